// Instantiation of the persistent solve kernel: double vectors, block sizes 17 .. 32.
#include "launch.cuh"
namespace bmr {
BMR_DEFINE_LAUNCHER(double, 32)
}  // namespace bmr
