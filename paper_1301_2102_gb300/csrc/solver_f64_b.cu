// Instantiations of the persistent solve kernel: double vectors, block sizes 5 .. 16.
#include "launch.cuh"
namespace bmr {
BMR_DEFINE_LAUNCHER(double, 8)
BMR_DEFINE_LAUNCHER(double, 16)
}  // namespace bmr
