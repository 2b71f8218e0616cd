// Instantiation of the persistent solve kernel: float vectors, block sizes 17 .. 32.
#include "launch.cuh"
namespace bmr {
BMR_DEFINE_LAUNCHER(float, 32)
}  // namespace bmr
