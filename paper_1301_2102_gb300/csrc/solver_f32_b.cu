// Instantiations of the persistent solve kernel: float vectors, block sizes 5 .. 16.
#include "launch.cuh"
namespace bmr {
BMR_DEFINE_LAUNCHER(float, 8)
BMR_DEFINE_LAUNCHER(float, 16)
}  // namespace bmr
