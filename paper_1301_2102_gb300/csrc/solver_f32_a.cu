// Instantiations of the persistent solve kernel: float vectors, block sizes up to 4.
#include "launch.cuh"
namespace bmr {
BMR_DEFINE_LAUNCHER(float, 1)
BMR_DEFINE_LAUNCHER(float, 2)
BMR_DEFINE_LAUNCHER(float, 4)
}  // namespace bmr
