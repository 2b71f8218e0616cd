// Instantiations of the persistent solve kernel: double vectors, block sizes up to 4.
#include "launch.cuh"
namespace bmr {
BMR_DEFINE_LAUNCHER(double, 1)
BMR_DEFINE_LAUNCHER(double, 2)
BMR_DEFINE_LAUNCHER(double, 4)
}  // namespace bmr
