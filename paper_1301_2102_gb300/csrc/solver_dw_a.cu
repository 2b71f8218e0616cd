// Instantiations of the persistent solve kernel: double-word vectors, block sizes up to 4.
#include "launch.cuh"
namespace bmr {
BMR_DEFINE_LAUNCHER(dw, 1)
BMR_DEFINE_LAUNCHER(dw, 2)
BMR_DEFINE_LAUNCHER(dw, 4)
}  // namespace bmr
