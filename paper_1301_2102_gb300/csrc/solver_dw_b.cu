// Instantiations of the persistent solve kernel: double-word vectors, block sizes 5 .. 16.
#include "launch.cuh"
namespace bmr {
BMR_DEFINE_LAUNCHER(dw, 8)
BMR_DEFINE_LAUNCHER(dw, 16)
}  // namespace bmr
