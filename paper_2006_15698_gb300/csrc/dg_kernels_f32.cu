// FP32 instantiation of the DG kernels (float state and volume/surface
// arithmetic; the time-step and integral reductions accumulate in double).
#include "dg_kernels.cuh"

namespace dg {
template struct Launch<float>;
}
