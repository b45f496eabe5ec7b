// FP32 instantiation of the DG kernels (float state and volume/surface
// arithmetic; the time-step and integral reductions accumulate in double).
// The per-degree stage paths are compiled in dg_f32_deg*.cu.
#include "dg_kernels.cuh"

namespace dg {
DG_INSTANTIATE_N(extern template, 1, float)
DG_INSTANTIATE_N(extern template, 2, float)
DG_INSTANTIATE_N(extern template, 3, float)
DG_INSTANTIATE_N(extern template, 4, float)
DG_INSTANTIATE_N(extern template, 5, float)
DG_INSTANTIATE_N(extern template, 6, float)
DG_INSTANTIATE_N(extern template, 7, float)
template struct Launch<float>;
}
