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

cudaError_t float_lambda(const Geo &g, const float *Q, unsigned long long *lam_bits, int *err,
                         cudaStream_t s)
{
    const long long nodes = g.E * (long long)(g.p + 1) * (g.p + 1) * (g.p + 1);
    cfl_kernel<float><<<grid_for(nodes, 256, 8LL * sm_count()), 256, 0, s>>>(Q, nodes, g.gamma, lam_bits,
                                                                     err);
    return cudaGetLastError();
}

cudaError_t float_stage(const Geo &g, const Ops<float> &T, const float *src, float *dst, float *dQ,
                        float A, float B, const double *dt, cudaStream_t s)
{
#define DG_CALL(NN) stage_n<NN, float>(g, T, src, dst, dQ, A, B, dt, s)
    DG_DISPATCH_P(g.p, DG_CALL)
#undef DG_CALL
}
}
