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
    cfl_kernel<float><<<grid_for(nodes, 256, 8LL * sm_count()), 256, 0, s>>>(
        Q, nodes, 0, nodes, g.gamma, lam_bits, err);
    return cudaGetLastError();
}

bool line_shape_info(int N, int *tx, int *ty)
{
    switch (N) {
#define DG_CASE(NN)                      \
    case NN:                             \
        *tx = LineShape<NN, 0>::TX;      \
        *ty = LineShape<NN, 0>::TY;      \
        return true;
        DG_CASE(1) DG_CASE(2) DG_CASE(3) DG_CASE(4) DG_CASE(5) DG_CASE(6) DG_CASE(7)
#undef DG_CASE
    default: return false;
    }
}

cudaError_t batch_line_stage(const LineItem *items, int nitems, const InstDev *inst, int N,
                             int parity, float A, float B, bool small, cudaStream_t s)
{
#define DG_CALL(NN) batch_line_n<NN, float>(items, nitems, inst, parity, A, B, small, s)
    DG_DISPATCH_P(N - 1, DG_CALL)
#undef DG_CALL
}

int batch_line_blocks_per_sm(int N, bool small)
{
    switch (N) {
    case 1: return batch_line_blocks_per_sm_n<1, float>(small);
    case 2: return batch_line_blocks_per_sm_n<2, float>(small);
    case 3: return batch_line_blocks_per_sm_n<3, float>(small);
    case 4: return batch_line_blocks_per_sm_n<4, float>(small);
    case 5: return batch_line_blocks_per_sm_n<5, float>(small);
    case 6: return batch_line_blocks_per_sm_n<6, float>(small);
    case 7: return batch_line_blocks_per_sm_n<7, float>(small);
    default: return 0;
    }
}

cudaError_t float_stage(const Geo &g, const Ops<float> &T, const float *src, float *dst, float *dQ,
                        float A, float B, const double *dt, cudaStream_t s)
{
#define DG_CALL(NN) stage_n<NN, float>(g, T, src, dst, dQ, A, B, dt, s)
    DG_DISPATCH_P(g.p, DG_CALL)
#undef DG_CALL
}
}
