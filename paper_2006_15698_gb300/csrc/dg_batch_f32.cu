// Batches of independent float meshes: the tile codes of the single-mesh
// tile kernel and the batched time-step kernels' launchers (a translation unit of its own, so that it compiles in
// parallel with the single-mesh float kernels).
#include "dg_kernels.cuh"

// ---------------------------------------------------------------------------
// batches (float form only)
// ---------------------------------------------------------------------------
namespace dg {

bool tile_code_info(int code, int *tx, int *ty, int *threads, size_t *smem)
{
    switch (code) {
#define DG_CASE(NN, VV)                                                        \
    case NN * 8 + VV: {                                                        \
        using SH = TileShape<NN, VV>;                                          \
        using FT = FusedTile<NN, SH::TX, SH::TY>;                              \
        *tx = SH::TX;                                                          \
        *ty = SH::TY;                                                          \
        *threads = FT::THREADS;                                                \
        *smem = FT::BYTES;                                                     \
        return true;                                                           \
    }
        DG_FOR_EACH_CODE(DG_CASE)
#undef DG_CASE
    default: return false;
    }
}

cudaError_t batch_lambda(const LambdaItem *items, int nitems, const InstDev *inst, int parity,
                         int *err, int grid, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    batched_lambda_kernel<<<grid, 256, 0, s>>>(items, nitems, inst, parity, err);
    return cudaGetLastError();
}

cudaError_t batch_dt(const InstDev *inst, int ninst, double cfl, cudaStream_t s)
{
    batched_cfl_finalize_kernel<<<(ninst + 127) / 128, 128, 0, s>>>(inst, ninst, cfl);
    return cudaGetLastError();
}

}  // namespace dg
