// Batches of independent float meshes: the persistent batched stage and CFL
// kernels' launchers (a translation unit of its own, so that it compiles in
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

int batch_code_class(int code) { return batch_class(code); }
int batch_class_threads(int cls) { return kBatchClassThreads[cls]; }

template <int CLASS>
static cudaError_t batch_stage_c(const BatchItem *items, int nitems, const InstDev *inst,
                                 int parity, float A, float B, int grid, size_t smem,
                                 cudaStream_t s)
{
    cudaError_t err = cudaFuncSetAttribute(batched_stage_kernel<1, CLASS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    batched_stage_kernel<1, CLASS><<<grid, kBatchClassThreads[CLASS], smem, s>>>(items, nitems,
                                                                                 inst, parity, A, B);
    return cudaGetLastError();
}

cudaError_t batch_stage(const BatchItem *items, int nitems, const InstDev *inst, int parity,
                        float A, float B, int cls, int grid, size_t smem, cudaStream_t s)
{
    return cls == 0 ? batch_stage_c<0>(items, nitems, inst, parity, A, B, grid, smem, s)
                    : batch_stage_c<1>(items, nitems, inst, parity, A, B, grid, smem, s);
}

int batch_stage_blocks_per_sm(int cls, size_t smem)
{
    const void *fn = cls == 0 ? (const void *)batched_stage_kernel<1, 0>
                              : (const void *)batched_stage_kernel<1, 1>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 1;
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kBatchClassThreads[cls], smem) !=
        cudaSuccess)
        return 1;
    return n < 1 ? 1 : n;
}

cudaError_t batch_cfl(const BatchItem *items, int nitems, const InstDev *inst, int ninst,
                      int parity, double cfl, int *err, int grid, int threads, cudaStream_t s)
{
    batched_cfl_kernel<<<grid, threads, 0, s>>>(items, nitems, inst, parity, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batched_cfl_finalize_kernel<<<(ninst + 127) / 128, 128, 0, s>>>(inst, ninst, cfl);
    return cudaGetLastError();
}

}  // namespace dg
