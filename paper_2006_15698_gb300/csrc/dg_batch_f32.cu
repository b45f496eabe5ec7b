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

template <int CLASS, typename Ix>
static cudaError_t batch_stage_c(const BatchItem *items, int nitems, const InstDev *inst,
                                 int parity, float A, float B, int grid, size_t smem,
                                 cudaStream_t s)
{
    cudaError_t err = cudaFuncSetAttribute(batched_stage_kernel<1, CLASS, Ix>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    batched_stage_kernel<1, CLASS, Ix><<<grid, kBatchClassThreads[CLASS], smem, s>>>(
        items, nitems, inst, parity, A, B);
    return cudaGetLastError();
}

cudaError_t batch_stage(const BatchItem *items, int nitems, const InstDev *inst, int parity,
                        float A, float B, int cls, bool small, int grid, size_t smem,
                        cudaStream_t s)
{
    if (small)
        return cls == 0 ? batch_stage_c<0, int>(items, nitems, inst, parity, A, B, grid, smem, s)
                        : batch_stage_c<1, int>(items, nitems, inst, parity, A, B, grid, smem, s);
    return cls == 0 ? batch_stage_c<0, long long>(items, nitems, inst, parity, A, B, grid, smem, s)
                    : batch_stage_c<1, long long>(items, nitems, inst, parity, A, B, grid, smem, s);
}

int batch_stage_blocks_per_sm(int cls, bool small, size_t smem)
{
    const void *fn = small ? (cls == 0 ? (const void *)batched_stage_kernel<1, 0, int>
                                       : (const void *)batched_stage_kernel<1, 1, int>)
                           : (cls == 0 ? (const void *)batched_stage_kernel<1, 0, long long>
                                       : (const void *)batched_stage_kernel<1, 1, long long>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 1;
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kBatchClassThreads[cls], smem) !=
        cudaSuccess)
        return 1;
    return n < 1 ? 1 : n;
}

cudaError_t batch_lambda(const BatchItem *items, int nitems, const InstDev *inst, int parity,
                         int *err, int grid, int threads, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    batched_cfl_kernel<<<grid, threads, 0, s>>>(items, nitems, inst, parity, err);
    return cudaGetLastError();
}

cudaError_t batch_dt(const InstDev *inst, int ninst, double cfl, cudaStream_t s)
{
    batched_cfl_finalize_kernel<<<(ninst + 127) / 128, 128, 0, s>>>(inst, ninst, cfl);
    return cudaGetLastError();
}

cudaError_t batch_cfl(const BatchItem *items, int nitems, const InstDev *inst, int ninst,
                      int parity, double cfl, int *err, int grid, int threads, cudaStream_t s)
{
    cudaError_t e = batch_lambda(items, nitems, inst, parity, err, grid, threads, s);
    if (e != cudaSuccess) return e;
    return batch_dt(inst, ninst, cfl, s);
}

}  // namespace dg
