// dg_internal.h -- structures shared between the host API (dg_api.cu) and the
// kernel translation units (dg_kernels_f64.cu, dg_kernels_f32.cu).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dg.h"

namespace dg {

constexpr int NF = 5;       // conserved fields (rho, rho u, rho v, rho w, rho E)
constexpr int NMAX = DG_MAX_P + 1;

// 1D operators of the collocated Gauss-Legendre basis, scaled by the
// element geometry, in the kernels' scalar type.  Passed to kernels by value
// (kernel parameter space), so every operand read is a constant-bank load.
//   D[d][i][a]  = g_d * w_a l_i'(xi_a) / w_i    weak derivative with the
//                                               inverse mass folded in
//   Lp[d][i]    = g_d * l_i(+1) / (2 w_i)       lift of the +d face flux
//   Lm[d][i]    = g_d * l_i(-1) / (2 w_i)       lift of the -d face flux
//                 (the 1/2 of the Lax-Friedrichs flux, stored as 2 F*)
//   lp[a], lm[a] = l_a(+1), l_a(-1)             trace interpolation
// with g_d = 2 / h_d the reference-to-physical factor of direction d.
template <typename real>
struct Ops {
    real D[3][NMAX][NMAX];
    real Lp[3][NMAX];
    real Lm[3][NMAX];
    real lp[NMAX];
    real lm[NMAX];
    real gamma, gm1;  // ratio of specific heats and gamma - 1, in the kernels' type
};

// Mesh geometry and sizes (plain values; also by value into kernels).
struct Geo {
    int nx, ny, nz, p;
    long long E;       // elements
    double x0, y0, z0;
    double hx, hy, hz;
    double gamma;
    double J;          // hx hy hz / 8
    double hmin;
    double xi[NMAX];   // Gauss-Legendre nodes on [-1, 1]
    double w[NMAX];    // Gauss-Legendre weights
    // z slabs (dg_mesh_set_zhalo): when zlo is set, the mesh's z neighbours
    // beyond its own layers are not the periodic wrap but another slab's
    // layers, known only by their face traces, [NF][nx*ny][N^2] scalars of
    // the state's type (face point j*N + i):
    //   zlo   traces at the +z end of the layer below layer 0
    //   zhi   traces at the -z end of the layer above layer nz-1
    //   zflux (double form) the interface fluxes of the -z face of layer 0,
    //         [NF][nx*ny][N^2], computed by the face kernel from zlo
    const void *zlo, *zhi;
    void *zflux;
};

// Per-kernel CUDA-event timing of a mesh handle (dg_profile_begin/end):
// when on, every kernel launch is bracketed by two events recorded on the
// launching stream; the pairs are summed per kernel kind on request.
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> ev;   // start/stop pairs, in launch order
    std::vector<int> kind;         // kernel kind of each pair
    std::vector<cudaEvent_t> pool; // recycled events

    cudaEvent_t take()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void start(int k, cudaStream_t s)
    {
        if (!on) return;
        cudaEvent_t e = take();
        cudaEventRecord(e, s);
        ev.push_back(e);
        kind.push_back(k);
    }
    void stop(cudaStream_t s)
    {
        if (!on) return;
        cudaEvent_t e = take();
        cudaEventRecord(e, s);
        ev.push_back(e);
    }
};

// Device workspace owned by a mesh handle.
// dg_advance_host's copy-back of the new state, overlapped with the last
// step's fifth stage (double state): that stage's volume kernel runs in
// `chunks` ranges of whole z layers, and after each range its part of every
// field plane is copied to `host` on `stream` (which waits on ev[c]).
struct CopyOut {
    void *host = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t *ev = nullptr;  // one per chunk
    int chunks = 0;
};

// dg_advance_host's copy-in of the state (double state): the state arrives
// on `stream` in `chunks` ranges of whole z layers (ev[c] recorded after
// range c; ev[chunks] marks the start), and the first time-step reduction and
// the first stage's face kernel follow it range by range.
struct CopyIn {
    const void *host = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t *ev = nullptr;  // chunks + 1
    int chunks = 0;
};

struct Work {
    const CopyOut *out = nullptr;           // set by dg_advance_host only
    const CopyIn *in = nullptr;             // set by dg_advance_host only
    bool first_face_done = false;           // the step's first face kernel already ran
    void *face_flux = nullptr;              // 3 * NF * E * N^2 scalars
    double *partials = nullptr;             // norms partial sums, kNormBlocks x 8
    unsigned long long *lam_bits = nullptr; // CFL maximum (bits of a positive double)
    int *err = nullptr;                     // sticky error flag
    void *qtmp = nullptr;                   // second state (float form's ping-pong)
    void *zflux = nullptr;                  // -z interface fluxes of layer 0 (z slabs, double)
    Prof *prof = nullptr;                   // kernel timing (host object)
};

constexpr int kNormBlocks = 1024;  // fixed partition of the norms reduction

// Streaming multiprocessors of the current device (queried once per device;
// a benign race: concurrent first calls store the same value).  Grid-stride
// kernels size their grids as a multiple of it.
inline int sm_count()
{
    constexpr int kDevices = 64;
    static int cache[kDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < kDevices && cache[dev] > 0) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
        n = 1;
    if (dev >= 0 && dev < kDevices) cache[dev] = n;
    return n;
}

// Tile variant of the float form's fused stage per N = p + 1 (process-wide
// tuning table, set through dg_set_tile_variant; read at each launch).
int tile_variant(int N);
// true when the single-mesh float stage of order N uses the column kernel
bool column_stage(int N);  // a column kernel (column or line form) runs the stage
bool line_stage(int N);    // ... and it is the line form

// tiles of TX x TY elements covering a mesh: ceil(nx/TX) x ceil(ny/TY) x nz
__host__ __device__ inline long long tile_count(const Geo &g, int TX, int TY)
{
    return (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY) * g.nz;
}

// ---- batches of independent float meshes (dg_batch_*) ----

// Device descriptor of one instance of a batch.
struct InstDev {
    Geo g;
    Ops<float> T;
    float *Q, *Qt, *dQ;            // state, second state, RK register
    double *dt;                    // this instance's time step (device)
    unsigned long long *lam_bits;  // CFL maximum slot
};

// One work item of a batch's time-step reduction: nodes [begin, end) of one
// instance (node index within a field plane).
struct LambdaItem {
    int inst;
    long long begin, end;
};
constexpr long long kLambdaNodes = 1 << 14;

// One work item of a batch's line-kernel stage: one (column, z chunk) CTA of
// one instance (block = column + chunk x columns, as in a single-mesh launch).
struct LineItem {
    int inst;
    int block;
    int zchunk;
};

// Cross-section (TX, TY) of the line kernel of order N (false if N unsupported).
bool line_shape_info(int N, int *tx, int *ty);
// CTAs of the batched line kernel of order N resident per SM (0 on error).
int batch_line_blocks_per_sm(int N, bool small);
// One float-form RK stage of every listed work item (all of order N) of a
// batch; small: every instance's offsets fit a 32-bit int.
cudaError_t batch_line_stage(const LineItem *items, int nitems, const InstDev *inst, int N,
                             int parity, float A, float B, bool small, cudaStream_t s);

// Host-side facts about a tile code (N * 8 + variant): tile shape, threads,
// dynamic shared memory of the fused stage; false for an unknown code.
bool tile_code_info(int code, int *tx, int *ty, int *threads, size_t *smem);

// Launchers of the batched time-step kernels (dg_batch_f32.cu): Lambda of
// the listed node ranges (parity 0: the current state is in Q, 1: in the
// second state Qt), then dt of every instance from its Lambda slot (which
// other launches may have filled).
cudaError_t batch_lambda(const LambdaItem *items, int nitems, const InstDev *inst, int parity,
                         int *err, int grid, cudaStream_t s);
cudaError_t batch_dt(const InstDev *inst, int ninst, double cfl, cudaStream_t s);

// Lambda (maximum wave-speed sum) of a float state merged into *lam_bits
// (no time step yet), and one float-form RK stage of a single mesh
// (src -> dst, dQ updated) with the degree's stage kernel: the launches of a
// batch's large instances.
cudaError_t float_lambda(const Geo &g, const float *Q, unsigned long long *lam_bits, int *err,
                         cudaStream_t s);
cudaError_t float_stage(const Geo &g, const Ops<float> &T, const float *src, float *dst, float *dQ,
                        float A, float B, const double *dt, cudaStream_t s);

// Launchers implemented per scalar type (dg_kernels_f64.cu / dg_kernels_f32.cu).
// Each returns cudaSuccess or the launch error.
template <typename real>
struct Launch {
    static cudaError_t init(const Geo &g, int kind, const double *params, real *Q, Work &w,
                            cudaStream_t s);
    static cudaError_t rhs(const Geo &g, const Ops<real> &ops, const real *Q, real *R, Work &w,
                           cudaStream_t s);
    static cudaError_t rk_step(const Geo &g, const Ops<real> &ops, real *Q, real *dQ,
                               const double *dt, Work &w, cudaStream_t s);
    static cudaError_t cfl(const Geo &g, const real *Q, double cfl, double *dt, Work &w,
                           cudaStream_t s);
    static cudaError_t norms(const Geo &g, const real *Q, const real *Qref, double *out, Work &w,
                             cudaStream_t s);
    // one LSERK45 stage (stage in 0..4) from Qin to Qout
    static cudaError_t rk_stage(const Geo &g, const Ops<real> &ops, const real *Qin, real *Qout,
                                real *dQ, const double *dt, int stage, Work &w, cudaStream_t s);
    // z-face traces of the first and last layers (z slabs)
    static cudaError_t ztraces(const Geo &g, const Ops<real> &ops, const real *Q, real *lo,
                               real *hi, cudaStream_t s);
    // nsteps x (cfl time step -> dts[k], LSERK45 step, integrals -> integ[k * DG_NORMS_LEN])
    static cudaError_t advance(const Geo &g, const Ops<real> &ops, real *Q, real *dQ, double cfl,
                               int nsteps, double *dts, double *integ, Work &w, cudaStream_t s);
};

}  // namespace dg
