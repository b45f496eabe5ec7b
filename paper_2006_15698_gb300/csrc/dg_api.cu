// dg_api.cu -- host side of the C ABI declared in include/dg.h: argument
// checks, the 1D operators of the collocated Gauss-Legendre basis, the mesh
// handle's device workspace, and dispatch to the per-precision launchers.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <algorithm>
#include <vector>

#include "dg_internal.h"

// ranges of z layers in which dg_advance_host (double state) moves the state:
// in, each range followed by the first reduction and face kernel over it;
// back, each range copied while the last stage computes the next ones
constexpr int kCopyChunks = 8;

struct dg_mesh {
    dg::Geo geo;
    dg_precision prec;
    dg::Ops<double> ops64;
    dg::Ops<float> ops32;
    dg::Work work;
    dg::Prof *prof;
    int device;
    size_t ws_bytes;
    // dg_advance_host: device time steps and integrals of the largest call
    // so far (allocated on first use)
    double *io = nullptr;
    size_t io_cap = 0;
    // dg_advance_host, double state: the copy stream and its events (created
    // on first use) for the copy-in overlapped with the first reduction and
    // face kernel, and the copy-back overlapped with the last stage
    // (copy-back: ranges 0..K-1 and the end; copy-in: K+1 .. 2K+1)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[2 * kCopyChunks + 2] = {};
};

namespace {

// ---------------------------------------------------------------------------
// 1D operators (Sec. II.B, Eq. 7): Gauss-Legendre rule by Newton iteration on
// P_N from Chebyshev starting points (long double), then the Lagrange basis in
// barycentric form (Berrut & Trefethen 2004):
//   lambda_j = 1 / prod_{k != j} (x_j - x_k)
//   l_j(x)   = [lambda_j / (x - x_j)] / sum_k [lambda_k / (x - x_k)]
//   l_j'(x_i) = (lambda_j / lambda_i) / (x_i - x_j)   (i != j),
//   l_i'(x_i) = -sum_{j != i} l_j'(x_i)
// ---------------------------------------------------------------------------
void gauss_legendre(int N, long double *x, long double *w)
{
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 0; k < N; ++k) {
        long double r = cosl(pi * (2 * k + 1) / (2.0L * N));  // Chebyshev point
        long double pn = 0, pn1 = 0;
        for (int it = 0; it < 200; ++it) {
            // P_N(r) and P_{N-1}(r) by Bonnet's recurrence
            long double a = 1, b = r;
            if (N == 1) { pn = r; pn1 = 1; }
            else {
                for (int m = 2; m <= N; ++m) {
                    long double c = ((2 * m - 1) * r * b - (m - 1) * a) / m;
                    a = b;
                    b = c;
                }
                pn = b;
                pn1 = a;
            }
            long double dp = N * (pn1 - r * pn) / (1 - r * r);  // P_N'(r)
            long double dr = pn / dp;
            r -= dr;
            if (fabsl(dr) < 1e-30L) break;
        }
        // recompute P_{N-1} at the converged root for the weight
        long double a = 1, b = r;
        for (int m = 2; m <= N; ++m) {
            long double c = ((2 * m - 1) * r * b - (m - 1) * a) / m;
            a = b;
            b = c;
        }
        long double pm1 = (N == 1) ? 1.0L : a;
        x[k] = r;
        w[k] = 2 * (1 - r * r) / ((long double)N * N * pm1 * pm1);
    }
    // ascending order
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j)
            if (x[j] < x[i]) {
                long double t = x[i]; x[i] = x[j]; x[j] = t;
                t = w[i]; w[i] = w[j]; w[j] = t;
            }
    if (N % 2 == 1) x[N / 2] = 0;  // the middle node is exactly 0 by symmetry
}

struct Basis {
    int N;
    long double x[dg::NMAX], w[dg::NMAX];
    long double Dm[dg::NMAX][dg::NMAX];  // Dm[i][j] = l_j'(x_i)
    long double ep[dg::NMAX], em[dg::NMAX];  // l_j(+1), l_j(-1)
};

void make_basis(int N, Basis &B)
{
    B.N = N;
    gauss_legendre(N, B.x, B.w);
    long double lam[dg::NMAX];
    for (int j = 0; j < N; ++j) {
        long double prod = 1;
        for (int k = 0; k < N; ++k)
            if (k != j) prod *= (B.x[j] - B.x[k]);
        lam[j] = 1 / prod;
    }
    for (int i = 0; i < N; ++i) {
        long double diag = 0;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            B.Dm[i][j] = (lam[j] / lam[i]) / (B.x[i] - B.x[j]);
            diag -= B.Dm[i][j];
        }
        B.Dm[i][i] = diag;
    }
    for (int s = 0; s < 2; ++s) {
        const long double X = s == 0 ? 1.0L : -1.0L;  // never a node of a Gauss rule
        long double den = 0;
        for (int k = 0; k < N; ++k) den += lam[k] / (X - B.x[k]);
        for (int j = 0; j < N; ++j) {
            long double v = (lam[j] / (X - B.x[j])) / den;
            if (s == 0) B.ep[j] = v; else B.em[j] = v;
        }
    }
}

template <typename real>
void fill_ops(const Basis &B, const double g[3], dg::Ops<real> &T)
{
    std::memset(&T, 0, sizeof(T));
    const int N = B.N;
    for (int d = 0; d < 3; ++d)
        for (int i = 0; i < N; ++i) {
            for (int a = 0; a < N; ++a)  // g * w_a l_i'(x_a) / w_i
                T.D[d][i][a] = (real)((long double)g[d] * B.w[a] * B.Dm[a][i] / B.w[i]);
            // lift vectors carry the 1/2 of the Lax-Friedrichs flux, whose
            // kernel stores 2 F*
            T.Lp[d][i] = (real)((long double)g[d] * B.ep[i] / B.w[i] / 2);
            T.Lm[d][i] = (real)((long double)g[d] * B.em[i] / B.w[i] / 2);
        }
    for (int a = 0; a < N; ++a) {
        T.lp[a] = (real)B.ep[a];
        T.lm[a] = (real)B.em[a];
    }
}

template <typename real>
void fill_gas(double gamma, dg::Ops<real> &T)
{
    T.gamma = (real)gamma;
    T.gm1 = (real)(gamma - 1.0);
}

dg_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return DG_OK;
    if (e == cudaErrorMemoryAllocation) return DG_ERR_OOM;
    if (e == cudaErrorNotSupported) return DG_ERR_UNSUPPORTED;  // a launcher's own refusal
    return DG_ERR_CUDA;
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

// state arrays start on a 16-byte boundary (vector loads of node lines)
bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" {

dg_status dg_mesh_create(int nx, int ny, int nz, int p, double x0, double y0, double z0,
                         double Lx, double Ly, double Lz, double gamma, dg_precision precision,
                         dg_mesh **out)
{
    if (!out) return DG_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return DG_ERR_ARG;
    if (!finite_pos(Lx) || !finite_pos(Ly) || !finite_pos(Lz)) return DG_ERR_ARG;
    if (!std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(z0)) return DG_ERR_ARG;
    if (!(std::isfinite(gamma) && gamma > 1.0)) return DG_ERR_ARG;
    if (precision != DG_FP64 && precision != DG_FP32) return DG_ERR_ARG;
    if (p < 0 || p > DG_MAX_P) return DG_ERR_UNSUPPORTED;
    const int N = p + 1;
    const long long E = (long long)nx * ny * nz;
    if (E * N * N * N >= (1LL << 40)) return DG_ERR_ARG;

    dg_mesh *m = new (std::nothrow) dg_mesh();
    if (!m) return DG_ERR_OOM;
    m->prof = new (std::nothrow) dg::Prof();
    if (!m->prof) { delete m; return DG_ERR_OOM; }
    m->work.prof = m->prof;
    m->prec = precision;
    dg::Geo &g = m->geo;
    g.nx = nx; g.ny = ny; g.nz = nz; g.p = p; g.E = E;
    g.x0 = x0; g.y0 = y0; g.z0 = z0;
    g.hx = Lx / nx; g.hy = Ly / ny; g.hz = Lz / nz;
    g.gamma = gamma;
    g.J = g.hx * g.hy * g.hz / 8.0;
    g.hmin = std::fmin(g.hx, std::fmin(g.hy, g.hz));
    Basis B;
    make_basis(N, B);
    for (int a = 0; a < N; ++a) {
        g.xi[a] = (double)B.x[a];
        g.w[a] = (double)B.w[a];
    }
    const double gf[3] = {2.0 / g.hx, 2.0 / g.hy, 2.0 / g.hz};
    fill_ops(B, gf, m->ops64);
    fill_ops(B, gf, m->ops32);
    fill_gas(gamma, m->ops64);
    fill_gas(gamma, m->ops32);

    cudaError_t err = cudaGetDevice(&m->device);
    if (err != cudaSuccess) { dg_mesh_destroy(m); return DG_ERR_CUDA; }
    const size_t esz = precision == DG_FP64 ? sizeof(double) : sizeof(float);
    // double form: the interface-flux buffer of the two-kernel stage;
    // float form: the second state of the fused single-pass stage
    const size_t fbytes =
        precision == DG_FP64 ? (size_t)3 * dg::NF * (size_t)E * N * N * esz : 0;
    const size_t tbytes =
        precision == DG_FP32 ? (size_t)dg::NF * (size_t)E * N * N * N * esz : 0;
    const size_t pbytes = (size_t)dg::kNormBlocks * 8 * sizeof(double);
    if (fbytes) err = cudaMalloc(&m->work.face_flux, fbytes);
    if (err == cudaSuccess && tbytes) err = cudaMalloc(&m->work.qtmp, tbytes);
    if (err == cudaSuccess) err = cudaMalloc((void **)&m->work.partials, pbytes);
    if (err == cudaSuccess) err = cudaMalloc((void **)&m->work.lam_bits, sizeof(unsigned long long));
    if (err == cudaSuccess) err = cudaMalloc((void **)&m->work.err, sizeof(int));
    if (err == cudaSuccess) err = cudaMemset(m->work.lam_bits, 0, sizeof(unsigned long long));
    if (err == cudaSuccess) err = cudaMemset(m->work.err, 0, sizeof(int));
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        dg_status st = cuda_status(err);
        cudaGetLastError();  // clear a sticky allocation error
        dg_mesh_destroy(m);
        return st;
    }
    m->ws_bytes = fbytes + tbytes + pbytes + sizeof(unsigned long long) + sizeof(int);
    *out = m;
    return DG_OK;
}

void dg_mesh_destroy(dg_mesh *m)
{
    if (!m) return;
    cudaDeviceSynchronize();
    cudaFree(m->work.face_flux);
    cudaFree(m->work.qtmp);
    cudaFree(m->work.zflux);
    cudaFree(m->work.partials);
    cudaFree(m->work.lam_bits);
    cudaFree(m->work.err);
    cudaFree(m->io);
    for (cudaEvent_t e : m->copy_ev)
        if (e) cudaEventDestroy(e);
    if (m->copy_stream) cudaStreamDestroy(m->copy_stream);
    if (m->prof) {
        for (cudaEvent_t e : m->prof->ev) cudaEventDestroy(e);
        for (cudaEvent_t e : m->prof->pool) cudaEventDestroy(e);
        delete m->prof;
    }
    delete m;
}

dg_status dg_mesh_sizes(const dg_mesh *m, int64_t *n_dof, int64_t *n_unknowns,
                        size_t *state_bytes, size_t *workspace_bytes)
{
    if (!m) return DG_ERR_ARG;
    const int N = m->geo.p + 1;
    const int64_t dof = (int64_t)m->geo.E * N * N * N;
    if (n_dof) *n_dof = dof;
    if (n_unknowns) *n_unknowns = dg::NF * dof;
    if (state_bytes)
        *state_bytes = (size_t)dg::NF * dof * (m->prec == DG_FP64 ? sizeof(double) : sizeof(float));
    if (workspace_bytes) *workspace_bytes = m->ws_bytes;
    return DG_OK;
}

dg_status dg_state_init(const dg_mesh *m, dg_init_kind kind, const double *params, int nparams,
                        void *Q, void *stream)
{
    if (!m || !Q) return DG_ERR_ARG;
    int need = kind == DG_INIT_UNIFORM ? 5 : kind == DG_INIT_VORTEX ? 7 : kind == DG_INIT_TGV ? 3 : -1;
    if (need < 0 || nparams < need || nparams > 8 || !params) return DG_ERR_ARG;
    double pr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < nparams; ++i) {
        if (!std::isfinite(params[i])) return DG_ERR_ARG;
        pr[i] = params[i];
    }
    dg::Work w = m->work;
    cudaError_t e = m->prec == DG_FP64
                        ? dg::Launch<double>::init(m->geo, kind, pr, (double *)Q, w, as_stream(stream))
                        : dg::Launch<float>::init(m->geo, kind, pr, (float *)Q, w, as_stream(stream));
    return cuda_status(e);
}

dg_status dg_rhs(const dg_mesh *m, const void *Q, void *R, void *stream)
{
    if (!m || !Q || !R || Q == R || !aligned16(Q) || !aligned16(R)) return DG_ERR_ARG;
    dg::Work w = m->work;
    cudaError_t e = m->prec == DG_FP64
                        ? dg::Launch<double>::rhs(m->geo, m->ops64, (const double *)Q, (double *)R,
                                                  w, as_stream(stream))
                        : dg::Launch<float>::rhs(m->geo, m->ops32, (const float *)Q, (float *)R, w,
                                                 as_stream(stream));
    return cuda_status(e);
}

dg_status dg_cfl_dt(const dg_mesh *m, const void *Q, double cfl, double *dt_dev, void *stream)
{
    if (!m || !Q || !dt_dev || !finite_pos(cfl)) return DG_ERR_ARG;
    dg::Work w = m->work;
    cudaError_t e = m->prec == DG_FP64
                        ? dg::Launch<double>::cfl(m->geo, (const double *)Q, cfl, dt_dev, w,
                                                  as_stream(stream))
                        : dg::Launch<float>::cfl(m->geo, (const float *)Q, cfl, dt_dev, w,
                                                 as_stream(stream));
    return cuda_status(e);
}

dg_status dg_rk_step(const dg_mesh *m, void *Q, void *dQ, const double *dt_dev, void *stream)
{
    if (!m || !Q || !dQ || !dt_dev || Q == dQ || !aligned16(Q) || !aligned16(dQ)) return DG_ERR_ARG;
    if (m->geo.zlo) return DG_ERR_UNSUPPORTED;  // a slab's halos change between stages
    dg::Work w = m->work;
    cudaError_t e = m->prec == DG_FP64
                        ? dg::Launch<double>::rk_step(m->geo, m->ops64, (double *)Q, (double *)dQ,
                                                      dt_dev, w, as_stream(stream))
                        : dg::Launch<float>::rk_step(m->geo, m->ops32, (float *)Q, (float *)dQ,
                                                     dt_dev, w, as_stream(stream));
    return cuda_status(e);
}

dg_status dg_advance(const dg_mesh *m, void *Q, void *dQ, double cfl, int nsteps, double *dts,
                     double *integ, void *stream)
{
    if (!m || !Q || !dQ || !dts || Q == dQ || !aligned16(Q) || !aligned16(dQ) || nsteps < 1 ||
        !(cfl > 0.0) || !std::isfinite(cfl))
        return DG_ERR_ARG;
    if (m->geo.zlo) return DG_ERR_UNSUPPORTED;  // a slab's halos change between stages
    dg::Work w = m->work;
    cudaError_t e = m->prec == DG_FP64
                        ? dg::Launch<double>::advance(m->geo, m->ops64, (double *)Q, (double *)dQ,
                                                      cfl, nsteps, dts, integ, w, as_stream(stream))
                        : dg::Launch<float>::advance(m->geo, m->ops32, (float *)Q, (float *)dQ,
                                                     cfl, nsteps, dts, integ, w, as_stream(stream));
    return cuda_status(e);
}

dg_status dg_advance_host(dg_mesh *m, void *Q_host, void *Q, void *dQ, double cfl, int nsteps,
                          double *dts_host, double *integ_host, void *stream)
{
    if (!m || !Q_host || !dts_host || !Q || !dQ || Q == dQ || !aligned16(Q) || !aligned16(dQ) ||
        nsteps < 1 || !(cfl > 0.0) || !std::isfinite(cfl))
        return DG_ERR_ARG;
    if (m->geo.zlo) return DG_ERR_UNSUPPORTED;
    const int N = m->geo.p + 1;
    const size_t per = (size_t)(1 + (integ_host ? DG_NORMS_LEN : 0));
    if ((size_t)nsteps > (SIZE_MAX / sizeof(double)) / per) return DG_ERR_ARG;
    const size_t need = (size_t)nsteps * per;
    if (need > m->io_cap) {
        cudaFree(m->io);
        m->io = nullptr;
        m->io_cap = 0;
        cudaError_t e = cudaMalloc((void **)&m->io, need * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();  // not sticky: the context stays usable
            return DG_ERR_OOM;
        }
        m->io_cap = need;
    }
    cudaStream_t s = as_stream(stream);
    const size_t bytes = (size_t)dg::NF * (size_t)m->geo.E * N * N * N *
                         (m->prec == DG_FP64 ? sizeof(double) : sizeof(float));
    double *dts = m->io, *integ = integ_host ? m->io + nsteps : nullptr;
    cudaError_t e = cudaSuccess;
    // the overlapped copy-back needs page-locked host memory (a copy into
    // pageable memory holds the host thread until it is done, which would
    // serialise the ranges)
    bool overlap = false;
    if (m->prec == DG_FP64) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, Q_host) == cudaSuccess)
            overlap = pa.type == cudaMemoryTypeHost;
        else
            cudaGetLastError();
    }
    if (overlap && !m->copy_stream) {
        e = cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking);
        for (int c = 0; c < 2 * kCopyChunks + 2 && e == cudaSuccess; ++c)
            e = cudaEventCreateWithFlags(&m->copy_ev[c], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (cudaEvent_t &ev : m->copy_ev)
                if (ev) { cudaEventDestroy(ev); ev = nullptr; }
            if (m->copy_stream) { cudaStreamDestroy(m->copy_stream); m->copy_stream = nullptr; }
            return DG_ERR_CUDA;
        }
    }
    if (!overlap) {
        e = cudaMemcpyAsync(Q, Q_host, bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (overlap) {
        // the state comes in range by range, the first reduction and face
        // kernel following it, and goes back range by range during the last
        // stage (kernels and floats as dg_advance; the copies on the mesh's
        // copy stream, joined into the caller's stream before the time steps)
        dg::CopyIn ci;
        ci.host = Q_host;
        ci.stream = m->copy_stream;
        ci.ev = m->copy_ev + kCopyChunks + 1;
        ci.chunks = kCopyChunks;
        dg::CopyOut co;
        co.host = Q_host;
        co.stream = m->copy_stream;
        co.ev = m->copy_ev;
        co.chunks = kCopyChunks;
        dg::Work w = m->work;
        w.in = &ci;
        w.out = &co;
        e = dg::Launch<double>::advance(m->geo, m->ops64, (double *)Q, (double *)dQ, cfl, nsteps,
                                        dts, integ, w, s);
        if (e == cudaSuccess) e = cudaEventRecord(m->copy_ev[kCopyChunks], m->copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->copy_ev[kCopyChunks], 0);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(m->copy_stream);
            return cuda_status(e);
        }
    } else {
        const dg_status st = dg_advance(m, Q, dQ, cfl, nsteps, dts, integ, stream);
        if (st != DG_OK) return st;
        e = cudaMemcpyAsync(Q_host, Q, bytes, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dts_host, dts, (size_t)nsteps * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && integ_host)
        e = cudaMemcpyAsync(integ_host, integ, (size_t)nsteps * DG_NORMS_LEN * sizeof(double),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(e);
}

dg_status dg_rk_stage(const dg_mesh *m, const void *Qin, void *Qout, void *dQ,
                      const double *dt_dev, int stage, void *stream)
{
    if (!m || !Qin || !Qout || !dQ || !dt_dev || stage < 0 || stage > 4) return DG_ERR_ARG;
    if (Qin == dQ || Qout == dQ || !aligned16(Qin) || !aligned16(Qout) || !aligned16(dQ))
        return DG_ERR_ARG;
    if (m->prec == DG_FP32 && Qin == Qout) return DG_ERR_ARG;
    dg::Work w = m->work;
    cudaError_t e = m->prec == DG_FP64
                        ? dg::Launch<double>::rk_stage(m->geo, m->ops64, (const double *)Qin,
                                                       (double *)Qout, (double *)dQ, dt_dev, stage,
                                                       w, as_stream(stream))
                        : dg::Launch<float>::rk_stage(m->geo, m->ops32, (const float *)Qin,
                                                      (float *)Qout, (float *)dQ, dt_dev, stage, w,
                                                      as_stream(stream));
    return cuda_status(e);
}

dg_status dg_mesh_set_zhalo(dg_mesh *m, const void *halo_lo, const void *halo_hi)
{
    if (!m || (!halo_lo) != (!halo_hi)) return DG_ERR_ARG;
    if (!halo_lo) {
        m->geo.zlo = m->geo.zhi = nullptr;
        m->geo.zflux = nullptr;
        return DG_OK;
    }
    if (m->prec == DG_FP32 && !dg::column_stage(m->geo.p + 1)) return DG_ERR_UNSUPPORTED;
    if (m->prec == DG_FP64 && !m->work.zflux) {
        const int N = m->geo.p + 1;
        const size_t bytes = (size_t)dg::NF * (size_t)m->geo.nx * m->geo.ny * N * N * sizeof(double);
        cudaError_t e = cudaMalloc(&m->work.zflux, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            m->work.zflux = nullptr;
            return cuda_status(e);
        }
        m->ws_bytes += bytes;
    }
    m->geo.zlo = halo_lo;
    m->geo.zhi = halo_hi;
    m->geo.zflux = m->work.zflux;
    return DG_OK;
}

dg_status dg_zhalo_traces(const dg_mesh *m, const void *Q, void *send_lo, void *send_hi,
                          void *stream)
{
    if (!m || !Q || !send_lo || !send_hi || send_lo == send_hi) return DG_ERR_ARG;
    cudaError_t e = m->prec == DG_FP64
                        ? dg::Launch<double>::ztraces(m->geo, m->ops64, (const double *)Q,
                                                      (double *)send_lo, (double *)send_hi,
                                                      as_stream(stream))
                        : dg::Launch<float>::ztraces(m->geo, m->ops32, (const float *)Q,
                                                     (float *)send_lo, (float *)send_hi,
                                                     as_stream(stream));
    return cuda_status(e);
}

dg_status dg_norms(const dg_mesh *m, const void *Q, const void *Qref, double *out, void *stream)
{
    if (!m || !Q || !out) return DG_ERR_ARG;
    dg::Work w = m->work;
    cudaError_t e = m->prec == DG_FP64
                        ? dg::Launch<double>::norms(m->geo, (const double *)Q,
                                                    (const double *)Qref, out, w, as_stream(stream))
                        : dg::Launch<float>::norms(m->geo, (const float *)Q, (const float *)Qref,
                                                   out, w, as_stream(stream));
    return cuda_status(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// dg_rhs_static: the right-hand side without any device allocation.  The
// interface-flux scratch is this file-scope device array; host code must not
// use its name as a device address (on the host it names a stand-in), so
// each device's address is looked up once with cudaGetSymbolAddress and
// passed to the kernels.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_face_scratch[DG_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void *g_static_addr[kMaxDevices] = {};  // per device, filled on first use

cudaError_t static_scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_face_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

dg_status dg_rhs_static(int nx, int ny, int nz, int p, double x0, double y0, double z0,
                        double Lx, double Ly, double Lz, double gamma, dg_precision precision,
                        const void *Q, void *R, void *stream)
{
    if (!Q || !R || Q == R || !aligned16(Q) || !aligned16(R)) return DG_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1) return DG_ERR_ARG;
    if (!finite_pos(Lx) || !finite_pos(Ly) || !finite_pos(Lz)) return DG_ERR_ARG;
    if (!std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(z0)) return DG_ERR_ARG;
    if (!(std::isfinite(gamma) && gamma > 1.0)) return DG_ERR_ARG;
    if (precision != DG_FP64 && precision != DG_FP32) return DG_ERR_ARG;
    if (p < 0 || p > DG_MAX_P) return DG_ERR_UNSUPPORTED;
    const int N = p + 1;
    const long long E = (long long)nx * ny * nz;
    if (E * N * N * N >= (1LL << 40)) return DG_ERR_ARG;
    // only the double form has interface-flux scratch (the float form's
    // single-pass stage keeps its interface fluxes in shared memory)
    if (precision == DG_FP64) {
        const double need = 3.0 * dg::NF * (double)E * N * N * (double)sizeof(double);
        if (need > (double)DG_STATIC_SCRATCH_BYTES) return DG_ERR_TOO_LARGE;
    }

    dg::Geo g{};
    g.nx = nx; g.ny = ny; g.nz = nz; g.p = p; g.E = E;
    g.x0 = x0; g.y0 = y0; g.z0 = z0;
    g.hx = Lx / nx; g.hy = Ly / ny; g.hz = Lz / nz;
    g.gamma = gamma;
    g.J = g.hx * g.hy * g.hz / 8.0;
    g.hmin = std::fmin(g.hx, std::fmin(g.hy, g.hz));
    Basis B;
    make_basis(N, B);
    for (int a = 0; a < N; ++a) {
        g.xi[a] = (double)B.x[a];
        g.w[a] = (double)B.w[a];
    }
    const double gf[3] = {2.0 / g.hx, 2.0 / g.hy, 2.0 / g.hz};

    dg::Work w;
    cudaError_t e = cudaSuccess;
    if (precision == DG_FP64) {
        e = static_scratch_address(&w.face_flux);
        if (e != cudaSuccess) return DG_ERR_CUDA;
        dg::Ops<double> ops;
        fill_ops(B, gf, ops);
        fill_gas(gamma, ops);
        e = dg::Launch<double>::rhs(g, ops, (const double *)Q, (double *)R, w, as_stream(stream));
    } else {
        dg::Ops<float> ops;
        fill_ops(B, gf, ops);
        fill_gas(gamma, ops);
        e = dg::Launch<float>::rhs(g, ops, (const float *)Q, (float *)R, w, as_stream(stream));
    }
    return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// tile-shape tuning table of the float form's fused stage
// ---------------------------------------------------------------------------
namespace dg {
static int g_tile_var[NMAX + 1] = {0, 0, 0, 0, 0, 0, 0, 0};
static int g_stage_kind[NMAX + 1] = {2, 2, 2, 2, 2, 2, 2, 2};
int tile_variant(int N) { return (N >= 1 && N <= NMAX) ? g_tile_var[N] : 0; }
bool column_stage(int N)
{
    return N >= 1 && N <= NMAX && (g_stage_kind[N] == DG_STAGE_COLUMN || g_stage_kind[N] == DG_STAGE_LINES);
}
bool line_stage(int N) { return N >= 1 && N <= NMAX && g_stage_kind[N] == DG_STAGE_LINES; }
}  // namespace dg

extern "C" {

int dg_tile_variant_count(int p)
{
    if (p < 0 || p > DG_MAX_P) return 0;
    int n = 0, tx, ty, th;
    size_t sm;
    while (n < 8 && dg::tile_code_info((p + 1) * 8 + n, &tx, &ty, &th, &sm)) ++n;
    return n;
}

dg_status dg_set_tile_variant(int p, int variant)
{
    if (p < 0 || p > DG_MAX_P) return DG_ERR_UNSUPPORTED;
    if (variant < 0 || variant >= dg_tile_variant_count(p)) return DG_ERR_ARG;
    dg::g_tile_var[p + 1] = variant;
    return DG_OK;
}

int dg_get_tile_variant(int p) { return (p < 0 || p > DG_MAX_P) ? -1 : dg::g_tile_var[p + 1]; }

dg_status dg_set_stage_kernel(int p, int kind)
{
    if (p < 0 || p > DG_MAX_P) return DG_ERR_UNSUPPORTED;
    if (kind != DG_STAGE_TILE && kind != DG_STAGE_COLUMN && kind != DG_STAGE_LINES)
        return DG_ERR_ARG;
    dg::g_stage_kind[p + 1] = kind;
    return DG_OK;
}

int dg_get_stage_kernel(int p) { return (p < 0 || p > DG_MAX_P) ? -1 : dg::g_stage_kind[p + 1]; }

dg_status dg_tile_shape(int p, int variant, int *tx, int *ty)
{
    if (!tx || !ty) return DG_ERR_ARG;
    int th;
    size_t sm;
    if (p < 0 || p > DG_MAX_P || !dg::tile_code_info((p + 1) * 8 + variant, tx, ty, &th, &sm))
        return DG_ERR_ARG;
    return DG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batches: many independent float meshes advanced by one launch per stage
// ---------------------------------------------------------------------------
struct dg_batch {
    int n = 0;
    std::vector<dg::InstDev> inst;      // host copy of the descriptors
    std::vector<dg::LambdaItem> items;  // node ranges of the shared instances (time steps)
    std::vector<dg::LineItem> litems;   // their stage work items, grouped by order N
    std::vector<long long> dofs;
    dg::InstDev *d_inst = nullptr;
    dg::LambdaItem *d_items = nullptr;
    dg::LineItem *d_litems = nullptr;
    int lbeg[dg::NMAX + 1] = {}, lend[dg::NMAX + 1] = {};  // work items of order N
    double *d_dt = nullptr;
    unsigned long long *d_lam = nullptr;
    int *d_err = nullptr;
    double *d_partials = nullptr;
    std::vector<void *> qt;             // second states owned by the batch
    int grid = 1;                   // CTAs of the time-step launch
    // capacities of the reusable device arrays (dg_batch_update): d_dt, d_lam,
    // d_inst (elements); d_items; d_litems
    size_t cap_inst[3] = {0, 0, 0}, cap_items = 0, cap_litems = 0;
    bool small = true;              // every instance's offsets fit a 32-bit int
    std::vector<int> direct;        // large instances: launched by themselves
    // streams the large instances' stage launches run on, concurrently with
    // each other and with the shared launches (forked from and joined to
    // the caller's stream every step); lane_of[k]: the lane of direct[k]
    static constexpr int kLanes = 4;
    int nlanes = 0;
    int group_lane[dg::NMAX + 1] = {};  // lane of the shared instances of order N
    cudaStream_t lane[kLanes] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kLanes] = {};
    std::vector<int> lane_of;
    // recorded graphs of one step (ends with the copy back) and of two steps
    // (ends in Q by itself), and the cfl they were recorded with
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
    double graph_cfl[3] = {-1.0, -1.0, -1.0};
};

namespace {

void batch_free(dg_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    for (int k = 1; k <= 2; ++k)
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    for (int k = 0; k < dg_batch::kLanes; ++k) {
        if (b->lane[k]) cudaStreamDestroy(b->lane[k]);
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    for (void *p : b->qt) cudaFree(p);
    cudaFree(b->d_inst);
    cudaFree(b->d_items);
    cudaFree(b->d_litems);
    cudaFree(b->d_dt);
    cudaFree(b->d_lam);
    cudaFree(b->d_err);
    cudaFree(b->d_partials);
    delete b;
}

// Instances of at least this many nodes run their own launches of the
// single-mesh stage kernels (inside the batch's step and graph, on the
// batch's lanes); the smaller ones share the batched line-kernel launches.
// Process-wide, read by dg_batch_create (dg_set_batch_direct_nodes).
std::atomic<long long> g_direct_nodes{1LL << 13};

// The kernels of `nsteps` (1 or 2) steps on stream s.  Per step: the CFL
// time step of every instance (read from the buffer holding the state), then
// five fused stages alternating between Q and the second state Qt.  One step
// ends in Qt and is followed by a copy back into Q (one memcpy per
// instance); two steps end in Q by themselves.
cudaError_t batch_enqueue(const dg_batch *b, double cfl, int nsteps, cudaStream_t s)
{
    static const double kA[5] = {0.0,
                                 -567301805773.0 / 1357537059087.0,
                                 -2404267990393.0 / 2016746695238.0,
                                 -3550918686646.0 / 2091501179385.0,
                                 -1275806237668.0 / 842570457699.0};
    static const double kB[5] = {1432997174477.0 / 9575080441755.0,
                                 5161836677717.0 / 13612068292357.0,
                                 1720146321549.0 / 2090206949498.0,
                                 3134564353537.0 / 4481467310338.0,
                                 2277821191437.0 / 14882151754819.0};
    const int ni = (int)b->items.size();
    cudaError_t e = cudaSuccess;
    int parity = 0;  // 0: the state is in Q at the start of the step
    for (int step = 0; step < nsteps && e == cudaSuccess; ++step) {
        e = dg::batch_lambda(b->d_items, ni, b->d_inst, parity, b->d_err, b->grid, s);
        for (size_t k = 0; k < b->direct.size() && e == cudaSuccess; ++k) {
            const dg::InstDev &I = b->inst[b->direct[k]];
            e = dg::float_lambda(I.g, parity == 0 ? I.Q : I.Qt, I.lam_bits, b->d_err, s);
        }
        if (e == cudaSuccess) e = dg::batch_dt(b->d_inst, b->n, cfl, s);
        // the large instances' five stages on their lanes, after the time steps
        if (e == cudaSuccess && b->nlanes > 0) {
            e = cudaEventRecord(b->fork_ev, s);
            for (int l = 0; l < b->nlanes && e == cudaSuccess; ++l)
                e = cudaStreamWaitEvent(b->lane[l], b->fork_ev, 0);
        }
        for (size_t k = 0; k < b->direct.size() && e == cudaSuccess; ++k) {
            const dg::InstDev &I = b->inst[b->direct[k]];
            for (int st = 0; st < 5 && e == cudaSuccess; ++st) {
                const int par = parity ^ (st & 1);
                e = dg::float_stage(I.g, I.T, par == 0 ? I.Q : I.Qt, par == 0 ? I.Qt : I.Q, I.dQ,
                                    (float)kA[st], (float)kB[st], I.dt,
                                    b->nlanes > 0 ? b->lane[b->lane_of[k]] : s);
            }
        }
        // the shared instances: per order N one launch per stage (one CTA per
        // instance, column and z chunk), on the order's lane (or the caller's
        // stream when the batch has a single unit of work)
        for (int N = 1; N <= dg::NMAX && e == cudaSuccess; ++N) {
            if (b->lend[N] <= b->lbeg[N]) continue;
            cudaStream_t ls = (b->nlanes > 0 && b->group_lane[N] >= 0) ? b->lane[b->group_lane[N]] : s;
            for (int st = 0; st < 5 && e == cudaSuccess; ++st)
                e = dg::batch_line_stage(b->d_litems + b->lbeg[N], b->lend[N] - b->lbeg[N],
                                         b->d_inst, N, parity ^ (st & 1), (float)kA[st],
                                         (float)kB[st], b->small, ls);
        }
        for (int l = 0; l < b->nlanes && e == cudaSuccess; ++l) {
            e = cudaEventRecord(b->join_ev[l], b->lane[l]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join_ev[l], 0);
        }
        parity ^= 1;  // five stages
    }
    if (parity == 1)
        for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
            const dg::InstDev &I = b->inst[i];
            const int N = I.g.p + 1;
            const size_t bytes = (size_t)dg::NF * (size_t)I.g.E * N * N * N * sizeof(float);
            e = cudaMemcpyAsync(I.Q, I.Qt, bytes, cudaMemcpyDeviceToDevice, s);
        }
    return e;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

dg_status check_instances(int n, const dg_instance *desc)
{
    if (n < 1 || !desc) return DG_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const dg_instance &d = desc[i];
        if (d.nx < 1 || d.ny < 1 || d.nz < 1 || !d.Q || !d.dQ || d.Q == d.dQ) return DG_ERR_ARG;
        if (d.Qt && (d.Qt == d.Q || d.Qt == d.dQ || !aligned16(d.Qt))) return DG_ERR_ARG;
        if (!aligned16(d.Q) || !aligned16(d.dQ)) return DG_ERR_ARG;
        if (!finite_pos(d.Lx) || !finite_pos(d.Ly) || !finite_pos(d.Lz)) return DG_ERR_ARG;
        if (!std::isfinite(d.x0) || !std::isfinite(d.y0) || !std::isfinite(d.z0)) return DG_ERR_ARG;
        if (!(std::isfinite(d.gamma) && d.gamma > 1.0)) return DG_ERR_ARG;
        if (d.p < 0 || d.p > DG_MAX_P) return DG_ERR_UNSUPPORTED;
        const long long E = (long long)d.nx * d.ny * d.nz;
        if (E * (d.p + 1) * (d.p + 1) * (d.p + 1) >= (1LL << 40)) return DG_ERR_ARG;
    }
    return DG_OK;
}

// a device array of at least `need` elements, reallocated (grown by half)
// only when the current one is too small
template <typename T>
cudaError_t ensure(T **p, size_t *cap, size_t need)
{
    if (need <= *cap) return cudaSuccess;
    const size_t c = std::max(need, *cap + *cap / 2);
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc((void **)p, c * sizeof(T));
    if (e == cudaSuccess) *cap = c;
    return e;
}

// (Re)build the batch for the instance list desc (validated): descriptors,
// work lists, lanes; device buffers and streams of an earlier list are
// reused where large enough.  Recorded graphs are dropped.
dg_status batch_assign(dg_batch *b, int n, const dg_instance *desc)
{
    for (int k = 1; k <= 2; ++k) {
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
        b->exec[k] = nullptr;
        b->graph_cfl[k] = -1.0;
    }
    for (void *p : b->qt) cudaFree(p);
    b->qt.clear();
    const long long direct_nodes = g_direct_nodes.load();
    b->n = n;
    b->inst.assign(n, dg::InstDev{});
    b->dofs.clear();
    b->direct.clear();
    b->items.clear();
    b->litems.clear();
    b->lane_of.clear();
    b->small = true;
    b->nlanes = 0;
    for (int N = 0; N <= dg::NMAX; ++N) b->lbeg[N] = b->lend[N] = b->group_lane[N] = 0;
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < n && err == cudaSuccess; ++i) {
        const dg_instance &d = desc[i];
        const int N = d.p + 1;
        dg::InstDev &I = b->inst[i];
        std::memset(&I, 0, sizeof(I));
        dg::Geo &g = I.g;
        g.nx = d.nx; g.ny = d.ny; g.nz = d.nz; g.p = d.p;
        g.E = (long long)d.nx * d.ny * d.nz;
        g.x0 = d.x0; g.y0 = d.y0; g.z0 = d.z0;
        g.hx = d.Lx / d.nx; g.hy = d.Ly / d.ny; g.hz = d.Lz / d.nz;
        g.gamma = d.gamma;
        g.J = g.hx * g.hy * g.hz / 8.0;
        g.hmin = std::fmin(g.hx, std::fmin(g.hy, g.hz));
        Basis B;
        make_basis(N, B);
        for (int a = 0; a < N; ++a) {
            g.xi[a] = (double)B.x[a];
            g.w[a] = (double)B.w[a];
        }
        const double gf[3] = {2.0 / g.hx, 2.0 / g.hy, 2.0 / g.hz};
        fill_ops(B, gf, I.T);
        fill_gas(d.gamma, I.T);
        I.Q = (float *)d.Q;
        I.dQ = (float *)d.dQ;
        const size_t bytes = (size_t)dg::NF * (size_t)g.E * N * N * N * sizeof(float);
        void *qt = d.Qt;
        if (!qt) {
            err = cudaMalloc(&qt, bytes);
            if (err == cudaSuccess) b->qt.push_back(qt);  // the batch's own
        }
        I.Qt = (float *)qt;
        b->dofs.push_back(g.E * N * N * N);
        if ((long long)dg::NF * g.E * N * N * N > 0x7fffffffLL) b->small = false;
    }
    if (err == cudaSuccess) err = ensure(&b->d_dt, &b->cap_inst[0], (size_t)n);
    if (err == cudaSuccess) err = ensure(&b->d_lam, &b->cap_inst[1], (size_t)n);
    if (err == cudaSuccess) err = ensure(&b->d_inst, &b->cap_inst[2], (size_t)n);
    if (err == cudaSuccess) err = cudaMemset(b->d_lam, 0, sizeof(unsigned long long) * n);
    if (err != cudaSuccess) return cuda_status(err);
    // time-step work list: every shared instance's nodes in ranges of at
    // most kLambdaNodes
    for (int i = 0; i < n; ++i) {
        dg::InstDev &I = b->inst[i];
        I.dt = b->d_dt + i;
        I.lam_bits = b->d_lam + i;
        if (b->dofs[i] >= direct_nodes) {  // own launches
            b->direct.push_back(i);
            continue;
        }
        for (long long t = 0; t < b->dofs[i]; t += dg::kLambdaNodes)
            b->items.push_back({i, t, std::min(b->dofs[i], t + dg::kLambdaNodes)});
        int lx, ly;
        if (!dg::line_shape_info(I.g.p + 1, &lx, &ly)) return DG_ERR_UNSUPPORTED;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // stage work items: the line kernel's columns of the shared instances,
    // each cut into z chunks.  Per order N one chunk length for all its
    // instances, chosen as a single mesh's launch chooses it: the length that
    // minimises (waves of the GPU's resident CTAs) x (layers per chunk + the
    // chunk's extra prologue layer) over the order's columns.
    for (int N = 1; N <= dg::NMAX; ++N) {
        std::vector<int> members;
        int maxz = 0;
        for (int i = 0; i < n; ++i)
            if (b->inst[i].g.p + 1 == N && b->dofs[i] < direct_nodes) {
                members.push_back(i);
                maxz = std::max(maxz, b->inst[i].g.nz);
            }
        if (members.empty()) continue;
        int lx, ly;
        dg::line_shape_info(N, &lx, &ly);
        const int per_sm = dg::batch_line_blocks_per_sm(N, b->small);
        const long long resident = (long long)std::max(1, sms) * std::max(1, per_sm);
        auto ncols = [&](int i) {
            const dg::Geo &g = b->inst[i].g;
            return (long long)((g.nx + lx - 1) / lx) * ((g.ny + ly - 1) / ly);
        };
        int best_zc = maxz;
        double best = -1.0;
        for (int zc = 1; zc <= maxz; ++zc) {
            long long ctas = 0;
            for (int i : members) ctas += ncols(i) * ((b->inst[i].g.nz + zc - 1) / zc);
            const double cost = (double)((ctas + resident - 1) / resident) * (zc + 1);
            if (best < 0.0 || cost < best) { best = cost; best_zc = zc; }
        }
        b->lbeg[N] = (int)b->litems.size();
        for (int i : members) {
            const int zc = std::min(best_zc, b->inst[i].g.nz);
            const long long nblk = ncols(i) * ((b->inst[i].g.nz + zc - 1) / zc);
            if (nblk > 0x7fffffffLL) return DG_ERR_ARG;
            for (long long k = 0; k < nblk; ++k) b->litems.push_back({i, (int)k, zc});
        }
        b->lend[N] = (int)b->litems.size();
    }
    if (b->litems.size() > 0x7fffffffULL || b->items.size() > 0x7fffffffULL) return DG_ERR_ARG;
    err = ensure(&b->d_items, &b->cap_items, b->items.size());
    if (err == cudaSuccess) err = ensure(&b->d_litems, &b->cap_litems, b->litems.size());
    if (err == cudaSuccess)
        err = cudaMemcpy(b->d_inst, b->inst.data(), sizeof(dg::InstDev) * n, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && !b->items.empty())
        err = cudaMemcpy(b->d_items, b->items.data(), sizeof(dg::LambdaItem) * b->items.size(),
                         cudaMemcpyHostToDevice);
    if (err == cudaSuccess && !b->litems.empty())
        err = cudaMemcpy(b->d_litems, b->litems.data(), sizeof(dg::LineItem) * b->litems.size(),
                         cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return cuda_status(err);
    // grid of the time-step reduction: as many CTAs as fit
    const int ni = (int)b->items.size();
    b->grid = (int)std::max<long long>(1, std::min<long long>((long long)sms * 8, (long long)ni));
    // lanes: the units of stage work -- each large instance; and, when there
    // is no large instance, the shared instances of each order N (one launch
    // per stage) -- largest first onto the least loaded lane.  Next to large
    // instances the orders' launches stay on the caller's stream, where they
    // overlap the lanes.
    std::vector<long long> unit_dof;  // direct instances first, then the orders
    std::vector<int> unit_N;
    for (int k : b->direct) {
        unit_dof.push_back(b->dofs[k]);
        unit_N.push_back(0);
    }
    for (int N = 1; N <= dg::NMAX && b->direct.empty(); ++N) {
        if (b->lend[N] <= b->lbeg[N]) continue;
        long long d = 0;
        for (int i = 0; i < n; ++i)
            if (b->inst[i].g.p + 1 == N && b->dofs[i] < direct_nodes) d += b->dofs[i];
        unit_dof.push_back(d);
        unit_N.push_back(N);
    }
    for (int N = 0; N <= dg::NMAX; ++N) b->group_lane[N] = -1;
    b->lane_of.assign(b->direct.size(), 0);
    if (unit_dof.size() > 1) {
        b->nlanes = (int)std::min<size_t>(dg_batch::kLanes, unit_dof.size());
        std::vector<int> order(unit_dof.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return unit_dof[x] > unit_dof[y]; });
        std::vector<long long> load(b->nlanes, 0);
        for (int k : order) {
            const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            if (unit_N[k] == 0) b->lane_of[k] = l;
            else b->group_lane[unit_N[k]] = l;
            load[l] += unit_dof[k];
        }
        if (!b->fork_ev) err = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
        for (int l = 0; l < b->nlanes && err == cudaSuccess; ++l) {
            if (b->lane[l]) continue;  // made for an earlier list
            err = cudaStreamCreateWithFlags(&b->lane[l], cudaStreamNonBlocking);
            if (err == cudaSuccess) err = cudaEventCreateWithFlags(&b->join_ev[l], cudaEventDisableTiming);
        }
        if (err != cudaSuccess) return cuda_status(err);
    }
    return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_batch_create(int n, const dg_instance *desc, dg_batch **out)
{
    if (!out) return DG_ERR_ARG;
    *out = nullptr;
    dg_status st = check_instances(n, desc);
    if (st != DG_OK) return st;
    dg_batch *b = new (std::nothrow) dg_batch();
    if (!b) return DG_ERR_OOM;
    cudaError_t err = cudaMalloc((void **)&b->d_err, sizeof(int));
    if (err == cudaSuccess)
        err = cudaMalloc((void **)&b->d_partials, (size_t)dg::kNormBlocks * 8 * sizeof(double));
    if (err == cudaSuccess) err = cudaMemset(b->d_err, 0, sizeof(int));
    st = err == cudaSuccess ? batch_assign(b, n, desc) : cuda_status(err);
    if (st != DG_OK) {
        cudaGetLastError();  // clear a sticky allocation error
        batch_free(b);
        return st;
    }
    *out = b;
    return DG_OK;
}

dg_status dg_batch_update(dg_batch *b, int n, const dg_instance *desc)
{
    if (!b) return DG_ERR_ARG;
    dg_status st = check_instances(n, desc);
    if (st != DG_OK) return st;
    st = batch_assign(b, n, desc);
    if (st != DG_OK) {
        cudaGetLastError();  // clear a sticky allocation error
        // a half-built list is never stepped: the batch holds no instances
        b->n = 0;
        b->inst.clear();
        b->dofs.clear();
        b->direct.clear();
        b->items.clear();
        b->litems.clear();
        b->lane_of.clear();
        b->nlanes = 0;
        for (int N = 0; N <= dg::NMAX; ++N) b->lbeg[N] = b->lend[N] = 0;
    }
    return st;
}

void dg_batch_destroy(dg_batch *b) { batch_free(b); }

dg_status dg_set_batch_direct_nodes(int64_t nodes)
{
    if (nodes < 0) return DG_ERR_ARG;
    g_direct_nodes.store((long long)nodes);
    return DG_OK;
}

int64_t dg_get_batch_direct_nodes(void) { return (int64_t)g_direct_nodes.load(); }

dg_status dg_batch_sizes(const dg_batch *b, int64_t *n_dof, int64_t *n_items)
{
    if (!b) return DG_ERR_ARG;
    long long s = 0;
    for (long long d : b->dofs) s += d;
    if (n_dof) *n_dof = s;
    if (n_items) *n_items = (int64_t)b->litems.size();
    return DG_OK;
}

dg_status dg_batch_state_init(const dg_batch *b, int idx, dg_init_kind kind, const double *params,
                              int nparams, void *stream)
{
    if (!b || idx < 0 || idx >= b->n) return DG_ERR_ARG;
    int need = kind == DG_INIT_UNIFORM ? 5 : kind == DG_INIT_VORTEX ? 7 : kind == DG_INIT_TGV ? 3 : -1;
    if (need < 0 || nparams < need || nparams > 8 || !params) return DG_ERR_ARG;
    double pr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < nparams; ++i) {
        if (!std::isfinite(params[i])) return DG_ERR_ARG;
        pr[i] = params[i];
    }
    dg::Work w;
    return cuda_status(dg::Launch<float>::init(b->inst[idx].g, kind, pr, b->inst[idx].Q, w,
                                               as_stream(stream)));
}

dg_status dg_batch_step(dg_batch *b, double cfl, int nsteps, int use_graph, void *stream)
{
    if (!b || !finite_pos(cfl) || nsteps < 0) return DG_ERR_ARG;
    if (b->n == 0) return DG_OK;  // no instances (after a failed dg_batch_update)
    cudaStream_t s = as_stream(stream);
    if (!use_graph) {
        cudaError_t e = cudaSuccess;
        for (int k = nsteps; k > 0 && e == cudaSuccess; k -= 2)
            e = batch_enqueue(b, cfl, k >= 2 ? 2 : 1, s);
        return cuda_status(e);
    }
    if (!s) return DG_ERR_ARG;  // capture needs a created stream, not the legacy default
    for (int k = nsteps; k > 0; k -= 2) {
        const int n = k >= 2 ? 2 : 1;
        if (!b->exec[n] || b->graph_cfl[n] != cfl) {
            if (b->exec[n]) {
                cudaGraphExecDestroy(b->exec[n]);
                b->exec[n] = nullptr;
            }
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return DG_ERR_CUDA;
            cudaError_t ek = batch_enqueue(b, cfl, n, s);
            e = cudaStreamEndCapture(s, &graph);
            if (ek != cudaSuccess || e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return DG_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&b->exec[n], graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                b->exec[n] = nullptr;
                return DG_ERR_CUDA;
            }
            b->graph_cfl[n] = cfl;
        }
        cudaError_t e = cudaGraphLaunch(b->exec[n], s);
        if (e != cudaSuccess) return DG_ERR_CUDA;
    }
    return DG_OK;
}

dg_status dg_batch_dt(const dg_batch *b, double *dt_host)
{
    if (!b || !dt_host) return DG_ERR_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(dt_host, b->d_dt, sizeof(double) * b->n, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

dg_status dg_batch_norms(const dg_batch *b, int idx, const void *Qref, double *out, void *stream)
{
    if (!b || idx < 0 || idx >= b->n || !out) return DG_ERR_ARG;
    dg::Work w;
    w.partials = b->d_partials;
    return cuda_status(dg::Launch<float>::norms(b->inst[idx].g, b->inst[idx].Q,
                                                (const float *)Qref, out, w, as_stream(stream)));
}

dg_status dg_batch_last_error(const dg_batch *b)
{
    if (!b) return DG_ERR_ARG;
    int flag = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return DG_ERR_CUDA;
    return flag ? DG_ERR_NONFINITE : DG_OK;
}

const char *dg_status_string(dg_status s)
{
    switch (s) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_UNSUPPORTED: return "unsupported polynomial degree";
    case DG_ERR_OOM: return "device allocation failed";
    case DG_ERR_CUDA: return "CUDA error";
    case DG_ERR_NONFINITE: return "non-positive or non-finite density or pressure";
    case DG_ERR_BOUNDS: return "index out of bounds";
    case DG_ERR_TIMEOUT: return "timeout";
    case DG_ERR_TOO_LARGE: return "problem larger than the static scratch of dg_rhs_static";
    }
    return "unknown status";
}

dg_status dg_profile_begin(dg_mesh *m)
{
    if (!m) return DG_ERR_ARG;
    dg::Prof &p = *m->prof;
    for (cudaEvent_t e : p.ev) p.pool.push_back(e);
    p.ev.clear();
    p.kind.clear();
    p.on = true;
    return DG_OK;
}

dg_status dg_profile_end(dg_mesh *m, double *ms, int64_t *launches)
{
    if (!m || !ms || !launches) return DG_ERR_ARG;
    dg::Prof &p = *m->prof;
    p.on = false;
    for (int k = 0; k < DG_PROFILE_KINDS; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    if (p.ev.size() != 2 * p.kind.size()) return DG_ERR_CUDA;
    for (size_t i = 0; i < p.kind.size(); ++i) {
        if (cudaEventSynchronize(p.ev[2 * i + 1]) != cudaSuccess) return DG_ERR_CUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1]) != cudaSuccess) return DG_ERR_CUDA;
        const int k = p.kind[i];
        if (k >= 0 && k < DG_PROFILE_KINDS) {
            ms[k] += t;
            launches[k] += 1;
        }
    }
    for (cudaEvent_t e : p.ev) p.pool.push_back(e);
    p.ev.clear();
    p.kind.clear();
    return DG_OK;
}

dg_status dg_last_error(const dg_mesh *m)
{
    if (!m) return DG_ERR_ARG;
    int flag = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, m->work.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(m->work.err, 0, sizeof(int));
    if (e != cudaSuccess) return DG_ERR_CUDA;
    return flag ? DG_ERR_NONFINITE : DG_OK;
}

}  // extern "C"
