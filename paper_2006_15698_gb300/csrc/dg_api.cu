// dg_api.cu -- host side of the C ABI declared in include/dg.h: argument
// checks, the 1D operators of the collocated Gauss-Legendre basis, the mesh
// handle's device workspace, and dispatch to the per-precision launchers.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "dg_internal.h"

struct dg_mesh {
    dg::Geo geo;
    dg_precision prec;
    dg::Ops<double> ops64;
    dg::Ops<float> ops32;
    dg::Work work;
    dg::Prof *prof;
    int device;
    size_t ws_bytes;
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
    cudaFree(m->work.partials);
    cudaFree(m->work.lam_bits);
    cudaFree(m->work.err);
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
    dg::Work w = m->work;
    cudaError_t e = m->prec == DG_FP64
                        ? dg::Launch<double>::rk_step(m->geo, m->ops64, (double *)Q, (double *)dQ,
                                                      dt_dev, w, as_stream(stream))
                        : dg::Launch<float>::rk_step(m->geo, m->ops32, (float *)Q, (float *)dQ,
                                                     dt_dev, w, as_stream(stream));
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
    const size_t esz = precision == DG_FP64 ? sizeof(double) : sizeof(float);
    const double need = 3.0 * dg::NF * (double)E * N * N * (double)esz;
    if (need > (double)DG_STATIC_SCRATCH_BYTES) return DG_ERR_TOO_LARGE;

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
    cudaError_t e = static_scratch_address(&w.face_flux);
    if (e != cudaSuccess) return DG_ERR_CUDA;
    if (precision == DG_FP64) {
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
