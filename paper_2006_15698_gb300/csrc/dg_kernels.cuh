// dg_kernels.cuh -- sm_103a kernels of the DG Euler right-hand side and its
// low-storage Runge-Kutta update, templated on the polynomial order and the
// scalar type.  Included by one translation unit per scalar type.
//
// One right-hand-side evaluation (Sec. II.B, Eq. 5 with collocated
// Gauss-Legendre quadrature) is two kernels:
//
//   face_flux_kernel   every unique face point of the mesh, once: the traces
//                      of the two neighbouring elements' polynomials
//                      (interpolated along the face-normal node line), and the
//                      local Lax-Friedrichs flux between them -> flux buffer.
//   volume_kernel      every node, once: the Euler flux vectors at the node
//                      (Eq. 2-3), the sum-factorised weak derivative
//                      sum_a D[i][a] F_a along each direction (staged through
//                      shared memory), the lift of the six face fluxes, and
//                      either the right-hand side itself or the RK stage
//                      update of (dQ, Q) in place.
//
// Every floating-point operation of the method is done exactly once per
// face point or node (no recomputation of traces or interface fluxes), which
// is what matters on this GPU's narrow FP64 pipe.  The in-place stage update
// is race-free because the only cross-element data of a stage (the interface
// fluxes) is complete before volume_kernel starts.
#pragma once

#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

#include "dg_internal.h"

namespace dg {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

template <int N>
struct Tile {
    static constexpr int N2 = N * N;
    static constexpr int N3 = N * N * N;
    // elements per CTA of volume_kernel: about 256 threads (one per node)
    // (p = 4: two elements, 250 threads, so that three CTAs of the FP64
    // volume kernel fit an SM's registers)
    static constexpr int EPB = N3 >= 128 ? 1 : (N3 >= 100 ? 2 : (N3 >= 64 ? 4 : (256 / N3)));
    // operator tables staged per CTA: D[3][N][N], Lp[3][N], Lm[3][N]
    static constexpr int OPS = 3 * N * N + 6 * N;
    static constexpr int THREADS = ((EPB * N3 + 31) / 32) * 32;
};

// index of (field n, element e, in-element node) in a state array
__device__ __forceinline__ long long sidx(int n, long long e, int node, long long E, int N3)
{
    return ((long long)n * E + e) * N3 + node;
}

// index in the interface-flux buffer F[d][n][e][face point]; the buffer
// holds twice the Lax-Friedrichs flux (the 1/2 is in the lift vectors)
__device__ __forceinline__ long long fidx(int d, int n, long long e, int pt, long long E, int N2)
{
    return ((long long)(d * NF + n) * E + e) * N2 + pt;
}

// periodic neighbour of element e in direction DIR, side +1 or -1
template <int DIR>
__device__ __forceinline__ long long neighbour(long long e, int side, const Geo &g)
{
    const long long nx = g.nx, nxy = (long long)g.nx * g.ny;
    if (DIR == 0) {
        long long ex = e % nx;
        if (side > 0) return ex == nx - 1 ? e - (nx - 1) : e + 1;
        return ex == 0 ? e + (nx - 1) : e - 1;
    } else if (DIR == 1) {
        long long ey = (e / nx) % g.ny;
        if (side > 0) return ey == g.ny - 1 ? e - (g.ny - 1) * nx : e + nx;
        return ey == 0 ? e + (g.ny - 1) * nx : e - nx;
    } else {
        long long ez = e / nxy;
        if (side > 0) return ez == g.nz - 1 ? e - (g.nz - 1) * nxy : e + nxy;
        return ez == 0 ? e + (g.nz - 1) * nxy : e - nxy;
    }
}

// ---------------------------------------------------------------------------
// Euler physics (Eq. 2-3) and the local Lax-Friedrichs flux
// ---------------------------------------------------------------------------

// 1/x for the positive densities of the flux evaluations.  Double: the
// hardware reciprocal approximation refined by two Newton-Raphson steps
// r <- r + r(1 - x r) (each squares the relative error, so the approximation's
// error falls below double rounding: the result is within 1 ulp of 1/x),
// four FMAs instead of a correctly rounded division.  Float: plain division.
__device__ __forceinline__ double recip(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }

// sqrt(a) for the positive, finite, normal a = gamma p / rho of the sound
// speed, on the FP64 pipe with fewer instructions than the correctly rounded
// square root: the hardware reciprocal-square-root approximation y ~ a^-1/2
// (rsqrt.approx.ftz.f64) starts the coupled iteration for g ~ sqrt(a) and
// h ~ 1/(2 sqrt(a)) (Goldschmidt's square-root iteration, as in P. Markstein,
// "IA-64 and Elementary Functions", Prentice Hall 2000): g = a y, h = y/2,
// r = 1/2 - g h, g <- g + g r, h <- h + h r (each squares the relative
// error), then one correction g <- g + h (a - g^2) with the residual formed
// exactly by an FMA.  The result is within one ulp of the correctly rounded
// root (checked against CUDA's sqrt on a sweep of inputs, dg_selfcheck_sqrt).
// a = 0 gives NaN (a zero pressure, which the time-step reduction reports as
// non-physical).
__device__ __forceinline__ double sqrt_pos(double a)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
    double g = a * y, h = 0.5 * y;
    const double r = fma(-g, h, 0.5);
    g = fma(g, r, g);
    h = fma(h, r, h);
    const double d = fma(-g, g, a);
    return fma(d, h, g);
}

// Local Lax-Friedrichs (Rusanov) flux through a face with normal +e_DIR,
// qL on the -side, qR on the +side (Sec. II.B; local dissipation speed):
//   F* = (F(qL) + F(qR))/2 - max(|u_n| + c)/2 (qR - qL)
// Returned as 2 F* (the factor 1/2 is folded into the lift vectors).  Each
// side's 1/rho, pressure and normal velocity are formed first and every flux
// component is evaluated where it is combined with the dissipation, so fewer
// values are live at once (the kernel's occupancy is register bound).
// (Double: one reciprocal 1/(rhoL rhoR) serves both densities, and the
// sound speeds use sqrt_pos; each result within a few ulp of the plain
// formulas, well inside the FP64 form's tolerance.)
template <int DIR, typename real>
__device__ __forceinline__ void lf_flux2(const real qL[NF], const real qR[NF], real gamma,
                                         real gm1, real f[NF])
{
    real rL, rR;
    if constexpr (sizeof(real) == 8) {
        const real rr = recip(qL[0] * qR[0]);
        rL = qR[0] * rr;
        rR = qL[0] * rr;
    } else {
        rL = recip(qL[0]);
        rR = recip(qR[0]);
    }
    const real pL = gm1 * (qL[4] - real(0.5) * (qL[1] * qL[1] + qL[2] * qL[2] + qL[3] * qL[3]) * rL);
    const real pR = gm1 * (qR[4] - real(0.5) * (qR[1] * qR[1] + qR[2] * qR[2] + qR[3] * qR[3]) * rR);
    const real uL = qL[1 + DIR] * rL, uR = qR[1 + DIR] * rR;
    real cL, cR;
    if constexpr (sizeof(real) == 8) {
        cL = sqrt_pos(gamma * pL * rL);
        cR = sqrt_pos(gamma * pR * rR);
    } else {
        cL = sqrt(gamma * pL * rL);
        cR = sqrt(gamma * pR * rR);
    }
    const real lam = fmax(fabs(uL) + cL, fabs(uR) + cR);
    // F(q)_n = q_n u_n (+ p for the normal momentum, + p u_n for the energy),
    // so F(qL)_n + F(qR)_n - lam (qR_n - qL_n) = qL_n (uL + lam) + qR_n (uR -
    // lam) + pressure terms: two FMA-pipe instructions per component instead
    // of four (the face kernel is FP64-pipe bound)
    const real aL = uL + lam, aR = uR - lam;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        if (n == DIR + 1) f[n] = fma(qL[n], aL, fma(qR[n], aR, pL + pR));
        else f[n] = fma(qL[n], aL, qR[n] * aR);
    }
    f[4] = fma(qL[4], aL, fma(pL, uL, fma(qR[4], aR, pR * uR)));
}

// ---------------------------------------------------------------------------
// interface fluxes
// ---------------------------------------------------------------------------

// Trace sum_c l[c] a[c * stride] of a face-normal node line (double form),
// every operation explicitly rounded in a fixed order, so that every kernel
// computing the trace of the same line (the face kernel, the z-slab trace
// kernel) gets the same value bit for bit.  (The float kernels' traces are
// line_dot, dg_column.cuh.)
template <int N>
__device__ __forceinline__ double trace_line(const double *l, const double *__restrict__ a,
                                             int stride)
{
    double s = __dmul_rn(l[0], __ldg(a));
#pragma unroll
    for (int c = 1; c < N; ++c) s = __fma_rn(l[c], __ldg(a + c * stride), s);
    return s;
}

// One thread per (direction, element, face point) of the element's +DIR face.
// Face point pt = t2*N + t1 where (t1, t2) are the two tangential node indices
// in (i, j, k) order.  The element is the left state, its +DIR neighbour the
// right state; each unique face of the periodic mesh is visited once.
// z slabs (g.zlo set): the +z face of the last layer takes its right state
// from the halo zhi, and layer 0's threads also evaluate their -z face
// (left state from the halo zlo) into g.zflux, with the same code.
template <int N, int DIR, typename real, bool HALO>
__device__ __forceinline__ void face_point(const real *__restrict__ Q, real *__restrict__ F,
                                           const Ops<real> &T, const Geo &g, long long e, int pt)
{
    constexpr int N2 = N * N, N3 = N * N * N;
    const int t1 = pt % N, t2 = pt / N;
    const int base = DIR == 0 ? (t2 * N + t1) * N : (DIR == 1 ? t2 * N2 + t1 : t2 * N + t1);
    constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? N : N2);
    const long long plane = (long long)g.nx * g.ny;
    const long long ez = DIR == 2 ? e / plane : 0;
    const bool slab = HALO && DIR == 2 && g.zlo != nullptr;
    const int faces = slab && ez == 0 ? 2 : 1;
#pragma unroll 1
    for (int side = 0; side < faces; ++side) {
        // side 0: the +DIR face (this element left); side 1: the -z face of
        // layer 0 of a slab (this element right, the halo left)
        real qL[NF], qR[NF];
        const long long en = neighbour<DIR>(e, +1, g);
        const long long h = ((long long)0 * plane + (e - ez * plane)) * N2 + pt;  // halo index of field 0
#pragma unroll
        for (int n = 0; n < NF; ++n) {
            const real *a = Q + sidx(n, e, base, g.E, N3);
            if (side == 0) {
                qL[n] = trace_line<N>(T.lp, a, stride);
                if (slab && ez == g.nz - 1)
                    qR[n] = static_cast<const real *>(g.zhi)[h + (long long)n * plane * N2];
                else
                    qR[n] = trace_line<N>(T.lm, Q + sidx(n, en, base, g.E, N3), stride);
            } else {
                qL[n] = static_cast<const real *>(g.zlo)[h + (long long)n * plane * N2];
                qR[n] = trace_line<N>(T.lm, a, stride);
            }
        }
        real f[NF];
        lf_flux2<DIR>(qL, qR, T.gamma, T.gm1, f);
        if (side == 0) {
#pragma unroll
            for (int n = 0; n < NF; ++n) F[fidx(DIR, n, e, pt, g.E, N2)] = f[n];
        } else {
#pragma unroll
            for (int n = 0; n < NF; ++n)
                static_cast<real *>(g.zflux)[h + (long long)n * plane * N2] = f[n];
        }
    }
}

// CTA shape of face_flux_kernel: EF consecutive elements and all three of
// their + faces, so each element's nodes are fetched from DRAM once and
// reused from L1 for its three directions.  Each direction owns a segment of
// SEG threads (EF N^2 face points rounded up to whole warps) so that every
// warp runs one direction's code path: on the narrow FP64 pipe a warp split
// across two directions would pay for both.
template <int N>
struct FaceTile {
    static constexpr int N2 = N * N;
    static constexpr int EF = N == 1 ? 32 : N == 2 ? 16 : N == 3 ? 7 : N == 4 ? 4 : N == 5 ? 5
                            : N == 6 ? 7 : 5;
    static constexpr int SEG = ((EF * N2 + 31) / 32) * 32;
    static constexpr int THREADS = 3 * SEG;
};

template <int N, typename real, bool HALO>
__global__ void __launch_bounds__(FaceTile<N>::THREADS, 1152 / FaceTile<N>::THREADS)
    face_flux_kernel(const real *__restrict__ Q, real *__restrict__ F, const Ops<real> T,
                     const Geo g, long long e_begin, long long e_end)
{
    constexpr int N2 = N * N, EF = FaceTile<N>::EF, SEG = FaceTile<N>::SEG;
    const int d = threadIdx.x / SEG;
    const int r = threadIdx.x - d * SEG;
    if (r >= EF * N2) return;
    const int el = r / N2;
    const int pt = r - el * N2;
    const long long e = e_begin + (long long)blockIdx.x * EF + el;
    if (e >= e_end) return;
    if (d == 0) face_point<N, 0, real, HALO>(Q, F, T, g, e, pt);
    else if (d == 1) face_point<N, 1, real, HALO>(Q, F, T, g, e, pt);
    else face_point<N, 2, real, HALO>(Q, F, T, g, e, pt);
}

// ---------------------------------------------------------------------------
// volume term, lift and stage update
// ---------------------------------------------------------------------------

// MODE 0: write R = dQ/dt.   MODE 1: LSERK stage, dQ <- A dQ + dt R,
// Q <- Q + B dQ, in place (first stage: A == 0 and dQ is not read).
template <int N, typename real, int MODE, bool HALO>
__global__ void __launch_bounds__(Tile<N>::THREADS)
    volume_kernel(const real *Qin, real *Out, real *dQ, const real *__restrict__ F,
                  const Ops<real> T, const Geo g, real A, real B, const double *__restrict__ dt,
                  long long e_begin, long long e_end)
{
    constexpr int N2 = N * N, N3 = N * N * N, EPB = Tile<N>::EPB;
    extern __shared__ unsigned char smem_raw[];
    real *sF = reinterpret_cast<real *>(smem_raw);  // [EPB][3][NF][N3]
    real *sD = sF + (size_t)EPB * 3 * NF * N3;        // [3][N][N]
    real *sLp = sD + 3 * N2;                           // [3][N]
    real *sLm = sLp + 3 * N;                           // [3][N]

    const int tid = threadIdx.x;
    const int el = tid / N3;
    const int node = tid - el * N3;
    const long long e = e_begin + (long long)blockIdx.x * EPB + el;
    const bool active = el < EPB && e < e_end;
    const int i = node % N, j = (node / N) % N, k = node / N2;

    // the operators, scaled once per CTA by dt for the stage update (so the
    // accumulated value is already dt * R) and by 1 for the rhs
    for (int t = tid; t < Tile<N>::OPS; t += blockDim.x) {
        const real sc = MODE == 1 ? real(*dt) : real(1);
        if (t < 3 * N2) sD[t] = sc * (&T.D[0][0][0])[(t / N2) * NMAX * NMAX + ((t % N2) / N) * NMAX + t % N];
        else if (t < 3 * N2 + 3 * N) { const int u = t - 3 * N2; sLp[u] = sc * T.Lp[u / N][u % N]; }
        else { const int u = t - 3 * N2 - 3 * N; sLm[u] = sc * T.Lm[u / N][u % N]; }
    }

    real q[NF];
    if (active) {
#pragma unroll
        for (int n = 0; n < NF; ++n) q[n] = Qin[sidx(n, e, node, g.E, N3)];
        // fluxes at this node (Eq. 2 with the closure of Eq. 3)
        const real gm1 = T.gm1;
        const real rinv = recip(q[0]);
        const real u = q[1] * rinv, v = q[2] * rinv, w = q[3] * rinv;
        const real p = gm1 * (q[4] - real(0.5) * (q[1] * u + q[2] * v + q[3] * w));
        const real ep = q[4] + p;
        real *s = sF + (size_t)el * 3 * NF * N3 + node;
        s[(0 * NF + 0) * N3] = q[1];
        s[(0 * NF + 1) * N3] = q[1] * u + p;
        s[(0 * NF + 2) * N3] = q[2] * u;
        s[(0 * NF + 3) * N3] = q[3] * u;
        s[(0 * NF + 4) * N3] = ep * u;
        s[(1 * NF + 0) * N3] = q[2];
        s[(1 * NF + 1) * N3] = q[1] * v;
        s[(1 * NF + 2) * N3] = q[2] * v + p;
        s[(1 * NF + 3) * N3] = q[3] * v;
        s[(1 * NF + 4) * N3] = ep * v;
        s[(2 * NF + 0) * N3] = q[3];
        s[(2 * NF + 1) * N3] = q[1] * w;
        s[(2 * NF + 2) * N3] = q[2] * w;
        s[(2 * NF + 3) * N3] = q[3] * w + p;
        s[(2 * NF + 4) * N3] = ep * w;
    }
    __syncthreads();
    if (!active) return;

    const long long exm = neighbour<0>(e, -1, g);
    const long long eym = neighbour<1>(e, -1, g);
    const long long ezm = neighbour<2>(e, -1, g);
    // z slabs: the -z face flux of layer 0 comes from the face kernel's zflux
    const long long plane = (long long)g.nx * g.ny;
    const real *fzm = F + fidx(2, 0, ezm, j * N + i, g.E, N2);
    long long fzm_stride = g.E * N2;  // between fields
    if (HALO && g.zflux != nullptr && e < plane) {
        fzm = static_cast<const real *>(g.zflux) + e * N2 + j * N + i;
        fzm_stride = plane * N2;
    }
    const int px = k * N + j, py = k * N + i, pz = j * N + i;
    const real *Dx = sD + 0 * N2 + i * N, *Dy = sD + 1 * N2 + j * N, *Dz = sD + 2 * N2 + k * N;

#pragma unroll
    for (int n = 0; n < NF; ++n) {
        const real *sx = sF + ((size_t)el * 3 + 0) * NF * N3 + n * N3;
        const real *sy = sF + ((size_t)el * 3 + 1) * NF * N3 + n * N3;
        const real *sz = sF + ((size_t)el * 3 + 2) * NF * N3 + n * N3;
        real acc = real(0);
        // sum-factorised weak derivative along x, y, z
#pragma unroll
        for (int a = 0; a < N; ++a) acc += Dx[a] * sx[(k * N + j) * N + a];
#pragma unroll
        for (int b = 0; b < N; ++b) acc += Dy[b] * sy[(k * N + b) * N + i];
#pragma unroll
        for (int c = 0; c < N; ++c) acc += Dz[c] * sz[(c * N + j) * N + i];
        // lift of the six interface fluxes (outward normal -> sign)
        acc -= sLp[0 * N + i] * __ldg(F + fidx(0, n, e, px, g.E, N2));
        acc += sLm[0 * N + i] * __ldg(F + fidx(0, n, exm, px, g.E, N2));
        acc -= sLp[1 * N + j] * __ldg(F + fidx(1, n, e, py, g.E, N2));
        acc += sLm[1 * N + j] * __ldg(F + fidx(1, n, eym, py, g.E, N2));
        acc -= sLp[2 * N + k] * __ldg(F + fidx(2, n, e, pz, g.E, N2));
        acc += sLm[2 * N + k] * __ldg(fzm + n * fzm_stride);

        const long long o = sidx(n, e, node, g.E, N3);
        if (MODE == 0) {
            Out[o] = acc;
        } else {
            // acc already carries dt (scaled operators)
            const real d = A == real(0) ? acc : A * dQ[o] + acc;
            dQ[o] = d;
            Out[o] = q[n] + B * d;
        }
    }
}

#include "dg_fused.cuh"
#include "dg_column.cuh"
#include "dg_lines.cuh"

// z slabs: the face traces a slab sends to its neighbours, one thread per
// (column element, face point): lo = layer 0's traces at its -z end,
// hi = the last layer's traces at its +z end, in the halo layout
// [NF][nx*ny][N^2], with the stage kernels' own trace arithmetic (double:
// trace_line as face_point; float: line_dot as the column kernels).
template <int N, typename real>
__global__ void __launch_bounds__(256) ztraces_kernel(const real *__restrict__ Q, real *lo,
                                                      real *hi, const Ops<real> T, const Geo g)
{
    constexpr int N2 = N * N, N3 = N * N * N;
    const long long plane = (long long)g.nx * g.ny;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= plane * N2) return;
    const long long col = t / N2;
    const int pt = (int)(t - col * N2);
    const long long top = col + (long long)(g.nz - 1) * plane;
#pragma unroll
    for (int n = 0; n < NF; ++n) {
        const real *a = Q + sidx(n, col, pt, g.E, N3), *b = Q + sidx(n, top, pt, g.E, N3);
        if constexpr (std::is_same<real, double>::value) {
            lo[(n * plane + col) * N2 + pt] = trace_line<N>(T.lm, a, N2);
            hi[(n * plane + col) * N2 + pt] = trace_line<N>(T.lp, b, N2);
        } else {
            float va[N], vb[N];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                va[c] = __ldg(a + c * N2);
                vb[c] = __ldg(b + c * N2);
            }
            lo[(n * plane + col) * N2 + pt] = line_dot<N>(T.lm, va);
            hi[(n * plane + col) * N2 + pt] = line_dot<N>(T.lp, vb);
        }
    }
}

// ---------------------------------------------------------------------------
// time step, integrals, initial states
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Wave-speed sum sum_d (|u_d| + c) of one node; false for rho <= 0, p <= 0 or NaN.
// Double state: every operation explicitly rounded (no FMA contraction) in a
// fixed order, so a node's speed is the same double on any conforming
// implementation of IEEE-754 arithmetic.
__device__ __forceinline__ bool node_speed(double r, double mx, double my, double mz, double E,
                                           double gamma, double &s)
{
    const double u = __ddiv_rn(mx, r), v = __ddiv_rn(my, r), w = __ddiv_rn(mz, r);
    const double uu = __dadd_rn(__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)), __dmul_rn(w, w));
    const double p = __dmul_rn(gamma - 1.0, __dsub_rn(E, __dmul_rn(__dmul_rn(0.5, r), uu)));
    if (!(r > 0.0) || !(p > 0.0)) return false;
    const double c = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), r));
    s = __dadd_rn(__dadd_rn(__dadd_rn(fabs(u), c), __dadd_rn(fabs(v), c)), __dadd_rn(fabs(w), c));
    return true;
}
// (float state: node_speed_f, with the float form's kernels)

// Float estimate of a double node's wave-speed sum, used only to skip the
// exact evaluation of nodes that cannot hold the maximum.  Returns true when
// the estimate is within kSpeedTol relative of the exact speed: every input
// inside [1e-9, 1e9] in magnitude (density) or below 1e9 (momenta, energy),
// so nothing overflows or goes subnormal in float; p >= E/100, so the
// cancellation E - |m|^2/(2 rho) costs at most a factor 100 (float relative
// error of p below 3e-5 for gamma <= 5/3, of c below half that); and a speed
// above 1e-20.  Any other node (including NaN, rho <= 0 or p <= 0) is
// evaluated exactly.
constexpr float kSpeedTol = 6e-5f;
__device__ __forceinline__ bool node_speed_estimate(double r, double mx, double my, double mz,
                                                    double E, float gamma, float &s)
{
    const float rf = (float)r, xf = (float)mx, yf = (float)my, zf = (float)mz, ef = (float)E;
    const float rinv = fast_rcp(rf);
    const float u = xf * rinv, v = yf * rinv, w = zf * rinv;
    const float p = (gamma - 1.0f) * (ef - 0.5f * rf * (u * u + v * v + w * w));
    const float c = fast_sqrt(gamma * p * rinv);
    s = (fabsf(u) + c) + (fabsf(v) + c) + (fabsf(w) + c);
    const float big = 1e9f;
    return rf >= 1e-9f && rf <= big && fabsf(xf) <= big && fabsf(yf) <= big &&
           fabsf(zf) <= big && fabsf(ef) <= big && p >= 0.01f * ef && s >= 1e-20f;
}

// One warp-synchronous step of the double-state Lambda reduction (all 32
// lanes call it together; `in` marks the lanes that hold a node).
//
// The exact speed (IEEE divisions and square root) costs about fifty
// FP64-pipe instructions, so each warp first estimates its 32 nodes' speeds
// in float and keeps R, the running maximum of its well-conditioned
// estimates.  Only nodes whose estimate reaches R (1 - 8 kSpeedTol), and the
// nodes without a trustworthy estimate, are evaluated exactly.  The node x
// holding the exact maximum S is always among them: its estimate is at least
// S (1 - tol) while R is at most S (1 + tol), and (1 - tol) >= (1 + tol)
// (1 - 8 tol).  The result is therefore the same double as the full
// evaluation, bit for bit.
__device__ __forceinline__ void pruned_speed_step(bool in, double r, double mx, double my,
                                                  double mz, double E, double gamma, float &R,
                                                  double &m, bool &bad)
{
    const float keep = 1.0f - 8.0f * kSpeedTol;
    float sf = 0.0f;
    bool ok = false;
    if (in) ok = node_speed_estimate(r, mx, my, mz, E, (float)gamma, sf);
    float wm = ok ? sf : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    R = fmaxf(R, wm);
    if (in && (!ok || sf >= R * keep)) {
        double s;
        if (node_speed(r, mx, my, mz, E, gamma, s)) m = fmax(m, s);
        else bad = true;
    }
}

// NaN-propagating block maximum of non-negative doubles (compared as bit
// patterns) merged into *lam_bits; a thread that saw a bad node raises *err
// and contributes a NaN, whose bit pattern is above every finite value.
// Called by every thread of the block (blockDim.x <= 256).
__device__ __forceinline__ void block_lambda(double m, bool bad, unsigned long long *lam_bits,
                                             int *err)
{
    __shared__ unsigned long long redb[8];
    if (bad) {
        atomicOr(err, 1);
        m = __longlong_as_double(0x7ff8000000000000LL);
    }
    unsigned long long b = (unsigned long long)__double_as_longlong(m);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
        b = x > b ? x : b;
    }
    if ((threadIdx.x & 31) == 0) redb[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long mb = redb[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mb = redb[w] > mb ? redb[w] : mb;
        atomicMax(lam_bits, mb);
    }
}

// Lambda = max over nodes of sum_d (|u_d| + c), reduced in double; a node with
// rho <= 0, p <= 0 or NaN contributes a NaN and raises the error flag.
// Double state: the float pre-filter above; float state: node speeds in float.
template <typename real>
__global__ void __launch_bounds__(256) cfl_kernel(const real *__restrict__ Q, long long nodes,
                                                  long long t_begin, long long t_end,
                                                  double gamma, unsigned long long *lam_bits,
                                                  int *err)
{
    // nodes t_begin .. t_end - 1 of every field (field stride: nodes)
    double m = 0.0;
    bool bad = false;
    if constexpr (std::is_same<real, double>::value) {
        const int lane = threadIdx.x & 31;
        const long long stride = (long long)gridDim.x * blockDim.x;  // a multiple of 32
        float R = 0.0f;
        // whole warps walk the nodes together, so the shuffles stay convergent
        for (long long tb = t_begin + (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
             tb < t_end; tb += stride) {
            const long long t = tb + lane;
            const bool in = t < t_end;
            double r = 1.0, mx = 0.0, my = 0.0, mz = 0.0, E = 0.0;
            if (in) {
                r = Q[t]; mx = Q[nodes + t]; my = Q[2 * nodes + t]; mz = Q[3 * nodes + t];
                E = Q[4 * nodes + t];
            }
            pruned_speed_step(in, r, mx, my, mz, E, gamma, R, m, bad);
        }
    } else {
        const float gf = (float)gamma;
        float mf = 0.0f;
        for (long long t = t_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x; t < t_end;
             t += (long long)gridDim.x * blockDim.x) {
            float sp;
            if (!node_speed_f(Q[t], Q[nodes + t], Q[2 * nodes + t], Q[3 * nodes + t],
                              Q[4 * nodes + t], gf, sp)) {
                bad = true;
                continue;
            }
            mf = fmaxf(mf, sp);
        }
        m = (double)mf;
    }
    block_lambda(m, bad, lam_bits, err);
}

static __global__ void cfl_finalize_kernel(unsigned long long *lam_bits, double cfl, double hmin,
                                    int p, double *dt)
{
    const double lam = __longlong_as_double((long long)*lam_bits);
    *dt = __ddiv_rn(__dmul_rn(cfl, hmin), __dmul_rn(2.0 * p + 1.0, lam));
    *lam_bits = 0ull;  // ready for the next reduction on this stream
}

// Pass 1 of the integrals: block b sums a fixed contiguous range of nodes in a
// fixed order (thread-strided, then a shared-memory tree), so the result does
// not depend on scheduling.  Values: I_0..I_4, KE, |Q-Qref|^2, |Qref|^2.
// Quadrature weight J w_i w_j w_k of every in-element node (passed by value,
// staged in shared memory by the kernel: threads index it by their own node).
struct NodeWeights {
    double w[NMAX * NMAX * NMAX];
};

// Float state: a thread's sums of w q are kept as unevaluated float pairs
// (hi + lo) with error-free transformations -- Knuth's TwoSum for the sums,
// the fma residual for the products, the double weight split into two floats
// -- so they carry about 48 bits without touching the FP64 pipe; each thread
// converts its pairs to double once, and everything after is double.
__device__ __forceinline__ void ff_accumulate(float &hi, float &lo, float wh, float wl, float x)
{
    // explicitly rounded operations: no contraction may merge them
    const float p = __fmul_rn(wh, x);
    const float e = fmaf(wh, x, -p);  // wh x - p, exactly
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));  // hi + p - s
    hi = s;
    lo += err + fmaf(wl, x, e);
}

// Shared per-block part of the integrals: the node weights (double, and split
// into two floats for the float state).
struct NormsShared {
    double red[8][256];
    double sw[NMAX * NMAX * NMAX];
    float swh[NMAX * NMAX * NMAX], swl[NMAX * NMAX * NMAX];
};

__device__ __forceinline__ void norms_stage_weights(NormsShared &sh, const NodeWeights &W, int N3)
{
    for (int t = threadIdx.x; t < N3; t += blockDim.x) {
        sh.sw[t] = W.w[t];
        sh.swh[t] = (float)W.w[t];
        sh.swl[t] = (float)(W.w[t] - (double)sh.swh[t]);
    }
    __syncthreads();
}

// One node's contribution to I_0..I_4 and KE (weight index nd).
template <typename real>
__device__ __forceinline__ void norms_node(const NormsShared &sh, int nd, const real qr[NF],
                                           double acc[8], float fh[6], float fl[6])
{
    if constexpr (sizeof(real) == 4) {
        const float wh = sh.swh[nd], wl = sh.swl[nd];
#pragma unroll
        for (int n = 0; n < NF; ++n) ff_accumulate(fh[n], fl[n], wh, wl, qr[n]);
        // the kinetic-energy density in float (the state's own precision)
        const float mm = __fadd_rn(__fadd_rn(__fmul_rn(qr[1], qr[1]), __fmul_rn(qr[2], qr[2])),
                                   __fmul_rn(qr[3], qr[3]));
        const float ke = __fmul_rn(__fmul_rn(0.5f, mm), fast_rcp(qr[0]));
        ff_accumulate(fh[5], fl[5], wh, wl, ke);
    } else {
        const double wq = sh.sw[nd];
#pragma unroll
        for (int n = 0; n < NF; ++n) acc[n] += wq * qr[n];
        acc[5] += wq * 0.5 * (qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]) * recip(qr[0]);
    }
}

// The block's sums (thread sums, then a fixed shared-memory tree) -> partials.
template <typename real>
__device__ __forceinline__ void norms_block_store(NormsShared &sh, double acc[8], const float fh[6],
                                                  const float fl[6], double *partials)
{
    if constexpr (sizeof(real) == 4) {
#pragma unroll
        for (int v = 0; v < 6; ++v) acc[v] = (double)fh[v] + (double)fl[v];
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) sh.red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int v = 0; v < 8; ++v) sh.red[v][threadIdx.x] += sh.red[v][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 8) partials[blockIdx.x * 8 + threadIdx.x] = sh.red[threadIdx.x][0];
}

// Nodes per thread per loop trip of the integral sweeps: their loads are all
// issued before any is used, for more DRAM requests in flight per thread.
template <typename real>
constexpr int kSweepU = sizeof(real) == 4 ? 4 : 2;

template <typename real>
__global__ void __launch_bounds__(256) norms_partial_kernel(const real *__restrict__ Q,
                                                            const real *__restrict__ Qref,
                                                            const Geo g, const NodeWeights W,
                                                            double *partials)
{
    constexpr int U = kSweepU<real>;
    __shared__ NormsShared sh;
    const int N = g.p + 1, N3 = N * N * N;
    norms_stage_weights(sh, W, N3);
    const long long nodes = g.E * N3;
    const long long chunk = (nodes + gridDim.x - 1) / gridDim.x;
    const long long beg = (long long)blockIdx.x * chunk;
    const long long end = beg + chunk < nodes ? beg + chunk : nodes;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float fh[6] = {0, 0, 0, 0, 0, 0}, fl[6] = {0, 0, 0, 0, 0, 0};
    // in-element node index of t, advanced by the stride without a division
    int node = (int)((beg + threadIdx.x) % N3);
    const int step = (int)(blockDim.x % N3);
    const int bd = blockDim.x;
    // the thread's nodes beg + threadIdx.x + k blockDim.x in order of k
    for (long long t0 = beg + threadIdx.x; t0 < end; t0 += (long long)U * bd) {
        real qr[U][NF];
        int nd[U];
        // loads of all U nodes first (indices past the end clamped to the
        // block's last node, so the loads need no branch)
#pragma unroll
        for (int u = 0; u < U; ++u) {
            long long t = t0 + (long long)u * bd;
            t = t < end ? t : end - 1;
            nd[u] = node;
            node += step;
            if (node >= N3) node -= N3;
#pragma unroll
            for (int n = 0; n < NF; ++n) qr[u][n] = Q[n * nodes + t];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long t = t0 + (long long)u * bd;
            if (t >= end) break;
            norms_node<real>(sh, nd[u], qr[u], acc, fh, fl);
            if (Qref) {
                const double wq = sh.sw[nd[u]];
#pragma unroll
                for (int n = 0; n < NF; ++n) {
                    const double q = (double)qr[u][n], r = (double)Qref[n * nodes + t];
                    acc[6] += wq * (q - r) * (q - r);
                    acc[7] += wq * r * r;
                }
            }
        }
    }
    norms_block_store<real>(sh, acc, fh, fl, partials);
}

// Step epilogue of dg_advance, one read of the state a step ends with: the
// integrals of the new state if NORMS (the partition, order and arithmetic
// of norms_partial_kernel without Qref, so the sums are those of dg_norms bit
// for bit) and, if CFL, its Lambda maximum for the next step's time step (the
// node speeds of cfl_kernel).
template <typename real, bool CFL, bool NORMS>
__global__ void __launch_bounds__(256) step_epilogue_kernel(const real *__restrict__ Q,
                                                            const Geo g, const NodeWeights W,
                                                            double *partials,
                                                            unsigned long long *lam_bits, int *err)
{
    constexpr int U = kSweepU<real>;
    __shared__ NormsShared sh;
    const int N = g.p + 1, N3 = N * N * N;
    norms_stage_weights(sh, W, N3);
    const long long nodes = g.E * N3;
    const long long chunk = (nodes + gridDim.x - 1) / gridDim.x;
    const long long beg = (long long)blockIdx.x * chunk;
    const long long end = beg + chunk < nodes ? beg + chunk : nodes;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float fh[6] = {0, 0, 0, 0, 0, 0}, fl[6] = {0, 0, 0, 0, 0, 0};
    double m = 0.0;
    float mf = 0.0f;
    bool bad = false;
    float R = 0.0f;
    const float gf = (float)g.gamma;
    int node = (int)((beg + threadIdx.x) % N3);
    const int step = (int)(blockDim.x % N3);
    const int bd = blockDim.x;
    const int lane = threadIdx.x & 31;
    // whole warps walk together (the double-state pre-filter shuffles); each
    // lane sees the nodes beg + threadIdx.x + k blockDim.x in order of k, as
    // in the integrals
    for (long long tb = beg + (threadIdx.x & ~31); tb < end; tb += (long long)U * bd) {
        real qr[U][NF];
        int nd[U];
        bool in[U];
        // loads of all U nodes first (indices past the end clamped to the
        // block's last node, so the loads need no branch)
#pragma unroll
        for (int u = 0; u < U; ++u) {
            long long t = tb + (long long)u * bd + lane;
            in[u] = t < end;
            t = in[u] ? t : end - 1;
            nd[u] = node;
            node += step;
            if (node >= N3) node -= N3;
#pragma unroll
            for (int n = 0; n < NF; ++n) qr[u][n] = Q[n * nodes + t];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if constexpr (NORMS) {
                if (in[u]) norms_node<real>(sh, nd[u], qr[u], acc, fh, fl);
            }
            if constexpr (CFL) {
                if constexpr (std::is_same<real, double>::value) {
                    pruned_speed_step(in[u], qr[u][0], qr[u][1], qr[u][2], qr[u][3], qr[u][4],
                                      g.gamma, R, m, bad);
                } else if (in[u]) {
                    float sp;
                    if (node_speed_f(qr[u][0], qr[u][1], qr[u][2], qr[u][3], qr[u][4], gf, sp))
                        mf = fmaxf(mf, sp);
                    else
                        bad = true;
                }
            }
        }
    }
    if constexpr (NORMS) norms_block_store<real>(sh, acc, fh, fl, partials);
    if constexpr (CFL) {
        if constexpr (sizeof(real) == 4) m = (double)mf;
        block_lambda(m, bad, lam_bits, err);
    }
}

// Pass 2: one block sums the partials in a fixed order.
static __global__ void __launch_bounds__(256) norms_final_kernel(const double *__restrict__ partials,
                                                          int nblocks, int has_ref, double *out)
{
    __shared__ double red[8][256];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] += partials[b * 8 + v];
#pragma unroll
    for (int v = 0; v < 8; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int v = 0; v < 8; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int v = 0; v < 6; ++v) out[v] = red[v][0];
        out[6] = has_ref ? sqrt(red[6][0]) / sqrt(red[7][0]) : 0.0;
    }
}

// Initial states at the nodes (kinds of dg_init_kind), evaluated in double.
struct InitParams {
    double v[8];
};

template <typename real>
__global__ void __launch_bounds__(256) init_kernel(const Geo g, int kind, const InitParams prm,
                                                   real *__restrict__ Q)
{
    const int N = g.p + 1, N3 = N * N * N;
    const long long nodes = g.E * N3;
    const double pi = 3.14159265358979323846;
    const double gam = g.gamma;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nodes;
         t += (long long)gridDim.x * blockDim.x) {
        const long long e = t / N3;
        const int node = (int)(t - e * N3);
        const int i = node % N, j = (node / N) % N, k = node / (N * N);
        const long long ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / ((long long)g.nx * g.ny);
        const double x = g.x0 + ((double)ex + 0.5 * (g.xi[i] + 1.0)) * g.hx;
        const double y = g.y0 + ((double)ey + 0.5 * (g.xi[j] + 1.0)) * g.hy;
        const double z = g.z0 + ((double)ez + 0.5 * (g.xi[k] + 1.0)) * g.hz;
        double rho, u, v, w, p;
        if (kind == DG_INIT_UNIFORM) {
            rho = prm.v[0]; u = prm.v[1]; v = prm.v[2]; w = prm.v[3]; p = prm.v[4];
        } else if (kind == DG_INIT_VORTEX) {
            const double beta = prm.v[0], tt = prm.v[6];
            const double Lx = g.hx * g.nx, Ly = g.hy * g.ny;
            double dx = x - prm.v[1] - prm.v[3] * tt;
            double dy = y - prm.v[2] - prm.v[4] * tt;
            dx -= Lx * round(dx / Lx);  // minimum image on the periodic box
            dy -= Ly * round(dy / Ly);
            const double r2 = dx * dx + dy * dy;
            const double ex1 = exp(0.5 * (1.0 - r2));
            u = prm.v[3] - beta / (2.0 * pi) * dy * ex1;
            v = prm.v[4] + beta / (2.0 * pi) * dx * ex1;
            w = prm.v[5];
            const double T = 1.0 - (gam - 1.0) * beta * beta / (8.0 * gam * pi * pi) * exp(1.0 - r2);
            rho = pow(T, 1.0 / (gam - 1.0));
            p = pow(rho, gam);
        } else {
            const double rho0 = prm.v[0], V0 = prm.v[1], Ma = prm.v[2];
            const double p0 = rho0 * V0 * V0 / (gam * Ma * Ma);
            u = V0 * sin(x) * cos(y) * cos(z);
            v = -V0 * cos(x) * sin(y) * cos(z);
            w = 0.0;
            p = p0 + rho0 * V0 * V0 / 16.0 * (cos(2.0 * x) + cos(2.0 * y)) * (cos(2.0 * z) + 2.0);
            rho = rho0 * p / p0;
        }
        Q[t] = (real)rho;
        Q[nodes + t] = (real)(rho * u);
        Q[2 * nodes + t] = (real)(rho * v);
        Q[3 * nodes + t] = (real)(rho * w);
        Q[4 * nodes + t] = (real)(p / (gam - 1.0) + 0.5 * rho * (u * u + v * v + w * w));
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

// Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage coefficients.
constexpr double kRkA[5] = {0.0,
                            -567301805773.0 / 1357537059087.0,
                            -2404267990393.0 / 2016746695238.0,
                            -3550918686646.0 / 2091501179385.0,
                            -1275806237668.0 / 842570457699.0};
constexpr double kRkB[5] = {1432997174477.0 / 9575080441755.0,
                            5161836677717.0 / 13612068292357.0,
                            1720146321549.0 / 2090206949498.0,
                            3134564353537.0 / 4481467310338.0,
                            2277821191437.0 / 14882151754819.0};

inline int grid_for(long long n, int threads, long long cap)
{
    long long b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// kernel kinds of the per-kernel timing (dg_profile_end)
enum { kKindFace = 0, kKindVolume = 1, kKindCfl = 2, kKindNorms = 3, kKindInit = 4, kKindStage = 5,
       kKindCopy = 6, kKindEpilogue = 7 };

struct ProfScope {
    Prof *p;
    cudaStream_t s;
    ProfScope(Prof *p_, int kind, cudaStream_t s_) : p(p_), s(s_)
    {
        if (p) p->start(kind, s);
    }
    ~ProfScope()
    {
        if (p) p->stop(s);
    }
};

constexpr long long kMaxGridX = 2147483647LL;

// the +faces of elements [e_begin, e_end) (the whole mesh: 0, g.E)
template <int N, typename real>
cudaError_t launch_face(const Geo &g, const Ops<real> &T, const real *Q, real *F, Prof *prof,
                        cudaStream_t s, long long e_begin = 0, long long e_end = -1)
{
    constexpr int EF = FaceTile<N>::EF;
    if (e_end < 0) e_end = g.E;
    const long long blocks = (e_end - e_begin + EF - 1) / EF;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > kMaxGridX) return cudaErrorInvalidConfiguration;
    ProfScope ps(prof, kKindFace, s);
    // z slabs (halos set) run their own instantiation, so that the periodic
    // kernel carries no halo code
    if (g.zlo != nullptr)
        face_flux_kernel<N, real, true><<<(unsigned)blocks, FaceTile<N>::THREADS, 0, s>>>(
            Q, F, T, g, e_begin, e_end);
    else
        face_flux_kernel<N, real, false><<<(unsigned)blocks, FaceTile<N>::THREADS, 0, s>>>(
            Q, F, T, g, e_begin, e_end);
    return cudaGetLastError();
}

// elements [e_begin, e_end) (the whole mesh: 0, g.E)
template <int N, typename real, int MODE>
cudaError_t launch_volume(const Geo &g, const Ops<real> &T, const real *Qin, real *Out, real *dQ,
                          const real *F, real A, real B, const double *dt, Prof *prof,
                          cudaStream_t s, long long e_begin = 0, long long e_end = -1)
{
    if (e_end < 0) e_end = g.E;
    constexpr int EPB = Tile<N>::EPB, THREADS = Tile<N>::THREADS, N3 = N * N * N;
    const size_t smem = ((size_t)EPB * 3 * NF * N3 + Tile<N>::OPS) * sizeof(real);
    // z slabs (halos set) run their own instantiation, as for the face kernel
    auto kernel = g.zflux != nullptr ? volume_kernel<N, real, MODE, true>
                                     : volume_kernel<N, real, MODE, false>;
    if (smem > 48 * 1024) {  // opt in above the default dynamic shared-memory limit
        cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
    }
    const long long blocks = (e_end - e_begin + EPB - 1) / EPB;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > kMaxGridX) return cudaErrorInvalidConfiguration;
    ProfScope ps(prof, kKindVolume, s);
    kernel<<<(unsigned)blocks, THREADS, smem, s>>>(Qin, Out, dQ, F, T, g, A, B, dt, e_begin, e_end);
    return cudaGetLastError();
}

template <int N, int V, int MODE, typename Ix>
cudaError_t launch_fused_ix(const Geo &g, const Ops<float> &T, const float *Qin, float *Out,
                            float *dQ, float A, float B, const double *dt, Prof *prof,
                            cudaStream_t s)
{
    using SH = TileShape<N, V>;
    using FT = FusedTile<N, SH::TX, SH::TY>;
    const size_t smem = FT::BYTES;
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(fused_stage_kernel<N, V, MODE, Ix>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
    }
    const long long blocks = tile_count(g, SH::TX, SH::TY);
    if (blocks > kMaxGridX) return cudaErrorInvalidConfiguration;
    ProfScope ps(prof, kKindStage, s);
    fused_stage_kernel<N, V, MODE, Ix><<<(unsigned)blocks, FT::THREADS, smem, s>>>(Qin, Out, dQ, T,
                                                                                    g, A, B, dt);
    return cudaGetLastError();
}

// 32-bit index arithmetic when every offset into the state arrays fits
template <int N, int V, int MODE>
cudaError_t launch_fused_v(const Geo &g, const Ops<float> &T, const float *Qin, float *Out,
                           float *dQ, float A, float B, const double *dt, Prof *prof,
                           cudaStream_t s)
{
    const long long floats = (long long)NF * g.E * N * N * N;
    if (floats <= 0x7fffffffLL)
        return launch_fused_ix<N, V, MODE, int>(g, T, Qin, Out, dQ, A, B, dt, prof, s);
    return launch_fused_ix<N, V, MODE, long long>(g, T, Qin, Out, dQ, A, B, dt, prof, s);
}

// the tile variant of order N selected for the single-mesh path (tuning table)
template <int N, int MODE>
cudaError_t launch_fused(const Geo &g, const Ops<float> &T, const float *Qin, float *Out,
                         float *dQ, float A, float B, const double *dt, Prof *prof,
                         cudaStream_t s)
{
    const int v = tile_variant(N);
    if constexpr (kTileVariants[N] > 2)
        if (v == 2) return launch_fused_v<N, (kTileVariants[N] > 2 ? 2 : 0), MODE>(g, T, Qin, Out, dQ, A, B, dt, prof, s);
    if constexpr (kTileVariants[N] > 1)
        if (v == 1) return launch_fused_v<N, (kTileVariants[N] > 1 ? 1 : 0), MODE>(g, T, Qin, Out, dQ, A, B, dt, prof, s);
    return launch_fused_v<N, 0, MODE>(g, T, Qin, Out, dQ, A, B, dt, prof, s);
}

// Column kernel launch (LINES: line_stage_kernel, else column_stage_kernel):
// the z range of every column is cut into chunks so that the number of CTAs
// fills the GPU's resident slots in whole waves (time ~ waves x (layers per
// chunk + the chunk's extra prologue layer)).
template <int N, int MODE, typename Ix, bool LINES>
cudaError_t launch_column_ix(const Geo &g, const Ops<float> &T, const float *Qin, float *Out,
                             float *dQ, float A, float B, const double *dt, Prof *prof,
                             cudaStream_t s)
{
    constexpr int TX = LINES ? LineShape<N, 0>::TX : ColShape<N, 0>::TX;
    constexpr int TY = LINES ? LineShape<N, 0>::TY : ColShape<N, 0>::TY;
    using LT = LineTile<N, TX, TY, LineShape<N, 0>::NS, LineShape<N, 0>::RPAD>;
    constexpr int THREADS = LINES ? LT::THREADS : ColTile<N, TX, TY>::THREADS;
    constexpr size_t BYTES = LINES ? LT::BYTES : ColTile<N, TX, TY>::BYTES;
    // a z slab's line kernel (halo reads compiled in) or the periodic one;
    // the column kernel tests for halos at run time
    const bool halo = LINES && g.zlo != nullptr;
    auto kernel = !LINES ? column_stage_kernel<N, 0, MODE, Ix>
                  : halo ? line_stage_kernel<N, 0, MODE, Ix, true>
                         : line_stage_kernel<N, 0, MODE, Ix, false>;
    // CTAs of this kernel resident on a device at once, per device and
    // variant (a benign race: concurrent first calls store the same value)
    constexpr int kDevices = 64;
    static int resident_of[2][kDevices] = {};
    if (BYTES > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)BYTES);
        if (err != cudaSuccess) return err;
    }
    int dev = 0;
    cudaError_t derr = cudaGetDevice(&dev);
    if (derr != cudaSuccess) return derr;
    int resident = dev < kDevices ? resident_of[halo][dev] : 0;
    if (resident == 0) {
        int sms = 0, per_sm = 0;
        cudaError_t err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (err == cudaSuccess)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, THREADS, BYTES);
        if (err != cudaSuccess) return err;
        resident = sms * (per_sm > 0 ? per_sm : 1);
        if (dev < kDevices) resident_of[halo][dev] = resident;
    }
    const long long ncols = (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int best_zc = g.nz;
    double best = -1.0;
    for (int nch = 1; nch <= g.nz && nch <= 64; ++nch) {
        const int zc = (g.nz + nch - 1) / nch;
        const long long ctas = ncols * ((g.nz + zc - 1) / zc);
        const double cost = (double)((ctas + resident - 1) / resident) * (zc + 1);
        if (best < 0.0 || cost < best) { best = cost; best_zc = zc; }
    }
    const long long blocks = ncols * ((g.nz + best_zc - 1) / best_zc);
    if (blocks > kMaxGridX) return cudaErrorInvalidConfiguration;
    ProfScope ps(prof, kKindStage, s);
    kernel<<<(unsigned)blocks, THREADS, BYTES, s>>>(Qin, Out, dQ, T, g, A, B, dt, best_zc);
    return cudaGetLastError();
}

// 32-bit index arithmetic when every offset into the state arrays fits
template <int N, int MODE>
cudaError_t launch_column(const Geo &g, const Ops<float> &T, const float *Qin, float *Out,
                          float *dQ, float A, float B, const double *dt, Prof *prof,
                          cudaStream_t s)
{
    const long long floats = (long long)NF * g.E * N * N * N;
    const bool lines = line_stage(N);
    if (floats <= 0x7fffffffLL)
        return lines ? launch_column_ix<N, MODE, int, true>(g, T, Qin, Out, dQ, A, B, dt, prof, s)
                     : launch_column_ix<N, MODE, int, false>(g, T, Qin, Out, dQ, A, B, dt, prof, s);
    return lines ? launch_column_ix<N, MODE, long long, true>(g, T, Qin, Out, dQ, A, B, dt, prof, s)
                 : launch_column_ix<N, MODE, long long, false>(g, T, Qin, Out, dQ, A, B, dt, prof, s);
}

// The float form runs the single-pass column stage (DRAM bound: one read of
// the state per stage); the double form the two-kernel stage (FP64-pipe
// bound: every interface flux evaluated once).
template <int N, typename real>
cudaError_t rhs_n(const Geo &g, const Ops<real> &T, const real *Q, real *R, Work &w,
                  cudaStream_t s)
{
    if constexpr (std::is_same<real, float>::value) {
        // z slabs: only the column kernels read the halo traces
        if (g.zlo != nullptr && !column_stage(N)) return cudaErrorNotSupported;
        if (column_stage(N))
            return launch_column<N, 0>(g, T, Q, R, nullptr, 0.0f, 0.0f, nullptr, w.prof, s);
        return launch_fused<N, 0>(g, T, Q, R, nullptr, 0.0f, 0.0f, nullptr, w.prof, s);
    } else {
        real *F = static_cast<real *>(w.face_flux);
        cudaError_t err = launch_face<N>(g, T, Q, F, w.prof, s);
        if (err != cudaSuccess) return err;
        return launch_volume<N, real, 0>(g, T, Q, R, nullptr, F, real(0), real(0), nullptr,
                                         w.prof, s);
    }
}

// The five float-form stages of one LSERK45 step, ping-ponging between two
// states: cur -> other -> cur -> other -> cur -> other, the step's result in
// other.  LAST_MODE 1: the fifth stage also leaves its dQ (dg_rk_step);
// 2: it writes only the new state (dg_advance: the next step's first stage,
// A_1 = 0, does not read dQ).
template <int N, int LAST_MODE>
cudaError_t float_step(const Geo &g, const Ops<float> &T, float *cur, float *other, float *dQ,
                       const double *dt, Work &w, cudaStream_t s)
{
    for (int st = 0; st < 5; ++st) {
        const float *src = (st % 2 == 0) ? cur : other;
        float *dst = (st % 2 == 0) ? other : cur;
        const float A = float(kRkA[st]), B = float(kRkB[st]);
        cudaError_t err;
        if (st == 4)
            err = column_stage(N) ? launch_column<N, LAST_MODE>(g, T, src, dst, dQ, A, B, dt, w.prof, s)
                                  : launch_fused<N, LAST_MODE>(g, T, src, dst, dQ, A, B, dt, w.prof, s);
        else
            err = column_stage(N) ? launch_column<N, 1>(g, T, src, dst, dQ, A, B, dt, w.prof, s)
                                  : launch_fused<N, 1>(g, T, src, dst, dQ, A, B, dt, w.prof, s);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// One LSERK45 step.  Float form: ping-pong between Q and the handle's second
// state; the fifth stage ends in the second state, copied back so that the
// result is in Q.
template <int N, typename real>
cudaError_t rk_n(const Geo &g, const Ops<real> &T, real *Q, real *dQ, const double *dt, Work &w,
                 cudaStream_t s)
{
    if constexpr (std::is_same<real, float>::value) {
        real *Tq = static_cast<real *>(w.qtmp);
        cudaError_t err = float_step<N, 1>(g, T, Q, Tq, dQ, dt, w, s);
        if (err != cudaSuccess) return err;
        const size_t bytes = (size_t)NF * (size_t)g.E * N * N * N * sizeof(real);
        ProfScope ps(w.prof, kKindCopy, s);
        return cudaMemcpyAsync(Q, Tq, bytes, cudaMemcpyDeviceToDevice, s);
    } else {
        real *F = static_cast<real *>(w.face_flux);
        for (int st = 0; st < 5; ++st) {
            cudaError_t err = cudaSuccess;
            if (st > 0 || !w.first_face_done) err = launch_face<N>(g, T, Q, F, w.prof, s);
            if (err != cudaSuccess) return err;
            if (st < 4 || w.out == nullptr) {
                err = launch_volume<N, real, 1>(g, T, Q, Q, dQ, F, real(kRkA[st]),
                                                real(kRkB[st]), dt, w.prof, s);
                if (err != cudaSuccess) return err;
                continue;
            }
            // the fifth stage in ranges of whole z layers, each range's part
            // of the new state copied to the host (w.out) on the copy stream
            // as soon as it is written, while the next ranges compute
            const CopyOut &co = *w.out;
            const long long plane = (long long)g.nx * g.ny, N3 = (long long)N * N * N;
            for (int c = 0; c < co.chunks; ++c) {
                const long long e0 = plane * ((long long)g.nz * c / co.chunks);
                const long long e1 = plane * ((long long)g.nz * (c + 1) / co.chunks);
                if (e1 <= e0) continue;
                err = launch_volume<N, real, 1>(g, T, Q, Q, dQ, F, real(kRkA[st]),
                                                real(kRkB[st]), dt, w.prof, s, e0, e1);
                if (err == cudaSuccess) err = cudaEventRecord(co.ev[c], s);
                if (err == cudaSuccess) err = cudaStreamWaitEvent(co.stream, co.ev[c], 0);
                for (int n = 0; n < NF && err == cudaSuccess; ++n) {
                    const long long off = ((long long)n * g.E + e0) * N3;
                    err = cudaMemcpyAsync(static_cast<real *>(co.host) + off, Q + off,
                                          (size_t)((e1 - e0) * N3) * sizeof(real),
                                          cudaMemcpyDeviceToHost, co.stream);
                }
                if (err != cudaSuccess) return err;
            }
        }
        return cudaSuccess;
    }
}

// One LSERK45 stage (st in 0..4) from Qin to Qout (dg_rk_stage): the double
// form's two kernels (Qin == Qout allowed: the interface fluxes are complete
// before the in-place update), or the float form's single-pass stage kernel
// (Qout a different buffer: neighbouring CTAs still read Qin).
template <int N, typename real>
cudaError_t rk_stage_n(const Geo &g, const Ops<real> &T, const real *Qin, real *Qout, real *dQ,
                       const double *dt, int st, Work &w, cudaStream_t s)
{
    if constexpr (std::is_same<real, float>::value) {
        if (g.zlo != nullptr && !column_stage(N)) return cudaErrorNotSupported;
        const float A = float(kRkA[st]), B = float(kRkB[st]);
        return column_stage(N) ? launch_column<N, 1>(g, T, Qin, Qout, dQ, A, B, dt, w.prof, s)
                               : launch_fused<N, 1>(g, T, Qin, Qout, dQ, A, B, dt, w.prof, s);
    } else {
        real *F = static_cast<real *>(w.face_flux);
        cudaError_t err = launch_face<N>(g, T, Qin, F, w.prof, s);
        if (err != cudaSuccess) return err;
        return launch_volume<N, real, 1>(g, T, Qin, Qout, dQ, F, real(kRkA[st]), real(kRkB[st]),
                                         dt, w.prof, s);
    }
}

// z slabs: the face traces of the first and last layers (ztraces_kernel)
template <int N, typename real>
cudaError_t ztraces_n(const Geo &g, const Ops<real> &T, const real *Q, real *lo, real *hi,
                      cudaStream_t s)
{
    const long long pts = (long long)g.nx * g.ny * N * N;
    const long long blocks = (pts + 255) / 256;
    if (blocks > kMaxGridX) return cudaErrorInvalidConfiguration;
    ztraces_kernel<N, real><<<(unsigned)blocks, 256, 0, s>>>(Q, lo, hi, T, g);
    return cudaGetLastError();
}

// One float-form RK stage (MODE 1) of a single mesh from src to dst with the
// stage kernel of the degree's table entry: the batch's launch path for
// instances large enough to fill the GPU by themselves.
template <int N, typename real>
cudaError_t stage_n(const Geo &g, const Ops<real> &T, const real *src, real *dst, real *dQ,
                    real A, real B, const double *dt, cudaStream_t s)
{
    if constexpr (std::is_same<real, float>::value) {
        return column_stage(N) ? launch_column<N, 1>(g, T, src, dst, dQ, A, B, dt, nullptr, s)
                               : launch_fused<N, 1>(g, T, src, dst, dQ, A, B, dt, nullptr, s);
    } else {
        return cudaErrorInvalidValue;
    }
}

// One float-form RK stage (MODE 1) of a batch's work items of order N: one
// launch of batched_line_kernel, one CTA per item.
template <int N, typename real>
cudaError_t batch_line_n(const LineItem *items, int nitems, const InstDev *inst, int parity,
                         float A, float B, bool small, cudaStream_t s)
{
    if constexpr (std::is_same<real, float>::value) {
        using LS = LineShape<N, 0>;
        using LT = LineTile<N, LS::TX, LS::TY, LS::NS, LS::RPAD>;
        if (nitems <= 0) return cudaSuccess;
        auto kernel = small ? batched_line_kernel<N, 1, int> : batched_line_kernel<N, 1, long long>;
        if (LT::BYTES > 48 * 1024) {
            cudaError_t err = cudaFuncSetAttribute(
                kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LT::BYTES);
            if (err != cudaSuccess) return err;
        }
        kernel<<<(unsigned)nitems, LT::THREADS, LT::BYTES, s>>>(items, inst, parity, A, B);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

// CTAs of batched_line_kernel<N> resident per SM (0 on error)
template <int N, typename real>
int batch_line_blocks_per_sm_n(bool small)
{
    if constexpr (std::is_same<real, float>::value) {
        using LS = LineShape<N, 0>;
        using LT = LineTile<N, LS::TX, LS::TY, LS::NS, LS::RPAD>;
        auto kernel = small ? batched_line_kernel<N, 1, int> : batched_line_kernel<N, 1, long long>;
        if (LT::BYTES > 48 * 1024 &&
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)LT::BYTES) != cudaSuccess)
            return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, LT::THREADS, LT::BYTES) !=
            cudaSuccess)
            return 0;
        return n;
    } else {
        return 0;
    }
}

// host table of the quadrature weight of every in-element node
inline NodeWeights node_weights(const Geo &g)
{
    NodeWeights W;
    const int N = g.p + 1;
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) W.w[(k * N + j) * N + i] = g.J * (g.w[i] * g.w[j] * g.w[k]);
    return W;
}

template <typename real, bool CFL, bool NORMS>
void launch_epilogue(const real *Q, const Geo &g, const NodeWeights &W, Work &w, cudaStream_t s)
{
    step_epilogue_kernel<real, CFL, NORMS><<<kNormBlocks, 256, 0, s>>>(Q, g, W, w.partials,
                                                                       w.lam_bits, w.err);
}

// nsteps steps of (time step, LSERK45 step, integrals); the end of a step and
// the start of the next share one pass over the state (step_epilogue_kernel).
template <int N, typename real>
cudaError_t advance_n(const Geo &g, const Ops<real> &T, real *Q, real *dQ, double cfl, int nsteps,
                      double *dts, double *integ, Work &w, cudaStream_t s);

#define DG_DISPATCH_P(p, CALL)            \
    switch (p) {                          \
    case 0: return CALL(1);               \
    case 1: return CALL(2);               \
    case 2: return CALL(3);               \
    case 3: return CALL(4);               \
    case 4: return CALL(5);               \
    case 5: return CALL(6);               \
    case 6: return CALL(7);               \
    default: return cudaErrorInvalidValue; \
    }

template <typename real>
cudaError_t Launch<real>::rhs(const Geo &g, const Ops<real> &T, const real *Q, real *R, Work &w,
                              cudaStream_t s)
{
#define DG_CALL(NN) rhs_n<NN, real>(g, T, Q, R, w, s)
    DG_DISPATCH_P(g.p, DG_CALL)
#undef DG_CALL
}

template <typename real>
cudaError_t Launch<real>::rk_step(const Geo &g, const Ops<real> &T, real *Q, real *dQ,
                                  const double *dt, Work &w, cudaStream_t s)
{
#define DG_CALL(NN) rk_n<NN, real>(g, T, Q, dQ, dt, w, s)
    DG_DISPATCH_P(g.p, DG_CALL)
#undef DG_CALL
}

template <typename real>
cudaError_t Launch<real>::cfl(const Geo &g, const real *Q, double cfl, double *dt, Work &w,
                              cudaStream_t s)
{
    const int N = g.p + 1;
    const long long nodes = g.E * N * N * N;
    ProfScope ps(w.prof, kKindCfl, s);
    cfl_kernel<real><<<grid_for(nodes, 256, 8LL * sm_count()), 256, 0, s>>>(
        Q, nodes, 0, nodes, g.gamma, w.lam_bits, w.err);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    cfl_finalize_kernel<<<1, 1, 0, s>>>(w.lam_bits, cfl, g.hmin, g.p, dt);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::norms(const Geo &g, const real *Q, const real *Qref, double *out,
                                Work &w, cudaStream_t s)
{
    const NodeWeights W = node_weights(g);
    ProfScope ps(w.prof, kKindNorms, s);
    norms_partial_kernel<real><<<kNormBlocks, 256, 0, s>>>(Q, Qref, g, W, w.partials);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    norms_final_kernel<<<1, 256, 0, s>>>(w.partials, kNormBlocks, Qref != nullptr, out);
    return cudaGetLastError();
}

template <typename real>
cudaError_t Launch<real>::init(const Geo &g, int kind, const double *params, real *Q, Work &w,
                               cudaStream_t s)
{
    InitParams prm{};  // params: 8 doubles, zero-padded by the caller
    for (int i = 0; i < 8; ++i) prm.v[i] = params[i];
    const int N = g.p + 1;
    const long long nodes = g.E * N * N * N;
    ProfScope ps(w.prof, kKindInit, s);
    init_kernel<real><<<grid_for(nodes, 256, 16LL * sm_count()), 256, 0, s>>>(g, kind, prm, Q);
    return cudaGetLastError();
}

// dg_advance_host's copy-in (double state): the host state arrives in ranges
// of whole z layers on the copy stream; the first time-step reduction runs
// over each range as it lands, and the first stage's face kernel over the
// elements of range c once range c + 1 (their +z neighbours) has landed too
// (the last range's neighbours are range 0).  The reduction's maximum is exact,
// so its partition does not change the time step.
template <int N, typename real>
cudaError_t copy_in_prologue(const Geo &g, const Ops<real> &T, real *Q, double cfl, double *dt,
                             Work &w, cudaStream_t s)
{
    const CopyIn &ci = *w.in;
    const long long plane = (long long)g.nx * g.ny, N3 = (long long)N * N * N;
    const long long nodes = g.E * N3;
    const int K = ci.chunks;
    auto lo = [&](int c) { return plane * ((long long)g.nz * c / K); };
    // the copy stream starts once the caller's earlier work on s is done
    cudaError_t err = cudaEventRecord(ci.ev[K], s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(ci.stream, ci.ev[K], 0);
    for (int c = 0; c < K && err == cudaSuccess; ++c) {
        const long long e0 = lo(c), e1 = lo(c + 1);
        for (int n = 0; n < NF && err == cudaSuccess && e1 > e0; ++n) {
            const long long off = ((long long)n * g.E + e0) * N3;
            err = cudaMemcpyAsync(Q + off, static_cast<const real *>(ci.host) + off,
                                  (size_t)((e1 - e0) * N3) * sizeof(real), cudaMemcpyHostToDevice,
                                  ci.stream);
        }
        if (err == cudaSuccess) err = cudaEventRecord(ci.ev[c], ci.stream);
    }
    if (err != cudaSuccess) return err;
    real *F = static_cast<real *>(w.face_flux);
    int pending = -1;  // a range whose face kernel waits for the next range
    for (int c = 0; c < K; ++c) {
        const long long e0 = lo(c), e1 = lo(c + 1);
        if (e1 <= e0) continue;
        err = cudaStreamWaitEvent(s, ci.ev[c], 0);
        if (err != cudaSuccess) return err;
        {
            ProfScope ps(w.prof, kKindCfl, s);
            cfl_kernel<real><<<grid_for((e1 - e0) * N3, 256, 8LL * sm_count()), 256, 0, s>>>(
                Q, nodes, e0 * N3, e1 * N3, g.gamma, w.lam_bits, w.err);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess && pending >= 0)
            err = launch_face<N>(g, T, Q, F, w.prof, s, lo(pending), lo(pending + 1));
        if (err != cudaSuccess) return err;
        pending = c;
    }
    // the last range's +z neighbours are layer 0, landed first
    if (pending >= 0) {
        err = launch_face<N>(g, T, Q, F, w.prof, s, lo(pending), lo(pending + 1));
        if (err != cudaSuccess) return err;
    }
    cfl_finalize_kernel<<<1, 1, 0, s>>>(w.lam_bits, cfl, g.hmin, g.p, dt);
    return cudaGetLastError();
}

template <int N, typename real>
cudaError_t advance_n(const Geo &g, const Ops<real> &T, real *Q, real *dQ, double cfl, int nsteps,
                      double *dts, double *integ, Work &w, cudaStream_t s)
{
    cudaError_t err = cudaSuccess;
    if constexpr (!std::is_same<real, float>::value) {
        if (w.in) err = copy_in_prologue<N, real>(g, T, Q, cfl, dts, w, s);
        else err = Launch<real>::cfl(g, Q, cfl, dts, w, s);
    } else {
        err = Launch<real>::cfl(g, Q, cfl, dts, w, s);
    }
    if (err != cudaSuccess) return err;
    const bool norms = integ != nullptr;
    if constexpr (!std::is_same<real, float>::value) {
        // double state: the integrals are FP64-pipe bound and the time step's
        // pre-filter is warp-synchronous; one pass doing both was measured
        // slower than the two passes, which it would only save one read of
        // the state
        for (int k = 0; k < nsteps; ++k) {
            // the copy-back of the new state (dg_advance_host) overlaps the
            // last step's fifth stage only
            Work wk = w;
            if (k + 1 < nsteps) wk.out = nullptr;
            wk.first_face_done = k == 0 && w.in != nullptr;
            err = rk_n<N, real>(g, T, Q, dQ, dts + k, wk, s);
            if (err != cudaSuccess) return err;
            if (norms) {
                err = Launch<real>::norms(g, Q, nullptr, integ + (size_t)k * DG_NORMS_LEN, w, s);
                if (err != cudaSuccess) return err;
            }
            if (k + 1 < nsteps) {
                err = Launch<real>::cfl(g, Q, cfl, dts + k + 1, w, s);
                if (err != cudaSuccess) return err;
            }
        }
        return cudaSuccess;
    } else {
        // float state: the steps alternate between Q and the second state
        // (each step's fifth stage writes only the new state, into the buffer
        // the step did not start from), and one read of each step's result
        // gives its integrals and the next time step; an odd number of steps
        // ends with a copy back into Q
        const NodeWeights W = node_weights(g);
        float *cur = Q, *other = static_cast<float *>(w.qtmp);
        for (int k = 0; k < nsteps; ++k) {
            err = float_step<N, 2>(g, T, cur, other, dQ, dts + k, w, s);
            if (err != cudaSuccess) return err;
            std::swap(cur, other);
            const bool more = k + 1 < nsteps;
            if (!more && !norms) break;
            {
                ProfScope ps(w.prof, kKindEpilogue, s);
                if (more && norms) launch_epilogue<float, true, true>(cur, g, W, w, s);
                else if (more) launch_epilogue<float, true, false>(cur, g, W, w, s);
                else launch_epilogue<float, false, true>(cur, g, W, w, s);
            }
            err = cudaGetLastError();
            if (err != cudaSuccess) return err;
            if (norms) {
                norms_final_kernel<<<1, 256, 0, s>>>(w.partials, kNormBlocks, 0, integ + (size_t)k * DG_NORMS_LEN);
                err = cudaGetLastError();
                if (err != cudaSuccess) return err;
            }
            if (more) {
                cfl_finalize_kernel<<<1, 1, 0, s>>>(w.lam_bits, cfl, g.hmin, g.p, dts + k + 1);
                err = cudaGetLastError();
                if (err != cudaSuccess) return err;
            }
        }
        if (cur != Q) {
            const size_t bytes = (size_t)NF * (size_t)g.E * N * N * N * sizeof(float);
            ProfScope ps(w.prof, kKindCopy, s);
            return cudaMemcpyAsync(Q, cur, bytes, cudaMemcpyDeviceToDevice, s);
        }
        return cudaSuccess;
    }
}

// Explicit instantiation of the per-degree launch paths of one scalar type:
// DG_INSTANTIATE_N(template, NN, real) defines them (one translation unit per
// group of degrees compiles them in parallel), DG_INSTANTIATE_N(extern
// template, NN, real) declares them elsewhere.
#define DG_INSTANTIATE_N(KW, NN, REAL)                                                        \
    KW cudaError_t rhs_n<NN, REAL>(const Geo &, const Ops<REAL> &, const REAL *, REAL *, Work &, \
                                   cudaStream_t);                                            \
    KW cudaError_t rk_n<NN, REAL>(const Geo &, const Ops<REAL> &, REAL *, REAL *,             \
                                  const double *, Work &, cudaStream_t);                     \
    KW cudaError_t advance_n<NN, REAL>(const Geo &, const Ops<REAL> &, REAL *, REAL *, double, \
                                       int, double *, double *, Work &, cudaStream_t);       \
    KW cudaError_t stage_n<NN, REAL>(const Geo &, const Ops<REAL> &, const REAL *, REAL *,     \
                                     REAL *, REAL, REAL, const double *, cudaStream_t);      \
    KW cudaError_t rk_stage_n<NN, REAL>(const Geo &, const Ops<REAL> &, const REAL *, REAL *,  \
                                        REAL *, const double *, int, Work &, cudaStream_t);  \
    KW cudaError_t ztraces_n<NN, REAL>(const Geo &, const Ops<REAL> &, const REAL *, REAL *,   \
                                       REAL *, cudaStream_t);                                \
    KW cudaError_t batch_line_n<NN, REAL>(const LineItem *, int, const InstDev *, int, float,  \
                                          float, bool, cudaStream_t);                        \
    KW int batch_line_blocks_per_sm_n<NN, REAL>(bool);

template <typename real>
cudaError_t Launch<real>::rk_stage(const Geo &g, const Ops<real> &T, const real *Qin, real *Qout,
                                   real *dQ, const double *dt, int stage, Work &w, cudaStream_t s)
{
#define DG_CALL(NN) rk_stage_n<NN, real>(g, T, Qin, Qout, dQ, dt, stage, w, s)
    DG_DISPATCH_P(g.p, DG_CALL)
#undef DG_CALL
}

template <typename real>
cudaError_t Launch<real>::ztraces(const Geo &g, const Ops<real> &T, const real *Q, real *lo,
                                  real *hi, cudaStream_t s)
{
#define DG_CALL(NN) ztraces_n<NN, real>(g, T, Q, lo, hi, s)
    DG_DISPATCH_P(g.p, DG_CALL)
#undef DG_CALL
}

template <typename real>
cudaError_t Launch<real>::advance(const Geo &g, const Ops<real> &T, real *Q, real *dQ, double cfl,
                                  int nsteps, double *dts, double *integ, Work &w, cudaStream_t s)
{
#define DG_CALL(NN) advance_n<NN, real>(g, T, Q, dQ, cfl, nsteps, dts, integ, w, s)
    DG_DISPATCH_P(g.p, DG_CALL)
#undef DG_CALL
}

}  // namespace dg
