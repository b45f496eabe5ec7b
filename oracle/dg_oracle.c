/*
 * dg_oracle.c -- plain, slow, FP64 CPU oracle for the DG Euler right-hand side
 * and its low-storage Runge-Kutta update (Kirby & Mavriplis, arXiv 2006.15698).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link or call this
 * file; only the tests, the smoke check and the CPU-baseline leg of the bench
 * use it.  It shares no code, header, table or constant generator with the
 * CUDA library: every number it uses (Gauss-Legendre nodes, Lagrange basis
 * values and derivatives, Runge-Kutta coefficients) is computed or written out
 * here, from the definitions cited beside each function.
 *
 * What it computes (paper Sec. II, Eqs. 1-7):
 *   conservative Euler system dQ/dt + div F(Q) = 0               (Eq. 1, Eq. 2)
 *   ideal-gas closure rho E = p/(gamma-1) + rho |u|^2 / 2          (Eq. 3)
 *   weak form per element, integrated by parts                    (Eq. 4, Eq. 5)
 *   Lax-Friedrichs interface flux F*                               (Sec. II.B)
 *   collocated nodal Lagrange basis on N = p+1 Gauss-Legendre points
 *   per direction, tensor product in 3D                            (Eq. 6, Eq. 7)
 *   five-stage, fourth-order low-storage explicit RK               (Sec. II.B, Sec. VI.A)
 *
 * Two independent evaluations of the semi-discrete right-hand side:
 *   O1 (dgo_rhs_o1): brute force.  The Lagrange basis, its gradient and the
 *      state are evaluated from the product formula Eq. 7 at every volume and
 *      face quadrature point, the full quadrature sums of Eq. 5 are formed for
 *      every test function, and the full (brute-force) mass matrix is solved.
 *   O2 (dgo_rhs_o2): the same quadrature written with the collocation identity
 *      psi_ijk(xi_abc) = delta_ia delta_jb delta_kc applied, as plain nested
 *      loops with every Jacobian and weight written out.
 *
 * Readings of points the paper leaves open (each is stated again where used):
 *   - Lax-Friedrichs is the local (Rusanov) form: the dissipation speed is the
 *     larger |u.n| + c of the two traces at each face quadrature point.
 *   - The velocities used in the pressure are the physical ones; the geometric
 *     factor 2/h multiplies the derivative of the flux only.
 *   - Boundary conditions are periodic in all three directions.
 *   - The RK scheme is Carpenter & Kennedy's 2N-storage (5,4) scheme.
 *   - The time-step rule is dt = CFL min(h) / ((2p+1) max_nodes sum_d(|u_d|+c)).
 *     The paper states none; parity for this rule is unpinned against the paper.
 *
 * Layout of a state array (shared interface with the tests, not arithmetic):
 *   Q[n][e][k][j][i], n = field (rho, rho u, rho v, rho w, rho E), element
 *   e = ex + nx*(ey + ny*ez), node (i,j,k) with i fastest.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (see oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NF 5
#define NMAX 9 /* the oracle itself supports p = 0..8 */

typedef struct {
    int nx, ny, nz, p;
    double x0, y0, z0;
    double Lx, Ly, Lz;
    double gamma;
} dgo_mesh;

/* ------------------------------------------------------------------------ */
/* 1D Gauss-Legendre quadrature and the Lagrange basis of Eq. 7             */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial P_n(x) and its derivative by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre_eval(int n, double x, double *P, double *dP)
{
    if (n == 0) { *P = 1.0; *dP = 0.0; return; }
    double pm1 = 1.0, pk = x;
    for (int k = 1; k < n; ++k) {
        double pk1 = ((2.0 * k + 1.0) * x * pk - k * pm1) / (k + 1.0);
        pm1 = pk;
        pk = pk1;
    }
    *P = pk;
    /* P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1), valid away from x = +-1 */
    *dP = n * (x * pk - pm1) / (x * x - 1.0);
}

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1], N points: the
 * roots of P_N found by Newton's method, weights w = 2 / ((1-x^2) P_N'(x)^2).
 * Returns 0 on success. */
int dgo_gl_nodes(int N, double *xi, double *w)
{
    if (N < 1 || N > NMAX) return 1;
    if (N == 1) { xi[0] = 0.0; w[0] = 2.0; return 0; }
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < N; ++k) {
        /* classical starting guess for the k-th largest root */
        double x = cos(pi * (k + 0.75) / (N + 0.5));
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre_eval(N, x, &P, &dP);
            double dx = P / dP;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        double P, dP;
        legendre_eval(N, x, &P, &dP);
        xi[N - 1 - k] = x; /* roots come largest first; store ascending */
        w[N - 1 - k] = 2.0 / ((1.0 - x * x) * dP * dP);
    }
    return 0;
}

/* Eq. 7: l_s(x) = prod_{i != s} (x - xi_i) / (xi_s - xi_i) */
double dgo_lagrange(int N, const double *xi, int s, double x)
{
    double v = 1.0;
    for (int i = 0; i < N; ++i)
        if (i != s) v *= (x - xi[i]) / (xi[s] - xi[i]);
    return v;
}

/* derivative of Eq. 7 by the product rule:
 * l_s'(x) = sum_{m != s} 1/(xi_s - xi_m) prod_{i != s, m} (x - xi_i)/(xi_s - xi_i) */
double dgo_lagrange_deriv(int N, const double *xi, int s, double x)
{
    double d = 0.0;
    for (int m = 0; m < N; ++m) {
        if (m == s) continue;
        double t = 1.0 / (xi[s] - xi[m]);
        for (int i = 0; i < N; ++i)
            if (i != s && i != m) t *= (x - xi[i]) / (xi[s] - xi[i]);
        d += t;
    }
    return d;
}

/* ------------------------------------------------------------------------ */
/* Euler flux (Eq. 2) with the ideal-gas closure (Eq. 3), and the local       */
/* Lax-Friedrichs interface flux                                             */
/* ------------------------------------------------------------------------ */

static double pressure(const double q[NF], double gamma)
{
    double rho = q[0];
    double u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
    /* Eq. 3 solved for p */
    return (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w));
}

/* F^d(Q), d = 0,1,2 for x,y,z: the d-th column of the flux matrix of Eq. 2.
 * rho u_d H = u_d (rho E + p). */
void dgo_flux(int d, const double q[NF], double gamma, double f[NF])
{
    double rho = q[0];
    double vel[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
    double p = pressure(q, gamma);
    double ud = vel[d];
    f[0] = rho * ud;
    for (int m = 0; m < 3; ++m)
        f[1 + m] = q[1 + m] * ud + (m == d ? p : 0.0);
    f[4] = (q[4] + p) * ud;
}

/* local Lax-Friedrichs (Rusanov) flux across a face whose normal is +e_d,
 * with qL on the side the normal points away from and qR on the other:
 *   F* = (F^d(qL) + F^d(qR))/2 - lambda (qR - qL)/2,
 *   lambda = max(|u_d| + c) over the two states, c = sqrt(gamma p / rho). */
void dgo_lf_flux(int d, const double qL[NF], const double qR[NF], double gamma,
                 double fs[NF])
{
    double fL[NF], fR[NF];
    dgo_flux(d, qL, gamma, fL);
    dgo_flux(d, qR, gamma, fR);
    double cL = sqrt(gamma * pressure(qL, gamma) / qL[0]);
    double cR = sqrt(gamma * pressure(qR, gamma) / qR[0]);
    double sL = fabs(qL[1 + d] / qL[0]) + cL;
    double sR = fabs(qR[1 + d] / qR[0]) + cR;
    double lam = sL > sR ? sL : sR;
    for (int n = 0; n < NF; ++n)
        fs[n] = 0.5 * (fL[n] + fR[n]) - 0.5 * lam * (qR[n] - qL[n]);
}

/* ------------------------------------------------------------------------ */
/* Mesh helpers                                                              */
/* ------------------------------------------------------------------------ */

static int mesh_ok(const dgo_mesh *m)
{
    return m && m->nx > 0 && m->ny > 0 && m->nz > 0 && m->p >= 0 &&
           m->p + 1 <= NMAX && m->Lx > 0 && m->Ly > 0 && m->Lz > 0 &&
           m->gamma > 1.0;
}

static int64_t n_elem(const dgo_mesh *m)
{
    return (int64_t)m->nx * m->ny * m->nz;
}

/* periodic neighbour of element (ex,ey,ez) shifted by s = +-1 in direction d */
static int64_t neighbour(const dgo_mesh *m, int ex, int ey, int ez, int d, int s)
{
    int c[3] = {ex, ey, ez};
    int n[3] = {m->nx, m->ny, m->nz};
    c[d] = (c[d] + s + n[d]) % n[d];
    return c[0] + (int64_t)m->nx * (c[1] + (int64_t)m->ny * c[2]);
}

/* index of value (field f, element e, node i,j,k) in Q[n][e][k][j][i] */
static size_t qidx(const dgo_mesh *m, int f, int64_t e, int i, int j, int k)
{
    int N = m->p + 1;
    return ((size_t)f * (size_t)n_elem(m) + (size_t)e) * (size_t)(N * N * N) +
           (size_t)((k * N + j) * N + i);
}

typedef struct {
    int N;
    double xi[NMAX], w[NMAX];
    double dl[NMAX][NMAX]; /* dl[s][a] = l_s'(xi_a) */
    double lp[NMAX], lm[NMAX]; /* l_s(+1), l_s(-1) */
} basis1d;

static void make_basis(int N, basis1d *b)
{
    b->N = N;
    dgo_gl_nodes(N, b->xi, b->w);
    for (int s = 0; s < N; ++s) {
        for (int a = 0; a < N; ++a)
            b->dl[s][a] = dgo_lagrange_deriv(N, b->xi, s, b->xi[a]);
        b->lp[s] = dgo_lagrange(N, b->xi, s, 1.0);
        b->lm[s] = dgo_lagrange(N, b->xi, s, -1.0);
    }
}

/* state at node (i,j,k) of element e */
static void load_node(const dgo_mesh *m, const double *Q, int64_t e, int i,
                      int j, int k, double q[NF])
{
    for (int f = 0; f < NF; ++f) q[f] = Q[qidx(m, f, e, i, j, k)];
}

/* trace of element e's polynomial on its face in direction d at side s
 * (s = +1: xi_d = +1, s = -1: xi_d = -1), at the face node (t1, t2), where
 * (t1, t2) are the two remaining indices in (i,j,k) order:
 * Q(face) = sum_a l_a(+-1) Q(node with index a along d). */
static void collocated_trace(const dgo_mesh *m, const basis1d *b, const double *Q,
                             int64_t e, int d, int s, int t1, int t2, double q[NF])
{
    const double *l = s > 0 ? b->lp : b->lm;
    for (int f = 0; f < NF; ++f) q[f] = 0.0;
    for (int a = 0; a < b->N; ++a) {
        int i, j, k;
        if (d == 0) { i = a; j = t1; k = t2; }
        else if (d == 1) { i = t1; j = a; k = t2; }
        else { i = t1; j = t2; k = a; }
        for (int f = 0; f < NF; ++f) q[f] += l[a] * Q[qidx(m, f, e, i, j, k)];
    }
}

/* A z-face trace held in a halo buffer H[f][ey*nx + ex][t2*N + t1] (the
 * layout of dgo_ztraces below). */
static void halo_trace(const dgo_mesh *m, const double *H, int ex, int ey, int t1, int t2,
                       double q[NF])
{
    const int N = m->p + 1;
    const size_t plane = (size_t)m->nx * (size_t)m->ny;
    const size_t col = (size_t)ey * (size_t)m->nx + (size_t)ex;
    for (int f = 0; f < NF; ++f) q[f] = H[((size_t)f * plane + col) * (size_t)(N * N) + (size_t)(t2 * N + t1)];
}

/* ------------------------------------------------------------------------ */
/* O2: collocated right-hand side, plain loops (Eq. 5 with psi(xi_abc) = delta) */
/* ------------------------------------------------------------------------ */

/* R = dQ/dt = M^{-1} (volume term - surface term), in the layout above.
 * For element e, node (i,j,k), field n, with J = hx hy hz / 8 and the x-faces'
 * surface Jacobian hy hz / 4 (and likewise for y, z):
 *   vol  = sum_a J w_a w_j w_k (2/hx) l_i'(xi_a) F^x_n(Q_ajk)
 *        + sum_b J w_i w_b w_k (2/hy) l_j'(xi_b) F^y_n(Q_ibk)
 *        + sum_c J w_i w_j w_c (2/hz) l_k'(xi_c) F^z_n(Q_ijc)
 *   surf = (hy hz/4) w_j w_k [ l_i(+1) F*x(+face)_jk - l_i(-1) F*x(-face)_jk ]
 *        + (same for y, z)
 *   R    = (vol - surf) / (J w_i w_j w_k)
 * where F*x(+face) is the Lax-Friedrichs flux through the element's +x face
 * (normal +x: the element is the left state, its +x neighbour the right) and
 * F*x(-face) the flux through its -x face (left state: the -x neighbour).
 * The outward normal on the -x face is -x, hence the sign of that term. */
/* O2 for one element e: out[n * N^3 + node] = R of field n at node (i,j,k). */
/* halo_lo / halo_hi (NULL: periodic in z) replace the traces of the -z
 * neighbour of layer 0 and of the +z neighbour of layer nz-1 (z slabs, below). */
static void rhs_o2_element(const dgo_mesh *m, const basis1d *bp, const double *Q, int64_t e,
                           const double *halo_lo, const double *halo_hi, double *out)
{
    const basis1d b = *bp;
    const int N = m->p + 1;
    const int N3 = N * N * N;
    const double h[3] = {m->Lx / m->nx, m->Ly / m->ny, m->Lz / m->nz};
    const double J = h[0] * h[1] * h[2] / 8.0;
    const double sJ[3] = {h[1] * h[2] / 4.0, h[0] * h[2] / 4.0, h[0] * h[1] / 4.0};
    const double gam = m->gamma;
    int ex = (int)(e % m->nx);
    int ey = (int)((e / m->nx) % m->ny);
    int ez = (int)(e / ((int64_t)m->nx * m->ny));
    double fx[NMAX * NMAX * NMAX][NF], fy[NMAX * NMAX * NMAX][NF], fz[NMAX * NMAX * NMAX][NF];
    /* fluxes at every node */
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                double q[NF];
                load_node(m, Q, e, i, j, k, q);
                int id = (k * N + j) * N + i;
                dgo_flux(0, q, gam, fx[id]);
                dgo_flux(1, q, gam, fy[id]);
                dgo_flux(2, q, gam, fz[id]);
            }
    /* interface fluxes on the six faces, fhat[d][side][t2*N+t1][n],
     * side 0 = -face, side 1 = +face */
    double fhat[3][2][NMAX * NMAX][NF];
    for (int d = 0; d < 3; ++d) {
        int64_t em = neighbour(m, ex, ey, ez, d, -1);
        int64_t ep = neighbour(m, ex, ey, ez, d, +1);
        for (int t2 = 0; t2 < N; ++t2)
            for (int t1 = 0; t1 < N; ++t1) {
                double qL[NF], qR[NF];
                /* -face: left = -neighbour at its +1 end, right = this at -1 */
                if (d == 2 && halo_lo && ez == 0)
                    halo_trace(m, halo_lo, ex, ey, t1, t2, qL);
                else
                    collocated_trace(m, &b, Q, em, d, +1, t1, t2, qL);
                collocated_trace(m, &b, Q, e, d, -1, t1, t2, qR);
                dgo_lf_flux(d, qL, qR, gam, fhat[d][0][t2 * N + t1]);
                /* +face: left = this at +1, right = +neighbour at -1 */
                collocated_trace(m, &b, Q, e, d, +1, t1, t2, qL);
                if (d == 2 && halo_hi && ez == m->nz - 1)
                    halo_trace(m, halo_hi, ex, ey, t1, t2, qR);
                else
                    collocated_trace(m, &b, Q, ep, d, -1, t1, t2, qR);
                dgo_lf_flux(d, qL, qR, gam, fhat[d][1][t2 * N + t1]);
            }
    }
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                for (int n = 0; n < NF; ++n) {
                    double vol = 0.0;
                    for (int a = 0; a < N; ++a)
                        vol += J * b.w[a] * b.w[j] * b.w[k] * (2.0 / h[0]) *
                               b.dl[i][a] * fx[(k * N + j) * N + a][n];
                    for (int bb = 0; bb < N; ++bb)
                        vol += J * b.w[i] * b.w[bb] * b.w[k] * (2.0 / h[1]) *
                               b.dl[j][bb] * fy[(k * N + bb) * N + i][n];
                    for (int c = 0; c < N; ++c)
                        vol += J * b.w[i] * b.w[j] * b.w[c] * (2.0 / h[2]) *
                               b.dl[k][c] * fz[(c * N + j) * N + i][n];
                    double surf = 0.0;
                    /* x faces: face node (t1,t2) = (j,k) */
                    surf += sJ[0] * b.w[j] * b.w[k] *
                            (b.lp[i] * fhat[0][1][k * N + j][n] -
                             b.lm[i] * fhat[0][0][k * N + j][n]);
                    /* y faces: face node (t1,t2) = (i,k) */
                    surf += sJ[1] * b.w[i] * b.w[k] *
                            (b.lp[j] * fhat[1][1][k * N + i][n] -
                             b.lm[j] * fhat[1][0][k * N + i][n]);
                    /* z faces: face node (t1,t2) = (i,j) */
                    surf += sJ[2] * b.w[i] * b.w[j] *
                            (b.lp[k] * fhat[2][1][j * N + i][n] -
                             b.lm[k] * fhat[2][0][j * N + i][n]);
                    double mass = J * b.w[i] * b.w[j] * b.w[k];
                    out[n * N3 + (k * N + j) * N + i] = (vol - surf) / mass;
                }
            }
}

/* R = dQ/dt = M^{-1} (volume term - surface term), in the layout above.
 * For element e, node (i,j,k), field n, with J = hx hy hz / 8 and the x-faces'
 * surface Jacobian hy hz / 4 (and likewise for y, z):
 *   vol  = sum_a J w_a w_j w_k (2/hx) l_i'(xi_a) F^x_n(Q_ajk)
 *        + sum_b J w_i w_b w_k (2/hy) l_j'(xi_b) F^y_n(Q_ibk)
 *        + sum_c J w_i w_j w_c (2/hz) l_k'(xi_c) F^z_n(Q_ijc)
 *   surf = (hy hz/4) w_j w_k [ l_i(+1) F*x(+face)_jk - l_i(-1) F*x(-face)_jk ]
 *        + (same for y, z)
 *   R    = (vol - surf) / (J w_i w_j w_k)
 * where F*x(+face) is the Lax-Friedrichs flux through the element's +x face
 * (normal +x: the element is the left state, its +x neighbour the right) and
 * F*x(-face) the flux through its -x face (left state: the -x neighbour).
 * The outward normal on the -x face is -x, hence the sign of that term. */
int dgo_rhs_o2(const dgo_mesh *m, const double *Q, double *R)
{
    if (!mesh_ok(m) || !Q || !R) return 1;
    const int N = m->p + 1;
    const int N3 = N * N * N;
    basis1d b;
    make_basis(N, &b);
    const int64_t E = n_elem(m);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        double out[NF * NMAX * NMAX * NMAX];
        rhs_o2_element(m, &b, Q, e, NULL, NULL, out);
        for (int n = 0; n < NF; ++n)
            for (int t = 0; t < N3; ++t) R[qidx(m, n, e, 0, 0, 0) + t] = out[n * N3 + t];
    }
    return 0;
}

/* O2 restricted to a list of elements (for sampled checks of large meshes):
 * R[n][s][k][j][i] for s = 0..nsel-1 is the right-hand side of element
 * elems[s]. */
int dgo_rhs_o2_elements(const dgo_mesh *m, const double *Q, int64_t nsel, const int64_t *elems,
                        double *R)
{
    if (!mesh_ok(m) || !Q || !R || !elems || nsel < 0) return 1;
    const int N = m->p + 1;
    const int N3 = N * N * N;
    for (int64_t s = 0; s < nsel; ++s)
        if (elems[s] < 0 || elems[s] >= n_elem(m)) return 1;
    basis1d b;
    make_basis(N, &b);
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < nsel; ++s) {
        double out[NF * NMAX * NMAX * NMAX];
        rhs_o2_element(m, &b, Q, elems[s], NULL, NULL, out);
        for (int n = 0; n < NF; ++n)
            for (int t = 0; t < N3; ++t) R[((size_t)n * nsel + s) * N3 + t] = out[n * N3 + t];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* O1: brute-force quadrature of Eq. 5 with the basis of Eq. 7                */
/* ------------------------------------------------------------------------ */

/* Value of element e's polynomial (all 5 fields) at reference point (r,s,t),
 * summing every nodal basis function l_i(r) l_j(s) l_k(t) (Eq. 6). */
static void eval_poly(const dgo_mesh *m, const double *xi, const double *Q,
                      int64_t e, double r, double s, double t, double q[NF])
{
    int N = m->p + 1;
    double lr[NMAX], ls[NMAX], lt[NMAX];
    for (int a = 0; a < N; ++a) {
        lr[a] = dgo_lagrange(N, xi, a, r);
        ls[a] = dgo_lagrange(N, xi, a, s);
        lt[a] = dgo_lagrange(N, xi, a, t);
    }
    for (int f = 0; f < NF; ++f) q[f] = 0.0;
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                double phi = lr[i] * ls[j] * lt[k];
                for (int f = 0; f < NF; ++f) q[f] += phi * Q[qidx(m, f, e, i, j, k)];
            }
}

/* Solve A x = b (n x n, row-major, overwritten) by Gaussian elimination with
 * partial pivoting; b holds nrhs right-hand sides as b[row*nrhs + c]. */
static int dense_solve(int n, double *A, double *b, int nrhs)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return 1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t;
            }
            for (int k = 0; k < nrhs; ++k) {
                double t = b[c * nrhs + k]; b[c * nrhs + k] = b[piv * nrhs + k]; b[piv * nrhs + k] = t;
            }
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            for (int k = 0; k < nrhs; ++k) b[r * nrhs + k] -= f * b[c * nrhs + k];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        for (int k = 0; k < nrhs; ++k) {
            double v = b[c * nrhs + k];
            for (int r = c + 1; r < n; ++r) v -= A[c * n + r] * b[r * nrhs + k];
            b[c * nrhs + k] = v / A[c * n + c];
        }
    }
    return 0;
}

/* dQ/dt from Eq. 5 by brute force: for every test function psi_ijk,
 *   vol_ijk  = sum over the N^3 volume quadrature points x_abc of
 *              J w_a w_b w_c F(Q(x_abc)) . grad psi_ijk(x_abc)
 *   surf_ijk = sum over the 6 faces and their N^2 face quadrature points of
 *              (face Jacobian) w w (F* . n) psi_ijk(face point)
 * with Q, psi and grad psi evaluated from Eq. 6/7 at each point and both face
 * traces evaluated as full polynomials, then M dQ/dt = vol - surf with the
 * brute-force mass matrix M_{ijk,i'j'k'} = sum J w w w psi_ijk psi_i'j'k'. */
int dgo_rhs_o1(const dgo_mesh *m, const double *Q, double *R)
{
    if (!mesh_ok(m) || !Q || !R) return 1;
    const int N = m->p + 1;
    const int N3 = N * N * N;
    double xi[NMAX], w[NMAX];
    dgo_gl_nodes(N, xi, w);
    const double h[3] = {m->Lx / m->nx, m->Ly / m->ny, m->Lz / m->nz};
    const double J = h[0] * h[1] * h[2] / 8.0;
    const double sJ[3] = {h[1] * h[2] / 4.0, h[0] * h[2] / 4.0, h[0] * h[1] / 4.0};
    const double gam = m->gamma;
    const int64_t E = n_elem(m);

    /* l_i(xi_a) and l_i'(xi_a) tabulated from Eq. 7 (not assumed to be delta) */
    double L[NMAX][NMAX], dL[NMAX][NMAX], Lpm[2][NMAX];
    for (int i = 0; i < N; ++i) {
        for (int a = 0; a < N; ++a) {
            L[i][a] = dgo_lagrange(N, xi, i, xi[a]);
            dL[i][a] = dgo_lagrange_deriv(N, xi, i, xi[a]);
        }
        Lpm[0][i] = dgo_lagrange(N, xi, i, -1.0);
        Lpm[1][i] = dgo_lagrange(N, xi, i, +1.0);
    }
    /* brute-force mass matrix (identical for every element of the mesh) */
    double *M = (double *)malloc(sizeof(double) * (size_t)N3 * N3);
    double *rhs = (double *)malloc(sizeof(double) * (size_t)N3 * NF);
    double *F = (double *)malloc(sizeof(double) * (size_t)N3 * 3 * NF);
    if (!M || !rhs || !F) { free(M); free(rhs); free(F); return 2; }

    /* interface flux at every face quadrature point of the element:
     * FS[((d*2 + side)*N*N + t2*N + t1)*NF + n], evaluated once per element */
    double *FS = (double *)malloc(sizeof(double) * (size_t)6 * N * N * NF);
    /* the brute-force mass matrix is the same for every element: build it once */
    double *M0 = (double *)malloc(sizeof(double) * (size_t)N3 * N3);
    if (!FS || !M0) { free(FS); free(M0); free(M); free(rhs); free(F); return 2; }
    for (int r = 0; r < N3; ++r) {
        int ri = r % N, rj = (r / N) % N, rk = r / (N * N);
        for (int c2 = 0; c2 < N3; ++c2) {
            int ci = c2 % N, cj = (c2 / N) % N, ck = c2 / (N * N);
            double s = 0.0;
            for (int c = 0; c < N; ++c)
                for (int bq = 0; bq < N; ++bq)
                    for (int a = 0; a < N; ++a)
                        s += J * w[a] * w[bq] * w[c] * L[ri][a] * L[rj][bq] *
                             L[rk][c] * L[ci][a] * L[cj][bq] * L[ck][c];
            M0[r * N3 + c2] = s;
        }
    }

    int status = 0;
    for (int64_t e = 0; e < E && status == 0; ++e) {
        int ex = (int)(e % m->nx);
        int ey = (int)((e / m->nx) % m->ny);
        int ez = (int)(e / ((int64_t)m->nx * m->ny));
        /* flux at every volume quadrature point, from the evaluated polynomial */
        for (int c = 0; c < N; ++c)
            for (int bq = 0; bq < N; ++bq)
                for (int a = 0; a < N; ++a) {
                    double q[NF];
                    eval_poly(m, xi, Q, e, xi[a], xi[bq], xi[c], q);
                    int pt = (c * N + bq) * N + a;
                    for (int d = 0; d < 3; ++d)
                        dgo_flux(d, q, gam, &F[(pt * 3 + d) * NF]);
                }
        /* interface fluxes: both traces evaluated as full polynomials */
        for (int d = 0; d < 3; ++d)
            for (int side = 0; side < 2; ++side) {
                double sgn = side ? 1.0 : -1.0; /* outward normal . e_d */
                int64_t enb = neighbour(m, ex, ey, ez, d, side ? +1 : -1);
                for (int t2 = 0; t2 < N; ++t2)
                    for (int t1 = 0; t1 < N; ++t1) {
                        double pin[3], pnb[3];
                        int tt[2] = {t1, t2}, u = 0;
                        for (int dd = 0; dd < 3; ++dd) {
                            if (dd == d) {
                                pin[dd] = sgn;
                                pnb[dd] = -sgn;
                            } else {
                                pin[dd] = xi[tt[u]];
                                pnb[dd] = xi[tt[u]];
                                ++u;
                            }
                        }
                        double qin[NF], qnb[NF];
                        double *fs = &FS[((d * 2 + side) * N * N + t2 * N + t1) * NF];
                        eval_poly(m, xi, Q, e, pin[0], pin[1], pin[2], qin);
                        eval_poly(m, xi, Q, enb, pnb[0], pnb[1], pnb[2], qnb);
                        if (side) dgo_lf_flux(d, qin, qnb, gam, fs);
                        else dgo_lf_flux(d, qnb, qin, gam, fs);
                    }
            }
        for (int tk = 0; tk < N; ++tk)
            for (int tj = 0; tj < N; ++tj)
                for (int ti = 0; ti < N; ++ti) {
                    int row = (tk * N + tj) * N + ti;
                    double acc[NF] = {0, 0, 0, 0, 0};
                    /* volume term */
                    for (int c = 0; c < N; ++c)
                        for (int bq = 0; bq < N; ++bq)
                            for (int a = 0; a < N; ++a) {
                                int pt = (c * N + bq) * N + a;
                                double wq = J * w[a] * w[bq] * w[c];
                                double gx = (2.0 / h[0]) * dL[ti][a] * L[tj][bq] * L[tk][c];
                                double gy = (2.0 / h[1]) * L[ti][a] * dL[tj][bq] * L[tk][c];
                                double gz = (2.0 / h[2]) * L[ti][a] * L[tj][bq] * dL[tk][c];
                                for (int n = 0; n < NF; ++n)
                                    acc[n] += wq * (F[(pt * 3 + 0) * NF + n] * gx +
                                                    F[(pt * 3 + 1) * NF + n] * gy +
                                                    F[(pt * 3 + 2) * NF + n] * gz);
                            }
                    /* surface term over the six faces */
                    int tix[3] = {ti, tj, tk};
                    for (int d = 0; d < 3; ++d)
                        for (int side = 0; side < 2; ++side) {
                            double sgn = side ? 1.0 : -1.0;
                            for (int t2 = 0; t2 < N; ++t2)
                                for (int t1 = 0; t1 < N; ++t1) {
                                    /* test function at the face point, from Eq. 7 */
                                    int tt[2] = {t1, t2}, u = 0;
                                    double psi = 1.0;
                                    for (int dd = 0; dd < 3; ++dd) {
                                        if (dd == d) {
                                            psi *= Lpm[side][tix[dd]];
                                        } else {
                                            psi *= dgo_lagrange(N, xi, tix[dd], xi[tt[u]]);
                                            ++u;
                                        }
                                    }
                                    const double *fs = &FS[((d * 2 + side) * N * N + t2 * N + t1) * NF];
                                    double wf = sJ[d] * w[t1] * w[t2];
                                    for (int n = 0; n < NF; ++n)
                                        acc[n] -= wf * sgn * fs[n] * psi;
                                }
                        }
                    for (int n = 0; n < NF; ++n) rhs[row * NF + n] = acc[n];
                }
        /* M x = rhs with a fresh copy of M (dense_solve overwrites it) */
        memcpy(M, M0, sizeof(double) * (size_t)N3 * N3);
        if (dense_solve(N3, M, rhs, NF)) { status = 3; break; }
        for (int r = 0; r < N3; ++r)
            for (int n = 0; n < NF; ++n)
                R[((size_t)n * (size_t)E + (size_t)e) * (size_t)N3 + (size_t)r] = rhs[r * NF + n];
    }
    free(FS);
    free(M0);
    free(M);
    free(rhs);
    free(F);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Low-storage Runge-Kutta, Carpenter & Kennedy (1994) 2N-storage (5,4)       */
/* ------------------------------------------------------------------------ */

/* Coefficients of the five-stage fourth-order 2N-storage scheme of
 * M. H. Carpenter and C. A. Kennedy, NASA TM-109112 (1994), the "LSERK45"
 * the paper integrates with (Sec. II.B, Sec. VI.A). */
static const double rk4a[5] = {
    0.0,
    -567301805773.0 / 1357537059087.0,
    -2404267990393.0 / 2016746695238.0,
    -3550918686646.0 / 2091501179385.0,
    -1275806237668.0 / 842570457699.0};
static const double rk4b[5] = {
    1432997174477.0 / 9575080441755.0,
    5161836677717.0 / 13612068292357.0,
    1720146321549.0 / 2090206949498.0,
    3134564353537.0 / 4481467310338.0,
    2277821191437.0 / 14882151754819.0};

void dgo_lserk_coeffs(double A[5], double B[5])
{
    for (int s = 0; s < 5; ++s) { A[s] = rk4a[s]; B[s] = rk4b[s]; }
}

typedef int (*dgo_rhs_fn)(void *ctx, const double *y, double *dydt);

/* One step of the 2N-storage scheme on y (length n), work array k (length n):
 * for s = 1..5:  k <- A_s k + dt f(y);  y <- y + B_s k.
 * A_1 = 0, so k's incoming contents are never read. */
/* stage s's update of the registers from f = dy/dt at the stage's start */
static void lserk_update(int64_t n, double *y, double *k, const double *f, double dt, int s)
{
    for (int64_t i = 0; i < n; ++i) {
        k[i] = (s == 0 ? 0.0 : rk4a[s] * k[i]) + dt * f[i];
        y[i] = y[i] + rk4b[s] * k[i];
    }
}

static int lserk_step(int64_t n, double *y, double *k, double *f, double dt,
                      dgo_rhs_fn rhs, void *ctx)
{
    for (int s = 0; s < 5; ++s) {
        int st = rhs(ctx, y, f);
        if (st) return st;
        lserk_update(n, y, k, f, dt, s);
    }
    return 0;
}

typedef int (*dgo_ode_cb)(int64_t n, const double *y, double *dydt);
typedef struct { dgo_ode_cb cb; int64_t n; } ode_ctx;
static int ode_rhs(void *ctx, const double *y, double *f)
{
    ode_ctx *c = (ode_ctx *)ctx;
    return c->cb(c->n, y, f);
}

/* The same stepper applied to a user ODE y' = cb(y) (used to pin the RK
 * coefficients by their order of accuracy and stability polynomial). */
int dgo_lserk_ode(int64_t n, double *y, int nsteps, double dt, dgo_ode_cb cb)
{
    double *k = (double *)calloc((size_t)n, sizeof(double));
    double *f = (double *)calloc((size_t)n, sizeof(double));
    if (!k || !f) { free(k); free(f); return 2; }
    ode_ctx c = {cb, n};
    int st = 0;
    for (int s = 0; s < nsteps && st == 0; ++s)
        st = lserk_step(n, y, k, f, dt, ode_rhs, &c);
    free(k);
    free(f);
    return st;
}

typedef struct { const dgo_mesh *m; int o1; } dg_ctx;
static int dg_rhs_cb(void *ctx, const double *y, double *f)
{
    dg_ctx *c = (dg_ctx *)ctx;
    return c->o1 ? dgo_rhs_o1(c->m, y, f) : dgo_rhs_o2(c->m, y, f);
}

static size_t state_len(const dgo_mesh *m)
{
    int N = m->p + 1;
    return (size_t)NF * (size_t)n_elem(m) * (size_t)(N * N * N);
}

/* nsteps LSERK45 steps of the O2 right-hand side with a fixed dt, in place on
 * Q.  dQ is the scheme's second register (length of Q; contents ignored on
 * entry, holds the last stage's increment on exit). */
int dgo_rk_steps(const dgo_mesh *m, double *Q, double *dQ, double dt, int nsteps)
{
    if (!mesh_ok(m) || !Q || !dQ) return 1;
    size_t n = state_len(m);
    double *f = (double *)malloc(sizeof(double) * n);
    if (!f) return 2;
    dg_ctx c = {m, 0};
    int st = 0;
    for (int s = 0; s < nsteps && st == 0; ++s)
        st = lserk_step((int64_t)n, Q, dQ, f, dt, dg_rhs_cb, &c);
    free(f);
    return st;
}

/* ------------------------------------------------------------------------ */
/* z slabs (Sec. III, Sec. IV: the mesh is partitioned and neighbouring      */
/* partitions exchange element face data every stage).  A slab is a mesh of  */
/* nz layers of a taller periodic box; its z neighbours beyond its own       */
/* layers belong to other slabs and enter only through their face traces.    */
/* ------------------------------------------------------------------------ */

/* The face traces a slab sends to its z neighbours, in the halo layout
 * H[f][ey*nx + ex][j*N + i]:
 *   lo = the traces of layer 0 at its -z end (the slab below needs them as
 *        its halo_hi),
 *   hi = the traces of layer nz-1 at its +z end (the slab above needs them
 *        as its halo_lo). */
int dgo_ztraces(const dgo_mesh *m, const double *Q, double *lo, double *hi)
{
    if (!mesh_ok(m) || !Q || !lo || !hi) return 1;
    const int N = m->p + 1;
    basis1d b;
    make_basis(N, &b);
    const size_t plane = (size_t)m->nx * (size_t)m->ny;
    for (size_t col = 0; col < plane; ++col)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                double ql[NF], qh[NF];
                collocated_trace(m, &b, Q, (int64_t)col, 2, -1, i, j, ql);
                collocated_trace(m, &b, Q, (int64_t)(col + (size_t)(m->nz - 1) * plane), 2, +1,
                                 i, j, qh);
                for (int f = 0; f < NF; ++f) {
                    lo[((size_t)f * plane + col) * (size_t)(N * N) + (size_t)(j * N + i)] = ql[f];
                    hi[((size_t)f * plane + col) * (size_t)(N * N) + (size_t)(j * N + i)] = qh[f];
                }
            }
    return 0;
}

/* O2 right-hand side of a slab: the trace of the -z neighbour of layer 0
 * is read from halo_lo, that of the +z neighbour of layer nz-1 from halo_hi
 * (layout of dgo_ztraces; both NULL: periodic in z, as dgo_rhs_o2). */
int dgo_rhs_o2_zhalo(const dgo_mesh *m, const double *Q, const double *halo_lo,
                     const double *halo_hi, double *R)
{
    if (!mesh_ok(m) || !Q || !R || (!halo_lo) != (!halo_hi)) return 1;
    const int N = m->p + 1;
    const int N3 = N * N * N;
    basis1d b;
    make_basis(N, &b);
    const int64_t E = n_elem(m);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        double out[NF * NMAX * NMAX * NMAX];
        rhs_o2_element(m, &b, Q, e, halo_lo, halo_hi, out);
        for (int n = 0; n < NF; ++n)
            for (int t = 0; t < N3; ++t) R[qidx(m, n, e, 0, 0, 0) + t] = out[n * N3 + t];
    }
    return 0;
}

/* Stage s (0..4) of the LSERK45 step of a slab, in place:
 * dQ <- A_s dQ + dt R(Q), Q <- Q + B_s dQ, with R from dgo_rhs_o2_zhalo
 * (five stages with periodic z are one dgo_rk_steps step). */
int dgo_rk_stage(const dgo_mesh *m, double *Q, double *dQ, double dt, int s,
                 const double *halo_lo, const double *halo_hi)
{
    if (!mesh_ok(m) || !Q || !dQ || s < 0 || s > 4) return 1;
    size_t n = state_len(m);
    double *f = (double *)malloc(sizeof(double) * n);
    if (!f) return 2;
    int st = dgo_rhs_o2_zhalo(m, Q, halo_lo, halo_hi, f);
    if (st == 0) lserk_update((int64_t)n, Q, dQ, f, dt, s);
    free(f);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Time-step rule, integrals, initial states                                 */
/* ------------------------------------------------------------------------ */

/* Reading (the paper gives no rule): Lambda = max over nodes of
 * sum_d (|u_d| + c), dt = cfl * min(hx,hy,hz) / ((2p+1) Lambda).
 * Writes Lambda to *lambda_out when non-null.  Returns dt, or -1 on a bad
 * argument or a non-positive density/pressure (NaN compares false). */
double dgo_cfl_dt(const dgo_mesh *m, const double *Q, double cfl, double *lambda_out)
{
    if (!mesh_ok(m) || !Q || !(cfl > 0)) return -1.0;
    int N = m->p + 1;
    int64_t E = n_elem(m);
    double lam = 0.0;
    int bad = 0;
    for (int64_t e = 0; e < E; ++e)
        for (int k = 0; k < N; ++k)
            for (int j = 0; j < N; ++j)
                for (int i = 0; i < N; ++i) {
                    double q[NF];
                    load_node(m, Q, e, i, j, k, q);
                    double p = pressure(q, m->gamma);
                    if (!(q[0] > 0) || !(p > 0)) { bad = 1; continue; }
                    double c = sqrt(m->gamma * p / q[0]);
                    double s = (fabs(q[1] / q[0]) + c) + (fabs(q[2] / q[0]) + c) +
                               (fabs(q[3] / q[0]) + c);
                    if (s > lam) lam = s;
                }
    if (bad) return -1.0;
    if (lambda_out) *lambda_out = lam;
    double h = m->Lx / m->nx;
    if (m->Ly / m->ny < h) h = m->Ly / m->ny;
    if (m->Lz / m->nz < h) h = m->Lz / m->nz;
    return cfl * h / ((2.0 * m->p + 1.0) * lam);
}

/* Quadrature integrals with the collocated GL rule (weight J w_i w_j w_k):
 *   out[0..4] = integral of each conserved field
 *   out[5]    = integral of the kinetic energy |rho u|^2 / (2 rho)
 *   out[6]    = relative L2 distance ||Q - Qref|| / ||Qref|| over all five
 *               fields (0 when Qref is NULL). */
int dgo_norms(const dgo_mesh *m, const double *Q, const double *Qref, double out[7])
{
    if (!mesh_ok(m) || !Q || !out) return 1;
    int N = m->p + 1;
    double xi[NMAX], w[NMAX];
    dgo_gl_nodes(N, xi, w);
    double h[3] = {m->Lx / m->nx, m->Ly / m->ny, m->Lz / m->nz};
    double J = h[0] * h[1] * h[2] / 8.0;
    int64_t E = n_elem(m);
    double I[NF] = {0, 0, 0, 0, 0}, ke = 0.0, dd = 0.0, rr = 0.0;
    for (int64_t e = 0; e < E; ++e)
        for (int k = 0; k < N; ++k)
            for (int j = 0; j < N; ++j)
                for (int i = 0; i < N; ++i) {
                    double wq = J * w[i] * w[j] * w[k];
                    double q[NF];
                    load_node(m, Q, e, i, j, k, q);
                    for (int n = 0; n < NF; ++n) I[n] += wq * q[n];
                    ke += wq * 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0];
                    if (Qref) {
                        double r[NF];
                        load_node(m, Qref, e, i, j, k, r);
                        for (int n = 0; n < NF; ++n) {
                            dd += wq * (q[n] - r[n]) * (q[n] - r[n]);
                            rr += wq * r[n] * r[n];
                        }
                    }
                }
    for (int n = 0; n < NF; ++n) out[n] = I[n];
    out[5] = ke;
    out[6] = Qref ? sqrt(dd) / sqrt(rr) : 0.0;
    return 0;
}

/* Initial states at the nodes, written as conservative variables.
 * kind 0, uniform:  params = {rho, u, v, w, p}.
 * kind 1, isentropic vortex, columnar along z (the classical Shu vortex):
 *   params = {beta, xc, yc, u_inf, v_inf, w_inf, t}; the state at time t is
 *   the t = 0 vortex carried by (u_inf, v_inf, w_inf), with minimum-image
 *   displacements on the periodic box:
 *     dx = x - xc - u_inf t, dy = y - yc - v_inf t (wrapped), r^2 = dx^2 + dy^2
 *     u = u_inf - beta/(2 pi) dy e^{(1-r^2)/2},  v = v_inf + beta/(2 pi) dx e^{(1-r^2)/2}
 *     w = w_inf,  T = 1 - (gamma-1) beta^2 / (8 gamma pi^2) e^{1-r^2}
 *     rho = T^{1/(gamma-1)},  p = rho^gamma.
 * kind 2, Taylor-Green vortex: params = {rho0, V0, Mach}:
 *     u = V0 sin x cos y cos z, v = -V0 cos x sin y cos z, w = 0,
 *     p0 = rho0 V0^2 / (gamma Mach^2),
 *     p = p0 + rho0 V0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2),  rho = rho0 p / p0.
 * Node coordinates: x = x0 + (ex + (xi_i + 1)/2) hx, likewise y and z. */
int dgo_state_init(const dgo_mesh *m, int kind, const double *params, int nparams,
                   double *Q)
{
    if (!mesh_ok(m) || !Q) return 1;
    if (kind == 0 && (nparams < 5 || !params)) return 1;
    if (kind == 1 && (nparams < 7 || !params)) return 1;
    if (kind == 2 && (nparams < 3 || !params)) return 1;
    if (kind < 0 || kind > 2) return 1;
    const double pi = 3.14159265358979323846;
    const double gam = m->gamma;
    int N = m->p + 1;
    double xi[NMAX], w[NMAX];
    dgo_gl_nodes(N, xi, w);
    double h[3] = {m->Lx / m->nx, m->Ly / m->ny, m->Lz / m->nz};
    int64_t E = n_elem(m);
    for (int64_t e = 0; e < E; ++e) {
        int ex = (int)(e % m->nx);
        int ey = (int)((e / m->nx) % m->ny);
        int ez = (int)(e / ((int64_t)m->nx * m->ny));
        for (int k = 0; k < N; ++k)
            for (int j = 0; j < N; ++j)
                for (int i = 0; i < N; ++i) {
                    double x = m->x0 + (ex + 0.5 * (xi[i] + 1.0)) * h[0];
                    double y = m->y0 + (ey + 0.5 * (xi[j] + 1.0)) * h[1];
                    double z = m->z0 + (ez + 0.5 * (xi[k] + 1.0)) * h[2];
                    double rho, u, v, ww, p;
                    if (kind == 0) {
                        rho = params[0]; u = params[1]; v = params[2];
                        ww = params[3]; p = params[4];
                    } else if (kind == 1) {
                        double beta = params[0], xc = params[1], yc = params[2];
                        double ui = params[3], vi = params[4], wi = params[5], t = params[6];
                        double dx = x - xc - ui * t, dy = y - yc - vi * t;
                        dx -= m->Lx * round(dx / m->Lx);
                        dy -= m->Ly * round(dy / m->Ly);
                        double r2 = dx * dx + dy * dy;
                        double g = exp(0.5 * (1.0 - r2));
                        u = ui - beta / (2.0 * pi) * dy * g;
                        v = vi + beta / (2.0 * pi) * dx * g;
                        ww = wi;
                        double T = 1.0 - (gam - 1.0) * beta * beta / (8.0 * gam * pi * pi) *
                                             exp(1.0 - r2);
                        rho = pow(T, 1.0 / (gam - 1.0));
                        p = pow(rho, gam);
                    } else {
                        double rho0 = params[0], V0 = params[1], Ma = params[2];
                        double p0 = rho0 * V0 * V0 / (gam * Ma * Ma);
                        u = V0 * sin(x) * cos(y) * cos(z);
                        v = -V0 * cos(x) * sin(y) * cos(z);
                        ww = 0.0;
                        p = p0 + rho0 * V0 * V0 / 16.0 * (cos(2.0 * x) + cos(2.0 * y)) *
                                     (cos(2.0 * z) + 2.0);
                        rho = rho0 * p / p0;
                    }
                    double q[NF] = {rho, rho * u, rho * v, rho * ww,
                                    p / (gam - 1.0) + 0.5 * rho * (u * u + v * v + ww * ww)};
                    for (int n = 0; n < NF; ++n) Q[qidx(m, n, e, i, j, k)] = q[n];
                }
    }
    return 0;
}

/* number of OpenMP threads the O2 loops would use (1 without OpenMP) */
#ifdef _OPENMP
#include <omp.h>
int dgo_num_threads(void) { return omp_get_max_threads(); }
void dgo_set_num_threads(int n) { if (n > 0) omp_set_num_threads(n); }
#else
int dgo_num_threads(void) { return 1; }
void dgo_set_num_threads(int n) { (void)n; }
#endif
