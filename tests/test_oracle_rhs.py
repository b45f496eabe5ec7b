"""Pins for the oracle's DG right-hand side (Eq. 5 with the basis of Eq. 7).

Free-stream preservation, discrete conservation on periodic meshes, axis
symmetries, the p = 0 reduction to the first-order Rusanov finite-volume
scheme, and agreement of the brute-force quadrature (O1) with the collocated
loops (O2).  A dropped term, a wrong sign, index or transposed operand in the
assembly breaks at least one of them.
"""
import numpy as np
import pytest

import oracle
from paper_2006_15698_gb300 import inputs


def _mesh(n, p, L=(1.0, 1.0, 1.0), **kw):
    if isinstance(n, int):
        n = (n, n, n)
    return oracle.Mesh(*n, p, Lx=L[0], Ly=L[1], Lz=L[2], **kw)


@pytest.mark.parametrize("p", range(0, 7))
def test_free_stream(p):
    m = _mesh((3, 2, 2), p, L=(1.5, 0.7, 2.0))
    for seed in range(3):
        Q = m.init("uniform", inputs.uniform_params(seed))
        R = m.rhs(Q)
        scale = np.max(np.abs(Q)) * 3 / min(m.box[3:]) * (p + 1) ** 2
        assert np.max(np.abs(R)) < 1e-13 * scale


@pytest.mark.parametrize("p", range(0, 7))
def test_conservation_random_data(p):
    # sum_e sum_ijk J w_i w_j w_k dQ/dt = 0 for every field on a periodic mesh,
    # even for non-smooth data: every face flux enters its two elements with
    # opposite signs and the volume term integrates the derivative of a test
    # function that sums to one.
    m = _mesh((3, 2, 2), p, L=(1.0, 2.0, 1.5))
    Q = inputs.random_state(m.shape, 11 + p)
    R = m.rhs(Q)
    I = m.norms(R)[:5]
    scale = np.sum(np.abs(R)) / R.size * np.prod(m.box[3:])
    assert np.max(np.abs(I)) < 1e-12 * scale


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("p", range(0, 7))
def test_o1_equals_o2(n, p):
    # n = 1 makes each element its own neighbour in every direction
    if n == 3 and p >= 5:
        pytest.skip("brute force too slow for 27 elements at p >= 5; covered at n <= 2")
    m = _mesh((n, n, max(1, n - 1)), p, L=(1.0, 1.3, 0.9))
    Q = inputs.random_state(m.shape, 100 * n + p)
    R1 = m.rhs(Q, "o1")
    R2 = m.rhs(Q, "o2")
    # a single p = 0 element is its own neighbour with equal traces: R = 0
    scale = max(np.linalg.norm(R2), 1e-300 if n * (p + 1) > 1 else np.linalg.norm(Q))
    err = np.linalg.norm(R1 - R2) / scale
    assert err < 1e-13, err


def _cyclic(A):
    """(x,y,z) -> (y,z,x) relabelling of a cubic mesh state: the new state at
    (x,y,z) is the old state at (y,z,x) with the momentum components
    reassigned (new m_x = old m_z, new m_y = old m_x, new m_z = old m_y)."""
    n = round(A.shape[1] ** (1 / 3))
    N = A.shape[2]
    B = A.reshape(5, n, n, n, N, N, N)  # (f, ez, ey, ex, k, j, i)
    B = B.transpose(0, 2, 3, 1, 5, 6, 4)
    B = B[[0, 3, 1, 2, 4]]
    return np.ascontiguousarray(B).reshape(A.shape)


def _mirror(A, d, nel):
    """Reflection x_d -> -x_d of a state: reverse element and node order along d
    and negate the d-momentum."""
    nx, ny, nz = nel
    N = A.shape[2]
    B = A.reshape(5, nz, ny, nx, N, N, N).copy()
    eax = {0: 3, 1: 2, 2: 1}[d]
    nax = {0: 6, 1: 5, 2: 4}[d]
    B = np.flip(np.flip(B, axis=eax), axis=nax)
    B[1 + d] *= -1
    return np.ascontiguousarray(B).reshape(A.shape)


@pytest.mark.parametrize("p", [0, 1, 2, 4])
def test_cyclic_axis_symmetry(p):
    m = _mesh(3, p)
    Q = inputs.random_state(m.shape, 5 + p)
    R = m.rhs(Q)
    Rp = m.rhs(_cyclic(Q))
    assert np.max(np.abs(Rp - _cyclic(R))) < 1e-12 * np.max(np.abs(R))


@pytest.mark.parametrize("p", [0, 1, 3])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_mirror_symmetry(p, d):
    nel = (3, 2, 4)
    m = _mesh(nel, p, L=(1.0, 0.8, 1.2))
    Q = inputs.random_state(m.shape, 40 + p + d)
    R = m.rhs(Q)
    Rm = m.rhs(_mirror(Q, d, nel))
    assert np.max(np.abs(Rm - _mirror(R, d, nel))) < 1e-12 * np.max(np.abs(R))


def _rusanov(qL, qR, d, gam=1.4):
    """Textbook Rusanov flux for the Euler equations (independent of the oracle)."""
    def prim(q):
        r = q[0]
        vel = q[1:4] / r
        p = (gam - 1) * (q[4] - 0.5 * r * np.sum(vel * vel, axis=0))
        return r, vel, p

    def phys(q):
        r, vel, p = prim(q)
        un = vel[d]
        f = np.empty_like(q)
        f[0] = r * un
        for k in range(3):
            f[1 + k] = q[1 + k] * un + (p if k == d else 0)
        f[4] = (q[4] + p) * un
        return f, np.abs(un) + np.sqrt(gam * p / r)

    fL, sL = phys(qL)
    fR, sR = phys(qR)
    return 0.5 * (fL + fR) - 0.5 * np.maximum(sL, sR) * (qR - qL)


@pytest.mark.parametrize("nel", [(2, 2, 2), (3, 2, 4), (5, 1, 1)])
def test_p0_is_first_order_rusanov_fv(nel):
    # with p = 0 the DG scheme is the cell-centred finite-volume scheme
    # dQ/dt = -sum_d (F*_{d+} - F*_{d-}) / h_d
    nx, ny, nz = nel
    L = (1.0, 0.5, 2.0)
    m = _mesh(nel, 0, L=L)
    Q = inputs.random_state(m.shape, 3)
    R = m.rhs(Q)
    U = Q.reshape(5, nz, ny, nx)
    h = (L[0] / nx, L[1] / ny, L[2] / nz)
    expect = np.zeros_like(U)
    for d, ax in ((0, 3), (1, 2), (2, 1)):
        Up = np.roll(U, -1, axis=ax)  # +d neighbour
        fplus = _rusanov(U, Up, d)
        fminus = np.roll(fplus, 1, axis=ax)
        expect -= (fplus - fminus) / h[d]
    assert np.max(np.abs(R.reshape(U.shape) - expect)) < 1e-13 * np.max(np.abs(expect))


# --------------------------------------------------------------------------
# Quadrature exactness (Sec. II.B, Eqs. 5-7): data for which every integral
# of the weak form is a polynomial that the N-point Gauss rule integrates
# exactly, so the discrete right-hand side must equal the exact one.
#
# Take a uniform velocity u0 and a density rho and total energy E that are
# continuous, periodic, piecewise polynomials of degree <= p per direction
# (the momentum is rho u0).  Then every Euler flux component is linear in
# (rho, E), hence of degree <= p per direction, and:
#   * the volume integrand F . grad psi has degree <= 2p+1 per direction,
#     the face integrand F . n psi and the mass integrand psi psi degree 2p:
#     all integrated exactly by N = p+1 Gauss points;
#   * the traces agree on both sides of every face (continuity), so the
#     Lax-Friedrichs dissipation vanishes and F* = F(Q);
#   * integrating by parts, M R = -int (div F) psi, and div F is itself of
#     degree <= p per direction, so R = -div F exactly at the nodes.
# The expected value below is -div F from the product rule on the known
# polynomials (numpy's Gauss nodes, no oracle code).
# --------------------------------------------------------------------------

def _periodic_profile(coef, ne, xi, h):
    """Values and x-derivatives at the nodes of a continuous periodic
    piecewise polynomial on ne (1 or 2) elements of size h: element e holds
    g(s_e xi) with s_e = (-1)^e, g(t) = sum_k coef[k] t^k (for ne = 1, g must
    be even so that g(-1) = g(+1)).  Returns arrays of shape (ne, N)."""
    g = np.polynomial.Polynomial(coef)
    dg = g.deriv()
    val = np.empty((ne, xi.size))
    der = np.empty((ne, xi.size))
    for e in range(ne):
        s = 1.0 if e % 2 == 0 else -1.0
        val[e] = g(s * xi)
        der[e] = dg(s * xi) * s * (2.0 / h)
    return val, der


def _exact_case(nel, p, box, seed, gam=1.4):
    """(Q, -div F) at the nodes of the mesh for the construction above."""
    N = p + 1
    xi, _ = np.polynomial.legendre.leggauss(N)
    rng = np.random.Generator(np.random.PCG64(seed))
    h = [box[3 + d] / nel[d] for d in range(3)]
    u0 = rng.uniform(-0.5, 0.5, 3)

    def field_profiles():
        prof = []
        for d in range(3):
            c = rng.uniform(-1.0, 1.0, N)
            if nel[d] == 1:
                c[1::2] = 0.0  # even: continuous across the periodic wrap
            # scaled so that |g| <= 1 on [-1, 1]
            c /= max(np.max(np.abs(np.polynomial.Polynomial(c)(np.linspace(-1, 1, 401)))), 1e-300)
            prof.append(_periodic_profile(c, nel[d], xi, h[d]))
        return prof

    def assemble(prof, base, amp):
        """base + amp * phi_x phi_y phi_z and its gradient, in the state layout
        (element e = ex + nx (ey + ny ez), node (i, j, k), i fastest)."""
        nx, ny, nz = nel
        (vx, dx), (vy, dy), (vz, dz) = prof
        # axes (ez, ey, ex, k, j, i)
        X = vx[None, None, :, None, None, :]
        Y = vy[None, :, None, None, :, None]
        Z = vz[:, None, None, :, None, None]
        dX = dx[None, None, :, None, None, :]
        dY = dy[None, :, None, None, :, None]
        dZ = dz[:, None, None, :, None, None]
        shp = (nz, ny, nx, N, N, N)
        f = base + amp * np.broadcast_to(X * Y * Z, shp)
        grad = [amp * np.broadcast_to(dX * Y * Z, shp), amp * np.broadcast_to(X * dY * Z, shp),
                amp * np.broadcast_to(X * Y * dZ, shp)]
        E = nx * ny * nz
        return f.reshape(E, N, N, N), [gg.reshape(E, N, N, N) for gg in grad]

    # rho in [0.7, 1.3], E in [2, 4]: density and pressure stay positive
    rho, drho = assemble(field_profiles(), 1.0, 0.3)
    En, dE = assemble(field_profiles(), 3.0, 1.0)
    uu = float(u0 @ u0)
    Q = np.empty((5,) + rho.shape)
    Q[0] = rho
    for k in range(3):
        Q[1 + k] = rho * u0[k]
    Q[4] = En
    dp = [(gam - 1.0) * (dE[d] - 0.5 * uu * drho[d]) for d in range(3)]
    R = np.empty_like(Q)
    R[0] = -sum(u0[d] * drho[d] for d in range(3))
    for k in range(3):
        R[1 + k] = -sum(u0[k] * u0[d] * drho[d] for d in range(3)) - dp[k]
    R[4] = -sum(u0[d] * (dE[d] + dp[d]) for d in range(3))
    # size of the individual terms summed into R: derivative ~ (2/h) N^2 |F|
    scale = 2.0 / min(h) * N * N * np.max(np.abs(Q)) * (1 + np.abs(u0).max()) ** 2
    return Q, R, scale


@pytest.mark.parametrize("p", range(0, 7))
@pytest.mark.parametrize("nel", [(1, 1, 1), (2, 1, 2), (2, 2, 2)])
def test_quadrature_exact_brute_force(nel, p):
    # O1 evaluates psi, grad psi and the state from Eq. 7 at every quadrature
    # point and forms the full sums of Eq. 5: it must reproduce -div F
    box = (0.0, 0.0, 0.0, 1.3, 0.8, 1.1)
    m = oracle.Mesh(*nel, p, *box)
    Q, R_exact, scale = _exact_case(nel, p, box, 17 * p + sum(nel))
    R1 = m.rhs(Q, "o1")
    # double rounding of ~N^2 terms of size <= scale/N^2: ~1e-16 scale observed
    assert np.max(np.abs(R1 - R_exact)) < 2e-15 * scale


@pytest.mark.parametrize("p", range(0, 7))
def test_quadrature_exact_collocated(p):
    # the same for the collocated loops O2 (the GPU's reference)
    nel = (2, 2, 2)
    box = (0.5, -0.2, 0.0, 0.9, 1.4, 1.2)
    m = oracle.Mesh(*nel, p, *box)
    Q, R_exact, scale = _exact_case(nel, p, box, 5 + p)
    R2 = m.rhs(Q)
    assert np.max(np.abs(R2 - R_exact)) < 2e-15 * scale


def test_quadrature_exact_case_is_not_trivial():
    # the construction exercises every field and every direction: the exact
    # right-hand side is far from zero in each field at p = 3
    nel, p, box = (2, 2, 2), 3, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
    Q, R, scale = _exact_case(nel, p, box, 1)
    for n in range(5):
        assert np.max(np.abs(R[n])) > 1e-3 * scale
