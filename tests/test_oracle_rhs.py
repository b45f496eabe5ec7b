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
