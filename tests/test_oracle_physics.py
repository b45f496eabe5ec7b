"""Pins for the oracle's initial states, quadrature integrals, time-step rule,
and the whole semi-discrete scheme through convergence to an exact solution.

The isentropic vortex is an exact solution of the Euler equations (Eq. 1-3):
the DG solution converges to it at high order only if the fluxes, the
Lax-Friedrichs interface flux, the assembly, the RK scheme and the vortex
formula are all right.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2006_15698_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GAM = 1.4


def _pressure(Q):
    r = Q[0]
    return (GAM - 1) * (Q[4] - 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / r)


def _vortex_run(n, p, T=0.5, cfl=0.3, L=16.0):
    m = oracle.Mesh(n, n, 1, p, Lx=L, Ly=L, Lz=L / n)
    prm = [3.0, 7.3, 8.6, 0.6, -0.4, 0.3, 0.0]
    Q = m.init("vortex", prm)
    dt, _ = m.cfl_dt(Q, cfl)
    ns = math.ceil(T / dt)
    Q, _ = m.rk_steps(Q, T / ns, ns)
    pe = list(prm)
    pe[6] = T
    return m.norms(Q, m.init("vortex", pe))[6]


@pytest.mark.slow
@pytest.mark.parametrize("p,ns", [(1, (16, 32, 64)), (2, (16, 32, 64)), (3, (8, 16, 32)), (4, (8, 16, 32))])
def test_vortex_convergence(p, ns):
    # relative L2 error against the exactly advected vortex at t = 0.5 on a
    # 16 x 16 periodic box (non-periodic tail of the vortex ~ 1e-14).  The
    # finest pair must converge at order >= p + 1/2 - 0.1 (the DG error bound
    # for smooth solutions is p + 1/2; p + 1 is typical).
    errs = [_vortex_run(n, p) for n in ns]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(r > 0.5 * (p + 1) for r in rates), (errs, rates)
    assert rates[-1] > p + 0.4, (errs, rates)


def test_cfl_golden():
    # rho = 1, p = 1/1.4 (c = 1): Lambda = |u|+|v|+|w| + 3c
    m = oracle.Mesh(2, 2, 2, 2, Lx=1.0, Ly=1.0, Lz=1.0)
    Q = m.init("uniform", [1.0, 0.0, 0.0, 0.0, 1 / 1.4])
    dt, lam = m.cfl_dt(Q, 0.6)
    assert abs(lam - 3.0) < 1e-14
    assert abs(dt - 0.6 * 0.5 / (5 * 3.0)) < 1e-16  # = 0.02
    Q = m.init("uniform", [1.0, 0.5, -1.0, 2.0, 1 / 1.4])
    dt, lam = m.cfl_dt(Q, 0.6)
    assert abs(lam - 6.5) < 1e-14
    assert abs(dt - 0.3 / 32.5) < 1e-16
    # the maximum over nodes: raise the speed at a single node
    Q = m.init("uniform", [1.0, 0.0, 0.0, 0.0, 1 / 1.4])
    Q[1, 5, 1, 2, 0] = 1.5  # u = 1.5 at one node, its pressure drops accordingly
    p_node = (GAM - 1) * (Q[4, 5, 1, 2, 0] - 0.5 * 1.5 ** 2)
    c_node = math.sqrt(GAM * p_node)
    assert 1.5 + 3 * c_node > 3.0
    dt, lam = m.cfl_dt(Q, 1.0)
    assert abs(lam - (1.5 + 3 * c_node)) < 1e-14
    # a non-positive pressure is reported as an error
    Q[4, 0, 0, 0, 0] = 0.0
    assert m.cfl_dt(Q, 1.0)[0] < 0


def test_norms_exact_for_polynomials():
    # the collocated N-point rule integrates tensor polynomials of degree
    # <= 2N-1 per direction exactly; node coordinates from numpy's leggauss
    nx, ny, nz, p = 3, 2, 2, 2
    N = p + 1
    box = (0.25, -1.0, 0.5, 1.5, 2.0, 1.0)
    m = oracle.Mesh(nx, ny, nz, p, *box)
    xg, _ = np.polynomial.legendre.leggauss(N)
    hx, hy, hz = box[3] / nx, box[4] / ny, box[5] / nz
    ez, ey, ex, k, j, i = np.meshgrid(range(nz), range(ny), range(nx), range(N), range(N), range(N),
                                      indexing="ij")
    x = box[0] + (ex + (xg[i] + 1) / 2) * hx
    y = box[1] + (ey + (xg[j] + 1) / 2) * hy
    z = box[2] + (ez + (xg[k] + 1) / 2) * hz
    Q = np.zeros((5, nz, ny, nx, N, N, N))
    Q[0] = 2.0 + 0 * x
    Q[1] = x ** 5
    Q[2] = x ** 2 * y ** 3 * z ** 4
    Q[3] = y ** 5 - z
    Q[4] = 10.0 + x * y * z
    Q = Q.reshape(5, nx * ny * nz, N, N, N)
    out = m.norms(Q)

    def I(f, a, b):  # exact integral of a monomial
        return (b ** (f + 1) - a ** (f + 1)) / (f + 1)

    X = (box[0], box[0] + box[3])
    Y = (box[1], box[1] + box[4])
    Z = (box[2], box[2] + box[5])
    vol = box[3] * box[4] * box[5]
    exact = [2.0 * vol,
             I(5, *X) * box[4] * box[5],
             I(2, *X) * I(3, *Y) * I(4, *Z),
             I(5, *Y) * box[3] * box[5] - I(1, *Z) * box[3] * box[4],
             10.0 * vol + I(1, *X) * I(1, *Y) * I(1, *Z)]
    assert np.max(np.abs(out[:5] - exact) / np.maximum(1, np.abs(exact))) < 1e-13
    # relative L2 distance: identical arrays give 0; Q vs Q/2 gives 1
    assert m.norms(Q, Q)[6] == 0.0
    assert abs(m.norms(Q, Q / 2)[6] - 1.0) < 1e-14


def test_norms_uniform_state():
    m = oracle.Mesh(2, 3, 1, 3, Lx=2.0, Ly=1.5, Lz=0.5)
    Q = m.init("uniform", [1.2, 0.5, -0.25, 1.0, 2.0])
    out = m.norms(Q)
    vol = 2.0 * 1.5 * 0.5
    rhoE = 2.0 / 0.4 + 0.5 * 1.2 * (0.25 + 0.0625 + 1.0)
    expect = np.array([1.2, 0.6, -0.3, 1.2, rhoE]) * vol
    assert np.max(np.abs(out[:5] - expect)) < 1e-13
    assert abs(out[5] - 0.5 * 1.2 * 1.3125 * vol) < 1e-13


def test_tgv_golden_point():
    row = [l.split() for l in open(os.path.join(GOLD, "tgv_point.txt")) if l.strip() and not l.startswith("#")][0]
    rho, u, v, w, p = (float(eval(t, {"sqrt": math.sqrt})) for t in row)
    # one p = 0 element of size 2pi centred at (pi/6, pi/6, 0)
    c = (math.pi / 6, math.pi / 6, 0.0)
    m = oracle.Mesh(1, 1, 1, 0, c[0] - math.pi, c[1] - math.pi, c[2] - math.pi,
                    2 * math.pi, 2 * math.pi, 2 * math.pi)
    Q = m.init("tgv", inputs.tgv_params(0.1))[:, 0, 0, 0, 0]
    expect = np.array([rho, rho * u, rho * v, rho * w, 2.5 * p + rho * 3 / 16])
    assert np.max(np.abs(Q - expect) / np.abs(expect).clip(1)) < 1e-14


@pytest.mark.parametrize("seed", range(3))
def test_vortex_isentropic_and_centre(seed):
    box = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)
    prm = inputs.vortex_params(seed, box)
    m = oracle.Mesh(4, 4, 2, 3, *box)
    Q = m.init("vortex", prm)
    rho = Q[0]
    p = _pressure(Q)
    assert np.max(np.abs(p - rho ** GAM)) < 1e-13  # isentropic: p = rho^gamma
    # velocity along z is the drift everywhere
    assert np.max(np.abs(Q[3] / Q[0] - prm[5])) < 1e-14
    # centre value: one p = 0 element centred on the vortex centre
    beta = prm[0]
    m1 = oracle.Mesh(1, 1, 1, 0, prm[1] - 5, prm[2] - 5, 0, 10, 10, 10)
    q = m1.init("vortex", prm)[:, 0, 0, 0, 0]
    rc = (1 - (GAM - 1) * beta ** 2 / (8 * GAM * math.pi ** 2) * math.e) ** (1 / (GAM - 1))
    assert abs(q[0] - rc) < 1e-14
    assert abs(q[1] / q[0] - prm[3]) < 1e-14 and abs(q[2] / q[0] - prm[4]) < 1e-14


def test_vortex_translation():
    # the state at time t equals the t = 0 state with the centre moved by
    # the drift times t, wrapped on the periodic box
    box = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)
    prm = inputs.vortex_params(4, box)
    m = oracle.Mesh(5, 5, 1, 2, *box)
    t = 13.7
    a = list(prm)
    a[6] = t
    b = list(prm)
    b[1] = (prm[1] + prm[3] * t) % 10.0
    b[2] = (prm[2] + prm[4] * t) % 10.0
    Qa = m.init("vortex", a)
    Qb = m.init("vortex", b)
    assert np.max(np.abs(Qa - Qb)) < 1e-11
