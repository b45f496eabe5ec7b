"""Planted mistakes in the oracle are caught by its pins.

Each case copies oracle/dg_oracle.c, plants one plausible mistake (a dropped
term, a wrong sign or index, a transposed operand, a wrong coefficient),
compiles the copy into a separate library on the CPU, and runs the pin
checks below against it: at least one must fail.  The unmodified oracle
passes all of them (first case).  The checks restate, in compact form, pins
of tests/test_oracle_*.py: hand-worked flux values, the Gauss rule, free
stream, conservation, p = 0 Rusanov finite volumes, brute force = collocated,
the RK stability polynomial, the CFL golden value and convergence to the
isentropic vortex.
"""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle.build import SRC, build_oracle
from paper_2006_15698_gb300 import inputs

MUTANTS = {
    "none": None,
    "lf_dissipation_sign": ("fs[n] = 0.5 * (fL[n] + fR[n]) - 0.5 * lam * (qR[n] - qL[n]);",
                            "fs[n] = 0.5 * (fL[n] + fR[n]) + 0.5 * lam * (qR[n] - qL[n]);"),
    "lift_minus_face_sign": ("(b.lp[i] * fhat[0][1][k * N + j][n] -\n",
                             "(b.lp[i] * fhat[0][1][k * N + j][n] +\n"),
    "pressure_half_dropped": ("return (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w));",
                              "return (gamma - 1.0) * (q[4] - rho * (u * u + v * v + w * w));"),
    "energy_flux_drops_p": ("f[4] = (q[4] + p) * ud;", "f[4] = q[4] * ud;"),
    "derivative_transposed": ("b.dl[i][a] * fx[(k * N + j) * N + a][n];",
                              "b.dl[a][i] * fx[(k * N + j) * N + a][n];"),
    "wrong_neighbour": ("collocated_trace(m, &b, Q, ep, d, -1, t1, t2, qR);",
                        "collocated_trace(m, &b, Q, em, d, -1, t1, t2, qR);"),
    "gauss_weight_factor": ("w[N - 1 - k] = 2.0 / ((1.0 - x * x) * dP * dP);",
                            "w[N - 1 - k] = 1.0 / ((1.0 - x * x) * dP * dP);"),
    "trace_uses_wrong_end": ("const double *l = s > 0 ? b->lp : b->lm;",
                             "const double *l = s > 0 ? b->lm : b->lp;"),
    "rk_coefficient_sign": ("-567301805773.0 / 1357537059087.0,", "567301805773.0 / 1357537059087.0,"),
    "rk_first_stage_weight": ("1432997174477.0 / 9575080441755.0,\n    5161836677717.0",
                              "1432997174477.0 / 9575080441756.0 * 1.001,\n    5161836677717.0"),
    "cfl_order_factor": ("return cfl * h / ((2.0 * m->p + 1.0) * lam);",
                         "return cfl * h / ((2.0 * m->p + 2.0) * lam);"),
    "vortex_velocity_sign": ("u = ui - beta / (2.0 * pi) * dy * g;", "u = ui + beta / (2.0 * pi) * dy * g;"),
    "sound_speed_gamma_dropped": ("double cL = sqrt(gamma * pressure(qL, gamma) / qL[0]);",
                                  "double cL = sqrt(pressure(qL, gamma) / qL[0]);"),
    # a wrong quadrature weight in the brute-force volume sums only
    "o1_volume_weight": ("double wq = J * w[a] * w[bq] * w[c];",
                         "double wq = J * w[a] * w[a] * w[c];"),
}

# pins that must be among the failures of a given mutant
MUST_CATCH = {"o1_volume_weight": "quadrature_exact"}


def _build(name):
    src = open(SRC).read()
    mut = MUTANTS[name]
    if mut is not None:
        old, new = mut
        assert src.count(old) >= 1, f"mutation site not found: {name}"
        src = src.replace(old, new, 1)
    d = tempfile.mkdtemp(prefix="dgo_mut_")
    path = os.path.join(d, "dg_oracle.c")
    with open(path, "w") as f:
        f.write(src)
    import oracle.build as ob
    saved = ob.SRC
    try:
        ob.SRC = path
        lib_path = build_oracle(force=True, out=os.path.join(d, "lib.so"))
    finally:
        ob.SRC = saved
    return oracle.load(lib_path)


def _checks(lib):
    """Names of the pin checks this library fails."""
    failed = []

    def check(name, fn):
        try:
            ok = fn()
        except Exception:
            ok = False
        if not ok:
            failed.append(name)

    q = np.array([2.0, 1.0, -2.0, 4.0, 12.75])
    check("flux_golden", lambda: np.allclose(oracle.flux(0, q, lib=lib), [1, 3.5, -1, 2, 7.875],
                                             atol=1e-13))
    qL = np.array([1, 0, 0, 0, 25 / 14])
    qR = np.array([1, 0.5, 0, 0, 25 / 14 + 1 / 8])
    check("lf_golden", lambda: np.allclose(oracle.lf_flux(0, qL, qR, lib=lib),
                                           [0.25, 5 / 7 - 0.25, 0, 0, 0.5625], atol=1e-13))
    check("gauss_rule", lambda: np.allclose(oracle.gl_nodes(5, lib=lib)[1],
                                            np.polynomial.legendre.leggauss(5)[1], atol=1e-14))
    m = oracle.Mesh(3, 2, 2, 3, Lx=1.0, Ly=1.3, Lz=0.9, lib=lib)
    Qf = m.init("uniform", inputs.uniform_params(1))
    check("free_stream", lambda: np.max(np.abs(m.rhs(Qf))) < 1e-11)
    Qr = inputs.random_state(m.shape, 9)

    def conservation():
        R = m.rhs(Qr)
        return np.max(np.abs(m.norms(R)[:5])) < 1e-11 * np.abs(R).mean() * 1.17

    check("conservation", conservation)

    def o1_o2():
        small = oracle.Mesh(2, 2, 1, 2, Lx=1.0, Ly=1.3, Lz=0.9, lib=lib)
        Q = inputs.random_state(small.shape, 4)
        R1, R2 = small.rhs(Q, "o1"), small.rhs(Q, "o2")
        return np.linalg.norm(R1 - R2) < 1e-12 * np.linalg.norm(R2)

    check("o1_equals_o2", o1_o2)

    def quadrature_exact():
        # continuous polynomial data with a uniform velocity: R = -div F
        # exactly (tests/test_oracle_rhs.py, quadrature exactness)
        from test_oracle_rhs import _exact_case
        nel, p, box = (2, 1, 2), 3, (0.0, 0.0, 0.0, 1.3, 0.8, 1.1)
        mm = oracle.Mesh(*nel, p, *box, lib=lib)
        Q, R, scale = _exact_case(nel, p, box, 3)
        return all(np.max(np.abs(mm.rhs(Q, form) - R)) < 2e-15 * scale for form in ("o1", "o2"))

    check("quadrature_exact", quadrature_exact)

    def p0_fv():
        mm = oracle.Mesh(3, 1, 1, 0, Lx=1.5, Ly=1.0, Lz=1.0, lib=lib)
        Q = inputs.random_state(mm.shape, 2)
        R = mm.rhs(Q).reshape(5, 3)
        U = Q.reshape(5, 3)

        def rus(a, b):
            def ph(x):
                r = x[0]; u = x[1] / r
                p = 0.4 * (x[4] - 0.5 * (x[1] ** 2 + x[2] ** 2 + x[3] ** 2) / r)
                f = np.array([x[1], x[1] * u + p, x[2] * u, x[3] * u, (x[4] + p) * u])
                return f, abs(u) + math.sqrt(1.4 * p / r)
            fa, sa = ph(a)
            fb, sb = ph(b)
            return 0.5 * (fa + fb) - 0.5 * max(sa, sb) * (b - a)

        exp = np.zeros_like(U)
        for e in range(3):
            fp = rus(U[:, e], U[:, (e + 1) % 3])
            fm = rus(U[:, (e - 1) % 3], U[:, e])
            exp[:, e] = -(fp - fm) / 0.5
        return np.max(np.abs(R - exp)) < 1e-12 * np.max(np.abs(exp))

    check("p0_rusanov", p0_fv)

    def stability():
        zs = [0.5 + 0.3j, -1.0 + 0.2j, -2.0 - 1.0j, 0.1 + 1.5j, -0.7 - 0.4j, 1.2 + 0.0j]
        R = []
        for z in zs:
            a, b = z.real, z.imag
            y = oracle.lserk_ode([1.0, 0.0], lambda y: np.array([a * y[0] - b * y[1], b * y[0] + a * y[1]]),
                                 1.0, 1, lib=lib)
            R.append(complex(y[0], y[1]))
        V = np.array([[z ** k for k in range(6)] for z in zs])
        c = np.linalg.solve(V, np.array(R))
        return np.allclose(c, [1, 1, 0.5, 1 / 6, 1 / 24, 1 / 200], atol=1e-12)

    check("rk_stability", stability)

    def cfl():
        mm = oracle.Mesh(2, 2, 2, 2, lib=lib)
        dt, lam = mm.cfl_dt(mm.init("uniform", [1.0, 0.5, -1.0, 2.0, 1 / 1.4]), 0.6)
        return abs(dt - 0.3 / 32.5) < 1e-15

    check("cfl_golden", cfl)

    def convergence():
        errs = []
        for n in (8, 16):
            mm = oracle.Mesh(n, n, 1, 2, Lx=16.0, Ly=16.0, Lz=16.0 / n, lib=lib)
            prm = [3.0, 7.3, 8.6, 0.6, -0.4, 0.3, 0.0]
            Q = mm.init("vortex", prm)
            dt = 0.5 / math.ceil(0.5 / (0.3 * (16.0 / n) / (5 * 7.0)))
            Q, _ = mm.rk_steps(Q, dt, int(round(0.5 / dt)))
            pe = list(prm)
            pe[6] = 0.5
            errs.append(mm.norms(Q, mm.init("vortex", pe))[6])
        return math.log2(errs[0] / errs[1]) > 2.0

    check("vortex_convergence", convergence)
    return failed


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    lib = _build(name)
    failed = _checks(lib)
    if MUTANTS[name] is None:
        assert failed == [], failed
    else:
        assert failed, f"mutant {name} passed every pin"
        if name in MUST_CATCH:
            assert MUST_CATCH[name] in failed, (name, failed)
