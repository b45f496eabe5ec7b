"""Seeded synthetic inputs, shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the DG method: it only draws numbers.  It
imports nothing from the CUDA binding or the oracle, so both sides can be fed
the same inputs without sharing code.

* ``splitmix64`` -- the counter-based generator of Steele, Lea & Flood (2014),
  used for the handful of per-case parameters (vortex strength, centre, drift).
* ``random_state`` -- a positive-density, positive-pressure conservative state
  per node, drawn from numpy's PCG64 (non-smooth data for parity tests).
"""
import numpy as np

NF = 5
MASK64 = (1 << 64) - 1


def splitmix64(state):
    """One step of splitmix64: returns (new_state, 64-bit output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def uniforms(seed, n):
    """n doubles uniform in [0, 1) from splitmix64 seeded with `seed` (53-bit mantissas)."""
    s = seed & MASK64
    out = []
    for _ in range(n):
        s, z = splitmix64(s)
        out.append((z >> 11) * (1.0 / (1 << 53)))
    return out


def vortex_params(seed, box=(0.0, 0.0, 0.0, 10.0, 10.0, 10.0), t=0.0):
    """Isentropic-vortex parameters {beta, xc, yc, u_inf, v_inf, w_inf, t} for a seed.

    beta ~ U[1, 5] (density stays positive for beta < ~10), the centre uniform
    in the box's x-y extent, the drift velocity uniform in [-1, 1]^3.
    """
    x0, y0, _z0, Lx, Ly, _Lz = box
    r = uniforms(seed, 6)
    beta = 1.0 + 4.0 * r[0]
    xc = x0 + Lx * r[1]
    yc = y0 + Ly * r[2]
    uinf, vinf, winf = (2.0 * r[3] - 1.0, 2.0 * r[4] - 1.0, 2.0 * r[5] - 1.0)
    return [beta, xc, yc, uinf, vinf, winf, float(t)]


def tgv_params(mach=0.1):
    """Taylor-Green parameters {rho0, V0, Mach}."""
    return [1.0, 1.0, float(mach)]


def uniform_params(seed):
    """A random uniform state {rho, u, v, w, p} with rho, p > 0."""
    r = uniforms(seed, 5)
    return [0.5 + r[0], 2.0 * r[1] - 1.0, 2.0 * r[2] - 1.0, 2.0 * r[3] - 1.0, 0.5 + 2.0 * r[4]]


def random_state(shape, seed, rho=(0.85, 1.15), vel=0.4, eint=(2.2, 2.8), dtype=np.float64):
    """Independent random conservative state at each node, Q[field][...].

    rho ~ U[rho], velocity components ~ U[-vel, vel], internal energy density
    rho*e ~ U[eint]; the total energy density is rho*e + |rho u|^2 / (2 rho),
    so density and pressure are positive at every node.  The default ranges
    are narrow enough that the polynomial's traces on element faces (which
    extrapolate the nodal values by up to a factor ~4 at p = 6) stay positive.
    """
    g = np.random.Generator(np.random.PCG64(seed))
    shp = tuple(shape[1:]) if shape[0] == NF else tuple(shape)
    r = g.uniform(rho[0], rho[1], shp)
    u = g.uniform(-vel, vel, (3,) + shp)
    ei = g.uniform(eint[0], eint[1], shp)
    Q = np.empty((NF,) + shp, dtype=np.float64)
    Q[0] = r
    Q[1:4] = r * u
    Q[4] = ei + 0.5 * r * (u * u).sum(axis=0)
    return Q.astype(dtype)
