"""Pins for the oracle's five-stage low-storage Runge-Kutta scheme (Sec. II.B, Sec. VI.A).

The coefficients (Carpenter & Kennedy 1994) are checked by what they must
achieve, through the same stepper the DG step uses: the linear stability
polynomial (order conditions up to fourth order) and fourth-order convergence
on a nonlinear system with a closed-form solution.
"""
import math

import numpy as np

import oracle


def _linear_step(z):
    # y' = lambda y, dt = 1, complex lambda written as a real 2-system
    a, b = z.real, z.imag

    def f(y):
        return np.array([a * y[0] - b * y[1], b * y[0] + a * y[1]])

    y = oracle.lserk_ode([1.0, 0.0], f, 1.0, 1)
    return complex(y[0], y[1])


def test_stability_polynomial():
    # one step on y' = lambda y multiplies y by R(z), z = lambda dt, a quintic.
    # Fourth order fixes its first five coefficients to 1, 1, 1/2, 1/6, 1/24.
    zs = [complex(np.cos(t), np.sin(t)) * r for t, r in
          [(0.3, 0.5), (1.9, 1.2), (2.8, 2.0), (3.1, 0.1), (-1.0, 0.7), (0.0, 1.5)]]
    R = np.array([_linear_step(z) for z in zs])
    V = np.array([[z ** k for k in range(6)] for z in zs])
    c = np.linalg.solve(V, R)
    expect = [1, 1, 0.5, 1 / 6, 1 / 24]
    assert np.max(np.abs(c[:5] - expect)) < 1e-12
    # the fifth coefficient of this scheme is 1/200
    assert abs(c[5] - 1 / 200) < 1e-12
    assert np.max(np.abs(c.imag)) < 1e-12


def test_fourth_order_nonlinear():
    # y' = -2 t y^2, t' = 1 (autonomous form of a non-autonomous problem),
    # y(0) = 1 -> y(t) = 1 / (1 + t^2)
    def f(y):
        return np.array([-2.0 * y[1] * y[0] ** 2, 1.0])

    errs = []
    for n in (10, 20, 40, 80):
        y = oracle.lserk_ode([1.0, 0.0], f, 2.0 / n, n)
        errs.append(abs(y[0] - 1 / 5))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(rates[1:]) > 3.8 and max(rates) < 4.3, rates


def test_coefficient_consistency():
    # sum of the effective stage weights equals 1 (first-order condition),
    # checked directly on the 2N-storage coefficients: one step of y' = 1 from 0
    y = oracle.lserk_ode([0.0], lambda y: np.array([1.0]), 0.37, 1)
    assert abs(y[0] - 0.37) < 1e-15
