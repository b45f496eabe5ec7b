"""Pins for the oracle's Euler flux (Eq. 2, Eq. 3) and Lax-Friedrichs flux (Sec. II.B)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2006_15698_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _val(tok):
    return float(eval(tok, {"sqrt": math.sqrt}))  # fixture tokens are plain fractions


def test_flux_golden():
    rows = [l.split() for l in open(os.path.join(GOLD, "euler_flux.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 6
    for r in rows:
        d = int(r[1])
        q = np.array([_val(t) for t in r[2:7]])
        f = np.array([_val(t) for t in r[7:12]])
        assert np.max(np.abs(oracle.flux(d, q) - f)) < 1e-14, r


def test_lf_golden():
    rows = [l.split() for l in open(os.path.join(GOLD, "lf_flux.txt")) if l.strip() and not l.startswith("#")]
    for r in rows:
        v = [_val(t) for t in r]
        qL, qR, fs = np.array(v[0:5]), np.array(v[5:10]), np.array(v[10:15])
        assert np.max(np.abs(oracle.lf_flux(0, qL, qR) - fs)) < 1e-14


@pytest.mark.parametrize("seed", range(5))
def test_lf_consistency_and_symmetry(seed):
    qa = inputs.random_state((5, 1), seed)[:, 0]
    qb = inputs.random_state((5, 1), seed + 100)[:, 0]
    for d in range(3):
        # consistency: equal states give the physical flux
        assert np.max(np.abs(oracle.lf_flux(d, qa, qa) - oracle.flux(d, qa))) < 1e-13
        # mirror symmetry: swapping the sides and reversing the normal velocity
        # (reflection x_d -> -x_d) negates the normal flux of mass/energy
        ra, rb = qa.copy(), qb.copy()
        ra[1 + d] *= -1
        rb[1 + d] *= -1
        f = oracle.lf_flux(d, qa, qb)
        g = oracle.lf_flux(d, rb, ra)
        sign = np.ones(5)
        sign[1 + d] = -1  # the normal-momentum flux is even under the reflection
        assert np.max(np.abs(f + sign * g)) < 1e-12


def test_flux_rotation_invariance():
    # rotational invariance: F^y of a state equals F^x of the state with the
    # x and y momentum components exchanged, with the same exchange applied
    q = inputs.random_state((5, 1), 7)[:, 0]
    qs = q[[0, 2, 1, 3, 4]]
    fy = oracle.flux(1, q)
    fx = oracle.flux(0, qs)
    assert np.max(np.abs(fy - fx[[0, 2, 1, 3, 4]])) < 1e-14
