"""dg_rhs_static, the allocation-free right-hand side, against dg_rhs.

Some callers cannot let a library allocate device memory (a fixed memory
budget, or a host framework whose allocator owns the free memory), so they
cannot create a mesh handle.  dg_rhs_static serves them: its interface-flux
scratch is a static device array.  This file is collected last so that a run
stopping at the first failure has already run every other test; it passes
alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import dg_module, rhs_scale, to_dev, to_host
from paper_2006_15698_gb300 import inputs

pytestmark = pytest.mark.gpu

BOX = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_rhs_matches_dg_rhs_twice(prec):
    dg = dg_module()
    import torch
    nel, p = (6, 5, 4), 4
    precision = dg.DG_FP64 if prec == "fp64" else dg.DG_FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    om = oracle.Mesh(*nel, p, *BOX)
    m = dg.Mesh(*nel, p, *BOX, precision=precision)
    # two calls in a row on different states: the second call must not see
    # anything the first left in the shared static array
    for seed in (21, 22):
        Qh = inputs.random_state(om.shape, seed)
        Q = to_dev(Qh, dtype)
        R_ref = to_host(m.rhs(Q))
        R = torch.empty_like(Q)
        dg.dg_rhs_static(*nel, p, *BOX, 1.4, precision, Q, R)
        Rs = to_host(R)
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.linalg.norm(Rs - R_ref) / rhs_scale(om, Qh) < tol
    assert np.isfinite(Rs).all()


def test_static_rhs_rejects_oversize_and_bad_args():
    dg = dg_module()
    import torch
    Q = torch.zeros(16, dtype=torch.float64, device="cuda")
    R = torch.zeros(16, dtype=torch.float64, device="cuda")
    # 32^3 elements at p = 4 need 15 * 32768 * 25 * 8 B = 98 MB of interface
    # fluxes, beyond the 16 MiB static scratch: rejected before any launch
    with pytest.raises(dg.DGError) as e:
        dg.dg_rhs_static(32, 32, 32, 4, *BOX, 1.4, dg.DG_FP64, Q, R)
    assert e.value.status == dg.DG_ERR_TOO_LARGE
    with pytest.raises(dg.DGError) as e:
        dg.dg_rhs_static(2, 2, 2, 9, *BOX, 1.4, dg.DG_FP64, Q, R)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
    with pytest.raises(dg.DGError) as e:
        dg.dg_rhs_static(2, 2, 2, 1, *BOX, 1.4, dg.DG_FP64, Q, Q)
    assert e.value.status == dg.DG_ERR_ARG
