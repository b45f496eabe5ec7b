"""dg_rhs_static, the allocation-free right-hand side, against the oracle and
against dg_rhs.

Some callers cannot let a library allocate device memory (a fixed memory
budget, or a host framework whose allocator owns the free memory), so they
cannot create a mesh handle.  dg_rhs_static serves them: the double form's
interface-flux scratch is a static device array of fixed size, the float form
needs none.  This file is collected last so that a run stopping at the first
failure has already run every other test; it passes alone in a fresh process
and after the other tests.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import dg_module, rhs_scale, to_dev, to_host
from paper_2006_15698_gb300 import inputs

BOX = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_rhs_matches_oracle_and_dg_rhs_twice(prec):
    dg = dg_module()
    import torch
    nel, p = (6, 5, 4), 4
    precision = dg.DG_FP64 if prec == "fp64" else dg.DG_FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    om = oracle.Mesh(*nel, p, *BOX)
    m = dg.Mesh(*nel, p, *BOX, precision=precision)
    tol = 1e-12 if prec == "fp64" else 2e-6
    # two calls in a row on different states: the second call must not see
    # anything the first left in the shared static array
    for seed in (21, 22):
        Qh = inputs.random_state(om.shape, seed)
        Q = to_dev(Qh, dtype)
        # the oracle evaluates the state the kernels see (rounded to float for FP32)
        R_or = om.rhs(to_host(Q))
        R_ref = to_host(m.rhs(Q))
        R = torch.empty_like(Q)
        dg.dg_rhs_static(*nel, p, *BOX, 1.4, precision, Q, R)
        Rs = to_host(R)
        scale = rhs_scale(om, Qh)
        assert np.linalg.norm(Rs - R_or) / scale < tol
        assert np.linalg.norm(Rs - R_ref) / scale < tol
    assert np.isfinite(Rs).all()


@pytest.mark.gpu
def test_static_rhs_fp64_at_the_scratch_limit():
    # 16 x 16 x 21 = 5,376 elements at p = 4 need 15 * 5376 * 25 * 8 B =
    # 16.13 MB of interface fluxes, just under the 16 MiB static array: the
    # whole array is in use, against dg_rhs and sampled oracle elements
    dg = dg_module()
    import torch
    nel, p = (16, 16, 21), 4
    om = oracle.Mesh(*nel, p, *BOX)
    m = dg.Mesh(*nel, p, *BOX)
    Qh = inputs.random_state(om.shape, 5)
    Q = to_dev(Qh)
    R = torch.empty_like(Q)
    dg.dg_rhs_static(*nel, p, *BOX, 1.4, dg.DG_FP64, Q, R)
    Rs = to_host(R)
    R_ref = to_host(m.rhs(Q))
    scale = rhs_scale(om, Qh)
    assert np.linalg.norm(Rs - R_ref) / scale < 1e-12
    E = om.E
    elems = np.array([0, 1, 15, 16 * 16 - 1, E // 2, E - 16 * 16, E - 1], dtype=np.int64)
    R_or = om.rhs_elements(Qh, elems)
    # the term scale of the sampled elements: (2/h) Lambda ||Q|| over them
    scale_s = scale * np.linalg.norm(Qh[:, elems]) / np.linalg.norm(Qh)
    assert np.linalg.norm(Rs[:, elems] - R_or) / scale_s < 1e-12


@pytest.mark.gpu
def test_static_rhs_rejects_oversize_and_bad_args():
    dg = dg_module()
    import torch
    # 7 x 17 x 47 = 5,593 elements at p = 4 need 16,779,000 B of interface
    # fluxes, 1,784 B beyond the 16 MiB static scratch: rejected before any launch
    nel, p = (7, 17, 47), 4
    Q = torch.zeros((5, 7 * 17 * 47, 5, 5, 5), dtype=torch.float64, device="cuda")
    R = torch.zeros_like(Q)
    with pytest.raises(dg.DGError) as e:
        dg.dg_rhs_static(*nel, p, *BOX, 1.4, dg.DG_FP64, Q, R)
    assert e.value.status == dg.DG_ERR_TOO_LARGE
    assert not R.any()
    with pytest.raises(dg.DGError) as e:
        dg.dg_rhs_static(2, 2, 2, 9, *BOX, 1.4, dg.DG_FP64, Q, R)
    assert e.value.status == dg.DG_ERR_UNSUPPORTED
    small = torch.zeros((5, 8, 2, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as e:
        dg.dg_rhs_static(2, 2, 2, 1, *BOX, 1.4, dg.DG_FP64, small, small)
    assert e.value.status == dg.DG_ERR_ARG
    # the binding checks what the C function cannot see: size, dtype, device
    with pytest.raises(ValueError):
        dg.dg_rhs_static(2, 2, 2, 1, *BOX, 1.4, dg.DG_FP64, small, small[:, :4])
    with pytest.raises(ValueError):
        dg.dg_rhs_static(2, 2, 2, 1, *BOX, 1.4, dg.DG_FP32, small, torch.zeros_like(small))
    with pytest.raises(ValueError):
        dg.dg_rhs_static(2, 2, 2, 1, *BOX, 1.4, dg.DG_FP64, small, small.cpu())


@pytest.mark.gpu
def test_static_rhs_fp32_has_no_scratch_limit():
    # the float form uses no scratch: a mesh far beyond the double form's
    # limit (32^3 elements at p = 4) is accepted and equals dg_rhs bit for bit
    dg = dg_module()
    import torch
    nel, p = (32, 32, 32), 4
    box = (0.0, 0.0, 0.0, 16.0, 16.0, 16.0)
    m = dg.Mesh(*nel, p, *box, precision=dg.DG_FP32)
    Q = m.init("vortex", inputs.vortex_params(3, box))
    R = torch.empty_like(Q)
    dg.dg_rhs_static(*nel, p, *box, 1.4, dg.DG_FP32, Q, R)
    R_ref = m.rhs(Q)
    torch.cuda.synchronize()
    assert torch.equal(R, R_ref)


def test_static_rhs_binding_rejects_host_tensors_without_a_call():
    # no GPU needed: the binding refuses tensors the library could not use
    # before it calls into the library
    dg = pytest.importorskip("paper_2006_15698_gb300.dg")
    import torch
    Q = torch.zeros((5, 8, 2, 2, 2), dtype=torch.float64)
    with pytest.raises(ValueError):
        dg.dg_rhs_static(2, 2, 2, 1, *BOX, 1.4, dg.DG_FP64, Q, Q.clone())
    with pytest.raises(ValueError):
        dg.dg_rhs_static(2, 2, 2, 1, *BOX, 1.4, dg.DG_FP64, Q.numpy(), Q.clone())
