"""dg_advance_host: the state in host memory, copied in, stepped and copied
back by one library call, equals dg_advance on the device copy bit for bit
(state, time steps, integrals), for both precisions and odd and even step
counts, with pinned and pageable host buffers (the double form's pinned
copy-back runs during the last stage, in ranges of z layers: meshes with
fewer layers than ranges, a ragged split and an even one); bad arguments
are refused before any copy."""
import pytest

import oracle
from gpu_helpers import dg_module, to_dev
from paper_2006_15698_gb300 import inputs

pytestmark = pytest.mark.gpu

BOX = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)


@pytest.mark.parametrize("prec,p,nel", [("fp64", 3, (4, 3, 5)), ("fp32", 3, (5, 4, 3)),
                                        ("fp32", 4, (3, 3, 2)), ("fp64", 1, (2, 5, 3)),
                                        ("fp64", 2, (3, 2, 11)), ("fp64", 4, (2, 2, 16))])
@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_host_call_equals_device_call(prec, p, nel, nsteps):
    dg = dg_module()
    import torch
    fp = dg.DG_FP64 if prec == "fp64" else dg.DG_FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    om = oracle.Mesh(*nel, p, *BOX)
    prm = inputs.vortex_params(11 + p, BOX)
    Q0 = to_dev(om.init("vortex", prm), dtype)
    m = dg.Mesh(*nel, p, *BOX, precision=fp)
    Qa, dQa = Q0.clone(), torch.zeros_like(Q0)
    dts_a, integ_a = m.advance(Qa, dQa, 0.5, nsteps)
    for pinned in (True, False):
        Qh = Q0.cpu().pin_memory() if pinned else Q0.cpu()
        Qd, dQd = torch.empty_like(Q0), torch.zeros_like(Q0)
        dts_h, integ_h = m.advance_host(Qh, Qd, dQd, 0.5, nsteps)
        assert not dts_h.is_cuda and not integ_h.is_cuda
        assert torch.equal(Qh, Qa.cpu()), pinned
        assert torch.equal(dts_h, dts_a.cpu()) and torch.equal(integ_h, integ_a.cpu())
    # no integrals requested
    Qh = Q0.cpu().pin_memory()
    dts_n, integ_n = m.advance_host(Qh, Qd, dQd, 0.5, nsteps, with_integrals=False)
    assert integ_n is None and torch.equal(dts_n, dts_a.cpu()) and torch.equal(Qh, Qa.cpu())
    assert m.last_error() == dg.DG_OK


def test_host_call_rejects_bad_arguments_before_copying():
    dg = dg_module()
    import torch
    m = dg.Mesh(3, 2, 2, 2, *BOX)
    Q = m.init("uniform", [1.0, 0.1, 0.2, 0.3, 1.0])
    dQ = torch.zeros_like(Q)
    Qh = torch.full_like(Q, 7.0).cpu()
    dts = torch.zeros(2, dtype=torch.float64)
    for args in ((Qh, Q, dQ, -1.0, 2), (Qh, Q, dQ, 0.5, 0), (Qh, Q, Q, 0.5, 2)):
        with pytest.raises(dg.DGError) as e:
            dg.dg_advance_host(m.h, args[0], args[1], args[2], args[3], args[4], dts, None)
        assert e.value.status == dg.DG_ERR_ARG
    torch.cuda.synchronize()
    # nothing was copied: the device state is still the uniform one
    assert torch.equal(Q, m.init("uniform", [1.0, 0.1, 0.2, 0.3, 1.0]))
    with pytest.raises(ValueError):
        m.advance_host(Q, Q, dQ, 0.5, 1)  # a device tensor as the host state
