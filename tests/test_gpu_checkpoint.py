"""Resume from a checkpoint on the GPU: n steps through dg_advance, or n/2
steps, a checkpoint written and read back into a new mesh, then n/2 more,
give the same state and time steps bit for bit (both precisions)."""
import pytest

import oracle
from gpu_helpers import dg_module, to_dev
from paper_2006_15698_gb300 import checkpoint, inputs

pytestmark = pytest.mark.gpu

BOX = (0.0, 0.0, 0.0, 10.0, 10.0, 10.0)


@pytest.mark.parametrize("prec,p,nel", [("fp64", 3, (4, 3, 5)), ("fp32", 4, (3, 4, 3)),
                                        ("fp32", 3, (5, 2, 4))])
def test_resume_continues_bit_for_bit(tmp_path, prec, p, nel):
    dg = dg_module()
    import torch
    fp = dg.DG_FP64 if prec == "fp64" else dg.DG_FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    om = oracle.Mesh(*nel, p, *BOX)
    Q0 = to_dev(om.init("vortex", inputs.vortex_params(21 + p, BOX)), dtype)
    m = dg.Mesh(*nel, p, *BOX, precision=fp)
    Qa, dQa = Q0.clone(), torch.zeros_like(Q0)
    dts_a, _ = m.advance(Qa, dQa, 0.5, 6)

    Qb, dQb = Q0.clone(), torch.zeros_like(Q0)
    dts_b1, _ = m.advance(Qb, dQb, 0.5, 3)
    path = str(tmp_path / "run.ck")
    checkpoint.save(path, m.spec, Qb, 3, float(dts_b1.sum()), extra={"dts": dts_b1.tolist()})
    del Qb, dQb
    m2, Qc, step, t, extra = checkpoint.restore(path)
    assert step == 3 and extra["dts"] == dts_b1.tolist() and m2.spec == m.spec
    dQc = torch.zeros_like(Qc)
    dts_c, _ = m2.advance(Qc, dQc, 0.5, 3)
    torch.cuda.synchronize()
    assert torch.equal(torch.cat([dts_b1, dts_c]), dts_a)
    assert torch.equal(Qc, Qa)
    assert t == float(dts_a[:3].sum())
