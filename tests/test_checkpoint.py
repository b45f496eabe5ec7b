"""Checkpoint files on the host (no GPU): a state, its step count, time and
mesh arguments survive a round trip exactly, and damaged or foreign files
are refused before anything is returned."""
import io
import json

import numpy as np
import pytest

from paper_2006_15698_gb300 import checkpoint

torch = pytest.importorskip("torch")

SPEC = dict(nx=3, ny=2, nz=4, p=2, x0=0.0, y0=0.0, z0=0.0, Lx=10.0, Ly=10.0, Lz=10.0,
            gamma=1.4, precision=0)


def _state(dtype, seed=0):
    g = torch.Generator().manual_seed(seed)
    return torch.rand((5, 24, 3, 3, 3), generator=g, dtype=torch.float64).to(dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_round_trip_is_exact(tmp_path, dtype):
    Q = _state(dtype)
    path = str(tmp_path / "ck")
    checkpoint.save(path, SPEC, Q, 17, 0.123456789, extra={"dts": [0.01, 0.02]})
    spec, Q2, step, t, extra = checkpoint.load(path)
    assert spec == SPEC and step == 17 and t == 0.123456789 and extra == {"dts": [0.01, 0.02]}
    assert Q2.dtype == dtype and torch.equal(Q2, Q)


def _rewrite(buf, mutate):
    buf.seek(0)
    with np.load(buf) as z:
        q, meta = np.array(z["Q"]), json.loads(bytes(z["meta"]).decode())
    q, meta = mutate(q, meta)
    out = io.BytesIO()
    np.savez(out, Q=q, meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8))
    out.seek(0)
    return out


def test_damaged_or_foreign_files_are_refused():
    buf = io.BytesIO()
    checkpoint.save(buf, SPEC, _state(torch.float64), 3, 1.0)

    def flip(q, meta):
        q = q.copy()
        q.reshape(-1)[5] += 1e-12
        return q, meta

    def fmt(q, meta):
        meta["format"] = 99
        return q, meta

    def mesh(q, meta):
        meta["spec"]["nz"] = 5
        return q, meta

    for mutate, what in ((flip, "checksum"), (fmt, "format"), (mesh, "fit")):
        with pytest.raises(ValueError, match=what):
            checkpoint.load(_rewrite(buf, mutate))
    with pytest.raises(ValueError):
        checkpoint.save(io.BytesIO(), SPEC, torch.zeros(5, 23, 3, 3, 3), 0, 0.0)
