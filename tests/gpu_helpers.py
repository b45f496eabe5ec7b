"""Shared helpers of the GPU parity tests: device round trips and the
scale the tolerances are measured against."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dg_module():
    require_gpu()
    from paper_2006_15698_gb300 import dg  # raises if the library is not built
    return dg


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def to_host(t):
    torch.cuda.synchronize()
    return t.detach().to("cpu", torch.float64).numpy()


def dev_scalar(x):
    return torch.tensor([float(x)], dtype=torch.float64, device="cuda")


def rhs_scale(om, Q):
    """Size of the individual terms summed into one right-hand-side value:
    (2/h_min) * Lambda * ||Q||, Lambda the largest sum of wave speeds (the
    oracle's CFL maximum).  Rounding in a sum of such terms is relative to
    this, not to the (possibly much smaller, cancelled) result."""
    hmin = min(om.box[3] / om.nx, om.box[4] / om.ny, om.box[5] / om.nz)
    _, lam = om.cfl_dt(Q, 1.0)
    return (2.0 / hmin) * lam * np.linalg.norm(Q)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
