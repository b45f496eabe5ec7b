"""Checkpoint and resume of a solution.

A checkpoint is one .npz file holding the state Q (the ABI layout, its own
dtype), the step count, the simulated time, the arguments of the mesh it
lives on (Mesh.spec) and a SHA-256 of the state's bytes.  The kernels are
deterministic (fixed reduction orders, no atomics in the arithmetic), so a
run resumed from a checkpoint continues bit for bit as the uninterrupted run
would have (tests/test_gpu_checkpoint.py).  Saving copies the state to the
host; loading checks the format, the shape against the mesh arguments and
the checksum before anything is returned.
"""
import hashlib
import json

import numpy as np

FORMAT = 1
NF = 5


def _state_shape(spec):
    N = int(spec["p"]) + 1
    return (NF, int(spec["nx"]) * int(spec["ny"]) * int(spec["nz"]), N, N, N)


def save(path, spec, Q, step, t, extra=None):
    """Write Q (a torch tensor or numpy array of the mesh's state shape), the
    step count and the time to `path` (a file name or a binary file object).
    `spec`: the mesh arguments (Mesh.spec); `extra`: JSON-serialisable data
    kept with the checkpoint (e.g. the time-step history)."""
    q = Q.detach().cpu().contiguous().numpy() if hasattr(Q, "detach") else np.ascontiguousarray(Q)
    if tuple(q.shape) != _state_shape(spec) and q.size != int(np.prod(_state_shape(spec))):
        raise ValueError(f"state of shape {q.shape} does not fit the mesh {spec}")
    meta = dict(format=FORMAT, spec=dict(spec), step=int(step), t=float(t), dtype=str(q.dtype),
                shape=list(q.shape), sha256=hashlib.sha256(q.tobytes()).hexdigest(),
                extra=extra or {})
    blob = np.frombuffer(json.dumps(meta, sort_keys=True).encode(), dtype=np.uint8)
    if isinstance(path, str):
        with open(path, "wb") as f:  # a handle: np.savez would append ".npz" to a bare name
            np.savez(f, Q=q, meta=blob)
    else:
        np.savez(path, Q=q, meta=blob)


def load(path):
    """Read a checkpoint: returns (spec, Q as a CPU torch tensor, step, t,
    extra).  Raises ValueError for another format, a state that does not
    fit the mesh arguments, or a checksum mismatch."""
    import torch
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        q = np.array(z["Q"])
    if meta.get("format") != FORMAT:
        raise ValueError(f"checkpoint format {meta.get('format')!r}, expected {FORMAT}")
    if str(q.dtype) != meta["dtype"] or list(q.shape) != meta["shape"]:
        raise ValueError("checkpoint state does not match its own description")
    if int(np.prod(q.shape)) != int(np.prod(_state_shape(meta["spec"]))):
        raise ValueError("checkpoint state does not fit its mesh")
    if hashlib.sha256(q.tobytes()).hexdigest() != meta["sha256"]:
        raise ValueError("checkpoint state fails its checksum")
    return meta["spec"], torch.from_numpy(q), meta["step"], meta["t"], meta["extra"]


def restore(path, device=None):
    """load() and recreate the mesh: returns (Mesh, Q on its device, step, t,
    extra)."""
    from . import dg
    spec, Q, step, t, extra = load(path)
    m = dg.Mesh(**spec, device=device)
    return m, Q.to(m.device).reshape(m.shape).contiguous(), step, t, extra
