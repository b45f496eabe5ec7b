"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/dg.h declares, and rejects bad arguments on the
host before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dg.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2006_15698_gb300.build import build
    return ctypes.CDLL(build())


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "dg_rk_step" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in dg.h but not exported"


def test_status_strings(lib):
    lib.dg_status_string.restype = ctypes.c_char_p
    for s in range(8):
        assert lib.dg_status_string(s)
    assert lib.dg_status_string(99) == b"unknown status"


def _create(lib, *a):
    h = ctypes.c_void_p()
    f = lib.dg_mesh_create
    f.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 7 + [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    f.restype = ctypes.c_int
    st = f(*a, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("args,status", [
    ((0, 1, 1, 2, 0, 0, 0, 1, 1, 1, 1.4, 0), 1),      # nx = 0
    ((1, 1, 1, 2, 0, 0, 0, -1, 1, 1, 1.4, 0), 1),     # Lx < 0
    ((1, 1, 1, 2, 0, 0, 0, 1, 1, 1, 1.0, 0), 1),      # gamma <= 1
    ((1, 1, 1, 2, 0, 0, 0, 1, 1, 1, 1.4, 7), 1),      # bad precision
    ((1, 1, 1, 7, 0, 0, 0, 1, 1, 1, 1.4, 0), 2),      # p > 6
    ((1, 1, 1, -1, 0, 0, 0, 1, 1, 1, 1.4, 0), 2),     # p < 0
    ((1 << 14, 1 << 14, 1 << 14, 6, 0, 0, 0, 1, 1, 1, 1.4, 0), 1),  # too many nodes
    ((1, 1, 1, 2, float("nan"), 0, 0, 1, 1, 1, 1.4, 0), 1),
])
def test_mesh_create_rejects_bad_arguments_on_host(lib, args, status):
    st, h = _create(lib, *args)
    assert st == status and not h.value


def test_null_handles_rejected(lib):
    for name, nargs in [("dg_rhs", 4), ("dg_rk_step", 5), ("dg_norms", 5), ("dg_cfl_dt", 5)]:
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        if name == "dg_cfl_dt":
            f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
            assert f(None, None, 0.5, None, None) == 1
        else:
            f.argtypes = [ctypes.c_void_p] * nargs
            assert f(*([None] * nargs)) == 1
    lib.dg_mesh_destroy.argtypes = [ctypes.c_void_p]
    lib.dg_mesh_destroy(None)  # NULL is ignored


def test_tuning_tables_validate_on_host(lib):
    """The process-wide tile-variant and stage-kernel tables: defaults,
    round trips, and host-side rejection of bad degrees and kinds."""
    lib.dg_set_stage_kernel.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.dg_get_stage_kernel.argtypes = [ctypes.c_int]
    lib.dg_set_tile_variant.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.dg_get_tile_variant.argtypes = [ctypes.c_int]
    lib.dg_tile_variant_count.argtypes = [ctypes.c_int]
    for p in range(7):
        assert lib.dg_get_stage_kernel(p) in (0, 1, 2)
        assert lib.dg_tile_variant_count(p) >= 1
    assert lib.dg_get_stage_kernel(-1) == -1 and lib.dg_get_stage_kernel(7) == -1
    assert lib.dg_set_stage_kernel(7, 0) == 2          # DG_ERR_UNSUPPORTED
    assert lib.dg_set_stage_kernel(3, 5) == 1          # DG_ERR_ARG
    saved = lib.dg_get_stage_kernel(3)
    assert lib.dg_set_stage_kernel(3, 0) == 0 and lib.dg_get_stage_kernel(3) == 0
    assert lib.dg_set_stage_kernel(3, 1) == 0 and lib.dg_get_stage_kernel(3) == 1
    assert lib.dg_set_stage_kernel(3, 2) == 0 and lib.dg_get_stage_kernel(3) == 2
    assert lib.dg_set_stage_kernel(3, 3) == 1
    lib.dg_set_stage_kernel(3, saved)
    assert lib.dg_set_tile_variant(3, lib.dg_tile_variant_count(3)) == 1
    lib.dg_set_batch_direct_nodes.argtypes = [ctypes.c_int64]
    lib.dg_get_batch_direct_nodes.restype = ctypes.c_int64
    saved = lib.dg_get_batch_direct_nodes()
    assert saved >= 0
    assert lib.dg_set_batch_direct_nodes(-1) == 1        # DG_ERR_ARG
    assert lib.dg_set_batch_direct_nodes(12345) == 0 and lib.dg_get_batch_direct_nodes() == 12345
    assert lib.dg_set_batch_direct_nodes(saved) == 0


def test_committed_tuning_table_applies():
    """The autotuner table shipped with the package names only known stage
    kernels and tile variants in range, and dg.load_tuning applies exactly
    those choices to the process-wide tables (host-only calls)."""
    from paper_2006_15698_gb300 import dg
    saved = {p: (dg.dg_get_tile_variant(p), dg.dg_get_stage_kernel(p)) for p in range(7)}
    try:
        table = dg.load_tuning()
        assert table is not None and table["degrees"]
        for p, ent in table["degrees"].items():
            p = int(p)
            assert ent["kernel"] in dg.STAGE_KINDS, ent
            assert 0 <= int(ent["variant"]) < dg.dg_tile_variant_count(p), ent
            assert dg.dg_get_stage_kernel(p) == dg.STAGE_KINDS[ent["kernel"]]
            assert dg.dg_get_tile_variant(p) == int(ent["variant"])
            assert list(dg.dg_tile_shape(p, int(ent["variant"]))) == list(ent["tile"])
    finally:
        for p, (v, k) in saved.items():
            dg.dg_set_tile_variant(p, v)
            dg.dg_set_stage_kernel(p, k)


def test_new_entry_points_reject_bad_arguments_on_host(lib):
    """The z-slab, batch-update, probe and self-check entry points validate
    their arguments before any CUDA call (no GPU needed)."""
    vp, i = ctypes.c_void_p, ctypes.c_int
    lib.dg_rk_stage.argtypes = [vp, vp, vp, vp, vp, i, vp]
    assert lib.dg_rk_stage(None, None, None, None, None, 0, None) == 1
    lib.dg_mesh_set_zhalo.argtypes = [vp, vp, vp]
    assert lib.dg_mesh_set_zhalo(None, None, None) == 1
    lib.dg_zhalo_traces.argtypes = [vp, vp, vp, vp, vp]
    assert lib.dg_zhalo_traces(None, None, None, None, None) == 1
    lib.dg_batch_update.argtypes = [vp, i, vp]
    assert lib.dg_batch_update(None, 1, None) == 1
    lib.dg_fma_throughput.argtypes = [i, vp, vp]
    assert lib.dg_fma_throughput(0, None, None) == 1
    lib.dg_dmma_throughput.argtypes = [i, vp, vp]
    assert lib.dg_dmma_throughput(2, None, None) == 1
    lib.dg_selfcheck_sqrt.argtypes = [vp, vp, vp, ctypes.c_int64, vp]
    assert lib.dg_selfcheck_sqrt(None, None, None, 4, None) == 1
    lib.dg_advance_host.argtypes = [vp, vp, vp, vp, ctypes.c_double, i, vp, vp, vp]
    assert lib.dg_advance_host(None, None, None, None, 0.5, 1, None, None, None) == 1
