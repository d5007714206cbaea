"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/dcd.h; the binding wraps each of them (no compute calls)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    text = (ROOT / "include" / "dcd.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dcd_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libdcd():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1904_08553_gb300 import dcd

    return dcd


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dcd_create", "dcd_apply_batch", "dcd_apply_batch_device", "dcd_update", "dcd_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libdcd):
    L = ctypes.CDLL(str(libdcd.LIB_PATH))
    for name in declared_functions():
        assert hasattr(L, name), name
    assert sorted(libdcd.EXPORTED) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(libdcd, name)), name


def test_status_text_and_defaults(libdcd):
    L = libdcd.lib()
    assert L.dcd_strerror(0) == b"ok"
    assert b"invalid" in L.dcd_strerror(-1)
    cfg = libdcd.dcd_config_default()
    assert (cfg.mode, cfg.max_iters, cfg.max_levels, cfg.tau_inv) == (2, 500, 64, 1_000_000)


def test_struct_layouts_match_header(libdcd):
    assert ctypes.sizeof(libdcd.Edge) == 12
    assert ctypes.sizeof(libdcd.Config) == 64
    # 14 int64 + double + 6 int64 + double + 16 float + 8 int64 + 2 float + 8 int64
    assert ctypes.sizeof(libdcd.StepStats) == 14 * 8 + 8 + 6 * 8 + 8 + 16 * 4 + 8 * 8 + 2 * 4 + 4 * 8 + 4 * 8


def test_create_rejects_bad_n_before_touching_the_device(libdcd):
    h = ctypes.c_void_p()
    L = libdcd.lib()
    assert L.dcd_create(0, None, None, ctypes.byref(h)) == libdcd.DCD_EINVAL
    assert L.dcd_create(-5, None, None, ctypes.byref(h)) == libdcd.DCD_EINVAL
    assert L.dcd_create(1 << 31, None, None, ctypes.byref(h)) == libdcd.DCD_EINVAL
    assert L.dcd_destroy(None) == 0


def test_create_rejects_bad_configurations_before_touching_the_device(libdcd):
    h = ctypes.c_void_p()
    L = libdcd.lib()
    cfg = libdcd.dcd_config_default()
    cfg.alg = 7  # unknown host method
    assert L.dcd_create(10, ctypes.byref(cfg), None, ctypes.byref(h)) == libdcd.DCD_EINVAL
    cfg.alg = libdcd.ALG_SLM  # smart local moving names n + v: n must stay below 2^30
    assert L.dcd_create(1 << 30, ctypes.byref(cfg), None, ctypes.byref(h)) == libdcd.DCD_EINVAL
    sizes = (ctypes.c_int64 * 2)(10, 20)
    g = ctypes.c_void_p()
    assert L.dcd_group_create(2, sizes, ctypes.byref(cfg), None, ctypes.byref(g)) == libdcd.DCD_EINVAL
    cfg = libdcd.dcd_config_default()
    for field in ("coarsen_full", "pass_loop"):  # switches take 0 or 1
        setattr(cfg, field, 2)
        assert L.dcd_create(10, ctypes.byref(cfg), None, ctypes.byref(h)) == libdcd.DCD_EINVAL
        setattr(cfg, field, 0)


def test_measurement_aids_reject_bad_arguments_before_touching_the_device(libdcd):
    """dcd_reserve and dcd_eval_bins check their arguments on the host: a NULL
    context or NULL outputs are refused with DCD_EINVAL, no CUDA call made."""
    L = libdcd.lib()
    assert L.dcd_reserve(None, 10, 10) == libdcd.DCD_EINVAL
    nb = ctypes.c_int32(0)
    buf = (ctypes.c_int64 * 12)()
    var = (ctypes.c_int32 * 12)()
    ms = (ctypes.c_float * 12)()
    assert L.dcd_eval_bins(None, 1, ctypes.byref(nb), var, buf, buf, ms) == libdcd.DCD_EINVAL
