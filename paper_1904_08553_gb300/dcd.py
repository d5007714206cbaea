"""Python binding of the C ABI in include/dcd.h (argument marshalling only).

Every step of the hot path runs in libdcd.so's CUDA kernels; this module
converts numpy arrays / torch tensors to pointers and status codes to
exceptions.  There is no fallback: if the library is missing or fails to load,
every call raises.

The module-level functions carry the C names (dcd_create, dcd_apply_batch,
dcd_update, ...).  ``Context`` bundles them for one dynamic graph.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libdcd.so"

DCD_OK, DCD_EINVAL, DCD_ENOMEM, DCD_ECUDA, DCD_ESTATE, DCD_EOVERFLOW, DCD_ETIMEOUT, DCD_EIO = (
    0, -1, -2, -3, -4, -5, -6, -7)
MODE_STATIC, MODE_BASE, MODE_DELTA, MODE_GIVEN_R, MODE_LEARNED = 0, 1, 2, 3, 4
ALG_LOUVAIN, ALG_SLM = 0, 1

EXPORTED = [
    "dcd_config_default", "dcd_create", "dcd_destroy", "dcd_apply_batch", "dcd_apply_batch_device",
    "dcd_update", "dcd_get_labels", "dcd_get_rset", "dcd_set_labels", "dcd_set_rset", "dcd_set_mode",
    "dcd_get_graph", "dcd_kernel_launches", "dcd_strerror", "dcd_last_cuda_error",
    "dcd_modularity_noalloc", "dcd_mlp_create", "dcd_mlp_destroy", "dcd_mlp_set_params",
    "dcd_mlp_get_params", "dcd_mlp_forward", "dcd_mlp_grad", "dcd_mlp_train",
    "dcd_set_screen", "dcd_set_collect", "dcd_get_screen_data",
    "dcd_group_create", "dcd_group_destroy", "dcd_group_apply_batch", "dcd_group_update",
    "dcd_set_bins", "dcd_get_bins", "dcd_autotune", "dcd_group_set_bins", "dcd_group_get_bins",
    "dcd_group_autotune", "dcd_save", "dcd_load", "dcd_get_state", "dcd_mlp_save",
    "dcd_mlp_load", "dcd_set_fault", "dcd_get_level0_bins", "dcd_eval_bins", "dcd_reserve",
]
MAX_BINS = 12
(LM_SEG16, LM_SEG32, LM_SEG64, LM_WARP128, LM_WARP256, LM_CTA512, LM_CTA1K, LM_CTA2K, LM_CTA4K,
 LM_HUB) = range(10)
LM_LIMIT = [16, 32, 64, 128, 256, 512, 1024, 2048, 4096, -1]
MLP_FEATURES, MLP_HIDDEN, MLP_PARAMS = 12, 64, 5057
NOALLOC_MAX_N = 1048056


class DcdError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {_lib_or_none_strerror(code)} ({code})"
        if code == DCD_ECUDA and _lib is not None:
            msg += f" [{_lib.dcd_last_cuda_error().decode()}]"
        super().__init__(msg)


class Edge(ctypes.Structure):
    _fields_ = [("u", ctypes.c_int32), ("v", ctypes.c_int32), ("w", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("tau_inv", ctypes.c_int32), ("alg", ctypes.c_int32), ("coarsen_full", ctypes.c_int32),
                ("pass_loop", ctypes.c_int32), ("reserved", ctypes.c_int32 * 9)]


_STAT_I64 = ["t", "n", "nnz", "m2", "r_size", "levels", "iters_total", "iters_level0", "moves_total",
             "edges_scanned", "verts_scanned", "communities", "n_lo", "n_hi"]
_STAT_F32 = ["ms_total", "ms_merge", "ms_screen", "ms_local_move", "ms_apply", "ms_coarsen", "ms_finish"]


class StepStats(ctypes.Structure):
    _fields_ = ([(k, ctypes.c_int64) for k in _STAT_I64] + [("q", ctypes.c_double)] +
                [("ins_records", ctypes.c_int64), ("del_records", ctypes.c_int64),
                 ("launches", ctypes.c_int64), ("r_screen", ctypes.c_int64), ("pool", ctypes.c_int64),
                 ("fallback", ctypes.c_int64), ("q_screen", ctypes.c_double)] +
                [(k, ctypes.c_float) for k in _STAT_F32] + [("ms_bin", ctypes.c_float * 4),
                                                            ("reserved_f", ctypes.c_float * 5),
                                                            ("edges_bin", ctypes.c_int64 * 4),
                                                            ("verts_bin", ctypes.c_int64 * 4),
                                                            ("ms_local_move0", ctypes.c_float),
                                                            ("reserved_g", ctypes.c_float),
                                                            ("edges_level0", ctypes.c_int64),
                                                            ("verts_level0", ctypes.c_int64),
                                                            ("refine_iters", ctypes.c_int64),
                                                            ("refine_moves", ctypes.c_int64),
                                                            ("coarse0_delta", ctypes.c_int64),
                                                            ("coarse0_entries", ctypes.c_int64),
                                                            ("edges_level0_screen", ctypes.c_int64),
                                                            ("verts_level0_screen", ctypes.c_int64)])

    @property
    def N(self) -> int:
        return (self.n_hi << 64) + (self.n_lo & ((1 << 64) - 1))

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("reserved_f", "reserved_g")}
        for k in ("ms_bin", "edges_bin", "verts_bin"):
            d[k] = list(d[k])
        d["N"] = self.N
        return d


_lib = None


def _lib_or_none_strerror(code: int) -> str:
    if _lib is None:
        return "error"
    return _lib.dcd_strerror(code).decode()


def lib():
    """Load libdcd.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(str(LIB_PATH))
        P, I64, I32, INT = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        sig = {
            "dcd_config_default": (None, [P]),
            "dcd_create": (INT, [I64, P, P, P]),
            "dcd_destroy": (INT, [P]),
            "dcd_apply_batch": (INT, [P, P, I64, P, I64]),
            "dcd_apply_batch_device": (INT, [P, P, I64, P, I64]),
            "dcd_update": (INT, [P, P, P, P]),
            "dcd_get_labels": (INT, [P, P]),
            "dcd_get_rset": (INT, [P, P]),
            "dcd_set_labels": (INT, [P, P]),
            "dcd_set_rset": (INT, [P, P]),
            "dcd_set_mode": (INT, [P, I32]),
            "dcd_get_graph": (INT, [P, P, P, P, P]),
            "dcd_kernel_launches": (I64, []),
            "dcd_modularity_noalloc": (INT, [I64, P, P, P, P, P, P, P]),
            "dcd_mlp_create": (INT, [ctypes.c_uint64, P, P]),
            "dcd_mlp_destroy": (INT, [P]),
            "dcd_mlp_set_params": (INT, [P, P]),
            "dcd_mlp_get_params": (INT, [P, P]),
            "dcd_mlp_forward": (INT, [P, P, I64, P]),
            "dcd_mlp_grad": (INT, [P, P, P, I64, P, P]),
            "dcd_mlp_train": (INT, [P, P, P, I64, I64, I32, ctypes.c_float, P]),
            "dcd_set_screen": (INT, [P, P, ctypes.c_float, ctypes.c_float, I32]),
            "dcd_set_collect": (INT, [P, I32]),
            "dcd_get_screen_data": (INT, [P, P, P, P, I64, P]),
            "dcd_group_create": (INT, [I32, P, P, P, P]),
            "dcd_group_destroy": (INT, [P]),
            "dcd_group_apply_batch": (INT, [P, I32, P, I64, P, I64]),
            "dcd_group_update": (INT, [P, P, P, P]),
            "dcd_set_bins": (INT, [P, I32, P, P]),
            "dcd_get_bins": (INT, [P, P, P, P]),
            "dcd_autotune": (INT, [P, I32, P]),
            "dcd_get_level0_bins": (INT, [P, P, P, P, P]),
            "dcd_eval_bins": (INT, [P, I32, P, P, P, P, P]),
            "dcd_reserve": (INT, [P, I64, I64]),
            "dcd_group_set_bins": (INT, [P, I32, P, P]),
            "dcd_group_get_bins": (INT, [P, P, P, P]),
            "dcd_group_autotune": (INT, [P, I32, P]),
            "dcd_save": (INT, [P, ctypes.c_char_p]),
            "dcd_load": (INT, [ctypes.c_char_p, P, P]),
            "dcd_get_state": (INT, [P, P, P, P]),
            "dcd_set_fault": (INT, [ctypes.c_char_p]),
            "dcd_mlp_save": (INT, [P, ctypes.c_char_p]),
            "dcd_mlp_load": (INT, [ctypes.c_char_p, P, P]),
            "dcd_strerror": (ctypes.c_char_p, [INT]),
            "dcd_last_cuda_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != DCD_OK:
        raise DcdError(rc, what)


def _ptr(x):
    """Address of a numpy array, a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _edges(a, name: str) -> np.ndarray:
    if a is None:
        return np.zeros((0, 3), np.int32)
    a = np.asarray(a)
    if a.ndim != 2 or a.shape[1] not in (2, 3):
        raise ValueError(f"{name} must be (k, 3) [u, v, w] or (k, 2) [u, v]")
    if a.shape[1] == 2:
        a = np.concatenate([a, np.ones((len(a), 1), a.dtype)], axis=1)
    return np.ascontiguousarray(a, dtype=np.int32)


# ---- C names -----------------------------------------------------------------

def dcd_config_default() -> Config:
    cfg = Config()
    lib().dcd_config_default(ctypes.byref(cfg))
    return cfg


def dcd_create(n: int, cfg: Config | None = None, stream=None):
    h = ctypes.c_void_p()
    _check(lib().dcd_create(int(n), ctypes.byref(cfg) if cfg is not None else None, _stream_ptr(stream),
                            ctypes.byref(h)), "dcd_create")
    return h


def dcd_destroy(h) -> None:
    _check(lib().dcd_destroy(h), "dcd_destroy")


def dcd_apply_batch(h, ins=None, dels=None) -> None:
    i3, d3 = _edges(ins, "ins"), _edges(dels, "dels")
    _check(lib().dcd_apply_batch(h, _ptr(i3), len(i3), _ptr(d3), len(d3)), "dcd_apply_batch")


def dcd_apply_batch_device(h, d_ins, n_ins: int, d_del, n_del: int) -> None:
    _check(lib().dcd_apply_batch_device(h, _ptr(d_ins), int(n_ins), _ptr(d_del), int(n_del)),
           "dcd_apply_batch_device")


def dcd_update(h, labels_out=None):
    q = ctypes.c_double()
    st = StepStats()
    _check(lib().dcd_update(h, _ptr(labels_out), ctypes.byref(q), ctypes.byref(st)), "dcd_update")
    return q.value, st


def dcd_get_labels(h, out) -> None:
    _check(lib().dcd_get_labels(h, _ptr(out)), "dcd_get_labels")


def dcd_get_rset(h, out) -> None:
    _check(lib().dcd_get_rset(h, _ptr(out)), "dcd_get_rset")


def dcd_set_labels(h, labels) -> None:
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    _check(lib().dcd_set_labels(h, _ptr(lab)), "dcd_set_labels")


def dcd_set_rset(h, r) -> None:
    rr = np.ascontiguousarray(r, dtype=np.uint8)
    _check(lib().dcd_set_rset(h, _ptr(rr)), "dcd_set_rset")


def dcd_set_mode(h, mode: int) -> None:
    _check(lib().dcd_set_mode(h, int(mode)), "dcd_set_mode")


def dcd_get_graph(h, n: int):
    nnz = ctypes.c_int64()
    _check(lib().dcd_get_graph(h, ctypes.byref(nnz), None, None, None), "dcd_get_graph")
    rp = np.zeros(n + 1, np.int64)
    col = np.zeros(nnz.value, np.int32)
    w = np.zeros(nnz.value, np.int32)
    _check(lib().dcd_get_graph(h, ctypes.byref(nnz), _ptr(rp), _ptr(col), _ptr(w)), "dcd_get_graph")
    return rp, col, w


def dcd_modularity_noalloc(n: int, d_row_ptr, d_col, d_w, d_labels, stream=None):
    """Q and 2m of a partition on a device CSR, without device allocation."""
    q = ctypes.c_double()
    m2 = ctypes.c_int64()
    _check(lib().dcd_modularity_noalloc(int(n), _ptr(d_row_ptr), _ptr(d_col), _ptr(d_w), _ptr(d_labels),
                                        _stream_ptr(stream), ctypes.byref(q), ctypes.byref(m2)),
           "dcd_modularity_noalloc")
    return q.value, m2.value


def dcd_kernel_launches() -> int:
    return int(lib().dcd_kernel_launches())


def dcd_set_screen(h, mlp_handle, theta_keep: float = 0.5, theta_add: float = 0.5, judge: bool = True) -> None:
    _check(lib().dcd_set_screen(h, mlp_handle, float(theta_keep), float(theta_add), int(bool(judge))),
           "dcd_set_screen")


def dcd_set_collect(h, on: bool = True) -> None:
    _check(lib().dcd_set_collect(h, int(bool(on))), "dcd_set_collect")


def dcd_get_screen_data(h, X_out=None, y_out=None, vertex_out=None, cap: int = 0) -> int:
    n = ctypes.c_int64()
    _check(lib().dcd_get_screen_data(h, _ptr(X_out), _ptr(y_out), _ptr(vertex_out), int(cap), ctypes.byref(n)),
           "dcd_get_screen_data")
    return n.value


def dcd_set_fault(spec: str | None) -> None:
    """Arm host-side fault injection ("alloc:N", "cuda:N", both comma-separated; None or "" disarms)."""
    _check(lib().dcd_set_fault(None if spec is None else spec.encode()), "dcd_set_fault")


def dcd_strerror(code: int) -> str:
    return lib().dcd_strerror(int(code)).decode()


def dcd_last_cuda_error() -> str:
    return lib().dcd_last_cuda_error().decode()


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream", None)


def _set_bins(fn, h, variants, his):
    v = np.ascontiguousarray(variants, dtype=np.int32)
    hi = np.ascontiguousarray(his, dtype=np.int64)
    if v.shape != hi.shape or v.ndim != 1:
        raise ValueError("variants and his must be 1-D of the same length")
    _check(fn(h, len(v), v.ctypes.data, hi.ctypes.data), "set_bins")


def _get_bins(fn, h):
    nb = ctypes.c_int32(0)
    v = np.zeros(MAX_BINS, np.int32)
    hi = np.zeros(MAX_BINS, np.int64)
    _check(fn(h, ctypes.byref(nb), v.ctypes.data, hi.ctypes.data), "get_bins")
    return v[:nb.value].tolist(), hi[:nb.value].tolist()


def _autotune(fn, h, reps):
    ms = ctypes.c_float(0.0)
    _check(fn(h, int(reps), ctypes.byref(ms)), "autotune")
    return ms.value


def dcd_set_bins(h, variants, his) -> None:
    _set_bins(lib().dcd_set_bins, h, variants, his)


def dcd_get_bins(h):
    return _get_bins(lib().dcd_get_bins, h)


def dcd_autotune(h, reps: int = 3) -> float:
    return _autotune(lib().dcd_autotune, h, reps)


def dcd_get_level0_bins(h):
    """Level 0 of the last update's local move: (count per bin, vertices one
    sweep of each bin's grid covers, whether the bins ran side by side)."""
    nb = ctypes.c_int32(0)
    cnt = np.zeros(MAX_BINS, np.int64)
    sw = np.zeros(MAX_BINS, np.int64)
    side = ctypes.c_int32(0)
    _check(lib().dcd_get_level0_bins(h, ctypes.byref(nb), cnt.ctypes.data, sw.ctypes.data, ctypes.byref(side)),
           "dcd_get_level0_bins")
    return cnt[:nb.value].tolist(), sw[:nb.value].tolist(), bool(side.value)


def dcd_reserve(h, nnz: int, records: int) -> None:
    _check(lib().dcd_reserve(h, int(nnz), int(records)), "dcd_reserve")


def dcd_eval_bins(h, reps: int = 3):
    """One local-move evaluation of every vertex of G_t under C_t, each bin's
    kernels timed alone: a list of (variant, vertices, entries, ms) per bin."""
    nb = ctypes.c_int32(0)
    var = np.zeros(MAX_BINS, np.int32)
    verts = np.zeros(MAX_BINS, np.int64)
    ent = np.zeros(MAX_BINS, np.int64)
    ms = np.zeros(MAX_BINS, np.float32)
    _check(lib().dcd_eval_bins(h, int(reps), ctypes.byref(nb), var.ctypes.data, verts.ctypes.data,
                               ent.ctypes.data, ms.ctypes.data), "dcd_eval_bins")
    return [(int(var[b]), int(verts[b]), int(ent[b]), float(ms[b])) for b in range(nb.value)]


def dcd_group_set_bins(h, variants, his) -> None:
    _set_bins(lib().dcd_group_set_bins, h, variants, his)


def dcd_group_get_bins(h):
    return _get_bins(lib().dcd_group_get_bins, h)


def dcd_group_autotune(h, reps: int = 3) -> float:
    return _autotune(lib().dcd_group_autotune, h, reps)


class _Bins:
    """Degree bins of the local-move kernels (dcd_set_bins / dcd_get_bins /
    dcd_autotune, or their group forms)."""

    _prefix = "dcd_"

    def set_bins(self, variants, his):
        _set_bins(getattr(lib(), self._prefix + "set_bins"), self._h, variants, his)

    def bins(self):
        return _get_bins(getattr(lib(), self._prefix + "get_bins"), self._h)

    def autotune(self, reps: int = 3) -> float:
        """Time each candidate bin plan on the current graph and keep the fastest;
        returns its time (ms) per local-move evaluation."""
        return _autotune(getattr(lib(), self._prefix + "autotune"), self._h, reps)


def _path(path) -> bytes:
    return os.fsencode(os.fspath(path))


def dcd_save(h, path) -> None:
    _check(lib().dcd_save(h, _path(path)), "dcd_save")


def dcd_load(path, stream=None):
    h = ctypes.c_void_p()
    _check(lib().dcd_load(_path(path), _stream_ptr(stream), ctypes.byref(h)), "dcd_load")
    return h


def dcd_get_state(h):
    """(n, t, mode) of a context."""
    n, t, mode = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib().dcd_get_state(h, ctypes.byref(n), ctypes.byref(t), ctypes.byref(mode)), "dcd_get_state")
    return n.value, t.value, mode.value


class Context(_Bins):
    """One dynamic graph on vertices [0, n) (dcd_ctx)."""

    def __init__(self, n: int, mode: int = MODE_DELTA, stream=None, max_iters: int = 500,
                 max_levels: int = 64, tau_inv: int = 1_000_000, alg: int = ALG_LOUVAIN,
                 coarsen_full: bool = False, pass_loop_host: bool = False):
        cfg = dcd_config_default()
        cfg.mode, cfg.max_iters, cfg.max_levels, cfg.tau_inv = mode, max_iters, max_levels, tau_inv
        cfg.alg = alg
        cfg.coarsen_full = 1 if coarsen_full else 0
        cfg.pass_loop = 1 if pass_loop_host else 0
        self.n = int(n)
        self._h = dcd_create(self.n, cfg, stream)

    @classmethod
    def load(cls, path, stream=None) -> "Context":
        """A context resumed from a dcd_save checkpoint."""
        h = dcd_load(path, stream)
        self = cls.__new__(cls)
        self._h = h
        self.n = dcd_get_state(h)[0]
        return self

    @property
    def t(self) -> int:
        """Time steps computed so far (the next update is step t + 1)."""
        return dcd_get_state(self._h)[1]

    def save(self, path) -> None:
        dcd_save(self._h, path)

    def level0_bins(self):
        """(count per bin, vertices per grid sweep, side by side) of the last
        update's level-0 local move."""
        return dcd_get_level0_bins(self._h)

    def reserve(self, nnz: int, records: int) -> None:
        """Reserve device memory for graphs of up to nnz directed entries and
        batches of up to `records` records (dcd_reserve)."""
        dcd_reserve(self._h, nnz, records)

    def eval_bins(self, reps: int = 3):
        """Each degree bin's local-move kernels timed alone on G_t under C_t:
        [(variant, vertices, entries, ms), ...] (dcd_eval_bins)."""
        return dcd_eval_bins(self._h, reps)

    def close(self):
        if getattr(self, "_h", None):
            dcd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def apply_batch(self, ins=None, dels=None):
        dcd_apply_batch(self._h, ins, dels)

    def apply_batch_device(self, d_ins, n_ins, d_del, n_del):
        dcd_apply_batch_device(self._h, d_ins, n_ins, d_del, n_del)

    def update(self, labels_out="host"):
        """Advance one step.  labels_out: "host" (numpy result), None, or a
        preallocated numpy array / CUDA tensor of n int32."""
        out = np.empty(self.n, np.int32) if isinstance(labels_out, str) else labels_out
        q, st = dcd_update(self._h, out)
        return out, q, st

    def labels(self) -> np.ndarray:
        out = np.empty(self.n, np.int32)
        dcd_get_labels(self._h, out)
        return out

    def rset(self) -> np.ndarray:
        out = np.empty(self.n, np.uint8)
        dcd_get_rset(self._h, out)
        return out

    def set_labels(self, labels):
        dcd_set_labels(self._h, labels)

    def set_rset(self, r):
        dcd_set_rset(self._h, r)

    def set_mode(self, mode: int):
        dcd_set_mode(self._h, mode)

    def graph(self):
        return dcd_get_graph(self._h, self.n)

    def set_screen(self, mlp, theta_keep=0.5, theta_add=0.5, judge=True):
        dcd_set_screen(self._h, None if mlp is None else mlp.handle, theta_keep, theta_add, judge)

    def set_collect(self, on=True):
        dcd_set_collect(self._h, on)

    def screen_data(self, with_labels=True):
        """(X, y or None, vertices) of the last update's pool, as numpy arrays."""
        n = dcd_get_screen_data(self._h)
        X = np.zeros((n, MLP_FEATURES), np.float32)
        y = np.zeros(n, np.float32) if with_labels else None
        v = np.zeros(n, np.int32)
        dcd_get_screen_data(self._h, X, y, v, n)
        return X, y, v


# ---- learned screen network -------------------------------------------------

def dcd_mlp_create(seed: int = 0, stream=None):
    h = ctypes.c_void_p()
    _check(lib().dcd_mlp_create(int(seed) & ((1 << 64) - 1), _stream_ptr(stream), ctypes.byref(h)),
           "dcd_mlp_create")
    return h


def dcd_mlp_destroy(h) -> None:
    _check(lib().dcd_mlp_destroy(h), "dcd_mlp_destroy")


def dcd_mlp_set_params(h, params) -> None:
    P = np.ascontiguousarray(params, dtype=np.float32)
    if P.size != MLP_PARAMS:
        raise ValueError(f"expected {MLP_PARAMS} parameters")
    _check(lib().dcd_mlp_set_params(h, _ptr(P)), "dcd_mlp_set_params")


def dcd_mlp_get_params(h) -> np.ndarray:
    P = np.zeros(MLP_PARAMS, np.float32)
    _check(lib().dcd_mlp_get_params(h, _ptr(P)), "dcd_mlp_get_params")
    return P


def dcd_mlp_forward(h, d_X, n: int, d_p) -> None:
    _check(lib().dcd_mlp_forward(h, _ptr(d_X), int(n), _ptr(d_p)), "dcd_mlp_forward")


def dcd_mlp_grad(h, d_X, d_y, n: int):
    G = np.zeros(MLP_PARAMS, np.float32)
    loss = ctypes.c_double()
    _check(lib().dcd_mlp_grad(h, _ptr(d_X), _ptr(d_y), int(n), _ptr(G), ctypes.byref(loss)), "dcd_mlp_grad")
    return G, loss.value


def dcd_mlp_train(h, d_X, d_y, n: int, batch: int, epochs: int, lr: float) -> float:
    loss = ctypes.c_double()
    _check(lib().dcd_mlp_train(h, _ptr(d_X), _ptr(d_y), int(n), int(batch), int(epochs), float(lr),
                               ctypes.byref(loss)), "dcd_mlp_train")
    return loss.value


class Mlp:
    """The learned screen's network (dcd_mlp)."""

    def __init__(self, seed: int = 0, stream=None):
        self._h = dcd_mlp_create(seed, stream)

    def close(self):
        if getattr(self, "_h", None):
            dcd_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    params = property(lambda self: dcd_mlp_get_params(self._h),
                      lambda self, p: dcd_mlp_set_params(self._h, p))

    def forward(self, d_X, n, d_p):
        dcd_mlp_forward(self._h, d_X, n, d_p)

    def grad(self, d_X, d_y, n):
        return dcd_mlp_grad(self._h, d_X, d_y, n)

    def train(self, d_X, d_y, n, batch=4096, epochs=1, lr=1e-3):
        return dcd_mlp_train(self._h, d_X, d_y, n, batch, epochs, lr)

    def save(self, path) -> None:
        dcd_mlp_save(self._h, path)

    @classmethod
    def load(cls, path, stream=None) -> "Mlp":
        """A network with the parameters of a dcd_mlp_save file."""
        self = cls.__new__(cls)
        self._h = dcd_mlp_load(path, stream)
        return self


def dcd_mlp_save(h, path) -> None:
    _check(lib().dcd_mlp_save(h, _path(path)), "dcd_mlp_save")


def dcd_mlp_load(path, stream=None):
    h = ctypes.c_void_p()
    _check(lib().dcd_mlp_load(_path(path), _stream_ptr(stream), ctypes.byref(h)), "dcd_mlp_load")
    return h


# ---- batched form ---------------------------------------------------------------

def dcd_group_create(sizes, cfg: Config | None = None, stream=None):
    n = np.ascontiguousarray(sizes, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(lib().dcd_group_create(len(n), _ptr(n), ctypes.byref(cfg) if cfg is not None else None,
                                  _stream_ptr(stream), ctypes.byref(h)), "dcd_group_create")
    return h


def dcd_group_destroy(h) -> None:
    _check(lib().dcd_group_destroy(h), "dcd_group_destroy")


def dcd_group_apply_batch(h, g: int, ins=None, dels=None) -> None:
    i3, d3 = _edges(ins, "ins"), _edges(dels, "dels")
    _check(lib().dcd_group_apply_batch(h, int(g), _ptr(i3), len(i3), _ptr(d3), len(d3)), "dcd_group_apply_batch")


def dcd_group_update(h, G: int, labels_out=None):
    q = np.zeros(G, np.float64)
    st = (StepStats * G)()
    _check(lib().dcd_group_update(h, _ptr(labels_out), _ptr(q), ctypes.cast(st, ctypes.c_void_p).value),
           "dcd_group_update")
    return q, list(st)


class Group(_Bins):
    """Many independent dynamic graphs advanced together (dcd_group)."""

    def __init__(self, sizes, mode: int = MODE_DELTA, stream=None):
        cfg = dcd_config_default()
        cfg.mode = mode
        self.sizes = np.asarray(sizes, dtype=np.int64)
        self.G = len(self.sizes)
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)])
        self._prefix = "dcd_group_"
        self._h = dcd_group_create(self.sizes, cfg, stream)

    def close(self):
        if getattr(self, "_h", None):
            dcd_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_batch(self, g, ins=None, dels=None):
        dcd_group_apply_batch(self._h, g, ins, dels)

    def update(self, labels_out="host"):
        out = np.empty(int(self.offsets[-1]), np.int32) if isinstance(labels_out, str) else labels_out
        q, st = dcd_group_update(self._h, self.G, out)
        return out, q, st
