"""CPU oracle for Delta-screening dynamic Louvain (arXiv 1904.08553).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs use it.  The CUDA
library never imports, links or calls anything here, and this package imports
nothing from the CUDA library.

The arithmetic lives in ``dcd_oracle.c`` (plain sequential C, exact integers);
this module only builds it with gcc and marshals numpy arrays through ctypes.

Parity status per function (pins in ``tests/test_oracle_pins.py``):
  modularity (Eq. 1)              pinned: closed forms, brute-force pairwise formula
  gain S (Sec. III-A, App. A)     pinned: exact Q difference, Lemma 3.2 / 3.4(B) identities
  local move / levels (Alg. 1)    pinned: invariants (no improving move, coarse Q = fine Q,
                                  m2 preserved, brute-force optimum bound, mode identities)
  screening inserts (Alg. 2)      pinned: hand-built cases
  deletion rule                   parity unpinned (the paper has no deletion rule)
  smart local moving (dSLM)       pinned: closed forms (split of a disconnected community),
                                  invariants (nesting, no improving move, coarse Q = fine Q)
  batch apply                     pinned: dictionary re-implementation of the edge set
  learned-screen pool, features   parity unpinned (not in the paper); cross-checked against a
                                  second implementation of the feature definitions
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "dcd_oracle.c"
_SRC_MLP = _HERE / "mlp_oracle.c"
_LIB = _HERE / "libdcd_oracle.so"

STATIC, BASE, DELTA, GIVEN_R = 0, 1, 2, 3
LOUVAIN, SLM = 0, 1  # host method of the multi-level run
MAX_ITERS = 500
MAX_LEVELS = 64


SANITIZE_FLAGS = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                  "-fno-sanitize-recover=undefined"]


def build_sanitized(out: Path) -> Path:
    """The same sources with AddressSanitizer and UndefinedBehaviorSanitizer,
    for a process that preloads the sanitizer runtime and points DCD_ORACLE_LIB
    at `out` (the sanitizer test does both)."""
    subprocess.check_call(
        ["gcc", *SANITIZE_FLAGS, "-std=gnu11", "-fPIC", "-shared", "-Wall", "-Wextra",
         "-Wno-unused-parameter", str(_SRC), str(_SRC_MLP), "-o", str(out), "-lm"]
    )
    return Path(out)


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (portable C: no target-specific flags)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < max(
        _SRC.stat().st_mtime, _SRC_MLP.stat().st_mtime, (_HERE / "dcd_oracle.h").stat().st_mtime
    ):
        tmp = _LIB.with_suffix(f".so.{os.getpid()}")
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall", "-Wextra",
             "-Wno-unused-parameter", str(_SRC), str(_SRC_MLP), "-o", str(tmp), "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "t", "n", "nnz", "m2", "r_size", "levels", "iters_total", "iters_level0",
        "moves_total", "edges_scanned", "communities", "n_lo", "n_hi")] + [("q", ctypes.c_double)] + [
        (name, ctypes.c_int64) for name in ("refine_iters", "refine_moves")]

    @property
    def N(self) -> int:
        return (self.n_hi << 64) + (self.n_lo & ((1 << 64) - 1))

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["N"] = self.N
        return d


_lib = None


def lib():
    global _lib
    if _lib is None:
        # DCD_ORACLE_LIB: another build of these sources (the sanitizer build)
        alt = os.environ.get("DCD_ORACLE_LIB")
        if not alt:
            build()
        L = ctypes.CDLL(alt or str(_LIB))
        P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        sig = {
            "orc_graph_new": (P, [I64, P, P, P]),
            "orc_graph_free": (None, [P]),
            "orc_graph_n": (I64, [P]),
            "orc_graph_nnz": (I64, [P]),
            "orc_graph_copy": (None, [P, P, P, P]),
            "orc_apply": (P, [P, P, I64, P, I64, P, P]),
            "orc_modularity": (D, [P, P, P, P, P]),
            "orc_gain": (None, [P, P, I32, I32, P, P]),
            "orc_local_move_pass": (I64, [P, P, P, P]),
            "orc_run_level": (I64, [P, P, P, I64, P, P]),
            "orc_coarsen": (P, [P, P, P]),
            "orc_screen": (ctypes.c_int, [P, P, P, P, I64, P, I64, P]),
            "orc_louvain": (ctypes.c_int, [P, P, P, P, P]),
            "orc_create": (P, [I64]),
            "orc_destroy": (None, [P]),
            "orc_apply_batch": (ctypes.c_int, [P, P, I64, P, I64]),
            "orc_update": (ctypes.c_int, [P, ctypes.c_int, P, P, P, P]),
            "orc_update_alg": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P, P, P]),
            "orc_slm": (ctypes.c_int, [P, P, P, P, P]),
            "orc_slm_refine": (I64, [P, P, P, P]),
            "orc_slm_level": (I64, [P, P, P, P]),
            "orc_get_rset": (ctypes.c_int, [P, P]),
            "orc_ctx_graph": (P, [P]),
            "orc_set_labels": (ctypes.c_int, [P, P]),
            "orc_clone": (P, [P]),
            "orc_mlp_nparams": (ctypes.c_int, []),
            "orc_bf16": (ctypes.c_float, [ctypes.c_float]),
            "orc_mlp_forward": (D, [P, P, P, I64, P]),
            "orc_mlp_grad": (D, [P, P, P, I64, P]),
            "orc_mlp_grad_exact": (D, [P, P, P, I64, P]),
            "orc_mlp_loss_exact": (D, [P, P, P, I64]),
            "orc_screen_features": (ctypes.c_int, [P, P, P, P, I64, P, I64, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _edges3(a, dtype=np.int32) -> np.ndarray:
    if a is None:
        return np.zeros((0, 3), dtype)
    return np.ascontiguousarray(np.asarray(a, dtype=dtype).reshape(-1, 3))


def _edges2(a) -> np.ndarray:
    if a is None:
        return np.zeros((0, 2), np.int32)
    a = np.asarray(a, dtype=np.int32)
    if a.ndim == 2 and a.shape[1] == 3:
        a = a[:, :2]
    return np.ascontiguousarray(a.reshape(-1, 2))


class Graph:
    """An oracle CSR graph (int64 row_ptr, int32 col, int64 w)."""

    def __init__(self, handle):
        if not handle:
            raise MemoryError("oracle graph allocation failed")
        self._h = handle

    @classmethod
    def from_csr(cls, n, row_ptr, col, w) -> "Graph":
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        c = np.ascontiguousarray(col, dtype=np.int32)
        ww = np.ascontiguousarray(w, dtype=np.int64)
        return cls(lib().orc_graph_new(int(n), _p(rp), _p(c), _p(ww)))

    @classmethod
    def empty(cls, n) -> "Graph":
        return cls(lib().orc_graph_new(int(n), None, None, None))

    @classmethod
    def from_edges(cls, n, edges) -> "Graph":
        """Undirected edges (u, v[, w]); duplicates add their weights."""
        e = np.asarray(edges, dtype=np.int64)
        if e.size and e.shape[1] == 2:
            e = np.concatenate([e, np.ones((len(e), 1), np.int64)], axis=1)
        g, err = cls.empty(n).apply(ins=e)
        if g is None:
            raise ValueError(f"bad edge list (error {err})")
        return g

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_graph_free(self._h)
            self._h = None

    @property
    def n(self) -> int:
        return int(lib().orc_graph_n(self._h))

    @property
    def nnz(self) -> int:
        return int(lib().orc_graph_nnz(self._h))

    def csr(self):
        n, nnz = self.n, self.nnz
        rp = np.zeros(n + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        w = np.zeros(nnz, np.int64)
        lib().orc_graph_copy(self._h, _p(rp), _p(col), _p(w))
        return rp, col, w

    def apply(self, ins=None, dels=None, want_present=False):
        ins3 = _edges3(ins)
        del2 = _edges2(dels)
        present = np.zeros(len(del2), np.uint8)
        err = ctypes.c_int(0)
        h = lib().orc_apply(self._h, _p(ins3), len(ins3), _p(del2), len(del2), _p(present),
                            ctypes.byref(err))
        g = Graph(h) if h else None
        if want_present:
            return g, err.value, present
        return g, err.value

    def modularity(self, labels):
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        m2 = ctypes.c_int64()
        lo = ctypes.c_int64()
        hi = ctypes.c_int64()
        q = lib().orc_modularity(self._h, _p(lab), ctypes.byref(m2), ctypes.byref(lo),
                                 ctypes.byref(hi))
        N = (hi.value << 64) + (lo.value & ((1 << 64) - 1))
        return q, N, m2.value

    def gain(self, labels, v, D) -> int:
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        lo = ctypes.c_int64()
        hi = ctypes.c_int64()
        lib().orc_gain(self._h, _p(lab), int(v), int(D), ctypes.byref(lo), ctypes.byref(hi))
        return (hi.value << 64) + (lo.value & ((1 << 64) - 1))

    def local_move_pass(self, labels, active=None):
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        out = np.zeros(self.n, np.int32)
        moves = lib().orc_local_move_pass(self._h, _p(lab), _p(act), _p(out))
        return out, int(moves)

    def run_level(self, labels, active=None, max_iters=MAX_ITERS):
        lab = np.array(labels, dtype=np.int32, copy=True)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        moves = ctypes.c_int64()
        edges = ctypes.c_int64()
        it = lib().orc_run_level(self._h, _p(lab), _p(act), int(max_iters), ctypes.byref(moves),
                                 ctypes.byref(edges))
        return lab, int(it), moves.value, edges.value

    def coarsen(self, labels):
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        cid = np.zeros(self.n, np.int32)
        g = Graph(lib().orc_coarsen(self._h, _p(lab), _p(cid)))
        return g, cid

    def slm(self, init=None, active=None):
        """Multi-level smart local moving (the dSLM-Delta-s host method)."""
        n = self.n
        ini = np.arange(n, dtype=np.int32) if init is None else np.ascontiguousarray(init, np.int32)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        out = np.zeros(n, np.int32)
        st = Stats()
        rc = lib().orc_slm(self._h, _p(ini), _p(act), _p(out), ctypes.byref(st))
        if rc != 0:
            raise RuntimeError(f"orc_slm failed: {rc}")
        return out, st

    def slm_refine(self, parent):
        """Sub-communities of each parent community (canonical), passes, moves."""
        par = np.ascontiguousarray(parent, dtype=np.int32)
        sub = np.zeros(self.n, np.int32)
        moves = ctypes.c_int64()
        it = lib().orc_slm_refine(self._h, _p(par), _p(sub), ctypes.byref(moves))
        return sub, int(it), moves.value

    def slm_level(self, labels, active=None):
        """SLM local moving of one level: (canonical labels, passes, moves)."""
        lab = np.array(labels, dtype=np.int32, copy=True)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        moves = ctypes.c_int64()
        it = lib().orc_slm_level(self._h, _p(lab), _p(act), ctypes.byref(moves))
        return lab, int(it), moves.value

    def louvain(self, init=None, active=None):
        n = self.n
        ini = np.arange(n, dtype=np.int32) if init is None else np.ascontiguousarray(init, np.int32)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        out = np.zeros(n, np.int32)
        st = Stats()
        rc = lib().orc_louvain(self._h, _p(ini), _p(act), _p(out), ctypes.byref(st))
        if rc != 0:
            raise RuntimeError(f"orc_louvain failed: {rc}")
        return out, st


def screen(g_prev: Graph, g_t: Graph, labels0, ins=None, dels=None) -> np.ndarray:
    lab = np.ascontiguousarray(labels0, dtype=np.int32)
    ins3 = _edges3(ins)
    del2 = _edges2(dels)
    r = np.zeros(g_t.n, np.uint8)
    rc = lib().orc_screen(g_prev._h, g_t._h, _p(lab), _p(ins3), len(ins3), _p(del2), len(del2),
                          _p(r))
    if rc != 0:
        raise RuntimeError(f"orc_screen failed: {rc}")
    return r


def screen_features(g_prev: Graph, g_t: Graph, labels0, ins, dels, rds):
    """(pool mask, X n x 12) of the learned screen's features."""
    lab = np.ascontiguousarray(labels0, dtype=np.int32)
    ins3 = _edges3(ins)
    del2 = _edges2(dels)
    r = np.ascontiguousarray(rds, dtype=np.uint8)
    pool = np.zeros(g_t.n, np.uint8)
    X = np.zeros((g_t.n, 12), np.float32)
    rc = lib().orc_screen_features(g_prev._h, g_t._h, _p(lab), _p(ins3), len(ins3), _p(del2), len(del2), _p(r),
                                   _p(pool), _p(X))
    if rc != 0:
        raise RuntimeError(f"orc_screen_features failed: {rc}")
    return pool, X


class Context:
    """Stateful incremental driver (Sec. III-D), the oracle twin of dcd_ctx."""

    def __init__(self, n: int):
        self._h = lib().orc_create(int(n))
        if not self._h:
            raise ValueError(f"bad vertex count {n}")
        self.n = int(n)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    def apply_batch(self, ins=None, dels=None) -> int:
        ins3 = _edges3(ins)
        del2 = _edges2(dels)
        return int(lib().orc_apply_batch(self._h, _p(ins3), len(ins3), _p(del2), len(del2)))

    def update(self, mode: int = DELTA, r_given=None, alg: int = LOUVAIN):
        labels = np.zeros(self.n, np.int32)
        q = ctypes.c_double()
        st = Stats()
        r = None if r_given is None else np.ascontiguousarray(r_given, dtype=np.uint8)
        rc = lib().orc_update_alg(self._h, int(alg), int(mode), _p(r), _p(labels), ctypes.byref(q),
                                  ctypes.byref(st))
        if rc != 0:
            raise RuntimeError(f"orc_update failed: {rc}")
        return labels, q.value, st

    def rset(self) -> np.ndarray:
        r = np.zeros(self.n, np.uint8)
        lib().orc_get_rset(self._h, _p(r))
        return r

    def graph_csr(self):
        h = lib().orc_ctx_graph(self._h)
        n = int(lib().orc_graph_n(h))
        nnz = int(lib().orc_graph_nnz(h))
        rp = np.zeros(n + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        w = np.zeros(nnz, np.int64)
        lib().orc_graph_copy(h, _p(rp), _p(col), _p(w))
        return rp, col, w

    def set_labels(self, labels) -> int:
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        return int(lib().orc_set_labels(self._h, _p(lab)))

    def clone(self) -> "Context":
        """A deep copy (G_t, C_t, R_t, t, staged batch): the next update of
        either copy gives the same result."""
        h = lib().orc_clone(self._h)
        if not h:
            raise MemoryError("oracle context copy failed")
        c = Context.__new__(Context)
        c._h = h
        c.n = self.n
        return c


# ---------------------------------------------------------------- learned screen (MLP)

MLP_FEATURES, MLP_HIDDEN = 12, 64


def mlp_nparams() -> int:
    return int(lib().orc_mlp_nparams())


def bf16(x: float) -> float:
    return float(lib().orc_bf16(float(x)))


def mlp_forward(params, X, y=None):
    """Probabilities (FP64, BF16-rounded operands) and mean BCE."""
    P = np.ascontiguousarray(params, np.float32)
    Xf = np.ascontiguousarray(X, np.float32).reshape(-1, MLP_FEATURES)
    yy = None if y is None else np.ascontiguousarray(y, np.float32)
    p = np.zeros(len(Xf), np.float64)
    loss = lib().orc_mlp_forward(_p(P), _p(Xf), _p(yy), len(Xf), _p(p))
    return p, loss


def mlp_grad(params, X, y):
    P = np.ascontiguousarray(params, np.float32)
    Xf = np.ascontiguousarray(X, np.float32).reshape(-1, MLP_FEATURES)
    yy = np.ascontiguousarray(y, np.float32)
    G = np.zeros(mlp_nparams(), np.float64)
    loss = lib().orc_mlp_grad(_p(P), _p(Xf), _p(yy), len(Xf), _p(G))
    return G, loss


def mlp_grad_exact(params, X, y):
    P = np.ascontiguousarray(params, np.float64)
    Xd = np.ascontiguousarray(X, np.float64).reshape(-1, MLP_FEATURES)
    yy = np.ascontiguousarray(y, np.float64)
    G = np.zeros(mlp_nparams(), np.float64)
    loss = lib().orc_mlp_grad_exact(_p(P), _p(Xd), _p(yy), len(Xd), _p(G))
    return G, loss


def mlp_loss_exact(params, X, y) -> float:
    P = np.ascontiguousarray(params, np.float64)
    Xd = np.ascontiguousarray(X, np.float64).reshape(-1, MLP_FEATURES)
    yy = np.ascontiguousarray(y, np.float64)
    return float(lib().orc_mlp_loss_exact(_p(P), _p(Xd), _p(yy), len(Xd)))
