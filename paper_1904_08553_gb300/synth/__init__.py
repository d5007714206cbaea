"""Seeded synthetic temporal graph streams (input generators only).

The generators hold none of the community-detection arithmetic; both the CUDA
library's tests/benchmark and the CPU oracle's tests draw their inputs here.
Each stream is a list of time steps, each a pair (inserts (k,3) int32 u,v,w;
deletes (k,2) int32 u,v).

Workload recipes (synthetic stand-ins for the paper's inputs, Sec. IV-A,
Table I; seed = 1904085530 + 1000 * workload + replica):

* ``sbm_10k``    -- 10,000 vertices, 100 planted blocks of 100; step 1 holds
  80,000 intra- and 20,000 inter-block distinct edges; 5 more steps each
  delete 1,000 existing edges and insert 5,000 new pairs (80 % intra).
* ``lfr_2m``     -- 2,000,000 vertices, degree exponent 2.5 on [20, 20000],
  community-size exponent 1.5 on [100, 50000], mixing 0.3, 63M edge events
  over 12 steps, 5 % drift and 2 % deletions per step.
* ``rmat``       -- R-MAT (0.57, 0.19, 0.19, 0.05), edge factor 16, weights
  1..8, 12 steps of 1 % inserts and 0.5 % deletes.
* ``batched_sbm`` -- independent SBMs with n log-uniform in [500, 200000],
  block sizes uniform in 20..2000, mean degree uniform in [8, 32], 80 % intra,
  6 steps of 3 % inserts and 1 % deletes after the initial load.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "synth.c"
_LIB = _HERE / "libdcdsynth.so"

SEED_BASE = 1904085530


def seed_for(workload: int, replica: int = 0) -> int:
    return SEED_BASE + 1000 * workload + replica


def build(force: bool = False) -> Path:
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".so.{os.getpid()}")
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall",
                               str(_SRC), "-o", str(tmp), "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        P, I64, I32, D, U64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                               ctypes.c_uint64)
        sig = {
            "dcdsyn_free": (None, [P]),
            "dcdsyn_n": (I64, [P]),
            "dcdsyn_steps": (I32, [P]),
            "dcdsyn_n_ins": (I64, [P, I32]),
            "dcdsyn_n_del": (I64, [P, I32]),
            "dcdsyn_copy_ins": (None, [P, I32, P]),
            "dcdsyn_copy_del": (None, [P, I32, P]),
            "dcdsyn_copy_planted": (None, [P, P]),
            "dcdsyn_sbm": (P, [U64, I64, I64, P, I64, I64, I32, I64, D, I64, D, D]),
            "dcdsyn_lfr": (P, [U64, I64, D, D, D, D, D, D, D, I64, I32, D, D]),
            "dcdsyn_rmat": (P, [U64, I32, I64, D, D, D, I32, I32, D, D]),
            "dcdsyn_batch_params": (I64, [U64, I32, D, D, I64, I64, D, D, P, P, P, P, I64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


@dataclass
class Stream:
    n: int
    steps: list  # list of (ins (k,3) int32, dels (k,2) int32)
    planted: np.ndarray

    @property
    def total_inserts(self) -> int:
        return sum(len(i) for i, _ in self.steps)


def _collect(h) -> Stream:
    if not h:
        raise ValueError("generator rejected its parameters")
    L = lib()
    try:
        n = int(L.dcdsyn_n(h))
        steps = []
        for t in range(int(L.dcdsyn_steps(h))):
            ni, nd = int(L.dcdsyn_n_ins(h, t)), int(L.dcdsyn_n_del(h, t))
            ins = np.zeros((ni, 3), np.int32)
            dels = np.zeros((nd, 2), np.int32)
            if ni:
                L.dcdsyn_copy_ins(h, t, ins.ctypes.data)
            if nd:
                L.dcdsyn_copy_del(h, t, dels.ctypes.data)
            steps.append((ins, dels))
        planted = np.zeros(n, np.int32)
        L.dcdsyn_copy_planted(h, planted.ctypes.data)
        return Stream(n, steps, planted)
    finally:
        L.dcdsyn_free(h)


def rebin(stream: Stream, k: int) -> Stream:
    """The same insert-only stream at a coarser temporal resolution: its steps
    merged into k consecutive groups (group g holds steps [g T / k, (g+1) T / k)
    rounded down).  Inserts commute, so every binning ends in the same graph;
    a stream with deletes is refused (a delete and an insert of one edge do not
    commute)."""
    T = len(stream.steps)
    if not 1 <= k <= T:
        raise ValueError(f"k must be in [1, {T}]")
    if any(len(d) for _, d in stream.steps):
        raise ValueError("rebinning needs an insert-only stream")
    bounds = [(g * T) // k for g in range(k + 1)]
    empty = np.zeros((0, 2), np.int32)
    steps = [(np.concatenate([stream.steps[t][0] for t in range(bounds[g], bounds[g + 1])]), empty)
             for g in range(k)]
    return Stream(stream.n, steps, stream.planted)


def sbm(seed: int, sizes, m_intra: int, m_inter: int, steps: int, ins_count: int = 0,
        ins_frac: float = 0.0, del_count: int = 0, del_frac: float = 0.0,
        intra_frac: float = 0.8) -> Stream:
    sz = np.ascontiguousarray(sizes, dtype=np.int64)
    n = int(sz.sum())
    return _collect(lib().dcdsyn_sbm(seed, n, len(sz), sz.ctypes.data, m_intra, m_inter, steps,
                                     ins_count, ins_frac, del_count, del_frac, intra_frac))


def sbm_10k(replica: int = 0, n: int = 10_000, blocks: int = 100, steps: int = 6) -> Stream:
    """Planted-partition SBM (mean intra-degree 16, inter-degree 4) + 5 update steps."""
    scale = n / 10_000
    return sbm(seed_for(0, replica), [n // blocks] * blocks, int(80_000 * scale),
               int(20_000 * scale), steps, ins_count=max(1, int(5_000 * scale)),
               del_count=max(1, int(1_000 * scale)), intra_frac=0.8)


def lfr(seed: int, n: int, n_events: int, steps: int = 12, g_deg: float = 2.5,
        kmin: float = 20.0, kmax: float = 20_000.0, g_com: float = 1.5, smin: float = 100.0,
        smax: float = 50_000.0, mu: float = 0.3, drift: float = 0.05,
        del_frac: float = 0.02) -> Stream:
    return _collect(lib().dcdsyn_lfr(seed, n, g_deg, kmin, kmax, g_com, smin, smax, mu,
                                     n_events, steps, drift, del_frac))


def lfr_2m(replica: int = 0, n: int = 2_000_000, events_per_vertex: float = 31.5,
           steps: int = 12, kmax: float = 20_000.0, smax: float = 50_000.0) -> Stream:
    """LFR-style stream shaped like sx-stackoverflow (2M vertices, 63M events)."""
    return lfr(seed_for(1, replica), n, int(round(events_per_vertex * n)), steps,
               kmax=min(kmax, n / 2), smax=min(smax, n / 4))


def rmat(seed: int, scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, wmax: int = 8, steps: int = 13, ins_frac: float = 0.01,
         del_frac: float = 0.005) -> Stream:
    return _collect(lib().dcdsyn_rmat(seed, scale, edge_factor, a, b, c, wmax, steps, ins_frac,
                                      del_frac))


def batched_params(seed: int, G: int = 512, nmin: float = 500, nmax: float = 200_000,
                   smin: int = 20, smax: int = 2000, dmin: float = 8, dmax: float = 32):
    n = np.zeros(G, np.int64)
    deg = np.zeros(G, np.float64)
    nb = np.zeros(G, np.int64)
    cap = int(G * (nmax / smin + 2))
    sizes = np.zeros(cap, np.int64)
    used = lib().dcdsyn_batch_params(seed, G, nmin, nmax, smin, smax, dmin, dmax, n.ctypes.data,
                                     deg.ctypes.data, nb.ctypes.data, sizes.ctypes.data, cap)
    if used < 0:
        raise RuntimeError("batch parameter buffer too small")
    out, off = [], 0
    for g in range(G):
        out.append((int(n[g]), float(deg[g]), sizes[off:off + nb[g]].copy()))
        off += int(nb[g])
    return out


def batched_sbm(replica: int = 0, G: int = 512, steps: int = 7, nmax: float = 200_000,
                intra_frac: float = 0.8, graphs=None) -> list:
    """Independent temporal SBMs of uneven sizes (initial load + steps-1 updates).
    ``graphs`` (indices into the G graphs) generates a subset; graph g is the
    same whichever subset it is generated in."""
    params = batched_params(seed_for(3, replica), G, nmax=nmax)
    streams = []
    for g, (n, deg, sizes) in enumerate(params):
        if graphs is not None and g not in graphs:
            continue
        m = int(round(n * deg / 2))
        m_intra = int(round(intra_frac * m))
        streams.append(sbm(seed_for(3, replica) * 7919 + g, sizes, m_intra, m - m_intra, steps,
                           ins_frac=0.03, del_frac=0.01, intra_frac=intra_frac))
    return streams
