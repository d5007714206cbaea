"""Parity at the benchmark's full size: the LFR-style stream with n = 2,000,000
and 63,000,000 edge events over 12 steps, run through the C ABI in the
configuration bench.py times (Delta-screening, bin plan autotuned after step 1).

The oracle cannot run Louvain at this size in seconds, so every step checks
what it can compute exactly at any size:
  * G_t: the CSR equals the oracle's batch merge, entry for entry;
  * R_t: equals the oracle's Delta-screening of the same batch (Algorithm 2 and
    the deletion rule) on the same G_{t-1}, G_t and C_{t-1};
  * Q: the library's exact N and 2m equal the oracle's Eq. 1 evaluation of the
    returned labels on G_t (so the tracked modularity is the true one);
  * the labels are canonical (every label is its community's smallest id).
"""
import numpy as np
import pytest

from test_gpu_parity import dcd  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

N_FULL = 2_000_000


def test_lfr_2m_full_size(dcd, orc):
    import bench

    s = bench.make_stream(N_FULL, bench.LFR_STEPS)
    n = s.n
    ctx = dcd.Context(n, mode=dcd.MODE_DELTA)
    g_prev = orc.Graph.empty(n)
    lab_prev = np.arange(n, dtype=np.int32)
    ids = np.arange(n, dtype=np.int32)
    for t, (ins, dels) in enumerate(s.steps):
        ctx.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        if t == 0:
            ctx.autotune(reps=2)
        g_t, err = g_prev.apply(ins, dels)
        assert err == 0
        # G_t
        rp, col, w = ctx.graph()
        orp, ocol, ow = g_t.csr()
        assert np.array_equal(rp, orp)
        assert np.array_equal(col, ocol)
        assert np.array_equal(w.astype(np.int64), ow)
        del rp, col, w, orp, ocol, ow
        # R_t
        if t > 0:
            r_ref = orc.screen(g_prev, g_t, lab_prev, ins, dels)
            assert np.array_equal(ctx.rset(), r_ref)
            assert st.r_size == int(r_ref.sum())
        # Q
        rq, rN, rm2 = g_t.modularity(lab)
        assert st.m2 == rm2 and st.N == rN
        assert abs(q - rq) <= 1e-12 * max(1.0, abs(rq))
        # canonical labels
        first = np.full(n, n, dtype=np.int64)
        np.minimum.at(first, lab, ids)
        assert np.array_equal(first[lab], lab.astype(np.int64))
        g_prev, lab_prev = g_t, lab
    ctx.close()
