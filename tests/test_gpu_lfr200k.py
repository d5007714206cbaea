"""Label-exact parity where the level-0 local move runs its full-size code
paths: the benchmark's LFR-style generator at n = 200,000 (6.3M edge events
over 12 steps, so about 6M directed entries by step 6), six steps of
Delta-screening (Algorithm 2, then Algorithm 1 over R_t) and one step of
dLouvain-base (R_t = V_t), against the oracle run on the same batches.

Labels, R_t, N, 2m, and the pass, move and level counts must be equal, bit
for bit, at every step.  The test also shows that it reached the paths the
small parity cases do not: at level 0 the active set holds at least 65,536
vertices (the degree bins then run side by side on their own streams), and
the most populated segment-per-vertex bins hold more vertices than one sweep
of their grid covers (the grid-stride loops run more than once per warp).
"""
import numpy as np
import pytest

from test_gpu_parity import assert_step_equal, dcd  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

N = 200_000
DELTA_STEPS = 6


def test_lfr_200k_label_exact(dcd, orc):
    import bench

    s = bench.make_stream(N, bench.LFR_STEPS)
    ctx = dcd.Context(N, mode=dcd.MODE_DELTA)
    ref = orc.Context(N)
    plan_var, _ = ctx.bins()
    multi_sweep = set()
    side_steps = 0
    for t in range(DELTA_STEPS + 1):
        base = t == DELTA_STEPS
        if base:
            ctx.set_mode(dcd.MODE_BASE)
        ins, dels = s.steps[t]
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        rlab, rq, rst = ref.update(orc.BASE if base else orc.DELTA)
        assert_step_equal(st, rst, lab, rlab, q, rq, ctx.rset(), ref.rset())
        cnt, sweep, side = ctx.level0_bins()
        assert sum(cnt) <= st.r_size
        if t > 0:
            assert sum(cnt) >= 65_536, cnt
            assert side
            side_steps += 1
        for b, (c, w) in enumerate(zip(cnt, sweep)):
            if c > w:
                multi_sweep.add(plan_var[b])
    assert side_steps == DELTA_STEPS
    # the segment kernels of the two most populated bins (rows of 17..32 and
    # 33..64 entries, two vertices a warp) each ran more than one sweep of
    # their grid in some step
    assert dcd.LM_SEG32 in multi_sweep, multi_sweep
    assert dcd.LM_SEG64 in multi_sweep, multi_sweep
    ctx.close()
