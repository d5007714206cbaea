"""Degree-bin plans of the local-move kernels: any valid plan gives the
oracle's labels and modularity bit for bit (the plan changes only which kernel
evaluates a vertex), the autotuner keeps one of its candidates, and invalid
plans are refused without changing the context."""
import numpy as np
import pytest

from test_gpu_parity import dcd  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def random_plan(dcd, rng):
    """Increasing bins, each within its variant's limit, ending in the hub variant."""
    limits = dcd.LM_LIMIT
    variants, his = [], []
    lo = 0
    for v in range(dcd.LM_HUB):
        if rng.random() < 0.5 or limits[v] <= lo:
            continue
        hi = int(rng.integers(lo + 1, limits[v] + 1))
        variants.append(v)
        his.append(hi)
        lo = hi
    variants.append(dcd.LM_HUB)
    his.append(-1)
    return variants, his


def lfr_small(synth):
    return synth.lfr(synth.seed_for(1, 7), n=20_000, n_events=400_000, steps=4, kmin=4, kmax=2000,
                     smin=20, smax=2000)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_any_plan_matches_oracle(dcd, orc, synth, seed):
    rng = np.random.default_rng(seed)
    s = lfr_small(synth)
    ctx = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    ref = orc.Context(s.n)
    for t, (ins, dels) in enumerate(s.steps):
        variants, his = random_plan(dcd, rng)
        ctx.set_bins(variants, his)
        assert ctx.bins() == (variants, his)
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        rlab, rq, rst = ref.update(orc.DELTA)
        assert np.array_equal(lab, rlab)
        assert abs(q - rq) <= 1e-12 * max(1.0, abs(rq))
        assert st.iters_total == rst.iters_total and st.moves_total == rst.moves_total
    ctx.close()


def test_hub_only_plan_matches_oracle(dcd, orc, synth):
    s = synth.sbm_10k(n=2000, blocks=20, steps=3)
    ctx = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    ref = orc.Context(s.n)
    ctx.set_bins([dcd.LM_HUB], [-1])
    for ins, dels in s.steps:
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, _ = ctx.update()
        rlab, rq, _ = ref.update(orc.DELTA)
        assert np.array_equal(lab, rlab) and abs(q - rq) <= 1e-12 * max(1.0, abs(rq))
    ctx.close()


def test_autotune_keeps_results(dcd, orc, synth):
    s = lfr_small(synth)
    ctx = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    ref = orc.Context(s.n)
    with pytest.raises(dcd.DcdError):
        ctx.autotune()  # no graph yet
    for t, (ins, dels) in enumerate(s.steps):
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, _ = ctx.update()
        rlab, rq, _ = ref.update(orc.DELTA)
        assert np.array_equal(lab, rlab) and abs(q - rq) <= 1e-12 * max(1.0, abs(rq))
        if t == 0:
            ms = ctx.autotune(reps=2)
            assert ms > 0.0
            variants, his = ctx.bins()
            assert variants[-1] == dcd.LM_HUB and his[-1] == -1
    ctx.close()


def test_group_autotune_keeps_results(dcd, orc, synth):
    streams = [synth.sbm_10k(replica=r, n=1500 + 500 * r, blocks=10 + r, steps=3) for r in range(3)]
    grp = dcd.Group([s.n for s in streams], mode=dcd.MODE_DELTA)
    refs = [orc.Context(s.n) for s in streams]
    for t in range(3):
        for g, s in enumerate(streams):
            grp.apply_batch(g, *s.steps[t])
            refs[g].apply_batch(*s.steps[t])
        lab, q, _ = grp.update()
        for g in range(3):
            rlab, rq, _ = refs[g].update(orc.DELTA)
            o = grp.offsets
            assert np.array_equal(lab[o[g]:o[g + 1]], rlab) and abs(q[g] - rq) <= 1e-12 * max(1.0, abs(rq))
        if t == 0:
            assert grp.autotune(reps=1) > 0.0
    grp.close()


# variant ids of include/dcd.h: 1 = DCD_LM_SEG32, 3 = DCD_LM_WARP128,
# 4 = DCD_LM_WARP256, 5 = DCD_LM_CTA512, 9 = DCD_LM_HUB
@pytest.mark.parametrize("variants,his", [
    ([], []),                                         # no bin
    ([1], [32]),                                      # last bin not the unbounded hub
    ([1, 9], [64, -1]),                               # above the segment variant's limit
    ([5, 3, 9], [20, 100, -1]),                       # valid: a CTA variant below a warp one
    ([4, 3, 9], [200, 100, -1]),                      # limits not increasing
    ([10, 9], [10, -1]),                              # unknown variant
    (list(range(9)) + [9, 9, 9, 9], [1] * 12 + [-1]),  # too many bins
])
def test_invalid_plans_are_refused(dcd, variants, his):
    ctx = dcd.Context(100)
    before = ctx.bins()
    if variants == [5, 3, 9]:
        ctx.set_bins(variants, his)  # increasing and within limits: accepted
        assert ctx.bins() == (variants, his)
        ctx.close()
        return
    with pytest.raises((dcd.DcdError, ValueError)):
        ctx.set_bins(variants, his)
    assert ctx.bins() == before
    ctx.close()


def test_eval_bins_counts_every_row_and_keeps_the_state(dcd, synth):
    """dcd_eval_bins times each bin alone on G_t under C_t: its vertex and
    entry counts cover every row of positive degree once, and the context
    (labels, graph) is unchanged by it."""
    s = lfr_small(synth)
    ctx = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    for ins, dels in s.steps[:2]:
        ctx.apply_batch(ins, dels)
        lab, _, _ = ctx.update()
    rp, col, w = ctx.graph()
    deg = np.diff(rp)
    plan = ctx.bins()
    rows = ctx.eval_bins(reps=2)
    assert [r[0] for r in rows] == plan[0]
    assert sum(r[1] for r in rows) == int((deg > 0).sum())
    assert sum(r[2] for r in rows) == int(deg.sum()) == len(col)
    lo = 0
    for (var, nv, ne, ms), hi in zip(rows, plan[1]):
        sel = (deg > lo) & ((deg <= hi) if hi >= 0 else True)
        assert nv == int(sel.sum()) and ne == int(deg[sel].sum())
        assert ms >= 0.0 and (ms > 0.0 or nv == 0)
        lo = hi
    assert np.array_equal(ctx.labels(), lab)
    rp2, col2, w2 = ctx.graph()
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2) and np.array_equal(w, w2)
    ctx.close()


def test_reserve_keeps_results_and_state(dcd, orc, synth):
    """dcd_reserve only pre-sizes buffers: a context that reserved memory
    before its first update, and one that reserved in the middle of the
    stream (G_t and a staged batch kept), give the oracle's results bit for
    bit; bad sizes are refused."""
    s = lfr_small(synth)
    nnz_max = 2 * sum(len(i) for i, _ in s.steps)
    rec_max = max(len(i) + len(d) for i, d in s.steps)
    a = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    a.reserve(nnz_max, rec_max)
    b = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    ref = orc.Context(s.n)
    for bad in ((-1, 10), (10, -1), (10, 1 << 30)):
        with pytest.raises(dcd.DcdError) as e:
            a.reserve(*bad)
        assert e.value.code == dcd.DCD_EINVAL
    for t, (ins, dels) in enumerate(s.steps):
        a.apply_batch(ins, dels)
        b.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        if t == 2:
            b.reserve(nnz_max, rec_max)  # a staged batch and G_{t-1} stay
        la, qa, sa = a.update()
        lb, qb, sb = b.update()
        rl, rq, _ = ref.update(orc.DELTA)
        assert np.array_equal(la, rl) and np.array_equal(lb, rl)
        assert abs(qa - rq) <= 1e-12 * max(1.0, abs(rq)) and qb == qa
        assert sa.nnz == sb.nnz
    a.close()
    b.close()
