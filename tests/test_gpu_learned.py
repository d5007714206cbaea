"""The learned screen end to end on the GPU: features and move labels against
the oracle, then a network trained on full re-evaluation runs that screens
fewer vertices than Delta-screening at the same modularity (within 1e-3)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dcd():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1904_08553_gb300 import dcd as m

    return m


def small_lfr(synth, replica, n=20_000, steps=6):
    return synth.lfr(synth.seed_for(4, replica), n=n, n_events=int(31.5 * n), steps=steps, kmax=n / 10,
                     smax=n / 20, smin=50)


def test_features_and_labels_match_oracle(dcd, orc, synth):
    s = small_lfr(synth, 0, n=4000, steps=4)
    ctx = dcd.Context(s.n, mode=dcd.MODE_BASE)
    ctx.set_collect(True)
    g_prev = orc.Graph.empty(s.n)
    labels = np.arange(s.n, dtype=np.int32)
    for t, (ins, dels) in enumerate(s.steps):
        ctx.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        g_t, err = g_prev.apply(ins, dels)
        assert err == 0
        if t > 0:
            X, y, v = ctx.screen_data()
            rds = orc.screen(g_prev, g_t, labels, ins, dels)
            pool, Xr = orc.screen_features(g_prev, g_t, labels, ins, dels, rds)
            assert sorted(v.tolist()) == np.nonzero(pool)[0].tolist()
            assert st.pool == len(v)
            np.testing.assert_allclose(X, Xr[v], rtol=2e-6, atol=1e-7)
            lev0, _, _, _ = g_t.run_level(labels)
            assert np.array_equal(y, (lev0[v] != labels[v]).astype(np.float32))
        g_prev, labels = g_t, lab


def test_learned_selection_matches_oracle(dcd, orc, synth):
    """R'_t of the learned screen against the oracle's selection: the oracle's
    pool and features, its FP64 network (BF16-rounded operands) and the same
    thresholds; every pool vertex whose score is clear of its threshold by
    more than the network tolerance (2e-2) must be selected alike, and no
    vertex outside the pool may be selected."""
    s = small_lfr(synth, 3, n=4000, steps=4)
    rng = np.random.default_rng(5)
    P = (rng.standard_normal(dcd.MLP_PARAMS) * 0.3).astype(np.float32)
    # centre the network's output on the first screened step (the oracle's
    # pool and scores): the output bias moves the median logit to 0, so both
    # thresholds below cut through the scores
    o = orc.Context(s.n)
    o.apply_batch(*s.steps[0])
    lab1, _, _ = o.update(orc.STATIC)
    g0, _ = orc.Graph.empty(s.n).apply(*s.steps[0])
    g1, _ = g0.apply(*s.steps[1])
    r1 = orc.screen(g0, g1, lab1, *s.steps[1])
    pool1, X1 = orc.screen_features(g0, g1, lab1, *s.steps[1], r1)
    p1, _ = orc.mlp_forward(P, X1[np.nonzero(pool1)[0]])
    p1 = np.clip(p1, 1e-6, 1 - 1e-6)
    P[-1] -= np.float32(np.median(np.log(p1 / (1 - p1))))
    mlp = dcd.Mlp(seed=1)
    mlp.params = P
    tk, ta = 0.4, 0.6
    ctx = dcd.Context(s.n, mode=dcd.MODE_LEARNED)
    ctx.set_screen(mlp, theta_keep=tk, theta_add=ta, judge=False)
    g_prev = orc.Graph.empty(s.n)
    labels = np.arange(s.n, dtype=np.int32)
    clear_total, near_total, picked = 0, 0, 0
    for t, (ins, dels) in enumerate(s.steps):
        ctx.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        g_t, err = g_prev.apply(ins, dels)
        assert err == 0
        if t > 0:
            rds = orc.screen(g_prev, g_t, labels, ins, dels)
            pool, X = orc.screen_features(g_prev, g_t, labels, ins, dels, rds)
            v = np.nonzero(pool)[0]
            p_ref, _ = orc.mlp_forward(P, X[v])
            thr = np.where(rds[v] != 0, tk, ta)
            want = p_ref >= thr
            got = ctx.rset()
            assert st.r_screen == int(rds.sum()) and st.pool == len(v)
            clear = np.abs(p_ref - thr) > 2e-2
            assert np.array_equal(got[v][clear] != 0, want[clear])
            outside = np.ones(s.n, bool)
            outside[v] = False
            assert not got[outside].any()
            clear_total += int(clear.sum())
            near_total += int((~clear).sum())
            picked += int(want.sum())
        g_prev, labels = g_t, lab
    ctx.close()
    # the comparison is not vacuous: most pool vertices are clear of their
    # threshold, and the selection keeps some vertices and drops others
    assert clear_total > 10 * max(near_total, 1)
    assert 0 < picked < clear_total + near_total


def collect(dcd, synth, replicas, n):
    Xs, ys = [], []
    for r in replicas:
        s = small_lfr(synth, r, n=n)
        ctx = dcd.Context(s.n, mode=dcd.MODE_BASE)
        ctx.set_collect(True)
        for t, (ins, dels) in enumerate(s.steps):
            ctx.apply_batch(ins, dels)
            ctx.update(labels_out=None)
            if t > 0:
                X, y, _ = ctx.screen_data()
                Xs.append(X)
                ys.append(y)
        ctx.close()
    return np.concatenate(Xs), np.concatenate(ys)


def test_trained_screen_prunes_r_at_equal_modularity(dcd, orc, synth):
    import torch

    X, y = collect(dcd, synth, range(1, 7), n=20_000)
    assert 0.0 < y.mean() < 1.0
    perm = np.random.default_rng(0).permutation(len(X))
    dX = torch.from_numpy(X[perm]).cuda()
    dy = torch.from_numpy(y[perm]).cuda()
    mlp = dcd.Mlp(seed=7)
    _, l0 = mlp.grad(dX, dy, len(X))
    mlp.train(dX, dy, len(X), batch=4096, epochs=6, lr=2e-3)
    _, l1 = mlp.grad(dX, dy, len(X))
    assert l1 < l0

    s = small_lfr(synth, 50, n=20_000)
    ctx = dcd.Context(s.n, mode=dcd.MODE_LEARNED)
    ctx.set_screen(mlp, theta_keep=0.3, theta_add=0.9, judge=True)
    ref = orc.Context(s.n)
    r_learned, r_screen = [], []
    for t, (ins, dels) in enumerate(s.steps):
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        if t == 0:
            ref.update(orc.STATIC)
            continue
        # the step the library kept is reproduced by the oracle from its R_t
        rl, rq, rst = ref.update(orc.GIVEN_R, ctx.rset())
        assert np.array_equal(lab, rl) and abs(q - rq) <= 1e-12 * max(1.0, abs(rq))
        if not st.fallback:
            assert q >= st.q_screen - 1e-3
        r_learned.append(st.r_size)
        r_screen.append(st.r_screen)
    assert np.mean(r_learned) < np.mean(r_screen)
