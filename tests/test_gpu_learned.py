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
