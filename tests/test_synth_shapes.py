"""The seeded generators against the recipes stated for them (the synthetic
stand-ins for the paper's datasets).  Each stream is replayed on a plain
Python edge set, independently of the generator and of both method
implementations: counts, distinctness, that deletes hit present edges and
inserts of the SBM absent ones, weights, self-loops, and the mixing of the
LFR-style stream."""
import numpy as np
import pytest


def key(u, v):
    return (int(u), int(v)) if u < v else (int(v), int(u))


def replay(stream, check_step):
    E = {}
    for t, (ins, dels) in enumerate(stream.steps):
        check_step(t, ins, dels, E)
        for u, v in dels:
            E.pop(key(u, v), None)
        for u, v, w in ins:
            k = key(u, v)
            E[k] = E.get(k, 0) + int(w)
    return E


def test_sbm_10k_recipe(synth):
    s = synth.sbm_10k()
    assert s.n == 10_000 and len(s.steps) == 6
    blocks = s.planted
    assert np.array_equal(np.bincount(blocks), np.full(100, 100))

    def check(t, ins, dels, E):
        assert np.all(ins[:, 2] == 1) and np.all(ins[:, 0] != ins[:, 1])
        pairs = {key(u, v) for u, v, _ in ins}
        assert len(pairs) == len(ins)  # distinct pairs
        intra = int((blocks[ins[:, 0]] == blocks[ins[:, 1]]).sum())
        if t == 0:
            assert len(dels) == 0 and intra == 80_000 and len(ins) - intra == 20_000
        else:
            dk = {key(u, v) for u, v in dels}
            assert len(dels) == 1_000 and len(dk) == 1_000 and dk <= set(E)
            assert len(ins) == 5_000 and intra == 4_000
            assert not (pairs & set(E))  # absent from G_{t-1}

    replay(s, check)


def test_lfr_recipe(synth):
    n, events, steps = 30_000, 450_000, 6
    s = synth.lfr(synth.seed_for(1, 31), n=n, n_events=events, steps=steps, kmin=4, kmax=3000, smin=20,
                  smax=3000)
    assert s.n == n and len(s.steps) == steps
    counts = [len(i) for i, _ in s.steps]
    assert sum(counts) == events  # one record per event, weight 1
    # each event picks its step uniformly: binomial counts
    mean, sd = events / steps, (events * (1 / steps) * (1 - 1 / steps)) ** 0.5
    assert all(abs(c - mean) < 5 * sd for c in counts)

    def check(t, ins, dels, E):
        assert np.all(ins[:, 2] == 1) and np.all(ins[:, 0] != ins[:, 1])
        assert ins[:, :2].min() >= 0 and ins[:, :2].max() < n
        dk = {key(u, v) for u, v in dels}
        assert len(dk) == len(dels) and dk <= set(E)
        if t == 0:
            assert len(dels) == 0
        else:
            # each distinct edge of G_{t-1} is deleted with probability 0.02
            assert abs(len(dels) - 0.02 * len(E)) <= 5 * (0.02 * 0.98 * len(E)) ** 0.5

    E = replay(s, check)
    # the last step's events use the final planted communities (drift happens
    # at the start of a step): 70 % are drawn inside the community, the rest
    # globally (which lands inside with a small probability)
    ins = s.steps[-1][0]
    intra = float(np.mean(s.planted[ins[:, 0]] == s.planted[ins[:, 1]]))
    assert 0.69 <= intra <= 0.76
    # heavy-tailed degrees from the power-law propensities
    deg = np.zeros(n, np.int64)
    for (u, v), w in E.items():
        deg[u] += 1
        deg[v] += 1
    assert deg.max() > 20 * np.median(deg)


def test_rmat_recipe(synth):
    scale, ef = 12, 16
    s = synth.rmat(synth.seed_for(2, 0), scale, edge_factor=ef, steps=4)

    def check(t, ins, dels, E):
        assert ins[:, 2].min() >= 1 and ins[:, 2].max() <= 8
        assert np.all(ins[:, 0] != ins[:, 1])  # self-loops dropped
        assert ins[:, :2].max() < (1 << scale)
        dk = {key(u, v) for u, v in dels}
        assert len(dk) == len(dels) and dk <= set(E)
        if t == 0:
            assert len(dels) == 0 and 0.99 * ef * (1 << scale) <= len(ins) <= ef * (1 << scale)
        else:
            # 1 % fresh samples (less the self-loops dropped), 0.5 % deletes
            assert 0.01 * len(E) - 10 <= len(ins) <= 0.01 * len(E) + 1
            assert abs(len(dels) - 0.005 * len(E)) <= 1

    replay(s, check)


def test_batched_parameters(synth):
    p = synth.batched_params(synth.seed_for(3, 0), G=512)
    assert len(p) == 512
    n = np.array([x[0] for x in p])
    deg = np.array([x[1] for x in p])
    assert n.min() >= 500 and n.max() <= 200_000
    # log-uniform: the mean of ln n is the midpoint of [ln 500, ln 200000]
    mid, half = (np.log(500) + np.log(200_000)) / 2, (np.log(200_000) - np.log(500)) / 2
    assert abs(np.log(n).mean() - mid) < 4 * half / np.sqrt(3 * 512)
    assert deg.min() >= 8 and deg.max() <= 32
    for ng, _, sizes in p:
        assert sizes.sum() == ng and sizes.min() >= 20 and sizes.max() <= 2000 + 19


@pytest.mark.parametrize("make", ["sbm", "lfr"])
def test_generators_are_seeded(synth, make):
    if make == "sbm":
        a, b = synth.sbm_10k(replica=3, n=2000, blocks=20, steps=3), synth.sbm_10k(replica=3, n=2000, blocks=20,
                                                                                       steps=3)
    else:
        kw = dict(n=5000, n_events=50_000, steps=3, kmin=4, kmax=500, smin=20, smax=500)
        a, b = synth.lfr(synth.seed_for(1, 9), **kw), synth.lfr(synth.seed_for(1, 9), **kw)
    assert np.array_equal(a.planted, b.planted)
    for (i1, d1), (i2, d2) in zip(a.steps, b.steps):
        assert np.array_equal(i1, i2) and np.array_equal(d1, d2)
