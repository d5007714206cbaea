"""Pins of the oracle's smart local moving (the paper's second host method,
dSLM-Delta-s) to facts that do not come from the oracle itself: closed forms
of modularity, exhaustive checks of the local-moving rule, brute force, and
the structure SLM's refinement must have.

The readings these pins follow are stated with the code:
  - SLM's local moving also offers an empty community, taken only when it beats
    every neighbouring community;
  - the refinement splits each community by local moving from singletons on
    the edges inside it, with the whole graph's degrees and 2m;
  - sub-communities are aggregated, each starting in its parent community.
"""
from fractions import Fraction

import numpy as np
import pytest

from test_oracle_pins import A_has, dense, n_pairwise, random_graph, set_partitions


def clique(base, s):
    return [(base + x, base + y) for x in range(s) for y in range(x + 1, s)]


@pytest.mark.parametrize("s", [3, 4, 5, 7])
def test_slm_splits_a_disconnected_community(orc, s):
    """Two disjoint s-cliques started in one community.  Neither local moving
    rule can split it vertex by vertex (leaving costs (s-1)^2 > 0 of 2 m^2 Q),
    so Louvain keeps Q = 0; SLM's refinement finds the two cliques and its
    coarse level moves one of them into an empty community: Q = 1/2."""
    n = 2 * s
    g = orc.Graph.from_edges(n, clique(0, s) + clique(s, s))
    init = np.zeros(n, np.int32)
    lab_l, st_l = g.louvain(init)
    assert (lab_l == 0).all() and st_l.q == 0.0
    lab, st = g.slm(init)
    assert (lab[:s] == 0).all() and (lab[s:] == s).all()
    # each clique holds half the edges and half the degree: 2 (1/2 - 1/4)
    assert Fraction(st.N, st.m2 * st.m2) == Fraction(1, 2)
    # why local moving alone cannot split it: a vertex leaving for an empty
    # community (label 1 is held by no vertex, so e_D = a_D = 0) gains
    # m2 (0 - e_C) - k (0 - a_C + k) with k = e_C = s - 1 and a_C = m2, that is
    # -(s - 1)^2
    assert g.gain(init, 0, 1) == -(s - 1) ** 2


@pytest.mark.parametrize("s", [3, 4, 6])
def test_slm_splits_two_joined_cliques_to_the_closed_form(orc, s):
    """Two s-cliques joined by one edge, started in one community: SLM ends
    with the two cliques, Q = 1/2 - 1/(s(s-1)+1) (the closed form of the
    Louvain pins), while Louvain from the same start cannot move."""
    n = 2 * s
    edges = clique(0, s) + clique(s, s) + [(s - 1, s)]
    g = orc.Graph.from_edges(n, edges)
    init = np.zeros(n, np.int32)
    lab_l, st_l = g.louvain(init)
    assert (lab_l == 0).all()
    lab, st = g.slm(init)
    assert (lab[:s] == 0).all() and (lab[s:] == s).all()
    assert Fraction(st.N, st.m2 * st.m2) == Fraction(1, 2) - Fraction(1, s * (s - 1) + 1)


def test_refinement_nests_in_the_parent_communities(orc):
    rng = np.random.default_rng(41)
    for trial in range(40):
        n = int(rng.integers(4, 40))
        edges = random_graph(rng, n, p=0.3)
        if not edges:
            continue
        g = orc.Graph.from_edges(n, edges)
        parent = rng.integers(0, max(1, n // 3), n).astype(np.int32)
        sub, it, moves = g.slm_refine(parent)
        for c in np.unique(sub):
            members = np.nonzero(sub == c)[0]
            assert members.min() == c  # canonical
            assert len(np.unique(parent[members])) == 1  # inside one parent
        # (sub-communities need not be connected: as in any local moving, a
        # vertex can join a community in the pass where its link to it leaves)
        # every parent community is covered by its sub-communities
        for p in np.unique(parent):
            assert set(np.unique(sub[parent == p]).tolist()) <= set(np.nonzero(parent == p)[0].tolist())


def test_refinement_from_a_single_community_has_no_improving_move(orc):
    """With one parent the refinement is SLM local moving from singletons on
    the whole graph; when it stops because no vertex moves, no neighbouring
    community and no empty community gives a positive gain (exhaustive, with
    the gain formula of the Louvain pins), except where the swap guard holds."""
    rng = np.random.default_rng(42)
    seen = 0
    for trial in range(40):
        n = int(rng.integers(6, 30))
        edges = random_graph(rng, n, p=0.25)
        if not edges:
            continue
        g = orc.Graph.from_edges(n, edges)
        sub, it, moves = g.slm_refine(np.zeros(n, np.int32))
        lab2, it2, mv2 = g.slm_level(sub)
        if mv2 != 0 or not (lab2 == sub).all():
            continue  # the refinement stopped by the tau rule
        seen += 1
        sizes = np.bincount(sub, minlength=n)
        empty = n  # unused label: e_D = a_D = 0
        for v in range(n):
            for D in set(sub.tolist()) - {int(sub[v])}:
                adjacent = any(sub[u] == D for u in range(n) if u != v and A_has(edges, v, u))
                guard = sizes[sub[v]] == 1 and sizes[D] == 1 and D > sub[v]
                assert g.gain(sub, v, D) <= 0 or guard or not adjacent
            if sizes[sub[v]] > 1:
                ext = np.append(sub, np.int32(empty))  # label n exists nowhere in the graph
                assert g.gain(ext[:n], v, empty) <= 0
    assert seen > 10


def test_slm_below_brute_force_optimum(orc):
    rng = np.random.default_rng(43)
    parts = {n: set_partitions(n) for n in (6, 8)}
    for n, trials in ((6, 6), (8, 4)):
        P = parts[n]
        for t in range(trials):
            edges = random_graph(rng, n, p=0.4)
            if not edges:
                continue
            A = dense(n, edges).astype(np.int64)
            k = A.sum(1)
            m2 = int(k.sum())
            B = m2 * A - np.outer(k, k)
            eq = P[:, :, None] == P[:, None, :]
            best = int((eq * B).sum((1, 2)).max())
            g = orc.Graph.from_edges(n, edges)
            lab, st = g.slm()
            assert st.m2 == m2 and st.N <= best
            Nref, _ = n_pairwise(dense(n, edges), lab)
            assert st.N == Nref


def test_slm_modes_reduce_like_louvain(orc, synth):
    """R = V reproduces dSLM-base, and dSLM-base from singletons reproduces a
    static SLM run, as for Louvain."""
    s = synth.sbm_10k(n=2000, blocks=20, steps=3)
    a, b = orc.Context(s.n), orc.Context(s.n)
    for ins, dels in s.steps:
        a.apply_batch(ins, dels)
        b.apply_batch(ins, dels)
        la, qa, sa = a.update(orc.BASE, alg=orc.SLM)
        lb, qb, sb = b.update(orc.GIVEN_R, np.ones(s.n, np.uint8), alg=orc.SLM)
        assert (la == lb).all() and qa == qb
    ins, dels = s.steps[0]
    c = orc.Context(s.n)
    c.apply_batch(ins, dels)
    lc, qc, _ = c.update(orc.STATIC, alg=orc.SLM)
    g = orc.Graph.from_edges(s.n, ins)
    lg, st = g.slm()
    assert (lc == lg).all() and qc == st.q


def test_dslm_delta_recovers_the_planted_sbm(orc, synth):
    s = synth.sbm_10k(n=2000, blocks=20, steps=3)
    ctx = orc.Context(s.n)
    for t, (ins, dels) in enumerate(s.steps):
        ctx.apply_batch(ins, dels)
        lab, q, st = ctx.update(orc.DELTA, alg=orc.SLM)
        if t == 0:
            for b in range(20):
                assert len(np.unique(lab[s.planted == b])) == 1
            assert st.communities == 20
        for c in np.unique(lab):
            assert np.nonzero(lab == c)[0].min() == c
    assert st.refine_iters > 0


def test_unknown_host_method_is_refused(orc):
    c = orc.Context(10)
    with pytest.raises(RuntimeError):
        c.update(orc.DELTA, alg=7)
