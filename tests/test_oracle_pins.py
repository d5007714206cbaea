"""Pins of the CPU oracle to facts the paper and the mathematics fix.

None of these tests compares the oracle with itself: every expected value comes
from a closed form, an independent formula (the pairwise form of Eq. 1), a
dictionary re-implementation, brute force, or an identity the paper states.
"""
from fractions import Fraction

import numpy as np
import pytest


# ---------------------------------------------------------------- helpers

def dense(n, edges):
    """Symmetric weight matrix of an undirected multigraph (duplicates add)."""
    A = np.zeros((n, n), dtype=object)
    for e in edges:
        u, v = int(e[0]), int(e[1])
        w = int(e[2]) if len(e) > 2 else 1
        A[u, v] += w
        A[v, u] += w
    return A


def n_pairwise(A, labels):
    """m2^2 * Q from the pairwise form Q = (1/2m) sum_ij (A_ij - k_i k_j / 2m) [c_i = c_j]."""
    n = A.shape[0]
    k = [sum(A[i, j] for j in range(n)) for i in range(n)]
    m2 = sum(k)
    N = 0
    for i in range(n):
        for j in range(n):
            if labels[i] == labels[j]:
                N += m2 * A[i, j] - k[i] * k[j]
    return N, m2


def random_graph(rng, n, p=0.5, wmax=3):
    edges = []
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < p:
                edges.append((u, v, int(rng.integers(1, wmax + 1))))
    return edges


def cliques_ring(K, s):
    E = []
    for c in range(K):
        b = c * s
        E += [(b + x, b + y) for x in range(s) for y in range(x + 1, s)]
        E.append((b + s - 1, ((c + 1) % K) * s))
    return E


def set_partitions(n):
    """All partitions of n items as restricted growth strings."""
    out = []
    a = [0] * n

    def rec(i, mx):
        if i == n:
            out.append(a.copy())
            return
        for c in range(mx + 2):
            a[i] = c
            rec(i + 1, max(mx, c))

    a[0] = 0
    rec(1, 0) if n > 1 else out.append([0])
    return np.array(out, dtype=np.int64)


# ---------------------------------------------------------------- Eq. (1)

@pytest.mark.parametrize("s", [3, 4, 5, 6, 8])
def test_two_cliques_closed_form(orc, s):
    edges = [(x, y) for x in range(s) for y in range(x + 1, s)]
    edges += [(s + x, s + y) for x in range(s) for y in range(x + 1, s)]
    edges.append((s - 1, s))
    g = orc.Graph.from_edges(2 * s, edges)
    cl = np.repeat([0, s], s).astype(np.int32)
    q, N, m2 = g.modularity(cl)
    assert Fraction(N, m2 * m2) == Fraction(1, 2) - Fraction(1, s * (s - 1) + 1)
    lab, st = g.louvain()
    assert (lab == cl).all()
    assert st.N == N


@pytest.mark.parametrize("K,s", [(3, 3), (4, 4), (6, 5), (10, 4), (8, 3), (16, 3), (30, 3), (12, 5)])
def test_ring_of_cliques(orc, K, s):
    g = orc.Graph.from_edges(K * s, cliques_ring(K, s))
    cl = np.repeat(np.arange(K) * s, s).astype(np.int32)
    m = K * (s * (s - 1) // 2 + 1)
    closed = K * (Fraction(s * (s - 1) // 2, m) - Fraction(s * (s - 1) + 2, 2 * m) ** 2)
    q, N, m2 = g.modularity(cl)
    assert Fraction(N, m2 * m2) == closed
    lab, st = g.louvain()
    if K <= s * (s - 1) + 2:
        # merging two neighbouring cliques gains 1/m - d^2/(2 m^2) <= 0 here
        assert (lab == cl).all()
        assert Fraction(st.N, st.m2 ** 2) == closed
    else:
        assert Fraction(st.N, st.m2 ** 2) > closed


def test_modularity_matches_pairwise_form(orc):
    rng = np.random.default_rng(1)
    for trial in range(60):
        n = int(rng.integers(2, 13))
        edges = random_graph(rng, n, p=float(rng.uniform(0.2, 0.9)))
        if not edges:
            continue
        g = orc.Graph.from_edges(n, edges)
        lab = rng.integers(0, n, n).astype(np.int32)
        q, N, m2 = g.modularity(lab)
        Nref, m2ref = n_pairwise(dense(n, edges), lab)
        assert (N, m2) == (Nref, m2ref)
        assert q == pytest.approx(float(Fraction(Nref, m2ref * m2ref)), rel=1e-15)


def test_modularity_empty_graph_is_zero(orc):
    g = orc.Graph.empty(5)
    q, N, m2 = g.modularity(np.arange(5, dtype=np.int32))
    assert (q, N, m2) == (0.0, 0, 0)


# ---------------------------------------------------------------- gain S

def test_gain_is_half_the_change_of_N(orc):
    rng = np.random.default_rng(2)
    for trial in range(40):
        n = int(rng.integers(3, 11))
        edges = random_graph(rng, n, p=0.5)
        if not edges:
            continue
        A = dense(n, edges)
        g = orc.Graph.from_edges(n, edges)
        lab = rng.integers(0, max(2, n // 2), n).astype(np.int32)
        N0, _ = n_pairwise(A, lab)
        for v in range(n):
            for D in set(lab.tolist()) | {int(rng.integers(0, n))}:
                S = g.gain(lab, v, D)
                after = lab.copy()
                after[v] = D
                N1, _ = n_pairwise(A, after)
                assert 2 * S == N1 - N0, (v, D)


def test_lemma_3_2_identity(orc):
    """i moves C -> D; a member i2 of C not adjacent to i loses exactly
    2 k_{i2} k_i of gain towards D (appendix proof of Lemma 3.2)."""
    rng = np.random.default_rng(3)
    checked = 0
    for trial in range(200):
        n = 12
        edges = random_graph(rng, n, p=0.3)
        if not edges:
            continue
        A = dense(n, edges)
        k = [sum(A[i, j] for j in range(n)) for i in range(n)]
        g = orc.Graph.from_edges(n, edges)
        lab = rng.integers(0, 3, n).astype(np.int32)
        i = int(rng.integers(0, n))
        C = lab[i]
        D = (C + 1) % 3
        for i2 in range(n):
            if i2 == i or lab[i2] != C or A[i, i2] != 0:
                continue
            before = g.gain(lab, i2, D)
            moved = lab.copy()
            moved[i] = D
            after = g.gain(moved, i2, D)
            assert after == before - 2 * k[i2] * k[i]
            checked += 1
    assert checked > 50


def test_lemma_3_4b_identity(orc):
    """k outside C(i) and C(j*), not adjacent to i: its gain towards C(j*)
    drops by exactly k_k k_i when i joins C(j*) (Lemma 3.4, case B; the
    paper writes an approximation, the integer identity is exact)."""
    rng = np.random.default_rng(4)
    checked = 0
    for trial in range(200):
        n = 12
        edges = random_graph(rng, n, p=0.3)
        if not edges:
            continue
        A = dense(n, edges)
        kk = [sum(A[i, j] for j in range(n)) for i in range(n)]
        g = orc.Graph.from_edges(n, edges)
        lab = rng.integers(0, 4, n).astype(np.int32)
        i = int(rng.integers(0, n))
        C = lab[i]
        D = (C + 1) % 4
        for k in range(n):
            if k == i or lab[k] in (C, D) or A[i, k] != 0:
                continue
            before = g.gain(lab, k, D)
            moved = lab.copy()
            moved[i] = D
            assert g.gain(moved, k, D) == before - kk[k] * kk[i]
            checked += 1
    assert checked > 50


# ---------------------------------------------------------------- Algorithm 1

def reference_pass(A, lab, active):
    """Decision rule restated with gains taken as half the change of the
    pairwise N: best neighbour community by gain, smallest label on ties,
    move only on a positive gain, singleton-swap guard."""
    n = A.shape[0]
    N0, _ = n_pairwise(A, lab)
    size = {c: int((lab == c).sum()) for c in set(lab.tolist())}
    out = lab.copy()
    for v in range(n):
        if active is not None and not active[v]:
            continue
        C = int(lab[v])
        cands = sorted({int(lab[u]) for u in range(n) if u != v and A[v, u] != 0} - {C})
        best, bestS = C, 0
        for D in cands:
            t = lab.copy()
            t[v] = D
            S = (n_pairwise(A, t)[0] - N0) // 2
            if S > bestS:
                best, bestS = D, S
        if best != C and size[C] == 1 and size[best] == 1 and best > C:
            best = C
        out[v] = best
    return out


def test_local_move_pass_rule(orc):
    rng = np.random.default_rng(5)
    for trial in range(25):
        n = int(rng.integers(4, 11))
        edges = random_graph(rng, n, p=0.45)
        if not edges:
            continue
        A = dense(n, edges)
        g = orc.Graph.from_edges(n, edges)
        for lab in (np.arange(n, dtype=np.int32), rng.integers(0, 3, n).astype(np.int32)):
            active = (rng.random(n) < 0.7).astype(np.uint8)
            out, moves = g.local_move_pass(lab, active)
            ref = reference_pass(A, lab, active)
            assert (out == ref).all()
            assert moves == int((ref != lab).sum())


def test_converged_level_has_no_improving_move(orc):
    rng = np.random.default_rng(6)
    seen = 0
    for trial in range(40):
        n = int(rng.integers(6, 30))
        edges = random_graph(rng, n, p=0.25)
        if not edges:
            continue
        g = orc.Graph.from_edges(n, edges)
        lab, it, moves, edges_scanned = g.run_level(np.arange(n, dtype=np.int32))
        out, mv = g.local_move_pass(lab)
        if mv != 0:
            continue  # stopped by the tau rule, not by a no-move pass
        seen += 1
        sizes = np.bincount(lab, minlength=n)
        for v in range(n):
            for D in set(lab.tolist()) - {int(lab[v])}:
                S = g.gain(lab, v, D)
                guard = sizes[lab[v]] == 1 and sizes[D] == 1 and D > lab[v]
                adjacent = any(lab[u] == D for u in range(n) if u != v and A_has(edges, v, u))
                assert S <= 0 or guard or not adjacent
    assert seen > 10


def A_has(edges, v, u):
    return any((a == v and b == u) or (a == u and b == v) for a, b, *_ in edges)


def test_coarsening_invariants(orc):
    rng = np.random.default_rng(7)
    for trial in range(30):
        n = int(rng.integers(3, 16))
        edges = random_graph(rng, n, p=0.4)
        if not edges:
            continue
        g = orc.Graph.from_edges(n, edges)
        lab = rng.integers(0, n, n).astype(np.int32)
        cg, cid = g.coarsen(lab)
        used = sorted(set(lab.tolist()))
        assert cg.n == len(used)
        assert (cid == np.array([used.index(x) for x in lab])).all()
        # coarse edges = sum of fine ordered pairs mapped by label rank
        agg = {}
        for u, v, w in edges:
            for a, b in ((u, v), (v, u)):
                key = (used.index(lab[a]), used.index(lab[b]))
                agg[key] = agg.get(key, 0) + w
        rp, col, w = cg.csr()
        got = {(u, int(col[e])): int(w[e]) for u in range(cg.n) for e in range(rp[u], rp[u + 1])}
        assert got == agg
        q0, N0, m20 = g.modularity(lab)
        q1, N1, m21 = cg.modularity(np.arange(cg.n, dtype=np.int32))
        assert (N0, m20) == (N1, m21)


def test_louvain_below_brute_force_optimum(orc):
    rng = np.random.default_rng(8)
    parts = {n: set_partitions(n) for n in (6, 8, 10)}
    for n, trials in ((6, 6), (8, 4), (10, 2)):
        P = parts[n]
        for t in range(trials):
            edges = random_graph(rng, n, p=0.4)
            if not edges:
                continue
            A = dense(n, edges).astype(np.int64)
            k = A.sum(1)
            m2 = int(k.sum())
            B = m2 * A - np.outer(k, k)
            best = -(1 << 62)
            for s in range(0, len(P), 20000):
                blk = P[s:s + 20000]
                eq = blk[:, :, None] == blk[:, None, :]
                best = max(best, int((eq * B).sum((1, 2)).max()))
            g = orc.Graph.from_edges(n, edges)
            lab, st = g.louvain()
            assert st.m2 == m2
            assert st.N <= best
            Nref, _ = n_pairwise(dense(n, edges), lab)
            assert st.N == Nref


# ---------------------------------------------------------------- batch apply

def test_apply_batch_against_dictionary(orc):
    rng = np.random.default_rng(9)
    n = 40
    g = orc.Graph.empty(n)
    ref = {}
    for step in range(30):
        ni, nd = int(rng.integers(0, 60)), int(rng.integers(0, 25))
        ins = []
        while len(ins) < ni:
            u, v = rng.integers(0, n, 2)
            if u != v:
                ins.append((int(u), int(v), int(rng.integers(1, 5))))
        keys = list(ref.keys())
        dels = []
        for x in range(nd):
            if keys and rng.random() < 0.8:
                a, b = keys[int(rng.integers(0, len(keys)))]
                dels.append((b, a) if rng.random() < 0.5 else (a, b))
            else:
                u, v = rng.integers(0, n, 2)
                if u != v:
                    dels.append((int(u), int(v)))
        present = [1 if (min(a, b), max(a, b)) in ref else 0 for a, b in dels]
        for a, b in dels:
            ref.pop((min(a, b), max(a, b)), None)
        for a, b, w in ins:
            key = (min(a, b), max(a, b))
            ref[key] = ref.get(key, 0) + w
        g, err, pres = g.apply(ins, dels, want_present=True)
        assert err == 0
        assert pres.tolist() == present
        rp, col, w = g.csr()
        got = {}
        for u in range(n):
            row = col[rp[u]:rp[u + 1]]
            assert (np.diff(row) > 0).all()
            for e in range(rp[u], rp[u + 1]):
                got[(u, int(col[e]))] = int(w[e])
        exp = {}
        for (a, b), w_ in ref.items():
            exp[(a, b)] = w_
            exp[(b, a)] = w_
        assert got == exp


@pytest.mark.parametrize("ins,dels", [
    ([(1, 1, 1)], []),
    ([(0, 5, 1)], []),
    ([(0, 1, 0)], []),
    ([(0, 1, -2)], []),
    ([], [(2, 2)]),
    ([], [(-1, 2)]),
])
def test_apply_batch_rejects_bad_input(orc, ins, dels):
    g = orc.Graph.from_edges(5, [(0, 1), (1, 2)])
    out, err = g.apply(ins, dels)
    assert out is None and err == -1
    ctx = orc.Context(5)
    assert ctx.apply_batch(ins, dels) == -1


# ---------------------------------------------------------------- Algorithm 2

def _two_communities():
    # community A = {0..4} (K5), community B = {5..9} (K5), bridge (4,5)
    E = [(x, y) for x in range(5) for y in range(x + 1, 5)]
    E += [(5 + x, 5 + y) for x in range(5) for y in range(x + 1, 5)]
    E.append((4, 5))
    lab = np.array([0] * 5 + [5] * 5 + [10, 11], np.int32)  # 10, 11 isolated
    return 12, E, lab


def test_screen_intra_community_insert_marks_nothing(orc):
    n, E, lab = _two_communities()
    gp = orc.Graph.from_edges(n, E)
    ins = [(0, 2, 1)]  # raises the multiplicity of an intra edge
    gt, err = gp.apply(ins)
    r = orc.screen(gp, gt, lab, ins)
    assert r.sum() == 0


def test_screen_empty_batch(orc):
    n, E, lab = _two_communities()
    gp = orc.Graph.from_edges(n, E)
    assert orc.screen(gp, gp, lab).sum() == 0


def test_screen_isolated_vertex_joins(orc):
    """Isolated i gets an edge to j in D: gain1 = w (m2 - a_D) > 0, so R gets
    {i, j} u Gamma(i) u D; no other vertex."""
    n, E, lab = _two_communities()
    gp = orc.Graph.from_edges(n, E)
    ins = [(10, 7, 1)]
    gt, err = gp.apply(ins)
    S = gt.gain(lab, 10, 5)
    q, N, m2 = gt.modularity(lab)
    aD = 2 * 10 + 1 + 1  # K5 degrees (20) + bridge (1) + new edge (1)
    assert S == 1 * (m2 - aD) and S > 0
    r = orc.screen(gp, gt, lab, ins)
    assert sorted(np.nonzero(r)[0].tolist()) == [5, 6, 7, 8, 9, 10]


def test_screen_defers_to_the_larger_gain(orc):
    """A source whose best gain is below the reverse gain adds nothing; the
    reverse orientation adds {j, i} u Gamma(j) u C(i) (Algorithm 2)."""
    rng = np.random.default_rng(10)
    found = 0
    for trial in range(3000):
        n = 10
        E = random_graph(rng, n, p=0.3, wmax=2)
        lab = rng.integers(0, 4, n).astype(np.int32)
        i, j = (int(x) for x in rng.choice(n, 2, replace=False))
        if lab[i] == lab[j]:
            continue
        gp = orc.Graph.from_edges(n, E) if E else orc.Graph.empty(n)
        ins = [(i, j, 1)]
        gt, err = gp.apply(ins)
        g1 = gt.gain(lab, i, lab[j])
        g2 = gt.gain(lab, j, lab[i])
        if not (0 < g1 < g2):
            continue
        r = orc.screen(gp, gt, lab, ins)
        rp, col, w = gt.csr()
        exp = {i, j} | set(col[rp[j]:rp[j + 1]].tolist()) | set(np.nonzero(lab == lab[i])[0].tolist())
        assert set(np.nonzero(r)[0].tolist()) == exp
        found += 1
        if found >= 10:
            break
    assert found >= 10


def test_screen_picks_best_sink(orc):
    """Isolated source with two sinks: j* is the sink of the larger gain, and
    only C(j*) is added whole; the other sink enters through Gamma(i)."""
    n, E, lab = _two_communities()
    gp = orc.Graph.from_edges(n, E)
    # vertex 10 gets edges into community 0 (weight 3) and community 5 (weight 1)
    ins = [(10, 1, 3), (10, 6, 1)]
    gt, err = gp.apply(ins)
    assert gt.gain(lab, 10, 0) > 0 and gt.gain(lab, 10, 0) > gt.gain(lab, 10, 5)
    # the sinks as sources: 1 defers to the larger reverse gain, 6 has none
    assert gt.gain(lab, 1, 10) < gt.gain(lab, 10, 0) and gt.gain(lab, 6, 10) <= 0
    r = orc.screen(gp, gt, lab, ins)
    assert set(np.nonzero(r)[0].tolist()) == {0, 1, 2, 3, 4, 6, 10}


def test_screen_deletion_rule(orc):
    """Deletion reading (not in the paper): an intra-community delete adds
    both endpoints and their neighbourhoods in G_t; an inter-community delete
    adds the two endpoints; deleting an absent edge adds nothing."""
    n, E, lab = _two_communities()
    gp = orc.Graph.from_edges(n, E)
    gt, err = gp.apply(None, [(0, 1)])
    r = orc.screen(gp, gt, lab, None, [(0, 1)])
    assert set(np.nonzero(r)[0].tolist()) == {0, 1, 2, 3, 4}
    gt, err = gp.apply(None, [(5, 4)])
    r = orc.screen(gp, gt, lab, None, [(5, 4)])
    assert set(np.nonzero(r)[0].tolist()) == {4, 5}
    gt, err = gp.apply(None, [(0, 9)])
    assert orc.screen(gp, gt, lab, None, [(0, 9)]).sum() == 0


# ---------------------------------------------------------------- Sec. III-D modes

def test_all_vertices_screen_reproduces_base(orc, synth):
    s = synth.sbm_10k(n=2000, blocks=20, steps=3)
    a, b = orc.Context(s.n), orc.Context(s.n)
    for t, (ins, dels) in enumerate(s.steps):
        a.apply_batch(ins, dels)
        b.apply_batch(ins, dels)
        la, qa, sa = a.update(orc.BASE)
        lb, qb, sb = b.update(orc.GIVEN_R, np.ones(s.n, np.uint8))
        assert (la == lb).all() and qa == qb


def test_base_from_singletons_reproduces_static(orc, synth):
    s = synth.sbm_10k(n=2000, blocks=20, steps=2)
    ins, dels = s.steps[0]
    a = orc.Context(s.n)
    a.apply_batch(ins, dels)
    la, qa, _ = a.update(orc.STATIC)
    b = orc.Context(s.n)
    b.set_labels(np.arange(s.n, dtype=np.int32))
    b.apply_batch(ins, dels)
    lb, qb, _ = b.update(orc.BASE)
    assert (la == lb).all() and qa == qb


def test_first_update_is_static_and_labels_canonical(orc, synth):
    s = synth.sbm_10k(n=1000, blocks=10, steps=1)
    ins, dels = s.steps[0]
    ctx = orc.Context(s.n)
    ctx.apply_batch(ins, dels)
    lab, q, st = ctx.update(orc.DELTA)
    g = orc.Graph.from_edges(s.n, ins)
    lab2, st2 = g.louvain()
    assert (lab == lab2).all() and q == st2.q
    for c in np.unique(lab):
        assert np.nonzero(lab == c)[0].min() == c
    assert st.r_size == s.n


def test_empty_step_has_empty_rset(orc, synth):
    s = synth.sbm_10k(n=1000, blocks=10, steps=1)
    ctx = orc.Context(s.n)
    ctx.apply_batch(*s.steps[0])
    lab1, q1, _ = ctx.update(orc.DELTA)
    lab2, q2, st = ctx.update(orc.DELTA)
    assert st.r_size == 0
    assert ctx.rset().sum() == 0
    assert q2 >= q1 - 1e-12


def test_planted_sbm_is_recovered(orc, synth):
    s = synth.sbm_10k(n=2000, blocks=20, steps=1)
    ctx = orc.Context(s.n)
    ctx.apply_batch(*s.steps[0])
    lab, q, st = ctx.update(orc.DELTA)
    # every planted block maps to one community
    for b in range(20):
        assert len(np.unique(lab[s.planted == b])) == 1
    assert st.communities == 20
