"""Pin of the oracle's learned-screen pool and features to a re-implementation
from their definitions: plain Python dictionaries for G_{t-1}, the batch and
G_t (deletes first, inserts add weight), and each of the twelve features
written out from its definition.  Nothing here calls the oracle's graph code
except orc_screen_features itself (and Graph.from_edges / apply to build its
inputs)."""
import math

import numpy as np


def key(u, v):
    return (u, v) if u < v else (v, u)


def apply_dict(E, ins, dels):
    E = dict(E)
    for u, v in dels:
        E.pop(key(int(u), int(v)), None)
    for u, v, w in ins:
        k = key(int(u), int(v))
        E[k] = E.get(k, 0) + int(w)
    return E


def rows(n, E):
    R = [dict() for _ in range(n)]
    for (u, v), w in E.items():
        R[u][v] = R[u].get(v, 0) + w
        R[v][u] = R[v].get(u, 0) + w
    return R


def features(n, E_prev, E_t, L, ins, dels, rds):
    """Pool and the twelve features of each pool vertex, in float64."""
    R = rows(n, E_t)
    k = [sum(r.values()) for r in R]
    m2 = sum(k)
    a, size = {}, {}
    for v in range(n):
        a[L[v]] = a.get(L[v], 0) + k[v]
        size[L[v]] = size.get(L[v], 0) + 1
    touched = set()
    for u, v, _ in ins:
        touched |= {int(u), int(v)}
    for u, v in dels:
        touched |= {int(u), int(v)}
    pool = {v for v in range(n) if rds[v]} | touched
    for v in touched:
        pool |= set(R[v])
    pool = {v for v in pool if len(R[v]) > 0}
    ins_sinks = [set() for _ in range(n)]
    wins = [0] * n
    for u, v, w in ins:
        u, v = int(u), int(v)
        ins_sinks[u].add(v)
        ins_sinks[v].add(u)
        wins[u] += int(w)
        wins[v] += int(w)
    del_sinks = [set() for _ in range(n)]
    for u, v in dels:
        u, v = int(u), int(v)
        if key(u, v) in E_prev:
            del_sinks[u].add(v)
            del_sinks[v].add(u)
    X = {}
    for v in pool:
        C = L[v]
        eC = sum(w for u, w in R[v].items() if u != v and L[u] == C)
        e_to = {}
        for u, w in R[v].items():
            if u != v and L[u] != C:
                e_to[L[u]] = e_to.get(L[u], 0) + w
        best, bestS = None, None
        for D in sorted(e_to):  # ties: the smaller label
            S = m2 * (e_to[D] - eC) - k[v] * (a[D] - a[C] + k[v])
            if best is None or S > bestS:
                best, bestS = D, S
        X[v] = [
            math.log1p(len(R[v])),
            math.log1p(k[v]),
            math.log1p(len(ins_sinks[v])),
            math.log1p(len(del_sinks[v])),
            min(wins[v] / k[v], 1.0),
            eC / k[v],
            (e_to[best] / k[v]) if best is not None else 0.0,
            (bestS / (k[v] * m2)) if best is not None else 0.0,
            a[C] / m2,
            (a[best] / m2) if best is not None else 0.0,
            math.log1p(size[C]),
            1.0 if rds[v] else 0.0,
        ]
    return X


def test_features_match_their_definitions(orc):
    rng = np.random.default_rng(51)
    checked = 0
    for trial in range(25):
        n = int(rng.integers(8, 40))
        E_prev = {}
        for _ in range(int(rng.integers(n, 4 * n))):
            u, v = rng.integers(0, n, 2)
            if u != v:
                E_prev[key(int(u), int(v))] = int(rng.integers(1, 4))
        edges_prev = [(u, v, w) for (u, v), w in E_prev.items()]
        g_prev = orc.Graph.from_edges(n, edges_prev)
        L = rng.integers(0, max(1, n // 4), n).astype(np.int32)
        # inserts: new pairs, existing pairs and repeats; deletes: present and absent
        ins = []
        for _ in range(int(rng.integers(1, n))):
            u, v = rng.integers(0, n, 2)
            if u != v:
                ins.append((int(u), int(v), int(rng.integers(1, 3))))
        present = list(E_prev)
        dels = [present[i] for i in rng.choice(len(present), min(len(present), 3), replace=False)] if present else []
        dels += [(int(u), int(v)) for u, v in rng.integers(0, n, (2, 2)) if u != v]
        ins_a = np.array(ins, np.int32).reshape(-1, 3)
        dels_a = np.array(dels, np.int32).reshape(-1, 2)
        g_t, err = g_prev.apply(ins_a, dels_a)
        assert err == 0
        rds = (rng.random(n) < 0.3).astype(np.uint8)
        pool, Xo = orc.screen_features(g_prev, g_t, L, ins_a, dels_a, rds)
        E_t = apply_dict(E_prev, ins, dels)
        X = features(n, E_prev, E_t, [int(x) for x in L], ins, dels, rds)
        assert set(np.nonzero(pool)[0].tolist()) == set(X)
        for v, row in X.items():
            np.testing.assert_allclose(Xo[v], np.array(row), rtol=2e-6, atol=1e-7)
            checked += 1
    assert checked > 200
