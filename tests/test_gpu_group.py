"""The batched form: independent graphs advanced together in one context give,
graph by graph, exactly the oracle's results (labels, Q, pass and level
counts, |R_t|)."""
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


@pytest.mark.parametrize("mode", ["delta", "base"])
def test_group_matches_oracle_graph_by_graph(dcd, orc, synth, mode):
    streams = synth.batched_sbm(replica=5, G=10, steps=4, nmax=6000)
    sizes = [s.n for s in streams]
    dm, om = {"delta": (dcd.MODE_DELTA, orc.DELTA), "base": (dcd.MODE_BASE, orc.BASE)}[mode]
    grp = dcd.Group(sizes, mode=dm)
    refs = [orc.Context(n) for n in sizes]
    off = grp.offsets
    for t in range(4):
        for g, s in enumerate(streams):
            ins, dels = s.steps[t]
            grp.apply_batch(g, ins, dels)
            refs[g].apply_batch(ins, dels)
        lab, q, st = grp.update()
        for g, ref in enumerate(refs):
            rl, rq, rst = ref.update(om)
            assert np.array_equal(lab[off[g]:off[g + 1]], rl), (t, g)
            assert abs(q[g] - rq) <= 1e-12 * max(1.0, abs(rq))
            assert st[g].N == rst.N and st[g].m2 == rst.m2
            assert st[g].levels == rst.levels
            assert st[g].iters_total == rst.iters_total
            assert st[g].iters_level0 == rst.iters_level0
            assert st[g].moves_total == rst.moves_total
            assert st[g].communities == rst.communities
            assert st[g].r_size == rst.r_size
            assert st[g].nnz == rst.nnz
    grp.close()


def test_group_with_an_empty_graph_and_bad_ids(dcd, orc):
    grp = dcd.Group([5, 300, 7])
    with pytest.raises(dcd.DcdError):
        grp.apply_batch(0, np.array([[0, 5, 1]], np.int32))
    with pytest.raises(dcd.DcdError):
        grp.apply_batch(3, np.array([[0, 1, 1]], np.int32))
    rng = np.random.default_rng(3)
    e = rng.integers(0, 300, (2000, 2))
    e = e[e[:, 0] != e[:, 1]]
    ins = np.concatenate([e, np.ones((len(e), 1), np.int64)], 1).astype(np.int32)
    grp.apply_batch(1, ins)
    grp.apply_batch(2, np.array([[0, 1, 3], [1, 2, 3], [0, 2, 3]], np.int32))
    lab, q, st = grp.update()
    ref = orc.Context(300)
    ref.apply_batch(ins)
    rl, rq, _ = ref.update(orc.DELTA)
    assert np.array_equal(lab[5:305], rl) and abs(q[1] - rq) <= 1e-12
    assert lab[:5].tolist() == list(range(5)) and q[0] == 0.0
    assert lab[305:].tolist() == [0, 0, 0, 3, 4, 5, 6]
