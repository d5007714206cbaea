"""Level-0 delta coarsening.  R_t only changes level 0 (Sec. III-D), so the
coarse graph of G_t under the level-0 labels is built from the previous
update's coarse graph (G_{t-1} under C_{t-1}), the batch's weight changes and
the rows of the vertices that level 0 moved, instead of from every entry of
G_t.  Each step must equal, bit for bit, both the same context with the
rebuild forced (coarsen_full) and the oracle; and the delta path must be the
one taken wherever its conditions hold."""
import numpy as np
import pytest

from test_gpu_parity import assert_step_equal, dcd  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def step_all(a, b, ref, omode, ins, dels):
    for x in (a, b, ref):
        x.apply_batch(ins, dels)
    la, qa, sa = a.update()
    lb, qb, sb = b.update()
    rl, rq, rs = ref.update(omode)
    assert_step_equal(sa, rs, la, rl, qa, rq, a.rset(), ref.rset())
    assert_step_equal(sb, rs, lb, rl, qb, rq, b.rset(), ref.rset())
    assert sb.coarse0_delta == 0
    return sa


def run(dcd, orc, stream, mode, omode, hook=None):
    a = dcd.Context(stream.n, mode=mode)
    b = dcd.Context(stream.n, mode=mode, coarsen_full=True)
    ref = orc.Context(stream.n)
    used, entries, nnz = [], [], []
    for t, (ins, dels) in enumerate(stream.steps):
        if hook:
            a = hook(t, a, b, ref)
        st = step_all(a, b, ref, omode, ins, dels)
        used.append(int(st.coarse0_delta))
        entries.append(int(st.coarse0_entries))
        nnz.append(int(st.nnz))
    a.close()
    b.close()
    return used, entries, nnz


@pytest.mark.parametrize("mode", ["delta", "base"])
def test_sbm_delta_coarsening_matches(dcd, orc, synth, mode):
    s = synth.sbm_10k(steps=8)
    m = {"delta": (dcd.MODE_DELTA, orc.DELTA), "base": (dcd.MODE_BASE, orc.BASE)}[mode]
    used, entries, nnz = run(dcd, orc, s, *m)
    # the first update starts from singletons; every later one takes the delta path
    assert used[0] == 0 and all(used[1:]), used
    assert all(e < z for e, z, u in zip(entries, nnz, used) if u), (entries, nnz)


def test_lfr_delta_coarsening_matches(dcd, orc, synth):
    s = synth.lfr(synth.seed_for(1, 9), n=30_000, n_events=600_000, steps=6, kmin=6, kmax=3000,
                  smin=30, smax=3000)
    used, _, _ = run(dcd, orc, s, dcd.MODE_DELTA, orc.DELTA)
    # step 1 leaves more than 4096 level-0 communities (no kept matrix for
    # step 2); from then on level 0 starts from C_{t-1}'s few communities
    assert used[:2] == [0, 0] and all(used[2:]), used


def test_rmat_delta_coarsening_matches(dcd, orc, synth):
    # deletions of existing edges: negative weight changes in the kept cells
    s = synth.rmat(synth.seed_for(2, 9), scale=12, edge_factor=8, steps=6, ins_frac=0.02, del_frac=0.05)
    used, _, _ = run(dcd, orc, s, dcd.MODE_DELTA, orc.DELTA)
    assert sum(used[1:]) >= 1, used


def test_set_labels_and_checkpoint_restart_the_rule(dcd, orc, synth, tmp_path):
    s = synth.sbm_10k(n=3000, blocks=30, steps=7)
    rng = np.random.default_rng(5)

    def hook(t, a, b, ref):
        if t == 3:  # replaced labels: the kept coarse graph no longer applies
            new = rng.integers(0, 60, s.n).astype(np.int32)
            for x in (a, b, ref):
                x.set_labels(new)
        if t == 5:  # a resumed context has no kept coarse graph
            p = tmp_path / "c.ckpt"
            a.save(p)
            a.close()
            a = dcd.Context.load(p)
        return a

    used, _, _ = run(dcd, orc, s, dcd.MODE_DELTA, orc.DELTA, hook)
    assert used == [0, 1, 1, 0, 1, 0, 1], used
