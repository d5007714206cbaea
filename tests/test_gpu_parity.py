"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer work (the CSR of G_t, R_t, labels, iteration and move counts) must be
bit-exact; modularity within 1e-12 relative (both sides convert the same exact
integers N and m2 to FP64, so in practice it is identical).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

QTOL = 1e-12


@pytest.fixture(scope="module")
def dcd():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1904_08553_gb300 import dcd as m

    return m


def oracle_csr_int32(rp, col, w):
    return rp, col, w.astype(np.int64)


def assert_step_equal(st, rst, lab, rlab, q, rq, rset=None, rrset=None):
    assert np.array_equal(lab, rlab), f"labels differ at {np.nonzero(lab != rlab)[0][:10]}"
    assert abs(q - rq) <= QTOL * max(1.0, abs(rq)), (q, rq)
    assert st.N == rst.N and st.m2 == rst.m2
    assert st.r_size == rst.r_size
    assert st.communities == rst.communities
    assert st.levels == rst.levels
    assert st.iters_total == rst.iters_total
    assert st.iters_level0 == rst.iters_level0
    assert st.moves_total == rst.moves_total
    assert st.edges_scanned == rst.edges_scanned
    if rset is not None:
        assert np.array_equal(rset, rrset)


def run_stream(dcd, orc, stream, mode, omode, check_graph=False, steps=None):
    ctx = dcd.Context(stream.n, mode=mode)
    ref = orc.Context(stream.n)
    for t, (ins, dels) in enumerate(stream.steps[:steps]):
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        rlab, rq, rst = ref.update(omode)
        assert_step_equal(st, rst, lab, rlab, q, rq, ctx.rset(), ref.rset())
        if check_graph:
            rp, col, w = ctx.graph()
            orp, ocol, ow = ref.graph_csr()
            assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(w, ow)
    ctx.close()
    return st


# ---------------------------------------------------------------- CSR merge

def test_csr_merge_matches_oracle(dcd, orc):
    rng = np.random.default_rng(11)
    n = 300
    ctx = dcd.Context(n, mode=dcd.MODE_BASE)
    ref = orc.Context(n)
    edges = set()
    for step in range(12):
        ins = []
        for _ in range(int(rng.integers(0, 400))):
            u, v = (int(x) for x in rng.integers(0, n, 2))
            if u != v:
                ins.append((u, v, int(rng.integers(1, 6))))
        dels = []
        cur = list(edges)
        for _ in range(int(rng.integers(0, 150))):
            if cur and rng.random() < 0.85:
                a, b = cur[int(rng.integers(0, len(cur)))]
                dels.append((b, a) if rng.random() < 0.5 else (a, b))
            else:
                u, v = (int(x) for x in rng.integers(0, n, 2))
                if u != v:
                    dels.append((u, v))
        # the same edge deleted and re-inserted in one step
        if cur:
            a, b = cur[0]
            dels.append((a, b))
            ins.append((b, a, 2))
        for a, b in dels:
            edges.discard((min(a, b), max(a, b)))
        for a, b, w in ins:
            edges.add((min(a, b), max(a, b)))
        ins = np.array(ins, np.int32).reshape(-1, 3)
        dels = np.array(dels, np.int32).reshape(-1, 2)
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        rlab, rq, rst = ref.update(orc.BASE)
        rp, col, w = ctx.graph()
        orp, ocol, ow = ref.graph_csr()
        assert np.array_equal(rp, orp)
        assert np.array_equal(col, ocol)
        assert np.array_equal(w.astype(np.int64), ow)
        assert_step_equal(st, rst, lab, rlab, q, rq)


def test_batches_concatenate_and_device_batches(dcd, orc, synth):
    import torch

    s = synth.sbm_10k(n=1000, blocks=10, steps=3)
    ctx = dcd.Context(s.n)
    ref = orc.Context(s.n)
    for t, (ins, dels) in enumerate(s.steps):
        half = len(ins) // 2
        if t % 2 == 0:
            ctx.apply_batch(ins[:half], dels)
            ctx.apply_batch(ins[half:], None)
        else:
            di = torch.from_numpy(np.ascontiguousarray(ins)).cuda()
            dd = torch.from_numpy(np.concatenate([dels, np.zeros((len(dels), 1), np.int32)], 1)).cuda()
            ctx.apply_batch_device(di, len(ins), dd, len(dels))
        ref.apply_batch(ins, dels)
        out = torch.empty(s.n, dtype=torch.int32, device="cuda")
        _, q, st = ctx.update(labels_out=out)
        rlab, rq, rst = ref.update(orc.DELTA)
        assert_step_equal(st, rst, out.cpu().numpy(), rlab, q, rq, ctx.rset(), ref.rset())


# ---------------------------------------------------------------- full path

@pytest.mark.parametrize("mode", ["delta", "base", "static"])
def test_sbm10k_stream_parity(dcd, orc, synth, mode):
    s = synth.sbm_10k()
    m = {"delta": (dcd.MODE_DELTA, orc.DELTA), "base": (dcd.MODE_BASE, orc.BASE),
         "static": (dcd.MODE_STATIC, orc.STATIC)}[mode]
    run_stream(dcd, orc, s, *m, check_graph=(mode == "delta"))


def test_lfr_small_parity(dcd, orc, synth):
    # degree spread 4..2000 exercises the warp, mid and large bins
    s = synth.lfr(synth.seed_for(1, 7), n=20_000, n_events=400_000, steps=4, kmin=4, kmax=2000,
                  smin=20, smax=2000)
    run_stream(dcd, orc, s, dcd.MODE_DELTA, orc.DELTA)


def test_rmat_small_parity(dcd, orc, synth):
    s = synth.rmat(synth.seed_for(2, 7), scale=12, edge_factor=8, steps=4, ins_frac=0.02, del_frac=0.01)
    run_stream(dcd, orc, s, dcd.MODE_DELTA, orc.DELTA)


def test_hub_vertex_uses_global_table(dcd, orc):
    # one vertex of degree 9000 (> 4096: table in global memory) + ring structure
    rng = np.random.default_rng(12)
    n = 12_000
    hub = 5
    ins = [(hub, v, int(rng.integers(1, 4))) for v in range(n) if v != hub and v % 4 != 1][:9000]
    ins += [(v, (v + 1) % n, 1) for v in range(0, n, 2)]
    ins += [(int(a), int(b), 1) for a, b in rng.integers(0, n, (20_000, 2)) if a != b]
    ins = np.array(ins, np.int32)
    steps = [(ins, np.zeros((0, 2), np.int32))]
    more = np.array([(hub, v, 2) for v in range(1, n, 4) if v != hub][:3000], np.int32)
    steps.append((more, ins[:500, :2].copy()))

    class S:
        pass

    s = S()
    s.n, s.steps = n, steps
    run_stream(dcd, orc, s, dcd.MODE_DELTA, orc.DELTA)


def test_several_hubs_over_steps(dcd, orc):
    # three hubs of 6,000..21,000 entries (rows split over several CTAs) that
    # are screening sources, j* of other sources and local-move vertices, over
    # steps that insert at and delete from them
    rng = np.random.default_rng(31)
    n = 40_000
    hubs = [7, 19_000, 33_333]
    degs = [21_000, 12_000, 6_000]
    ins = []
    for h, d in zip(hubs, degs):
        nb = rng.choice(n, size=d, replace=False)
        ins += [(h, int(v), int(rng.integers(1, 5))) for v in nb if v != h]
    ins += [(int(a), int(b), 1) for a, b in rng.integers(0, n, (60_000, 2)) if a != b]
    ins += [(v, v + 1, 2) for v in range(0, n - 1, 3)]
    ins = np.array(ins, np.int32)
    steps = [(ins, np.zeros((0, 2), np.int32))]
    for t in range(3):
        add = [(hubs[t % 3], int(v), 1) for v in rng.integers(0, n, 2_500) if v != hubs[t % 3]]
        add += [(int(a), int(b), 1) for a, b in rng.integers(0, n, (5_000, 2)) if a != b]
        dels = ins[rng.choice(len(ins), size=1_500, replace=False), :2]
        steps.append((np.array(add, np.int32), dels.copy()))

    class S:
        pass

    s = S()
    s.n, s.steps = n, steps
    run_stream(dcd, orc, s, dcd.MODE_DELTA, orc.DELTA)


def test_wide_gain_path(dcd, orc, synth):
    # weights near 2^20 push 2m above 2^31: the 128-bit gain path
    s = synth.sbm_10k(n=2000, blocks=20, steps=3)
    rng = np.random.default_rng(13)
    steps = []
    for ins, dels in s.steps:
        ins = ins.copy()
        ins[:, 2] = rng.integers(1 << 19, 1 << 20, len(ins))
        steps.append((ins, dels))

    class S:
        pass

    w = S()
    w.n, w.steps = s.n, steps
    st = run_stream(dcd, orc, w, dcd.MODE_DELTA, orc.DELTA)
    assert st.m2 >= (1 << 31)


def test_given_rset_mode(dcd, orc, synth):
    s = synth.sbm_10k(n=2000, blocks=20, steps=3)
    rng = np.random.default_rng(14)
    ctx = dcd.Context(s.n, mode=dcd.MODE_GIVEN_R)
    ref = orc.Context(s.n)
    for t, (ins, dels) in enumerate(s.steps):
        r = (rng.random(s.n) < 0.3).astype(np.uint8)
        ctx.set_rset(r)
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        rlab, rq, rst = ref.update(orc.GIVEN_R if t else orc.STATIC, r if t else None)
        assert_step_equal(st, rst, lab, rlab, q, rq)


# ---------------------------------------------------------------- edge cases

def test_empty_graph_and_empty_steps(dcd, orc):
    ctx = dcd.Context(50)
    ref = orc.Context(50)
    for t in range(3):
        lab, q, st = ctx.update()
        rlab, rq, rst = ref.update(orc.DELTA)
        assert_step_equal(st, rst, lab, rlab, q, rq)
        assert q == 0.0 and np.array_equal(lab, np.arange(50))
    ins = np.array([[1, 2, 1], [2, 3, 1], [1, 3, 1], [10, 11, 4]], np.int32)
    ctx.apply_batch(ins)
    ref.apply_batch(ins)
    lab, q, st = ctx.update()
    rlab, rq, rst = ref.update(orc.DELTA)
    assert_step_equal(st, rst, lab, rlab, q, rq, ctx.rset(), ref.rset())
    # delete everything again
    ctx.apply_batch(None, ins[:, :2])
    ref.apply_batch(None, ins[:, :2])
    lab, q, st = ctx.update()
    rlab, rq, rst = ref.update(orc.DELTA)
    assert_step_equal(st, rst, lab, rlab, q, rq, ctx.rset(), ref.rset())
    assert st.nnz == 0


def test_single_vertex_graph(dcd):
    ctx = dcd.Context(1)
    lab, q, st = ctx.update()
    assert lab.tolist() == [0] and q == 0.0


def test_invalid_batches_leave_state_unchanged(dcd, orc):
    import torch

    ctx = dcd.Context(100)
    ins = np.array([[0, 1, 1], [1, 2, 1], [2, 0, 1]], np.int32)
    ctx.apply_batch(ins)
    lab0, q0, st0 = ctx.update()
    g0 = ctx.graph()
    for bad in ([[3, 3, 1]], [[0, 100, 1]], [[0, 5, 0]], [[-1, 5, 1]]):
        with pytest.raises(dcd.DcdError) as ei:
            ctx.apply_batch(np.array(bad, np.int32))
        assert ei.value.code == dcd.DCD_EINVAL
    # a bad device batch is caught inside dcd_update
    di = torch.tensor([[4, 5, 1], [7, 7, 1]], dtype=torch.int32, device="cuda")
    ctx.apply_batch_device(di, 2, None, 0)
    with pytest.raises(dcd.DcdError) as ei:
        ctx.update()
    assert ei.value.code == dcd.DCD_EINVAL
    g1 = ctx.graph()
    assert all(np.array_equal(a, b) for a, b in zip(g0, g1))
    assert np.array_equal(ctx.labels(), lab0)
    # the next valid step works
    ctx.apply_batch(np.array([[4, 5, 1]], np.int32))
    lab, q, st = ctx.update()
    assert st.t == 2


def test_weight_overflow_is_reported(dcd):
    ctx = dcd.Context(10)
    big = np.array([[0, 1, 2_000_000_000]], np.int32)
    ctx.apply_batch(big)
    ctx.update()
    ctx.apply_batch(big)
    with pytest.raises(dcd.DcdError) as ei:
        ctx.update()
    assert ei.value.code == dcd.DCD_EOVERFLOW
    rp, col, w = ctx.graph()
    assert w.tolist() == [2_000_000_000, 2_000_000_000]


def test_set_labels_mid_stream(dcd, orc, synth):
    # replacing C_t between steps: the next step's level-0 sums start from the
    # new labels (the kept sum of the old ones must not be reused)
    s = synth.sbm_10k(n=2000, blocks=20, steps=5)
    ctx = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    ref = orc.Context(s.n)
    rng = np.random.default_rng(41)
    for t, (ins, dels) in enumerate(s.steps):
        if t in (2, 4):
            new = rng.integers(0, 40, s.n).astype(np.int32)
            ctx.set_labels(new)
            ref.set_labels(new)
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        rlab, rq, rst = ref.update(orc.DELTA)
        assert_step_equal(st, rst, lab, rlab, q, rq, ctx.rset(), ref.rset())
    ctx.close()


def test_host_pass_loop_matches_oracle(dcd, orc, synth):
    """dcd_config.pass_loop = 1: the host enqueues each local-move pass
    instead of one graph launch per level.  The results are the oracle's, and
    equal the device loop's bit for bit, with the same level-0 bin record."""
    s = synth.lfr(synth.seed_for(1, 7), n=20_000, n_events=400_000, steps=4, kmin=4, kmax=2000,
                  smin=20, smax=2000)
    a = dcd.Context(s.n, mode=dcd.MODE_DELTA, pass_loop_host=True)
    b = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    ref = orc.Context(s.n)
    for ins, dels in s.steps:
        for x in (a, b, ref):
            x.apply_batch(ins, dels)
        la, qa, sa = a.update()
        lb, qb, sb = b.update()
        rl, rq, rs = ref.update(orc.DELTA)
        assert_step_equal(sa, rs, la, rl, qa, rq, a.rset(), ref.rset())
        assert np.array_equal(la, lb) and qa == qb
        assert (sa.iters_total, sa.moves_total, sa.levels) == (sb.iters_total, sb.moves_total, sb.levels)
        assert a.level0_bins() == b.level0_bins()
    a.close()
    b.close()


@pytest.mark.parametrize("mode", ["delta", "base"])
def test_first_pass_proposals_from_screening(dcd, orc, synth, mode):
    """A Delta-screening update's first level-0 pass reads the state the
    screening reads (C_{t-1} and its sums on G_t), so the screening hands over
    its proposals for the sources whose rows it sums and the pass skips those
    rows.  The results stay the oracle's, bit for bit; the hand-over covers
    part of one pass in DELTA mode and nothing in BASE mode (no screening) or
    in the static first update."""
    s = synth.lfr(synth.seed_for(1, 7), n=20_000, n_events=400_000, steps=4, kmin=4, kmax=2000,
                  smin=20, smax=2000)
    m, om = {"delta": (dcd.MODE_DELTA, orc.DELTA), "base": (dcd.MODE_BASE, orc.BASE)}[mode]
    ctx = dcd.Context(s.n, mode=m)
    ref = orc.Context(s.n)
    for t, (ins, dels) in enumerate(s.steps):
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        rlab, rq, rst = ref.update(om)
        assert_step_equal(st, rst, lab, rlab, q, rq, ctx.rset(), ref.rset())
        one_pass_v = st.verts_level0 // max(st.iters_level0, 1)
        one_pass_e = st.edges_level0 // max(st.iters_level0, 1)
        if mode == "delta" and t > 0:
            assert 0 < st.verts_level0_screen <= one_pass_v, (st.verts_level0_screen, one_pass_v)
            assert 0 < st.edges_level0_screen <= one_pass_e
        else:
            assert st.verts_level0_screen == 0 and st.edges_level0_screen == 0
    ctx.close()
