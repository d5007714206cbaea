"""dSLM-Delta-s on the GPU (the paper's second host method, Sec. III-D): the
smart-local-moving run through the C ABI against the oracle's restatement
(oracle/dcd_oracle.c, orc_slm), bit for bit: labels, R_t, N and 2m, levels,
passes of the main local moving and of the refinements, and moves, at every
step of SBM, LFR and R-MAT streams in Delta-screening, base and static
modes, on the 64-bit and the 128-bit gain paths."""
import numpy as np
import pytest

from test_gpu_parity import QTOL, dcd  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def run_slm(dcd, orc, stream, mode, omode, steps=None):
    ctx = dcd.Context(stream.n, mode=mode, alg=dcd.ALG_SLM)
    ref = orc.Context(stream.n)
    for ins, dels in stream.steps[:steps]:
        ctx.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = ctx.update()
        rlab, rq, rst = ref.update(omode, alg=orc.SLM)
        assert np.array_equal(lab, rlab), f"labels differ at {np.nonzero(lab != rlab)[0][:10]}"
        assert abs(q - rq) <= QTOL * max(1.0, abs(rq)), (q, rq)
        assert st.N == rst.N and st.m2 == rst.m2
        assert st.r_size == rst.r_size
        assert st.communities == rst.communities
        assert st.levels == rst.levels
        assert st.iters_total == rst.iters_total and st.iters_level0 == rst.iters_level0
        assert st.moves_total == rst.moves_total
        assert st.edges_scanned == rst.edges_scanned
        assert st.refine_iters == rst.refine_iters and st.refine_moves == rst.refine_moves
        assert np.array_equal(ctx.rset(), ref.rset())
    ctx.close()
    return st


@pytest.mark.parametrize("mode", ["delta", "base", "static"])
def test_slm_sbm_stream(dcd, orc, synth, mode):
    s = synth.sbm_10k(n=3000, blocks=30, steps=4)
    m = {"delta": (dcd.MODE_DELTA, orc.DELTA), "base": (dcd.MODE_BASE, orc.BASE),
         "static": (dcd.MODE_STATIC, orc.STATIC)}[mode]
    run_slm(dcd, orc, s, *m)


def test_slm_lfr_with_long_rows(dcd, orc, synth):
    # degrees up to 2000: rows above 256 entries take the CTA kernel
    s = synth.lfr(synth.seed_for(1, 8), n=8_000, n_events=160_000, steps=4, kmin=4, kmax=2000, smin=20, smax=800)
    st = run_slm(dcd, orc, s, dcd.MODE_DELTA, orc.DELTA)
    assert st.refine_iters > 0


def test_slm_rmat(dcd, orc, synth):
    s = synth.rmat(synth.seed_for(2, 8), scale=11, edge_factor=8, steps=3, ins_frac=0.02, del_frac=0.01)
    run_slm(dcd, orc, s, dcd.MODE_DELTA, orc.DELTA)


def test_slm_wide_gain_path(dcd, orc, synth):
    # weights near 2^20 push 2m above 2^31: the 128-bit gain path
    s = synth.sbm_10k(n=1500, blocks=15, steps=3)
    rng = np.random.default_rng(23)
    steps = []
    for ins, dels in s.steps:
        ins = ins.copy()
        ins[:, 2] = rng.integers(1 << 19, 1 << 20, len(ins))
        steps.append((ins, dels))

    class S:
        pass

    w = S()
    w.n, w.steps = s.n, steps
    st = run_slm(dcd, orc, w, dcd.MODE_DELTA, orc.DELTA)
    assert st.m2 >= (1 << 31)


def test_slm_refuses_training_data_collection(dcd):
    # the learned screen's move labels are defined on Louvain's level 0
    ctx = dcd.Context(100, mode=dcd.MODE_DELTA, alg=dcd.ALG_SLM)
    ctx.set_collect(True)
    ctx.apply_batch(np.array([[0, 1, 1], [1, 2, 1]], np.int32))
    ctx.update()  # step 1 is static (no collection)
    ctx.apply_batch(np.array([[2, 3, 1]], np.int32))
    with pytest.raises(dcd.DcdError) as ei:
        ctx.update()
    assert ei.value.code == dcd.DCD_ESTATE
    ctx.set_collect(False)
    ctx.apply_batch(np.array([[2, 3, 1]], np.int32))  # a failed update consumes its batch
    lab, q, st = ctx.update()
    assert st.t == 2 and lab[3] == lab[2]
    ctx.close()
