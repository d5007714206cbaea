"""The oracle's context copy (timing infrastructure of the CPU baseline): a
copy taken between steps, and one taken with a batch staged, continue the
stream exactly as the original does."""
import numpy as np


def test_clone_continues_like_the_original(orc, synth):
    s = synth.sbm_10k(n=1500, blocks=15, steps=4)
    a = orc.Context(s.n)
    for ins, dels in s.steps[:2]:
        a.apply_batch(ins, dels)
        a.update(orc.DELTA)
    b = a.clone()
    ins, dels = s.steps[2]
    a.apply_batch(ins, dels)
    c = a.clone()  # staged batch copied too
    b.apply_batch(ins, dels)
    outs = [x.update(orc.DELTA) for x in (a, b, c)]
    for lab, q, st in outs[1:]:
        assert np.array_equal(lab, outs[0][0])
        assert q == outs[0][1]
        assert st.iters_total == outs[0][2].iters_total and st.r_size == outs[0][2].r_size
    assert np.array_equal(a.rset(), b.rset()) and np.array_equal(a.rset(), c.rset())
    # the copies are independent: advancing one leaves the other as it was
    ins, dels = s.steps[3]
    b.apply_batch(ins, dels)
    lb, _, _ = b.update(orc.DELTA)
    a.apply_batch(ins, dels)
    la, _, _ = a.update(orc.DELTA)
    assert np.array_equal(la, lb)
