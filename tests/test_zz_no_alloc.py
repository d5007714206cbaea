"""The allocation-free modularity entry point.

dcd_modularity_noalloc serves callers that cannot allocate device memory when
they need an answer (memory held by another allocator, or code that must not
call cudaMalloc/cudaFree).  Its scratch is a fixed device array shared by all
calls, so this test calls it twice in a row on the same inputs and checks both
answers against the oracle's Eq. 1 evaluation of the same partition on the
same graph (and against the Q and 2m that dcd_update reported for it).  It
also checks what the entry point exists for: the device's free memory does
not change across its calls, and a call succeeds while the library's next
device allocation is armed to fail.  The file name keeps it last in
collection order.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_modularity_matches_oracle(orc):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1904_08553_gb300 import dcd, synth

    s = synth.sbm_10k(n=5000, blocks=50, steps=3)
    ctx = dcd.Context(s.n)
    g = orc.Graph.empty(s.n)
    for ins, dels in s.steps:
        ctx.apply_batch(ins, dels)
        labels, q_upd, st = ctx.update()
        g, err = g.apply(ins, dels)
        assert err == 0
    rp, col, w = ctx.graph()
    ctx.close()
    q_ref, _, m2_ref = g.modularity(labels)
    dev = torch.device("cuda", 0)
    d_rp = torch.from_numpy(rp).to(dev)
    d_col = torch.from_numpy(col).to(dev)
    d_w = torch.from_numpy(w).to(dev)
    d_lab = torch.from_numpy(labels).to(dev)
    ones = torch.arange(s.n, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    dcd.dcd_modularity_noalloc(s.n, d_rp, d_col, d_w, d_lab)  # first call on the device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(2):  # the shared scratch must not carry state between calls
        q, m2 = dcd.dcd_modularity_noalloc(s.n, d_rp, d_col, d_w, d_lab)
        assert m2 == m2_ref == st.m2
        assert abs(q - q_ref) <= 1e-12 * max(1.0, abs(q_ref)), (q, q_ref)
        assert abs(q - q_upd) <= 1e-12 * max(1.0, abs(q_upd)), (q, q_upd)
    # a second partition (singletons) right after: no stale sums from the first
    q1, _ = dcd.dcd_modularity_noalloc(s.n, d_rp, d_col, d_w, ones)
    q1_ref, _, _ = g.modularity(np.arange(s.n, dtype=np.int32))
    assert abs(q1 - q1_ref) <= 1e-12
    # the library's next device allocation fails: this call makes none
    dcd.dcd_set_fault("alloc:1")
    try:
        q2, _ = dcd.dcd_modularity_noalloc(s.n, d_rp, d_col, d_w, d_lab)
    finally:
        dcd.dcd_set_fault(None)
    assert abs(q2 - q_ref) <= 1e-12 * max(1.0, abs(q_ref))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    # argument checks, all before any device work
    with pytest.raises(dcd.DcdError) as ei:
        dcd.dcd_modularity_noalloc(dcd.NOALLOC_MAX_N + 1, d_rp, d_col, d_w, d_lab)
    assert ei.value.code == dcd.DCD_EINVAL
    for args in ((None, d_col, d_w, d_lab), (d_rp, None, d_w, d_lab), (d_rp, d_col, None, d_lab),
                 (d_rp, d_col, d_w, None)):
        with pytest.raises(dcd.DcdError) as ei:
            dcd.dcd_modularity_noalloc(s.n, *args)
        assert ei.value.code == dcd.DCD_EINVAL
    bad = d_lab.clone()
    bad[3] = s.n + 7
    with pytest.raises(dcd.DcdError) as ei:
        dcd.dcd_modularity_noalloc(s.n, d_rp, d_col, d_w, bad)
    assert ei.value.code == dcd.DCD_EINVAL
