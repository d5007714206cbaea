"""The allocation-free modularity entry point against the library's own update.

dcd_modularity_noalloc serves callers that cannot allocate device memory when
they need an answer (memory held by another allocator, or code that must not
call cudaMalloc/cudaFree).  Its scratch is a fixed device array shared by all
calls, so this test calls it twice in a row on the same inputs and checks both
answers against the Q and 2m that dcd_update reported for the same labels.
The file name keeps it last in collection order.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_modularity_matches_update():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1904_08553_gb300 import dcd, synth

    s = synth.sbm_10k(n=5000, blocks=50, steps=3)
    ctx = dcd.Context(s.n)
    for ins, dels in s.steps:
        ctx.apply_batch(ins, dels)
        labels, q_ref, st = ctx.update()
    rp, col, w = ctx.graph()
    ctx.close()
    dev = torch.device("cuda", 0)
    d_rp = torch.from_numpy(rp).to(dev)
    d_col = torch.from_numpy(col).to(dev)
    d_w = torch.from_numpy(w).to(dev)
    d_lab = torch.from_numpy(labels).to(dev)
    torch.cuda.synchronize()
    for _ in range(2):  # the shared scratch must not carry state between calls
        q, m2 = dcd.dcd_modularity_noalloc(s.n, d_rp, d_col, d_w, d_lab)
        assert m2 == st.m2
        assert abs(q - q_ref) <= 1e-12 * max(1.0, abs(q_ref)), (q, q_ref)
    # a second partition (singletons) right after: no stale sums from the first
    q1, _ = dcd.dcd_modularity_noalloc(s.n, d_rp, d_col, d_w, torch.arange(s.n, dtype=torch.int32, device=dev))
    k = np.diff(rp) * 0
    for u in range(s.n):
        k[u] = w[rp[u]:rp[u + 1]].sum()
    expect = -float((k.astype(np.float64) ** 2).sum()) / float(st.m2) ** 2
    assert abs(q1 - expect) <= 1e-12
    with pytest.raises(dcd.DcdError) as ei:
        dcd.dcd_modularity_noalloc(dcd.NOALLOC_MAX_N + 1, d_rp, d_col, d_w, d_lab)
    assert ei.value.code == dcd.DCD_EINVAL
    bad = d_lab.clone()
    bad[3] = s.n + 7
    with pytest.raises(dcd.DcdError) as ei:
        dcd.dcd_modularity_noalloc(s.n, d_rp, d_col, d_w, bad)
    assert ei.value.code == dcd.DCD_EINVAL
