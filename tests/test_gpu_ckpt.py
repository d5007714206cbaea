"""Checkpoint / resume on the GPU: a context saved mid-stream and loaded again
continues exactly as the saved one (labels, modularity, R_t and the step
statistics, bit for bit) and as the oracle; damaged files are refused; the
learned screen's network survives a save / load with identical outputs."""
import struct

import numpy as np
import pytest

from test_gpu_parity import assert_step_equal, dcd  # noqa: F401  (fixture + helper)

pytestmark = pytest.mark.gpu


def fnv_words(data: bytes) -> int:
    h = 1469598103934665603
    for (x,) in struct.iter_unpack("<Q", data):
        h = ((h ^ x) * 1099511628211) & ((1 << 64) - 1)
    return h


def lfr_small(synth):
    return synth.lfr(synth.seed_for(1, 11), n=20_000, n_events=400_000, steps=6, kmin=4, kmax=2000,
                     smin=20, smax=2000)


def test_resume_mid_stream_is_bit_identical(dcd, orc, synth, tmp_path):
    s = lfr_small(synth)
    a = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    ref = orc.Context(s.n)
    cut = 3
    for ins, dels in s.steps[:cut]:
        a.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        a.update()
        ref.update(orc.DELTA)
    a.set_bins([dcd.LM_SEG32, dcd.LM_WARP256, dcd.LM_CTA4K, dcd.LM_HUB], [32, 256, 4096, -1])
    path = tmp_path / "mid.ckpt"
    a.save(path)
    g_a, lab_a, r_a = a.graph(), a.labels(), a.rset()

    b = dcd.Context.load(path)
    assert (b.n, b.t) == (s.n, cut)
    assert b.bins() == a.bins()
    for x, y in zip(b.graph(), g_a):
        assert np.array_equal(x, y)
    assert np.array_equal(b.labels(), lab_a) and np.array_equal(b.rset(), r_a)

    for ins, dels in s.steps[cut:]:
        for c in (a, b):
            c.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        la, qa, sa = a.update()
        lb, qb, sb = b.update()
        rl, rq, rs = ref.update(orc.DELTA)
        assert_step_equal(sb, sa, lb, la, qb, qa, b.rset(), a.rset())
        assert qb == qa and sb.t == sa.t
        assert_step_equal(sb, rs, lb, rl, qb, rq, b.rset(), ref.rset())
    a.close()
    b.close()


def test_save_before_the_first_update_resumes_statically(dcd, orc, synth, tmp_path):
    s = synth.sbm_10k(n=3000, blocks=15, steps=2)
    a = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    a.save(tmp_path / "t0.ckpt")
    b = dcd.Context.load(tmp_path / "t0.ckpt")
    assert b.t == 0
    ref = orc.Context(s.n)
    for ins, dels in s.steps:
        b.apply_batch(ins, dels)
        ref.apply_batch(ins, dels)
        lab, q, st = b.update()
        rlab, rq, rst = ref.update(orc.DELTA)
        assert_step_equal(st, rst, lab, rlab, q, rq, b.rset(), ref.rset())
    a.close()
    b.close()


def test_save_refuses_a_staged_batch(dcd, synth, tmp_path):
    s = synth.sbm_10k(n=2000, blocks=10, steps=2)
    c = dcd.Context(s.n)
    c.apply_batch(*s.steps[0])
    with pytest.raises(dcd.DcdError) as e:
        c.save(tmp_path / "staged.ckpt")
    assert e.value.code == dcd.DCD_ESTATE
    assert not (tmp_path / "staged.ckpt").exists()
    c.update()
    c.save(tmp_path / "staged.ckpt")
    assert (tmp_path / "staged.ckpt").exists() and not (tmp_path / "staged.ckpt.tmp").exists()
    c.close()


def sections(n, nnz):
    """(offset, size) of the padded sections of a checkpoint with R_t."""
    pad = lambda b: (b + 7) // 8 * 8  # noqa: E731
    off, out = 256, {}
    for name, size in (("rp", 8 * (n + 1)), ("col", 4 * nnz), ("w", 4 * nnz), ("labels", 4 * n), ("rset", n)):
        out[name] = (off, size)
        off += pad(size)
    out["sum"] = (off, 8)
    return out


@pytest.mark.parametrize("damage", ["flip", "truncate", "trailing", "col_range", "self_loop", "col_order",
                                    "weight", "label", "rp_end", "rset_byte"])
def test_damaged_checkpoint_is_refused(dcd, synth, tmp_path, damage):
    s = synth.sbm_10k(n=2000, blocks=10, steps=2)
    c = dcd.Context(s.n)
    for st in s.steps:
        c.apply_batch(*st)
        c.update()
    good = tmp_path / "good.ckpt"
    c.save(good)
    nnz = len(c.graph()[1])
    c.close()
    data = bytearray(good.read_bytes())
    sec = sections(s.n, nnz)
    assert len(data) == sec["sum"][0] + 8
    col0, w0, rp0, lab0, r0 = sec["col"][0], sec["w"][0], sec["rp"][0], sec["labels"][0], sec["rset"][0]
    row0 = struct.unpack_from("<q", data, rp0 + 8)[0]  # entries of row 0
    assert row0 >= 2
    refix = True
    if damage == "flip":
        data[col0 + 4 * (nnz // 2)] ^= 0x40
        refix = False  # the checksum catches it
    elif damage == "truncate":
        data = data[:-20]
        refix = False
    elif damage == "trailing":
        data += b"\0"
        refix = False
    elif damage == "col_range":
        struct.pack_into("<i", data, col0, s.n)
    elif damage == "self_loop":
        struct.pack_into("<i", data, col0, 0)  # row 0's first entry pointing at vertex 0
    elif damage == "col_order":
        a, b = struct.unpack_from("<ii", data, col0)
        struct.pack_into("<ii", data, col0, b, a)
    elif damage == "weight":
        struct.pack_into("<i", data, w0 + 4, 0)
    elif damage == "label":
        struct.pack_into("<i", data, lab0 + 8, -1)
    elif damage == "rp_end":
        struct.pack_into("<q", data, rp0 + 8 * s.n, nnz - 2)
    elif damage == "rset_byte":
        data[r0 + 5] = 2
    if refix:  # a valid checksum, so only the entry checks can refuse it
        struct.pack_into("<Q", data, sec["sum"][0], fnv_words(bytes(data[:sec["sum"][0]])))
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(data))
    with pytest.raises(dcd.DcdError) as e:
        dcd.Context.load(bad)
    assert e.value.code == dcd.DCD_EINVAL
    # the good file still loads
    dcd.Context.load(good).close()


def test_learned_mode_needs_the_network_again(dcd, synth, tmp_path):
    s = synth.sbm_10k(n=2000, blocks=10, steps=3)
    c = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    c.apply_batch(*s.steps[0])
    c.update()
    c.set_mode(dcd.MODE_LEARNED)
    c.save(tmp_path / "l.ckpt")
    b = dcd.Context.load(tmp_path / "l.ckpt")
    b.apply_batch(*s.steps[1])
    with pytest.raises(dcd.DcdError) as e:
        b.update()
    assert e.value.code == dcd.DCD_ESTATE
    # the failed attempt consumed its batch and left G and C as loaded
    b.set_mode(dcd.MODE_DELTA)
    b.apply_batch(*s.steps[1])
    c.set_mode(dcd.MODE_DELTA)
    c.apply_batch(*s.steps[1])
    la, qa, _ = c.update()
    lb, qb, _ = b.update()
    assert np.array_equal(la, lb) and qa == qb
    c.close()
    b.close()


def test_network_round_trip(dcd, tmp_path):
    import torch

    m = dcd.Mlp(seed=123)
    p = m.params
    p[:] = np.random.default_rng(5).normal(0, 0.3, p.size).astype(np.float32)
    m.params = p
    m.save(tmp_path / "net.mlp")
    m2 = dcd.Mlp.load(tmp_path / "net.mlp")
    assert np.array_equal(m2.params, m.params)
    X = torch.randn(10_000, dcd.MLP_FEATURES, device="cuda")
    p1 = torch.empty(10_000, device="cuda")
    p2 = torch.empty(10_000, device="cuda")
    m.forward(X, 10_000, p1)
    m2.forward(X, 10_000, p2)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
    m.close()
    m2.close()
