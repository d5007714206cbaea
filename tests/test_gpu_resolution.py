"""The temporal-resolution sweep (Sec. IV-C) on the GPU: one insert-only
stream rebinned into k steps for several k, each binning run with
dLouvain-base and dLouvain-Delta-s through the C ABI, against the oracle run
on the same binnings.  Every step's labels, |R_t| and Q must agree (labels bit
for bit, Q within 1e-12), and so must the sweep's rows (mean Q, mean |R_t| / n)
that bench.py --workload resolution reports."""
import numpy as np
import pytest

from test_gpu_parity import dcd  # noqa: F401  (fixture)
from test_resolution_sweep import OracleCtx, fine_stream

pytestmark = pytest.mark.gpu

KS = (1, 2, 4, 7, 14, 28)


def test_sweep_matches_oracle(dcd, orc, synth):
    import bench

    fine = fine_stream(synth, n=4000, events=60_000)
    seen = {"gpu": [], "oracle": []}

    class GpuCtx:
        def __init__(self, n, mode):
            self.c = dcd.Context(n, mode={"base": dcd.MODE_BASE, "delta": dcd.MODE_DELTA}[mode])
            self.log = []
            seen["gpu"].append(self.log)

        def step(self, ins, dels):
            self.c.apply_batch(ins, dels)
            lab, q, st = self.c.update()
            self.log.append((lab, q, st.r_size))
            return q, st.ms_total, st.r_size

        def close(self):
            self.c.close()

    class OrcCtx(OracleCtx):
        def __init__(self, n, mode):
            super().__init__(orc, n, mode)
            self.log = []
            seen["oracle"].append(self.log)

        def step(self, ins, dels):
            self.c.apply_batch(ins, dels)
            lab, q, st = self.c.update(self.mode)
            self.log.append((lab, q, st.r_size))
            return q, 0.0, st.r_size

    rows_g = bench.resolution_sweep(GpuCtx, fine, KS, ("base", "delta"))
    rows_o = bench.resolution_sweep(OrcCtx, fine, KS, ("base", "delta"))
    assert len(seen["gpu"]) == len(seen["oracle"]) == 2 * len(KS)
    for lg, lo in zip(seen["gpu"], seen["oracle"]):
        assert len(lg) == len(lo)
        for (lab, q, r), (rlab, rq, rr) in zip(lg, lo):
            assert np.array_equal(lab, rlab)
            assert abs(q - rq) <= 1e-12 * max(1.0, abs(rq))
            assert r == rr
    for rg, ro in zip(rows_g, rows_o):
        assert (rg["steps"], rg["mode"]) == (ro["steps"], ro["mode"])
        assert abs(rg["mean_q"] - ro["mean_q"]) <= 1e-12
        assert rg["mean_r_fraction"] == ro["mean_r_fraction"]
    # Delta-screening re-evaluates fewer vertices than the base method at some
    # resolution of this stream (the point of the sweep)
    by = {(r["steps"], r["mode"]): r for r in rows_g}
    assert any(by[(k, "delta")]["mean_r_fraction"] < by[(k, "base")]["mean_r_fraction"] for k in KS if k > 1)
