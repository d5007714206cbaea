"""The temporal-resolution sweep (Sec. IV-C) on the CPU: rebinning keeps the
insert-only stream's events, in order, in k non-empty consecutive steps, and
the sweep core runs every binning and mode (here through the oracle; bench.py
runs it through the library with --workload resolution)."""
import time

import numpy as np
import pytest


def fine_stream(synth, n=2000, events=24_000):
    return synth.lfr(synth.seed_for(5, 9), n=n, n_events=events, steps=28, kmin=4, kmax=400, smin=20, smax=400,
                     drift=0.0, del_frac=0.0)


def test_rebin_keeps_the_stream(synth):
    fine = fine_stream(synth)
    assert all(len(d) == 0 for _, d in fine.steps)
    seq = np.concatenate([i for i, _ in fine.steps])
    for k in (1, 2, 3, 5, 7, 12, 28):
        s = synth.rebin(fine, k)
        assert len(s.steps) == k and all(len(i) > 0 and len(d) == 0 for i, d in s.steps)
        assert np.array_equal(np.concatenate([i for i, _ in s.steps]), seq)
    for bad in (0, 29):
        with pytest.raises(ValueError):
            synth.rebin(fine, bad)
    with pytest.raises(ValueError):
        synth.rebin(synth.sbm_10k(n=1000, blocks=10, steps=3), 2)  # has deletes


class OracleCtx:
    def __init__(self, orc, n, mode):
        self.c = orc.Context(n)
        self.mode = {"base": orc.BASE, "delta": orc.DELTA}[mode]

    def step(self, ins, dels):
        self.c.apply_batch(ins, dels)
        t0 = time.perf_counter()
        _, q, st = self.c.update(self.mode)
        return q, (time.perf_counter() - t0) * 1e3, st.r_size

    def close(self):
        pass


def test_sweep_core_runs_every_binning_and_mode(orc, synth):
    import bench

    fine = fine_stream(synth)
    ks = (1, 2, 7, 28)
    rows = bench.resolution_sweep(lambda n, mode: OracleCtx(orc, n, mode), fine, ks, ("base", "delta"))
    assert [(r["steps"], r["mode"]) for r in rows] == [(k, m) for k in ks for m in ("base", "delta")]
    by = {(r["steps"], r["mode"]): r for r in rows}
    for k in ks:
        b, d = by[(k, "base")], by[(k, "delta")]
        assert b["mean_r_fraction"] == 1.0  # dLouvain-base evaluates every vertex
        assert 0.0 < d["mean_r_fraction"] <= 1.0
        assert 0.0 < b["mean_q"] < 1.0 and 0.0 < d["mean_q"] < 1.0
    # one step is the static run in both modes
    assert by[(1, "base")]["mean_q"] == by[(1, "delta")]["mean_q"]
    assert by[(1, "delta")]["mean_r_fraction"] == 1.0
