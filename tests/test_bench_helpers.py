"""Host-side helpers of bench.py: the timed schedule replays the
configuration's steps after the warm-up, and the level-0 roofline counts only
the rows the local-move kernels read (not the first-pass rows whose proposals
the screening supplied)."""
from types import SimpleNamespace


def test_timed_schedule_replays_the_configuration():
    import bench

    assert bench.timed_schedule(3, 8) == [list(range(4, 12))]
    segs = bench.timed_schedule(5, 20)
    assert sum(len(s) for s in segs) == 20
    assert all(s[0] == 6 and s[-1] <= 11 for s in segs)


def test_level0_bytes_excludes_the_screened_first_pass():
    import bench

    st = SimpleNamespace(edges_level0=1000, verts_level0=100, edges_level0_screen=300, verts_level0_screen=20)
    assert bench.level0_bytes(st) == bench.BYTES_PER_ENTRY * 700 + bench.BYTES_PER_VERTEX * 80


def test_kernel_rows_skip_empty_bins():
    import bench

    rows = bench.kernel_rows([(0, 10, 100, 0.5), (1, 0, 0, 0.0)], peak=1000.0)
    assert len(rows) == 1
    r = rows[0]
    assert r["bytes"] == bench.BYTES_PER_ENTRY * 100 + bench.BYTES_PER_VERTEX * 10
    assert abs(r["gbs"] - r["bytes"] / 0.5e-3 / 1e9) < 1e-9 and abs(r["frac"] - r["gbs"] / 1000.0) < 1e-12
