"""Error paths under host-side fault injection: every device allocation and
every checked CUDA call of a step is made to fail in turn (the call is not
made; no GPU is faulted).  Each failed call must leave the context exactly as
it was -- G_t, C_t, R_t, t -- and once the injector is disarmed the stream must
continue exactly as a context that never failed, and as the oracle."""
import numpy as np
import pytest

from test_gpu_parity import assert_step_equal, dcd  # noqa: F401  (fixture + helper)

pytestmark = pytest.mark.gpu

CAP = 5000  # more checked calls than one small step makes


@pytest.fixture(autouse=True)
def disarm(dcd):
    dcd.dcd_set_fault(None)
    yield
    dcd.dcd_set_fault(None)


def snapshot(c):
    n, t, mode = dcd_state(c)
    rp, col, w = c.graph()
    return dict(t=t, mode=mode, rp=rp, col=col, w=w, labels=c.labels(), rset=c.rset(), bins=c.bins())


def dcd_state(c):
    from paper_1904_08553_gb300 import dcd as m

    return m.dcd_get_state(c._h)


def assert_same_state(a, b):
    assert a.keys() == b.keys()
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(a[k], b[k]), k
        else:
            assert a[k] == b[k], k


def sweep_update(dcd, c, batch, kind):
    """Fail the N-th event of `kind` in one update, for N = 1, 2, ... until the
    update completes without reaching it.  Returns (failures seen, result)."""
    before = snapshot(c)
    for N in range(1, CAP):
        c.apply_batch(*batch)
        dcd.dcd_set_fault(f"{kind}:{N}")
        try:
            res = c.update()
        except dcd.DcdError as e:
            dcd.dcd_set_fault(None)
            assert e.code == (dcd.DCD_ENOMEM if kind == "alloc" else dcd.DCD_ECUDA), (N, e)
            assert_same_state(snapshot(c), before)
            continue
        dcd.dcd_set_fault(None)
        return N - 1, res
    raise AssertionError(f"{kind}: more than {CAP} events in one update")


@pytest.mark.parametrize("kind", ["cuda", "alloc"])
def test_every_failure_point_of_an_update_rolls_back(dcd, orc, synth, kind):
    s = synth.lfr(synth.seed_for(1, 12), n=3000, n_events=40_000, steps=4, kmin=4, kmax=400, smin=20, smax=400)
    c = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    ref = orc.Context(s.n)
    for t, batch in enumerate(s.steps):
        ref.apply_batch(*batch)
        rlab, rq, rst = ref.update(orc.DELTA)
        if t in (0, 2):  # the static first step and a Delta-screening step
            fails, (lab, q, st) = sweep_update(dcd, c, batch, kind)
            assert fails > (10 if kind == "alloc" else 50)
        else:
            c.apply_batch(*batch)
            lab, q, st = c.update()
        assert_step_equal(st, rst, lab, rlab, q, rq, c.rset(), ref.rset())
    c.close()


def test_failed_apply_batch_stages_nothing(dcd, orc, synth):
    s = synth.sbm_10k(n=2000, blocks=10, steps=3)
    c = dcd.Context(s.n, mode=dcd.MODE_DELTA)
    ref = orc.Context(s.n)
    for batch in s.steps:
        for N in range(1, CAP):
            dcd.dcd_set_fault(f"cuda:{N}")
            try:
                c.apply_batch(*batch)
            except dcd.DcdError as e:
                assert e.code == dcd.DCD_ECUDA
                continue
            finally:
                dcd.dcd_set_fault(None)
            break
        # the successful call is the only one staged
        ref.apply_batch(*batch)
        lab, q, st = c.update()
        rlab, rq, rst = ref.update(orc.DELTA)
        assert_step_equal(st, rst, lab, rlab, q, rq, c.rset(), ref.rset())
    c.close()


def test_group_update_rolls_back(dcd, orc, synth):
    streams = [synth.sbm_10k(replica=r, n=800 + 400 * r, blocks=6 + r, steps=3) for r in range(3)]
    grp = dcd.Group([s.n for s in streams], mode=dcd.MODE_DELTA)
    refs = [orc.Context(s.n) for s in streams]
    o = grp.offsets
    for t in range(3):
        for g, s in enumerate(streams):
            refs[g].apply_batch(*s.steps[t])
        expect = [refs[g].update(orc.DELTA) for g in range(3)]
        for N in range(1, CAP, 7 if t else 1):
            for g, s in enumerate(streams):
                grp.apply_batch(g, *s.steps[t])
            dcd.dcd_set_fault(f"cuda:{N}")
            try:
                lab, q, _ = grp.update()
            except dcd.DcdError as e:
                assert e.code == dcd.DCD_ECUDA
                continue
            finally:
                dcd.dcd_set_fault(None)
            break
        for g in range(3):
            rlab, rq, _ = expect[g]
            assert np.array_equal(lab[o[g]:o[g + 1]], rlab) and abs(q[g] - rq) <= 1e-12 * max(1.0, abs(rq))
    grp.close()


def test_failed_save_keeps_the_old_file(dcd, synth, tmp_path):
    s = synth.sbm_10k(n=2000, blocks=10, steps=3)
    c = dcd.Context(s.n)
    c.apply_batch(*s.steps[0])
    c.update()
    path = tmp_path / "c.ckpt"
    c.save(path)
    old = path.read_bytes()
    c.apply_batch(*s.steps[1])
    c.update()
    failures = 0
    for N in range(1, CAP):
        dcd.dcd_set_fault(f"cuda:{N}")
        try:
            c.save(path)
        except dcd.DcdError as e:
            assert e.code == dcd.DCD_ECUDA
            failures += 1
            assert path.read_bytes() == old and not (tmp_path / "c.ckpt.tmp").exists()
            continue
        finally:
            dcd.dcd_set_fault(None)
        break
    assert failures >= 3
    assert path.read_bytes() != old
    b = dcd.Context.load(path)
    assert np.array_equal(b.labels(), c.labels())
    for N in range(1, 40):  # a failed load creates nothing and reports the failure
        dcd.dcd_set_fault(f"alloc:{N}")
        try:
            dcd.Context.load(path).close()
        except dcd.DcdError as e:
            assert e.code in (dcd.DCD_ENOMEM, dcd.DCD_ECUDA)
        finally:
            dcd.dcd_set_fault(None)
    b.close()
    c.close()
