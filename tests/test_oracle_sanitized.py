"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a build of
the same C sources with both sanitizers runs every oracle entry point on small
streams in a child process.  Any out-of-bounds access, use after free, signed
overflow, misaligned or invalid shift aborts it with a report."""
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent

SCRIPT = r'''
import numpy as np
import oracle as orc
from paper_1904_08553_gb300 import synth

synth.lib()
s = synth.lfr(synth.seed_for(1, 21), n=3000, n_events=40_000, steps=4, kmin=4, kmax=500, smin=20, smax=500)
for alg in (orc.LOUVAIN, orc.SLM):
    for mode in (orc.STATIC, orc.BASE, orc.DELTA):
        c = orc.Context(s.n)
        for ins, dels in s.steps:
            c.apply_batch(ins, dels)
            lab, q, st = c.update(mode, alg=alg)
            c.rset()
        c.graph_csr()
        c.set_labels(lab)
g_prev = orc.Graph.empty(s.n)
lab = np.arange(s.n, dtype=np.int32)
for ins, dels in s.steps:
    g_t, err = g_prev.apply(ins, dels)
    assert err == 0
    r = orc.screen(g_prev, g_t, lab, ins, dels)
    orc.screen_features(g_prev, g_t, lab, ins, dels, r)
    lab2 = g_t.louvain(lab, r)[0]
    g_t.modularity(lab2)
    g_t.coarsen(lab2)
    g_t.run_level(lab2.copy())
    g_t.local_move_pass(lab2.copy())
    g_t.gain(lab2, 0, int(lab2[1]))
    g_t.slm(lab, r)
    g_t.slm_refine(lab2)
    g_t.slm_level(lab2, r)
    g_prev, lab = g_t, lab2
P = np.random.default_rng(0).normal(0, 0.2, orc.mlp_nparams()).astype(np.float32)
X = np.random.default_rng(1).normal(0, 1, (257, 12)).astype(np.float32)
y = (np.random.default_rng(2).random(257) < 0.3).astype(np.float32)
orc.mlp_forward(P, X, y)
orc.mlp_grad(P, X, y)
orc.mlp_grad_exact(P, X, y)
orc.mlp_loss_exact(P, X, y)
print("sanitized oracle ok")
'''


def runtime(name):
    p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    asan = runtime("libasan.so")
    if asan is None:
        pytest.skip("no AddressSanitizer runtime for this gcc")
    sys.path.insert(0, str(ROOT))
    import oracle

    lib = oracle.build_sanitized(tmp_path / "liboracle_san.so")
    env = dict(os.environ, LD_PRELOAD=asan, DCD_ORACLE_LIB=str(lib),
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", PYTHONPATH=str(ROOT))
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=600,
                       cwd=str(ROOT))
    report = r.stderr[-4000:]
    assert r.returncode == 0, report
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, report
    assert "sanitized oracle ok" in r.stdout


PLANTED = r'''
#include <limits.h>
int oob_read(int i) { int a[4] = {1, 2, 3, 4}; volatile int* p = a; return p[i]; }
int add_one(int x) { return x + 1; }
'''


@pytest.mark.parametrize("call", ["oob_read(4)", "add_one(2147483647)"])
def test_the_harness_catches_a_planted_mistake(tmp_path, call):
    """The same flags, preload and options on a planted out-of-bounds read and
    signed overflow: the child must abort with the sanitizer's report."""
    asan = runtime("libasan.so")
    if asan is None:
        pytest.skip("no AddressSanitizer runtime for this gcc")
    sys.path.insert(0, str(ROOT))
    import oracle

    src = tmp_path / "planted.c"
    src.write_text(PLANTED)
    lib = tmp_path / "libplanted.so"
    subprocess.check_call(["gcc", *oracle.SANITIZE_FLAGS, "-fPIC", "-shared", str(src), "-o", str(lib)])
    script = f"import ctypes; L = ctypes.CDLL({str(lib)!r}); print(L.{call})"
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=120)
    # whichever sanitizer sees it first (UBSan's bounds check or ASan) reports and stops the child
    assert r.returncode != 0, r.stdout
    assert "runtime error" in r.stderr or "AddressSanitizer" in r.stderr, r.stderr[-2000:]
