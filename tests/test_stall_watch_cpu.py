"""The stagnation watch that ends an FP32-mixed stage (stall_step, shared by
the single-cell loops on host and device and by the batched engine's device
and host loop tests), compiled for the host from the same header and driven
with error sequences whose outcome follows from its stated rule: a new low is
the first error or one below 0.99 times the last low; the watch trips once
`window` iterations pass without one, or, when widening, max(window, twice
the longest gap between lows)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2409_10774_gb300", "csrc")


@pytest.fixture(scope="module")
def watch(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    inc = [f"-I{CSRC}"]
    for d in ("/usr/local/cuda/include", os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")):
        if os.path.isdir(d):
            inc.append(f"-I{d}")
    exe = str(tmp_path_factory.mktemp("watch") / "stall_watch_check")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-x", "c++", *inc, os.path.join(HERE, "stall_watch_check.cpp"),
                        "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("the shared header does not compile for the host here: " + r.stderr[:200])

    def run(errs, window, adapt):
        inp = f"{window} {int(adapt)} {len(errs)}\n" + "\n".join(repr(float(e)) for e in errs) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
        return tuple(int(v) for v in out)
    return run


def test_steady_decrease_never_trips(watch):
    errs = 1e-2 * 0.98 ** np.arange(500)
    assert watch(errs, 64, False) == (0, 500, 1)


def test_flat_error_trips_after_the_window(watch):
    errs = np.full(300, 3e-6)
    assert watch(errs, 64, False)[0] == 65      # last low at iteration 1
    assert watch(errs, 128, True)[0] == 129     # no gap seen: the window itself


def test_a_drop_under_one_percent_is_no_new_low(watch):
    errs = 1e-3 * 0.995 ** np.arange(200)       # 0.5 % per iteration
    tripped, it_ref, _ = watch(errs, 10, False)
    # lows at 1, 3, 5, ... (two steps make 0.99 x): never 10 iterations without one
    assert tripped == 0 and it_ref in (199, 200)


def test_widening_follows_the_longest_gap(watch):
    # a 5 % drop every 100 iterations: the fixed window of 64 trips, the
    # widening one (128, then twice the 100-iteration gap) keeps going
    errs = np.array([1e-3 * 0.95 ** (i // 100) for i in range(600)])
    assert watch(errs, 64, False)[0] == 65
    tripped, it_ref, gap = watch(errs, 128, True)
    assert tripped == 0 and gap == 100 and it_ref == 501
    # a low is accepted before the window is checked: lows at 1, 41, 121
    # (gaps 40 and 80, the second exactly the window max(64, 2 x 40)), then
    # none: the watch trips 2 x 80 iterations after the last low
    lows = {1: 1e-3, 41: 9e-4, 121: 8e-4}
    seq, cur = [], None
    for it in range(1, 500):
        cur = lows.get(it, cur)
        seq.append(cur)
    assert watch(np.array(seq), 64, True) == (121 + 160, 121, 80)
    # a gap beyond the widened window trips it before the late low arrives
    lows = {1: 1e-3, 11: 9e-4, 41: 8e-4, 131: 7e-4}   # gaps 10, 30, then 90 > max(64, 60)
    seq, cur = [], None
    for it in range(1, 300):
        cur = lows.get(it, cur)
        seq.append(cur)
    assert watch(np.array(seq), 64, True) == (41 + 64, 41, 30)
