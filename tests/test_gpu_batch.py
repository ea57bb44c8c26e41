"""Batched solves and the continuous-batching server, through the C ABI.

* Batched FP64 solves agree with the FP64 oracle item by item (lockstep,
  <= 1e-11 relative, as for single solves).
* A cell's batched result does not depend on the other cells of the batch:
  alone and in a mix of other sizes, precisions and error metrics, every
  output is bit-identical.  Against mp_solve (a separately compiled form of
  the same kernels, whose reductions sum in another order) results agree to
  rounding.
* Failures stay per item (invalid input, non-convergence), matching mp_solve.
* The server admits requests while others run (their rounds overlap on the
  device), and each request's result is the same alone and in the mix; the
  HBM budget bounds what is resident at once.
"""
import threading
import time

import numpy as np
import pytest

import workloads as W
from parity_helpers import compare_solves as _compare_solves
from oracle import solver as OS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_FIELD_KEYS = ("e", "g", "t", "m", "p", "q")
_STEP_KEYS = ("T", "M", "Eavg", "Gavg", "P", "Q", "Teq", "Meq", "err", "iters")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_10774_gb300 as M
    return M.Context(0)


def _small_batch(count, sizes, n_steps, tol, seed=None):
    return W.workload_batch(count=count, sizes=sizes, n_steps=n_steps, tol=tol,
                            seed=W.seed_for(3) + 17 if seed is None else seed)


def _assert_identical(a, b, fields=True):
    assert a["status"] == b["status"]
    assert a["steps_done"] == b["steps_done"] and a["failed_step"] == b["failed_step"]
    for k in _STEP_KEYS:
        assert np.array_equal(a[k], b[k]), k
    if fields:
        for k in _FIELD_KEYS:
            assert np.array_equal(a["final"][k], b["final"][k]), k


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_batch_fp64_matches_oracle_lockstep(ctx):
    import paper_2409_10774_gb300 as M
    probs = _small_batch(4, (8, 12, 16), 3, 1e-8)
    refs = [OS.solve(p) for p in probs]
    assert all(r["status"] == "ok" for r in refs)
    res = M.mp_batch_solve(ctx, probs, precision=0, fields=True,
                           lockstep_iters=[r["iters"] for r in refs])
    for p, r, g in zip(probs, refs, res):
        assert g["status"] == "ok", p["name"]
        assert list(g["iters"]) == list(r["iters"])
        _compare_solves(g, r, 1e-11, 1e-11)


def test_batch_fp32_matches_oracle(ctx):
    """FP32-mixed batch within the FP32 tolerances (lockstep with the oracle)."""
    import paper_2409_10774_gb300 as M
    probs = _small_batch(3, (12, 16), 3, 1e-6, seed=W.seed_for(3) + 29)
    refs = [OS.solve(p) for p in probs]
    res = M.mp_batch_solve(ctx, probs, precision=1, fields=True,
                           lockstep_iters=[r["iters"] for r in refs])
    for r, g in zip(refs, res):
        assert g["status"] == "ok"
        _compare_solves(g, r, 1e-6, 1e-5)


def test_batch_item_alone_equals_item_in_mix(ctx):
    import paper_2409_10774_gb300 as M
    probs = _small_batch(6, (8, 12, 16, 24), 4, 1e-6)
    x = probs[2]
    alone = M.mp_batch_solve(ctx, [x], precision=1, fields=True)[0]
    assert alone["status"] == "ok"
    avg = dict(probs[3])
    avg["err_kind"] = "average"
    mix = [probs[1], avg, x, probs[4], probs[3]]
    precs = [1, 0, 1, 1, 0]
    res = M.mp_batch_solve(ctx, mix, precision=precs, fields=[True, False, True, False, True])
    assert [r["status"] for r in res] == ["ok"] * 5
    _assert_identical(res[2], alone)
    # and again, in another order and with x twice
    res2 = M.mp_batch_solve(ctx, [x, probs[3], x], precision=[1, 0, 1], fields=True)
    _assert_identical(res2[0], alone)
    _assert_identical(res2[2], alone)


def test_batch_agrees_with_single_solve(ctx):
    """mp_solve and the batch run separately compiled forms of the same
    kernels (one cell per launch vs. a work list of cells) and sum their
    reductions in other orders: the same iterations give the same results to
    rounding - the tolerances of the oracle comparisons."""
    import paper_2409_10774_gb300 as M
    probs = _small_batch(3, (12, 16), 4, 1e-6, seed=W.seed_for(3) + 5)
    for precision, tol_hom, tol_fields in ((0, 1e-11, 1e-11), (1, 1e-6, 1e-5)):
        res = M.mp_batch_solve(ctx, probs, precision=precision, fields=True)
        for p, b in zip(probs, res):
            s = M.mp_solve(ctx, p, precision=precision, fields=True, lockstep_iters=b["iters"])
            assert s["status"] == b["status"] == "ok"
            _compare_solves(b, s, tol_hom, tol_fields, h=p["h"])


def test_batch_failures_stay_per_item(ctx):
    import paper_2409_10774_gb300 as M
    probs = _small_batch(3, (8, 12), 3, 1e-6, seed=W.seed_for(3) + 41)
    bad = dict(probs[1])
    bad["phase"] = np.full_like(probs[1]["phase"], 7)  # phase id beyond the table
    stuck = dict(probs[2])
    stuck["tol"] = 1e-15
    stuck["max_iter"] = 3
    res = M.mp_batch_solve(ctx, [probs[0], bad, stuck], precision=1)
    assert res[0]["status"] == "ok"
    assert res[1]["status"] == "invalid_arg" and res[1]["steps_done"] == 0
    assert res[2]["status"] == "not_converged"
    single = M.mp_solve(ctx, stuck, precision=1)
    assert single["status"] == "not_converged"
    assert res[2]["failed_step"] == single["failed_step"] == 1
    assert res[2]["steps_done"] == single["steps_done"] == 1
    assert list(res[2]["iters"]) == list(single["iters"]) == [3]
    # same iterate sequence, but the batched and the single-cell kernels are
    # separately compiled and sum their FP64 reductions in another order, and
    # the FP32 fields carry that difference: agreement to FP32 rounding
    assert _rel(res[2]["T"], single["T"]) <= 1e-6
    alone = M.mp_batch_solve(ctx, [probs[0]], precision=1)[0]
    _assert_identical(res[0], alone, fields=False)


def test_server_results_same_alone_and_in_mix(ctx):
    """Requests submitted while another is running join its rounds; each
    result equals the one it gets alone."""
    import paper_2409_10774_gb300 as M
    long_req = W.workload_serving_request(0, sizes=(32,))
    # a fixed, long iteration schedule keeps it on the device while the others arrive
    lock = [150] * (len(long_req["time"]) - 1)
    short = _small_batch(3, (12, 16), 3, 1e-6, seed=W.seed_for(4) + 3)
    alone_long = M.mp_batch_solve(ctx, [long_req], precision=1, lockstep_iters=[lock])[0]
    alone_short = M.mp_batch_solve(ctx, short, precision=1, fields=True)
    with M.Server(ctx, budget_bytes=512 << 20) as srv:
        t_long = srv.submit(long_req, precision=1, lockstep_iters=lock)
        # wait until the long request is resident and iterating, then add the others
        deadline = time.time() + 60
        while srv.stats()["rounds"] < 3 and time.time() < deadline:
            time.sleep(0.002)
        tickets = [srv.submit(p, precision=1, fields=True) for p in short]
        got_short = [srv.wait(t) for t in tickets]
        got_long = srv.wait(t_long)
        st = srv.stats()
    assert st["peak_resident"] >= 2, st
    assert st["completed"] == 4 and st["queued"] == 0
    _assert_identical(got_long, alone_long, fields=False)
    for g, a in zip(got_short, alone_short):
        _assert_identical(g, a)


def test_server_concurrent_submitters(ctx):
    import paper_2409_10774_gb300 as M
    probs = _small_batch(8, (8, 12, 16), 2, 1e-6, seed=W.seed_for(4) + 11)
    alone = M.mp_batch_solve(ctx, probs, precision=1)
    out = [None] * len(probs)
    with M.Server(ctx, budget_bytes=256 << 20) as srv:
        def worker(i):
            out[i] = srv.wait(srv.submit(probs[i], precision=1))
        ths = [threading.Thread(target=worker, args=(i,)) for i in range(len(probs))]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
    for a, b in zip(out, alone):
        _assert_identical(a, b, fields=False)


def test_server_budget_bounds_residency(ctx):
    import paper_2409_10774_gb300 as M
    from paper_2409_10774_gb300 import binding as B
    probs = _small_batch(3, (16,), 2, 1e-8, seed=W.seed_for(4) + 19)
    alone = M.mp_batch_solve(ctx, probs, precision=0)
    # one 16^3 FP64 cell needs ~2.7 MB: a 4 MiB budget holds one at a time
    with M.Server(ctx, budget_bytes=4 << 20) as srv:
        ts = [srv.submit(p, precision=0) for p in probs]
        got = [srv.wait(t) for t in ts]
        st = srv.stats()
        big = W.workload_serving_request(1, sizes=(64,))
        with pytest.raises(B.MicropolarError) as ei:
            srv.submit(big, precision=1)
        assert ei.value.status == 6
    assert st["peak_resident"] == 1
    for g, a in zip(got, alone):
        assert g["status"] == "ok"
        _assert_identical(g, a, fields=False)


def test_server_wait_timeout_and_cancel(ctx):
    import paper_2409_10774_gb300 as M
    from paper_2409_10774_gb300 import binding as B
    req = W.workload_serving_request(2, sizes=(64,))
    srv = M.Server(ctx, budget_bytes=256 << 20)
    t = srv.submit(req, precision=0)
    with pytest.raises(B.MicropolarError) as ei:
        srv.wait(t, timeout_ms=0)
    assert ei.value.status == 8
    r = srv.wait(t, timeout_ms=-1)
    assert r["status"] == "ok" and r["steps_done"] == len(req["time"]) - 1
    # destroy with work queued and resident: returns, nothing left behind
    for _ in range(3):
        srv.submit(req, precision=1)
    srv.close()


def _truncate(problem, n_steps):
    p = dict(problem)
    p["time"] = problem["time"][: n_steps + 1]
    p["E"] = problem["E"][: n_steps + 1]
    p["G"] = problem["G"][: n_steps + 1]
    return p


def test_batch_fp32_escalates_stagnating_cells(ctx):
    """A strongly plastic cell whose FP32 iteration stalls above the tolerance
    of the local error measure continues those increments in the increment
    form (and, should that stall too, in FP64) and converges; it agrees with
    the plain FP64 solve to the tolerance's level and is the same alone and
    beside another cell."""
    import paper_2409_10774_gb300 as M
    p = _truncate(W.workload_serving_request(0), 3)
    st = {}
    r32 = M.mp_batch_solve(ctx, [p], precision=1, stats=st)[0]
    r64 = M.mp_batch_solve(ctx, [p], precision=0)[0]
    assert r32["status"] == "ok" and r64["status"] == "ok"
    assert st["delta_switches"] > 0
    assert st["escalations"] == int((r32["iters_fp64"] > 0).sum())
    assert np.all(r32["iters_fp64"] <= r32["iters"])
    assert list(r64["iters_fp64"]) == list(r64["iters"])
    assert np.all(r32["err"] <= p["tol"])
    assert _rel(r32["T"], r64["T"]) <= 1e-5
    other = _small_batch(1, (16,), 3, 1e-6, seed=W.seed_for(4) + 23)[0]
    mix = M.mp_batch_solve(ctx, [other, p], precision=1)
    _assert_identical(mix[1], r32, fields=False)
