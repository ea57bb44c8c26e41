"""FP32-mixed increments that stall above the tolerance, in the single-cell
solver: the serving workload's first request (RSA spheres at contrast 10,
strongly plastic) stalls at the FP32 rounding floor of the local error
measure at tolerance 1e-6.  Its increments continue in the increment form
and finish in FP64; the cell then returns to FP32 for the next increment.

* the solve ends ok where the plain FP32 loop would spend its 10^4
  iterations, with iters_fp64 <= iters and some increments finished in FP64;
* its homogenized stress agrees with the plain FP64 solve to the
  early-stopping level of a run stopped at the tolerance (1e-5 relative);
* the loop decided on the device (graph WHILE node, the stagnation watch in
  the loop-deciding reduction) and the loop decided on the host (per-kernel
  timing forces it) take the same decisions and give bit-identical results;
* a checkpoint taken between increments resumes to the same results,
  iters_fp64 included.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_10774_gb300 as M
    return M.Context(0)


def _request(n_steps=4):
    p = dict(W.workload_serving_request(0))
    p["time"], p["E"], p["G"] = p["time"][: n_steps + 1], p["E"][: n_steps + 1], p["G"][: n_steps + 1]
    return p


def _run(ctx, p, profile):
    import paper_2409_10774_gb300 as M
    r = M.Rve(ctx, p, precision=1)
    r.profile(profile)
    r.run(len(p["time"]) - 1)
    out = r.results()
    r.close()
    return out


def test_single_cell_finishes_stalled_increments_in_fp64(ctx):
    import paper_2409_10774_gb300 as M
    p = _request()
    r32 = M.mp_solve(ctx, p, precision=1)
    r64 = M.mp_solve(ctx, p, precision=0)
    assert r32["status"] == "ok" and r64["status"] == "ok"
    assert np.all(r32["iters_fp64"] <= r32["iters"])
    assert (r32["iters_fp64"] > 0).any(), (r32["iters"], r32["iters_fp64"])
    assert np.all(r32["err"] <= p["tol"])
    assert list(r64["iters_fp64"]) == list(r64["iters"])
    rel = np.abs(r32["T"] - r64["T"]).max() / np.abs(r64["T"]).max()
    assert rel <= 1e-5, rel


def test_device_and_host_loops_agree_through_the_stages(ctx):
    p = _request(3)
    dev = _run(ctx, p, profile=False)
    host = _run(ctx, p, profile=True)
    assert (dev["iters_fp64"] > 0).any()
    for k in ("iters", "iters_fp64", "T", "M", "Eavg", "P", "Q", "Teq", "Meq", "err"):
        assert np.array_equal(dev[k], host[k]), k


def test_checkpoint_keeps_fp64_counts(ctx):
    import paper_2409_10774_gb300 as M
    p = _request(4)
    a = M.Rve(ctx, p, precision=1)
    a.run(2)
    image = a.checkpoint()
    a.run(2)
    ra = a.results()
    a.close()
    b = M.Rve(ctx, p, precision=1)
    b.resume(image)
    b.run(2)
    rb = b.results()
    b.close()
    for k in ("iters", "iters_fp64", "T", "P", "err"):
        assert np.array_equal(ra[k], rb[k]), k
