"""GPU parity of the error measure (eq. err with eq. err_local and
eq. err_average) iteration by iteration: the CUDA path, run in lockstep with
the oracle, records eq. err and its four per-field terms (e, t, gamma, m) for
every fixed-point iteration (mp_rve_trace); they must be the oracle's.

Tolerances: in FP64 both sides' iterates agree to ~1e-13 of the fields, so an
error value, a difference of two iterates over a mean, agrees to that over
its own size (1e-4 relative near err ~ 1e-8, far better early on).  In FP32
the iterates round at ~1e-7 of the fields, so the error values are compared
while they are well above that (oracle err > 1e-3) at 1 % of their size.
"""
import numpy as np
import pytest

import workloads as W
from oracle import solver as OS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_10774_gb300 as M
    return M.Context(0)


def _problem(kind):
    p = dict(W.workload_centered_sphere(ref_kind="midrange", n_steps=4))
    p["err_kind"] = kind
    # a mean curvature, so that the curvature and couple-stress terms have
    # their own denominators rather than the floored ones
    p["G"] = np.array(p["E"]) * 0.0
    p["G"][:, 0, 1] = np.linspace(0.0, 0.002, len(p["time"]))
    return p


def _oracle_rows(ref):
    rows = []
    for s, (errs, parts) in enumerate(zip(ref["err_history"], ref["err_parts"])):
        for i, (e, pt) in enumerate(zip(errs, parts)):
            rows.append((s + 1, i + 1, e) + tuple(pt))
    return np.array(rows)


@pytest.mark.parametrize("kind", ["local", "average"])
@pytest.mark.parametrize("precision", [0, 1])
def test_error_trace_matches_oracle(ctx, kind, precision):
    import paper_2409_10774_gb300 as M
    p = _problem(kind)
    ref = OS.solve(p)
    assert ref["status"] == "ok"
    want = _oracle_rows(ref)
    rve = M.Rve(ctx, p, precision=precision, lockstep_iters=ref["iters"])
    rve.trace(True)
    assert rve.run(len(ref["iters"])) == 0
    got = rve.trace_read()
    rve.close()
    assert got.shape == want.shape
    np.testing.assert_array_equal(got[:, :2], want[:, :2])
    if precision == 0:
        bound = 1e-4 * np.abs(want[:, 2:]) + 1e-12
        assert np.all(np.abs(got[:, 2:] - want[:, 2:]) <= bound)
    else:
        big = want[:, 2] > 1e-3
        assert big.sum() >= 4
        d = np.abs(got[big, 2:] - want[big, 2:])
        assert np.all(d <= 1e-2 * np.abs(want[big, 2:]) + 1e-6)
    # the two measures differ (the average of the per-voxel norms is below their maximum)
    if kind == "average":
        loc = OS.solve(dict(p, err_kind="local"), lockstep_iters=ref["iters"])
        assert np.all(np.array(loc["err_history"][0]) > np.array(ref["err_history"][0]))
