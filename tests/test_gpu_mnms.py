"""The numerically manufactured solution MNMS-II of Appendix D.1 on the CUDA
path (FP64): the manufactured stresses enter the polarization as the source
of eq. manufactured_polarization_stress (mp_problem.tau_m / mu_m), and every
field of every one of the 100 increments must lie within the paper's printed
bound of 1e-9 of the manufactured solution (fixture
tests/golden/mnms_appendix_d1.json), single and as batched copies, and agree
with the oracle's run of the same problem.
"""
import json
import os

import numpy as np
import pytest

from oracle import mnms
from oracle import solver as OS
from parity_helpers import compare_solves

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_10774_gb300 as M
    return M.Context(0)


@pytest.fixture(scope="module")
def case():
    spec = json.load(open(os.path.join(GOLDEN, "mnms_appendix_d1.json")))
    prob = mnms.problem(n_steps=spec["n_steps"], tol=spec["tolerance"])
    tm, mm = mnms.manufactured_stresses(prob["time"])
    prob = dict(prob, tau_m=tm, mu_m=mm)
    ref = OS.solve(prob, source=lambda s: (tm[s], mm[s]))
    assert ref["status"] == "ok"
    e1, g1 = mnms.unit_rate_fields()
    return spec, prob, ref, tm, mm, e1, g1


def _worst(fin, s, prob, tm, mm, e1, g1):
    ts = prob["time"][s]
    return max(np.abs(fin["e"] - ts * e1).max(), np.abs(fin["g"] - ts * g1).max(),
               np.abs(fin["t"] - tm[s]).max(), np.abs(fin["m"] - mm[s]).max())


def test_mnms_every_increment_within_printed_bound(ctx, case):
    import paper_2409_10774_gb300 as M
    spec, prob, ref, tm, mm, e1, g1 = case
    rve = M.Rve(ctx, prob, precision=0)
    worst = 0.0
    for s in range(1, spec["n_steps"] + 1):
        assert rve.run(1) == 0
        res = rve.results(fields=True)
        worst = max(worst, _worst(res["final"], s, prob, tm, mm, e1, g1))
    rve.close()
    assert worst < spec["max_abs_error_bound"], worst
    fin = res["final"]
    assert (fin["p"] > 0).all() and (fin["q"] > 0).all()  # plastic at both levels


def test_mnms_matches_oracle_run(ctx, case):
    import paper_2409_10774_gb300 as M
    spec, prob, ref, tm, mm, e1, g1 = case
    res = M.mp_solve(ctx, prob, precision=0, fields=True, lockstep_iters=ref["iters"])
    assert res["status"] == "ok"
    compare_solves(res, ref, 1e-11, 1e-11, h=prob["h"])
    free = M.mp_solve(ctx, prob, precision=0)
    assert np.abs(free["iters"] - ref["iters"]).max() <= 1


def test_mnms_batched_copies(ctx, case):
    import paper_2409_10774_gb300 as M
    spec, prob, ref, tm, mm, e1, g1 = case
    single = M.mp_solve(ctx, prob, precision=0, fields=True)
    out = M.mp_batch_solve(ctx, [prob] * 4, precision=0, fields=True)
    for r in out:
        assert r["status"] == "ok"
        assert _worst(r["final"], spec["n_steps"], prob, tm, mm, e1, g1) < spec["max_abs_error_bound"]
        np.testing.assert_array_equal(r["final"]["e"], out[0]["final"]["e"])
        assert np.abs(r["T"] - single["T"]).max() <= 1e-12 * np.abs(single["T"]).max()

