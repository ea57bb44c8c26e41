"""The launch-schedule autotuner: a new cell shape's candidate schedules
(pass-A rows per work item; fused spectral pass or separate column passes)
are timed on the cell's first increment, the fastest kept and cached in the
context.  Schedules only split the work differently, so the solve's results
agree with the default schedule's to rounding, and with the oracle as
always."""
import numpy as np
import pytest

import workloads as W
from oracle import solver as OS
from parity_helpers import compare_solves

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problem(n):
    rng = np.random.default_rng(17)
    phase = (rng.uniform(size=(n[2], n[1], n[0])) < 0.35).astype(np.uint16)
    rows = [dict(W.generators._matrix_row()), dict(W.generators._matrix_row(2.0))]
    rows[1]["elastic"] = 1
    phases = W.phase_record(rows)
    Ef = np.array([[0.004, 0.001, 0.0], [0.0, -0.001, 0.0], [0.0, 0.0, 0.001]])
    time, E, G = W.ramp_path(2, Ef, None)
    return W.generators._problem(n, phase, phases, time, E, G, 1e-8, ref_kind="midrange")


@pytest.mark.parametrize("n,precision", [((16, 16, 16), 0), ((24, 12, 8), 1), ((2, 256, 256), 1)])
def test_tuned_schedule_gives_the_same_solve(n, precision):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_10774_gb300 as M
    p = _problem(n)
    ref = OS.solve(p, fft="library", lockstep_iters=[6, 6])
    plain = M.Context(0)
    plain.set_autotune(False)
    tuned = M.Context(0)
    out = {}
    for name, ctx in (("plain", plain), ("tuned", tuned)):
        rve = M.Rve(ctx, p, precision=precision, lockstep_iters=ref["iters"])
        cfg = rve.config()
        assert rve.run(len(ref["iters"])) == 0
        out[name] = (cfg, rve.results(fields=True))
        rve.close()
    assert not out["plain"][0]["tuned"]
    default_rows = out["plain"][0]["rows_per_item"]
    cfg = out["tuned"][0]
    assert cfg["rows_per_item"] in {default_rows, max(default_rows // 2, 1), max(default_rows // 4, 1)}
    tol_h, tol_f = (1e-11, 1e-11) if precision == 0 else (1e-6, 1e-5)
    for name in ("plain", "tuned"):
        compare_solves(out[name][1], ref, tol_h, tol_f, h=p["h"])
    # a second cell of the shape takes the cached schedule
    rve = M.Rve(tuned, p, precision=precision)
    again = rve.config()
    rve.close()
    assert again["rows_per_item"] == cfg["rows_per_item"] and again["fused_spectral"] == cfg["fused_spectral"]
