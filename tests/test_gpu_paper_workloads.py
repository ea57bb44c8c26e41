"""The paper's own experiments on the CUDA path, as batched workloads
(workloads/paper_cases.py), each checked against the oracle and against the
behaviour the paper reports.

* Micro-plastic ratcheting (Sec. 3.2, Table 2): 4^3 laminate, one-second
  cycles of E12 at rates +-1.  The macro level stays elastic (P = 0, T_eq
  below t_Y), the micro level yields every cycle (Q grows), and the stress
  shows a hysteresis loop that the all-elastic variant does not have; over 50
  cycles with t_Y = 1.9, Q grows linearly and P stays zero without micro
  hardening, while with m_H = 0.0025 macro plasticity appears.
* Length-scale sweep (Sec. 3.3, Table 3) as batched dataset generation over
  (l_e, l_p), with the curvature load Gamma11: M11 at the last step hardly
  depends on the lengths, T32 falls as l_e grows.
* Iterations against the hardening contrast (Sec. 3.4, Table 5): more
  fixed-point iterations as phase 2's hardening x goes to zero.
* The Cauchy-limit phases (Table 1) and the average error measure
  (eq. err_average, Appendix D.2) in lockstep with the oracle.
"""
import numpy as np
import pytest

from oracle import solver as OS
from parity_helpers import compare_solves
from workloads import paper_cases as PC

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2409_10774_gb300 as M
    return M.Context(0)


def _truncate(p, n_steps):
    q = dict(p)
    q["time"], q["E"], q["G"] = p["time"][: n_steps + 1], p["E"][: n_steps + 1], p["G"][: n_steps + 1]
    return q


# ---------------------------------------------------------------- Sec. 3.2

def test_ratcheting_matches_oracle_lockstep(ctx):
    import paper_2409_10774_gb300 as M
    p = _truncate(PC.workload_ratcheting(n_cycles=2), 200)
    ref = OS.solve(p, fft="library")
    assert ref["status"] == "ok"
    res = M.mp_solve(ctx, p, precision=0, fields=True, lockstep_iters=ref["iters"])
    compare_solves(res, ref, 1e-11, 1e-11, h=p["h"])


def _loop_gap(res, p, cycle):
    """T12 on loading minus T12 on unloading at E12 = 0.25 of one cycle."""
    up, down = 100 * cycle + 24, 100 * cycle + 74
    assert np.isclose(p["E"][up + 1][0, 1], 0.25) and np.isclose(p["E"][down + 1][0, 1], 0.25)
    return res["T"][up][0, 1] - res["T"][down][0, 1]


def test_ratcheting_batch_shows_micro_plastic_hysteresis(ctx):
    import paper_2409_10774_gb300 as M
    cases = [PC.workload_ratcheting(n_cycles=10), PC.workload_ratcheting(n_cycles=10, elastic=True),
             PC.workload_ratcheting(n_cycles=50, tY=1.9, mH=0.0),
             PC.workload_ratcheting(n_cycles=50, tY=1.9, mH=0.0025)]
    out = M.mp_batch_solve(ctx, cases, precision=1)
    for r in out:
        assert r["status"] == "ok"
    micro, elastic, soft0, soft1 = out
    tY, mY = 2.5, 0.005
    # 10 cycles: macro elastic, micro plastic every cycle, a hysteresis loop
    assert micro["P"].max() == 0.0 and micro["Teq"].max() < tY
    assert micro["Meq"].max() > mY
    q_end = micro["Q"][99::100]
    assert np.all(np.diff(q_end) > 0) and np.all(np.diff(micro["Q"]) >= -1e-12)
    scale = np.abs(micro["T"][:, 0, 1]).max()
    for c in range(1, 10):
        assert _loop_gap(micro, cases[0], c) > 1e-2 * scale
    # the elastic comparison: no loop, no plastic strain
    assert elastic["P"].max() == 0.0 and elastic["Q"].max() == 0.0
    for c in range(1, 10):
        assert abs(_loop_gap(elastic, cases[1], c)) <= 1e-5 * scale
    # 50 cycles, t_Y = 1.9: no micro hardening keeps the macro level elastic
    # while Q grows linearly; with micro hardening macro plasticity appears
    assert soft0["P"].max() == 0.0
    dq = np.diff(soft0["Q"][99::100])
    assert dq.min() > 0 and dq.max() <= 1.05 * dq.min()
    assert soft0["Meq"].max() <= mY * (1 + 1e-6)
    assert soft1["P"][-1] > 0.0


# ---------------------------------------------------------------- Sec. 3.3

def test_length_scale_sweep_batch(ctx):
    """The sweep as one batch.  The corner l_e = 0.1, l_p = 1 is left out: its
    elastic moduli (gamma / l_e^2 = 100, 200) against the post-yield tangent
    make the basic scheme contract so slowly that its first increment needs
    more than the 10^4 iterations allowed per increment (in FP64 as well; the
    paper notes the scheme's dependence on the stiffness contrast)."""
    import paper_2409_10774_gb300 as M
    lengths = (0.1, 0.4, 1.0)
    grid = [(le, lp) for le in lengths for lp in lengths if not (le == 0.1 and lp == 1.0)]
    cases = [PC.workload_length_scales(le, lp) for le, lp in grid]
    out = M.mp_batch_solve(ctx, cases, precision=1)
    for p, r in zip(cases, out):
        assert r["status"] == "ok", (p["name"], r["status"], r["steps_done"])
    T32 = {k: r["T"][-1][2, 1] for k, r in zip(grid, out)}
    M11 = {k: r["M"][-1][0, 0] for k, r in zip(grid, out)}
    m = np.array(list(M11.values()))
    # the curvature load path is active and the micropolar response hardly
    # depends on the lengths (Table 3 keeps gamma, b fixed): near-constant M11
    assert m.min() > 0 and np.ptp(m) <= 0.1 * m.mean()
    # elastically stiffer (larger T32) at smaller l_e, for every l_p
    for lp in lengths:
        col = [T32[(le, lp)] for le in lengths if (le, lp) in T32]
        assert all(a > b for a, b in zip(col, col[1:])), (lp, col)
    # l_e ~ l_p << L: the macro stress dominates the couple stress (the paper
    # prints T32 ~ 14 against M11 ~ 0.5 there, on its own four-sphere cell)
    assert T32[(0.1, 0.1)] > 10 * M11[(0.1, 0.1)]
    assert 5.0 < T32[(0.1, 0.1)] < 40.0 and 0.2 < M11[(0.1, 0.1)] < 1.5


@pytest.mark.parametrize("le,lp", [(1.0, 0.1), (0.4, 0.4)])
def test_length_scale_cells_match_oracle(ctx, le, lp):
    import paper_2409_10774_gb300 as M
    p = PC.workload_length_scales(le, lp, n_steps=10)
    ref = OS.solve(p, fft="library")
    assert ref["status"] == "ok"
    res = M.mp_solve(ctx, p, precision=0, fields=True, lockstep_iters=ref["iters"])
    compare_solves(res, ref, 1e-11, 1e-11, h=p["h"])
    batched = M.mp_batch_solve(ctx, [p], precision=0, lockstep_iters=[ref["iters"]])[0]
    compare_solves(batched, ref, 1e-11, h=p["h"])


# ---------------------------------------------------------------- Sec. 3.4

def test_iterations_grow_as_hardening_contrast_grows(ctx):
    import paper_2409_10774_gb300 as M
    cases = [PC.workload_hardening_contrast(x) for x in PC.TABLE5_X]
    out = M.mp_batch_solve(ctx, cases, precision=0)
    total = [int(np.sum(r["iters"])) for r in out]
    for r in out:
        assert r["status"] == "ok"
    # x ascending: non-increasing iteration totals, strictly more at x = 0 than at x = 0.1
    assert all(a >= b for a, b in zip(total, total[1:])), total
    assert total[0] > 2 * total[-1], total
    # against the oracle: the iteration totals (counts per increment shift by a
    # few where a slow contraction crosses the tolerance at a slightly other
    # iterate, which then changes the next increments' starting points) and,
    # in lockstep, the results
    for k in (0, len(cases) - 1):
        ref = OS.solve(cases[k], fft="library")
        assert ref["status"] == "ok"
        assert abs(total[k] - int(np.sum(ref["iters"]))) <= 0.05 * np.sum(ref["iters"])
        lock = M.mp_solve(ctx, cases[k], precision=0, lockstep_iters=ref["iters"])
        compare_solves(lock, ref, 1e-10, h=cases[k]["h"])


# ---------------------------------------------------------------- Sec. 3.1 and Appendix D.2

@pytest.mark.parametrize("cauchy", [True, False])
def test_table1_phases_match_oracle(ctx, cauchy):
    import paper_2409_10774_gb300 as M
    p = PC.workload_cauchy_limit(cauchy=cauchy)
    ref = OS.solve(p, fft="library")
    assert ref["status"] == "ok" and ref["P"][-1] > 0
    res = M.mp_solve(ctx, p, precision=0, fields=True, lockstep_iters=ref["iters"])
    compare_solves(res, ref, 1e-11, 1e-11, h=p["h"])


@pytest.mark.parametrize("geometry", ["laminate", "sphere"])
def test_calculation_verification_average_error(ctx, geometry):
    import paper_2409_10774_gb300 as M
    p = PC.workload_calculation_verification(geometry)
    assert p["err_kind"] == "average"
    ref = OS.solve(p, fft="library")
    assert ref["status"] == "ok"
    res = M.mp_solve(ctx, p, precision=0, fields=True, lockstep_iters=ref["iters"])
    compare_solves(res, ref, 1e-11, 1e-11, h=p["h"])
    free = M.mp_solve(ctx, p, precision=0)
    assert np.abs(free["iters"] - ref["iters"]).max() <= 1
    assert np.all(free["err"] <= p["tol"])
