"""Pins of the oracle's error measures (eq. err, err_local, err_average), its
homogenized equivalent stresses (T_eq, M_eq) and its step predictor
(Algorithm 2) against values worked out by hand or fixed by the mathematics.

* eq. err_average divides the voxel average of ||a_new - a_old|| by the norm
  of the average of a_new; eq. err_local uses the voxel maximum instead.  A
  two-voxel field is worked by hand, including the floored curvature
  denominator of a load without mean curvature.
* For a homogeneous cell the fields are uniform and T_eq, M_eq are the
  equivalent stresses of the closed-form elastic stresses, t_eq = |e12|
  sqrt(2 a1 mu (mu + kappa)) for a pure e12 strain and m_eq = |g12|
  sqrt(b1 gamma (beta + gamma)) for a pure gamma12 curvature (eq. equiv_stress
  and equiv_couple_stress with a2 = a1 mu / kappa, b2 = b1 (gamma + beta) /
  (gamma - beta)); on a plastic step T_eq = t_Y + t_H P (the returned stress
  lies on the yield surface, eq. radius_1).
* The linear-extrapolation predictor e' = e_n + ratio (e_n - e_{n-1}),
  ratio = (t_{n+1} - t_n) / (t_n - t_{n-1}), is exact for a linear elastic
  cell under a proportional load, whatever the step sizes: on a non-uniform
  time grid the first fixed-point iteration of every increment after the
  first changes nothing (its error is at the level of the converged
  tolerance), while the first increment (predictor E) does.
"""
import numpy as np
import pytest

import workloads as W
from oracle import solver


def _field(vals):
    """(1, 1, 2, 3, 3) field from two voxel tensors."""
    return np.asarray(vals, dtype=np.float64).reshape(1, 1, 2, 3, 3)


def _two_voxel_case(h):
    z = np.zeros((3, 3))
    e0 = np.zeros((3, 3)); e0[0, 0] = 3.0; e0[0, 1] = 4.0           # ||e0|| = 5
    g0 = np.zeros((3, 3)); g0[1, 2] = 0.6; g0[2, 1] = 0.8           # ||g0|| = 1, <g> = 0 below
    t1 = np.zeros((3, 3)); t1[1, 1] = 6.0; t1[2, 2] = 8.0           # ||t1|| = 10
    dt = np.zeros((3, 3)); dt[2, 2] = 2.0
    new = dict(e=_field([e0, z]), g=_field([g0, -g0]), t=_field([z, t1]), m=_field([z, z]))
    old = dict(e=_field([z, z]), g=_field([z, z]), t=_field([z, t1 - dt]), m=_field([z, z]))
    return new, old


@pytest.mark.parametrize("h", [1.0, 0.5])
def test_error_measures_by_hand(h):
    new, old = _two_voxel_case(h)
    # means: ||<e>|| = 2.5, ||<t>|| = 5, <g> = 0, <m> = 0
    den_e = max(2.5, h * 0.0)          # = 2.5
    den_g = max(0.0, 2.5 / h)          # floored through the voxel size
    den_t = max(5.0, 0.0 / h)          # = 5
    # per-voxel ||delta||: e (5, 0), g (1, 1), t (0, 2), m (0, 0)
    local = {"e": 5.0 / den_e, "g": 1.0 / den_g, "t": 2.0 / den_t, "m": 0.0}
    average = {"e": 2.5 / den_e, "g": 1.0 / den_g, "t": 1.0 / den_t, "m": 0.0}
    for kind, want in (("local", local), ("average", average)):
        err, parts = solver.error_measure(new, old, kind, h)
        for a in ("e", "g", "t", "m"):
            assert parts[a] == pytest.approx(want[a], rel=1e-15, abs=1e-300), (kind, a)
        assert err == pytest.approx(max(want.values()), rel=1e-15)
    # the two measures differ on this field (a mean taken for a max, or the
    # reverse, fails one of the two sets above)
    assert local["e"] != average["e"] and local["t"] != average["t"]


def test_error_measure_zero_over_zero_is_zero():
    z = np.zeros((1, 1, 2, 3, 3))
    fields = dict(e=z, g=z, t=z, m=z)
    err, parts = solver.error_measure(fields, fields, "average", 1.0)
    assert err == 0.0 and all(v == 0.0 for v in parts.values())


def _homogeneous(row, Ef, Gf, n_steps, tol=1e-12, n=(2, 2, 2)):
    phases = W.phase_record([row])
    phase = np.zeros((n[2], n[1], n[0]), np.uint16)
    time, E, G = W.ramp_path(n_steps, Ef, Gf)
    return W.generators._problem(n, phase, phases, time, E, G, tol, err_kind="average")


def test_equivalent_stress_averages_closed_form_elastic():
    row = dict(W.generators._matrix_row())
    row.update(alpha=0.4, beta=0.9, gamma=1.5, a1=1.3, b1=0.7, elastic=1)
    eps, kap_g = 0.003, 0.002
    Ef = np.zeros((3, 3)); Ef[0, 1] = eps
    Gf = np.zeros((3, 3)); Gf[0, 1] = kap_g
    res = solver.solve(_homogeneous(row, Ef, Gf, 2))
    assert res["status"] == "ok"
    mu, kappa, a1 = row["mu"], row["kappa"], row["a1"]
    beta, gamma, b1 = row["beta"], row["gamma"], row["b1"]
    for s, frac in enumerate((0.5, 1.0)):
        teq = frac * eps * np.sqrt(2.0 * a1 * mu * (mu + kappa))
        meq = frac * kap_g * np.sqrt(b1 * gamma * (beta + gamma))
        assert res["Teq"][s] == pytest.approx(teq, rel=1e-12)
        assert res["Meq"][s] == pytest.approx(meq, rel=1e-12)
        assert res["P"][s] == 0.0 and res["Q"][s] == 0.0


def test_equivalent_stress_averages_on_the_yield_surface():
    """A plastic homogeneous step: the returned stress lies on the yield
    surfaces, so <t_eq> = t_Y + t_H <p> and <m_eq> = m_Y + m_H <q>."""
    row = dict(W.generators._matrix_row())
    row.update(beta=0.6, gamma=1.5, tH=0.8, mH=0.5)
    Ef = np.array([[0.004, 0.006, 0.0], [0.0, -0.002, 0.0], [0.0, 0.0, 0.0]])
    Gf = np.array([[0.0, 0.02, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.01]])
    res = solver.solve(_homogeneous(row, Ef, Gf, 3))
    assert res["status"] == "ok"
    assert res["P"][-1] > 0.0 and res["Q"][-1] > 0.0
    assert res["Teq"][-1] == pytest.approx(row["tY"] + row["tH"] * res["P"][-1], rel=1e-12)
    assert res["Meq"][-1] == pytest.approx(row["mY"] + row["mH"] * res["Q"][-1], rel=1e-12)


def test_predictor_is_exact_for_linear_elastic_proportional_load():
    rng = np.random.default_rng(5)
    n = (6, 4, 4)
    phase = (rng.uniform(size=(n[2], n[1], n[0])) < 0.4).astype(np.uint16)
    rows = [dict(W.generators._matrix_row(), elastic=1), dict(W.generators._matrix_row(1.7), elastic=1)]
    rows[0]["beta"] = 0.7
    phases = W.phase_record(rows)
    time = np.array([0.0, 0.1, 0.3, 0.35, 0.7, 0.8])  # step-size ratios 2, 0.25, 7, 2/7
    Ef = np.array([[0.004, 0.002, 0.0], [0.001, -0.001, 0.0], [0.0, 0.0, 0.002]])
    Gf = np.array([[0.0, 0.003, 0.0], [0.0, 0.0, 0.0], [-0.002, 0.0, 0.001]])
    E = time[:, None, None] * Ef[None]
    G = time[:, None, None] * Gf[None]
    tol = 1e-13
    prob = W.generators._problem(n, phase, phases, time, E, G, tol, ref_kind="midrange")
    res = solver.solve(prob)
    assert res["status"] == "ok"
    first = [h[0] for h in res["err_history"]]
    assert first[0] > 1e-3                  # predictor E at the first increment is not the solution
    for s in range(1, len(first)):
        assert first[s] < 1e-10, (s, first[s])
        assert res["iters"][s] == 1


def test_error_floors_from_the_loading_history():
    """A field whose mean is zero now (the unloaded state of a cyclic load)
    is measured against the largest mean it reached at earlier steps."""
    new, old = _two_voxel_case(1.0)
    z = np.zeros_like(new["e"])
    zero_mean = dict(new, e=new["e"] - new["e"].mean(axis=(0, 1, 2)))  # <e> = 0 now
    err, parts = solver.error_measure(zero_mean, dict(old, e=z), "local", 1.0)
    assert parts["e"] == np.inf                              # no floor: undefined
    err, parts = solver.error_measure(zero_mean, dict(old, e=z), "local", 1.0, {"e": 4.0})
    d = np.sqrt((zero_mean["e"] ** 2).sum(axis=(-1, -2))).max()
    assert parts["e"] == pytest.approx(d / 4.0, rel=1e-15)
    # a history floor below the current mean changes nothing
    _, p0 = solver.error_measure(new, old, "local", 1.0)
    _, p1 = solver.error_measure(new, old, "local", 1.0, {"e": 1.0, "t": 1.0, "g": 0.0, "m": 0.0})
    assert p0 == p1


def test_cyclic_load_through_zero_converges():
    """Sec. 3.2's cycles return the mean strain to zero; with the history
    floors the fixed-point loop still converges there (a linear elastic
    laminate, whose unloaded state is exactly the zero state)."""
    from workloads import paper_cases as PC
    p = PC.workload_ratcheting(n_cycles=2, elastic=True)
    res = solver.solve(p, fft="library")
    assert res["status"] == "ok"
    back = 99  # E12 = 0 at the end of the first cycle
    assert np.abs(res["T"][back]).max() < 1e-6 * np.abs(res["T"]).max()
