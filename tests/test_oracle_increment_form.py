"""The increment form of the fixed-point iteration, on the oracle (FP64, CPU).

The batched GPU engine continues an FP32 cell that has reached the rounding
floor of its transforms in the increment form
    e^{i+1} = e^i + F^-1[G(F(tau^i - tau^{i-1}))]
(G the Green operator of Sec. 2.4 with its sign, applied to the change of the
polarization instead of the polarization).  Because G is linear and e^i is
itself E + F^-1[G(F tau^{i-1})], this is the same iteration as Algorithm 2's
full form in exact arithmetic.  Here both forms run side by side in FP64 with
the oracle's own steps and must give the same iterates to rounding; a wrong
sign, a dropped mean or an off-by-one in tau^{i-1} fails it.
"""
import numpy as np

import workloads as W
from oracle import solver as OS
from oracle.constitutive import radial_return_field
from oracle.green import GreenOperator, wavevectors


def _plastic_problem():
    # one large increment so that the matrix yields within the first step
    p = W.workload_centered_sphere(n=8, radius=2.5, n_steps=1, tol=1e-10, ref_kind="midrange")
    p = dict(p)
    p["E"] = np.array(p["E"]) * 4.0
    return p


def _run(problem, n_total, n_full, drop_previous=False):
    """n_total iterations of step 1; iterations n_full.. use the increment form
    (drop_previous: the planted mistake of transforming tau^i instead of
    tau^i - tau^{i-1})."""
    n, h = problem["n"], problem["h"]
    pm, phases = problem["phase"], problem["phases"]
    E, G = problem["E"][1], problem["G"][1]
    A0, B0 = OS.reference_tensors(problem)
    xi, active = wavevectors(n, h)
    green = GreenOperator(xi, active, A0, B0)
    shape = (n[2], n[1], n[0])
    z9 = np.zeros(shape + (3, 3))
    z = np.zeros(shape)
    e = np.broadcast_to(E, shape + (3, 3)).copy()
    g = np.broadcast_to(G, shape + (3, 3)).copy()
    t, m, p, q = radial_return_field(e, g, z9, z9, z9, z9, z, z, pm, phases)
    tau_prev = mu_prev = None
    for i in range(n_total):
        tau, mu = OS.polarization(t, m, e, g, A0, B0)
        if i < n_full:
            e_new, g_new = OS.fixed_point_update(tau, mu, E, G, green)
        else:
            dtau = tau if drop_previous else tau - tau_prev
            dmu = mu if drop_previous else mu - mu_prev
            de, dg = OS.fixed_point_update(dtau, dmu, 0.0 * E, 0.0 * G, green)
            e_new, g_new = e + de, g + dg
        tau_prev, mu_prev = tau, mu
        t, m, p, q = radial_return_field(e_new, g_new, z9, z9, z9, z9, z, z, pm, phases)
        e, g = e_new, g_new
    return dict(e=e, g=g, t=t, m=m, p=p, q=q)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_increment_form_equals_full_form():
    prob = _plastic_problem()
    full = _run(prob, 12, 12)
    inc = _run(prob, 12, 3)
    assert full["p"].max() > 0.0, "the workload must be plastic"
    for k in ("e", "g", "t", "m", "p", "q"):
        assert _rel(inc[k], full[k]) < 1e-11, k
    # the increment form keeps the prescribed mean strain
    assert np.allclose(inc["e"].mean(axis=(0, 1, 2)), prob["E"][1], rtol=0, atol=1e-15)


def test_increment_form_needs_the_previous_polarization():
    """Planted mistake: transforming tau^i itself in the increment form (the
    full-form polarization added to e^i) must be caught by the comparison."""
    prob = _plastic_problem()
    full = _run(prob, 12, 12)
    wrong = _run(prob, 12, 3, drop_previous=True)
    assert _rel(wrong["e"], full["e"]) > 1e-3
