"""Pins of the oracle's Algorithm 2 against results the paper or the
mathematics fixes.

* P1/P2 homogeneous medium and the 1-voxel grid: uniform fields, <e> = E,
  one iteration per step, the elastic stress in closed form.
* P7 the numerically manufactured solution of Appendix D.1: every field
  within the paper's printed bound 1e-9 of the manufactured one.
* P8 brute force: for elastic phases the converged fixed point equals the
  direct solution of the discrete (trigonometric Galerkin) balance equations.
* P10 laminate: fields depend on the normal coordinate only and the traction
  t_1l is uniform (eq. momemtum_balance).
* P11/P12 classical limit: with vanishing curvature moduli the homogenized
  stress approaches an independently written classical J2 Moulinec-Suquet
  scheme, and the size effect decays monotonically as the intrinsic length
  l (alpha = beta = gamma = mu l^2) goes to zero.
* P13 translation invariance; and the recorded divergence of the paper's
  mean reference medium on the centred-sphere workload.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import mnms, solver

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sym(V):
    return 0.5 * (V + np.swapaxes(V, -1, -2))


def _skw(V):
    return 0.5 * (V - np.swapaxes(V, -1, -2))


def _tr(V):
    return np.trace(V, axis1=-2, axis2=-1)


def _c(row, key):
    return np.asarray(row[key])[..., None, None]


def _elastic_t(row, e):
    """eq. elast_constitutive_iso written out (scalar or per-voxel moduli)."""
    return (_c(row, "lambda") * _tr(e)[..., None, None] * np.eye(3) + 2 * _c(row, "mu") * _sym(e)
            + 2 * _c(row, "kappa") * _skw(e))


def _elastic_m(row, g):
    return (_c(row, "alpha") * _tr(g)[..., None, None] * np.eye(3)
            + (_c(row, "beta") + _c(row, "gamma")) * _sym(g)
            + (_c(row, "beta") - _c(row, "gamma")) * _skw(g))


# ---------------------------------------------------------------- P1 / P2

@pytest.mark.parametrize("n", [(1, 1, 1), (4, 2, 6)])
def test_homogeneous_medium_gives_uniform_fields(n):
    row = dict(W.generators._matrix_row())
    row["alpha"] = 0.4
    phases = W.phase_record([row])
    phase = np.zeros((n[2], n[1], n[0]), np.uint16)
    Ef = np.array([[0.004, 0.002, 0.0], [0.0, -0.001, 0.0], [0.001, 0.0, 0.0]])
    Gf = np.array([[0.0, 0.003, 0.0], [0.0, 0.0, 0.0], [-0.002, 0.0, 0.001]])
    time, E, G = W.ramp_path(5, Ef, Gf)
    prob = W.generators._problem(n, phase, phases, time, E, G, 1e-10)
    res = solver.solve(prob, keep_fields=True)
    assert res["status"] == "ok"
    assert list(res["iters"]) == [1] * 5
    for s in range(5):
        f = res["fields"][s]
        np.testing.assert_allclose(f["e"], np.broadcast_to(E[s + 1], f["e"].shape), atol=1e-17)
        np.testing.assert_allclose(f["g"], np.broadcast_to(G[s + 1], f["g"].shape), atol=1e-17)
        assert np.ptp(f["t"], axis=(0, 1, 2)).max() < 1e-15
        assert res["err"][s] < 1e-12
    # the first increment is elastic: T = A E, M = B Gamma in closed form
    r0 = phases[0]
    np.testing.assert_allclose(res["T"][0], _elastic_t(r0, E[1]), atol=1e-16)
    np.testing.assert_allclose(res["M"][0], _elastic_m(r0, G[1]), atol=1e-16)
    assert res["P"][-1] > 0.0  # later increments are plastic


# ---------------------------------------------------------------- P7 MNMS

def test_mnms_appendix_d1_within_printed_bound():
    spec = json.load(open(os.path.join(GOLDEN, "mnms_appendix_d1.json")))
    cols = ("lambda", "mu", "kappa", "alpha", "beta", "gamma", "tY", "tH", "mY", "mH", "a1", "b1")
    for idx, key in ((0, "phase1"), (1, "phase2")):
        for c in cols:
            assert mnms.PHASES[idx][c] == spec[key][c]
    np.testing.assert_array_equal(mnms.E_RATE, np.array(spec["E_rate"]))
    np.testing.assert_array_equal(mnms.G_RATE, np.array(spec["Gamma_rate"]))
    prob = mnms.problem(n_steps=spec["n_steps"], tol=spec["tolerance"])
    assert prob["n"] == tuple(spec["grid"])
    tm, mm = mnms.manufactured_stresses(prob["time"])
    e1, g1 = mnms.unit_rate_fields()
    res = solver.solve(prob, source=lambda s: (tm[s], mm[s]), keep_fields=True)
    assert res["status"] == "ok"
    worst = 0.0
    for s in range(1, spec["n_steps"] + 1):
        f = res["fields"][s - 1]
        ts = prob["time"][s]
        worst = max(worst, np.abs(f["e"] - ts * e1).max(), np.abs(f["g"] - ts * g1).max(),
                    np.abs(f["t"] - tm[s]).max(), np.abs(f["m"] - mm[s]).max())
    assert worst < spec["max_abs_error_bound"], worst
    # the manufactured state is genuinely plastic at both levels
    fin = res["fields"][-1]
    assert (fin["p"] > 0).all() and (fin["q"] > 0).all()


# ---------------------------------------------------------------- P8 brute force

def _brute_force_elastic(prob, s):
    """Direct solve of the discrete balance equations at step s for elastic
    phases: unknown displacement / micro-rotation amplitudes on the non-zero,
    non-Nyquist frequencies; numpy.fft serves as the (library) transform."""
    n = prob["n"]
    shape = (n[2], n[1], n[0])
    h = prob["h"]
    f1 = np.fft.fftfreq(n[0]) * n[0]
    f2 = np.fft.fftfreq(n[1]) * n[1]
    f3 = np.fft.fftfreq(n[2]) * n[2]
    K3, K2, K1 = np.meshgrid(f3, f2, f1, indexing="ij")
    ok = (K1 ** 2 + K2 ** 2 + K3 ** 2) > 0
    for F, N in ((K1, n[0]), (K2, n[1]), (K3, n[2])):
        if N % 2 == 0:
            ok &= np.abs(F) != N // 2
    xi = np.stack([2 * np.pi * K1 / (n[0] * h), 2 * np.pi * K2 / (n[1] * h),
                   2 * np.pi * K3 / (n[2] * h)], axis=-1)
    idx = np.argwhere(ok)
    na = len(idx)
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    rows = prob["phases"][prob["phase"]]
    E, G = prob["E"][s], prob["G"][s]

    def fields(x):
        eh = np.zeros(shape + (3, 3), complex)
        gh = np.zeros(shape + (3, 3), complex)
        for j, (a, b, c) in enumerate(idx):
            u, ph = x[6 * j:6 * j + 3], x[6 * j + 3:6 * j + 6]
            k = xi[a, b, c]
            eh[a, b, c] = 1j * np.outer(k, u) + np.einsum("lkm,m->kl", eps, ph)
            gh[a, b, c] = 1j * np.outer(ph, k)
        e = E + np.fft.ifftn(eh, axes=(0, 1, 2))
        g = G + np.fft.ifftn(gh, axes=(0, 1, 2))
        return e, g

    def residual(x):
        e, g = fields(x)
        t = _elastic_t(rows, e)
        m = _elastic_m(rows, g)
        th = np.fft.fftn(t, axes=(0, 1, 2))
        mh = np.fft.fftn(m, axes=(0, 1, 2))
        r = []
        for (a, b, c) in idx:
            k = xi[a, b, c]
            r.append(1j * k @ th[a, b, c])
            r.append(1j * k @ mh[a, b, c] + np.einsum("lkm,km->l", eps, th[a, b, c]))
        return np.concatenate(r)

    r0 = residual(np.zeros(6 * na, complex))
    M = np.zeros((6 * na, 6 * na), complex)
    for c in range(6 * na):
        x = np.zeros(6 * na, complex)
        x[c] = 1.0
        M[:, c] = residual(x) - r0
    x = np.linalg.solve(M, -r0)
    e, g = fields(x)
    return e.real, g.real, np.abs(e.imag).max()


def test_elastic_fixed_point_equals_direct_solve():
    rows = [dict(W.generators._matrix_row()), dict(W.generators._matrix_row(1.8))]
    rows[1]["beta"] = 1.2  # gamma - beta > 0 in both phases
    for r in rows:
        r["elastic"] = 1
    phases = W.phase_record(rows)
    phase = W.sphere_map((4, 4, 4), (2.0, 2.0, 2.0), 1.3)
    Ef = np.array([[0.01, 0.004, 0.0], [0.0, -0.003, 0.002], [0.001, 0.0, 0.005]])
    Gf = np.array([[0.0, 0.02, 0.0], [0.0, 0.0, 0.01], [-0.01, 0.0, 0.03]])
    time, E, G = W.ramp_path(1, Ef, Gf)
    prob = W.generators._problem((4, 4, 4), phase, phases, time, E, G, 1e-14)
    res = solver.solve(prob, keep_fields=True)
    assert res["status"] == "ok"
    e_ref, g_ref, imag = _brute_force_elastic(prob, 1)
    assert imag < 1e-14
    f = res["fields"][0]
    assert np.abs(f["e"] - e_ref).max() < 1e-12 * np.abs(e_ref).max()
    assert np.abs(f["g"] - g_ref).max() < 1e-12 * np.abs(g_ref).max()


# ---------------------------------------------------------------- P10 laminate

def test_laminate_traction_continuity():
    table = json.load(open(os.path.join(GOLDEN, "tables.json")))
    cols = table["columns"]
    rows = [dict(zip(cols, table["table4"][k])) for k in ("phase1", "phase2")]
    phases = W.phase_record(rows)
    n = (8, 2, 2)
    phase = W.laminate_map(n, axis=0)
    Ef = np.zeros((3, 3)); Ef[0, 2] = 0.6; Ef[0, 0] = 0.2
    Gf = np.zeros((3, 3)); Gf[2, 1] = 0.6
    time, E, G = W.ramp_path(4, Ef, Gf)
    prob = W.generators._problem(n, phase, phases, time, E, G, 1e-12, h=1.0 / 8)
    res = solver.solve(prob, keep_fields=True)
    assert res["status"] == "ok"
    f = res["fields"][-1]
    assert f["p"].max() > 0 and f["q"].max() > 0
    for key in ("e", "g", "t", "m"):
        # independent of x2, x3 (axes 0, 1 of the (N3, N2, N1) arrays)
        assert np.ptp(f[key], axis=(0, 1)).max() < 1e-12
    t1 = f["t"][..., 0, :]
    scale = np.abs(f["t"]).max()
    assert np.ptp(t1, axis=(0, 1, 2)).max() < 1e-9 * scale


# ---------------------------------------------------------------- P11 / P12 classical limit

def _classical_ms(phase_map, rows, time, E, tol, lam0, mu0, h=1.0):
    """Classical small-strain J2 basic scheme (Moulinec-Suquet 1998) with the
    same predictor, error measure and Nyquist treatment: test-only code."""
    N3, N2, N1 = phase_map.shape
    f1 = np.fft.fftfreq(N1) * N1
    f2 = np.fft.fftfreq(N2) * N2
    f3 = np.fft.fftfreq(N3) * N3
    K3, K2, K1 = np.meshgrid(f3, f2, f1, indexing="ij")
    xi = np.stack([2 * np.pi * K1 / (N1 * h), 2 * np.pi * K2 / (N2 * h), 2 * np.pi * K3 / (N3 * h)], -1)
    ok = (K1 ** 2 + K2 ** 2 + K3 ** 2) > 0
    for F, N in ((K1, N1), (K2, N2), (K3, N3)):
        if N % 2 == 0:
            ok &= np.abs(F) != N // 2
    k2 = np.where(ok, (xi ** 2).sum(-1), 1.0)
    d = np.eye(3)
    G0 = (np.einsum("ki,...h,...j->...khij", d, xi, xi) + np.einsum("hi,...k,...j->...khij", d, xi, xi)
          + np.einsum("kj,...h,...i->...khij", d, xi, xi) + np.einsum("hj,...k,...i->...khij", d, xi, xi)
          ) / (4 * mu0 * k2[..., None, None, None, None])
    G0 -= ((lam0 + mu0) / (mu0 * (lam0 + 2 * mu0)) * np.einsum("...i,...j,...k,...h->...khij", xi, xi, xi, xi)
           / (k2 ** 2)[..., None, None, None, None])
    G0[~ok] = 0.0
    lam = rows["lambda"][phase_map]; mu = rows["mu"][phase_map]
    tY = np.where(rows["elastic"][phase_map] != 0, np.inf, rows["tY"][phase_map])
    tH = rows["tH"][phase_map]
    shape = phase_map.shape

    def C(eps, lm, m):
        return lm[..., None, None] * _tr(eps)[..., None, None] * d + 2 * m[..., None, None] * eps

    def rr(eps, eps_n, sig_n, p_n):
        s_tr = sig_n + C(eps - eps_n, lam, mu)
        dev = s_tr - _tr(s_tr)[..., None, None] * d / 3
        seq = np.sqrt(1.5 * (dev * dev).sum((-1, -2)))
        R = tY + tH * p_n
        pl = seq >= R
        dp = np.where(pl, (seq - np.where(pl, R, 0.0)) / (3 * mu + tH), 0.0)
        f = np.where(pl, (np.where(pl, R, 0.0) + tH * dp) / np.where(pl, seq, 1.0), 1.0)
        return _tr(s_tr)[..., None, None] * d / 3 + f[..., None, None] * dev, p_n + dp

    z = np.zeros(shape + (3, 3))
    eps_c = [z, z]
    sig_n, eps_n, p_n = z, z, np.zeros(shape)
    T = []
    for s in range(1, len(time)):
        if s == 1:
            eps = np.broadcast_to(E[s], z.shape).copy()
        else:
            r = (time[s] - time[s - 1]) / (time[s - 1] - time[s - 2])
            eps = eps_c[-1] + r * (eps_c[-1] - eps_c[-2])
        sig, p = rr(eps, eps_n, sig_n, p_n)
        err = 2 * tol
        while err > tol:
            tau = sig - (lam0 * _tr(eps)[..., None, None] * d + 2 * mu0 * eps)
            th = np.fft.fftn(tau, axes=(0, 1, 2))
            eh = -np.einsum("...khij,...ij->...kh", G0, th)
            eps_new = E[s] + np.fft.ifftn(eh, axes=(0, 1, 2)).real
            sig_new, p = rr(eps_new, eps_n, sig_n, p_n)
            de = np.sqrt(((eps_new - eps) ** 2).sum((-1, -2))).max() / np.linalg.norm(eps_new.mean((0, 1, 2)))
            ds = np.sqrt(((sig_new - sig) ** 2).sum((-1, -2))).max() / np.linalg.norm(sig_new.mean((0, 1, 2)))
            err = max(de, ds)
            eps, sig = eps_new, sig_new
        eps_c.append(eps)
        sig_n, eps_n, p_n = sig, eps, p
        T.append(sig.mean((0, 1, 2)))
    return np.array(T)


def _sphere_problem(ell, kappa=None):
    rows = [dict(W.generators._matrix_row()), dict(W.generators._matrix_row(2.5))]
    rows[1]["elastic"] = 1
    for r in rows:
        r["alpha"] = r["beta"] = r["gamma"] = r["mu"] * ell * ell
        r["mY"] = 1e3  # the micro level stays elastic
        if kappa is not None:
            r["kappa"] = kappa
    phases = W.phase_record(rows)
    phase = W.sphere_map((8, 8, 8), (4.0, 4.0, 4.0), 2.5)
    Ef = np.array([[0.004, 0.0015, 0.0], [0.0015, 0.0, 0.0], [0.0, 0.0, -0.001]])  # symmetric
    time, E, G = W.ramp_path(4, Ef)
    return W.generators._problem((8, 8, 8), phase, phases, time, E, G, 1e-9, ref_kind="midrange")


def test_size_effect_vanishes_as_intrinsic_length_goes_to_zero():
    prob0 = _sphere_problem(1.0)
    lam0, mu0 = solver.reference_moduli(prob0)[:2]
    T_cl = _classical_ms(prob0["phase"], prob0["phases"], prob0["time"], prob0["E"], 1e-10, lam0, mu0)
    gaps = []
    for ell in (1.0, 0.3, 0.1, 0.03):
        res = solver.solve(_sphere_problem(ell))
        assert res["status"] == "ok"
        gaps.append(np.abs(res["T"][-1] - T_cl[-1]).max() / np.abs(T_cl[-1]).max())
    assert all(b < a for a, b in zip(gaps, gaps[1:])), gaps
    assert gaps[0] > 1e-3 and gaps[-1] < 3e-4, gaps


def test_cauchy_limit_parameters_approach_classical_scheme():
    table = json.load(open(os.path.join(GOLDEN, "tables.json")))
    cols = table["columns"]
    rows = [dict(zip(cols, table["table1"][k])) for k in ("cauchy_phase1", "cauchy_phase2")]
    phases = W.phase_record(rows)
    phase = W.sphere_map((8, 8, 8), (4.0, 4.0, 4.0), 2.5)
    Ef = np.zeros((3, 3)); Ef[0, 1] = Ef[1, 0] = 0.4   # Cauchy convention E12 = E21
    time, E, G = W.ramp_path(4, Ef)
    prob = W.generators._problem((8, 8, 8), phase, phases, time, E, G, 1e-9, h=1.0 / 8,
                                 ref_kind="midrange")
    res = solver.solve(prob)
    assert res["status"] == "ok" and res["P"][-1] > 0
    lam0, mu0 = solver.reference_moduli(prob)[:2]
    T_cl = _classical_ms(phase, phases, time, E, 1e-10, lam0, mu0, h=1.0 / 8)
    assert np.abs(res["T"] - T_cl).max() < 2e-3 * np.abs(T_cl).max()


# ---------------------------------------------------------------- P13 and F2

def test_translation_invariance():
    rng = np.random.default_rng(5)
    phase = (rng.uniform(size=(6, 4, 8)) < 0.3).astype(np.uint16)
    rows = [dict(W.generators._matrix_row()), dict(W.generators._matrix_row(1.5))]
    rows[1]["beta"] = 1.5
    phases = W.phase_record(rows)
    Ef = np.array([[0.006, 0.002, 0.0], [0.0, 0.0, 0.001], [0.0, 0.0, 0.0]])
    time, E, G = W.ramp_path(3, Ef)
    a = W.generators._problem((8, 4, 6), phase, phases, time, E, G, 1e-10, ref_kind="midrange")
    b = dict(a)
    b["phase"] = np.roll(phase, (2, 1, 3), axis=(0, 1, 2))
    ra = solver.solve(a, keep_fields=True)
    rb = solver.solve(b, keep_fields=True)
    assert list(ra["iters"]) == list(rb["iters"])
    np.testing.assert_allclose(ra["T"], rb["T"], atol=1e-13)
    np.testing.assert_allclose(ra["M"], rb["M"], atol=1e-13)
    np.testing.assert_allclose(np.roll(ra["final"]["t"], (2, 1, 3), axis=(0, 1, 2)), rb["final"]["t"],
                               atol=1e-12)
    # dissipation >= 0: plastic strains never decrease (eq. reduced_dissipation_ineq)
    assert np.all(np.diff(ra["P"]) >= 0)


def test_mean_reference_diverges_on_centred_sphere_midrange_converges():
    p = W.workload_centered_sphere()
    res = solver.solve(p, max_steps=3)
    assert res["status"] == "diverged" and res["failed_step"] <= 3
    p["ref_kind"] = "midrange"
    res = solver.solve(p, max_steps=2)
    assert res["status"] == "ok"


def test_centred_sphere_symmetry_under_uniaxial_strain():
    """P13: a sphere centred in the cell (voxel centres at i + 1/2) under E11
    alone.  The phase map is invariant under the reflections x_j -> L - x_j
    and under swapping y and z, and so is the load: <t22> = <t33>, the
    off-diagonal averages vanish, and so does the mean couple stress (no
    curvature load), to rounding; the plastic strain never decreases."""
    p = W.workload_centered_sphere(n=8, radius=2.5, n_steps=3, tol=1e-10, ref_kind="midrange")
    assert np.array_equal(p["phase"], np.transpose(p["phase"], (1, 0, 2)))   # z <-> y
    assert np.array_equal(p["phase"], p["phase"][::-1, ::-1, ::-1])
    res = solver.solve(p)
    assert res["status"] == "ok" and res["P"][-1] > 0.0
    T, M = res["T"], res["M"]
    scale = np.abs(T).max()
    np.testing.assert_allclose(T[:, 1, 1], T[:, 2, 2], rtol=0, atol=1e-12 * scale)
    off = T.copy()
    for k in range(3):
        off[:, k, k] = 0.0
    assert np.abs(off).max() <= 1e-12 * scale
    assert np.abs(M).max() <= 1e-12 * scale * p["h"]
    assert np.all(np.diff(res["P"]) >= 0) and np.all(np.diff(res["Q"]) >= 0)
