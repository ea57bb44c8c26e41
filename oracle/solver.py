"""Algorithm 2: micropolar elastoplastic FFT-based basic scheme (FP64).

Test infrastructure only (see the package docstring).

Problem dictionaries come from ``workloads``: grid ``n = (N1, N2, N3)``,
voxel size ``h``, ``phase`` map (N3, N2, N1), ``phases`` table, ``time``
(n_steps + 1), ``E`` and ``G`` (n_steps + 1, 3, 3), ``tol``, ``err_kind``
('local' = eq. err_local, 'average' = eq. err_average), ``ref_kind``
('mean' = Alg. 2 reference medium, 'midrange', 'explicit' with
``ref_moduli``), ``max_iter``.

Step s = 1..n_steps of this module is the paper's time index n = s + 1; the
zero initial state sits at s = 0 (Alg. 2, initialisation line).

Readings where the paper is silent or degenerate (each also stated where it
is used):
* err denominators: ||<gamma>|| vanishes whenever the mean curvature is zero
  (and likewise for the other fields under other loads).  Each denominator is
  floored by its dimensional partner through the voxel size h:
      den_e = max(|<e>|, h |<gamma>|),   den_gamma = max(|<gamma>|, |<e>| / h),
      den_t = max(|<t>|, |<m>| / h),     den_m = max(|<m>|, h |<t>|),
  where, so that a cyclic load passing through a zero mean (the unloaded state
  of Sec. 3.2, or a mean stress changing sign) keeps a finite measure, each
  |<a>| is the larger of the field's mean norm now and the largest one it
  reached at any earlier converged step of the load path (the scale of the
  loading history; zero at the first step).
  A zero numerator over a zero denominator counts as zero.
* divergence: a non-finite error, or one above ``div_limit`` (default 1e6),
  stops the solve with status 'diverged'; more than ``max_iter`` iterations in
  a step stops it with status 'not_converged'.
"""
from __future__ import annotations

import numpy as np

from . import fft as offt
from .constitutive import (apply_A, apply_B, equivalent_fields, radial_return_field,
                           stiffness_A, stiffness_B)
from .green import GreenOperator, wavevectors

MODULI = ("lambda", "mu", "kappa", "alpha", "beta", "gamma")


def reference_moduli(problem):
    """Six reference moduli (lambda0, mu0, kappa0, alpha0, beta0, gamma0).

    'mean': <A(x)>, <B(x)> over the voxels (Alg. 2); the stiffness tensors are
    linear in the moduli, so this is the voxel average of each modulus.
    'midrange': (min + max) / 2 of each modulus over the phases present.
    'explicit': ``problem['ref_moduli']``."""
    kind = problem.get("ref_kind", "mean")
    phases = problem["phases"]
    pm = problem["phase"]
    if kind == "explicit":
        return tuple(float(v) for v in problem["ref_moduli"])
    present, counts = np.unique(pm, return_counts=True)
    out = []
    for f in MODULI:
        vals = np.array([phases[int(i)][f] for i in present])
        if kind == "mean":
            out.append(float(np.sum(vals * counts) / pm.size))
        elif kind == "midrange":
            out.append(float(0.5 * (vals.min() + vals.max())))
        else:
            raise ValueError(f"unknown ref_kind {kind}")
    return tuple(out)


def reference_tensors(problem):
    """A0, B0 as 4th-order tensors.  For 'mean' the tensor average <A(x)> is
    formed literally from the per-phase tensors and volume fractions."""
    kind = problem.get("ref_kind", "mean")
    if kind == "mean":
        pm = problem["phase"]
        phases = problem["phases"]
        present, counts = np.unique(pm, return_counts=True)
        A0 = np.zeros((3, 3, 3, 3))
        B0 = np.zeros((3, 3, 3, 3))
        for i, c in zip(present, counts):
            r = phases[int(i)]
            A0 += (c / pm.size) * stiffness_A(r["lambda"], r["mu"], r["kappa"])
            B0 += (c / pm.size) * stiffness_B(r["alpha"], r["beta"], r["gamma"])
        return A0, B0
    lam, mu, kap, al, be, ga = reference_moduli(problem)
    return stiffness_A(lam, mu, kap), stiffness_B(al, be, ga)


def _norm(V):
    """||V|| = sqrt(V_kl V_kl) per voxel (Sec. 2.4)."""
    return np.sqrt(np.einsum("...kl,...kl->...", V, V))


def error_measure(new, old, kind, h, history=None):
    """eq. err with eq. err_local ('local') or eq. err_average ('average').

    ``new`` / ``old``: dicts with fields 'e', 't', 'g', 'm' (N3, N2, N1, 3, 3);
    ``history``: the largest ||<a>|| of each field at earlier converged steps
    (the denominator floors of the module docstring), or None.
    Returns (err, per-field dict)."""
    hist = history or {}
    # each field's magnitude: its mean now or the largest earlier one
    means = {a: max(_norm(new[a].mean(axis=(0, 1, 2))), hist.get(a, 0.0)) for a in ("e", "t", "g", "m")}
    den = {
        "e": max(means["e"], h * means["g"]),
        "g": max(means["g"], means["e"] / h),
        "t": max(means["t"], means["m"] / h),
        "m": max(means["m"], h * means["t"]),
    }
    parts = {}
    for a in ("e", "t", "g", "m"):
        d = _norm(new[a] - old[a])
        num = float(d.max()) if kind == "local" else float(d.mean())
        if den[a] == 0.0:
            parts[a] = 0.0 if num == 0.0 else np.inf
        else:
            parts[a] = num / den[a]
    return max(parts.values()), parts


def polarization(t, m, e, g, A0, B0, tau_m=None, mu_m=None):
    """tau = t - A0 e, mu = m - B0 gamma (eq. micropolar_polarizatons); with the
    manufactured stresses of eq. manufactured_polarization_stress subtracted
    when given (Appendix D.1)."""
    tau = t - apply_A(A0, e)
    mu = m - apply_B(B0, g)
    if tau_m is not None:
        tau = tau - tau_m
        mu = mu - mu_m
    return tau, mu


def _library_fftn(x):
    return np.fft.fftn(x, axes=(0, 1, 2))


def _library_ifftn(x):
    return np.fft.ifftn(x, axes=(0, 1, 2))


# The discrete Fourier transform of the scheme (same convention, unnormalised
# forward, 1/V inverse), evaluated by the oracle's own FFT ("own", default)
# or by numpy's FFT library routine ("library"), which computes the same
# transform (tests/test_oracle_fft_green.py checks the two against each other
# and against the brute-force triple sum) and is used for long reference runs.
FFT_BACKENDS = {"own": (offt.fftn, offt.ifftn), "library": (_library_fftn, _library_ifftn)}


def fixed_point_update(tau, mu, E, G, green, fft="own"):
    """One Lippmann-Schwinger update (Alg. 2 while-loop, transform / contract /
    inverse-transform steps): e = E + F^-1[G(tau^, mu^)], gamma likewise."""
    fwd, inv = FFT_BACKENDS[fft]
    tau_hat = fwd(tau)
    mu_hat = fwd(mu)
    e_hat, g_hat = green(tau_hat, mu_hat)
    e = E + inv(e_hat).real
    g = G + inv(g_hat).real
    return e, g


def averages(fields, phase_map, phases):
    """Homogenized outputs of one converged step (Sec. 3.2 and 3.3):
    T = <t>, M = <m>, <e>, <gamma>, P = <p>, Q = <q>, T_eq = <t_eq(t)>,
    M_eq = <m_eq(m)>."""
    teq, meq = equivalent_fields(fields["t"], fields["m"], phase_map, phases)
    return dict(T=fields["t"].mean(axis=(0, 1, 2)), M=fields["m"].mean(axis=(0, 1, 2)),
                Eavg=fields["e"].mean(axis=(0, 1, 2)), Gavg=fields["g"].mean(axis=(0, 1, 2)),
                P=float(fields["p"].mean()), Q=float(fields["q"].mean()),
                Teq=float(teq.mean()), Meq=float(meq.mean()))


def solve(problem, lockstep_iters=None, source=None, keep_fields=False, div_limit=1e6,
          max_steps=None, callback=None, fft="own"):
    """Run Algorithm 2 on ``problem``.

    lockstep_iters: optional per-step iteration counts; when given, each step
        runs exactly that many while-loop iterations (the error is still
        computed and reported).
    source: optional callable s -> (tau_m, mu_m) manufactured stress fields for
        step s (Appendix D.1, eq. manufactured_polarization_stress).
    keep_fields: store the converged fields of every step in the result.
    max_steps: stop after this many steps (bounded samples).
    callback: optional callable(step, iteration, err) called after every
        iteration (used for timing samples).
    fft: 'own' (the oracle's FFT) or 'library' (numpy's), see FFT_BACKENDS.

    Returns a dict with per-step arrays and the final fields."""
    n = problem["n"]
    h = problem["h"]
    pm = problem["phase"]
    phases = problem["phases"]
    time = problem["time"]
    Ep, Gp = problem["E"], problem["G"]
    tol = problem["tol"]
    kind = problem.get("err_kind", "local")
    max_iter = problem.get("max_iter", 10000)
    n_steps = len(time) - 1 if max_steps is None else min(max_steps, len(time) - 1)

    A0, B0 = reference_tensors(problem)
    xi, active = wavevectors(n, h)
    green = GreenOperator(xi, active, A0, B0)
    shape = (n[2], n[1], n[0])
    z9 = np.zeros(shape + (3, 3))
    # initial state (Alg. 2): all fields zero at time index 0
    hist = dict(e=z9.copy(), g=z9.copy(), t=z9.copy(), m=z9.copy(),
                p=np.zeros(shape), q=np.zeros(shape))
    committed = [dict(e=z9.copy(), g=z9.copy())]  # converged e, gamma per step (s = 0 first)
    scale = dict(e=0.0, t=0.0, g=0.0, m=0.0)       # largest ||<a>|| of the converged steps so far

    res = dict(T=[], M=[], Eavg=[], Gavg=[], P=[], Q=[], Teq=[], Meq=[], err=[], iters=[],
               err_history=[], err_parts=[], status="ok", failed_step=-1, fields=[])
    for s in range(1, n_steps + 1):
        E = Ep[s]
        G = Gp[s]
        # predictor (Alg. 2): E at the first step, linear extrapolation after
        if s == 1:
            e = np.broadcast_to(E, shape + (3, 3)).copy()
            g = np.broadcast_to(G, shape + (3, 3)).copy()
        else:
            ratio = (time[s] - time[s - 1]) / (time[s - 1] - time[s - 2])
            e = committed[s - 1]["e"] + ratio * (committed[s - 1]["e"] - committed[s - 2]["e"])
            g = committed[s - 1]["g"] + ratio * (committed[s - 1]["g"] - committed[s - 2]["g"])
        t, m, p, q = radial_return_field(e, g, hist["e"], hist["g"], hist["t"], hist["m"],
                                         hist["p"], hist["q"], pm, phases)
        tau_m = mu_m = None
        if source is not None:
            tau_m, mu_m = source(s)
        err = 2.0 * tol
        it = 0
        errs = []
        parts_s = []
        target = None if lockstep_iters is None else int(lockstep_iters[s - 1])
        while (err > tol) if target is None else (it < target):
            if target is None and it >= max_iter:
                res["status"] = "not_converged"
                res["failed_step"] = s
                break
            tau, mu = polarization(t, m, e, g, A0, B0, tau_m, mu_m)
            e_new, g_new = fixed_point_update(tau, mu, E, G, green, fft)
            t_new, m_new, p_new, q_new = radial_return_field(
                e_new, g_new, hist["e"], hist["g"], hist["t"], hist["m"], hist["p"], hist["q"],
                pm, phases)
            err, parts = error_measure(dict(e=e_new, t=t_new, g=g_new, m=m_new),
                                       dict(e=e, t=t, g=g, m=m), kind, h, scale)
            e, g, t, m, p, q = e_new, g_new, t_new, m_new, p_new, q_new
            it += 1
            errs.append(err)
            parts_s.append((parts["e"], parts["t"], parts["g"], parts["m"]))
            if callback is not None:
                callback(s, it, err)
            if not np.isfinite(err) or err > div_limit:
                res["status"] = "diverged"
                res["failed_step"] = s
                break
        res["iters"].append(it)
        res["err"].append(err)
        res["err_history"].append(errs)
        res["err_parts"].append(parts_s)
        # commit (Alg. 2, last line of the time loop)
        hist = dict(e=e, g=g, t=t, m=m, p=p, q=q)
        committed.append(dict(e=e, g=g))
        avg = averages(hist, pm, phases)
        for k, v in avg.items():
            res[k].append(v)
        for a, key in (("e", "Eavg"), ("t", "T"), ("g", "Gavg"), ("m", "M")):
            scale[a] = max(scale[a], float(_norm(avg[key])))
        if keep_fields:
            res["fields"].append({k: v.copy() for k, v in hist.items()})
        if res["status"] != "ok":
            break
    for k in ("T", "M", "Eavg", "Gavg"):
        res[k] = np.array(res[k])
    for k in ("P", "Q", "Teq", "Meq", "err"):
        res[k] = np.array(res[k], dtype=np.float64)
    res["iters"] = np.array(res["iters"], dtype=np.int64)
    res["final"] = hist
    res["ref_moduli"] = reference_moduli(problem)
    return res
