"""Seeded inputs of the paper's own experiments (Sec. 3 and Appendix D.2).

Phase parameters are the paper's tables; where the paper's geometry is not
given (the four-sphere cell of Sec. 3.3) a seeded synthetic one with the
stated size and volume fraction stands in.  Load paths follow the stated
rates, time steps and step counts.  No function here computes any part of the
solver.

Readings:
* Table 5 lists phase 1 with beta = 0.5 > gamma = 0.1, which violates the
  bound gamma - beta >= 0 (eq. energetic_bounds; b2 would be negative).  As for
  every other drawn or listed parameter set, beta := min(beta, gamma) is
  applied (here beta = 0.1), recorded in the case's name.
* Table 3 gives lambda = mu = kappa = gamma / l_e^2 and a = b l_p^2 with b = 1.5,
  beta = gamma / 2, the rest as listed.
* The ratcheting cycle (Sec. 3.2) of one second loads E12 at rate +1 for its
  first half and unloads at rate -1 for its second half.
* The orientation of the ratcheting laminate is not stated.  Its layers are
  taken normal to x2: with layers normal to x1 the traction t_1l is uniform
  and, because mu = kappa in Table 2, the skew stress is uniform too, so the
  couple stress stays zero under E12, whereas the section requires a geometry
  whose heterogeneity activates it.
"""
from __future__ import annotations

import numpy as np

from .generators import _paint_sphere, _problem, laminate_map, phase_record, seed_for

COLUMNS = ("lambda", "mu", "kappa", "alpha", "beta", "gamma", "tY", "tH", "mY", "mH", "a1", "b1")


def _row(values, elastic=0):
    r = dict(zip(COLUMNS, (float(v) for v in values)))
    r["elastic"] = elastic
    return r


# Table 1 (micropolar-res1): phases 1, 2 and the Cauchy-limit phases
TABLE1 = {"phase1": (1.0, 1.0, 1.0, 0.0, 0.0, 1.0, 0.5, 0.125, 0.5, 0.125, 1.5, 1.5),
          "phase2": (2.0, 2.0, 2.0, 0.0, 0.0, 2.0, 0.75, 0.25, 0.75, 0.25, 1.5, 1.5),
          "cauchy_phase1": (1.0, 1.0, 0.0001, 0.0, 0.0, 0.0001, 0.5, 0.125, 1000.0, 0.0, 1.5, 1000.0),
          "cauchy_phase2": (2.0, 2.0, 0.0001, 0.0, 0.0, 0.0001, 0.75, 0.25, 1000.0, 0.0, 1.5, 1000.0)}
# Table 2 (micropolar_phases_racheting)
TABLE2 = {"phase1": (1.0, 1.0, 1.0, 0.0, 1.0, 2.0, 2.5, 0.0, 0.005, 0.0025, 1.5, 1.5),
          "phase2": (2.0, 2.0, 2.0, 0.0, 2.0, 4.0, 2.5, 0.0, 0.005, 0.0025, 1.5, 1.5)}
# Table 3 (sizeeffect): gamma, beta = gamma / 2, tY, tH, mY, mH and b per phase
TABLE3 = {"phase1": {"gamma": 1.0, "tY": 0.5, "tH": 0.125, "mY": 0.5, "mH": 0.125, "b": 1.5},
          "phase2": {"gamma": 2.0, "tY": 0.75, "tH": 0.25, "mY": 0.75, "mH": 0.25, "b": 1.5}}
# Table 4 (comput)
TABLE4 = {"phase1": (1.0, 1.0, 1.0, 0.0, 0.5, 1.0, 0.5, 0.125, 0.5, 0.125, 1.5, 1.5),
          "phase2": (2.0, 2.0, 2.0, 0.0, 1.0, 2.0, 0.75, 0.25, 0.75, 0.25, 1.5, 1.5)}
# Table 5 (iter_step); phase 2's tH = mH = x
TABLE5 = {"phase1": (1.0, 1.0, 1.0, 0.0, 0.5, 0.1, 0.5, 0.1, 0.5, 0.1, 1.5, 1.5),
          "phase2": (1.0, 1.0, 1.0, 0.0, 0.5, 1.0, 0.5, None, 0.5, None, 1.5, 1.5)}
TABLE5_X = (0.0, 0.001, 0.005, 0.01, 0.05, 0.1)


def _rate_path(n_steps, dt, E_rate=None, G_rate=None):
    time = dt * np.arange(n_steps + 1)
    E = np.zeros((n_steps + 1, 3, 3))
    G = np.zeros((n_steps + 1, 3, 3))
    if E_rate is not None:
        E = time[:, None, None] * np.asarray(E_rate, dtype=np.float64)[None]
    if G_rate is not None:
        G = time[:, None, None] * np.asarray(G_rate, dtype=np.float64)[None]
    return time, E, G


def _unit(k, l, value=1.0):
    a = np.zeros((3, 3))
    a[k, l] = value
    return a


# ---------------------------------------------------------------- Sec. 3.2 ratcheting

def cyclic_shear_path(n_cycles=10, steps_per_cycle=100, rate=1.0, comp=(0, 1)):
    """One-second cycles: E_comp rises at +rate for half a cycle and falls at
    -rate for the other half (dt = 1 / steps_per_cycle)."""
    n_steps = n_cycles * steps_per_cycle
    dt = 1.0 / steps_per_cycle
    time = dt * np.arange(n_steps + 1)
    phase_in_cycle = time - np.floor(time + 1e-12)
    up = np.minimum(phase_in_cycle, 1.0 - phase_in_cycle)
    up[np.isclose(phase_in_cycle, 0.0)] = 0.0
    E = np.zeros((n_steps + 1, 3, 3))
    E[:, comp[0], comp[1]] = rate * up
    return time, E, np.zeros_like(E)


def workload_ratcheting(n_cycles=10, tY=None, mH=None, elastic=False, tol=1e-5):
    """Sec. 3.2: 4 x 4 x 4 laminate at 50 % volume fraction, cell side L = 1,
    Table 2 phases, 10 one-second cycles of E12 at rates +-1 with dt = 0.01,
    eq. err_local at 1e-5.  tY / mH override both phases (the 50-cycle variants
    of the same section use tY = 1.9 with mH = 0 or mH = 0.0025); elastic makes
    both phases elastic (the non-dissipative comparison)."""
    rows = []
    for k in ("phase1", "phase2"):
        r = _row(TABLE2[k], elastic=1 if elastic else 0)
        if tY is not None:
            r["tY"] = float(tY)
        if mH is not None:
            r["mH"] = float(mH)
        rows.append(r)
    n = (4, 4, 4)
    time, E, G = cyclic_shear_path(n_cycles)
    name = f"ratchet-{n_cycles}c" + ("-elastic" if elastic else "") + (f"-tY{tY}" if tY is not None else "") \
        + (f"-mH{mH}" if mH is not None else "")
    return _problem(n, laminate_map(n, axis=1), phase_record(rows), time, E, G, tol, h=0.25, name=name)


# ---------------------------------------------------------------- Sec. 3.3 length scales

def four_sphere_map(n=16, volume_fraction=0.2, seed=None):
    """Four equal periodic non-overlapping spheres at the given volume fraction
    (the paper's positions are not given: seeded positions stand in)."""
    seed = seed_for(5) if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    nvox = n ** 3
    radius = (volume_fraction * nvox / (4 * 4.0 / 3.0 * np.pi)) ** (1.0 / 3.0)
    for _ in range(10000):
        centres = rng.uniform(0.0, n, (4, 3))
        ok = True
        for i in range(4):
            for j in range(i):
                d = centres[i] - centres[j]
                d -= n * np.round(d / n)
                if np.sqrt((d * d).sum()) < 2 * radius + 1.0:
                    ok = False
        if ok:
            break
    phase = np.zeros((n, n, n), dtype=np.uint16)
    for c in centres:
        _paint_sphere(phase, (n, n, n), c, radius, 1)
    return phase


def table3_phases(l_e, l_p):
    rows = []
    for k in ("phase1", "phase2"):
        t = TABLE3[k]
        g = t["gamma"]
        m = g / (l_e * l_e)
        rows.append({"lambda": m, "mu": m, "kappa": m, "alpha": 0.0, "beta": g / 2.0, "gamma": g,
                     "tY": t["tY"], "tH": t["tH"], "mY": t["mY"], "mH": t["mH"],
                     "a1": t["b"] * l_p * l_p, "b1": t["b"], "elastic": 0})
    return phase_record(rows)


def workload_length_scales(l_e, l_p, n=16, n_steps=100, tol=1e-5):
    """Sec. 3.3: 16^3 matrix with four spherical inclusions (20 % volume
    fraction), cell side L = 1, Table 3 phases at (l_e, l_p), monotonic
    E32 and Gamma11 at unit rates, dt = 0.01, 100 steps, eq. err_local 1e-5."""
    time, E, G = _rate_path(n_steps, 0.01, _unit(2, 1), _unit(0, 0))
    return _problem((n, n, n), four_sphere_map(n), table3_phases(l_e, l_p), time, E, G, tol, h=1.0 / n,
                    name=f"length-scales-le{l_e:g}-lp{l_p:g}", l_e=l_e, l_p=l_p)


# ---------------------------------------------------------------- Sec. 3.4 scaling and iterations

def workload_laminate_scaling(n, n_steps=100, tol=1e-5, err_kind="local"):
    """Sec. 3.4: 50 % laminate of n^3 voxels (1, 8, 64, ... voxels), cell side
    L = 1, Table 4 phases, E13 and Gamma32 at unit rates, dt = 0.01, 100
    steps, eq. err_local 1e-5."""
    phases = phase_record([_row(TABLE4["phase1"]), _row(TABLE4["phase2"])])
    shape = (n, n, n)
    phase = laminate_map(shape) if n > 1 else np.zeros((1, 1, 1), np.uint16)
    time, E, G = _rate_path(n_steps, 0.01, _unit(0, 2), _unit(2, 1))
    return _problem(shape, phase, phases, time, E, G, tol, h=1.0 / n, err_kind=err_kind,
                    name=f"laminate-scaling-{n}^3")


def workload_hardening_contrast(x, n=8, n_steps=100, tol=1e-8):
    """Sec. 3.4 / Table 5: the 512-voxel 50 % laminate, phase 2 hardening
    tH = mH = x, phase 1 with beta := min(beta, gamma) (see the module
    docstring), E13 and Gamma32 at unit rates, dt = 0.01, 100 steps,
    eq. err_local 1e-8."""
    r1 = _row(TABLE5["phase1"])
    r1["beta"] = min(r1["beta"], r1["gamma"])
    vals = list(TABLE5["phase2"])
    r2 = _row([x if v is None else v for v in vals])
    shape = (n, n, n)
    time, E, G = _rate_path(n_steps, 0.01, _unit(0, 2), _unit(2, 1))
    return _problem(shape, laminate_map(shape), phase_record([r1, r2]), time, E, G, tol, h=1.0 / n,
                    name=f"hardening-x{x:g}-beta1-clamped", x=x)


# ---------------------------------------------------------------- Sec. 3.1 Cauchy limit, App. D.2

def workload_cauchy_limit(n=8, n_steps=20, tol=1e-6, cauchy=True):
    """Sec. 3.1 phases (Table 1) on a 50 % laminate: the micropolar phases
    under E12 at unit rate, or the Cauchy-limit phases under E12 = E21 at
    unit rates (the paper's two loadings), dt = 0.01, eq. err_local."""
    keys = ("cauchy_phase1", "cauchy_phase2") if cauchy else ("phase1", "phase2")
    phases = phase_record([_row(TABLE1[keys[0]]), _row(TABLE1[keys[1]])])
    rate = _unit(0, 1) + (_unit(1, 0) if cauchy else 0.0)
    shape = (n, n, n)
    time, E, G = _rate_path(n_steps, 0.01, rate)
    return _problem(shape, laminate_map(shape), phases, time, E, G, tol, h=1.0 / n,
                    name=("cauchy" if cauchy else "micropolar") + f"-laminate-{n}^3")


def workload_calculation_verification(geometry="laminate", n=8, n_steps=20, tol=1e-4):
    """Appendix D.2: 50 % laminate or centred sphere of radius L / 4, Table 1
    phases, E12 at unit rate, dt = 0.01, eq. err_average at 1e-4."""
    phases = phase_record([_row(TABLE1["phase1"]), _row(TABLE1["phase2"])])
    shape = (n, n, n)
    if geometry == "laminate":
        phase = laminate_map(shape)
    else:
        phase = np.zeros((n, n, n), np.uint16)
        _paint_sphere(phase, shape, (n / 2, n / 2, n / 2), n / 4.0, 1)
    time, E, G = _rate_path(n_steps, 0.01, _unit(0, 1))
    return _problem(shape, phase, phases, time, E, G, tol, h=1.0 / n, err_kind="average",
                    name=f"calc-verification-{geometry}-{n}^3")
