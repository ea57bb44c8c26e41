"""Seeded generators for voxel microstructures, phase tables and load paths.

Geometry follows the paper's description of its inputs: a voxelised image
holding a phase (or grain) ID per voxel (Sec. 1), per-phase isotropic
micropolar moduli and yield/hardening parameters (Tables 1-5), and a
macroscopic strain / curvature history E(t), Gamma(t) (Alg. 2 inputs).

Conventions
-----------
* Grid ``n = (N1, N2, N3)``; arrays are C-ordered ``[x3][x2][x1]`` so that x1
  is the fastest (contiguous) axis.  Voxel centres sit at ``(i + 1/2) h``.
* A load path is ``time`` (n_steps + 1 values, ``time[0] = 0``) plus ``E`` and
  ``G`` of shape ``(n_steps + 1, 3, 3)`` (row index k, column index l of
  E_kl), with the zero initial state at index 0.
* Phase tables are numpy structured arrays with the fields of ``PHASE_FIELDS``;
  ``elastic = 1`` marks a phase that never yields.

No function here computes any part of the solver.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2409_10774

PHASE_FIELDS = ("lambda", "mu", "kappa", "alpha", "beta", "gamma",
                "tY", "tH", "mY", "mH", "a1", "b1", "elastic")

PHASE_DTYPE = np.dtype([(f, np.float64) for f in PHASE_FIELDS[:-1]] + [("elastic", np.int32)])


def seed_for(config: int, replica: int = 0) -> int:
    """Seed convention shared by every generator call."""
    return SEED_BASE + 1000 * config + replica


def phase_record(rows):
    """Build a phase table from a list of dicts (missing 'elastic' -> 0)."""
    table = np.zeros(len(rows), dtype=PHASE_DTYPE)
    for i, r in enumerate(rows):
        for f in PHASE_FIELDS:
            table[i][f] = r.get(f, 0)
    return table


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def _centres(n):
    """Voxel-centre coordinates (in voxel units) along x1, x2, x3."""
    return [np.arange(n[a]) + 0.5 for a in range(3)]


def _periodic_dist2(n, c):
    """Squared minimum-image distance from every voxel centre to point c.

    Returns an array of shape (N3, N2, N1)."""
    parts = []
    for a in range(3):
        d = _centres(n)[a] - c[a]
        d = d - n[a] * np.round(d / n[a])
        parts.append(d * d)
    return parts[2][:, None, None] + parts[1][None, :, None] + parts[0][None, None, :]


def sphere_map(n, centre, radius, inside=1, outside=0, periodic=False):
    """Phase map with one sphere (voxel centres within ``radius`` of centre)."""
    n = tuple(int(v) for v in n)
    if periodic:
        d2 = _periodic_dist2(n, centre)
    else:
        x1, x2, x3 = _centres(n)
        d2 = ((x3[:, None, None] - centre[2]) ** 2 + (x2[None, :, None] - centre[1]) ** 2
              + (x1[None, None, :] - centre[0]) ** 2)
    out = np.full((n[2], n[1], n[0]), outside, dtype=np.uint16)
    out[d2 <= radius * radius] = inside
    return out


def laminate_map(n, axis=0, fraction=0.5):
    """Two-phase laminate with layer normal along ``axis`` (0 -> x1)."""
    n = tuple(int(v) for v in n)
    out = np.zeros((n[2], n[1], n[0]), dtype=np.uint16)
    cut = int(round(fraction * n[axis]))
    sl = [slice(None)] * 3
    sl[2 - axis] = slice(cut, None)
    out[tuple(sl)] = 1
    return out


def _paint_sphere(phase, n, c, radius, value=1):
    """Set ``value`` at every voxel whose centre lies within ``radius`` of c
    (minimum-image distance), visiting only the periodic box around c.
    Returns the number of voxels that changed to ``value``."""
    idx = []
    for a in range(3):
        lo = int(np.floor(c[a] - radius - 0.5)) - 1
        hi = int(np.ceil(c[a] + radius + 0.5)) + 1
        if hi - lo >= n[a]:
            i = np.arange(n[a])
        else:
            i = np.arange(lo, hi + 1) % n[a]
        d = (i + 0.5) - c[a]
        d = d - n[a] * np.round(d / n[a])
        idx.append((i, d * d))
    (i1, d1), (i2, d2), (i3, d3) = idx
    inside = (d3[:, None, None] + d2[None, :, None] + d1[None, None, :]) <= radius * radius
    sub = phase[np.ix_(i3, i2, i1)]
    changed = int(np.count_nonzero(inside & (sub != value)))
    sub[inside] = value
    phase[np.ix_(i3, i2, i1)] = sub
    return changed


def rsa_sphere_map(n, radius, volume_fraction, seed, max_tries=200000):
    """Random sequential addition of periodic, non-overlapping equal spheres.

    Centres are uniform in the cell; a candidate is accepted if its
    minimum-image distance to every accepted centre is at least 2 r.  Spheres
    are added until the voxel volume fraction reaches ``volume_fraction``.
    Returns (phase map, centres)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = tuple(int(v) for v in n)
    L = np.array(n, dtype=np.float64)
    centres = np.empty((0, 3))
    phase = np.zeros((n[2], n[1], n[0]), dtype=np.uint16)
    size = phase.size
    filled = 0
    tries = 0
    while filled / size < volume_fraction:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("RSA did not reach the requested volume fraction")
        c = rng.uniform(0.0, 1.0, 3) * L
        if len(centres):
            d = c[None, :] - centres
            d -= L * np.round(d / L)
            if np.any((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]) < (2.0 * radius) ** 2):
                continue
        centres = np.vstack([centres, c[None, :]])
        filled += _paint_sphere(phase, n, c, radius)
    return phase, centres


def voronoi_seeds(n_cells, box, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 1.0, (n_cells, 3)) * float(box)


def voronoi_map(n, seeds, scale=1.0):
    """Periodic Voronoi tessellation: each voxel gets the index of its nearest
    seed (minimum-image distance, ties to the lowest index).  ``scale`` (one
    number, or one per axis) maps seed coordinates into this grid's voxel
    units (1/4 for the 64^3 regeneration of a 256^3 cell)."""
    n = tuple(int(v) for v in n)
    best = np.full((n[2], n[1], n[0]), np.inf)
    owner = np.zeros((n[2], n[1], n[0]), dtype=np.uint16)
    for i, s in enumerate(np.asarray(seeds) * scale):
        d2 = _periodic_dist2(n, s)
        closer = d2 < best
        best[closer] = d2[closer]
        owner[closer] = i
    return owner


def random_sphere_map(n, count, r_lo, r_hi, rng):
    """``count`` periodic spheres with radii U[r_lo, r_hi]; overlap allowed."""
    n = tuple(int(v) for v in n)
    phase = np.zeros((n[2], n[1], n[0]), dtype=np.uint16)
    for _ in range(count):
        c = rng.uniform(0.0, 1.0, 3) * np.array(n, dtype=np.float64)
        r = rng.uniform(r_lo, r_hi)
        phase[_periodic_dist2(n, c) <= r * r] = 1
    return phase


# --------------------------------------------------------------------------
# load paths
# --------------------------------------------------------------------------

def ramp_path(n_steps, E_final=None, G_final=None, t_final=1.0):
    """Monotonic proportional ramp from zero in ``n_steps`` equal increments."""
    time = np.linspace(0.0, t_final, n_steps + 1)
    frac = time / t_final
    E = np.zeros((n_steps + 1, 3, 3))
    G = np.zeros((n_steps + 1, 3, 3))
    if E_final is not None:
        E = frac[:, None, None] * np.asarray(E_final, dtype=np.float64)[None]
    if G_final is not None:
        G = frac[:, None, None] * np.asarray(G_final, dtype=np.float64)[None]
    return time, E, G


def two_leg_path(n1, leg1, n2, leg2):
    """Ramp to ``leg1`` in n1 increments, then add ``leg2`` in n2 increments
    while holding leg1 (equal time increments throughout)."""
    n_steps = n1 + n2
    time = np.linspace(0.0, 1.0, n_steps + 1)
    E = np.zeros((n_steps + 1, 3, 3))
    leg1 = np.asarray(leg1, dtype=np.float64)
    leg2 = np.asarray(leg2, dtype=np.float64)
    for s in range(n_steps + 1):
        if s <= n1:
            E[s] = leg1 * (s / n1)
        else:
            E[s] = leg1 + leg2 * ((s - n1) / n2)
    return time, E, np.zeros_like(E)


def _unit_direction(rng):
    v = rng.standard_normal(9)
    return (v / np.linalg.norm(v)).reshape(3, 3)


# --------------------------------------------------------------------------
# the benchmark workloads
# --------------------------------------------------------------------------

MATRIX = dict(lam=20.0, mu=12.0, kappa=3.0, alpha=1.5, beta=1.5, gamma=1.5,
              tY=0.05, tH=1.0, mY=0.05, mH=1.0, a1=1.5, b1=1.5)


def _matrix_row(scale=1.0):
    m = MATRIX
    return {"lambda": m["lam"] * scale, "mu": m["mu"] * scale, "kappa": m["kappa"] * scale,
            "alpha": m["alpha"] * scale, "beta": m["beta"] * scale, "gamma": m["gamma"] * scale,
            "tY": m["tY"], "tH": m["tH"], "mY": m["mY"], "mH": m["mH"], "a1": m["a1"], "b1": m["b1"]}


def _problem(n, phase, phases, time, E, G, tol, h=1.0, name="", **kw):
    p = dict(n=tuple(int(v) for v in n), h=float(h), phase=np.ascontiguousarray(phase, dtype=np.uint16),
             phases=phases, time=np.asarray(time, dtype=np.float64),
             E=np.asarray(E, dtype=np.float64), G=np.asarray(G, dtype=np.float64),
             tol=float(tol), err_kind="local", ref_kind="mean", ref_moduli=None,
             max_iter=10000, name=name)
    p.update(kw)
    return p


def workload_centered_sphere(n=16, radius=4.0, n_steps=10, tol=1e-8, ref_kind="mean"):
    """One centred elastic spherical inclusion in an elastoplastic matrix,
    uniaxial E11 ramp to 0.5 %, zero mean curvature."""
    phase = sphere_map((n, n, n), (n / 2, n / 2, n / 2), radius, inside=1, outside=0)
    incl = {"lambda": 60.0, "mu": 40.0, "kappa": 10.0, "alpha": 5.0, "beta": 5.0, "gamma": 5.0,
            "tY": 0.0, "tH": 0.0, "mY": 0.0, "mH": 0.0, "a1": 1.5, "b1": 1.5, "elastic": 1}
    phases = phase_record([_matrix_row(), incl])
    E = np.zeros((3, 3)); E[0, 0] = 0.005
    time, Ep, Gp = ramp_path(n_steps, E)
    return _problem((n, n, n), phase, phases, time, Ep, Gp, tol, ref_kind=ref_kind,
                    name=f"centered-sphere-{n}^3")


def workload_rsa_spheres(n=64, radius=6.0, volume_fraction=0.30, contrast=10.0, tol=1e-6,
                         seed=None, ref_kind="mean", n1=17, n2=8):
    """Seeded non-overlapping monodisperse spheres (RSA) at stiffness contrast
    ``contrast``; E11 to 1 % then E12 to 0.5 %."""
    seed = seed_for(1) if seed is None else seed
    phase, _ = rsa_sphere_map((n, n, n), radius, volume_fraction, seed)
    incl = _matrix_row(contrast)
    incl["elastic"] = 1
    phases = phase_record([_matrix_row(), incl])
    leg1 = np.zeros((3, 3)); leg1[0, 0] = 0.01
    leg2 = np.zeros((3, 3)); leg2[0, 1] = 0.005
    time, E, G = two_leg_path(n1, leg1, n2, leg2)
    return _problem((n, n, n), phase, phases, time, E, G, tol, ref_kind=ref_kind,
                    name=f"rsa-spheres-{n}^3")


def voronoi_phase_table(n_cells, seed):
    """Per-cell parameters drawn U[0.8, 1.2] x matrix values; beta is clamped
    to min(beta, gamma) so that gamma - beta >= 0 holds in every cell."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    rows = []
    m = _matrix_row()
    for _ in range(n_cells):
        r = dict(m)
        for f in ("lambda", "mu", "kappa", "alpha", "beta", "gamma", "tY", "mY"):
            r[f] = m[f] * rng.uniform(0.8, 1.2)
        r["beta"] = min(r["beta"], r["gamma"])
        rows.append(r)
    return phase_record(rows)


def workload_voronoi(n=256, n_cells=200, n_steps=20, tol=1e-6, seed=None, cell_box=256,
                     ref_kind="mean", shape=None):
    """Periodic Voronoi polycrystal-like cell.  Seeds live in a box of side
    ``cell_box`` voxels; generating at ``n = cell_box / 4`` gives the
    downsampled regeneration of the same tessellation and the same cell
    parameters.  ``shape = (N1, N2, N3)`` instead of ``n`` maps the seed box
    onto a box-shaped grid, each axis scaled by its own N / cell_box (the same
    grains, stretched; smaller grids of the 256^3 cell's kernels)."""
    seed = seed_for(2) if seed is None else seed
    seeds = voronoi_seeds(n_cells, cell_box, seed)
    if shape is None:
        dims, scale, tag = (n, n, n), n / cell_box, f"{n}^3"
    else:
        dims = tuple(int(v) for v in shape)
        scale = np.asarray(dims, dtype=np.float64) / cell_box
        tag = "x".join(str(v) for v in dims)
    phase = voronoi_map(dims, seeds, scale=scale)
    phases = voronoi_phase_table(n_cells, seed)
    E = np.zeros((3, 3)); E[0, 0] = 0.01
    time, Ep, Gp = ramp_path(n_steps, E)
    return _problem(dims, phase, phases, time, Ep, Gp, tol, ref_kind=ref_kind,
                    name=f"voronoi{n_cells}-{tag}")


def workload_batch(count=512, seed=None, sizes=(16, 24, 32, 48), n_steps=10, tol=1e-6,
                   ref_kind="midrange"):
    """Batch of RVEs of uneven size: 1-8 overlapping periodic spheres of
    radius U[3, 8], intrinsic length l ~ logU[0.1, 10] voxels entering as
    alpha = beta = gamma = mu_phase * l^2, random unit strain direction of norm
    0.5 %, zero curvature."""
    seed = seed_for(3) if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        k = int(rng.integers(1, 9))
        phase = random_sphere_map((n, n, n), k, 3.0, 8.0, rng)
        ell = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        mat = _matrix_row()
        incl = {"lambda": 60.0, "mu": 40.0, "kappa": 10.0, "tY": 0.0, "tH": 0.0, "mY": 0.0,
                "mH": 0.0, "a1": 1.5, "b1": 1.5, "elastic": 1}
        for r in (mat, incl):
            r["alpha"] = r["beta"] = r["gamma"] = r["mu"] * ell * ell
        phases = phase_record([mat, incl])
        E = 0.005 * _unit_direction(rng)
        time, Ep, Gp = ramp_path(n_steps, E)
        out.append(_problem((n, n, n), phase, phases, time, Ep, Gp, tol, ref_kind=ref_kind,
                            name=f"batch-{i}-{n}^3", length_scale=ell))
    return out


def workload_serving_request(index, seed=None, sizes=(32, 64, 96, 128), tol=1e-6,
                             ref_kind="midrange"):
    """One serving request: RSA spheres (r = 6, vf 0.3) at contrast 10, a
    random strain direction of norm 0.5 % reached in 5-20 increments."""
    seed = seed_for(4, index) if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.choice(sizes))
    n_steps = int(rng.integers(5, 21))
    phase, _ = rsa_sphere_map((n, n, n), 6.0, 0.30, seed + 7)
    incl = _matrix_row(10.0)
    incl["elastic"] = 1
    phases = phase_record([_matrix_row(), incl])
    E = 0.005 * _unit_direction(rng)
    time, Ep, Gp = ramp_path(n_steps, E)
    return _problem((n, n, n), phase, phases, time, Ep, Gp, tol, ref_kind=ref_kind,
                    name=f"request-{index}-{n}^3")


# --------------------------------------------------------------------------
# random material-point states (radial-return unit tests)
# --------------------------------------------------------------------------

def random_material_states(count, seed, strain_scale=0.01, history_scale=0.01,
                           p_scale=0.01):
    """Random inputs of the material-point update: current total strains e,
    curvatures g, the previous converged e_n, g_n, stresses t_n, m_n and
    equivalent plastic strains p_n, q_n >= 0.  Tensors have shape (count,3,3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    e = strain_scale * rng.standard_normal((count, 3, 3))
    g = strain_scale * rng.standard_normal((count, 3, 3))
    e_n = e + 0.3 * strain_scale * rng.standard_normal((count, 3, 3))
    g_n = g + 0.3 * strain_scale * rng.standard_normal((count, 3, 3))
    t_n = history_scale * rng.standard_normal((count, 3, 3))
    m_n = history_scale * rng.standard_normal((count, 3, 3))
    p_n = p_scale * rng.uniform(0.0, 1.0, count)
    q_n = p_scale * rng.uniform(0.0, 1.0, count)
    return dict(e=e, g=g, e_n=e_n, g_n=g_n, t_n=t_n, m_n=m_n, p_n=p_n, q_n=q_n)
