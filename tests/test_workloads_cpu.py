"""The seeded input generators (host logic, no method arithmetic).

The benchmark and the parity tests rely on these recipes: the same seed gives
the same inputs, the geometries have the structure their docstrings state
(periodic non-overlapping RSA spheres at the requested volume fraction, a
periodic nearest-seed Voronoi tessellation whose 64^3 regeneration matches
the 256^3 cell, admissible per-grain moduli), and the load paths end at the
stated macroscopic strain.
"""
import numpy as np
import pytest

import workloads as W
from workloads import generators as G


def test_same_seed_same_inputs():
    a = W.workload_serving_request(3)
    b = W.workload_serving_request(3)
    c = W.workload_serving_request(4)
    assert a["n"] == b["n"] and np.array_equal(a["phase"], b["phase"]) and np.array_equal(a["E"], b["E"])
    assert not (a["n"] == c["n"] and np.array_equal(a["phase"], c["phase"]))


def test_rsa_spheres_periodic_non_overlapping_at_the_fraction():
    n = (40, 40, 40)
    r, vf = 4.0, 0.2
    phase, centres = G.rsa_sphere_map(n, r, vf, seed=11)
    L = np.array(n, dtype=float)
    d = centres[:, None, :] - centres[None, :, :]
    d -= L * np.round(d / L)
    dist = np.sqrt((d * d).sum(-1)) + np.eye(len(centres)) * 1e9
    assert dist.min() >= 2.0 * r
    frac = phase.mean()
    assert vf <= frac < vf + 0.05
    # every inclusion voxel lies within r of a centre (minimum image), every
    # other voxel farther from all of them
    x = np.stack(np.meshgrid(*[np.arange(k) + 0.5 for k in n[::-1]], indexing="ij"), -1)[..., ::-1]
    dd = x[:, :, :, None, :] - centres[None, None, None, :, :]
    dd -= L * np.round(dd / L)
    near = ((dd * dd).sum(-1) <= r * r).any(-1)
    assert np.array_equal(near, phase == 1)


def test_voronoi_nearest_seed_and_regeneration():
    seeds = G.voronoi_seeds(12, 64, seed=5)
    owner = G.voronoi_map((16, 16, 16), seeds, scale=16 / 64)
    assert set(np.unique(owner)) <= set(range(12))
    rng = np.random.default_rng(0)
    for _ in range(50):
        z, y, x = rng.integers(0, 16, 3)
        p = np.array([x + 0.5, y + 0.5, z + 0.5])
        d = p[None, :] - seeds * (16 / 64)
        d -= 16 * np.round(d / 16)
        d2 = (d * d).sum(1)
        assert d2[owner[z, y, x]] == pytest.approx(d2.min())
    # the 64^3 regeneration of the 256^3 cell: same seeds and grain table
    a = W.workload_voronoi(n=64, n_cells=200)
    t = G.voronoi_phase_table(200, W.seed_for(2))
    assert np.array_equal(a["phases"], t)
    assert np.all(a["phases"]["gamma"] >= a["phases"]["beta"])
    assert a["E"][-1][0, 0] == pytest.approx(0.01) and np.count_nonzero(a["E"][-1]) == 1


def test_batch_and_serving_recipes():
    probs = W.workload_batch(count=24)
    assert len(probs) == 24
    for p in probs:
        assert p["n"][0] in (16, 24, 32, 48) and p["n"][0] == p["n"][1] == p["n"][2]
        assert len(p["time"]) == 11
        assert np.linalg.norm(p["E"][-1]) == pytest.approx(0.005)
        assert np.count_nonzero(p["G"]) == 0
        assert 0.1 <= p["length_scale"] <= 10.0
        ph = p["phases"]
        assert np.allclose(ph["alpha"], ph["mu"] * p["length_scale"] ** 2)
    for i in range(6):
        q = W.workload_serving_request(i)
        assert q["n"][0] in (32, 64, 96, 128)
        assert 5 <= len(q["time"]) - 1 <= 20
        assert np.linalg.norm(q["E"][-1]) == pytest.approx(0.005)


def test_ramp_path_is_linear_from_zero():
    Ef = np.array([[0.004, 0.001, 0.0], [0.0, -0.001, 0.0], [0.0, 0.0, 0.002]])
    time, E, Gm = G.ramp_path(4, Ef)
    assert time[0] == 0.0 and np.all(np.diff(time) > 0)
    assert np.array_equal(E[0], np.zeros((3, 3))) and np.allclose(E[-1], Ef)
    assert np.allclose(E[2], 0.5 * Ef)
    assert np.count_nonzero(Gm) == 0


def test_box_shaped_voronoi_regenerations():
    """A box-shaped grid maps the same seed box onto each axis with its own
    scale: the cubic shape reproduces the cubic generator, and a box shape
    keeps the grain table and every grain that the scaled seeds reach."""
    cube = W.workload_voronoi(n=16)
    box = W.workload_voronoi(shape=(16, 16, 16))
    assert np.array_equal(cube["phase"], box["phase"])
    assert box["name"] == "voronoi200-16x16x16"
    thin = W.workload_voronoi(shape=(32, 8, 16))
    assert thin["n"] == (32, 8, 16) and thin["phase"].shape == (16, 8, 32)
    assert len(thin["phases"]) == len(cube["phases"])
    # nearest-seed check at a few voxels, seeds scaled per axis
    seeds = G.voronoi_seeds(200, 256, G.seed_for(2)) * (np.array([32, 8, 16]) / 256.0)
    rng = np.random.default_rng(0)
    for _ in range(20):
        z, y, x = (int(rng.integers(16)), int(rng.integers(8)), int(rng.integers(32)))
        c = np.array([x + 0.5, y + 0.5, z + 0.5])
        d = c[None, :] - seeds
        d -= np.array([32, 8, 16]) * np.round(d / np.array([32, 8, 16]))
        assert thin["phase"][z, y, x] == int(np.argmin((d * d).sum(axis=1)))
