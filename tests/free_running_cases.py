"""Recipes of the free-running parity cases (shared by the script that writes
their oracle references, tests/golden/make_free_running.py, and the GPU test
that compares the CUDA path with them).  Only inputs: no method arithmetic.

* rsa64: the 64^3 cell of random non-overlapping spheres (radius 6, volume
  fraction 0.3, stiffness contrast 10) under E11 to 1 % and then E12 to
  0.5 %, in 3 + 2 increments (the configuration's 17 + 8, coarsened so that
  the oracle's converged reference run stays within minutes).
* voronoi64: the 64^3 regeneration of the 256^3 Voronoi cell (same 200 seeds
  scaled by 1/4, same grain parameters), the first 8 of its 20 increments of
  E11 to 1 % (past first yield).
* request0: the serving workload's first request (RSA spheres, random strain
  direction), first 3 increments: a strongly plastic cell on which the FP32
  iteration stalls above the tolerance and continues in the increment form.
"""
import numpy as np

import workloads as W

ORACLE_TOL = 1e-10   # the references are converged far below the GPU runs' tolerance
SAMPLES = 2048       # voxels whose final fields are stored


def _truncate(problem, n_steps):
    p = dict(problem)
    p["time"] = np.asarray(problem["time"])[: n_steps + 1]
    p["E"] = np.asarray(problem["E"])[: n_steps + 1]
    p["G"] = np.asarray(problem["G"])[: n_steps + 1]
    return p


def problem(name):
    """The case's problem at its own tolerance (the GPU run's)."""
    if name == "rsa64":
        return W.workload_rsa_spheres(n=64, n1=3, n2=2, ref_kind="midrange")
    if name == "voronoi64":
        return _truncate(W.workload_voronoi(n=64), 8)
    if name == "request0":
        return _truncate(W.workload_serving_request(0), 3)
    raise KeyError(name)


def sample_voxels(problem, seed=2409):
    nv = int(np.prod(problem["n"]))
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(nv, min(SAMPLES, nv), replace=False))


CASES = ("rsa64", "voronoi64", "request0")
