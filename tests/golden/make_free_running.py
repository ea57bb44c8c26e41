"""Writes the oracle references of the free-running parity cases
(tests/free_running_cases.py): the FP64 oracle run to an error of 1e-10, its
per-increment homogenized results and iteration counts, and its final fields
on a seeded sample of voxels, with the full fields' L2 norms.

Calls only the oracle (numpy's FFT as its transform step, see
oracle.solver.FFT_BACKENDS).  Usage:

    python tests/golden/make_free_running.py [case ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import free_running_cases as FC  # noqa: E402
from oracle import solver  # noqa: E402


def write(name):
    prob = dict(FC.problem(name))
    prob["tol"] = FC.ORACLE_TOL
    t0 = time.time()
    res = solver.solve(prob, fft="library")
    if res["status"] != "ok":
        raise RuntimeError(f"{name}: oracle {res['status']}")
    fin = res["final"]
    idx = FC.sample_voxels(prob)
    z, y, x = np.unravel_index(idx, (prob["n"][2], prob["n"][1], prob["n"][0]))
    out = {k: np.asarray(res[k]) for k in ("T", "M", "Eavg", "Gavg", "P", "Q", "Teq", "Meq", "err", "iters")}
    out["ref_moduli"] = np.asarray(res["ref_moduli"])
    out["sample"] = idx
    for k in ("e", "g", "t", "m", "p", "q"):
        out["sample_" + k] = fin[k][z, y, x]
        out["norm_" + k] = np.linalg.norm(fin[k])
    out["oracle_tol"] = FC.ORACLE_TOL
    path = os.path.join(HERE, f"free_running_{name}.npz")
    np.savez_compressed(path, **out)
    print(f"{name}: {int(np.sum(res['iters']))} iterations, {time.time() - t0:.0f} s -> {path}")


if __name__ == "__main__":
    for name in sys.argv[1:] or FC.CASES:
        write(name)
