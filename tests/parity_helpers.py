"""Comparison of a GPU solve result with the oracle's (shared by the GPU test files)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def compare_solves(res, ref, tol_hom, tol_fields=None, h=1.0):
    """Homogenized results within tol_hom of the oracle, relative to each
    quantity's magnitude; couple-stress quantities are measured against
    max(|M|, h |T|) (a couple stress is a stress times a length), so that a
    load without curvature, whose M is pure rounding, is not compared to zero."""
    assert res["steps_done"] == len(ref["iters"])
    scaleT = max(np.abs(ref["T"]).max(), 1e-300)
    scaleM = max(np.abs(ref["M"]).max(), h * scaleT)
    assert np.abs(res["T"] - ref["T"]).max() <= tol_hom * scaleT
    assert np.abs(res["M"] - ref["M"]).max() <= tol_hom * scaleM
    # Q (a plastic curvature, 1 / length) is floored by its dimensional
    # partner P / h, as M is by h T
    scales = {"P": np.abs(ref["P"]).max(), "Q": max(np.abs(ref["Q"]).max(), np.abs(ref["P"]).max() / h),
              "Teq": np.abs(ref["Teq"]).max(), "Meq": max(np.abs(ref["Meq"]).max(), h * np.abs(ref["Teq"]).max())}
    for k, sc in scales.items():
        assert np.abs(res[k] - ref[k]).max() <= tol_hom * max(sc, 1e-300), k
    scaleE = np.abs(ref["Eavg"]).max()
    assert np.abs(res["Eavg"] - ref["Eavg"]).max() <= tol_hom * scaleE
    if tol_fields is not None:
        fin, rf = res["final"], ref["final"]
        for k in ("e", "t"):
            assert rel_l2(fin[k], rf[k]) <= tol_fields, k
        # curvature / couple stress against their dimensional partners
        for k, partner, f in (("g", "e", 1.0 / h), ("m", "t", h)):
            err = np.linalg.norm(fin[k] - rf[k])
            den = max(np.linalg.norm(rf[k]), f * np.linalg.norm(rf[partner]))
            assert err <= tol_fields * den, k

