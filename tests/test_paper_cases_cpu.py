"""The inputs of the paper's experiments (workloads/paper_cases.py) against
the tables transcribed in tests/golden/tables.json (Tables 1-5) and the
stated geometries and load paths (Sec. 3.2-3.4, Appendix D.2)."""
import json
import os

import numpy as np
import pytest

from workloads import paper_cases as PC

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tables():
    return json.load(open(os.path.join(GOLDEN, "tables.json")))


def test_tables_match_the_transcription(tables):
    for key, ours in (("table1", PC.TABLE1), ("table2", PC.TABLE2), ("table4", PC.TABLE4),
                      ("table5", PC.TABLE5)):
        for phase, row in ours.items():
            assert list(row) == tables[key][phase], (key, phase)
    assert list(PC.TABLE5_X) == tables["table5"]["x"]
    cols = tables["table3"]["columns"]
    for phase in ("phase1", "phase2"):
        t = PC.TABLE3[phase]
        assert [t[c] for c in cols] == tables["table3"][phase]


def test_ratcheting_cycles():
    p = PC.workload_ratcheting(n_cycles=10)
    assert p["n"] == (4, 4, 4) and len(p["time"]) == 1001
    np.testing.assert_allclose(np.diff(p["time"]), 0.01)
    e12 = p["E"][:, 0, 1]
    # rate +1 for the first half of every one-second cycle, -1 for the second
    rates = np.diff(e12) / 0.01
    for c in range(10):
        np.testing.assert_allclose(rates[100 * c:100 * c + 50], 1.0)
        np.testing.assert_allclose(rates[100 * c + 50:100 * c + 100], -1.0)
    mask = np.ones((3, 3), bool); mask[0, 1] = False
    assert np.abs(p["E"][:, mask]).max() == 0.0 and np.abs(p["G"]).max() == 0.0
    assert p["phase"].mean() == 0.5
    # layers normal to x2: the phase depends on x2 only
    assert np.ptp(p["phase"], axis=(0, 2)).max() == 0 and np.ptp(p["phase"], axis=1).min() == 1


def test_length_scale_case():
    p = PC.workload_length_scales(0.25, 0.5)
    assert p["n"] == (16, 16, 16) and abs(p["phase"].mean() - 0.2) < 0.02
    r = p["phases"]
    assert np.allclose(r["mu"], r["gamma"] / 0.25 ** 2) and np.allclose(r["a1"], 1.5 * 0.5 ** 2)
    assert np.allclose(p["E"][-1][2, 1], 1.0) and np.allclose(p["G"][-1][0, 0], 1.0)


def test_hardening_case_clamps_beta():
    p = PC.workload_hardening_contrast(0.005)
    assert p["n"] == (8, 8, 8) and p["tol"] == 1e-8
    r = p["phases"]
    assert r[0]["beta"] == r[0]["gamma"] == 0.1
    assert r[1]["tH"] == r[1]["mH"] == 0.005
