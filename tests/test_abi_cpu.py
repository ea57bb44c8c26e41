"""CPU-side checks of the C ABI library: it builds, loads, exports every symbol
declared in include/micropolar.h, validates problems without a GPU, and
refuses to compute without one (no CPU fallback)."""
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "micropolar.h")


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._build_module().build()


def _declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:mp_status|void|int32_t|int64_t|const char\*)\s+(mp_\w+)\s*\(",
                                 src, flags=re.M)))


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (mp_\w+)$", out, flags=re.M))
    declared = _declared_symbols()
    assert len(declared) >= 15
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    from paper_2409_10774_gb300 import binding
    assert set(binding.EXPORTED) == set(declared)


def test_binding_loads_and_reports_version(lib_path):
    import paper_2409_10774_gb300 as M
    assert M.mp_abi_version() == 2


def test_validation_without_gpu(lib_path):
    import paper_2409_10774_gb300 as M
    p = W.workload_centered_sphere()
    assert M.mp_validate(p)[0] == 0
    # unsupported size (a prime factor 5)
    q = dict(p)
    q["n"] = (10, 16, 16)
    q["phase"] = np.zeros((16, 16, 10), np.uint16)
    assert M.mp_validate(q)[0] == 3
    # gamma < beta violates the energetic bounds (eq. energetic_bounds)
    ph = p["phases"].copy()
    ph[0]["beta"] = 2.0
    assert M.mp_validate(dict(p, phases=ph))[0] == 2
    # zero yield stress is rejected (0/0 in the return factor)
    ph = p["phases"].copy()
    ph[0]["tY"] = 0.0
    assert M.mp_validate(dict(p, phases=ph))[0] == 1
    # phase id out of range
    pm = p["phase"].copy()
    pm[0, 0, 0] = 7
    assert M.mp_validate(dict(p, phase=pm))[0] == 1
    # non-increasing time
    t = p["time"].copy()
    t[3] = t[2]
    assert M.mp_validate(dict(p, time=t))[0] == 1
    # gamma == beta is admitted (the skew couple stress then vanishes)
    assert (p["phases"]["beta"] == p["phases"]["gamma"]).all()
    # a manufactured source needs both its fields, finite
    nsrc = np.zeros((len(p["time"]),) + p["phase"].shape + (3, 3))
    assert M.mp_validate(dict(p, tau_m=nsrc, mu_m=nsrc))[0] == 0
    st, msg = M.mp_validate(dict(p, tau_m=nsrc))
    assert st == 1 and "together" in msg
    bad = nsrc.copy()
    bad[2, 0, 0, 0, 1, 1] = np.nan
    assert M.mp_validate(dict(p, tau_m=nsrc, mu_m=bad))[0] == 1
    # precision 0, 1 and 2 are the accepted arithmetics
    assert M.mp_validate(p, precision=2)[0] == 0
    assert M.mp_validate(p, precision=3)[0] == 1


def test_no_cpu_fallback(lib_path):
    import torch
    import paper_2409_10774_gb300 as M
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(M.MicropolarError) as ei:
        M.Context(use_torch_allocator=False)
    assert ei.value.status == 10
