"""Build-time checks of the CUDA kernels (no GPU needed: nvcc cross-compiles).

The tiled kernels take the opt-in shared-memory maximum minus a reserve for
their static shared memory (cell descriptor, reduction words); a kernel whose
static shared memory outgrew the reserve would make every launch fail with
'invalid argument'.  This compiles the kernels with ptxas' resource report
and checks each kernel's static shared memory against the reserve declared in
the source.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_10774_gb300", "csrc")


def _nvcc():
    return shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)


@pytest.mark.skipif(_nvcc() is None, reason="nvcc not available")
def test_static_shared_memory_fits_the_reserve(tmp_path):
    src = os.path.join(CSRC, "mp_kernels.cu")
    text = open(src).read()
    reserve = int(re.search(r"kSmemStaticReserve\s*=\s*(\d+)", text).group(1))
    out = subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                          "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v",
                          "-c", src, "-o", str(tmp_path / "k.o")], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr[-2000:]
    name, seen = None, {}
    for line in out.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and name:
            sm = re.search(r"(\d+) bytes smem", line)
            seen[name] = (int(m.group(1)), int(sm.group(1)) if sm else 0)
            name = None
    tiled = {k: v for k, v in seen.items() if re.search(r"k_(pass_a|fft_y|green_z)", k)}
    assert len(tiled) >= 20, sorted(seen)
    for k, (regs, smem) in tiled.items():
        assert smem <= reserve, (k, smem, reserve)
        assert regs <= 255, (k, regs)
