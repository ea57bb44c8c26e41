"""The binding refuses device arguments whose size does not match the call,
before anything reaches the library (a short tensor would be read or written
out of bounds by the kernels).  Runs without a GPU: CPU tensors of the right
size are refused as well, for not being on the device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _binding():
    try:
        from paper_2409_10774_gb300 import binding as B
    except ImportError as exc:  # library not built
        pytest.skip(str(exc))
    return B


def test_green_apply_refuses_wrong_sizes():
    B = _binding()
    n = (4, 4, 2)
    good = torch.zeros((2, 4, 4, 3, 3), dtype=torch.float32)
    short = torch.zeros((2, 4, 3, 3, 3), dtype=torch.float32)
    for fn in (B.mp_green_apply, B.mp_green_apply_static):
        with pytest.raises(ValueError, match="elements"):
            fn(None, 1, n, 1.0, (1, 1, 1, 1, 1, 1), short, good)
        with pytest.raises(ValueError, match="elements"):
            fn(None, 1, n, 1.0, (1, 1, 1, 1, 1, 1), good, short)
        with pytest.raises(ValueError, match="dtype"):
            fn(None, 0, n, 1.0, (1, 1, 1, 1, 1, 1), good, good)
        with pytest.raises(ValueError, match="CUDA"):
            fn(None, 1, n, 1.0, (1, 1, 1, 1, 1, 1), good, good)
    with pytest.raises(ValueError, match="e_out"):
        B.mp_green_apply_static(None, 1, n, 1.0, (1, 1, 1, 1, 1, 1), good, good, e_out=short)


def test_radial_return_refuses_wrong_sizes():
    B = _binding()
    import workloads as W
    count = 5
    phases = W.phase_record([W.generators._matrix_row()])
    ph = torch.zeros(count, dtype=torch.int16)
    t9 = torch.zeros((count, 3, 3), dtype=torch.float32)
    s9 = torch.zeros((count - 1, 3, 3), dtype=torch.float32)
    pq = torch.zeros(count, dtype=torch.float64)
    with pytest.raises(ValueError, match="g_n"):
        B.mp_radial_return(None, 1, ph, phases, t9, t9, t9, s9, t9, t9, pq, pq)
    with pytest.raises(ValueError, match="q_n"):
        B.mp_radial_return(None, 1, ph, phases, t9, t9, t9, t9, t9, t9, pq, pq[:3])
    with pytest.raises(ValueError, match="phase"):
        B.mp_radial_return(None, 1, ph[:2], phases, t9, t9, t9, t9, t9, t9, pq, pq)
    with pytest.raises(ValueError, match="phase"):
        B.mp_radial_return(None, 1, ph.float(), phases, t9, t9, t9, t9, t9, t9, pq, pq)
    with pytest.raises(ValueError, match="CUDA"):
        B.mp_radial_return(None, 1, ph, phases, t9, t9, t9, t9, t9, t9, pq, pq)
