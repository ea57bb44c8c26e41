"""GB300-native micropolar elastoplastic FFT-based solver (sm_103a).

The solver of Francis, Lebensohn, Pourahmadian and Dingreville: the
FFT-based basic scheme with time stepping (their Algorithm 2) around the
closed-form micropolar radial return (their Algorithm 1), run entirely in
hand-written CUDA kernels behind the C ABI of ``include/micropolar.h``.
``binding`` is the thin Python layer over that ABI.
"""
from .binding import (  # noqa: F401
    Context,
    MicropolarError,
    Rve,
    Server,
    mp_abi_version,
    mp_batch_solve,
    mp_green_apply,
    mp_radial_return,
    mp_rve_create,
    mp_solve,
    mp_validate,
)

__all__ = ["Context", "MicropolarError", "Rve", "Server", "mp_abi_version", "mp_batch_solve",
           "mp_green_apply", "mp_radial_return", "mp_rve_create", "mp_solve", "mp_validate"]
