"""ctypes binding of the C ABI declared in include/micropolar.h.

Argument marshalling only: every step of the solver runs in the CUDA kernels
of ``libmicropolar_gb300.so``.  Functions keep the C names (``mp_solve``,
``mp_rve_create``, ...) and take / return numpy arrays (host data) or torch
CUDA tensors (device data).  PyTorch supplies device memory (through the
library's allocator callbacks) and streams.  There is no CPU fallback: if the
library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

LIB_PATH = _build.LIB_PATH

# status codes (mp_status)
MP_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "inadmissible", 3: "unsupported_size",
                4: "not_converged", 5: "diverged", 6: "oom", 7: "cuda", 8: "timeout",
                9: "cancelled", 10: "no_device"}
ERR_KIND = {"local": 0, "average": 1}
REF_KIND = {"mean": 0, "midrange": 1, "explicit": 2}

EXPORTED = ("mp_abi_version", "mp_create", "mp_destroy", "mp_last_error", "mp_validate",
            "mp_solve", "mp_rve_create", "mp_rve_run", "mp_rve_results", "mp_rve_reset",
            "mp_rve_steps_done", "mp_rve_iterations", "mp_rve_destroy", "mp_rve_profile",
            "mp_rve_profile_read", "mp_radial_return", "mp_green_apply", "mp_green_apply_static",
            "mp_rve_trace", "mp_rve_trace_read", "mp_checkpoint", "mp_resume", "mp_batch_solve",
            "mp_server_create", "mp_server_submit", "mp_server_wait",
            "mp_server_query", "mp_server_destroy", "mp_set_autotune", "mp_rve_config")
MP_STATIC_SCRATCH_BYTES = 8 * 1024 * 1024
KERNEL_CLASSES = ("fft_y_fwd", "green_z", "fft_y_inv", "pass_a", "reduce", "start", "commit", "spectral")


class MicropolarError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class mp_phase(C.Structure):
    _fields_ = [(f, C.c_double) for f in ("lambda_", "mu", "kappa", "alpha", "beta", "gamma",
                                          "tY", "tH", "mY", "mH", "a1", "b1")] + \
               [("elastic", C.c_int32), ("reserved", C.c_int32)]


class mp_problem(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("h", C.c_double), ("phase", C.POINTER(C.c_uint16)),
                ("n_phases", C.c_int32), ("phases", C.POINTER(mp_phase)), ("n_steps", C.c_int32),
                ("time", C.POINTER(C.c_double)), ("E", C.POINTER(C.c_double)),
                ("G", C.POINTER(C.c_double)), ("tol", C.c_double), ("err_kind", C.c_int32),
                ("max_iter", C.c_int32), ("ref_kind", C.c_int32),
                ("ref_moduli", C.POINTER(C.c_double)), ("precision", C.c_int32),
                ("lockstep_iters", C.POINTER(C.c_int32)), ("div_limit", C.c_double),
                ("tau_m", C.POINTER(C.c_double)), ("mu_m", C.POINTER(C.c_double))]


_DP = C.POINTER(C.c_double)


class mp_result(C.Structure):
    _fields_ = [("T", _DP), ("M", _DP), ("Eavg", _DP), ("Gavg", _DP), ("P", _DP), ("Q", _DP),
                ("Teq", _DP), ("Meq", _DP), ("err", _DP), ("iters", C.POINTER(C.c_int32)),
                ("iters_fp64", C.POINTER(C.c_int32)),
                ("e", _DP), ("g", _DP), ("t", _DP), ("m", _DP), ("p", _DP), ("q", _DP),
                ("steps_done", C.c_int32), ("failed_step", C.c_int32),
                ("ref_moduli_used", C.c_double * 6)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class mp_alloc(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class mp_batch_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("rounds", "rounds_fp64", "voxel_iters", "voxel_iters_fp64",
                                         "escalations", "delta_switches")]


class mp_server_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_resident", C.c_int32), ("reserved", C.c_int32)]


class mp_server_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "completed", "queued", "resident", "peak_resident",
                                         "rounds", "voxel_iters")] + \
               [("budget_bytes", C.c_size_t), ("resident_bytes", C.c_size_t)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    V, P = C.c_void_p, C.POINTER
    sig = {
        "mp_abi_version": (C.c_int32, []),
        "mp_create": (C.c_int, [P(V), C.c_int32, P(mp_alloc)]),
        "mp_destroy": (None, [V]),
        "mp_last_error": (C.c_char_p, [V]),
        "mp_validate": (C.c_int, [P(mp_problem), C.c_char_p, C.c_size_t]),
        "mp_solve": (C.c_int, [V, P(mp_problem), P(mp_result), V]),
        "mp_rve_create": (C.c_int, [V, P(mp_problem), P(V), V]),
        "mp_rve_run": (C.c_int, [V, C.c_int32, V]),
        "mp_rve_results": (C.c_int, [V, P(mp_result), V]),
        "mp_rve_reset": (C.c_int, [V, V]),
        "mp_rve_steps_done": (C.c_int32, [V]),
        "mp_rve_iterations": (C.c_int64, [V]),
        "mp_rve_destroy": (None, [V]),
        "mp_rve_profile": (C.c_int, [V, C.c_int32]),
        "mp_rve_profile_read": (C.c_int, [V, P(C.c_double), P(C.c_int64), C.c_int32]),
        "mp_radial_return": (C.c_int, [V, C.c_int32, C.c_int64, V, C.c_int32, P(mp_phase)] + [V] * 6
                             + [V, V, V, V, V, V, V]),
        "mp_green_apply": (C.c_int, [V, C.c_int32, P(C.c_int32), C.c_double, P(C.c_double), V, V, V, V, V]),
        "mp_green_apply_static": (C.c_int, [V, C.c_int32, P(C.c_int32), C.c_double, P(C.c_double), V, V, V, V,
                                            V]),
        "mp_rve_trace": (C.c_int, [V, C.c_int32]),
        "mp_checkpoint": (C.c_int, [V, V, P(C.c_size_t), V]),
        "mp_resume": (C.c_int, [V, V, C.c_size_t, V]),
        "mp_rve_trace_read": (C.c_int64, [V, P(C.c_double), C.c_int64, C.c_int32]),
        "mp_batch_solve": (C.c_int, [V, P(P(mp_problem)), C.c_int32, P(mp_result), P(C.c_int), V,
                                     P(mp_batch_stats)]),
        "mp_server_create": (C.c_int, [V, P(mp_server_opts), P(V)]),
        "mp_server_submit": (C.c_int, [V, P(mp_problem), P(mp_result), P(C.c_uint64)]),
        "mp_server_wait": (C.c_int, [V, C.c_uint64, C.c_int32]),
        "mp_server_query": (C.c_int, [V, P(mp_server_stats)]),
        "mp_server_destroy": (None, [V]),
        "mp_set_autotune": (C.c_int, [V, C.c_int32]),
        "mp_rve_config": (C.c_int, [V, P(C.c_int32), C.c_int32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def last_error(ctx=None) -> str:
    msg = LIB.mp_last_error(ctx)
    return msg.decode() if msg else ""


# ---------------------------------------------------------------- marshalling helpers

def phase_table(phases) -> "C.Array":
    """numpy structured phase table (workloads.PHASE_FIELDS) -> mp_phase[]."""
    arr = (mp_phase * len(phases))()
    for i, r in enumerate(phases):
        arr[i] = mp_phase(float(r["lambda"]), float(r["mu"]), float(r["kappa"]), float(r["alpha"]),
                          float(r["beta"]), float(r["gamma"]), float(r["tY"]), float(r["tH"]),
                          float(r["mY"]), float(r["mH"]), float(r["a1"]), float(r["b1"]),
                          int(r["elastic"]), 0)
    return arr


def _dptr(a):
    return a.ctypes.data_as(_DP)


class _Problem:
    """Keeps the host arrays of an mp_problem alive while it is in use."""

    def __init__(self, problem, precision=None, lockstep_iters=None, div_limit=0.0):
        p = problem
        n = tuple(int(v) for v in p["n"])
        self.phase = np.ascontiguousarray(p["phase"], dtype=np.uint16).reshape(-1)
        if self.phase.size != n[0] * n[1] * n[2]:
            raise ValueError("phase map size does not match n")
        self.phases = phase_table(p["phases"])
        self.time = np.ascontiguousarray(p["time"], dtype=np.float64)
        n_steps = self.time.size - 1
        self.E = np.ascontiguousarray(np.asarray(p["E"], dtype=np.float64).reshape(n_steps + 1, 9))
        self.G = np.ascontiguousarray(np.asarray(p["G"], dtype=np.float64).reshape(n_steps + 1, 9))
        self.ref = None
        if p.get("ref_moduli") is not None:
            self.ref = np.ascontiguousarray(p["ref_moduli"], dtype=np.float64)
        # manufactured source (both or neither; the library checks the pairing)
        self.tau_m = self.mu_m = None
        nel = (n_steps + 1) * n[0] * n[1] * n[2] * 9
        for key in ("tau_m", "mu_m"):
            if p.get(key) is not None:
                arr = np.ascontiguousarray(p[key], dtype=np.float64).reshape(-1)
                if arr.size != nel:
                    raise ValueError(f"{key} must hold (n_steps + 1) * N1*N2*N3 * 9 values")
                setattr(self, key, arr)
        self.lock = None
        if lockstep_iters is not None:
            self.lock = np.ascontiguousarray(lockstep_iters, dtype=np.int32)
        prec = p.get("precision", 1) if precision is None else precision
        self.st = mp_problem()
        self.st.n = (C.c_int32 * 3)(*n)
        self.st.h = float(p["h"])
        self.st.phase = self.phase.ctypes.data_as(C.POINTER(C.c_uint16))
        self.st.n_phases = len(p["phases"])
        self.st.phases = self.phases
        self.st.n_steps = n_steps
        self.st.time = _dptr(self.time)
        self.st.E = _dptr(self.E)
        self.st.G = _dptr(self.G)
        self.st.tol = float(p["tol"])
        self.st.err_kind = ERR_KIND[p.get("err_kind", "local")]
        self.st.max_iter = int(p.get("max_iter", 10000))
        self.st.ref_kind = REF_KIND[p.get("ref_kind", "mean")]
        self.st.ref_moduli = _dptr(self.ref) if self.ref is not None else None
        self.st.precision = int(prec)
        self.st.lockstep_iters = self.lock.ctypes.data_as(C.POINTER(C.c_int32)) if self.lock is not None else None
        self.st.div_limit = float(div_limit)
        self.st.tau_m = _dptr(self.tau_m) if self.tau_m is not None else None
        self.st.mu_m = _dptr(self.mu_m) if self.mu_m is not None else None
        self.n = n
        self.n_steps = n_steps


class _Result:
    def __init__(self, n, n_steps, fields):
        ns = max(n_steps, 1)
        nv = n[0] * n[1] * n[2]
        self.arrs = {k: np.zeros((ns, 9)) for k in ("T", "M", "Eavg", "Gavg")}
        self.arrs.update({k: np.zeros(ns) for k in ("P", "Q", "Teq", "Meq", "err")})
        self.iters = np.zeros(ns, dtype=np.int32)
        self.iters64 = np.zeros(ns, dtype=np.int32)
        self.fields = {}
        if fields:
            self.fields = {k: np.zeros((nv, 9)) for k in ("e", "g", "t", "m")}
            self.fields.update({k: np.zeros(nv) for k in ("p", "q")})
        self.st = mp_result()
        for k, a in self.arrs.items():
            setattr(self.st, k, _dptr(a))
        self.st.iters = self.iters.ctypes.data_as(C.POINTER(C.c_int32))
        self.st.iters_fp64 = self.iters64.ctypes.data_as(C.POINTER(C.c_int32))
        for k, a in self.fields.items():
            setattr(self.st, k, _dptr(a))
        self.n = n

    def to_dict(self, status):
        ns = self.st.steps_done
        out = {k: v[:ns].copy() for k, v in self.arrs.items()}
        for k in ("T", "M", "Eavg", "Gavg"):
            out[k] = out[k].reshape(ns, 3, 3)
        out["iters"] = self.iters[:ns].astype(np.int64)
        out["iters_fp64"] = self.iters64[:ns].astype(np.int64)
        out["steps_done"] = ns
        out["failed_step"] = self.st.failed_step
        out["ref_moduli"] = tuple(self.st.ref_moduli_used)
        out["status"] = STATUS_NAMES.get(status, str(status))
        n = self.n
        if self.fields and ns > 0:
            fin = {}
            for k in ("e", "g", "t", "m"):
                fin[k] = self.fields[k].reshape(n[2], n[1], n[0], 3, 3)
            for k in ("p", "q"):
                fin[k] = self.fields[k].reshape(n[2], n[1], n[0])
            out["final"] = fin
        return out


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# ---------------------------------------------------------------- context

class Context:
    """mp_create / mp_destroy with PyTorch's caching allocator as device memory."""

    def __init__(self, device=0, use_torch_allocator=True):
        self.device = int(device)
        self._alloc = None
        ptr = C.c_void_p()
        alloc_p = None
        if use_torch_allocator:
            import torch

            dev = self.device

            def _a(nbytes, user):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev))
                except RuntimeError:
                    return 0

            def _f(p, nbytes, user):
                torch.cuda.caching_allocator_delete(int(p))

            self._afn = ALLOC_FN(_a)
            self._ffn = FREE_FN(_f)
            self._alloc = mp_alloc(self._afn, self._ffn, None)
            alloc_p = C.byref(self._alloc)
        st = LIB.mp_create(C.byref(ptr), self.device, alloc_p)
        if st != MP_OK:
            raise MicropolarError(st, last_error(None))
        self.ptr = ptr

    def close(self):
        if getattr(self, "ptr", None):
            LIB.mp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self):
        return last_error(self.ptr)

    def set_autotune(self, enable=True):
        """mp_set_autotune: time candidate launch schedules for new cell shapes."""
        st = LIB.mp_set_autotune(self.ptr, 1 if enable else 0)
        if st != MP_OK:
            raise MicropolarError(st, self.error())


# ---------------------------------------------------------------- entry points

def mp_abi_version():
    return LIB.mp_abi_version()


def mp_validate(problem, precision=None):
    pr = _Problem(problem, precision)
    buf = C.create_string_buffer(512)
    st = LIB.mp_validate(C.byref(pr.st), buf, 512)
    return st, buf.value.decode()


_HARD_ERRORS = (1, 2, 3, 6, 7, 8, 9, 10)


def mp_solve(ctx, problem, precision=None, fields=False, lockstep_iters=None, div_limit=0.0,
             stream=None):
    """Whole solve; returns a dict shaped like the oracle's result (per-step
    arrays, 'final' fields when requested, 'status')."""
    pr = _Problem(problem, precision, lockstep_iters, div_limit)
    rs = _Result(pr.n, pr.n_steps, fields)
    st = LIB.mp_solve(ctx.ptr, C.byref(pr.st), C.byref(rs.st), _stream_handle(stream))
    if st in _HARD_ERRORS:
        raise MicropolarError(st, ctx.error())
    return rs.to_dict(st)


class Rve:
    """Device-resident cell: mp_rve_create / run / results / reset / destroy."""

    def __init__(self, ctx, problem, precision=None, lockstep_iters=None, div_limit=0.0, stream=None):
        self.ctx = ctx
        self._pr = _Problem(problem, precision, lockstep_iters, div_limit)
        self.ptr = C.c_void_p()
        st = LIB.mp_rve_create(ctx.ptr, C.byref(self._pr.st), C.byref(self.ptr), _stream_handle(stream))
        if st != MP_OK:
            raise MicropolarError(st, ctx.error())

    def run(self, n_steps, stream=None):
        st = LIB.mp_rve_run(self.ptr, int(n_steps), _stream_handle(stream))
        if st in _HARD_ERRORS:
            raise MicropolarError(st, self.ctx.error())
        self._run_status = st
        return st

    def results(self, fields=False, stream=None):
        rs = _Result(self._pr.n, self._pr.n_steps, fields)
        st = LIB.mp_rve_results(self.ptr, C.byref(rs.st), _stream_handle(stream))
        if st != MP_OK:
            raise MicropolarError(st, self.ctx.error())
        return rs.to_dict(MP_OK if rs.st.failed_step == 0 else getattr(self, "_run_status", 4))

    def reset(self, stream=None):
        LIB.mp_rve_reset(self.ptr, _stream_handle(stream))

    def profile(self, enable=True):
        st = LIB.mp_rve_profile(self.ptr, 1 if enable else 0)
        if st != MP_OK:
            raise MicropolarError(st, self.ctx.error())

    def profile_read(self, reset=False):
        """{kernel class: (milliseconds, launches)}."""
        k = len(KERNEL_CLASSES)
        ms = (C.c_double * k)()
        ln = (C.c_int64 * k)()
        LIB.mp_rve_profile_read(self.ptr, ms, ln, 1 if reset else 0)
        return {name: (ms[i], ln[i]) for i, name in enumerate(KERNEL_CLASSES)}

    def checkpoint(self, stream=None):
        """The cell's committed state as bytes (mp_checkpoint)."""
        n = C.c_size_t(0)
        st = LIB.mp_checkpoint(self.ptr, None, C.byref(n), _stream_handle(stream))
        if st != MP_OK:
            raise MicropolarError(st, self.ctx.error())
        buf = C.create_string_buffer(n.value)
        st = LIB.mp_checkpoint(self.ptr, buf, C.byref(n), _stream_handle(stream))
        if st != MP_OK:
            raise MicropolarError(st, self.ctx.error())
        return buf.raw[: n.value]

    def resume(self, image, stream=None):
        """Load a checkpoint image taken from a cell of the same problem (mp_resume)."""
        buf = C.create_string_buffer(bytes(image), len(image))
        st = LIB.mp_resume(self.ptr, buf, len(image), _stream_handle(stream))
        if st != MP_OK:
            raise MicropolarError(st, self.ctx.error())

    def trace(self, enable=True):
        """Record (increment, iteration, err, err_e, err_t, err_gamma, err_m) per iteration."""
        st = LIB.mp_rve_trace(self.ptr, 1 if enable else 0)
        if st != MP_OK:
            raise MicropolarError(st, self.ctx.error())

    def trace_read(self, clear=True):
        n = LIB.mp_rve_trace_read(self.ptr, None, 0, 0)
        buf = np.zeros((max(n, 1), 7))
        LIB.mp_rve_trace_read(self.ptr, buf.ctypes.data_as(_DP), n, 1 if clear else 0)
        return buf[:n]

    def config(self):
        """The cell's launch schedule (mp_rve_config)."""
        cfg = (C.c_int32 * 6)()
        LIB.mp_rve_config(self.ptr, cfg, 6)
        return {"rows_per_item": cfg[0], "fused_spectral": bool(cfg[1]), "grid_a": cfg[2], "grid_y": cfg[3],
                "grid_z": cfg[4], "tuned": bool(cfg[5])}

    @property
    def steps_done(self):
        return LIB.mp_rve_steps_done(self.ptr)

    @property
    def iterations(self):
        return LIB.mp_rve_iterations(self.ptr)

    def close(self):
        if getattr(self, "ptr", None):
            LIB.mp_rve_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp_rve_create(ctx, problem, precision=None, lockstep_iters=None, div_limit=0.0, stream=None):
    return Rve(ctx, problem, precision, lockstep_iters, div_limit, stream)


def _real(precision):
    import torch
    return torch.float64 if precision == 0 else torch.float32


def _check_dev(specs):
    """Device pointers of the tensors in `specs` = [(tensor, dtype, numel,
    name), ...] after checking everything the kernels rely on: each is a
    contiguous CUDA tensor of its dtype holding exactly `numel` elements (the
    kernels read and write that many, so a shorter tensor would be accessed
    out of bounds).  Sizes and dtypes of all arguments are checked before
    their placement."""
    import torch
    for t, dtype, numel, name in specs:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name}: expected a torch tensor")
        if t.numel() != numel:
            raise ValueError(f"{name}: expected {numel} elements, got {t.numel()} (shape {tuple(t.shape)})")
        if dtype is not None and t.dtype != dtype:
            raise ValueError(f"{name}: expected dtype {dtype}, got {t.dtype}")
    for t, _, _, name in specs:
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous CUDA tensor")
    return [C.c_void_p(t.data_ptr()) for t, _, _, _ in specs]


def mp_radial_return(ctx, precision, phase, phases, e, g, e_n, g_n, t_n, m_n, p_n, q_n, stream=None):
    """Algorithm 1 on device tensors (count, 3, 3) of the precision's real type;
    phase: uint16-valued int32/int16 CUDA tensor is converted to a uint16 view
    when given as torch.int16; p_n, q_n float64.  Returns (t, m, p, q)."""
    import torch
    R = _real(precision)
    count = int(e.shape[0])
    if not isinstance(phase, torch.Tensor) or phase.is_floating_point() or phase.element_size() != 2:
        raise ValueError("phase: expected a 16-bit integer tensor")
    ptrs = _check_dev([(phase, None, count, "phase")]
                      + [(x, R, 9 * count, nm) for x, nm in ((e, "e"), (g, "g"), (e_n, "e_n"), (g_n, "g_n"),
                                                             (t_n, "t_n"), (m_n, "m_n"))]
                      + [(x, torch.float64, count, nm) for x, nm in ((p_n, "p_n"), (q_n, "q_n"))])
    ph_ptr, args, pq = ptrs[0], ptrs[1:7], ptrs[7:9]
    ph = phase_table(phases)
    t = torch.empty_like(e)
    m = torch.empty_like(g)
    p = torch.empty(count, dtype=torch.float64, device=e.device)
    q = torch.empty(count, dtype=torch.float64, device=e.device)
    st = LIB.mp_radial_return(ctx.ptr, int(precision), int(count), ph_ptr,
                              len(phases), ph, *args, *pq, C.c_void_p(t.data_ptr()),
                              C.c_void_p(m.data_ptr()), C.c_void_p(p.data_ptr()),
                              C.c_void_p(q.data_ptr()), _stream_handle(stream))
    if st != MP_OK:
        raise MicropolarError(st, ctx.error())
    return t, m, p, q


def mp_green_apply(ctx, precision, n, h, ref_moduli, tau, mu, stream=None):
    """Fluctuations (e~, gamma~) of the polarization fields tau, mu: device
    tensors (N3, N2, N1, 3, 3) of the precision's real type."""
    R = _real(precision)
    nel = 9 * int(n[0]) * int(n[1]) * int(n[2])
    ptau, pmu = _check_dev([(tau, R, nel, "tau"), (mu, R, nel, "mu")])
    import torch
    e = torch.empty_like(tau)
    g = torch.empty_like(mu)
    nn = (C.c_int32 * 3)(*[int(v) for v in n])
    ref = (C.c_double * 6)(*[float(v) for v in ref_moduli])
    st = LIB.mp_green_apply(ctx.ptr, int(precision), nn, float(h), ref, ptau, pmu,
                            C.c_void_p(e.data_ptr()), C.c_void_p(g.data_ptr()), _stream_handle(stream))
    if st != MP_OK:
        raise MicropolarError(st, ctx.error())
    return e, g


def mp_green_apply_static(ctx, precision, n, h, ref_moduli, tau, mu, e_out=None, g_out=None,
                          stream=None):
    """Same result as mp_green_apply, computed without any device allocation
    inside the library (its scratch is a static device array of
    MP_STATIC_SCRATCH_BYTES).  The caller passes the output tensors; when they
    are omitted this wrapper allocates them with torch before the call."""
    R = _real(precision)
    nel = 9 * int(n[0]) * int(n[1]) * int(n[2])
    import torch
    if e_out is None:
        e_out = torch.empty_like(tau)
    if g_out is None:
        g_out = torch.empty_like(mu)
    ptau, pmu, pe, pg = _check_dev([(tau, R, nel, "tau"), (mu, R, nel, "mu"), (e_out, R, nel, "e_out"),
                                    (g_out, R, nel, "g_out")])
    nn = (C.c_int32 * 3)(*[int(v) for v in n])
    ref = (C.c_double * 6)(*[float(v) for v in ref_moduli])
    st = LIB.mp_green_apply_static(ctx.ptr, int(precision), nn, float(h), ref, ptau, pmu, pe, pg,
                                   _stream_handle(stream))
    if st != MP_OK:
        raise MicropolarError(st, ctx.error())
    return e_out, g_out


# ---------------------------------------------------------------- batched solves and serving

def _per_item(value, count):
    if isinstance(value, (list, tuple)):
        if len(value) != count:
            raise ValueError("per-problem argument list has the wrong length")
        return list(value)
    return [value] * count


def mp_batch_solve(ctx, problems, precision=None, fields=False, lockstep_iters=None, div_limit=0.0,
                   stream=None, stats=None):
    """Solve many cells together (mp_batch_solve).  `precision`, `fields`,
    `lockstep_iters` and `div_limit` are one value for all problems or a list
    with one entry per problem.  Returns one result dict per problem, shaped
    like mp_solve's, each with its own 'status'; a dict passed as `stats`
    receives the call's work counters."""
    count = len(problems)
    precs = _per_item(precision, count)
    fl = _per_item(fields, count)
    locks = lockstep_iters if (isinstance(lockstep_iters, (list, tuple)) and lockstep_iters
                               and not np.isscalar(lockstep_iters[0])) else [lockstep_iters] * count
    divs = _per_item(div_limit, count)
    prs = [_Problem(p, precs[i], locks[i], divs[i]) for i, p in enumerate(problems)]
    rss = [_Result(pr.n, pr.n_steps, fl[i]) for i, pr in enumerate(prs)]
    parr = (C.POINTER(mp_problem) * max(count, 1))(*[C.pointer(pr.st) for pr in prs])
    rarr = (mp_result * max(count, 1))()
    for i, rs in enumerate(rss):
        rarr[i] = rs.st
    status = (C.c_int * max(count, 1))()
    bst = mp_batch_stats()
    st = LIB.mp_batch_solve(ctx.ptr, parr, count, rarr, status, _stream_handle(stream), C.byref(bst))
    if stats is not None:
        stats.update({k: getattr(bst, k) for k, _ in mp_batch_stats._fields_})
    if st == 1 and count and all(status[i] == 0 for i in range(count)):
        raise MicropolarError(st, ctx.error())
    out = []
    for i, rs in enumerate(rss):
        rs.st = rarr[i]
        out.append(rs.to_dict(status[i]))
    return out


class Server:
    """mp_server_*: continuous-batching solve server on one device."""

    def __init__(self, ctx, budget_bytes=0, max_resident=0):
        self.ctx = ctx
        opts = mp_server_opts(int(budget_bytes), int(max_resident), 0)
        self.ptr = C.c_void_p()
        st = LIB.mp_server_create(ctx.ptr, C.byref(opts), C.byref(self.ptr))
        if st != MP_OK:
            raise MicropolarError(st, ctx.error())
        self._pending = {}

    def submit(self, problem, precision=None, fields=False, lockstep_iters=None, div_limit=0.0):
        pr = _Problem(problem, precision, lockstep_iters, div_limit)
        rs = _Result(pr.n, pr.n_steps, fields)
        ticket = C.c_uint64()
        st = LIB.mp_server_submit(self.ptr, C.byref(pr.st), C.byref(rs.st), C.byref(ticket))
        if st != MP_OK:
            raise MicropolarError(st, last_error(None))
        self._pending[ticket.value] = rs
        return ticket.value

    def wait(self, ticket, timeout_ms=-1):
        """Result dict of `ticket` (its 'status' names the outcome); raises
        MicropolarError(MP_E_TIMEOUT) when it has not ended in time."""
        st = LIB.mp_server_wait(self.ptr, C.c_uint64(ticket), int(timeout_ms))
        if st == 8 and ticket in self._pending:
            # either the wait expired or the solve itself timed out on the device
            msg = last_error(None)
            if "not finished within" in msg:
                raise MicropolarError(st, msg)
        if st == 1:
            raise MicropolarError(st, last_error(None))
        rs = self._pending.pop(ticket)
        return rs.to_dict(st)

    def stats(self):
        s = mp_server_stats()
        LIB.mp_server_query(self.ptr, C.byref(s))
        return {k: getattr(s, k) for k, _ in mp_server_stats._fields_}

    def close(self):
        if self.ptr:
            LIB.mp_server_destroy(self.ptr)
            self.ptr = C.c_void_p()
            self._pending.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
