"""ctypes binding of the C ABI in include/mcmg.h (argument marshalling only).

Every computation runs in the CUDA library ``libmcmg.so`` built in-tree by
``build.py``; this module only converts Python / numpy / torch arguments into
plain pointers and sizes.  There is no CPU fallback: ``load()`` raises when
the library is missing.

Device buffers are torch tensors on the CUDA device (complex64 for
single-precision fields, complex128 for the solve's f and u); host buffers are
numpy arrays or CPU tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmcmg.so")

MAX_LEVELS = 8
MCMG_OK, MCMG_PENDING = 0, 1
MCMG_ERR_SHAPE = -2
STATUS = {0: "OK", 1: "PENDING", -1: "ERR_ARG", -2: "ERR_SHAPE", -3: "ERR_OOM", -4: "ERR_CUDA",
          -5: "ERR_NOT_CONVERGED", -6: "ERR_TIMEOUT", -7: "ERR_NUMERIC", -8: "ERR_BUSY"}
FP32, BF16, FP32_TC = 0, 1, 2   # mcmg_precision
SOLVE_STATIONARY = 1
SOLVE_BORN = 2


class McmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Medium(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("c", C.POINTER(C.c_double)),
                ("sponge_width", C.c_int), ("gamma_max", C.c_double)]


class Weights(C.Structure):
    _fields_ = [("levels", C.c_int), ("channels", C.c_int * MAX_LEVELS),
                ("nu_pre", C.c_int * MAX_LEVELS), ("nu_post", C.c_int * MAX_LEVELS),
                ("feat_sl", C.c_double), ("feat_eps", C.c_double),
                ("sl_shift_re", C.c_double), ("sl_shift_im", C.c_double),
                ("precision", C.c_int), ("blob", C.POINTER(C.c_double)), ("blob_len", C.c_size_t)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart_m", C.c_int), ("max_iters", C.c_int),
                ("nrhs", C.c_int), ("flags", C.c_int), ("stream", C.c_void_p)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("rel_residual", C.c_double),
                ("t_solve_s", C.c_double), ("converged", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_SIGS = {
    "mcmg_ctx_create": [C.c_int, C.c_size_t, C.POINTER(_P)],
    "mcmg_ctx_destroy": [_P],
    "mcmg_ctx_memory": [_P, C.POINTER(C.c_size_t)],
    "mcmg_setup": [_P, C.POINTER(Medium), C.c_double, C.POINTER(Weights), C.POINTER(_P)],
    "mcmg_destroy": [_P],
    "mcmg_vcycle": [_P, _P, _P, C.c_int, _P],
    "mcmg_solve": [_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveInfo)],
    "mcmg_solve_host": [_P, _P, _P, C.POINTER(SolveOpts), C.POINTER(SolveInfo)],
    "mcmg_submit": [_P, _P, _P, _P, C.POINTER(SolveOpts), C.POINTER(C.c_uint64)],
    "mcmg_poll": [_P, C.c_uint64, C.POINTER(SolveInfo)],
    "mcmg_drain": [_P],
    "mcmg_apply_A": [_P, _P, _P, C.c_int, C.c_int, _P],
    "mcmg_device_error": [_P, C.POINTER(C.c_int)],
    "mcmg_get_feature": [_P, C.c_int, C.c_int, _P],
    "mcmg_lift": [_P, _P, _P, C.c_int, _P],
    "mcmg_project": [_P, _P, _P, C.c_int, _P],
    "mcmg_smooth": [_P, C.c_int, C.c_int, _P, _P, _P, C.c_int, _P],
    "mcmg_residual": [_P, C.c_int, _P, _P, _P, C.c_int, _P],
    "mcmg_residual_restrict": [_P, C.c_int, _P, _P, _P, C.c_int, _P],
    "mcmg_prolong_add": [_P, C.c_int, _P, _P, C.c_int, _P],
    "mcmg_coarse_basis": [_P, C.c_int, C.c_longlong, C.c_int, _P, _P],
    "mcmg_apply_G": [_P, _P, _P],
    "mcmg_cgs2": [_P, _P, C.c_int, C.c_size_t, _P, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "mcmg_cgs2_noalloc": [_P, C.c_int, C.c_size_t, _P, C.POINTER(C.c_double),
                          C.POINTER(C.c_double), _P],
    "mcmg_server_batching": [_P, C.c_int, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)],
    "mcmg_kernel_shape_count": [C.c_int],
    "mcmg_get_kernel_shape": [_P, C.c_int, C.c_int, C.POINTER(C.c_int)],
    "mcmg_set_kernel_shape": [_P, C.c_int, C.c_int, C.c_int],
    "mcmg_fp32_ffma_tflops": [_P, C.POINTER(C.c_double)],
    "mcmg_kernel_launches": [],
    "mcmg_last_error": [],
    "mcmg_version": [],
}

_lib = None


def declared_symbols():
    """Entry points declared in include/mcmg.h (parsed from the header text)."""
    import re
    hdr = os.path.join(os.path.dirname(HERE), "include", "mcmg.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"\b(mcmg_[A-Za-z0-9_]+)\s*\(", txt)))


def load(path: str = LIB_PATH):
    """Load libmcmg.so and declare every entry point.  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} not built; run paper_2606_30495_b300/build.py")
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        if name in ("mcmg_last_error", "mcmg_version"):
            fn.restype = C.c_char_p
        elif name == "mcmg_kernel_launches":
            fn.restype = C.c_uint64
        else:
            fn.restype = C.c_int
    _lib = lib
    return lib


def _check(st):
    if st not in (MCMG_OK,):
        raise McmgError(st, _lib.mcmg_last_error().decode())
    return st


def ptr(t) -> int:
    """Data pointer of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


# operations with interchangeable kernel shapes
OP_SMOOTH, OP_RESIDUAL, OP_RESTRICT, OP_PROLONG = 0, 1, 2, 3


def kernel_shape_count(op: int) -> int:
    return int(load().mcmg_kernel_shape_count(op))


def kernel_launches() -> int:
    return int(load().mcmg_kernel_launches())


def _stream(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


# ---------------------------------------------------------------- weights ---

def pack_weights(w: dict):
    """Pack a weight dict (layout of inputs.make_weights) into the float64 blob
    order of mcmg.h.  Returns (Weights struct, blob) -- keep both alive."""
    parts = []

    def real(a):
        parts.append(np.ascontiguousarray(a, dtype=np.float64).reshape(-1))

    def cplx(a):
        a = np.ascontiguousarray(a, dtype=np.complex128)
        parts.append(a.view(np.float64).reshape(-1))

    L = w["levels"]
    real(w["flift_w"]); real(w["flift_b"])
    for l in range(L):
        lv = w["lvl"][l]
        cplx(lv["W"]); cplx(lv["KA"]); cplx(lv["KS"]); cplx(lv["Wsm"])
        real(lv["fs_w"]); real(lv["fs_b"])
        if l < L - 1:
            cplx(lv["R"]); cplx(lv["P"]); real(lv["fa_w"]); real(lv["fa_b"])
    cplx(w["lift"]); cplx(w["proj"])
    blob = np.concatenate(parts)
    s = Weights()
    s.levels = L
    for l in range(L):
        s.channels[l] = w["channels"][l]
        s.nu_pre[l] = w["nu_pre"][l]
        s.nu_post[l] = w["nu_post"][l]
    s.feat_sl = w["feat_sl"]
    s.feat_eps = w["feat_eps"]
    s.sl_shift_re, s.sl_shift_im = w["sl_shift"]
    s.precision = w.get("precision", FP32)
    s.blob = blob.ctypes.data_as(C.POINTER(C.c_double))
    s.blob_len = blob.size
    return s, blob


# ---------------------------------------------------------------- objects ---

def fp32_ffma_tflops(stream=None) -> float:
    """Measured FP32 FFMA rate of the current device (TFLOP/s)."""
    v = C.c_double()
    _check(load().mcmg_fp32_ffma_tflops(_stream(stream), C.byref(v)))
    return v.value


def cgs2_noalloc(V, w, stream=None):
    """mcmg_cgs2_noalloc: CGS2 of w against the rows of V with no device
    allocation (scratch in a static device array).  Returns (h, ||w||)."""
    import torch
    lib = load()
    if V.dim() != 2 or not V.is_cuda or not w.is_cuda or V.device != w.device:
        raise ValueError("V ([k][n]) and w ([n]) must be CUDA tensors on one device")
    if V.dtype != torch.complex64 or w.dtype != torch.complex64:
        raise ValueError("V and w must be complex64")
    if not V.is_contiguous() or not w.is_contiguous():
        raise ValueError("V and w must be contiguous")
    k, n = V.shape[0], V.shape[1]
    if w.numel() != n:
        raise ValueError(f"w has {w.numel()} elements, V's rows have {n}")
    hbuf = np.zeros(2 * k)
    nrm = C.c_double()
    with torch.cuda.device(V.device):
        _check(lib.mcmg_cgs2_noalloc(ptr(V), k, n, ptr(w),
                                     hbuf.ctypes.data_as(C.POINTER(C.c_double)), C.byref(nrm),
                                     _stream(stream)))
    return hbuf.view(np.complex128), nrm.value


class Context:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = load()
        self.h = _P()
        _check(self.lib.mcmg_ctx_create(device, hbm_budget_bytes, C.byref(self.h)))

    def memory(self) -> int:
        v = C.c_size_t()
        _check(self.lib.mcmg_ctx_memory(self.h, C.byref(v)))
        return v.value

    def submit(self, handle, f, u, tol=1e-6, restart_m=20, max_iters=0, nrhs=1, flags=0,
               stream=None) -> int:
        """Queue a solve; it reads f and u after the work enqueued so far on
        `stream` (default: torch's current stream), which wrote them."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        o = SolveOpts(tol, restart_m, max_iters, nrhs, flags, _stream(stream))
        t = C.c_uint64()
        _check(self.lib.mcmg_submit(self.h, handle.h, ptr(f), ptr(u), C.byref(o), C.byref(t)))
        return t.value

    def batching(self, enable=None):
        """Switch cross-request batching (True / False, None: unchanged);
        returns (cohort V-cycles run, requests they held)."""
        r, m = C.c_uint64(), C.c_uint64()
        e = -1 if enable is None else int(bool(enable))
        _check(self.lib.mcmg_server_batching(self.h, e, C.byref(r), C.byref(m)))
        return r.value, m.value

    def poll(self, ticket: int):
        """(status, info dict); status MCMG_PENDING while running."""
        info = SolveInfo()
        st = self.lib.mcmg_poll(self.h, ticket, C.byref(info))
        if st < 0 and st not in (-5, -7):
            raise McmgError(st, self.lib.mcmg_last_error().decode())
        return st, info.as_dict()

    def drain(self):
        _check(self.lib.mcmg_drain(self.h))

    def close(self):
        if self.h:
            self.lib.mcmg_ctx_destroy(self.h)
            self.h = _P()


class Handle:
    """One medium set up with one weight set (Algorithm 1 run on the device)."""

    def __init__(self, ctx: Context, c: np.ndarray, omega: float, sponge_width: int,
                 gamma_max: float, weights: dict, precision: int = FP32):
        self.ctx = ctx
        self.lib = ctx.lib
        c = np.ascontiguousarray(c, dtype=np.float64)
        self.shape = c.shape
        m = Medium()
        m.dim = c.ndim
        for a, n in enumerate(c.shape):
            m.n[a] = n
        m.c = c.ctypes.data_as(C.POINTER(C.c_double))
        m.sponge_width = sponge_width
        m.gamma_max = gamma_max
        ws, self._blob = pack_weights({**weights, "precision": precision})
        self.h = _P()
        _check(self.lib.mcmg_setup(ctx.h, C.byref(m), omega, C.byref(ws), C.byref(self.h)))
        self.levels = weights["levels"]
        self.channels = list(weights["channels"])
        self.nu_pre = list(weights["nu_pre"])
        self.nu_post = list(weights["nu_post"])

    def level_shape(self, l):
        return tuple(n >> l for n in self.shape)

    def vcycle(self, r, e, nrhs=1, stream=None):
        _check(self.lib.mcmg_vcycle(self.h, ptr(r), ptr(e), nrhs, _stream(stream)))

    def solve(self, f, u, tol=1e-6, restart_m=20, max_iters=0, nrhs=1, flags=0, stream=None):
        o = SolveOpts(tol, restart_m, max_iters, nrhs, flags, _stream(stream))
        info = SolveInfo()
        st = self.lib.mcmg_solve(self.h, ptr(f), ptr(u), C.byref(o), C.byref(info))
        if st not in (MCMG_OK, -5):
            _check(st)
        return st, info.as_dict()

    def solve_host(self, f, u, tol=1e-6, restart_m=20, max_iters=0, nrhs=1, flags=0):
        o = SolveOpts(tol, restart_m, max_iters, nrhs, flags)
        info = SolveInfo()
        st = self.lib.mcmg_solve_host(self.h, ptr(f), ptr(u), C.byref(o), C.byref(info))
        if st not in (MCMG_OK, -5):
            _check(st)
        return st, info.as_dict()

    def kernel_shape(self, level, op=0) -> int:
        v = C.c_int()
        _check(self.lib.mcmg_get_kernel_shape(self.h, level, op, C.byref(v)))
        return v.value

    def set_kernel_shape(self, level, op, shape) -> bool:
        """Use CUDA-core shape `shape` for operation op (-1: setup's choice).
        False when the shape cannot run on this level's channels."""
        st = self.lib.mcmg_set_kernel_shape(self.h, level, op, shape)
        if st == MCMG_ERR_SHAPE:
            return False
        _check(st)
        return True

    def device_error(self) -> int:
        v = C.c_int()
        _check(self.lib.mcmg_device_error(self.h, C.byref(v)))
        return v.value

    def apply_A(self, x, y, fp64=False, nrhs=1, stream=None):
        _check(self.lib.mcmg_apply_A(self.h, ptr(x), ptr(y), int(fp64), nrhs, _stream(stream)))

    def get_feature(self, level, which, out):
        _check(self.lib.mcmg_get_feature(self.h, level, which, ptr(out)))

    def lift(self, r, r1, nrhs=1, stream=None):
        _check(self.lib.mcmg_lift(self.h, ptr(r), ptr(r1), nrhs, _stream(stream)))

    def project(self, e1, e, nrhs=1, stream=None):
        _check(self.lib.mcmg_project(self.h, ptr(e1), ptr(e), nrhs, _stream(stream)))

    def smooth(self, level, step, r, e_in, e_out, nrhs=1, stream=None):
        _check(self.lib.mcmg_smooth(self.h, level, step, ptr(r), None if e_in is None else ptr(e_in),
                                    ptr(e_out), nrhs, _stream(stream)))

    def residual(self, level, r, e, t, nrhs=1, stream=None):
        """t = r - A_l(e) on `level` (enqueued on `stream`)."""
        _check(self.lib.mcmg_residual(self.h, level, ptr(r), ptr(e), ptr(t), nrhs,
                                      _stream(stream)))

    def residual_restrict(self, level, r, e, rc, nrhs=1, stream=None):
        _check(self.lib.mcmg_residual_restrict(self.h, level, ptr(r), ptr(e), ptr(rc), nrhs,
                                               _stream(stream)))

    def prolong_add(self, level, ec, e, nrhs=1, stream=None):
        _check(self.lib.mcmg_prolong_add(self.h, level, ptr(ec), ptr(e), nrhs, _stream(stream)))

    def apply_G(self, x, stream=None):
        """x <- G x in place (the Born-series Green operator; x complex128)."""
        _check(self.lib.mcmg_apply_G(self.h, ptr(x), _stream(stream)))

    def coarse_basis(self, level, node, channel, out, stream=None):
        """Raw coarse-basis response of (level, node, channel) into `out`
        (complex64, finest grid)."""
        _check(self.lib.mcmg_coarse_basis(self.h, level, node, channel, ptr(out), _stream(stream)))

    def cgs2(self, V, w):
        k = V.shape[0]
        n = V.shape[1]
        hbuf = np.zeros(2 * k)
        nrm = C.c_double()
        _check(self.lib.mcmg_cgs2(self.h, ptr(V), k, n, ptr(w),
                                  hbuf.ctypes.data_as(C.POINTER(C.c_double)), C.byref(nrm)))
        return hbuf.view(np.complex128), nrm.value

    def close(self):
        if self.h:
            self.lib.mcmg_destroy(self.h)
            self.h = _P()
