"""Python binding of libcsc.so (include/csc.h): argument marshalling only.

Every array argument may be a torch tensor (CUDA or CPU) or a numpy array; it must be contiguous
and float32 (mu: float64). The library itself decides whether a pointer is host or device memory.
All computation runs in the library's CUDA kernels; if libcsc.so is missing this module raises at
import: there is no fallback.

Functions carry the C names (csc_init, csc_code, csc_learn, csc_objective, csc_destroy,
csc_last_error, csc_version); ``Solver`` wraps a context.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcsc.so")

CSC_OK = 0
STATUS_NAMES = {0: "CSC_OK", 1: "CSC_ERR_ARG", 2: "CSC_ERR_SHAPE", 3: "CSC_ERR_WORKSPACE", 4: "CSC_ERR_CUDA",
                5: "CSC_ERR_NONFINITE", 6: "CSC_ERR_NOT_CONVERGED", 7: "CSC_ERR_TIMEOUT",
                8: "CSC_ERR_UNSUPPORTED"}
CSC_FP32 = 0
CSC_MIXED_BF16 = 1
CSC_MIXED_TF32 = 2
CSC_FLAG_GRAPH = 1
CSC_FLAG_CHECK_FINITE = 2
CSC_FLAG_CG_STRICT = 4
CSC_FLAG_SYMMETRIC_BOUNDARY = 8
CSC_FLAG_SPATIAL = 16


class CscError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class csc_params(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int), ("K", ctypes.c_int), ("fs", ctypes.c_int * 2),
                ("beta", ctypes.c_double), ("rho", ctypes.c_double), ("cg_max", ctypes.c_int),
                ("cg_tol", ctypes.c_double), ("precision", ctypes.c_int), ("flags", ctypes.c_int),
                ("deterministic", ctypes.c_int)]


class csc_timing(ctypes.Structure):
    _fields_ = [("sweep_ms", ctypes.c_double), ("sweep_launches", ctypes.c_int), ("learn_ms", ctypes.c_double),
                ("learn_calls", ctypes.c_int), ("kernel_launches", ctypes.c_longlong)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is not built; run paper_1709_09479_gb300.build.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.csc_init.argtypes = [ctypes.POINTER(csc_params), i, ctypes.POINTER(i), vp, ctypes.POINTER(vp)]
    lib.csc_init.restype = i
    lib.csc_code.argtypes = [vp, vp, vp, vp, vp, i]
    lib.csc_code.restype = i
    lib.csc_learn.argtypes = [vp, vp, vp, vp, vp, i, ctypes.POINTER(i)]
    lib.csc_learn.restype = i
    lib.csc_objective.argtypes = [vp, vp, vp, vp, ctypes.POINTER(d)]
    lib.csc_objective.restype = i
    lib.csc_destroy.argtypes = [vp]
    lib.csc_destroy.restype = None
    lib.csc_last_error.argtypes = [vp]
    lib.csc_last_error.restype = ctypes.c_char_p
    lib.csc_timing_enable.argtypes = [vp, i]
    lib.csc_timing_enable.restype = i
    lib.csc_timing_read.argtypes = [vp, ctypes.POINTER(csc_timing)]
    lib.csc_timing_read.restype = i
    lib.csc_init_uneven.argtypes = [ctypes.POINTER(csc_params), i, ctypes.POINTER(i), vp, ctypes.POINTER(vp)]
    lib.csc_init_uneven.restype = i
    lib.csc_init_video.argtypes = [ctypes.POINTER(csc_params), i, i, ctypes.POINTER(i), vp, ctypes.POINTER(vp)]
    lib.csc_init_video.restype = i
    lib.csc_describe.argtypes = [vp, ctypes.c_char_p, i]
    lib.csc_describe.restype = i
    lib.csc_tape_bytes.argtypes = [vp, i, i]
    lib.csc_tape_bytes.restype = ctypes.c_size_t
    lib.csc_code_unrolled.argtypes = [vp, vp, vp, vp, vp, i, i, vp]
    lib.csc_code_unrolled.restype = i
    lib.csc_code_backward.argtypes = [vp, vp, vp, vp, i, i, vp, vp, vp]
    lib.csc_code_backward.restype = i
    lib.csc_synthesize.argtypes = [vp, vp, vp, vp]
    lib.csc_synthesize.restype = i
    lib.csc_synthesize_backward.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.csc_synthesize_backward.restype = i
    lib.csc_code_noalloc.argtypes = [ctypes.POINTER(csc_params), i, ctypes.POINTER(i), vp, vp, vp, vp, vp, i]
    lib.csc_code_noalloc.restype = i
    lib.csc_learn_stats.argtypes = [vp, vp, vp, vp, vp]
    lib.csc_learn_stats.restype = i
    lib.csc_learn_solve.argtypes = [vp, vp, vp, vp, vp, i, ctypes.POINTER(i)]
    lib.csc_learn_solve.restype = i
    lib.csc_check.argtypes = [vp]
    lib.csc_check.restype = i
    lib.csc_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    lib.csc_set_wait_limit.restype = i
    lib.csc_version.argtypes = []
    lib.csc_version.restype = ctypes.c_char_p
    return lib


LIB = _load()


def _ptr(a, dtype):
    """Data pointer of a contiguous torch tensor / numpy array of the given dtype (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
        return a.ctypes.data
    import torch
    want = torch.float32 if dtype == np.float32 else torch.float64
    if not isinstance(a, torch.Tensor) or a.dtype != want or not a.is_contiguous():
        raise TypeError(f"expected a contiguous torch tensor of {want}")
    return a.data_ptr()


def _check(status, ctx=None):
    if status != CSC_OK:
        raise CscError(status, csc_last_error(ctx))


def csc_version() -> str:
    return LIB.csc_version().decode()


def csc_last_error(ctx=None) -> str:
    return LIB.csc_last_error(ctx).decode()


def csc_init(J, K, fs, dims, n_images, beta, rho, cg_max=100, cg_tol=1e-6, precision=CSC_FP32,
             stream=None, flags=0):
    """Create a context; returns an opaque handle (int). ``stream``: cudaStream_t as int or None."""
    p = csc_params(J, K, (ctypes.c_int * 2)(*fs), beta, rho, cg_max, cg_tol, precision, flags, 1)
    dims_arr = (ctypes.c_int * 2)(*dims)
    out = ctypes.c_void_p()
    _check(LIB.csc_init(ctypes.byref(p), n_images, dims_arr, stream, ctypes.byref(out)))
    return out.value


def csc_init_uneven(J, K, fs, dims_list, beta, rho, precision=CSC_FP32, stream=None, flags=0):
    """Context for images of different sizes; dims_list = [(H, W), ...] in image order."""
    p = csc_params(J, K, (ctypes.c_int * 2)(*fs), beta, rho, 1, 1e-6, precision, flags, 1)
    flat = [int(v) for hw in dims_list for v in hw]
    arr = (ctypes.c_int * len(flat))(*flat)
    out = ctypes.c_void_p()
    _check(LIB.csc_init_uneven(ctypes.byref(p), len(dims_list), arr, stream, ctypes.byref(out)))
    return out.value


def csc_init_video(J, K, fs, ft, dims, n_videos, beta, rho, stream=None, cg_max=100, cg_tol=1e-6, flags=0):
    """Context for n_videos tensors J x T x H x W (dims = (T, H, W)), filters ft x fh x fw (fs = (fh, fw))."""
    p = csc_params(J, K, (ctypes.c_int * 2)(*fs), beta, rho, cg_max, cg_tol, CSC_FP32, flags, 1)
    dims_arr = (ctypes.c_int * 3)(*dims)
    out = ctypes.c_void_p()
    _check(LIB.csc_init_video(ctypes.byref(p), ft, n_videos, dims_arr, stream, ctypes.byref(out)))
    return out.value


def csc_describe(ctx) -> str:
    buf = ctypes.create_string_buffer(512)
    _check(LIB.csc_describe(ctx, buf, 512), ctx)
    return buf.value.decode()


def csc_destroy(ctx):
    LIB.csc_destroy(ctx)


def csc_code(ctx, x, d, v, z=None, iters=1):
    _check(LIB.csc_code(ctx, _ptr(x, np.float32), _ptr(d, np.float32), _ptr(v, np.float32),
                        _ptr(z, np.float32), iters), ctx)


def csc_learn(ctx, x, z, d, mu, steps):
    its = (ctypes.c_int * max(steps, 1))()
    _check(LIB.csc_learn(ctx, _ptr(x, np.float32), _ptr(z, np.float32), _ptr(d, np.float32),
                         _ptr(mu, np.float64), steps, its), ctx)
    return list(its)[:steps]


def csc_learn_stats(ctx, x, z, C, b):
    """This context's sums over its images: lags C [K][K][2fh-1][2fw-1] and right-hand side b [K][J][fh][fw]."""
    _check(LIB.csc_learn_stats(ctx, _ptr(x, np.float32), _ptr(z, np.float32), _ptr(C, np.float32),
                               _ptr(b, np.float32)), ctx)


def csc_learn_solve(ctx, C, b, d, mu, steps):
    """Learning steps from given (reduced) C and b; returns the CG iterations of each step."""
    its = (ctypes.c_int * max(steps, 1))()
    _check(LIB.csc_learn_solve(ctx, _ptr(C, np.float32), _ptr(b, np.float32), _ptr(d, np.float32),
                               _ptr(mu, np.float64), steps, its), ctx)
    return list(its)[:steps]


def csc_objective(ctx, x, d, z) -> float:
    out = ctypes.c_double()
    _check(LIB.csc_objective(ctx, _ptr(x, np.float32), _ptr(d, np.float32), _ptr(z, np.float32),
                             ctypes.byref(out)), ctx)
    return out.value


def _raw_ptr(a):
    """Data pointer of a device tensor of any dtype (the unrolled-coding tape)."""
    return a.data_ptr()


def csc_tape_bytes(ctx, iters, every) -> int:
    return int(LIB.csc_tape_bytes(ctx, iters, every))


def csc_code_unrolled(ctx, x, d, v, z, iters, every, tape):
    _check(LIB.csc_code_unrolled(ctx, _ptr(x, np.float32), _ptr(d, np.float32), _ptr(v, np.float32),
                                 _ptr(z, np.float32), iters, every, _raw_ptr(tape)), ctx)


def csc_code_backward(ctx, x, d, tape, iters, every, gz, gx, gd):
    _check(LIB.csc_code_backward(ctx, _ptr(x, np.float32), _ptr(d, np.float32), _raw_ptr(tape), iters, every,
                                 _ptr(gz, np.float32), _ptr(gx, np.float32), _ptr(gd, np.float32)), ctx)


def csc_synthesize(ctx, d, z, out):
    _check(LIB.csc_synthesize(ctx, _ptr(d, np.float32), _ptr(z, np.float32), _ptr(out, np.float32)), ctx)


def csc_synthesize_backward(ctx, d, z, gout, gz, gd):
    _check(LIB.csc_synthesize_backward(ctx, _ptr(d, np.float32), _ptr(z, np.float32), _ptr(gout, np.float32),
                                       _ptr(gz, np.float32), _ptr(gd, np.float32)), ctx)


def csc_code_noalloc(J, K, fs, dims, n_images, beta, rho, x, d, v, z=None, iters=1, stream=None):
    """The context-free, allocation-free coding call (device arrays only; see include/csc.h)."""
    p = csc_params(J, K, (ctypes.c_int * 2)(*fs), beta, rho, 1, 1e-6, CSC_FP32, 0, 1)
    dims_arr = (ctypes.c_int * 2)(*dims)
    if stream is None:
        stream = _current_stream()
    _check(LIB.csc_code_noalloc(ctypes.byref(p), n_images, dims_arr, stream, _ptr(x, np.float32),
                                _ptr(d, np.float32), _ptr(v, np.float32), _ptr(z, np.float32), iters))


def csc_check(ctx):
    """Synchronise and raise CscError(CSC_ERR_NONFINITE) if the latest csc_code met a non-finite value."""
    _check(LIB.csc_check(ctx), ctx)


def csc_set_wait_limit(ctx, clocks):
    """Testing aid: bound the learning CG's exchange waits to `clocks` SM cycles (0: default)."""
    _check(LIB.csc_set_wait_limit(ctx, int(clocks)), ctx)


def csc_timing_enable(ctx, enable=True):
    _check(LIB.csc_timing_enable(ctx, 1 if enable else 0), ctx)


def csc_timing_read(ctx) -> dict:
    t = csc_timing()
    _check(LIB.csc_timing_read(ctx, ctypes.byref(t)), ctx)
    return {"sweep_ms": t.sweep_ms, "sweep_launches": t.sweep_launches, "learn_ms": t.learn_ms,
            "learn_calls": t.learn_calls, "kernel_launches": t.kernel_launches}


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


class Solver:
    """One context: N images of size dims = (H, W), K filters of support fs with J channels."""

    def __init__(self, *, J, K, fs, dims=None, n_images=None, beta, rho, cg_max=100, cg_tol=1e-6,
                 precision=CSC_FP32, stream=None, flags=0, dims_list=None, ft=None):
        """dims + n_images: a batch of equal sizes; dims_list: one (H, W) per image (uneven batch);
        ft + dims = (T, H, W): n_images videos with filters of ft time taps (3-D transforms)."""
        self.J, self.K, self.fs = J, K, tuple(fs)
        self.beta, self.rho = beta, rho
        if stream is None:
            stream = _current_stream()
        if ft is not None:
            self.dims, self.N, self.ft = tuple(dims), n_images, ft
            self.ctx = csc_init_video(J, K, fs, ft, dims, n_images, beta, rho, stream, cg_max, cg_tol, flags)
        elif dims_list is not None:
            self.dims_list = [tuple(hw) for hw in dims_list]
            self.N, self.dims = len(self.dims_list), None
            self.ctx = csc_init_uneven(J, K, fs, self.dims_list, beta, rho, precision, stream, flags)
        else:
            self.dims, self.N = tuple(dims), n_images
            self.ctx = csc_init(J, K, fs, dims, n_images, beta, rho, cg_max, cg_tol, precision, stream, flags)

    def code(self, x, d, v, z=None, iters=1):
        csc_code(self.ctx, x, d, v, z, iters)

    def learn(self, x, z, d, mu, steps):
        return csc_learn(self.ctx, x, z, d, mu, steps)

    def learn_stats(self, x, z, C, b):
        csc_learn_stats(self.ctx, x, z, C, b)

    def learn_solve(self, C, b, d, mu, steps):
        return csc_learn_solve(self.ctx, C, b, d, mu, steps)

    def stats_shapes(self):
        """Shapes of csc_learn_stats' outputs: C (K, K, 2fh-1, 2fw-1) and b (K, J, fh, fw)."""
        fh, fw = self.fs
        return (self.K, self.K, 2 * fh - 1, 2 * fw - 1), (self.K, self.J, fh, fw)

    def objective(self, x, d, z):
        return csc_objective(self.ctx, x, d, z)

    def describe(self):
        return csc_describe(self.ctx)

    def check(self):
        csc_check(self.ctx)

    def set_wait_limit(self, clocks):
        csc_set_wait_limit(self.ctx, clocks)

    def timing_enable(self, enable=True):
        csc_timing_enable(self.ctx, enable)

    def timing_read(self):
        return csc_timing_read(self.ctx)

    def close(self):
        if self.ctx:
            csc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
