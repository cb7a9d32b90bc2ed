"""GB300 tridiagonal partition solver: Python binding of the C ABI (include/tdp.h).

Every numerical step runs in the CUDA kernels of ``libtdp.so``; this module
only marshals arguments (torch tensors -> device pointers, the current torch
stream) and raises on error codes.  There is no CPU fallback: importing the
package fails when the library cannot be loaded, and every call needs CUDA
tensors.

Names follow the C ABI (``tdp_solve``, ``tdp_solve_batched``, ...); the
lower-case helpers ``solve``, ``solve_batched``, ... allocate the output and
pick defaults.  ``TridiagonalSolve`` is the autograd Function (forward: the
partition solve; backward: the transposed solve of ``tdp_solve_backward``).
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))

F64, F32, F32_REFINE = 0, 1, 2
_ERRORS = {1: "EINVAL", 2: "ECUDA", 3: "ESINGULAR", 4: "ETIMEOUT", 5: "ENOMEM"}
OK, EINVAL, ECUDA, ESINGULAR, ETIMEOUT, ENOMEM = range(6)
ST_FALLBACK = 8  # status bit: the windowed pass fell back to the exact binary64 solve


class TdpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"TDP_{_ERRORS.get(code, code)}: {msg}")
        self.code = code


def _load() -> ctypes.CDLL:
    path = _build.LIB
    sources = [os.path.join(_build.CSRC, f) for f in os.listdir(_build.CSRC)] + [
        os.path.join(_build.ROOT, "include", "tdp.h")]
    if os.environ.get("TDP_REBUILD") == "1" or _build._stale(path, sources):
        _build.build()  # incremental: only stale translation units are compiled
    lib = ctypes.CDLL(path)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.tdp_solve.argtypes = [P, P, P, P, P, I64, I32, I32, I32, P]
    lib.tdp_solve_batched.argtypes = [P, I32, I64, P, P, P, P, P, I32, I32, I32, P]
    lib.tdp_solve_strided.argtypes = [I32, I64, I64, I64, P, P, P, P, P, I32, I32, I32, P]
    lib.tdp_solve_backward.argtypes = [P, I32, I64, P, P, P, P, P, P, P, P, P, I32, I32, P]
    lib.tdp_predict_s.argtypes = [I64, I32, I32]
    lib.tdp_predict_s.restype = I32
    lib.tdp_load_table.argtypes = [ctypes.c_char_p]
    lib.tdp_reserve.argtypes = [I64, I32, I32, I32, P]
    lib.tdp_status.argtypes = [P]
    lib.tdp_set_checked.argtypes = [ctypes.c_int]
    lib.tdp_set_checked.restype = None
    lib.tdp_last_error.restype = ctypes.c_char_p
    lib.tdp_launch_count.restype = I64
    lib.tdp_thomas_batched.argtypes = [P, I32, I64, P, P, P, P, P, I32, P]
    lib.tdp_stage1.argtypes = [P, P, P, P, I64, I32, I32, P, P, P, P, P]
    lib.tdp_profile_enable.argtypes = [ctypes.c_int]
    lib.tdp_profile_enable.restype = None
    lib.tdp_profile_summary.argtypes = [ctypes.c_char_p, I64]
    lib.tdp_profile_summary.restype = I64
    lib.tdp_solve_noalloc.argtypes = [P, P, P, P, P, I64, I32, I32, P]
    lib.tdp_set_tuning.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.tdp_predict_s_batched.argtypes = [P, I32, I32, P, P]
    lib.tdp_get_tuning.argtypes = [ctypes.c_int]
    lib.tdp_solve_const.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, I64, I32, I64, I64,
                                     I32, I32, I32, P]
    lib.tdp_predict_r.argtypes = [I64, I32, I32]
    lib.tdp_predict_r.restype = I32
    lib.tdp_load_rtable.argtypes = [ctypes.c_char_p]
    lib.tdp_recursion_plan.argtypes = [I64, I32, I32, I32, P, I32]
    lib.tdp_recursion_plan.restype = I32
    lib.tdp_solve_multi.argtypes = [P, P, P, P, P, I64, I32, I64, I64, I32, I32, P]
    lib.tdp_solve_host.argtypes = [P, P, P, P, P, I64, I32, I32, I32, P]
    lib.tdp_status_code.argtypes = [ctypes.c_uint32]
    lib.tdp_last_status_bits.restype = ctypes.c_uint32
    lib.tdp_fp64_fma_rate.argtypes = [P, P, P]
    return lib


LIB = _load()

# Every symbol the header declares (checked by the tests).
SYMBOLS = ("tdp_solve", "tdp_solve_batched", "tdp_solve_strided", "tdp_solve_backward", "tdp_predict_s",
           "tdp_load_table", "tdp_reserve", "tdp_status", "tdp_set_checked", "tdp_last_error",
           "tdp_launch_count", "tdp_thomas_batched", "tdp_stage1", "tdp_profile_enable", "tdp_profile_summary",
           "tdp_solve_noalloc", "tdp_set_tuning", "tdp_get_tuning", "tdp_predict_s_batched", "tdp_predict_r",
           "tdp_load_rtable", "tdp_recursion_plan", "tdp_solve_const", "tdp_solve_multi", "tdp_solve_host",
           "tdp_status_code", "tdp_last_status_bits", "tdp_fp64_fma_rate")

(TUNE_SMEM_BUDGET, TUNE_S_REC, TUNE_S_TAIL, TUNE_VTILE, TUNE_COOP) = range(5)
(TUNE_REFINE3, TUNE_RECURSION, TUNE_R, TUNE_SEGMENTED, TUNE_PER_SYSTEM_S, TUNE_IFACE32, TUNE_REFINE_KEPT,
 TUNE_COOP_REG, TUNE_BATCH_FLAT, TUNE_VTILE_B, TUNE_VTILE_L, TUNE_WINDOW, TUNE_WINDOW_HALO, TUNE_WAIT_LOG2,
 TUNE_WAIT_NEVER, TUNE_WINDOW_SW, TUNE_WINDOW32, TUNE_WINDOW_PREFETCH, TUNE_WINDOW_HALO32,
 TUNE_WINDOW_SW32) = range(9, 29)
RETIRED_TUNING_KEYS = (5, 6, 7, 8)


def _check(rc: int):
    if rc != 0:
        raise TdpError(rc, LIB.tdp_last_error().decode())


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("tdp: tensors must live on a CUDA device (no CPU path)")
    if not t.is_contiguous():
        raise ValueError("tdp: tensors must be contiguous")
    return t.data_ptr()


def _dtype_code(t: torch.Tensor, refine: bool) -> int:
    if t.dtype == torch.float64:
        return F32_REFINE if refine else F64
    if t.dtype == torch.float32:
        if refine:
            raise ValueError("tdp: refinement needs float64 storage")
        return F32
    raise TypeError(f"tdp: unsupported dtype {t.dtype}")


# ----------------------------------------------------------------------------
# C ABI, one to one (tensors or raw device pointers)
# ----------------------------------------------------------------------------
def tdp_solve(a, b, c, d, x, n, s, dtype, refine_iters=0, stream=None):
    _check(LIB.tdp_solve(_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x), int(n), int(s), int(dtype),
                         int(refine_iters), _stream(stream)))


def tdp_solve_noalloc(a, b, c, d, x, n, s, dtype, stream=None):
    """Allocation-free single-system solve (static 16 MiB device scratch)."""
    _check(LIB.tdp_solve_noalloc(_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x), int(n), int(s), int(dtype),
                                 _stream(stream)))


def tdp_solve_batched(offsets, batch, total_n, a, b, c, d, x, s, dtype, refine_iters=0, stream=None):
    _check(LIB.tdp_solve_batched(_ptr(offsets), int(batch), int(total_n), _ptr(a), _ptr(b), _ptr(c), _ptr(d),
                                 _ptr(x), int(s), int(dtype), int(refine_iters), _stream(stream)))


def tdp_solve_strided(batch, n, sys_stride, elem_stride, a, b, c, d, x, s, dtype, refine_iters=0, stream=None):
    _check(LIB.tdp_solve_strided(int(batch), int(n), int(sys_stride), int(elem_stride), _ptr(a), _ptr(b), _ptr(c),
                                 _ptr(d), _ptr(x), int(s), int(dtype), int(refine_iters), _stream(stream)))


def tdp_solve_backward(offsets, batch, total_n, a, b, c, x, g, grad_a, grad_b, grad_c, grad_d, s, dtype,
                       stream=None):
    _check(LIB.tdp_solve_backward(_ptr(offsets), int(batch), int(total_n), _ptr(a), _ptr(b), _ptr(c), _ptr(x),
                                  _ptr(g), _ptr(grad_a), _ptr(grad_b), _ptr(grad_c), _ptr(grad_d), int(s),
                                  int(dtype), _stream(stream)))


def tdp_thomas_batched(offsets, batch, total_n, a, b, c, d, x, dtype, stream=None):
    _check(LIB.tdp_thomas_batched(_ptr(offsets), int(batch), int(total_n), _ptr(a), _ptr(b), _ptr(c), _ptr(d),
                                  _ptr(x), int(dtype), _stream(stream)))


def tdp_stage1(a, b, c, d, n, s, dtype, ra, rb, rc, rd, stream=None):
    _check(LIB.tdp_stage1(_ptr(a), _ptr(b), _ptr(c), _ptr(d), int(n), int(s), int(dtype), _ptr(ra), _ptr(rb),
                          _ptr(rc), _ptr(rd), _stream(stream)))


def tdp_predict_s(n: int, batch: int = 1, dtype: int = F64) -> int:
    return int(LIB.tdp_predict_s(int(n), int(batch), int(dtype)))


def tdp_predict_s_batched(offsets, batch, dtype, s_out, stream=None):
    _check(LIB.tdp_predict_s_batched(_ptr(offsets), int(batch), int(dtype), _ptr(s_out), _stream(stream)))


def tdp_load_table(path: str):
    _check(LIB.tdp_load_table(path.encode()))


def tdp_solve_const(a, b, c, d, x, n, batch, sys_stride, elem_stride, s, dtype, refine_iters=0, stream=None):
    _check(LIB.tdp_solve_const(float(a), float(b), float(c), _ptr(d), _ptr(x), int(n), int(batch), int(sys_stride),
                               int(elem_stride), int(s), int(dtype), int(refine_iters), _stream(stream)))


def tdp_solve_host(a, b, c, d, x, n, s=0, dtype=F64, refine_iters=0, stream=None):
    """tdp_solve on CPU tensors (pinned memory lets the copies overlap the solve)."""
    for t in (a, b, c, d, x):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("tdp_solve_host takes contiguous host tensors")
    _check(LIB.tdp_solve_host(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                              ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                              ctypes.c_void_p(x.data_ptr()), int(n), int(s), int(dtype), int(refine_iters),
                              _stream(stream)))


def tdp_solve_multi(a, b, c, d, x, n, nrhs, ldd, ldx, s=0, dtype=F64, stream=None):
    """A X = D for nrhs columns (column j of d / x at element j*ldd / j*ldx)."""
    _check(LIB.tdp_solve_multi(_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x), int(n), int(nrhs), int(ldd), int(ldx),
                               int(s), int(dtype), _stream(stream)))


def tdp_predict_r(n: int, batch: int = 1, dtype: int = F64) -> int:
    return int(LIB.tdp_predict_r(int(n), int(batch), int(dtype)))


def tdp_load_rtable(path: str):
    _check(LIB.tdp_load_rtable(path.encode()))


def tdp_recursion_plan(n: int, s: int, R: int = -1, dtype: int = F64) -> list:
    """Sub-system sizes of the recursive steps of the paper's schedule (host only)."""
    buf = (ctypes.c_int32 * 16)()
    k = int(LIB.tdp_recursion_plan(int(n), int(s), int(R), int(dtype), ctypes.cast(buf, ctypes.c_void_p), 16))
    if k < 0:
        raise TdpError(1, "tdp_recursion_plan: bad arguments")
    return [int(buf[i]) for i in range(k)]


def tdp_reserve(total_n, batch, s, dtype, stream=None):
    _check(LIB.tdp_reserve(int(total_n), int(batch), int(s), int(dtype), _stream(stream)))


def tdp_status(stream=None):
    _check(LIB.tdp_status(_stream(stream)))


def tdp_set_checked(on: bool):
    LIB.tdp_set_checked(1 if on else 0)


def tdp_set_tuning(key: int, value: int):
    _check(LIB.tdp_set_tuning(int(key), int(value)))


def tdp_get_tuning(key: int) -> int:
    return int(LIB.tdp_get_tuning(int(key)))


def tdp_last_error() -> str:
    return LIB.tdp_last_error().decode()


def tdp_launch_count() -> int:
    return int(LIB.tdp_launch_count())


def tdp_profile_enable(on: bool):
    LIB.tdp_profile_enable(1 if on else 0)


def tdp_fp64_fma_rate(stream=None):
    """(binary64 FMAs per second, milliseconds of the timed launch) measured on
    the current device by the library's diagnostic kernel."""
    rate = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    _check(LIB.tdp_fp64_fma_rate(ctypes.addressof(rate), ctypes.addressof(ms), _stream(stream)))
    return rate.value, ms.value


def tdp_profile_summary() -> dict:
    """{kernel name: (launches, total ms)} of the launches recorded since
    profiling was enabled (waits for their events)."""
    n = int(LIB.tdp_profile_summary(None, 0))
    buf = ctypes.create_string_buffer(n + 1)
    LIB.tdp_profile_summary(buf, n + 1)
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


# ----------------------------------------------------------------------------
# Convenience wrappers
# ----------------------------------------------------------------------------
def solve(a, b, c, d, s: int = 0, refine: bool = False, refine_iters: int = 1, out=None, stream=None):
    """x with A x = d for one system (CUDA tensors of equal length and dtype)."""
    x = torch.empty_like(d) if out is None else out
    tdp_solve(a, b, c, d, x, d.numel(), s, _dtype_code(d, refine), refine_iters if refine else 0, stream)
    return x


def solve_batched(offsets, a, b, c, d, s: int = 0, refine: bool = False, refine_iters: int = 1, out=None,
                  stream=None):
    """Systems stored back to back; ``offsets`` is an int64 CUDA tensor of B+1 entries."""
    x = torch.empty_like(d) if out is None else out
    tdp_solve_batched(offsets, offsets.numel() - 1, d.numel(), a, b, c, d, x, s, _dtype_code(d, refine),
                      refine_iters if refine else 0, stream)
    return x


def solve_strided(batch, n, sys_stride, elem_stride, a, b, c, d, s: int = 0, refine: bool = False,
                  refine_iters: int = 1, out=None, stream=None):
    x = torch.empty_like(d) if out is None else out
    tdp_solve_strided(batch, n, sys_stride, elem_stride, a, b, c, d, x, s, _dtype_code(d, refine),
                      refine_iters if refine else 0, stream)
    return x


def thomas_batched(offsets, a, b, c, d, out=None, stream=None):
    x = torch.empty_like(d) if out is None else out
    tdp_thomas_batched(offsets, offsets.numel() - 1, d.numel(), a, b, c, d, x, _dtype_code(d, False), stream)
    return x


def solve_backward(offsets, a, b, c, x, g, s: int = 0, refine: bool = False, stream=None):
    """(grad_a, grad_b, grad_c, grad_d) of L given x = A^{-1} d and g = dL/dx;
    ``refine`` (float64 tensors): the transposed solve in binary32 with one
    binary64 correction."""
    ga, gb, gc, gd = (torch.empty_like(x) for _ in range(4))
    tdp_solve_backward(offsets, offsets.numel() - 1, x.numel(), a, b, c, x, g, ga, gb, gc, gd, s,
                       _dtype_code(x, refine), stream)
    return ga, gb, gc, gd


class CapturedSolve:
    """A solve captured into a CUDA graph.

    ``fn(stream)`` must queue one solve on ``stream`` (for example a
    ``tdp_solve_batched`` call on fixed buffers).  It runs once un-captured
    (which sizes the library's workspace for that stream), then once under
    capture; ``replay()`` re-runs the captured kernels on the same buffers.
    Checked mode must be off while capturing (it synchronises).
    """

    def __init__(self, fn, stream=None):
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            fn(self.stream)
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            fn(self.stream)
        self.stream.synchronize()

    def replay(self):
        self.graph.replay()


class TridiagonalSolve(torch.autograd.Function):
    """x = A^{-1} d for back-to-back systems; differentiable in a, b, c, d.

    The forward pass keeps x; the backward pass solves A^T lambda = g with the
    same partition kernels and forms the diagonal gradients on the device.
    """

    @staticmethod
    def forward(ctx, offsets, a, b, c, d, s=0, refine=False):
        x = solve_batched(offsets, a, b, c, d, s=s, refine=refine)
        ctx.save_for_backward(offsets, a, b, c, x)
        ctx.s = s
        ctx.refine = refine
        return x

    @staticmethod
    def backward(ctx, g):
        offsets, a, b, c, x = ctx.saved_tensors
        ga, gb, gc, gd = solve_backward(offsets, a, b, c, x, g.contiguous(), s=ctx.s, refine=ctx.refine)
        return None, ga, gb, gc, gd, None, None


def tridiagonal_solve(a, b, c, d, offsets=None, s: int = 0, refine: bool = False):
    """Differentiable solve; ``offsets`` defaults to one system; ``refine``
    (float64 tensors): forward and adjoint solves in binary32 with one
    binary64 correction."""
    if offsets is None:
        offsets = torch.tensor([0, d.numel()], dtype=torch.int64, device=d.device)
    return TridiagonalSolve.apply(offsets, a, b, c, d, s, refine)
