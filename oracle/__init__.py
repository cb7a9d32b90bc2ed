"""CPU oracle for the tridiagonal partition method (arXiv 2510.27351).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  The product library
(``paper_2510_27351_gb300``) never imports it, and it imports nothing from the
product: the two share no code.

The numerical routines live in ``oracle.c`` (plain C, binary64 / long double)
and are loaded through ctypes from ``liboracle.so`` (built by ``build()``).
The size-choice oracle (1-nearest-neighbour, label correction, the paper's
interval rule) is plain Python in ``predictor.py``.

Every function states the passage of the paper it follows and what pins it;
see the comments in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_f = ctypes.POINTER(ctypes.c_float)
_i64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (no GPU code involved)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    I64 = ctypes.c_int64
    lib.or_thomas.argtypes = [I64, _d, _d, _d, _d, _d]
    lib.or_thomas_f32.argtypes = [I64, _f, _f, _f, _f, _f]
    lib.or_thomas_batched.argtypes = [ctypes.c_int32, _i64, _i64, I64, _d, _d, _d, _d, _d]
    lib.or_partition.argtypes = [I64, I64, _d, _d, _d, _d, _d, _d, _d, _d, _d, _i64, _i64]
    lib.or_dense_ld_full.argtypes = [I64, _d, _d, _d]
    lib.or_dense_ld.argtypes = [I64, _d, _d, _d, _d, _d]
    lib.or_residual.argtypes = [I64, _d, _d, _d, _d, _d, _d]
    lib.or_residual.restype = None
    lib.or_matvec.argtypes = [I64, _d, _d, _d, _d, _d]
    lib.or_matvec.restype = None
    lib.or_refine.argtypes = [I64, _d, _d, _d, _d, _d, ctypes.c_int, ctypes.c_double, _d,
                              ctypes.POINTER(ctypes.c_int)]
    lib.or_adjoint.argtypes = [I64, _d, _d, _d, _d, _d, _d, _d, _d, _d, _d]
    lib.or_dst_const.argtypes = [I64, ctypes.c_double, _d, _d]
    lib.or_dst_const.restype = None
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_SO))
    return _lib


def _p(x, ptr=_d):
    return x.ctypes.data_as(ptr)


def _c64(*arrs):
    return [np.ascontiguousarray(v, dtype=np.float64) for v in arrs]


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc == 1:
        raise OracleError(f"{what}: zero pivot")
    if rc == 2:
        raise OracleError(f"{what}: bad argument")


def thomas(a, b, c, d):
    """x = A^{-1} d by sequential binary64 Thomas."""
    a, b, c, d = _c64(a, b, c, d)
    x = np.empty_like(d)
    _check(_load().or_thomas(len(d), _p(a), _p(b), _p(c), _p(d), _p(x)), "thomas")
    return x


def thomas_f32(a, b, c, d):
    """Thomas in binary32 arithmetic."""
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float32) for v in (a, b, c, d))
    x = np.empty_like(d)
    _check(_load().or_thomas_f32(len(d), _p(a, _f), _p(b, _f), _p(c, _f), _p(d, _f), _p(x, _f)), "thomas_f32")
    return x


def thomas_batched(a, b, c, d, offsets=None, base=None, length=None, elem_stride=1):
    """Thomas per system; either contiguous ``offsets`` or (base, length, stride)."""
    a, b, c, d = _c64(a, b, c, d)
    if offsets is not None:
        offsets = np.asarray(offsets, dtype=np.int64)
        base = offsets[:-1].copy()
        length = np.diff(offsets)
    base = np.ascontiguousarray(base, dtype=np.int64)
    length = np.ascontiguousarray(length, dtype=np.int64)
    x = np.zeros_like(d)
    _check(_load().or_thomas_batched(len(base), _p(base, _i64), _p(length, _i64), int(elem_stride),
                                     _p(a), _p(b), _p(c), _p(d), _p(x)), "thomas_batched")
    return x


def partition(a, b, c, d, s):
    """Non-recursive partition method (Sec. I).  Returns (x, reduced) where
    reduced = dict(a, b, c, d, idx) is the interface system of Stage 2."""
    a, b, c, d = _c64(a, b, c, d)
    n = len(d)
    mmax = 2 * ((n + s - 1) // s)
    x = np.empty_like(d)
    ra, rb, rc, rd = (np.zeros(mmax) for _ in range(4))
    ridx = np.zeros(mmax, dtype=np.int64)
    M = np.zeros(1, dtype=np.int64)
    _check(_load().or_partition(n, int(s), _p(a), _p(b), _p(c), _p(d), _p(x), _p(ra), _p(rb), _p(rc), _p(rd),
                                _p(ridx, _i64), _p(M, _i64)), "partition")
    m = int(M[0])
    return x, dict(a=ra[:m], b=rb[:m], c=rc[:m], d=rd[:m], idx=ridx[:m])


def dense_ld_full(A, rhs):
    """Dense long-double Gaussian elimination with partial pivoting."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    x = np.empty_like(rhs)
    _check(_load().or_dense_ld_full(len(rhs), _p(A), _p(rhs), _p(x)), "dense_ld_full")
    return x


def dense_ld(a, b, c, d):
    a, b, c, d = _c64(a, b, c, d)
    x = np.empty_like(d)
    _check(_load().or_dense_ld(len(d), _p(a), _p(b), _p(c), _p(d), _p(x)), "dense_ld")
    return x


def residual(a, b, c, d, x):
    """r = d - A x (long-double accumulation)."""
    a, b, c, d, x = _c64(a, b, c, d, x)
    r = np.empty_like(d)
    _load().or_residual(len(d), _p(a), _p(b), _p(c), _p(d), _p(x), _p(r))
    return r


def matvec(a, b, c, x):
    a, b, c, x = _c64(a, b, c, x)
    y = np.empty_like(x)
    _load().or_matvec(len(x), _p(a), _p(b), _p(c), _p(x), _p(y))
    return y


def refine(a, b, c, d, max_iter=4, tol=1e-14):
    """binary32 Thomas + binary64 residual refinement; returns (x, history)."""
    a, b, c, d = _c64(a, b, c, d)
    x = np.empty_like(d)
    hist = np.zeros(max_iter + 1)
    it = ctypes.c_int(0)
    _check(_load().or_refine(len(d), _p(a), _p(b), _p(c), _p(d), _p(x), int(max_iter), float(tol), _p(hist),
                             ctypes.byref(it)), "refine")
    return x, hist[: it.value + 1]


def adjoint(a, b, c, x, g):
    """lambda = A^{-T} g and the gradients of L with dL/dx = g."""
    a, b, c, x, g = _c64(a, b, c, x, g)
    n = len(x)
    lam, ga, gb, gc, gd = (np.empty(n) for _ in range(5))
    _check(_load().or_adjoint(n, _p(a), _p(b), _p(c), _p(x), _p(g), _p(lam), _p(ga), _p(gb), _p(gc), _p(gd)),
           "adjoint")
    return dict(lam=lam, a=ga, b=gb, c=gc, d=gd)


def adjoint_batched(a, b, c, x, g, offsets):
    out = {k: np.empty(len(x)) for k in ("lam", "a", "b", "c", "d")}
    for j in range(len(offsets) - 1):
        s, e = int(offsets[j]), int(offsets[j + 1])
        r = adjoint(a[s:e], b[s:e], c[s:e], x[s:e], g[s:e])
        for k in out:
            out[k][s:e] = r[k]
    return out


def dst_const(n, r, d):
    """Closed-form solve of tridiag(-r, 1+2r, -r) x = d via the sine basis."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    x = np.empty_like(d)
    _load().or_dst_const(int(n), float(r), _p(d), _p(x))
    return x


def heat_step(a, b, c, u):
    """One implicit heat step (a benchmark workload, not in the paper): solve
    along every row, then along every column, with Thomas per line.  Arrays
    are (n, n) row-major."""
    n = u.shape[0]
    flat = lambda v: np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    A, B, C, U = flat(a), flat(b), flat(c), flat(u)
    rows = thomas_batched(A, B, C, U, base=np.arange(n) * n, length=np.full(n, n), elem_stride=1)
    cols = thomas_batched(A, B, C, rows, base=np.arange(n), length=np.full(n, n), elem_stride=n)
    return rows.reshape(n, n), cols.reshape(n, n)


def rel_err(x, ref):
    """||x - ref||_inf / ||ref||_inf."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(ref))) if ref.size else 1.0
    return float(np.max(np.abs(x - ref))) / (den if den > 0 else 1.0) if ref.size else 0.0


if __name__ == "__main__":
    build(force=True)
    print(_SO, file=sys.stderr)
