"""Seeded synthetic inputs for the tridiagonal solver (numpy only).

This module draws random numbers and assembles test systems.  It holds none of
the solver's arithmetic: it is shared by the CPU oracle's tests, the GPU tests
and the benchmark so that both sides see bit-identical inputs.

Generator
---------
A counter-based splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  The i-th draw of stream ``k``
under seed ``seed`` is ``mix64(key + (i + 1) * GAMMA)`` with
``key = mix64(seed * GAMMA + k)``; ``mix64`` is the splitmix64 finaliser.
Uniform doubles take the top 53 bits: ``(z >> 11) * 2**-53`` in [0, 1).

Streams: 0 = a, 1 = b, 2 = c, 3 = x*, 4 = system sizes, 5/6 = normal draws,
7 = heat field, 8/9 = exponents and zeros of ``binade_edges``.

Workloads (value distributions of the benchmark configurations)
---------------------------------------------------------------
* ``single``: b ~ U[4, 8], a, c ~ U[-1, 1], a[0] = c[N-1] = 0 (strictly
  diagonally dominant), x* ~ U[-1, 1], d = A x* in binary64.
* ``batched``: ``B`` systems, sizes N_j = round(exp(U(ln lo, ln hi))) clamped
  to [lo, hi], drawn before the values; values as ``single`` over the
  concatenation, with a = 0 at each system start and c = 0 at each end.
* ``adjoint``: ``batched`` of equal sizes plus loss weights w ~ N(0, 1)
  (Box-Muller on two uniform streams).
* ``heat``: the implicit heat step on an n x n grid: b = 1 + 2r, a = c = -r,
  Dirichlet zeros outside the grid (the solver ignores a at a line's first
  row and c at its last, so one materialised diagonal serves the row and the
  column sweep), field u ~ U[0, 1].
* ``binade_edges``: ``single``'s matrix with x* of signed powers of two
  2^k, k uniform in {-3, ..., 3}, and zeros (probability 1/10), d = A x*.
* ``weak``: near-weakly-dominant systems: a, c ~ U[-1, 1] as ``single`` /
  ``batched``, b = (|a| + |c|)(1 + margin) (every row dominant by the
  relative margin only; optionally every column as well), x* ~ U[-1, 1],
  d = A x*.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_A, STREAM_B, STREAM_C, STREAM_X, STREAM_N, STREAM_G1, STREAM_G2, STREAM_U, STREAM_E, STREAM_Z = range(10)
STREAM_RHS = 16  # right-hand-side columns use streams 16, 17, ...


def mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def raw64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` draws of stream ``stream`` beginning at counter ``start``."""
    with np.errstate(over="ignore"):
        key = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GAMMA + np.uint64(stream))
        ctr = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        return mix64(key + ctr * GAMMA)


def uniform(seed: int, stream: int, count: int, lo: float = 0.0, hi: float = 1.0, start: int = 0) -> np.ndarray:
    u = (raw64(seed, stream, count, start) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, count: int) -> np.ndarray:
    """Box-Muller normals from streams 5 and 6."""
    u1 = uniform(seed, STREAM_G1, count)
    u2 = uniform(seed, STREAM_G2, count)
    u1 = np.where(u1 <= 0.0, 2.0 ** -53, u1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class System:
    """Concatenated tridiagonal systems (contiguous, uneven sizes)."""

    a: np.ndarray
    b: np.ndarray
    c: np.ndarray
    d: np.ndarray
    xstar: np.ndarray
    offsets: np.ndarray  # int64, length B+1, offsets[0] = 0

    @property
    def n(self) -> int:
        return int(self.offsets[-1])

    @property
    def batch(self) -> int:
        return len(self.offsets) - 1

    def astype(self, dtype) -> "System":
        return System(*(v.astype(dtype) for v in (self.a, self.b, self.c, self.d, self.xstar)), self.offsets)


def _ends(offsets: np.ndarray):
    """First and last rows of the non-empty systems."""
    offsets = np.asarray(offsets, dtype=np.int64)
    keep = offsets[1:] > offsets[:-1]
    return offsets[:-1][keep], offsets[1:][keep] - 1


def matvec(a, b, c, x, offsets) -> np.ndarray:
    """d = A x for concatenated systems (couplings across systems dropped)."""
    a = a.copy()
    c = c.copy()
    first, last = _ends(offsets)
    a[first] = 0.0
    c[last] = 0.0
    d = b * x
    d[1:] += a[1:] * x[:-1]
    d[:-1] += c[:-1] * x[1:]
    return d


def _values(seed: int, offsets: np.ndarray) -> System:
    n = int(offsets[-1])
    a = uniform(seed, STREAM_A, n, -1.0, 1.0)
    b = uniform(seed, STREAM_B, n, 4.0, 8.0)
    c = uniform(seed, STREAM_C, n, -1.0, 1.0)
    first, last = _ends(offsets)
    a[first] = 0.0
    c[last] = 0.0
    x = uniform(seed, STREAM_X, n, -1.0, 1.0)
    d = matvec(a, b, c, x, offsets)
    return System(a, b, c, d, x, offsets.astype(np.int64))


def weak(n: int = 0, margin: float = 1e-3, seed: int = 0, sizes=None, columns: bool = False) -> System:
    """One system of n rows (or concatenated systems of the given sizes) in
    which every row is diagonally dominant by the relative margin only:
    b = (|a| + |c|)(1 + margin) with a, c ~ U[-1, 1] (zero at system ends).
    With ``columns`` every column is dominant too (so is the transpose):
    b_i = max(|a_i| + |c_i|, |c_{i-1}| + |a_{i+1}|)(1 + margin)."""
    if sizes is None:
        if n < 1:
            raise ValueError("n must be >= 1")
        sizes = [n]
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    S = _values(seed, offsets)
    row = np.abs(S.a) + np.abs(S.c)
    if columns:
        col = np.zeros_like(row)
        col[1:] += np.abs(S.c[:-1])
        col[:-1] += np.abs(S.a[1:])
        row = np.maximum(row, col)
    b = row * (1.0 + margin)
    d = matvec(S.a, b, S.c, S.xstar, offsets)
    return System(S.a, b, S.c, d, S.xstar, S.offsets)


def single(n: int, seed: int = 0) -> System:
    """One strictly diagonally dominant system with a manufactured solution."""
    if n < 1:
        raise ValueError("n must be >= 1")
    return _values(seed, np.array([0, n], dtype=np.int64))


def binade_edges(n: int, seed: int = 0) -> System:
    """``single``'s matrix with a solution of signed powers of two and zeros:
    x*_i = +-2^k, k uniform in {-3, ..., 3}, x*_i = 0 with probability 1/10."""
    S = single(n, seed)
    u = uniform(seed, STREAM_E, n)
    k = np.floor(u * 14.0).astype(np.int64)  # 0..13: sign from the parity, exponent from the rest
    x = np.ldexp(np.where(k % 2 == 0, 1.0, -1.0), k // 2 - 3)
    x[uniform(seed, STREAM_Z, n) < 0.1] = 0.0
    d = matvec(S.a, S.b, S.c, x, S.offsets)
    return System(S.a, S.b, S.c, d, x, S.offsets)


def batch_sizes(batch: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    """Log-uniform sizes in [lo, hi]."""
    u = uniform(seed, STREAM_N, batch)
    sizes = np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.clip(sizes, lo, hi)


def batched(batch: int = 4096, lo: int = 64, hi: int = 65536, seed: int = 0, sizes=None) -> System:
    """``batch`` independent systems of log-uniform (or given) sizes."""
    if sizes is None:
        sizes = batch_sizes(batch, lo, hi, seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    return _values(seed, offsets)


def uniform_batch(batch: int, n: int, seed: int = 0) -> System:
    return batched(sizes=np.full(batch, n, dtype=np.int64), seed=seed)


def loss_weights(n: int, seed: int = 0) -> np.ndarray:
    """w ~ N(0, 1) for the loss L = sum(w * x)."""
    return normal(seed, n)


@dataclass
class Heat:
    """Implicit heat step on an n x n grid, lines along rows then columns."""

    n: int
    r: float
    u: np.ndarray  # (n, n) row-major field
    a: np.ndarray  # (n, n) diagonals, same layout as u
    b: np.ndarray
    c: np.ndarray


def heat(n: int = 2048, r: float = 0.5, seed: int = 0) -> Heat:
    u = uniform(seed, STREAM_U, n * n).reshape(n, n)
    a = np.full((n, n), -r)
    b = np.full((n, n), 1.0 + 2.0 * r)
    c = np.full((n, n), -r)
    return Heat(n, r, u, a, b, c)


def rhs_columns(n: int, nrhs: int, seed: int = 0) -> np.ndarray:
    """nrhs right-hand sides of n rows for one matrix, each U[-1, 1]
    (column j from stream 16 + j); shape (nrhs, n)."""
    return np.stack([uniform(seed, STREAM_RHS + j, n, -1.0, 1.0) for j in range(nrhs)])
