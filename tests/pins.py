"""Checks that pin the CPU oracle to facts outside itself.

Each ``pin_*`` function returns a list of failure messages (empty = holds).
``test_oracle_pins.py`` asserts every pin holds for the committed oracle;
``test_oracle_mutants.py`` plants plausible mistakes in a copy of the oracle
source and asserts that some pin catches each one.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

import oracle
import workloads as W


def _fail(cond, msg, out):
    if not cond:
        out.append(msg)


def dense_matrix(a, b, c):
    n = len(b)
    A = np.diag(np.asarray(b, dtype=np.float64))
    if n > 1:
        A += np.diag(np.asarray(a[1:], dtype=np.float64), -1) + np.diag(np.asarray(c[:-1], dtype=np.float64), 1)
    return A


def pin_dense_vs_lapack():
    """Long-double elimination agrees with LAPACK on random dense systems."""
    out = []
    rng = np.random.default_rng(1)
    for n in (1, 2, 7, 20):
        A = rng.uniform(-1, 1, (n, n)) + n * np.eye(n)
        rhs = rng.uniform(-1, 1, n)
        x = oracle.dense_ld_full(A, rhs)
        ref = np.linalg.solve(A, rhs)
        _fail(oracle.rel_err(x, ref) < 1e-13, f"dense n={n}: {oracle.rel_err(x, ref):.2e}", out)
    # a system that needs pivoting
    A = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    rhs = np.array([1.0, 2.0, 3.0])
    x = oracle.dense_ld_full(A, rhs)
    _fail(oracle.rel_err(x, np.linalg.solve(A, rhs)) < 1e-14, "dense pivoting case", out)
    return out


def pin_thomas_vs_dense():
    """Thomas vs long-double dense elimination, n <= 64, several seeds."""
    out = []
    for seed in range(4):
        for n in (1, 2, 3, 5, 17, 64):
            S = W.single(n, seed)
            x = oracle.thomas(S.a, S.b, S.c, S.d)
            ref = oracle.dense_ld(S.a, S.b, S.c, S.d)
            e = oracle.rel_err(x, ref)
            _fail(e <= 1e-14, f"thomas vs dense n={n} seed={seed}: {e:.2e}", out)
    return out


def pin_thomas_vs_lapack_banded():
    """Thomas vs LAPACK's banded solver (general a, c; nonzero a[0], c[n-1] ignored)."""
    out = []
    for n in (2, 9, 1000):
        S = W.single(n, 7)
        a, c = S.a.copy(), S.c.copy()
        a[0], c[-1] = 3.0, -5.0  # must be ignored
        ab = np.zeros((3, n))
        ab[0, 1:] = c[:-1]
        ab[1] = S.b
        ab[2, :-1] = a[1:]
        ref = scipy.linalg.solve_banded((1, 1), ab, S.d)
        x = oracle.thomas(a, S.b, c, S.d)
        _fail(oracle.rel_err(x, ref) <= 1e-14, f"thomas vs banded n={n}", out)
    return out


def pin_thomas_manufactured():
    """||x - x*|| within kappa * eps bound for the benchmark distribution."""
    out = []
    S = W.single(100_000, 3)
    x = oracle.thomas(S.a, S.b, S.c, S.d)
    _fail(oracle.rel_err(x, S.xstar) <= 1e-14, "thomas manufactured", out)
    return out


def pin_dst():
    """Thomas and the sine-basis closed form agree; the closed form agrees with
    dense elimination on a small case (both sides pinned)."""
    out = []
    for n, tol in ((16, 1e-14), (256, 1e-13)):
        d = W.uniform(11, 9, n)
        r = 0.5
        a = np.full(n, -r)
        b = np.full(n, 1 + 2 * r)
        c = np.full(n, -r)
        xd = oracle.dst_const(n, r, d)
        xt = oracle.thomas(a, b, c, d)
        _fail(oracle.rel_err(xt, xd) <= tol, f"thomas vs dst n={n}: {oracle.rel_err(xt, xd):.2e}", out)
        if n <= 64:
            xl = oracle.dense_ld(a, b, c, d)
            _fail(oracle.rel_err(xd, xl) <= 1e-14, "dst vs dense", out)
    return out


def pin_partition_vs_thomas():
    """Partition method reaches the plain solution (exact method, Sec. I)."""
    out = []
    for n in (1, 2, 3, 4, 5, 31, 32, 33, 64, 100, 1000, 4097):
        S = W.single(n, n)
        xt = oracle.thomas(S.a, S.b, S.c, S.d)
        for s in (2, 3, 4, 5, 8, 32, 1000):
            x, _ = oracle.partition(S.a, S.b, S.c, S.d, s)
            e = oracle.rel_err(x, xt)
            _fail(e <= 1e-13, f"partition n={n} s={s}: {e:.2e}", out)
    return out


def pin_partition_special_cases():
    """s >= n: two interface unknowns (x[0], x[n-1]); s == 2: interface
    system is A itself (no interiors)."""
    out = []
    S = W.single(50, 4)
    x, red = oracle.partition(S.a, S.b, S.c, S.d, 64)
    _fail(list(red["idx"]) == [0, 49], "s>=n interface indices", out)
    _fail(oracle.rel_err(x, oracle.thomas(S.a, S.b, S.c, S.d)) <= 1e-14, "s>=n equals thomas", out)
    x, red = oracle.partition(S.a, S.b, S.c, S.d, 2)
    a0, c0 = S.a.copy(), S.c.copy()
    a0[0], c0[-1] = 0.0, 0.0
    ok = (np.array_equal(red["a"], a0) and np.array_equal(red["b"], S.b) and np.array_equal(red["c"], c0)
          and np.array_equal(red["d"], S.d) and np.array_equal(red["idx"], np.arange(50)))
    _fail(ok, "s==2 interface system is A", out)
    return out


def pin_schur_complement():
    """The interface system equals the Schur complement of A onto the
    interface indices, formed densely with numpy (independent formula)."""
    out = []
    for n, s in ((40, 8), (37, 5), (12, 3), (9, 4)):
        S = W.single(n, 100 + n)
        _, red = oracle.partition(S.a, S.b, S.c, S.d, s)
        A = dense_matrix(S.a, S.b, S.c)
        I = np.asarray(red["idx"])
        J = np.array(sorted(set(range(n)) - set(I.tolist())), dtype=int)
        if len(J):
            AJJ_inv = np.linalg.inv(A[np.ix_(J, J)])
            Sc = A[np.ix_(I, I)] - A[np.ix_(I, J)] @ AJJ_inv @ A[np.ix_(J, I)]
            rs = S.d[I] - A[np.ix_(I, J)] @ AJJ_inv @ S.d[J]
        else:
            Sc, rs = A[np.ix_(I, I)], S.d[I]
        M = len(I)
        R = np.zeros((M, M))
        for j in range(M):
            R[j, j] = red["b"][j]
            if j > 0:
                R[j, j - 1] = red["a"][j]
            if j < M - 1:
                R[j, j + 1] = red["c"][j]
        _fail(np.max(np.abs(R - Sc)) <= 1e-13 * np.max(np.abs(Sc)), f"schur matrix n={n} s={s}", out)
        _fail(np.max(np.abs(red["d"] - rs)) <= 1e-13 * np.max(np.abs(rs)), f"schur rhs n={n} s={s}", out)
        # tridiagonal: no coupling beyond the neighbours
        off = Sc - np.triu(np.tril(Sc, 1), -1)
        _fail(np.max(np.abs(off)) <= 1e-14 * np.max(np.abs(Sc)), "schur complement tridiagonal", out)
    return out


def pin_reduced_dominance():
    """Interface system strictly diagonally dominant when A is (Sec. I)."""
    out = []
    S = W.single(5000, 5)
    for s in (4, 32, 100):
        _, red = oracle.partition(S.a, S.b, S.c, S.d, s)
        M = len(red["b"])
        off = np.abs(red["a"]) + np.abs(red["c"])
        off[0] -= abs(red["a"][0])
        off[M - 1] -= abs(red["c"][M - 1])
        _fail(bool(np.all(np.abs(red["b"]) > off)), f"dominance s={s}", out)
    return out


def pin_refine():
    """FP32 start within 1e-5; refinement reaches the FP64 answer within
    1e-12 and the residual shrinks by about kappa*eps32 per step."""
    out = []
    S = W.single(20_000, 6)
    xt = oracle.thomas(S.a, S.b, S.c, S.d)
    x32 = oracle.thomas_f32(S.a, S.b, S.c, S.d).astype(np.float64)
    _fail(oracle.rel_err(x32, xt) <= 1e-5, "fp32 thomas 1e-5", out)
    _fail(oracle.rel_err(x32, xt) >= 1e-9, "fp32 thomas is really single precision", out)
    x, hist = oracle.refine(S.a, S.b, S.c, S.d, max_iter=4, tol=1e-14)
    _fail(oracle.rel_err(x, xt) <= 1e-12, f"refined error {oracle.rel_err(x, xt):.2e}", out)
    _fail(len(hist) >= 2 and hist[0] > 1e-9, "needs at least one correction", out)
    _fail(all(hist[k + 1] <= max(1e-3 * hist[k], 1e-15) for k in range(len(hist) - 1)), f"contraction {hist}", out)
    # residual of the refined x, by an independent long-double evaluation
    r = oracle.residual(S.a, S.b, S.c, S.d, x)
    _fail(np.max(np.abs(r)) / np.max(np.abs(S.d)) <= 1e-14, "refined residual", out)
    return out


def pin_adjoint():
    """<w, x> = <lambda, d>; gradients vs dense numpy and central differences."""
    out = []
    n = 64
    S = W.single(n, 8)
    w = W.loss_weights(n, 8)
    x = oracle.thomas(S.a, S.b, S.c, S.d)
    g = oracle.adjoint(S.a, S.b, S.c, x, w)
    _fail(abs(np.dot(w, x) - np.dot(g["lam"], S.d)) <= 1e-13 * abs(np.dot(w, x)) + 1e-15, "adjoint identity", out)
    A = dense_matrix(S.a, S.b, S.c)
    lam = np.linalg.solve(A.T, w)
    _fail(oracle.rel_err(g["lam"], lam) <= 1e-13, "lambda vs dense", out)
    G = -np.outer(lam, x)
    ref_a = np.concatenate([[0.0], np.diag(G, -1)])
    ref_c = np.concatenate([np.diag(G, 1), [0.0]])
    for k, ref in (("a", ref_a), ("b", np.diag(G)), ("c", ref_c), ("d", lam)):
        _fail(oracle.rel_err(g[k], ref) <= 1e-13, f"grad {k} vs dense", out)
    # central finite differences, h = 1e-6, on every entry
    h = 1e-6
    L = lambda a, b, c, d: float(np.dot(w, oracle.thomas(a, b, c, d)))
    worst = 0.0
    for name in ("a", "b", "c", "d"):
        for i in range(n):
            if (name == "a" and i == 0) or (name == "c" and i == n - 1):
                continue
            args = {k: getattr(S, k).copy() for k in "abcd"}
            args[name][i] += h
            lp = L(args["a"], args["b"], args["c"], args["d"])
            args[name][i] -= 2 * h
            lm = L(args["a"], args["b"], args["c"], args["d"])
            fd = (lp - lm) / (2 * h)
            scale = max(abs(g[name][i]), 1e-3)
            worst = max(worst, abs(fd - g[name][i]) / scale)
    _fail(worst <= 1e-6, f"finite differences {worst:.2e}", out)
    return out


def pin_batched():
    """Batched Thomas equals Thomas on each system (contiguous and strided)."""
    out = []
    Sb = W.batched(6, 1, 40, seed=2)
    x = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
    for j in range(Sb.batch):
        s, e = Sb.offsets[j], Sb.offsets[j + 1]
        ref = oracle.dense_ld(Sb.a[s:e], Sb.b[s:e], Sb.c[s:e], Sb.d[s:e])
        _fail(oracle.rel_err(x[s:e], ref) <= 1e-14, f"batched system {j}", out)
    H = W.heat(32, 0.5, 3)
    rows, cols = oracle.heat_step(H.a, H.b, H.c, H.u)
    for i in range(32):
        _fail(oracle.rel_err(rows[i], oracle.dst_const(32, 0.5, H.u[i])) <= 1e-14, f"heat row {i}", out)
        _fail(oracle.rel_err(cols[:, i], oracle.dst_const(32, 0.5, rows[:, i])) <= 1e-14, f"heat col {i}", out)
    return out


ALL_PINS = [
    pin_dense_vs_lapack,
    pin_thomas_vs_dense,
    pin_thomas_vs_lapack_banded,
    pin_thomas_manufactured,
    pin_dst,
    pin_partition_vs_thomas,
    pin_partition_special_cases,
    pin_schur_complement,
    pin_reduced_dominance,
    pin_refine,
    pin_adjoint,
    pin_batched,
]
