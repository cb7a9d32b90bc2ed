"""CUDA path vs the oracle on nearly weakly dominant systems, through the C ABI.

The benchmark inputs are strongly dominant (|a| + |c| <= b / 2).  Here every
row is dominant by a small margin only, which is where unpivoted eliminations
see their largest pivot growth, the reciprocals their smallest pivots, and
the interface systems (dominant whenever the whole system is, Sec. I) their
smallest dominance margin:

* random systems with b = (|a| + |c|)(1 + 1e-3): single, batched (as one
  system and with the block map), adjoint;
* the implicit heat step tridiag(-r, 1 + 2r, -r) at large time steps,
  r = 100 and r = 1000, with materialised diagonals (rows and the strided
  column sweep) and on the constant-coefficient path.

Tolerances scale with a bound on the condition number (a reading: the
paper's tolerances are stated for its well-conditioned inputs).  For the
random systems the diagonally scaled matrix D^-1 A = I + E has
||E||_inf <= 1 / (1 + m), so kappa_inf(D^-1 A) <= (2 + m) / m; for the heat
step kappa_inf(A) <= 1 + 4r (||A^-1||_inf <= 1 since every row is dominant by
1).  binary64: max(1e-12, kappa * 1e-15); binary32 before refinement:
kappa * 1e-6; binary32 + three binary64 corrections (one correction contracts
the error by about kappa * 2^-24 only): max(1e-12, kappa * 1e-15).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

MARGIN = 1e-3
KAPPA_WEAK = (2 + MARGIN) / MARGIN
ITERS = 3


def tol(code, kappa):
    return kappa * 1e-6 if code == 1 else max(1e-12, kappa * 1e-15)


@pytest.fixture(scope="module")
def tdp():
    import torch

    import paper_2510_27351_gb300 as tdp

    assert torch.cuda.is_available()
    tdp.tdp_set_checked(True)
    yield tdp
    tdp.tdp_set_checked(False)


def dev(x, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def per_system_err(x, ref, offsets):
    """Largest relative infinity-norm error over the systems of a batch."""
    worst = 0.0
    for j in range(len(offsets) - 1):
        lo, hi = int(offsets[j]), int(offsets[j + 1])
        if hi > lo:
            worst = max(worst, oracle.rel_err(x[lo:hi], ref[lo:hi]))
    return worst


def _dt(code):
    import torch

    return torch.float32 if code == 1 else torch.float64


@pytest.mark.parametrize("code", [0, 1, 2])
def test_weak_single(tdp, code):
    import torch

    for n in (5, 1000, 100_003, 1 << 20):
        S = W.weak(n, MARGIN, seed=n + 1)
        ref = oracle.thomas(S.a, S.b, S.c, S.d)
        a, b, c, d = (dev(v, _dt(code)) for v in (S.a, S.b, S.c, S.d))
        for s in (8, 16, 32, 0):
            x = torch.empty_like(d)
            tdp.tdp_solve(a, b, c, d, x, n, s, code, ITERS if code == 2 else 0)
            torch.cuda.synchronize()
            e = oracle.rel_err(host(x), ref)
            assert e <= tol(code, KAPPA_WEAK), (n, s, e)


@pytest.mark.parametrize("code", [0, 1, 2])
def test_weak_batched(tdp, code):
    """Large systems (solved as one block-diagonal system) and small ones
    (block map), every system held to the tolerance on its own."""
    import torch

    for Sb in (W.weak(sizes=W.batch_sizes(24, 4096, 65536, seed=3), margin=MARGIN, seed=3),
               W.weak(sizes=W.batch_sizes(300, 2, 3000, seed=4), margin=MARGIN, seed=4)):
        ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
        a, b, c, d = (dev(v, _dt(code)) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
        off = dev(Sb.offsets)
        for s in (16, 0):
            x = torch.empty_like(d)
            tdp.tdp_solve_batched(off, Sb.batch, Sb.n, a, b, c, d, x, s, code, ITERS if code == 2 else 0)
            torch.cuda.synchronize()
            e = per_system_err(host(x), ref, Sb.offsets)
            assert e <= tol(code, KAPPA_WEAK), (Sb.batch, s, e)


@pytest.mark.parametrize("code", [0, 1, 2])
def test_weak_adjoint(tdp, code):
    """A^T has the columns of A as rows, so these systems are made dominant by
    columns too (by the same margin): the bound on kappa then holds for A^T.
    code 2 (one binary64 correction): the windowed pass rejects these rows
    (the decay across its halo is too slow) and the exact binary64 solve
    answers."""
    import torch

    sizes = [64, 3, 8192, 1000, 2]
    Sb = W.weak(sizes=sizes, margin=MARGIN, seed=6, columns=True)
    x = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
    g = W.loss_weights(Sb.n, seed=6)
    ref = oracle.adjoint_batched(Sb.a, Sb.b, Sb.c, x, g, Sb.offsets)
    a, b, c, X, G = (dev(v, _dt(code)) for v in (Sb.a, Sb.b, Sb.c, x, g))
    outs = [torch.empty_like(X) for _ in range(4)]
    tdp.tdp_solve_backward(dev(Sb.offsets), len(sizes), Sb.n, a, b, c, X, G, *outs, 16, code)
    torch.cuda.synchronize()
    for k, o in zip("abcd", outs):
        e = per_system_err(host(o), ref[k], Sb.offsets)
        assert e <= tol(code, KAPPA_WEAK), (k, e)


@pytest.mark.parametrize("r", [100.0, 1000.0])
@pytest.mark.parametrize("code", [0, 1, 2])
def test_heat_step_large_time_step(tdp, r, code):
    """Rows, then the stride-n column sweep, with materialised diagonals; then
    the same step on the constant-coefficient path.  Each line against the
    oracle's Thomas and, for the rows, the sine-basis closed form."""
    import torch

    n = 512
    kappa = 1 + 4 * r
    H = W.heat(n, r, seed=7)
    rows_ref, cols_ref = oracle.heat_step(H.a, H.b, H.c, H.u)
    u = H.u.reshape(-1)
    dst_rows = np.concatenate([oracle.dst_const(n, r, u[i * n:(i + 1) * n]) for i in range(n)])
    assert oracle.rel_err(rows_ref.reshape(-1), dst_rows) <= 1e-12  # the two oracles agree
    it = ITERS if code == 2 else 0
    a, b, c, U = (dev(v.reshape(-1), _dt(code)) for v in (H.a, H.b, H.c, H.u))
    rows = torch.empty_like(U)
    tdp.tdp_solve_strided(n, n, n, 1, a, b, c, U, rows, 16, code, it)
    cols = torch.empty_like(U)
    tdp.tdp_solve_strided(n, n, 1, n, a, b, c, rows, cols, 16, code, it)
    torch.cuda.synchronize()
    assert oracle.rel_err(host(rows), rows_ref.reshape(-1)) <= tol(code, kappa)
    assert oracle.rel_err(host(cols), cols_ref.reshape(-1)) <= 2 * tol(code, kappa)
    # the same rows as one batch of back-to-back systems (single-system tiles)
    off = dev(np.arange(n + 1, dtype=np.int64) * n)
    x = torch.empty_like(U)
    tdp.tdp_solve_batched(off, n, n * n, a, b, c, U, x, 0, code, it)
    torch.cuda.synchronize()
    assert oracle.rel_err(host(x), rows_ref.reshape(-1)) <= tol(code, kappa)
    # constant coefficients
    rows_c = torch.empty_like(U)
    tdp.tdp_solve_const(-r, 1 + 2 * r, -r, U, rows_c, n, n, n, 1, 0, code, it)
    cols_c = torch.empty_like(U)
    tdp.tdp_solve_const(-r, 1 + 2 * r, -r, rows_c, cols_c, n, n, 1, n, 0, code, it)
    torch.cuda.synchronize()
    assert oracle.rel_err(host(rows_c), dst_rows) <= tol(code, kappa)
    assert oracle.rel_err(host(cols_c), cols_ref.reshape(-1)) <= 2 * tol(code, kappa)
