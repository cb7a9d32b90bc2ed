"""The windowed single pass of TDP_F32_REFINE against the oracle, through the C ABI.

The pass solves every tile of rows inside a window with halo rows on both
sides (binary32 eliminations, binary64 residual and corrections, one read of
the inputs) and checks, per tile, that the window's rows are diagonally
dominant and that the decay of A^-1 across the halo bounds the windowed
solution's distance from x by 2^-45 ||x||_inf.  A tile that fails sets the
fallback bit of the status word and the exact binary64 solve answers.

Tolerances (relative infinity norm against the oracle's binary64 Thomas):
1e-12 with at least one correction, 1e-5 without (the binary32 solve alone).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdp():
    import torch

    import paper_2510_27351_gb300 as tdp

    assert torch.cuda.is_available()
    tdp.tdp_set_checked(True)
    assert tdp.tdp_get_tuning(tdp.TUNE_WINDOW) == 1
    yield tdp
    tdp.tdp_set_checked(False)


def dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def per_system_err(x, ref, offsets):
    worst = 0.0
    for j in range(len(offsets) - 1):
        lo, hi = int(offsets[j]), int(offsets[j + 1])
        if hi > lo:
            worst = max(worst, oracle.rel_err(x[lo:hi], ref[lo:hi]))
    return worst


def solve(tdp, a, b, c, d, n, iters):
    import torch

    A, B, C, D = (dev(v) for v in (a, b, c, d))
    x = torch.full_like(D, float("nan"))
    tdp.tdp_solve(A, B, C, D, x, n, 0, tdp.F32_REFINE, iters)
    torch.cuda.synchronize()
    return host(x), tdp.LIB.tdp_last_status_bits()


TILE = 256 * 7 - 2 * 48  # owned rows per tile at the default geometry (refinement: 7 rows per thread, 48 halo rows)
TILE32 = 256 * 5 - 2 * 32  # the binary32 pass on short systems (5 rows per thread, 32 halo rows)


@pytest.mark.parametrize("iters", [0, 1, 2])
def test_window_single_sizes(tdp, iters):
    """Sizes around tile boundaries, one row, odd ends; every tile passes."""
    tol = 1e-5 if iters == 0 else 1e-12
    for n in (1, 2, 3, 5, 47, 48, 49, 97, TILE - 1, TILE, TILE + 1, 2 * TILE + 3, 100_003, (1 << 20) + 1):
        S = W.single(n, seed=n + 13)
        ref = oracle.thomas(S.a, S.b, S.c, S.d)
        x, bits = solve(tdp, S.a, S.b, S.c, S.d, n, iters)
        assert np.all(np.isfinite(x)), n
        assert not bits & tdp.ST_FALLBACK, n
        e = oracle.rel_err(x, ref)
        assert e <= tol, (n, iters, e)


def test_window_matches_exact_schedule(tdp):
    """The windowed pass and the exact three-pass schedule (TDP_TUNE_WINDOW =
    0) agree with each other and with x* to the refinement's accuracy."""
    import torch

    n = 3_000_017
    S = W.single(n, seed=5)
    ref = oracle.thomas(S.a, S.b, S.c, S.d)
    xw, bits = solve(tdp, S.a, S.b, S.c, S.d, n, 1)
    assert not bits & tdp.ST_FALLBACK
    tdp.tdp_set_tuning(tdp.TUNE_WINDOW, 0)
    try:
        A, B, C, D = (dev(v) for v in (S.a, S.b, S.c, S.d))
        x3 = torch.empty_like(D)
        tdp.tdp_solve(A, B, C, D, x3, n, 24, tdp.F32_REFINE, 1)
        torch.cuda.synchronize()
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_WINDOW, 1)
    assert oracle.rel_err(xw, ref) <= 1e-12
    assert oracle.rel_err(host(x3), ref) <= 1e-12
    assert oracle.rel_err(xw, S.xstar) <= 1e-12


@pytest.mark.parametrize("code", [2, 1])
def test_window_adjoint_reads_transposed_windows(tdp, code):
    """The adjoints of binary32 + one correction (code 2) and of binary32
    storage (code 1) solve A^T lambda = g on the windowed passes, whose windows
    read A^T's diagonals straight from a and c (c 16 bytes early, a as usual,
    both cut at every system's ends): batches of uneven sizes, tiny systems at
    tile and halo boundaries, and one system of many tiles, against the
    oracle's gradients per system and against the exact schedule (the
    windowed pass switched off: transposed copies)."""
    import torch

    knob, tol, dt = ((tdp.TUNE_WINDOW, 1e-12, torch.float64) if code == 2 else
                     (tdp.TUNE_WINDOW32, 1e-5, torch.float32))
    Sl = W.batched(600, 2, 20000, seed=12)
    for sizes in ([5000, 1, 2, 3, 1697, 1696, 1695, 48, 47, 3000, 64, 3264, 3265, 3263],
                  [1_000_003], list(Sl.offsets[1:] - Sl.offsets[:-1])):
        Sb = W.batched(sizes=[int(v) for v in sizes], seed=13)
        x = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
        g = W.loss_weights(Sb.n, seed=13)
        ref = oracle.adjoint_batched(Sb.a, Sb.b, Sb.c, x, g, Sb.offsets)
        a, b, c, X, G = (torch.from_numpy(np.ascontiguousarray(v)).to("cuda", dt) for v in (Sb.a, Sb.b, Sb.c, x, g))
        got = {}
        for win in (1, 0):
            tdp.tdp_set_tuning(knob, win)
            try:
                outs = [torch.full_like(X, float("nan")) for _ in range(4)]
                tdp.tdp_solve_backward(dev(Sb.offsets), Sb.batch, Sb.n, a, b, c, X, G, *outs, 0, code)
                torch.cuda.synchronize()
            finally:
                tdp.tdp_set_tuning(knob, 1)
            if win:
                assert not tdp.LIB.tdp_last_status_bits() & tdp.ST_FALLBACK
            got[win] = [host(o) for o in outs]
        for k, o1, o0 in zip("abcd", got[1], got[0]):
            assert per_system_err(o1, ref[k], Sb.offsets) <= tol, (len(sizes), k)
            assert per_system_err(o0, ref[k], Sb.offsets) <= tol, (len(sizes), k)


def test_window_batches(tdp):
    """Batches solved as one system through the windowed pass: log-uniform
    sizes, and tiny, one-row and empty systems (cut points inside windows and
    halos); every system against the oracle on its own."""
    import torch

    for Sb in (W.batched(256, 64, 65536, seed=3), W.batched(sizes=[0, 1, 2, 3, 0, 5, 64, 1, 1700, 47, 48, 0],
                                                            seed=4),
               W.batched(3000, 2, 200, seed=6)):
        ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
        A, B, C, D = (dev(v) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
        for iters in (1, 2):
            x = torch.full_like(D, float("nan"))
            tdp.tdp_solve_batched(dev(Sb.offsets), Sb.batch, Sb.n, A, B, C, D, x, 0, tdp.F32_REFINE, iters)
            torch.cuda.synchronize()
            assert not tdp.LIB.tdp_last_status_bits() & tdp.ST_FALLBACK
            e = per_system_err(host(x), ref, Sb.offsets)
            assert e <= 1e-12, (Sb.batch, iters, e)


@pytest.mark.parametrize("k,fallback", [(-800, False), (800, False), (-1000, True), (1000, True)])
def test_window_scaled_right_hand_side(tdp, k, fallback):
    """d scaled by 2^k (x* with it, exactly): the window's binary32 copies of
    d and x carry the scale 2^-m, m the exponent of the window's largest |d|,
    so the pass answers for |m| <= 850 (a binary32 copy of d 2^-800 alone would
    be zero) and falls back beyond; binary64 accuracy either way."""
    n = 300_007
    S = W.single(n, seed=29)
    d = np.ldexp(S.d, k)
    ref = oracle.thomas(S.a, S.b, S.c, d)
    x, bits = solve(tdp, S.a, S.b, S.c, d, n, 1)
    assert bool(bits & tdp.ST_FALLBACK) == fallback
    assert oracle.rel_err(x, ref) <= 1e-12
    assert oracle.rel_err(x, np.ldexp(S.xstar, k)) <= 1e-12


def test_window_matrix_entries_outside_binary32_range(tdp):
    """Off-diagonal entries below the binary32 range (every 7th row's a and
    c times 2^-300: their binary32 copies are zero or subnormal, and the
    binary64 residual restores them), and a whole system scaled by 2^500
    (|b| above 1e30: every tile falls back) or 2^-500; binary64 accuracy."""
    n = 200_003
    S = W.single(n, seed=41)
    a, c = S.a.copy(), S.c.copy()
    a[::7] = np.ldexp(a[::7], -300)
    c[::7] = np.ldexp(c[::7], -300)
    d = W.matvec(a, S.b, c, S.xstar, S.offsets)
    x, bits = solve(tdp, a, S.b, c, d, n, 1)
    assert not bits & tdp.ST_FALLBACK
    assert oracle.rel_err(x, oracle.thomas(a, S.b, c, d)) <= 1e-12
    for k in (500, -500):
        A, B, C, D = (np.ldexp(v, k) for v in (S.a, S.b, S.c, S.d))
        x, bits = solve(tdp, A, B, C, D, n, 1)
        assert bits & tdp.ST_FALLBACK
        assert oracle.rel_err(x, oracle.thomas(A, B, C, D)) <= 1e-12


def test_window_zero_and_quiet_right_hand_sides(tdp):
    """d = 0 gives x = 0 exactly; a system whose second half has d 2^-200
    smaller is solved to binary64 accuracy, the quiet half (away from the
    tile that holds both scales) to its own scale."""
    n = 100_003
    S = W.single(n, seed=31)
    x, bits = solve(tdp, S.a, S.b, S.c, np.zeros(n), n, 1)
    assert not bits & tdp.ST_FALLBACK
    assert np.all(x == 0.0)
    d = S.d.copy()
    h = n // 2
    d[h:] = np.ldexp(d[h:], -200)
    ref = oracle.thomas(S.a, S.b, S.c, d)
    x, bits = solve(tdp, S.a, S.b, S.c, d, n, 1)
    assert not bits & tdp.ST_FALLBACK
    assert oracle.rel_err(x, ref) <= 1e-12
    q = h + 2 * TILE
    assert oracle.rel_err(x[q:], ref[q:]) <= 1e-12


@pytest.mark.parametrize("spread,fallback", [(20, False), (300, True)])
def test_window_batch_of_mixed_scales(tdp, spread, fallback):
    """Systems whose right-hand sides are scaled by 2^-spread, 1, 2^spread in
    turn, every system against the oracle on its own.  Neighbours within 2^40
    share windows; 2^300 apart, a window that holds both falls back (the
    smaller system's residual would fall below the binary32 range)."""
    import torch

    Sb = W.batched(64, 64, 20000, seed=33)
    d = Sb.d.copy()
    for j in range(Sb.batch):
        lo, hi = int(Sb.offsets[j]), int(Sb.offsets[j + 1])
        d[lo:hi] = np.ldexp(d[lo:hi], spread * (j % 3 - 1))
    ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, d, offsets=Sb.offsets)
    A, B, C, D = (dev(v) for v in (Sb.a, Sb.b, Sb.c, d))
    x = torch.full_like(D, float("nan"))
    tdp.tdp_solve_batched(dev(Sb.offsets), Sb.batch, Sb.n, A, B, C, D, x, 0, tdp.F32_REFINE, 1)
    torch.cuda.synchronize()
    assert bool(tdp.LIB.tdp_last_status_bits() & tdp.ST_FALLBACK) == fallback
    e = per_system_err(host(x), ref, Sb.offsets)
    assert e <= 1e-12, (spread, e)


def test_window_update_near_binade_edges(tdp):
    """x* of signed powers of two and zeros: the binary32 solution lies on or
    next to the ends of its binade and at zero, where the correction is added
    by the binary64 pipe (the integer update would leave the binade)."""
    n = 200_003
    S = W.binade_edges(n, seed=37)
    ref = oracle.thomas(S.a, S.b, S.c, S.d)
    for iters in (1, 2):
        x, bits = solve(tdp, S.a, S.b, S.c, S.d, n, iters)
        assert not bits & tdp.ST_FALLBACK
        assert oracle.rel_err(x, ref) <= 1e-12
        assert oracle.rel_err(x, S.xstar) <= 1e-12


@pytest.mark.parametrize("knob", ["window_off", "recursion"])
def test_exact_refinement_schedules_at_any_scale(tdp, knob):
    """The exact refinement schedules (windowed pass off, or the paper's
    recursion schedule) narrow d to binary32 without a scale: a system with a
    nonzero |d| outside [2^-70, 2^70] sets the gate of the exact binary64
    solve after them (fallback bit), single and batched; inside, no fallback."""
    import torch

    key = tdp.TUNE_WINDOW if knob == "window_off" else tdp.TUNE_RECURSION
    old = tdp.tdp_get_tuning(key)
    tdp.tdp_set_tuning(key, 0 if knob == "window_off" else 1)
    try:
        n = 200_003
        S = W.single(n, seed=47)
        for k, fallback in ((0, False), (-300, True), (300, True)):
            d = np.ldexp(S.d, k)
            x, bits = solve(tdp, S.a, S.b, S.c, d, n, 1)
            assert bool(bits & tdp.ST_FALLBACK) == fallback, k
            assert oracle.rel_err(x, oracle.thomas(S.a, S.b, S.c, d)) <= 1e-12, k
        Sb = W.batched(40, 64, 9000, seed=48)
        d = Sb.d.copy()
        lo, hi = int(Sb.offsets[7]), int(Sb.offsets[8])
        d[lo:hi] = np.ldexp(d[lo:hi], -200)
        A, B, C, D = (dev(v) for v in (Sb.a, Sb.b, Sb.c, d))
        x = torch.full_like(D, float("nan"))
        tdp.tdp_solve_batched(dev(Sb.offsets), Sb.batch, Sb.n, A, B, C, D, x, 0, tdp.F32_REFINE, 1)
        torch.cuda.synchronize()
        assert tdp.LIB.tdp_last_status_bits() & tdp.ST_FALLBACK
        ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, d, offsets=Sb.offsets)
        assert per_system_err(host(x), ref, Sb.offsets) <= 1e-12
    finally:
        tdp.tdp_set_tuning(key, old)


def test_window_bad_offsets(tdp):
    import torch

    Sb = W.batched(sizes=[10, 20], seed=1)
    A, B, C, D = (dev(v) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
    x = torch.empty_like(D)
    for bad in ([0, 20, 10], [1, 10, 30], [0, 10, 29]):
        with pytest.raises(tdp.TdpError) as ei:
            tdp.tdp_solve_batched(dev(np.array(bad, dtype=np.int64)), 2, 30, A, B, C, D, x, 0, tdp.F32_REFINE, 1)
        assert ei.value.code == tdp.EINVAL


def test_bad_offsets_inside_large_batches(tdp):
    """Offsets that are unsorted, past the end or negative in the middle of a
    batch of large systems (the cut points fall inside the windows and tiles
    of the windowed passes and of the binary64 flat batch) are reported as
    TDP_EINVAL by every precision; the kernels' cuts stay inside their tiles."""
    import torch

    Sb = W.batched(sizes=[5000] * 8, seed=2)
    good = Sb.offsets.copy()
    for code, dt, iters in ((tdp.F64, torch.float64, 0), (tdp.F32, torch.float32, 0),
                            (tdp.F32_REFINE, torch.float64, 1)):
        A, B, C, D = (torch.from_numpy(v).to("cuda", dt) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
        x = torch.empty_like(D)
        for j, v in ((3, 31_000), (3, 10 ** 9), (3, -7), (6, 2)):
            bad = good.copy()
            bad[j] = v
            with pytest.raises(tdp.TdpError) as ei:
                tdp.tdp_solve_batched(dev(bad), Sb.batch, Sb.n, A, B, C, D, x, 0, code, iters)
            assert ei.value.code == tdp.EINVAL, (code, j, v)
        x = torch.full_like(D, float("nan"))
        tdp.tdp_solve_batched(dev(good), Sb.batch, Sb.n, A, B, C, D, x, 0, code, iters)
        torch.cuda.synchronize()
        ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=good)
        assert per_system_err(host(x), ref, good) <= (1e-5 if code == tdp.F32 else 1e-12), code


def test_window_heat_step_passes_its_bound(tdp):
    """tridiag(-r, 1 + 2r, -r) at r = 0.5: every factor of the decay bound,
    |a| / (|b| - |c|) = r / (1 + r), is 1/3, and 48 halo rows give
    3^-48 < 2^-46, so the windowed pass answers."""
    n = 1 << 20
    r = 0.5
    a = np.full(n, -r)
    b = np.full(n, 1 + 2 * r)
    c = np.full(n, -r)
    d = W.uniform(9, 5, n, 0.0, 1.0)
    ref = oracle.thomas(a, b, c, d)
    x, bits = solve(tdp, a, b, c, d, n, 1)
    assert not bits & tdp.ST_FALLBACK
    assert oracle.rel_err(x, ref) <= 1e-12


def test_window_falls_back_on_a_weak_region(tdp):
    """A strongly dominant system with one nearly weakly dominant stretch of
    5000 rows: the tiles around it fail the decay bound, the exact binary64
    solve answers (fallback bit set), and the answer matches the oracle.
    A shorter halo (16 rows) fails the bound on ordinary tiles as well."""
    n = 1_000_003
    S = W.single(n, seed=17)
    a, c = S.a.copy(), S.c.copy()
    b = S.b.copy()
    lo, hi = 500_000, 505_000
    b[lo:hi] = (np.abs(a[lo:hi]) + np.abs(c[lo:hi])) * (1 + 1e-3)
    d = W.matvec(a, b, c, S.xstar, S.offsets)
    ref = oracle.thomas(a, b, c, d)
    x, bits = solve(tdp, a, b, c, d, n, 1)
    assert bits & tdp.ST_FALLBACK
    assert oracle.rel_err(x, ref) <= 1e-12
    # an input that is not diagonally dominant at all: fallback, still exact (binary64)
    b2 = S.b.copy()
    b2[123_456] = 0.25  # |a| + |c| may exceed b here
    d2 = W.matvec(S.a, b2, S.c, S.xstar, S.offsets)
    ref2 = oracle.thomas(S.a, b2, S.c, d2)
    x2, bits2 = solve(tdp, S.a, b2, S.c, d2, n, 1)
    if abs(S.a[123_456]) + abs(S.c[123_456]) > 0.25:
        assert bits2 & tdp.ST_FALLBACK
    assert oracle.rel_err(x2, ref2) <= 1e-12
    old = tdp.tdp_get_tuning(tdp.TUNE_WINDOW_HALO)
    tdp.tdp_set_tuning(tdp.TUNE_WINDOW_HALO, 16)
    try:
        x3, _ = solve(tdp, S.a, S.b, S.c, S.d, n, 1)
        assert oracle.rel_err(x3, oracle.thomas(S.a, S.b, S.c, S.d)) <= 1e-12
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_WINDOW_HALO, old)


@pytest.mark.parametrize("pinned", [True, False])
def test_window_host_arrays_with_fallback(tdp, pinned):
    """tdp_solve_host streams the windowed pass chunk by chunk; when a tile
    fails, the exact solve rewrites x after every chunk has been copied out:
    straight into the caller's pinned array, or through the device copy for a
    pageable one.  A system with one weak stretch (fallback) and one without."""
    import torch

    n = 1_000_003
    S = W.single(n, seed=43)
    b = S.b.copy()
    lo, hi = 700_000, 704_000
    b[lo:hi] = (np.abs(S.a[lo:hi]) + np.abs(S.c[lo:hi])) * (1 + 1e-3)
    d = W.matvec(S.a, b, S.c, S.xstar, S.offsets)
    for bb, dd, fallback in ((S.b, S.d, False), (b, d, True)):
        ref = oracle.thomas(S.a, bb, S.c, dd)
        hs = [torch.from_numpy(np.ascontiguousarray(v)) for v in (S.a, bb, S.c, dd)]
        hx = torch.full((n,), float("nan"), dtype=torch.float64)
        if pinned:
            hs = [h.pin_memory() for h in hs]
            hx = hx.pin_memory()
        tdp.tdp_solve_host(*hs, hx, n, 0, tdp.F32_REFINE, 1)
        torch.cuda.synchronize()
        assert bool(tdp.LIB.tdp_last_status_bits() & tdp.ST_FALLBACK) == fallback
        assert oracle.rel_err(hx.numpy(), ref) <= 1e-12, (pinned, fallback)


def test_window_fallback_timeout_reported(tdp):
    """The fallback's grid barrier made unreachable (testing key): its wait
    runs out and the call reports TDP_ETIMEOUT; with the gate clear the
    fallback returns at once and never waits."""
    n = 200_003
    S = W.weak(n, 1e-3, seed=2)
    G = W.single(n, seed=2)
    old = (tdp.tdp_get_tuning(tdp.TUNE_WAIT_NEVER), tdp.tdp_get_tuning(tdp.TUNE_WAIT_LOG2))
    tdp.tdp_set_tuning(tdp.TUNE_WAIT_LOG2, 14)
    tdp.tdp_set_tuning(tdp.TUNE_WAIT_NEVER, 1)
    try:
        with pytest.raises(tdp.TdpError) as ei:
            solve(tdp, S.a, S.b, S.c, S.d, n, 1)
        assert ei.value.code == tdp.ETIMEOUT
        x, bits = solve(tdp, G.a, G.b, G.c, G.d, n, 1)  # every tile passes: no barrier is reached
        assert not bits & tdp.ST_FALLBACK
        assert oracle.rel_err(x, oracle.thomas(G.a, G.b, G.c, G.d)) <= 1e-12
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_WAIT_NEVER, old[0])
        tdp.tdp_set_tuning(tdp.TUNE_WAIT_LOG2, old[1])


def solve32(tdp, a, b, c, d, n, offsets=None):
    import torch

    A, B, C, D = (dev(np.asarray(v, dtype=np.float32)) for v in (a, b, c, d))
    x = torch.full_like(D, float("nan"))
    if offsets is None:
        tdp.tdp_solve(A, B, C, D, x, n, 0, tdp.F32, 0)
    else:
        tdp.tdp_solve_batched(dev(offsets), len(offsets) - 1, n, A, B, C, D, x, 0, tdp.F32, 0)
    torch.cuda.synchronize()
    return host(x), tdp.LIB.tdp_last_status_bits()


def test_window_binary32_storage(tdp):
    """Binary32 storage through the windowed pass (no refinement; the
    window's bound is 2^-30 ||x||): tile-boundary sizes, a batch with tiny and
    empty systems, and inputs that fail the bound (fallback: the exact
    binary64 solve, rounded to binary32).  Tolerance 1e-5 against the
    oracle's binary64 Thomas of the binary32-rounded inputs.  The heat step
    at r = 1 (decay factor 1/2 per row: 2^-32 over the 32 halo rows) passes."""
    # (longer systems take longer windows: 9 rows per thread from about 1e6
    # rows, 11 from about 1.25e6, 13 from about 1.5e6 on 152 SMs)
    for n in (1, 2, 3, 5, 97, TILE32 - 1, TILE32, TILE32 + 1, 2 * TILE32 + 3, 100_003, (1 << 20) + 1, 1_300_007,
              1_500_001, (1 << 22) + 5):
        S = W.single(n, seed=n + 29)
        a, b, c, d = (v.astype(np.float32).astype(np.float64) for v in (S.a, S.b, S.c, S.d))
        x, bits = solve32(tdp, a, b, c, d, n)
        assert not bits & tdp.ST_FALLBACK, n
        assert oracle.rel_err(x, oracle.thomas(a, b, c, d)) <= 1e-5, n
    Sb = W.batched(sizes=[0, 1, 2, 3, 0, 5, 64, 1, 1700, 47, 48, 0, 5000, 300], seed=8)
    a, b, c, d = (v.astype(np.float32).astype(np.float64) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
    x, bits = solve32(tdp, a, b, c, d, Sb.n, Sb.offsets)
    assert not bits & tdp.ST_FALLBACK
    assert per_system_err(x, oracle.thomas_batched(a, b, c, d, offsets=Sb.offsets), Sb.offsets) <= 1e-5
    Sw = W.weak(200_003, 1e-3, seed=9)
    a, b, c, d = (v.astype(np.float32).astype(np.float64) for v in (Sw.a, Sw.b, Sw.c, Sw.d))
    x, bits = solve32(tdp, a, b, c, d, Sw.n)
    assert bits & tdp.ST_FALLBACK
    assert oracle.rel_err(x, oracle.thomas(a, b, c, d)) <= 1e-5
    n = 1 << 20
    a, b, c = np.full(n, -1.0), np.full(n, 3.0), np.full(n, -1.0)
    d = W.uniform(9, 5, n, 0.0, 1.0).astype(np.float32).astype(np.float64)
    x, bits = solve32(tdp, a, b, c, d, n)
    assert not bits & tdp.ST_FALLBACK
    assert oracle.rel_err(x, oracle.thomas(a, b, c, d)) <= 1e-5
