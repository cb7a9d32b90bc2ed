"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances (relative, infinity norm against the oracle's binary64 answer):
binary64 1e-12, binary32 before refinement 1e-5, binary32 + binary64
refinement 1e-12.  Interface systems are compared row-normalised (each row
divided by its diagonal: the interface equations are unique up to scaling).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-12}


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
    """Largest relative infinity-norm error over the systems of a batch (so
    that a short system's error is not hidden behind a long one's norm)."""
    worst = 0.0
    for j in range(len(offsets) - 1):
        lo, hi = int(offsets[j]), int(offsets[j + 1])
        if hi > lo:
            worst = max(worst, oracle.rel_err(x[lo:hi], ref[lo:hi]))
    return worst


def _solve(tdp, S, s, code, iters=1):
    import torch

    dt = torch.float32 if code == 1 else torch.float64
    a, b, c, d = (dev(v, dt) for v in (S.a, S.b, S.c, S.d))
    x = torch.empty_like(d)
    tdp.tdp_solve(a, b, c, d, x, S.n, s, code, iters if code == 2 else 0)
    torch.cuda.synchronize()
    return host(x)


SIZES = [1, 2, 3, 4, 5, 31, 32, 33, 63, 64, 65, 1000, 4097, 65536, 100_003]
SUBS = [2, 3, 4, 7, 8, 16, 32, 64, 100, 1024]


@pytest.mark.parametrize("code", [0, 1, 2])
@pytest.mark.parametrize("n", SIZES)
def test_single_vs_oracle(tdp, n, code):
    S = W.single(n, seed=n)
    ref = oracle.thomas(S.a, S.b, S.c, S.d)
    for s in SUBS:
        x = _solve(tdp, S, s, code)
        e = oracle.rel_err(x, ref)
        assert e <= TOL[code], (n, s, code, e)


@pytest.mark.parametrize("code", [1, 2])
def test_exact_schedules_vs_oracle(tdp, code):
    """The exact binary32 and binary32 + refinement schedules (the windowed
    passes off: Stage 1, the binary64 interface recursion, Stage 3; the
    three-pass refinement) against the oracle, every size and sub-system size
    of test_single_vs_oracle."""
    keys = (tdp.TUNE_WINDOW, tdp.TUNE_WINDOW32)
    old = [tdp.tdp_get_tuning(k) for k in keys]
    for k in keys:
        tdp.tdp_set_tuning(k, 0)
    try:
        for n in SIZES:
            S = W.single(n, seed=n + 1)
            ref = oracle.thomas(S.a, S.b, S.c, S.d)
            for s in SUBS:
                e = oracle.rel_err(_solve(tdp, S, s, code), ref)
                assert e <= TOL[code], (n, s, e)
    finally:
        for k, v in zip(keys, old):
            tdp.tdp_set_tuning(k, v)


def test_fp32_really_single_precision(tdp):
    S = W.single(50_000, seed=3)
    ref = oracle.thomas(S.a, S.b, S.c, S.d)
    e32 = oracle.rel_err(_solve(tdp, S, 32, 1), ref)
    e0 = oracle.rel_err(_solve(tdp, S, 32, 2, iters=0), ref)
    e1 = oracle.rel_err(_solve(tdp, S, 32, 2, iters=1), ref)
    e2 = oracle.rel_err(_solve(tdp, S, 32, 2, iters=2), ref)
    assert 1e-9 < e32 <= 1e-5 and 1e-9 < e0 <= 1e-5
    assert e1 <= 1e-12 and e2 <= 1e-13
    assert e2 <= e1 <= e0


def test_predicted_s(tdp):
    S = W.single(70_001, seed=9)
    ref = oracle.thomas(S.a, S.b, S.c, S.d)
    for code in (0, 1, 2):
        assert oracle.rel_err(_solve(tdp, S, 0, code), ref) <= TOL[code]


def _normalise(a, b, c, d):
    return a / b, c / b, d / b


@pytest.mark.parametrize("code", [0, 1])
def test_stage1_interface_system(tdp, code):
    import torch

    for n, s in ((1000, 8), (1027, 32), (33, 4), (64, 64), (9, 2), (10, 3)):
        S = W.single(n, seed=n + s)
        dt = torch.float32 if code == 1 else torch.float64
        a, b, c, d = (dev(v, dt) for v in (S.a, S.b, S.c, S.d))
        m = (n + s - 1) // s
        R = [torch.zeros(2 * m, dtype=torch.float64, device="cuda") for _ in range(4)]
        tdp.tdp_stage1(a, b, c, d, n, s, code, *R)
        torch.cuda.synchronize()
        ra, rb, rc, rd = (host(t) for t in R)
        src = S if code == 0 else S.astype(np.float32).astype(np.float64)
        _, red = oracle.partition(src.a, src.b, src.c, src.d, s)
        # the library emits two rows per block; a one-row last block gets an identity row
        keep = np.ones(2 * m, dtype=bool)
        if n % s == 1:
            keep[-1] = False
            assert ra[-1] == 0 and rb[-1] == 1 and rc[-1] == 0 and rd[-1] == 0
        g = _normalise(ra[keep], rb[keep], rc[keep], rd[keep])
        o = _normalise(red["a"], red["b"], red["c"], red["d"])
        tol = 1e-13 if code == 0 else 2e-6
        for u, v in zip(g, o):
            assert np.max(np.abs(u - v)) <= tol * max(1.0, np.max(np.abs(v))), (n, s)


@pytest.mark.parametrize("code", [0, 1, 2])
def test_batched_uneven(tdp, code):
    import torch

    sizes = [0, 1, 2, 3, 5, 64, 65, 127, 1000, 0, 4097, 31, 32, 33, 1]
    Sb = W.batched(sizes=sizes, seed=4)
    ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
    dt = torch.float32 if code == 1 else torch.float64
    a, b, c, d = (dev(v, dt) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
    off = dev(Sb.offsets)
    for s in (2, 4, 32, 100):
        x = torch.empty_like(d)
        tdp.tdp_solve_batched(off, len(sizes), Sb.n, a, b, c, d, x, s, code, 1 if code == 2 else 0)
        torch.cuda.synchronize()
        e = per_system_err(host(x), ref, Sb.offsets)
        assert e <= TOL[code], (s, e)


def test_batched_log_uniform_small(tdp):
    import torch

    Sb = W.batched(256, 64, 65536, seed=0)
    ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
    a, b, c, d = (dev(v) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
    off = dev(Sb.offsets)
    for code in (0, 2):
        x = torch.empty_like(d)
        tdp.tdp_solve_batched(off, Sb.batch, Sb.n, a, b, c, d, x, 0, code, 1 if code == 2 else 0)
        torch.cuda.synchronize()
        assert per_system_err(host(x), ref, Sb.offsets) <= 1e-12


def test_bad_offsets_reported(tdp):
    import torch

    Sb = W.batched(sizes=[10, 20], seed=1)
    a, b, c, d = (dev(v) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
    x = torch.empty_like(d)
    for bad in ([0, 20, 10], [1, 10, 30], [0, 10, 29]):
        off = dev(np.array(bad, dtype=np.int64))
        with pytest.raises(tdp.TdpError) as ei:
            tdp.tdp_solve_batched(off, 2, 30, a, b, c, d, x, 4, 0, 0)
        assert ei.value.code == 1


def test_zero_pivot_reported(tdp):
    import torch

    S = W.single(100, seed=2)
    b = S.b.copy()
    b[40] = 0.0
    a = S.a.copy()
    c = S.c.copy()
    a[40] = 0.0
    c[40] = 0.0  # row 40 reads 0 = d[40]: singular
    A, B, C, D = (dev(v) for v in (a, b, c, S.d))
    x = torch.empty_like(D)
    with pytest.raises(tdp.TdpError) as ei:
        tdp.tdp_solve(A, B, C, D, x, 100, 8, 0, 0)
    assert ei.value.code == 3


def test_thomas_baseline(tdp):
    import torch

    Sb = W.batched(sizes=[1, 2, 3, 100, 4000, 0, 7], seed=5)
    ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
    for code, dt, tol in ((0, torch.float64, 1e-14), (1, torch.float32, 1e-5)):
        a, b, c, d = (dev(v, dt) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
        x = torch.empty_like(d)
        tdp.tdp_thomas_batched(dev(Sb.offsets), Sb.batch, Sb.n, a, b, c, d, x, code)
        torch.cuda.synchronize()
        assert oracle.rel_err(host(x), ref) <= tol


@pytest.mark.parametrize("code", [0, 1, 2])
def test_strided_heat_step(tdp, code):
    import torch

    n = 256
    H = W.heat(n, 0.5, seed=1)
    rows_ref, cols_ref = oracle.heat_step(H.a, H.b, H.c, H.u)
    dt = torch.float32 if code == 1 else torch.float64
    a, b, c, u = (dev(v.reshape(-1), dt) for v in (H.a, H.b, H.c, H.u))
    rows = torch.empty_like(u)
    tdp.tdp_solve_strided(n, n, n, 1, a, b, c, u, rows, 16, code, 1 if code == 2 else 0)
    cols = torch.empty_like(u)
    tdp.tdp_solve_strided(n, n, 1, n, a, b, c, rows, cols, 16, code, 1 if code == 2 else 0)
    torch.cuda.synchronize()
    assert oracle.rel_err(host(rows), rows_ref.reshape(-1)) <= TOL[code]
    assert oracle.rel_err(host(cols), cols_ref.reshape(-1)) <= 2 * TOL[code]


@pytest.mark.parametrize("code", [0, 1, 2])
def test_strided_layouts(tdp, code):
    """Strided batches beyond the square grid: the interleaved layout (element
    i of system j at j + i*es, gathered by tiled transposes) with ragged tiles
    (37 systems of 1000 rows, es = 37 and es = 40 with padding), and a padded
    row-major layout (j*ss + i, ss = n + 3); every system against the oracle."""
    import torch

    dt = torch.float32 if code == 1 else torch.float64
    for batch, n, ss, es in ((37, 1000, 1, 37), (37, 1000, 1, 40), (5, 3001, 3004, 1), (64, 33, 1, 64)):
        size = (batch - 1) * ss + (n - 1) * es + 1
        S = W.batched(sizes=[n] * batch, seed=batch + n)
        arrs = []
        for v, fill in ((S.a, 0.0), (S.b, 1.0), (S.c, 0.0), (S.d, 0.0)):
            buf = np.full(size, fill)
            for j in range(batch):
                buf[j * ss + np.arange(n) * es] = v[j * n:(j + 1) * n]
            arrs.append(torch.from_numpy(buf).to("cuda", dt))
        x = torch.full((size,), float("nan"), dtype=dt, device="cuda")
        tdp.tdp_solve_strided(batch, n, ss, es, *arrs, x, 0, code, 1 if code == 2 else 0)
        torch.cuda.synchronize()
        xs = host(x)
        ref = oracle.thomas_batched(S.a, S.b, S.c, S.d, offsets=S.offsets)
        for j in range(batch):
            got = xs[j * ss + np.arange(n) * es]
            assert oracle.rel_err(got, ref[j * n:(j + 1) * n]) <= TOL[code], (batch, n, ss, es, j)


@pytest.mark.parametrize("code", [0, 1, 2])
def test_backward_vs_oracle(tdp, code):
    """code 2: binary64 arrays, the transposed solve in binary32 with one
    binary64 correction (the windowed pass)."""
    import torch

    sizes = [64, 1, 2, 300, 129]
    Sb = W.batched(sizes=sizes, seed=6)
    x = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
    g = W.loss_weights(Sb.n, seed=6)
    ref = oracle.adjoint_batched(Sb.a, Sb.b, Sb.c, x, g, Sb.offsets)
    dt = torch.float32 if code == 1 else torch.float64
    a, b, c, X, G = (dev(v, dt) for v in (Sb.a, Sb.b, Sb.c, x, g))
    outs = [torch.empty_like(X) for _ in range(4)]
    tdp.tdp_solve_backward(dev(Sb.offsets), len(sizes), Sb.n, a, b, c, X, G, *outs, 8, code)
    torch.cuda.synchronize()
    tol = 1e-5 if code == 1 else 1e-12
    for k, o in zip("abcd", outs):
        assert oracle.rel_err(host(o), ref[k]) <= tol, k


@pytest.mark.parametrize("refine", [False, True])
@pytest.mark.parametrize("n", [64, 100_003])
def test_autograd_function(tdp, refine, n):
    import torch

    S = W.single(n, seed=8)
    w = W.loss_weights(n, seed=8)
    a, b, c, d = (dev(v).requires_grad_(True) for v in (S.a, S.b, S.c, S.d))
    x = tdp.tridiagonal_solve(a, b, c, d, s=8 if n == 64 else 0, refine=refine)
    loss = (dev(w) * x).sum()
    loss.backward()
    xo = oracle.thomas(S.a, S.b, S.c, S.d)
    ref = oracle.adjoint(S.a, S.b, S.c, xo, w)
    assert oracle.rel_err(host(x.detach()), xo) <= 1e-12
    for k, t in zip("abcd", (a, b, c, d)):
        assert oracle.rel_err(host(t.grad), ref[k]) <= 1e-12, k


def test_device_size_model_matches_host(tdp, tmp_path):
    import torch

    Sb = W.batched(300, 16, 1 << 20, seed=9)
    off = dev(Sb.offsets)
    out = torch.zeros(Sb.batch, dtype=torch.int32, device="cuda")
    sizes = np.diff(Sb.offsets)
    for table in (None, "0 100 1 4\n0 3000 1 8\n0 40000 1 16\n0 1000000 1 32\n0 300 300 6\n0 100000 300 24\n"):
        if table is not None:
            p = tmp_path / "t.txt"
            p.write_text(table)
            tdp.tdp_load_table(str(p))
        try:
            tdp.tdp_predict_s_batched(off, Sb.batch, 0, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            ref = [tdp.tdp_predict_s(int(n), Sb.batch, 0) for n in sizes]
            assert list(got) == ref
        finally:
            tdp.tdp_load_table("")


def test_batched_per_system_sizes(tdp, tmp_path):
    import torch

    p = tmp_path / "t.txt"
    p.write_text("0 64 4096 4\n0 2000 4096 8\n0 20000 4096 32\n2 64 4096 8\n2 50000 4096 16\n")
    tdp.tdp_load_table(str(p))
    old = tdp.tdp_get_tuning(tdp.TUNE_PER_SYSTEM_S)
    tdp.tdp_set_tuning(tdp.TUNE_PER_SYSTEM_S, 1)
    try:
        Sb = W.batched(512, 64, 65536, seed=11)
        ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
        a, b, c, d = (dev(v) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
        off = dev(Sb.offsets)
        for code in (0, 2):
            x = torch.empty_like(d)
            tdp.tdp_solve_batched(off, Sb.batch, Sb.n, a, b, c, d, x, 0, code, 1 if code == 2 else 0)
            torch.cuda.synchronize()
            assert per_system_err(host(x), ref, Sb.offsets) <= 1e-12, code
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_PER_SYSTEM_S, old)
        tdp.tdp_load_table("")


def test_cuda_graph_capture_and_autotune(tdp):
    import torch

    from paper_2510_27351_gb300 import tune

    Sb = W.batched(128, 64, 8192, seed=12)
    a, b, c, d = (dev(v) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
    off = dev(Sb.offsets)
    x = torch.empty_like(d)
    tdp.tdp_set_checked(False)
    shape = (tdp.tdp_get_tuning(tdp.TUNE_WINDOW_SW), tdp.tdp_get_tuning(tdp.TUNE_WINDOW_HALO),
             tdp.tdp_get_tuning(tdp.TUNE_SMEM_BUDGET))
    try:
        # the refinement's batches take the windowed pass: its block shape is tuned
        s, budget, ms = tune.autotune_batched(off, a, b, c, d, x, 2, 1, s_grid=(8, 16), budgets=(32768, 65536))
        assert s == 0 and ms > 0
        assert tdp.tdp_get_tuning(tdp.TUNE_WINDOW_SW) in (5, 7)
        assert tdp.tdp_get_tuning(tdp.TUNE_WINDOW_HALO) in (32, 48, 64)
        # the exact schedule's (s, shared-memory budget)
        tdp.tdp_set_tuning(tdp.TUNE_WINDOW, 0)
        try:
            s2, budget, ms2 = tune.autotune_batched(off, a, b, c, d, x, 2, 1, s_grid=(8, 16),
                                                    budgets=(32768, 65536))
        finally:
            tdp.tdp_set_tuning(tdp.TUNE_WINDOW, 1)
        assert s2 in (8, 16) and budget in (32768, 65536) and ms2 > 0
        graph = tdp.CapturedSolve(lambda st: tdp.tdp_solve_batched(off, Sb.batch, Sb.n, a, b, c, d, x, s, 2, 1, st))
        for seed in (1, 2):  # new right-hand sides in the captured buffers
            d2 = W.matvec(Sb.a, Sb.b, Sb.c, W.uniform(seed, 9, Sb.n, -1, 1), Sb.offsets)
            d.copy_(dev(d2))
            x.zero_()
            graph.replay()
            torch.cuda.synchronize()
            ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, d2, offsets=Sb.offsets)
            assert oracle.rel_err(host(x), ref) <= 1e-12
        tdp.tdp_status()
    finally:
        tdp.tdp_set_checked(True)
        tdp.tdp_set_tuning(tdp.TUNE_WINDOW_SW, shape[0])
        tdp.tdp_set_tuning(tdp.TUNE_WINDOW_HALO, shape[1])
        tdp.tdp_set_tuning(tdp.TUNE_SMEM_BUDGET, shape[2])


@pytest.mark.parametrize("code", [0, 1, 2])
def test_paper_recursion_schedule(tdp, code):
    """The recursive variant (Sec. III) with R forced to 0..5 and predicted:
    R recursive steps with the paper's sub-system sizes, then the last
    interface system solved directly; every R gives x = A^-1 d."""
    import torch

    old = (tdp.tdp_get_tuning(tdp.TUNE_RECURSION), tdp.tdp_get_tuning(tdp.TUNE_R))
    tdp.tdp_set_tuning(tdp.TUNE_RECURSION, 1)
    try:
        for n in (1000, 100_003, 1 << 20):
            S = W.single(n, seed=n + 3)
            ref = oracle.thomas(S.a, S.b, S.c, S.d)
            for R in (-1, 0, 1, 2, 3, 5):
                tdp.tdp_set_tuning(tdp.TUNE_R, R)
                for s in (4, 8, 32):
                    e = oracle.rel_err(_solve(tdp, S, s, code), ref)
                    assert e <= TOL[code], (n, R, s, e)
        Sb = W.batched(64, 64, 65536, seed=8)
        refb = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
        dt = torch.float32 if code == 1 else torch.float64
        a, b, c, d = (dev(v, dt) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
        for R in (0, 2):
            tdp.tdp_set_tuning(tdp.TUNE_R, R)
            x = torch.empty_like(d)
            tdp.tdp_solve_batched(dev(Sb.offsets), Sb.batch, Sb.n, a, b, c, d, x, 0, code, 1 if code == 2 else 0)
            torch.cuda.synchronize()
            assert oracle.rel_err(host(x), refb) <= TOL[code], R
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_RECURSION, old[0])
        tdp.tdp_set_tuning(tdp.TUNE_R, old[1])


def _const_ref(a, b, c, d2, n, batch, ss, es):
    """Oracle Thomas on materialised constant diagonals for the strided layout."""
    size = int((batch - 1) * ss + (n - 1) * es + 1)
    A, B, C = np.full(size, a), np.full(size, b), np.full(size, c)
    base = np.arange(batch, dtype=np.int64) * ss
    return oracle.thomas_batched(A, B, C, d2, base=base, length=np.full(batch, n), elem_stride=es)


@pytest.mark.parametrize("code", [0, 1, 2])
def test_constant_coefficients_vs_oracle(tdp, code):
    """tdp_solve_const against Thomas on the materialised diagonals: one system,
    back-to-back systems and interleaved systems (the column sweep layout),
    sizes with a ragged last block, every s from 2 to 512."""
    import torch

    dt = torch.float32 if code == 1 else torch.float64
    a, b, c = -0.45, 2.1, -0.55
    for n, batch, layout in ((1, 1, "seq"), (2, 3, "seq"), (3, 2, "int"), (5, 7, "int"), (64, 1, "seq"),
                             (1000, 5, "seq"), (4099, 33, "int"), (100_003, 2, "seq")):
        ss, es = (n, 1) if layout == "seq" else (1, batch)
        size = (batch - 1) * ss + (n - 1) * es + 1
        d2 = W.uniform(n + batch, 5, size, -1, 1)
        ref = _const_ref(a, b, c, d2, n, batch, ss, es)
        D = dev(d2, dt)
        for s in (2, 3, 4, 8, 16, 32, 64, 100, 512, 0):
            x = torch.zeros_like(D)
            tdp.tdp_solve_const(a, b, c, D, x, n, batch, ss, es, s, code, 1 if code == 2 else 0)
            torch.cuda.synchronize()
            e = oracle.rel_err(host(x), ref)
            assert e <= TOL[code], (n, batch, layout, s, e)


@pytest.mark.parametrize("k", [-300, 300])
def test_constant_coefficients_at_any_scale(tdp, k):
    """Binary64 storage (TDP_F32_REFINE runs binary64 arithmetic on the
    constant path): d scaled by 2^k, far outside the binary32 range, solved to
    1e-12 against Thomas on the materialised diagonals of the scaled input."""
    import torch

    a, b, c = -0.45, 2.1, -0.55
    n, batch = 4099, 9
    d2 = np.ldexp(W.uniform(17, 5, n * batch, -1, 1), k)
    ref = _const_ref(a, b, c, d2, n, batch, n, 1)
    D = dev(d2)
    for code in (0, 2):
        x = torch.zeros_like(D)
        tdp.tdp_solve_const(a, b, c, D, x, n, batch, n, 1, 0, code, 1 if code == 2 else 0)
        torch.cuda.synchronize()
        assert oracle.rel_err(host(x), ref) <= 1e-12, code


def test_constant_heat_step_closed_form(tdp):
    """The implicit heat step (b = 1 + 2r, a = c = -r) along rows then columns
    against the sine-basis closed form of tridiag(-r, 1+2r, -r)."""
    import torch

    n, r = 512, 0.5
    H = W.heat(n, r, seed=2)
    u = H.u.reshape(-1)
    rows_ref = np.concatenate([oracle.dst_const(n, r, u[i * n:(i + 1) * n]) for i in range(n)])
    cols_ref = np.stack([oracle.dst_const(n, r, rows_ref.reshape(n, n)[:, j]) for j in range(n)], axis=1).reshape(-1)
    U = dev(u)
    rows = torch.empty_like(U)
    tdp.tdp_solve_const(-r, 1 + 2 * r, -r, U, rows, n, n, n, 1, 0, 2, 1)
    cols = torch.empty_like(U)
    tdp.tdp_solve_const(-r, 1 + 2 * r, -r, rows, cols, n, n, 1, n, 0, 2, 1)
    torch.cuda.synchronize()
    assert oracle.rel_err(host(rows), rows_ref) <= 1e-12
    assert oracle.rel_err(host(cols), cols_ref) <= 1e-12


@pytest.mark.parametrize("code", [0, 1, 2])
def test_segmented_interface_solve(tdp, code):
    """Batches of >= 32 systems solve their interface systems one CTA per
    system (TDP_TUNE_SEGMENTED): interface systems from a few rows (warp
    cyclic reduction only) to tens of thousands (two levels on chip), empty
    and one-row systems; the same answer with the knob on and off."""
    import torch

    sizes = [0, 1, 2, 3, 40, 100, 1000, 5000, 20000, 65536] * 4
    Sb = W.batched(sizes=sizes, seed=21)
    ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
    dt = torch.float32 if code == 1 else torch.float64
    a, b, c, d = (dev(v, dt) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
    off = dev(Sb.offsets)
    old = tdp.tdp_get_tuning(tdp.TUNE_SEGMENTED)
    try:
        for seg in (1, 0):
            tdp.tdp_set_tuning(tdp.TUNE_SEGMENTED, seg)
            for s in (4, 16, 0):
                x = torch.full_like(d, float("nan"))
                tdp.tdp_solve_batched(off, Sb.batch, Sb.n, a, b, c, d, x, s, code, 1 if code == 2 else 0)
                torch.cuda.synchronize()
                assert oracle.rel_err(host(x), ref) <= TOL[code], (seg, s)
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_SEGMENTED, old)


@pytest.mark.parametrize("kept", [0, 1])
def test_refinement_last_pass_variants(tdp, kept):
    """Both forms of the refinement's last pass (re-solve from a, b, c and the
    binary32 residual, or elementwise from the kept binary32 coefficients),
    single systems with ragged last blocks and a batch with empty, one-row
    and two-row systems."""
    import torch

    old = tdp.tdp_get_tuning(tdp.TUNE_REFINE_KEPT)
    tdp.tdp_set_tuning(tdp.TUNE_REFINE_KEPT, kept)
    try:
        for n in (1, 2, 3, 5, 33, 1000, 4097, 100_003):
            S = W.single(n, seed=100 + n)
            ref = oracle.thomas(S.a, S.b, S.c, S.d)
            for s in (2, 3, 8, 24, 32, 100):
                for iters in (1, 2):
                    e = oracle.rel_err(_solve(tdp, S, s, 2, iters), ref)
                    assert e <= TOL[2], (kept, n, s, iters, e)
        sizes = [0, 1, 2, 3, 5, 64, 65, 127, 1000, 0, 4097, 31, 32, 33, 1]
        Sb = W.batched(sizes=sizes, seed=5)
        ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
        a, b, c, d = (dev(v) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
        off = dev(Sb.offsets)
        for s in (2, 4, 24, 100):
            x = torch.empty_like(d)
            tdp.tdp_solve_batched(off, len(sizes), Sb.n, a, b, c, d, x, s, 2, 1)
            torch.cuda.synchronize()
            e = oracle.rel_err(host(x), ref)
            assert e <= TOL[2], (kept, s, e)
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_REFINE_KEPT, old)


@pytest.mark.parametrize("key,value", [("TUNE_VTILE", 0), ("TUNE_COOP_REG", 0), ("TUNE_IFACE32", 1),
                                       ("TUNE_VTILE_B", 0), ("TUNE_VTILE_L", 0)])
def test_tuning_variants(tdp, key, value):
    """Non-default kernel choices give the same answers: register-staged
    tiles instead of the interleaved cp.async tiles, the one-launch tail
    without register-resident blocks, the first interface level of the
    binary32 solves in binary32 arithmetic,
    binary32 full blocks on the interleaved tiles.  Sizes reach the
    interface levels above 2^19 rows."""
    k = getattr(tdp, key)
    old = tdp.tdp_get_tuning(k)
    tdp.tdp_set_tuning(k, value)
    try:
        for n in (1000, 100_003, 1 << 20, 1 << 22):
            S = W.single(n, seed=7 + n)
            ref = oracle.thomas(S.a, S.b, S.c, S.d)
            for code in (0, 1, 2):
                for s in (8, 24, 32):
                    e = oracle.rel_err(_solve(tdp, S, s, code), ref)
                    assert e <= TOL[code], (key, value, n, code, s, e)
    finally:
        tdp.tdp_set_tuning(k, old)


@pytest.mark.parametrize("code", [0, 1, 2])
def test_batched_as_one_system(tdp, code):
    """Batches of large systems are solved as one block-diagonal system
    (couplings across system boundaries cut inside the tiles, or zeroed
    copies for the refinement); blocks straddle boundaries, empty and
    one-row systems sit between large ones.  The same batch with the block
    map (TUNE_BATCH_FLAT = 0) must agree."""
    import torch

    sizes = [5000, 1, 0, 8193, 4096, 12000, 2, 7, 9999, 3, 6500]
    Sb = W.batched(sizes=sizes, seed=11)
    assert Sb.n >= 4096 * len(sizes)
    ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
    dt = torch.float32 if code == 1 else torch.float64
    a, b, c, d = (dev(v, dt) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
    # the ignored entries a[first row], c[last row] of every system hold garbage
    for j in range(len(sizes)):
        lo, hi = int(Sb.offsets[j]), int(Sb.offsets[j + 1])
        if hi > lo:
            a[lo] = 3.5
            c[hi - 1] = -2.25
    off = dev(Sb.offsets)
    old = tdp.tdp_get_tuning(tdp.TUNE_BATCH_FLAT)
    try:
        # refinement: one correction cuts inside the tiles, two work on zeroed copies
        runs = [(flat, s, it) for flat in (1, 0) for s in (0, 4, 8, 12, 24, 100)
                for it in ((1, 2) if code == 2 else (0,))]
        for flat, s, it in runs:
            tdp.tdp_set_tuning(tdp.TUNE_BATCH_FLAT, flat)
            x = torch.empty_like(d)
            tdp.tdp_solve_batched(off, len(sizes), Sb.n, a, b, c, d, x, s, code, it)
            torch.cuda.synchronize()
            got = host(x)
            for j in range(len(sizes)):
                lo, hi = int(Sb.offsets[j]), int(Sb.offsets[j + 1])
                if hi > lo:
                    e = oracle.rel_err(got[lo:hi], ref[lo:hi])
                    assert e <= TOL[code], (flat, s, it, j, e)
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_BATCH_FLAT, old)


def test_padded_binary32_tiles_match_interleaved_tiles(tdp):
    """Binary32 storage: Stage 1 and Stage 3 on padded block-major tiles
    (TUNE_VTILE_L = 1) run the sweeps of the interleaved tiles
    (TUNE_VTILE_L = 0), so the answers agree bit for bit: single systems
    with and without a ragged last block (lean sweeps for full blocks, the
    per-row sweeps for the ragged one), sub-systems up to 1024 rows (fewer
    than 32 blocks per tile), and a batch solved as one system (cuts inside
    the tiles)."""
    import torch

    old = tdp.tdp_get_tuning(tdp.TUNE_VTILE_L)
    old_w = tdp.tdp_get_tuning(tdp.TUNE_WINDOW32)
    tdp.tdp_set_tuning(tdp.TUNE_WINDOW32, 0)  # the tiles belong to the exact binary32 path
    cases = [W.single(n, seed=n) for n in (1, 2, 3, 5, 7, 1000, 4096, 4099, 100_003, 1 << 20, (1 << 22) + 37)]
    Sb = W.batched(sizes=[5000, 1, 0, 8193, 4096, 12000, 2, 7, 9999, 3, 6500], seed=11)
    try:
        for S in cases + [Sb]:
            a, b, c, d = (dev(v, torch.float32) for v in (S.a, S.b, S.c, S.d))
            batched = S is Sb
            off = dev(Sb.offsets) if batched else None
            for s in (4, 8, 24, 64, 100, 1024):
                got = {}
                for v in (0, 1):
                    tdp.tdp_set_tuning(tdp.TUNE_VTILE_L, v)
                    x = torch.full_like(d, float("nan"))
                    if batched:
                        tdp.tdp_solve_batched(off, Sb.batch, Sb.n, a, b, c, d, x, s, 1, 0)
                    else:
                        tdp.tdp_solve(a, b, c, d, x, S.n, s, 1, 0)
                    torch.cuda.synchronize()
                    got[v] = host(x)
                assert np.array_equal(got[1], got[0]), (S.n, s)
                ref = (oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets) if batched
                       else oracle.thomas(S.a, S.b, S.c, S.d))
                assert oracle.rel_err(got[1], ref) <= TOL[1], (S.n, s)
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_VTILE_L, old)
        tdp.tdp_set_tuning(tdp.TUNE_WINDOW32, old_w)


@pytest.mark.parametrize("code", [0, 1])
def test_many_rhs_vs_oracle(tdp, code):
    """tdp_solve_multi: every column against the oracle's Thomas, ragged last
    blocks, padded leading dimensions (d's padding holds nan, x's padding must
    stay untouched), and a case with enough small columns for the per-column
    interface solves."""
    import torch

    dt = torch.float32 if code == 1 else torch.float64
    cases = [(n, nrhs, s) for n in (1, 2, 3, 5, 33, 1000, 4097, 100_003) for nrhs in (1, 3, 8)
             for s in (2, 3, 8, 32, 100)] + [(200, 40, 8), (5000, 33, 16)]
    for n, nrhs, s in cases:
        S = W.single(n, seed=n)
        D = W.rhs_columns(n, nrhs, seed=n)
        v = 4 if code == 1 else 2  # columns start on 16-byte boundaries
        ldd, ldx = -(-(n + 3) // v) * v, -(-(n + 5) // v) * v
        dpad = np.full((nrhs, ldd), np.nan)
        dpad[:, :n] = D
        a, b, c = (dev(v, dt) for v in (S.a, S.b, S.c))
        d = dev(dpad.reshape(-1), dt)
        x = torch.full((nrhs * ldx,), 7.0, dtype=dt, device="cuda")
        tdp.tdp_solve_multi(a, b, c, d, x, n, nrhs, ldd, ldx, s, code)
        torch.cuda.synchronize()
        X = host(x).reshape(nrhs, ldx)
        assert (X[:, n:] == 7.0).all(), (n, nrhs, s)
        for j in range(nrhs):
            ref = oracle.thomas(S.a, S.b, S.c, D[j])
            e = oracle.rel_err(X[j, :n], ref)
            assert e <= TOL[code], (n, nrhs, s, j, e)


def test_randomised_configurations(tdp):
    """Seeded random mix of sizes, sub-system sizes, precisions and entry
    points (single, batched with and without the one-system form, many
    right-hand sides), every answer against the oracle."""
    import random

    import torch

    rng = random.Random(2024)
    for case in range(60):
        code = rng.choice([0, 1, 2])
        dt = torch.float32 if code == 1 else torch.float64
        it = rng.choice([1, 2]) if code == 2 else 0
        kind = rng.choice(["single", "batched", "multi"]) if code != 2 else rng.choice(["single", "batched"])
        s = rng.choice([0, 2, 3, 4, 5, 8, 12, 16, 20, 24, 32, 48, 64, 100])
        if kind == "single":
            n = int(round(2 ** rng.uniform(0, 17)))
            S = W.single(n, seed=case)
            x = _solve(tdp, S, s, code, it)
            assert oracle.rel_err(x, oracle.thomas(S.a, S.b, S.c, S.d)) <= TOL[code], (case, n, s, code)
        elif kind == "batched":
            sizes = [int(round(2 ** rng.uniform(0, 14))) for _ in range(rng.randint(1, 40))]
            if rng.random() < 0.3:
                sizes[rng.randrange(len(sizes))] = 0
            Sb = W.batched(sizes=sizes, seed=case)
            if Sb.n == 0:
                continue
            ref = oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)
            a, b, c, d = (dev(v, dt) for v in (Sb.a, Sb.b, Sb.c, Sb.d))
            x = torch.empty_like(d)
            tdp.tdp_solve_batched(dev(Sb.offsets), len(sizes), Sb.n, a, b, c, d, x, s, code, it)
            torch.cuda.synchronize()
            got = host(x)
            for j in range(len(sizes)):
                lo, hi = int(Sb.offsets[j]), int(Sb.offsets[j + 1])
                if hi > lo:
                    assert oracle.rel_err(got[lo:hi], ref[lo:hi]) <= TOL[code], (case, sizes, s, code, j)
        else:
            n = int(round(2 ** rng.uniform(0, 15)))
            nrhs = rng.randint(1, 12)
            v = 4 if code == 1 else 2
            ld = -(-n // v) * v
            S = W.single(n, seed=case)
            D = W.rhs_columns(n, nrhs, seed=case)
            dpad = np.zeros((nrhs, ld))
            dpad[:, :n] = D
            a, b, c = (dev(vv, dt) for vv in (S.a, S.b, S.c))
            d = dev(dpad.reshape(-1), dt)
            x = torch.zeros_like(d)  # the padding past n stays as it is
            tdp.tdp_solve_multi(a, b, c, d, x, n, nrhs, ld, ld, s, code)
            torch.cuda.synchronize()
            X = host(x).reshape(nrhs, ld)
            for j in range(nrhs):
                ref = oracle.thomas(S.a, S.b, S.c, D[j])
                assert oracle.rel_err(X[j, :n], ref) <= TOL[code], (case, n, nrhs, s, code, j)


@pytest.mark.parametrize("code", [0, 1, 2])
def test_solve_host_arrays(tdp, code):
    """tdp_solve_host: host arrays in and out (pinned and pageable), the
    chunked copy/compute pipeline giving exactly tdp_solve's answer, and the
    oracle's within tolerance."""
    import torch

    dt = torch.float32 if code == 1 else torch.float64
    it = 1 if code == 2 else 0
    for n, s in ((1, 0), (1000, 8), (100_003, 16), (100_003, 12), ((1 << 22) + 777, 0), ((1 << 22) + 5, 64)):
        S = W.single(n, seed=n)
        ref = oracle.thomas(S.a, S.b, S.c, S.d)
        for pinned in (True, False):
            hs = [torch.from_numpy(getattr(S, k)).to(dt) for k in "abcd"]
            if pinned:
                hs = [h.pin_memory() for h in hs]
            hx = torch.empty_like(hs[0])
            if pinned:
                hx = hx.pin_memory()
            tdp.tdp_solve_host(*hs, hx, n, s, code, it)
            torch.cuda.synchronize()
            got = hx.double().numpy()
            assert oracle.rel_err(got, ref) <= TOL[code], (n, s, code, pinned)
            dev_x = torch.empty(n, dtype=dt, device="cuda")
            tdp.tdp_solve(*[h.cuda() for h in hs], dev_x, n, s, code, it)
            torch.cuda.synchronize()
            assert np.array_equal(host(dev_x), got), (n, s, code, pinned)


def test_device_wait_timeout_reported(tdp):
    """Failure detection without a GPU fault: with the testing key
    TDP_TUNE_WAIT_NEVER the grid barrier of the one-launch interface solve
    waits for an arrival that never comes; every wait gives up after
    2^14 cycles, the kernel returns, and the call reports TDP_ETIMEOUT.  The
    context stays usable: the same solve then matches the oracle."""
    import torch

    n, s = 1 << 20, 16  # interface system of 131,072 rows: one cooperative launch
    S = W.single(n, seed=31)
    ref = oracle.thomas(S.a, S.b, S.c, S.d)
    old = (tdp.tdp_get_tuning(tdp.TUNE_WAIT_NEVER), tdp.tdp_get_tuning(tdp.TUNE_WAIT_LOG2),
           tdp.tdp_get_tuning(tdp.TUNE_WINDOW32))
    tdp.tdp_set_tuning(tdp.TUNE_WAIT_LOG2, 14)
    tdp.tdp_set_tuning(tdp.TUNE_WAIT_NEVER, 1)
    # the windowed passes wait on no grid barrier unless they fall back
    # (tests/test_gpu_window.py makes that fallback's wait run out): binary32
    # here takes the exact schedule
    tdp.tdp_set_tuning(tdp.TUNE_WINDOW32, 0)
    try:
        for code in (0, 1):
            with pytest.raises(tdp.TdpError) as ei:
                _solve(tdp, S, s, code)
            assert ei.value.code == tdp.ETIMEOUT, code
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_WAIT_NEVER, old[0])
        tdp.tdp_set_tuning(tdp.TUNE_WAIT_LOG2, old[1])
        tdp.tdp_set_tuning(tdp.TUNE_WINDOW32, old[2])
    for code in (0, 2):
        assert oracle.rel_err(_solve(tdp, S, s, code), ref) <= TOL[code]
    # unchecked mode: the call returns at once and tdp_status reports the timeout later
    tdp.tdp_set_checked(False)
    tdp.tdp_set_tuning(tdp.TUNE_WAIT_LOG2, 14)
    tdp.tdp_set_tuning(tdp.TUNE_WAIT_NEVER, 1)
    try:
        _solve(tdp, S, s, 0)
        with pytest.raises(tdp.TdpError) as ei:
            tdp.tdp_status()
        assert ei.value.code == tdp.ETIMEOUT
        tdp.tdp_status()  # cleared by the read
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_WAIT_NEVER, old[0])
        tdp.tdp_set_tuning(tdp.TUNE_WAIT_LOG2, old[1])
        tdp.tdp_set_checked(True)


def test_device_size_model_matches_the_oracle_knn(tdp):
    """The size model's inference kernel (tdp_predict_s_batched, one system
    per thread) against the oracle's 1-NN over the built-in table (Sec. II-E:
    log2 N and log2 batch features, ties to the larger s): every table size,
    sizes between and around them, for several batch sizes."""
    import os

    import torch

    from oracle import predictor as P

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    rows = P.load_table(os.path.join(root, "paper_2510_27351_gb300", "data", "table_gb300.txt"))
    for dt in (0, 1, 2):
        mine = [(int(r[1]), int(r[2]), int(r[3])) for r in rows if int(r[0]) == dt]
        ns = sorted({n for n, _, _ in mine})
        queries = set(ns) | {1, 2, 100, 1 << 29}
        queries |= {int((x * y) ** 0.5) for x, y in zip(ns, ns[1:])}
        queries |= {n + 1 for n in ns} | {n - 1 for n in ns}
        queries = sorted(q for q in queries if q >= 1)
        for batch in (1, 2, 64, 1024, 4096):
            groups = [[q] for q in queries] if batch == 1 else [[queries[i % len(queries)] for i in range(batch)]]
            for sizes in groups:
                off = np.zeros(len(sizes) + 1, dtype=np.int64)
                np.cumsum(np.asarray(sizes, dtype=np.int64), out=off[1:])
                out = torch.zeros(len(sizes), dtype=torch.int32, device="cuda")
                tdp.tdp_predict_s_batched(dev(off), len(sizes), dt, out)
                torch.cuda.synchronize()
                got = out.cpu().numpy()
                for q, g in zip(sizes, got):
                    want = P.knn_predict([r[0] for r in mine], [r[2] for r in mine], q, k=1,
                                         train_batches=[r[1] for r in mine], query_batch=len(sizes))
                    assert int(g) == want, (dt, q, len(sizes), int(g), want)


def test_adjoint_central_differences(tdp):
    """The adjoint through the autograd Function against central differences
    on the device (h = 1e-6, every entry of a, b, c and d): systems of N = 64
    drawn like the 1024 x 8192 differentiation workload, loss L = sum(w x),
    w ~ N(0, 1).  All 2 x 4 x 64 perturbed systems of one base system are
    solved as one batch.  Agreement to 1e-6 relative (truncation O(h^2) and
    rounding O(eps / h) are both far below)."""
    import torch

    n, h = 64, 1e-6
    Sb = W.uniform_batch(4, n, seed=41)
    wts = W.loss_weights(Sb.n, seed=41)
    for j in range(4):
        lo, hi = j * n, (j + 1) * n
        base = [v[lo:hi].copy() for v in (Sb.a, Sb.b, Sb.c, Sb.d)]
        w = wts[lo:hi]
        ts = [dev(v).requires_grad_(True) for v in base]
        x = tdp.tridiagonal_solve(*ts, s=8)
        (dev(w) * x).sum().backward()
        grads = [host(t.grad) for t in ts]
        # batch of perturbed copies: for each array k and entry i, +h then -h
        P = 2 * 4 * n
        A = np.tile(base[0], P); B = np.tile(base[1], P); C = np.tile(base[2], P); D = np.tile(base[3], P)
        arrs = (A, B, C, D)
        q = 0
        for k in range(4):
            for i in range(n):
                for sign in (1.0, -1.0):
                    arrs[k][q * n + i] += sign * h
                    q += 1
        off = np.arange(P + 1, dtype=np.int64) * n
        X = torch.empty(P * n, dtype=torch.float64, device="cuda")
        tdp.tdp_solve_batched(dev(off), P, P * n, dev(A), dev(B), dev(C), dev(D), X, 8, tdp.F64, 0)
        torch.cuda.synchronize()
        L = (host(X).reshape(P, n) * w[None, :]).sum(axis=1)
        fd = ((L[0::2] - L[1::2]) / (2 * h)).reshape(4, n)
        for k in range(4):
            g = grads[k].copy()
            if k == 0:
                g[0] = fd[k][0]  # a[0] is ignored by the solver: no dependence, zero gradient both ways
            if k == 2:
                g[-1] = fd[k][-1]
            scale = np.max(np.abs(grads[k]))
            assert np.max(np.abs(fd[k] - g)) <= 1e-6 * scale, ("abcd"[k], j, np.max(np.abs(fd[k] - g)) / scale)
            if k == 0:
                assert grads[0][0] == 0.0 and abs(fd[0][0]) <= 1e-6 * scale
            if k == 2:
                assert grads[2][-1] == 0.0 and abs(fd[2][-1]) <= 1e-6 * scale
