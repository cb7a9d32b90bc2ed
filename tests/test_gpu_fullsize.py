"""CUDA path vs the CPU oracle at the benchmark's full sizes, element by
element, in the launch configuration the benchmark times (s = 0: the size
model's choice; one binary64 correction for the refinement).

* one system of 2^26 unknowns: binary64, binary32 storage, binary32 + one
  binary64 correction;
* 4096 systems of log-uniform sizes in [64, 65536] (seed 0): binary64 and
  binary32 + correction;
* the adjoint of 1024 systems of 8192;
* the implicit heat step on a 2048 x 2048 grid (rows, then columns) with
  materialised diagonals and with the constant-coefficient entry.

The oracle (binary64 Thomas in C) solves every system in full, so nothing is
sampled.  Tolerances as in test_gpu_parity.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-12}
N_FULL = 1 << 26


@pytest.fixture(scope="module")
def tdp():
    import torch

    import paper_2510_27351_gb300 as tdp

    assert torch.cuda.is_available()
    tdp.tdp_set_checked(True)
    yield tdp
    tdp.tdp_set_checked(False)


@pytest.fixture(scope="module")
def single_full():
    S = W.single(N_FULL, seed=0)
    return S, oracle.thomas(S.a, S.b, S.c, S.d)


@pytest.fixture(scope="module")
def batched_full():
    Sb = W.batched(4096, 64, 65536, seed=0)
    return Sb, oracle.thomas_batched(Sb.a, Sb.b, Sb.c, Sb.d, offsets=Sb.offsets)


def _dev(x, dtype):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


@pytest.mark.parametrize("code", [0, 1, 2])
def test_single_system_2e26(tdp, single_full, code):
    import torch

    S, ref = single_full
    dt = torch.float32 if code == 1 else torch.float64
    a, b, c, d = (_dev(getattr(S, k), dt) for k in "abcd")
    x = torch.empty_like(d)
    tdp.tdp_solve(a, b, c, d, x, S.n, 0, code, 1 if code == 2 else 0)
    torch.cuda.synchronize()
    got = x.double().cpu().numpy()
    del a, b, c, d, x
    assert np.isfinite(got).all()
    e = oracle.rel_err(got, ref)
    assert e <= TOL[code], (code, e)


@pytest.mark.parametrize("code", [0, 2])
def test_batched_4096_log_uniform(tdp, batched_full, code):
    import torch

    Sb, ref = batched_full
    a, b, c, d = (_dev(getattr(Sb, k), torch.float64) for k in "abcd")
    off = torch.from_numpy(Sb.offsets).cuda()
    x = torch.empty_like(d)
    tdp.tdp_solve_batched(off, Sb.batch, Sb.n, a, b, c, d, x, 0, code, 1 if code == 2 else 0)
    torch.cuda.synchronize()
    got = x.cpu().numpy()
    # per system, so that a small system's error is not hidden by a large one's norm
    worst = 0.0
    for j in range(Sb.batch):
        lo, hi = int(Sb.offsets[j]), int(Sb.offsets[j + 1])
        worst = max(worst, oracle.rel_err(got[lo:hi], ref[lo:hi]))
    assert worst <= TOL[code], (code, worst)


@pytest.fixture(scope="module")
def adjoint_full():
    Sa = W.uniform_batch(1024, 8192, seed=0)
    x = oracle.thomas_batched(Sa.a, Sa.b, Sa.c, Sa.d, offsets=Sa.offsets)
    g = W.loss_weights(Sa.n, seed=0)
    return Sa, x, g, oracle.adjoint_batched(Sa.a, Sa.b, Sa.c, x, g, Sa.offsets)


@pytest.mark.parametrize("code", [0, 2])
def test_adjoint_1024x8192(tdp, adjoint_full, code):
    """code 2: the transposed solve in binary32 with one binary64 correction."""
    import torch

    Sa, x, g, ref = adjoint_full
    a, b, c, X, G = (_dev(v, torch.float64) for v in (Sa.a, Sa.b, Sa.c, x, g))
    outs = [torch.empty_like(X) for _ in range(4)]
    tdp.tdp_solve_backward(torch.from_numpy(Sa.offsets).cuda(), Sa.batch, Sa.n, a, b, c, X, G, *outs, 0, code)
    torch.cuda.synchronize()
    for k, o in zip("abcd", outs):
        assert oracle.rel_err(o.cpu().numpy(), ref[k]) <= 1e-12, k


@pytest.fixture(scope="module")
def heat_full():
    H = W.heat(2048, 0.5, seed=0)
    rows_ref, cols_ref = oracle.heat_step(H.a, H.b, H.c, H.u)
    return H, rows_ref.reshape(-1), cols_ref.reshape(-1)


@pytest.mark.parametrize("code", [0, 2])
def test_heat_step_2048(tdp, heat_full, code):
    import torch

    H, rows_ref, cols_ref = heat_full
    n = 2048
    a, b, c, u = (_dev(v.reshape(-1), torch.float64) for v in (H.a, H.b, H.c, H.u))
    it = 1 if code == 2 else 0
    rows = torch.empty_like(u)
    tdp.tdp_solve_strided(n, n, n, 1, a, b, c, u, rows, 0, code, it)
    cols = torch.empty_like(u)
    tdp.tdp_solve_strided(n, n, 1, n, a, b, c, rows, cols, 0, code, it)
    torch.cuda.synchronize()
    assert oracle.rel_err(rows.cpu().numpy(), rows_ref) <= TOL[code]
    assert oracle.rel_err(cols.cpu().numpy(), cols_ref) <= 2 * TOL[code]


@pytest.mark.parametrize("code,s", [(0, 16), (2, 64), (0, 0), (2, 0)])
def test_constant_heat_step_2048(tdp, heat_full, code, s):
    import torch

    H, rows_ref, cols_ref = heat_full
    n, r = 2048, 0.5
    u = _dev(H.u.reshape(-1), torch.float64)
    it = 1 if code == 2 else 0
    rows = torch.empty_like(u)
    tdp.tdp_solve_const(-r, 1 + 2 * r, -r, u, rows, n, n, n, 1, s, code, it)
    cols = torch.empty_like(u)
    tdp.tdp_solve_const(-r, 1 + 2 * r, -r, rows, cols, n, n, 1, n, s, code, it)
    torch.cuda.synchronize()
    assert oracle.rel_err(rows.cpu().numpy(), rows_ref) <= TOL[code]
    assert oracle.rel_err(cols.cpu().numpy(), cols_ref) <= 2 * TOL[code]


@pytest.mark.parametrize("code", [1, 2])
def test_binary64_interface_levels_2e26(tdp, single_full, code):
    """The binary32 solves with every interface level in binary64
    (TUNE_IFACE32 = 0) meet the same tolerance as the default schedule."""
    old = tdp.tdp_get_tuning(tdp.TUNE_IFACE32)
    tdp.tdp_set_tuning(tdp.TUNE_IFACE32, 0)
    try:
        test_single_system_2e26(tdp, single_full, code)
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_IFACE32, old)


def test_many_rhs_2e22x16(tdp):
    """16 right-hand sides of one 2^22-row system (2^26 unknowns in all),
    binary64, every element against the oracle."""
    import torch

    n, nrhs = 1 << 22, 16
    S = W.single(n, seed=3)
    D = W.rhs_columns(n, nrhs, seed=3)
    a, b, c = (_dev(v, torch.float64) for v in (S.a, S.b, S.c))
    d = _dev(D.reshape(-1), torch.float64)
    x = torch.empty_like(d)
    tdp.tdp_solve_multi(a, b, c, d, x, n, nrhs, n, n, 0, 0)
    torch.cuda.synchronize()
    X = x.cpu().numpy().reshape(nrhs, n)
    for j in range(nrhs):
        assert oracle.rel_err(X[j], oracle.thomas(S.a, S.b, S.c, D[j])) <= 1e-12, j


@pytest.mark.parametrize("code", [0, 2])
def test_single_system_2e28_largest_swept(tdp, code):
    """The largest size of the size-model sweeps, 2^28 unknowns (2 GiB per
    binary64 array): every element against the oracle, so that no index of
    the kernels or the interface levels overflows at the top of the range."""
    import os

    import torch

    n = 1 << 28
    free, _ = torch.cuda.mem_get_info()
    try:
        host_bytes = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        host_bytes = 0
    if free < 40 * (1 << 30) or host_bytes < 48 * (1 << 30):
        pytest.skip("needs 40 GiB of free device memory and 48 GiB of host memory")
    S = W.single(n, seed=5)
    ref = oracle.thomas(S.a, S.b, S.c, S.d)
    a, b, c, d = (_dev(getattr(S, k), torch.float64) for k in "abcd")
    del S
    x = torch.empty_like(d)
    tdp.tdp_solve(a, b, c, d, x, n, 0, code, 1 if code == 2 else 0)
    torch.cuda.synchronize()
    got = x.cpu().numpy()
    del a, b, c, d, x
    torch.cuda.empty_cache()
    assert oracle.rel_err(got, ref) <= TOL[code]
