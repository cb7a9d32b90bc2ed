"""The allocation-free entry point, tdp_solve_noalloc.

It exists for callers that cannot allocate device memory when they solve
(latency-critical loops where a cudaMalloc would synchronise the device, or
a host memory pool that owns all device memory): its scratch is a static
16 MiB device array inside the library.  These tests call it through the C
ABI and compare it with tdp_solve and with the oracle's binary64 Thomas
solve, within the tolerances the other GPU tests use (binary64 1e-12,
binary32 1e-5, relative infinity norm), on two calls in a row, so that state
the shared array keeps from one call cannot leak into the next.  The file is
collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _rel(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def tdp():
    import torch

    import paper_2510_27351_gb300 as tdp

    assert torch.cuda.is_available()
    tdp.tdp_set_checked(True)
    yield tdp
    tdp.tdp_set_checked(False)


@pytest.mark.parametrize("code,tol", [(0, 1e-12), (1, 1e-5)])
def test_noalloc_matches_tdp_solve_twice(tdp, code, tol):
    import torch

    dt = torch.float64 if code == 0 else torch.float32
    for n, s, seed in ((1_000_003, 32, 11), (65_536, 16, 12)):  # two calls in a row, different systems
        S = W.single(n, seed=seed)
        a, b, c, d = (torch.from_numpy(v).to("cuda", dt) for v in (S.a, S.b, S.c, S.d))
        x_ref = torch.empty_like(d)
        tdp.tdp_solve(a, b, c, d, x_ref, n, s, code, 0)
        x = torch.full_like(d, float("nan"))
        rc = tdp.LIB.tdp_solve_noalloc(a.data_ptr(), b.data_ptr(), c.data_ptr(), d.data_ptr(), x.data_ptr(), n, s,
                                       code, torch.cuda.current_stream().cuda_stream)
        assert rc == 0, tdp.tdp_last_error()
        torch.cuda.synchronize()
        ref = x_ref.double().cpu().numpy()
        got = x.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) <= tol, (n, s, _rel(got, ref))
        assert _rel(got, oracle.thomas(S.a, S.b, S.c, S.d)) <= tol, (n, s)
        assert _rel(got, S.xstar) <= (1e-12 if code == 0 else 1e-5)


def test_noalloc_rejects_oversized_systems(tdp):
    import torch

    n = 4_000_000  # beyond the static scratch at s = 32
    a = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = tdp.LIB.tdp_solve_noalloc(a.data_ptr(), a.data_ptr(), a.data_ptr(), a.data_ptr(), a.data_ptr(), n, 32, 0,
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == 1
    assert "needs" in tdp.tdp_last_error() and "static scratch" in tdp.tdp_last_error()
    # refinement is not offered by this entry point
    rc = tdp.LIB.tdp_solve_noalloc(a.data_ptr(), a.data_ptr(), a.data_ptr(), a.data_ptr(), a.data_ptr(), 1000, 32, 2,
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == 1


def test_noalloc_reports_a_device_timeout(tdp):
    """A bounded device wait that runs out inside the allocation-free call
    (the grid barrier of the one-launch interface solve, made unreachable by
    the testing key TDP_TUNE_WAIT_NEVER) comes back as TDP_ETIMEOUT in
    checked mode, like tdp_solve; afterwards the same call succeeds again."""
    import torch

    n, s = 1 << 20, 16  # interface system of 131,072 rows: solved in one cooperative launch
    S = W.single(n, seed=21)
    a, b, c, d = (torch.from_numpy(v).cuda() for v in (S.a, S.b, S.c, S.d))
    x = torch.empty_like(d)
    st = torch.cuda.current_stream().cuda_stream
    args = (a.data_ptr(), b.data_ptr(), c.data_ptr(), d.data_ptr(), x.data_ptr(), n, s, 0, st)
    old = (tdp.tdp_get_tuning(tdp.TUNE_WAIT_NEVER), tdp.tdp_get_tuning(tdp.TUNE_WAIT_LOG2))
    tdp.tdp_set_tuning(tdp.TUNE_WAIT_LOG2, 14)
    tdp.tdp_set_tuning(tdp.TUNE_WAIT_NEVER, 1)
    try:
        assert tdp.LIB.tdp_solve_noalloc(*args) == tdp.ETIMEOUT
        assert "timed out" in tdp.tdp_last_error()
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_WAIT_NEVER, old[0])
        tdp.tdp_set_tuning(tdp.TUNE_WAIT_LOG2, old[1])
    assert tdp.LIB.tdp_solve_noalloc(*args) == tdp.OK, tdp.tdp_last_error()
    torch.cuda.synchronize()
    assert _rel(x.cpu().numpy(), oracle.thomas(S.a, S.b, S.c, S.d)) <= 1e-12
