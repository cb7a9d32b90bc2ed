"""The C ABI library on the host: it loads, exports every declared symbol,
and rejects bad arguments before touching a device (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tdp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tdp_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2510_27351_gb300 as tdp

    lib = ctypes.CDLL(tdp._build.LIB)
    names = _declared()
    assert "tdp_solve" in names and "tdp_predict_s" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(tdp.SYMBOLS) == names


def test_bad_arguments_rejected_on_host():
    import paper_2510_27351_gb300 as tdp

    lib = tdp.LIB
    # n < 1
    assert lib.tdp_solve(16, 16, 16, 16, 16, 0, 4, 0, 0, 0) == 1
    assert "n must be" in tdp.tdp_last_error()
    # s out of range
    assert lib.tdp_solve(16, 16, 16, 16, 16, 10, 1, 0, 0, 0) == 1
    assert lib.tdp_solve(16, 16, 16, 16, 16, 10, 2000, 0, 0, 0) == 1
    # null and misaligned pointers
    assert lib.tdp_solve(0, 16, 16, 16, 16, 10, 4, 0, 0, 0) == 1
    assert "null" in tdp.tdp_last_error()
    assert lib.tdp_solve(24, 16, 16, 16, 16, 10, 4, 0, 0, 0) == 1
    assert "aligned" in tdp.tdp_last_error()
    # bad dtype and refinement count
    assert lib.tdp_solve(16, 16, 16, 16, 16, 10, 4, 7, 0, 0) == 1
    assert lib.tdp_solve(16, 16, 16, 16, 16, 10, 4, 2, 9, 0) == 1
    # batched: batch < 1, null offsets
    assert lib.tdp_solve_batched(16, 0, 10, 16, 16, 16, 16, 16, 4, 0, 0, 0) == 1
    assert lib.tdp_solve_batched(0, 1, 10, 16, 16, 16, 16, 16, 4, 0, 0, 0) == 1
    # constant coefficients: s too large, zero stride, overlapping systems, aliasing, misaligned
    f = lib.tdp_solve_const
    assert f(-1.0, 4.0, -1.0, 16, 32, 10, 2, 10, 1, 600, 0, 0, 0) == 1
    assert f(-1.0, 4.0, -1.0, 16, 32, 10, 2, 0, 1, 4, 0, 0, 0) == 1
    assert f(-1.0, 4.0, -1.0, 16, 32, 10, 2, 5, 1, 4, 0, 0, 0) == 1
    assert "overlap" in tdp.tdp_last_error()
    assert f(-1.0, 4.0, -1.0, 16, 16, 10, 2, 10, 1, 4, 0, 0, 0) == 1
    assert f(-1.0, 4.0, -1.0, 20, 32, 10, 2, 10, 1, 4, 0, 0, 0) == 1
    assert "aligned" in tdp.tdp_last_error()
    # strided: bad strides
    assert lib.tdp_solve_strided(2, 8, -1, 1, 16, 16, 16, 16, 16, 4, 0, 0, 0) == 1
    # backward refuses an unknown dtype
    assert lib.tdp_solve_backward(16, 1, 8, 16, 16, 16, 16, 16, 0, 0, 0, 0, 4, 5, 0) == 1
    assert "dtype" in tdp.tdp_last_error()
    # many right-hand sides: (a, b, c, d, x, n, nrhs, ldd, ldx, s, dtype, stream)
    m = lib.tdp_solve_multi
    assert m(16, 16, 16, 1 << 20, 1 << 24, 10, 0, 10, 10, 4, 0, 0) == 1      # nrhs < 1
    assert m(16, 16, 16, 1 << 20, 1 << 24, 10, 2, 9, 10, 4, 0, 0) == 1       # ldd < n
    assert m(16, 16, 16, 1 << 20, 1 << 24, 10, 2, 10, 10, 4, 2, 0) == 1      # refinement dtype
    assert m(16, 16, 16, 1 << 20, (1 << 20) + 128, 10, 2, 10, 10, 4, 0, 0) == 1
    assert "overlap" in tdp.tdp_last_error()
    assert m(16, 16, 16, 1 << 20, (1 << 24) + 8, 10, 2, 10, 10, 4, 0, 0) == 1
    assert "aligned" in tdp.tdp_last_error()
    assert m(16, 16, 16, 1 << 20, 1 << 24, 11, 2, 11, 12, 4, 0, 0) == 1     # odd column stride
    assert "16-byte" in tdp.tdp_last_error()
    # host arrays: (a, b, c, d, x, n, s, dtype, refine_iters, stream)
    h = lib.tdp_solve_host
    assert h(16, 16, 16, 0, 1 << 24, 10, 4, 0, 0, 0) == 1
    assert "null" in tdp.tdp_last_error()
    assert h(16, 16, 16, 1 << 20, (1 << 20) + 8, 10, 4, 0, 0, 0) == 1
    assert "overlaps" in tdp.tdp_last_error()
    assert h(16, 16, 16, 1 << 20, 1 << 24, 0, 4, 0, 0, 0) == 1


def test_predictor_is_host_only_and_valid():
    import paper_2510_27351_gb300 as tdp

    for n in (1, 64, 4500, 65536, 1 << 20, 1 << 26):
        for dt in (0, 1, 2):
            s = tdp.tdp_predict_s(n, 1, dt)
            assert 2 <= s <= 1024


def test_predictor_table_loading(tmp_path):
    import paper_2510_27351_gb300 as tdp

    p = tmp_path / "t.txt"
    p.write_text("# dtype n batch s\n0 1024 1 8\n0 1048576 1 64\n0 1048576 4096 16\n")
    tdp.tdp_load_table(str(p))
    try:
        assert tdp.tdp_predict_s(1000, 1, 0) == 8
        assert tdp.tdp_predict_s(1 << 21, 1, 0) == 64
        assert tdp.tdp_predict_s(1 << 20, 4000, 0) == 16
        # equal distance in log2 N: the larger s wins
        assert tdp.tdp_predict_s(32768, 1, 0) == 64
        bad = tmp_path / "bad.txt"
        bad.write_text("0 1024 1 1\n")
        with pytest.raises(tdp.TdpError):
            tdp.tdp_load_table(str(bad))
        with pytest.raises(tdp.TdpError):
            tdp.tdp_load_table(str(tmp_path / "missing.txt"))
        assert tdp.tdp_predict_s(1000, 1, 0) == 8  # unchanged by the failed loads
    finally:
        tdp.tdp_load_table("")


def test_tuning_knobs_validate_and_round_trip():
    import paper_2510_27351_gb300 as tdp

    old = tdp.tdp_get_tuning(tdp.TUNE_S_REC)
    try:
        tdp.tdp_set_tuning(tdp.TUNE_S_REC, 16)
        assert tdp.tdp_get_tuning(tdp.TUNE_S_REC) == 16
        with pytest.raises(tdp.TdpError):
            tdp.tdp_set_tuning(tdp.TUNE_S_REC, 2)  # would not shrink the interface system
        with pytest.raises(tdp.TdpError):
            tdp.tdp_set_tuning(99, 1)
        assert tdp.tdp_get_tuning(99) == -1
        assert tdp.tdp_get_tuning(tdp.TUNE_S_REC) == 16
        # every key the header declares answers with its default range
        defaults = {tdp.TUNE_IFACE32: 0, tdp.TUNE_REFINE_KEPT: 1, tdp.TUNE_SEGMENTED: 1, tdp.TUNE_REFINE3: 1,
                    tdp.TUNE_PER_SYSTEM_S: 0, tdp.TUNE_VTILE: 1, tdp.TUNE_COOP: 1, tdp.TUNE_COOP_REG: 1,
                    tdp.TUNE_BATCH_FLAT: 1, tdp.TUNE_VTILE_B: 1, tdp.TUNE_VTILE_L: 1, tdp.TUNE_WINDOW: 1,
                    tdp.TUNE_WINDOW32: 1,
                    tdp.TUNE_WAIT_NEVER: 0}
        for key, v in defaults.items():
            assert tdp.tdp_get_tuning(key) in (0, 1) and tdp.tdp_get_tuning(key) == v, key
        assert tdp.tdp_get_tuning(tdp.TUNE_WINDOW_HALO) == 48
        assert tdp.tdp_get_tuning(tdp.TUNE_WAIT_LOG2) == 31
        assert tdp.tdp_get_tuning(tdp.TUNE_WINDOW_SW) == 7
        assert tdp.tdp_get_tuning(tdp.TUNE_WINDOW_PREFETCH) == 128
        assert tdp.tdp_get_tuning(tdp.TUNE_WINDOW_HALO32) == 32
        assert tdp.tdp_get_tuning(tdp.TUNE_WINDOW_SW32) == 13
        # the binary32 interface level is off by default: every interface
        # level of every precision runs in binary64 (the reduced system's
        # stability is what binary64 is kept for)
        for key in tdp.RETIRED_TUNING_KEYS:
            assert tdp.tdp_get_tuning(key) == -1
            with pytest.raises(tdp.TdpError, match="retired"):
                tdp.tdp_set_tuning(key, 0)
        with pytest.raises(tdp.TdpError):
            tdp.tdp_set_tuning(tdp.TUNE_WINDOW_HALO, 8)
        with pytest.raises(tdp.TdpError):
            tdp.tdp_set_tuning(tdp.TUNE_WAIT_LOG2, 41)
        with pytest.raises(tdp.TdpError):
            tdp.tdp_set_tuning(tdp.TUNE_IFACE32, 2)
        with pytest.raises(tdp.TdpError):
            tdp.tdp_set_tuning(tdp.TUNE_VTILE_L, 2)
        tdp.tdp_set_tuning(tdp.TUNE_VTILE_L, 0)
        assert tdp.tdp_get_tuning(tdp.TUNE_VTILE_L) == 0
        tdp.tdp_set_tuning(tdp.TUNE_VTILE_L, 1)
        assert tdp.tdp_get_tuning(tdp.TUNE_WINDOW_SW32 + 1) == -1
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_S_REC, old)


def test_recursion_depth_model_and_plan_match_the_oracle(tmp_path):
    """Host-only: tdp_predict_r without table rows follows the paper's
    intervals of optimum R, and tdp_recursion_plan follows the paper's rule
    for the sizes of the recursive steps (the oracle gets the library's size
    model as its size predictor, so only the rule is compared)."""
    import paper_2510_27351_gb300 as tdp
    from oracle import predictor as P

    gold = os.path.join(ROOT, "tests", "golden")
    rule = [(int(float(r[0])), int(r[1])) for r in P.load_table(os.path.join(gold, "interval_rule_R.txt"))]
    empty = tmp_path / "empty.txt"
    empty.write_text("# no rows\n")
    tdp.tdp_load_rtable(str(empty))
    try:
        for n in (1, 1000, 1e5, 2.2e6, 2.25e6, 2.3e6, 4.8e6, 4.9e6, 5e6, 9.6e6, 9.7e6, 1e7, 1e8, 1 << 28):
            assert tdp.tdp_predict_r(int(n)) == P.interval_rule_r(int(n), rule), n
    finally:
        tdp.tdp_load_rtable("")
    p = tmp_path / "r.txt"
    p.write_text("0 1048576 1 2\n0 67108864 1 4\n")
    tdp.tdp_load_rtable(str(p))
    try:
        assert tdp.tdp_predict_r(1 << 20) == 2 and tdp.tdp_predict_r(1 << 26) == 4
        assert tdp.tdp_predict_r(1 << 23) == 4  # equal log2 distance: the larger R
        bad = tmp_path / "bad.txt"
        bad.write_text("0 1024 1 13\n")
        with pytest.raises(tdp.TdpError):
            tdp.tdp_load_rtable(str(bad))
    finally:
        tdp.tdp_load_rtable("")
    pred = lambda M: tdp.tdp_predict_s(M, 1, tdp.F64)  # noqa: E731
    for n in (100, 5000, 1 << 20, 4_500_000, 1 << 26):
        for s in (2, 8, 24, 64):
            for R in range(6):
                assert tdp.tdp_recursion_plan(n, s, R) == P.recursive_sizes(n, s, R, pred), (n, s, R)
    assert tdp.LIB.tdp_recursion_plan(0, 8, 1, 0, 0, 0) == -1


def test_builtin_predictor_matches_the_oracle_knn():
    """tdp_predict_s with the built-in table is the oracle's 1-NN over the
    same rows (log2 N and log2 batch features, ties to the larger s), query
    by query: every table size, sizes between them, sizes outside the table,
    batch sizes on and between the table's buckets."""
    import paper_2510_27351_gb300 as tdp
    from oracle import predictor as P

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    rows = P.load_table(os.path.join(root, "paper_2510_27351_gb300", "data", "table_gb300.txt"))
    for dt in (0, 1, 2):
        mine = [(int(r[1]), int(r[2]), int(r[3])) for r in rows if int(r[0]) == dt]
        assert mine, dt
        ns = sorted({n for n, _, _ in mine})
        queries = set(ns) | {1, 2, 100, 1 << 29, 3 << 28}
        queries |= {int((x * y) ** 0.5) for x, y in zip(ns, ns[1:])}
        queries |= {n + 1 for n in ns} | {n - 1 for n in ns}
        for batch in (1, 2, 64, 100, 1024, 2000, 4096, 10000):
            for n in sorted(queries):
                want = P.knn_predict([r[0] for r in mine], [r[2] for r in mine], n, k=1,
                                     train_batches=[r[1] for r in mine], query_batch=batch)
                assert tdp.tdp_predict_s(n, batch, dt) == want, (dt, n, batch)


def test_builtin_recursion_depth_model_matches_the_oracle_knn():
    """tdp_predict_r with the built-in table is the oracle's 1-NN over the same
    rows (R = -1 is the library's default schedule), query by query."""
    import paper_2510_27351_gb300 as tdp
    from oracle import predictor as P

    rows = P.load_table(os.path.join(ROOT, "paper_2510_27351_gb300", "data", "table_r_gb300.txt"))
    for dt in sorted({int(r[0]) for r in rows}):
        mine = [(int(r[1]), int(r[2]), int(r[3])) for r in rows if int(r[0]) == dt]
        ns = sorted({n for n, _, _ in mine})
        queries = set(ns) | {1, 1000, 1 << 29} | {int((x * y) ** 0.5) for x, y in zip(ns, ns[1:])}
        for n in sorted(queries):
            want = P.knn_predict([r[0] for r in mine], [r[2] for r in mine], n, k=1,
                                 train_batches=[r[1] for r in mine], query_batch=1)
            assert tdp.tdp_predict_r(n, 1, dt) == want, (dt, n)


def test_status_word_maps_to_return_codes():
    """Host-only: every bit of the device status word maps to its return
    code, with the precedence argument error > timeout > pivot failure that
    tdp_status, checked-mode solves and tdp_solve_noalloc share."""
    import paper_2510_27351_gb300 as tdp

    SING, TIME, BAD = 1, 2, 4
    assert tdp.LIB.tdp_status_code(0) == tdp.OK
    assert tdp.LIB.tdp_status_code(SING) == tdp.ESINGULAR
    assert tdp.LIB.tdp_status_code(TIME) == tdp.ETIMEOUT
    assert tdp.LIB.tdp_status_code(BAD) == tdp.EINVAL
    assert tdp.LIB.tdp_status_code(SING | TIME) == tdp.ETIMEOUT
    assert tdp.LIB.tdp_status_code(SING | BAD) == tdp.EINVAL
    assert tdp.LIB.tdp_status_code(SING | TIME | BAD) == tdp.EINVAL
