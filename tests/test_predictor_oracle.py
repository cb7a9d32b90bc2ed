"""The size-choice oracle against the paper's printed tables (Sec. II, IV-B)."""
import os

import pytest

from oracle import predictor as P

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = P.load_table(os.path.join(GOLD, "table1_fp64_opt_s.txt"))
    return [int(float(r[0])) for r in rows], [int(r[1]) for r in rows], [int(r[4]) for r in rows], rows


def _rule():
    return [(int(float(r[0])), int(r[1])) for r in P.load_table(os.path.join(GOLD, "interval_rule_fp64.txt"))]


def _table4():
    rows = P.load_table(os.path.join(GOLD, "table4_fp32_times.txt"))
    times = []
    for r in rows:
        t = {}
        if r[4] != "-":
            for kv in r[4:]:
                s, v = kv.split(":")
                t[int(s)] = float(v)
        else:
            t = {int(r[1]): 1.0}
        times.append(t)
    return rows, times


def test_interval_rule_matches_corrected_table1():
    sizes, _, corrected, _ = _table1()
    rule = _rule()
    assert [P.interval_rule(n, rule) for n in sizes] == corrected


def test_knn_recovers_training_labels_and_interval_rule():
    sizes, _, corrected, _ = _table1()
    rule = _rule()
    for n, lab in zip(sizes, corrected):
        assert P.knn_predict(sizes, corrected, n, 1) == lab
    # geometric midpoints of neighbouring table sizes inside one interval
    for n0, n1, l0, l1 in zip(sizes, sizes[1:], corrected, corrected[1:]):
        if l0 == l1:
            q = (n0 * n1) ** 0.5
            assert P.knn_predict(sizes, corrected, q, 1) == P.interval_rule(q, rule) == l0


def test_knn_tie_breaks_to_larger_size():
    assert P.knn_predict([64, 256], [4, 8], 128, 1) == 8  # equidistant in log2
    assert P.knn_predict([64, 256, 1024], [4, 16, 8], 128, 2) == 16


def test_grid_search_finds_k1_on_corrected_labels():
    sizes, _, corrected, _ = _table1()
    k, acc = P.grid_search_k(sizes, corrected)
    assert k == 1  # Sec. II-E: k = 1 was found
    tr_s, tr_l, te_s, te_l = P.split_3to1(sizes, corrected, seed=0)
    assert set(tr_l) == set(corrected)
    assert len(te_s) == len(sizes) // 4


def test_null_accuracy_table1_is_most_frequent_class_share():
    _, observed, corrected, _ = _table1()
    # the most frequent corrected size is 32 (12 of 37 rows)
    assert P.null_accuracy(corrected) == pytest.approx(12 / 37)


def test_fp32_transcription_matches_printed_differences():
    rows, times = _table4()
    for r, t in zip(rows, times):
        if r[3] != "-":
            obs, cor = int(r[1]), int(r[2])
            assert t[obs] - t[cor] == pytest.approx(float(r[3]), abs=2e-6 * max(1.0, t[obs]))


def test_label_correction_reproduces_table4():
    rows, times = _table4()
    raw, corrected = P.correct_labels(times, tol=0.05)
    assert raw == [int(r[1]) for r in rows]
    assert corrected == [int(r[2]) for r in rows]
    # every corrected label is non-decreasing in N and within 5% of the best
    assert all(x <= y for x, y in zip(corrected, corrected[1:]))
    for t, s in zip(times, corrected):
        assert t[s] <= 1.05 * min(t.values())


def _table_r():
    rows = P.load_table(os.path.join(GOLD, "table_opt_R.txt"))
    return [int(float(r[0])) for r in rows], [int(r[1]) for r in rows]


def _rule_r():
    return [(int(float(r[0])), int(r[1])) for r in P.load_table(os.path.join(GOLD, "interval_rule_R.txt"))]


def test_interval_rule_r_reproduces_table_of_optimum_r():
    sizes, labels = _table_r()
    rule = _rule_r()
    assert [P.interval_rule_r(n, rule) for n in sizes] == labels
    assert P.interval_rule_r(2_250_000, rule) == 1  # between two intervals: the larger R
    assert P.interval_rule_r(1e9, rule) == 3


def test_r_knn_reproduces_the_intervals():
    """Sec. III-A: a 1-NN model over the listed sizes; inside every interval of
    the table it returns that interval's R, and it reproduces its training
    labels.  (Held-out accuracy depends on the split: sizes at an interval's
    edge have their nearest neighbour across the edge.)"""
    sizes, labels = _table_r()
    assert [P.knn_predict(sizes, labels, n) for n in sizes] == labels
    probes = {150_000: 0, 1_500_000: 0, 2_450_000: 1, 3_500_000: 1, 6_500_000: 2, 9_000_000: 2, 3e7: 3, 5e8: 3}
    for n, r in probes.items():
        assert P.knn_predict(sizes, labels, n) == r, n


def test_recursive_sizes_follow_the_rule():
    """Sec. III-B: step 1 uses 10 when R >= 2; every other step uses the size
    model on the interface system it partitions (here a stub: 32 below 2^20
    rows, 64 above); each step turns M rows into 2 ceil(M / m)."""
    stub = lambda M: 32 if M < (1 << 20) else 64  # noqa: E731
    n, s = 1 << 24, 16
    M1 = 2 * (n // s)  # 2^21 rows
    assert P.recursive_sizes(n, s, 0, stub) == []
    assert P.recursive_sizes(n, s, 1, stub) == [64]  # R = 1: the model on M1
    assert P.recursive_sizes(n, s, 2, stub) == [10, 32]  # 2 ceil(2^21 / 10) = 419432 rows < 2^20
    sizes = P.recursive_sizes(n, s, 8, stub)
    M = M1
    for m in sizes:
        M = 2 * -(-M // m)
    assert sizes[0] == 10 and all(m in (32, 64) for m in sizes[1:]) and M <= 64
    assert len(sizes) < 8  # stops once the interface system has at most 64 rows
