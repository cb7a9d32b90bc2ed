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
