"""The library's size-model code (tune.py) against the oracle and the paper."""
import os
import random

import pytest

from oracle import predictor as P

GOLD = os.path.join(os.path.dirname(__file__), "golden")


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


def test_correct_reproduces_paper_table4():
    from paper_2510_27351_gb300 import tune

    rows, times = _table4()
    raw, cor = tune.correct(times, tol=0.05)
    assert raw == [int(r[1]) for r in rows]
    assert cor == [int(r[2]) for r in rows]


def test_correct_matches_oracle_on_random_sweeps():
    from paper_2510_27351_gb300 import tune

    rng = random.Random(3)
    grid = [4, 8, 16, 20, 32, 64]
    for _ in range(200):
        n = rng.randint(2, 12)
        times = []
        for i in range(n):
            best = rng.choice(grid)
            t = {s: 1.0 + rng.uniform(0, 0.12) + 0.02 * abs(grid.index(s) - grid.index(best)) for s in grid}
            times.append(t)
        try:
            ref = P.correct_labels(times, tol=0.05)
        except RuntimeError:
            with pytest.raises(ValueError):
                tune.correct(times, tol=0.05)
            continue
        assert tune.correct(times, tol=0.05) == ref


def test_nearest_matches_oracle():
    from paper_2510_27351_gb300 import tune

    rng = random.Random(5)
    for _ in range(100):
        train = [(rng.randint(64, 1 << 26), rng.choice([1, 16, 4096]), rng.choice([4, 8, 16, 32, 64]))
                 for _ in range(rng.randint(1, 20))]
        for _ in range(10):
            n, b = rng.randint(1, 1 << 27), rng.choice([1, 16, 4096, 100])
            ref = P.knn_predict([t[0] for t in train], [t[2] for t in train], n, 1,
                                train_batches=[t[1] for t in train], query_batch=b)
            assert tune.nearest(train, n, b) == ref


def test_evaluate_protocol_on_synthetic_sweep():
    from paper_2510_27351_gb300 import tune

    rows = []
    for k in range(37):
        n = int(2 ** (10 + k / 2))
        opt = 8 if n < 2 ** 14 else 16 if n < 2 ** 20 else 32
        for s in (8, 16, 32, 64):
            rows.append({"dtype": 0, "n": n, "batch": 1, "s": s, "ms": 1.0 + 0.1 * abs(s - opt) / opt})
    rep = tune.evaluate(rows)["f64/batch1"]
    assert rep["accuracy_corrected"] >= 0.8
    assert rep["max_time_loss"] <= 0.25
    table = tune.build_table(rows)
    assert len(table) == 37 and all(r[3] in (8, 16, 32) for r in table)


def test_recursion_depth_table_and_evaluation():
    """tune.py's R pipeline on synthetic timings: the fastest R per size (ties
    to the larger R, the default schedule R = -1 excluded), and an evaluation
    whose losses are measured against that fastest R."""
    from paper_2510_27351_gb300 import tune

    rows = []
    for k, n in enumerate([1 << e for e in range(14, 26)]):
        best = 0 if n < (1 << 18) else 1 if n < (1 << 22) else 3
        for r in (-1, 0, 1, 2, 3):
            ms = 1.0 + abs(r - best) * 0.1 if r >= 0 else 1.05
            if r == best + 1 and best == 0:
                ms = 1.0  # a tie: the larger R wins
            rows.append({"dtype": 0, "n": n, "batch": 1, "R": r, "s": 8, "ms": ms})
    table = tune.build_rtable(rows)
    lab = {n: r for _, n, _, r in table}
    assert lab[1 << 14] == 1 and lab[1 << 20] == 1 and lab[1 << 24] == 3
    rep = tune.evaluate_r(rows)["f64/batch1"]
    assert rep["n_sizes"] == 12 and 0.0 <= rep["accuracy"] <= 1.0
    assert rep["mean_time_loss"] >= 0.0
    assert all(abs(v - 1.0 / 1.05) < 1e-12 for v in rep["best_over_default_all"].values())


def test_precision_transfer_study_on_synthetic_sweeps():
    """evaluate_transfer: a source precision with the same timings as the
    target transfers perfectly; one whose optimum is shifted loses exactly the
    target's time ratio at every size."""
    from paper_2510_27351_gb300 import tune

    sizes = [1 << k for k in range(10, 20)]
    rows = []
    for n in sizes:
        for s in (8, 16, 32):
            t_a = 1.0 + abs(s - 16) / 16          # optimum 16 for dtypes 0 and 1
            t_c = 1.0 + abs(s - 32) / 32          # optimum 32 for dtype 2
            rows += [{"dtype": 0, "n": n, "batch": 1, "s": s, "ms": t_a},
                     {"dtype": 1, "n": n, "batch": 1, "s": s, "ms": t_a},
                     {"dtype": 2, "n": n, "batch": 1, "s": s, "ms": t_c}]
    rep = tune.evaluate_transfer(rows)
    same = rep["f64->f32/batch1"]
    assert same["accuracy"] == 1.0 and same["mean_time_loss"] == 0.0
    shifted = rep["f64->f32_refine/batch1"]
    assert shifted["accuracy"] == 0.0
    assert shifted["mean_time_loss"] == pytest.approx(1.5 - 1.0)  # s = 16 on a target whose best is 32
    assert shifted["best_fixed_s"] == 32 and shifted["target_loo_mean_time_loss"] == 0.0
    assert set(rep) == {f"{a}->{b}/batch1" for a in ("f64", "f32", "f32_refine")
                        for b in ("f64", "f32", "f32_refine") if a != b}


def test_committed_tables_are_derived_from_the_committed_sweeps(tmp_path):
    """The size table compiled into the library (tdp_table.inc), its text copy
    and the recursion-depth table are exactly what tune.py derives from the
    committed GB300 sweeps: a re-sweep that was not turned into tables, or a
    hand-edited table, fails here."""
    from paper_2510_27351_gb300 import tune

    pkg = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2510_27351_gb300")
    data = os.path.join(pkg, "data")
    cases = [(tune.build_table, tune.write_table, "sweep_gb300.jsonl", "table_gb300.txt", "tdp_table.inc"),
             (tune.build_rtable, tune.write_rtable, "sweep_r_gb300.jsonl", "table_r_gb300.txt", "tdp_rtable.inc")]
    for build, write, sweep, txt, inc in cases:
        out_txt, out_inc = str(tmp_path / txt), str(tmp_path / inc)
        write(build(tune.load_sweep(os.path.join(data, sweep))), out_txt, out_inc)
        with open(out_txt) as f1, open(os.path.join(data, txt)) as f2:
            assert f1.read() == f2.read(), txt
        with open(out_inc) as f1, open(os.path.join(pkg, "csrc", inc)) as f2:
            assert f1.read() == f2.read(), inc


def test_committed_evaluations_are_reproduced_from_the_committed_sweeps():
    """The committed evaluation reports (size model, recursion depth model,
    transfer between precisions) are what tune.py computes from the committed
    sweeps (fixed split seed)."""
    import json

    from paper_2510_27351_gb300 import tune

    data = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2510_27351_gb300", "data")
    rows = tune.load_sweep(os.path.join(data, "sweep_gb300.jsonl"))
    rrows = tune.load_sweep(os.path.join(data, "sweep_r_gb300.jsonl"))
    for got, name in ((tune.evaluate(rows), "evaluation_gb300.json"),
                      (tune.evaluate_transfer(rows), "evaluation_transfer_gb300.json"),
                      (tune.evaluate_r(rrows), "evaluation_r_gb300.json")):
        with open(os.path.join(data, name)) as f:
            assert json.loads(json.dumps(got)) == json.load(f), name
