"""Sub-system-size model: timing sweeps on the GPU, label correction, 1-NN.

This is the GB300 counterpart of the paper's heuristic (Sec. II-D, II-E,
IV-B): time the solver for every sub-system size s of a grid at many sizes
N, take the fastest s per N, correct the labels towards a trend, and fit a
1-nearest-neighbour classifier N -> s (one per precision; the batch size is
a second feature for batched solves).  The library's predictor
(``tdp_predict_s``, host and device) reads the resulting table.

    python -m paper_2510_27351_gb300.tune sweep --out sweep.jsonl
    python -m paper_2510_27351_gb300.tune table --sweep sweep.jsonl --out table.txt --inc csrc/tdp_table.inc
    python -m paper_2510_27351_gb300.tune evaluate --sweep sweep.jsonl

The sweep appends one JSON line per (dtype, n, batch, s) so that a killed
sweep resumes where it stopped.

The number of recursive steps R of the paper's recursive variant (Sec. III)
gets the same treatment: ``sweep-r`` times the paper's schedule for every R of
a grid (and the library's default schedule, recorded as R = -1), ``rtable``
writes the fastest R per size for ``tdp_predict_r``, ``evaluate-r`` reports the
1-NN accuracy, the time lost against the fastest R and the comparison with the
default schedule.

    python -m paper_2510_27351_gb300.tune sweep-r --out sweep_r.jsonl
    python -m paper_2510_27351_gb300.tune rtable --sweep sweep_r.jsonl --out table_r.txt --inc csrc/tdp_rtable.inc
    python -m paper_2510_27351_gb300.tune evaluate-r --sweep sweep_r.jsonl
"""
from __future__ import annotations

import argparse
import json
import math
import os
import random
import sys
from collections import defaultdict

S_GRID = (4, 8, 12, 16, 20, 24, 32, 40, 48, 64, 96, 128)
R_GRID = (0, 1, 2, 3, 4, 5)
DTYPES = {0: "f64", 1: "f32", 2: "f32_refine"}
TOL = 0.05  # labels within 5 % of the fastest count as near-optimal
TOL_FLAT = 0.03  # the flat fallback only smooths labels within 3 % of the fastest


# ---------------------------------------------------------------------------
# label correction (Sec. II-E)
# ---------------------------------------------------------------------------
def correct(times, tol: float = TOL):
    """``times``: per ascending size, a dict {s: time}.  Returns (raw, corrected).

    Raw label: the fastest s (ties to the larger s).  Corrected: among the
    sizes within ``tol`` of the fastest, a non-decreasing sequence over N with
    the fewest label changes, preferring larger labels (compared from the
    largest N down), then the least total relative loss.
    """
    n = len(times)
    raw = []
    cand = []
    for t in times:
        best = min(t.values())
        raw.append(max((s for s in t if t[s] == best)))
        cand.append({s: t[s] / best - 1.0 for s in t if t[s] <= (1.0 + tol) * best})
    # state per position: label -> (changes, labels from the end (negated), loss, path)
    table = [None] * n
    table[n - 1] = {s: (0, (-s,), lo, [s]) for s, lo in cand[n - 1].items()}
    for i in range(n - 2, -1, -1):
        cur = {}
        for s, lo in cand[i].items():
            best = None
            for s2, (ch, neg, loss, path) in table[i + 1].items():
                if s2 < s:
                    continue
                key = (ch + (1 if s2 != s else 0), neg + (-s,), loss + lo)
                if best is None or key < best[:3]:
                    best = key + (path + [s],)
            if best is not None:
                cur[s] = best
        table[i] = cur
    if not table[0]:
        raise ValueError("no non-decreasing label sequence within the tolerance")
    final = min(table[0].values(), key=lambda v: v[:3])
    return raw, final[3][::-1]


# ---------------------------------------------------------------------------
# 1-nearest neighbour (Sec. II-E) in log2 features
# ---------------------------------------------------------------------------
def nearest(train, n, batch=1):
    """train: list of (n, batch, s).  The label of the closest row in
    (log2 n, log2 batch); equal distances go to the larger s."""
    ln, lb = math.log2(max(1, n)), math.log2(max(1, batch))
    best, lab = None, None
    for tn, tb, s in train:
        dist = (math.log2(tn) - ln) ** 2 + (math.log2(tb) - lb) ** 2
        if best is None or dist < best or (dist == best and s > lab):
            best, lab = dist, s
    return lab


def load_sweep(path):
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line:
                rows.append(json.loads(line))
    return rows


def grouped(rows):
    """{(dtype, batch): [(n, {s: ms}), ...] ascending n}."""
    g = defaultdict(lambda: defaultdict(dict))
    for r in rows:
        g[(r["dtype"], r["batch"])][r["n"]][r["s"]] = r["ms"]
    return {k: sorted(v.items()) for k, v in g.items()}


def correct_flat(times, tol: float = TOL):
    """Labels within ``tol`` of the fastest at every N with the fewest label
    changes over N (no monotonicity), then the least total relative loss."""
    cand = []
    for t in times:
        best = min(t.values())
        cand.append({s: t[s] / best - 1.0 for s in t if t[s] <= (1.0 + tol) * best})
    prev = {s: (0, lo, [s]) for s, lo in cand[0].items()}
    for i in range(1, len(times)):
        cur = {}
        for s, lo in cand[i].items():
            best = None
            for sp, (ch, loss, path) in prev.items():
                key = (ch + (1 if sp != s else 0), loss + lo)
                if best is None or key < best[:2] or (key == best[:2] and sp > best[2][-1]):
                    best = key + (path + [s],)
            cur[s] = best
        prev = cur
    return min(prev.values(), key=lambda v: (v[0], v[1], -v[2][-1]))[2]


def correct_relaxed(times, tol: float = TOL, tol_flat: float = TOL_FLAT):
    """The paper's correction (non-decreasing labels, ``correct``) when a
    sequence within ``tol`` exists; otherwise, since the optimum need not grow
    with N on every GPU, the flattest labels within ``tol_flat``
    (``correct_flat``).  Without a trend to restore, the fallback only removes
    label changes that buy less than ``tol_flat``: with 5 % it kept one label
    over sizes where another was faster by up to 4.6 % at every size.
    Returns (raw, corrected, rule) with rule "monotone" or "flat"."""
    raw = [max((s for s in tm if tm[s] == min(tm.values()))) for tm in times]
    try:
        return correct(times, tol)[0], correct(times, tol)[1], "monotone"
    except ValueError:
        return raw, correct_flat(times, tol_flat), "flat"


def build_table(rows):
    """Rows (dtype, n, batch, s) of the corrected labels."""
    out = []
    for (dt, batch), series in sorted(grouped(rows).items()):
        sizes = [n for n, _ in series]
        raw, cor, _ = correct_relaxed([t for _, t in series])
        out += [(dt, n, batch, s) for n, s in zip(sizes, cor)]
    return out


def write_table(table, path_txt=None, path_inc=None):
    if path_txt:
        with open(path_txt, "w") as fh:
            fh.write("# dtype n batch s   (GB300 sweep, corrected labels)\n")
            for dt, n, b, s in table:
                fh.write(f"{dt} {n} {b} {s}\n")
    if path_inc:
        with open(path_inc, "w") as fh:
            fh.write("// Built-in predictor table: (dtype, n, batch, s) rows, the corrected labels of\n"
                     "// the GB300 timing sweep written by paper_2510_27351_gb300/tune.py.  A dtype\n"
                     "// with no rows falls back to the paper's interval rule.\n"
                     "static const Row kBuiltinTable[] = {\n")
            for dt, n, b, s in table:
                fh.write(f"    {{{dt}, {float(n)!r}, {float(b)!r}, {s}}},\n")
            fh.write("};\n")


def evaluate(rows, seed=0):
    """The paper's protocol per (dtype, batch): shuffled 3:1 split keeping every
    class in training, 1-NN accuracy on observed and corrected labels, null
    accuracy, and the time lost by the prediction against the sweep optimum."""
    report = {}
    for (dt, batch), series in sorted(grouped(rows).items()):
        sizes = [n for n, _ in series]
        times = [t for _, t in series]
        raw, cor, tol_used = correct_relaxed(times)
        idx = list(range(len(sizes)))
        rng = random.Random(seed)
        for _ in range(1000):
            rng.shuffle(idx)
            k = len(idx) // 4
            test, train = idx[:k], idx[k:]
            if set(cor[i] for i in train) == set(cor) and set(raw[i] for i in train) == set(raw):
                break
        acc = {}
        for name, lab in (("observed", raw), ("corrected", cor)):
            tr = [(sizes[i], batch, lab[i]) for i in train]
            acc[name] = sum(nearest(tr, sizes[i], batch) == lab[i] for i in test) / max(1, len(test))
        mode = max(set(cor), key=cor.count)
        null = sum(cor[i] == mode for i in test) / max(1, len(test))
        tr = [(sizes[i], batch, cor[i]) for i in train]
        losses = []
        for i in test:
            sp = nearest(tr, sizes[i], batch)
            t = times[i]
            losses.append(t.get(sp, float("inf")) / min(t.values()) - 1.0)
        # leave-one-out over every size: the prediction from all other labels
        loo = []
        for i in range(len(sizes)):
            tr_i = [(sizes[j], batch, cor[j]) for j in range(len(sizes)) if j != i]
            loo.append(times[i][nearest(tr_i, sizes[i], batch)] / min(times[i].values()) - 1.0)
        report[f"{DTYPES.get(dt, dt)}/batch{batch}"] = {
            "n_sizes": len(sizes), "accuracy_observed": acc["observed"], "accuracy_corrected": acc["corrected"],
            "null_accuracy": null, "max_time_loss": max(losses) if losses else 0.0,
            "mean_time_loss": sum(losses) / max(1, len(losses)), "loo_mean_time_loss": sum(loo) / len(loo),
            "loo_max_time_loss": max(loo), "correction_rule": tol_used,
            "test_sizes": [sizes[i] for i in sorted(test)]}
    return report


def evaluate_transfer(rows):
    """Does a size model trained on one precision serve another (the paper's
    question of reusing a table across precisions, Sec. IV)?  For every batch
    group and every ordered pair of precisions (source, target) swept at the
    same sizes: 1-NN on all of the source's corrected labels, predicted at the
    target's sizes, against the target's own labels and timings.  Reported:
    label accuracy, mean and maximum time loss against the target's fastest s,
    and, for scale, the target's own leave-one-out loss and the loss of the
    best single s for every size."""
    groups = grouped(rows)
    labels = {}
    for key, series in groups.items():
        labels[key] = correct_relaxed([t for _, t in series])[1]
    report = {}
    for (dt_t, batch), series in sorted(groups.items()):
        sizes = [n for n, _ in series]
        times = [t for _, t in series]
        cor_t = labels[(dt_t, batch)]
        own = []
        for i in range(len(sizes)):
            tr_i = [(sizes[j], batch, cor_t[j]) for j in range(len(sizes)) if j != i]
            own.append(times[i][nearest(tr_i, sizes[i], batch)] / min(times[i].values()) - 1.0)
        common = set.intersection(*(set(t) for t in times))
        fixed = min(common, key=lambda s: sum(t[s] / min(t.values()) for t in times)) if common else None
        fixed_loss = [t[fixed] / min(t.values()) - 1.0 for t in times] if fixed else []
        for (dt_s, batch_s), series_s in sorted(groups.items()):
            if batch_s != batch or dt_s == dt_t:
                continue
            tr = [(n, batch, s) for (n, _), s in zip(series_s, labels[(dt_s, batch)])]
            pred = [nearest(tr, n, batch) for n in sizes]
            loss = [t.get(p, float("inf")) / min(t.values()) - 1.0 for p, t in zip(pred, times)]
            report[f"{DTYPES.get(dt_s, dt_s)}->{DTYPES.get(dt_t, dt_t)}/batch{batch}"] = {
                "n_sizes": len(sizes),
                "accuracy": sum(p == c for p, c in zip(pred, cor_t)) / len(sizes),
                "mean_time_loss": sum(loss) / len(loss), "max_time_loss": max(loss),
                "target_loo_mean_time_loss": sum(own) / len(own), "target_loo_max_time_loss": max(own),
                "best_fixed_s": fixed, "best_fixed_s_mean_time_loss": sum(fixed_loss) / max(1, len(fixed_loss)),
                "predicted": dict(zip(map(str, sizes), pred)), "target_labels": dict(zip(map(str, sizes), cor_t))}
    return report


# ---------------------------------------------------------------------------
# autotuner for a given batch (GPU)
# ---------------------------------------------------------------------------
_AUTOTUNE_CACHE = {}


def _timed_ms(fn, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune_window(offsets, a, b, c, d, x, dtype, refine_iters=0, sw_grid=(5, 7), halos=(32, 48, 64), reps=3):
    """Pick the windowed pass's block shape (rows per thread, halo rows) for
    ``tdp_solve_batched`` on this batch by timing every pair (a halo too short
    for the batch's decay shows up as the time of the exact fallback), set
    the knobs TDP_TUNE_WINDOW_SW and TDP_TUNE_WINDOW_HALO (binary32 + refinement)
    or TDP_TUNE_WINDOW_HALO32 (binary32) and return (rows per thread, halo,
    ms).  Cached per (dtype, total rows, batch)."""
    import paper_2510_27351_gb300 as tdp

    batch, total = offsets.numel() - 1, d.numel()
    hkey = tdp.TUNE_WINDOW_HALO32 if int(dtype) == tdp.F32 else tdp.TUNE_WINDOW_HALO
    key = ("window", int(dtype), int(total), int(batch), int(refine_iters))
    if key not in _AUTOTUNE_CACHE:
        old = (tdp.tdp_get_tuning(tdp.TUNE_WINDOW_SW), tdp.tdp_get_tuning(hkey))
        best = None
        try:
            for sw in sw_grid:
                for h in halos:
                    tdp.tdp_set_tuning(tdp.TUNE_WINDOW_SW, sw)
                    tdp.tdp_set_tuning(hkey, h)
                    ms = _timed_ms(lambda: tdp.tdp_solve_batched(offsets, batch, total, a, b, c, d, x, 0, dtype,
                                                                 refine_iters), reps)
                    if best is None or ms < best[2]:
                        best = (sw, h, ms)
        finally:
            tdp.tdp_set_tuning(tdp.TUNE_WINDOW_SW, old[0])
            tdp.tdp_set_tuning(hkey, old[1])
        _AUTOTUNE_CACHE[key] = best
    sw, h, ms = _AUTOTUNE_CACHE[key]
    tdp.tdp_set_tuning(tdp.TUNE_WINDOW_SW, sw)
    tdp.tdp_set_tuning(hkey, h)
    return sw, h, ms


def autotune_batched(offsets, a, b, c, d, x, dtype, refine_iters=0, s_grid=(8, 12, 16, 24, 32, 48),
                     budgets=(32 * 1024, 64 * 1024, 100 * 1024), reps=3):
    """Pick (s, shared-memory budget per CTA) for ``tdp_solve_batched`` on
    this batch by timing every pair, set the budget knob and return
    (s, budget, ms).  Results are cached per (dtype, total rows, batch).
    A precision whose batches take the windowed pass (binary32 + refinement,
    binary32; s does not apply there) gets its block shape tuned instead
    (autotune_window) and (0, the current budget, ms) back."""
    import torch

    import paper_2510_27351_gb300 as tdp

    batch, total = offsets.numel() - 1, d.numel()
    windowed = ((int(dtype) == tdp.F32_REFINE and tdp.tdp_get_tuning(tdp.TUNE_WINDOW))
                or (int(dtype) == tdp.F32 and tdp.tdp_get_tuning(tdp.TUNE_WINDOW32)))
    if windowed:
        _, _, ms = autotune_window(offsets, a, b, c, d, x, dtype, refine_iters, reps=reps)
        return 0, tdp.tdp_get_tuning(tdp.TUNE_SMEM_BUDGET), ms
    key = (int(dtype), int(total), int(batch), int(refine_iters))
    if key in _AUTOTUNE_CACHE:
        s, budget, ms = _AUTOTUNE_CACHE[key]
        tdp.tdp_set_tuning(tdp.TUNE_SMEM_BUDGET, budget)
        return s, budget, ms
    old = tdp.tdp_get_tuning(tdp.TUNE_SMEM_BUDGET)
    best = None
    try:
        for budget in budgets:
            tdp.tdp_set_tuning(tdp.TUNE_SMEM_BUDGET, budget)
            for s in s_grid:
                fn = lambda: tdp.tdp_solve_batched(offsets, batch, total, a, b, c, d, x, s, dtype, refine_iters)
                fn()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                if best is None or ms < best[2]:
                    best = (s, budget, ms)
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_SMEM_BUDGET, old)
    _AUTOTUNE_CACHE[key] = best
    tdp.tdp_set_tuning(tdp.TUNE_SMEM_BUDGET, best[1])
    return best


# ---------------------------------------------------------------------------
# the sweep (GPU)
# ---------------------------------------------------------------------------
def sweep(out, dtypes=(0, 1, 2), log2_lo=10.0, log2_hi=28.0, step=0.5, batches=(1,), trials=5, s_grid=S_GRID,
          max_rows=1 << 28):
    """Time every s of the grid for every size, batch and precision: one solve
    captured into a CUDA graph and replayed (device time only, no host launch
    gaps, which dominate at small sizes), the fastest of ``trials`` timed
    trials of about 20 ms each (launch noise only ever adds time).  The
    binary32 + refinement rows time the exact three-pass schedule, the one
    that uses s, and so do the binary32 rows (the windowed passes have a
    fixed geometry)."""
    import torch

    import paper_2510_27351_gb300 as tdp

    done = set()
    if os.path.exists(out):
        for r in load_sweep(out):
            done.add((r["dtype"], r["n"], r["batch"], r["s"]))
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    stream = torch.cuda.Stream()  # one stream: the library keeps one workspace per stream
    sizes = []
    x = log2_lo
    while x <= log2_hi + 1e-9:
        sizes.append(int(round(2 ** x)))
        x += step
    keys = (tdp.TUNE_WINDOW, tdp.TUNE_WINDOW32)  # the windowed passes ignore s: time the exact schedules
    old_window = [tdp.tdp_get_tuning(k) for k in keys]
    for k in keys:
        tdp.tdp_set_tuning(k, 0)
    try:
        with open(out, "a") as fh:
            for batch in batches:
                for n in sizes:
                    total = n * batch
                    if total > max_rows:
                        continue
                    for dt in dtypes:
                        todo = [s for s in s_grid if (dt, n, batch, s) not in done and s <= max(4, n)]
                        if not todo:
                            continue
                        a, b, c, d = _random_system(total, dt, g, dev)
                        xo = torch.empty_like(d)
                        off = torch.arange(batch + 1, device=dev, dtype=torch.int64) * n
                        it = 1 if dt == 2 else 0
                        for s in todo:
                            if batch == 1:
                                fn = lambda st: tdp.tdp_solve(a, b, c, d, xo, total, s, dt, it, st)
                            else:
                                fn = lambda st: tdp.tdp_solve_batched(off, batch, total, a, b, c, d, xo, s, dt, it,
                                                                      st)
                            ms = _graph_time_ms(tdp, fn, stream, trials)
                            fh.write(json.dumps({"dtype": dt, "n": n, "batch": batch, "s": s, "ms": ms}) + "\n")
                            fh.flush()
                        del a, b, c, d, xo
                        torch.cuda.empty_cache()
    finally:
        for k, v in zip(keys, old_window):
            tdp.tdp_set_tuning(k, v)


def _graph_time_ms(tdp, fn, stream, trials):
    """Milliseconds per solve: fn(stream) captured into a CUDA graph, replayed
    back to back; the fastest of ``trials`` trials of about 20 ms."""
    import torch

    graph = tdp.CapturedSolve(fn, stream)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        stream.synchronize()
        reps = int(max(3, min(500, 20.0 / max(1e-3, e0.elapsed_time(e1)))))
        best = float("inf")
        for _ in range(trials):
            e0.record(stream)
            for _ in range(reps):
                graph.replay()
            e1.record(stream)
            stream.synchronize()
            best = min(best, e0.elapsed_time(e1) / reps)
    del graph
    return best


def autotune_const(fn, s_grid=(8, 16, 32, 64, 128), reps=10):
    """Fastest s for a constant-coefficient solve: ``fn(s)`` queues the solve(s)
    with sub-system size s on the current stream; every s of the grid is timed
    (CUDA events) after one untimed call.  Returns (s, ms)."""
    best = None
    for s in s_grid:
        ms = _time_ms(lambda: fn(s), reps)
        if best is None or ms < best[1]:
            best = (s, ms)
    return best


# ---------------------------------------------------------------------------
# number of recursive steps (Sec. III)
# ---------------------------------------------------------------------------
def _random_system(total, dt, g, dev):
    import torch

    st = torch.float32 if dt == 1 else torch.float64
    a = torch.rand(total, generator=g, device=dev, dtype=st) * 2 - 1
    b = torch.rand(total, generator=g, device=dev, dtype=st) * 4 + 4
    c = torch.rand(total, generator=g, device=dev, dtype=st) * 2 - 1
    d = torch.rand(total, generator=g, device=dev, dtype=st) * 2 - 1
    return a, b, c, d


def _time_ms(fn, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def sweep_r(out, dtypes=(0, 2), log2_lo=14.0, log2_hi=28.0, step=0.5, reps=5, r_grid=R_GRID):
    """Time one system per size with the paper's recursion schedule for every R
    of r_grid, and with the default schedule (recorded as R = -1); s is the
    size model's choice."""
    import torch

    import paper_2510_27351_gb300 as tdp

    done = set()
    if os.path.exists(out):
        for r in load_sweep(out):
            done.add((r["dtype"], r["n"], r["R"]))
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    sizes = []
    x = log2_lo
    while x <= log2_hi + 1e-9:
        sizes.append(int(round(2 ** x)))
        x += step
    old = (tdp.tdp_get_tuning(tdp.TUNE_RECURSION), tdp.tdp_get_tuning(tdp.TUNE_R))
    try:
        with open(out, "a") as fh:
            for n in sizes:
                for dt in dtypes:
                    todo = [r for r in (-1,) + tuple(r_grid) if (dt, n, r) not in done]
                    if not todo:
                        continue
                    a, b, c, d = _random_system(n, dt, g, dev)
                    xo = torch.empty_like(d)
                    s = tdp.tdp_predict_s(n, 1, dt)
                    it = 1 if dt == 2 else 0
                    for r in todo:
                        tdp.tdp_set_tuning(tdp.TUNE_RECURSION, 0 if r < 0 else 1)
                        tdp.tdp_set_tuning(tdp.TUNE_R, max(r, -1))
                        ms = min(_time_ms(lambda: tdp.tdp_solve(a, b, c, d, xo, n, s, dt, it),
                                          reps if n >= (1 << 20) else 4 * reps) for _ in range(3))
                        fh.write(json.dumps({"dtype": dt, "n": n, "batch": 1, "R": r, "s": s, "ms": ms}) + "\n")
                        fh.flush()
                    del a, b, c, d, xo
                    torch.cuda.empty_cache()
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_RECURSION, old[0])
        tdp.tdp_set_tuning(tdp.TUNE_R, old[1])


def grouped_r(rows):
    """{(dtype, batch): [(n, {R: ms}), ...]} sorted by n; R = -1 is the default schedule."""
    acc = defaultdict(lambda: defaultdict(dict))
    for r in rows:
        acc[(r["dtype"], r["batch"])][r["n"]][r["R"]] = r["ms"]
    return {k: sorted(v.items()) for k, v in acc.items()}


def best_r(times):
    """Fastest R >= 0 (ties to the larger R)."""
    cand = {r: t for r, t in times.items() if r >= 0}
    tmin = min(cand.values())
    return max(r for r, t in cand.items() if t == tmin)


def r_labels(series):
    """Observed (fastest) and corrected R per size: the label correction of the
    size model (within TOL of the fastest, trend-consistent) applied to the
    times of the paper's schedule, R >= 0."""
    times = [{r: t for r, t in tm.items() if r >= 0} for _, tm in series]
    raw = [best_r(t) for t in times]
    _, cor, rule = correct_relaxed(times)
    return raw, cor, rule


def build_rtable(rows):
    out = []
    for (dt, batch), series in sorted(grouped_r(rows).items()):
        _, cor, _ = r_labels(series)
        out += [(dt, n, batch, r) for (n, _), r in zip(series, cor)]
    return out


def write_rtable(table, path_txt=None, path_inc=None):
    if path_txt:
        with open(path_txt, "w") as fh:
            fh.write("# dtype n batch R   (GB300 sweep of the number of recursive steps, corrected labels)\n")
            for dt, n, b, r in table:
                fh.write(f"{dt} {n} {b} {r}\n")
    if path_inc:
        with open(path_inc, "w") as fh:
            fh.write("// Recursion-depth table (dtype, n, batch, R): the number of recursive steps per\n"
                     "// size from the GB300 sweep written by paper_2510_27351_gb300/tune.py (within 5 %\n"
                     "// of the fastest R, corrected towards the trend like the size model's labels).\n"
                     "const RRow kBuiltinRTable[] = {\n")
            for dt, n, b, r in table:
                fh.write(f"    {{{dt}, {float(n)!r}, {float(b)!r}, {r}}},\n")
            fh.write("};\n")


def evaluate_r(rows, seed=0):
    """Per dtype: shuffled 3:1 split keeping every R in training, 1-NN accuracy
    and null accuracy (Sec. III-A), the time lost by the predicted R against the
    fastest R, and the paper's schedule with the predicted R against the
    library's default schedule, on the held-out sizes."""
    report = {}
    for (dt, batch), series in sorted(grouped_r(rows).items()):
        sizes = [n for n, _ in series]
        times = [t for _, t in series]
        raw, lab, rule = r_labels(series)
        idx = list(range(len(sizes)))
        rng = random.Random(seed)
        for _ in range(1000):
            rng.shuffle(idx)
            k = len(idx) // 4
            test, train = idx[:k], idx[k:]
            if set(lab[i] for i in train) == set(lab):
                break
        tr = [(sizes[i], batch, lab[i]) for i in train]
        pred = {i: nearest(tr, sizes[i], batch) for i in test}
        mode = max(set(lab), key=lab.count)
        losses = [times[i][pred[i]] / times[i][raw[i]] - 1.0 for i in test]
        vs_default = [times[i][pred[i]] / times[i][-1] for i in test if -1 in times[i]]
        tr_raw = [(sizes[i], batch, raw[i]) for i in train]
        report[f"{DTYPES.get(dt, dt)}/batch{batch}"] = {
            "n_sizes": len(sizes), "labels_observed": dict(zip(map(str, sizes), raw)),
            "labels": dict(zip(map(str, sizes), lab)), "correction_rule": rule,
            "accuracy_observed": sum(nearest(tr_raw, sizes[i], batch) == raw[i] for i in test) / max(1, len(test)),
            "accuracy": sum(pred[i] == lab[i] for i in test) / max(1, len(test)),
            "null_accuracy": sum(lab[i] == mode for i in test) / max(1, len(test)),
            "max_time_loss": max(losses) if losses else 0.0, "mean_time_loss": sum(losses) / max(1, len(losses)),
            "predicted_over_default_mean": sum(vs_default) / max(1, len(vs_default)),
            "best_over_default_all": {str(n): t[best_r(t)] / t[-1] for n, t in zip(sizes, times) if -1 in t},
            "test_sizes": [sizes[i] for i in sorted(test)]}
    return report


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    p = sub.add_parser("sweep")
    p.add_argument("--out", required=True)
    p.add_argument("--dtypes", default="0,1,2")
    p.add_argument("--lo", type=float, default=10.0)
    p.add_argument("--hi", type=float, default=28.0)
    p.add_argument("--step", type=float, default=0.5)
    p.add_argument("--batches", default="1")
    p.add_argument("--trials", type=int, default=5)
    p = sub.add_parser("table")
    p.add_argument("--sweep", required=True)
    p.add_argument("--out")
    p.add_argument("--inc")
    p = sub.add_parser("evaluate")
    p.add_argument("--sweep", required=True)
    p = sub.add_parser("sweep-r")
    p.add_argument("--out", required=True)
    p.add_argument("--dtypes", default="0,2")
    p.add_argument("--lo", type=float, default=14.0)
    p.add_argument("--hi", type=float, default=28.0)
    p.add_argument("--step", type=float, default=0.5)
    p.add_argument("--reps", type=int, default=5)
    p = sub.add_parser("rtable")
    p.add_argument("--sweep", required=True)
    p.add_argument("--out")
    p.add_argument("--inc")
    p = sub.add_parser("evaluate-r")
    p.add_argument("--sweep", required=True)
    p = sub.add_parser("evaluate-transfer")
    p.add_argument("--sweep", required=True)
    args = ap.parse_args(argv)
    if args.cmd == "sweep":
        sweep(args.out, tuple(int(v) for v in args.dtypes.split(",")), args.lo, args.hi, args.step,
              tuple(int(v) for v in args.batches.split(",")), args.trials)
    elif args.cmd == "table":
        write_table(build_table(load_sweep(args.sweep)), args.out, args.inc)
    elif args.cmd == "evaluate":
        print(json.dumps(evaluate(load_sweep(args.sweep)), indent=1))
    elif args.cmd == "sweep-r":
        sweep_r(args.out, tuple(int(v) for v in args.dtypes.split(",")), args.lo, args.hi, args.step, args.reps)
    elif args.cmd == "rtable":
        write_rtable(build_rtable(load_sweep(args.sweep)), args.out, args.inc)
    elif args.cmd == "evaluate-transfer":
        print(json.dumps(evaluate_transfer(load_sweep(args.sweep)), indent=1))
    else:
        print(json.dumps(evaluate_r(load_sweep(args.sweep)), indent=1))


if __name__ == "__main__":
    sys.exit(main())
