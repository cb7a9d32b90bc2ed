"""Oracle for the sub-system-size choice (paper Sec. II-D, II-E, IV-B).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain Python, no
numerical library beyond numpy; every routine is a brute-force statement of
the rule it implements.

* ``interval_rule``: the piecewise-constant rule N -> s read off Table I
  (Sec. II-D).
* ``knn_predict``: k-nearest-neighbour classification (Sec. II-E: the mode of
  the labels of the k closest training sizes; k = 1 was found best).  The
  feature is log2 N (plus log2 batch when the table has batch sizes); the
  paper used the SLAE size itself, but sizes here span 2^10 .. 2^28, so
  distances are taken between their logarithms (a reading of Sec. II-E).
  Ties in distance are broken towards the larger s, ties in the vote likewise.
* ``correct_labels``: the label correction of Sec. II-E.  The paper replaces
  noisy per-size optima by near-optimal sizes that follow the trend; its
  reading here: among the sizes whose time is within ``tol`` of the fastest
  at that N, choose a label sequence that is non-decreasing in N with the
  fewest changes, then the larger labels, then the least summed time loss.
* ``split_3to1`` / ``grid_search_k`` / ``accuracy`` / ``null_accuracy``:
  the evaluation protocol of Sec. II-E (shuffled 3:1 split keeping every
  class in training, k searched in [1, #classes] by cross-validation).
* ``interval_rule_r``: the number of recursive steps R read off the paper's
  table of optimum R (Sec. III-A); ``knn_predict`` serves its 1-NN model too.
* ``recursive_sizes``: the sub-system sizes of the R recursive steps
  (Sec. III-B): the first step 10 when R >= 2, every other step the size
  model applied to the interface system that step partitions.
"""
from __future__ import annotations

import math
import random
from collections import Counter

import numpy as np


def interval_rule(n: float, table) -> int:
    """table = [(N_upper, s), ...] ascending; returns s for N (Sec. II-D)."""
    for upper, s in table:
        if n <= upper:
            return int(s)
    return int(table[-1][1])


def _features(sizes, batches=None):
    f = [[math.log2(float(n))] for n in sizes]
    if batches is not None:
        for row, bt in zip(f, batches):
            row.append(math.log2(float(bt)))
    return f


def knn_predict(train_sizes, train_labels, query_size, k: int = 1, train_batches=None, query_batch=None):
    """Label of ``query_size`` by k-NN over log2 features (brute force)."""
    feats = _features(train_sizes, train_batches)
    q = _features([query_size], None if query_batch is None else [query_batch])[0]
    dist = []
    for f, lab in zip(feats, train_labels):
        dist.append((sum((fi - qi) ** 2 for fi, qi in zip(f, q)), -int(lab), int(lab)))
    dist.sort()  # nearest first; equal distance -> larger label first
    top = [lab for _, _, lab in dist[:k]]
    votes = Counter(top)
    best = max(votes.values())
    # mode of the k labels; a tied vote goes to the larger size
    return max(lab for lab, v in votes.items() if v == best)


def accuracy(train_sizes, train_labels, test_sizes, test_labels, k: int = 1) -> float:
    if len(test_sizes) == 0:
        return 1.0
    hits = sum(knn_predict(train_sizes, train_labels, n, k) == int(lab) for n, lab in zip(test_sizes, test_labels))
    return hits / len(test_sizes)


def null_accuracy(test_labels, train_labels=None) -> float:
    """Accuracy of always predicting the most frequent size (Sec. II-E)."""
    ref = train_labels if train_labels is not None else test_labels
    mode = Counter(int(v) for v in ref).most_common(1)[0][0]
    return sum(int(v) == mode for v in test_labels) / max(1, len(test_labels))


def split_3to1(sizes, labels, seed: int = 0, max_tries: int = 1000):
    """Shuffled 3:1 train/test split with every class present in training."""
    idx = list(range(len(sizes)))
    classes = set(int(v) for v in labels)
    rng = random.Random(seed)
    n_test = len(idx) // 4
    for _ in range(max_tries):
        rng.shuffle(idx)
        test, train = idx[:n_test], idx[n_test:]
        if set(int(labels[i]) for i in train) == classes:
            pick = lambda ids, arr: [arr[i] for i in ids]
            return pick(train, sizes), pick(train, labels), pick(test, sizes), pick(test, labels)
    raise RuntimeError("no split keeps every class in training")


def grid_search_k(sizes, labels, folds: int = 5):
    """k in [1, #classes] maximising mean cross-validated accuracy; the
    smallest such k wins a tie."""
    n_classes = len(set(int(v) for v in labels))
    n = len(sizes)
    best_k, best_acc = 1, -1.0
    for k in range(1, n_classes + 1):
        accs = []
        for f in range(folds):
            te = [i for i in range(n) if i % folds == f]
            tr = [i for i in range(n) if i % folds != f]
            if not te or len(tr) < k:
                continue
            accs.append(accuracy([sizes[i] for i in tr], [labels[i] for i in tr],
                                 [sizes[i] for i in te], [labels[i] for i in te], k))
        acc = float(np.mean(accs)) if accs else 0.0
        if acc > best_acc + 1e-12:
            best_k, best_acc = k, acc
    return best_k, best_acc


def correct_labels(times, tol: float = 0.05):
    """Trend-consistent labels from per-size timings (Sec. II-E).

    ``times``: list over ascending N of dicts {s: time}.  An entry with one
    key only (no timings known) fixes the label.  Returns (raw, corrected).

    Among the sizes within ``tol`` of the fastest at each N, the corrected
    sequence is non-decreasing in N and, in this order of preference, has
    (1) the fewest changes of label, (2) the larger labels, compared from the
    largest N downwards (the paper's speed-ups come from moving to larger
    sizes), (3) the smallest summed relative time loss.
    """
    raw = [min(t, key=lambda s: (t[s], -s)) for t in times]
    cands = []
    for t in times:
        tmin = min(t.values())
        cands.append({s: t[s] / tmin - 1.0 for s in t if t[s] <= (1.0 + tol) * tmin})
    n = len(times)
    # backward dynamic programme; key = (changes, -labels from the end, loss)
    best = [dict() for _ in range(n)]
    for s, loss in cands[-1].items():
        best[-1][s] = (0, (-s,), loss, (s,))
    for i in range(n - 2, -1, -1):
        for s, loss in cands[i].items():
            opt = None
            for sn, (ch, neg, lo, seq) in best[i + 1].items():
                if sn < s:
                    continue
                c = (ch + (sn != s), neg + (-s,), lo + loss, seq + (s,))
                if opt is None or c[:3] < opt[:3]:
                    opt = c
            if opt is not None:
                best[i][s] = opt
    if not best[0]:
        raise RuntimeError("no non-decreasing label sequence within tolerance")
    final = min(best[0].values(), key=lambda v: v[:3])
    return raw, list(final[3])[::-1]


def interval_rule_r(n: float, table) -> int:
    """table = [(N_upper, R), ...] ascending; returns R for N, the last R + 1
    above the last bound (Sec. III-A)."""
    for upper, r in table:
        if n <= upper:
            return int(r)
    return int(table[-1][1]) + 1


def recursive_sizes(n: int, s: int, R: int, predict_s, base_rows: int = 64):
    """Sub-system sizes m_1..m_R of the recursive steps for one system of n
    unknowns partitioned with s (Sec. III-B).  The interface system of a
    partition into ceil(M/m) blocks has 2 ceil(M/m) rows.  Steps stop early
    once the interface system has at most ``base_rows`` rows or the step
    would form a single block (nothing left to reduce)."""
    sizes = []
    M = 2 * math.ceil(n / s)
    for level in range(1, R + 1):
        if M <= base_rows:
            break
        m = 10 if (level == 1 and R >= 2) else int(predict_s(M))
        m = max(m, 3)
        if m >= M:
            break
        sizes.append(m)
        M = 2 * math.ceil(M / m)
    return sizes


def load_table(path):
    """Rows of a whitespace table, '#' comments skipped."""
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows
