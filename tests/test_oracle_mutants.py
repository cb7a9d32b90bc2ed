"""Planted mistakes: each plausible slip in the oracle must trip a pin.

Every case copies oracle.c, applies one textual mutation (a flipped sign, a
wrong index, a dropped term, a transposed operand, ...), compiles the copy
with gcc into a temporary library, swaps it in for the oracle's library and
runs the pins of tests/pins.py until one fails.  Nothing touches a GPU.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
from pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "thomas_pivot_sign": ("den = b[i] - a[i] * cp[i - 1];", "den = b[i] + a[i] * cp[i - 1];"),
    "thomas_backsub_index": ("x[i] = dp[i] - cp[i] * x[i + 1];", "x[i] = dp[i] - cp[i + 1] * x[i + 1];"),
    "thomas_f32_reciprocal": ("cp[i] = (i < n - 1 ? c[i] : 0.0f) / den;", "cp[i] = (i < n - 1 ? c[i] : 0.0f) * den;"),
    "partition_dropped_rhs_term": ("D2[M] = d[L] - c[L] * g[0];", "D2[M] = d[L];"),
    "partition_swapped_spikes": ("B2[M] = b[L] + c[L] * v[0];\n    C2[M] = c[L] * w[0];",
                                 "B2[M] = b[L] + c[L] * w[0];\n    C2[M] = c[L] * v[0];"),
    "partition_spike_sign": ("rhs[0] = -a[L + 1];", "rhs[0] = a[L + 1];"),
    "partition_stage3_wrong_end": ("rhs[ni - 1] -= c[R - 1] * x[R];", "rhs[ni - 1] -= c[R - 1] * x[L];"),
    "partition_last_row_coupling": ("A2[M] = a[R] * v[ni - 1];", "A2[M] = a[R] * w[ni - 1];"),
    "dense_pivot_choice": ("if (v > best) { best = v; p = i; }", "if (v < best) { best = v; p = i; }"),
    "adjoint_untransposed": ("ta[i] = (i > 0) ? c[i - 1] : 0.0;", "ta[i] = (i > 0) ? a[i] : 0.0;"),
    "adjoint_grad_sign": ("gb[i] = -lam[i] * x[i];", "gb[i] = lam[i] * x[i];"),
    "adjoint_grad_index": ("gc[i] = (i < n - 1) ? -lam[i] * x[i + 1] : 0.0;",
                           "gc[i] = (i < n - 1) ? -lam[i + 1] * x[i] : 0.0;"),
    "refine_residual_index": ("if (i > 0) acc -= a[i] * x[i - 1];", "if (i > 0) acc -= a[i] * x[i];"),
    "dst_eigenvalue": ("1.0L + 4.0L * (long double)r * sj * sj", "1.0L + 2.0L * (long double)r * sj * sj"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found in oracle.c"
    src = src.replace(old, new, 1)
    c_path = tmp_path / "mutant.c"
    so_path = tmp_path / "libmutant.so"
    c_path.write_text(src)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", str(so_path), str(c_path), "-lm"])
    lib = oracle._configure(ctypes.CDLL(str(so_path)))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = []
    for pin in ALL_PINS:
        try:
            failures = pin()
        except Exception as exc:  # a zero pivot or a crash of the checker counts
            failures = [f"raised {exc!r}"]
        if failures:
            caught.append((pin.__name__, failures[0]))
            break
    assert caught, f"no pin catches the planted mistake {name}"
