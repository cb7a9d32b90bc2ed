"""The seeded input generator (shared by the oracle's and the GPU's tests)."""
import numpy as np

import workloads as W


def _splitmix64_next(state):
    """Reference splitmix64 step written with Python integers."""
    M = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & M
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return state, z ^ (z >> 31)


def test_splitmix64_known_answer():
    # first output of splitmix64 from state 0 (published test value)
    _, z = _splitmix64_next(0)
    assert z == 0xE220A8397B1DCDAF
    assert int(W.mix64(np.uint64(0x9E3779B97F4A7C15))) == 0xE220A8397B1DCDAF


def test_counter_stream_matches_sequential_generator():
    seed, stream = 5, 2
    key = int(W.mix64(np.uint64(seed) * W.GAMMA + np.uint64(stream)))
    st, ref = key, []
    for _ in range(10):
        st, z = _splitmix64_next(st)
        ref.append(z)
    assert [int(v) for v in W.raw64(seed, stream, 10)] == ref
    assert [int(v) for v in W.raw64(seed, stream, 4, start=6)] == ref[6:]


def test_distributions_and_structure():
    S = W.single(4096, 0)
    assert S.a[0] == 0.0 and S.c[-1] == 0.0
    assert np.all((S.b >= 4) & (S.b < 8))
    assert np.all(np.abs(S.a) <= 1) and np.all(np.abs(S.c) <= 1)
    assert np.all(np.abs(S.b) > np.abs(S.a) + np.abs(S.c))
    Sb = W.batched(4096, 64, 65536, 0)
    sizes = np.diff(Sb.offsets)
    assert sizes.min() >= 64 and sizes.max() <= 65536
    # log-uniform: median near sqrt(64 * 65536) = 2048
    assert 1200 < np.median(sizes) < 3500
    assert np.all(Sb.a[Sb.offsets[:-1]] == 0) and np.all(Sb.c[Sb.offsets[1:] - 1] == 0)
    w = W.loss_weights(100_000, 0)
    assert abs(w.mean()) < 0.02 and abs(w.std() - 1) < 0.02
