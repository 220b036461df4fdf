"""The seeded input generator that the oracle and the CUDA path share: counter-based splitmix64
(Steele, Lea & Flood 2014), uniforms from the top 53 bits, Box-Muller normals."""
import math

import numpy as np

from synth import rng


def _splitmix64_reference(seed, n):
    """splitmix64 as published: the state advances by the golden-gamma increment, each output is
    the state passed through the two xor-shift-multiply rounds and a final xor-shift."""
    mask = (1 << 64) - 1
    state = seed & mask
    out = []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_published_outputs():
    """Seed 0: the first outputs of the published generator."""
    assert [int(v) for v in rng.raw64(0, 4)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_streams_match_the_scalar_definition():
    for key in (1, 0xDEADBEEF, rng.derive_key(7, "w", 3)):
        ref = _splitmix64_reference(key, 257)
        assert [int(v) for v in rng.raw64(key, 257)] == ref
        # a window at an offset is the same stream
        assert [int(v) for v in rng.raw64(key, 5, offset=100)] == ref[100:105]


def test_uniforms_and_normals():
    key = rng.derive_key(0, "test")
    u = rng.uniform01(key, 1 << 20)
    assert u.min() > 0.0 and u.max() < 1.0
    v = rng.raw64(key, 4)
    assert np.array_equal(u[:4], ((v >> np.uint64(11)).astype(np.float64) + 0.5) / 2.0 ** 53)
    n = u.size
    assert abs(u.mean() - 0.5) < 5 / math.sqrt(12 * n)
    assert abs(u.var() - 1 / 12) < 1e-3
    z = rng.normal(key, 1 << 20)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 1e-2
    # Box-Muller of the first pair, written out
    u1, u2 = rng.uniform01(key, 2)
    assert z[0] == np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    assert np.array_equal(rng.normal(key, 3, offset=5), rng.normal(key, 8)[5:])


def test_derived_keys_are_distinct_and_stable():
    keys = {rng.derive_key(s, t) for s in range(4) for t in ("a", "b", "weights", 0, 1)}
    assert len(keys) == 20
    assert rng.derive_key(3, "x") == rng.derive_key(3, "x")
    assert rng.derive_key(3, "x", "y") != rng.derive_key(3, "y", "x")
