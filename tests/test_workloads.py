"""The seeded input generator shared by the oracle and the GPU side: its SplitMix64
finaliser against the published outputs, the uniform and normal transforms, and the
determinism and shapes of the workloads."""
import os

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def test_splitmix64_matches_published_outputs():
    want = [int(line, 16) for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        got = [int(W._mix(np.array([g * np.uint64(i)], dtype=np.uint64))[0])
               for i in range(1, len(want) + 1)]
    assert got == want


def test_streams_are_counter_based_and_distinct():
    a = W.raw_stream(7, 1, 10)
    assert np.array_equal(a[3:], W.raw_stream(7, 1, 7, offset=3))  # any index, directly
    assert not np.array_equal(a, W.raw_stream(7, 2, 10))
    assert not np.array_equal(a, W.raw_stream(8, 1, 10))


def test_uniform_and_normal_transforms():
    u = W.uniform(3, 1, 200000, -1.0, 1.0)
    assert u.min() > -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    z = W.normal(3, 2, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_workloads_are_deterministic_and_sized():
    p1, p2 = W.workload1(), W.workload1()
    assert np.array_equal(p1.kappa, p2.kappa) and np.array_equal(p1.f, p2.f)
    assert p1.N == 65 ** 2 and p1.r == 8 and p1.agg.min() == 0 and p1.agg.max() == 7
    q = W.workload2(64)
    assert q.kappa.shape == (64 * 64,) and q.f.shape == (65 * 65,)
    assert np.all(q.kappa > 0)
