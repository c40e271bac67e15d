"""Pins for oracle.rng: published Philox vectors, sampler invariants, normal law."""

import os

import numpy as np
from scipy import stats

from oracle import rng as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def load_kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answer_vectors():
    kat = load_kat()
    assert len(kat) == 3
    for ctr, key, out in kat:
        got = R.philox4x32_10(np.array(ctr, dtype=np.uint64), key)
        assert [int(x) for x in got] == out


def test_philox_vectorised_matches_scalar_calls():
    ctr = np.array([[i, 7, i * 3, 2] for i in range(50)], dtype=np.uint64)
    batch = R.philox4x32_10(ctr, (123, 456))
    for i in range(50):
        np.testing.assert_array_equal(batch[i], R.philox4x32_10(ctr[i], (123, 456)))


def test_block_sampler_distinct_in_range_and_full_permutation():
    for n in [1, 2, 3, 5, 17, 64, 1000, 4097]:
        for t in [0, 1, 9]:
            B = R.sample_block(n, n, seed=11, t=t)
            assert sorted(B.tolist()) == list(range(n))     # b = n: a permutation
    B = R.sample_block(100000, 3000, seed=5, t=2)
    assert len(np.unique(B)) == 3000 and B.min() >= 0 and B.max() < 100000


def test_block_sampler_is_uniform_over_rows():
    n, b, T = 40, 10, 4000
    counts = np.zeros(n)
    for t in range(T):
        counts[R.sample_block(n, b, seed=3, t=t)] += 1
    expected = T * b / n
    chi2 = np.sum((counts - expected) ** 2 / expected)
    assert stats.chi2.sf(chi2, n - 1) > 1e-3
    first = np.array([R.sample_block(n, 2, seed=3, t=t) for t in range(T)])
    diff = (first[:, 1] - first[:, 0]) % n
    cnt = np.bincount(diff, minlength=n)[1:]
    exp2 = T / (n - 1)
    assert stats.chi2.sf(np.sum((cnt - exp2) ** 2 / exp2), n - 2) > 1e-3


def test_normals_follow_standard_normal_law():
    z = R.normals(200000, seed=7, t=3, stream=R.OMEGA)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    z2 = R.normals(200000, seed=7, t=3, stream=R.V0)
    z3 = R.normals(200000, seed=7, t=4, stream=R.OMEGA)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.01
    assert abs(np.corrcoef(z, z3)[0, 1]) < 0.01


def test_box_muller_words_map_as_documented():
    w = R.philox4x32_10(np.array([1, 5, 0, R.V0], dtype=np.uint64), R.seed_key(99))
    u = (w.astype(np.float64) + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2 * np.log(u[2]))
    expect = rad * np.sin(2 * np.pi * u[3])          # element 7 = word pair (2,3), odd
    got = R.normals(8, seed=99, t=5, stream=R.V0)[7]
    assert abs(got - expect) < 1e-15


def test_omega_scaling():
    Om = R.sample_omega(4000, 8, seed=1, t=0)
    np.testing.assert_allclose(np.diag(Om.T @ Om), 1.0, atol=0.08)
