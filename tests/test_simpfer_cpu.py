"""The CPU Simpfer baseline (``oracle/simpfer_cpu.c``, Algorithms 1-3 in
float64 with exact tie decisions) against the definition.

It serves as the CPU baseline of bench.py and as an exact method for full
result sets at sizes the brute-force oracle cannot reach, so it is pinned here
to the brute force (Definition 2) on tiny inputs, including exact ties.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import rmips_oracle as O
from oracle import simpfer_cpu as S
from paper_2110_07131_gb300 import datagen


def _fsign(u, a, b):
    s = sum(Fraction(float(x)) * (Fraction(float(y)) - Fraction(float(z))) for x, y, z in zip(u, a, b))
    return (s > 0) - (s < 0)


def test_expansion_sign_is_exact():
    rng = np.random.default_rng(0)
    for _ in range(200):
        d = int(rng.integers(1, 80))
        u, a, b = ((rng.standard_normal(d) * 2.0 ** rng.integers(-60, 60, d)).astype(np.float32) for _ in range(3))
        assert S.exact_sign(u, a, b) == _fsign(u, a, b)
    # cancellation far below float64 resolution, and exact ties
    u = np.array([1.0, 1.0, 1.0], np.float32)
    a = np.array([1.0, 2.0 ** -30, -(2.0 ** -30) + 2.0 ** -54], np.float32)
    b = np.array([1.0, 2.0 ** -30, -(2.0 ** -30)], np.float32)
    assert S.exact_sign(u, a, b) == 1 and S.exact_sign(u, b, a) == -1 and S.exact_sign(u, a, a) == 0
    u = np.array([3.0e38, 1.4e-45, -3.0e38, 1.0], np.float32)
    a = np.array([3.0e38, 1.4e-45, 3.0e38, 2.0 ** -60], np.float32)
    b = np.array([3.0e38, 0.0, 3.0e38, 0.0], np.float32)
    assert S.exact_sign(u, a, b) == _fsign(u, a, b) == 1


@pytest.fixture(scope="module")
def tiny():
    Q, P = datagen.make_problem(2000, 1000, 50, 0)
    qs, _ = datagen.queries_from_items(P, 12, 0)
    qs = np.concatenate([qs, datagen.random_queries(4, 50, 0), np.zeros((1, 50), np.float32)])
    return Q, P, qs, O.counts_greater_multi(Q, P, qs)


@pytest.mark.parametrize("p_prime,bs", [(100, 32), (0, 32), (10, 20), (100, 1), (1000, 256)])
def test_simpfer_cpu_equals_definition(tiny, p_prime, bs):
    Q, P, qs, counts = tiny
    idx = S.SimpferCPU(Q, P, k_max=25, p_prime=p_prime, block_size=bs)
    for j in range(len(qs)):
        for k in (1, 10, 25):
            got = idx.query(qs[j], k)
            assert np.array_equal(got, np.nonzero(counts[j] < k)[0]), (p_prime, bs, j, k)
    idx.close()


def test_simpfer_cpu_thread_counts_agree(tiny):
    Q, P, qs, counts = tiny
    idx = S.SimpferCPU(Q, P, k_max=25)
    for j in range(4):
        st1, stn = {}, {}
        one = idx.query(qs[j], 10, threads=1, stats=st1)
        many = idx.query(qs[j], 10, threads=0, stats=stn)
        assert np.array_equal(one, many) and np.array_equal(one, np.nonzero(counts[j] < 10)[0])
        assert st1 == stn                            # the per-block work does not depend on the threads
    idx.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_simpfer_cpu_on_exact_ties(seed):
    Q, P = datagen.integer_problem(300, 80, 4, seed, lim=2)
    qs = np.concatenate([P[:15], Q[:5]])
    counts = O.counts_greater_multi(Q, P, qs)
    for p_prime in (8, 0):
        idx = S.SimpferCPU(Q, P, k_max=12, p_prime=p_prime, block_size=16)
        for j in range(len(qs)):
            for k in (1, 3, 12):
                assert np.array_equal(idx.query(qs[j], k), np.nonzero(counts[j] < k)[0]), (seed, p_prime, j, k)
        idx.close()


def test_simpfer_cpu_prunes_and_uses_the_lemmas(tiny):
    Q, P, qs, _ = tiny
    idx = S.SimpferCPU(Q, P, k_max=25)
    tot = dict(pruned_blocks=0, lemma1_no=0, lemma2_yes=0, scanned=0)
    for j in range(len(qs)):
        st = {}
        idx.query(qs[j], 10, stats=st)
        for key in tot:
            tot[key] += st[key]
    assert tot["pruned_blocks"] > 0 and tot["lemma1_no"] > 0 and tot["scanned"] > 0
    with pytest.raises(ValueError):
        idx.query(qs[0], 26)
    idx.close()
