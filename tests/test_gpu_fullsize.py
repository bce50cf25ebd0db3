"""Parity at the benchmark's full size (|Q| = 1M, |P| = 500k, d = 50), through
the same batched call bench.py times.  The oracle decides sampled users one by
one; properties that hold at any size cover the rest."""
import numpy as np
import pytest

from oracle import rmips_oracle as O
from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu

N, M, D, K, KMAX, SEED = 1_000_000, 500_000, 50, 10, 25, 3


@pytest.fixture(scope="module")
def big():
    Q, P = datagen.make_problem(N, M, D, SEED)
    index = rmips.rmips_build_index(Q, P, k_max=KMAX)
    qs, _ = datagen.queries_from_items(P, 2000, SEED)
    yield Q, P, qs, index
    index.close()


def test_full_size_sampled_users_match_oracle(big):
    Q, P, qs, index = big
    ids, offs = rmips.rmips_query_batch(index, qs, np.full(len(qs), K, np.int32))
    rng = np.random.default_rng(11)
    # the queries with the largest results and a few random ones
    sizes = np.diff(offs)
    pick = np.unique(np.concatenate([np.argsort(-sizes)[:2], rng.choice(len(qs), 3, replace=False)]))
    for j in pick:
        got = ids[offs[j]:offs[j + 1]]
        sample = np.unique(np.concatenate([got[:150], rng.choice(N, 150, replace=False)]))
        truth = O.decide_users(Q, P, qs[j], K, sample)
        assert np.array_equal(np.intersect1d(sample, got), sample[truth]), j


def test_full_size_single_and_batched_paths_agree(big):
    _, _, qs, index = big
    ids, offs = rmips.rmips_query_batch(index, qs[:64], np.full(64, K, np.int32))
    for j in range(0, 64, 4):
        assert np.array_equal(rmips.rmips_query(index, qs[j], K), ids[offs[j]:offs[j + 1]])


def test_full_size_monotone_in_k(big):
    _, _, qs, index = big
    sub = qs[:500]
    prev = None
    for k in (1, 5, 10, 11, 25):
        ids, offs = rmips.rmips_query_batch(index, sub, np.full(len(sub), k, np.int32))
        cur = [ids[offs[j]:offs[j + 1]] for j in range(len(sub))]
        if prev is not None:
            for a, b in zip(prev, cur):
                assert np.isin(a, b).all()
        prev = cur


def test_full_size_mixed_k_batch(big):
    _, _, qs, index = big
    ks = datagen.random_ks(len(qs), 1, KMAX, SEED)
    ids, offs = rmips.rmips_query_batch(index, qs, ks)
    for j in range(0, len(qs), 97):
        assert np.array_equal(rmips.rmips_query(index, qs[j], int(ks[j])), ids[offs[j]:offs[j + 1]])
