"""Parity at the benchmark's full size (|Q| = 1M, |P| = 500k, d = 50), through
the same batched call bench.py times, for float32 (TF32 tiles), BF16 and FP16
indexes.

Two independent references:
* the CPU Simpfer (``oracle/simpfer_cpu.c``: Algorithms 1-3 in float64 with
  exact tie decisions, pinned to the definition on small inputs) gives the
  FULL result set of every checked query, every one of the 1M users;
* the brute-force oracle decides, per query, every returned user (up to 1,500
  of them), every user whose u.q lies within the filter's error bound of its
  k-th bounds (the pairs the filter sends to the exact recheck) and 10,000
  uniform users.
The 20 queries are 10 random items of P and 10 random N(0, I/d) vectors."""
import numpy as np
import pytest

from oracle import rmips_oracle as O
from oracle import simpfer_cpu as S
from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu

N, M, D, K, KMAX, SEED = 1_000_000, 500_000, 50, 10, 25, 3
# relative error bounds of the batched filter's tiles (TF32 for float32 indexes)
REL = {"fp32": 0.00198, "bf16": 0.00788, "fp16": 0.000995}


@pytest.fixture(scope="module")
def data():
    Q, P = datagen.make_problem(N, M, D, SEED)
    qi, _ = datagen.queries_from_items(P, 2000, SEED)
    q20 = np.concatenate([qi[:10], datagen.random_queries(10, D, SEED)])
    cpu = S.SimpferCPU(Q, P, k_max=KMAX, p_prime=100)
    truth = {k: [cpu.query(q, k) for q in q20] for k in (1, K, KMAX)}
    yield Q, P, qi, q20, cpu, truth
    cpu.close()


@pytest.fixture(scope="module")
def indexes(data):
    Q, P = data[0], data[1]
    built = {}

    def get(name):
        if name not in built:
            if name == "noblocks":
                built[name] = rmips.rmips_build_index(Q, P, k_max=KMAX, block_filter=False)
            else:
                built[name] = rmips.rmips_build_index(Q, P, k_max=KMAX, precision=name)
        return built[name]
    yield get
    for ix in built.values():
        ix.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_full_size_full_sets_equal_cpu_simpfer(data, indexes, precision):
    _, _, _, q20, _, truth = data
    index = indexes(precision)
    for k in (1, K, KMAX):
        ids, offs = rmips.rmips_query_batch(index, q20, np.full(len(q20), k, np.int32))
        for j in range(len(q20)):
            assert np.array_equal(ids[offs[j]:offs[j + 1]], truth[k][j]), (precision, k, j)
    for j in range(0, len(q20), 3):                        # the one-launch single-query path
        assert np.array_equal(rmips.rmips_query(index, q20[j], K), truth[K][j]), (precision, j)


def test_full_size_sampled_users_match_brute_force(data, indexes):
    Q, P, _, q20, _, truth = data
    rng = np.random.default_rng(11)
    uniform = rng.choice(N, 10_000, replace=False)
    qn = np.linalg.norm(q20.astype(np.float64), axis=1)
    got, per_query = {}, [set(uniform.tolist()) for _ in q20]
    for precision in ("fp32", "bf16", "fp16"):
        index = indexes(precision)
        ids, offs = rmips.rmips_query_batch(index, q20, np.full(len(q20), K, np.int32))
        got[precision] = [ids[offs[j]:offs[j + 1]] for j in range(len(q20))]
        # pairs the filter cannot decide in O(1): u.q within its error bound
        # of the index's interval [lo_k, hi_k] of u's k-th largest product
        permQ = rmips.rmips_index_export(index, "permQ")
        lo = rmips.rmips_index_export(index, "lo")[K - 1].astype(np.float64)
        hi = rmips.rmips_index_export(index, "hi")[K - 1].astype(np.float64)
        Us = Q[permQ].astype(np.float64)
        un = np.linalg.norm(Us, axis=1)
        G = Us @ q20.astype(np.float64).T
        for j in range(len(q20)):
            e = 1.05 * REL[precision] * un * qn[j] + 1e-30
            near = np.nonzero((G[:, j] >= lo - e) & (G[:, j] <= hi + e))[0]
            per_query[j].update(permQ[near].tolist())
            ret = got[precision][j]
            per_query[j].update((ret if len(ret) <= 1500 else rng.choice(ret, 1500, replace=False)).tolist())
    users = np.array(sorted(set().union(*per_query)), dtype=np.int64)
    yes = O.decide_users_multi(Q, P, q20, K, users, threads=16, chunk=1024)
    for j in range(len(q20)):
        sample = np.array(sorted(per_query[j]), dtype=np.int64)
        exp = users[yes[j]]
        exp = exp[np.isin(exp, sample)]
        # the brute force and the CPU Simpfer agree on the sample ...
        assert np.array_equal(exp, np.intersect1d(truth[K][j], sample)), j
        # ... and so does every GPU path
        for precision in got:
            assert np.array_equal(np.intersect1d(got[precision][j], sample), exp), (precision, j)
    assert len(users) >= 10_000


def test_full_size_mixed_k_batch_matches_cpu_simpfer(data, indexes):
    # the batching workload: 10,000 queries with k uniform in 1..25 in one call
    _, _, qi, _, cpu, _ = data
    qs = np.concatenate([qi, qi[::-1], qi, qi, qi])[:10_000]
    ks = datagen.random_ks(len(qs), 1, KMAX, SEED)
    for precision in ("fp32", "bf16"):
        ids, offs = rmips.rmips_query_batch(indexes(precision), qs, ks)
        for j in np.random.default_rng(5).choice(len(qs), 20, replace=False):
            assert np.array_equal(ids[offs[j]:offs[j + 1]], cpu.query(qs[j], int(ks[j]))), (precision, j)


def test_full_size_without_blocks_matches_cpu_simpfer(data, indexes):
    _, _, _, q20, _, truth = data
    index = indexes("noblocks")
    ids, offs = rmips.rmips_query_batch(index, q20, np.full(len(q20), K, np.int32))
    for j in range(len(q20)):
        assert np.array_equal(ids[offs[j]:offs[j + 1]], truth[K][j]), j
    assert np.array_equal(rmips.rmips_query(index, q20[0], K), truth[K][0])


def test_full_size_monotone_in_k(data, indexes):
    _, _, qi, _, _, _ = data
    index = indexes("fp32")
    sub = qi[:500]
    prev = None
    for k in (1, 5, 10, 11, 25):
        ids, offs = rmips.rmips_query_batch(index, sub, np.full(len(sub), k, np.int32))
        cur = [ids[offs[j]:offs[j + 1]] for j in range(len(sub))]
        if prev is not None:
            for a, b in zip(prev, cur):
                assert np.isin(a, b).all()
        prev = cur
