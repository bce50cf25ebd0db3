"""CUDA path vs the CPU oracle: exact-set parity, through the C ABI."""
import numpy as np
import pytest

from oracle import rmips_oracle as O
from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    cfg = datagen.CONFIGS["tiny"]
    Q, P = datagen.make_problem(cfg["n"], cfg["m"], cfg["d"], cfg["seed"])
    qs, qidx = datagen.queries_from_items(P, cfg["nq"], cfg["seed"])
    rq = datagen.random_queries(10, cfg["d"], cfg["seed"])
    allq = np.concatenate([qs, rq])
    counts = O.counts_greater_multi(Q, P, allq)          # [nq, n] exact c(u)
    return Q, P, allq, counts


def _check_all(index, allq, counts, ks):
    for k in ks:
        ids, offs = rmips.rmips_query_batch(index, allq, np.full(len(allq), k, np.int32))
        for j in range(len(allq)):
            exp = np.nonzero(counts[j] < k)[0]
            got = ids[offs[j]:offs[j + 1]]
            assert np.array_equal(got, exp), (k, j, len(got), len(exp))


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("p_prime", [0, 100])
def test_tiny_config_parity(tiny, precision, p_prime):
    Q, P, allq, counts = tiny
    index = rmips.rmips_build_index(Q, P, k_max=25, p_prime=p_prime, precision=precision)
    _check_all(index, allq, counts, (1, 5, 10, 25))
    index.close()


def test_tiny_config_parity_cuda_core_batches(tiny):
    Q, P, allq, counts = tiny
    for p_prime in (0, 100):
        index = rmips.rmips_build_index(Q, P, k_max=25, p_prime=p_prime, batch_tensor_cores=False,
                                        build_tensor_cores=False)
        _check_all(index, allq, counts, (1, 10, 25))


def test_mixed_k_batch_tensor_and_cuda_cores_agree(tiny):
    Q, P, allq, counts = tiny
    ks = datagen.random_ks(len(allq), 1, 25, 0)
    for tc in (True, False):
        index = rmips.rmips_build_index(Q, P, k_max=25, batch_tensor_cores=tc)
        ids, offs = rmips.rmips_query_batch(index, allq, ks)
        for j in range(len(allq)):
            assert np.array_equal(ids[offs[j]:offs[j + 1]], np.nonzero(counts[j] < ks[j])[0])


@pytest.mark.parametrize("bs", [64, 256])
def test_block_sizes(tiny, bs):
    Q, P, allq, counts = tiny
    index = rmips.rmips_build_index(Q, P, k_max=25, block_size=bs)
    _check_all(index, allq, counts, (3, 10))


@pytest.mark.parametrize("p_prime", [0, 100])
def test_single_query_api_matches(tiny, p_prime):
    Q, P, allq, counts = tiny
    index = rmips.rmips_build_index(Q, P, k_max=25, p_prime=p_prime)
    for j in range(0, len(allq), 7):
        for k in (1, 10, 25):
            got = rmips.rmips_query(index, allq[j], k)
            assert np.array_equal(got, np.nonzero(counts[j] < k)[0])
            # alternate with batches on the same index: shared workspaces stay consistent
            ids, offs = rmips.rmips_query_batch(index, allq[j:j + 2], k)
            assert np.array_equal(ids[offs[0]:offs[1]], got)


@pytest.mark.parametrize("build_tc,precision", [(True, "fp32"), (False, "fp32"), (True, "bf16"), (True, "fp16")])
def test_index_arrays_match_oracle(tiny, build_tc, precision):
    # the candidate selection runs on tensor cores in TF32, BF16 or FP16 (the
    # index's precision) or on CUDA cores; the bounds are rigorous either way
    Q, P, _, _ = tiny
    k_max = 25
    index = rmips.rmips_build_index(Q, P, k_max=k_max, build_tensor_cores=build_tc, precision=precision)
    assert rmips.rmips_index_get_info(index)["build_kind"] == (
        {"fp32": 0, "bf16": 1, "fp16": 2}[precision] if build_tc else -1)
    permQ = rmips.rmips_index_export(index, "permQ")
    permP = rmips.rmips_index_export(index, "permP")
    assert np.array_equal(permQ, O.norm_order(Q))
    assert np.array_equal(permP, O.norm_order(P))
    v = O.kth_values(Q[permQ], P, k_max)                   # [n, k_max] float64
    lo = rmips.rmips_index_export(index, "lo").T
    hi = rmips.rmips_index_export(index, "hi").T
    scale = np.abs(Q[permQ]).astype(np.float64) @ np.abs(P).astype(np.float64).max(axis=0)
    tol = 1e-12 * scale[:, None]
    assert (lo <= v + tol).all() and (hi >= v - tol).all()
    assert (hi - lo <= 1e-5 * (1 + np.abs(v))).all()      # bounds are tight
    LB = rmips.rmips_index_export(index, "LB")
    hdr = rmips.rmips_index_export(index, "hdr")
    for b in range(LB.shape[1]):
        assert np.array_equal(LB[:, b], lo[32 * b:32 * b + 32].min(axis=0))
    nrm = O.norms_fp64(Q[permQ])
    assert (hdr >= nrm[::32]).all() and (hdr <= nrm[::32] * (1 + 1e-6)).all()
    assert rmips.rmips_index_get_info(index)["incomplete"] == 0


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("p_prime", [0, 8])
def test_integer_ties_exact(precision, p_prime):
    Q, P = datagen.integer_problem(300, 90, 8, 5, lim=2)
    qs = np.concatenate([P[:12], Q[:4], np.zeros((1, 8), np.float32)])
    counts = O.counts_greater_multi(Q, P, qs)
    index = rmips.rmips_build_index(Q, P, k_max=12, p_prime=p_prime, precision=precision)
    _check_all(index, qs, counts, (1, 2, 5, 12))


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_massive_ties_use_scan_fallback(precision):
    # components in {-1, 0, 1}, d = 3: only 7 distinct inner products, so the
    # values at ranks k_max..32 tie and completeness cannot be proven
    Q, P = datagen.integer_problem(400, 120, 3, 8, lim=1)
    qs = np.concatenate([P[:10], Q[:3]])
    counts = O.counts_greater_multi(Q, P, qs)
    index = rmips.rmips_build_index(Q, P, k_max=12, precision=precision)
    assert rmips.rmips_index_get_info(index)["incomplete"] > 0
    _check_all(index, qs, counts, (1, 4, 12))


@pytest.mark.parametrize("n,m,d,k_max", [(1, 1, 3, 1), (31, 3, 5, 5), (33, 40, 7, 8), (1007, 31, 50, 25),
                                         (70, 2, 64, 25), (257, 129, 128, 4)])
def test_ragged_sizes(n, m, d, k_max):
    Q, P = datagen.make_problem(n, m, d, 17)
    qs = np.concatenate([P[:2], datagen.random_queries(2, d, 3)])
    counts = O.counts_greater_multi(Q, P, qs)
    for p_prime in (0, 2):
        index = rmips.rmips_build_index(Q, P, k_max=k_max, p_prime=p_prime)
        _check_all(index, qs, counts, sorted({1, k_max}))


def test_zero_and_scaled_queries(tiny):
    Q, P, _, _ = tiny
    index = rmips.rmips_build_index(Q, P, k_max=25)
    qs = np.stack([np.zeros(50, np.float32), P[3] * 8.0, P[5] * 0.125, -P[9]]).astype(np.float32)
    counts = O.counts_greater_multi(Q, P, qs)
    _check_all(index, qs, counts, (1, 10, 25))


def test_errors(tiny):
    Q, P, allq, _ = tiny
    index = rmips.rmips_build_index(Q, P, k_max=10)
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query(index, allq[0], 0)
    assert e.value.status == 2
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query(index, allq[0], 11)
    assert e.value.status == 2
    bad = allq[0].copy()
    bad[3] = np.nan
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query(index, bad, 5)
    assert e.value.status == 3
    # the index stays usable after an error
    qbig = (allq[1] * 4.0).astype(np.float32)           # a large norm: many users
    full = rmips.rmips_query(index, qbig, 10)
    assert len(full) > 1
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query(index, qbig, 10, capacity=len(full) - 1)
    assert e.value.status == 5
    assert np.array_equal(rmips.rmips_query(index, qbig, 10, capacity=len(full)), full)
    ids, offs = rmips.rmips_query_batch(index, np.stack([allq[0], qbig]), 10)
    assert np.array_equal(ids[offs[1]:offs[2]], full)
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query_batch(index, np.stack([allq[0], qbig]), 10, capacity=len(full) - 1)
    assert e.value.status == 5
    Qb = Q.copy()
    Qb[7, 2] = np.inf
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_build_index(Qb, P, k_max=10)
    assert e.value.status == 3


def test_fp16_index_refuses_values_beyond_its_range(tiny):
    # an FP16 copy of |x| > 65504 would be infinite and break the filter's
    # bounds: the build and the queries refuse such values (status 3); a
    # float32 index answers them exactly
    Q, P, allq, _ = tiny
    Qb = Q.copy()
    Qb[11, 4] = 70000.0
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_build_index(Qb, P, k_max=10, precision="fp16")
    assert e.value.status == 3
    index16 = rmips.rmips_build_index(Q, P, k_max=10, precision="fp16")
    q = allq[2].copy()
    q[5] = 70000.0
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query(index16, q, 5)
    assert e.value.status == 3
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query_batch(index16, np.stack([allq[0], q]), 5)
    assert e.value.status == 3
    ok = rmips.rmips_query(index16, allq[0], 5)           # still usable
    index32 = rmips.rmips_build_index(Q, P, k_max=10)
    assert np.array_equal(rmips.rmips_query(index32, allq[0], 5), ok)
    got = rmips.rmips_query(index32, q, 5)
    exp = np.nonzero(O.counts_greater_multi(Q, P, q[None, :])[0] < 5)[0]
    assert np.array_equal(got, exp)


def test_segments(tiny):
    Q, P, allq, counts = tiny
    index = rmips.rmips_build_index(Q, P, k_max=25)
    rng = np.random.default_rng(0)
    subset = np.sort(rng.choice(Q.shape[0], 700, replace=False))
    for j in range(0, 40, 3):
        exp = np.nonzero(counts[j] < 25)[0]
        got = rmips.rmips_query(index, allq[j], 25, segment=(500, 1500))
        assert np.array_equal(got, exp[(exp >= 500) & (exp < 1500)])
        got = rmips.rmips_query(index, allq[j], 25, segment=subset)
        assert np.array_equal(got, np.intersect1d(exp, subset))
    ids, offs = rmips.rmips_query_batch(index, allq[:6], 25, segments=[None, (0, 10), subset, None, (1990, 2000), subset])
    for j, sg in enumerate([None, (0, 10), subset, None, (1990, 2000), subset]):
        exp = np.nonzero(counts[j] < 25)[0]
        if isinstance(sg, tuple):
            exp = exp[(exp >= sg[0]) & (exp < sg[1])]
        elif sg is not None:
            exp = np.intersect1d(exp, sg)
        assert np.array_equal(ids[offs[j]:offs[j + 1]], exp)


def test_device_pointers(tiny):
    torch = pytest.importorskip("torch")
    Q, P, allq, counts = tiny
    dQ, dP = torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda()
    index = rmips.rmips_build_index(dQ, dP, k_max=25)
    dq = torch.from_numpy(allq[:20]).cuda()
    dk = torch.full((20,), 10, dtype=torch.int32, device="cuda")
    out = torch.empty(20 * 2000, dtype=torch.int64, device="cuda")
    ids, offs = rmips.rmips_query_batch(index, dq, dk, out=out)
    ids = ids.cpu().numpy()
    for j in range(20):
        assert np.array_equal(ids[offs[j]:offs[j + 1]], np.nonzero(counts[j] < 10)[0])
    out1 = torch.empty(2000, dtype=torch.int64, device="cuda")
    got = rmips.rmips_query(index, dq[3], 10, out=out1)
    assert np.array_equal(got.cpu().numpy(), np.nonzero(counts[3] < 10)[0])


def test_large_result_bitmap_path():
    # a query with a huge norm is in the top-k of most users: > 8192 results
    Q, P = datagen.make_problem(40000, 500, 16, 2)
    q = (P[0] * 200.0).astype(np.float32)
    counts = O.counts_greater(Q, P, q)
    index = rmips.rmips_build_index(Q, P, k_max=5)
    got = rmips.rmips_query(index, q, 5)
    exp = np.nonzero(counts < 5)[0]
    assert len(exp) > 8192
    assert np.array_equal(got, exp)
    # the batched path sorts such a result in global scratch memory
    ids, offs = rmips.rmips_query_batch(index, np.stack([q, P[1], q]), 5)
    assert np.array_equal(ids[offs[0]:offs[1]], exp)
    assert np.array_equal(ids[offs[2]:offs[3]], exp)


def test_plain_config_sum_identity_and_samples():
    cfg = datagen.CONFIGS["plain"]
    n, m, d = cfg["n"], cfg["m"], cfg["d"]
    Q, P = datagen.make_problem(n, m, d, cfg["seed"])
    index = rmips.rmips_build_index(Q, P, k_max=25)
    # Every item as a query: each user has exactly k items whose top-k holds it.
    for k in (1, 10):
        ids, offs = rmips.rmips_query_batch(index, P, np.full(m, k, np.int32))
        assert offs[-1] == n * k
    qs, _ = datagen.queries_from_items(P, 6, cfg["seed"])
    rng = np.random.default_rng(5)
    for j, q in enumerate(qs):
        for k in cfg["ks"][::2]:
            got = rmips.rmips_query(index, q, k)
            sample = np.unique(np.concatenate([got, rng.choice(n, 150, replace=False)]))
            truth = O.decide_users(Q, P, q, k, sample)
            assert np.array_equal(sample[truth], got), (j, k)


def test_batch_with_many_large_results():
    # more large-result queries than the batched emitter's 64 bitmaps: several rounds
    Q, P = datagen.make_problem(20000, 400, 8, 4)
    qs = np.concatenate([(P[:70] * 500.0).astype(np.float32), P[70:90]])
    counts = O.counts_greater_multi(Q, P, qs)
    index = rmips.rmips_build_index(Q, P, k_max=5)
    ids, offs = rmips.rmips_query_batch(index, qs, np.full(len(qs), 5, np.int32))
    big = 0
    for j in range(len(qs)):
        exp = np.nonzero(counts[j] < 5)[0]
        big += len(exp) > 8192
        assert np.array_equal(ids[offs[j]:offs[j + 1]], exp), j
    assert big > 64


def test_precision_modes_return_identical_sets():
    # d = 64 with queries from P and random N(0, I/d) queries, as in the
    # precision workload: BF16 / FP16 tensor-core filtering must not change
    # any result, only how many pairs need the exact recheck
    n, m, d = 40000, 20000, 64
    Q, P = datagen.make_problem(n, m, d, 2)
    qs = np.concatenate([datagen.queries_from_items(P, 300, 2)[0], datagen.random_queries(300, d, 2)])
    ks = datagen.random_ks(len(qs), 1, 25, 2)
    res = {}
    for prec in ("fp32", "bf16", "fp16"):
        index = rmips.rmips_build_index(Q, P, k_max=25, precision=prec)
        ids, offs = rmips.rmips_query_batch(index, qs, ks)
        res[prec] = [ids[offs[j]:offs[j + 1]] for j in range(len(qs))]
        st = rmips.rmips_last_query_stats(index)
        res[prec + "_todo"] = st["todo"]
        index.close()
    for j in range(len(qs)):
        assert np.array_equal(res["bf16"][j], res["fp32"][j]), j
        assert np.array_equal(res["fp16"][j], res["fp32"][j]), j
    assert res["bf16_todo"] >= res["fp16_todo"]          # coarser format, more rechecks
    rng = np.random.default_rng(3)
    for j in rng.choice(len(qs), 4, replace=False):
        got = res["fp32"][j]
        sample = np.unique(np.concatenate([got[:100], rng.choice(n, 100, replace=False)]))
        truth = O.decide_users(Q, P, qs[j], int(ks[j]), sample)
        assert np.array_equal(np.intersect1d(sample, got), sample[truth])


def test_async_batch_matches_sync_and_reports_on_device():
    torch = pytest.importorskip("torch")
    Q, P = datagen.make_problem(20000, 5000, 50, 13)
    index = rmips.rmips_build_index(Q, P, k_max=25)
    qs, _ = datagen.queries_from_items(P, 3000, 13)
    ks = datagen.random_ks(len(qs), 1, 25, 13)
    ids_ref, offs_ref = rmips.rmips_query_batch(index, qs, ks)
    total = int(offs_ref[-1])
    dev = torch.device("cuda")
    dq, dk = torch.from_numpy(qs).to(dev), torch.from_numpy(ks).to(dev)
    stream = torch.cuda.current_stream()
    rmips.rmips_profile_enable(index, True)
    outs = []
    for _ in range(2):                                   # two calls in a row on one workspace
        out = torch.full((total + 7,), -1, dtype=torch.int64, device=dev)
        offs = torch.empty(len(qs) + 1, dtype=torch.int64, device=dev)
        done = torch.full((2,), -1, dtype=torch.int64, device=dev)
        rmips.rmips_query_batch_async(index, dq, dk, out, offs, done, stream)
        outs.append((out, offs, done))
    ids_sync, _ = rmips.rmips_query_batch(index, qs[:100], ks[:100])   # a synchronous call in between
    torch.cuda.synchronize()
    for out, offs, done in outs:
        assert done.tolist() == [0, total]
        assert np.array_equal(offs.cpu().numpy(), offs_ref)
        assert np.array_equal(out[:total].cpu().numpy(), ids_ref)
    assert np.array_equal(ids_sync, ids_ref[:offs_ref[100]])
    prof = rmips.rmips_profile_read(index)
    assert prof["mfilter_launches"] >= 2 and prof["mfilter_pairs"] > 0 and prof["mfilter_ms"] > 0
    rmips.rmips_profile_enable(index, False)
    # device-side errors arrive in done
    small = torch.empty(max(1, total // 2), dtype=torch.int64, device=dev)
    offs = torch.empty(len(qs) + 1, dtype=torch.int64, device=dev)
    done = torch.empty(2, dtype=torch.int64, device=dev)
    rmips.rmips_query_batch_async(index, dq, dk, small, offs, done, stream)
    torch.cuda.synchronize()
    assert done.tolist() == [5, total] and int(offs[-1]) == total
    bad = dk.clone()
    bad[7] = 26
    rmips.rmips_query_batch_async(index, dq, bad, outs[0][0], offs, done, stream)
    torch.cuda.synchronize()
    assert int(done[0]) == 2
    with pytest.raises(rmips.RmipsError):
        rmips.rmips_query_batch_async(index, qs, ks, outs[0][0], offs, done, stream)   # host arrays
    index.close()


def test_async_batches_on_two_streams_overlap_correctly():
    # consecutive batches queued on two streams in turn run on two workspaces
    # at once (each replaying its own graphs after two uses); every batch must
    # still return exactly the synchronous answer, including batches of
    # another size in between
    torch = pytest.importorskip("torch")
    Q, P = datagen.make_problem(30000, 6000, 50, 29)
    index = rmips.rmips_build_index(Q, P, k_max=25)
    qs, _ = datagen.queries_from_items(P, 8 * 1200, 29)
    ks = datagen.random_ks(len(qs), 1, 25, 29)
    sizes = [1200, 1200, 1200, 1200, 700, 1200, 1200, 1200]
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    refs = [rmips.rmips_query_batch(index, qs[a:a + n], ks[a:a + n]) for a, n in zip(starts, sizes)]
    dev = torch.device("cuda")
    dq, dk = torch.from_numpy(qs).to(dev), torch.from_numpy(ks).to(dev)
    streams = [torch.cuda.current_stream(), torch.cuda.Stream()]
    outs = []
    for rnd in range(2):
        for i, (a, n) in enumerate(zip(starts, sizes)):
            total = int(refs[i][1][-1])
            out = torch.full((total + 5,), -1, dtype=torch.int64, device=dev)
            offs = torch.empty(n + 1, dtype=torch.int64, device=dev)
            done = torch.full((2,), -1, dtype=torch.int64, device=dev)
            rmips.rmips_query_batch_async(index, dq[a:a + n], dk[a:a + n], out, offs, done, streams[i & 1])
            outs.append((i, out, offs, done))
    torch.cuda.synchronize()
    for i, out, offs, done in outs:
        ids_ref, offs_ref = refs[i]
        total = int(offs_ref[-1])
        assert done.tolist() == [0, total], i
        assert np.array_equal(offs.cpu().numpy(), offs_ref), i
        assert np.array_equal(out[:total].cpu().numpy(), ids_ref), i
    index.close()


def test_graph_replay_with_same_and_changing_batches():
    """Passes with unchanged arguments replay captured graphs (from the second
    identical call on); new query data under the same arguments, and changed
    sizes, must still give the single-query answers."""
    Q, P = datagen.make_problem(20000, 5000, 50, 17)
    index = rmips.rmips_build_index(Q, P, k_max=25)
    qa, _ = datagen.queries_from_items(P, 1500, 17)
    qb, _ = datagen.queries_from_items(P, 1500, 18)
    ks = datagen.random_ks(1500, 1, 25, 17)
    ref = {}
    for name, qs in (("a", qa), ("b", qb)):
        ref[name] = [rmips.rmips_query(index, qs[j], int(ks[j])) for j in range(0, 1500, 37)]
    seq = [("a", 1500), ("a", 1500), ("a", 1500), ("b", 1500), ("b", 1500), ("a", 700), ("a", 700), ("b", 1500)]
    for name, nq in seq:
        qs = qa if name == "a" else qb
        ids, offs = rmips.rmips_query_batch(index, qs[:nq], ks[:nq])
        for r, j in enumerate(range(0, nq, 37)):
            assert np.array_equal(ids[offs[j]:offs[j + 1]], ref[name][r]), (name, nq, j)
    index.close()


@pytest.mark.parametrize("bs", [32, 128])
def test_no_block_filter_gives_the_same_answers(bs):
    """Lemma 3 only skips work: switching it off (every block bound -inf) must
    not change any answer, single or batched."""
    Q, P = datagen.make_problem(6000, 2000, 50, 23)
    on = rmips.rmips_build_index(Q, P, k_max=25, block_size=bs)
    off = rmips.rmips_build_index(Q, P, k_max=25, block_size=bs, block_filter=False)
    assert (rmips.rmips_index_export(off, "LB") == -np.inf).all()
    qs, _ = datagen.queries_from_items(P, 300, 23)
    ks = datagen.random_ks(len(qs), 1, 25, 23)
    a = rmips.rmips_query_batch(on, qs, ks)
    b = rmips.rmips_query_batch(off, qs, ks)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for j in range(0, len(qs), 29):
        assert np.array_equal(rmips.rmips_query(off, qs[j], int(ks[j])), a[0][a[1][j]:a[1][j + 1]])
    on.close()
    off.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_pair_list_overflow_splits_the_pass(monkeypatch, precision):
    # Ties-heavy data leaves many (user, query) pairs undecided by the O(1)
    # tests.  With the pair list shrunk to 64 entries a whole-batch pass
    # overflows it; the call runs the batch again in smaller passes (down to
    # the per-query path) and must still return the oracle's sets.
    monkeypatch.setenv("RMIPS_PAIR_LIST_CAP", "64")
    Q, P = datagen.integer_problem(400, 120, 3, 8, lim=1)
    qs = np.concatenate([P, Q[:40]])
    counts = O.counts_greater_multi(Q, P, qs)
    index = rmips.rmips_build_index(Q, P, k_max=12, precision=precision)
    for k in (1, 4, 12):
        ids, offs = rmips.rmips_query_batch(index, qs, np.full(len(qs), k, np.int32))
        for j in range(len(qs)):
            assert np.array_equal(ids[offs[j]:offs[j + 1]], np.nonzero(counts[j] < k)[0]), (k, j)
    # with the default list, one pass of the same batch holds more than 64
    # undecided pairs: the small list really overflowed above
    monkeypatch.delenv("RMIPS_PAIR_LIST_CAP")
    big = rmips.rmips_build_index(Q, P, k_max=12, precision=precision)
    rmips.rmips_query_batch(big, qs, np.full(len(qs), 12, np.int32))
    assert rmips.rmips_last_query_stats(big)["todo"] > 64
    big.close()
    index.close()


@pytest.mark.parametrize("p_prime", [0, 100])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_async_single_queries_back_to_back(tiny, p_prime, precision):
    # rmips_query_async: device buffers, no host wait; many calls queued back
    # to back on one stream (the workspaces alternate) give the oracle's sets
    torch = pytest.importorskip("torch")
    Q, P, allq, counts = tiny
    index = rmips.rmips_build_index(Q, P, k_max=25, p_prime=p_prime, precision=precision)
    dq = torch.from_numpy(allq).cuda()
    nq = len(allq)
    outs = torch.full((nq, 2000), -1, dtype=torch.int64, device="cuda")
    dones = torch.full((nq, 2), -7, dtype=torch.int64, device="cuda")
    st = torch.cuda.Stream()
    ks = [1 + (j * 7) % 25 for j in range(nq)]
    with torch.cuda.stream(st):
        for j in range(nq):
            rmips.rmips_query_async(index, dq[j], ks[j], outs[j], dones[j], stream=st)
    st.synchronize()
    d = dones.cpu().numpy()
    o = outs.cpu().numpy()
    assert (d[:, 0] == 0).all(), d[:, 0]
    for j in range(nq):
        assert np.array_equal(o[j, :d[j, 1]], np.nonzero(counts[j] < ks[j])[0]), (j, ks[j])
    # too small an output buffer: the status says so and the size needed is reported
    small = torch.empty(1, dtype=torch.int64, device="cuda")
    done = torch.zeros(2, dtype=torch.int64, device="cuda")
    j = int(np.argmax((counts < 25).sum(axis=1)))
    rmips.rmips_query_async(index, dq[j], 25, small, done)
    torch.cuda.synchronize()
    assert done.cpu().tolist() == [5, int((counts[j] < 25).sum())]
    with pytest.raises(rmips.RmipsError):
        rmips.rmips_query_async(index, dq[0], 26, outs[0], dones[0])
    index.close()


def test_single_query_kernel_ragged_spans():
    # users not a multiple of the kernel's span (ten chunks of 32 users: 320),
    # one short of and just past one and two spans, blocks of every size, and
    # the largest results (bitmap emit): the one-launch kernel against the oracle
    for n, m, d, bs in ((1, 3, 5, 32), (255, 40, 50, 32), (257, 60, 50, 64), (319, 50, 50, 32),
                        (321, 60, 50, 64), (641, 70, 50, 32), (9000, 300, 64, 256), (700, 90, 128, 128)):
        Q, P = datagen.make_problem(n, m, d, 23)
        qs = np.concatenate([P[:3] * 6.0, datagen.random_queries(2, d, 5), np.zeros((1, d), np.float32)])
        counts = O.counts_greater_multi(Q, P, qs)
        index = rmips.rmips_build_index(Q, P, k_max=min(25, m), block_size=bs)
        for j in range(len(qs)):
            for k in sorted({1, min(25, m)}):
                assert np.array_equal(rmips.rmips_query(index, qs[j], k), np.nonzero(counts[j] < k)[0]), (n, j, k)
        index.close()
