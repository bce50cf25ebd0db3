"""rmips_query_noalloc gives the same answers as rmips_query.

The allocation-free entry point exists for callers that cannot allocate
device memory during a query: code whose device memory is owned by another
allocator (a framework's caching allocator that has reserved the free memory)
and latency-critical serving threads, where cudaMalloc / cudaFree can stall
the whole device.  Its scratch is one fixed device array shared by every call,
so two calls in a row must not see each other's leftovers.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu


def test_noalloc_matches_rmips_query_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    Q, P = datagen.make_problem(5000, 2000, 50, 21)
    index = rmips.rmips_build_index(Q, P, k_max=25)
    qs, _ = datagen.queries_from_items(P, 6, 21)
    qs = np.concatenate([qs, (P[:1] * 6.0).astype(np.float32)])   # one query with a large result
    out = torch.empty(5000, dtype=torch.int64, device="cuda")
    for q in qs:
        dq = torch.from_numpy(q).cuda()
        for k in (1, 10, 25):
            ref = rmips.rmips_query(index, q, k)
            for _ in range(2):
                out.fill_(-7)
                cnt = rmips.rmips_query_noalloc(index, dq, k, out)
                assert cnt == len(ref)
                assert np.array_equal(out[:cnt].cpu().numpy(), ref)
    index.close()


def test_noalloc_capacity_and_limits():
    torch = pytest.importorskip("torch")
    Q, P = datagen.make_problem(3000, 500, 16, 5)
    index = rmips.rmips_build_index(Q, P, k_max=10)
    q = (P[0] * 8.0).astype(np.float32)
    ref = rmips.rmips_query(index, q, 10)
    assert len(ref) > 2
    small = torch.full((len(ref) - 1,), -7, dtype=torch.int64, device="cuda")
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query_noalloc(index, q, 10, small)
    assert e.value.status == 5
    assert (small == -7).all()                      # nothing written on a capacity error
    out = torch.empty(len(ref), dtype=torch.int64, device="cuda")
    assert rmips.rmips_query_noalloc(index, q, 10, out) == len(ref)
    assert np.array_equal(out.cpu().numpy(), ref)
    index.close()
    # more users than the fixed scratch holds: a clear error, no work
    Qb, Pb = datagen.make_problem((1 << 20) + 1, 8, 4, 1)
    big = rmips.rmips_build_index(Qb, Pb, k_max=4)
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query_noalloc(big, Pb[0], 2, torch.empty(8, dtype=torch.int64, device="cuda"))
    assert e.value.status == 1
    big.close()
