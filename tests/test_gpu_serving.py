"""Serving loop: each request's result is the same alone and in the mix."""
import threading

import numpy as np
import pytest

from oracle import rmips_oracle as O
from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    Q, P = datagen.make_problem(3000, 1500, 50, 9)
    index = rmips.rmips_build_index(Q, P, k_max=25)
    yield Q, P, index
    index.close()


def _requests(P, n_req, seed):
    rng = np.random.default_rng(seed)
    qs, _ = datagen.queries_from_items(P, n_req, seed)
    ks = rng.integers(1, 26, n_req)
    segs = []
    for j in range(n_req):
        r = j % 4
        if r == 1:
            a = int(rng.integers(0, 3000))
            segs.append((a, a + int(rng.integers(1, 3000))))      # uneven id ranges
        elif r == 2:
            segs.append(np.sort(rng.choice(3000, int(rng.integers(1, 2000)), replace=False)))
        else:
            segs.append(None)
    return qs, ks, segs


def test_results_identical_alone_and_in_the_mix(setup):
    Q, P, index = setup
    qs, ks, segs = _requests(P, 600, 1)
    alone = [rmips.rmips_query(index, qs[j], int(ks[j]), segment=segs[j]) for j in range(len(qs))]
    srv = rmips.Server(index, max_batch=64, max_wait_us=300, streams=3)
    got = [None] * len(qs)
    errs = []

    def client(lo, hi):
        try:
            tickets = [(j, srv.submit(qs[j], int(ks[j]), segs[j])) for j in range(lo, hi)]
            for j, t in tickets:
                got[j], lat = srv.wait(t)
                assert lat >= 0.0
        except Exception as e:                # surfaced below
            errs.append(e)

    threads = [threading.Thread(target=client, args=(i * 150, (i + 1) * 150)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errs, errs
    for j in range(len(qs)):
        assert np.array_equal(got[j], alone[j]), j
    st = srv.stats()
    assert st["completed"] == len(qs) and st["pending"] == 0
    assert st["batches"] >= 1 and st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    srv.close()


def test_batched_requests_match_oracle(setup):
    Q, P, index = setup
    qs, ks, _ = _requests(P, 200, 2)
    srv = rmips.Server(index, max_batch=128, max_wait_us=1000, streams=2)
    tickets = srv.submit_many(qs, ks.astype(np.int32))
    counts = O.counts_greater_multi(Q, P, qs)
    for j, t in enumerate(tickets[:100]):
        ids, _ = srv.wait(int(t))
        assert np.array_equal(ids, np.nonzero(counts[j] < ks[j])[0])
    ids, offs, lat = srv.wait_many(tickets[100:])
    for j in range(100, 200):
        assert np.array_equal(ids[offs[j - 100]:offs[j - 99]], np.nonzero(counts[j] < ks[j])[0])
    assert (lat >= 0).all()
    srv.close()


def test_admission_and_bad_requests_do_not_stop_the_loop(setup):
    Q, P, index = setup
    srv = rmips.Server(index, max_batch=32, max_wait_us=100000, streams=1, max_pending=8)
    with pytest.raises(rmips.RmipsError) as e:
        srv.submit_many(P[:20], 5)
    assert e.value.status == 9                    # admission refused, nothing queued
    with pytest.raises(rmips.RmipsError) as e:
        srv.submit(P[0], 0)
    assert e.value.status == 2
    bad = P[1].copy()
    bad[4] = np.inf
    with pytest.raises(rmips.RmipsError) as e:
        srv.submit(bad, 3)
    assert e.value.status == 3
    t = srv.submit(P[2], 7)
    try:                                          # a poll: finished or not yet, never another error
        ids, _ = srv.wait(t, timeout_ms=0)
    except rmips.RmipsError as e:
        assert e.status == 6
        ids, _ = srv.wait(t)
    assert np.array_equal(ids, rmips.rmips_query(index, P[2], 7))
    st = srv.stats()
    assert st["rejected"] == 20 and st["completed"] == 1
    srv.close()


def test_small_result_budget_falls_back_per_request(setup):
    Q, P, index = setup
    qs, ks, _ = _requests(P, 40, 3)
    # a result buffer of 64 ids, with reservations of one id per request: the
    # 40 requests are admitted, but their batches hold more results than the
    # buffer and are re-run request by request
    srv = rmips.Server(index, max_batch=40, max_wait_us=2000, streams=1, max_device_bytes=64 * 8,
                       result_ids_per_request=1)
    tickets = srv.submit_many(qs, ks.astype(np.int32))
    for j, t in enumerate(tickets):
        ids, _ = srv.wait(int(t))
        assert np.array_equal(ids, rmips.rmips_query(index, qs[j], int(ks[j])))
    assert srv.stats()["batches_one_by_one"] >= 1
    with pytest.raises(rmips.RmipsError) as e:
        srv.wait(12345678)
    assert e.value.status == 1
    srv.close()


def test_fp16_out_of_range_request_is_refused_alone():
    # On an FP16 index a query value beyond 65504 has no FP16 copy.  The
    # server refuses that request at submission, so the requests it would
    # have been batched with still complete with their exact answers.
    Q, P = datagen.make_problem(2000, 1000, 50, 11)
    index = rmips.rmips_build_index(Q, P, k_max=25, precision="fp16")
    srv = rmips.Server(index, max_batch=64, max_wait_us=20000, streams=1)
    qs, _ = datagen.queries_from_items(P, 12, 11)
    good = [srv.submit(qs[j], 10) for j in range(6)]
    bad = qs[6].copy()
    bad[3] = np.float32(70000.0)
    with pytest.raises(rmips.RmipsError) as e:
        srv.submit(bad, 10)
    assert e.value.status == 3
    with pytest.raises(rmips.RmipsError) as e:           # all or none: nothing of this call is queued
        srv.submit_many(np.stack([qs[7], bad]), 10)
    assert e.value.status == 3
    good += [srv.submit(qs[j], 10) for j in range(8, 12)]
    counts = O.counts_greater_multi(Q, P, np.concatenate([qs[:6], qs[8:12]]))
    for j, t in enumerate(good):
        ids, _ = srv.wait(t)
        assert np.array_equal(ids, np.nonzero(counts[j] < 10)[0]), j
    st = srv.stats()
    assert st["completed"] == 10 and st["pending"] == 0
    srv.close()
    index.close()


def test_registered_segments_and_id_lists_are_answered_in_the_batch(setup):
    Q, P, index = setup
    rng = np.random.default_rng(21)
    srv = rmips.Server(index, max_batch=256, max_wait_us=3000, streams=2)
    subsets = [np.sort(rng.choice(3000, s, replace=False)) for s in (5, 700, 2999)]
    handles = [srv.add_segment(np.concatenate([x, x[:3]])) for x in subsets]   # duplicates are dropped
    qs, ks, _ = _requests(P, 90, 22)
    segs = [("registered", handles[j % 3]) if j % 2 == 0 else subsets[j % 3] for j in range(len(qs))]
    tickets = srv.submit_many(qs, ks.astype(np.int32), segs)
    ids, offs, _ = srv.wait_many(tickets)
    for j in range(len(qs)):
        alone = rmips.rmips_query(index, qs[j], int(ks[j]), segment=subsets[j % 3])
        assert np.array_equal(ids[offs[j]:offs[j + 1]], alone), j
    st = srv.stats()
    assert st["batches"] <= 3 and st["batches_one_by_one"] == 0     # no single-query detour
    with pytest.raises(rmips.RmipsError) as e:
        srv.submit(qs[0], 5, ("registered", 17))
    assert e.value.status == 1
    srv.close()


def test_admission_by_result_memory(setup):
    Q, P, index = setup
    # one stream, a result buffer of 200 ids, 50 ids reserved per request:
    # at most four requests can be queued or running at once
    srv = rmips.Server(index, max_batch=64, max_wait_us=200000, streams=1, max_device_bytes=200 * 8,
                       result_ids_per_request=50)
    st = srv.stats()
    assert st["reservable_ids"] == 200
    t4 = srv.submit_many(P[:4], 10)
    assert srv.stats()["reserved_ids"] == 200
    with pytest.raises(rmips.RmipsError) as e:
        srv.submit(P[4], 10)
    assert e.value.status == 9
    # a request whose segment is smaller reserves less
    small = srv.stats()
    ids, offs, _ = srv.wait_many(t4)
    for j in range(4):
        assert np.array_equal(ids[offs[j]:offs[j + 1]], rmips.rmips_query(index, P[j], 10))
    assert srv.stats()["reserved_ids"] == 0
    t = srv.submit(P[5], 10, segment=(0, 20))               # 20 users: reserves 20 ids
    assert srv.stats()["reserved_ids"] == 20
    got, _ = srv.wait(t)
    assert np.array_equal(got, rmips.rmips_query(index, P[5], 10, segment=(0, 20)))
    assert small["rejected"] == 1
    srv.close()


def test_small_batches_run_as_single_launches(setup):
    # every batch of up to 64 requests goes through the one-launch kernel on
    # the slot's stream; segments of every kind, mixed k: the same results
    Q, P, index = setup
    srv = rmips.Server(index, max_batch=64, max_wait_us=500, streams=2, single_max=64)
    qs, ks, segs = _requests(P, 160, 31)
    h = srv.add_segment(np.arange(0, 3000, 3))
    segs = [("registered", h) if j % 5 == 4 else sg for j, sg in enumerate(segs)]
    tickets = [srv.submit(qs[j], int(ks[j]), segs[j]) for j in range(len(qs))]
    for j, t in enumerate(tickets):
        ids, _ = srv.wait(t)
        sg = np.arange(0, 3000, 3) if j % 5 == 4 else segs[j]
        assert np.array_equal(ids, rmips.rmips_query(index, qs[j], int(ks[j]), segment=sg)), j
    st = srv.stats()
    assert st["completed"] == len(qs) and st["batches_one_by_one"] == 0
    srv.close()


def test_spinning_server_and_greedy_dispatch_give_the_same_results(setup):
    # spin_us polls instead of blocking; max_wait_us = 0 closes a batch as
    # soon as a stream slot is free: the answers are the same
    Q, P, index = setup
    qs, ks, segs = _requests(P, 120, 41)
    srv = rmips.Server(index, max_batch=64, max_wait_us=0, streams=2, spin_us=300)
    tickets = [srv.submit(qs[j], int(ks[j]), segs[j]) for j in range(len(qs))]
    for j, t in enumerate(tickets):
        ids, _ = srv.wait(t)
        assert np.array_equal(ids, rmips.rmips_query(index, qs[j], int(ks[j]), segment=segs[j])), j
    more = srv.submit_many(qs[:40], ks[:40].astype(np.int32))
    ids, offs, _ = srv.wait_many(more)
    for j in range(40):
        assert np.array_equal(ids[offs[j]:offs[j + 1]], rmips.rmips_query(index, qs[j], int(ks[j])))
    with pytest.raises(rmips.RmipsError) as e:
        rmips.Server(index, spin_us=-1)
    assert e.value.status == 1
    srv.close()
