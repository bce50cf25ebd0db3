"""Pins for the CPU oracle against what the paper and the mathematics fix.

Nothing here touches the CUDA library; all of it runs on the CPU.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import rmips_oracle as O
from paper_2110_07131_gb300 import datagen

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1.json")


def _fdot(u, x):
    """Exact rational inner product, written independently of the oracle."""
    acc = Fraction(0)
    for a, b in zip(u, x):
        acc += Fraction(float(a)) * Fraction(float(b))
    return acc


def _brute(Q, P, q, k):
    """All-rational brute force of Definition 2 (strict tie rule)."""
    res = []
    for i in range(Q.shape[0]):
        g = _fdot(Q[i], q)
        above = sum(1 for j in range(P.shape[0]) if _fdot(Q[i], P[j]) > g)
        if above < k:
            res.append(i)
    return res


@pytest.fixture(scope="module")
def table1():
    with open(GOLD) as f:
        g = json.load(f)
    Q = np.array([g["Q"][f"u{i}"] for i in range(1, 5)], dtype=np.float32)
    P = np.array([g["P"][f"p{i}"] for i in range(1, 6)], dtype=np.float32)
    return g, Q, P


def _names(ids, prefix):
    return [f"{prefix}{i + 1}" for i in ids]


# ---------------------------------------------------------------------------
# Table 1 / Example 1
# ---------------------------------------------------------------------------
def test_table1_inner_products_match_hand_table(table1):
    g, Q, P = table1
    S = Q.astype(np.float64) @ P.astype(np.float64).T
    for i in range(4):
        for j in range(5):
            assert S[i, j] == pytest.approx(g["hand_inner_products"][f"u{i+1}"][f"p{j+1}"], abs=1e-5)


def test_table1_printed_answers(table1):
    g, Q, P = table1
    # Example 1: q = p5 gives {u3, u4}; q = p1 gives nothing.
    assert _names(O.reverse_kmips(Q, P, P[4], 1), "u") == g["printed_results_k1"]["p5"]
    assert _names(O.reverse_kmips(Q, P, P[0], 1), "u") == g["printed_results_k1"]["p1"]


def test_table1_printed_p2_answer_conflicts_with_printed_vectors(table1):
    g, Q, P = table1
    # The printed MIPS column names p2 for u2, but the printed vectors give p3.
    assert _fdot(Q[1], P[2]) > _fdot(Q[1], P[1])
    assert g["printed_results_k1"]["p2"] == ["u2"]
    assert _names(O.reverse_kmips(Q, P, P[1], 1), "u") == []


@pytest.mark.parametrize("k", [1, 2, 3])
def test_table1_derived_answers(table1, k):
    g, Q, P = table1
    exp = g["derived_results"][f"k{k}"]
    for j in range(5):
        assert _names(O.reverse_kmips(Q, P, P[j], k), "u") == exp[f"p{j+1}"], (k, j)
        assert _names(_brute(Q, P, P[j], k), "u") == exp[f"p{j+1}"]


# ---------------------------------------------------------------------------
# Brute force on tiny inputs, exact ties, special cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_rational_brute_force_mf(seed):
    Q, P = datagen.make_problem(17, 13, 5, seed)
    qs = np.concatenate([P[:3], datagen.random_queries(2, 5, seed)])
    for q in qs:
        for k in (1, 2, 4, 13, 14):
            assert O.reverse_kmips(Q, P, q, k).tolist() == _brute(Q, P, q, k)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_matches_rational_brute_force_integer_ties(seed):
    Q, P = datagen.integer_problem(20, 15, 4, seed, lim=2)
    qs = np.concatenate([P[:4], np.zeros((1, 4), np.float32), Q[:2]])
    for q in qs:
        for k in (1, 2, 3, 7, 15, 16):
            assert O.reverse_kmips(Q, P, q, k).tolist() == _brute(Q, P, q, k)


def test_ties_are_exercised_by_integer_fixture():
    Q, P = datagen.integer_problem(20, 15, 4, 0, lim=2)
    S = Q @ P.T
    g = Q @ P[0]
    assert ((S == g[:, None]).sum(axis=1) >= 2).any()


def test_near_tie_needs_exact_fallback():
    # u.p and u.q differ by 2^-60 relative: invisible to a float64 dot.
    u = np.array([1.0, 1.0, 1.0], np.float32)
    q = np.array([1.0, 2.0 ** -30, -(2.0 ** -30)], np.float32)
    p = np.array([1.0, 2.0 ** -30, -(2.0 ** -30) + 2.0 ** -54], np.float32)
    assert float(p[2]) != float(q[2])
    P = np.stack([p, np.array([0.0, 0.0, 0.0], np.float32)])
    Q = u[None, :]
    exact = _fdot(u, p) > _fdot(u, q)
    assert O.counts_greater(Q, P, q)[0] == int(exact)


def test_k_at_least_m_returns_everyone():
    Q, P = datagen.make_problem(40, 9, 6, 5)
    every = list(range(40))
    assert O.reverse_kmips(Q, P, datagen.random_queries(1, 6, 1)[0], 10).tolist() == every
    # q in P: its own copy never counts, so k = m already returns everyone.
    assert O.reverse_kmips(Q, P, P[3], 9).tolist() == every


def test_zero_query_counts_positive_products():
    Q, P = datagen.integer_problem(30, 12, 5, 9, lim=2)
    q = np.zeros(5, np.float32)
    for k in (1, 3, 6):
        exp = [i for i in range(30) if sum(1 for j in range(12) if _fdot(Q[i], P[j]) > 0) < k]
        assert O.reverse_kmips(Q, P, q, k).tolist() == exp


def test_monotone_in_k():
    Q, P = datagen.make_problem(300, 120, 8, 3)
    for q in P[:5]:
        prev = set()
        for k in range(1, 30):
            cur = set(O.reverse_kmips(Q, P, q, k).tolist())
            assert prev <= cur
            prev = cur


@pytest.mark.parametrize("k", [1, 5, 10])
def test_sum_identity_over_all_items(k):
    # With no ties, each user has exactly k items whose top-k contains them.
    n, m = 400, 150
    Q, P = datagen.make_problem(n, m, 8, 7)
    res = O.reverse_kmips_multi(Q, P, P, k)
    assert sum(len(r) for r in res) == n * k


def test_permutation_and_power_of_two_scaling_invariance():
    Q, P = datagen.make_problem(200, 80, 6, 11)
    q = P[7]
    base = O.reverse_kmips(Q, P, q, 4)
    rng = np.random.default_rng(0)
    pq = rng.permutation(200)
    pp = rng.permutation(80)
    r = O.reverse_kmips(Q[pq], P[pp], q, 4)
    assert sorted(pq[r].tolist()) == base.tolist()
    # exact scaling by powers of two: items and query together, users alone
    assert O.reverse_kmips(Q, P * 4.0, q * 4.0, 4).tolist() == base.tolist()
    assert O.reverse_kmips(Q * 0.5, P, q, 4).tolist() == base.tolist()


def test_alternative_tie_reading_differs_only_on_ties():
    Q, P = datagen.make_problem(100, 40, 6, 2)
    q = P[5]
    assert (O.counts_greater(Q, P, q) ==
            O.counts_greater(Q, P, q, tie_rule="ge_excl", q_items=[5])).all()
    Qi, Pi = datagen.integer_problem(30, 20, 3, 4, lim=2)
    a = O.counts_greater(Qi, Pi, Pi[0])
    b = O.counts_greater(Qi, Pi, Pi[0], tie_rule="ge_excl", q_items=[0])
    assert (b >= a).all() and (b > a).any()


def test_decide_users_agrees_with_full_set():
    Q, P = datagen.make_problem(120, 50, 6, 8)
    q = P[2]
    full = set(O.reverse_kmips(Q, P, q, 3).tolist())
    users = np.array([0, 5, 17, 33, 90, 119])
    dec = O.decide_users(Q, P, q, 3, users)
    assert [bool(x) for x in dec] == [int(u) in full for u in users]


# ---------------------------------------------------------------------------
# Algorithm 1 (index) and the lemmas
# ---------------------------------------------------------------------------
def test_norm_order_matches_exact_squared_norms():
    Q, _ = datagen.make_problem(60, 1, 7, 4)
    sq = [sum(Fraction(float(x)) ** 2 for x in row) for row in Q]
    exp = sorted(range(60), key=lambda i: (-sq[i], i))
    assert O.norm_order(Q).tolist() == exp


def test_norm_order_ties_by_id():
    X = np.array([[1, 0], [0, 1], [0, 2], [-1, 0]], np.float32)
    assert O.norm_order(X).tolist() == [2, 0, 1, 3]


@pytest.mark.parametrize("p_prime", [None, 8, 3])
def test_index_lower_bound_arrays(p_prime):
    Q, P = datagen.make_problem(45, 20, 5, 6)
    k_max = 5
    ix = O.build_index(Q, P, k_max, p_prime=p_prime, block_size=8)
    Ps = P[ix["permP"]]
    pp = 20 if p_prime is None else p_prime
    for i, u in enumerate(Q[ix["permQ"]]):
        vals = sorted((_fdot(u, Ps[j]) for j in range(pp)), reverse=True)
        for j in range(k_max):
            if j < pp:
                assert ix["L"][i, j] == pytest.approx(float(vals[j]), abs=1e-12)
            else:
                assert ix["L"][i, j] == -np.inf
    # Equation 1: block arrays are the minima over the block, headers the first norm
    for b in range(ix["LB"].shape[0]):
        lo, hi = 8 * b, min(45, 8 * b + 8)
        assert (ix["LB"][b] == ix["L"][lo:hi].min(axis=0)).all()
        assert ix["hdr"][b] == ix["normQ"][lo] == ix["normQ"][lo:hi].max()


@pytest.mark.parametrize("seed", [0, 1])
def test_lemmas_are_sound(seed):
    n, m, d, k_max = 256, 100, 6, 6
    Q, P = datagen.make_problem(n, m, d, seed)
    ix = O.build_index(Q, P, k_max, p_prime=12, block_size=16)
    Qs, nQ, nP = ix["Qs"], ix["normQ"], ix["normP"]
    for q in np.concatenate([P[:6], datagen.random_queries(3, d, seed)]):
        nq = float(np.linalg.norm(q.astype(np.float64)))
        gam = Qs.astype(np.float64) @ q.astype(np.float64)
        for k in (1, 3, 6):
            truth = O.counts_greater(Qs, P, q) < k
            lem1 = gam < ix["L"][:, k - 1] - 1e-9
            assert not (lem1 & truth).any()                     # Lemma 1: no
            lem2 = gam > nQ * nP[k - 1] + 1e-9
            assert not (lem2 & ~truth).any()                    # Lemma 2: yes
            for b in range(ix["LB"].shape[0]):                  # Lemma 3: block no
                if ix["hdr"][b] * nq < ix["LB"][b, k - 1] - 1e-9:
                    assert not truth[16 * b:16 * b + 16].any()


@pytest.mark.parametrize("seed,p_prime,bs", [(0, None, 8), (1, 10, 4), (2, 3, 16), (3, 25, 5)])
def test_simpfer_equals_definition(seed, p_prime, bs):
    Q, P = datagen.make_problem(90, 40, 5, seed)
    ix = O.build_index(Q, P, 10, p_prime=p_prime, block_size=bs)
    qs = np.concatenate([P[:4], datagen.random_queries(2, 5, seed)])
    for q in qs:
        for k in (1, 4, 10):
            st = {}
            got = O.simpfer_query(ix, q, k, st)
            assert got.tolist() == O.reverse_kmips(Q, P, q, k).tolist()


def test_simpfer_on_integer_ties():
    Q, P = datagen.integer_problem(50, 18, 3, 1, lim=2)
    ix = O.build_index(Q, P, 6, p_prime=8, block_size=8)
    for q in P[:6]:
        for k in (1, 2, 6):
            assert O.simpfer_query(ix, q, k).tolist() == _brute(Q, P, q, k)


def test_linear_scan_reads_negative_products():
    # every product is negative: a threshold that starts at 0 would never move
    u = np.array([1.0, 0.0], np.float32)
    Ps = np.array([[-1.0, 0.0], [-2.0, 1.0], [-3.0, 0.0]], np.float32)
    nP = O.norms_fp64(Ps)
    order = np.argsort(-nP, kind="stable")
    q = np.array([-2.5, 0.0], np.float32)
    # products: -1, -2, -3 vs u.q = -2.5  -> two items above
    assert O.linear_scan(u, Ps[order], nP[order], q, 2) == 0
    assert O.linear_scan(u, Ps[order], nP[order], q, 3) == 1


# ---------------------------------------------------------------------------
# Definition 1 for every user (top-k MIPS join)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_topk_mips_matches_hand_table(table1, k):
    g, Q, P = table1
    hand = g["hand_inner_products"]
    got = O.topk_mips(Q, P, k)
    for i in range(4):
        row = hand[f"u{i + 1}"]
        want = sorted(row, key=lambda name: (-row[name], int(name[1:])))[:k]
        assert _names(got[i], "p") == want


def test_topk_mips_top1_is_the_printed_mips_column_except_u2(table1):
    g, Q, P = table1
    got = O.topk_mips(Q, P, 1)
    for i in range(4):
        name = f"u{i + 1}"
        if name == "u2":        # printed p2, but the printed vectors give p3 (10.00 > 9.85)
            assert _names(got[i], "p") == ["p3"]
        else:
            assert _names(got[i], "p") == [g["printed_mips_column"][name]]


def _brute_topk(Q, P, k):
    out = []
    for i in range(Q.shape[0]):
        vals = [(_fdot(Q[i], P[j]), j) for j in range(P.shape[0])]
        vals.sort(key=lambda t: (-t[0], t[1]))
        out.append([j for _, j in vals[:k]])
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_topk_mips_matches_rational_brute_force(seed):
    Q, P = datagen.make_problem(11, 17, 5, seed)
    Qi, Pi = datagen.integer_problem(9, 14, 4, seed, lim=2)        # many exact ties
    for A, B in ((Q, P), (Qi, Pi)):
        for k in (1, 3, 7, B.shape[0]):
            assert O.topk_mips(A, B, k).tolist() == _brute_topk(A, B, k)


def test_topk_mips_agrees_with_reverse_kmips_without_ties():
    """For tie-free data, p is in the top-k of u exactly when u is in R_k(p)."""
    Q, P = datagen.make_problem(40, 25, 6, 7)
    for k in (1, 4, 9):
        top = O.topk_mips(Q, P, k)
        for j in range(P.shape[0]):
            users = set(O.reverse_kmips(Q, P, P[j], k).tolist())
            assert users == {i for i in range(Q.shape[0]) if j in top[i]}


# ---------------------------------------------------------------------------
# kth_values: the j-th largest u.p (Definition 1's ranks, which Algorithm 1's
# lower-bound array L holds), against a rational sort written here
# ---------------------------------------------------------------------------
def _rational_kth(Q, P, k_max):
    """Exact j-th largest u.p per user (rational sort), None past |P|."""
    out = []
    for u in Q:
        vals = sorted((_fdot(u, p) for p in P), reverse=True)
        out.append([vals[j] if j < len(vals) else None for j in range(k_max)])
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_kth_values_integer_ties_are_exact(seed):
    # small-integer vectors: every float64 product sum is exact, and equal
    # products are frequent, so the j-th value must equal the rational one
    Q, P = datagen.integer_problem(12, 15, 6, seed, lim=2)
    got = O.kth_values(Q, P, 9)
    exp = _rational_kth(Q, P, 9)
    for i in range(Q.shape[0]):
        for j in range(9):
            assert Fraction(got[i, j]) == exp[i][j], (i, j)
    # the ranks are descending and ties repeat the same value
    assert np.all(np.diff(got, axis=1) <= 0)
    assert any(got[i, j] == got[i, j + 1] for i in range(12) for j in range(8))


@pytest.mark.parametrize("seed", [2, 3])
def test_kth_values_mf_within_float64_bound(seed):
    Q, P = datagen.make_problem(10, 40, 50, seed)
    k_max = 25
    got = O.kth_values(Q, P, k_max)
    exp = _rational_kth(Q, P, k_max)
    d = Q.shape[1]
    gam = d * 2.0 ** -53 / (1 - d * 2.0 ** -53)
    for i in range(Q.shape[0]):
        # a float64 sum of exact float32 products is within gam * sum|u_i p_i|
        # of the exact value, so each order statistic moves by at most the
        # largest such error over the items
        tol = gam * float(np.max(np.abs(Q[i].astype(np.float64)) @ np.abs(P.astype(np.float64)).T))
        for j in range(k_max):
            assert abs(Fraction(got[i, j]) - exp[i][j]) <= Fraction(tol), (i, j)
    # an off-by-one in the rank would move every entry by a whole gap
    gaps = [float(exp[0][j] - exp[0][j + 1]) for j in range(k_max - 1)]
    assert min(gaps) > 1e3 * gam


def test_kth_values_pad_with_minus_inf_past_the_item_count():
    Q, P = datagen.make_problem(6, 4, 8, 5)
    got = O.kth_values(Q, P, 7)
    exp = _rational_kth(Q, P, 7)
    assert got.shape == (6, 7)
    assert np.all(np.isneginf(got[:, 4:]))
    for i in range(6):
        for j in range(4):
            assert abs(Fraction(got[i, j]) - exp[i][j]) < Fraction(1, 10 ** 9)


# ---------------------------------------------------------------------------
# decide_users_multi (the k-th-largest form of Definition 2, many queries)
# against the counting form
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("chunk", [7, 512])
def test_decide_users_multi_equals_counting_mf(chunk):
    Q, P = datagen.make_problem(600, 300, 50, 4)
    qs, _ = datagen.queries_from_items(P, 8, 4)
    qs = np.concatenate([qs, datagen.random_queries(3, 50, 4), np.zeros((1, 50), np.float32)])
    counts = O.counts_greater_multi(Q, P, qs)
    users = np.random.default_rng(0).choice(600, 250, replace=False)
    for ks in (1, 10, 25, np.arange(1, 13)):
        kk = np.broadcast_to(np.asarray(ks), (len(qs),))
        got = O.decide_users_multi(Q, P, qs, kk, users, threads=3, chunk=chunk)
        exp = counts[:, users] < kk[:, None]
        assert np.array_equal(got, exp), ks


@pytest.mark.parametrize("seed", [0, 1])
def test_decide_users_multi_equals_counting_integer_ties(seed):
    # many exact ties at the k-th value: the exact band path decides them
    Q, P = datagen.integer_problem(200, 60, 4, seed, lim=2)
    qs = np.concatenate([P[:10], Q[:3]])
    counts = O.counts_greater_multi(Q, P, qs)
    users = np.arange(200)
    for k in (1, 2, 5, 12, 60, 61):
        got = O.decide_users_multi(Q, P, qs, k, users, threads=2, chunk=64)
        assert np.array_equal(got, counts < k), k
