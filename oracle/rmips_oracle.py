"""CPU oracle for exact reverse k-MIPS -- test infrastructure, not product code.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` import this module.  It shares no code with the CUDA library and
never calls it.

What it computes (Definition 2 of the paper, "Reverse k-MIPS problem"): for a
query item q, the users u of Q whose k-MIPS result over ``P + {q}`` contains q.
The rule for ties between q and an item (Definition 2 does not fix it) is the
one this package uses throughout: q is kept in u's top-k unless at least k items
of P have an inner product with u that is *strictly* larger than ``u.q``::

    c(u) = #{ p in P : u.p > u.q },     u in R(q, k)  <=>  c(u) < k

This is the only reading under which the worked example of Table 1 holds with
``q = p5`` (q's own copy in P ties with q and must not push q out).

Arithmetic: every inner product of two float32 vectors is formed in float64
(each product of two float32 numbers is exact in float64).  Whenever a float64
comparison is within its rounding-error bound, the comparison is redone in exact
rational arithmetic (``fractions.Fraction``), so the returned sets are those of
exact arithmetic on the float32 inputs.

``topk_mips`` is Definition 1 itself (the k-MIPS of every user, the join
that the index's candidates come from).

Parity pins (see ``tests/test_oracle.py``): the printed vectors of Table 1,
an all-``Fraction`` brute force on tiny inputs, integer fixtures with exact ties,
monotonicity in k, the identity ``sum_{q in P} |R_k(q)| = n k`` for tie-free
data, the k >= m and q = 0 special cases, and soundness of every pruning lemma.
``simpfer_query`` (Algorithm 3 with Algorithm 2) is pinned by equality with the
definition.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

__all__ = [
    "norms_fp64", "norm_order", "exact_dot", "exact_sign_diff",
    "counts_greater", "counts_greater_multi", "reverse_kmips", "reverse_kmips_multi",
    "decide_users", "decide_users_multi", "build_index", "linear_scan", "simpfer_query", "kth_values",
    "topk_mips",
]

_U64 = 2.0 ** -53


# ---------------------------------------------------------------------------
# Norms and the norm order of Algorithm 1 (pre-processing, steps 1-2)
# ---------------------------------------------------------------------------
def norms_fp64(X: np.ndarray) -> np.ndarray:
    """Euclidean norm of every row, float64, squares summed in index order.

    Algorithm 1 first computes ``||u_i||`` for every user and ``||p_j||`` for
    every item.  Each square of a float32 is exact in float64; the running sum
    is rounded once per dimension, in the order 0, 1, ..., d-1.
    """
    X64 = np.asarray(X, dtype=np.float64)
    acc = np.zeros(X64.shape[0], dtype=np.float64)
    for i in range(X64.shape[1]):
        acc = acc + X64[:, i] * X64[:, i]
    return np.sqrt(acc)


def norm_order(X: np.ndarray) -> np.ndarray:
    """Row ids in descending order of ``norms_fp64`` (ties: ascending id).

    Algorithm 1 sorts Q and P in descending order of norm; the paper does not
    say how equal norms are ordered, so the lower row id goes first.
    """
    nrm = norms_fp64(X)
    ids = np.arange(X.shape[0])
    return np.lexsort((ids, -nrm)).astype(np.int64)


# ---------------------------------------------------------------------------
# Exact rational arithmetic for near-ties
# ---------------------------------------------------------------------------
def exact_dot(u, x) -> Fraction:
    """``u . x`` as an exact rational number (float32 inputs are exact)."""
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, x)), Fraction(0))


def exact_sign_diff(u, a, b) -> int:
    """Sign of ``u.a - u.b`` in exact arithmetic: -1, 0 or +1.

    When a and b hold the same values, ``u.a - u.b`` is exactly zero (this is
    the tie between a query and its own copy in P), so no rational arithmetic
    is needed.
    """
    if np.array_equal(np.asarray(a, dtype=np.float32), np.asarray(b, dtype=np.float32)):
        return 0
    diff = exact_dot(u, a) - exact_dot(u, b)
    return (diff > 0) - (diff < 0)


def _fp64_bound(d: int) -> float:
    """Bound factor for a float64 difference of two length-d dot products.

    A float64 dot product of float32 vectors has error at most
    ``gamma_d * sum|u_i x_i|`` (Higham, Accuracy and Stability of Numerical
    Algorithms, Sec. 3.1) in any summation order; the difference adds one more
    rounding.  A factor 4 over ``(d + 2) u`` covers the computed (not exact)
    absolute sums and the subtraction.
    """
    return 4.0 * (d + 2) * _U64


# ---------------------------------------------------------------------------
# The definition: c(u) = #{p : u.p > u.q}
# ---------------------------------------------------------------------------
def counts_greater_multi(Q: np.ndarray, P: np.ndarray, qs: np.ndarray,
                         tie_rule: str = "strict", q_items=None,
                         chunk_elems: int = 1 << 24) -> np.ndarray:
    """``c[j, u] = #{p in P : u.p > u.q_j}`` in exact arithmetic, for every query.

    ``tie_rule="strict"`` is Definition 2 under the strict reading (the one
    this package implements).  ``tie_rule="ge_excl"`` is the alternative
    reading that counts ``u.p >= u.q`` but skips q's own row of P
    (``q_items[j]``, or -1 when q is not an item).  Inputs are float32.
    """
    Q = np.asarray(Q, dtype=np.float32)
    P = np.asarray(P, dtype=np.float32)
    qs = np.atleast_2d(np.asarray(qs, dtype=np.float32))
    Q64, P64, qs64 = (x.astype(np.float64) for x in (Q, P, qs))
    n, d = Q64.shape
    m = P64.shape[0]
    nq = qs64.shape[0]
    if q_items is None:
        q_items = [-1] * nq
    G = _fp64_bound(d)
    gam = Q64 @ qs64.T                         # [n, nq]   u.q
    agam = np.abs(Q64) @ np.abs(qs64).T        # [n, nq]   sum |u_i q_i|
    counts = np.zeros((nq, n), dtype=np.int64)
    step = max(1, chunk_elems // max(1, n))
    for p0 in range(0, m, step):
        p1 = min(m, p0 + step)
        S = Q64 @ P64[p0:p1].T                 # [n, mc]   u.p
        A = np.abs(Q64) @ np.abs(P64[p0:p1]).T
        for j in range(nq):
            diff = S - gam[:, j:j + 1]
            bound = G * (A + agam[:, j:j + 1])
            # clear of the bound: the float64 sign is the exact sign
            counts[j] += (diff > bound).sum(axis=1)
            near_u, near_p = np.nonzero(np.abs(diff) <= bound)
            for u, pc in zip(near_u.tolist(), near_p.tolist()):
                p = p0 + pc
                if tie_rule == "ge_excl" and p == q_items[j]:
                    continue
                s = exact_sign_diff(Q[u], P[p], qs[j])
                if s > 0 or (tie_rule == "ge_excl" and s == 0):
                    counts[j, u] += 1
    return counts


def counts_greater(Q, P, q, **kw) -> np.ndarray:
    """``c(u)`` for every user and one query q."""
    return counts_greater_multi(Q, P, np.atleast_2d(q), **kw)[0]


def reverse_kmips(Q, P, q, k: int, **kw) -> np.ndarray:
    """Definition 2: ascending ids of users whose top-k over ``P + {q}`` holds q."""
    c = counts_greater(Q, P, q, **kw)
    return np.nonzero(c < k)[0].astype(np.int64)


def reverse_kmips_multi(Q, P, qs, ks, **kw) -> list:
    """``reverse_kmips`` for many queries (one matrix product over P)."""
    c = counts_greater_multi(Q, P, qs, **kw)
    ks = np.broadcast_to(np.asarray(ks), (c.shape[0],))
    return [np.nonzero(c[j] < ks[j])[0].astype(np.int64) for j in range(c.shape[0])]


def decide_users(Q, P, q, k: int, users) -> np.ndarray:
    """Yes/no of Definition 2 for the listed users only (for sampled checks)."""
    users = np.asarray(users, dtype=np.int64)
    c = counts_greater(np.asarray(Q)[users], P, q)
    return c < k


def decide_users_multi(Q, P, qs, ks, users, threads: int = 8, chunk: int = 512) -> np.ndarray:
    """Yes/no of Definition 2 for every (query j, listed user), many queries at once.

    Uses the identity ``c(u) < k  <=>  v_k(u) <= u.q`` where ``v_k(u)`` is the
    k-th largest ``u.p`` over P (counted with multiplicity): if the k-th
    largest product is at most ``u.q``, only the k-1 above it can be strictly
    above ``u.q``; if it is larger, the k largest all are.  Each listed user's
    products with all of P are formed once in float64 and its K = max(ks)
    largest are kept, so every query is decided from them:

    * ``t_k > u.q + E`` (E covers the float64 error of both sides): no;
    * ``t_k < u.q - E``: yes;
    * otherwise the items whose product may reach ``u.q`` are compared with q
      exactly (rational arithmetic), reading the user's whole row again when
      they do not all lie among the K kept.

    Returns a bool array ``[len(qs), len(users)]``.
    """
    from concurrent.futures import ThreadPoolExecutor
    Q = np.asarray(Q, dtype=np.float32)
    P = np.asarray(P, dtype=np.float32)
    qs = np.atleast_2d(np.asarray(qs, dtype=np.float32))
    users = np.asarray(users, dtype=np.int64)
    nq, m, d = qs.shape[0], P.shape[0], P.shape[1]
    ks = np.broadcast_to(np.asarray(ks, dtype=np.int64), (nq,))
    K = int(min(m, ks.max()))
    P64 = P.astype(np.float64)
    q64 = qs.astype(np.float64)
    G = _fp64_bound(d)
    pmax = float(norms_fp64(P).max()) * (1 + 1e-12)
    out = np.zeros((nq, users.shape[0]), dtype=bool)

    def top(rows):
        S = rows @ P64.T                                  # [r, m]
        if K >= m:
            idx = np.broadcast_to(np.arange(m), S.shape)
        else:
            idx = np.argpartition(S, m - K, axis=1)[:, m - K:]
        val = np.take_along_axis(S, idx, axis=1)
        order = np.argsort(-val, axis=1, kind="stable")
        return np.take_along_axis(val, order, axis=1), np.take_along_axis(np.asarray(idx), order, axis=1)

    with ThreadPoolExecutor(max(1, threads)) as ex:
        for c0 in range(0, users.shape[0], chunk):
            ids = users[c0:c0 + chunk]
            U = Q[ids]
            U64 = U.astype(np.float64)
            parts = np.array_split(np.arange(ids.shape[0]), max(1, min(threads, ids.shape[0])))
            res = list(ex.map(lambda r: top(U64[r]), parts))
            tv = np.concatenate([r[0] for r in res])      # [r, K] descending float64 products
            ti = np.concatenate([r[1] for r in res])      # their items
            gam = U64 @ q64.T                             # [r, nq] u.q
            agam = np.abs(U64) @ np.abs(q64).T
            unorm = norms_fp64(U) * (1 + 1e-12)
            for j in range(nq):
                k = int(ks[j])
                if k > m:                                 # fewer than k items exist: always yes
                    out[j, c0:c0 + ids.shape[0]] = True
                    continue
                E = G * (agam[:, j] + unorm * pmax)       # float64 error of u.q plus that of any u.p
                tk = tv[:, k - 1]
                no = tk > gam[:, j] + E
                yes = tk < gam[:, j] - E
                out[j, c0:c0 + ids.shape[0]] = yes
                for r in np.nonzero(~(no | yes))[0].tolist():
                    lo = gam[r, j] - E[r]
                    if K < m and tv[r, K - 1] >= lo:      # the band reaches past the kept items
                        row = P64 @ U64[r]
                        cand = np.nonzero(row >= lo)[0]
                    else:
                        cand = ti[r][tv[r] >= lo]
                    above = sum(1 for p in cand.tolist() if exact_sign_diff(U[r], P[p], qs[j]) > 0)
                    out[j, c0 + r] = above < k
    return out


def kth_values(Q, P, k_max: int) -> np.ndarray:
    """``v[i, j-1]`` = the j-th largest ``u_i . p`` over P (float64), j = 1..k_max.

    Entries past |P| are ``-inf``.
    """
    Q64 = np.asarray(Q, dtype=np.float64)
    P64 = np.asarray(P, dtype=np.float64)
    S = Q64 @ P64.T
    kk = min(k_max, S.shape[1])
    part = -np.sort(-S, axis=1)[:, :kk]
    out = np.full((Q64.shape[0], k_max), -np.inf)
    out[:, :kk] = part
    return out


def topk_mips(Q, P, k: int) -> np.ndarray:
    """Definition 1 (k-MIPS) for every user: ``out[i]`` holds the ids of the k
    items with the largest ``u_i . p``, in descending order of ``u_i . p``;
    equal products are ordered by ascending item id.  Exact: items whose
    float64 products lie within the float64 error bound of the k-th largest
    are ordered in rational arithmetic.  k <= |P|.
    """
    Q = np.asarray(Q, dtype=np.float32)
    P = np.asarray(P, dtype=np.float32)
    n, m = Q.shape[0], P.shape[0]
    Q64, P64 = Q.astype(np.float64), P.astype(np.float64)
    S = Q64 @ P64.T
    A = np.abs(Q64) @ np.abs(P64).T
    f = _fp64_bound(Q.shape[1])
    out = np.empty((n, k), dtype=np.int64)
    for i in range(n):
        order = np.lexsort((np.arange(m), -S[i]))
        kth = S[i, order[k - 1]]
        slack = f * A[i].max()
        near = np.nonzero(S[i] >= kth - 2 * slack)[0]      # every item that may rank in the top k
        exact = {int(j): exact_dot(Q[i], P[j]) for j in near}
        ranked = sorted(exact, key=lambda j: (-exact[j], j))
        out[i] = ranked[:k]
    return out


# ---------------------------------------------------------------------------
# Algorithm 1: the lower-bound arrays and the blocks
# ---------------------------------------------------------------------------
def build_index(Q, P, k_max: int, p_prime=None, block_size: int = 32) -> dict:
    """Algorithm 1 (pre-processing), in float64.

    1. norms of every user and item, 2. both sets sorted by descending norm,
    3. ``P'`` = the first ``p_prime`` sorted items (all of P when None),
    4. ``L_i^j`` = the j-th largest ``u_i . p`` over ``P'`` (``-inf`` when
       ``|P'| < j``), 5. blocks of ``block_size`` consecutive sorted users with
    ``L^j(B) = min_{u_i in B} L_i^j`` (Equation 1).  Positions are 0-based.
    """
    Q = np.asarray(Q, dtype=np.float32)
    P = np.asarray(P, dtype=np.float32)
    n, m = Q.shape[0], P.shape[0]
    permQ = norm_order(Q)
    permP = norm_order(P)
    Qs, Ps = Q[permQ], P[permP]
    nQ, nP = norms_fp64(Qs), norms_fp64(Ps)
    pp = m if p_prime is None else min(int(p_prime), m)
    Pp = Ps[:pp].astype(np.float64)
    S = Qs.astype(np.float64) @ Pp.T
    kk = min(k_max, pp)
    order = np.argsort(-S, axis=1, kind="stable")[:, :kk]
    L = np.full((n, k_max), -np.inf)
    L_item = np.full((n, k_max), -1, dtype=np.int64)
    L[:, :kk] = np.take_along_axis(S, order, axis=1)
    L_item[:, :kk] = order
    nb = (n + block_size - 1) // block_size
    LB = np.empty((nb, k_max))
    hdr = np.empty(nb)
    for b in range(nb):
        lo, hi = b * block_size, min(n, (b + 1) * block_size)
        LB[b] = L[lo:hi].min(axis=0)
        hdr[b] = nQ[lo]
    return dict(permQ=permQ, permP=permP, Qs=Qs, Ps=Ps, normQ=nQ, normP=nP, L=L,
                L_item=L_item, LB=LB, hdr=hdr, block_size=block_size, p_prime=pp,
                k_max=k_max)


# ---------------------------------------------------------------------------
# Algorithms 2 and 3 (online phase), restated for the strict tie rule
# ---------------------------------------------------------------------------
def _cmp(u, a, b, bound_scale: float) -> int:
    """Sign of ``u.a - u.b``: float64 when clear of its error bound, else exact."""
    u64 = u.astype(np.float64)
    diff = float(u64 @ a.astype(np.float64) - u64 @ b.astype(np.float64))
    bound = bound_scale * float(np.abs(u64) @ (np.abs(a.astype(np.float64)) + np.abs(b.astype(np.float64))))
    if diff > bound:
        return 1
    if diff < -bound:
        return -1
    return exact_sign_diff(u, a, b)


def linear_scan(u: np.ndarray, Ps: np.ndarray, normP: np.ndarray, q: np.ndarray, k: int) -> int:
    """Algorithm 2 (Linear-scan) for one user: 1 = yes, 0 = no.

    Items are visited in descending norm.  Corollary 1: once
    ``||u|| ||p_j|| <= u.q`` no later item can beat q, so the answer is yes.
    Corollary 2: once k items are strictly above ``u.q`` the answer is no.
    Readings that differ from the printed algorithm: the running threshold
    starts at minus infinity (the printed 0 would ignore negative products),
    and reaching the end of P means yes (the printed algorithm has no final
    return).  The norm test is made with a relative margin so that the
    irrational ``||u|| ||p_j||`` never decides a true tie the wrong way.
    """
    d = u.shape[0]
    G = _fp64_bound(d)
    u64 = u.astype(np.float64)
    gamma = float(u64 @ q.astype(np.float64))
    gamma_lo = gamma - G * float(np.abs(u64) @ np.abs(q.astype(np.float64)))
    nu = float(np.sqrt(u64 @ u64))
    above = 0
    for j in range(Ps.shape[0]):
        if gamma_lo >= nu * normP[j] * (1.0 + 8 * (d + 2) * _U64):        # Corollary 1
            return 1
        if _cmp(u, Ps[j], q, G) > 0:
            above += 1
            if above >= k:                                             # Corollary 2
                return 0
    return 1


def simpfer_query(index: dict, q: np.ndarray, k: int, stats: dict | None = None) -> np.ndarray:
    """Algorithm 3 (Simpfer) on an index from ``build_index``; returns ascending original ids.

    For each block: Lemma 3 prunes the block when ``||u_first|| ||q|| < L^k(B)``;
    for each remaining user, Lemma 1 answers no when ``u.q < L_i^k``, Lemma 2
    answers yes when ``u.q >= ||u|| ||p_k||``, and Algorithm 2 decides the rest.
    Under the strict tie rule a user with ``u.q = L_i^k`` can still be a yes, so
    Lemmas 1 and 3 prune only on strict inequality.  Tests of ``u.q`` against
    an ``L`` entry are made exactly (``L_i^k`` is ``u.p`` for a known item p);
    tests against a product of norms carry a relative margin.
    """
    Qs, Ps = index["Qs"], index["Ps"]
    nQ, nP = index["normQ"], index["normP"]
    L, L_item, LB, hdr = index["L"], index["L_item"], index["LB"], index["hdr"]
    b = index["block_size"]
    n, d = Qs.shape
    G = _fp64_bound(d)
    marg = 8 * (d + 2) * _U64
    q = np.asarray(q, dtype=np.float32)
    q64 = q.astype(np.float64)
    nq = float(np.sqrt(q64 @ q64))
    k_max = L.shape[1]
    if not 1 <= k <= k_max:
        raise ValueError("k must be in [1, k_max]")
    st = dict(blocks_pruned=0, lemma1_no=0, lemma2_yes=0, scanned=0)
    out = []
    for blk in range(LB.shape[0]):
        if hdr[blk] * nq * (1.0 + marg) < LB[blk, k - 1]:              # Lemma 3 (strict)
            st["blocks_pruned"] += 1
            continue
        for i in range(blk * b, min(n, (blk + 1) * b)):
            u = Qs[i]
            it = L_item[i, k - 1]
            if it >= 0 and _cmp(u, q, Ps[it], G) < 0:                  # Lemma 1 (strict)
                st["lemma1_no"] += 1
                continue
            u64 = u.astype(np.float64)
            gamma_lo = float(u64 @ q64) - G * float(np.abs(u64) @ np.abs(q64))
            pk = nP[k - 1] if k - 1 < nP.shape[0] else 0.0
            if gamma_lo >= nQ[i] * pk * (1.0 + marg):                    # Lemma 2
                st["lemma2_yes"] += 1
                out.append(i)
                continue
            st["scanned"] += 1
            if linear_scan(u, Ps, nP, q, k):
                out.append(i)
    if stats is not None:
        stats.update(st)
    return np.sort(index["permQ"][np.asarray(out, dtype=np.int64)]) if out else np.zeros(0, np.int64)
