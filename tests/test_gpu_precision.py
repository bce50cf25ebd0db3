"""The precision workload at its stated size: |Q| = 500k, |P| = 100k, d = 64,
k = 10, 2,000 queries drawn from P plus 2,000 random N(0, I/d) queries, with
the filter's products in TF32 (float32 index), BF16 and FP16 on tensor cores,
FP32 accumulation and the exact recheck of every pair within the error bound.

Every one of the 4,000 result sets is compared, whole, with the CPU Simpfer
(float64 with exact tie decisions, pinned to the definition), and the largest
error of the tensor-core inner products against float64 is measured on tiles
of the workload's own users and queries."""
import numpy as np
import pytest

from oracle import simpfer_cpu as S
from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu

N, M, D, K, KMAX, SEED = 500_000, 100_000, 64, 10, 25, 2
BOUND = {"tf32": 0.00198, "bf16": 0.00788, "fp16": 0.000995}


@pytest.fixture(scope="module")
def data():
    Q, P = datagen.make_problem(N, M, D, SEED)
    qi, _ = datagen.queries_from_items(P, 2000, SEED)
    qs = np.concatenate([qi, datagen.random_queries(2000, D, SEED)])
    cpu = S.SimpferCPU(Q, P, k_max=KMAX, p_prime=100)
    truth = [cpu.query(q, K) for q in qs]
    cpu.close()
    return Q, P, qs, truth


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_precision_config_every_set_equals_cpu_simpfer(data, precision):
    Q, P, qs, truth = data
    index = rmips.rmips_build_index(Q, P, k_max=KMAX, precision=precision)
    ids, offs = rmips.rmips_query_batch(index, qs, np.full(len(qs), K, np.int32))
    bad = [j for j in range(len(qs)) if not np.array_equal(ids[offs[j]:offs[j + 1]], truth[j])]
    assert not bad, (precision, bad[:10])
    assert sum(len(t) for t in truth) > 0
    index.close()


@pytest.mark.parametrize("kind", ["tf32", "bf16", "fp16"])
def test_precision_config_inner_product_error(data, kind):
    # tiles of the workload: the 128 largest-norm users and random ones,
    # against item and random queries
    torch = pytest.importorskip("torch")
    Q, P, qs, _ = data
    un = np.linalg.norm(Q.astype(np.float64), axis=1)
    rng = np.random.default_rng(3)
    worst = 0.0
    for users in (np.argsort(-un)[:128], rng.choice(N, 128, replace=False)):
        for q0 in (0, 2000, 1000):
            A, B = Q[users], qs[q0:q0 + 64]
            dA, dB = torch.from_numpy(np.ascontiguousarray(A)).cuda(), torch.from_numpy(np.ascontiguousarray(B)).cuda()
            dD = torch.zeros((128, 64), dtype=torch.float32, device="cuda")
            rmips.rmips_debug_tc_tile(dA, dB, dD, kind=kind)
            ref = A.astype(np.float64) @ B.astype(np.float64).T
            nrm = np.linalg.norm(A.astype(np.float64), axis=1)[:, None] * np.linalg.norm(B.astype(np.float64), axis=1)
            worst = max(worst, float((np.abs(dD.cpu().numpy() - ref) / nrm).max()))
    assert 0 < worst <= BOUND[kind] / 2, (kind, worst)
