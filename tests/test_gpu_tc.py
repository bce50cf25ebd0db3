"""Tensor-core (tcgen05) tiles used by the batched filter, against float64.

The batched filter charges each inner product an error of at most
``rel * ||u|| ||q||`` (TF32 0.00198, BF16 0.00788, FP16 0.000995, derived from
the operand formats and a float32 accumulator).  The tiles here run real data
through the same shared-memory layout, descriptors, MMAs and TMEM loads; the
observed error must stay within half of that budget.
"""
import numpy as np
import pytest

from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu

BOUND = {"tf32": 0.00198, "bf16": 0.00788, "fp16": 0.000995}


@pytest.mark.parametrize("kind", ["tf32", "bf16", "fp16"])
@pytest.mark.parametrize("data", ["gauss", "mf"])
def test_tc_tile_error_within_half_the_bound(kind, data):
    torch = pytest.importorskip("torch")
    if data == "gauss":
        rng = np.random.default_rng(0)
        A = rng.standard_normal((128, 64)).astype(np.float32)
        B = rng.standard_normal((64, 64)).astype(np.float32)
    else:                                   # MF-like rows, d = 50 padded with zeros (the filter's case)
        Q, P = datagen.make_problem(128, 64, 50, 3)
        A = np.zeros((128, 64), np.float32)
        B = np.zeros((64, 64), np.float32)
        A[:, :50], B[:, :50] = Q, P
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dD = torch.zeros((128, 64), dtype=torch.float32, device="cuda")
    rmips.rmips_debug_tc_tile(dA, dB, dD, kind=kind)
    D = dD.cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    norms = np.linalg.norm(A.astype(np.float64), axis=1)[:, None] * np.linalg.norm(B.astype(np.float64), axis=1)[None, :]
    rel = np.abs(D - ref) / norms
    assert rel.max() <= BOUND[kind] / 2, rel.max()
    assert rel.max() > 0                    # the tile really ran in reduced precision


def test_swapped_descriptor_offsets_give_wrong_products():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    A = rng.standard_normal((128, 64)).astype(np.float32)
    B = rng.standard_normal((64, 64)).astype(np.float32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dD = torch.zeros((128, 64), dtype=torch.float32, device="cuda")
    rmips.rmips_debug_tc_tile(dA, dB, dD, kind="tf32", lbo=2048, sbo=128)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.abs(dD.cpu().numpy() - ref).max() > 1.0
