"""Tensor-core (tcgen05, TF32) tile used by the batched filter vs float64."""
import numpy as np
import pytest

from paper_2110_07131_gb300 import rmips

pytestmark = pytest.mark.gpu


def test_tc_tile_matches_fp64_within_tf32_bound():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    A = rng.standard_normal((128, 64)).astype(np.float32)
    B = rng.standard_normal((64, 64)).astype(np.float32)
    A[:, 50:] = 0.0                       # the filter pads d = 50 to K = 64 with zeros
    B[:, 50:] = 0.0
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dD = torch.zeros((128, 64), dtype=torch.float32, device="cuda")
    rmips.rmips_debug_tc_tile(dA, dB, dD)
    D = dD.cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    rel = np.abs(D - ref) / scale
    # TF32 keeps 10 fraction bits: each operand is within 2^-10 (relative) of
    # its float32 value, so the product error is below 2^-9 of |a||b|.
    assert rel.max() <= 2.0 ** -9
    assert rel.max() > 0                  # the tile really ran in reduced precision
