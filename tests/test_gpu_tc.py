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



# Largest relative operand-rounding error each format can make, placed on every
# entry of a tile with all products positive, so the errors add up coherently:
#  - TF32: 1 + 2^-10 - 2^-23 loses ~2^-10 if the conversion truncates, and
#    1 + 2^-11 + 2^-22 loses ~2^-11 if it rounds to nearest;
#  - BF16 / FP16 (rounded to nearest): just above the midpoint between 1 and
#    the next value of the format.
WORST = {"tf32": [1 + 2.0 ** -10 - 2.0 ** -23, 1 + 2.0 ** -11 + 2.0 ** -22],
         "bf16": [1 + 2.0 ** -8 + 2.0 ** -20],
         "fp16": [1 + 2.0 ** -11 + 2.0 ** -20]}


def _tile_rel_err(A, B, kind):
    torch = pytest.importorskip("torch")
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dD = torch.zeros((128, 64), dtype=torch.float32, device="cuda")
    rmips.rmips_debug_tc_tile(dA, dB, dD, kind=kind)
    D = dD.cpu().numpy().astype(np.float64)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = A64 @ B64.T
    norms = np.linalg.norm(A64, axis=1)[:, None] * np.linalg.norm(B64, axis=1)[None, :]
    return np.abs(D - ref) / norms


@pytest.mark.parametrize("kind", ["tf32", "bf16", "fp16"])
def test_tc_tile_adversarial_error_within_the_bound(kind):
    """The error bound of each kind (operand rounding, exact products, the
    accumulation assumption) against tiles built to reach it."""
    rng = np.random.default_rng(7)
    worst = np.zeros(0)
    for v in WORST[kind]:
        # coherent rounding: every entry the worst value, scaled by powers of
        # two per row (exact), all 64 columns used
        A = np.full((128, 64), v, np.float32) * (2.0 ** rng.integers(-4, 5, (128, 1))).astype(np.float32)
        B = np.full((64, 64), v, np.float32) * (2.0 ** rng.integers(-4, 5, (64, 1))).astype(np.float32)
        rel = _tile_rel_err(A, B, kind)
        assert rel.max() <= BOUND[kind], (kind, v, rel.max())
        worst = np.concatenate([worst, rel.ravel()])
    # the bound is not loose on these tiles: the coherent case reaches at
    # least 45 % of it (TF32 rounded to nearest) and up to 99 % (BF16)
    assert worst.max() >= 0.45 * BOUND[kind], (kind, worst.max())
    # mixed exponents (within each format's normal range) and cancellation
    span = 5 if kind == "fp16" else 12
    A = (rng.standard_normal((128, 64)) * 2.0 ** rng.integers(-span, span + 1, (128, 64))).astype(np.float32)
    B = (rng.standard_normal((64, 64)) * 2.0 ** rng.integers(-span, span + 1, (64, 64))).astype(np.float32)
    assert _tile_rel_err(A, B, kind).max() <= BOUND[kind]
    sgn = np.where(np.arange(64) % 2 == 0, 1.0, -1.0).astype(np.float32)
    B = (A[:64] * sgn[None, :]).astype(np.float32)             # u.q = sum of +-u_i^2: heavy cancellation
    B[:, 1::2] = np.nextafter(B[:, 1::2], np.float32(0))        # cancel up to the last bits
    assert _tile_rel_err(A, B, kind).max() <= BOUND[kind]
