"""k-MIPS of every user (Definition 1) from the index: the top-k join."""
import numpy as np
import pytest

from oracle import rmips_oracle as O
from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu


def _exact_desc(Q, P, i, ids):
    return sorted((O.exact_dot(Q[i], P[j]) for j in ids), reverse=True)


def test_join_matches_oracle():
    Q, P = datagen.make_problem(3000, 1500, 50, 41)
    index = rmips.rmips_build_index(Q, P, k_max=25)
    for k in (1, 10, 25):
        got = rmips.rmips_topk_join(index, k)
        want = O.topk_mips(Q, P, k)
        assert np.array_equal(got, want), k
    index.close()


def test_join_with_exact_ties_returns_a_valid_top_k():
    """Integer data has many equal products: the ids of tied items may differ
    from the oracle's, the products (and their order) may not."""
    Q, P = datagen.integer_problem(600, 300, 4, 3, lim=2)
    index = rmips.rmips_build_index(Q, P, k_max=20)
    for k in (1, 5, 20):
        got = rmips.rmips_topk_join(index, k)
        want = O.topk_mips(Q, P, k)
        for i in range(Q.shape[0]):
            assert len(set(got[i].tolist())) == k and got[i].min() >= 0 and got[i].max() < P.shape[0]
            vals = [O.exact_dot(Q[i], P[j]) for j in got[i]]
            assert vals == sorted(vals, reverse=True), i
            assert vals == _exact_desc(Q, P, i, want[i]), i
    index.close()


def test_join_device_output_and_errors():
    torch = pytest.importorskip("torch")
    Q, P = datagen.make_problem(2000, 800, 16, 9)
    index = rmips.rmips_build_index(Q, P, k_max=10)
    out = torch.full((2000, 7), -1, dtype=torch.int64, device="cuda")
    rmips.rmips_topk_join(index, 7, out=out)
    assert np.array_equal(out.cpu().numpy(), O.topk_mips(Q, P, 7))
    for k in (0, 11):
        with pytest.raises(rmips.RmipsError) as e:
            rmips.rmips_topk_join(index, k)
        assert e.value.status == 2
    small = rmips.rmips_build_index(Q, P, k_max=10, p_prime=100)
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_topk_join(small, 5)
    assert e.value.status == 1
    index.close()
    small.close()
