"""Index persistence (save / load) and the rebuild with a larger k_max."""
import numpy as np
import pytest

from oracle import rmips_oracle as O
from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_saved_index_answers_identically(tmp_path, precision):
    Q, P = datagen.make_problem(8000, 3000, 50, 31)
    index = rmips.rmips_build_index(Q, P, k_max=12, precision=precision)
    qs, _ = datagen.queries_from_items(P, 400, 31)
    ks = datagen.random_ks(len(qs), 1, 12, 31)
    ids, offs = rmips.rmips_query_batch(index, qs, ks)
    path = str(tmp_path / "index.bin")
    rmips.rmips_index_save(index, path)
    loaded = rmips.rmips_index_load(path)
    a, b = rmips.rmips_index_get_info(index), rmips.rmips_index_get_info(loaded)
    for key in ("n", "m", "d", "k_max", "block_size", "precision", "n_blocks", "p_prime", "incomplete"):
        assert a[key] == b[key], key
    ids2, offs2 = rmips.rmips_query_batch(loaded, qs, ks)
    assert np.array_equal(offs, offs2) and np.array_equal(ids, ids2)
    for j in range(0, len(qs), 53):
        assert np.array_equal(rmips.rmips_query(loaded, qs[j], int(ks[j])), ids[offs[j]:offs[j + 1]])
    index.close()
    loaded.close()


def test_truncated_file_is_refused(tmp_path):
    Q, P = datagen.make_problem(2000, 800, 16, 3)
    index = rmips.rmips_build_index(Q, P, k_max=5)
    path = tmp_path / "index.bin"
    rmips.rmips_index_save(index, str(path))
    data = path.read_bytes()
    cut = tmp_path / "cut.bin"
    cut.write_bytes(data[: len(data) // 2])
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_index_load(str(cut))
    assert e.value.status == 1
    index.close()


@pytest.mark.parametrize("p_prime", [0, 100])
def test_rebuild_serves_larger_k(p_prime):
    Q, P = datagen.make_problem(3000, 1500, 50, 5)
    index = rmips.rmips_build_index(Q, P, k_max=5, p_prime=p_prime)
    qs, _ = datagen.queries_from_items(P, 12, 5)
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_query(index, qs[0], 20)
    assert e.value.status == 2
    big = rmips.rmips_index_rebuild(index, 25)
    assert rmips.rmips_index_get_info(big)["k_max"] == 25
    counts = O.counts_greater_multi(Q, P, qs)
    for j in range(len(qs)):
        for k in (3, 20, 25):
            assert np.array_equal(rmips.rmips_query(big, qs[j], k), np.nonzero(counts[j] < k)[0]), (j, k)
    ks = np.array([25, 1, 20, 7, 25, 13, 5, 22, 9, 25, 2, 18], np.int32)
    ids, offs = rmips.rmips_query_batch(big, qs, ks)
    for j in range(len(qs)):
        assert np.array_equal(ids[offs[j]:offs[j + 1]], np.nonzero(counts[j] < ks[j])[0]), j
    assert np.array_equal(rmips.rmips_query(index, qs[1], 5), np.nonzero(counts[1] < 5)[0])   # old index intact
    index.close()
    big.close()
