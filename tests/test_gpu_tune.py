"""The autotuner: tuned and default launch choices return the oracle's sets,
and the choices are cached in the tune file and saved with the index."""
import numpy as np
import pytest

from oracle import rmips_oracle as O
from paper_2110_07131_gb300 import datagen, rmips

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    Q, P = datagen.make_problem(6000, 3000, 50, 31)
    qs, _ = datagen.queries_from_items(P, 40, 31)
    qs = np.concatenate([qs, datagen.random_queries(8, 50, 31)])
    return Q, P, qs, O.counts_greater_multi(Q, P, qs)


def _check(index, qs, counts):
    ks = datagen.random_ks(len(qs), 1, 25, 4)
    ids, offs = rmips.rmips_query_batch(index, qs, ks)
    for j in range(len(qs)):
        assert np.array_equal(ids[offs[j]:offs[j + 1]], np.nonzero(counts[j] < ks[j])[0]), j
    for j in range(0, len(qs), 5):
        assert np.array_equal(rmips.rmips_query(index, qs[j], 10), np.nonzero(counts[j] < 10)[0]), j


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_tuned_and_default_choices_give_the_oracle_sets(data, tmp_path, precision):
    Q, P, qs, counts = data
    cache = str(tmp_path / "tune.txt")
    default = rmips.rmips_build_index(Q, P, k_max=25, precision=precision)
    _check(default, qs, counts)
    tuned = rmips.rmips_build_index(Q, P, k_max=25, precision=precision, tune_cache=cache)
    info = rmips.rmips_index_get_info(tuned)
    assert info["tuned"] == 1 and info["block_size"] in (32, 64, 128, 256)
    assert info["batch_stages"] in (4, 8, 12) and info["single_stages"] >= 1
    _check(tuned, qs, counts)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and f"bs={info['block_size']}" in lines[0]
    # a second build reads the cache instead of searching
    again = rmips.rmips_build_index(Q, P, k_max=25, precision=precision, tune_cache=cache)
    info2 = rmips.rmips_index_get_info(again)
    assert info2["tuned"] == 2
    for key in ("block_size", "batch_stages", "single_stages"):
        assert info2[key] == info[key]
    assert len(open(cache).read().splitlines()) == 1
    # tuning an index after its build (no cache: a search) keeps it exact
    info3 = rmips.rmips_index_tune(default, None)
    assert info3["tuned"] == 1
    _check(default, qs, counts)
    for ix in (default, tuned, again):
        ix.close()


def test_tuned_choices_are_saved_with_the_index(data, tmp_path):
    Q, P, qs, counts = data
    index = rmips.rmips_build_index(Q, P, k_max=25, autotune=True)
    info = rmips.rmips_index_get_info(index)
    path = str(tmp_path / "ix.rmips")
    rmips.rmips_index_save(index, path)
    loaded = rmips.rmips_index_load(path)
    linfo = rmips.rmips_index_get_info(loaded)
    for key in ("tuned", "block_size", "batch_stages", "single_stages", "n_blocks"):
        assert linfo[key] == info[key], key
    _check(loaded, qs, counts)
    bigger = rmips.rmips_index_rebuild(loaded, 28)
    assert rmips.rmips_index_get_info(bigger)["batch_stages"] == info["batch_stages"]
    for ix in (index, loaded, bigger):
        ix.close()
