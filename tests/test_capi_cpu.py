"""Host-side checks of the C-ABI library (no GPU needed, no device compute)."""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from paper_2110_07131_gb300 import datagen, rmips

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "rmips.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rmips_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return rmips.load_library()


def test_library_exports_every_declared_function(lib):
    names = _declared_functions()
    assert len(names) >= 10
    raw = ctypes.CDLL(rmips.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name
    assert sorted(names) == sorted(rmips.EXPORTED_SYMBOLS)


def test_status_strings(lib):
    assert rmips.rmips_status_string(0) == "ok"
    assert "capacity" in rmips.rmips_status_string(5)
    assert rmips.rmips_status_string(99) == "unknown status"


def _fsign(u, a, b):
    s = sum(Fraction(float(x)) * (Fraction(float(y)) - Fraction(float(z))) for x, y, z in zip(u, a, b))
    return (s > 0) - (s < 0)


def test_exact_sign_matches_rationals_random(lib):
    rng = np.random.default_rng(0)
    for _ in range(300):
        d = int(rng.integers(1, 70))
        u, a, b = (rng.standard_normal(d).astype(np.float32) for _ in range(3))
        assert rmips.rmips_exact_sign_host(u, a, b) == _fsign(u, a, b)


def test_exact_sign_ties_and_extremes(lib):
    Q, P = datagen.integer_problem(8, 8, 16, 3, lim=3)
    for u in Q:
        for a in P:
            for b in P:
                assert rmips.rmips_exact_sign_host(u, a, b) == _fsign(u, a, b)
    big = np.float32(3.0e38)
    tiny = np.float32(1.4e-45)        # smallest subnormal
    u = np.array([big, tiny, -big, 1.0], np.float32)
    a = np.array([big, tiny, big, 2.0 ** -60], np.float32)
    b = np.array([big, 0.0, big, 0.0], np.float32)
    assert rmips.rmips_exact_sign_host(u, a, b) == _fsign(u, a, b) == 1
    # cancellation far below float64 resolution
    u = np.array([1.0, 1.0, 1.0], np.float32)
    a = np.array([1.0, 2.0 ** -30, -(2.0 ** -30) + 2.0 ** -54], np.float32)
    b = np.array([1.0, 2.0 ** -30, -(2.0 ** -30)], np.float32)
    assert rmips.rmips_exact_sign_host(u, a, b) == 1
    assert rmips.rmips_exact_sign_host(u, b, a) == -1
    assert rmips.rmips_exact_sign_host(u, a, a) == 0


def test_exact_sign_full_dimension(lib):
    rng = np.random.default_rng(1)
    for d in (128, 256):
        u = (rng.standard_normal(d) * 2.0 ** rng.integers(-100, 100, d)).astype(np.float32)
        a = (rng.standard_normal(d) * 2.0 ** rng.integers(-100, 100, d)).astype(np.float32)
        b = a.copy()
        b[d // 2] = np.nextafter(b[d // 2], np.float32(np.inf))
        assert rmips.rmips_exact_sign_host(u, a, b) == _fsign(u, a, b)


def test_index_load_refuses_foreign_files_without_a_gpu(tmp_path):
    """The file header is checked before any device call."""
    from paper_2110_07131_gb300 import rmips
    bogus = tmp_path / "not_an_index.bin"
    bogus.write_bytes(b"hello, this is not an index" * 10)
    for path in (str(bogus), str(tmp_path / "missing.bin")):
        with pytest.raises(rmips.RmipsError) as e:
            rmips.rmips_index_load(path)
        assert e.value.status == 1
