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


PTR_CLASS_TEST = r"""
#include <cstdio>
#include "ptr_class.h"
using namespace rmips;
int main() {
  // cudaMemoryType values: 0 unregistered, 1 pinned host, 2 device, 3 managed
  if (ptr_class_of(0, -2, 0) != PTR_HOST) return 1;
  if (ptr_class_of(1, 0, 0) != PTR_HOST) return 2;
  if (ptr_class_of(2, 0, 0) != PTR_DEVICE) return 3;
  if (ptr_class_of(2, 1, 0) != PTR_OTHER_DEVICE) return 4;   // memory of GPU 1, index on GPU 0
  if (ptr_class_of(2, 0, 3) != PTR_OTHER_DEVICE) return 5;
  if (ptr_class_of(2, 3, 3) != PTR_DEVICE) return 6;
  if (ptr_class_of(3, 1, 0) != PTR_DEVICE) return 7;         // managed memory is reachable
  std::printf("ptr class ok\n");
  return 0;
}
"""


def test_pointer_of_another_gpu_is_refused(tmp_path):
    """The entry points refuse device memory of a GPU other than the index's
    (a kernel on the index's GPU cannot write there).  The decision is made on
    the attributes cudaPointerGetAttributes reports; here it is fed the
    attributes of a pointer on another device, with no GPU involved."""
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = tmp_path / "ptr.cpp"
    src.write_text(PTR_CLASS_TEST)
    exe = tmp_path / "ptr"
    r = subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-I",
                        os.path.join(ROOT, "paper_2110_07131_gb300", "csrc"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=30)
    assert r.returncode == 0 and "ptr class ok" in r.stdout, (r.returncode, r.stdout)
    # every entry point that takes a caller buffer runs the check
    csrc = os.path.join(ROOT, "paper_2110_07131_gb300", "csrc")
    text = "".join(open(os.path.join(csrc, f)).read() for f in os.listdir(csrc) if f.endswith(".cu"))
    assert text.count("check_ptr_device(") + text.count("ptr_class(") >= 12


# ---------------------------------------------------------------------------
# Index files: every header field and the index arrays are checked on the
# host, before any device call, so these run without a GPU
# ---------------------------------------------------------------------------
def _fnv1a(b: bytes) -> int:
    h = 1469598103934665603
    for x in b:
        h ^= x
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _index_file(n=4, m=3, d=2, k_max=2, bs=32, nb=None, pp=None, precision=0, full_p=1, batch_tc=1,
                no_blocks=0, has_qh=0, has_qtc=0, incomplete=0, pn0=1.0, tune=0, narrays=None,
                permQ=None, permP=None, cand=None, corrupt_hash=False, magic=b"RMIPSIX3"):
    import struct
    nb = (n + bs - 1) // bs if nb is None else nb
    pp = m if pp is None else pp
    pad = 32 * d
    arrays = [np.zeros(n * d + pad, np.float32), np.zeros(m * d + pad, np.float32),
              np.ones(n, np.float32), np.ones(m, np.float32),
              np.arange(n, dtype=np.int32) if permQ is None else np.asarray(permQ, np.int32),
              np.arange(m, dtype=np.int32) if permP is None else np.asarray(permP, np.int32),
              np.zeros(k_max * n * 2, np.float32), np.zeros(k_max * nb, np.float32), np.ones(nb, np.float32)]
    if full_p:
        c = np.full(n * 32, -1, np.int32)
        c[:m] = np.arange(m)
        arrays += [c if cand is None else np.asarray(cand, np.int32), np.zeros(n * 32 * 2, np.float32),
                   np.zeros(n, np.uint8)]
    if has_qh:
        arrays.append(np.zeros(n * d + pad, np.float16))
    narrays = len(arrays) if narrays is None else narrays
    out = bytearray(magic)
    out += struct.pack("<5q", n, m, nb, pp, incomplete)
    out += struct.pack("<10i", d, k_max, bs, precision, full_p, batch_tc, no_blocks, has_qh, has_qtc, narrays)
    out += struct.pack("<fi", pn0, tune)
    assert len(out) == 96
    for i, a in enumerate(arrays):
        b = a.tobytes()
        out += struct.pack("<q", len(b)) + b
        h = _fnv1a(b) ^ (1 if (corrupt_hash and i == 2) else 0)
        out += struct.pack("<Q", h)
    return bytes(out)


def test_index_file_crafted_by_the_test_is_accepted_up_to_the_device(tmp_path):
    # the reference file passes every host check: loading it only fails (if at
    # all) when it reaches the device, which this machine may not have
    p = tmp_path / "ok.rmips"
    p.write_bytes(_index_file())
    try:
        idx = rmips.rmips_index_load(str(p))
        idx.close()
    except rmips.RmipsError as e:
        assert e.status in (4, 7), (e.status, str(e))


@pytest.mark.parametrize("field", [
    dict(bs=48), dict(nb=2), dict(precision=7), dict(pp=5), dict(pp=2), dict(full_p=2),
    dict(batch_tc=3), dict(no_blocks=-1), dict(has_qh=1), dict(has_qtc=1, d=80), dict(incomplete=9),
    dict(pn0=float("nan")), dict(tune=1), dict(tune=9 << 8), dict(tune=3 << 16), dict(tune=1 << 24),
    dict(narrays=3), dict(k_max=40), dict(d=0),
    dict(magic=b"RMIPSIX2"), dict(permQ=[0, 1, 1, 3]), dict(permQ=[0, 1, 2, 4]), dict(permP=[2, 0, -1]),
    dict(cand=[5] + [-1] * 127), dict(corrupt_hash=True)])
def test_index_file_with_an_inconsistent_field_is_refused(tmp_path, field):
    p = tmp_path / "bad.rmips"
    p.write_bytes(_index_file(**field))
    with pytest.raises(rmips.RmipsError) as e:
        rmips.rmips_index_load(str(p))
    assert e.value.status == 1, (field, e.value.status, str(e.value))


def test_truncated_or_padded_index_file_is_refused(tmp_path):
    good = _index_file()
    for name, data in (("short", good[:-9]), ("long", good + b"\0"), ("header", good[:50])):
        p = tmp_path / f"{name}.rmips"
        p.write_bytes(data)
        with pytest.raises(rmips.RmipsError) as e:
            rmips.rmips_index_load(str(p))
        assert e.value.status == 1, name
