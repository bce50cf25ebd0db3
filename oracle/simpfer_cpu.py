"""Python side of the CPU Simpfer baseline (``simpfer_cpu.c``) -- test
infrastructure, not product code.

``build()`` compiles ``simpfer_cpu.c`` with the host C compiler (OpenMP when
available) into ``oracle/libsimpfer_cpu.so``; ``SimpferCPU`` builds the index
of Algorithm 1 and answers queries with Algorithm 3 on the host cores.  Only
the test-suite, ``__graft_entry__`` and ``bench.py``'s CPU-baseline legs use
it; it shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "simpfer_cpu.c")
LIB = os.path.join(HERE, "libsimpfer_cpu.so")

_lib = None
OPENMP = None


class _Stats(C.Structure):
    _fields_ = [("pruned_blocks", C.c_int64), ("lemma1_no", C.c_int64), ("lemma2_yes", C.c_int64),
                ("scanned", C.c_int64), ("scanned_items", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the library if it is missing or older than its source."""
    global OPENMP
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("no C compiler for the CPU Simpfer baseline")
    base = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", SRC, "-o", LIB + ".tmp",
            "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    OPENMP = r.returncode == 0
    if r.returncode != 0:                       # no OpenMP on this host: one thread
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"building simpfer_cpu failed:\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(LIB)
        P, I64, I32 = C.c_void_p, C.c_int64, C.c_int
        lib.simpfer_build.argtypes = [P, I64, P, I64, I32, I32, I64, I32, I32]
        lib.simpfer_build.restype = P
        lib.simpfer_query.argtypes = [P, P, I32, P, I64, I32, C.POINTER(_Stats)]
        lib.simpfer_query.restype = I64
        lib.simpfer_free.argtypes = [P]
        lib.simpfer_max_threads.restype = I32
        lib.simpfer_openmp.restype = I32
        lib.simpfer_exact_sign.argtypes = [P, P, P, I32]
        lib.simpfer_exact_sign.restype = I32
        lib.simpfer_blocks.argtypes = [P]
        lib.simpfer_blocks.restype = I64
        _lib = lib
    return _lib


def openmp() -> bool:
    """Whether the loaded library was compiled with OpenMP."""
    return bool(_load().simpfer_openmp())


def max_threads() -> int:
    return int(_load().simpfer_max_threads())


def exact_sign(u, a, b) -> int:
    """Sign of ``u.a - u.b`` by the expansion arithmetic (exact)."""
    lib = _load()
    u, a, b = (np.ascontiguousarray(x, dtype=np.float32) for x in (u, a, b))
    return int(lib.simpfer_exact_sign(u.ctypes.data, a.ctypes.data, b.ctypes.data, u.shape[0]))


class SimpferCPU:
    """Algorithm 1 on construction, Algorithm 3 per query (host cores)."""

    def __init__(self, Q, P, k_max: int, p_prime: int = 100, block_size: int = 32, threads: int = 0):
        lib = _load()
        self._Q = np.ascontiguousarray(Q, dtype=np.float32)
        self._P = np.ascontiguousarray(P, dtype=np.float32)
        self.n, self.d = self._Q.shape
        self.m = self._P.shape[0]
        self.k_max = k_max
        self.h = lib.simpfer_build(self._Q.ctypes.data, self.n, self._P.ctypes.data, self.m, self.d, k_max,
                                   int(p_prime), block_size, int(threads))
        if not self.h:
            raise ValueError("bad arguments for the CPU Simpfer index")
        self._Q = self._P = None                       # the index keeps its own sorted copies

    def query(self, q, k: int, threads: int = 0, stats: dict | None = None) -> np.ndarray:
        """Ascending ids of Definition 2's result (strict tie rule)."""
        lib = _load()
        q = np.ascontiguousarray(q, dtype=np.float32)
        st = _Stats()
        cap = 1 << 16
        while True:
            out = np.empty(cap, dtype=np.int64)
            cnt = lib.simpfer_query(self.h, q.ctypes.data, int(k), out.ctypes.data, cap, int(threads),
                                    C.byref(st))
            if cnt < 0:
                raise ValueError("k outside [1, k_max]")
            if cnt <= cap:
                break
            cap = int(cnt)
        if stats is not None:
            stats.update({f: int(getattr(st, f)) for f, _ in _Stats._fields_})
            stats["blocks"] = int(lib.simpfer_blocks(self.h))
        return out[:cnt].copy()

    def close(self):
        if self.h:
            _load().simpfer_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
