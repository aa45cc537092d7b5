"""ctypes wrapper of numarck_cpu.c, the multi-threaded C implementation of the compression path
used as the all-cores CPU baseline of the benchmark.

TEST AND BENCHMARK INFRASTRUCTURE ONLY (like the oracle in this directory): only the test suite
and bench.py's cpu_baseline leg use it. It is compiled here with gcc from its C source (plain C,
POSIX threads, -ffp-contract=off, no fast-math) and shares no code with the GPU library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "numarck_cpu.c")
LIB = os.path.join(_HERE, "_build", "libnumarck_cpu.so")
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-pthread"]

_lib = None


def build(force: bool = False) -> str:
    """Compiles the library (if it is missing or older than its source)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i64, i32, sz, d = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t,
                               ctypes.c_double)
        L.ncpu_compress_bound.argtypes = [i64, i32, i32, i64]
        L.ncpu_compress_bound.restype = sz
        L.ncpu_compress.argtypes = [vp, vp, i64, i32, i32, d, i32, i64, i32, vp, sz,
                                    ctypes.POINTER(sz)]
        L.ncpu_compress.restype = i32
        L.ncpu_decompress.argtypes = [vp, sz, vp, vp, i64, i32]
        L.ncpu_decompress.restype = i32
        _lib = L
    return _lib


def threads_available() -> int:
    return len(os.sched_getaffinity(0))


def compress(prev: np.ndarray, cur: np.ndarray, E: float, B: int, anchor: int = 0,
             block_bytes: int = 1 << 20, threads: int | None = None) -> bytes:
    prev = np.ascontiguousarray(prev)
    cur = np.ascontiguousarray(cur)
    assert prev.dtype == cur.dtype and prev.dtype in (np.float32, np.float64)
    dtype = 1 if prev.dtype == np.float64 else 0
    n = prev.size
    cap = lib().ncpu_compress_bound(n, dtype, B, block_bytes)
    out = np.empty(max(cap, 1), dtype=np.uint8)
    size = ctypes.c_size_t(0)
    rc = lib().ncpu_compress(prev.ctypes.data, cur.ctypes.data, n, dtype, B, float(E), anchor,
                             block_bytes, threads or threads_available(), out.ctypes.data, cap,
                             ctypes.byref(size))
    if rc != 0:
        raise RuntimeError(f"ncpu_compress: status {rc}")
    return out[: size.value].tobytes()


def decompress(blob: bytes, prev: np.ndarray, threads: int | None = None) -> np.ndarray:
    prev = np.ascontiguousarray(prev)
    out = np.empty_like(prev)
    buf = np.frombuffer(blob, dtype=np.uint8)
    rc = lib().ncpu_decompress(buf.ctypes.data, buf.size, prev.ctypes.data, out.ctypes.data,
                               prev.size, threads or threads_available())
    if rc != 0:
        raise RuntimeError(f"ncpu_decompress: status {rc}")
    return out
