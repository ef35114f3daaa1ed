"""Seeded synthetic inputs for suffix-array construction (ctypes over gen.c).

Holds no suffix-sorting arithmetic: the CPU oracle and the CUDA path both
take their inputs from here and share nothing else.

Recipes (see gen.h): 1 uniform DNA, 2 Zipf(1.1) base repeated 256x with
0.1% substitutions per copy, 3 order-3 Markov DNA with 5% copied segments,
4 a batch of log-uniform-length DNA texts, 5 a Poisson request stream.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgbsagen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libgbsagen.so (plain gcc, no contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, "gen.h")))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, p = ctypes.c_uint64, ctypes.c_void_p
        for name in ("gen_dna_uniform", "gen_zipf_repeats", "gen_zipf_iid",
                     "gen_bytes_uniform"):
            getattr(lib, name).argtypes = [u64, u64, p]
            getattr(lib, name).restype = None
        lib.gen_markov_dna.argtypes = [u64, u64, p, p]
        lib.gen_markov_dna.restype = None
        lib.gen_batch_lengths.argtypes = [u64, ctypes.c_uint32, u64, u64, p]
        lib.gen_batch_lengths.restype = None
        lib.gen_request_stream.argtypes = [u64, ctypes.c_uint32, ctypes.c_double,
                                           u64, u64, p, p, p]
        lib.gen_request_stream.restype = None
        lib.gen_log.argtypes = [ctypes.c_double]
        lib.gen_log.restype = ctypes.c_double
        lib.gen_exp.argtypes = [ctypes.c_double]
        lib.gen_exp.restype = ctypes.c_double
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def text(recipe: str, seed: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
    """One text of n bytes.

    recipe: "dna" (1), "zipf_repeats" (2), "markov" (3), "zipf" (i.i.d.
    Zipf bytes, the byte half of 5) or "bytes" (uniform 0..255).
    """
    lib = _load()
    if out is None:
        out = np.empty(n, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.size >= n and out.flags.c_contiguous
    if n == 0:
        return out[:0]
    if recipe == "dna":
        lib.gen_dna_uniform(seed, n, _ptr(out))
    elif recipe == "zipf_repeats":
        lib.gen_zipf_repeats(seed, n, _ptr(out))
    elif recipe == "markov":
        scratch = np.empty(n, dtype=np.uint8)
        lib.gen_markov_dna(seed, n, _ptr(out), _ptr(scratch))
    elif recipe == "zipf":
        lib.gen_zipf_iid(seed, n, _ptr(out))
    elif recipe == "bytes":
        lib.gen_bytes_uniform(seed, n, _ptr(out))
    else:
        raise ValueError(f"unknown recipe {recipe!r}")
    return out[:n]


def batch_lengths(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Recipe 4 lengths: log-uniform in [lo, hi]."""
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    if count:
        lib.gen_batch_lengths(seed, count, lo, hi, _ptr(out))
    return out


def batch(seed: int, count: int, lo: int, hi: int):
    """Recipe 4: (flat uint8 texts, uint64 offsets[count+1]); text k is
    uniform DNA drawn with seed (seed * 1_000_003 + k)."""
    lengths = batch_lengths(seed, count, lo, hi)
    offsets = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(lengths, out=offsets[1:])
    flat = np.empty(int(offsets[-1]), dtype=np.uint8)
    for k in range(count):
        a, b = int(offsets[k]), int(offsets[k + 1])
        if b > a:
            text("dna", seed * 1_000_003 + k, b - a, out=flat[a:b])
    return flat, offsets


def request_stream(seed: int, count: int, lam: float, lo: int, hi: int):
    """Recipe 5: (arrival seconds, sizes, kinds) for count requests."""
    lib = _load()
    t = np.empty(count, dtype=np.float64)
    s = np.empty(count, dtype=np.uint64)
    k = np.empty(count, dtype=np.uint8)
    if count:
        lib.gen_request_stream(seed, count, lam, lo, hi, _ptr(t), _ptr(s), _ptr(k))
    return t, s, k


def request_text(seed: int, index: int, size: int, kind: int) -> np.ndarray:
    """The text of request `index` of a recipe-5 stream."""
    return text("dna" if kind == 0 else "zipf", seed * 7_919 + index, size)


def log(x: float) -> float:
    return _load().gen_log(x)


def exp(x: float) -> float:
    return _load().gen_exp(x)
