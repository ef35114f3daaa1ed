"""CPU oracle for suffix-array construction — TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
reference legs may import this package. The CUDA library never does: the
two share no code, headers or helpers.

ctypes bindings over oracle.c (plain sequential C, integer only), which
follows Section 2 (definition of SA/ISA and the $ sentinel) and Section 2.1
(prefix doubling: Algorithms 1, 2, 4, 5 and 6, and its a-fold form of
the Prefix Quadrupling subsection) of Bingmann, Gog & Kurpicz,
"Scalable Construction of Text Indexes" (arXiv 1610.03007).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")


def _lib_path(mutant: int) -> str:
    return os.path.join(_HERE, "liboracle.so" if mutant == 0 else f"liboracle_m{mutant}.so")


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile oracle.c (gcc, -O2) into liboracle.so, or a planted-mutant
    build liboracle_m<k>.so used only by the pin tests."""
    out = _lib_path(mutant)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           f"-DORACLE_MUTANT={mutant}", "-o", tmp, _SRC])
    os.replace(tmp, out)
    return out


MUTANTS = (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16)


class Oracle:
    """One loaded build of the oracle (mutant 0 is the real one)."""

    def __init__(self, mutant: int = 0):
        lib = ctypes.CDLL(build(mutant))
        p, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.oracle_naive_sa.argtypes = [p, i64, p]
        lib.oracle_naive_sa.restype = None
        lib.oracle_pd_sa.argtypes = [p, i64, i64, p, p, p, i64]
        lib.oracle_pd_sa.restype = i64
        lib.oracle_pq_sa.argtypes = [p, i64, i64, i64, p, p, p, i64]
        lib.oracle_pq_sa.restype = i64
        lib.oracle_check_sa.argtypes = [p, i64, p, p]
        lib.oracle_check_sa.restype = ctypes.c_int
        lib.oracle_check_permutation.argtypes = [p, i64, p]
        lib.oracle_check_permutation.restype = ctypes.c_int
        lib.oracle_check_adjacent.argtypes = [p, i64, p, p, i64]
        lib.oracle_check_adjacent.restype = i64
        lib.oracle_suffix_rank.argtypes = [p, i64, i64]
        lib.oracle_suffix_rank.restype = i64
        lib.oracle_bwt.argtypes = [p, i64, p, p, p]
        lib.oracle_bwt.restype = None
        lib.oracle_lcp_pair.argtypes = [p, i64, i64, i64]
        lib.oracle_lcp_pair.restype = i64
        lib.oracle_lcp.argtypes = [p, i64, p, p]
        lib.oracle_lcp.restype = None
        lib.oracle_dc7_names.argtypes = [p, i64, p]
        lib.oracle_dc7_names.restype = i64
        lib.oracle_bwt_invert.argtypes = [p, i64, i64, p]
        lib.oracle_bwt_invert.restype = ctypes.c_int
        self._lib = lib
        self.mutant = mutant

    @staticmethod
    def _text(t) -> np.ndarray:
        if isinstance(t, (bytes, bytearray, str)):
            t = t.encode("latin-1") if isinstance(t, str) else bytes(t)
            return np.frombuffer(t, dtype=np.uint8).copy()
        a = np.ascontiguousarray(t, dtype=np.uint8)
        return a

    def naive_sa(self, t) -> np.ndarray:
        """SA by its definition: a comparison sort of all suffixes (Section 2)."""
        T = self._text(t)
        sa = np.empty(T.size, dtype=np.uint32)
        self._lib.oracle_naive_sa(T.ctypes.data, T.size, sa.ctypes.data)
        return sa

    def pd_sa(self, t, h0: int = 1, trace_cap: int = 0, a: int = 2):
        """Prefix doubling with discarding (Section 2.1, Algorithms 1/2/4/5/6);
        a = 3 or 4 ranks a-tuples of names per round (Prefix Quadrupling).

        Returns (sa, isa, rounds, trace) where trace has shape
        (min(rounds+1, trace_cap), n): names after the initial naming and
        after each refinement round."""
        T = self._text(t)
        n = T.size
        sa = np.empty(n, dtype=np.uint32)
        isa = np.empty(n, dtype=np.uint32)
        trace = np.zeros((max(trace_cap, 0), n), dtype=np.uint32)
        tp = trace.ctypes.data if trace_cap > 0 else None
        if a == 2:
            rounds = self._lib.oracle_pd_sa(T.ctypes.data, n, h0, sa.ctypes.data,
                                            isa.ctypes.data, tp, trace_cap)
        else:
            rounds = self._lib.oracle_pq_sa(T.ctypes.data, n, h0, a, sa.ctypes.data,
                                            isa.ctypes.data, tp, trace_cap)
            if rounds < 0:
                raise ValueError(f"multiplier a={a} outside [2, 4]")
        return sa, isa, int(rounds), trace[: min(rounds + 1, trace_cap)]

    def check_sa(self, t, sa) -> tuple[int, int]:
        """Burkhardt-Kaerkkaeinen checker: (code, bad index); code 0 = valid."""
        T = self._text(t)
        s = np.ascontiguousarray(sa, dtype=np.uint32)
        if s.size != T.size:
            return 1, -1
        bad = ctypes.c_int64(-1)
        code = self._lib.oracle_check_sa(T.ctypes.data, T.size, s.ctypes.data,
                                         ctypes.byref(bad))
        return int(code), int(bad.value)

    def check_permutation(self, sa) -> int:
        """0 if SA is a permutation of [0, len(SA)), else 1."""
        s = np.ascontiguousarray(sa, dtype=np.uint32)
        bad = ctypes.c_int64(-1)
        return int(self._lib.oracle_check_permutation(s.ctypes.data, s.size, ctypes.byref(bad)))

    def check_adjacent(self, t, sa, idx) -> int:
        T = self._text(t)
        s = np.ascontiguousarray(sa, dtype=np.uint32)
        ix = np.ascontiguousarray(idx, dtype=np.int64)
        return int(self._lib.oracle_check_adjacent(T.ctypes.data, T.size, s.ctypes.data,
                                                   ix.ctypes.data, ix.size))

    def suffix_rank(self, t, i: int) -> int:
        T = self._text(t)
        return int(self._lib.oracle_suffix_rank(T.ctypes.data, T.size, i))

    def bwt(self, t, sa):
        T = self._text(t)
        s = np.ascontiguousarray(sa, dtype=np.uint32)
        out = np.empty(T.size + 1, dtype=np.uint8)
        prim = ctypes.c_int64(0)
        self._lib.oracle_bwt(T.ctypes.data, T.size, s.ctypes.data, out.ctypes.data,
                             ctypes.byref(prim))
        return out, int(prim.value)

    def lcp_pair(self, t, a: int, b: int) -> int:
        """Longest common prefix of suffixes a and b (the definition)."""
        T = self._text(t)
        return int(self._lib.oracle_lcp_pair(T.ctypes.data, T.size, a, b))

    def lcp(self, t, sa) -> np.ndarray:
        """LCP array of T for its suffix array sa (lcp[0] = 0)."""
        T = self._text(t)
        s = np.ascontiguousarray(sa, dtype=np.uint32)
        out = np.zeros(T.size, dtype=np.uint32)
        self._lib.oracle_lcp(T.ctypes.data, T.size, s.ctypes.data, out.ctypes.data)
        return out

    def dc7_names(self, t) -> np.ndarray:
        """DC7's first recursion text: names of the samples i = 0, 1, 3
        (mod 7), i <= n, class by class (Section 2.2)."""
        T = self._text(t)
        out = np.zeros(3 * (T.size // 7 + 1), dtype=np.uint32)
        m = self._lib.oracle_dc7_names(T.ctypes.data, T.size, out.ctypes.data)
        return out[:m]

    def bwt_invert(self, bwt, primary: int) -> np.ndarray:
        b = np.ascontiguousarray(bwt, dtype=np.uint8)
        n = b.size - 1
        out = np.empty(max(n, 0), dtype=np.uint8)
        rc = self._lib.oracle_bwt_invert(b.ctypes.data, n, primary, out.ctypes.data)
        if rc != 0:
            raise ValueError("BWT inversion failed")
        return out


_default = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(0)
    return _default
