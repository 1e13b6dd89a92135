"""ctypes front end of the plain CPU oracle in ``oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the product package never imports it.

The C file restates the GateKeeper-GPU filter of arxiv 2103.14978 one base per
byte (Sec. 2.1 masks, amendment, AND and windowed count; Sec. 3.3 undefined
bases; Sec. 3.4 leading/trailing improvement) and a textbook Levenshtein
distance (the ground truth of Sec. 4.4).  This module only compiles it with
gcc, loads it and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

RUNS4 = 0  # runs of 1s per 4-base window (default reading of Sec. 2.1)
POPCOUNT = 1  # number of 1s in the final vector
RUNS = 2  # runs of 1s over the whole vector

FLAG_NO_EDGE_FIX = 1  # the original GateKeeper: no Sec. 3.4 improvement

UNDEFINED = 0xFFFF  # edits of a pair holding a non-ACGT base (Sec. 3.3)
INVALID = 0xFFFE  # edits of a pair whose read id / window is out of range

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u16p = ctypes.POINTER(ctypes.c_uint16)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.gko_code.argtypes = [ctypes.c_ubyte]
            L.gko_code.restype = ctypes.c_int
            L.gko_shifted_mask.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, _u8p]
            L.gko_amend.argtypes = [_u8p, ctypes.c_int]
            L.gko_edge_fix.argtypes = [_u8p, ctypes.c_int, ctypes.c_int]
            L.gko_count.argtypes = [_u8p, ctypes.c_int, ctypes.c_int]
            L.gko_count.restype = ctypes.c_int
            L.gko_final_vector.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p]
            L.gko_final_vector.restype = ctypes.c_int
            L.gko_filter_pair.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, _u8p, _u16p]
            L.gko_filter_batch.argtypes = [ctypes.c_void_p, _u64p, _u16p, ctypes.c_uint64,
                                           ctypes.c_void_p, ctypes.c_uint64, _u32p, _u32p, _u8p,
                                           ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                           _u8p, _u16p, ctypes.c_int]
            L.gko_filter_batch.restype = ctypes.c_int
            L.gko_levenshtein.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
            L.gko_levenshtein.restype = ctypes.c_int
            L.gko_levenshtein_batch.argtypes = [ctypes.c_void_p, _u64p, _u16p, ctypes.c_void_p, _u32p, _u32p,
                                                ctypes.c_uint64, _i32p, ctypes.c_int]
            L.gko_levenshtein_batch.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _bits(s: str) -> np.ndarray:
    return np.frombuffer(s.encode(), dtype=np.uint8) - ord("0")


def _str(bits: np.ndarray) -> str:
    return "".join("1" if b else "0" for b in bits)


# ---- single steps (used by the worked-example pins) ----------------------

def shifted_mask(R: str, G: str, s: int) -> str:
    """Mask of the read shifted by s bases against the segment (Sec. 2.1)."""
    m = len(R)
    assert len(G) == m
    M = np.zeros(max(m, 1), np.uint8)
    lib().gko_shifted_mask(R.encode(), G.encode(), m, s, _ptr(M, _u8p))
    return _str(M[:m])


def amend(bits: str) -> str:
    """Amendment of one mask (Sec. 2.1); bits as a '0'/'1' string."""
    M = np.ascontiguousarray(_bits(bits)) if bits else np.zeros(1, np.uint8)
    lib().gko_amend(_ptr(M, _u8p), len(bits))
    return _str(M[: len(bits)])


def edge_fix(bits: str, s: int) -> str:
    """Leading/trailing improvement of one amended mask (Sec. 3.4)."""
    M = np.ascontiguousarray(_bits(bits)) if bits else np.zeros(1, np.uint8)
    lib().gko_edge_fix(_ptr(M, _u8p), len(bits), s)
    return _str(M[: len(bits)])


def count(bits: str, mode: int = RUNS4) -> int:
    """Error count of a final vector (Sec. 2.1)."""
    M = np.ascontiguousarray(_bits(bits)) if bits else np.zeros(1, np.uint8)
    return lib().gko_count(_ptr(M, _u8p), len(bits), mode)


def final_vector(R: str, G: str, e: int, flags: int = 0):
    """AND of the 2e+1 amended, edge-fixed masks, or None if undefined."""
    m = len(R)
    assert len(G) == m
    F = np.zeros(max(m, 1), np.uint8)
    if lib().gko_final_vector(R.encode(), G.encode(), m, e, flags, _ptr(F, _u8p)):
        return None
    return _str(F[:m])


def filter_pair(R: str, G: str, e: int, mode: int = RUNS4, flags: int = 0):
    """(accept, edits) of one pair."""
    m = len(R)
    assert len(G) == m
    a = np.zeros(1, np.uint8)
    ed = np.zeros(1, np.uint16)
    lib().gko_filter_pair(R.encode(), G.encode(), m, e, mode, flags, _ptr(a, _u8p), _ptr(ed, _u16p))
    return int(a[0]), int(ed[0])


def levenshtein(a: str, b: str) -> int:
    return lib().gko_levenshtein(a.encode(), len(a), b.encode(), len(b))


# ---- batches ---------------------------------------------------------------

def filter_batch(reads: np.ndarray, read_start: np.ndarray, read_len: np.ndarray,
                 ref: np.ndarray, pair_read: np.ndarray, pair_off: np.ndarray, e,
                 mode: int = RUNS4, flags: int = 0, threads: int | None = None):
    """Filter many pairs.  ``reads``/``ref`` are uint8 ASCII buffers, read r is
    ``reads[read_start[r] : read_start[r] + read_len[r]]``.  ``e`` is an int or a
    uint8 array (one per pair).  Returns (accept uint8[n], edits uint16[n],
    threads used)."""
    reads = np.ascontiguousarray(reads, dtype=np.uint8)
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    read_start = np.ascontiguousarray(read_start, dtype=np.uint64)
    read_len = np.ascontiguousarray(read_len, dtype=np.uint16)
    pair_read = np.ascontiguousarray(pair_read, dtype=np.uint32)
    pair_off = np.ascontiguousarray(pair_off, dtype=np.uint32)
    n = pair_read.shape[0]
    assert pair_off.shape[0] == n
    if np.isscalar(e) or np.ndim(e) == 0:
        pe, fixed_e = None, int(e)
    else:
        pe = np.ascontiguousarray(e, dtype=np.uint8)
        assert pe.shape[0] == n
        fixed_e = 0
    accept = np.zeros(n, np.uint8)
    edits = np.zeros(n, np.uint16)
    threads = threads or os.cpu_count() or 1
    used = lib().gko_filter_batch(
        reads.ctypes.data, _ptr(read_start, _u64p), _ptr(read_len, _u16p), read_len.shape[0],
        ref.ctypes.data, ref.shape[0], _ptr(pair_read, _u32p), _ptr(pair_off, _u32p),
        _ptr(pe, _u8p) if pe is not None else None, fixed_e, n, mode, flags,
        _ptr(accept, _u8p), _ptr(edits, _u16p), threads)
    return accept, edits, used


def levenshtein_batch(reads, read_start, read_len, ref, pair_read, pair_off, threads=None):
    """Edit distance of every pair's read against its reference window."""
    reads = np.ascontiguousarray(reads, dtype=np.uint8)
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    read_start = np.ascontiguousarray(read_start, dtype=np.uint64)
    read_len = np.ascontiguousarray(read_len, dtype=np.uint16)
    pair_read = np.ascontiguousarray(pair_read, dtype=np.uint32)
    pair_off = np.ascontiguousarray(pair_off, dtype=np.uint32)
    n = pair_read.shape[0]
    dist = np.zeros(n, np.int32)
    lib().gko_levenshtein_batch(reads.ctypes.data, _ptr(read_start, _u64p), _ptr(read_len, _u16p),
                                ref.ctypes.data, _ptr(pair_read, _u32p), _ptr(pair_off, _u32p), n,
                                _ptr(dist, _i32p), threads or os.cpu_count() or 1)
    return dist
