"""Python binding of libgk (include/gk.h): argument marshalling only.

Every function forwards to the C entry point of the same name; all filter
work runs in the library's CUDA kernels.  Device buffers are torch tensors,
streams are torch streams.  There is no fallback: if libgk.so is missing or
fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

GK_MAX_LEN = 512
GK_OK, GK_EINVAL, GK_ERANGE, GK_ENOMEM, GK_ECUDA = 0, -1, -2, -3, -4
GK_COUNT_RUNS4, GK_COUNT_POPCOUNT = 0, 1
GK_FLAG_NO_EDGE_FIX = 1
GK_FLAG_RESULT_BYTE = 2
GK_PIPE_SLICED = 4
GK_PIPE_READ_STARTS = 8
GK_RESULT_MAX_COUNT, GK_RESULT_UNDEFINED, GK_RESULT_INVALID = 253, 254, 255
GK_EDITS_UNDEFINED, GK_EDITS_INVALID = 0xFFFF, 0xFFFE

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgk.so")

_lock = threading.Lock()
_lib = None

_c = ctypes


class PipeDesc(ctypes.Structure):
    """gk_pipe_desc_t: sizes, read length and thresholds of a streamed pipe."""
    _fields_ = [("max_reads", ctypes.c_uint64), ("ascii_stride", ctypes.c_uint64), ("read_len", ctypes.c_uint32),
                ("max_pairs", ctypes.c_uint64), ("n_thresholds", ctypes.c_uint32), ("thresholds", ctypes.c_void_p),
                ("count_mode", ctypes.c_int), ("flags", ctypes.c_uint32), ("n_slots", ctypes.c_uint32)]


_SIGS = {
    "gk_last_error": ([], _c.c_char_p),
    "gk_version": ([], _c.c_int),
    "gk_encode": ([_c.c_void_p, _c.c_uint64, _c.c_void_p, _c.c_uint16, _c.c_uint64, _c.c_void_p,
                   _c.c_uint32, _c.c_void_p, _c.c_int, _c.c_void_p], _c.c_int),
    "gk_load_reference": ([_c.c_void_p, _c.c_uint64, _c.c_int, _c.c_void_p, _c.POINTER(_c.c_void_p)],
                          _c.c_int),
    "gk_free_reference": ([_c.c_void_p], None),
    "gk_reference_info": ([_c.c_void_p, _c.POINTER(_c.c_uint64), _c.POINTER(_c.c_uint64)], _c.c_int),
    "gk_filter": ([_c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_uint64, _c.c_void_p, _c.c_uint32,
                   _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_uint64, _c.c_int,
                   _c.c_uint32, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p], _c.c_int),
    "gk_filter_sweep": ([_c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_uint64, _c.c_void_p, _c.c_uint32,
                         _c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_uint32, _c.c_uint64, _c.c_int, _c.c_uint32,
                         _c.c_void_p, _c.c_void_p, _c.c_uint64, _c.c_void_p, _c.c_void_p], _c.c_int),
    "gk_filter_ascii": ([_c.c_void_p, _c.c_void_p, _c.c_uint64, _c.c_uint64, _c.c_uint32, _c.c_void_p,
                         _c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_uint64, _c.c_int, _c.c_uint32, _c.c_void_p,
                         _c.c_void_p, _c.c_void_p, _c.c_void_p], _c.c_int),
    "gk_sliced_bytes": ([_c.c_uint64, _c.c_uint32], _c.c_uint64),
    "gk_slice": ([_c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_uint64, _c.c_void_p, _c.c_uint32, _c.c_void_p,
                  _c.c_void_p, _c.c_uint64, _c.c_void_p, _c.c_uint64, _c.c_void_p, _c.c_void_p], _c.c_int),
    "gk_filter_sliced": ([_c.c_void_p, _c.c_uint64, _c.c_uint64, _c.c_uint32, _c.c_uint32, _c.c_int, _c.c_uint32,
                          _c.c_void_p, _c.c_void_p, _c.c_void_p], _c.c_int),
    "gk_filter_sliced_sweep": ([_c.c_void_p, _c.c_uint64, _c.c_uint64, _c.c_uint32, _c.c_uint32, _c.c_uint32,
                                _c.c_int, _c.c_uint32, _c.c_void_p, _c.c_void_p, _c.c_uint64, _c.c_void_p,
                                _c.c_void_p], _c.c_int),
    "gk_probe_alu": ([_c.c_int, _c.c_uint32, _c.c_uint32, _c.c_uint32, _c.c_void_p, _c.c_void_p], _c.c_int),
    "gk_filter_batched_workspace": ([_c.c_uint64], _c.c_uint64),
    "gk_filter_batched": ([_c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_uint64, _c.c_void_p, _c.c_void_p,
                           _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_uint64, _c.c_int,
                           _c.c_uint32, _c.c_void_p, _c.c_void_p, _c.c_uint64, _c.c_void_p, _c.c_void_p,
                           _c.c_void_p, _c.c_void_p], _c.c_int),
    "gk_filter_batched_noalloc": ([_c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_uint64, _c.c_void_p,
                                   _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_uint32,
                                   _c.c_uint64, _c.c_int, _c.c_uint32, _c.c_void_p, _c.c_void_p,
                                   _c.c_void_p, _c.c_void_p, _c.c_void_p], _c.c_int),
    "gk_rebase_pairs": ([_c.c_void_p, _c.c_void_p, _c.c_uint64, _c.c_void_p, _c.c_void_p, _c.c_void_p,
                         _c.c_uint32, _c.c_void_p], _c.c_int),
    "gk_expand_pairs": ([_c.c_void_p, _c.c_void_p, _c.c_uint64, _c.c_void_p, _c.c_void_p, _c.c_void_p,
                         _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p,
                         _c.c_uint32, _c.c_uint64, _c.c_void_p], _c.c_int),
    "gk_copy_many": ([_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_int, _c.c_void_p], _c.c_int),
    "gk_gather": ([_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_uint32, _c.c_void_p], _c.c_int),
    "gk_pipe_create": ([_c.c_void_p, _c.POINTER(PipeDesc), _c.POINTER(_c.c_void_p)], _c.c_int),
    "gk_pipe_submit": ([_c.c_void_p, _c.c_void_p, _c.c_uint64, _c.c_void_p, _c.c_void_p, _c.c_uint64,
                        _c.c_void_p, _c.c_void_p, _c.POINTER(_c.c_uint64)], _c.c_int),
    "gk_pipe_wait": ([_c.c_void_p, _c.c_uint64], _c.c_int),
    "gk_pipe_destroy": ([_c.c_void_p], None),
}

GK_NOALLOC_MAX_PAIRS = 1_000_000
GK_SLICED_MAX_LEN = 255
GK_SLICED_MAX_SHIFT = 15
GK_SWEEP_MAX_SHIFT = 30
GK_GATHER_MAX_BYTES = 65536


class Tiling(ctypes.Structure):
    """gk_tiling_t: words per lane, pairs per tile, persistent grid shape."""
    _fields_ = [("words_per_thread", ctypes.c_uint32), ("tile_pairs", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("warps_per_block", ctypes.c_uint32)]

    def astuple(self):
        return (self.words_per_thread, self.tile_pairs, self.blocks_per_sm, self.warps_per_block)

    def __repr__(self):
        return "Tiling(wpt=%d, tile=%d, blocks/SM=%d, warps/block=%d)" % self.astuple()


class GKError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libgk error {code}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded libgk.so.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -m paper_2103_14978_gb300.build` (no CPU fallback exists)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(rc: int):
    if rc != GK_OK:
        raise GKError(rc, lib().gk_last_error().decode())


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dptr(t: torch.Tensor | None, dtype: torch.dtype, name: str, numel: int | None = None) -> int | None:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    return t.data_ptr()


def words_for(m: int) -> int:
    return max(1, -(-int(m) // 32))


class Reference:
    """A reference genome encoded once and resident on the current device."""

    def __init__(self, handle: int, n_bases: int, n_undefined: int, device: int):
        self.handle = handle
        self.n_bases = n_bases
        self.n_undefined = n_undefined
        self.device = device

    def close(self):
        if self.handle:
            gk_free_reference(self)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gk_load_reference(ascii, stream=None) -> Reference:
    """Encode ``ascii`` (a uint8 numpy array / host tensor, or a CUDA uint8
    tensor) and keep it resident (gk_load_reference)."""
    if isinstance(ascii, np.ndarray):
        ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
        if not ascii.flags.writeable:
            ascii = ascii.copy()
        ascii = torch.from_numpy(ascii)
    if ascii.dtype != torch.uint8 or not ascii.is_contiguous():
        raise TypeError("reference must be a contiguous uint8 array")
    h = ctypes.c_void_p()
    _check(lib().gk_load_reference(ascii.data_ptr(), ascii.numel(), 1 if ascii.is_cuda else 0,
                                   _stream(stream), ctypes.byref(h)))
    nb, nu = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().gk_reference_info(h, ctypes.byref(nb), ctypes.byref(nu)))
    return Reference(h.value, nb.value, nu.value, torch.cuda.current_device())


def gk_free_reference(ref: Reference):
    lib().gk_free_reference(ref.handle)


def gk_encode(ascii: torch.Tensor, n_seq: int, ascii_stride: int, lens: torch.Tensor | None = None,
              fixed_len: int = 0, stride_words: int | None = None, packed: torch.Tensor | None = None,
              nflag: torch.Tensor | None = None, stream=None):
    """2-bit planes of n_seq sequences (gk_encode).  Device tensors run the
    device encoder on ``stream``; host tensors run the host encoder.  Returns
    (packed int32 [n_seq * stride_words * 2], nflag uint8 [n_seq])."""
    on_device = ascii.is_cuda
    if stride_words is None:
        stride_words = words_for(fixed_len if lens is None else GK_MAX_LEN)
    dev = ascii.device
    if packed is None:
        packed = torch.empty(n_seq * stride_words * 2, dtype=torch.int32, device=dev)
    if nflag is None:
        nflag = torch.empty(n_seq, dtype=torch.uint8, device=dev)
    for t, name in ((packed, "packed"), (nflag, "nflag")) + (((lens, "lens"),) if lens is not None else ()):
        if t.is_cuda != on_device:
            raise TypeError(f"{name} must live where ascii lives")
    if not ascii.is_contiguous() or ascii.dtype != torch.uint8:
        raise TypeError("ascii must be contiguous uint8")
    need = (n_seq - 1) * ascii_stride + (fixed_len if lens is None else ascii_stride)
    if n_seq and ascii.numel() < need:
        raise ValueError("ascii is shorter than n_seq sequences")
    if packed.numel() < n_seq * stride_words * 2 or nflag.numel() < n_seq:
        raise ValueError("output buffers too small")
    if lens is not None and (lens.dtype != torch.int16 or lens.numel() < n_seq):
        raise TypeError("lens must hold n_seq int16 (read as uint16) lengths")
    _check(lib().gk_encode(ascii.data_ptr(), ascii_stride, lens.data_ptr() if lens is not None else None,
                           fixed_len, n_seq, packed.data_ptr(), stride_words, nflag.data_ptr(),
                           1 if on_device else 0, _stream(stream) if on_device else None))
    return packed, nflag


def gk_filter(ref: Reference, reads: torch.Tensor, stride_words: int, n_reads: int,
              read_nflag: torch.Tensor | None, m: int, pair_read: torch.Tensor, pair_off: torch.Tensor,
              e, count_mode: int = GK_COUNT_RUNS4, flags: int = 0, accept: torch.Tensor | None = None,
              edits: torch.Tensor | None = None, err_count: torch.Tensor | None = None, stream=None):
    """Filter pairs of read length m (gk_filter).  ``e`` is an int or a CUDA
    uint8 tensor (one threshold per pair).  ``pair_read``/``pair_off`` are
    int32 CUDA tensors read as uint32.  Returns (accept uint8, edits int16 read
    as uint16); with GK_FLAG_RESULT_BYTE, (result bytes uint8, None)."""
    n = pair_read.numel()
    dev = pair_read.device
    result_byte = bool(flags & GK_FLAG_RESULT_BYTE)
    if accept is None:
        accept = torch.empty(n, dtype=torch.uint8, device=dev)
    if edits is None and not result_byte:
        edits = torch.empty(n, dtype=torch.int16, device=dev)
    if m > 0 and reads.numel() < n_reads * stride_words * 2:
        raise ValueError("reads holds fewer than n_reads * stride_words * 2 words")
    pe = None
    fixed_e = 0
    if isinstance(e, torch.Tensor):
        pe = _dptr(e, torch.uint8, "e", n)
    else:
        fixed_e = int(e)
    _check(lib().gk_filter(
        ref.handle, _dptr(reads, torch.int32, "reads"), stride_words, n_reads,
        _dptr(read_nflag, torch.uint8, "read_nflag", n_reads), m,
        _dptr(pair_read, torch.int32, "pair_read"), _dptr(pair_off, torch.int32, "pair_off", n),
        pe, fixed_e, n, count_mode, flags, _dptr(accept, torch.uint8, "accept", n),
        None if result_byte else _dptr(edits, torch.int16, "edits", n),
        _dptr(err_count, torch.int32, "err_count", 1), _stream(stream)))
    return accept, (None if result_byte else edits)


def gk_filter_sweep(ref: Reference, reads: torch.Tensor, stride_words: int, n_reads: int,
                    read_nflag: torch.Tensor | None, m: int, pair_read: torch.Tensor, pair_off: torch.Tensor,
                    e_lo: int, e_hi: int, count_mode: int = GK_COUNT_RUNS4, flags: int = 0,
                    accept: torch.Tensor | None = None, edits: torch.Tensor | None = None,
                    out_stride: int | None = None, err_count: torch.Tensor | None = None, stream=None):
    """gk_filter at every threshold e_lo..e_hi in one launch
    (gk_filter_sweep).  Returns (accept, edits) as views of shape
    (e_hi - e_lo + 1, n_pairs) over threshold-major buffers (rows out_stride
    elements apart), or (result bytes, None) with GK_FLAG_RESULT_BYTE."""
    n = pair_read.numel()
    dev = pair_read.device
    result_byte = bool(flags & GK_FLAG_RESULT_BYTE)
    n_e = int(e_hi) - int(e_lo) + 1
    if out_stride is None:
        out_stride = max(-(-n // 16) * 16, 1)
    need = (n_e - 1) * out_stride + n if n_e > 0 else 0
    if accept is None:
        accept = torch.empty(max(need, n_e * out_stride, 1), dtype=torch.uint8, device=dev)
    if edits is None and not result_byte:
        edits = torch.empty(max(need, n_e * out_stride, 1), dtype=torch.int16, device=dev)
    if m > 0 and reads.numel() < n_reads * stride_words * 2:
        raise ValueError("reads holds fewer than n_reads * stride_words * 2 words")
    _check(lib().gk_filter_sweep(
        ref.handle, _dptr(reads, torch.int32, "reads"), stride_words, n_reads,
        _dptr(read_nflag, torch.uint8, "read_nflag", n_reads), m, _dptr(pair_read, torch.int32, "pair_read"),
        _dptr(pair_off, torch.int32, "pair_off", n), int(e_lo), int(e_hi), n, count_mode, flags,
        _dptr(accept, torch.uint8, "accept", need),
        None if result_byte else _dptr(edits, torch.int16, "edits", need), out_stride,
        _dptr(err_count, torch.int32, "err_count", 1), _stream(stream)))
    rows = lambda t: t.as_strided((n_e, n), (out_stride, 1))  # noqa: E731
    return rows(accept), (None if result_byte else rows(edits))


def gk_filter_ascii(ref: Reference, ascii: torch.Tensor, ascii_stride: int, n_reads: int, m: int,
                    pair_read: torch.Tensor, pair_off: torch.Tensor, e, count_mode: int = GK_COUNT_RUNS4,
                    flags: int = 0, accept: torch.Tensor | None = None, edits: torch.Tensor | None = None,
                    err_count: torch.Tensor | None = None, stream=None):
    """Filter pairs whose reads are ASCII rows on the device, encoding them in
    the filter kernel (gk_filter_ascii).  Same arguments and results as
    gk_filter, with the uint8 CUDA tensor ``ascii`` (n_reads rows of
    ascii_stride bytes) in place of the packed reads."""
    n = pair_read.numel()
    dev = pair_read.device
    result_byte = bool(flags & GK_FLAG_RESULT_BYTE)
    if accept is None:
        accept = torch.empty(n, dtype=torch.uint8, device=dev)
    if edits is None and not result_byte:
        edits = torch.empty(n, dtype=torch.int16, device=dev)
    pe = None
    fixed_e = 0
    if isinstance(e, torch.Tensor):
        pe = _dptr(e, torch.uint8, "e", n)
    else:
        fixed_e = int(e)
    _check(lib().gk_filter_ascii(
        ref.handle, _dptr(ascii, torch.uint8, "ascii", n_reads * ascii_stride if m > 0 else 0), ascii_stride,
        n_reads, m, _dptr(pair_read, torch.int32, "pair_read"), _dptr(pair_off, torch.int32, "pair_off", n),
        pe, fixed_e, n, count_mode, flags, _dptr(accept, torch.uint8, "accept", n),
        None if result_byte else _dptr(edits, torch.int16, "edits", n),
        _dptr(err_count, torch.int32, "err_count", 1), _stream(stream)))
    return accept, (None if result_byte else edits)


def sliced_supported(m: int, e: int) -> bool:
    """Whether gk_filter_sliced filters read length m at threshold e."""
    return 1 <= m <= GK_SLICED_MAX_LEN and min(int(e), m - 1) <= GK_SLICED_MAX_SHIFT


def gk_sliced_bytes(n_pairs: int, m: int) -> int:
    return int(lib().gk_sliced_bytes(n_pairs, m))


def gk_slice(ref: Reference, reads: torch.Tensor, stride_words: int, n_reads: int,
             read_nflag: torch.Tensor | None, m: int, pair_read: torch.Tensor, pair_off: torch.Tensor,
             out: torch.Tensor | None = None, err_count: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Gather and transpose a batch of pairs into a sliced buffer (gk_slice);
    returns the buffer (a uint8 CUDA tensor, ``out`` when given)."""
    n = pair_read.numel()
    nbytes = gk_sliced_bytes(n, m) if n else 0
    if out is None:
        out = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=pair_read.device)
    if reads.numel() < n_reads * stride_words * 2:
        raise ValueError("reads holds fewer than n_reads * stride_words * 2 words")
    _check(lib().gk_slice(
        ref.handle, _dptr(reads, torch.int32, "reads"), stride_words, n_reads,
        _dptr(read_nflag, torch.uint8, "read_nflag", n_reads), m,
        _dptr(pair_read, torch.int32, "pair_read"), _dptr(pair_off, torch.int32, "pair_off", n), n,
        _dptr(out, torch.uint8, "out", nbytes), out.numel(), _dptr(err_count, torch.int32, "err_count", 1),
        _stream(stream)))
    return out


def gk_filter_sliced(sliced: torch.Tensor, n_pairs: int, m: int, e: int, count_mode: int = GK_COUNT_RUNS4,
                     flags: int = 0, accept: torch.Tensor | None = None, edits: torch.Tensor | None = None,
                     stream=None):
    """Filter a sliced batch at threshold ``e`` (gk_filter_sliced).  Returns
    (accept uint8, edits int16 read as uint16), or (result bytes, None) with
    GK_FLAG_RESULT_BYTE, as gk_filter."""
    dev = sliced.device
    result_byte = bool(flags & GK_FLAG_RESULT_BYTE)
    if accept is None:
        accept = torch.empty(n_pairs, dtype=torch.uint8, device=dev)
    if edits is None and not result_byte:
        edits = torch.empty(n_pairs, dtype=torch.int16, device=dev)
    _check(lib().gk_filter_sliced(
        _dptr(sliced, torch.uint8, "sliced"), sliced.numel(), n_pairs, m, int(e), count_mode, flags,
        _dptr(accept, torch.uint8, "accept", n_pairs),
        None if result_byte else _dptr(edits, torch.int16, "edits", n_pairs), _stream(stream)))
    return accept, (None if result_byte else edits)


def gk_filter_sliced_sweep(sliced: torch.Tensor, n_pairs: int, m: int, e_lo: int, e_hi: int,
                           count_mode: int = GK_COUNT_RUNS4, flags: int = 0, accept: torch.Tensor | None = None,
                           edits: torch.Tensor | None = None, out_stride: int | None = None,
                           err_count: torch.Tensor | None = None, stream=None):
    """Filter a sliced batch at every threshold e_lo..e_hi
    (gk_filter_sliced_sweep).  Returns (accept, edits) as views of shape
    (e_hi - e_lo + 1, n_pairs) over the threshold-major buffers (rows
    out_stride elements apart), or (result bytes, None) with
    GK_FLAG_RESULT_BYTE; row e - e_lo holds threshold e's results."""
    dev = sliced.device
    result_byte = bool(flags & GK_FLAG_RESULT_BYTE)
    n_e = int(e_hi) - int(e_lo) + 1
    if out_stride is None:
        out_stride = -(-n_pairs // 16) * 16
    need = (n_e - 1) * out_stride + n_pairs if n_e > 0 else 0
    if accept is None:
        accept = torch.empty(max(need, n_e * out_stride, 1), dtype=torch.uint8, device=dev)
    if edits is None and not result_byte:
        edits = torch.empty(max(need, n_e * out_stride, 1), dtype=torch.int16, device=dev)
    _check(lib().gk_filter_sliced_sweep(
        _dptr(sliced, torch.uint8, "sliced"), sliced.numel(), n_pairs, m, int(e_lo), int(e_hi), count_mode,
        flags, _dptr(accept, torch.uint8, "accept", need),
        None if result_byte else _dptr(edits, torch.int16, "edits", need), out_stride,
        _dptr(err_count, torch.int32, "err_count", 1), _stream(stream)))
    rows = lambda t: t.as_strided((n_e, n_pairs), (out_stride, 1))  # noqa: E731
    return rows(accept), (None if result_byte else rows(edits))


def gk_filter_batched_workspace(n_pairs: int) -> int:
    return int(lib().gk_filter_batched_workspace(n_pairs))


def gk_filter_batched(ref: Reference, reads: torch.Tensor, stride_words: int, n_reads: int,
                      read_len: torch.Tensor, read_nflag: torch.Tensor | None, pair_read: torch.Tensor,
                      pair_off: torch.Tensor, e, tiling: Tiling, workspace: torch.Tensor,
                      count_mode: int = GK_COUNT_RUNS4, flags: int = 0, accept: torch.Tensor | None = None,
                      edits: torch.Tensor | None = None, err_count: torch.Tensor | None = None, stream=None):
    """Filter pairs of mixed read lengths in one persistent launch
    (gk_filter_batched).  ``read_len`` is an int16 CUDA tensor (uint16
    values); ``workspace`` a uint8 CUDA tensor of at least
    gk_filter_batched_workspace(n) bytes.  Returns (accept, edits); with
    GK_FLAG_RESULT_BYTE, (result bytes, None) unless ``edits`` is given."""
    n = pair_read.numel()
    dev = pair_read.device
    if accept is None:
        accept = torch.empty(n, dtype=torch.uint8, device=dev)
    if edits is None and not flags & GK_FLAG_RESULT_BYTE:
        edits = torch.empty(n, dtype=torch.int16, device=dev)
    if reads.numel() < n_reads * stride_words * 2:
        raise ValueError("reads holds fewer than n_reads * stride_words * 2 words")
    pe, fixed_e = (_dptr(e, torch.uint8, "e", n), 0) if isinstance(e, torch.Tensor) else (None, int(e))
    _check(lib().gk_filter_batched(
        ref.handle, _dptr(reads, torch.int32, "reads"), stride_words, n_reads,
        _dptr(read_len, torch.int16, "read_len", n_reads), _dptr(read_nflag, torch.uint8, "read_nflag", n_reads),
        _dptr(pair_read, torch.int32, "pair_read"), _dptr(pair_off, torch.int32, "pair_off", n), pe, fixed_e, n,
        count_mode, flags, ctypes.byref(tiling), _dptr(workspace, torch.uint8, "workspace"), workspace.numel(),
        _dptr(accept, torch.uint8, "accept", n), _dptr(edits, torch.int16, "edits", n),
        _dptr(err_count, torch.int32, "err_count", 1), _stream(stream)))
    return accept, edits


def gk_filter_batched_noalloc(ref: Reference, reads: torch.Tensor, stride_words: int, n_reads: int,
                              read_len: torch.Tensor, read_nflag: torch.Tensor | None, pair_read: torch.Tensor,
                              pair_off: torch.Tensor, e, tiling: Tiling, accept: torch.Tensor,
                              edits: torch.Tensor, count_mode: int = GK_COUNT_RUNS4, flags: int = 0,
                              err_count: torch.Tensor | None = None, stream=None):
    """gk_filter_batched without a workspace, for callers that must not
    allocate device memory while filtering: the library keeps a fixed scratch
    array of its own (at most GK_NOALLOC_MAX_PAIRS pairs per call; calls that
    overlap on the GPU race on it).  The caller provides the outputs."""
    n = pair_read.numel()
    if reads.numel() < n_reads * stride_words * 2:
        raise ValueError("reads holds fewer than n_reads * stride_words * 2 words")
    pe, fixed_e = (_dptr(e, torch.uint8, "e", n), 0) if isinstance(e, torch.Tensor) else (None, int(e))
    _check(lib().gk_filter_batched_noalloc(
        ref.handle, _dptr(reads, torch.int32, "reads"), stride_words, n_reads,
        _dptr(read_len, torch.int16, "read_len", n_reads), _dptr(read_nflag, torch.uint8, "read_nflag", n_reads),
        _dptr(pair_read, torch.int32, "pair_read"), _dptr(pair_off, torch.int32, "pair_off", n), pe, fixed_e, n,
        count_mode, flags, ctypes.byref(tiling), _dptr(accept, torch.uint8, "accept", n),
        _dptr(edits, torch.int16, "edits", n), _dptr(err_count, torch.int32, "err_count", 1), _stream(stream)))
    return accept, edits


GK_SEG_NO_N = 0x10000


def gk_expand_pairs(pair_read: torch.Tensor, pair_e: torch.Tensor, read_start: torch.Tensor,
                    seg_read_end: torch.Tensor, seg_pair_end: torch.Tensor, seg_read_slot: torch.Tensor,
                    seg_start_base: torch.Tensor, seg_e: torch.Tensor, n_reads: int | None = None,
                    seg_read_info: torch.Tensor | None = None, read_len: torch.Tensor | None = None,
                    read_nflag: torch.Tensor | None = None, stream=None):
    """Per-pair read ids (read-buffer rows) and thresholds of the pairs of
    n_segs requests from their reads' start offsets (gk_expand_pairs):
    segment i owns reads [seg_read_end[i-1], seg_read_end[i]) at rows
    seg_read_slot[i] + k and pairs [seg_pair_end[i-1], seg_pair_end[i]);
    read_start[row] - seg_start_base[i] is the read's first pair within its
    request.  With ``seg_read_info`` (int32: a shared read length in bits
    0..15, GK_SEG_NO_N) the rows' lengths and N flags of such segments are
    written too.  int64 / int32 / uint8 CUDA tensors as in gk.h."""
    n_segs = seg_read_end.numel()
    n = pair_read.numel()
    if n_reads is None:
        n_reads = int(seg_read_end[-1].item()) if n_segs else 0
    _check(lib().gk_expand_pairs(_dptr(pair_read, torch.int32, "pair_read"), _dptr(pair_e, torch.uint8, "pair_e", n),
                                 n, _dptr(read_start, torch.int32, "read_start"),
                                 _dptr(seg_read_end, torch.int64, "seg_read_end"),
                                 _dptr(seg_pair_end, torch.int64, "seg_pair_end", n_segs),
                                 _dptr(seg_read_slot, torch.int64, "seg_read_slot", n_segs),
                                 _dptr(seg_start_base, torch.int32, "seg_start_base", n_segs),
                                 _dptr(seg_e, torch.uint8, "seg_e", n_segs),
                                 _dptr(seg_read_info, torch.int32, "seg_read_info", n_segs),
                                 _dptr(read_len, torch.int16, "read_len"), _dptr(read_nflag, torch.uint8, "read_nflag"),
                                 n_segs, n_reads, _stream(stream)))


def gk_rebase_pairs(pair_read: torch.Tensor, seg_end: torch.Tensor, seg_delta: torch.Tensor,
                    pair_e: torch.Tensor | None = None, seg_e: torch.Tensor | None = None, stream=None):
    """Add request i's offset seg_delta[i] to the read ids of its pairs
    [seg_end[i-1], seg_end[i]) in place and, if ``pair_e`` is given, write its
    threshold seg_e[i] into them (gk_rebase_pairs)."""
    n_segs = seg_end.numel()
    n = pair_read.numel()
    _check(lib().gk_rebase_pairs(_dptr(pair_read, torch.int32, "pair_read"),
                                 _dptr(pair_e, torch.uint8, "pair_e", n), n,
                                 _dptr(seg_end, torch.int64, "seg_end"), _dptr(seg_delta, torch.int64, "seg_delta", n_segs),
                                 _dptr(seg_e, torch.uint8, "seg_e", n_segs), n_segs, _stream(stream)))


H2D, D2H, D2D = 1, 2, 3


def gk_copy_many(dst: np.ndarray, src: np.ndarray, nbytes: np.ndarray, kind: int, stream=None):
    """Enqueue len(dst) copies (uint64 address arrays) with one call."""
    dst = np.ascontiguousarray(dst, np.uint64)
    src = np.ascontiguousarray(src, np.uint64)
    nbytes = np.ascontiguousarray(nbytes, np.uint64)
    _check(lib().gk_copy_many(dst.ctypes.data, src.ctypes.data, nbytes.ctypes.data, dst.shape[0], kind,
                              _stream(stream)))


def gather_chunks(dst: np.ndarray, src: np.ndarray, nbytes: np.ndarray, chunk: int = GK_GATHER_MAX_BYTES):
    """Split copies (uint64 address / size arrays) into gk_gather entries of
    at most ``chunk`` bytes; returns the (dst, src, bytes) entry arrays."""
    dst = np.asarray(dst, np.uint64)
    src = np.asarray(src, np.uint64)
    nb = np.asarray(nbytes, np.uint64)
    keep = nb > 0
    dst, src, nb = dst[keep], src[keep], nb[keep]
    k = ((nb + np.uint64(chunk - 1)) // np.uint64(chunk)).astype(np.int64)
    first = np.repeat(np.cumsum(k) - k, k)
    which = np.repeat(np.arange(k.shape[0]), k)
    off = (np.arange(int(k.sum()), dtype=np.int64) - first).astype(np.uint64) * np.uint64(chunk)
    size = np.minimum(nb[which] - off, np.uint64(chunk))
    return dst[which] + off, src[which] + off, size


def gk_gather(dst: torch.Tensor, src: torch.Tensor, nbytes: torch.Tensor, n: int, stream=None):
    """One kernel doing n copies (gk_gather).  The three tables are int64
    tensors the device can read (CUDA, or pinned host), left unchanged until
    the kernel has run; entries come from gather_chunks."""
    for t, name in ((dst, "dst"), (src, "src"), (nbytes, "nbytes")):
        if t.dtype != torch.int64 or not t.is_contiguous() or t.numel() < n:
            raise ValueError(f"gk_gather: {name} must be a contiguous int64 tensor of >= n entries")
        if not (t.is_cuda or t.is_pinned()):
            raise ValueError(f"gk_gather: {name} must be device memory or pinned host memory")
    _check(lib().gk_gather(dst.data_ptr(), src.data_ptr(), nbytes.data_ptr(), int(n), _stream(stream)))


GK_PROBE_LOP3, GK_PROBE_SHF, GK_PROBE_MIX = 0, 1, 2


def _hptr(x, dtypes, name: str, numel: int) -> int | None:
    """Address of a contiguous host buffer (numpy array or CPU tensor) of one
    of `dtypes` holding at least `numel` elements."""
    if numel == 0:
        return None
    if isinstance(x, torch.Tensor):
        if x.is_cuda or not x.is_contiguous() or x.dtype not in dtypes:
            raise TypeError(f"{name} must be a contiguous host tensor of {dtypes}")
        n = x.numel()
        ptr = x.data_ptr()
    elif isinstance(x, np.ndarray):  # either signedness of the element width
        width = torch.empty(0, dtype=dtypes[0]).element_size()
        if not x.flags.c_contiguous or x.dtype.kind not in "iu" or x.dtype.itemsize != width:
            raise TypeError(f"{name} must be a contiguous host array of {width}-byte integers")
        n = x.size
        ptr = x.ctypes.data
    else:
        raise TypeError(f"{name} must be a numpy array or a CPU tensor")
    if n < numel:
        raise ValueError(f"{name} holds {n} elements, needs {numel}")
    return ptr


class Pipe:
    """gk_pipe_*: a streamed host pipeline over fixed-length reads.  Each
    ``submit`` enqueues one batch (host ASCII reads and pairs in, results of
    every threshold out, threshold-major) and returns its ticket; ``wait``
    blocks until that batch's results are in its host buffers.  Host buffers
    should be page-locked (``tensor.pin_memory()``) for the copies to overlap
    the filtering; the pipe keeps them referenced until they are waited on."""

    def __init__(self, ref: Reference, max_reads: int, ascii_stride: int, read_len: int, max_pairs: int,
                 thresholds, count_mode: int = GK_COUNT_RUNS4, flags: int = 0, n_slots: int = 3):
        th = np.ascontiguousarray(np.asarray(thresholds), dtype=np.uint8)
        desc = PipeDesc(max_reads, ascii_stride, read_len, max_pairs, th.size, th.ctypes.data, count_mode, flags,
                        n_slots)
        h = ctypes.c_void_p()
        _check(lib().gk_pipe_create(ref.handle, ctypes.byref(desc), ctypes.byref(h)))
        self.handle = h.value
        self.ref = ref
        self.ascii_stride = ascii_stride
        self.n_thresholds = int(th.size)
        self.result_byte = bool(flags & GK_FLAG_RESULT_BYTE)
        self.read_starts = bool(flags & GK_PIPE_READ_STARTS)
        self._held = {}

    def submit(self, ascii, n_reads: int, pair_read, pair_off, accept_out, edits_out) -> int:
        """pair_read: a read id per pair, or with GK_PIPE_READ_STARTS one
        start per read (read i's pairs are pair_read[i] .. pair_read[i+1]-1)."""
        n_pairs = int(pair_off.shape[0]) if pair_off is not None else 0
        i32 = (torch.int32,)
        n_link = n_reads if self.read_starts else n_pairs
        args = (_hptr(ascii, (torch.uint8,), "ascii", n_reads * self.ascii_stride), n_reads,
                _hptr(pair_read, i32, "pair_read", n_link), _hptr(pair_off, i32, "pair_off", n_pairs), n_pairs,
                _hptr(accept_out, (torch.uint8,), "accept_out", self.n_thresholds * n_pairs),
                None if self.result_byte else
                _hptr(edits_out, (torch.int16,), "edits_out", self.n_thresholds * n_pairs))
        t = ctypes.c_uint64()
        _check(lib().gk_pipe_submit(self.handle, *args, ctypes.byref(t)))
        self._held[t.value] = (ascii, pair_read, pair_off, accept_out, edits_out)
        return t.value

    def wait(self, ticket: int):
        _check(lib().gk_pipe_wait(self.handle, ticket))
        for k in [k for k in self._held if k <= ticket]:
            del self._held[k]

    def close(self):
        if self.handle:
            lib().gk_pipe_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def gk_probe_alu(kind: int, iters: int, blocks: int, threads: int, sink: torch.Tensor, stream=None):
    """Enqueue the integer-throughput probe (include/gk_probe.h); issues
    blocks * threads * iters * 64 ops."""
    _check(lib().gk_probe_alu(kind, iters, blocks, threads, _dptr(sink, torch.int32, "sink", 1),
                              _stream(stream)))


def version() -> int:
    return lib().gk_version()
