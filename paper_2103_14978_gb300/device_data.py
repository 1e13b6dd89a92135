"""Moves a workload onto the device: reads are uploaded as ASCII and packed by
the library's device encoder (gk_encode), pairs become int32 tensors holding
uint32 values.  Host-side marshalling only."""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import gk


@dataclasses.dataclass
class DeviceReads:
    packed: torch.Tensor       # int32 [n_reads * stride_words * 2]
    nflag: torch.Tensor        # uint8 [n_reads]
    stride_words: int
    n_reads: int
    read_len: np.ndarray       # host copy of the lengths (uint16)


@dataclasses.dataclass
class DevicePairs:
    pair_read: torch.Tensor    # int32 (uint32 values)
    pair_off: torch.Tensor     # int32 (uint32 values)
    pair_e: torch.Tensor | None  # uint8
    n_pairs: int


def as_i32(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32))


def as_i16(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16))


def upload_reads(reads_ascii: np.ndarray, read_len: np.ndarray, stride: int, device="cuda",
                 stride_words: int | None = None, stream=None) -> DeviceReads:
    n = int(read_len.shape[0])
    fixed = bool(n) and bool((read_len == read_len[0]).all())
    sw = stride_words or gk.words_for(int(read_len.max()) if n else 1)
    asc = torch.from_numpy(np.ascontiguousarray(reads_ascii, dtype=np.uint8)).to(device)
    lens = None if fixed else as_i16(read_len).to(device)
    packed, nflag = gk.gk_encode(asc, n, stride, lens=lens, fixed_len=int(read_len[0]) if fixed else 0,
                                 stride_words=sw, stream=stream)
    return DeviceReads(packed, nflag, sw, n, np.asarray(read_len, np.uint16))


def upload_pairs(pair_read: np.ndarray, pair_off: np.ndarray, pair_e: np.ndarray | None,
                 device="cuda") -> DevicePairs:
    return DevicePairs(as_i32(pair_read).to(device), as_i32(pair_off).to(device),
                       None if pair_e is None else torch.from_numpy(np.ascontiguousarray(pair_e, np.uint8)).to(device),
                       int(pair_read.shape[0]))


def edits_u16(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint16)
