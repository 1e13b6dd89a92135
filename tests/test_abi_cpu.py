"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every symbol include/*.h declares, rejects bad
arguments before touching the device, and its host encoder writes the 2-bit
code of Sec. 2.1 (A=00 C=01 G=10 T=11)."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def libgk():
    from paper_2103_14978_gb300 import build, gk

    build.build()
    return gk


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(gk_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_declared_symbols(libgk):
    names = declared_symbols()
    assert {"gk_encode", "gk_load_reference", "gk_filter", "gk_free_reference"} <= set(names)
    L = ctypes.CDLL(libgk.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", libgk.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gk_\w+)", out))
    assert set(names) <= exported
    # the binding wraps exactly what the header declares (besides probes)
    assert set(libgk.exported_symbols()) <= set(names)


def test_library_is_sm103a(libgk):
    out = subprocess.run(["cuobjdump", "--list-elf", libgk.LIB_PATH], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_version_and_error_reporting(libgk):
    L = libgk.lib()
    assert L.gk_version() >= 100
    # null reference handle: rejected on the host, message set
    rc = L.gk_filter(None, None, 1, 1, None, 100, None, None, None, 2, 10, 0, 0, None, None, None, None)
    assert rc == libgk.GK_EINVAL
    assert b"reference" in L.gk_last_error()
    rc = L.gk_load_reference(None, 10, 0, None, ctypes.byref(ctypes.c_void_p()))
    assert rc == libgk.GK_EINVAL
    # zero pairs / zero sequences enqueue nothing and succeed
    assert L.gk_encode(None, 1, None, 1, 0, None, 1, None, 0, None) == libgk.GK_OK


def test_encode_argument_checks(libgk):
    L = libgk.lib()
    buf = np.zeros(64, np.uint8)
    out = np.zeros(64, np.uint32)
    fl = np.zeros(4, np.uint8)
    p = lambda a: a.ctypes.data
    assert L.gk_encode(p(buf), 8, None, 600, 1, p(out), 1, p(fl), 0, None) == libgk.GK_ERANGE
    assert L.gk_encode(p(buf), 8, None, 16, 1, p(out), 1, p(fl), 0, None) == libgk.GK_EINVAL  # len > stride
    assert L.gk_encode(p(buf), 40, None, 40, 1, p(out), 1, p(fl), 0, None) == libgk.GK_EINVAL  # 1 word < 40
    assert L.gk_encode(p(buf), 8, None, 8, 1, p(out), 0, p(fl), 0, None) == libgk.GK_EINVAL
    assert L.gk_encode(p(buf), 8, None, 8, 1, p(out), 1, None, 0, None) == libgk.GK_EINVAL


def _decode(packed, n, stride_words, lens):
    """Read the planes back as bases with the paper's code table."""
    out = []
    for s in range(n):
        chars = []
        for i in range(int(lens[s])):
            w, b = divmod(i, 32)
            hi = (int(packed[(s * stride_words + w) * 2]) >> b) & 1
            lo = (int(packed[(s * stride_words + w) * 2 + 1]) >> b) & 1
            chars.append("ACGT"[2 * hi + lo])
        out.append("".join(chars))
    return out


def test_host_encoder_matches_code_table(libgk):
    rng = np.random.default_rng(1)
    n, stride = 300, 150
    lens = rng.integers(0, stride + 1, n).astype(np.uint16)
    asc = rng.choice(np.frombuffer(b"ACGTacgt", np.uint8), n * stride)
    n_pos = rng.integers(0, n * stride, 40)
    asc[n_pos] = ord("N")
    sw = 5
    packed = np.full(n * sw * 2, 0xDEADBEEF, np.uint32)
    nflag = np.full(n, 7, np.uint8)
    rc = libgk.lib().gk_encode(asc.ctypes.data, stride, lens.ctypes.data, 0, n, packed.ctypes.data, sw,
                               nflag.ctypes.data, 0, None)
    assert rc == 0
    got = _decode(packed, n, sw, lens)
    for s in range(n):
        raw = bytes(asc[s * stride: s * stride + lens[s]]).decode().upper()
        has_n = "N" in raw
        assert nflag[s] == int(has_n)
        assert got[s] == raw.replace("N", "A")
        # bits past the length are zero, in every word of the stride
        for i in range(int(lens[s]), sw * 32):
            w, b = divmod(i, 32)
            assert (packed[(s * sw + w) * 2] >> b) & 1 == 0
            assert (packed[(s * sw + w) * 2 + 1] >> b) & 1 == 0


def test_pipe_rejects_bad_arguments_on_host(libgk):
    L = libgk.lib()
    h = ctypes.c_void_p()
    assert L.gk_pipe_create(None, None, ctypes.byref(h)) == libgk.GK_EINVAL
    assert b"gk_pipe_create" in L.gk_last_error()
    t = ctypes.c_uint64()
    assert L.gk_pipe_submit(None, None, 0, None, None, 0, None, None, ctypes.byref(t)) == libgk.GK_EINVAL
    assert L.gk_pipe_wait(None, 0) == libgk.GK_EINVAL
    L.gk_pipe_destroy(None)  # ignored


def test_expand_pairs_host_checks(libgk):
    """gk_expand_pairs: nothing to do for no pairs; a missing table is
    rejected before any device work."""
    L = libgk.lib()
    assert L.gk_expand_pairs(None, None, 0, None, None, None, None, None, None, None, None, None, 0, 0, None) == libgk.GK_OK
    assert L.gk_expand_pairs(None, None, 10, None, None, None, None, None, None, None, None, None, 1, 3, None) == libgk.GK_EINVAL
    assert b"gk_expand_pairs" in L.gk_last_error()


def test_sliced_sizes_and_host_checks(libgk):
    """gk_sliced_bytes follows the documented layout; gk_slice and
    gk_filter_sliced reject bad arguments before any device work."""
    L = libgk.lib()
    for n, m in ((1, 1), (31, 100), (32, 100), (33, 150), (1024, 250), (20_000_000, 100), (5, 255)):
        groups = -(-n // 32)
        pitch = -(-groups // 32) * 32
        assert L.gk_sliced_bytes(n, m) == (2 * (m + 24) + 1) * pitch * 8 + 16, (n, m)
    assert L.gk_sliced_bytes(0, 100) == 0 and L.gk_sliced_bytes(10, 0) == 0 and L.gk_sliced_bytes(10, 256) == 0
    buf = ctypes.c_void_p(16)  # never dereferenced: every call below fails its host checks
    cap = L.gk_sliced_bytes(64, 100)
    E, R = libgk.GK_EINVAL, libgk.GK_ERANGE
    assert L.gk_filter_sliced(buf, cap, 64, 0, 3, 0, 0, buf, buf, None) == R  # m = 0
    assert L.gk_filter_sliced(buf, cap, 64, 256, 3, 0, 0, buf, buf, None) == R  # m > 255
    assert L.gk_filter_sliced(buf, cap, 64, 100, 16, 0, 0, buf, buf, None) == R  # min(e, m-1) > 15
    assert L.gk_filter_sliced(buf, cap, 64, 100, 3, 0, libgk.GK_FLAG_NO_EDGE_FIX, buf, buf, None) == E
    assert L.gk_filter_sliced(buf, cap, 64, 100, 3, 7, 0, buf, buf, None) == E  # count mode
    assert L.gk_filter_sliced(buf, cap - 8, 64, 100, 3, 0, 0, buf, buf, None) == E  # buffer too small
    assert L.gk_filter_sliced(None, cap, 64, 100, 3, 0, 0, buf, buf, None) == E
    assert L.gk_filter_sliced(buf, cap, 64, 100, 253, 0, libgk.GK_FLAG_RESULT_BYTE, buf, None, None) == R
    assert b"gk_filter_sliced" in L.gk_last_error()
    assert L.gk_filter_sliced(buf, cap, 0, 100, 3, 0, 0, None, None, None) == libgk.GK_OK  # nothing to do
    assert L.gk_slice(None, None, 4, 1, None, 100, None, None, 64, buf, cap, None, None) == E  # no reference
    fs = L.gk_filter_sweep
    assert fs(None, None, 4, 1, None, 100, buf, buf, 0, 3, 64, 0, 0, buf, buf, 64, None, None) == E  # no reference
    sw = L.gk_filter_sliced_sweep
    assert sw(buf, cap, 64, 100, 0, 16, 0, 0, buf, buf, 64, None, None) == R  # min(e_hi, m-1) > 15
    assert sw(buf, cap, 64, 100, 5, 4, 0, 0, buf, buf, 64, None, None) == E  # e_lo > e_hi
    assert sw(buf, cap, 64, 100, 0, 256, 0, 0, buf, buf, 64, None, None) == R
    assert sw(buf, cap, 64, 0, 0, 3, 0, 0, buf, buf, 64, None, None) == R  # m = 0
    assert sw(buf, cap, 64, 100, 0, 10, 0, 0, buf, buf, 63, None, None) == E  # out_stride < n_pairs
    assert sw(buf, cap - 8, 64, 100, 0, 10, 0, 0, buf, buf, 64, None, None) == E  # buffer too small
    assert sw(buf, cap, 64, 100, 0, 10, 0, libgk.GK_FLAG_NO_EDGE_FIX, buf, buf, 64, None, None) == E
    assert sw(buf, cap, 64, 100, 0, 10, 9, 0, buf, buf, 64, None, None) == E  # count mode
    assert sw(None, cap, 64, 100, 0, 10, 0, 0, buf, buf, 64, None, None) == E
    assert sw(buf, cap, 64, 100, 0, 10, 0, 0, buf, None, 64, None, None) == E  # edits needed
    assert sw(buf, cap, 64, 20, 0, 253, 0, libgk.GK_FLAG_RESULT_BYTE, buf, None, 64, None, None) == R
    assert b"gk_filter_sliced_sweep" in L.gk_last_error()
    assert sw(buf, cap, 0, 100, 0, 10, 0, 0, None, None, 0, None, None) == libgk.GK_OK  # nothing to do
    assert libgk.sliced_supported(100, 15) and not libgk.sliced_supported(100, 16)
    assert libgk.sliced_supported(5, 255) and not libgk.sliced_supported(17, 255)  # min(e, m-1)
    assert not libgk.sliced_supported(0, 0) and not libgk.sliced_supported(256, 0)
