"""The suffix sort's key arithmetic (csrc/suffix_sort.cu) run on the CPU.

ConstructSA (Section 3) sorts each suffix first by a 63-bit key: its first H
codes (H = 29 two-bit or 14 four-bit codes), zeroed at and past its
terminator, above a length field (min(len, H), or 29 when the suffix has at
least H symbols).  The bucket split then numbers the buckets (the first P
codes p, l = min(len, P)) densely, in key order, by a closed form (Legendre's
formula for base 4; its base-sigma form for 4-bit codes).

Pinned here against plain definitions, not against the closed forms:
* every valid bucket (p, l) -- the codes of p at and past l are zero -- is
  listed and ordered as the keys order them, and each must get its index in
  that list (exhaustively: 5,592,405 buckets for 2-bit codes; for 4-bit
  codes sigma = 7, 12 and 16, with the longest bucket prefix whose numbers
  fit 24 bits);
* keys read from random packed text with terminators must equal keys built
  symbol by symbol from the unpacked codes.
The device functions are cut out of the CUDA source and compiled for the
host with tests/emu/cuda_emu.h.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "keys_emulation.cpp")
kH0 = 29
kShortFlag = 0x80000000
kDigitBits = 24


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("keysemu")
    src = open(os.path.join(CSRC, "suffix_sort.cu")).read()
    (d / "constants.inc").write_text(_cut(src, "constexpr int kThreads = 256;", "// Key geometry per code width"))
    (d / "keys.inc").write_text(_cut(src, "// Key geometry per code width",
                                     "// Element of block position t for the bucket split"))
    lib = d / "libkeysemu.so"
    subprocess.check_call(["g++", "-O2", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    L.emu_bucket_digit.argtypes = [U64, P, P]
    L.emu_bucket_digit_sigma.argtypes = [U64, P, U32, U32, P]
    L.emu_keys.argtypes = [I, P, U64, P, U64, U64, P, P, P]
    for f in (L.emu_bucket_digit, L.emu_bucket_digit_sigma, L.emu_keys):
        f.restype = I
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def valid_buckets(base: int, P: int):
    """Every bucket (p, l), l <= P, whose codes at and past l are zero, in
    the order of the keys that fall in them: by the P codes p (read as a
    base-`base` number, first code most significant), then by l."""
    ps, ls = [], []
    for l in range(P + 1):
        step = base ** (P - l)  # codes l .. P-1 zero: p a multiple of base^(P - l)
        p = np.arange(0, base ** P, step, dtype=np.int64)
        ps.append(p)
        ls.append(np.full(p.size, l, np.int8))
    p, l = np.concatenate(ps), np.concatenate(ls)
    order = np.lexsort((l, p))
    return p[order], l[order].astype(np.int64)


def packed_head(p, base, P, kb):
    """The P codes of p (base-`base` digits, first code most significant)
    packed kb bits each, first code in the highest bits."""
    head = np.zeros(p.size, np.uint64)
    x = p.copy()
    for q in range(P):  # least significant digit = last code
        head |= (x % base).astype(np.uint64) << np.uint64(kb * q)
        x //= base
    return head


def make_keys(head, l, H, kb, P, symbols, rng):
    """Keys whose first P codes are `head` and whose length is l (< P) or at
    least P.  A short bucket's key has only zeros after its l codes; a long
    one gets random further codes and a length field of P .. H - 1 (codes
    from there on zero) or kH0 (at least H symbols)."""
    n = head.size
    long_ = l == P
    fl = rng.integers(P, H + 1, size=n)
    field = np.where(long_, np.where(fl == H, kH0, fl), l)
    ncodes = np.where(long_, fl, l)  # symbols before the terminator (H: at least H)
    key = head.copy()
    for q in range(P, H):
        c = rng.integers(0, symbols, size=n).astype(np.uint64)
        key = (key << np.uint64(kb)) | np.where(q < ncodes, c, np.uint64(0))
    return (key << np.uint64(5)) | field.astype(np.uint64)


def test_bucket_numbers_two_bit_codes_are_dense_and_ordered(emu):
    P, H = 11, 29
    rng = np.random.default_rng(5)
    p, l = valid_buckets(4, P)
    assert p.size == sum(4 ** k for k in range(P + 1)) == 5_592_405
    keys = make_keys(packed_head(p, 4, P, 2), l, H, 2, P, 4, rng)
    out = np.empty(p.size, np.uint32)
    assert emu.emu_bucket_digit(p.size, _p(keys), _p(out)) == 0
    want = np.arange(p.size, dtype=np.uint32) | np.where(l < P, kShortFlag, 0).astype(np.uint32)
    assert np.array_equal(out, want)
    assert int((out & ~np.uint32(kShortFlag)).max()) < 1 << kDigitBits


def bucket_codes_for(sigma: int) -> int:
    """The longest bucket prefix (at most H = 14 codes) whose valid buckets,
    sum of sigma^l over l <= P, all get numbers below 2^24."""
    P = 1
    while P + 1 <= 14 and sum(sigma ** k for k in range(P + 2)) <= 1 << kDigitBits:
        P += 1
    return P


@pytest.mark.parametrize("sigma", [7, 12, 16])
def test_bucket_numbers_base_sigma_are_dense_and_ordered(emu, sigma):
    H = 14
    P = bucket_codes_for(sigma)
    rng = np.random.default_rng(sigma)
    p, l = valid_buckets(sigma, P)
    keys = make_keys(packed_head(p, sigma, P, 4), l, H, 4, P, sigma, rng)
    out = np.empty(p.size, np.uint32)
    assert emu.emu_bucket_digit_sigma(p.size, _p(keys), sigma, P, _p(out)) == 0
    want = np.arange(p.size, dtype=np.uint32) | np.where(l < P, kShortFlag, 0).astype(np.uint32)
    assert np.array_equal(out, want)
    assert int((out & ~np.uint32(kShortFlag)).max()) < 1 << kDigitBits


def pack(codes, kb):
    """Codes into 32-bit words, first code in the most significant bits."""
    per = 32 // kb
    n = codes.size
    words = np.zeros((n + per - 1) // per, np.uint64)
    for j in range(per):
        part = codes[j::per].astype(np.uint64)
        words[:part.size] |= part << np.uint64(32 - kb * (j + 1))
    return words.astype(np.uint32)


@pytest.mark.parametrize("kb,sigma", [(2, 4), (4, 5), (4, 16)])
def test_keys_from_packed_text(emu, kb, sigma):
    H = 29 if kb == 2 else 14
    rng = np.random.default_rng(100 + kb + sigma)
    # reads of mixed lengths (0 .. 3H) each followed by a terminator
    lens = rng.integers(0, 3 * H, size=400)
    lens[:5] = [0, 1, H - 1, H, H + 1]
    n = int(lens.sum() + lens.size)
    codes = rng.integers(0, sigma, size=n)
    term = np.zeros(n, bool)
    term[np.cumsum(lens + 1) - 1] = True
    # the packed text's code at a terminator is arbitrary: the key must not see it
    text = pack(codes, kb)
    bits = np.zeros((n + 31) // 32, np.uint32)
    for j in np.nonzero(term)[0]:
        bits[j >> 5] |= np.uint32(1 << (j & 31))
    pos = np.arange(n, dtype=np.uint64)
    init = np.empty(n, np.uint64)
    with_len = np.empty(n, np.uint64)
    assert emu.emu_keys(kb, _p(text), text.size, _p(bits), bits.size, n, _p(pos), _p(init), _p(with_len)) == 0
    # expected, symbol by symbol
    next_term = np.empty(n, np.int64)
    nxt = n
    for j in range(n - 1, -1, -1):
        if term[j]:
            nxt = j
        next_term[j] = nxt
    for t in range(n):
        ln = int(next_term[t] - t)
        field = ln if ln < H else kH0
        k = 0
        for q in range(H):
            c = int(codes[t + q]) if q < ln and t + q < n else 0
            k = (k << kb) | c
        want = (k << 5) | field
        assert int(init[t]) == want, (t, ln)
    assert np.array_equal(with_len, init)
