"""The read packing (csrc/pack.cu) run on the CPU.

An append's reads become the text T = S_0 $_0 S_1 $_1 ... (Section 2): read
j's symbol k sits at position offsets[j] + j + k and its terminator at
offsets[j+1] + j.  Each symbol is stored as its index in the alphabet, in
2-bit codes (16 per 32-bit word) or 4-bit codes (8 per word), the first
position in the most significant bits; the terminator positions are the
set bits of a bitmap (bit q of word w for position 32 w + q) and hold code
0 in the text.  A byte outside the alphabet sets bit 0 of the error word.

Checked against that layout built position by position in numpy (the
layout the key tests read), for the whole text and for a range of words.
The kernels' text is cut out of the CUDA source and compiled for the host
with tests/emu/cuda_emu.h.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "pack_emulation.cpp")
SENTINEL = 0x5A5A5A5A


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("packemu")
    src = open(os.path.join(CSRC, "pack.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_kernels.cuh")).read()
    (d / "alphabet.inc").write_text(_cut(hdr, "struct Alphabet16 {", "// pack.cu:"))
    (d / "pack.inc").write_text(_cut(src, "// One thread per 32 positions", "}  // namespace\n\nvoid launch_pack_w"))
    lib = d / "libpackemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    L.emu_pack.argtypes = [I, P, U64, P, U64, U64, P, I, P, P, P, U64, U64]
    L.emu_pack.restype = I
    return L


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def make_reads(rng, alphabet, m, foreign=None):
    lens = rng.integers(0, 70, size=m)
    lens[:3] = [0, 1, 0]
    lut = np.frombuffer(alphabet, np.uint8)
    reads = lut[rng.integers(0, len(alphabet), size=int(lens.sum()))].copy()
    if foreign is not None and reads.size:
        reads[reads.size // 2] = foreign
    return reads, np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)


def expected_layout(reads, offsets, alphabet, code_bits):
    """Codes and terminator bits position by position, then packed."""
    m = offsets.size - 1
    npos = reads.size + m
    codes = np.zeros(npos, np.int64)
    term = np.zeros(npos, bool)
    code_of = {b: i for i, b in enumerate(alphabet)}
    for j in range(m):
        a, b = int(offsets[j]), int(offsets[j + 1])
        for k in range(b - a):
            codes[a + j + k] = code_of.get(int(reads[a + k]), 0)
        term[b + j] = True
    per = 32 // code_bits
    words = (npos + 31) // 32
    text = np.zeros(words * 32 // per, np.uint64)
    for t in range(npos):
        text[t // per] |= np.uint64(codes[t]) << np.uint64(32 - code_bits * (t % per + 1))
    bits = np.zeros(words, np.uint64)
    for t in np.nonzero(term)[0]:
        bits[t >> 5] |= np.uint64(1 << (t & 31))
    return npos, text.astype(np.uint32), bits.astype(np.uint32)


def run(emu, code_bits, reads, offsets, alphabet, w_begin=0, w_end=None):
    m = offsets.size - 1
    npos = reads.size + m
    words = (npos + 31) // 32
    w_end = words if w_end is None else w_end
    per = 2 if code_bits == 2 else 4
    text = np.full(words * per, SENTINEL, np.uint32)
    term = np.full(words, SENTINEL, np.uint32)
    err = np.zeros(1, np.uint32)
    alpha = np.frombuffer(alphabet, np.uint8).copy()
    assert emu.emu_pack(code_bits, _p(reads), reads.size, _p(offsets), m, npos, _p(alpha), len(alphabet), _p(text),
                        _p(term), _p(err), w_begin, w_end) == 0
    return text, term, int(err[0])


@pytest.mark.parametrize("code_bits,alphabet", [(2, b"ACGT"), (2, b"AC"), (4, b"ACGTNRYKMSW"),
                                                (4, bytes(range(65, 81)))])
def test_text_and_terminator_bitmap(emu, code_bits, alphabet):
    rng = np.random.default_rng(len(alphabet) * 10 + code_bits)
    reads, offsets = make_reads(rng, alphabet, 300)
    npos, want_text, want_term = expected_layout(reads, offsets, alphabet, code_bits)
    assert npos % 32 != 0
    text, term, err = run(emu, code_bits, reads, offsets, alphabet)
    assert err == 0
    assert np.array_equal(text, want_text)
    assert np.array_equal(term, want_term)
    # a range of words: only those are written
    words = (npos + 31) // 32
    w0, w1 = 5, min(words, 17)
    per = 2 if code_bits == 2 else 4
    text, term, err = run(emu, code_bits, reads, offsets, alphabet, w0, w1)
    assert np.array_equal(text[w0 * per:w1 * per], want_text[w0 * per:w1 * per])
    assert np.array_equal(term[w0:w1], want_term[w0:w1])
    assert np.all(text[:w0 * per] == SENTINEL) and np.all(text[w1 * per:] == SENTINEL)
    assert np.all(term[:w0] == SENTINEL) and np.all(term[w1:] == SENTINEL)


@pytest.mark.parametrize("code_bits,alphabet,foreign", [(2, b"ACGT", ord("N")), (2, b"AC", ord("G")),
                                                        (4, b"ACGTN", ord("x"))])
def test_a_byte_outside_the_alphabet_sets_the_error_bit(emu, code_bits, alphabet, foreign):
    rng = np.random.default_rng(foreign)
    reads, offsets = make_reads(rng, alphabet, 50, foreign=foreign)
    _, _, err = run(emu, code_bits, reads, offsets, alphabet)
    assert err == 1
