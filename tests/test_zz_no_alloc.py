"""sbwt_bwt_noalloc: the BWT of a small read set for callers that cannot
allocate device memory (their device memory belongs to another framework's
pool, or allocation is forbidden after start-up).  It works from one fixed
device array instead of cudaMalloc, so its output must equal, byte for byte,
what the allocating entry points (sbwt_create + sbwt_append + sbwt_get_bwt)
produce for the same reads -- on consecutive calls too, since every call
reuses the same array."""
import numpy as np
import pytest

import paper_1410_0562_gb300 as sb
import readgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sb.build()
    sb.load()


def allocating_bwt(reads, offsets, alphabet=b"ACGT"):
    idx = sb.SetBWT(alphabet)
    idx.append(reads, offsets)
    out = idx.bwt()
    idx.close()
    return out


def test_two_calls_in_a_row_match_the_allocating_path():
    # a larger set first, then a smaller one: the second call must not see
    # anything the first left behind in the shared array
    big_r, big_o = readgen.ragged_reads(1500, 0, 150, seed=21, p_empty=0.05, p_repeat=0.05)
    small_r, small_o = readgen.uniform_reads(300, 100, seed=22)
    assert int(big_o[-1]) + len(big_o) - 1 <= sb.SBWT_NOALLOC_MAX_SUFFIXES
    first = sb.sbwt_bwt_noalloc(b"ACGT", big_r, big_o)
    second = sb.sbwt_bwt_noalloc(b"ACGT", small_r, small_o)
    assert np.array_equal(first, allocating_bwt(big_r, big_o))
    assert np.array_equal(second, allocating_bwt(small_r, small_o))


def test_other_alphabet_and_size_limit():
    reads, off = readgen.ragged_reads(200, 0, 60, seed=23, alphabet=b"ACG")
    assert np.array_equal(sb.sbwt_bwt_noalloc(b"ACG", reads, off), allocating_bwt(reads, off, b"ACG"))
    # one suffix past the fixed maximum is refused before any GPU work
    L = sb.SBWT_NOALLOC_MAX_SUFFIXES
    too_big = np.full(L, ord("A"), np.uint8)
    with pytest.raises(sb.SbwtError) as e:
        sb.sbwt_bwt_noalloc(b"ACGT", too_big, np.array([0, L], np.uint64))
    assert e.value.code == sb.SBWT_EINVAL
    # exactly at the maximum is accepted
    at_max = np.full(L - 1, ord("C"), np.uint8)
    at_max[::7] = ord("A")
    off = np.array([0, L - 1], np.uint64)
    assert np.array_equal(sb.sbwt_bwt_noalloc(b"ACGT", at_max, off), allocating_bwt(at_max, off))


def raw_call(alphabet, reads, offsets, cap):
    """sbwt_bwt_noalloc through ctypes with a caller-chosen output size."""
    import ctypes
    reads = np.ascontiguousarray(reads, np.uint8)
    offsets = np.ascontiguousarray(offsets, np.uint64)
    out = np.zeros(max(cap, 1), np.uint8)
    got = ctypes.c_uint64()
    rc = sb.load().sbwt_bwt_noalloc(alphabet, ctypes.c_void_p(reads.ctypes.data),
                                    ctypes.c_void_p(offsets.ctypes.data), len(offsets) - 1,
                                    ctypes.c_void_p(out.ctypes.data), cap, ctypes.byref(got), None)
    return rc, got.value, out[: min(cap, got.value)]


def test_error_paths_and_the_reused_error_word():
    reads, off = readgen.ragged_reads(400, 1, 120, seed=24)
    n = int(off[-1]) + len(off) - 1
    # output buffer one byte short: nothing computed, the needed size reported
    rc, got, _ = raw_call(b"ACGT", reads, off, n - 1)
    assert rc == sb.SBWT_ERANGE and got == n
    # a byte outside the alphabet is found by the packing kernel and reported
    # through the error word the calls share
    bad = reads.copy()
    bad[len(bad) // 2] = ord("N")
    rc, _, _ = raw_call(b"ACGT", bad, off, n)
    assert rc == sb.SBWT_EINVAL
    # the next clean call starts from a cleared error word and matches
    rc, got, out = raw_call(b"ACGT", reads, off, n)
    assert rc == sb.SBWT_OK and got == n
    assert np.array_equal(out, allocating_bwt(reads, off))


def test_calls_allocate_no_device_memory():
    import torch
    a_r, a_o = readgen.ragged_reads(900, 0, 200, seed=25, p_empty=0.02, p_repeat=0.05)
    b_r, b_o = readgen.uniform_reads(700, 90, seed=26)
    expect_a, expect_b = allocating_bwt(a_r, a_o), allocating_bwt(b_r, b_o)
    torch.cuda.synchronize()
    # the first calls do the per-device set-up (and load the kernels they use)
    sb.sbwt_bwt_noalloc(b"ACGT", a_r, a_o)
    sb.sbwt_bwt_noalloc(b"ACGT", b_r, b_o)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    got_a = sb.sbwt_bwt_noalloc(b"ACGT", a_r, a_o)
    got_b = sb.sbwt_bwt_noalloc(b"ACGT", b_r, b_o)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    assert np.array_equal(got_a, expect_a) and np.array_equal(got_b, expect_b)
