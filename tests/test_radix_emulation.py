"""One radix pass (csrc/radix.cu) run on the CPU: its counting phases and its scatter.

The upsweep counts the digits of each chunk of whole 2048-key tiles (a
persistent grid of G CTAs, chunk c holding tiles [c per, (c+1) per) of the
ceil(n / 2048) tiles) and adds them to the pass's digit totals; the chunk
scan turns the G x 256 counts into each (chunk, digit)'s first output slot:
the number of keys with a smaller digit plus the keys of the same digit in
earlier chunks, which is what a stable counting sort gives.  The kernels'
text is cut out of the CUDA source and compiled for the host with
tests/emu/cuda_emu.h (the one inline-PTX load becomes two plain loads).
The downsweep's tile copies and their mbarrier are inline PTX in helper
functions; the harness gives host versions of those helpers (the copy done
at once, completing its bytes on the barrier's phase) and checks the bulk
copies' 16-byte rule, so a whole pass runs and is compared with a stable
counting sort.
Checked against numpy on keys whose count is not a multiple of the tile,
with grids that leave the last chunks empty.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1410_0562_gb300", "csrc")
EMU = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emu", "radix_emulation.cpp")
TILE = 2048


def _cut(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("radixemu")
    src = open(os.path.join(CSRC, "radix.cu")).read()
    hdr = open(os.path.join(CSRC, "sbwt_internal.cuh")).read()
    (d / "radix_hdr.inc").write_text(_cut(hdr, "constexpr int kRadixBits = 8;", "size_t radix_temp_words(uint64_t cap);"))
    (d / "scan.inc").write_text(_cut(hdr, "struct SumOp {", "// Launch bookkeeping"))
    (d / "radix_consts.inc").write_text(_cut(src, "constexpr int kThreads = 256;", "// Chunk c of a grid"))
    count = _cut(src, "// Chunk c of a grid", "// The scatter of one pass over this CTA's chunk")
    ptx = 'asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));'
    assert ptx in count
    (d / "radix_count.inc").write_text(count.replace(ptx, "a = p[0];\n    b = p[1];"))
    down = _cut(src, "// The scatter of one pass over this CTA's chunk",
                "// ---------------------------------------------------------------------------\n// Fused sort")
    dyn = "extern __shared__ __align__(128) unsigned char smem[];"
    assert down.count(dyn) == 1
    (d / "radix_down.inc").write_text(down.replace(dyn, "unsigned char* smem = g_dyn_smem;"))
    (d / "radix_fused_scan.inc").write_text(_cut(src, "// Output offsets of every (chunk, digit) from the chunk counts",
                                                 "template <class KeyT>\n__global__ void __launch_bounds__(kThreads, 3) "
                                                 "radix_sort_fused_kernel("))
    lib = d / "libradixemu.so"
    subprocess.check_call(["g++", "-O1", "-std=c++20", "-shared", "-fPIC", "-pthread", "-I", str(d), "-o", str(lib),
                           EMU])
    L = ctypes.CDLL(str(lib))
    P, U32, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
    L.emu_radix_count.argtypes = [P, U32, I, U32, P, P]
    L.emu_radix_count.restype = I
    L.emu_radix_pass.argtypes = [P, P, U32, I, U32, I, P, P, P]
    L.emu_radix_pass.restype = I
    L.emu_fused_sort.argtypes = [P, P, U32, I, I, U32, P, P, P]
    L.emu_fused_sort.restype = I
    return L


def chunk_of(n: int, grid: int) -> np.ndarray:
    """Chunk of every key index under the kernels' tiling."""
    ntiles = (n + TILE - 1) // TILE
    per = (ntiles + grid - 1) // grid
    return (np.arange(n) // TILE) // per


@pytest.mark.parametrize("n,grid,shift", [(50_001, 7, 0), (50_001, 40, 8), (6_000, 5, 16), (2_048, 3, 0), (0, 4, 0)])
def test_chunk_offsets_are_those_of_a_stable_counting_sort(emu, n, grid, shift):
    rng = np.random.default_rng(n + grid + shift)
    # a skewed digit mix (a few digits take most keys) as in the bucket split
    digits = np.where(rng.random(n) < 0.5, rng.integers(0, 4, n), rng.integers(0, 256, n)).astype(np.uint64)
    keys = (digits << np.uint64(shift)) | (rng.integers(0, 1 << 20, n).astype(np.uint64) << np.uint64(40))
    offsets = np.zeros(grid * 256, np.uint32)
    next_totals = np.full(256, 99, np.uint32)
    kp = keys if n else np.zeros(1, np.uint64)
    assert emu.emu_radix_count(ctypes.c_void_p(kp.ctypes.data), n, shift, grid,
                               ctypes.c_void_p(offsets.ctypes.data), ctypes.c_void_p(next_totals.ctypes.data)) == 0
    assert not next_totals.any()
    if n == 0:
        return
    chunks = chunk_of(n, grid)
    used = int(chunks.max()) + 1
    start = np.concatenate([[0], np.cumsum(np.bincount(digits.astype(np.int64), minlength=256))[:-1]])
    counts = np.zeros((grid, 256), np.int64)
    np.add.at(counts, (chunks, digits.astype(np.int64)), 1)
    want = start[None, :] + np.cumsum(counts, axis=0) - counts
    got = offsets.reshape(grid, 256).astype(np.int64)
    # chunks past the last tile hold nothing and are left alone
    assert np.array_equal(got[:used], want[:used])
    # the offsets place every key once: a stable counting sort by digit
    order = np.empty(n, np.int64)
    nxt = got[:used].copy()
    for i in range(n):
        c, dg = chunks[i], int(digits[i])
        order[nxt[c, dg]] = i
        nxt[c, dg] += 1
    assert np.array_equal(order, np.argsort(digits, kind="stable"))


@pytest.mark.timeout(600)
@pytest.mark.parametrize("n,grid,shift,pairs", [(50_001, 7, 0, 0), (50_001, 40, 8, 1), (6_000, 5, 16, 0),
                                                (2_048, 3, 0, 1), (3 * TILE, 2, 24, 1), (1, 1, 0, 0), (0, 4, 0, 1)])
def test_one_pass_is_a_stable_counting_sort(emu, n, grid, shift, pairs):
    """The whole pass (upsweep, chunk scan, downsweep with its bulk-copied
    tiles) puts every key, and its value, where a stable counting sort by
    the pass's digit does."""
    rng = np.random.default_rng(n + 3 * grid + shift)
    digits = np.where(rng.random(n) < 0.5, rng.integers(0, 4, n), rng.integers(0, 256, n)).astype(np.uint64)
    keys = (digits << np.uint64(shift)) | (rng.integers(0, 1 << 20, n).astype(np.uint64) << np.uint64(40))
    keys |= rng.integers(0, 1 << 8, n).astype(np.uint64) << np.uint64(32 if shift != 32 else 0)
    vals = rng.permutation(n).astype(np.uint32)
    out_k = np.zeros(max(n, 1), np.uint64)
    out_v = np.zeros(max(n, 1), np.uint32)
    err = np.zeros(1, np.uint32)
    kp = keys if n else np.zeros(1, np.uint64)
    vp = vals if n else np.zeros(1, np.uint32)
    rc = emu.emu_radix_pass(ctypes.c_void_p(kp.ctypes.data), ctypes.c_void_p(vp.ctypes.data), n, shift, grid, pairs,
                            ctypes.c_void_p(out_k.ctypes.data), ctypes.c_void_p(out_v.ctypes.data),
                            ctypes.c_void_p(err.ctypes.data))
    assert rc == 0, "a bulk copy broke the 16-byte rule"
    assert err[0] == 0
    order = np.argsort(digits, kind="stable")
    assert np.array_equal(out_k[:n], keys[order])
    if pairs:
        assert np.array_equal(out_v[:n], vals[order])


@pytest.mark.timeout(600)
@pytest.mark.parametrize("n,grid,begin,passes", [(20_001, 5, 0, 3), (9_000, 20, 8, 2), (2_048, 3, 0, 1),
                                                 (12_000, 4, 4, 4), (1, 2, 0, 3)])
def test_fused_sort_passes_sort_stably_by_all_their_bits(emu, n, grid, begin, passes):
    """The fused sort's phases (upsweep, the two-step chunk scan of chunk
    groups, downsweep) run pass after pass with keys and values ping-ponging
    between the two arrays: the result is a stable sort by bits [begin,
    begin + 8 passes)."""
    rng = np.random.default_rng(n + grid + passes)
    width = 8 * passes
    field = np.where(rng.random(n) < 0.4, rng.integers(0, 16, n), rng.integers(0, 1 << width, n)).astype(np.uint64)
    keys = (field << np.uint64(begin)) | (rng.integers(0, 1 << 10, n).astype(np.uint64) << np.uint64(begin + width))
    keys |= rng.integers(0, 1 << begin, n).astype(np.uint64) if begin else np.uint64(0)
    vals = rng.permutation(n).astype(np.uint32)
    out_k = np.zeros(n, np.uint64)
    out_v = np.zeros(n, np.uint32)
    err = np.zeros(1, np.uint32)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    assert emu.emu_fused_sort(p(keys), p(vals), n, begin, passes, grid, p(out_k), p(out_v), p(err)) == 0
    assert err[0] == 0
    order = np.argsort(field, kind="stable")
    assert np.array_equal(out_k, keys[order]) and np.array_equal(out_v, vals[order])
