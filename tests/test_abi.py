"""The C ABI without a GPU: libsbwt.so builds, loads, exports every entry
point include/sbwt.h declares, and rejects bad arguments on the host before
touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1410_0562_gb300 as sb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sbwt.h")


@pytest.fixture(scope="module")
def lib():
    sb.build()
    return sb.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sbwt_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sbwt_create", "sbwt_append", "sbwt_get_bwt", "sbwt_rank"):
        assert required in names
    assert sorted(sb.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5, -99):
        assert isinstance(sb.strerror(code), str) and sb.strerror(code)


@pytest.mark.parametrize("alpha", [b"", b"ACGTN", b"CA", b"AAC", b"A$", b"ACC", b"ABCDEFGHIJKLMNOPQ",
                                   b"ABCDEFGH$"])
def test_create_rejects_bad_alphabet(lib, alpha):
    h = ctypes.c_void_p()
    assert lib.sbwt_create(alpha, 0, ctypes.byref(h)) == sb.SBWT_EINVAL
    assert not h.value


def test_create_does_not_touch_the_gpu(lib):
    # works on a machine without a GPU: device state is created lazily
    for alpha in (b"A", b"AC", b"ACG", b"ACGT", b"abn", b"imps", b"ACGNT", b"ABCDEFGHIJKLMNOP"):
        h = sb.sbwt_create(alpha)
        assert sb.sbwt_size(h) == (0, 0)
        sb.sbwt_reset(h)
        sb.sbwt_destroy(h)
    sb.sbwt_destroy(None)


def test_create_ex_rejects_bad_options(lib):
    for kw in ({"index_bits": 16}, {"block_suffixes": (1 << 31) + 1}):
        with pytest.raises(sb.SbwtError) as e:
            sb.sbwt_create_ex(b"ACGT", **kw)
        assert e.value.code == sb.SBWT_EINVAL


def test_append_rejects_bad_offsets_on_the_host(lib):
    h = sb.sbwt_create(b"ACGT")
    reads = np.frombuffer(b"ACGTACGT", np.uint8)
    for off in ([1, 4, 8], [0, 5, 4, 8], [0, 9, 8]):
        with pytest.raises(sb.SbwtError) as e:
            sb.sbwt_append(h, reads, np.array(off, np.uint64))
        assert e.value.code == sb.SBWT_EINVAL
    assert sb.sbwt_size(h) == (0, 0)
    # m = 0 is a no-op that needs no device
    sb.sbwt_append(h, reads, np.array([0], np.uint64))
    assert sb.sbwt_size(h) == (0, 0)
    sb.sbwt_destroy(h)


def test_queries_validate_on_the_host(lib):
    h = sb.sbwt_create(b"ACGT")
    with pytest.raises(sb.SbwtError):
        sb.sbwt_rank(h, ord("N"), 0)
    with pytest.raises(sb.SbwtError):
        sb.sbwt_rank(h, ord("A"), 1)  # k > n = 0
    assert len(sb.sbwt_get_bwt(h)) == 0
    with pytest.raises(sb.SbwtError):
        sb.sbwt_get_stage(h, sb.SBWT_STAGE_SA)  # capture is off
    sb.sbwt_destroy(h)


def test_no_cpu_fallback_without_a_device(lib):
    """On a machine without a GPU a valid append must fail loudly with
    SBWT_EDEVICE; it must never compute the BWT on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = sb.sbwt_create(b"ACGT")
    with pytest.raises(sb.SbwtError) as e:
        sb.sbwt_append(h, np.frombuffer(b"ACGT", np.uint8), np.array([0, 4], np.uint64))
    assert e.value.code == sb.SBWT_EDEVICE
    assert sb.sbwt_size(h) == (0, 0)
    sb.sbwt_destroy(h)


def test_index_width_is_checked_on_the_host(lib):
    """With 32-bit row indices an append that would reach 2^32 - 1 rows is
    refused before any device work; with automatic width it passes that
    check (and then needs the device).  The reads are three of 2^31 - 2
    bases in lazily mapped zero pages that the refused call never reads."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the automatic-width append would run")
    L = (1 << 31) - 2
    reads = np.zeros(3 * L, np.uint8)
    off = np.array([0, L, 2 * L, 3 * L], np.uint64)
    h = sb.sbwt_create_ex(b"ACGT", index_bits=32)
    with pytest.raises(sb.SbwtError) as e:
        sb.sbwt_append(h, reads, off)
    assert e.value.code == sb.SBWT_EINVAL
    assert sb.sbwt_size(h) == (0, 0)
    sb.sbwt_destroy(h)
    h = sb.sbwt_create_ex(b"ACGT", index_bits=0)
    with pytest.raises(sb.SbwtError) as e:
        sb.sbwt_append(h, reads, off)
    assert e.value.code == sb.SBWT_EDEVICE
    sb.sbwt_destroy(h)


def test_load_checks_the_file_before_any_device_work(lib, tmp_path):
    """Missing file -> SBWT_EIO; not an index file, a flipped byte or a
    truncated file -> SBWT_EINVAL; a valid file of an empty index reaches the
    device step (SBWT_EDEVICE here, without a GPU)."""
    with pytest.raises(sb.SbwtError) as e:
        sb.SetBWT.load(tmp_path / "missing.sbwt")
    assert e.value.code == sb.SBWT_EIO
    junk = tmp_path / "junk.sbwt"
    junk.write_bytes(b"not an index" * 20)
    with pytest.raises(sb.SbwtError) as e:
        sb.SetBWT.load(junk)
    assert e.value.code == sb.SBWT_EINVAL
    good = tmp_path / "empty.sbwt"
    sb.SetBWT(b"ACGT").save(good)  # never appended: no device work
    data = bytearray(good.read_bytes())
    assert data[:8] == b"SBWTIDX1"
    flipped = tmp_path / "flipped.sbwt"
    bad = bytearray(data)
    bad[100] ^= 1
    flipped.write_bytes(bytes(bad))
    truncated = tmp_path / "truncated.sbwt"
    truncated.write_bytes(bytes(data[:-9]))
    for path in (flipped, truncated):
        with pytest.raises(sb.SbwtError) as e:
            sb.SetBWT.load(path)
        assert e.value.code == sb.SBWT_EINVAL
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(sb.SbwtError) as e:
            sb.SetBWT.load(good)
        assert e.value.code == sb.SBWT_EDEVICE


def test_wide_alphabet_file_layout(lib, tmp_path):
    """An index of 5 to 16 symbols is written as file version 2: the 88-byte
    header (symbols 5.. after the first four), one 64-byte block, one
    superblock and C[] of 16 counters each, the checksum."""
    import struct
    path = tmp_path / "wide.sbwt"
    sb.SetBWT(b"ACGNT").save(path)  # never appended: no device work
    data = path.read_bytes()
    assert data[:8] == b"SBWTIDX1"
    version, sigma = struct.unpack_from("<II", data, 8)
    assert (version, sigma) == (2, 5)
    assert data[16:20] == b"ACGN" and data[56:57] == b"T"
    assert len(data) == 88 + 64 + 16 * 8 + 16 * 8 + 8
    narrow = tmp_path / "narrow.sbwt"
    sb.SetBWT(b"ACGT").save(narrow)
    assert struct.unpack_from("<II", narrow.read_bytes(), 8) == (3, 4)
    assert struct.unpack_from("<I", narrow.read_bytes(), 68) == (64,)
    assert len(narrow.read_bytes()) == 88 + 32 + 4 * 8 + 4 * 8 + 8
    # sampling 128 and 256: blocks of 7 and 13 words
    for rows, words in ((128, 7), (256, 13)):
        f = tmp_path / f"narrow{rows}.sbwt"
        sb.SetBWT(b"ACGT", occ_sampling=rows).save(f)
        assert struct.unpack_from("<I", f.read_bytes(), 68) == (rows,)
        assert len(f.read_bytes()) == 88 + 8 * words + 4 * 8 + 4 * 8 + 8
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(sb.SbwtError) as e:  # the file checks pass; the device step fails
            sb.SetBWT.load(path)
        assert e.value.code == sb.SBWT_EDEVICE


def test_save_rejects_null_path(lib):
    idx = sb.SetBWT(b"ACGT")
    assert lib.sbwt_save(idx.handle, None) == sb.SBWT_EINVAL


def test_noalloc_rejects_sizes_that_would_wrap(lib):
    """sbwt_bwt_noalloc checks its size limit on the host before any device
    work, with offsets whose sums would wrap past 2^64."""
    out = np.zeros(16, np.uint8)
    got = ctypes.c_uint64()
    top = np.iinfo(np.uint64).max
    for offs in ([0, top], [0, top, top], [0, top - 1, top], [0, sb.SBWT_NOALLOC_MAX_SUFFIXES]):
        o = np.array(offs, np.uint64)
        rc = lib.sbwt_bwt_noalloc(b"ACGT", ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(o.ctypes.data),
                                  len(o) - 1, ctypes.c_void_p(out.ctypes.data), 16, ctypes.byref(got), None)
        assert rc == sb.SBWT_EINVAL, offs
    # more reads than the maximum can hold terminators for
    m = sb.SBWT_NOALLOC_MAX_SUFFIXES + 1
    o = np.zeros(m + 1, np.uint64)
    rc = lib.sbwt_bwt_noalloc(b"ACGT", ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(o.ctypes.data), m,
                              ctypes.c_void_p(out.ctypes.data), 16, ctypes.byref(got), None)
    assert rc == sb.SBWT_EINVAL


def test_occurrence_sampling_option(lib):
    """64, 128 and 256 rows per occurrence block for up to 4 symbols; 5 to 16
    symbols take 64 only; any other value is refused."""
    for rows in (0, 64, 128, 256):
        sb.SetBWT(b"ACGT", occ_sampling=rows).close()
    for rows in (1, 32, 96, 192, 512):
        with pytest.raises(sb.SbwtError) as e:
            sb.SetBWT(b"ACGT", occ_sampling=rows)
        assert e.value.code == sb.SBWT_EINVAL
    sb.SetBWT(b"ACGNT", occ_sampling=64).close()
    with pytest.raises(sb.SbwtError) as e:
        sb.SetBWT(b"ACGNT", occ_sampling=128)
    assert e.value.code == sb.SBWT_ENOTSUP


def fnv1a(data: bytes) -> int:
    h = 1469598103934665603
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_version_1_file_passes_the_checks(lib, tmp_path):
    """A file of the first layout (2-bit codes interleaved in 64-row blocks,
    version 1) is still read: its checks pass before the device step."""
    import struct
    header = bytearray(88)
    header[:8] = b"SBWTIDX1"
    struct.pack_into("<II4sI", header, 8, 1, 4, b"ACGT", 32)
    struct.pack_into("<QQQQ", header, 24, 0, 0, 1, 1)  # n, m, one block, one superblock
    body = bytes(header) + bytes(32) + bytes(32) + bytes(32)
    path = tmp_path / "v1.sbwt"
    path.write_bytes(body + struct.pack("<Q", fnv1a(body)))
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(sb.SbwtError) as e:
            sb.SetBWT.load(path)
        assert e.value.code == sb.SBWT_EDEVICE
    # a wrong checksum is refused before any device work
    path.write_bytes(body + struct.pack("<Q", fnv1a(body) ^ 1))
    with pytest.raises(sb.SbwtError) as e:
        sb.SetBWT.load(path)
    assert e.value.code == sb.SBWT_EINVAL
