"""sbwt_save / sbwt_load: a saved and reloaded index answers like the one
that wrote it, and later appends continue it exactly (checked against the
oracle's BWT of all reads)."""
import numpy as np
import pytest

import oracle
import paper_1410_0562_gb300 as sb
import readgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sb.build()
    sb.load()


def concat(parts):
    reads = np.concatenate([r for r, _ in parts])
    lengths = np.concatenate([np.diff(o.astype(np.int64)) for _, o in parts])
    return reads, readgen.offsets_from_lengths(lengths)


@pytest.mark.parametrize("index_bits,host_tier", [(32, 0), (64, 0), (32, 3)])
def test_round_trip_then_append(tmp_path, index_bits, host_tier):
    a = readgen.ragged_reads(700, 0, 160, seed=71, p_empty=0.02, p_repeat=0.05)
    b = readgen.ragged_reads(500, 1, 120, seed=72)
    idx = sb.SetBWT(b"ACGT", index_bits=index_bits, block_suffixes=30_000)
    idx.append(*a)
    path = tmp_path / "idx.sbwt"
    idx.save(path)
    back = sb.SetBWT.load(path, block_suffixes=30_000, host_tier=host_tier)
    assert back.size() == idx.size()
    assert np.array_equal(back.bwt(), idx.bwt())
    n, _ = idx.size()
    ks = np.arange(0, n + 1, 37, dtype=np.uint64)
    for c in b"ACGT$":
        cs = np.full(len(ks), c, np.uint8)
        assert np.array_equal(back.rank_batch(cs, ks), idx.rank_batch(cs, ks))
    pats = [b"A", b"ACG", b"TTT", b"GATTACA", b""]
    assert np.array_equal(back.count(pats), idx.count(pats))
    if host_tier == 3:
        hbm, host = sb.sbwt_memory(back.handle)
        assert host > 0
    # appends continue the read ids of the saved index
    idx.append(*b)
    back.append(*b)
    expect = oracle.bwt(*concat([a, b]))
    assert np.array_equal(idx.bwt(), expect)
    assert np.array_equal(back.bwt(), expect)


def test_empty_index_round_trip(tmp_path):
    path = tmp_path / "empty.sbwt"
    sb.SetBWT(b"ACG").save(path)
    back = sb.SetBWT.load(path)
    assert back.size() == (0, 0)
    r = readgen.uniform_reads(50, 30, seed=5, alphabet=b"ACG")
    back.append(*r)
    assert np.array_equal(back.bwt(), oracle.bwt(*r, alphabet=b"ACG"))


@pytest.mark.parametrize("sampling", [128, 256])
def test_round_trip_other_samplings(tmp_path, sampling):
    a = readgen.ragged_reads(900, 0, 150, seed=73, p_empty=0.02)
    idx = sb.SetBWT(b"ACGT", occ_sampling=sampling, block_suffixes=25_000)
    idx.append(*a)
    path = tmp_path / "idx.sbwt"
    idx.save(path)
    back = sb.SetBWT.load(path)
    assert np.array_equal(back.bwt(), oracle.bwt(*a))
    with pytest.raises(sb.SbwtError):  # the file's sampling decides
        sb.SetBWT.load(path, occ_sampling=64 if sampling != 64 else 128)


def test_version_1_file_is_converted(tmp_path):
    """A file in the first layout (2-bit codes interleaved in blocks of 64
    rows, version 1), written here from the oracle's B, loads into the
    bit-plane layout and answers like a built index."""
    import struct
    a = readgen.ragged_reads(800, 0, 140, seed=74, p_empty=0.02)
    B = oracle.bwt(*a)
    n, m = len(B), len(a[1]) - 1
    code = np.zeros(256, np.uint64)
    for i, c in enumerate(b"ACGT"):
        code[c] = i
    nb = (n >> 6) + 1
    c = np.zeros(nb * 64, np.uint64)
    d = np.zeros(nb * 64, np.uint64)
    c[:n] = code[B]
    d[:n] = B == ord("$")
    c = c.reshape(nb, 64)
    d = d.reshape(nb, 64)
    sym0 = np.bitwise_or.reduce(c[:, :32] << (2 * np.arange(32)).astype(np.uint64), axis=1)
    sym1 = np.bitwise_or.reduce(c[:, 32:] << (2 * np.arange(32)).astype(np.uint64), axis=1)
    dm = np.bitwise_or.reduce(d << np.arange(64).astype(np.uint64), axis=1)
    cnt = np.stack([((c == k) & (d == 0)).sum(axis=1) for k in range(4)], axis=1).astype(np.int64)
    excl = np.cumsum(cnt, axis=0) - cnt
    first = (np.arange(nb) // 1024) * 1024
    rel = (excl - excl[first]).astype(np.uint64)
    packed = rel[:, 0] | (rel[:, 1] << np.uint64(16)) | (rel[:, 2] << np.uint64(32)) | (rel[:, 3] << np.uint64(48))
    blocks = np.stack([sym0, sym1, dm, packed], axis=1).astype("<u8")
    nsb = (nb + 1023) // 1024
    sbc = np.zeros((nsb, 4), np.uint64)
    tot = np.stack([np.count_nonzero(B == x) for x in b"ACGT"])
    for s_ in range(1, nsb):
        chunk = B[: s_ << 16]
        sbc[s_] = [np.count_nonzero(chunk == x) for x in b"ACGT"]
    C = np.array([m, m + tot[0], m + tot[0] + tot[1], m + tot[0] + tot[1] + tot[2]], np.uint64)
    header = bytearray(88)
    header[:8] = b"SBWTIDX1"
    struct.pack_into("<II4sI", header, 8, 1, 4, b"ACGT", 0)
    struct.pack_into("<QQQQ", header, 24, n, m, nb, nsb)
    body = bytes(header) + blocks.tobytes() + sbc.astype("<u8").tobytes() + C.astype("<u8").tobytes()
    h = 1469598103934665603
    for byte in body:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    path = tmp_path / "v1.sbwt"
    path.write_bytes(body + struct.pack("<Q", h))
    back = sb.SetBWT.load(path)
    assert back.size() == (n, m)
    assert np.array_equal(back.bwt(), B)
    b = readgen.ragged_reads(300, 1, 100, seed=75)
    back.append(*b)
    assert np.array_equal(back.bwt(), oracle.bwt(*concat([a, b])))
