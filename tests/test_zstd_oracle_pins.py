"""Pins of the oracle's Zstandard mask frames (Sec. III-C: the zero bitmask
packed into bytes and compressed with Zstd; Sec. III-D: a P scan's mask XORed
with the previous one first).

The frames are pinned to things other than the oracle itself:
  - libzstd (an independent Zstandard implementation, through ctypes)
    restores every frame the oracle writes, on inputs chosen to reach every
    block kind and both forms of the Huffman tree description;
  - a frame derived by hand from RFC 8878 (tests/golden/zstd_frame_*.txt);
  - the Huffman streams cost what an optimal Huffman code costs (a textbook
    heap construction here), when the length limit does not bind;
  - the masks in a coded stream are exactly the packed zero bitmasks of the
    quantized scans (XORed for P), as libzstd decompresses them.
"""
import ctypes
import ctypes.util
import heapq
import os

import numpy as np
import pytest

import oracle
from tests import golden_io

ZSTD = ctypes.util.find_library("zstd")


def _libzstd():
    if ZSTD is None:
        pytest.skip("libzstd is not installed")
    z = ctypes.CDLL(ZSTD)
    sz, vp = ctypes.c_size_t, ctypes.c_void_p
    z.ZSTD_decompress.restype, z.ZSTD_decompress.argtypes = sz, [vp, sz, vp, sz]
    z.ZSTD_isError.restype, z.ZSTD_isError.argtypes = ctypes.c_uint, [sz]
    return z


def decompress(frame: bytes, n: int):
    z = _libzstd()
    src = np.frombuffer(frame, dtype=np.uint8).copy()
    out = np.zeros(n + 64, dtype=np.uint8)
    k = z.ZSTD_decompress(out.ctypes.data, out.nbytes, src.ctypes.data, len(src))
    return None if z.ZSTD_isError(k) else out[:k].tobytes()


def inputs():
    """Byte strings of several sizes and statistics: sparse masks (I and
    P), uniform bytes, one value, a small alphabet, Fibonacci counts (an
    optimal code deeper than 11 bits)."""
    rng = np.random.default_rng(11)
    fib = [1, 1]
    while len(fib) < 24:
        fib.append(fib[-1] + fib[-2])
    fibsyms = np.repeat(np.arange(24, dtype=np.uint8) * 9 + 30, fib)
    out = []
    for n in (1, 2, 3, 64, 700, 1023, 1024, 1025, 4099, 8192, 8193, 20000, 40000):
        out.append(("mask12", np.packbits(rng.random(8 * n) < 0.12, bitorder="little")[:n]))
        out.append(("uniform", rng.integers(0, 256, n, dtype=np.uint8)))
        out.append(("same", np.full(n, 0xA5, np.uint8)))
        out.append(("small", rng.integers(0, 3, n).astype(np.uint8)))
        out.append(("p", ((rng.random(n) < 0.02) * rng.integers(1, 256, n)).astype(np.uint8)))
        out.append(("fib", np.resize(rng.permutation(fibsyms), n)))
    return [(k, b.tobytes()) for k, b in out]


def blocks(frame: bytes):
    """(type, literal size format, tree form, stream bytes, block input) of
    each block, from the headers alone."""
    assert frame[:4] == bytes.fromhex("28b52ffd") and frame[4] == 0xA0
    pos, out = 9, []
    while True:
        bh = int.from_bytes(frame[pos:pos + 3], "little")
        last, t, size = bh & 1, (bh >> 1) & 3, bh >> 3
        pos += 3
        if t == 2:
            sf = (frame[pos] >> 2) & 3
            lh = 3 if sf <= 1 else (4 if sf == 2 else 5)
            bits = 10 if sf <= 1 else (14 if sf == 2 else 18)
            h = int.from_bytes(frame[pos:pos + lh], "little")
            rs, cs = (h >> 4) & ((1 << bits) - 1), (h >> (4 + bits)) & ((1 << bits) - 1)
            hb = frame[pos + lh]
            tree = 1 + (hb - 127 + 1) // 2 if hb >= 128 else 1 + hb
            streams = cs - tree - (6 if sf else 0)
            out.append(("compressed", sf, "direct" if hb >= 128 else "fse", streams, rs))
            pos += size
        elif t == 1:
            out.append(("rle", None, None, 0, size))
            pos += 1
        else:
            out.append(("raw", None, None, 0, size))
            pos += size
        if last:
            return out, pos


def huffman_bits(data: bytes) -> int:
    """Bits of an optimal (unrestricted) Huffman code of the bytes."""
    cnt = np.bincount(np.frombuffer(data, dtype=np.uint8), minlength=256)
    h = [int(c) for c in cnt if c]
    if len(h) < 2:
        return len(data)
    heapq.heapify(h)
    total = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        total += a + b
        heapq.heappush(h, a + b)
    return total


def max_huffman_depth(data: bytes) -> int:
    cnt = np.bincount(np.frombuffer(data, dtype=np.uint8), minlength=256)
    h = [(int(c), 0) for c in cnt if c]
    heapq.heapify(h)
    while len(h) > 1:
        (a, da), (b, db) = heapq.heappop(h), heapq.heappop(h)
        heapq.heappush(h, (a + b, max(da, db) + 1))
    return h[0][1]


# ---------------------------------------------------------------- golden
def test_golden_frame_by_hand():
    src, want, ends = b"", b"", []
    with open(os.path.join(golden_io.GOLDEN, "zstd_frame_64_two_symbols.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "in":
                src += bytes(int(x, 16) for x in line[1:])
            elif line[0] == "bytes":
                want += bytes(int(x, 16) for x in line[1:])
            elif line[0] == "ends":
                ends = [int(x) for x in line[1:]]
    frame, got_ends = oracle.zstd_frame(src)
    assert frame == want, frame.hex(" ")
    assert got_ends == ends
    assert oracle.zstd_read(want, len(src)) == src
    assert decompress(want, len(src)) == src


# ---------------------------------------------------------------- libzstd
@pytest.mark.parametrize("kind", ["mask12", "uniform", "same", "small", "p", "fib"])
def test_libzstd_restores_every_frame(kind):
    for k, data in inputs():
        if k != kind:
            continue
        frame, ends = oracle.zstd_frame(data)
        assert decompress(frame, len(data)) == data, (kind, len(data))
        assert oracle.zstd_read(frame, len(data)) == data
        bl, end = blocks(frame)
        assert end == len(frame) and ends[-1] == len(frame)
        assert len(bl) == len(ends) == max(1, -(-len(data) // 8192))
        assert sum(b[4] for b in bl) == len(data)


def test_every_block_kind_and_tree_form_is_reached():
    seen = set()
    for _, data in inputs():
        frame, _ = oracle.zstd_frame(data)
        for t, sf, tree, _, _ in blocks(frame)[0]:
            seen.add((t, sf, tree))
    for want in [("raw", None, None), ("rle", None, None), ("compressed", 0, "direct"), ("compressed", 2, "direct"),
                 ("compressed", 0, "fse"), ("compressed", 2, "fse")]:
        assert want in seen, want


def test_block_choice():
    # all equal -> RLE; uniform bytes do not shrink -> Raw; a compressed
    # block is always smaller than its input
    frame, _ = oracle.zstd_frame(bytes([7]) * 9000)
    assert [b[0] for b in blocks(frame)[0]] == ["rle", "rle"]
    rng = np.random.default_rng(3)
    frame, _ = oracle.zstd_frame(rng.integers(0, 256, 5000, dtype=np.uint8).tobytes())
    assert [b[0] for b in blocks(frame)[0]] == ["raw"]
    for _, data in inputs():
        frame, _ = oracle.zstd_frame(data)
        for t, _, _, _, n in blocks(frame)[0]:
            assert t != "compressed" or n > 4


# ---------------------------------------------------------------- Huffman
def test_huffman_streams_cost_an_optimal_code():
    checked = 0
    for kind, data in inputs():
        frame, _ = oracle.zstd_frame(data)
        for j, (t, sf, _, streams, n) in enumerate(blocks(frame)[0]):
            if t != "compressed":
                continue
            blk = data[8192 * j:8192 * j + n]
            if max_huffman_depth(blk) > 11:
                continue
            opt = huffman_bits(blk)
            if sf == 0:  # one stream: the optimal bits plus the end mark
                assert streams == (opt + 1 + 7) // 8, (kind, n)
            else:  # four streams, each closed by an end mark
                assert (opt + 4 + 7) // 8 <= streams <= (opt + 4) // 8 + 4, (kind, n)
            checked += 1
    assert checked > 20


def test_length_limit_keeps_codes_within_11_bits():
    data = [d for k, d in inputs() if k == "fib" and len(d) >= 8192][0][:8192]
    assert max_huffman_depth(data) > 11  # the unrestricted optimum is deeper
    frame, _ = oracle.zstd_frame(data)
    (t, _, _, streams, _), = blocks(frame)[0]
    assert t == "compressed"
    assert decompress(frame, len(data)) == data
    assert oracle.zstd_read(frame, len(data)) == data  # the reader refuses codes over 11 bits
    assert streams * 8 >= huffman_bits(data)


# ---------------------------------------------------------------- reader
def test_reader_rejects_damaged_frames():
    rng = np.random.default_rng(5)
    data = np.packbits(rng.random(8 * 20000) < 0.1, bitorder="little").tobytes()
    frame, _ = oracle.zstd_frame(data)
    assert oracle.zstd_read(frame, len(data)) == data
    assert oracle.zstd_read(frame, len(data) + 1) is None  # content size differs
    for cut in (0, 4, 9, 11, len(frame) // 2, len(frame) - 1):
        assert oracle.zstd_read(frame[:cut], len(data)) is None
    assert oracle.zstd_read(frame + b"\0", len(data)) is None
    for at, v in ((0, 0x29), (4, 0x20), (4, 0x60)):
        bad = bytearray(frame)
        bad[at] = v
        assert oracle.zstd_read(bytes(bad), len(data)) is None


# ---------------------------------------------------------------- in a stream
def _quantized_zero_bytes(plane, s, P):
    m = (1 << (8 * s)) - 1
    q = np.minimum(((plane.astype(np.int64) & m) + P // 2) // P, m // P)
    H, W = q.shape
    rb = (W + 7) // 8
    bits = np.zeros((H, 8 * rb), dtype=bool)
    bits[:, :W] = q == 0
    return np.packbits(bits, axis=1, bitorder="little").reshape(-1)


@pytest.mark.parametrize("H,W,force", [(3, 37, -1), (16, 512, 1), (40, 1700, 0)])
def test_stream_masks_are_the_packed_zero_masks(H, W, force):
    rng = np.random.default_rng(H * W)
    attrs = [(4, 10), (1, 1)]
    scans = []
    base = [rng.integers(0, 60000, (H, W), dtype=np.uint32), rng.integers(0, 256, (H, W)).astype(np.uint8)]
    for t in range(4):
        sc = []
        for a, (s, _) in enumerate(attrs):
            v = base[a].copy()
            v[rng.random((H, W)) < 0.15] = 0
            sc.append(v)
        scans.append(sc)
    buf, lens, modes = oracle.encode_sequence(H, W, attrs, scans, force_mode=force, stages=oracle.ZSTD_MASK)
    planes, _ = oracle.decode_sequence(H, W, attrs, buf, len(scans), stages=oracle.ZSTD_MASK)
    pos = 16 + 8 * len(attrs)
    assert buf[18] == 4  # the stage-flag byte carries bit 2
    rb = (W + 7) // 8
    nblk = -(-H * rb // 8192)
    for t in range(len(scans)):
        fh = buf[pos:pos + 8 + 12 * len(attrs)]
        sp = pos + len(fh)
        for a, (s, P) in enumerate(attrs):
            mode = fh[8 + 12 * a]
            sec = int.from_bytes(fh[12 + 12 * a:16 + 12 * a], "little")
            z0 = sp + 8 * H
            fb = int.from_bytes(buf[z0:z0 + 4], "little")
            frame = buf[z0 + 4 + 4 * nblk:z0 + 4 + 4 * nblk + fb]
            want = _quantized_zero_bytes(scans[t][a], s, P)
            if mode == 1:
                want = want ^ _quantized_zero_bytes(scans[t - 1][a], s, P)
            assert decompress(frame, H * rb) == want.tobytes(), (t, a)
            ends = [int.from_bytes(buf[z0 + 4 + 4 * j:z0 + 8 + 4 * j], "little") for j in range(nblk)]
            assert ends[-1] == fb
            sp += sec
        pos = sp
        for a, (s, P) in enumerate(attrs):
            m = (1 << (8 * s)) - 1
            q = np.minimum(((scans[t][a].astype(np.int64) & m) + P // 2) // P, m // P)
            assert np.array_equal(planes[t][a].astype(np.int64), q * P)
    assert pos == len(buf)


def test_zstd_mask_needs_the_mask_stage():
    with pytest.raises(ValueError):
        oracle.Codec(2, 8, [(2, 1)], stages=oracle.ZSTD_MASK | oracle.NO_MASK)


def test_reader_accepts_only_the_writers_subset():
    # valid Zstandard frames that the writer never produces are refused by
    # the reader: a block split other than 8192 bytes, and libzstd's own
    # frames (LZ sequences); libzstd itself restores both
    rng = np.random.default_rng(8)
    data = np.packbits(rng.random(8 * 9000) < 0.1, bitorder="little").tobytes()
    n = len(data)
    # two Raw blocks of 4096 bytes and one of 808: 28 b5 2f fd a0 <n>, blocks
    frame = bytes.fromhex("28b52ffda0") + n.to_bytes(4, "little")
    cuts = [0, 4096, 8192, n]
    for j in range(3):
        size = cuts[j + 1] - cuts[j]
        frame += (int(j == 2) | (size << 3)).to_bytes(3, "little") + data[cuts[j]:cuts[j + 1]]
    assert decompress(frame, n) == data
    assert oracle.zstd_read(frame, n) is None
    z = _libzstd()
    sz, vp = ctypes.c_size_t, ctypes.c_void_p
    z.ZSTD_compress.restype, z.ZSTD_compress.argtypes = sz, [vp, sz, vp, sz, ctypes.c_int]
    src = np.frombuffer(data, dtype=np.uint8).copy()
    dst = np.zeros(2 * n + 1024, dtype=np.uint8)
    k = z.ZSTD_compress(dst.ctypes.data, dst.nbytes, src.ctypes.data, n, 3)
    lib_frame = dst[:k].tobytes()
    assert decompress(lib_frame, n) == data
    assert oracle.zstd_read(lib_frame, n) is None
