"""The stream inspector (paper_2209_08196_gb300.streaminfo) against streams
whose layout is known: the hand-derived fixtures in tests/golden/ (each
section's mask part, block headers and bodies read off the byte listing) and
oracle streams, where the coded counts recovered from the zero masks must equal the frame
headers' nnz."""
import numpy as np
import pytest

import oracle
from paper_2209_08196_gb300 import streaminfo
from tests import golden_io


def _stream(name):
    _, _, _, frames = golden_io.load(name)
    return b"".join(f["bytes"] for f in frames), frames


def test_golden_exceptions_stream_parts():
    # H = 1, W = 8, no zeros: row table 8, class word 4, one block header 4,
    # body 12 (low bits 4, positions 4, high parts 4)
    buf, _ = _stream("stream_1x8_u16_exceptions.txt")
    head, secs = streaminfo.sections(buf)
    assert (head["H"], head["W"], head["A"]) == (1, 8, 1)
    (s,) = secs
    assert (s.mode, s.nnz, s.bytes) == (0, 8, 28)
    assert (s.table_bytes, s.mask_bytes, s.header_bytes, s.body_bytes) == (8, 4, 4, 12)


def test_golden_ipp_stream_modes_and_literal_mask():
    # frame 1 repeats frame 0 (class-0 XOR word, empty body); frame 2's XOR
    # mask is one literal word
    buf, frames = _stream("stream_1x16_u32_ipp.txt")
    _, secs = streaminfo.sections(buf)
    assert [s.mode for s in secs] == [f["mode"][0] for f in frames]
    assert secs[1].mask_bytes == 4 and secs[1].body_bytes == 0
    assert secs[2].mask_bytes == 8


def test_golden_streams_parts_add_up():
    for name in golden_io.names():
        buf, frames = _stream(name)
        _, secs = streaminfo.sections(buf)
        assert len(secs) == len(frames) * len(frames[0]["in"]), name
        for s in secs:
            assert s.coded == s.nnz, name
            assert s.body_bytes >= 0, name


def test_oracle_streams_parts_add_up_and_counts_match_nnz():
    rng = np.random.default_rng(3)
    H, W, attrs = 6, 200, [(4, 10), (2, 1), (1, 1)]
    base = [rng.integers(1, 1 << (8 * s), size=(H, W)).astype(np.int64) for s, _ in attrs]
    scans = []
    for t in range(5):
        planes = []
        for (s, _), b in zip(attrs, base):
            x = np.clip(b + rng.integers(-3, 4, size=b.shape) * (t % 2), 0, (1 << (8 * s)) - 1)
            x[rng.random(x.shape) < 0.3] = 0
            planes.append(x.astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[s]))
        scans.append(planes)
    for force in (-1, 1):
        buf, _, modes = oracle.encode_sequence(H, W, attrs, scans, force_mode=force)
        _, secs = streaminfo.sections(buf)
        assert [s.mode for s in secs] == [m for mm in modes for m in mm]
        for s in secs:
            # the coded count recovered from the masks (P: after undoing the
            # XOR with the previous scan's mask) is the frame header's nnz
            assert s.coded == s.nnz
            assert s.header_bytes >= 4 * ((s.nnz + 127) // 128) and s.body_bytes >= 0
        per = streaminfo.mask_bytes_per_frame(buf)
        assert len(per) == len(scans) and all(m > 0 for m in per)


def test_zstd_mask_streams_parts_add_up():
    # the section's mask as one Zstandard frame (Sec. III-C): the masks read
    # back from the frames give each row's coded count, and they add up to nnz
    import ctypes.util
    if ctypes.util.find_library("zstd") is None:
        pytest.skip("libzstd is not installed")
    rng = np.random.default_rng(4)
    H, W, attrs = 9, 300, [(4, 10), (1, 1)]
    base = [rng.integers(1, 1 << (8 * s), size=(H, W)).astype(np.int64) for s, _ in attrs]
    scans = []
    for t in range(4):
        planes = []
        for (s, _), b in zip(attrs, base):
            x = b.copy()
            x[rng.random(x.shape) < 0.25] = 0
            planes.append(x.astype({1: np.uint8, 2: np.uint16, 4: np.uint32}[s]))
        scans.append(planes)
    for force in (-1, 0, 1):
        buf, _, modes = oracle.encode_sequence(H, W, attrs, scans, force_mode=force, stages=oracle.ZSTD_MASK)
        head, secs = streaminfo.sections(buf)
        assert head["stages"] == [4, 4]
        assert [s.mode for s in secs] == [m for mm in modes for m in mm]
        for s in secs:
            assert s.coded == s.nnz
            assert s.bytes == s.table_bytes + s.mask_bytes + s.header_bytes + s.body_bytes
