"""Host-side inspection of a Jiffy stream: where its bytes go.

Walks the stream's structures (stream header, frame headers, per-attribute
sections with their row tables and row chunks) and reports, per section, the
mode (I or P, Sec. III-C / III-D) and how its bytes split into the row table,
the zero-mask part (class words and literal mask words, or the section's
Zstandard frame), the packing blocks' headers and their bodies. This is a
reader of the byte layout, for reports and analysis (for instance the size of
the mask part against another mask coder); it decodes no values and checks
only what it needs to walk. Streams with the Zstandard mask are read with the
host's libzstd (through ctypes), which must then be installed.
"""
from __future__ import annotations

import ctypes
import ctypes.util
from dataclasses import dataclass

import numpy as np

MAGIC = 0x3159464A  # "JFY1"
STAGE_NO_MASK = 1
FLAG_ZSTD_MASK = 4   # stage-flag bit of the stream header: the mask is one Zstandard frame per section
ZSTD_BLOCK = 8192    # mask bytes per block of that frame


def _zstd_decompress(frame: bytes, n: int) -> np.ndarray:
    path = ctypes.util.find_library("zstd")
    if path is None:
        raise RuntimeError("reading a stream with the Zstandard mask needs libzstd")
    z = ctypes.CDLL(path)
    sz, vp = ctypes.c_size_t, ctypes.c_void_p
    z.ZSTD_decompress.restype, z.ZSTD_decompress.argtypes = sz, [vp, sz, vp, sz]
    z.ZSTD_isError.restype, z.ZSTD_isError.argtypes = ctypes.c_uint, [sz]
    src = np.frombuffer(frame, dtype=np.uint8).copy()
    out = np.zeros(max(n, 1), dtype=np.uint8)
    k = z.ZSTD_decompress(out.ctypes.data, out.nbytes, src.ctypes.data, len(src))
    if z.ZSTD_isError(k) or k != n:
        raise ValueError("a mask frame does not decompress to the section's mask")
    return out[:n]


@dataclass
class SectionInfo:
    frame: int
    attr: int
    mode: int            # 0 = I, 1 = P
    nnz: int             # samples coded
    bytes: int           # whole section
    table_bytes: int     # row table (8 per row)
    mask_bytes: int      # class words + literal mask words, all rows
    header_bytes: int    # packing block headers, all rows
    body_bytes: int      # packing block bodies, all rows
    coded: int           # samples coded according to the zero masks (equals nnz in a valid stream)


_SHIFTS = np.arange(0, 32, 2, dtype=np.uint64)[None, :]


def _popcount32(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint64)
    x = x - ((x >> 1) & 0x55555555)
    x = (x & 0x33333333) + ((x >> 2) & 0x33333333)
    x = (x + (x >> 4)) & 0x0F0F0F0F
    return ((x * 0x01010101) & 0xFFFFFFFF) >> 24


def sections(buf: bytes, n_frames: int | None = None) -> tuple[dict, list[SectionInfo]]:
    """(stream header fields, [SectionInfo]) of a stream that starts with a
    stream header. n_frames: stop after that many frames (default: all)."""
    if len(buf) % 4:
        raise ValueError("a stream is a whole number of 32-bit words")
    w = np.frombuffer(buf, dtype="<u4")
    if int(w[0]) != MAGIC or (int(w[1]) & 0xFFFF) != 1:
        raise ValueError("not a version-1 Jiffy stream")
    A = int(w[1]) >> 16
    H, W = int(w[2]), int(w[3])
    attr_words = [int(w[4 + 2 * a]) for a in range(A)]
    head = {"A": A, "H": H, "W": W, "dtype_bytes": [x & 0xFF for x in attr_words],
            "stages": [(x >> 16) & 0xFF for x in attr_words], "precision": [int(w[5 + 2 * a]) for a in range(A)]}
    nw = (W + 31) // 32
    last_valid = (1 << (W % 32)) - 1 if W % 32 else 0xFFFFFFFF
    prev = [np.zeros((H, nw), dtype=np.uint32) for _ in range(A)]  # each attribute's last zero masks
    prev_bits = [np.zeros((H, W), dtype=bool) for _ in range(A)]     # the same, with the Zstandard mask
    rb = (W + 7) // 8
    at = 16 + 8 * A
    out = []
    t = 0
    while at < len(buf) and (n_frames is None or t < n_frames):
        fw = at // 4
        fbytes = int(w[fw])
        sec = at + 8 + 12 * A
        for a in range(A):
            mode = int(w[fw + 2 + 3 * a]) & 0xFF
            sbytes = int(w[fw + 3 + 3 * a])
            nnz = int(w[fw + 4 + 3 * a])
            no_mask = head["stages"][a] & STAGE_NO_MASK
            zmask = head["stages"][a] & FLAG_ZSTD_MASK
            ncls = 0 if (no_mask or zmask) else (nw + 15) // 16
            ends = w[sec // 4:sec // 4 + 2 * H:2].astype(np.int64)
            starts = np.concatenate([[0], ends[:-1]])
            data = sec + 8 * H
            mask_b = head_b = coded = 0
            masks = prev[a]
            if zmask:  # u32 frame bytes, u32 block ends, the frame, padding
                nblk = max(1, -(-(H * rb) // ZSTD_BLOCK))
                fb = int(w[data // 4])
                f0 = data + 4 + 4 * nblk
                part = (4 + 4 * nblk + fb + 3) & ~3
                packed = _zstd_decompress(buf[f0:f0 + fb], H * rb).reshape(H, rb)
                bits = np.unpackbits(packed, axis=1, bitorder="little")[:, :W].astype(bool)
                if mode == 1:
                    bits ^= prev_bits[a]
                prev_bits[a] = bits
                n_rows = W - bits.sum(axis=1)
                mask_b = part
                head_b = int(sum(4 * ((int(n) + 127) // 128) for n in n_rows))
                coded = int(n_rows.sum())
                chunks = int(ends[-1]) if H else 0
                out.append(SectionInfo(t, a, mode, nnz, sbytes, 8 * H, mask_b, head_b, chunks - head_b, coded))
                sec += sbytes
                continue
            for r in range(H):
                c0 = (data + int(starts[r])) // 4
                if no_mask:
                    n = W
                    nlit = 0
                else:
                    cw = w[c0:c0 + ncls].astype(np.uint64)
                    kinds = ((cw[:, None] >> _SHIFTS) & 3).reshape(-1)[:nw]
                    nlit = int((kinds == 2).sum())
                    # the mask words as written (class 1: every valid bit set;
                    # class 2: the literals in order), then, for P, the XOR
                    # with the previous scan's mask undone (Sec. III-D)
                    words = np.zeros(nw, dtype=np.uint32)
                    words[kinds == 1] = 0xFFFFFFFF
                    if kinds[-1] == 1:
                        words[-1] = last_valid
                    words[kinds == 2] = w[c0 + ncls:c0 + ncls + nlit]
                    if mode == 1:
                        words ^= masks[r]
                    masks[r] = words
                    n = W - int(_popcount32(words).sum())
                mask_b += 4 * (ncls + nlit)
                head_b += 4 * ((n + 127) // 128)
                coded += n
            chunks = int(ends[-1]) if H else 0
            out.append(SectionInfo(t, a, mode, nnz, sbytes, 8 * H, mask_b, head_b, chunks - mask_b - head_b,
                                   coded))
            sec += sbytes
        at += fbytes  # frame bytes run from the frame header to the end of its sections
        t += 1
    return head, out


def mask_bytes_per_frame(buf: bytes, n_frames: int | None = None) -> list[int]:
    """Bytes of the zero-mask parts of each frame (all attributes)."""
    _, secs = sections(buf, n_frames)
    per = {}
    for s in secs:
        per[s.frame] = per.get(s.frame, 0) + s.mask_bytes
    return [per[t] for t in sorted(per)]
