"""Python handle on the Jiffy oracle (plain single-threaded C, jiffy_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it to check and time the CUDA library.
The library itself never imports this package. Nothing here is shared with
the CUDA path: the C file is compiled on its own with gcc.

The oracle follows the paper (Ford & Ford, arXiv 2209.08196) step by step:
quantization (Sec. III-A/B), zero bitmask (Sec. III-C), trial I/P selection
(Sec. III-E), mask XOR (Sec. III-D), compaction, residual, delta, ZigZag
(Eq. 1) and PFOR-style packing (Sec. II). A stream may drop the mask, delta or
ZigZag stage (the ablated codecs of Sec. IV-H, Table IV).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jiffy_oracle.c")
_SRC_STD = os.path.join(_HERE, "jiffy_std_oracle.c")
_SRC_ZSTD = os.path.join(_HERE, "jiffy_zstd_oracle.c")
_LIB = os.path.join(_HERE, "libjiffy_oracle.so")

ERR_CAPACITY = 2
ERR_CORRUPT = 3

# stage switches of a stream (Table IV ablations)
NO_MASK = 1
NO_DELTA = 2
NO_ZIGZAG = 4
# not an ablation: the mask coded the paper's way, one Zstandard frame per section (Sec. III-C)
ZSTD_MASK = 8

_DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no target-specific flags)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_STD), os.path.getmtime(_SRC_ZSTD))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp,
                               _SRC, _SRC_STD, _SRC_ZSTD, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u32, i32, u64, i64, vp, sz = (ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t)
        L.jo_quantize.restype = u32
        L.jo_quantize.argtypes = [u32, u32, u32]
        L.jo_zigzag.restype = u32
        L.jo_zigzag.argtypes = [i32]
        L.jo_unzigzag.restype = i32
        L.jo_unzigzag.argtypes = [u32]
        L.jo_block_body_bytes.restype = u32
        L.jo_block_body_bytes.argtypes = [vp, u32, u32]
        L.jo_best_b.restype = u32
        L.jo_best_b.argtypes = [vp, u32]
        L.jo_pack_block.restype = u32
        L.jo_pack_block.argtypes = [vp, u32, u32, vp]
        L.jo_create.restype = vp
        L.jo_create.argtypes = [u32, u32, u32, vp, vp, u32, i32, u32]
        L.jo_destroy.restype = None
        L.jo_destroy.argtypes = [vp]
        L.jo_reset.restype = None
        L.jo_reset.argtypes = [vp]
        L.jo_encode.restype = i64
        L.jo_encode.argtypes = [vp, vp, vp, sz, vp]
        L.jo_decode.restype = i64
        L.jo_decode.argtypes = [vp, vp, sz, vp]
        L.jo_trial_cost.restype = u64
        L.jo_trial_cost.argtypes = [u32, u32, u32, u32, u32, vp, vp, ctypes.c_int]
        L.jo_section_split.restype = u64
        L.jo_section_split.argtypes = [u32, u32, u32, u32, vp, vp, ctypes.c_int, vp, vp]
        L.jz_frame_bound.restype = sz
        L.jz_frame_bound.argtypes = [sz]
        L.jz_block_count.restype = sz
        L.jz_block_count.argtypes = [sz]
        L.jz_write_frame.restype = sz
        L.jz_write_frame.argtypes = [vp, sz, vp, vp]
        L.jz_read_frame.restype = sz
        L.jz_read_frame.argtypes = [vp, sz, vp, sz, vp, sz]
        L.js_azimuth.restype = u32
        L.js_azimuth.argtypes = [i64, i64]
        L.js_elevation.restype = i32
        L.js_elevation.argtypes = [i64, i64, i64]
        L.js_isqrt.restype = u64
        L.js_isqrt.argtypes = [u64, u64]
        L.js_quantize_attr.restype = u32
        L.js_quantize_attr.argtypes = [ctypes.c_float, ctypes.c_float, u32]
        L.js_standardize.restype = ctypes.c_int
        L.js_standardize.argtypes = [vp, u32, u32, u32, vp, ctypes.c_double, ctypes.c_int, ctypes.c_float, u32, u32,
                                     u32, vp, u32, vp, vp, vp, vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def quantize(v: int, P: int, s: int) -> int:
    return lib().jo_quantize(v, P, s)


def zigzag(x: int) -> int:
    return lib().jo_zigzag(x)


def unzigzag(z: int) -> int:
    return lib().jo_unzigzag(z)


def block_body_bytes(z, b: int) -> int:
    z = np.ascontiguousarray(z, dtype=np.uint32)
    return lib().jo_block_body_bytes(_ptr(z), len(z), b)


def best_b(z) -> int:
    z = np.ascontiguousarray(z, dtype=np.uint32)
    return lib().jo_best_b(_ptr(z), len(z))


def pack_block(z, b: int) -> bytes:
    z = np.ascontiguousarray(z, dtype=np.uint32)
    out = np.zeros(4 + 4 * 128 + 4 * 32 + 4 * 128 + 64, dtype=np.uint8)
    n = lib().jo_pack_block(_ptr(z), len(z), b, _ptr(out))
    return out[:n].tobytes()


def trial_cost(cur: np.ndarray, prev: np.ndarray, P: int, mode: int, test_lines: int = 4) -> int:
    H, W = cur.shape
    cur = np.ascontiguousarray(cur)
    prev = np.ascontiguousarray(prev, dtype=cur.dtype)
    return lib().jo_trial_cost(H, W, cur.itemsize, P, test_lines, _ptr(cur), _ptr(prev), mode)


def section_split(cur: np.ndarray, prev: np.ndarray, P: int, mode: int):
    """(section bytes, mask-part bytes, block bytes) of one attribute-scan coded in a forced mode."""
    H, W = cur.shape
    cur = np.ascontiguousarray(cur)
    prev = np.ascontiguousarray(prev, dtype=cur.dtype)
    m = ctypes.c_uint64(0)
    d = ctypes.c_uint64(0)
    sec = lib().jo_section_split(H, W, cur.itemsize, P, _ptr(cur), _ptr(prev), mode,
                                 ctypes.addressof(m), ctypes.addressof(d))
    return sec, m.value, d.value


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__("oracle error %d" % code)
        self.code = code


class Codec:
    """One stateful oracle stream (encoder or decoder role; the state is the
    previous scan's quantized values, Sec. III-D)."""

    def __init__(self, H: int, W: int, attrs, test_lines: int = 4, force_mode: int = -1, stages: int = 0):
        self.H, self.W = H, W
        self.attrs = [(int(s), int(p)) for s, p in attrs]
        self.A = len(self.attrs)
        dt = np.array([s for s, _ in self.attrs], dtype=np.uint8)
        pr = np.array([p for _, p in self.attrs], dtype=np.uint32)
        self._h = lib().jo_create(H, W, self.A, _ptr(dt), _ptr(pr), test_lines, force_mode, stages)
        if not self._h:
            raise ValueError("invalid oracle configuration")

    def close(self):
        if self._h:
            lib().jo_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def reset(self):
        lib().jo_reset(self._h)

    def bound(self) -> int:
        nw = (self.W + 31) // 32
        row = 4 * ((nw + 15) // 16) + 4 * nw + 4 * ((self.W + 127) // 128) + 4 * self.W
        # + 16 + 8 per Zstandard mask block: the option's index, frame and block headers, padding
        nblk = max(1, -(-(self.H * ((self.W + 7) // 8)) // 8192))
        return 16 + 8 * self.A + 8 + 12 * self.A + self.A * (8 * self.H + self.H * row + 16 + 8 * nblk)

    def encode(self, planes, return_modes: bool = False):
        arrs = []
        for (s, _), p in zip(self.attrs, planes):
            a = np.ascontiguousarray(p, dtype=_DT[s])
            assert a.shape == (self.H, self.W)
            arrs.append(a)
        ptrs = (ctypes.c_void_p * self.A)(*[_ptr(a) for a in arrs])
        out = np.zeros(self.bound(), dtype=np.uint8)
        modes = np.zeros(self.A, dtype=np.uint8)
        n = lib().jo_encode(self._h, ptrs, _ptr(out), out.nbytes, _ptr(modes))
        if n < 0:
            raise OracleError(-n)
        b = out[:n].tobytes()
        return (b, [int(m) for m in modes]) if return_modes else b

    def decode(self, buf: bytes):
        """Decodes one frame (plus the stream header before the first one);
        returns (planes, bytes consumed)."""
        src = np.frombuffer(buf, dtype=np.uint8)
        if src.size == 0:
            src = np.zeros(1, dtype=np.uint8)
        outs = [np.zeros((self.H, self.W), dtype=_DT[s]) for s, _ in self.attrs]
        ptrs = (ctypes.c_void_p * self.A)(*[_ptr(o) for o in outs])
        n = lib().jo_decode(self._h, _ptr(src), len(buf), ptrs)
        if n < 0:
            raise OracleError(-n)
        return outs, int(n)


def encode_sequence(H, W, attrs, scans, test_lines=4, force_mode=-1, stages=0):
    """Encodes scans (a list of per-scan plane lists) as one stream; returns
    (bytes of the whole stream, per-frame byte lengths, per-frame modes)."""
    c = Codec(H, W, attrs, test_lines, force_mode, stages)
    parts, lens, modes = [], [], []
    for planes in scans:
        b, m = c.encode(planes, return_modes=True)
        parts.append(b)
        lens.append(len(b))
        modes.append(m)
    c.close()
    return b"".join(parts), lens, modes


def decode_sequence(H, W, attrs, buf: bytes, n_scans: int, stages: int = 0):
    c = Codec(H, W, attrs, stages=stages)
    out, pos = [], 0
    for _ in range(n_scans):
        planes, n = c.decode(buf[pos:])
        out.append(planes)
        pos += n
    c.close()
    return out, pos


# ---------------------------------------------------------------- standardization (Sec. III-A)
ANGLE_UNITS = 1 << 32  # binary angle units per turn


def zstd_frame(data: bytes):
    """The oracle's Zstandard frame of data (the mask frames of Sec. III-C):
    (frame bytes, [end of each block, from the frame's start])."""
    src = np.frombuffer(bytes(data), dtype=np.uint8).copy()
    n = len(src)
    L = lib()
    out = np.zeros(L.jz_frame_bound(n), dtype=np.uint8)
    ends = np.zeros(max(1, L.jz_block_count(n)), dtype=np.uint32)
    k = L.jz_write_frame(_ptr(src), n, _ptr(out), _ptr(ends))
    return out[:k].tobytes(), [int(e) for e in ends]


def zstd_read(frame: bytes, n: int):
    """The oracle's reader of its own frames: n bytes, or None when the frame
    is malformed or outside the subset the writer uses."""
    src = np.frombuffer(bytes(frame), dtype=np.uint8).copy()
    out = np.zeros(max(1, n), dtype=np.uint8)
    L = lib()
    nb = L.jz_block_count(n)
    ends = np.zeros(nb, dtype=np.uint32)
    k = L.jz_read_frame(_ptr(src) if len(src) else None, len(src), _ptr(out), n, _ptr(ends), nb)
    return out[:n].tobytes() if k and k == len(src) else None


def azimuth(X: int, Y: int) -> int:
    """CORDIC azimuth of the integer vector (X, Y), binary angle in [0, 2^32)."""
    return lib().js_azimuth(X, Y)


def elevation(X: int, Y: int, Z: int) -> int:
    """CORDIC elevation of (sqrt(X^2 + Y^2), Z), signed binary angle."""
    return lib().js_elevation(X, Y, Z)


def isqrt(n: int) -> int:
    """floor(sqrt(n)) for n < 2^126."""
    return lib().js_isqrt(n >> 64, n & ((1 << 64) - 1))


def quantize_attr(v: float, scale: float, nbytes: int) -> int:
    return lib().js_quantize_attr(v, scale, nbytes)


def standardize(xyz, H: int, W: int, beam_alt, az0: float = 0.0, clockwise: bool = False, units_per_m: float = 1000.0,
                range_bytes: int = 4, min_range: int = 0, max_range: int = 0xFFFFFFFF, attrs=()):
    """Standardizes one scan: xyz (n x 3 float32, metres) -> (range image,
    [attribute images]). attrs: list of (values (n float32), bytes, scale)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    n = xyz.shape[0]
    alt = np.ascontiguousarray(beam_alt, dtype=np.float64)
    assert alt.shape == (H,)
    rng_out = np.zeros((H, W), dtype=_DT[range_bytes])
    A = len(attrs)
    vals = [np.ascontiguousarray(v, dtype=np.float32) for v, _, _ in attrs]
    outs = [np.zeros((H, W), dtype=_DT[b]) for _, b, _ in attrs]
    vp = (ctypes.c_void_p * max(A, 1))(*[_ptr(v) for v in vals])
    op = (ctypes.c_void_p * max(A, 1))(*[_ptr(o) for o in outs])
    nb = np.array([b for _, b, _ in attrs] or [4], dtype=np.uint32)
    sc = np.array([s for _, _, s in attrs] or [1.0], dtype=np.float32)
    src = xyz if n else np.zeros((1, 3), dtype=np.float32)
    rc = lib().js_standardize(_ptr(src), n, H, W, _ptr(alt), az0, int(clockwise), units_per_m, range_bytes,
                              min_range, max_range, _ptr(rng_out), A, vp, _ptr(nb), _ptr(sc), op)
    if rc != 0:
        raise ValueError("invalid standardization arguments")
    return rng_out, outs
