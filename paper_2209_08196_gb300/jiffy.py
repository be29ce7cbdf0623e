"""Python binding of the Jiffy C ABI (include/jiffy.h), argument marshalling
only: every step of encode and decode runs in the CUDA kernels of
libjiffy_gb300.so. PyTorch supplies device memory and streams.

The functions keep the C names. Planes are CUDA tensors of H x W samples
with 1, 2 or 4 bytes per element (uint8, int16/uint16, int32/uint32: only
the bytes matter); byte buffers are uint8 CUDA tensors. There is no CPU
fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libjiffy_gb300.so")

JIFFY_ENCODER, JIFFY_DECODER = 0, 1
STATUS = {
    0: "JIFFY_OK", 1: "JIFFY_ERR_INVALID_ARG", 2: "JIFFY_ERR_CAPACITY", 3: "JIFFY_ERR_CORRUPT",
    4: "JIFFY_ERR_STATE", 5: "JIFFY_ERR_TIMEOUT", 6: "JIFFY_ERR_CUDA", 7: "JIFFY_ERR_NOMEM",
}


class JiffyError(RuntimeError):
    def __init__(self, status: int, what: str = "", required: int | None = None):
        self.status = status
        self.name = STATUS.get(status, str(status))
        self.required = required
        super().__init__("%s%s: %s" % (what + ": " if what else "", self.name, _lib().jiffy_status_string(status).decode()))


class _AttrDesc(ctypes.Structure):
    _fields_ = [("dtype_bytes", ctypes.c_uint32), ("precision", ctypes.c_uint32)]


class _Options(ctypes.Structure):
    _fields_ = [("test_lines", ctypes.c_uint32), ("force_mode", ctypes.c_int32), ("stages", ctypes.c_uint32)]


class _SensorDesc(ctypes.Structure):
    _fields_ = [("H", ctypes.c_uint32), ("W", ctypes.c_uint32), ("beam_altitude", ctypes.POINTER(ctypes.c_double)),
                ("azimuth0", ctypes.c_double), ("clockwise", ctypes.c_int32), ("units_per_m", ctypes.c_float),
                ("range_bytes", ctypes.c_uint32), ("min_range", ctypes.c_uint32), ("max_range", ctypes.c_uint32)]


class _PointAttr(ctypes.Structure):
    _fields_ = [("values", ctypes.c_void_p), ("out", ctypes.c_void_p), ("scale", ctypes.c_float),
                ("dtype_bytes", ctypes.c_uint32)]


# stage switches (jiffy_options.stages): the ablated codecs of Sec. IV-H
STAGE_NO_MASK = 1
STAGE_NO_DELTA = 2
STAGE_NO_ZIGZAG = 4
STAGE_ZSTD_MASK = 8  # the zero mask as one Zstandard frame per section (Sec. III-C)


_L = None
_ENC_BATCH_ADDR = _DEC_BATCH_ADDR = None


def _lib() -> ctypes.CDLL:
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libjiffy_gb300.so is not built (run paper_2209_08196_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, i32, sz, u64p = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)
        L.jiffy_status_string.restype = ctypes.c_char_p
        L.jiffy_status_string.argtypes = [ctypes.c_int]
        L.jiffy_stream_create.restype = ctypes.c_int
        L.jiffy_stream_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, u32, u32, u32, ctypes.POINTER(_AttrDesc),
                                          ctypes.POINTER(_Options), ctypes.c_int]
        L.jiffy_stream_destroy.restype = None
        L.jiffy_stream_destroy.argtypes = [vp]
        L.jiffy_stream_reset.restype = ctypes.c_int
        L.jiffy_stream_reset.argtypes = [vp]
        L.jiffy_stream_frame_index.restype = u32
        L.jiffy_stream_frame_index.argtypes = [vp]
        L.jiffy_stream_set_profiling.restype = ctypes.c_int
        L.jiffy_stream_set_profiling.argtypes = [vp, ctypes.c_int]
        L.jiffy_stream_kernel_times.restype = u32
        L.jiffy_stream_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), u32]
        L.jiffy_max_encoded_size.restype = sz
        L.jiffy_max_encoded_size.argtypes = [u32, u32, u32, ctypes.POINTER(_AttrDesc), u32]
        L.jiffy_encode.restype = ctypes.c_int
        L.jiffy_encode.argtypes = [vp, ctypes.POINTER(vp), vp, sz, ctypes.POINTER(sz), vp]
        L.jiffy_encode_seq.restype = ctypes.c_int
        L.jiffy_encode_seq.argtypes = [vp, u32, ctypes.POINTER(vp), vp, sz, u64p, ctypes.POINTER(sz), vp]
        L.jiffy_decode.restype = ctypes.c_int
        L.jiffy_decode.argtypes = [vp, vp, sz, ctypes.POINTER(vp), vp]
        L.jiffy_decode_seq.restype = ctypes.c_int
        L.jiffy_decode_seq.argtypes = [vp, u32, vp, sz, u64p, ctypes.POINTER(vp), vp]
        L.jiffy_decode_frame_noalloc.restype = ctypes.c_int
        L.jiffy_encode_seq_async.argtypes = [vp, u32, ctypes.POINTER(vp), vp, sz, vp, vp]
        L.jiffy_encode_seq_async.restype = ctypes.c_int
        L.jiffy_decode_seq_async.argtypes = [vp, u32, vp, sz, vp, ctypes.POINTER(vp), vp]
        L.jiffy_decode_seq_async.restype = ctypes.c_int
        L.jiffy_stream_wait.argtypes = [vp]
        L.jiffy_stream_wait.restype = ctypes.c_int
        L.jiffy_decode_frame_noalloc.argtypes = [vp, sz, u32, u32, u32, ctypes.POINTER(_AttrDesc), u32, u32,
                                                 ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        L.jiffy_batch_create.restype = ctypes.c_int
        L.jiffy_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
        L.jiffy_batch_destroy.restype = None
        L.jiffy_batch_destroy.argtypes = [vp]
        L.jiffy_batch_set_profiling.restype = ctypes.c_int
        L.jiffy_batch_set_profiling.argtypes = [vp, ctypes.c_int]
        L.jiffy_batch_kernel_times.restype = u32
        L.jiffy_batch_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), u32]
        pp = ctypes.POINTER(vp)
        L.jiffy_encode_batch.restype = ctypes.c_int
        L.jiffy_encode_batch.argtypes = [vp, u32, pp, ctypes.POINTER(u32), pp, pp, ctypes.POINTER(sz), pp,
                                         ctypes.POINTER(sz), ctypes.POINTER(ctypes.c_int), vp]
        L.jiffy_decode_batch.restype = ctypes.c_int
        L.jiffy_decode_batch.argtypes = [vp, u32, pp, ctypes.POINTER(u32), pp, ctypes.POINTER(sz), pp, pp,
                                         ctypes.POINTER(ctypes.c_int), vp]
        L.jiffy_encode_batch_async.restype = ctypes.c_int
        L.jiffy_encode_batch_async.argtypes = L.jiffy_encode_batch.argtypes
        L.jiffy_decode_batch_async.restype = ctypes.c_int
        L.jiffy_decode_batch_async.argtypes = L.jiffy_decode_batch.argtypes
        L.jiffy_batch_wait.restype = ctypes.c_int
        L.jiffy_batch_wait.argtypes = [vp]
        # the same batched entry points over plain addresses (array-marshalled calls)
        global _ENC_BATCH_ADDR, _DEC_BATCH_ADDR
        _ENC_BATCH_ADDR = ctypes.CFUNCTYPE(ctypes.c_int, vp, u32, *([vp] * 9))(("jiffy_encode_batch_async", L))
        _DEC_BATCH_ADDR = ctypes.CFUNCTYPE(ctypes.c_int, vp, u32, *([vp] * 8))(("jiffy_decode_batch_async", L))
        L.jiffy_batch_set_graphs.restype = ctypes.c_int
        L.jiffy_batch_set_graphs.argtypes = [vp, ctypes.c_int]
        L.jiffy_batch_set_autotune.restype = ctypes.c_int
        L.jiffy_batch_set_autotune.argtypes = [vp, ctypes.c_int]
        L.jiffy_batch_set_launch.restype = ctypes.c_int
        L.jiffy_batch_set_launch.argtypes = [vp, ctypes.c_int, u32, u32, u32]
        L.jiffy_batch_info.restype = ctypes.c_int
        L.jiffy_batch_info.argtypes = [vp, u64p, u32]
        L.jiffy_stream_copy_state.restype = ctypes.c_int
        L.jiffy_stream_copy_state.argtypes = [vp, vp, vp]
        L.jiffy_stream_state_size.restype = sz
        L.jiffy_stream_state_size.argtypes = [vp]
        L.jiffy_stream_save_state.restype = ctypes.c_int
        L.jiffy_stream_save_state.argtypes = [vp, vp, sz]
        L.jiffy_stream_load_state.restype = ctypes.c_int
        L.jiffy_stream_load_state.argtypes = [vp, vp, sz]
        L.jiffy_stream_device_bytes.restype = sz
        L.jiffy_stream_device_bytes.argtypes = [vp]
        L.jiffy_stream_test_withhold_row.argtypes = [vp, u32]
        L.jiffy_standardizer_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_SensorDesc), ctypes.c_int]
        L.jiffy_standardizer_destroy.restype = None
        L.jiffy_standardizer_destroy.argtypes = [vp]
        L.jiffy_standardize.argtypes = [vp, vp, u32, vp, u32, ctypes.POINTER(_PointAttr), vp]
        L.jiffy_standardize_seq.argtypes = [vp, u32, vp, u64p, vp, u32, ctypes.POINTER(_PointAttr), vp]
        _L = L
    return _L


def loaded_library_path() -> str:
    _lib()
    return LIB_PATH


def _attrs(attrs):
    arr = (_AttrDesc * len(attrs))()
    for i, (s, p) in enumerate(attrs):
        arr[i].dtype_bytes = int(s)
        arr[i].precision = int(p)
    return arr


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _check_plane(t: torch.Tensor, H: int, W: int, s: int, what: str):
    if not t.is_cuda or t.element_size() != s or not t.is_contiguous() or t.numel() != H * W:
        raise ValueError("%s: expected a contiguous CUDA tensor of %d x %d %d-byte samples, got %s %s %s"
                         % (what, H, W, s, tuple(t.shape), t.dtype, t.device))


class Handle:
    """An opaque jiffy_stream* with the configuration it was created with."""

    def __init__(self, ptr, role, H, W, attrs, device):
        self.ptr, self.role, self.H, self.W, self.attrs, self.device = ptr, role, H, W, list(attrs), device
        self._ptr_cache = {}  # (T, attribute base addresses) -> ctypes pointer array

    @property
    def A(self):
        return len(self.attrs)

    def __del__(self):
        if getattr(self, "ptr", None) and _L is not None:
            _L.jiffy_stream_destroy(self.ptr)
            self.ptr = None


def jiffy_stream_create(role: int, H: int, W: int, attrs, test_lines: int = 4, force_mode: int = -1,
                        device: int = 0, stages: int = 0) -> Handle:
    L = _lib()
    h = ctypes.c_void_p()
    opt = _Options(test_lines, force_mode, stages)
    st = L.jiffy_stream_create(ctypes.byref(h), role, H, W, len(attrs), _attrs(attrs), ctypes.byref(opt), device)
    if st != 0:
        raise JiffyError(st, "jiffy_stream_create")
    return Handle(h.value, role, H, W, attrs, device)


def jiffy_stream_destroy(h: Handle):
    if h.ptr:
        _lib().jiffy_stream_destroy(h.ptr)
        h.ptr = None


def jiffy_stream_reset(h: Handle):
    st = _lib().jiffy_stream_reset(h.ptr)
    if st != 0:
        raise JiffyError(st, "jiffy_stream_reset")


def jiffy_stream_frame_index(h: Handle) -> int:
    return _lib().jiffy_stream_frame_index(h.ptr)


def jiffy_stream_set_profiling(h: Handle, enable: bool = True):
    st = _lib().jiffy_stream_set_profiling(h.ptr, int(bool(enable)))
    if st != 0:
        raise JiffyError(st, "jiffy_stream_set_profiling")


def jiffy_stream_kernel_times(h: Handle):
    """Device ms of each kernel of the last call (launch order)."""
    buf = (ctypes.c_float * 8)()
    n = _lib().jiffy_stream_kernel_times(h.ptr, buf, 8)
    return [float(buf[i]) for i in range(min(n, 8))]


def jiffy_max_encoded_size(H: int, W: int, attrs, n_scans: int = 1) -> int:
    return _lib().jiffy_max_encoded_size(H, W, len(attrs), _attrs(attrs), n_scans)


def _ptr_array(tensors):
    return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])


def jiffy_encode(h: Handle, planes, out: torch.Tensor, stream=None) -> int:
    """Encodes one scan (list of A planes) into out (uint8 CUDA tensor);
    returns the bytes written."""
    for a, (p, (s, _)) in enumerate(zip(planes, h.attrs)):
        _check_plane(p, h.H, h.W, s, "plane %d" % a)
    n = ctypes.c_size_t(0)
    st = _lib().jiffy_encode(h.ptr, _ptr_array(planes), out.data_ptr(), out.numel() * out.element_size(),
                             ctypes.byref(n), _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_encode", required=n.value if st == 2 else None)
    return n.value


def _seq_planes(h: Handle, planes):
    """planes: list over attributes of T x H x W tensors, or list over scans
    of lists over attributes. Returns (T, flat scan-major list)."""
    if isinstance(planes[0], torch.Tensor) and len(planes) == h.A and planes[0].dim() == 3:
        T = planes[0].shape[0]
        flat = []
        for t in range(T):
            for a in range(h.A):
                flat.append(planes[a][t])
        return T, flat
    T = len(planes)
    return T, [p for scan in planes for p in scan]


def _seq_ptrs(h: Handle, planes, what: str):
    """(T, ctypes array of the T * A plane pointers, scan-major). A list over
    attributes of contiguous T x H x W tensors is checked once per attribute
    and addressed by arithmetic; any other form is checked plane by plane."""
    if isinstance(planes[0], torch.Tensor) and len(planes) == h.A and planes[0].dim() == 3:
        T = planes[0].shape[0]
        bases, steps = [], []
        for a, (p, (s, _)) in enumerate(zip(planes, h.attrs)):
            if p.shape[0] != T or not p.is_cuda or p.element_size() != s or not p.is_contiguous() or \
                    p.shape[1] * p.shape[2] != h.H * h.W:
                raise ValueError("%s %d: expected a contiguous CUDA tensor of %d x %d x %d %d-byte samples, got %s %s"
                                 % (what, a, T, h.H, h.W, s, tuple(p.shape), p.dtype))
            bases.append(p.data_ptr())
            steps.append(h.H * h.W * s)
        key = (T, tuple(bases))
        arr = h._ptr_cache.get(key)
        if arr is None:
            A = h.A
            ptrs = [bases[a] + t * steps[a] for t in range(T) for a in range(A)]
            arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
            if len(h._ptr_cache) >= 8:
                h._ptr_cache.clear()
            h._ptr_cache[key] = arr
        return T, arr
    T, flat = _seq_planes(h, planes)
    for i, p in enumerate(flat):
        _check_plane(p, h.H, h.W, h.attrs[i % h.A][0], "%s %d" % (what, i))
    return T, _ptr_array(flat)


def jiffy_encode_seq(h: Handle, planes, out: torch.Tensor, stream=None):
    """Encodes T consecutive scans in one pass; returns (total bytes, list of
    T + 1 frame offsets)."""
    T, arr = _seq_ptrs(h, planes, "plane")
    offs = (ctypes.c_uint64 * (T + 1))()
    n = ctypes.c_size_t(0)
    st = _lib().jiffy_encode_seq(h.ptr, T, arr, out.data_ptr(), out.numel() * out.element_size(),
                                 offs, ctypes.byref(n), _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_encode_seq", required=n.value if st == 2 else None)
    return n.value, list(offs)


def jiffy_encode_seq_async(h: Handle, planes, out: torch.Tensor, offsets_dev: torch.Tensor, stream=None):
    """Enqueues the encode of T consecutive scans without waiting; the T + 1
    frame offsets (the last = bytes written) go to offsets_dev, a device
    int64 tensor of at least T + 1 entries. Device errors come back from
    jiffy_stream_wait."""
    T, arr = _seq_ptrs(h, planes, "plane")
    if offsets_dev.numel() < T + 1 or offsets_dev.element_size() != 8 or not offsets_dev.is_cuda:
        raise ValueError("offsets_dev: a device tensor of T + 1 64-bit entries")
    st = _lib().jiffy_encode_seq_async(h.ptr, T, arr, out.data_ptr(), out.numel() * out.element_size(),
                                       offsets_dev.data_ptr(), _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_encode_seq_async")


def jiffy_decode_seq_async(h: Handle, buf: torch.Tensor, offsets_dev: torch.Tensor, planes_out, stream=None):
    """Enqueues the decode of T frames of buf whose offsets are in the device
    tensor offsets_dev (as jiffy_encode_seq_async writes them); the kernel
    checks them against buf's size. Device errors come back from
    jiffy_stream_wait."""
    T, arr = _seq_ptrs(h, planes_out, "output plane")
    if offsets_dev.numel() < T + 1 or offsets_dev.element_size() != 8 or not offsets_dev.is_cuda:
        raise ValueError("offsets_dev: a device tensor of T + 1 64-bit entries")
    st = _lib().jiffy_decode_seq_async(h.ptr, T, buf.data_ptr(), buf.numel() * buf.element_size(),
                                       offsets_dev.data_ptr(), arr, _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_decode_seq_async")


def jiffy_stream_wait(h: Handle):
    """Waits for the stream's enqueue-only calls; raises the error the device
    reported for any of them (the stream must then be reset)."""
    st = _lib().jiffy_stream_wait(h.ptr)
    if st != 0:
        raise JiffyError(st, "jiffy_stream_wait")


def jiffy_decode(h: Handle, buf: torch.Tensor, length: int, planes_out, stream=None):
    """Decodes one frame of `length` bytes at the start of buf into planes_out."""
    for a, (p, (s, _)) in enumerate(zip(planes_out, h.attrs)):
        _check_plane(p, h.H, h.W, s, "output plane %d" % a)
    st = _lib().jiffy_decode(h.ptr, buf.data_ptr(), length, _ptr_array(planes_out), _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_decode")


def jiffy_decode_seq(h: Handle, buf: torch.Tensor, length: int, offsets, planes_out, stream=None):
    """Decodes T frames whose byte offsets (T + 1 entries) are `offsets`."""
    T, arr = _seq_ptrs(h, planes_out, "output plane")
    if len(offsets) != T + 1:
        raise ValueError("need T + 1 frame offsets")
    offs = (ctypes.c_uint64 * (T + 1))(*[int(o) for o in offsets])
    st = _lib().jiffy_decode_seq(h.ptr, T, buf.data_ptr(), length, offs, arr, _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_decode_seq")


def jiffy_decode_frame_noalloc(buf: torch.Tensor, length: int, H: int, W: int, attrs, scan_index: int,
                               prev_planes, planes_out, stream=None, stages: int = 0):
    """Decodes one frame without a stream handle and without allocating
    device memory (for callers that may not allocate once running). Pass the
    previous frame's decoded planes as prev_planes (or None when the frame has
    no P attribute; planes_out itself decodes in place) and the stream's stage
    switches."""
    for a, (p, (s, _)) in enumerate(zip(planes_out, attrs)):
        _check_plane(p, H, W, s, "output plane %d" % a)
    prev = None
    if prev_planes is not None:
        for a, (p, (s, _)) in enumerate(zip(prev_planes, attrs)):
            _check_plane(p, H, W, s, "previous plane %d" % a)
        prev = _ptr_array(prev_planes)
    st = _lib().jiffy_decode_frame_noalloc(buf.data_ptr(), length, H, W, len(attrs), _attrs(attrs), scan_index,
                                           stages, prev, _ptr_array(planes_out), _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_decode_frame_noalloc")


class Batch:
    """An opaque jiffy_batch*: scratch of many-stream calls on one device."""

    def __init__(self, ptr, device):
        self.ptr, self.device = ptr, device

    def __del__(self):
        if getattr(self, "ptr", None) and _L is not None:
            _L.jiffy_batch_destroy(self.ptr)
            self.ptr = None


def jiffy_batch_create(device: int = 0) -> Batch:
    h = ctypes.c_void_p()
    st = _lib().jiffy_batch_create(ctypes.byref(h), device)
    if st != 0:
        raise JiffyError(st, "jiffy_batch_create")
    return Batch(h.value, device)


def jiffy_batch_destroy(b: Batch):
    if b.ptr:
        _lib().jiffy_batch_destroy(b.ptr)
        b.ptr = None


def jiffy_batch_set_profiling(b: Batch, enable: bool = True):
    st = _lib().jiffy_batch_set_profiling(b.ptr, int(bool(enable)))
    if st != 0:
        raise JiffyError(st, "jiffy_batch_set_profiling")


def jiffy_batch_kernel_times(b: Batch):
    buf = (ctypes.c_float * 8)()
    n = _lib().jiffy_batch_kernel_times(b.ptr, buf, 8)
    return [float(buf[i]) for i in range(min(n, 8))]


class BatchError(JiffyError):
    """A batched call failed for some streams; .statuses has one code per
    stream (0 = that stream succeeded and advanced)."""

    def __init__(self, status, what, statuses, required=None, result=None):
        super().__init__(status, what)
        self.statuses = list(statuses)
        self.required = required
        self.result = result  # array-marshalled encode: (bytes, offsets, starts) of the streams that succeeded


def jiffy_batch_set_graphs(b: Batch, enable: bool = True):
    st = _lib().jiffy_batch_set_graphs(b.ptr, int(bool(enable)))
    if st != 0:
        raise JiffyError(st, "jiffy_batch_set_graphs")


def jiffy_batch_set_autotune(b: Batch, enable: bool = True):
    st = _lib().jiffy_batch_set_autotune(b.ptr, int(bool(enable)))
    if st != 0:
        raise JiffyError(st, "jiffy_batch_set_autotune")


def jiffy_batch_set_launch(b: Batch, role: int, warps_per_cta: int = 0, ctas_per_sm: int = 0,
                           items_per_ticket: int = 0):
    st = _lib().jiffy_batch_set_launch(b.ptr, role, warps_per_cta, ctas_per_sm, items_per_ticket)
    if st != 0:
        raise JiffyError(st, "jiffy_batch_set_launch")


BATCH_INFO = ("calls", "graph_captures", "graph_replays", "tunings", "tuned_classes",
              "warps_per_cta", "ctas_per_sm", "items_per_ticket", "grid")


def jiffy_batch_info(b: Batch) -> dict:
    buf = (ctypes.c_uint64 * len(BATCH_INFO))()
    st = _lib().jiffy_batch_info(b.ptr, buf, len(BATCH_INFO))
    if st != 0:
        raise JiffyError(st, "jiffy_batch_info")
    return {k: int(v) for k, v in zip(BATCH_INFO, buf)}


def jiffy_stream_copy_state(dst: Handle, src: Handle, stream=None):
    st = _lib().jiffy_stream_copy_state(dst.ptr, src.ptr, _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_stream_copy_state")


def jiffy_stream_save_state(h: Handle) -> bytes:
    """The stream's state (previous scan as decoded and frame counter) as
    bytes, for checkpoint / resume."""
    n = _lib().jiffy_stream_state_size(h.ptr)
    buf = (ctypes.c_uint8 * n)()
    st = _lib().jiffy_stream_save_state(h.ptr, buf, n)
    if st != 0:
        raise JiffyError(st, "jiffy_stream_save_state")
    return bytes(buf)


def jiffy_stream_load_state(h: Handle, state: bytes):
    """Restores a state saved by jiffy_stream_save_state into a stream of the
    same configuration; its next frame continues the saved stream."""
    buf = (ctypes.c_uint8 * len(state)).from_buffer_copy(state) if state else (ctypes.c_uint8 * 1)()
    st = _lib().jiffy_stream_load_state(h.ptr, buf, len(state))
    if st != 0:
        raise JiffyError(st, "jiffy_stream_load_state")


def jiffy_stream_test_withhold_row(h: Handle, row_item: int):
    """Test hook: the stream's next call leaves row item `row_item` unpublished
    (a row that waits on it gives up after the bounded wait: JIFFY_ERR_TIMEOUT)."""
    st = _lib().jiffy_stream_test_withhold_row(h.ptr, row_item)
    if st != 0:
        raise JiffyError(st, "jiffy_stream_test_withhold_row")


def jiffy_stream_device_bytes(h: Handle) -> int:
    return _lib().jiffy_stream_device_bytes(h.ptr)


def _addr(a) -> int:
    return ctypes.cast(a, ctypes.c_void_p).value


class _EncCall:
    """Marshalled arguments of one batched encode (kept alive until it ends)."""

    def __init__(self, handles, planes, outs):
        n = len(handles)
        flats = [_seq_ptrs(h, pl, "plane") for h, pl in zip(handles, planes)]
        self.n = n
        self.streams = (ctypes.c_void_p * n)(*[h.ptr for h in handles])
        self.n_scans = (ctypes.c_uint32 * n)(*[T for T, _ in flats])
        self.parr = [arr for _, arr in flats]
        self.planes = (ctypes.c_void_p * n)(*[_addr(a) for a in self.parr])
        self.outs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        self.caps = (ctypes.c_size_t * n)(*[o.numel() * o.element_size() for o in outs])
        self.offs = [(ctypes.c_uint64 * (T + 1))() for T, _ in flats]
        self.offs_pp = (ctypes.c_void_p * n)(*[_addr(a) for a in self.offs])
        self.lens = (ctypes.c_size_t * n)()
        self.sts = (ctypes.c_int * n)()

    def args(self, b, stream):
        return (b.ptr, self.n, self.streams, self.n_scans, self.planes, self.outs, self.caps, self.offs_pp,
                self.lens, self.sts, _stream_ptr(stream))

    def result(self):
        return [(self.lens[i], list(self.offs[i])) for i in range(self.n)]


class _DecCall:
    def __init__(self, handles, bufs, lengths, offsets, planes_out):
        n = len(handles)
        flats = [_seq_ptrs(h, pl, "output plane") for h, pl in zip(handles, planes_out)]
        for (T, _), o in zip(flats, offsets):
            if len(o) != T + 1:
                raise ValueError("need T + 1 frame offsets")
        self.n = n
        self.streams = (ctypes.c_void_p * n)(*[h.ptr for h in handles])
        self.n_frames = (ctypes.c_uint32 * n)(*[T for T, _ in flats])
        self.ins = (ctypes.c_void_p * n)(*[x.data_ptr() for x in bufs])
        self.lens = (ctypes.c_size_t * n)(*[int(x) for x in lengths])
        self.offs = [(ctypes.c_uint64 * len(o))(*[int(v) for v in o]) for o in offsets]
        self.offs_pp = (ctypes.c_void_p * n)(*[_addr(a) for a in self.offs])
        self.parr = [arr for _, arr in flats]
        self.planes = (ctypes.c_void_p * n)(*[_addr(a) for a in self.parr])
        self.sts = (ctypes.c_int * n)()

    def args(self, b, stream):
        return (b.ptr, self.n, self.streams, self.n_frames, self.ins, self.lens, self.offs_pp, self.planes,
                self.sts, _stream_ptr(stream))


def jiffy_encode_batch(b: Batch, handles, planes, outs, stream=None):
    """Encodes, per stream i, the scans planes[i] (as for jiffy_encode_seq)
    into outs[i], all streams in one pass. Returns a list of (bytes, frame
    offsets) per stream."""
    c = _EncCall(handles, planes, outs)
    st = _lib().jiffy_encode_batch(*c.args(b, stream))
    if st != 0:
        raise BatchError(st, "jiffy_encode_batch", list(c.sts), required=list(c.lens))
    return c.result()


def jiffy_decode_batch(b: Batch, handles, bufs, lengths, offsets, planes_out, stream=None):
    """Decodes, per stream i, the frames of bufs[i] (lengths[i] bytes, frame
    offsets offsets[i]) into planes_out[i], all streams in one pass."""
    c = _DecCall(handles, bufs, lengths, offsets, planes_out)
    st = _lib().jiffy_decode_batch(*c.args(b, stream))
    if st != 0:
        raise BatchError(st, "jiffy_decode_batch", list(c.sts))


def jiffy_encode_batch_async(b: Batch, handles, planes, outs, stream=None):
    """Enqueues a batched encode and returns at once; jiffy_batch_wait(b)
    returns its result (as jiffy_encode_batch does)."""
    c = _EncCall(handles, planes, outs)
    st = _lib().jiffy_encode_batch_async(*c.args(b, stream))
    if st != 0:
        raise BatchError(st, "jiffy_encode_batch_async", list(c.sts))
    b.pending = ("encode", c)


def jiffy_decode_batch_async(b: Batch, handles, bufs, lengths, offsets, planes_out, stream=None):
    c = _DecCall(handles, bufs, lengths, offsets, planes_out)
    st = _lib().jiffy_decode_batch_async(*c.args(b, stream))
    if st != 0:
        raise BatchError(st, "jiffy_decode_batch_async", list(c.sts))
    b.pending = ("decode", c)


class _ArrayCall:
    """A batched call marshalled from numpy arrays of addresses (kept alive
    until it ends). Frame offsets of stream i sit in offs[starts[i]:]."""

    def __init__(self, n, keep, offs, starts, lens, sts):
        self.n, self.keep, self.offs, self.starts, self.lens, self.sts = n, keep, offs, starts, lens, sts

    def result(self):
        return self.lens, self.offs, self.starts


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def jiffy_encode_batch_async_arrays(b: Batch, streams, n_scans, plane_tables, outs, caps, stream=None):
    """jiffy_encode_batch_async with its per-stream arguments given as numpy
    arrays, for callers that issue many batches over fixed buffers (a serving
    engine): stream handle addresses (Handle.ptr), scan counts, addresses of
    plane pointer tables (each holds n_scans[i] * A device pointers,
    scan-major, kept alive by the caller), output buffer addresses and
    capacities in bytes. Nothing is checked here beyond what the C ABI checks.
    jiffy_batch_wait(b) then returns (bytes per stream, frame offsets,
    start of each stream's offsets) as numpy arrays."""
    _lib()
    streams, tables, outs, caps = _u64(streams), _u64(plane_tables), _u64(outs), _u64(caps)
    n_scans = np.ascontiguousarray(n_scans, dtype=np.uint32)
    n = len(streams)
    if not (len(n_scans) == len(tables) == len(outs) == len(caps) == n):
        raise ValueError("per-stream arrays differ in length")
    starts = np.zeros(n, dtype=np.int64)
    np.cumsum(n_scans[:-1].astype(np.int64) + 1, out=starts[1:])
    offs = np.zeros(int(n_scans.sum()) + n, dtype=np.uint64)
    offs_pp = _u64(offs.ctypes.data + 8 * starts)
    lens = np.zeros(n, dtype=np.uint64)
    sts = np.zeros(n, dtype=np.int32)
    keep = (streams, n_scans, tables, outs, caps, offs_pp)
    st = _ENC_BATCH_ADDR(b.ptr, n, streams.ctypes.data, n_scans.ctypes.data, tables.ctypes.data, outs.ctypes.data,
                         caps.ctypes.data, offs_pp.ctypes.data, lens.ctypes.data, sts.ctypes.data,
                         _stream_ptr(stream))
    if st != 0:
        raise BatchError(st, "jiffy_encode_batch_async", sts.tolist())
    b.pending = ("encode", _ArrayCall(n, keep, offs, starts, lens, sts))


def jiffy_decode_batch_async_arrays(b: Batch, streams, n_frames, ins, in_lens, offsets, offset_starts, plane_tables,
                                    stream=None):
    """jiffy_decode_batch_async with numpy arrays: stream handle addresses,
    frame counts, input buffer addresses and lengths, all streams' frame
    offsets in one uint64 array (stream i's n_frames[i] + 1 offsets start at
    offset_starts[i]) and addresses of output plane pointer tables
    (n_frames[i] * A pointers each, kept alive by the caller)."""
    _lib()
    streams, ins, in_lens, tables = _u64(streams), _u64(ins), _u64(in_lens), _u64(plane_tables)
    n_frames = np.ascontiguousarray(n_frames, dtype=np.uint32)
    offsets = _u64(offsets)
    n = len(streams)
    if not (len(n_frames) == len(ins) == len(in_lens) == len(tables) == len(offset_starts) == n):
        raise ValueError("per-stream arrays differ in length")
    starts = np.asarray(offset_starts, dtype=np.int64)
    if n and (starts.min() < 0 or (starts + n_frames.astype(np.int64) + 1).max() > len(offsets)):
        raise ValueError("frame offsets out of range")
    offs_pp = _u64(offsets.ctypes.data + 8 * starts)
    sts = np.zeros(n, dtype=np.int32)
    keep = (streams, n_frames, ins, in_lens, offsets, offs_pp, tables)
    st = _DEC_BATCH_ADDR(b.ptr, n, streams.ctypes.data, n_frames.ctypes.data, ins.ctypes.data, in_lens.ctypes.data,
                         offs_pp.ctypes.data, tables.ctypes.data, sts.ctypes.data, _stream_ptr(stream))
    if st != 0:
        raise BatchError(st, "jiffy_decode_batch_async", sts.tolist())
    b.pending = ("decode", _ArrayCall(n, keep, offsets, starts, None, sts))


def plane_table(planes):
    """A ctypes table of device pointers (for the array-marshalled calls);
    its address is ctypes.addressof(table). The caller keeps the planes and
    the table alive."""
    return (ctypes.c_void_p * len(planes))(*[p.data_ptr() for p in planes])


def jiffy_batch_wait(b: Batch):
    """Waits for the batch's enqueued call; returns the encode result (list of
    (bytes, frame offsets), or for an array-marshalled call (bytes, offsets,
    starts) as numpy arrays) or None for a decode."""
    kind, c = getattr(b, "pending", None) or (None, None)
    st = _lib().jiffy_batch_wait(b.ptr)
    b.pending = None
    if st != 0:
        sts = c.sts.tolist() if isinstance(c, _ArrayCall) else (list(c.sts) if c else [])
        req = res = None
        if kind == "encode":
            req = c.lens.tolist() if isinstance(c, _ArrayCall) else list(c.lens)
            res = c.result() if isinstance(c, _ArrayCall) else None
        raise BatchError(st, "jiffy_batch_wait", sts, required=req, result=res)
    return c.result() if kind == "encode" else None


TORCH_DTYPE = {1: torch.uint8, 2: torch.int16, 4: torch.int32}


def empty_planes(h: Handle, T: int | None = None, device=None):
    """Output planes for h: a list over attributes of (T x) H x W tensors."""
    dev = device if device is not None else torch.device("cuda", h.device)
    shape = (h.H, h.W) if T is None else (T, h.H, h.W)
    return [torch.empty(shape, dtype=TORCH_DTYPE[s], device=dev) for s, _ in h.attrs]


# ---- input standardization (Sec. III-A): Cartesian points -> range image


class Standardizer:
    """An opaque jiffy_standardizer* for one sensor."""

    def __init__(self, ptr, H, W, range_bytes, device):
        self.ptr, self.H, self.W, self.range_bytes, self.device = ptr, H, W, range_bytes, device

    def __del__(self):
        if getattr(self, "ptr", None) and _L is not None:
            _L.jiffy_standardizer_destroy(self.ptr)
            self.ptr = None


def jiffy_standardizer_create(H: int, W: int, beam_altitude, azimuth0: float = 0.0, clockwise: bool = False,
                              units_per_m: float = 1000.0, range_bytes: int = 4, min_range: int = 0,
                              max_range: int = 0xFFFFFFFF, device: int = 0) -> Standardizer:
    alt = (ctypes.c_double * H)(*[float(a) for a in beam_altitude])
    d = _SensorDesc(H, W, alt, azimuth0, 1 if clockwise else 0, units_per_m, range_bytes, min_range, max_range)
    h = ctypes.c_void_p()
    st = _lib().jiffy_standardizer_create(ctypes.byref(h), ctypes.byref(d), device)
    if st != 0:
        raise JiffyError(st, "jiffy_standardizer_create")
    return Standardizer(h.value, H, W, range_bytes, device)


def jiffy_standardizer_destroy(h: Standardizer):
    if h.ptr:
        _lib().jiffy_standardizer_destroy(h.ptr)
        h.ptr = None


def jiffy_standardize(h: Standardizer, xyz: torch.Tensor, range_out: torch.Tensor, attrs=(), stream=None):
    """xyz: n x 3 float32 CUDA tensor (metres); range_out: H x W CUDA tensor of
    range_bytes samples; attrs: (values (n float32), out (H x W), scale)
    triples. Stream-ordered, does not wait."""
    if xyz.dtype != torch.float32 or not xyz.is_cuda or not xyz.is_contiguous() or xyz.numel() % 3:
        raise ValueError("xyz: expected a contiguous CUDA float32 tensor of n x 3 coordinates")
    n = xyz.numel() // 3
    _check_plane(range_out, h.H, h.W, h.range_bytes, "range_out")
    arr = (_PointAttr * max(len(attrs), 1))()
    for i, (v, o, scale) in enumerate(attrs):
        if v.dtype != torch.float32 or not v.is_cuda or not v.is_contiguous() or v.numel() != n:
            raise ValueError("attribute %d: expected %d contiguous CUDA float32 values" % (i, n))
        _check_plane(o, h.H, h.W, o.element_size(), "attribute %d out" % i)
        arr[i] = _PointAttr(v.data_ptr(), o.data_ptr(), float(scale), o.element_size())
    st = _lib().jiffy_standardize(h.ptr, xyz.data_ptr() if n else None, n, range_out.data_ptr(), len(attrs), arr,
                                  _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_standardize")


def jiffy_standardize_seq(h: Standardizer, xyz: torch.Tensor, offsets, range_out: torch.Tensor, attrs=(),
                          stream=None):
    """Several scans in one pass: xyz holds all scans' points (N x 3 float32),
    scan t = rows offsets[t]:offsets[t+1]; range_out and each attribute out
    are T x H x W; attrs: (values (N float32), out, scale) triples."""
    T = len(offsets) - 1
    if xyz.dtype != torch.float32 or not xyz.is_cuda or not xyz.is_contiguous() or xyz.numel() % 3:
        raise ValueError("xyz: expected a contiguous CUDA float32 tensor of N x 3 coordinates")
    n = xyz.numel() // 3
    if T < 1 or offsets[0] < 0 or offsets[-1] > n:
        raise ValueError("offsets: expected T + 1 point indices within xyz")

    def check_out(t, what):
        if not t.is_cuda or not t.is_contiguous() or t.numel() != T * h.H * h.W:
            raise ValueError("%s: expected a contiguous CUDA tensor of %d x %d x %d samples" % (what, T, h.H, h.W))
    check_out(range_out, "range_out")
    if range_out.element_size() != h.range_bytes:
        raise ValueError("range_out: expected %d-byte samples" % h.range_bytes)
    arr = (_PointAttr * max(len(attrs), 1))()
    for i, (v, o, scale) in enumerate(attrs):
        if v.dtype != torch.float32 or not v.is_cuda or not v.is_contiguous() or v.numel() != n:
            raise ValueError("attribute %d: expected %d contiguous CUDA float32 values" % (i, n))
        check_out(o, "attribute %d out" % i)
        arr[i] = _PointAttr(v.data_ptr(), o.data_ptr(), float(scale), o.element_size())
    offs = (ctypes.c_uint64 * (T + 1))(*[int(x) for x in offsets])
    st = _lib().jiffy_standardize_seq(h.ptr, T, xyz.data_ptr() if n else None, offs, range_out.data_ptr(),
                                      len(attrs), arr, _stream_ptr(stream))
    if st != 0:
        raise JiffyError(st, "jiffy_standardize_seq")
