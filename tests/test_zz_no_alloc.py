"""The allocation-free decode entry point (jiffy_decode_frame_noalloc).

It serves callers that may not allocate device memory while they run (fixed
footprint real-time stacks, hosts whose allocator owns the device memory).
This file checks, through the C ABI, that it decodes exactly what the regular
handle-based jiffy_decode decodes, frame after frame (an I frame, then P
frames that need the previous frame's planes), including two calls in a row on
the shared scratch array. Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2209_08196_gb300 import build as jbuild  # noqa: E402
from paper_2209_08196_gb300 import jiffy as J  # noqa: E402

jbuild.build()

SIGNED = {1: np.uint8, 2: np.int16, 4: np.int32}


def _scans(H, W, attrs, T, seed):
    rng = np.random.default_rng(seed)
    base = []
    for s, _ in attrs:
        v = rng.integers(1, 1 << (8 * s), size=(H, W), dtype=np.uint64)
        v[rng.random((H, W)) < 0.2] = 0
        base.append(v)
    scans = []
    for t in range(T):
        planes = []
        for (s, _), b in zip(attrs, base):
            x = np.clip(b.astype(np.int64) + rng.integers(-1, 2, size=b.shape) * (t % 2), 0, (1 << (8 * s)) - 1)
            x[rng.random(x.shape) < 0.01] = 0
            planes.append(torch.from_numpy(x.astype(SIGNED[s])).cuda())
        scans.append(planes)
    return scans


def _encode_frames(H, W, attrs, scans):
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs)
    frames = []
    for planes in scans:
        out = torch.empty(J.jiffy_max_encoded_size(H, W, attrs, 1), dtype=torch.uint8, device="cuda")
        n = J.jiffy_encode(enc, planes, out)
        frames.append((out, n))
    return frames


def test_noalloc_decode_matches_handle_decode():
    H, W, attrs = 16, 1024, [(4, 10), (2, 1), (1, 1)]
    scans = _scans(H, W, attrs, 4, seed=5)
    frames = _encode_frames(H, W, attrs, scans)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs)
    prev = None
    saw_p = False
    for t, (buf, n) in enumerate(frames):
        want = J.empty_planes(dec)
        J.jiffy_decode(dec, buf, n, want)
        got = J.empty_planes(dec)
        J.jiffy_decode_frame_noalloc(buf, n, H, W, attrs, t, prev, got)
        for a in range(len(attrs)):
            assert torch.equal(got[a], want[a]), "scan %d attribute %d" % (t, a)
        # a second call in a row on the same frame: the shared scratch keeps
        # the previous call's contents and must not change the result
        again = J.empty_planes(dec)
        J.jiffy_decode_frame_noalloc(buf, n, H, W, attrs, t, prev, again)
        for a in range(len(attrs)):
            assert torch.equal(again[a], want[a]), "repeat, scan %d attribute %d" % (t, a)
        mode_bytes = buf[16 + 8 * len(attrs) if t == 0 else 0:][8:8 + 12 * len(attrs)].cpu().numpy()[::12]
        saw_p |= bool((mode_bytes == 1).any())
        prev = got
    assert saw_p, "the sequence should contain P frames"


def test_noalloc_rejects_out_of_limit_sizes_and_missing_previous_planes():
    H, W, attrs = 8, 256, [(4, 1)]
    scans = _scans(H, W, attrs, 2, seed=6)
    scans[1] = [p.clone() for p in scans[0]]  # identical scan: P is chosen
    frames = _encode_frames(H, W, attrs, scans)
    out = [torch.empty((H, W), dtype=torch.int32, device="cuda")]
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_decode_frame_noalloc(frames[1][0], frames[1][1], H, W, attrs, 1, None, out)
    assert ei.value.status == 4  # JIFFY_ERR_STATE: a P frame needs the previous planes
    big = [(1, 1)] * 17  # more attributes than the scratch array holds
    outs = [torch.empty((1, 8), dtype=torch.uint8, device="cuda") for _ in big]
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_decode_frame_noalloc(frames[0][0], frames[0][1], 1, 8, big, 0, None, outs)
    assert ei.value.status == 1  # JIFFY_ERR_INVALID_ARG
