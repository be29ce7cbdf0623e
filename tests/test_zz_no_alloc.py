"""The allocation-free decode entry point (jiffy_decode_frame_noalloc).

It serves callers that may not allocate device memory while they run (fixed
footprint real-time stacks, hosts whose allocator owns the device memory).
This file checks, through the C ABI, that it decodes exactly what the oracle
decodes, frame after frame (an I frame, then P frames that need the previous
frame's planes), including two calls in a row on the shared scratch array, a
stream with stage switches (the ablated codecs) past its first frame, and a
decode in place over the previous planes. Kept in a file of its own that
pytest collects last.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2209_08196_gb300 import build as jbuild  # noqa: E402
from paper_2209_08196_gb300 import jiffy as J  # noqa: E402

jbuild.build()

NP = {1: np.uint8, 2: np.uint16, 4: np.uint32}
SIGNED = {1: np.uint8, 2: np.int16, 4: np.int32}
TDT = {1: torch.uint8, 2: torch.int16, 4: torch.int32}


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
            planes.append(x.astype(NP[s]))
        scans.append(planes)
    return scans


def _oracle_frames(H, W, attrs, scans, force_mode=-1, stages=0):
    """The oracle's stream as (device bytes, length, scan index) per frame and
    its decoded planes."""
    buf, lens, modes = oracle.encode_sequence(H, W, attrs, scans, force_mode=force_mode, stages=stages)
    planes, _ = oracle.decode_sequence(H, W, attrs, buf, len(scans), stages=stages)
    frames, at = [], 0
    for t, n in enumerate(lens):
        dev = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
        dev[:n] = torch.from_numpy(np.frombuffer(buf[at:at + n], dtype=np.uint8).copy())
        frames.append((dev, n))
        at += n
    return frames, planes, modes


def _out(H, W, attrs):
    return [torch.empty((H, W), dtype=TDT[s], device="cuda") for s, _ in attrs]


def _np(t, s):
    return t.cpu().numpy().view(NP[s])


def test_noalloc_decode_matches_oracle_frame_after_frame():
    H, W, attrs = 16, 1024, [(4, 10), (2, 1), (1, 1)]
    scans = _scans(H, W, attrs, 4, seed=5)
    frames, want, modes = _oracle_frames(H, W, attrs, scans)
    assert any(m == 1 for mm in modes for m in mm), "the sequence should contain P frames"
    prev = None
    for t, (buf, n) in enumerate(frames):
        got = _out(H, W, attrs)
        J.jiffy_decode_frame_noalloc(buf, n, H, W, attrs, t, prev, got)
        for a, (s, _) in enumerate(attrs):
            assert np.array_equal(_np(got[a], s), want[t][a]), "scan %d attribute %d" % (t, a)
        # a second call in a row on the same frame: the shared scratch keeps
        # the previous call's contents and must not change the result
        again = _out(H, W, attrs)
        J.jiffy_decode_frame_noalloc(buf, n, H, W, attrs, t, prev, again)
        for a, (s, _) in enumerate(attrs):
            assert np.array_equal(_np(again[a], s), want[t][a]), "repeat, scan %d attribute %d" % (t, a)
        prev = got


@pytest.mark.parametrize("stages", [1, 2, 4, 6, 7])
def test_noalloc_decodes_ablated_streams_past_their_first_frame(stages):
    # stage switches (Sec. IV-H ablations) live in the stream header only;
    # frames after the first decode with the switches the caller passes
    H, W, attrs = 8, 300, [(2, 1), (4, 10)]
    scans = _scans(H, W, attrs, 3, seed=20 + stages)
    frames, want, modes = _oracle_frames(H, W, attrs, scans, force_mode=1, stages=stages)
    prev = None
    for t, (buf, n) in enumerate(frames):
        got = _out(H, W, attrs)
        J.jiffy_decode_frame_noalloc(buf, n, H, W, attrs, t, prev, got, stages=stages)
        for a, (s, _) in enumerate(attrs):
            assert np.array_equal(_np(got[a], s), want[t][a]), "scan %d attribute %d" % (t, a)
        prev = got
    # the first frame's header carries the switches: others are CORRUPT
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_decode_frame_noalloc(frames[0][0], frames[0][1], H, W, attrs, 0, None, _out(H, W, attrs), stages=0)
    assert ei.value.name == "JIFFY_ERR_CORRUPT"


def test_noalloc_decodes_in_place_over_the_previous_planes():
    H, W, attrs = 16, 512, [(4, 10), (2, 1)]
    scans = _scans(H, W, attrs, 3, seed=31)
    frames, want, modes = _oracle_frames(H, W, attrs, scans, force_mode=1)
    planes = _out(H, W, attrs)
    J.jiffy_decode_frame_noalloc(frames[0][0], frames[0][1], H, W, attrs, 0, None, planes)
    for t in (1, 2):  # P frames decoded over the previous frame's planes
        J.jiffy_decode_frame_noalloc(frames[t][0], frames[t][1], H, W, attrs, t, planes, planes)
        for a, (s, _) in enumerate(attrs):
            assert np.array_equal(_np(planes[a], s), want[t][a]), "scan %d attribute %d" % (t, a)


def test_noalloc_rejects_out_of_limit_sizes_and_missing_previous_planes():
    H, W, attrs = 8, 256, [(4, 1)]
    scans = _scans(H, W, attrs, 2, seed=6)
    scans[1] = [p.copy() for p in scans[0]]  # identical scan: P is chosen
    frames, _, modes = _oracle_frames(H, W, attrs, scans)
    assert modes[1][0] == 1
    out = _out(H, W, attrs)
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_decode_frame_noalloc(frames[1][0], frames[1][1], H, W, attrs, 1, None, out)
    assert ei.value.status == 4  # JIFFY_ERR_STATE: a P frame needs the previous planes
    big = [(1, 1)] * 17  # more attributes than the scratch array holds
    outs = [torch.empty((1, 8), dtype=torch.uint8, device="cuda") for _ in big]
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_decode_frame_noalloc(frames[0][0], frames[0][1], 1, 8, big, 0, None, outs)
    assert ei.value.status == 1  # JIFFY_ERR_INVALID_ARG
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_decode_frame_noalloc(frames[0][0], frames[0][1], H, W, attrs, 0, None, out, stages=8)
    assert ei.value.status == 1  # unknown stage switch
