"""GPU: the enqueue-only sequence calls (jiffy_encode_seq_async /
jiffy_decode_seq_async / jiffy_stream_wait). An encode and the decode of its
stream run back to back on one CUDA stream with the frame offsets handed over
in device memory; the bytes and planes must be the oracle's, P frames must
chain across calls, and errors found on the device (offsets that leave the
buffer, a too small output) come back from jiffy_stream_wait without a
fault, after which a reset stream codes correctly again."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2209_08196_gb300 import build as jbuild  # noqa: E402
from paper_2209_08196_gb300 import jiffy as J  # noqa: E402
from paper_2209_08196_gb300 import synth  # noqa: E402
from tests.gpu_util import to_dev, to_np  # noqa: E402

jbuild.build()


def workload(n_scans, H=32, W=1024, seed=3):
    cfg = synth.config_multi_attr(n_scans=n_scans, H=H, W=W, seed=seed)
    return cfg, synth.attr_descs(cfg), synth.ScanSequence(cfg).scans()


def stacked(scans, attrs):
    return [torch.stack([to_dev(s[a]) for s in scans]) for a in range(len(attrs))]


def test_async_round_trip_matches_oracle_over_steps():
    cfg, attrs, scans = workload(6)
    H, W, T = cfg.H, cfg.W, len(scans)
    want, _, _ = oracle.encode_sequence(H, W, attrs, scans)
    want_planes, _ = oracle.decode_sequence(H, W, attrs, want, T)
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs)
    planes = stacked(scans, attrs)
    out = torch.zeros(J.jiffy_max_encoded_size(H, W, attrs, T), dtype=torch.uint8, device="cuda")
    d_offs = torch.zeros(T + 1, dtype=torch.int64, device="cuda")
    outs = J.empty_planes(dec, T)
    for _ in range(3):  # several steps in flight before the first wait
        J.jiffy_stream_reset(enc)
        J.jiffy_stream_reset(dec)
        J.jiffy_encode_seq_async(enc, planes, out, d_offs)
        J.jiffy_decode_seq_async(dec, out, d_offs, outs)
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    offs = [int(x) for x in d_offs.cpu()]
    assert out[:offs[-1]].cpu().numpy().tobytes() == want
    for t in range(T):
        for a, (s, _) in enumerate(attrs):
            assert np.array_equal(to_np(outs[a][t], s), want_planes[t][a]), (t, a)


def test_timed_async_calls_replay_graphs_with_their_own_timing_events():
    # kernel timing on: every enqueue-only call records its kernel times with
    # the next event set of a ring of 16, while the call's launch sequence is
    # replayed from one captured graph whose timing nodes are pointed at that
    # set; 20 steps in flight go round the ring, and the bytes, planes and
    # kernel times stay right
    cfg, attrs, scans = workload(4, seed=12)
    H, W, T = cfg.H, cfg.W, len(scans)
    want, _, _ = oracle.encode_sequence(H, W, attrs, scans)
    want_planes, _ = oracle.decode_sequence(H, W, attrs, want, T)
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs)
    J.jiffy_stream_set_profiling(enc, True)
    J.jiffy_stream_set_profiling(dec, True)
    planes = stacked(scans, attrs)
    out = torch.zeros(J.jiffy_max_encoded_size(H, W, attrs, T), dtype=torch.uint8, device="cuda")
    d_offs = torch.zeros(T + 1, dtype=torch.int64, device="cuda")
    outs = J.empty_planes(dec, T)
    for _ in range(20):
        J.jiffy_stream_reset(enc)
        J.jiffy_stream_reset(dec)
        J.jiffy_encode_seq_async(enc, planes, out, d_offs)
        J.jiffy_decode_seq_async(dec, out, d_offs, outs)
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    te, td = J.jiffy_stream_kernel_times(enc), J.jiffy_stream_kernel_times(dec)
    assert len(te) == 3 and all(t > 0 for t in te) and len(td) == 1 and td[0] > 0
    offs = [int(x) for x in d_offs.cpu()]
    assert out[:offs[-1]].cpu().numpy().tobytes() == want
    for t in range(T):
        for a, (s, _) in enumerate(attrs):
            assert np.array_equal(to_np(outs[a][t], s), want_planes[t][a]), (t, a)


def test_async_calls_chain_p_frames_across_calls():
    # two calls of 3 scans each, no reset between them: the second call's
    # first frame predicts from the first call's last scan (Sec. III-D)
    cfg, attrs, scans = workload(6, seed=8)
    H, W = cfg.H, cfg.W
    want, lens, _ = oracle.encode_sequence(H, W, attrs, scans, force_mode=1)
    want_planes, _ = oracle.decode_sequence(H, W, attrs, want, 6)
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, force_mode=1)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, force_mode=1)
    got = b""
    for t0, part in ((0, scans[:3]), (3, scans[3:])):
        out = torch.zeros(J.jiffy_max_encoded_size(H, W, attrs, 3), dtype=torch.uint8, device="cuda")
        d_offs = torch.zeros(4, dtype=torch.int64, device="cuda")
        outs = J.empty_planes(dec, 3)
        J.jiffy_encode_seq_async(enc, stacked(part, attrs), out, d_offs)
        J.jiffy_decode_seq_async(dec, out, d_offs, outs)
        J.jiffy_stream_wait(enc)
        J.jiffy_stream_wait(dec)
        n = int(d_offs[-1])
        got += out[:n].cpu().numpy().tobytes()
        for t in range(3):
            for a, (s, _) in enumerate(attrs):
                assert np.array_equal(to_np(outs[a][t], s), want_planes[t0 + t][a]), (t0 + t, a)
    assert got == want


@pytest.mark.parametrize("case", ["beyond", "misaligned", "overlap"])
def test_async_decode_rejects_bad_device_offsets(case):
    cfg, attrs, scans = workload(2, seed=9)
    H, W = cfg.H, cfg.W
    # frame offsets from the oracle's per-frame lengths (the first frame's
    # length includes the stream header)
    buf, lens, _ = oracle.encode_sequence(H, W, attrs, scans)
    offs = [16 + 8 * len(attrs)]
    for k, n in enumerate(lens):
        offs.append((offs[-1] if k else 0) + n)
    assert offs[-1] == len(buf)
    bad = list(offs)
    if case == "beyond":
        bad[2] = len(buf) + 4096
    elif case == "misaligned":
        bad[1] += 2
    else:
        bad[1] = bad[0]  # a frame shorter than its header
    src = torch.from_numpy(np.frombuffer(buf, dtype=np.uint8).copy()).cuda()
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs)
    outs = J.empty_planes(dec, 2)
    J.jiffy_decode_seq_async(dec, src, torch.tensor(bad, dtype=torch.int64, device="cuda"), outs)
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_stream_wait(dec)
    assert ei.value.name == "JIFFY_ERR_CORRUPT"
    # a reset stream decodes the good offsets
    J.jiffy_stream_reset(dec)
    J.jiffy_decode_seq_async(dec, src, torch.tensor(offs, dtype=torch.int64, device="cuda"), outs)
    J.jiffy_stream_wait(dec)
    want, _ = oracle.decode_sequence(H, W, attrs, buf, 2)
    for t in range(2):
        for a, (s, _) in enumerate(attrs):
            assert np.array_equal(to_np(outs[a][t], s), want[t][a])


def test_async_encode_capacity_error_is_reported_by_wait():
    cfg, attrs, scans = workload(2, seed=10)
    H, W = cfg.H, cfg.W
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs)
    small = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    d_offs = torch.zeros(3, dtype=torch.int64, device="cuda")
    J.jiffy_encode_seq_async(enc, stacked(scans, attrs), small, d_offs)
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_stream_wait(enc)
    assert ei.value.name == "JIFFY_ERR_CAPACITY"
    J.jiffy_stream_reset(enc)
    out = torch.zeros(J.jiffy_max_encoded_size(H, W, attrs, 2), dtype=torch.uint8, device="cuda")
    J.jiffy_encode_seq_async(enc, stacked(scans, attrs), out, d_offs)
    J.jiffy_stream_wait(enc)
    want, _, _ = oracle.encode_sequence(H, W, attrs, scans)
    assert out[:int(d_offs[-1])].cpu().numpy().tobytes() == want
