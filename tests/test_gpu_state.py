"""GPU: checkpoint / resume (jiffy_stream_save_state / jiffy_stream_load_state).
A stream saved after some frames and restored into a new handle continues the
saved stream: the encoder's next frames, P frames included, are the bytes the
oracle writes for the uninterrupted sequence, and a restored decoder (or a
decoder restored from an encoder's state) decodes the rest of it. Saved states
of another configuration, damaged ones and states of streams with calls in
flight are refused without touching the stream."""
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


def workload(n_scans, seed):
    cfg = synth.config_multi_attr(n_scans=n_scans, H=16, W=512, seed=seed)
    return cfg, synth.attr_descs(cfg), synth.ScanSequence(cfg).scans()


def dev_scans(scans):
    return [[to_dev(p) for p in s] for s in scans]


def encode(h, scans, H, W, attrs):
    out = torch.zeros(J.jiffy_max_encoded_size(H, W, attrs, len(scans)), dtype=torch.uint8, device="cuda")
    n, offs = J.jiffy_encode_seq(h, dev_scans(scans), out)
    return out[:n].cpu().numpy().tobytes(), offs


@pytest.mark.parametrize("force", [1, -1])
def test_encoder_resumes_from_a_saved_state(force):
    cfg, attrs, scans = workload(6, seed=31)
    H, W = cfg.H, cfg.W
    want, _, modes = oracle.encode_sequence(H, W, attrs, scans, force_mode=force)
    a = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, force_mode=force)
    part1, _ = encode(a, scans[:3], H, W, attrs)
    state = J.jiffy_stream_save_state(a)
    assert len(state) == 28 + 8 * len(attrs) + sum(H * W * s for s, _ in attrs)
    b = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, force_mode=force)
    J.jiffy_stream_load_state(b, state)
    assert J.jiffy_stream_frame_index(b) == 3
    part2, _ = encode(b, scans[3:], H, W, attrs)
    assert part1 + part2 == want
    if force == 1:
        assert all(m == 1 for mm in modes[3:] for m in mm)  # the resumed frames predict from the saved scan


def test_decoder_resumes_from_a_decoder_or_an_encoder_state():
    cfg, attrs, scans = workload(6, seed=32)
    H, W = cfg.H, cfg.W
    buf, lens, _ = oracle.encode_sequence(H, W, attrs, scans, force_mode=1)
    want, _ = oracle.decode_sequence(H, W, attrs, buf, 6)
    head = 16 + 8 * len(attrs)
    offs = [head]
    for k, n in enumerate(lens):
        offs.append((offs[-1] if k else 0) + n)
    dev_buf = torch.from_numpy(np.frombuffer(buf, dtype=np.uint8).copy()).cuda()
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, force_mode=1)
    outs = J.empty_planes(dec, 3)
    J.jiffy_decode_seq(dec, dev_buf, offs[3], offs[:4], outs)
    saved_dec = J.jiffy_stream_save_state(dec)
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, force_mode=1)
    J.jiffy_encode_seq(enc, dev_scans(scans[:3]),
                       torch.zeros(J.jiffy_max_encoded_size(H, W, attrs, 3), dtype=torch.uint8, device="cuda"))
    saved_enc = J.jiffy_stream_save_state(enc)
    rest = dev_buf[offs[3]:].clone()
    rest_offs = [o - offs[3] for o in offs[3:]]
    for state in (saved_dec, saved_enc):
        d2 = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, force_mode=1)
        J.jiffy_stream_load_state(d2, state)
        outs2 = J.empty_planes(d2, 3)
        J.jiffy_decode_seq(d2, rest, rest_offs[-1], rest_offs, outs2)
        for t in range(3):
            for k, (s, _) in enumerate(attrs):
                assert np.array_equal(to_np(outs2[k][t], s), want[3 + t][k]), (t, k)


def test_state_errors_leave_the_stream_untouched():
    cfg, attrs, scans = workload(2, seed=33)
    H, W = cfg.H, cfg.W
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs)
    encode(enc, scans[:1], H, W, attrs)
    state = J.jiffy_stream_save_state(enc)
    other = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W * 2, attrs)
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_stream_load_state(other, state)
    assert ei.value.name == "JIFFY_ERR_INVALID_ARG"
    fresh = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs)
    for bad in (b"XXXX" + state[4:], state[:-4], state + b"\0\0\0\0", b""):
        with pytest.raises(J.JiffyError) as ei:
            J.jiffy_stream_load_state(fresh, bad)
        assert ei.value.name == "JIFFY_ERR_CORRUPT"
    assert J.jiffy_stream_frame_index(fresh) == 0
    # enqueue-only calls in flight: save and load wait for jiffy_stream_wait
    planes = [torch.stack([to_dev(s[a]) for s in scans]) for a in range(len(attrs))]
    out = torch.zeros(J.jiffy_max_encoded_size(H, W, attrs, 2), dtype=torch.uint8, device="cuda")
    d_offs = torch.zeros(3, dtype=torch.int64, device="cuda")
    J.jiffy_encode_seq_async(fresh, planes, out, d_offs)
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_stream_save_state(fresh)
    assert ei.value.name == "JIFFY_ERR_STATE"
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_stream_load_state(fresh, state)
    assert ei.value.name == "JIFFY_ERR_STATE"
    J.jiffy_stream_wait(fresh)
    assert J.jiffy_stream_frame_index(fresh) == 2
    J.jiffy_stream_load_state(fresh, state)
    assert J.jiffy_stream_frame_index(fresh) == 1
