"""GPU parity: the CUDA library (through the C ABI) against the oracle.

Integer codec, so the bar is exact: identical bytes from the encoder,
identical planes from the decoder. Sizes span several rows, blocks of 128
and ragged tails; the edge cases are the degenerate scans the method has
(all zero, all maximal, one row, one column, widths off the 32-bit grid,
large precisions, static scenes that select P)."""
import numpy as np
import pytest

import oracle
from tests import golden_io

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2209_08196_gb300 import build as jbuild  # noqa: E402
from paper_2209_08196_gb300 import jiffy as J  # noqa: E402
from paper_2209_08196_gb300 import synth  # noqa: E402
from tests.gpu_util import TORCH_DT, GpuCodec  # noqa: E402

jbuild.build()
DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def rand_scan(rng, H, W, s, zero_frac, hi=None):
    hi = hi or (1 << (8 * s))
    v = rng.integers(1, hi, size=(H, W), dtype=np.uint64)
    v[rng.random((H, W)) < zero_frac] = 0
    return v.astype(DT[s])


def drift(rng, base, s, amount, zero_frac=0.05):
    x = base.astype(np.int64) + rng.integers(-amount, amount + 1, size=base.shape)
    x = np.clip(x, 0, (1 << (8 * s)) - 1).astype(DT[s])
    x[rng.random(x.shape) < zero_frac] = 0
    return x


def check_stream(H, W, attrs, scans, test_lines=4, force_mode=-1, seq=False, stages=0):
    """Encodes scans with oracle and GPU, compares bytes frame by frame and
    the decoded planes; seq=True uses the one-pass sequence entry points."""
    ref = oracle.Codec(H, W, attrs, test_lines, force_mode, stages)
    refd = oracle.Codec(H, W, attrs, test_lines, force_mode, stages)
    gpu = GpuCodec(H, W, attrs, test_lines, force_mode, stages)
    ref_frames = [ref.encode(s) for s in scans]
    if seq:
        buf, offs = gpu.encode_seq(scans)
        gpu_frames = [buf[(0 if t == 0 else offs[t]):offs[t + 1]] for t in range(len(scans))]
        assert buf == b"".join(ref_frames)
        dec = gpu.decode_seq(buf, offs)
    else:
        gpu_frames = [gpu.encode(s) for s in scans]
        dec = [gpu.decode(f) for f in gpu_frames]
    for t, (g, r) in enumerate(zip(gpu_frames, ref_frames)):
        assert g == r, "frame %d differs (gpu %d bytes, oracle %d bytes)" % (t, len(g), len(r))
    for t, f in enumerate(ref_frames):
        want, _ = refd.decode(f)
        for a in range(len(attrs)):
            assert np.array_equal(dec[t][a], want[a]), "decoded frame %d attr %d differs" % (t, a)
    return ref_frames


@pytest.mark.parametrize("name", golden_io.names())
def test_golden_streams_on_gpu(name):
    H, W, attrs, frames = golden_io.load(name)
    opt = golden_io.options(name)
    gpu = GpuCodec(H, W, attrs, 4, opt["force_mode"], opt["stages"])
    for f in frames:
        b = gpu.encode(f["in"])
        assert b == f["bytes"], (b.hex(" "), f["bytes"].hex(" "))
        out = gpu.decode(b)
        for o, w in zip(out, f["out"]):
            assert np.array_equal(o, w)


@pytest.mark.parametrize("seed", range(8))
def test_random_sequences_match_oracle(seed):
    rng = np.random.default_rng(1000 + seed)
    H = int(rng.choice([1, 2, 3, 7, 16, 33]))
    W = int(rng.choice([1, 5, 31, 32, 33, 100, 128, 129, 257, 1000, 2048]))
    A = int(rng.integers(1, 4))
    attrs = [(int(rng.choice([1, 2, 4])), int(rng.choice([1, 1, 3, 10, 255, 4096]))) for _ in range(A)]
    force = int(rng.choice([-1, -1, -1, 0, 1]))
    base = [rand_scan(rng, H, W, s, float(rng.choice([0.0, 0.1, 0.5, 0.95]))) for s, _ in attrs]
    scans = []
    for t in range(5):
        scans.append([drift(rng, b, s, int(rng.choice([0, 1, 3, 1000])), 0.05) for b, (s, _) in zip(base, attrs)])
    check_stream(H, W, attrs, scans, force_mode=force, seq=bool(seed % 2))


def test_static_scene_selects_p_and_matches():
    rng = np.random.default_rng(7)
    H, W = 16, 1024
    attrs = [(4, 10), (2, 1), (1, 1)]
    base = [rand_scan(rng, H, W, s, 0.2) for s, _ in attrs]
    scans = [[drift(rng, b, s, 1 if t % 2 else 0, 0.01) for b, (s, _) in zip(base, attrs)] for t in range(6)]
    ref = oracle.Codec(H, W, attrs)
    modes = [ref.encode(s, return_modes=True)[1] for s in scans]
    assert any(m == 1 for mm in modes for m in mm)  # P is exercised
    check_stream(H, W, attrs, scans)
    check_stream(H, W, attrs, scans, seq=True)


@pytest.mark.parametrize("case", ["zeros", "max", "one_row", "one_col", "big_precision", "tiny_w"])
def test_degenerate_scans(case):
    rng = np.random.default_rng(11)
    if case == "zeros":
        H, W, attrs = 4, 300, [(4, 1), (1, 7)]
        scans = [[np.zeros((H, W), DT[s]) for s, _ in attrs] for _ in range(3)]
    elif case == "max":
        H, W, attrs = 3, 200, [(4, 1), (2, 3), (1, 1)]
        scans = [[np.full((H, W), (1 << (8 * s)) - 1, DT[s]) for s, _ in attrs] for _ in range(3)]
        scans[1][0][1, 5] = 0
    elif case == "one_row":
        H, W, attrs = 1, 4096, [(4, 10)]
        scans = [[rand_scan(rng, H, W, 4, 0.3, 10**6)] for _ in range(3)]
    elif case == "one_col":
        H, W, attrs = 64, 1, [(2, 1)]
        scans = [[rand_scan(rng, H, W, 2, 0.3)] for _ in range(3)]
    elif case == "big_precision":
        H, W, attrs = 5, 100, [(4, 0x80000000), (4, 0xC0000001), (4, 3000000000), (4, 65537)]
        scans = [[rand_scan(rng, H, W, 4, 0.2) for _ in attrs] for _ in range(3)]
    else:
        H, W, attrs = 9, 3, [(1, 2), (4, 5)]
        scans = [[rand_scan(rng, H, W, s, 0.4) for s, _ in attrs] for _ in range(4)]
    check_stream(H, W, attrs, scans)
    check_stream(H, W, attrs, scans, seq=True)


@pytest.mark.parametrize("shape", ["max_w", "max_h"])
def test_maximum_shapes(shape):
    # the largest row (W = 16384: 128 blocks per row, one warp per CTA) and the
    # most rows (H = 4096) the library accepts, both modes, several attributes
    rng = np.random.default_rng(21)
    H, W = (2, 16384) if shape == "max_w" else (4096, 40)
    attrs = [(4, 10), (2, 1), (1, 3)]
    base = [rand_scan(rng, H, W, s, 0.1) for s, _ in attrs]
    scans = [[drift(rng, b, s, t, 0.05) for b, (s, _) in zip(base, attrs)] for t in range(3)]
    check_stream(H, W, attrs, scans, seq=True)
    check_stream(H, W, attrs, scans, force_mode=1)


def test_test_lines_option():
    rng = np.random.default_rng(12)
    H, W, attrs = 40, 512, [(4, 10)]
    base = rand_scan(rng, H, W, 4, 0.2, 10**6)
    scans = [[drift(rng, base, 4, 2 * t, 0.02)] for t in range(4)]
    for L in (1, 4, 7, 40, 64):
        check_stream(H, W, attrs, scans, test_lines=L, seq=True)


def test_synthetic_small_range_full_size():
    cfg = synth.config_small_range()  # 16 scans of 64 x 1024, range, 10 mm
    scans = synth.ScanSequence(cfg).scans()
    check_stream(cfg.H, cfg.W, synth.attr_descs(cfg), scans, seq=True)


@pytest.mark.parametrize("maker", [synth.config_multi_attr, synth.config_low_coherence])
def test_synthetic_multi_attr_and_low_coherence(maker):
    cfg = maker(n_scans=3)
    scans = synth.ScanSequence(cfg).scans()
    check_stream(cfg.H, cfg.W, synth.attr_descs(cfg), scans, seq=True)


@pytest.mark.parametrize("lines", ["H", "10H"])
def test_brute_force_choice_over_every_row(lines):
    # test_lines >= H: every scanline is a test row, the brute-force I/P choice
    cfg = synth.config_multi_attr(n_scans=3)
    scans = synth.ScanSequence(cfg).scans()
    L = cfg.H if lines == "H" else 10 * cfg.H
    check_stream(cfg.H, cfg.W, synth.attr_descs(cfg), scans, test_lines=L, seq=True)


def test_sequence_equals_single_calls_and_state_carries_across_calls():
    rng = np.random.default_rng(13)
    H, W, attrs = 8, 700, [(4, 10), (2, 1)]
    base = [rand_scan(rng, H, W, s, 0.1) for s, _ in attrs]
    scans = [[drift(rng, b, s, t % 3, 0.02) for b, (s, _) in zip(base, attrs)] for t in range(7)]
    one = GpuCodec(H, W, attrs)
    singles = [one.encode(s) for s in scans]
    many = GpuCodec(H, W, attrs)
    b1, o1 = many.encode_seq(scans[:3])
    b2, o2 = many.encode_seq(scans[3:])
    assert b1 + b2 == b"".join(singles)
    dec = GpuCodec(H, W, attrs)
    out1 = dec.decode_seq(b1, o1)
    out2 = dec.decode_seq(b2, o2)
    refd = oracle.Codec(H, W, attrs)
    for t, f in enumerate(singles):
        want, _ = refd.decode(f)
        got = (out1 + out2)[t]
        for a in range(len(attrs)):
            assert np.array_equal(got[a], want[a])


def test_capacity_error_reports_size_and_keeps_state():
    rng = np.random.default_rng(14)
    H, W, attrs = 4, 256, [(4, 1)]
    s0, s1 = [rand_scan(rng, H, W, 4, 0.1)], [rand_scan(rng, H, W, 4, 0.1)]
    a, b = GpuCodec(H, W, attrs), GpuCodec(H, W, attrs)
    a.encode(s0)
    b.encode(s0)
    small = torch.zeros(64, dtype=torch.uint8, device="cuda")
    from tests.gpu_util import to_dev
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_encode(a.enc, [to_dev(s1[0])], small)
    assert ei.value.status == 2
    want = b.encode(s1)
    assert ei.value.required == len(want)
    assert a.encode(s1) == want


def test_corrupt_streams_are_rejected_without_faults():
    rng = np.random.default_rng(15)
    H, W, attrs = 6, 500, [(4, 10), (1, 1)]
    scans = [[rand_scan(rng, H, W, s, 0.2) for s, _ in attrs] for _ in range(2)]
    good = GpuCodec(H, W, attrs).encode(scans[0])
    A = len(attrs)
    fh = 16 + 8 * A             # frame header follows the stream header
    sec = fh + 8 + 12 * A       # first section (row table)
    cases = []
    b = bytearray(good); b[0] ^= 1; cases.append(bytes(b))                # magic
    b = bytearray(good); b[fh + 4] ^= 1; cases.append(bytes(b))           # scan index
    b = bytearray(good); b[fh + 8] = 2; cases.append(bytes(b))            # mode
    b = bytearray(good); b[fh + 12] ^= 4; cases.append(bytes(b))          # section bytes
    b = bytearray(good); b[sec] ^= 8; cases.append(bytes(b))              # row end
    b = bytearray(good); b[sec + 8 * H] = 0xFF; cases.append(bytes(b))    # class word: invalid class
    b = bytearray(good); b[16 + 4] ^= 1; cases.append(bytes(b))           # precision differs
    for bad in cases:
        g = GpuCodec(H, W, attrs)
        with pytest.raises(J.JiffyError) as ei:
            g.decode(bad)
        assert ei.value.status == 3
        with pytest.raises(oracle.OracleError):
            oracle.Codec(H, W, attrs).decode(bad)
    # truncated: the frame length no longer matches
    with pytest.raises(J.JiffyError):
        GpuCodec(H, W, attrs).decode(good[:-4])
    # the decoder still works after errors
    g = GpuCodec(H, W, attrs)
    out = g.decode(good)
    want, _ = oracle.Codec(H, W, attrs).decode(good)
    for o, w in zip(out, want):
        assert np.array_equal(o, w)


def test_full_size_multi_attribute_sequence_sampled_against_oracle():
    """The benchmark's launch configuration: 100 scans of 128 x 2048 with five
    attributes in one encode pass and one decode pass. Every frame must round
    trip exactly (q * P); sampled frames are re-coded by the oracle from
    their predecessor and must match byte for byte (except the scan index)."""
    cfg = synth.config_multi_attr()
    seq = synth.ScanSequence(cfg, device="cuda")
    attrs = synth.attr_descs(cfg)
    T, H, W = cfg.n_scans, cfg.H, cfg.W
    planes = [[None] * len(attrs) for _ in range(T)]
    for t in range(T):
        planes[t] = seq.scan(t, as_numpy=False)
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs)
    cap = J.jiffy_max_encoded_size(H, W, attrs, T)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    n, offs = J.jiffy_encode_seq(enc, planes, out)
    outs = J.empty_planes(dec, T)
    J.jiffy_decode_seq(dec, out, n, offs, outs)
    for a, (s, P) in enumerate(attrs):
        mask = (1 << (8 * s)) - 1
        v = torch.stack([planes[t][a] for t in range(T)]).to(torch.int64) & mask
        q = torch.clamp((v + P // 2) // P, max=mask // P)
        assert torch.equal((outs[a].to(torch.int64) & mask), q * P), "attribute %d" % a
    host = out[:n].cpu().numpy().tobytes()
    for t in (0, 1, 37, 99):
        ref = oracle.Codec(H, W, attrs)
        prev = [p.cpu().numpy().view(DT[s]) for p, (s, _) in zip(planes[t - 1], attrs)] if t else None
        cur = [p.cpu().numpy().view(DT[s]) for p, (s, _) in zip(planes[t], attrs)]
        if prev is not None:
            ref.encode(prev)
        want = ref.encode(cur)
        if t:
            got = bytearray(host[offs[t]:offs[t + 1]])
            assert len(got) == len(want)
            got[4:8] = want[4:8]  # scan index: the oracle started this stream at t - 1
            assert bytes(got) == want, "frame %d" % t
        else:
            assert host[:offs[1]] == want


@pytest.mark.parametrize("force", [-1, 1])
def test_full_width_parked_scene_with_p_frames_against_oracle(force):
    """The parked scene (sensor at rest, 90 % of the dropouts on fixed pixels,
    10 mm range noise) at full width, through the enqueue-only calls: the P
    path (Sec. III-D: temporal residuals, mask XOR) at the benchmark's row
    width. With the trial, the second-return range is coded P in every frame
    after the first; forced, every attribute is. Whole stream compared with
    the oracle's, every frame decoded exactly."""
    cfg = synth.config_multi_attr(n_scans=8)
    cfg.speed_mps = 0.0
    cfg.persistent_dropout = 0.9
    cfg.range_noise_mm = 10.0
    seq = synth.ScanSequence(cfg, device="cuda")
    attrs = synth.attr_descs(cfg)
    T, H, W = cfg.n_scans, cfg.H, cfg.W
    scans = [seq.scan(t, as_numpy=False) for t in range(T)]
    host = [[p.cpu().numpy().view(DT[s]) for p, (s, _) in zip(sc, attrs)] for sc in scans]
    want, _, modes = oracle.encode_sequence(H, W, attrs, host, force_mode=force)
    assert all(modes[t][1] == 1 for t in range(1, T))
    want_planes, _ = oracle.decode_sequence(H, W, attrs, want, T)
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, force_mode=force)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, force_mode=force)
    planes = [torch.stack([scans[t][a] for t in range(T)]) for a in range(len(attrs))]
    out = torch.empty(J.jiffy_max_encoded_size(H, W, attrs, T), dtype=torch.uint8, device="cuda")
    d_offs = torch.zeros(T + 1, dtype=torch.int64, device="cuda")
    outs = J.empty_planes(dec, T)
    J.jiffy_encode_seq_async(enc, planes, out, d_offs)
    J.jiffy_decode_seq_async(dec, out, d_offs, outs)
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    assert out[:int(d_offs[-1])].cpu().numpy().tobytes() == want
    for t in range(T):
        for a, (s, _) in enumerate(attrs):
            assert np.array_equal(outs[a][t].cpu().numpy().view(DT[s]), want_planes[t][a]), (t, a)


@pytest.mark.parametrize("stages", range(1, 8))
@pytest.mark.parametrize("force", [-1, 0, 1])
def test_ablated_codecs_match_oracle(stages, force):
    # the stage switches of the Sec. IV-H ablations: bytes and planes equal
    # the oracle's for every stage set, in both entry points, across several
    # blocks and a ragged tail, with zeros, maxima and P frames
    rng = np.random.default_rng(300 + 3 * stages + force)
    H, W = 9, 1000
    attrs = [(4, 7), (2, 1), (1, 1)]
    base = [rand_scan(rng, H, W, s, 0.2) for s, _ in attrs]
    scans = []
    for t in range(4):
        planes = [drift(rng, b, s, 3, 0.1) for b, (s, _) in zip(base, attrs)]
        if t == 2:
            planes[1][0, :] = 0xFFFF  # maximal values: wide exceptions without ZigZag
        scans.append(planes)
    check_stream(H, W, attrs, scans, force_mode=force, seq=bool(stages % 2), stages=stages)


@pytest.mark.parametrize("stages", [1, 5, 7])
def test_ablated_codecs_on_the_benchmark_shape(stages):
    cfg = synth.config_multi_attr(n_scans=3, H=128, W=2048)
    seq = synth.ScanSequence(cfg).scans()
    check_stream(cfg.H, cfg.W, synth.attr_descs(cfg), seq, force_mode=0 if stages & 4 else -1, seq=True,
                 stages=stages)


def test_bounded_wait_runs_out_and_the_stream_recovers():
    # failure made on the host: one decoder row withholds its completion flag,
    # so the same row of the next (P) frame waits until the bounded device
    # wait gives up; the call reports a timeout, the stream's state is
    # unchanged and the device stays usable (the same frames decode next)
    rng = np.random.default_rng(77)
    H, W, attrs = 8, 512, [(2, 1), (1, 1)]
    base = [rand_scan(rng, H, W, s, 0.1) for s, _ in attrs]
    scans = [[drift(rng, b, s, 1, 0.0) for b, (s, _) in zip(base, attrs)] for _ in range(3)]
    gpu = GpuCodec(H, W, attrs, force_mode=1)  # frames 1 and 2 are P
    buf, offs = gpu.encode_seq(scans)
    assert buf == oracle.encode_sequence(H, W, attrs, scans, force_mode=1)[0]
    src = torch.from_numpy(np.frombuffer(buf, dtype=np.uint8).copy()).cuda()
    outs = [torch.empty((3, H, W), dtype=TORCH_DT[s], device="cuda") for s, _ in attrs]
    J.jiffy_stream_test_withhold_row(gpu.dec, 5)  # attribute 0, scan 0, row 5
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_decode_seq(gpu.dec, src, len(buf), offs, outs)
    assert ei.value.name == "JIFFY_ERR_TIMEOUT"
    assert J.jiffy_stream_frame_index(gpu.dec) == 0
    dec = gpu.decode_seq(buf, offs)  # same frames, no hook: decodes and matches the oracle
    want, _ = oracle.decode_sequence(H, W, attrs, buf, 3)
    for t in range(3):
        for a in range(len(attrs)):
            assert np.array_equal(dec[t][a], want[t][a])


def test_encoder_carry_wait_runs_out_and_the_stream_recovers():
    # only row 0 has nonzero samples, so a row r >= 5 finds no kept sample
    # among the 2048 samples before it (the direct search) and its delta
    # carry comes from the look-back over the earlier rows' last residuals;
    # one row withholds its status (host-side hook), the rows after it give
    # up after the bounded wait, the call reports a timeout and leaves the
    # stream as it was
    rng = np.random.default_rng(78)
    H, W, attrs = 8, 512, [(2, 1)]
    v = rand_scan(rng, H, W, 2, 0.05)
    v[1:, :] = 0
    gpu = GpuCodec(H, W, attrs)
    J.jiffy_stream_test_withhold_row(gpu.enc, 2)  # scan 0, row 2
    with pytest.raises(J.JiffyError) as ei:
        gpu.encode([v])
    assert ei.value.name == "JIFFY_ERR_TIMEOUT"
    assert J.jiffy_stream_frame_index(gpu.enc) == 0
    assert gpu.encode([v]) == oracle.Codec(H, W, attrs).encode([v])
