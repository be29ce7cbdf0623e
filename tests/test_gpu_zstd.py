"""GPU: the Zstandard mask (Sec. III-C: the zero bitmask packed into bytes and
compressed with Zstd, XORed with the previous scan's for P, Sec. III-D) against
the oracle. Bytes must be identical and the planes must round trip.

Cases: row widths whose byte rows are not whole words, sections of several
8192-byte blocks (up to 256), masks that give RLE, Raw and Compressed blocks
with direct and FSE-coded Huffman weights, one and four streams; I, P and
trial modes; the single-call, sequence, enqueue-only (graph replay) and
batched entry points; the stage switches combined with it; malformed frames
rejected without faults. libzstd restores
every mask frame the GPU writes to the packed zero masks of the inputs."""
import ctypes
import ctypes.util

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2209_08196_gb300 import build as jbuild  # noqa: E402
from paper_2209_08196_gb300 import jiffy as J  # noqa: E402
from paper_2209_08196_gb300 import streaminfo, synth  # noqa: E402
from tests.gpu_util import TORCH_DT, GpuCodec, to_dev, to_np  # noqa: E402
from tests.test_gpu_parity import check_stream, drift, rand_scan  # noqa: E402

jbuild.build()
Z = J.STAGE_ZSTD_MASK
DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def masked_scans(rng, H, W, attrs, T, kind):
    """T scans whose zero masks give the block kinds asked for."""
    base = [rand_scan(rng, H, W, s, 0.0) for s, _ in attrs]
    scans = []
    for t in range(T):
        planes = []
        for b, (s, _) in zip(base, attrs):
            x = drift(rng, b, s, 2, 0.0)
            x[x == 0] = 1
            if kind == "sparse":      # 12 % zeros: Compressed, FSE weights
                x[rng.random(x.shape) < 0.12] = 0
            elif kind == "half":      # 50 % zeros: Raw
                x[rng.random(x.shape) < 0.5] = 0
            elif kind == "none":      # no zeros: RLE (and all-zero P masks)
                pass
            elif kind == "low7":      # zeros only off bit 7 of each byte: direct weights
                cols = (np.arange(W) % 8) != 7
                x[(rng.random(x.shape) < 0.1) & cols[None, :]] = 0
            elif kind == "rows":      # whole zero rows and runs (structured)
                x[rng.integers(0, H, max(1, H // 4))] = 0
                x[:, :W // 5] = 0
            planes.append(x)
        scans.append(planes)
    return scans


@pytest.mark.parametrize("H,W", [(1, 16), (3, 37), (9, 1000), (16, 512), (40, 1700), (64, 2048), (1, 16384)])
@pytest.mark.parametrize("force", [-1, 0, 1])
def test_shapes_and_modes_match_oracle(H, W, force):
    rng = np.random.default_rng(H * 7919 + W + force)
    attrs = [(4, 10), (2, 1), (1, 1)]
    scans = masked_scans(rng, H, W, attrs, 4, "sparse")
    check_stream(H, W, attrs, scans, force_mode=force, seq=(H + W) % 2 == 0, stages=Z)
    check_stream(H, W, attrs, scans, force_mode=force, seq=(H + W) % 2 == 1, stages=Z)


@pytest.mark.parametrize("kind", ["sparse", "half", "none", "low7", "rows"])
def test_block_kinds_match_oracle_and_libzstd(kind):
    rng = np.random.default_rng(["sparse", "half", "none", "low7", "rows"].index(kind) + 500)
    H, W, attrs = 48, 1400, [(2, 1), (1, 1)]  # 8400 mask bytes: a full block and a short one
    scans = masked_scans(rng, H, W, attrs, 3, kind)
    frames = check_stream(H, W, attrs, scans, stages=Z, seq=True)
    buf = b"".join(frames)
    _, secs = streaminfo.sections(buf)  # reads every frame back with libzstd
    for s in secs:
        assert s.coded == s.nnz
    if ctypes.util.find_library("zstd") is None:
        return
    z = ctypes.CDLL(ctypes.util.find_library("zstd"))
    z.ZSTD_decompress.restype = ctypes.c_size_t
    z.ZSTD_decompress.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t]
    rb = (W + 7) // 8
    nblk = -(-H * rb // 8192)
    pos, prev = 16 + 8 * len(attrs), None
    for t, sc in enumerate(scans):
        fh = buf[pos:pos + 8 + 12 * len(attrs)]
        sp = pos + len(fh)
        packed = []
        for a, (s, P) in enumerate(attrs):
            mode = fh[8 + 12 * a]
            sb = int.from_bytes(fh[12 + 12 * a:16 + 12 * a], "little")
            zp = sp + 8 * H
            fb = int.from_bytes(buf[zp:zp + 4], "little")
            frame = np.frombuffer(buf[zp + 4 + 4 * nblk:zp + 4 + 4 * nblk + fb], dtype=np.uint8).copy()
            bits = np.zeros((H, 8 * rb), dtype=bool)
            bits[:, :W] = sc[a] == 0
            want = np.packbits(bits, axis=1, bitorder="little").reshape(-1)
            packed.append(want)
            if mode == 1:
                want = want ^ prev[a]
            out = np.zeros(H * rb + 16, dtype=np.uint8)
            k = z.ZSTD_decompress(out.ctypes.data, out.nbytes, frame.ctypes.data, fb)
            assert k == H * rb and np.array_equal(out[:k], want), (t, a)
            sp += sb
        prev = packed
        pos = sp


@pytest.mark.parametrize("extra", [J.STAGE_NO_DELTA, J.STAGE_NO_ZIGZAG, J.STAGE_NO_DELTA | J.STAGE_NO_ZIGZAG])
def test_with_other_stage_switches(extra):
    rng = np.random.default_rng(40 + extra)
    H, W, attrs = 9, 1000, [(4, 7), (2, 1), (1, 1)]
    scans = masked_scans(rng, H, W, attrs, 4, "sparse")
    for force in (-1, 0, 1):
        check_stream(H, W, attrs, scans, force_mode=force, seq=True, stages=Z | extra)


def test_benchmark_shape_sequence():
    cfg = synth.config_multi_attr(n_scans=4, H=128, W=2048)
    scans = synth.ScanSequence(cfg).scans()
    check_stream(cfg.H, cfg.W, synth.attr_descs(cfg), scans, seq=True, stages=Z)
    check_stream(cfg.H, cfg.W, synth.attr_descs(cfg), scans, force_mode=1, seq=True, stages=Z)


def test_batched_streams_with_and_without_the_zstd_mask():
    rng = np.random.default_rng(77)
    cfgs = [(16, 1024, [(4, 10), (1, 1)], Z), (8, 300, [(2, 1)], 0), (40, 1700, [(4, 10)], Z)]
    T = 3
    b = J.jiffy_batch_create()
    encs, decs, planes, outs, scans_all = [], [], [], [], []
    for H, W, attrs, st in cfgs:
        encs.append(J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, stages=st))
        decs.append(J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, stages=st))
        scans = masked_scans(rng, H, W, attrs, T, "sparse")
        scans_all.append(scans)
        planes.append([[to_dev(p) for p in s] for s in scans])
        outs.append(torch.zeros(J.jiffy_max_encoded_size(H, W, attrs, T), dtype=torch.uint8, device="cuda"))
    res = J.jiffy_encode_batch(b, encs, planes, outs)
    bufs, lens, offs, pout = [], [], [], []
    for (H, W, attrs, st), scans, (n, off), o in zip(cfgs, scans_all, res, outs):
        want, _, _ = oracle.encode_sequence(H, W, attrs, scans, stages=st)
        assert o[:n].cpu().numpy().tobytes() == want
        bufs.append(o)
        lens.append(n)
        offs.append(off)
        pout.append([torch.empty((T, H, W), dtype=TORCH_DT[s], device="cuda") for s, _ in attrs])
    J.jiffy_decode_batch(b, decs, bufs, lens, offs, pout)
    for (H, W, attrs, st), scans, po in zip(cfgs, scans_all, pout):
        for t in range(T):
            for a, (s, P) in enumerate(attrs):
                m = (1 << (8 * s)) - 1
                q = np.minimum(((scans[t][a].astype(np.int64) & m) + P // 2) // P, m // P)
                assert np.array_equal(to_np(po[a][t], s).astype(np.int64), q * P)


def test_malformed_frames_are_rejected_without_faults():
    rng = np.random.default_rng(9)
    H, W, attrs = 40, 1700, [(4, 10), (1, 1)]
    scans = masked_scans(rng, H, W, attrs, 1, "sparse")
    good = GpuCodec(H, W, attrs, stages=Z).encode(scans[0])
    A = len(attrs)
    sec = 16 + 8 * A + 8 + 12 * A
    zp = sec + 8 * H
    nblk = -(-H * ((W + 7) // 8) // 8192)
    fz = zp + 4 + 4 * nblk
    cases = []
    for at, x in ((fz, 1), (fz + 4, 0x40), (fz + 5, 1), (zp + 4, 4), (zp, 4), (fz + 9, 6), (fz + 30, 0x55),
                  (fz + 200, 0xFF)):
        b = bytearray(good)
        b[at] ^= x
        cases.append(bytes(b))
    for bad in cases:
        try:
            want_err = False
            oracle.Codec(H, W, attrs, stages=Z).decode(bad)
        except oracle.OracleError:
            want_err = True
        g = GpuCodec(H, W, attrs, stages=Z)
        if want_err:
            with pytest.raises(J.JiffyError) as ei:
                g.decode(bad)
            assert ei.value.status == 3
        else:  # a change the format cannot see (a literal code) decodes as the oracle decodes it
            out = g.decode(bad)
            ref, _ = oracle.Codec(H, W, attrs, stages=Z).decode(bad)
            for o, w in zip(out, ref):
                assert np.array_equal(o, w)
    # a class-coded decoder refuses the stream, and the stream still decodes
    with pytest.raises(J.JiffyError):
        GpuCodec(H, W, attrs).decode(good)
    out = GpuCodec(H, W, attrs, stages=Z).decode(good)
    want, _ = oracle.Codec(H, W, attrs, stages=Z).decode(good)
    for o, w in zip(out, want):
        assert np.array_equal(o, w)


def test_options_that_cannot_be_combined():
    with pytest.raises(J.JiffyError):
        J.jiffy_stream_create(J.JIFFY_ENCODER, 4, 64, [(2, 1)], stages=Z | J.STAGE_NO_MASK)
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = [torch.zeros((4, 64), dtype=torch.int16, device="cuda")]
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_decode_frame_noalloc(buf, 64, 4, 64, [(2, 1)], 0, None, out, stages=Z)
    assert ei.value.name == "JIFFY_ERR_INVALID_ARG"


def test_large_sections_of_many_blocks():
    # 1024 x 16384: 2 MiB of mask bytes per section, 256 blocks (the writer's
    # and the reader's grids run 256 blocks deep; the block-end index has 256
    # entries); an I frame, then P
    rng = np.random.default_rng(123)
    H, W, attrs = 1024, 16384, [(1, 1)]
    b = rng.integers(1, 256, size=(H, W)).astype(np.uint8)
    scans = []
    for t in range(2):
        x = b.copy()
        x[rng.random((H, W)) < 0.1] = 0
        scans.append([x])
    check_stream(H, W, attrs, scans, force_mode=1, seq=True, stages=Z)


def test_enqueue_only_pair_replays_graphs():
    # the enqueue-only pair with the frame offsets left on the device; calls
    # after the first replay the stream's captured launch sequence
    rng = np.random.default_rng(321)
    H, W, attrs, T = 32, 1000, [(4, 10), (2, 1), (1, 1)], 4
    scans = masked_scans(rng, H, W, attrs, T, "sparse")
    want, _, _ = oracle.encode_sequence(H, W, attrs, scans, stages=Z)
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, stages=Z)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, stages=Z)
    planes = [[to_dev(p) for p in s] for s in scans]
    out = torch.zeros(J.jiffy_max_encoded_size(H, W, attrs, T), dtype=torch.uint8, device="cuda")
    d_offs = torch.zeros(T + 1, dtype=torch.int64, device="cuda")
    outs = J.empty_planes(dec, T)
    for _ in range(3):
        J.jiffy_stream_reset(enc)
        J.jiffy_stream_reset(dec)
        outs[0].zero_()
        J.jiffy_encode_seq_async(enc, planes, out, d_offs)
        J.jiffy_decode_seq_async(dec, out, d_offs, outs)
        J.jiffy_stream_wait(enc)
        J.jiffy_stream_wait(dec)
        assert out[:int(d_offs[T])].cpu().numpy().tobytes() == want
        for t in range(T):
            for a, (s, P) in enumerate(attrs):
                m = (1 << (8 * s)) - 1
                q = np.minimum(((scans[t][a].astype(np.int64) & m) + P // 2) // P, m // P)
                assert np.array_equal(to_np(outs[a][t], s).astype(np.int64), q * P), (t, a)
