"""GPU parity of the many-stream entry points (jiffy_encode_batch /
jiffy_decode_batch) against the oracle.

Several sensors of different shapes, attribute sets and scan counts are coded
in one launch sequence; each stream's bytes must equal what the oracle writes
for that stream alone, across successive calls (state carried per stream),
and a stream that fails inside a batch must leave the others, and its own
state, intact."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2209_08196_gb300 import build as jbuild  # noqa: E402
from paper_2209_08196_gb300 import jiffy as J  # noqa: E402
from tests.gpu_util import TORCH_DT, to_dev, to_np  # noqa: E402

jbuild.build()
DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}

# (H, W, attrs): mixed row counts, ragged widths, 1..3 attributes of all sizes
SENSORS = [
    (16, 1024, [(4, 10), (2, 1), (1, 1)]),
    (32, 500, [(4, 4)]),
    (8, 2048, [(2, 3), (4, 1)]),
    (5, 97, [(1, 1), (1, 2)]),
]


def make_scans(rng, H, W, attrs, T):
    base = []
    for s, _ in attrs:
        v = rng.integers(1, 1 << (8 * s), size=(H, W), dtype=np.uint64)
        v[rng.random((H, W)) < 0.15] = 0
        base.append(v.astype(np.int64))
    scans = []
    for t in range(T):
        planes = []
        for (s, _), b in zip(attrs, base):
            x = np.clip(b + rng.integers(-2, 3, size=b.shape) * (t % 3), 0, (1 << (8 * s)) - 1)
            x[rng.random(x.shape) < 0.02] = 0
            planes.append(x.astype(DT[s]))
        scans.append(planes)
    return scans


class Fleet:
    """One encoder, decoder and oracle pair per sensor (stages: optional
    per-sensor stage switches)."""

    def __init__(self, sensors, stages=None):
        self.sensors = sensors
        st = stages or [0] * len(sensors)
        self.enc = [J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, a, stages=g) for (H, W, a), g in zip(sensors, st)]
        self.dec = [J.jiffy_stream_create(J.JIFFY_DECODER, H, W, a, stages=g) for (H, W, a), g in zip(sensors, st)]
        self.ref = [oracle.Codec(H, W, a, stages=g) for (H, W, a), g in zip(sensors, st)]
        self.refd = [oracle.Codec(H, W, a, stages=g) for (H, W, a), g in zip(sensors, st)]
        self.b = J.jiffy_batch_create()

    def encode(self, scans_per_stream, caps=None):
        planes = [[[to_dev(p) for p in sc] for sc in scans] for scans in scans_per_stream]
        outs = []
        for i, ((H, W, a), scans) in enumerate(zip(self.sensors, scans_per_stream)):
            cap = J.jiffy_max_encoded_size(H, W, a, len(scans)) if caps is None else caps[i]
            outs.append(torch.zeros(cap, dtype=torch.uint8, device="cuda"))
        res = J.jiffy_encode_batch(self.b, self.enc, planes, outs)
        return [(o[:n].cpu().numpy().tobytes(), offs) for o, (n, offs) in zip(outs, res)]


@pytest.mark.parametrize("stages", [None, [0, 7, 1, 6]])
def test_batch_encode_decode_matches_oracle_over_calls(stages):
    # stages: streams of the full codec and ablated ones (Sec. IV-H) in the
    # same launches (the kernels that read stage switches then run every
    # segment, the full-codec ones included)
    rng = np.random.default_rng(11)
    fleet = Fleet(SENSORS, stages)
    T_calls = [[1, 3, 2, 4], [2, 1, 3, 1], [3, 2, 1, 2]]
    saw_p = False
    for Ts in T_calls:
        scans = [make_scans(rng, H, W, a, T) for (H, W, a), T in zip(SENSORS, Ts)]
        got = fleet.encode(scans)
        bufs, offsets, planes_out = [], [], []
        for i, ((H, W, a), sc) in enumerate(zip(SENSORS, scans)):
            parts = [fleet.ref[i].encode(s, return_modes=True) for s in sc]
            saw_p |= any(m == 1 for _, modes in parts for m in modes)
            want = b"".join(b for b, _ in parts)
            buf, offs = got[i]
            assert buf == want, "stream %d: batch bytes differ from the oracle" % i
            bufs.append(torch.from_numpy(np.frombuffer(buf, dtype=np.uint8).copy()).cuda())
            offsets.append(offs)
            planes_out.append([torch.empty((len(sc), H, W), dtype=TORCH_DT[s], device="cuda") for s, _ in a])
        J.jiffy_decode_batch(fleet.b, fleet.dec, bufs, [len(x) for x, _ in got], offsets, planes_out)
        for i, ((H, W, a), sc) in enumerate(zip(SENSORS, scans)):
            buf, offs = got[i]
            for t in range(len(sc)):
                frame = buf[(offs[t] if t else 0):offs[t + 1]]
                want, _ = fleet.refd[i].decode(frame)
                for k, (s, _) in enumerate(a):
                    assert np.array_equal(to_np(planes_out[i][k][t], s), want[k]), (i, t, k)
        for i, T in enumerate(Ts):
            assert J.jiffy_stream_frame_index(fleet.enc[i]) == J.jiffy_stream_frame_index(fleet.dec[i])
    assert saw_p, "the sequences should select P for some attribute"


def test_mixed_row_widths_in_one_call_match_oracle():
    # rows wider than 2048 columns next to narrower ones: the encoder runs the
    # narrow segments' rows in a launch of their own (wide ones after), and
    # the segments are numbered narrow first whatever the call's order
    rng = np.random.default_rng(19)
    sensors = [(4, 3000, [(4, 10), (2, 1)]), (8, 500, [(4, 4)]), (2, 5000, [(1, 1)]), (6, 2048, [(2, 3)]),
               (3, 2049, [(4, 1)])]
    fleet = Fleet(sensors)
    for Ts in ([2, 1, 3, 1, 2], [1, 2, 1, 2, 1]):
        scans = [make_scans(rng, H, W, a, T) for (H, W, a), T in zip(sensors, Ts)]
        got = fleet.encode(scans)
        bufs, offsets, planes_out = [], [], []
        for i, ((H, W, a), sc) in enumerate(zip(sensors, scans)):
            want = b"".join(fleet.ref[i].encode(x) for x in sc)
            assert got[i][0] == want, "stream %d" % i
            bufs.append(torch.from_numpy(np.frombuffer(got[i][0], dtype=np.uint8).copy()).cuda())
            offsets.append(got[i][1])
            planes_out.append([torch.empty((len(sc), H, W), dtype=TORCH_DT[x], device="cuda") for x, _ in a])
        J.jiffy_decode_batch(fleet.b, fleet.dec, bufs, [len(x) for x, _ in got], offsets, planes_out)
        for i, ((H, W, a), sc) in enumerate(zip(sensors, scans)):
            buf, offs = got[i]
            for t in range(len(sc)):
                want, _ = fleet.refd[i].decode(buf[(offs[t] if t else 0):offs[t + 1]])
                for k, (x, _) in enumerate(a):
                    assert np.array_equal(to_np(planes_out[i][k][t], x), want[k]), (i, t, k)


def test_batch_equals_per_stream_calls():
    rng = np.random.default_rng(12)
    scans = [make_scans(rng, H, W, a, 3) for H, W, a in SENSORS]
    fleet = Fleet(SENSORS)
    got = fleet.encode(scans)
    for i, (H, W, a) in enumerate(SENSORS):
        h = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, a)
        out = torch.zeros(J.jiffy_max_encoded_size(H, W, a, 3), dtype=torch.uint8, device="cuda")
        n, offs = J.jiffy_encode_seq(h, [[to_dev(p) for p in s] for s in scans[i]], out)
        assert out[:n].cpu().numpy().tobytes() == got[i][0]
        assert offs == got[i][1]


def test_failing_stream_keeps_others_and_its_state():
    rng = np.random.default_rng(13)
    fleet = Fleet(SENSORS[:3])
    scans = [make_scans(rng, H, W, a, 2) for H, W, a in SENSORS[:3]]
    caps = [J.jiffy_max_encoded_size(H, W, a, 2) for H, W, a in SENSORS[:3]]
    caps[1] = 64  # too small for stream 1
    with pytest.raises(J.BatchError) as ei:
        fleet.encode(scans, caps)
    assert ei.value.status == 2
    assert ei.value.statuses == [0, 2, 0]
    assert ei.value.required[1] > 64
    assert [J.jiffy_stream_frame_index(h) for h in fleet.enc] == [2, 0, 2]
    # streams 0 and 2 advanced (their oracle twins too); stream 1 starts over
    for i in (0, 2):
        for s in scans[i]:
            fleet.ref[i].encode(s)
    again = [make_scans(rng, H, W, a, 1) for H, W, a in SENSORS[:3]]
    again[1] = scans[1]
    got = fleet.encode(again)
    for i in range(3):
        want = b"".join(fleet.ref[i].encode(s) for s in again[i])
        assert got[i][0] == want, i


def test_batch_rejects_repeated_stream_and_wrong_role():
    H, W, a = SENSORS[0]
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, a)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, a)
    b = J.jiffy_batch_create()
    sc = [to_dev(p) for p in make_scans(np.random.default_rng(1), H, W, a, 1)[0]]
    out = [torch.zeros(J.jiffy_max_encoded_size(H, W, a, 1), dtype=torch.uint8, device="cuda") for _ in range(2)]
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_encode_batch(b, [enc, enc], [[sc], [sc]], out)
    assert ei.value.status == 1
    with pytest.raises(J.JiffyError) as ei:
        J.jiffy_encode_batch(b, [enc, dec], [[sc], [sc]], out)
    assert ei.value.status == 4
    assert J.jiffy_stream_frame_index(enc) == 0


def _oracle_bytes(fleet, i, scans):
    return b"".join(fleet.ref[i].encode(s) for s in scans)


def test_graph_replay_matches_oracle():
    rng = np.random.default_rng(14)
    fleet = Fleet(SENSORS)
    J.jiffy_batch_set_graphs(fleet.b, True)
    for call in range(3):
        scans = [make_scans(rng, H, W, a, 2) for H, W, a in SENSORS]
        got = fleet.encode(scans)
        for i in range(len(SENSORS)):
            assert got[i][0] == _oracle_bytes(fleet, i, scans[i]), (call, i)
    # each call captures or replays its table slot's sequence: one capture
    # per slot (one or two slots), the rest replays
    info = J.jiffy_batch_info(fleet.b)
    assert info["graph_captures"] + info["graph_replays"] == 3 and 1 <= info["graph_captures"] <= 2, info
    # a different shape captures again
    scans = [make_scans(rng, H, W, a, 1) for H, W, a in SENSORS]
    got = fleet.encode(scans)
    for i in range(len(SENSORS)):
        assert got[i][0] == _oracle_bytes(fleet, i, scans[i])
    assert J.jiffy_batch_info(fleet.b)["graph_captures"] == info["graph_captures"] + 1


@pytest.mark.parametrize("wpc,ctas", [(1, 1), (2, 0), (4, 1), (4, 2)])
def test_every_encode_launch_configuration_codes_the_same_bytes(wpc, ctas):
    rng = np.random.default_rng(15)
    fleet = Fleet(SENSORS)
    J.jiffy_batch_set_launch(fleet.b, J.JIFFY_ENCODER, wpc, ctas, 0)
    scans = [make_scans(rng, H, W, a, 3) for H, W, a in SENSORS]
    got = fleet.encode(scans)
    info = J.jiffy_batch_info(fleet.b)
    assert info["warps_per_cta"] == wpc and (ctas == 0 or info["ctas_per_sm"] <= ctas)
    for i in range(len(SENSORS)):
        assert got[i][0] == _oracle_bytes(fleet, i, scans[i])


@pytest.mark.parametrize("wpc,ctas,ipt", [(1, 1, 1), (8, 0, 16), (2, 2, 64), (4, 0, 3)])
def test_every_decode_launch_configuration_decodes_the_same(wpc, ctas, ipt):
    rng = np.random.default_rng(16)
    fleet = Fleet(SENSORS)
    scans = [make_scans(rng, H, W, a, 4) for H, W, a in SENSORS]
    got = fleet.encode(scans)
    J.jiffy_batch_set_launch(fleet.b, J.JIFFY_DECODER, wpc, ctas, ipt)
    bufs = [torch.from_numpy(np.frombuffer(x, dtype=np.uint8).copy()).cuda() for x, _ in got]
    outs = [[torch.empty((4, H, W), dtype=TORCH_DT[s], device="cuda") for s, _ in a] for H, W, a in SENSORS]
    J.jiffy_decode_batch(fleet.b, fleet.dec, bufs, [len(x) for x, _ in got], [o for _, o in got], outs)
    info = J.jiffy_batch_info(fleet.b)
    assert info["warps_per_cta"] == wpc and info["items_per_ticket"] == ipt, info
    for i, (H, W, a) in enumerate(SENSORS):
        want, _ = oracle.decode_sequence(H, W, a, got[i][0], 4)
        for t in range(4):
            for k, (s, _) in enumerate(a):
                assert np.array_equal(to_np(outs[i][k][t], s), want[t][k]), (i, t, k)


def test_autotune_keeps_bytes_and_records_a_choice():
    rng = np.random.default_rng(17)
    fleet = Fleet(SENSORS)
    J.jiffy_batch_set_autotune(fleet.b, True)
    for call in range(2):
        scans = [make_scans(rng, H, W, a, 2) for H, W, a in SENSORS]
        got = fleet.encode(scans)
        for i in range(len(SENSORS)):
            assert got[i][0] == _oracle_bytes(fleet, i, scans[i]), (call, i)
    info = J.jiffy_batch_info(fleet.b)
    assert info["tunings"] == 1 and info["tuned_classes"] == 1, info


def test_async_calls_on_two_batches_overlap_and_match():
    rng = np.random.default_rng(18)
    half = [SENSORS[:2], SENSORS[2:]]
    fleets = [Fleet(h) for h in half]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for call in range(3):
        scans = [[make_scans(rng, H, W, a, 2) for H, W, a in h] for h in half]
        outs, keep = [], []
        for f, sc, cs in zip(fleets, scans, streams):
            planes = [[[to_dev(p) for p in s] for s in x] for x in sc]
            o = [torch.zeros(J.jiffy_max_encoded_size(H, W, a, 2), dtype=torch.uint8, device="cuda")
                 for H, W, a in f.sensors]
            torch.cuda.synchronize()
            J.jiffy_encode_batch_async(f.b, f.enc, planes, o, stream=cs)
            outs.append(o)
            keep.append(planes)
        for f, o, sc in zip(fleets, outs, scans):
            res = J.jiffy_batch_wait(f.b)
            for i, (n, _) in enumerate(res):
                assert o[i][:n].cpu().numpy().tobytes() == _oracle_bytes(f, i, sc[i]), (call, i)


def test_async_call_blocks_its_streams_until_waited():
    H, W, a = SENSORS[1]
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, a)
    b1, b2 = J.jiffy_batch_create(), J.jiffy_batch_create()
    sc = [[to_dev(p) for p in make_scans(np.random.default_rng(2), H, W, a, 1)[0]]]
    o = [torch.zeros(J.jiffy_max_encoded_size(H, W, a, 1), dtype=torch.uint8, device="cuda")]
    J.jiffy_encode_batch_async(b1, [enc], [sc], o)
    with pytest.raises(J.JiffyError) as ei:  # the stream is in flight in b1
        J.jiffy_encode_batch(b2, [enc], [sc], o)
    assert ei.value.status == 4
    with pytest.raises(J.JiffyError) as ei:  # b1 has an unfinished call
        J.jiffy_encode_batch_async(b1, [enc], [sc], o)
    assert ei.value.status == 4
    J.jiffy_batch_wait(b1)
    assert J.jiffy_stream_frame_index(enc) == 1


def test_decoder_takes_over_from_encoder_state():
    """A decode request for the frame an encoder codes next: copy the
    encoder's state into a decoder first (both hold the previous scan as
    decoded), then decode the new frame alone."""
    rng = np.random.default_rng(19)
    H, W, a = SENSORS[0]
    scans = make_scans(rng, H, W, a, 5)
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, a)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, a)
    ref = oracle.Codec(H, W, a)
    refd = oracle.Codec(H, W, a)
    cap = J.jiffy_max_encoded_size(H, W, a, 1)
    for t, sc in enumerate(scans):
        want_bytes = ref.encode(sc)
        want_planes, _ = refd.decode(want_bytes)
        out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        if t in (0, 3, 4):
            J.jiffy_stream_copy_state(dec, enc)
        n = J.jiffy_encode(enc, [to_dev(p) for p in sc], out)
        assert out[:n].cpu().numpy().tobytes() == want_bytes
        if t in (0, 3, 4):
            got = J.empty_planes(dec)
            J.jiffy_decode(dec, out, n, got)
            for k, (s, _) in enumerate(a):
                assert np.array_equal(to_np(got[k], s), want_planes[k]), (t, k)
    other = J.jiffy_stream_create(J.JIFFY_DECODER, H, W + 1, a)
    with pytest.raises(J.JiffyError):
        J.jiffy_stream_copy_state(other, enc)


def test_array_marshalled_calls_match_oracle_over_calls():
    # jiffy_*_batch_async_arrays: per-stream arguments as numpy arrays of
    # addresses, plane tables built once; bytes, offsets and decoded planes
    # equal the oracle's over calls of different scan counts
    import ctypes
    rng = np.random.default_rng(17)
    fleet = Fleet(SENSORS)
    for Ts in ([2, 1, 3, 1], [1, 2, 1, 3]):
        scans = [make_scans(rng, H, W, a, T) for (H, W, a), T in zip(SENSORS, Ts)]
        dev = [[to_dev(p) for sc in ss for p in sc] for ss in scans]  # scan-major planes per stream
        tabs = [J.plane_table(d) for d in dev]
        outs = [torch.zeros(J.jiffy_max_encoded_size(H, W, a, T), dtype=torch.uint8, device="cuda")
                for (H, W, a), T in zip(SENSORS, Ts)]
        J.jiffy_encode_batch_async_arrays(fleet.b, [h.ptr for h in fleet.enc], Ts,
                                          [ctypes.addressof(t) for t in tabs], [o.data_ptr() for o in outs],
                                          [o.numel() for o in outs])
        lens, offs, starts = J.jiffy_batch_wait(fleet.b)
        bufs = []
        for i, ((H, W, a), sc) in enumerate(zip(SENSORS, scans)):
            want = b"".join(fleet.ref[i].encode(s) for s in sc)
            got = outs[i][:int(lens[i])].cpu().numpy().tobytes()
            assert got == want, "stream %d" % i
            o = offs[starts[i]:starts[i] + Ts[i] + 1].tolist()
            assert o[-1] == len(want)
            bufs.append(got)
        planes_out = [[torch.empty((H, W), dtype=TORCH_DT[s], device="cuda") for _ in range(T) for s, _ in a]
                      for (H, W, a), T in zip(SENSORS, Ts)]
        dtabs = [J.plane_table(p) for p in planes_out]
        J.jiffy_decode_batch_async_arrays(fleet.b, [h.ptr for h in fleet.dec], Ts, [o.data_ptr() for o in outs],
                                          lens, offs, starts, [ctypes.addressof(t) for t in dtabs])
        assert J.jiffy_batch_wait(fleet.b) is None
        for i, ((H, W, a), sc) in enumerate(zip(SENSORS, scans)):
            o = offs[starts[i]:starts[i] + Ts[i] + 1].tolist()
            for t in range(Ts[i]):
                want, _ = fleet.refd[i].decode(bufs[i][(o[t] if t else 0):o[t + 1]])
                for k, (s, _) in enumerate(a):
                    assert np.array_equal(to_np(planes_out[i][t * len(a) + k], s), want[k]), (i, t, k)


def test_tune_cache_keeps_tuned_launches_for_the_next_batch(tmp_path, monkeypatch):
    # JIFFY_TUNE_CACHE: the first batch tunes its shape classes and writes
    # them out; a batch created afterwards loads them and tunes nothing,
    # coding the same bytes
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("JIFFY_TUNE_CACHE", str(path))
    rng = np.random.default_rng(18)
    scans = [make_scans(rng, H, W, a, 2) for H, W, a in SENSORS]
    first = Fleet(SENSORS)
    J.jiffy_batch_set_autotune(first.b, True)
    got1 = first.encode(scans)
    assert J.jiffy_batch_info(first.b)["tunings"] >= 1
    lines = path.read_text().splitlines()
    assert lines and all(ln.startswith("jiffy-tune 1 ") for ln in lines)
    second = Fleet(SENSORS)
    J.jiffy_batch_set_autotune(second.b, True)
    got2 = second.encode(scans)
    info = J.jiffy_batch_info(second.b)
    assert info["tunings"] == 0 and info["tuned_classes"] >= 1
    assert [b for b, _ in got2] == [b for b, _ in got1]
    for i, ((H, W, a), sc) in enumerate(zip(SENSORS, scans)):
        assert got1[i][0] == b"".join(first.ref[i].encode(x) for x in sc)
    # a damaged file only means tuning anew
    path.write_text("jiffy-tune 1 garbage\n")
    third = Fleet(SENSORS)
    J.jiffy_batch_set_autotune(third.b, True)
    assert [b for b, _ in third.encode(scans)] == [b for b, _ in got1]
    assert J.jiffy_batch_info(third.b)["tunings"] >= 1


def test_many_stream_workload_sampled_against_oracle():
    # the many-stream configuration (uneven shapes from 16x1024 to 128x4096,
    # attribute sets {range}, {range, signal}, all five; 8 scans each) in one
    # batched call each way; sampled streams, the widest among them, checked
    # byte for byte and plane for plane against the oracle
    from paper_2209_08196_gb300 import synth
    cfgs = [synth.batch_stream_config(i, base_seed=77, n_scans=8) for i in range(24)]
    encs, decs, planes, outs, attrs_l = [], [], [], [], []
    for c in cfgs:
        at = synth.attr_descs(c)
        attrs_l.append(at)
        seq = synth.ScanSequence(c, device="cuda")
        sc = [seq.scan(t, as_numpy=False) for t in range(c.n_scans)]
        planes.append([torch.stack([sc[t][a] for t in range(c.n_scans)]) for a in range(len(at))])
        encs.append(J.jiffy_stream_create(J.JIFFY_ENCODER, c.H, c.W, at))
        decs.append(J.jiffy_stream_create(J.JIFFY_DECODER, c.H, c.W, at))
        outs.append(torch.empty(J.jiffy_max_encoded_size(c.H, c.W, at, c.n_scans), dtype=torch.uint8, device="cuda"))
    b = J.jiffy_batch_create()
    res = J.jiffy_encode_batch(b, encs, planes, outs)
    dec_planes = [J.empty_planes(d, c.n_scans) for d, c in zip(decs, cfgs)]
    J.jiffy_decode_batch(b, decs, outs, [n for n, _ in res], [o for _, o in res], dec_planes)
    widest = max(range(len(cfgs)), key=lambda i: cfgs[i].H * cfgs[i].W * len(attrs_l[i]))
    for i in sorted({0, 5, 11, 17, widest}):
        c, at = cfgs[i], attrs_l[i]
        host = [[to_np(planes[i][a][t], s) for a, (s, _) in enumerate(at)] for t in range(c.n_scans)]
        want, _, _ = oracle.encode_sequence(c.H, c.W, at, host)
        n, offs = res[i]
        assert outs[i][:n].cpu().numpy().tobytes() == want, i
        ref_planes, _ = oracle.decode_sequence(c.H, c.W, at, want, c.n_scans)
        for t in range(c.n_scans):
            for a, (s, _) in enumerate(at):
                assert np.array_equal(to_np(dec_planes[i][a][t], s), ref_planes[t][a]), (i, t, a)
