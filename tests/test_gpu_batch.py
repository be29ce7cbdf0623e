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
    """One encoder, decoder and oracle pair per sensor."""

    def __init__(self, sensors):
        self.sensors = sensors
        self.enc = [J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, a) for H, W, a in sensors]
        self.dec = [J.jiffy_stream_create(J.JIFFY_DECODER, H, W, a) for H, W, a in sensors]
        self.ref = [oracle.Codec(H, W, a) for H, W, a in sensors]
        self.refd = [oracle.Codec(H, W, a) for H, W, a in sensors]
        self.b = J.jiffy_batch_create()

    def encode(self, scans_per_stream, caps=None):
        planes = [[[to_dev(p) for p in sc] for sc in scans] for scans in scans_per_stream]
        outs = []
        for i, ((H, W, a), scans) in enumerate(zip(self.sensors, scans_per_stream)):
            cap = J.jiffy_max_encoded_size(H, W, a, len(scans)) if caps is None else caps[i]
            outs.append(torch.zeros(cap, dtype=torch.uint8, device="cuda"))
        res = J.jiffy_encode_batch(self.b, self.enc, planes, outs)
        return [(o[:n].cpu().numpy().tobytes(), offs) for o, (n, offs) in zip(outs, res)]


def test_batch_encode_decode_matches_oracle_over_calls():
    rng = np.random.default_rng(11)
    fleet = Fleet(SENSORS)
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
