"""GPU: the top of the stream-size sweep on the high-sparsity, low-coherence
workload. 4 GiB of raw planes (3277 scans of 128 x 2048: range u32 at 1 mm
precision + reflectivity u8, 40 % zeros in random discs, random yaw and
translation, so the trial mostly picks I frames) go through one encode call
and one decode call, enqueue-only on one CUDA stream as the benchmark's sweep
runs them. The encoder's row slots and the output capacity pass 2^32 bytes,
so 64-bit offsets are exercised. The round trip must be the identity
(precision 1), and sampled frames, re-coded by the oracle from their
predecessor, must match the GPU's bytes (except the scan index)."""
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

jbuild.build()

DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def test_low_coherence_4gib_stream_sampled_against_oracle():
    H, W = 128, 2048
    n = -(-4096 * 2**20 // (H * W * 5))  # scans of 4 GiB of raw planes
    cfg = synth.config_low_coherence(seed=7, n_scans=n)
    attrs = synth.attr_descs(cfg)
    seq = synth.ScanSequence(cfg, device="cuda")
    planes = [torch.empty((n, H, W), dtype=torch.int32, device="cuda"),
              torch.empty((n, H, W), dtype=torch.uint8, device="cuda")]
    for t in range(n):
        for a, p in enumerate(seq.scan(t, as_numpy=False)):
            planes[a][t].copy_(p)
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs)
    out = torch.empty(J.jiffy_max_encoded_size(H, W, attrs, n), dtype=torch.uint8, device="cuda")
    assert out.numel() > 2**32
    outs = J.empty_planes(dec, n)
    d_offs = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    J.jiffy_encode_seq_async(enc, planes, out, d_offs)
    J.jiffy_decode_seq_async(dec, out, d_offs, outs)
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    for a in range(2):
        assert torch.equal(outs[a], planes[a]), "attribute %d" % a
    offs = [int(x) for x in d_offs.cpu()]
    rng = np.random.default_rng(11)
    sample = sorted({0, 1, n // 2, n - 2, n - 1, *rng.integers(2, n - 2, size=3).tolist()})
    for t in sample:
        ref = oracle.Codec(H, W, attrs)
        if t:
            ref.encode([planes[a][t - 1].cpu().numpy().view(DT[s]) for a, (s, _) in enumerate(attrs)])
        want = ref.encode([planes[a][t].cpu().numpy().view(DT[s]) for a, (s, _) in enumerate(attrs)])
        lo = offs[t] if t else 0
        got = bytearray(out[lo:offs[t + 1]].cpu().numpy().tobytes())
        assert len(got) == len(want), "frame %d" % t
        if t:
            got[4:8] = want[4:8]  # scan index: the oracle started this stream at t - 1
        assert bytes(got) == want, "frame %d" % t
