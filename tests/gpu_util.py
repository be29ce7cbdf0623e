"""Helpers for the GPU tests: run the CUDA library on numpy scans."""
import numpy as np
import torch

from paper_2209_08196_gb300 import jiffy as J

NP_DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}
TORCH_DT = {1: torch.uint8, 2: torch.int16, 4: torch.int32}


def to_dev(x: np.ndarray) -> torch.Tensor:
    s = x.dtype.itemsize
    signed = {1: np.uint8, 2: np.int16, 4: np.int32}[s]
    return torch.from_numpy(np.ascontiguousarray(x).view(signed)).cuda()


def to_np(t: torch.Tensor, s: int) -> np.ndarray:
    return t.cpu().numpy().view(NP_DT[s])


class GpuCodec:
    def __init__(self, H, W, attrs, test_lines=4, force_mode=-1, stages=0):
        self.H, self.W, self.attrs = H, W, attrs
        self.enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, test_lines, force_mode, stages=stages)
        self.dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, test_lines, force_mode, stages=stages)

    def encode(self, planes):
        dev = [to_dev(p) for p in planes]
        cap = J.jiffy_max_encoded_size(self.H, self.W, self.attrs, 1)
        out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        n = J.jiffy_encode(self.enc, dev, out)
        return out[:n].cpu().numpy().tobytes()

    def encode_seq(self, scans):
        T = len(scans)
        dev = [[to_dev(p) for p in s] for s in scans]
        cap = J.jiffy_max_encoded_size(self.H, self.W, self.attrs, T)
        out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        n, offs = J.jiffy_encode_seq(self.enc, dev, out)
        return out[:n].cpu().numpy().tobytes(), offs

    def decode(self, buf: bytes):
        src = torch.from_numpy(np.frombuffer(buf, dtype=np.uint8).copy()).cuda()
        outs = [torch.empty((self.H, self.W), dtype=TORCH_DT[s], device="cuda") for s, _ in self.attrs]
        J.jiffy_decode(self.dec, src, len(buf), outs)
        return [to_np(o, s) for o, (s, _) in zip(outs, self.attrs)]

    def decode_seq(self, buf: bytes, offsets):
        T = len(offsets) - 1
        src = torch.from_numpy(np.frombuffer(buf, dtype=np.uint8).copy()).cuda()
        outs = [torch.empty((T, self.H, self.W), dtype=TORCH_DT[s], device="cuda") for s, _ in self.attrs]
        J.jiffy_decode_seq(self.dec, src, len(buf), offsets, outs)
        return [[to_np(outs[a][t], s) for a, (s, _) in enumerate(self.attrs)] for t in range(T)]
