"""Seeded synthetic LiDAR scans shaped like the paper's workloads.

Stand-in for the paper's Ouster driving / infrastructure / drone datasets
(Sec. IV-B, Tables I and II), which are not available here. A spinning sensor
with H beams (elevations evenly spaced over [-22.5, 22.5] degrees) and W
azimuth columns casts rays into a scene made of a ground plane at z = -1.8 m
and 40 axis-aligned boxes (sides 1-10 m) resting on the ground, centred within
80 m of the start. Boxes are recycled modulo a 160 m window around the sensor
so the density stays constant over long runs. Range is the first hit in mm
(uint32); returns beyond 120 m and dropped returns are 0 (the invalid
sentinel, Sec. III-A). Attributes follow the scan types of Sec. IV-B: a
second-return range at depth discontinuities, signal (uint16, reflectivity /
r^2 with Poisson noise), reflectivity (uint8, per object +/- 3) and ambient
near-infrared (uint16, smooth field + Gaussian noise).

This module holds no codec arithmetic: it only makes raw sensor planes. It
runs on the CPU or, for large benchmark workloads, on a CUDA device through
PyTorch tensor operations; random draws come from seeded generators.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

RANGE, RANGE2, SIGNAL, REFLECTIVITY, AMBIENT = "range", "range2", "signal", "reflectivity", "ambient"

# attribute -> (bytes per sample, precision used by the workloads)
ATTR_DTYPE = {RANGE: 4, RANGE2: 4, SIGNAL: 2, REFLECTIVITY: 1, AMBIENT: 2}
_TORCH_DT = {1: torch.uint8, 2: torch.int16, 4: torch.int32}
_NP_DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}

MAX_RANGE_M = 120.0


@dataclass
class SensorConfig:
    H: int
    W: int
    attrs: tuple = (RANGE,)
    precisions: tuple = (10,)
    n_scans: int = 16
    dropout: float = 0.08          # i.i.d. dropout probability
    persistent_dropout: float = 0.0  # share of the dropouts on a fixed pixel set (same every scan)
    range_noise_mm: float = 0.0    # Gaussian range noise, standard deviation in mm
    target_zero_frac: float | None = None   # tune dropouts so range has this zero fraction
    disc_zero_frac: float = 0.0    # clustered dropouts: discs of radius 5..40 px
    speed_mps: float = 10.0        # forward motion along +x
    random_motion: bool = False    # random translation direction + yaw per scan
    yaw_rate_dps: float = 0.0      # max |yaw rate| for random_motion
    wall: bool = False             # enclosing wall at 110 m (removes sky zeros)
    rate_hz: float = 10.0
    seed: int = 0
    extra: dict = field(default_factory=dict)


def config_small_range(seed=0, n_scans=16, H=64, W=1024):
    """16 scans of 64 x 1024, range only, 10 mm precision, 8 % dropouts."""
    return SensorConfig(H=H, W=W, attrs=(RANGE,), precisions=(10,), n_scans=n_scans,
                        dropout=0.08, speed_mps=10.0, seed=seed)


def config_multi_attr(seed=0, n_scans=100, H=128, W=2048):
    """100 scans of 128 x 2048: dual range (10 mm), signal, reflectivity,
    ambient; 12 % zeros in range."""
    return SensorConfig(H=H, W=W, attrs=(RANGE, RANGE2, SIGNAL, REFLECTIVITY, AMBIENT),
                        precisions=(10, 10, 1, 1, 1), n_scans=n_scans, dropout=0.0,
                        target_zero_frac=0.12, speed_mps=10.0, wall=True, seed=seed)


def config_low_coherence(seed=0, n_scans=200, H=128, W=2048):
    """128 x 2048 range (1 mm) + reflectivity, 40 % zeros in discs, random yaw
    (+-30 deg/s) and 3 m/s translation in a random direction."""
    return SensorConfig(H=H, W=W, attrs=(RANGE, REFLECTIVITY), precisions=(1, 1),
                        n_scans=n_scans, dropout=0.0, disc_zero_frac=0.40, speed_mps=3.0,
                        random_motion=True, yaw_rate_dps=30.0, wall=True, seed=seed)


# attribute sets and shapes of the many-stream workloads
BATCH_SHAPES = ((16, 1024), (32, 1024), (64, 1024), (64, 2048), (128, 2048), (128, 4096))
BATCH_ATTR_SETS = ((RANGE,), (RANGE, SIGNAL), (RANGE, RANGE2, SIGNAL, REFLECTIVITY, AMBIENT))


def batch_stream_config(stream: int, base_seed: int = 1000, n_scans: int = 8):
    """Stream `stream` of the many-stream workload: shape and attribute set
    drawn uniformly from the sets above with seed base_seed + stream."""
    rng = np.random.default_rng(base_seed + stream)
    H, W = BATCH_SHAPES[rng.integers(len(BATCH_SHAPES))]
    attrs = BATCH_ATTR_SETS[rng.integers(len(BATCH_ATTR_SETS))]
    prec = tuple(10 if a in (RANGE, RANGE2) else 1 for a in attrs)
    return SensorConfig(H=H, W=W, attrs=attrs, precisions=prec, n_scans=n_scans, dropout=0.0,
                        target_zero_frac=0.12, speed_mps=10.0, wall=True, seed=base_seed + stream)


class ScanSequence:
    """Generates the scans of one sensor stream, one scan at a time.

    scan(t) returns a list of planes (one per attribute, H x W, dtypes
    uint32 / uint16 / uint8 as numpy arrays on CPU, or torch tensors on the
    requested device with the same bytes: torch has no uint16/uint32 for all
    ops, so the device tensors are int16 / int32 views of the same bits).
    """

    def __init__(self, cfg: SensorConfig, device: str = "cpu"):
        self.cfg = cfg
        self.device = torch.device(device)
        rng = np.random.default_rng(cfg.seed)
        self._rng = rng
        nb = 40
        self.box_size = rng.uniform(1.0, 10.0, size=(nb, 3)).astype(np.float32)
        rad = 80.0 * np.sqrt(rng.uniform(0.0, 1.0, size=nb))
        ang = rng.uniform(0.0, 2 * math.pi, size=nb)
        cx, cy = rad * np.cos(ang), rad * np.sin(ang)
        # keep a clear lane around the driving line so the sensor is not inside a box
        lane = 3.0 + self.box_size[:, 1] / 2
        cy = np.where(np.abs(cy) < lane, np.sign(cy + 1e-9) * lane, cy)
        self.box_c = np.stack([cx, cy], axis=1).astype(np.float32)
        self.box_refl = rng.integers(20, 250, size=nb).astype(np.float32)
        self.ground_refl = 40.0
        self.wall_refl = 90.0
        # ambient field: a few low-frequency sinusoids over (row, column)
        self.amb_k = rng.uniform(0.5, 3.0, size=(4, 2)).astype(np.float32)
        self.amb_phase = rng.uniform(0, 2 * math.pi, size=4).astype(np.float32)
        self.amb_amp = rng.uniform(100.0, 400.0, size=4).astype(np.float32)
        # ego trajectory
        T = cfg.n_scans
        pos = np.zeros((T, 2), dtype=np.float64)
        yaw = np.zeros(T, dtype=np.float64)
        dt = 1.0 / cfg.rate_hz
        for t in range(1, T):
            if cfg.random_motion:
                d = rng.uniform(0, 2 * math.pi)
                pos[t] = pos[t - 1] + cfg.speed_mps * dt * np.array([math.cos(d), math.sin(d)])
                yaw[t] = yaw[t - 1] + math.radians(rng.uniform(-cfg.yaw_rate_dps, cfg.yaw_rate_dps)) * dt
            else:
                pos[t] = pos[t - 1] + np.array([cfg.speed_mps * dt, 0.0])
                yaw[t] = yaw[t - 1]
        self.pos, self.yaw = pos, yaw
        self.scan_seeds = rng.integers(0, 2**31 - 1, size=T)
        H, W = cfg.H, cfg.W
        el = np.radians(np.linspace(22.5, -22.5, H)) if H > 1 else np.zeros(1)
        self._el = torch.tensor(el, dtype=torch.float32, device=self.device)
        self._az0 = torch.arange(W, dtype=torch.float32, device=self.device) * (2 * math.pi / W)
        # pixels that return nothing in every scan (persistent dropouts): a fixed
        # uniform draw per stream, thresholded by the scan's dropout rate
        self._persist_u = None
        if cfg.persistent_dropout > 0:
            gp = torch.Generator(device="cpu").manual_seed(int(cfg.seed) * 7919 + 17)
            self._persist_u = torch.rand((H, W), generator=gp)

    # -- geometry -----------------------------------------------------------
    def _cast(self, t: int):
        """First and second hit distance along every ray and the reflectivity
        of the first hit. Boxes are intersected a group at a time (slab test
        on a box x H x W grid); the nearest and second nearest of ground,
        boxes and wall are kept as running minima, ties going to the earlier
        surface (ground, then boxes in order, then wall)."""
        cfg = self.cfg
        dev = self.device
        ox, oy = float(self.pos[t, 0]), float(self.pos[t, 1])
        az = self._az0 + float(self.yaw[t])
        ce = torch.cos(self._el)[:, None]
        dx = ce * torch.cos(az)[None, :]
        dy = ce * torch.sin(az)[None, :]
        dz = torch.sin(self._el)[:, None].expand_as(dx)
        big = torch.tensor(float("inf"), device=dev)
        # ground plane z = -1.8
        tg = torch.where(dz < -1e-6, -1.8 / torch.where(dz < -1e-6, dz, -torch.ones_like(dz)), big)
        # boxes, recycled modulo a 160 m window around the sensor
        inv = [1.0 / torch.where(d.abs() < 1e-9, torch.full_like(d, 1e-9), d) for d in (dx, dy, dz)]
        # box bounds relative to the sensor, in float32 like the box tables
        c, sz = self.box_c, self.box_size
        cx = ox + ((c[:, 0] - ox + 80.0) % 160.0) - 80.0
        cy = oy + ((c[:, 1] - oy + 80.0) % 160.0) - 80.0
        lo = np.stack([cx - sz[:, 0] / 2 - ox, cy - sz[:, 1] / 2 - oy, np.full(len(cx), -1.8, np.float32)], 1)
        hi = np.stack([cx + sz[:, 0] / 2 - ox, cy + sz[:, 1] / 2 - oy, -1.8 + sz[:, 2]], 1)
        lo = torch.tensor(lo, dtype=torch.float32, device=dev)[:, :, None, None]
        hi = torch.tensor(hi, dtype=torch.float32, device=dev)[:, :, None, None]
        refl_tab = torch.tensor([self.ground_refl] + [float(r) for r in self.box_refl] + [self.wall_refl],
                                dtype=torch.float32, device=dev)
        best, second, first = tg, torch.full_like(tg, float("inf")), torch.zeros(tg.shape, dtype=torch.int64,
                                                                                 device=dev)
        nb = lo.shape[0]
        step = nb if dev.type == "cuda" else 40  # boxes per slab test (CPU: cache-sized groups)

        def merge(hits, base):
            # fold a group of surfaces (in order) into the running nearest and
            # second nearest; a tie keeps the earlier surface as the nearest
            nonlocal best, second, first
            gb, gi = hits.min(0)
            if hits.shape[0] > 1:
                idx = torch.arange(hits.shape[0], device=dev)[:, None, None]
                gs = torch.where(idx == gi[None], big, hits).min(0).values
            else:
                gs = torch.full_like(gb, float("inf"))
            closer = gb < best
            second = torch.where(closer, torch.minimum(best, gs), torch.minimum(second, gb))
            first = torch.where(closer, gi + base, first)
            best = torch.where(closer, gb, best)

        for k0 in range(0, nb, step):
            tmin = tmax = None
            for ax in range(3):
                t1 = lo[k0:k0 + step, ax] * inv[ax]
                t2 = hi[k0:k0 + step, ax] * inv[ax]
                a, b = torch.minimum(t1, t2), torch.maximum(t1, t2)
                tmin = a if tmin is None else torch.maximum(tmin, a)
                tmax = b if tmax is None else torch.minimum(tmax, b)
            merge(torch.where((tmax >= tmin) & (tmin > 0), tmin, big), 1 + k0)
        if cfg.wall:  # enclosing wall of radius 110 m, 60 m tall
            ch = torch.sqrt(dx * dx + dy * dy).clamp_min(1e-6)
            tw = 110.0 / ch
            merge(torch.where(dz * tw < 60.0, tw, big)[None], 1 + nb)
        refl = refl_tab[first]
        return best, second, refl

    # -- attributes ----------------------------------------------------------
    def scan(self, t: int, as_numpy: bool = True):
        cfg = self.cfg
        dev = self.device
        H, W = cfg.H, cfg.W
        g = torch.Generator(device="cpu").manual_seed(int(self.scan_seeds[t]))
        best, second, refl = self._cast(t)
        valid = best <= MAX_RANGE_M
        # dropouts
        drop = torch.zeros((H, W), dtype=torch.bool)
        p = cfg.dropout
        if cfg.target_zero_frac is not None:
            f0 = 1.0 - float(valid.float().mean())
            p = max(0.0, (cfg.target_zero_frac - f0) / max(1e-9, 1.0 - f0))
        if p > 0 and self._persist_u is not None:
            drop |= self._persist_u < p * cfg.persistent_dropout
            drop |= torch.rand((H, W), generator=g) < p * (1.0 - cfg.persistent_dropout)
        elif p > 0:
            drop |= torch.rand((H, W), generator=g) < p
        if cfg.disc_zero_frac > 0:
            drop |= self._discs(g, cfg.disc_zero_frac)
        valid = valid & ~drop.to(dev)
        r_m = best
        if cfg.range_noise_mm > 0:
            r_m = best + torch.randn((H, W), generator=g).to(dev) * (cfg.range_noise_mm / 1000.0)
        r_mm = torch.where(valid, torch.round(r_m * 1000.0).clamp_min(1.0), torch.zeros_like(best))
        out = []
        for a in cfg.attrs:
            if a == RANGE:
                v = r_mm
            elif a == RANGE2:
                # second return at depth discontinuities (object edges)
                rr = torch.where(best <= MAX_RANGE_M, best, torch.full_like(best, 1e9))
                # depth discontinuities: a jump of more than 0.5 m to a horizontal
                # neighbour or 2.5 m to a vertical one (about 5 % of pixels)
                edge = torch.zeros_like(valid)
                edge[:, 1:] |= (rr[:, :-1] - rr[:, 1:]).abs() > 0.5
                edge[:, :-1] |= (rr[:, 1:] - rr[:, :-1]).abs() > 0.5
                edge[1:, :] |= (rr[:-1, :] - rr[1:, :]).abs() > 2.5
                edge[:-1, :] |= (rr[1:, :] - rr[:-1, :]).abs() > 2.5
                ok = valid & edge & (second <= MAX_RANGE_M)
                v = torch.where(ok, torch.round(second * 1000.0), torch.zeros_like(second))
            elif a == SIGNAL:
                lam = 1000.0 * refl / best.clamp_min(1.0) ** 2
                noise = torch.poisson(lam.clamp(0, 60000).cpu(), generator=g).to(dev)
                v = torch.where(valid, noise.clamp(1, 65535), torch.zeros_like(noise))
            elif a == REFLECTIVITY:
                jit = torch.randint(-3, 4, (H, W), generator=g).to(dev).float()
                v = torch.where(valid, (refl + jit).clamp(1, 255), torch.zeros_like(refl))
            elif a == AMBIENT:
                rows = torch.arange(H, device=dev, dtype=torch.float32)[:, None] / max(H, 1)
                cols = torch.arange(W, device=dev, dtype=torch.float32)[None, :] / max(W, 1)
                f = torch.full((H, W), 1500.0, device=dev)
                for k in range(4):
                    f = f + float(self.amb_amp[k]) * torch.sin(
                        2 * math.pi * (float(self.amb_k[k, 0]) * rows + float(self.amb_k[k, 1]) * cols)
                        + float(self.amb_phase[k]) + 0.05 * t)
                n = torch.randn((H, W), generator=g).to(dev) * 20.0
                v = (f + n).round().clamp(1, 65535)
            else:
                raise ValueError(a)
            s = ATTR_DTYPE[a]
            v = v.to(torch.int64)
            if as_numpy:
                out.append(v.cpu().numpy().astype(_NP_DT[s]))
            else:
                # same bits in a signed container of the same width
                if s == 4:
                    v = torch.where(v >= 2**31, v - 2**32, v)
                elif s == 2:
                    v = torch.where(v >= 2**15, v - 2**16, v)
                out.append(v.to(_TORCH_DT[s]).contiguous())
        return out

    def _discs(self, g: torch.Generator, frac: float):
        """Clustered dropouts: random discs (radius 5..40 px, centres uniform
        over the image) are added until they cover at least `frac` of the
        pixels. Each disc only touches its bounding window."""
        H, W = self.cfg.H, self.cfg.W
        m = np.zeros((H, W), dtype=bool)
        covered, need = 0, frac * (H * W)
        for _ in range(100000):
            if covered >= need:
                break
            cy = float(torch.randint(0, H, (1,), generator=g))
            cx = float(torch.randint(0, W, (1,), generator=g))
            rad = 5.0 + 35.0 * float(torch.rand(1, generator=g))
            r0, r1 = max(0, int(math.floor(cy - rad))), min(H, int(math.ceil(cy + rad)) + 1)
            c0, c1 = max(0, int(math.floor(cx - rad))), min(W, int(math.ceil(cx + rad)) + 1)
            rows = np.arange(r0, r1, dtype=np.float32)[:, None]
            cols = np.arange(c0, c1, dtype=np.float32)[None, :]
            disc = (rows - np.float32(cy)) ** 2 + (cols - np.float32(cx)) ** 2 <= np.float32(rad * rad)
            win = m[r0:r1, c0:c1]
            covered += int(np.count_nonzero(disc & ~win))
            win |= disc
        return torch.from_numpy(m)

    def scans(self, as_numpy: bool = True):
        return [self.scan(t, as_numpy) for t in range(self.cfg.n_scans)]


def attr_descs(cfg: SensorConfig):
    """[(bytes per sample, precision)] of a configuration's attributes."""
    return [(ATTR_DTYPE[a], int(p)) for a, p in zip(cfg.attrs, cfg.precisions)]
