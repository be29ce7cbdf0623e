"""GPU parity of input standardization (Sec. III-A): the CUDA kernels
(through the C ABI) against the standardization oracle, element by element.
Every decision is integer arithmetic on both sides, so the bar is exact:
identical range and attribute images, including collisions, points on pixel
boundaries, out-of-range and invalid points, every sample size, clockwise
sensors, an azimuth origin, ragged and maximal shapes and an empty scan."""
import math

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
NP = {1: np.uint8, 2: np.uint16, 4: np.uint32}
TD = {1: torch.uint8, 2: torch.int16, 4: torch.int32}


def beams(H, lo=-22.5, hi=22.5):
    return np.radians(np.linspace(hi, lo, H))


def run_gpu(h, xyz, attrs, H, W, range_bytes):
    x = torch.from_numpy(np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)).cuda()
    r = torch.full((H, W), 7, dtype=TD[range_bytes], device="cuda")  # overwritten everywhere
    outs = []
    args = []
    for v, b, s in attrs:
        o = torch.full((H, W), 5, dtype=TD[b], device="cuda")
        outs.append(o)
        args.append((torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda(), o, s))
    J.jiffy_standardize(h, x, r, args)
    torch.cuda.synchronize()
    return (r.cpu().numpy().view(NP[range_bytes]), [o.cpu().numpy().view(NP[b]) for o, (_, b, _) in zip(outs, attrs)])


def check(xyz, H, W, alt, attrs=(), **kw):
    h = J.jiffy_standardizer_create(H, W, alt, **kw)
    rb = kw.get("range_bytes", 4)
    got_r, got_a = run_gpu(h, xyz, attrs, H, W, rb)
    okw = {("az0" if k == "azimuth0" else k): v for k, v in kw.items()}
    want_r, want_a = oracle.standardize(xyz, H, W, alt, attrs=attrs, **okw)
    assert np.array_equal(got_r, want_r), "range image differs at %d pixels" % int((got_r != want_r).sum())
    for a, (g, w) in enumerate(zip(got_a, want_a)):
        assert np.array_equal(g, w), "attribute %d differs" % a
    return h, want_r


def cloud(rng, n, spread=60.0):
    xyz = rng.normal(0.0, spread, size=(n, 3)).astype(np.float32)
    xyz[:, 2] *= 0.2
    return xyz


def test_random_clouds_with_collisions_and_invalid_points():
    rng = np.random.default_rng(1)
    H, W = 24, 100  # W off every power of two
    alt = beams(H)
    xyz = cloud(rng, 50_003)
    xyz = np.concatenate([xyz, xyz[:500]])  # exact duplicates: the first index wins
    xyz[rng.integers(0, len(xyz), 50)] = np.nan
    xyz[rng.integers(0, len(xyz), 50), 0] = 5e6  # out of the coordinate range
    xyz[rng.integers(0, len(xyz), 50)] = 0.0
    attrs = [(rng.normal(100, 80, len(xyz)).astype(np.float32), 1, 1.0),
             (rng.uniform(-5, 70000, len(xyz)).astype(np.float32), 2, 1.0),
             (rng.uniform(0, 1e5, len(xyz)).astype(np.float32), 4, 37.5)]
    check(xyz, H, W, alt, attrs, min_range=500, max_range=150000)


@pytest.mark.parametrize("range_bytes", [2, 4])
@pytest.mark.parametrize("clockwise", [False, True])
def test_sensor_options(range_bytes, clockwise):
    rng = np.random.default_rng(2 + range_bytes + clockwise)
    H, W = 32, 1024
    check(cloud(rng, 40_000, 30.0), H, W, beams(H, -16.6, 16.6), range_bytes=range_bytes, clockwise=clockwise,
          azimuth0=1.234, units_per_m=500.0)


def test_points_on_pixel_boundaries():
    # azimuths exactly on column edges and elevations exactly on the midpoints
    # between beams: the integer arithmetic decides identically on both sides
    H, W = 16, 360
    alt = beams(H, -15.0, 15.0)
    pts = []
    for b in range(H + 1):
        e = alt[0] + 0.5 * (alt[0] - alt[1]) if b == 0 else (
            alt[-1] - 0.5 * (alt[-2] - alt[-1]) if b == H else 0.5 * (alt[b - 1] + alt[b]))
        for c in range(0, W, 7):
            a = c * 2 * math.pi / W
            for r in (3.0, 17.25, 99.999):
                pts.append([r * math.cos(e) * math.cos(a), r * math.cos(e) * math.sin(a), r * math.sin(e)])
    xyz = np.array(pts, np.float32)
    check(xyz, H, W, alt)
    check(xyz, H, W, alt, clockwise=True, azimuth0=-0.5 * 2 * math.pi / W)


def test_synthetic_scan_round_trip_and_parity():
    # a scan of the multi-attribute workload turned into points (float32
    # metres at the pixel centres' directions), standardized back
    cfg = synth.config_multi_attr(n_scans=1, H=128, W=2048)
    seq = synth.ScanSequence(cfg)
    r_mm, _, signal = seq.scan(0)[:3]
    H, W = cfg.H, cfg.W
    alt = np.radians(np.linspace(22.5, -22.5, H))
    rows, cols = np.nonzero(r_mm)
    r = r_mm[rows, cols].astype(np.float64) / 1000.0
    az = (cols + 0.5) * 2 * math.pi / W
    el = alt[rows]
    xyz = np.stack([r * np.cos(el) * np.cos(az), r * np.cos(el) * np.sin(az), r * np.sin(el)], 1).astype(np.float32)
    perm = np.random.default_rng(3).permutation(len(xyz))
    xyz = xyz[perm]
    sig = signal[rows, cols].astype(np.float32)[perm]
    _, want = check(xyz, H, W, alt, [(sig, 2, 1.0)])
    # the image comes back: same valid pixels, ranges within the float32 rounding
    assert np.array_equal(want > 0, r_mm > 0)
    assert np.abs(want.astype(np.int64) - r_mm.astype(np.int64)).max() <= 1


def test_repeated_calls_reuse_the_pixel_table_and_empty_scans():
    rng = np.random.default_rng(4)
    H, W = 8, 256
    alt = beams(H)
    h = J.jiffy_standardizer_create(H, W, alt)
    for n in (20_000, 0, 777, 20_000):
        xyz = cloud(rng, n, 20.0)
        got, _ = run_gpu(h, xyz, (), H, W, 4)
        want, _ = oracle.standardize(xyz, H, W, alt)
        assert np.array_equal(got, want), n
        if n == 0:
            assert not got.any()


def test_many_scans_in_one_call():
    # uneven point counts (one scan empty), attributes, and a second call with
    # more scans than the first (the pixel table grows)
    rng = np.random.default_rng(6)
    H, W = 16, 700
    alt = beams(H)
    h = J.jiffy_standardizer_create(H, W, alt, range_bytes=2, max_range=65000)
    for counts in ([3000, 0, 12345, 1, 999], [5000] * 3 + [0] * 2 + [7777] * 6):
        clouds = [cloud(rng, c, 25.0) for c in counts]
        vals = [rng.uniform(0, 400, c).astype(np.float32) for c in counts]
        offs = np.concatenate([[0], np.cumsum(counts)]).tolist()
        T = len(counts)
        xyz = torch.from_numpy(np.concatenate(clouds).reshape(-1, 3)).cuda()
        v = torch.from_numpy(np.concatenate(vals)).cuda()
        r = torch.full((T, H, W), 3, dtype=torch.int16, device="cuda")
        o = torch.full((T, H, W), 3, dtype=torch.uint8, device="cuda")
        J.jiffy_standardize_seq(h, xyz, offs, r, [(v, o, 0.5)])
        torch.cuda.synchronize()
        r, o = r.cpu().numpy().view(np.uint16), o.cpu().numpy()
        for t in range(T):
            wr, (wa,) = oracle.standardize(clouds[t], H, W, alt, range_bytes=2, max_range=65000,
                                           attrs=[(vals[t], 1, 0.5)])
            assert np.array_equal(r[t], wr), (counts, t)
            assert np.array_equal(o[t], wa), (counts, t)


@pytest.mark.parametrize("H,W", [(64, 16384), (4096, 64)])
def test_largest_shapes(H, W):
    # the widest rows, and the most beams (4096 rows: the row search over
    # 4095 midpoints spaced 1.1e-4 rad apart)
    rng = np.random.default_rng(5 + H)
    xyz = cloud(rng, 1_500_000, 40.0)
    check(xyz, H, W, beams(H), [(rng.uniform(0, 300, len(xyz)).astype(np.float32), 1, 1.0)])


def test_invalid_sensors_are_rejected():
    with pytest.raises(J.JiffyError):
        J.jiffy_standardizer_create(4, 16, beams(4)[::-1])  # increasing beams
    with pytest.raises(J.JiffyError):
        J.jiffy_standardizer_create(4, 16, beams(4), range_bytes=1)
    with pytest.raises(J.JiffyError):
        J.jiffy_standardizer_create(4, 16, beams(4), units_per_m=0.0)
    with pytest.raises(J.JiffyError):  # beyond +-90 degrees
        J.jiffy_standardizer_create(3, 16, [1.7, 0.0, -0.1])
