"""Pins for the standardization oracle (Sec. III-A: Cartesian points ->
spherical coordinates -> rows by altitude, columns by azimuth -> quantized
unsigned samples, 0 = no valid measurement). Each test checks it against
something other than itself: Python's exact integer square root, the
library arctangent within the CORDIC error bound (6e-8 rad), scans built pixel by pixel
from known angles, and the stated rules for collisions, range limits, the
field of view and attribute rounding."""
import math

import numpy as np
import pytest

import oracle

TURN = oracle.ANGLE_UNITS


def angle_err(binary, rad):
    d = (binary / TURN * 2 * math.pi - rad) % (2 * math.pi)
    return min(d, 2 * math.pi - d)


def test_isqrt_is_exact():
    rng = np.random.default_rng(1)
    vals = [0, 1, 2, 3, 4, 15, 16, 17, (1 << 64) - 1, 1 << 64, (1 << 126) - 1]
    for _ in range(2000):
        v = int(rng.integers(0, 1 << 62)) * int(rng.integers(1, 1 << 62)) + int(rng.integers(0, 1 << 60))
        vals.append(v % (1 << 126))
        r = math.isqrt(vals[-1])
        vals += [r * r, r * r - 1 if r else 0, (r + 1) * (r + 1) - 1]
    for v in vals:
        if v < (1 << 126):
            assert oracle.isqrt(v) == math.isqrt(v), v


def test_cordic_angles_within_bound_of_atan2():
    # 30 CORDIC steps in 32-bit integers on vectors normalised to 29 bits:
    # residual angle after the last step, table rounding and shift truncation
    # stay below 6e-8 rad (a 2048-column pixel is 3.1e-3 rad wide)
    rng = np.random.default_rng(2)
    cases = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, -1), (2**31 - 1, 1), (1, -(2**31 - 1))]
    for _ in range(3000):
        mag = 1 << int(rng.integers(0, 31))
        cases.append((int(rng.integers(-mag, mag + 1)), int(rng.integers(-mag, mag + 1))))
    for X, Y in cases:
        if X == 0 and Y == 0:
            continue
        assert angle_err(oracle.azimuth(X, Y), math.atan2(Y, X)) < 6e-8, (X, Y)
    for _ in range(3000):
        mag = 1 << int(rng.integers(1, 31))
        X, Y, Z = (int(rng.integers(-mag, mag + 1)) for _ in range(3))
        if X == 0 and Y == 0 and Z == 0:
            continue
        e = oracle.elevation(X, Y, Z)
        assert abs(e / TURN * 2 * math.pi - math.atan2(Z, math.hypot(X, Y))) < 6e-8, (X, Y, Z)
    assert oracle.azimuth(0, 0) == 0 and oracle.elevation(0, 0, 0) == 0


def sensor(H, lo=-22.5, hi=22.5):
    return np.radians(np.linspace(hi, lo, H))


def points_at(rows, cols, ranges_m, alt, W, az0=0.0):
    """Points in the middle of the given pixels at the given ranges."""
    el = alt[rows]
    az = az0 + (np.asarray(cols) + 0.5) * 2 * math.pi / W
    r = np.asarray(ranges_m, dtype=np.float64)
    xyz = np.stack([r * np.cos(el) * np.cos(az), r * np.cos(el) * np.sin(az), r * np.sin(el)], axis=1)
    return xyz.astype(np.float32)


def test_points_built_at_pixel_centres_land_in_their_pixels():
    rng = np.random.default_rng(3)
    H, W = 16, 512
    alt = sensor(H)
    rows = np.repeat(np.arange(H), W)
    cols = np.tile(np.arange(W), H)
    r_m = rng.uniform(1.0, 100.0, H * W)
    keep = rng.random(H * W) < 0.8
    xyz = points_at(rows[keep], cols[keep], r_m[keep], alt, W)
    perm = rng.permutation(len(xyz))  # input order does not matter
    img, _ = oracle.standardize(xyz[perm], H, W, alt)
    want = np.zeros((H, W), np.int64)
    want[rows[keep], cols[keep]] = np.round(r_m[keep] * 1000)
    got = img.astype(np.int64)
    assert np.array_equal(got == 0, want == 0)
    assert np.abs(got - want).max() <= 1  # float32 coordinates round to the nearest mm
    # the exact value: nearest integer to the norm of the rounded coordinates
    X = np.rint(xyz[perm].astype(np.float32) * np.float32(1000)).astype(np.int64)
    n = (X * X).sum(axis=1)
    r = np.array([math.isqrt(int(v)) for v in n])
    R = r + ((n - r * r) > r)
    pr, pc = rows[keep][perm], cols[keep][perm]
    assert np.array_equal(got[pr, pc], R)


def test_nearest_point_wins_then_lowest_index():
    H, W = 4, 64
    alt = sensor(H)
    xyz = points_at([1, 1, 1, 2, 2], [5, 5, 5, 9, 9], [30.0, 20.0, 25.0, 10.0, 10.0], alt, W)
    vals = np.array([1, 2, 3, 4, 5], np.float32)
    img, (a,) = oracle.standardize(xyz, H, W, alt, attrs=[(vals, 1, 1.0)])
    assert img[1, 5] == 20000 and a[1, 5] == 2
    assert img[2, 9] == 10000 and a[2, 9] == 4  # equal ranges: the earlier point
    assert np.count_nonzero(img) == 2 and np.count_nonzero(a) == 2


def test_range_limits_and_field_of_view_drop_points():
    H, W = 8, 128
    alt = sensor(H, -10.0, 10.0)
    step = math.radians(20.0 / 7)
    xyz = points_at([0, 1, 2, 3], [0, 1, 2, 3], [0.5, 50.0, 150.0, 20.0], alt, W)
    img, _ = oracle.standardize(xyz, H, W, alt, min_range=1000, max_range=100000)
    assert [int(img[i, i]) for i in range(4)] == [0, 50000, 0, 20000]
    # just inside / outside the top row's half spacing above the first beam
    el_in, el_out = alt[0] + 0.49 * step, alt[0] + 0.51 * step
    az = 0.5 * 2 * math.pi / W  # middle of column 0
    pts = np.array([[10 * math.cos(e) * math.cos(az), 10 * math.cos(e) * math.sin(az), 10 * math.sin(e)]
                    for e in (el_in, el_out)], np.float32)
    img, _ = oracle.standardize(pts, H, W, alt)
    assert np.count_nonzero(img) == 1 and img[0, 0] == 10000
    # 16-bit range images drop ranges that do not fit
    img, _ = oracle.standardize(points_at([4, 5], [7, 8], [60.0, 70.0], alt, W), H, W, alt, range_bytes=2)
    assert img.dtype == np.uint16 and img[4, 7] == 60000 and img[5, 8] == 0


def test_azimuth_origin_and_direction():
    H, W = 2, 360
    alt = sensor(H, -1.0, 1.0)
    xyz = points_at([0, 0, 1], [10, 100, 359], [5.0, 6.0, 7.0], alt, W)
    base, _ = oracle.standardize(xyz, H, W, alt)
    # az0 three columns further: every column index drops by 3 (cyclically)
    shifted, _ = oracle.standardize(xyz, H, W, alt, az0=3 * 2 * math.pi / W)
    assert np.array_equal(shifted, np.roll(base, -3, axis=1))
    # a clockwise sensor sees column c where a counterclockwise one sees W-1-c
    cw, _ = oracle.standardize(xyz, H, W, alt, clockwise=True)
    assert np.array_equal(cw, base[:, ::-1])


def test_attribute_quantization_rounds_half_even_and_clamps():
    q = oracle.quantize_attr
    assert [q(v, 1.0, 1) for v in (0.5, 1.5, 2.5, 2.4999, 254.5, 255.5, 300.0, -3.0, float("nan"))] == \
        [0, 2, 2, 2, 254, 255, 255, 0, 0]
    assert q(1.25, 4.0, 2) == 5 and q(1e9, 1.0, 2) == 65535 and q(1e12, 1.0, 4) == 0xFFFFFFFF


def test_no_points_and_invalid_coordinates():
    H, W = 3, 40
    alt = sensor(H)
    img, (a,) = oracle.standardize(np.zeros((0, 3), np.float32), H, W, alt, attrs=[(np.zeros(0, np.float32), 2, 1.0)])
    assert not img.any() and not a.any()
    bad = np.array([[np.nan, 1, 1], [3e6, 0, 0], [np.inf, 0, 0], [0, 0, 0]], np.float32)
    img, _ = oracle.standardize(bad, H, W, alt)
    assert not img.any()
    with pytest.raises(ValueError):  # beams must be strictly decreasing
        oracle.standardize(bad, H, W, alt[::-1])
    with pytest.raises(ValueError):  # and within +-90 degrees
        oracle.standardize(bad, H, W, np.array([1.7, 0.0, -0.1]))
