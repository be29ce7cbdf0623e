"""Pins for the oracle: each test checks it against something other than
itself -- the paper's Eq. 1 values, the quantization error bound (Sec. III-B,
Fig. 4), hand-worked byte streams (tests/golden), closed forms for special
scans, exhaustive searches and round trips (Sec. III-C: decoding reverses
encoding exactly)."""
import numpy as np
import pytest

import oracle
from tests import golden_io

DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def quantize_plane(v, P, s):
    return np.array([oracle.quantize(int(x), P, s) for x in v.ravel()], dtype=np.uint64).reshape(v.shape)


# ---------------------------------------------------------------- golden
@pytest.mark.parametrize("name", golden_io.names())
def test_golden_stream(name):
    H, W, attrs, frames = golden_io.load(name)
    opt = golden_io.options(name)
    enc = oracle.Codec(H, W, attrs, 4, opt["force_mode"], opt["stages"])
    dec = oracle.Codec(H, W, attrs, stages=opt["stages"])
    for f in frames:
        b, modes = enc.encode(f["in"], return_modes=True)
        assert modes == f["mode"]
        assert b == f["bytes"], (b.hex(" "), f["bytes"].hex(" "))
        planes, n = dec.decode(b)
        assert n == len(b)
        for p, o in zip(planes, f["out"]):
            assert np.array_equal(p, o)


# ---------------------------------------------------------------- Eq. 1
def test_zigzag_eq1_values():
    # Eq. 1: ZigZag(x) = 2|x| + 1 if x < 0, 2|x| otherwise
    assert [oracle.zigzag(x) for x in (0, 1, -1, 2, -2, 3, -3)] == [0, 2, 3, 4, 5, 6, 7]
    assert oracle.zigzag(1000) == 2000 and oracle.zigzag(-1000) == 2001


def test_zigzag_is_a_bijection_mod_2_32():
    xs = list(range(-70000, 70001)) + [2**31 - 1, -(2**31 - 1), -(2**31), 2**30, -(2**30)]
    zs = [oracle.zigzag(x) for x in xs]
    assert len(set(zs)) == len(zs)
    assert all(oracle.unzigzag(z) == x for x, z in zip(xs, zs))
    # the top of the range wraps modulo 2^32
    assert oracle.zigzag(-(2**31)) == 1
    assert oracle.zigzag(2**31 - 1) == 2**32 - 2
    assert oracle.zigzag(-(2**31 - 1)) == 2**32 - 1
    rng = np.random.default_rng(1)
    for z in rng.integers(0, 2**32, size=20000, dtype=np.uint64):
        assert oracle.zigzag(oracle.unzigzag(int(z))) == int(z)


# ---------------------------------------------------------------- quantizer
def test_quantize_is_nearest_multiple_ties_up():
    rng = np.random.default_rng(2)
    for _ in range(20000):
        s = int(rng.choice([1, 2, 4]))
        vmax = (1 << (8 * s)) - 1
        P = int(rng.choice([1, 2, 3, 5, 10, 16, 100, 1000, 12345]))
        v = int(rng.integers(0, vmax + 1))
        q = oracle.quantize(v, P, s)
        if P == 1:
            assert q == v
        assert q * P <= vmax
        cands = [c for c in range(max(0, v // P - 1), v // P + 3) if c * P <= vmax]
        best = min(cands, key=lambda c: (abs(v - c * P), -c))  # nearest, ties to the larger
        assert q == best, (v, P, s, q, best)
        if (v + P // 2) // P <= vmax // P:  # not clamped: the Fig. 4 bound
            assert abs(v - q * P) * 2 <= P


# ---------------------------------------------------------------- PFOR blocks
def test_block_cost_equals_packed_length_and_best_b_is_exhaustive_min():
    rng = np.random.default_rng(3)
    for it in range(600):
        n = int(rng.integers(1, 129))
        kind = it % 4
        if kind == 0:
            z = rng.integers(0, 2 ** int(rng.integers(0, 33)), size=n, dtype=np.uint64)
        elif kind == 1:  # mostly small with a few outliers
            z = rng.integers(0, 16, size=n, dtype=np.uint64)
            k = int(rng.integers(0, 6))
            z[rng.integers(0, n, size=k)] = rng.integers(0, 2**32, size=k, dtype=np.uint64)
        elif kind == 2:
            z = np.zeros(n, dtype=np.uint64)
        else:
            z = rng.integers(0, 2**32, size=n, dtype=np.uint64)
        z = z.astype(np.uint32)
        wmax = max(int(x).bit_length() for x in z)
        sizes = []
        for b in range(0, wmax + 1):
            packed = oracle.pack_block(z, b)
            assert oracle.block_body_bytes(z, b) == len(packed) - 4
            assert packed[0] == b and packed[3] == 0
            sizes.append(len(packed) - 4)
        b_star = oracle.best_b(z)
        assert b_star == int(np.argmin(sizes))  # argmin returns the first (smallest b) minimum


def test_pack_block_bit_layout_by_hand():
    # b = 4, values 1..8 -> nibbles LSB first: 0x87654321
    z = np.arange(1, 9, dtype=np.uint32)
    assert oracle.pack_block(z, 4) == bytes([4, 0, 0, 0, 0x21, 0x43, 0x65, 0x87])
    # b = 0 with all zeros: empty body
    assert oracle.pack_block(np.zeros(128, np.uint32), 0) == bytes([0, 0, 0, 0])


# ---------------------------------------------------------------- trial == brute force
def random_scan(rng, H, W, s, zero_frac, scale):
    v = rng.integers(1, scale, size=(H, W), dtype=np.uint64)
    v[rng.random((H, W)) < zero_frac] = 0
    return v.astype(DT[s])


@pytest.mark.parametrize("H", [1, 2, 3, 4])
def test_trial_equals_bruteforce_when_all_rows_are_test_rows(H):
    # Sec. III-E: the trial codes a few scanlines without the mask; with H <= 4
    # test lines it codes every line, so it must equal coding the whole scan
    # both ways and keeping the smaller data part (brute force, mask excluded).
    rng = np.random.default_rng(10 + H)
    for it in range(40):
        W = int(rng.choice([1, 7, 31, 32, 33, 100, 128, 129, 300]))
        s = int(rng.choice([1, 2, 4]))
        P = int(rng.choice([1, 3, 10]))
        scale = {1: 256, 2: 65536, 4: 200000}[s]
        prev = random_scan(rng, H, W, s, 0.2, scale)
        cur = prev.copy()
        noise = rng.integers(-3, 4, size=cur.shape)
        cur = np.clip(cur.astype(np.int64) + noise * (it % 3), 0, scale - 1).astype(DT[s])
        cur[rng.random((H, W)) < 0.1] = 0
        data = {}
        for mode in (0, 1):
            trial = oracle.trial_cost(cur, prev, P, mode)
            _, mask_b, data_b = oracle.section_split(cur, prev, P, mode)
            assert trial == data_b
            data[mode] = data_b
        c = oracle.Codec(H, W, [(s, P)])
        c.encode([prev])
        _, modes = c.encode([cur], return_modes=True)
        assert modes == [1 if data[1] < data[0] else 0]


def test_trial_reads_only_the_test_rows():
    # test rows floor((2k+1)H/(2L)), L = 4: rows 2, 6, 10, 14 of a 16-row scan
    rng = np.random.default_rng(5)
    prev = random_scan(rng, 16, 64, 4, 0.1, 100000)
    cur = random_scan(rng, 16, 64, 4, 0.1, 100000)
    base = [oracle.trial_cost(cur, prev, 1, m) for m in (0, 1)]
    for r in range(16):
        mod = cur.copy()
        mod[r] = (mod[r].astype(np.uint64) * 7 + 12345).astype(np.uint32)
        costs = [oracle.trial_cost(mod, prev, 1, m) for m in (0, 1)]
        if r in (2, 6, 10, 14):
            assert costs != base
        else:
            assert costs == base


# ---------------------------------------------------------------- closed forms
def test_identical_scan_in_p_mode_has_empty_bodies():
    rng = np.random.default_rng(6)
    H, W = 5, 300
    v = random_scan(rng, H, W, 4, 0.3, 10**6)
    sec, mask_b, data_b = oracle.section_split(v, v, 7, 1)
    q = quantize_plane(v, 7, 4)
    nw = (W + 31) // 32
    nb = sum((int((q[r] != 0).sum()) + 127) // 128 for r in range(H))
    assert mask_b == H * 4 * ((nw + 15) // 16)  # every coded word is 0: class words only
    assert data_b == 4 * nb  # every block: b = 0, no exceptions, empty body
    assert sec == 8 * H + mask_b + data_b


def test_constant_row_in_i_mode():
    # one row of 128 equal nonzero values c: d = c, 0, 0, ...; z = 2c, 0, ...
    # -> b = 0 with one exception of width W(2c): 4 + 4 + 4*ceil(W/32) bytes
    for c in (1, 5, 1000, 2**20):
        v = np.full((1, 128), c, dtype=np.uint32)
        _, mask_b, data_b = oracle.section_split(v, v, 1, 0)
        hb = (2 * c).bit_length()
        assert mask_b == 4
        assert data_b == 4 + 4 + 4 * ((hb + 31) // 32)


def test_all_zero_scan_is_class_words_only():
    for W in (1, 8, 32, 33, 40, 512, 1000):
        v = np.zeros((3, W), dtype=np.uint16)
        c = oracle.Codec(3, W, [(2, 1)])
        b = c.encode([v])
        nw = (W + 31) // 32
        sec = 8 * 3 + 3 * 4 * ((nw + 15) // 16)
        assert len(b) == (16 + 8) + (8 + 12) + sec
        # every class is 1 (all valid bits of the word set)
        cls = np.frombuffer(b[44 + 24:44 + 24 + 4 * ((nw + 15) // 16)], dtype=np.uint32)
        bits = []
        for j in range(nw):
            bits.append((int(cls[j // 16]) >> (2 * (j % 16))) & 3)
        assert bits == [1] * nw


# ---------------------------------------------------------------- round trips
@pytest.mark.parametrize("seed", range(6))
def test_round_trip_random_sequences(seed):
    rng = np.random.default_rng(100 + seed)
    H = int(rng.choice([1, 2, 5, 16]))
    W = int(rng.choice([1, 31, 32, 33, 129, 256, 1000]))
    A = int(rng.integers(1, 4))
    attrs = [(int(rng.choice([1, 2, 4])), int(rng.choice([1, 2, 10, 255]))) for _ in range(A)]
    force = int(rng.choice([-1, -1, 0, 1]))
    enc = oracle.Codec(H, W, attrs, force_mode=force)
    dec = oracle.Codec(H, W, attrs)
    base = [random_scan(rng, H, W, s, 0.3, 1 << (8 * s)) for s, _ in attrs]
    for t in range(5):
        planes = []
        for (s, P), b in zip(attrs, base):
            x = b.astype(np.int64) + rng.integers(-2, 3, size=b.shape) * (t % 2)
            x = np.clip(x, 0, (1 << (8 * s)) - 1).astype(DT[s])
            x[rng.random(x.shape) < 0.05] = 0
            if t == 3:
                x[:] = (1 << (8 * s)) - 1  # maximum values
            planes.append(x)
        buf = enc.encode(planes)
        out, n = dec.decode(buf)
        assert n == len(buf)
        for (s, P), x, o in zip(attrs, planes, out):
            q = quantize_plane(x, P, s)
            assert np.array_equal(o.astype(np.uint64), q * P)


def test_round_trip_synthetic_multi_attribute():
    from paper_2209_08196_gb300 import synth
    cfg = synth.config_multi_attr(n_scans=3, H=8, W=512)
    seq = synth.ScanSequence(cfg).scans()
    attrs = synth.attr_descs(cfg)
    buf, lens, modes = oracle.encode_sequence(cfg.H, cfg.W, attrs, seq)
    out, pos = oracle.decode_sequence(cfg.H, cfg.W, attrs, buf, len(seq))
    assert pos == len(buf) == sum(lens)
    for t in range(len(seq)):
        for a, (s, P) in enumerate(attrs):
            assert np.array_equal(out[t][a].astype(np.uint64), quantize_plane(seq[t][a], P, s) * P)


def test_static_scene_prefers_p_and_reset_restarts_with_i():
    # Sec. III-D: a static scene makes successive scans near-identical
    rng = np.random.default_rng(8)
    v = random_scan(rng, 16, 256, 4, 0.2, 100000)
    c = oracle.Codec(16, 256, [(4, 1)])
    modes = [c.encode([v], return_modes=True)[1][0] for _ in range(3)]
    assert modes == [0, 1, 1]
    c.reset()
    b, m = c.encode([v], return_modes=True)
    assert m == [0] and b[:4] == b"JFY1"


def test_capacity_error_leaves_state_unchanged():
    rng = np.random.default_rng(9)
    v0 = random_scan(rng, 4, 64, 2, 0.2, 60000)
    v1 = random_scan(rng, 4, 64, 2, 0.2, 60000)
    a = oracle.Codec(4, 64, [(2, 1)])
    b = oracle.Codec(4, 64, [(2, 1)])
    a.encode([v0])
    b.encode([v0])
    import ctypes
    out = np.zeros(16, np.uint8)
    planes = (ctypes.c_void_p * 1)(v1.ctypes.data)
    rc = oracle.lib().jo_encode(a._h, planes, out.ctypes.data, 16, None)
    assert rc == -oracle.ERR_CAPACITY
    assert a.encode([v1]) == b.encode([v1])


def test_corrupt_streams_are_rejected():
    rng = np.random.default_rng(11)
    v = random_scan(rng, 3, 100, 4, 0.2, 10**6)
    buf = oracle.Codec(3, 100, [(4, 10)]).encode([v])
    for cut in (0, 10, 30, 50, len(buf) - 1):
        with pytest.raises(oracle.OracleError):
            oracle.Codec(3, 100, [(4, 10)]).decode(buf[:cut])
    bad = bytearray(buf)
    bad[0] ^= 1  # magic
    with pytest.raises(oracle.OracleError):
        oracle.Codec(3, 100, [(4, 10)]).decode(bytes(bad))
    with pytest.raises(oracle.OracleError):  # precision differs from the stream's
        oracle.Codec(3, 100, [(4, 11)]).decode(buf)


# ---------------------------------------------------------------- ablations (Sec. IV-H, Table IV)
def _read_bits(words, pos, n):
    """n bits of a little-endian bit stream held in u32 words, from bit pos."""
    v = 0
    for k in range(n):
        p = pos + k
        v |= ((int(words[p // 32]) >> (p % 32)) & 1) << k
    return v


def _unmasked_row_values(buf, H, W, A, a, frame_start):
    """Reads the packed values of every row of attribute a of the frame at
    frame_start in a stream without the mask stage, straight from the bytes:
    row table, block headers {b, e, hb, 0}, low bits, exception positions
    and high parts."""
    u32 = lambda o: int.from_bytes(buf[o:o + 4], "little")
    sec = frame_start + 8 + 12 * A
    for aa in range(a):
        sec += u32(frame_start + 12 + 12 * aa)
    data = sec + 8 * H
    rows, begin = [], 0
    for r in range(H):
        end = u32(sec + 8 * r)
        chunk = np.frombuffer(buf[data + begin:data + end], dtype="<u4")
        nb = (W + 127) // 128
        pos = nb
        z = []
        for g in range(nb):
            h = int(chunk[g])
            b, e, hb = h & 255, (h >> 8) & 255, (h >> 16) & 255
            m = min(128, W - 128 * g)
            body = chunk[pos:]
            vals = [_read_bits(body, i * b, b) for i in range(m)]
            low = (m * b + 31) // 32
            if e:
                pbytes = body[low:].tobytes()
                highs = body[low + (e + 3) // 4:]
                for j in range(e):
                    vals[pbytes[j]] |= _read_bits(highs, j * hb, hb) << b
            pos += low + ((e + 3) // 4 + (e * hb + 31) // 32 if e else 0)
            z += vals
        assert pos == len(chunk)
        rows.append(z)
        begin = end
    return rows


def _zz(x):
    x = int(np.int64(np.int32(np.uint32(x & 0xFFFFFFFF))))  # two's complement value
    return (2 * abs(x) + (1 if x < 0 else 0)) & 0xFFFFFFFF   # Eq. 1, modulo 2^32


@pytest.mark.parametrize("stages", [1, 3, 5, 7])
def test_unmasked_streams_pack_the_definition_of_each_stage(stages):
    # without the mask every sample is coded (zeros too); the packed values
    # are the residuals (I: q), deltaed over the flat vector unless the delta
    # is off, ZigZag coded (Eq. 1) unless ZigZag is off
    rng = np.random.default_rng(20 + stages)
    H, W, P = 3, 300, 3
    v = random_scan(rng, H, W, 2, 0.25, 60000)
    buf = oracle.Codec(H, W, [(2, P)], force_mode=0, stages=stages).encode([v])
    assert buf[16 + 1] == (0 if stages & 4 else 1) and buf[16 + 2] == stages & 3
    rows = _unmasked_row_values(buf, H, W, 1, 0, 24)
    e = [int(x) for x in quantize_plane(v, P, 2).ravel()]
    want, prev = [], 0
    for x in e:
        d = x if stages & 2 else (x - prev) & 0xFFFFFFFF
        want.append(d if stages & 4 else _zz(d))
        prev = x
    assert sum(rows, []) == want


def test_unmasked_p_frame_packs_every_temporal_difference():
    rng = np.random.default_rng(31)
    H, W = 2, 200
    v0 = random_scan(rng, H, W, 4, 0.3, 10**6)
    v1 = v0.copy()
    v1[rng.random(v1.shape) < 0.2] = 0  # new dropouts stay in the residual stream
    c = oracle.Codec(H, W, [(4, 1)], force_mode=1, stages=7)
    c.encode([v0])
    buf = c.encode([v1])
    rows = _unmasked_row_values(buf, H, W, 1, 0, 0)
    assert sum(rows, []) == [(int(a) - int(b)) & 0xFFFFFFFF for a, b in zip(v1.ravel(), v0.ravel())]


def test_mask_stage_off_on_a_scan_without_zeros_only_drops_the_class_words():
    # no zero sample: the masked stream's rows carry all-zero class words
    # (ceil(nw/16) per row) before the same blocks
    rng = np.random.default_rng(32)
    H, W = 4, 700
    v = rng.integers(1, 50000, size=(H, W)).astype(np.uint16)
    a = oracle.Codec(H, W, [(2, 1)], force_mode=0).encode([v])
    b = oracle.Codec(H, W, [(2, 1)], force_mode=0, stages=1).encode([v])
    ncls = ((W + 31) // 32 + 15) // 16
    assert len(a) - len(b) == 4 * ncls * H
    u32 = lambda buf, o: int.from_bytes(buf[o:o + 4], "little")
    sa, sb = 24 + 20 + 8 * H, 24 + 20 + 8 * H
    ba = bb = 0
    for r in range(H):
        ea, eb = u32(a, 24 + 20 + 8 * r), u32(b, 24 + 20 + 8 * r)
        assert a[sa + ba:sa + ba + 4 * ncls] == bytes(4 * ncls)
        assert a[sa + ba + 4 * ncls:sa + ea] == b[sb + bb:sb + eb]
        assert u32(a, 24 + 20 + 8 * r + 4) == u32(b, 24 + 20 + 8 * r + 4)  # same carries
        ba, bb = ea, eb


@pytest.mark.parametrize("stages", range(8))
@pytest.mark.parametrize("force", [-1, 0, 1])
def test_round_trip_every_stage_set(stages, force):
    rng = np.random.default_rng(40 + 3 * stages + force)
    H, W = 5, 77
    attrs = [(4, 3), (2, 1), (1, 2)]
    enc = oracle.Codec(H, W, attrs, force_mode=force, stages=stages)
    dec = oracle.Codec(H, W, attrs, stages=stages)
    base = [random_scan(rng, H, W, s, 0.3, 1 << (8 * s)) for s, _ in attrs]
    for t in range(4):
        planes = []
        for s, b in zip((4, 2, 1), base):
            x = np.clip(b.astype(np.int64) + rng.integers(-3, 4, size=b.shape), 0, (1 << (8 * s)) - 1).astype(DT[s])
            x[rng.random(x.shape) < 0.1] = 0
            planes.append(x)
        buf = enc.encode(planes)
        out, n = dec.decode(buf)
        assert n == len(buf)
        for (s, P), x, o in zip(attrs, planes, out):
            assert np.array_equal(o.astype(np.uint64), quantize_plane(x, P, s) * P)


def test_stage_set_is_part_of_the_stream_header():
    rng = np.random.default_rng(41)
    v = random_scan(rng, 2, 64, 2, 0.2, 60000)
    buf = oracle.Codec(2, 64, [(2, 1)], stages=3).encode([v])
    with pytest.raises(oracle.OracleError):  # a decoder of the full codec refuses it
        oracle.Codec(2, 64, [(2, 1)]).decode(buf)
    zbuf = oracle.Codec(2, 64, [(2, 1)], stages=oracle.ZSTD_MASK).encode([v])
    with pytest.raises(oracle.OracleError):  # and a stream with the Zstandard mask
        oracle.Codec(2, 64, [(2, 1)]).decode(zbuf)
    for bad in (16, oracle.ZSTD_MASK | oracle.NO_MASK):
        with pytest.raises(ValueError):
            oracle.Codec(2, 64, [(2, 1)], stages=bad)
