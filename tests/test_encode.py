"""BF16 / FP8-E4M3 navigation encoders against the formats' definitions
(hand-worked values, ties-to-even cases, saturation, round trips)."""
import numpy as np

import oracle
import paper_2507_10070_b300 as ann


def test_bf16_round_to_nearest_even():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 0.0, 3.0e38], np.float32)
    got = oracle.decode_bf16(ann.encode_bf16(x))
    assert got[0] == 1.0
    assert got[1] == 1.0                      # tie: to the even mantissa (0)
    assert got[2] == 1 + 2 ** -6              # tie between mantissas 1 and 2: to 2
    assert got[3] == -2.5 and got[4] == 0.0
    rng = np.random.default_rng(0)
    y = rng.normal(size=100_000).astype(np.float32)
    dy = oracle.decode_bf16(ann.encode_bf16(y))
    assert np.all(np.abs(dy - y) <= 2.0 ** -8 * np.abs(y.astype(np.float64)))   # half an ulp


def test_fp8_e4m3_hand_values():
    vals = {1.0: 0x38, -2.0: 0xC0, 448.0: 0x7E, 500.0: 0x7E, -1e9: 0xFE, 0.0: 0x00,
            2.0 ** -9: 0x01, 7 * 2.0 ** -9: 0x07, 2.0 ** -6: 0x08,
            2.0 ** -10: 0x00,            # half the smallest subnormal: tie to even (0)
            3 * 2.0 ** -10: 0x02,        # 1.5 subnormal steps: tie to even (2)
            7.5 * 2.0 ** -9: 0x08,       # between 7 steps and the smallest normal: even (8)
            1 + 1 / 16: 0x38,            # tie between 1.0 and 1.125: even (1.0)
            1 + 3 / 16: 0x3A,            # tie between 1.125 and 1.25: even (1.25)
            0.3: 0x2A}                   # 0.3 = 1.2 * 2^-2 -> 1.25 * 2^-2 (mantissa field 2)
    x = np.array(list(vals), np.float32)
    assert ann.encode_fp8e4m3(x).tolist() == list(vals.values())


def test_fp8_e4m3_round_trip_and_error():
    codes = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], np.uint8)   # all but NaN
    dec = oracle.decode_fp8e4m3(codes)
    assert np.array_equal(ann.encode_fp8e4m3(dec.astype(np.float32)), codes)
    assert np.isnan(oracle.decode_fp8e4m3(np.array([0x7F, 0xFF], np.uint8))).all()
    rng = np.random.default_rng(1)
    y = rng.uniform(-1, 1, 100_000).astype(np.float32)
    s = 64.0
    dy = oracle.decode_fp8e4m3(ann.encode_fp8e4m3(y, s), s)
    normal = np.abs(y) * s >= 2.0 ** -6
    assert np.all(np.abs(dy - y)[normal] <= 2.0 ** -4 * np.abs(y[normal]))        # half an ulp
    assert np.all(np.abs(dy - y)[~normal] <= 2.0 ** -10 / s + 1e-12)
