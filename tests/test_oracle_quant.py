"""Pins of the oracle's rounding into the sketch number formats."""
import numpy as np

from oracle.quant import round_to


def test_f32_is_ieee_cast():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(50000) * np.exp(rng.uniform(-80, 80, 50000))
    assert np.array_equal(round_to(x, "f32"), x.astype(np.float32).astype(np.float64))


def test_bf16_hand_values():
    import torch
    assert float.fromhex("0x1.fep127") == torch.finfo(torch.bfloat16).max
    u = 2.0 ** -8
    x = np.array([1 + u, 1 + 3 * u, 1 + 2 * u, -(1 + 1.5 * u), 2.0 ** -133, 2.0 ** -134,
                  3 * 2.0 ** -134, 2.0 ** 128, float.fromhex("0x1.fep127"),
                  float.fromhex("0x1.ffp127"), float.fromhex("0x1.fefffp127"), 0.0, -0.0])
    want = np.array([1.0, 1 + 4 * u, 1 + 2 * u, -(1 + 2 * u), 2.0 ** -133, 0.0,
                     2.0 ** -132, np.inf, float.fromhex("0x1.fep127"), np.inf,
                     float.fromhex("0x1.fep127"), 0.0, -0.0])
    got = round_to(x, "bf16")
    assert np.array_equal(got, want)
    assert np.signbit(got[-1])


def _e4m3_values():
    vals = set()
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue            # NaN encoding
            v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
            vals.add(v)
            vals.add(-v)
    return np.array(sorted(vals))


def test_e4m3_nearest_even_brute_force():
    grid = _e4m3_values()
    assert grid.max() == 448.0 and np.all(round_to(grid, "e4m3") == grid)
    rng = np.random.default_rng(2)
    x = rng.uniform(-460, 460, 20000) * np.exp(rng.uniform(-12, 0, 20000))
    got = round_to(x, "e4m3")
    for xi, gi in zip(x[:4000], got[:4000]):
        if abs(xi) > 448:
            assert gi == np.sign(xi) * 448
            continue
        d = np.abs(grid - xi)
        best = grid[d == d.min()]
        if best.size == 1:
            assert gi == best[0]
        else:   # tie: even significand
            assert gi in best


def test_bf16_matches_direct_rne_not_double_rounding():
    # 0x1.deffffc9...p-15 rounds down in one step; through fp32 it would tie up
    x = float.fromhex("-0x1.deffffc94b117p-15")
    assert round_to(np.array([x]), "bf16")[0] == float.fromhex("-0x1.dep-15")


# ---- precision forms of the pass: BF16x2 split and per-tile E4M3 ----------
from oracle.quant import (e4m3_decode, e4m3_encode, fp8_dequantize_bf16,  # noqa: E402
                          fp8_tile_quantize, split_bf16x2)


def test_bf16x2_split_bound_and_exact_cases():
    rng = np.random.default_rng(3)
    A = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    A = A.astype(np.float64)
    hi, lo = split_bf16x2(A)
    # both halves are bfloat16 values, hi is the bf16 rounding of A
    assert np.array_equal(round_to(hi, "bf16"), hi) and np.array_equal(round_to(lo, "bf16"), lo)
    assert np.array_equal(hi, round_to(A, "bf16"))
    # A - hi has at most 16 significant bits left; lo rounds it to 8: 2^-17 relative
    assert np.all(np.abs(A - (hi + lo)) <= 2.0 ** -17 * np.abs(A) * (1 + 1e-12))
    # bf16-representable inputs split with lo = 0
    b = round_to(A[:1000], "bf16")
    h2, l2 = split_bf16x2(b)
    assert np.array_equal(h2, b) and not np.any(l2)
    # a value needing exactly 16 bits is carried exactly
    x = 1.0 + 2.0 ** -7 + 2.0 ** -15
    h3, l3 = split_bf16x2(np.array([x]))
    assert h3[0] + l3[0] == x


def test_e4m3_codes_golden():
    # OCP FP8 E4M3 code points: bias 7, 3 mantissa bits, 0x7e = 448, NaN 0x7f
    vals = np.array([0.0, 1.0, 448.0, 2.0 ** -9, 2.0 ** -6, 1.75, -2.0, 0.875 * 2.0 ** -6, 240.0])
    codes = np.array([0x00, 0x38, 0x7E, 0x01, 0x08, 0x3E, 0xC0, 0x07, 0x77], dtype=np.uint8)
    assert np.array_equal(e4m3_encode(vals), codes)
    assert np.array_equal(e4m3_decode(codes), vals)
    assert np.isnan(e4m3_decode(np.array([0x7F, 0xFF], dtype=np.uint8))).all()
    allv = _e4m3_values()
    assert np.array_equal(e4m3_decode(e4m3_encode(allv)), allv)


def test_fp8_tile_quantize_properties():
    rng = np.random.default_rng(9)
    M = rng.standard_normal((300, 200)).astype(np.float32).astype(np.float64)
    M[128:256, 128:200] = 0.0                     # an all-zero tile: scale 1
    M[0, 0] = 1e4                                 # a large entry sets its tile's scale
    q, s = fp8_tile_quantize(M)
    assert s.shape == (3, 2) and s[1, 1] == 1.0
    assert np.array_equal(round_to(q, "e4m3"), q)
    assert np.abs(q).max() <= 448.0
    for bi in range(3):
        for bj in range(2):
            t = M[bi * 128:(bi + 1) * 128, bj * 128:(bj + 1) * 128]
            qt = q[bi * 128:(bi + 1) * 128, bj * 128:(bj + 1) * 128]
            mx = np.abs(t).max()
            if mx == 0:
                continue
            assert s[bi, bj] == float(np.float32(np.float32(mx) / np.float32(448.0)))
            # the largest entry lands on +-448 (up to the binary32 division)
            assert abs(np.abs(qt).max() - 448.0) <= 448.0 * 2.0 ** -4
            # relative error of the dequantised tile: e4m3 half-ulp 2^-4 (normal
            # range) + subnormal floor 2^-10 * s + the bf16 rounding 2^-8
            D = fp8_dequantize_bf16(qt, s[bi:bi + 1, bj:bj + 1])
            err = np.abs(D - t)
            bound = (2.0 ** -4 + 2.0 ** -8 + 2.0 ** -12) * np.abs(t) + 2.0 ** -10 * s[bi, bj] * 1.01
            assert np.all(err <= bound)
