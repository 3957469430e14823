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
