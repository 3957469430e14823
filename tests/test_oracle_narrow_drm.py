"""Pins of the oracle's DRMs in a narrow number format (bf16, e4m3).

The tensor cores multiply the dense tensor by Khatri-Rao blocks stored in the
plan's format, so the DRM the method applies is the stored block: the exact
product of the rounded per-mode factors, rounded once more (Sec. 7, Khatri-Rao
sketchings).  Three facts fix that reading independently of the oracle's own
code:
  * a hand-worked two-mode block, whose rounded entries (including two
    round-half-to-even ties) are written out below;
  * each stored block is within the format's unit roundoff of the exact
    Khatri-Rao product (2^-8 relative for bf16, 2^-4 for e4m3 plus the
    subnormal half-spacing 2^-10);
  * generalised Nystrom recovery (Sec. 4 recovery phase) is exact for a tensor
    whose TTN ranks equal the targets only when every node uses one X_t and
    one Y_t for Omega_t, Psi_t and its parent's Psi: the narrow-format DRMs
    recover such a tensor to 1e-12, and mixing the two Y blocks of the pass
    side's child (exact product in Omega, stored block in the parent's Psi)
    breaks it.
"""
import numpy as np
import pytest

import workloads as W
from oracle import sttnn as OS
from oracle import ttnn as O
from oracle.quant import round_to
from oracle.tree import Tree


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_pass_block_worked_example_bf16():
    # bf16 keeps 8 significant bits (7 after the point)
    a = np.array([[1.0 + 2.0 ** -7], [3.0]])
    b = np.array([[1.0 + 2.0 ** -7], [1.5]])
    # exact products, rows (i_a, i_b) with i_b fastest:
    #   (1 + 2^-7)^2      = 1 + 2^-6 + 2^-14   -> 1 + 2^-6      (2^-14 < half ulp)
    #   (1 + 2^-7) * 1.5  = 1 + 2^-1 + 2^-7 + 2^-8: a tie between
    #                       1.5078125 (odd last bit) and 1.515625 (even) -> 1.515625
    #   3 * (1 + 2^-7)    = 2 * the previous value                   -> 3.03125
    #   3 * 1.5           = 4.5 (exact)
    want = np.array([[1.015625], [1.515625], [3.03125], [4.5]])
    got = O.pass_block([a, b], "bf16")
    assert np.array_equal(got, want)
    exact = np.array([[(1 + 2.0 ** -7) ** 2], [(1 + 2.0 ** -7) * 1.5], [3 * (1 + 2.0 ** -7)], [4.5]])
    assert np.max(np.abs(got - exact) / exact) <= 2.0 ** -8
    # binary64 blocks are the exact product
    assert np.array_equal(O.pass_block([a, b], "f64"), exact)


def test_pass_block_worked_example_e4m3():
    # e4m3 keeps 4 significant bits: 1.125 * 1.125 = 1.265625 -> 1.25;
    # 1.125 * 1.5 = 1.6875 is a tie between 1.625 (odd) and 1.75 (even) -> 1.75
    a = np.array([[1.125], [1.5]])
    b = np.array([[1.125]])
    got = O.pass_block([a, b], "e4m3")
    assert np.array_equal(got, np.array([[1.25], [1.75]]))


TREES = [("binary4", W.balanced_binary(4), [5, 6, 5, 6]),
         ("tt4", W.tensor_train(4), [5, 4, 5, 4]),
         ("toy6", W.toy_tree(), [3, 4, 3, 4, 3, 4])]


def _tree(tr, dims, r, p):
    n = len(tr[0])
    return Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
@pytest.mark.parametrize("variant", ["ttnn", "sttnn"])
@pytest.mark.parametrize("name,tr,dims", TREES, ids=[t[0] for t in TREES])
def test_stored_blocks_within_unit_roundoff_of_exact_product(name, tr, dims, variant, fmt):
    t = _tree(tr, dims, 3, 2)
    drm = O.Drm(t, 31, fmt, variant)
    u, tiny = (2.0 ** -8, 0.0) if fmt == "bf16" else (2.0 ** -4, 2.0 ** -10)
    blocks = [(drm.BRX, [drm.X[mu] for mu in drm.Rmodes]),
              (drm.BLX, [drm.X[mu] for mu in drm.Lmodes])]
    if drm.Yside is not None:
        c = t.node(drm.ychild)
        blocks.append((drm.Yside, [drm.Y[mu] for mu in range(c.lo, c.hi)]))
    for stored, facs in blocks:
        exact = O.kr(facs)
        assert np.all(np.abs(stored - exact) <= u * np.abs(exact) + tiny)
        # and it is a rounding, not the exact product (the test would not bite otherwise)
        if len(facs) > 1:
            assert not np.array_equal(stored, exact)
    # the per-mode factors themselves are rounded once from binary64
    d64 = O.Drm(t, 31, "f64", variant)
    for mu in range(t.d):
        assert np.array_equal(drm.X[mu], round_to(d64.X[mu], fmt))
        assert np.array_equal(drm.Y[mu], round_to(d64.Y[mu], fmt))


def _sketch(variant):
    return O.sketch_ttnn if variant == "ttnn" else OS.sketch_sttnn


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
@pytest.mark.parametrize("variant", ["ttnn", "sttnn"])
@pytest.mark.parametrize("name,tr,dims", TREES, ids=[t[0] for t in TREES])
def test_narrow_drms_recover_exact_rank_tensor(name, tr, dims, variant, fmt):
    """TTN ranks equal to the targets (3), p = 2: the recovery is exact up to
    binary64 rounding with the narrow-format DRMs of either variant."""
    n = len(tr[0])
    T, _ = W.exact_ttn(tr, dims, [3] * n, 17)
    t = _tree(tr, dims, 3, 2)
    drm = O.Drm(t, 41, fmt, variant)
    cores, info = O.recover(t, *_sketch(variant)(T, t, drm))
    assert _rel(O.reconstruct(t, cores), T) <= 1e-12
    assert all(k == 3 for k in info.values())


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_mixed_y_blocks_break_exact_recovery(fmt):
    """Negative control: Omega of the pass side's Y child taken with the exact
    Khatri-Rao product while the root's Psi uses the stored block -- one
    plausible way to get the rule wrong -- is no longer exact."""
    tr, dims = W.balanced_binary(4), [5, 6, 5, 6]
    T, _ = W.exact_ttn(tr, dims, [3] * 7, 17)
    t = _tree(tr, dims, 3, 2)
    drm = O.Drm(t, 41, fmt, "ttnn")
    assert drm.Yside is not None
    Om, Ps, Pr = O.sketch_ttnn(T, t, drm)
    v = drm.ychild
    nd = t.node(v)
    G = O.unfold(T, nd.lo, nd.hi) @ drm.Xt(v)
    Om_bad = dict(Om)
    Om_bad[v] = O.kr([drm.Y[mu] for mu in range(nd.lo, nd.hi)])[:, :nd.s].T @ G
    good, _ = O.recover(t, Om, Ps, Pr)
    bad, _ = O.recover(t, Om_bad, Ps, Pr)
    assert _rel(O.reconstruct(t, good), T) <= 1e-12
    assert _rel(O.reconstruct(t, bad), T) > 1e-6
