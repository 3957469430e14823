"""Precision forms of the first-level pass on the GPU against the oracle:
BF16x2 split (binary32 tensor as bf16 hi + lo on the tensor cores) and FP8
E4M3 with one binary32 scale per 128 x 128 tile (dequantised to bfloat16 on
chip).  All calls go through the C ABI."""
import numpy as np
import pytest

import workloads as W
from oracle import quant as Q
from oracle import sttnn as OS
from oracle import ttnn as O
from oracle.tree import Tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run, rel  # noqa: E402

# binary roots: the pass matrix is (first root child's modes) x (the rest)
CASES = {
    "bin5_960x960": (W.balanced_binary(5), [8, 12, 10, 24, 40], 4, 2),
    "bin4_r20": (W.balanced_binary(4), [16, 16, 32, 32], 20, 10),
    "bin4_80x2560": (W.balanced_binary(4), [8, 10, 40, 64], 6, 4),
    "bin4_64x4096": (W.balanced_binary(4), [8, 8, 64, 64], 6, 4),
}


def _otree(tr, dims, r, p):
    n = len(tr[0])
    return Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])


def _nl(run, dims):
    root = [nd for nd in run.nodes if nd["parent"] < 0][0]
    first = min((nd for nd in run.nodes if nd["parent"] == root["user_index"]),
                key=lambda nd: nd["mode_lo"])
    return int(np.prod(dims[first["mode_lo"]:first["mode_hi"]]))


def _sketch(variant, T, t, drm):
    return (O.sketch_ttnn if variant == api.VARIANT_TTNN else OS.sketch_sttnn)(T, t, drm)


def _worst(run, want):
    Om, Ps, Pr = want
    gOm, gPs, gPr = run.sketches()
    w = max(max(rel(gOm[v], Om[v]), rel(gPs[v], Ps[v])) for v in Om)
    return max(w, rel(gPr, Pr))


@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
@pytest.mark.parametrize("case", sorted(CASES))
def test_bf16x2_pass_matches_oracle(case, variant):
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    T = W.gaussian(dims, 5).astype(np.float32).astype(np.float64)
    run = Run(tr, dims, [r] * n, [p] * n, 31, dtype=api.BF16X2, variant=variant)
    try:
        api.ttnn_update_dense(run.state, torch.from_numpy(T.astype(np.float32)).cuda())
        assert api.ttnn_plan_pass_counts(run.plan) == (1, 0)
        t = _otree(tr, dims, r, p)
        drm = O.Drm(t, 31, "bf16", "sttnn" if variant else "ttnn")
        hi, lo = Q.split_bf16x2(T)
        assert _worst(run, _sketch(variant, hi + lo, t, drm)) <= 1e-5
        # the split carries ~16 significand bits: close to the unsplit tensor
        assert _worst(run, _sketch(variant, T, t, drm)) <= 1e-4
        run.recover()
    finally:
        run.close()


@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
@pytest.mark.parametrize("case", sorted(CASES))
def test_fp8_pass_matches_oracle(case, variant):
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    T = W.gaussian(dims, 6).astype(np.float32).astype(np.float64)
    run = Run(tr, dims, [r] * n, [p] * n, 32, dtype=api.E4M3, variant=variant)
    try:
        nl = _nl(run, dims)
        q, s = Q.fp8_tile_quantize(T.reshape(nl, -1))
        qb = torch.from_numpy(Q.e4m3_encode(q).reshape(-1)).cuda()
        sc = torch.from_numpy(s.astype(np.float32).reshape(-1)).cuda()
        api.ttnn_update_dense(run.state, qb, tile_scale=sc)
        assert api.ttnn_plan_pass_counts(run.plan) == (1, 0)
        t = _otree(tr, dims, r, p)
        drm = O.Drm(t, 32, "e4m3", "sttnn" if variant else "ttnn")
        D = Q.fp8_dequantize_bf16(q, s).reshape(dims)
        assert _worst(run, _sketch(variant, D, t, drm)) <= 1e-5
        run.recover()
    finally:
        run.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp8_quantize_bitwise(case):
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    T = (W.gaussian(dims, 8) * np.exp(np.random.default_rng(1).uniform(-6, 6, dims)))
    T = T.astype(np.float32).astype(np.float64)
    T.reshape(-1)[:300] = 0.0
    run = Run(tr, dims, [r] * n, [p] * n, 1, dtype=api.E4M3)
    try:
        nl = _nl(run, dims)
        q, s = Q.fp8_tile_quantize(T.reshape(nl, -1))
        src = torch.from_numpy(T.astype(np.float32)).cuda()
        dst = torch.empty(T.size, dtype=torch.uint8, device="cuda")
        sc = torch.empty(s.size, dtype=torch.float32, device="cuda")
        api.ttnn_fp8_quantize(run.plan, src, dst, sc)
        torch.cuda.synchronize()
        assert np.array_equal(dst.cpu().numpy(), Q.e4m3_encode(q).reshape(-1))
        assert np.array_equal(sc.cpu().numpy().astype(np.float64), s.reshape(-1))
    finally:
        run.close()


def test_fp8_box_update_and_quantize_extent():
    # a box of the tensor: quantised over the box's own pass matrix
    tr, dims, r, p = CASES["bin4_80x2560"]
    n = len(tr[0])
    off, ext = [0, 3, 8, 0], [8, 5, 16, 64]       # box pass matrix 40 x 1024
    rng = np.random.default_rng(2)
    B = rng.standard_normal(ext).astype(np.float32).astype(np.float64)
    run = Run(tr, dims, [r] * n, [p] * n, 3, dtype=api.E4M3)
    try:
        nlb = ext[0] * ext[1]
        src = torch.from_numpy(B.astype(np.float32)).cuda()
        dst = torch.empty(B.size, dtype=torch.uint8, device="cuda")
        ntile = -(-nlb // 128) * -(-(B.size // nlb) // 128)
        sc = torch.empty(ntile, dtype=torch.float32, device="cuda")
        api.ttnn_fp8_quantize(run.plan, src, dst, sc, extent=ext)
        api.ttnn_update_dense(run.state, dst, off, ext, tile_scale=sc)
        q, s = Q.fp8_tile_quantize(B.reshape(nlb, -1))
        D = W.embed_box(dims, off, ext, Q.fp8_dequantize_bf16(q, s).reshape(ext))
        t = _otree(tr, dims, r, p)
        assert _worst(run, O.sketch_ttnn(D, t, O.Drm(t, 3, "e4m3"))) <= 1e-5
    finally:
        run.close()


def test_bf16x2_box_update():
    tr, dims, r, p = CASES["bin5_960x960"]
    n = len(tr[0])
    off, ext = [2, 0, 1, 8, 0], [4, 12, 6, 8, 40]
    B = np.random.default_rng(3).standard_normal(ext).astype(np.float32).astype(np.float64)
    run = Run(tr, dims, [r] * n, [p] * n, 4, dtype=api.BF16X2)
    try:
        api.ttnn_update_dense(run.state, torch.from_numpy(B.astype(np.float32)).cuda(), off, ext)
        hi, lo = Q.split_bf16x2(B)
        t = _otree(tr, dims, r, p)
        want = O.sketch_ttnn(W.embed_box(dims, off, ext, hi + lo), t, O.Drm(t, 4, "bf16"))
        assert _worst(run, want) <= 1e-5
    finally:
        run.close()


def test_narrow_formats_reject_unsupported_shapes():
    # E4M3 needs 16-byte rows of the pass matrix (24 columns do not give them):
    # the plan is refused, as no whole-tensor update could run
    tr, dims = W.tensor_train(4), [16, 16, 16, 24]
    n = len(tr[0])
    with pytest.raises(api.TtnnError) as ei:
        Run(tr, dims, [6] * n, [3] * n, 1, dtype=api.E4M3)
    assert ei.value.status == 7
    # a supported shape without tile scales is an argument error
    tr, dims, r, p = CASES["bin5_960x960"]
    n = len(tr[0])
    run = Run(tr, dims, [r] * n, [p] * n, 1, dtype=api.E4M3)
    try:
        data = torch.zeros(int(np.prod(dims)), dtype=torch.uint8, device="cuda")
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_update_dense(run.state, data)
        assert ei.value.status == 1
        assert not np.any(run.state_host())
    finally:
        run.close()


@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
@pytest.mark.parametrize("fixed", ["right", "left"])
def test_rank_one_boxes_narrow_formats(fixed, variant):
    # boxes fixing every mode of one pass side take the rank-one path in the
    # BF16x2 (split rows) and E4M3 (dequantised rows) formats as well
    tr, dims, r, p = CASES["bin4_80x2560"]      # left modes {0, 1}, right {2, 3}
    n = len(tr[0])
    t = _otree(tr, dims, r, p)
    rng = np.random.default_rng(9)
    fix = [2, 3] if fixed == "right" else [0, 1]
    off = [int(rng.integers(0, d)) if mu in fix else 1 for mu, d in enumerate(dims)]
    ext = [1 if mu in fix else dims[mu] - 1 for mu in range(4)]
    B = rng.standard_normal(ext).astype(np.float32).astype(np.float64)
    nlb = ext[0] * ext[1]
    # BF16x2
    run = Run(tr, dims, [r] * n, [p] * n, 41, dtype=api.BF16X2, variant=variant)
    try:
        api.ttnn_update_dense(run.state, torch.from_numpy(B.astype(np.float32)).cuda(), off, ext,
                              lam=0.5)
        hi, lo = Q.split_bf16x2(B)
        drm = O.Drm(t, 41, "bf16", "sttnn" if variant else "ttnn")
        want = _sketch(variant, 0.5 * W.embed_box(dims, off, ext, hi + lo), t, drm)
        assert _worst(run, want) <= 1e-5
    finally:
        run.close()
    # E4M3, quantised over the box's own pass matrix
    run = Run(tr, dims, [r] * n, [p] * n, 42, dtype=api.E4M3, variant=variant)
    try:
        src = torch.from_numpy(B.astype(np.float32)).cuda()
        dst = torch.empty(B.size, dtype=torch.uint8, device="cuda")
        ntile = -(-nlb // 128) * -(-(B.size // nlb) // 128)
        sc = torch.empty(ntile, dtype=torch.float32, device="cuda")
        api.ttnn_fp8_quantize(run.plan, src, dst, sc, extent=ext)
        api.ttnn_update_dense(run.state, dst, off, ext, tile_scale=sc)
        q, s = Q.fp8_tile_quantize(B.reshape(nlb, -1))
        D = W.embed_box(dims, off, ext, Q.fp8_dequantize_bf16(q, s).reshape(ext))
        drm = O.Drm(t, 42, "e4m3", "sttnn" if variant else "ttnn")
        assert _worst(run, _sketch(variant, D, t, drm)) <= 1e-5
    finally:
        run.close()
