"""Parity at the full benchmark size, in the configuration bench.py times:
the dense order-5 64^5 tensor 1/sum(x) on [1,2]^5 (binary64 -> binary32 and
the form's storage, as the bench builds it), balanced binary tree
((0,1),2),(3,4), r = 20, p = 10, one whole-tensor update then recovery.
Every form the bench times is checked: BF16 TTNN and STTNN (tcgen05 pass),
FP32 plain (tensor-core pass: binary32 data and DRM blocks each split into
bf16 hi + lo, three products), the BF16x2 split and FP8 E4M3 with per-tile scales
(converter passes).  Each form's sketches are compared with the oracle run
on the tensor that form sketches, then the recovered cores' reconstructions
are compared.  Needs ~40 GB of host memory and a few minutes of host time
for the oracle."""
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

D, N, RANK, OVER, SEED = 5, 64, 20, 10, 2024   # the bench configuration

_CACHE = {}


def _t32():
    """The binary32 tensor of the bench (binary64 values, as f64 array)."""
    if "t32" not in _CACHE:
        _CACHE["t32"] = Q.round_to(W.inv_sum(D, N), "f32")
    return _CACHE["t32"]


def _tree():
    tr = W.balanced_binary(D)
    n = len(tr[0])
    return tr, n, Tree(tr[0], tr[1], [N] * D, [RANK] * n, [OVER] * n, tr[2])


def _check(dtype, variant, dev, Ts, fmt, sk_tol, rec_tol, tile_scale=None):
    """Runs one whole-tensor update + recovery and compares with the oracle
    run on Ts (the tensor the form sketches) with the fmt DRMs."""
    tr, n, t = _tree()
    run = Run(tr, [N] * D, [RANK] * n, [OVER] * n, SEED, dtype=dtype, variant=variant)
    try:
        api.ttnn_update_dense(run.state, dev, tile_scale=tile_scale)
        tc, simt = api.ttnn_plan_pass_counts(run.plan)
        assert (tc, simt) == (1, 0)          # every form on the tensor-core pass
        gOm, gPs, gPr = run.sketches()
        cores = run.recover()
        vname = "sttnn" if variant == api.VARIANT_STTNN else "ttnn"
        drm = O.Drm(t, SEED, fmt, vname)
        Om, Ps, Pr = (OS.sketch_sttnn if vname == "sttnn" else O.sketch_ttnn)(Ts, t, drm)
        worst = max(max(rel(gOm[v], Om[v]), rel(gPs[v], Ps[v])) for v in t.sketched())
        worst = max(worst, rel(gPr, Pr))
        assert worst <= sk_tol, worst
        want = O.reconstruct(t, O.recover(t, Om, Ps, Pr)[0])
        got = O.reconstruct(t, cores)
        assert rel(got, want) <= rec_tol, rel(got, want)
        return got, want
    finally:
        run.close()


@pytest.mark.timeout(1200)
@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
def test_full_size_bf16_sketches_and_recovery_match_oracle(variant):
    Tq = Q.round_to(_t32(), "bf16")
    dev = torch.from_numpy(Tq.astype(np.float32)).cuda().to(torch.bfloat16)
    # binary32 accumulation over up to 2^18 terms per product: 2e-5;
    # reconstructions within 1e-4
    got, want = _check(api.BF16, variant, dev, Tq, "bf16", 2e-5, 1e-4)
    del dev
    torch.cuda.empty_cache()
    # the approximation error itself is the method's, not the kernels':
    # the GPU and the oracle land on the same value (about 2e-2 here, the
    # bfloat16 storage noise of the input amplified by the recovery)
    assert abs(rel(got, Tq) - rel(want, Tq)) <= 1e-3 * rel(want, Tq)


@pytest.mark.timeout(1200)
def test_full_size_fp32_plain_matches_oracle():
    T32 = _t32()
    dev = torch.from_numpy(T32.astype(np.float32)).cuda()
    # the FP32 plain form's stated tolerance: 1e-4 relative Frobenius
    _check(api.F32, api.VARIANT_TTNN, dev, T32, "f32", 1e-4, 1e-4)
    del dev
    torch.cuda.empty_cache()


@pytest.mark.timeout(1200)
def test_full_size_bf16x2_split_matches_oracle():
    T32 = _t32()
    hi, lo = Q.split_bf16x2(T32)
    dev = torch.from_numpy(T32.astype(np.float32)).cuda()
    # two products (hi and lo) per entry accumulated in binary32: 5e-5
    _check(api.BF16X2, api.VARIANT_TTNN, dev, hi + lo, "bf16", 5e-5, 1e-4)
    del dev
    torch.cuda.empty_cache()


@pytest.mark.timeout(1200)
def test_full_size_fp8_quantize_and_pass_match_oracle():
    T32 = _t32()
    nl = N ** 3                                   # rows of the pass matrix (modes 0-2)
    src = torch.from_numpy(T32.astype(np.float32)).cuda()
    ntile = (nl // 128) * (T32.size // nl // 128)
    q8 = torch.empty(T32.size, dtype=torch.uint8, device="cuda")
    sc = torch.empty(ntile, dtype=torch.float32, device="cuda")
    tr, n, _ = _tree()
    probe = Run(tr, [N] * D, [RANK] * n, [OVER] * n, SEED, dtype=api.E4M3)
    try:
        api.ttnn_fp8_quantize(probe.plan, src, q8, sc)
        torch.cuda.synchronize()
    finally:
        probe.close()
    del src
    q, s = Q.fp8_tile_quantize(T32.reshape(nl, -1))
    # the quantiser is bit-exact at full size
    assert np.array_equal(sc.cpu().numpy().astype(np.float64), s.reshape(-1))
    qh, qf = q8.cpu().numpy(), q.reshape(-1)
    step = 1 << 25
    for k in range(0, qf.size, step):
        assert np.array_equal(qh[k:k + step], Q.e4m3_encode(qf[k:k + step]))
    del qh, qf
    Dq = Q.fp8_dequantize_bf16(q, s).reshape([N] * D)
    del q
    _check(api.E4M3, api.VARIANT_TTNN, q8, Dq, "e4m3", 2e-5, 1e-4, tile_scale=sc)
    del q8
    torch.cuda.empty_cache()
