"""GPU path against the FP64 oracle, element by element, on seeded inputs
(ragged sizes, several tree shapes, both variants, every number format the
SIMT path runs).  All calls go through the C ABI (libttnn.so)."""
import numpy as np
import pytest

import workloads as W
from oracle import philox
from oracle import sttnn as OS
from oracle import ttnn as O
from oracle.tree import Tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run, rel  # noqa: E402

FMT = {api.F64: "f64", api.F32: "f32", api.BF16: "bf16", api.E4M3: "e4m3"}

CASES = {
    "binary4": (W.balanced_binary(4), [7, 5, 6, 4], 3, 2),
    "toy6": (W.toy_tree(), [3, 4, 3, 5, 4, 3], 2, 2),
    "tt5": (W.tensor_train(5), [4, 3, 5, 3, 4], 2, 1),
    "tucker4": (W.tucker(4), [5, 4, 6, 3], 2, 2),
    "binary5": (W.balanced_binary(5), [6, 7, 5, 8, 6], 4, 2),
}


def _otree(tr, dims, r, p):
    n = len(tr[0])
    return Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])


def _dev(T, dtype):
    t = torch.from_numpy(np.ascontiguousarray(T)).cuda()
    if dtype == api.F64:
        return t.double(), T
    if dtype == api.F32:
        t = t.float()
    else:
        t = t.float().to(torch.bfloat16)
    return t, t.double().cpu().numpy()


@pytest.mark.parametrize("seed", [0, 1, 2 ** 40 + 3])
@pytest.mark.parametrize("fmt", [0, 1, 2, 3])
def test_philox_generator_bitwise(seed, fmt):
    for kind, ident, rows, cols in [(1, 0, 37, 24), (2, 5, 129, 48), (3, 77, 8, 5), (1, 3, 1000, 1)]:
        dst = torch.empty(rows * cols, dtype=torch.float64, device="cuda")
        api.ttnn_philox_gaussian(seed, kind, ident, rows, cols, fmt, dst)
        got = dst.cpu().numpy().reshape(rows, cols)
        want = philox.gaussian_matrix(seed, kind, ident, rows, cols)
        from oracle.quant import round_to
        want = round_to(want, FMT[fmt])
        assert np.array_equal(got, want), (seed, fmt, kind, np.abs(got - want).max())


@pytest.mark.parametrize("dtype", [api.F64, api.F32, api.BF16])
def test_plan_factors_bitwise(dtype):
    tr, dims, r, p = CASES["toy6"]
    run = Run(tr, dims, [r] * len(tr[0]), [p] * len(tr[0]), 1234, dtype=dtype)
    try:
        t = _otree(tr, dims, r, p)
        drm = O.Drm(t, 1234, FMT[dtype])
        for mu in range(len(dims)):
            for which, want in ((1, drm.X[mu]), (2, drm.Y[mu])):
                rows, cols = api.ttnn_plan_factor(run.plan, which, mu)
                dst = torch.empty(rows * cols, dtype=torch.float64, device="cuda")
                api.ttnn_plan_factor(run.plan, which, mu, dst)
                assert np.array_equal(dst.cpu().numpy().reshape(rows, cols), want)
        for v in t.sketched():
            lex = t.node(v).lex
            rows, cols = api.ttnn_plan_factor(run.plan, 3, lex)
            dst = torch.empty(rows * cols, dtype=torch.float64, device="cuda")
            api.ttnn_plan_factor(run.plan, 3, lex, dst)
            assert np.array_equal(dst.cpu().numpy().reshape(rows, cols), drm.XT[v])
    finally:
        run.close()


def _compare_sketches(run, t, T, drm, variant, tol):
    Om, Ps, Pr = (O.sketch_ttnn if variant == api.VARIANT_TTNN else OS.sketch_sttnn)(T, t, drm)
    gOm, gPs, gPr = run.sketches()
    worst = 0.0
    for v in t.sketched():
        worst = max(worst, rel(gOm[v], Om[v]), rel(gPs[v], Ps[v]))
    worst = max(worst, rel(gPr, Pr))
    assert worst <= tol, worst
    return worst


@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("dtype,tol", [(api.F64, 1e-12), (api.F32, 1e-5), (api.BF16, 1e-5)])
def test_sketches_match_oracle(case, variant, dtype, tol):
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    T = W.gaussian(dims, 17)
    dev, Tq = _dev(T, dtype)
    run = Run(tr, dims, [r] * n, [p] * n, 99, dtype=dtype, variant=variant)
    try:
        api.ttnn_update_dense(run.state, dev)
        t = _otree(tr, dims, r, p)
        drm = O.Drm(t, 99, FMT[dtype], "sttnn" if variant else "ttnn")
        _compare_sketches(run, t, Tq, drm, variant, tol)
    finally:
        run.close()


@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
@pytest.mark.parametrize("case", sorted(CASES))
def test_recovery_matches_oracle_f64(case, variant):
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    T, _ = W.exact_ttn(tr, dims, [max(1, r - 1)] * n, 5, noise=1e-3)
    run = Run(tr, dims, [r] * n, [p] * n, 7, dtype=api.F64, variant=variant)
    try:
        api.ttnn_update_dense(run.state, torch.from_numpy(T).cuda())
        cores = run.recover()
        t = _otree(tr, dims, r, p)
        drm = O.Drm(t, 7, "f64", "sttnn" if variant else "ttnn")
        sk = (O.sketch_ttnn if variant == 0 else OS.sketch_sttnn)(T, t, drm)
        ocores, kept = O.recover(t, *sk)
        rg, ro = O.reconstruct(t, cores), O.reconstruct(t, ocores)
        assert rel(rg, ro) <= 1e-10
        for v in t.sketched():
            assert run.nodes[v]["kept_rank"] == kept[v]
    finally:
        run.close()


@pytest.mark.parametrize("noise,tol", [(0.0, 1e-12), (1e-8, 1e-6)])
def test_exact_recovery_order4_24(noise, tol):
    """Order-4 24^4 exact TTN, ranks 5, l = 5, FP64, one update."""
    tr = W.balanced_binary(4)
    dims = [24] * 4
    T, _ = W.exact_ttn(tr, dims, [5] * 7, 1000, noise=noise)
    run = Run(tr, dims, [5] * 7, [5] * 7, 2000, dtype=api.F64)
    try:
        api.ttnn_update_dense(run.state, torch.from_numpy(T).cuda())
        t = _otree(tr, dims, 5, 5)
        R = O.reconstruct(t, run.recover())
        assert rel(R, T) <= tol
    finally:
        run.close()


@pytest.mark.parametrize("dtype,tol", [(api.F64, 1e-12), (api.F32, 1e-5)])
def test_box_updates_are_linear(dtype, tol):
    """Sketch of a sum of sub-block updates = sum of their sketches (Sec. 4
    streaming) = sketch of the whole tensor."""
    tr, dims, r, p = CASES["toy6"]
    n = len(tr[0])
    rng = np.random.default_rng(3)
    T = np.zeros(dims)
    run = Run(tr, dims, [r] * n, [p] * n, 5, dtype=dtype)
    try:
        for k in range(6):
            off = [int(rng.integers(0, d)) for d in dims]
            ext = [int(rng.integers(1, d - o + 1)) for d, o in zip(dims, off)]
            data = rng.standard_normal(ext)
            lam = float(rng.uniform(-2, 2))
            dev, dq = _dev(data, dtype)
            api.ttnn_update_dense(run.state, dev, offset=off, extent=ext, lam=lam)
            T[tuple(slice(o, o + e) for o, e in zip(off, ext))] += lam * dq
        t = _otree(tr, dims, r, p)
        drm = O.Drm(t, 5, FMT[dtype])
        _compare_sketches(run, t, T, drm, 0, tol)
    finally:
        run.close()


def test_state_checkpoint_resume_and_axpy():
    tr, dims, r, p = CASES["binary4"]
    n = len(tr[0])
    T1, T2 = W.gaussian(dims, 1), W.gaussian(dims, 2)
    a = Run(tr, dims, [r] * n, [p] * n, 9, dtype=api.F64)
    b = Run(tr, dims, [r] * n, [p] * n, 9, dtype=api.F64)
    try:
        api.ttnn_update_dense(a.state, torch.from_numpy(T1).cuda())
        snap = a.state_host()
        api.ttnn_update_dense(a.state, torch.from_numpy(T2).cuda())
        full = a.state_host()
        api.ttnn_state_load(b.state, snap.copy())
        api.ttnn_update_dense(b.state, torch.from_numpy(T2).cuda())
        assert np.array_equal(b.state_host(), full)          # bitwise resume
        api.ttnn_state_zero(b.state)
        api.ttnn_update_dense(b.state, torch.from_numpy(T2).cuda(), lam=-1.0)
        api.ttnn_state_axpy(a.state, b.state, 1.0)           # a = S(T1) + S(T2) - S(T2)
        assert np.allclose(a.state_host(), snap, rtol=0, atol=1e-12 * np.abs(snap).max())
    finally:
        a.close()
        b.close()


def test_profiling_intervals_and_launch_counter():
    tr, dims, r, p = CASES["binary4"]
    n = len(tr[0])
    run = Run(tr, dims, [r] * n, [p] * n, 3, dtype=api.F32)
    try:
        T = torch.from_numpy(W.gaussian(dims, 4)).float().cuda()
        api.ttnn_profile(run.plan, True)
        l0 = api.ttnn_kernel_launches()
        for _ in range(2):
            api.ttnn_update_dense(run.state, T)
            run.recover()
        assert api.ttnn_kernel_launches() > l0
        for ph in range(3):
            ms, cnt = api.ttnn_profile_read(run.plan, ph)
            assert cnt == 2 and ms > 0
        assert api.ttnn_profile_read(run.plan, 0) == (0.0, 0)
        api.ttnn_profile(run.plan, False)
    finally:
        run.close()


TC_CASES = {
    # (tree, dims, r, p): pass-matrix sizes nL x nR are multiples of 8 so the
    # BF16 plans take the tensor-core pass; several 128-row blocks, ragged tails
    "bin5_960x960": (W.balanced_binary(5), [8, 12, 10, 24, 40], 4, 2),
    "bin5_512x1600": (W.balanced_binary(5), [8, 8, 8, 40, 40], 5, 3),
    "tt4_4096x24": (W.tensor_train(4), [16, 16, 16, 24], 6, 3),
    "bin4_r20": (W.balanced_binary(4), [16, 16, 32, 32], 20, 10),
    # four 1024-column chunks: the chunk CTAs form clusters and sum D1 on chip
    "bin4_64x4096": (W.balanced_binary(4), [8, 8, 64, 64], 6, 4),
    # three chunks: no cluster shape, partial sums through global memory
    "bin4_80x2560": (W.balanced_binary(4), [8, 10, 40, 64], 6, 4),
    # no left-side block (w_L = 0): the pass Y side is an identity leaf, so
    # the pass forms D1 only (TTNN; the STTNN plans keep both products)
    "tt4_wl0_1024x16": (W.tensor_train(4), [8, 16, 8, 16], 12, 6),
    "tucker4_wl0_3072x16": (W.tucker(4), [24, 16, 8, 16], 16, 8),
}


@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
@pytest.mark.parametrize("case", sorted(TC_CASES))
def test_tensor_core_pass_matches_oracle_and_simt(case, variant):
    tr, dims, r, p = TC_CASES[case]
    n = len(tr[0])
    T = W.gaussian(dims, 23)
    dev, Tq = _dev(T, api.BF16)
    tc = Run(tr, dims, [r] * n, [p] * n, 77, dtype=api.BF16, variant=variant)
    simt = Run(tr, dims, [r] * n, [p] * n, 77, dtype=api.BF16, variant=variant,
               flags=api.FLAG_SIMT_PASS)
    try:
        api.ttnn_profile(tc.plan, True)
        api.ttnn_update_dense(tc.state, dev)
        api.ttnn_update_dense(simt.state, dev)
        t = _otree(tr, dims, r, p)
        drm = O.Drm(t, 77, "bf16", "sttnn" if variant else "ttnn")
        assert api.ttnn_plan_pass_counts(tc.plan) == (1, 0)
        assert api.ttnn_plan_pass_counts(simt.plan) == (0, 1)
        _compare_sketches(tc, t, Tq, drm, variant, 1e-5)
        a, b = tc.state_host(), simt.state_host()
        assert rel(a, b) <= 1e-5
        # recovery reports no device-side timeout from the pass
        tc.recover()
    finally:
        tc.close()
        simt.close()


@pytest.mark.parametrize("case", ["tt4_wl0_1024x16", "tucker4_wl0_3072x16", "tt4_4096x24"])
def test_tensor_core_slices_match_oracle_and_simt(case):
    # one slice per mode (that mode fixed): slices whose pass matrix keeps
    # 16-byte rows take the tensor-core pass, with or without a D2 product
    tr, dims, r, p = TC_CASES[case]
    n = len(tr[0])
    t = _otree(tr, dims, r, p)
    drm = O.Drm(t, 31, "bf16", "ttnn")
    rng = np.random.default_rng(8)
    for mu in range(len(dims)):
        off, ext = [0] * len(dims), list(dims)
        off[mu], ext[mu] = int(rng.integers(0, dims[mu])), 1
        data = rng.standard_normal(ext)
        dev, dq = _dev(data, api.BF16)
        tc = Run(tr, dims, [r] * n, [p] * n, 31, dtype=api.BF16)
        simt = Run(tr, dims, [r] * n, [p] * n, 31, dtype=api.BF16, flags=api.FLAG_SIMT_PASS)
        try:
            api.ttnn_update_dense(tc.state, dev, off, ext, lam=0.5)
            api.ttnn_update_dense(simt.state, dev, off, ext, lam=0.5)
            if mu < len(dims) - 1:
                assert api.ttnn_plan_pass_counts(tc.plan) == (1, 0), mu
            _compare_sketches(tc, t, 0.5 * W.embed_box(dims, off, ext, dq), drm,
                              api.VARIANT_TTNN, 1e-5)
            assert rel(tc.state_host(), simt.state_host()) <= 1e-5
        finally:
            tc.close()
            simt.close()


def _pass_sides(tr, variant):
    """Modes of the two first-level pass sides: the root's children split
    into a left group (all but the last child for TTNN with three or more
    children, else the first child) and the rest."""
    ch, modes = W.children_of(tr[0], tr[1])
    kids = ch[list(tr[0]).index(-1)]
    a = 1 if variant == api.VARIANT_STTNN or len(kids) == 2 else len(kids) - 1
    left = sorted(m for c in kids[:a] for m in modes[c])
    right = sorted(m for c in kids[a:] for m in modes[c])
    return left, right


@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
@pytest.mark.parametrize("case", ["binary4", "toy6", "tt5"])
@pytest.mark.parametrize("dtype,tol", [(api.F64, 1e-12), (api.F32, 1e-5), (api.BF16, 1e-5)])
def test_rank_one_boxes_match_oracle(case, variant, dtype, tol):
    # boxes that fix every mode of one pass side: one product is rank one
    # (a broadcast in the walk), the other a matrix-vector product read
    # straight from the cached whole-tensor side block
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    left, right = _pass_sides(tr, variant)
    rng = np.random.default_rng(12)
    t = _otree(tr, dims, r, p)
    drm = O.Drm(t, 61, FMT[dtype], "sttnn" if variant else "ttnn")
    for fixed in (right, left):
        off = [int(rng.integers(0, d)) if mu in fixed else int(rng.integers(0, 2))
               for mu, d in enumerate(dims)]
        ext = [1 if mu in fixed else dims[mu] - off[mu] for mu in range(len(dims))]
        data = rng.standard_normal(ext)
        dev, dq = _dev(data, dtype)
        run = Run(tr, dims, [r] * n, [p] * n, 61, dtype=dtype, variant=variant)
        simt = Run(tr, dims, [r] * n, [p] * n, 61, dtype=dtype, variant=variant,
                   flags=api.FLAG_SIMT_PASS)
        try:
            api.ttnn_update_dense(run.state, dev, off, ext, lam=-1.5)
            api.ttnn_update_dense(simt.state, dev, off, ext, lam=-1.5)
            _compare_sketches(run, t, -1.5 * W.embed_box(dims, off, ext, dq), drm, variant, tol)
            assert rel(run.state_host(), simt.state_host()) <= tol
        finally:
            run.close()
            simt.close()


@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
def test_rank_deficient_recovery_truncates_like_oracle(variant):
    """True ranks 2 below the target 4 (no noise): Omega_v is rank deficient,
    the certified R^-1 path must refuse and the Jacobi eps-pseudo-inverse must
    drop the same directions as the oracle; the tensor is still reproduced."""
    tr = W.toy_tree()
    dims = [5, 4, 5, 4, 5, 4]
    n = len(tr[0])
    T, _ = W.exact_ttn(tr, dims, [2] * n, 3)
    run = Run(tr, dims, [4] * n, [3] * n, 9, dtype=api.F64, variant=variant)
    try:
        api.ttnn_update_dense(run.state, torch.from_numpy(T).cuda())
        cores = run.recover()
        t = _otree(tr, dims, 4, 3)
        drm = O.Drm(t, 9, "f64", "sttnn" if variant else "ttnn")
        sk = (O.sketch_ttnn if variant == 0 else OS.sketch_sttnn)(T, t, drm)
        _, kept = O.recover(t, *sk)
        truncated = 0
        for v in t.sketched():
            nd = run.nodes[v]
            assert nd["kept_rank"] == kept[v]
            if kept[v] < nd["r"]:
                truncated += 1
                assert nd["jacobi_sweeps"] > 0
        assert truncated > 0
        assert rel(O.reconstruct(t, cores), T) <= 1e-10
    finally:
        run.close()


@pytest.mark.parametrize("case", ["bin4_64x4096", "bin5_512x1600"])
def test_cluster_and_global_partial_sums_are_bitwise_equal(case):
    """The chunk partials of D1 are summed in the same order on chip (cluster)
    and by the last CTA of each row block through L2, so the two paths agree
    bit for bit."""
    tr, dims, r, p = TC_CASES[case]
    n = len(tr[0])
    dev, _ = _dev(W.gaussian(dims, 31), api.BF16)
    a = Run(tr, dims, [r] * n, [p] * n, 5, dtype=api.BF16)
    b = Run(tr, dims, [r] * n, [p] * n, 5, dtype=api.BF16, flags=api.FLAG_CLUSTER_REDUCE)
    try:
        api.ttnn_update_dense(a.state, dev)
        api.ttnn_update_dense(b.state, dev)
        assert np.array_equal(a.state_host(), b.state_host())
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_near_full_box_update(case):
    """A box one index short of the tensor on one mode generates its DRM
    blocks into the workspace (the cached whole-tensor blocks do not apply):
    the plan's workspace must hold it; the sketch matches the oracle."""
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    off = [0] * len(dims)
    ext = list(dims)
    off[-1], ext[-1] = 1, dims[-1] - 1
    B = W.gaussian(ext, 41)
    run = Run(tr, dims, [r] * n, [p] * n, 12, dtype=api.F64)
    try:
        api.ttnn_update_dense(run.state, torch.from_numpy(np.ascontiguousarray(B)).cuda(), off, ext)
        t = _otree(tr, dims, r, p)
        _compare_sketches(run, t, W.embed_box(dims, off, ext, B), O.Drm(t, 12, "f64"),
                          api.VARIANT_TTNN, 1e-12)
    finally:
        run.close()


def test_shard_state_tensor_aliases_the_state():
    """The tensor the all-reduce works on is the state itself: scaling it in
    place scales the sketches; with one rank the all-reduce is the identity."""
    from paper_2412_06111_gb300 import shard
    tr, dims, r, p = CASES["binary4"]
    n = len(tr[0])
    for dtype in (api.F64, api.F32):
        run = Run(tr, dims, [r] * n, [p] * n, 2, dtype=dtype)
        try:
            api.ttnn_update_dense(run.state, _dev(W.gaussian(dims, 3), dtype)[0])
            before = run.state_host()
            t = shard.state_tensor(run.plan, run.state)
            assert t.numel() == before.size
            assert np.array_equal(t.cpu().numpy().astype(np.float64), before)
            t.mul_(2.0)
            shard.allreduce_state_(run.plan, run.state)
            assert np.array_equal(run.state_host(), 2.0 * before)
        finally:
            run.close()
