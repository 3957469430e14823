"""Unstructured Gaussian DRMs on the GPU (TTNN_FLAG_DENSE_DRM): every node
draws its own X_t, Y_t (Sec. 4 eq. (sketch)), as Thm 6.6 assumes.  Sketches
and recoveries against the oracle's DenseDrm, the expected error bound of
Thm 6.6 over 30 seeds of GPU runs, and the updates this form refuses.  All
calls go through the C ABI."""
import numpy as np
import pytest

import workloads as W
from oracle import bounds as BD
from oracle import ttnn as O
from oracle.tree import Tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run, rel  # noqa: E402

CASES = {
    "binary4": (W.balanced_binary(4), [7, 5, 6, 4], 3, 2),
    "toy6": (W.toy_tree(), [3, 4, 3, 5, 4, 3], 2, 2),
    "tt5": (W.tensor_train(5), [4, 3, 5, 3, 4], 2, 1),
    "tucker4": (W.tucker(4), [5, 4, 6, 3], 2, 2),
    "binary5": (W.balanced_binary(5), [6, 7, 5, 8, 6], 4, 2),
}
FMT = {api.F64: "f64", api.F32: "f32"}
TDT = {api.F64: torch.float64, api.F32: torch.float32}


def _otree(tr, dims, r, p):
    n = len(tr[0])
    return Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])


@pytest.mark.parametrize("dtype,tol", [(api.F64, 1e-12), (api.F32, 1e-5)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_dense_drm_sketches_match_oracle(case, dtype, tol):
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    T = W.gaussian(dims, 17)
    Tq = T if dtype == api.F64 else T.astype(np.float32).astype(np.float64)
    run = Run(tr, dims, [r] * n, [p] * n, 99, dtype=dtype, flags=api.FLAG_DENSE_DRM)
    try:
        api.ttnn_update_dense(run.state, torch.from_numpy(np.ascontiguousarray(Tq)).to("cuda", TDT[dtype]),
                              lam=-0.75)
        t = _otree(tr, dims, r, p)
        Om, Ps, Pr = O.sketch_ttnn(Tq, t, O.DenseDrm(t, 99, FMT[dtype]))
        gOm, gPs, gPr = run.sketches()
        for v in Om:
            assert rel(gOm[v], -0.75 * Om[v]) <= tol, ("Omega", v)
            assert rel(gPs[v], -0.75 * Ps[v]) <= tol, ("Psi", v)
        assert rel(gPr, -0.75 * Pr) <= tol
        # the Khatri-Rao plan of the same seed sketches something else
        kr = O.sketch_ttnn(Tq, t, O.Drm(t, 99, FMT[dtype]))
        v = t.sketched()[0]
        assert rel(kr[0][v], Om[v]) > 0.1
    finally:
        run.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_dense_drm_recovery_matches_oracle_f64(case):
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    T, _ = W.exact_ttn(tr, dims, [max(1, r - 1)] * n, 5, noise=1e-3)
    run = Run(tr, dims, [r] * n, [p] * n, 7, dtype=api.F64, flags=api.FLAG_DENSE_DRM)
    try:
        api.ttnn_update_dense(run.state, torch.from_numpy(T).cuda())
        cores = run.recover()
        t = _otree(tr, dims, r, p)
        oc, kept = O.recover(t, *O.sketch_ttnn(T, t, O.DenseDrm(t, 7)))
        assert rel(O.reconstruct(t, cores), O.reconstruct(t, oc)) <= 1e-10
        for v in t.sketched():
            assert run.nodes[v]["kept_rank"] == kept[v]
    finally:
        run.close()


def test_expected_error_bound_thm_6_6_on_gpu_runs():
    """Mean error of 30 GPU recoveries with independent Gaussian DRMs (seeds
    500..529) below the right-hand side of Thm 6.6 (r^ = 2 < r - 1 = 3,
    p = 3 >= 2), each run equal to the oracle's."""
    tr = W.balanced_binary(3)
    dims = [8, 8, 8]
    T, _ = W.exact_ttn(tr, dims, [3] * 5, 5, noise=0.2)
    t = _otree(tr, dims, 4, 3)
    rhat = {v: 2 for v in t.sketched()}
    dev = torch.from_numpy(T).cuda()
    errs = []
    for seed in range(30):
        run = Run(tr, dims, [4] * 5, [3] * 5, 500 + seed, dtype=api.F64, flags=api.FLAG_DENSE_DRM)
        try:
            api.ttnn_update_dense(run.state, dev)
            R = O.reconstruct(t, run.recover())
        finally:
            run.close()
        oc, _ = O.recover(t, *O.sketch_ttnn(T, t, O.DenseDrm(t, 500 + seed)))
        assert rel(R, O.reconstruct(t, oc)) <= 1e-10
        errs.append(np.linalg.norm(R - T))
    assert np.mean(errs) <= BD.expected(T, t, rhat)


def test_dense_drm_refused_updates_and_plans():
    tr, dims, r, p = CASES["binary4"]
    n = len(tr[0])
    with pytest.raises(api.TtnnError) as ei:          # narrow formats use tensor-core blocks
        api.ttnn_plan_create(tr, dims, [r] * n, [p] * n, 1, sketch_dtype=api.BF16,
                             flags=api.FLAG_DENSE_DRM)
    assert ei.value.status == 7
    with pytest.raises(api.TtnnError) as ei:          # STTNN contracts per-mode groups
        api.ttnn_plan_create(tr, dims, [r] * n, [p] * n, 1, sketch_dtype=api.F64,
                             variant=api.VARIANT_STTNN, flags=api.FLAG_DENSE_DRM)
    assert ei.value.status == 7
    run = Run(tr, dims, [r] * n, [p] * n, 1, dtype=api.F64, flags=api.FLAG_DENSE_DRM)
    try:
        box = torch.zeros([2, 2, 2, 2], dtype=torch.float64, device="cuda")
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_update_dense(run.state, box, [0, 0, 0, 0], [2, 2, 2, 2])
        assert ei.value.status == 7
        fac = [torch.zeros(m, 1, dtype=torch.float64, device="cuda") for m in dims]
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_update_cp(run.state, [1.0], fac)
        assert ei.value.status == 7
        torch.cuda.synchronize()
        assert not np.any(run.state_host())
    finally:
        run.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_ttn_hmt_matches_oracle(case):
    """TTN-HMT (Sec. 8 comparator) on the GPU: Householder range finders on
    the plan's unstructured sketches, cores against the oracle's (compared
    through their reconstructions), exact for TTN ranks at the targets."""
    from oracle import baselines as B
    tr, dims, r, p = CASES[case]
    n = len(tr[0])
    t = _otree(tr, dims, r, p)
    run = Run(tr, dims, [r] * n, [p] * n, 13, dtype=api.F64, flags=api.FLAG_DENSE_DRM)
    try:
        for T in (W.gaussian(dims, 5), W.exact_ttn(tr, dims, [r] * n, 6)[0]):
            out = torch.zeros(run.sizes[2], dtype=torch.float64, device="cuda")
            api.ttnn_hmt(run.plan, torch.from_numpy(T).cuda(), out)
            host = out.cpu().numpy()
            got = {nd["user_index"]: host[nd["core_offset"]:nd["core_offset"] + nd["core_elems"]]
                   .reshape(nd["core_shape"]) for nd in run.nodes}
            want = B.ttn_hmt(T, t, O.DenseDrm(t, 13))
            rg = O.reconstruct(t, got)
            assert rel(rg, O.reconstruct(t, want)) <= 1e-10
        assert rel(rg, T) <= 1e-10            # the exact-rank tensor
    finally:
        run.close()


def test_hilbert_ttnn_sttnn_hmt_against_oracle():
    """The paper's first experiment in miniature (Hilbert 1/(1 + sum i),
    example tree, Gaussian sketches): TTNN with unstructured DRMs and TTN-HMT
    on the GPU equal the oracle's; the errors of both, and of TTN-SVD, are
    the paper's comparison (TTN-HMT slightly more accurate than TTNN)."""
    from oracle import baselines as B
    tr = W.toy_tree()
    n = len(tr[0])
    dims = [10] * 6
    T = W.hilbert(6, 10)
    r, p = 5, 5
    t = _otree(tr, dims, r, p)
    run = Run(tr, dims, [r] * n, [p] * n, 21, dtype=api.F64, flags=api.FLAG_DENSE_DRM)
    try:
        dev = torch.from_numpy(T).cuda()
        api.ttnn_update_dense(run.state, dev)
        g_ttnn = O.reconstruct(t, run.recover())
        out = torch.zeros(run.sizes[2], dtype=torch.float64, device="cuda")
        api.ttnn_hmt(run.plan, dev, out)
        host = out.cpu().numpy()
        g_hmt = O.reconstruct(t, {nd["user_index"]: host[nd["core_offset"]:nd["core_offset"] +
                                                            nd["core_elems"]].reshape(nd["core_shape"])
                                  for nd in run.nodes})
    finally:
        run.close()
    drm = O.DenseDrm(t, 21)
    o_ttnn = O.reconstruct(t, O.recover(t, *O.sketch_ttnn(T, t, drm))[0])
    o_hmt = O.reconstruct(t, B.ttn_hmt(T, t, drm))
    assert rel(g_ttnn, o_ttnn) <= 1e-8 and rel(g_hmt, o_hmt) <= 1e-10
    e_svd = rel(B.hsvd(T, t), T)
    e_ttnn, e_hmt = rel(g_ttnn, T), rel(g_hmt, T)
    # every method is at least as far from T as the quasi-optimal TTN-SVD
    # allows (within sqrt(#edges) of the best approximation of these ranks)
    assert min(e_ttnn, e_hmt) >= e_svd / np.sqrt(n - 1)
