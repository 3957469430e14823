"""Parity of the streamed order-6 workload at full size: a 32^6 tensor that
arrives as additive updates, each one rank-2 CP term (N(0,1) factors) plus
one dense 32^3 box of N(0, 0.01) noise on three random modes (BF16 data),
tensor-train (caterpillar) tree, r = 16, p = 8, BF16 plan, 256 updates
through ttnn_update_cp / ttnn_update_dense.  The accumulated sketches are
compared with the oracle's sketches of the summed dense tensor (Sec. 4:
streaming by linearity), then the recovered cores' reconstructions.

The two kinds of update use the plan's DRM as the library defines it: a
dense box multiplies the stored Khatri-Rao blocks on the tensor cores, a CP
term uses the stored per-mode factors with exact Khatri-Rao products (the
oracle's Drm variants "ttnn" and "round").  Needs ~40 GB of host memory."""
import numpy as np
import pytest

import workloads as W
from oracle import ttnn as O
from oracle.quant import round_to
from oracle.tree import Tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run, rel  # noqa: E402

D, N, R, P, SEED, NUPD = 6, 32, 16, 8, 2027, 256


@pytest.mark.timeout(1500)
def test_streamed_cp_plus_box_updates_match_oracle_full_size():
    tr = W.tensor_train(D)
    n = len(tr[0])
    dims = [N] * D
    ups = W.streaming_updates(dims, NUPD, 1003)
    run = Run(tr, dims, [R] * n, [P] * n, SEED, dtype=api.BF16)
    try:
        boxes = []
        for u in ups:
            fac = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in u["cp_factors"]]
            api.ttnn_update_cp(run.state, list(u["cp_weights"]), fac)
            b = torch.from_numpy(np.ascontiguousarray(u["box_data"])).cuda().to(torch.bfloat16)
            api.ttnn_update_dense(run.state, b, u["box_offset"], u["box_extent"])
            boxes.append(b.double().cpu().numpy())
        gOm, gPs, gPr = run.sketches()
        cores = run.recover()
    finally:
        run.close()
    t = Tree(tr[0], tr[1], dims, [R] * n, [P] * n, tr[2])
    # the CP terms summed: one CP tensor of rank 2 * NUPD, formed as one
    # product of two Khatri-Rao matrices (modes 0-2 x modes 3-5)
    A = [np.hstack([u["cp_factors"][mu] * np.asarray(u["cp_weights"])[None, :] if mu == 0
                    else u["cp_factors"][mu] for u in ups]) for mu in range(D)]
    T = (O.kr(A[:3]) @ O.kr(A[3:]).T).reshape(dims)
    cOm, cPs, cPr = O.sketch_ttnn(T, t, O.Drm(t, SEED, "bf16", "round"))
    T[...] = 0.0
    for u, b in zip(ups, boxes):
        sl = tuple(slice(o, o + e) for o, e in zip(u["box_offset"], u["box_extent"]))
        T[sl] += b
    bOm, bPs, bPr = O.sketch_ttnn(T, t, O.Drm(t, SEED, "bf16", "ttnn"))
    Om = {v: cOm[v] + bOm[v] for v in cOm}
    Ps = {v: cPs[v] + bPs[v] for v in cPs}
    Pr = cPr + bPr
    # binary32 accumulation of 256 updates' contributions
    worst = max(max(rel(gOm[v], Om[v]), rel(gPs[v], Ps[v])) for v in t.sketched())
    worst = max(worst, rel(gPr, Pr))
    assert worst <= 1e-5, worst
    del T
    want = O.reconstruct(t, O.recover(t, Om, Ps, Pr)[0])
    got = O.reconstruct(t, cores)
    assert rel(got, want) <= 1e-4, rel(got, want)
    # the boxes really were bfloat16 values (the data the oracle saw)
    assert all(np.array_equal(b, round_to(b, "bf16")) for b in boxes[:4])
