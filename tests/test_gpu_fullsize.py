"""Parity at the full benchmark size, in the configuration bench.py times:
the dense order-5 64^5 tensor 1/sum(x) on [1,2]^5 (binary64 -> binary32 ->
bfloat16, as the bench builds it), balanced binary tree ((0,1),2),(3,4),
r = 20, p = 10, BF16 plan (tcgen05 first-level pass), TTNN.  Every sketch is
compared with the oracle run on the same tensor, then the recovered cores'
reconstructions are compared.  Needs ~30 GB of host memory and a minute or
two of host time for the oracle."""
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

D, N, RANK, OVER, SEED = 5, 64, 20, 10, 2024   # the bench configuration


@pytest.mark.timeout(1200)
def test_full_size_bf16_sketches_and_recovery_match_oracle():
    tr = W.balanced_binary(D)
    n = len(tr[0])
    dims = [N] * D
    # input: built on the host, rounded as the bench rounds it
    T = round_to(round_to(W.inv_sum(D, N), "f32"), "bf16")
    dev = torch.from_numpy(T.astype(np.float32)).cuda().to(torch.bfloat16)
    run = Run(tr, dims, [RANK] * n, [OVER] * n, SEED, dtype=api.BF16)
    try:
        api.ttnn_update_dense(run.state, dev)
        assert api.ttnn_plan_pass_counts(run.plan) == (1, 0)
        del dev
        torch.cuda.empty_cache()
        gOm, gPs, gPr = run.sketches()
        cores = run.recover()
        t = Tree(tr[0], tr[1], dims, [RANK] * n, [OVER] * n, tr[2])
        drm = O.Drm(t, SEED, "bf16")
        Om, Ps, Pr = O.sketch_ttnn(T, t, drm)
        worst = max(max(rel(gOm[v], Om[v]), rel(gPs[v], Ps[v])) for v in t.sketched())
        worst = max(worst, rel(gPr, Pr))
        # binary32 accumulation over up to 2^18 terms per product
        assert worst <= 2e-5, worst
        want = O.reconstruct(t, O.recover(t, Om, Ps, Pr)[0])
        got = O.reconstruct(t, cores)
        assert rel(got, want) <= 1e-4, rel(got, want)
        # the approximation error itself is the method's, not the kernels':
        # the GPU and the oracle land on the same value (about 2e-2 here, the
        # bfloat16 storage noise of the input amplified by the recovery)
        assert abs(rel(got, T) - rel(want, T)) <= 1e-3 * rel(want, T)
    finally:
        run.close()
