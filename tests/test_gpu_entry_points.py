"""Composite entry points on the GPU against the oracle: sttnn_run (one
dense STTNN sketch pass + recovery, Sec. 5) on several trees and formats.
All calls go through the C ABI."""
import numpy as np
import pytest

import workloads as W
from oracle import sttnn as OS
from oracle import ttnn as O
from oracle.quant import round_to
from oracle.tree import Tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import rel  # noqa: E402

CASES = {
    "toy6_f64": (W.toy_tree(), [3, 4, 3, 5, 4, 3], 2, 2, api.F64),
    "bin5_f32": (W.balanced_binary(5), [6, 7, 5, 8, 6], 4, 2, api.F32),
    "bin4_bf16_tc": (W.balanced_binary(4), [16, 16, 32, 32], 6, 4, api.BF16),
}
FMT = {api.F64: "f64", api.F32: "f32", api.BF16: "bf16"}
TDT = {api.F64: torch.float64, api.F32: torch.float32, api.BF16: torch.bfloat16}
# reconstruction tolerance: the task's 1e-10 for binary64 runs, 1e-4 otherwise
TOL = {api.F64: 1e-10, api.F32: 1e-4, api.BF16: 1e-4}


@pytest.mark.parametrize("case", sorted(CASES))
def test_sttnn_run_matches_oracle(case):
    tr, dims, r, p, dt = CASES[case]
    n = len(tr[0])
    T, _ = W.exact_ttn(tr, dims, [max(1, r - 1)] * n, 9)
    Tq = T if dt == api.F64 else round_to(round_to(T, "f32"), FMT[dt])
    plan = api.ttnn_plan_create(tr, dims, [r] * n, [p] * n, 55, variant=api.VARIANT_STTNN,
                                sketch_dtype=dt)
    try:
        ce = api.ttnn_plan_sizes(plan)[2]
        out = torch.zeros(ce, dtype=torch.float64, device="cuda")
        dev = torch.from_numpy(np.ascontiguousarray(Tq)).cuda().to(TDT[dt])
        api.sttnn_run(plan, dev, out)
        host = out.cpu().numpy()
        nodes = [api.ttnn_plan_node(plan, v) for v in range(n)]
        got = {nd["user_index"]: host[nd["core_offset"]:nd["core_offset"] + nd["core_elems"]]
               .reshape(nd["core_shape"]) for nd in nodes}
        t = Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])
        drm = O.Drm(t, 55, FMT[dt], "sttnn")
        want = O.recover(t, *OS.sketch_sttnn(Tq, t, drm))[0]
        rg, rw = O.reconstruct(t, got), O.reconstruct(t, want)
        assert rel(rg, rw) <= TOL[dt], rel(rg, rw)
        # binary64: TTN ranks r - 1 below the targets, so the recovery is exact
        if dt == api.F64:
            assert rel(rg, Tq) <= 1e-10
        if dt == api.BF16:
            assert api.ttnn_plan_pass_counts(plan) == (1, 0)
    finally:
        api.ttnn_plan_destroy(plan)
