"""eps-truncated output on the GPU (TTNN_FLAG_TRUNCATE): the directions the
eps-pseudo-inverse drops are cut from the cores (Sec. 4 recovery, eq.
(stabilized_nystrom)).  Core shapes against the oracle's truncated recovery,
reconstructions against the oracle and against the untruncated run.  All
calls go through the C ABI."""
import numpy as np
import pytest

import workloads as W
from oracle import sttnn as OS
from oracle import ttnn as O
from oracle.tree import Tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run, rel  # noqa: E402

CASES = {
    "toy6": (W.toy_tree(), [5, 4, 5, 4, 5, 4]),
    "binary5": (W.balanced_binary(5), [6, 7, 5, 8, 6]),
    "tt5": (W.tensor_train(5), [5, 4, 6, 4, 5]),
}


@pytest.mark.parametrize("variant", [api.VARIANT_TTNN, api.VARIANT_STTNN])
@pytest.mark.parametrize("case", sorted(CASES))
def test_truncated_cores_have_kept_ranks(case, variant):
    tr, dims = CASES[case]
    n = len(tr[0])
    T, _ = W.exact_ttn(tr, dims, [2] * n, 3)           # true ranks 2 below the targets 4
    t = Tree(tr[0], tr[1], dims, [4] * n, [3] * n, tr[2])
    cut = Run(tr, dims, [4] * n, [3] * n, 9, dtype=api.F64, variant=variant,
              flags=api.FLAG_TRUNCATE)
    full = Run(tr, dims, [4] * n, [3] * n, 9, dtype=api.F64, variant=variant)
    try:
        dev = torch.from_numpy(T).cuda()
        api.ttnn_update_dense(cut.state, dev)
        api.ttnn_update_dense(full.state, dev)
        gc, gf = cut.recover(), full.recover()
        vname = "sttnn" if variant else "ttnn"
        sk = (OS.sketch_sttnn if variant else O.sketch_ttnn)(T, t, O.Drm(t, 9, "f64", vname))
        oc, kept = O.recover(t, *sk, truncate=True)
        assert min(kept.values()) < 4
        for v in range(n):
            assert gc[v].shape == oc[v].shape, (v, gc[v].shape, oc[v].shape)
            if t.node(v).parent >= 0 and not t.node(v).identity:
                assert cut.nodes[v]["kept_rank"] == kept[v]
        rc = O.reconstruct(t, gc)
        assert rel(rc, O.reconstruct(t, oc)) <= 1e-10
        assert rel(rc, O.reconstruct(t, gf)) <= 1e-10
        assert rel(rc, T) <= 1e-10
        # fewer numbers than the padded cores
        assert sum(c.size for c in gc.values()) < sum(c.size for c in gf.values())
    finally:
        cut.close()
        full.close()


def test_truncation_is_a_no_op_at_full_rank():
    tr, dims = CASES["binary5"]
    n = len(tr[0])
    T = W.gaussian(dims, 4)
    cut = Run(tr, dims, [3] * n, [2] * n, 5, dtype=api.F64, flags=api.FLAG_TRUNCATE)
    full = Run(tr, dims, [3] * n, [2] * n, 5, dtype=api.F64)
    try:
        dev = torch.from_numpy(T).cuda()
        api.ttnn_update_dense(cut.state, dev)
        api.ttnn_update_dense(full.state, dev)
        gc, gf = cut.recover(), full.recover()
        for v in range(n):
            assert gc[v].shape == gf[v].shape
        t = Tree(tr[0], tr[1], dims, [3] * n, [2] * n, tr[2])
        assert rel(O.reconstruct(t, gc), O.reconstruct(t, gf)) <= 1e-12
    finally:
        cut.close()
        full.close()
