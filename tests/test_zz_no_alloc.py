"""ttnn_update_dense_static (scratch in static device memory, no allocation)
against ttnn_update_dense on the same plan and inputs, through the C ABI.

Collected last on purpose: it must pass in a fresh process and after every
other test of the suite."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run, rel  # noqa: E402

TOL = {api.F64: 1e-12, api.F32: 1e-5, api.BF16: 1e-5}

CASES = {
    # tensor-core pass (BF16), whole tensor
    "bf16_bin4_r20": (W.balanced_binary(4), [16, 16, 32, 32], 20, 10, api.BF16, None),
    # SIMT pass (FP32), whole tensor
    "f32_bin5": (W.balanced_binary(5), [6, 7, 5, 8, 6], 4, 2, api.F32, None),
    # FP64 box update: the box's DRM blocks live in the scratch too
    "f64_toy6_box": (W.toy_tree(), [3, 4, 3, 5, 4, 3], 2, 2, api.F64,
                     ([1, 0, 1, 2, 0, 1], [2, 4, 2, 3, 3, 2])),
}


def _dev(T, dtype):
    t = torch.from_numpy(np.ascontiguousarray(T)).cuda()
    if dtype == api.F64:
        return t.double()
    if dtype == api.F32:
        return t.float()
    return t.float().to(torch.bfloat16)


@pytest.mark.parametrize("case", sorted(CASES))
def test_static_update_matches_update_dense_twice(case):
    tr, dims, r, p, dtype, box = CASES[case]
    n = len(tr[0])
    run = Run(tr, dims, [r] * n, [p] * n, 4242, dtype=dtype)
    other = api.ttnn_state_create(run.plan)
    try:
        for call, (seed, lam) in enumerate(((101, 1.0), (202, -0.75))):
            shape = dims if box is None else box[1]
            data = _dev(W.gaussian(shape, seed), dtype)
            off, ext = (None, None) if box is None else box
            api.ttnn_state_zero(run.state)
            api.ttnn_state_zero(other)
            api.ttnn_update_dense(other, data, off, ext, lam=lam)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            plan0 = api.ttnn_plan_device_bytes(run.plan)
            api.ttnn_update_dense_static(run.state, data, off, ext, lam=lam)
            torch.cuda.synchronize()
            if call == 1:
                # the second call (the block's address already known) allocates
                # nothing: device memory and the plan's footprint are unchanged
                assert torch.cuda.mem_get_info()[0] == free0
                assert api.ttnn_plan_device_bytes(run.plan) == plan0
            got = run.state_host()
            buf = np.zeros_like(got, dtype=np.float64 if run.sizes[1] == 8 else np.float32)
            api.ttnn_state_save(other, buf)
            want = buf.astype(np.float64)
            assert np.linalg.norm(want) > 0
            assert rel(got, want) <= TOL[dtype], (case, call, rel(got, want))
    finally:
        api.ttnn_state_destroy(other)
        run.close()


def test_static_update_rejects_oversized_scratch():
    # 96^4 BF16 with r = 20, p = 10 needs about 44 MiB of scratch (> 32 MiB)
    tr, dims = W.balanced_binary(4), [96, 96, 96, 96]
    n = len(tr[0])
    run = Run(tr, dims, [20] * n, [10] * n, 7, dtype=api.BF16)
    try:
        data = torch.zeros(dims, dtype=torch.bfloat16, device="cuda")
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_update_dense_static(run.state, data)
        assert ei.value.status == 1 and "scratch" in str(ei.value)
        torch.cuda.synchronize()
        assert not np.any(run.state_host())
    finally:
        run.close()
