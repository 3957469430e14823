"""Failure paths on the GPU, made without a GPU fault: a device wait that is
given no time at all (TTNN_FLAG_WAIT_TEST) and device allocations that fail
on request (ttnn_debug_fail_alloc).  Each test checks the status the library
returns, that nothing was changed, and that the CUDA context is still usable
afterwards.  All calls go through the C ABI."""
import numpy as np
import pytest

import workloads as W
from oracle import rounding as OR
from oracle import ttnn as O
from oracle.quant import round_to
from oracle.tree import Tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run, rel  # noqa: E402

ENOMEM, ETIMEOUT = 2, 5


def _otree(tr, dims, r, p):
    n = len(tr[0])
    return Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])


def test_pass_wait_running_out_reports_timeout_and_context_survives():
    tr, dims, r, p = W.balanced_binary(4), [16, 16, 32, 32], 6, 4
    n = len(tr[0])
    T = W.gaussian(dims, 5)
    Tq = round_to(round_to(T, "f32"), "bf16")
    dev = torch.from_numpy(Tq.astype(np.float32)).cuda().to(torch.bfloat16)
    bad = Run(tr, dims, [r] * n, [p] * n, 3, dtype=api.BF16, flags=api.FLAG_WAIT_TEST)
    good = Run(tr, dims, [r] * n, [p] * n, 3, dtype=api.BF16)
    try:
        api.ttnn_update_dense(bad.state, dev)
        assert api.ttnn_plan_pass_counts(bad.plan) == (1, 0)
        core = torch.zeros(bad.sizes[2], dtype=torch.float64, device="cuda")
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_recover(bad.state, core)
        assert ei.value.status == ETIMEOUT
        # reported once: the device word was cleared
        api.ttnn_plan_sync(bad.plan)
        # the context is intact: a normal plan on the same data matches the oracle
        api.ttnn_update_dense(good.state, dev)
        t = _otree(tr, dims, r, p)
        Om, Ps, Pr = O.sketch_ttnn(Tq, t, O.Drm(t, 3, "bf16"))
        gOm, gPs, gPr = good.sketches()
        for v in Om:
            assert rel(gOm[v], Om[v]) <= 1e-5 and rel(gPs[v], Ps[v]) <= 1e-5
        assert rel(gPr, Pr) <= 1e-5
        good.recover()
    finally:
        bad.close()
        good.close()


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_injected_allocation_failures_in_plan_creation():
    tr, dims, r, p = W.balanced_binary(4), [16, 16, 32, 32], 6, 4
    n = len(tr[0])

    def sweep():
        k = 1
        while True:
            api.ttnn_debug_fail_alloc(k)
            try:
                plan = api.ttnn_plan_create(tr, dims, [r] * n, [p] * n, 3, sketch_dtype=api.BF16)
            except api.TtnnError as e:
                assert e.status == ENOMEM and "injected" in str(e)
                k += 1
                assert k < 64
                continue
            api.ttnn_debug_fail_alloc(0)
            api.ttnn_plan_destroy(plan)
            return k

    try:
        k1 = sweep()
        before = _free_bytes()
        k2 = sweep()
        after = _free_bytes()
    finally:
        api.ttnn_debug_fail_alloc(0)
    # every allocation of a plan was made to fail once; nothing leaked
    assert k1 == k2 and k1 >= 5
    assert before - after <= (4 << 20)


def test_injected_allocation_failure_leaves_state_unchanged():
    """A TTN-format update whose workspace must grow: the failed growth
    returns ENOMEM, launches nothing and keeps the plan's old workspace; the
    same update then succeeds and matches the oracle."""
    tr, dims, r, p = W.balanced_binary(5), [6, 7, 5, 8, 6], 4, 2
    n = len(tr[0])
    rng = np.random.default_rng(21)
    cores = W.ttn_cores(tr, dims, [24] * n, rng)
    dcores = [torch.from_numpy(np.ascontiguousarray(cores[v])).cuda() for v in range(n)]
    run = Run(tr, dims, [r] * n, [p] * n, 42, dtype=api.F64, flags=api.FLAG_STRUCTURED_ONLY)
    try:
        # a first, small update fills the state
        small = W.ttn_cores(tr, dims, [1] * n, np.random.default_rng(3))
        api.ttnn_update_ttn(run.state, [torch.from_numpy(np.ascontiguousarray(small[v])).cuda()
                                        for v in range(n)], [1] * n)
        before = run.state_host().copy()
        ws0 = api.ttnn_plan_device_bytes(run.plan)[1]
        api.ttnn_debug_fail_alloc(1)
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_update_ttn(run.state, dcores, [24] * n)
        api.ttnn_debug_fail_alloc(0)
        assert ei.value.status == ENOMEM
        assert np.array_equal(run.state_host(), before)
        assert api.ttnn_plan_device_bytes(run.plan)[1] == ws0
        api.ttnn_update_ttn(run.state, dcores, [24] * n)
        assert api.ttnn_plan_device_bytes(run.plan)[1] > ws0
        t = _otree(tr, dims, r, p)
        drm = O.Drm(t, 42, "f64", "round")
        a = OR.sketch_ttn_input(small, t, drm)
        b = OR.sketch_ttn_input(cores, t, drm)
        Om, Ps, Pr = run.sketches()
        for v in a[0]:
            assert rel(Om[v], a[0][v] + b[0][v]) <= 1e-12
            assert rel(Ps[v], a[1][v] + b[1][v]) <= 1e-12
        assert rel(Pr, a[2] + b[2]) <= 1e-12
        # state creation under injection
        api.ttnn_debug_fail_alloc(1)
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_state_create(run.plan)
        assert ei.value.status == ENOMEM
    finally:
        api.ttnn_debug_fail_alloc(0)
        run.close()
