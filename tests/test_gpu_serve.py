"""Serving loop on the GPU: streams of different trees, sizes and formats
updated through one server (batched, walks merged across streams) end with
the same sketches, bit for bit, as the same updates applied alone with
ttnn_update_dense; recoveries on request match ttnn_recover; admission by
device memory; bounded waits.  All calls go through the C ABI."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run  # noqa: E402

STREAMS = [
    # tree, dims, r, p, dtype
    (W.balanced_binary(4), [16, 16, 32, 32], 6, 3, api.BF16),
    (W.tensor_train(5), [6, 5, 7, 5, 6], 3, 2, api.F64),
    (W.tucker(4), [8, 9, 10, 8], 3, 2, api.F32),
    (W.toy_tree(), [4, 5, 4, 6, 5, 4], 2, 2, api.F32),
    (W.balanced_binary(5), [8, 12, 10, 24, 40], 4, 2, api.BF16),
]

TDT = {api.F64: torch.float64, api.F32: torch.float32, api.BF16: torch.bfloat16}


def _slice_updates(dims, k, rng):
    """k updates: slices (one mode fixed) and small boxes, N(0,1) data."""
    out = []
    for i in range(k):
        d = len(dims)
        if i % 2 == 0:
            mu = int(rng.integers(0, d))
            off = [0] * d
            ext = list(dims)
            off[mu] = int(rng.integers(0, dims[mu]))
            ext[mu] = 1
        else:
            ext = [int(rng.integers(1, n + 1)) for n in dims]
            off = [int(rng.integers(0, n - e + 1)) for n, e in zip(dims, ext)]
        out.append((off, ext, rng.standard_normal(ext), float(rng.uniform(0.5, 1.5))))
    return out


def _state(plan, st):
    n, eb, _, _ = api.ttnn_plan_sizes(plan)
    buf = np.zeros(n, dtype=np.float64 if eb == 8 else np.float32)
    api.ttnn_state_save(st, buf)
    return buf


def test_mixed_streams_equal_alone_bitwise():
    srv = api.ttnn_server_create(64 << 30, max_batch=8)
    rng = np.random.default_rng(0)
    alone, sids, work = [], [], []
    try:
        for j, (tr, dims, r, p, dt) in enumerate(STREAMS):
            n = len(tr[0])
            sids.append(api.ttnn_server_open(srv, tr, dims, [r] * n, [p] * n, 100 + j,
                                             sketch_dtype=dt))
            alone.append(Run(tr, dims, [r] * n, [p] * n, 100 + j, dtype=dt))
            ups = _slice_updates(dims, 12, rng)
            work.append([(off, ext, torch.from_numpy(np.ascontiguousarray(x)).to("cuda", TDT[dt]), lam)
                         for off, ext, x, lam in ups])
        # interleave the streams' requests; keep tickets and data alive
        tickets = []
        for i in range(12):
            for j in range(len(STREAMS)):
                off, ext, x, lam = work[j][i]
                tickets.append(api.ttnn_server_submit(srv, sids[j], x, off, ext, lam=lam))
        cores_srv = []
        for j in range(len(STREAMS)):
            ce = api.ttnn_plan_sizes(alone[j].plan)[2]
            c = torch.zeros(ce, dtype=torch.float64, device="cuda")
            cores_srv.append(c)
            tickets.append(api.ttnn_server_recover(srv, sids[j], c))
        for t in tickets:
            assert api.ttnn_server_wait(srv, t) == 0
        # the same updates alone, in the same order
        for j in range(len(STREAMS)):
            for off, ext, x, lam in work[j]:
                api.ttnn_update_dense(alone[j].state, x, off, ext, lam=lam)
        torch.cuda.synchronize()
        for j in range(len(STREAMS)):
            got = _state(alone[j].plan, api.ttnn_server_stream_state(srv, sids[j]))
            want = _state(alone[j].plan, alone[j].state)
            assert np.array_equal(got, want), j
            ce = api.ttnn_plan_sizes(alone[j].plan)[2]
            c = torch.zeros(ce, dtype=torch.float64, device="cuda")
            api.ttnn_recover(alone[j].state, c)
            assert torch.equal(c, cores_srv[j]), j
        rep = api.ttnn_server_stats(srv)
        assert rep["completed_updates"] == 12 * len(STREAMS)
        assert rep["completed_recoveries"] == len(STREAMS)
        assert rep["failed"] == 0 and rep["open_streams"] == len(STREAMS)
        # batches merged several streams' walks
        assert rep["batches"] < rep["completed_updates"] + rep["completed_recoveries"]
    finally:
        api.ttnn_server_destroy(srv)
        for a in alone:
            a.close()


def test_admission_by_device_memory_and_close():
    tr, dims, r, p, dt = STREAMS[0]
    n = len(tr[0])
    probe = api.ttnn_server_create(64 << 30)
    try:
        s0 = api.ttnn_server_open(probe, tr, dims, [r] * n, [p] * n, 1, sketch_dtype=dt)
        need = api.ttnn_server_stats(probe)["device_bytes"]
        assert need > 0
        api.ttnn_server_close(probe, s0)
        assert api.ttnn_server_stats(probe)["device_bytes"] == 0
    finally:
        api.ttnn_server_destroy(probe)
    srv = api.ttnn_server_create(need + need // 2)       # room for one stream
    try:
        a = api.ttnn_server_open(srv, tr, dims, [r] * n, [p] * n, 1, sketch_dtype=dt)
        with pytest.raises(api.TtnnError) as ei:
            api.ttnn_server_open(srv, tr, dims, [r] * n, [p] * n, 2, sketch_dtype=dt)
        assert ei.value.status == 6                        # EBUSY
        api.ttnn_server_close(srv, a)
        b = api.ttnn_server_open(srv, tr, dims, [r] * n, [p] * n, 2, sketch_dtype=dt)
        assert b != a
    finally:
        api.ttnn_server_destroy(srv)


def test_request_errors_and_bounded_waits():
    tr, dims, r, p, dt = STREAMS[2]
    n = len(tr[0])
    srv = api.ttnn_server_create(64 << 30)
    try:
        s = api.ttnn_server_open(srv, tr, dims, [r] * n, [p] * n, 5, sketch_dtype=dt)
        x = torch.zeros(dims, dtype=torch.float32, device="cuda")
        with pytest.raises(api.TtnnError) as ei:          # box outside the tensor
            api.ttnn_server_submit(srv, s, x, [1, 0, 0, 0], dims)
        assert ei.value.status == 1
        with pytest.raises(api.TtnnError) as ei:          # unknown stream
            api.ttnn_server_submit(srv, s + 7, x)
        assert ei.value.status == 1
        with pytest.raises(api.TtnnError) as ei:          # unknown ticket
            api.ttnn_server_wait(srv, 123456, 1000)
        assert ei.value.status == 1
        t = api.ttnn_server_submit(srv, s, x)
        assert api.ttnn_server_wait(srv, t, 5_000_000) == 0
        with pytest.raises(api.TtnnError) as ei:          # reported once
            api.ttnn_server_wait(srv, t, 1000)
        assert ei.value.status == 1
    finally:
        api.ttnn_server_destroy(srv)
