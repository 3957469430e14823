"""Serving loop on the GPU: streams of different trees, sizes and formats
updated through one server (batched, walks merged across streams) end with
the same sketches, bit for bit, as the same updates applied alone with
ttnn_update_dense; recoveries on request match ttnn_recover; admission by
device memory; bounded waits.  All calls go through the C ABI."""
import numpy as np
import pytest

import workloads as W
from oracle import ttnn as O
from oracle.tree import Tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2412_06111_gb300 import api  # noqa: E402

from _lib_util import Run, rel  # noqa: E402

STREAMS = [
    # tree, dims, r, p, dtype
    (W.balanced_binary(4), [16, 16, 32, 32], 6, 3, api.BF16),
    (W.tensor_train(5), [6, 5, 7, 5, 6], 3, 2, api.F64),
    (W.tucker(4), [8, 9, 10, 8], 3, 2, api.F32),
    (W.toy_tree(), [4, 5, 4, 6, 5, 4], 2, 2, api.F32),
    (W.balanced_binary(5), [8, 12, 10, 24, 40], 4, 2, api.BF16),
]

TDT = {api.F64: torch.float64, api.F32: torch.float32, api.BF16: torch.bfloat16}
FMT = {api.F64: "f64", api.F32: "f32", api.BF16: "bf16"}
# sketches: binary64 summation order only; binary32 accumulation otherwise
SK_TOL = {api.F64: 1e-12, api.F32: 1e-5, api.BF16: 1e-5}
# reconstructions of the recovered TTN (the task's 1e-10 for binary64 runs,
# 1e-4 for the binary32-accumulated forms)
REC_TOL = {api.F64: 1e-10, api.F32: 1e-4, api.BF16: 1e-4}


def _oracle_check(j, work, state_host, cores_dev, plan):
    """The stream's state and recovered cores against the oracle run on the
    sum of its updates (each box embedded in zeros, data in the stream's
    number format, weighted by lambda: Sec. 4 streaming by linearity)."""
    tr, dims, r, p, dt = STREAMS[j]
    n = len(tr[0])
    t = Tree(tr[0], tr[1], dims, [r] * n, [p] * n, tr[2])
    H = np.zeros(dims)
    for off, ext, x, lam in work:
        xq = x.double().cpu().numpy()
        sl = tuple(slice(o, o + e) for o, e in zip(off, ext))
        H[sl] += lam * xq
    drm = O.Drm(t, 100 + j, FMT[dt])
    Om, Ps, Pr = O.sketch_ttnn(H, t, drm)
    nodes = [api.ttnn_plan_node(plan, v) for v in range(n)]
    for nd in nodes:
        v = nd["user_index"]
        if nd["parent"] < 0:
            got = state_host[nd["psi_offset"]:nd["psi_offset"] + nd["psi_elems"]]
            assert rel(got, Pr.ravel()) <= SK_TOL[dt], (j, "Psi_root")
            continue
        if nd["identity"]:
            continue
        om = state_host[nd["omega_offset"]:nd["omega_offset"] + nd["omega_elems"]]
        ps = state_host[nd["psi_offset"]:nd["psi_offset"] + nd["psi_elems"]]
        assert rel(om, Om[v].ravel()) <= SK_TOL[dt], (j, "Omega", v)
        assert rel(ps, Ps[v].ravel()) <= SK_TOL[dt], (j, "Psi", v)
    host = cores_dev.cpu().numpy()
    got = {nd["user_index"]: host[nd["core_offset"]:nd["core_offset"] + nd["core_elems"]]
           .reshape(nd["core_shape"]) for nd in nodes}
    want = O.recover(t, Om, Ps, Pr)[0]
    assert rel(O.reconstruct(t, got), O.reconstruct(t, want)) <= REC_TOL[dt], j


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
    # one worker: requests that arrive while it works queue up and are batched
    srv = api.ttnn_server_create(64 << 30, max_batch=8, workers=1)
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
            # and both equal the oracle's sketch and recovery of the same updates
            _oracle_check(j, work[j], got.astype(np.float64), cores_srv[j], alone[j].plan)
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


@pytest.mark.parametrize("cap,scap", [(3, 0), (0, 2)])
def test_back_pressure_bounds_outstanding_requests(cap, scap):
    # queue_capacity bounds the requests outstanding (queued or on the
    # device), stream_queue_capacity those of one stream: submits beyond
    # either are refused with EBUSY, the client waits
    # for its oldest ticket and submits again; no update is lost or applied
    # twice (the state equals the same updates applied alone)
    tr, dims, r, p, dt = STREAMS[4]
    n = len(tr[0])
    srv = api.ttnn_server_create(64 << 30, max_batch=4, queue_capacity=cap, workers=1,
                                 stream_queue_capacity=scap)
    alone = Run(tr, dims, [r] * n, [p] * n, 300, dtype=dt)
    rng = np.random.default_rng(3)
    try:
        sid = api.ttnn_server_open(srv, tr, dims, [r] * n, [p] * n, 300, sketch_dtype=dt)
        work = [(off, ext, torch.from_numpy(np.ascontiguousarray(x)).to("cuda", TDT[dt]), lam)
                for off, ext, x, lam in _slice_updates(dims, 40, rng)]
        outstanding, refused = [], 0
        for off, ext, x, lam in work:
            while True:
                try:
                    outstanding.append(api.ttnn_server_submit(srv, sid, x, off, ext, lam=lam))
                    break
                except api.TtnnError as e:
                    assert e.status == 6                   # EBUSY
                    assert len(outstanding) >= 1
                    refused += 1
                    assert api.ttnn_server_wait(srv, outstanding.pop(0)) == 0
            assert api.ttnn_server_stats(srv)["queued"] <= max(cap, scap)
        for t in outstanding:
            assert api.ttnn_server_wait(srv, t) == 0
        assert refused > 0
        for off, ext, x, lam in work:
            api.ttnn_update_dense(alone.state, x, off, ext, lam=lam)
        torch.cuda.synchronize()
        got = _state(alone.plan, api.ttnn_server_stream_state(srv, sid))
        want = _state(alone.plan, alone.state)
        assert np.array_equal(got, want)
        assert api.ttnn_server_stats(srv)["completed_updates"] == len(work)
    finally:
        api.ttnn_server_destroy(srv)
        alone.close()


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
    # room for one stream beside the library's 32 MiB static scratch block,
    # which the server counts against its budget
    srv = api.ttnn_server_create(need + need // 2 + (32 << 20))
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
