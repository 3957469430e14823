"""Benchmark of the TTNN sketching hot path on one GB300 (or N, weak scaling).

Workload: dense order-5 tensor 64^5 (1.07e9 entries) sampled from
f(x) = 1/(x_1 + ... + x_5) on the uniform grid of [1, 2]^5, generated on the
device and resident in HBM (2.1 GB as BF16, 4.3 GB as FP32 -- larger than the
129 MB L2, so no flush is needed between steps); balanced binary tree
((1,2),3),(4,5); target ranks 20, oversampling 10.

One step = one pass of the whole hot path over the tensor: ttnn_update_dense
(first-level pass, tree walk, accumulation) + ttnn_recover (FP64 QR,
eps-pseudo-inverse, core assembly).  The headline `value` is the BF16 form's
tensor bytes streamed per second; the FP32 plain form and STTNN (BF16) are
measured the same way and reported beside it.

--impl reference times the FP64 CPU oracle (the reference arm)
on a bounded sample of the same workload on the host cores.
"""
import argparse
import collections
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D, NMODE, RANK, OVERSAMPLE, SEED = 5, 64, 20, 10, 2024
METRIC = "TTNN sketch GB/s streamed (% roofline) BF16 vs FP32; p50/p99 update latency"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), float(j["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _pass_traffic():
    """DRAM bytes per pass_kernel launch from the committed ncu summary, or
    None once the kernel's sources differ from the ones that were profiled."""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    prof = os.path.join(root, "profiles", "pass_kernel_64p5_bf16.md")
    h = hashlib.sha256()
    try:
        text = open(prof).read()
        for f in ("pass_tc.cu", "tc_ptx.cuh"):
            h.update(open(os.path.join(root, "paper_2412_06111_gb300", "csrc", f), "rb").read())
    except OSError:
        return None
    digest = h.hexdigest()
    vals = {}
    for line in text.splitlines():
        key, sep, val = line.partition(": ")
        if sep and key in ("traffic-bytes-per-launch", "source-sha256-prefix"):
            vals[key] = val.strip()
    prefix = vals.get("source-sha256-prefix", "")
    if not prefix or not digest.startswith(prefix):
        return None
    try:
        return int(vals["traffic-bytes-per-launch"])
    except (KeyError, ValueError):
        return None


def _dist():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, ws


def _barrier(ws):
    import torch
    if ws > 1:
        torch.distributed.barrier()


def _max_over_ranks(x, ws):
    import torch
    if ws == 1:
        return x
    # NCCL reduces device tensors; gloo (CPU ranks) host tensors
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


SAMPLES, SAMPLE_SEED = 20000, 77


def _ttn_sample_error(api, plan, tree, cores_dev, ws, rank):
    """Final relative error of the recovered TTN against the exact binary64
    values of 1/sum(x) at SAMPLES seeded indices (host evaluation of the
    cores: leaf slices, then each transfer tensor against its children)."""
    parent, leaf_modes, _ = tree
    nn = len(parent)
    nodes = [api.ttnn_plan_node(plan, v) for v in range(nn)]
    host = cores_dev.cpu().numpy()
    dims, _ = _geometry(ws, rank)
    rng = np.random.default_rng(SAMPLE_SEED)
    idx = np.stack([rng.integers(0, dims[m], size=SAMPLES) for m in range(D)], axis=1)
    grid = np.stack([idx[:, m] / (dims[m] - 1) for m in range(D)], axis=1)
    exact = 1.0 / (1.0 + grid).sum(axis=1)
    ch = {v: sorted([c for c in range(nn) if parent[c] == v], key=lambda c: nodes[c]["mode_lo"])
          for v in range(nn)}
    letters = "bcdefghijk"

    def val(v):
        nd = nodes[v]
        core = host[nd["core_offset"]:nd["core_offset"] + nd["core_elems"]].reshape(nd["core_shape"])
        if not ch[v]:
            lo, hi = nd["mode_lo"], nd["mode_hi"]
            flat = np.ravel_multi_index(tuple(idx[:, lo:hi].T), [dims[m] for m in range(lo, hi)])
            return core.reshape(core.shape[0], -1)[:, flat].T
        vecs = [val(c) for c in ch[v]]
        m = len(vecs)
        head = "" if parent[v] < 0 else "a"
        spec = head + letters[:m] + "," + ",".join("s" + letters[k] for k in range(m)) + "->s" + head
        return np.einsum(spec, core, *vecs, optimize=True)

    root = parent.index(-1)
    approx = val(root)
    return float(np.linalg.norm(approx - exact) / np.linalg.norm(exact))


def _oracle_error():
    """The FP64 oracle's error on the same samples (tests/golden, written by
    a script that calls only the oracle), or None."""
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                     "fullsize_oracle_error.txt")
    try:
        for line in open(p):
            if line.startswith("sampled_rel_error:"):
                return float(line.split(":", 1)[1])
    except OSError:
        pass
    return None


def _geometry(ws, rank):
    """Global dims (mode 0 of n*ws points) and this rank's mode-0 slab."""
    from paper_2412_06111_gb300 import shard
    dims = [NMODE * ws] + [NMODE] * (D - 1)
    off, ext = shard.shard_box(dims, ws, rank, 0)
    return dims, (None, None) if ws == 1 else (off, ext)


def run_form(api, W, dtype, variant, steps, warmup, ws, torch, data, quantize=False, rank=0):
    """Times `steps` whole-path steps on device-resident data.  Returns a dict.
    quantize: `data` is binary32 and is first quantised to E4M3 tiles with the
    plan (timed apart: the producer's step, not the sketch's)."""
    from paper_2412_06111_gb300 import shard
    log("form dtype", dtype, "variant", variant)
    tr = W.balanced_binary(D)
    n = len(tr[0])
    dims, (off, ext) = _geometry(ws, rank)
    # the passes leave a few SMs free for the recovery that overlaps them
    plan = api.ttnn_plan_create(tr, dims, [RANK] * n, [OVERSAMPLE] * n, SEED, variant=variant,
                                sketch_dtype=dtype, flags=api.FLAG_RESERVE_SMS)
    # the update path (pass, walk) on a high-priority stream: when its blocks
    # and the overlapping recovery's wait for the same SMs, the update's go
    # first (the recovery has a whole step of slack)
    base = torch.cuda.current_stream()
    main = torch.cuda.Stream(priority=-1)
    main.wait_stream(base)
    torch.cuda.set_stream(main)
    side = torch.cuda.Stream()
    upd_done = torch.cuda.Event()
    rec_done = [torch.cuda.Event(), torch.cuda.Event()]
    for e in rec_done:
        e.record(main)

    def step(k=0, sync=False):
        """One whole-path step on state k % 2.  Pipelined (sync=False): the
        update runs on the main stream, the recovery of its state on a side
        stream, overlapping the next step's update (on the other state)."""
        st = states[k % 2]
        main.wait_event(rec_done[k % 2])           # the recovery that last read this state
        api.ttnn_state_zero(st)
        api.ttnn_update_dense(st, data, off, ext, tile_scale=scale)
        if ws > 1:
            shard.allreduce_state_(plan, st)       # the one exchange: sum of sketches
        if sync:
            api.ttnn_recover(st, cores)            # waits, reads the kept ranks back
            return
        upd_done.record(main)
        side.wait_event(upd_done)
        api.ttnn_recover_async(st, cores, stream=side)
        rec_done[k % 2].record(side)

    states = [api.ttnn_state_create(plan), api.ttnn_state_create(plan)]
    state = states[0]
    scale, quant_ms = None, None
    if quantize:
        nl = NMODE ** ((D + 1) // 2)        # the slab's pass-matrix rows (mode 0 is in L)
        nrt, nct = -(-nl // 128), -(-(data.numel() // nl) // 128)
        q8 = torch.empty(data.numel(), dtype=torch.uint8, device="cuda")
        scale = torch.empty(nrt * nct, dtype=torch.float32, device="cuda")
        api.ttnn_fp8_quantize(plan, data, q8, scale, extent=ext)
        torch.cuda.synchronize()
        qa, qb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        qa.record()
        api.ttnn_fp8_quantize(plan, data, q8, scale, extent=ext)
        qb.record()
        torch.cuda.synchronize()
        quant_ms = qa.elapsed_time(qb)
        data = q8
    ce = api.ttnn_plan_sizes(plan)[2]
    cores = torch.zeros(ce, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    log("plan and state ready")
    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    log("warm-up done")
    api.ttnn_profile(plan, True)
    for ph in range(4):
        api.ttnn_profile_read(plan, ph)
    l0 = api.ttnn_kernel_launches()
    _barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        step(k)
    for e in rec_done:
        stream.wait_event(e)                       # the last recoveries are inside the region
    e1.record(stream)
    torch.cuda.synchronize()
    api.ttnn_plan_sync(plan)
    _barrier(ws)
    ms = e0.elapsed_time(e1) / steps
    launches = api.ttnn_kernel_launches() - l0
    # latency of one update + recovery round trip (host wall clock, waited on)
    lat = []
    for _ in range(steps):
        t0 = time.perf_counter()
        step(sync=True)
        lat.append((time.perf_counter() - t0) * 1e3)
    passes = api.ttnn_plan_pass_counts(plan)
    api.ttnn_profile(plan, False)
    prof = [api.ttnn_profile_read(plan, ph) for ph in range(4)]
    err = _ttn_sample_error(api, plan, tr, cores, ws, rank) if NMODE == 64 else None
    for st in states:
        api.ttnn_state_destroy(st)
    api.ttnn_plan_destroy(plan)
    torch.cuda.synchronize()
    torch.cuda.set_stream(base)
    lat.sort()
    return {"ms_per_step": ms, "launches": launches, "tc_passes": passes[0], "simt_passes": passes[1],
            "pass_ms": prof[0][0] / max(prof[0][1], 1), "walk_ms": prof[1][0] / max(prof[1][1], 1),
            "recover_ms": prof[2][0] / max(prof[2][1], 1),
            "pass_kernel_ms": prof[3][0] / max(prof[3][1], 1) if prof[3][1] else None,
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "quantize_ms": quant_ms, "rel_error": err}


def run_e2e(api, W, dtype, steps, warmup, torch, host, ws=1, rank=0):
    """Same metric through the public API from pinned host memory: H2D copy of
    the tensor (this rank's slab), update, (all-reduce,) recovery, D2H copy of
    the cores every step.  The copy of step k+1's input (on a copy stream,
    into the other of two device buffers) overlaps step k's compute, as a
    streaming caller would run it; every copy and every step is inside the
    timed region."""
    from paper_2412_06111_gb300 import shard
    tr = W.balanced_binary(D)
    n = len(tr[0])
    dims, (off, ext) = _geometry(ws, rank)
    plan = api.ttnn_plan_create(tr, dims, [RANK] * n, [OVERSAMPLE] * n, SEED, sketch_dtype=dtype)
    state = api.ttnn_state_create(plan)
    ce = api.ttnn_plan_sizes(plan)[2]
    cores = torch.zeros(ce, dtype=torch.float64, device="cuda")
    cores_h = torch.zeros(ce, dtype=torch.float64).pin_memory()
    bufs = [torch.empty_like(host, device="cuda") for _ in range(2)]
    comp = torch.cuda.current_stream()
    cstream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    for e in freed:
        e.record(comp)

    def issue_copy(k):
        b = k % 2
        with torch.cuda.stream(cstream):
            cstream.wait_event(freed[b])
            bufs[b].copy_(host, non_blocking=True)
            copied[b].record(cstream)

    def step(k, last):
        b = k % 2
        if not last:
            issue_copy(k + 1)        # next input streams in while this step computes
        comp.wait_event(copied[b])
        api.ttnn_state_zero(state)
        api.ttnn_update_dense(state, bufs[b], off, ext)
        if ws > 1:
            shard.allreduce_state_(plan, state)
        freed[b].record(comp)
        api.ttnn_recover(state, cores)
        cores_h.copy_(cores, non_blocking=True)

    def run(k_steps):
        issue_copy(0)
        for k in range(k_steps):
            step(k, k == k_steps - 1)

    run(warmup)
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    api.ttnn_state_destroy(state)
    api.ttnn_plan_destroy(plan)
    return ms, host.numel() * host.element_size(), ce * 8


def run_config1(api, W, torch, n_lat=200):
    """Plain TTNN in binary64 on a 24^4 tensor with exact TTN ranks 5 on the
    balanced tree ((1,2),(3,4)) (N(0,1) cores) plus Gaussian noise of relative
    Frobenius norm 1e-8; target ranks 5, oversampling 5; the whole tensor in
    one update.  Host round-trip latency of the update and of the recovery
    (each waited on), with the Khatri-Rao and the unstructured Gaussian DRMs,
    and the relative error of the recovered TTN on 20000 seeded entries."""
    d, n, r, p = 4, 24, 5, 5
    tr = W.balanced_binary(d)
    nn = len(tr[0])
    dims = [n] * d
    T, _ = W.exact_ttn(tr, dims, [r] * nn, 1001, noise=1e-8)
    dev = torch.from_numpy(np.ascontiguousarray(T)).cuda()
    out = {"workload": "24^4 exact TTN ranks 5 + 1e-8 noise, FP64, r = 5, p = 5, one update"}
    for name, flags in (("kr", 0), ("gaussian", api.FLAG_DENSE_DRM)):
        plan = api.ttnn_plan_create(tr, dims, [r] * nn, [p] * nn, SEED + 1, sketch_dtype=api.F64,
                                    flags=flags)
        st = api.ttnn_state_create(plan)
        cores = torch.zeros(api.ttnn_plan_sizes(plan)[2], dtype=torch.float64, device="cuda")
        up, rec, dev_up, host_up = [], [], [], []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(n_lat + 5):
            api.ttnn_state_zero(st)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0.record()
            api.ttnn_update_dense(st, dev)
            e1.record()
            th = time.perf_counter()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            api.ttnn_recover(st, cores)
            t2 = time.perf_counter()
            if i >= 5:
                up.append((t1 - t0) * 1e6)
                rec.append((t2 - t1) * 1e6)
                dev_up.append(e0.elapsed_time(e1) * 1e3)
                host_up.append((th - t0) * 1e6)
        for v in (up, rec, dev_up, host_up):
            v.sort()
        err = _sampled_error(api, plan, tr, cores, dims, lambda idx: T[tuple(idx.T)])
        out[name] = {"update_us": {"p50": up[len(up) // 2], "p99": up[int(0.99 * len(up))],
                                   "device_p50": dev_up[len(dev_up) // 2],
                                   "host_call_p50": host_up[len(host_up) // 2]},
                     "recover_us": {"p50": rec[len(rec) // 2], "p99": rec[int(0.99 * len(rec))]},
                     "rel_error": err}
        api.ttnn_state_destroy(st)
        api.ttnn_plan_destroy(plan)
    return out


def run_streaming(api, W, torch, n_updates=4096, n_lat=256):
    """Streamed order-6 workload: 32^6 caterpillar (tensor train, identity
    single-mode leaves), r = 16, s = 24, BF16 plan; each update is one rank-2
    CP term (N(0,1) factors, binary64) plus one 32^3 box of N(0, 0.01) noise
    on 3 uniformly chosen modes (the others fixed at uniform indices).
    Throughput over n_updates back to back; latency over n_lat synchronised
    updates.  Inputs resident on the device."""
    d, n = 6, 32
    tr = W.tensor_train(d)
    nn = len(tr[0])
    dims = [n] * d
    plan = api.ttnn_plan_create(tr, dims, [16] * nn, [8] * nn, SEED + 3, sketch_dtype=api.BF16)
    state = api.ttnn_state_create(plan)
    g = torch.Generator(device="cuda").manual_seed(1003)
    facs = torch.randn(n_updates, d, n, 2, dtype=torch.float64, device="cuda", generator=g)
    boxes = (torch.randn(n_updates, n * n * n, device="cuda", generator=g) * 0.1).to(torch.bfloat16)
    rng = np.random.default_rng(1003)
    geo = []
    for _ in range(n_updates):
        modes = sorted(rng.choice(d, size=3, replace=False).tolist())
        off = [int(rng.integers(0, n)) for _ in range(d)]
        ext = [1] * d
        for mu in modes:
            ext[mu], off[mu] = n, 0
        geo.append((off, ext))
    flist = [[facs[i, mu] for mu in range(d)] for i in range(n_updates)]

    def one(i):
        api.ttnn_update_cp(state, [1.0, 1.0], flist[i])
        off, ext = geo[i]
        api.ttnn_update_dense(state, boxes[i], off, ext)

    for i in range(16):
        one(i)
    torch.cuda.synchronize()
    l0 = api.ttnn_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for i in range(n_updates):
        one(i)
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    launches = api.ttnn_kernel_launches() - l0
    lat = []
    for i in range(n_lat):
        t1 = time.perf_counter()
        one(i)
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t1) * 1e6)
    lat.sort()
    cores = torch.zeros(api.ttnn_plan_sizes(plan)[2], dtype=torch.float64, device="cuda")
    r0 = time.perf_counter()
    api.ttnn_recover(state, cores)
    rec_ms = (time.perf_counter() - r0) * 1e3
    api.ttnn_state_destroy(state)
    api.ttnn_plan_destroy(plan)
    # against binary64: the first n_err updates applied to a binary64 and to
    # a BF16 plan (same tree, ranks and seed; the boxes hold bfloat16
    # values, exact in both), the recovered TTNs compared on 20000 seeded
    # entries
    # (E4M3: each box quantised with its per-tile scales first)
    n_err = 1024
    idx = _sample_idx(dims)
    vals, notes = {}, {}
    q8 = torch.empty(n * n * n, dtype=torch.uint8, device="cuda")
    qs = torch.empty(4096, dtype=torch.float32, device="cuda")
    for name, dt in (("f64", api.F64), ("bf16", api.BF16), ("e4m3", api.E4M3)):
        try:
            pl = api.ttnn_plan_create(tr, dims, [16] * nn, [8] * nn, SEED + 3, sketch_dtype=dt)
            s_ = api.ttnn_state_create(pl)
            for i in range(n_err):
                api.ttnn_update_cp(s_, [1.0, 1.0], flist[i])
                off, ext = geo[i]
                if dt == api.E4M3:
                    api.ttnn_fp8_quantize(pl, boxes[i].float(), q8, qs, extent=ext)
                    api.ttnn_update_dense(s_, q8, off, ext, tile_scale=qs)
                else:
                    api.ttnn_update_dense(s_, boxes[i] if dt == api.BF16 else boxes[i].double(),
                                          off, ext)
            c_ = torch.zeros(api.ttnn_plan_sizes(pl)[2], dtype=torch.float64, device="cuda")
            api.ttnn_recover(s_, c_)
            vals[name] = _ttn_entries(api, pl, tr, c_, dims, idx)
            api.ttnn_state_destroy(s_)
            api.ttnn_plan_destroy(pl)
        except api.TtnnError as e:
            notes[name] = str(e)
    rel = lambda a: (float(np.linalg.norm(vals[a] - vals["f64"]) / np.linalg.norm(vals["f64"]))
                     if a in vals and "f64" in vals else None)
    err64 = rel("bf16")
    err8 = rel("e4m3")
    upd_bytes = n * n * n * 2 + d * n * 2 * 8
    return {"workload": "32^6 tensor train r=16 s=24 BF16; update = rank-2 CP + 32^3 box",
            "updates": n_updates, "updates_per_s": n_updates / (ms * 1e-3),
            "host_wall_updates_per_s": n_updates / wall,
            "update_gbs": n_updates * upd_bytes / (ms * 1e-3) / 1e9,
            "launches_per_update": launches / n_updates,
            "latency_us": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
            "recover_ms": rec_ms,
            "vs_f64": {"note": f"recovered TTN after the first {n_err} updates, BF16 and E4M3 "
                               "(per-tile scales) plans against the binary64 plan, 20000 seeded "
                               "entries; each plan's DRM is rounded to its format, and this "
                               "tensor (a sum of rank-2 terms) is far from rank 16, so the "
                               "difference includes that of two rank-16 approximations taken "
                               "with different DRMs", "bf16_rel_diff": err64, "e4m3_rel_diff": err8,
                       "errors": notes}}


def _ttn_inner(parent, ch, A, B):
    """Frobenius inner product of two TTNs on one tree (cores: root
    (R_c..), transfer (R_v, R_c..), leaf (R_v, n..)): Gram matrices of the
    two networks' node bases, leaves first, then the root's scalar."""
    order, stack = [], [parent.index(-1)]
    while stack:
        v = stack.pop()
        order.append(v)
        stack.extend(ch[v])
    M = {}
    for v in reversed(order):
        a, b = np.asarray(A[v]), np.asarray(B[v])
        if not ch[v]:
            M[v] = a.reshape(a.shape[0], -1) @ b.reshape(b.shape[0], -1).T
            continue
        head = 0 if parent[v] < 0 else 1
        x = b
        for k, c in enumerate(ch[v]):          # B's child axes into A's rank spaces
            x = np.moveaxis(np.tensordot(M[c], x, axes=([1], [head + k])), 0, head + k)
        if head:
            M[v] = np.tensordot(a, x, axes=(list(range(1, a.ndim)), list(range(1, a.ndim))))
        else:
            M[v] = np.array(np.sum(a * x))
    return float(M[order[0]])


def run_rounding(api, W, torch, steps=5, warmup=3):
    """TTN rounding (Sec. 7, sketches of a tensor already in TTN format):
    order 8, modes 64, balanced binary tree, every edge of rank 200 (a
    dominant rank-30 network, norm 100, in direct sum with a rank-170 noise
    network, norm 1), recompressed to ranks 30 with p = 15.  One step =
    ttnn_update_ttn of the whole network into a zeroed state + recovery,
    binary64 cores resident on the device; BF16 and FP32 plans (binary32
    walk in both; the BF16 plan's DRM factors are bfloat16 values)."""
    d, n, rdom, rnoise, r, p = 8, 64, 30, 170, 30, 15
    tr = W.balanced_binary(d)
    nn = len(tr[0])
    dims = [n] * d
    cores = W.rounding_input(tr, dims, rdom, rnoise, 1005)
    dev = [torch.from_numpy(np.ascontiguousarray(cores[v])).cuda() for v in range(nn)]
    in_bytes = sum(c.numel() * 8 for c in dev)
    walk_bytes = 2 * sum(c.numel() for c in dev) * 4      # two sweeps over binary32 copies
    # dominant GEMM flops of the sweeps: every core against its sketch
    # blocks, up (r + s columns) and down (r columns)
    flops = sum(2.0 * c.numel() * (r + (r + p) + r) for c in dev)
    ch, _ = W.children_of(tr[0], tr[1])
    tt = _ttn_inner(tr[0], ch, cores, cores)
    out = {"workload": f"TTN order {d}, modes {n}, balanced binary tree, edge ranks {rdom + rnoise} "
                       f"({rdom} dominant x100 + {rnoise} noise) -> ranks {r}, p = {p}",
           "input_bytes": in_bytes, "walk_bytes": walk_bytes}
    for name, dt in (("bf16", api.BF16), ("fp32", api.F32)):
        plan = api.ttnn_plan_create(tr, dims, [r] * nn, [p] * nn, SEED + 5, sketch_dtype=dt,
                                    flags=api.FLAG_STRUCTURED_ONLY)
        st = api.ttnn_state_create(plan)
        ce = api.ttnn_plan_sizes(plan)[2]
        outc = torch.zeros(ce, dtype=torch.float64, device="cuda")

        def step():
            api.ttnn_state_zero(st)
            api.ttnn_update_ttn(st, dev, [rdom + rnoise] * nn)
            api.ttnn_recover_async(st, outc)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        api.ttnn_plan_sync(plan)
        ms = e0.elapsed_time(e1) / steps
        host = outc.cpu().numpy()
        nodes = [api.ttnn_plan_node(plan, v) for v in range(nn)]
        got = {nd["user_index"]: host[nd["core_offset"]:nd["core_offset"] + nd["core_elems"]]
               .reshape(nd["core_shape"]) for nd in nodes}
        err = float(np.sqrt(max(tt - 2 * _ttn_inner(tr[0], ch, cores, got) +
                                _ttn_inner(tr[0], ch, got, got), 0.0) / tt))
        tf = flops / (ms * 1e-3) / 1e12
        out[name] = {"ms_per_rounding": ms, "input_gbs": in_bytes / (ms * 1e-3) / 1e9,
                     "walk_gbs": walk_bytes / (ms * 1e-3) / 1e9, "rel_error": err,
                     "roofline": {"bound": "alu", "achieved": tf, "peak": FFMA_TFLOPS,
                                  "unit": "TFLOP/s", "frac": tf / FFMA_TFLOPS,
                                  "flops": flops, "note": "binary32 FFMA peak from unit counts "
                                  "and clocks; whole rounding (sweeps, QR, assembly) timed"}}
        api.ttnn_state_destroy(st)
        api.ttnn_plan_destroy(plan)
    out["noise_level"] = 0.01
    # the paper's TTN-rounding workload (Sec. 8, second experiment) at its
    # size: the example tree, modes 500, rank 70, orthogonal-CP transfer
    # tensors with cubic decay, Haar leaves -> ranks 20, p = 10, binary64
    tr6 = W.toy_tree()
    n6 = len(tr6[0])
    dims6 = [500] * 6
    c6 = W.orthogonal_cp_ttn(tr6, dims6, 70, lambda i: 1.0 / i ** 3, 1006)
    d6 = [torch.from_numpy(np.ascontiguousarray(c6[v])).cuda() for v in range(n6)]
    ch6, _ = W.children_of(tr6[0], tr6[1])
    tt6 = _ttn_inner(tr6[0], ch6, c6, c6)
    plan = api.ttnn_plan_create(tr6, dims6, [20] * n6, [10] * n6, SEED + 6, sketch_dtype=api.F64,
                                flags=api.FLAG_STRUCTURED_ONLY)
    st = api.ttnn_state_create(plan)
    outc = torch.zeros(api.ttnn_plan_sizes(plan)[2], dtype=torch.float64, device="cuda")

    def step6():
        api.ttnn_state_zero(st)
        api.ttnn_update_ttn(st, d6, [70] * n6)
        api.ttnn_recover_async(st, outc)

    for _ in range(warmup):
        step6()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step6()
    e1.record()
    torch.cuda.synchronize()
    api.ttnn_plan_sync(plan)
    host = outc.cpu().numpy()
    nodes = [api.ttnn_plan_node(plan, v) for v in range(n6)]
    got = {nd["user_index"]: host[nd["core_offset"]:nd["core_offset"] + nd["core_elems"]]
           .reshape(nd["core_shape"]) for nd in nodes}
    err6 = float(np.sqrt(max(tt6 - 2 * _ttn_inner(tr6[0], ch6, c6, got) +
                             _ttn_inner(tr6[0], ch6, got, got), 0.0) / tt6))
    out["paper_workload"] = {
        "workload": "example tree, modes 500 (5^6 x 10^9 entries never formed), TTN rank 70, "
                    "orthogonal-CP cores with sigma_i = i^-3, Haar leaves -> ranks 20, p = 10, FP64",
        "ms_per_rounding": e0.elapsed_time(e1) / steps, "rel_error": err6,
        "input_bytes": sum(c.numel() * 8 for c in d6)}
    api.ttnn_state_destroy(st)
    api.ttnn_plan_destroy(plan)
    return out


def _ttn_entries(api, plan, tree, cores_dev, dims, idx):
    """Entries of the recovered TTN at the multi-indices idx (samples x d):
    host evaluation of the cores (leaf slices, then each transfer tensor
    against its children's vectors)."""
    parent, leaf_modes, _ = tree
    nn = len(parent)
    nodes = [api.ttnn_plan_node(plan, v) for v in range(nn)]
    host = cores_dev.cpu().numpy()
    ch = {v: sorted([c for c in range(nn) if parent[c] == v], key=lambda c: nodes[c]["mode_lo"])
          for v in range(nn)}
    letters = "bcdefghijk"

    def val(v):
        nd = nodes[v]
        core = host[nd["core_offset"]:nd["core_offset"] + nd["core_elems"]].reshape(nd["core_shape"])
        if not ch[v]:
            lo, hi = nd["mode_lo"], nd["mode_hi"]
            flat = np.ravel_multi_index(tuple(idx[:, lo:hi].T), [dims[m] for m in range(lo, hi)])
            return core.reshape(core.shape[0], -1)[:, flat].T
        vecs = [val(c) for c in ch[v]]
        m = len(vecs)
        head = "" if parent[v] < 0 else "a"
        spec = head + letters[:m] + "," + ",".join("s" + letters[k] for k in range(m)) + "->s" + head
        return np.einsum(spec, core, *vecs, optimize=True)

    return val(parent.index(-1))


def _sample_idx(dims, samples=20000, seed=77):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, n, size=samples) for n in dims], axis=1)


def _sampled_error(api, plan, tree, cores_dev, dims, exact, samples=20000, seed=77):
    """Relative error of the recovered TTN on `samples` seeded entries against
    exact(idx)."""
    idx = _sample_idx(dims, samples, seed)
    approx = _ttn_entries(api, plan, tree, cores_dev, dims, idx)
    want = exact(idx)
    return float(np.linalg.norm(approx - want) / np.linalg.norm(want))


def run_hilbert(api, W, torch, steps=3, warmup=2, r=10, p=5):
    """The paper's first experiment (Sec. 8): the 6D Hilbert tensor
    1/(1 + i_1 + .. + i_6) with modes 20 on the paper's example tree, ranks
    r, oversampling p, binary64: TTNN and STTNN with Khatri-Rao DRMs, TTNN
    with unstructured Gaussian DRMs (the paper's sketches for this
    experiment) and TTN-HMT on the same sketches, each timed (whole-tensor
    update + recovery, or the two passes of TTN-HMT) and its error measured
    on 20000 seeded entries."""
    tr = W.toy_tree()
    nn = len(tr[0])
    dims = [20] * 6
    dev = torch.from_numpy(W.hilbert(6, 20)).cuda()
    exact = lambda idx: 1.0 / (1.0 + idx.sum(axis=1))
    out = {"workload": f"Hilbert 20^6 (FP64, {dev.numel() * 8 / 1e6:.0f} MB), example tree, "
                       f"r = {r}, p = {p}"}
    for name, variant, flags, hmt in (("ttnn_kr", api.VARIANT_TTNN, 0, False),
                                      ("sttnn_kr", api.VARIANT_STTNN, 0, False),
                                      ("ttnn_gaussian", api.VARIANT_TTNN, api.FLAG_DENSE_DRM, False),
                                      ("ttn_hmt_gaussian", api.VARIANT_TTNN, api.FLAG_DENSE_DRM, True)):
        plan = api.ttnn_plan_create(tr, dims, [r] * nn, [p] * nn, SEED + 7, variant=variant,
                                    sketch_dtype=api.F64, flags=flags)
        st = api.ttnn_state_create(plan)
        cores = torch.zeros(api.ttnn_plan_sizes(plan)[2], dtype=torch.float64, device="cuda")

        def step():
            if hmt:
                api.ttnn_hmt(plan, dev, cores)
            else:
                api.ttnn_state_zero(st)
                api.ttnn_update_dense(st, dev)
                api.ttnn_recover_async(st, cores)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        api.ttnn_plan_sync(plan)
        out[name] = {"ms": e0.elapsed_time(e1) / steps,
                     "rel_error": _sampled_error(api, plan, tr, cores, dims, exact)}
        api.ttnn_state_destroy(st)
        api.ttnn_plan_destroy(plan)
    return out


# binary32 FMA peak of a GB300: 152 SMs x 128 FMA lanes x 2 flops x 2.07 GHz
FFMA_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
SERVE_QUEUE = 1024     # requests outstanding in the server (back-pressure beyond)
SERVE_STREAM_QUEUE = 4   # ... and per stream
EBUSY = 6


def run_serving(api, W, torch, n_streams=256, rate=22000.0, seconds=60.0):
    """Serving mix: n_streams resident BF16 streams of mixed order, sizes,
    trees and ranks (workloads.serving_stream_spec; streams whose device
    footprint exceeds 512 MiB are redrawn), fed a Poisson stream of N(0,1)
    slices (one mode fixed at a uniform index) at `rate`/s for `seconds`.
    The server holds at most SERVE_QUEUE outstanding requests, and
    SERVE_STREAM_QUEUE per stream: a submit beyond either is refused (EBUSY)
    and the client waits for that stream's oldest outstanding ticket (or the
    busiest stream's) before retrying, which bounds the latency at full load."""
    rng = np.random.default_rng(1004)
    srv = api.ttnn_server_create(160 << 30, max_batch=64, queue_capacity=SERVE_QUEUE, workers=8,
                                 stream_queue_capacity=SERVE_STREAM_QUEUE)
    outstanding = collections.defaultdict(collections.deque)   # stream -> tickets in order
    stats = {"throttled": 0, "throttle_s": 0.0, "failed": 0, "errors": {}}

    def finish(t):
        st = api.ttnn_server_wait(srv, t, 120_000_000)
        if st != 0:
            stats["failed"] += 1
            key = f"{st}: {api.last_error_message()}"
            stats["errors"][key] = stats["errors"].get(key, 0) + 1

    def submit(sid, dm, mu, idx):
        off = [0] * len(dm)
        ext = list(dm)
        off[mu], ext[mu] = idx, 1
        while True:
            try:
                outstanding[sid].append(api.ttnn_server_submit(srv, sid, buf, off, ext))
                return
            except api.TtnnError as e:
                if e.status != EBUSY:
                    raise
                q = outstanding[sid] if outstanding[sid] else max(outstanding.values(), key=len)
                if not q:
                    raise
                stats["throttled"] += 1
                tw = time.perf_counter()
                finish(q.popleft())
                stats["throttle_s"] += time.perf_counter() - tw

    def drain():
        """Waits for every outstanding ticket; returns the time at which all
        were done (a stream's requests complete in order, so its last ticket
        done means all of its tickets are: those are waited on first, the
        rest are then only collected)."""
        for q in outstanding.values():
            if q:
                finish(q.pop())
        t_done = time.perf_counter()
        for q in outstanding.values():
            while q:
                finish(q.popleft())
        return t_done

    sids, dims_of = [], []
    t_open = time.perf_counter()
    tries = 0
    while len(sids) < n_streams and tries < 20 * n_streams:
        tries += 1
        sp = W.serving_stream_spec(rng)
        nn = len(sp["tree"][0])
        before = api.ttnn_server_stats(srv)["device_bytes"]
        try:
            sid = api.ttnn_server_open(srv, sp["tree"], sp["dims"], [sp["r"]] * nn, [sp["p"]] * nn,
                                       SEED + len(sids), sketch_dtype=api.BF16)
        except api.TtnnError:
            continue
        if api.ttnn_server_stats(srv)["device_bytes"] - before > (512 << 20):
            api.ttnn_server_close(srv, sid)
            continue
        sids.append(sid)
        dims_of.append(sp["dims"])
    open_s = time.perf_counter() - t_open
    n_streams = len(sids)
    max_slice = max(int(np.prod(dm)) // min(dm) for dm in dims_of)
    buf = torch.randn(max_slice, device="cuda").to(torch.bfloat16)
    arrivals = W.poisson_slices(rng, n_streams, dims_of, rate, seconds)
    tickets = []
    # warm-up: one slice per stream
    for j, sid in enumerate(sids):
        ext = list(dims_of[j])
        ext[0] = 1
        tickets.append(api.ttnn_server_submit(srv, sid, buf, None, ext))
    for t in tickets:
        api.ttnn_server_wait(srv, t, 60_000_000)
    api.ttnn_server_stats(srv, reset=True)
    late = 0
    t0 = time.perf_counter()
    for (ta, s_, mu, idx) in arrivals:
        while True:
            now = time.perf_counter() - t0
            if now >= ta:
                break
        if now - ta > 1e-3:
            late += 1
        submit(sids[s_], dims_of[s_], mu, idx)
    wall = drain() - t0
    rep = api.ttnn_server_stats(srv)
    dev_bytes = rep["device_bytes"]
    offered = dict(throttled=stats["throttled"], throttle_s=stats["throttle_s"])
    # capacity: the same kind of slices submitted back to back (the queue
    # stays full; the client is held back by EBUSY), completion rate until
    # the last one is done
    api.ttnn_server_stats(srv, reset=True)
    stats["throttled"], stats["throttle_s"] = 0, 0.0
    burst = [(s_, mu, idx) for (_, s_, mu, idx) in arrivals[:100000]]
    t1 = time.perf_counter()
    for (s_, mu, idx) in burst:
        submit(sids[s_], dims_of[s_], mu, idx)
    cap_s = drain() - t1
    cap = api.ttnn_server_stats(srv)
    api.ttnn_server_destroy(srv)
    return {"workload": f"{n_streams} streams (d 3-6, n in 16..128, binary/TT/Tucker, r 4-32, "
                        f"p=r/2, BF16), Poisson slices at {rate:.0f}/s for {seconds:.0f} s",
            "offered_per_s": len(arrivals) / seconds, "target_per_s": 20000,
            "drain_s": wall - seconds, "completed": rep["completed_updates"],
            "completed_per_s": rep["completed_updates"] / wall,
            "failed": stats["failed"] + rep["failed"],
            "update_gbs": rep["update_bytes"] / wall / 1e9,
            "latency_us": {"p50": rep["p50_us"], "p99": rep["p99_us"], "max": rep["max_us"]},
            "batches": rep["batches"],
            "updates_per_batch": rep["completed_updates"] / max(rep["batches"], 1),
            "late_submits": late, "open_s": open_s, "queue_capacity": SERVE_QUEUE,
            "stream_queue_capacity": SERVE_STREAM_QUEUE,
            "throttled_submits": offered["throttled"], "throttle_wait_s": offered["throttle_s"],
            "worker_host_s": rep["worker_host_s"], "wall_s": wall, "errors": stats["errors"],
            "device_gb": dev_bytes / 1e9,
            "capacity": {"note": "the first slices of the same arrival list submitted back to "
                                 "back; submits beyond the queue capacity wait (EBUSY) for the "
                                 "oldest outstanding ticket",
                         "updates": cap["completed_updates"], "per_s": cap["completed_updates"] / cap_s,
                         "batches": cap["batches"],
                         "updates_per_batch": cap["completed_updates"] / max(cap["batches"], 1),
                         "p50_us": cap["p50_us"], "p99_us": cap["p99_us"], "max_us": cap["max_us"],
                         "throttled_submits": stats["throttled"]}}


def cpu_oracle_sample(max_seconds=25.0):
    """The FP64 oracle (as it stands) on a bounded sample of the workload: the
    same tree/ranks on a 16 x 64^4 slab (a quarter) of the tensor."""
    import numpy as np

    import workloads as W
    from oracle import ttnn as O
    from oracle.tree import Tree
    tr = W.balanced_binary(D)
    n = len(tr[0])
    slab = min(16, NMODE)
    ext = [slab] + [NMODE] * (D - 1)
    full = 1.0 + np.arange(NMODE) / (NMODE - 1)
    x0 = full[:slab]
    s = x0.reshape(slab, 1, 1, 1, 1) + 0.0
    for mu in range(1, D):
        sh = [1] * D
        sh[mu] = NMODE
        s = s + full.reshape(sh)
    T = (1.0 / s).astype(np.float32).astype(np.float64)
    t = Tree(tr[0], tr[1], ext, [RANK] * n, [OVERSAMPLE] * n, tr[2])
    reps, t_tot = 0, 0.0
    while True:
        t0 = time.perf_counter()
        O.ttnn(T, t, SEED, "f32")
        t_tot += time.perf_counter() - t0
        reps += 1
        if t_tot > max_seconds * 0.5 or reps >= 3:
            break
    sec = t_tot / reps
    nbytes = T.size * 4
    return {"value": nbytes / sec / 1e9, "unit": "GB/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{slab}x{NMODE}^4 slab of the {NMODE}^5 tensor (FP32 values, {T.size} entries), TTNN "
                      f"sketch + recovery in FP64 numpy, mean of {reps} run(s), {sec:.2f} s each"}


def main():
    global NMODE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson serving run (60 s: the stated serving config)")
    ap.add_argument("--no-serving", action="store_true",
                    help="leave out the streamed-update and serving-mix legs (extra keys)")
    ap.add_argument("--nmode", type=int, default=NMODE, help="mode size (64 = the stated workload)")
    ap.add_argument("--headline-only", action="store_true",
                    help="time only one form's step (default the BF16 TTNN headline; no other "
                         "forms, e2e or serving legs; e.g. for profiling)")
    ap.add_argument("--form", default="bf16", choices=["bf16", "sttnn", "fp32", "bf16x2", "fp8"],
                    help="the form --headline-only times")
    ap.add_argument("--leg", default=None,
                    choices=["config1", "streaming", "serving", "rounding", "hilbert"],
                    help="run only this extra leg and print its JSON (e.g. for profiling)")
    args = ap.parse_args()
    NMODE = args.nmode
    warmup = max(3, args.warmup)

    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return
        per = []
        for _ in range(args.steps):
            per.append(cpu_oracle_sample(max_seconds=10.0))
        v = statistics.median(p["value"] for p in per)
        cb = dict(per[0])
        cb["value"] = v
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": 0,
                          "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": f"order-5 {NMODE}^5 inv-sum, binary tree, r=20 "
                                                 f"l=10 (bounded {min(16, NMODE)}x{NMODE}^4 slab "
                                                 "per step on host cores)"},
                          "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch

    import workloads as W
    from paper_2412_06111_gb300 import api
    rank, ws = _dist()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    hbm, bf16_tf, peak_src = _peaks()
    if args.leg:
        if rank == 0:
            legs = {"config1": lambda: run_config1(api, W, torch),
                    "streaming": lambda: run_streaming(api, W, torch),
                    "serving": lambda: run_serving(api, W, torch, seconds=args.serve_seconds),
                    "rounding": lambda: run_rounding(api, W, torch),
                    "hilbert": lambda: run_hilbert(api, W, torch)}
            with Clocks(dev) as clk:
                res = legs[args.leg]()
            print(json.dumps({"leg": args.leg, args.leg: res, "clocks": clk.summary()}))
        return
    N = NMODE ** D
    a32 = W.inv_sum_slab_torch(D, NMODE, ws, rank, "cuda", torch.float32)
    if args.headline_only:
        # one form, holding only the tensor that form reads
        dt, var, narrow, quant = {"bf16": (api.BF16, api.VARIANT_TTNN, True, False),
                                  "sttnn": (api.BF16, api.VARIANT_STTNN, True, False),
                                  "fp32": (api.F32, api.VARIANT_TTNN, False, False),
                                  "bf16x2": (api.BF16X2, api.VARIANT_TTNN, False, False),
                                  "fp8": (api.E4M3, api.VARIANT_TTNN, False, True)}[args.form]
        data = a32.to(torch.bfloat16) if narrow else a32
        del a32
        torch.cuda.empty_cache()
        with Clocks(dev) as clk:
            bf = run_form(api, W, dt, var, args.steps, warmup, ws, torch, data, quantize=quant,
                          rank=rank)
        ms = _max_over_ranks(bf["ms_per_step"], ws)
        if rank == 0:
            eb, dts = {"bf16": (2, "bf16"), "sttnn": (2, "bf16"), "fp32": (4, "f32"),
                       "bf16x2": (4, "f32"), "fp8": (1, "e4m3")}[args.form]
            print(json.dumps({"metric": METRIC, "value": N * eb * ws / (ms * 1e-3) / 1e9,
                              "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
                              "warmup": warmup, "ms_per_step": ms, "dtype": dts,
                              "headline_only": True, "form": args.form,
                              "phases_ms": {"pass": bf["pass_ms"], "walk": bf["walk_ms"],
                                            "recover": bf["recover_ms"]},
                              "clocks": clk.summary()}))
        return
    a16 = a32.to(torch.bfloat16)
    log("tensor ready", N)
    with Clocks(dev) as clk:
        bf = run_form(api, W, api.BF16, api.VARIANT_TTNN, args.steps, warmup, ws, torch, a16,
                      rank=rank)
    k = max(3, args.steps // 2)
    f32 = run_form(api, W, api.F32, api.VARIANT_TTNN, k, warmup, ws, torch, a32, rank=rank)
    x2 = run_form(api, W, api.BF16X2, api.VARIANT_TTNN, k, warmup, ws, torch, a32, rank=rank)
    f8 = run_form(api, W, api.E4M3, api.VARIANT_TTNN, k, warmup, ws, torch, a32, quantize=True,
                  rank=rank)
    st = run_form(api, W, api.BF16, api.VARIANT_STTNN, k, warmup, ws, torch, a16, rank=rank)
    host16 = a16.cpu().pin_memory()
    del a32
    e2e_ms, h2d, d2h = run_e2e(api, W, api.BF16, k, 2, torch, host16, ws, rank)
    e2e_ms = _max_over_ranks(e2e_ms, ws)
    ms = _max_over_ranks(bf["ms_per_step"], ws)
    value = N * 2 * ws / (ms * 1e-3) / 1e9
    # the roofline's kernel: the tensor-core pass kernel alone (its average
    # launch, CUDA events on its stream); the pass phase adds the reduction
    # of the D2 row-group partials
    kern_ms = bf["pass_kernel_ms"] or bf["pass_ms"]
    pass_gbs = N * 2 / (kern_ms * 1e-3) / 1e9
    traffic = _pass_traffic() if NMODE == 64 else None
    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": (f"dense order-5 {NMODE * ws}x{NMODE}^4" if ws > 1 else
                                f"dense order-5 {NMODE}^5") +
                               " f(x)=1/sum(x) on [1,2]^5, balanced binary tree, "
                               "ranks 20, oversampling 10, TTNN, one whole-tensor update + recovery "
                               "per step", "global_batch": 1, "l2": "inputs larger than L2 (2.1 GB)",
                   "parallelism": "single GPU" if ws == 1 else
                   f"sharded{ws}: each rank owns a 64^5 mode-0 slab of a ({NMODE}*{ws})x{NMODE}^4 "
                   "tensor; one NCCL sum all-reduce of the sketch state per step; recovery on "
                   "every rank"},
        "roofline": {"bound": "hbm", "achieved": pass_gbs, "peak": hbm, "unit": "GB/s",
                     "frac": pass_gbs / hbm, "traffic": traffic,
                     "kernel": "tc::pass_kernel (first-level pass)", "kernel_ms": kern_ms,
                     "pass_phase_ms": bf["pass_ms"],
                     "pass_phase_frac": N * 2 / (bf["pass_ms"] * 1e-3) / 1e9 / hbm,
                     "peak_source": peak_src},
        "e2e": {"value": N * 2 * ws / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(bf["launches"]),
        "clocks": clk.summary(),
        "latency_ms": {"p50": bf["p50_ms"], "p99": bf["p99_ms"]},
        "phases_ms": {"pass": bf["pass_ms"], "walk": bf["walk_ms"], "recover": bf["recover_ms"]},
        "pass_path": {"tensor_core": bf["tc_passes"], "simt": bf["simt_passes"]},
        "rel_error": {"note": "final relative error of the recovered TTN vs the exact binary64 "
                              f"tensor on {SAMPLES} seeded entries",
                      "fp64_oracle": _oracle_error(), "bf16": bf["rel_error"],
                      "fp32_plain": f32["rel_error"], "bf16x2_split": x2["rel_error"],
                      "fp8_e4m3": f8["rel_error"], "sttnn_bf16": st["rel_error"]},
        "fp32_plain": {"value": N * 4 / (f32["ms_per_step"] * 1e-3) / 1e9, "unit": "GB/s",
                       "ms_per_step": f32["ms_per_step"], "pass_ms": f32["pass_ms"]},
        "sttnn_bf16": {"value": N * 2 / (st["ms_per_step"] * 1e-3) / 1e9, "unit": "GB/s",
                       "ms_per_step": st["ms_per_step"], "pass_ms": st["pass_ms"]},
        "bf16x2_split": {"value": N * 4 / (x2["ms_per_step"] * 1e-3) / 1e9, "unit": "GB/s",
                         "ms_per_step": x2["ms_per_step"], "pass_ms": x2["pass_ms"],
                         "pass_gbs": N * 4 / (x2["pass_ms"] * 1e-3) / 1e9},
        "fp8_e4m3": {"value": N * 1 / (f8["ms_per_step"] * 1e-3) / 1e9, "unit": "GB/s",
                     "ms_per_step": f8["ms_per_step"], "pass_ms": f8["pass_ms"],
                     "pass_gbs": N * 1 / (f8["pass_ms"] * 1e-3) / 1e9,
                     "quantize_ms": f8["quantize_ms"]},
    }
    if rank == 0 and not args.no_serving:
        log("config-1 leg")
        out["config1"] = run_config1(api, W, torch)
        log("streaming leg")
        out["streaming"] = run_streaming(api, W, torch)
        log("serving leg")
        out["serving"] = run_serving(api, W, torch, seconds=args.serve_seconds)
        log("rounding leg")
        out["rounding"] = run_rounding(api, W, torch)
        log("hilbert leg")
        out["hilbert"] = run_hilbert(api, W, torch)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle_sample()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
