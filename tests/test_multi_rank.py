"""The N > 1 path on CPU ranks (gloo): each rank sketches its own slab of the
tensor (the oracle stands in for the device update of that box), one sum
all-reduce through the package's shard helpers gives every rank the sketch of
the whole tensor (linearity, Sec. 4), and recovery from it reproduces the
single-process result.  Also: the slabs partition the tensor."""
import os
import socket

import numpy as np
import pytest

import workloads as W
from oracle import ttnn as O
from oracle.tree import Tree
from paper_2412_06111_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_boxes_partition():
    for dims in ([7, 5, 6], [3, 4, 5, 6], [64, 2]):
        for world in (1, 2, 3, 5, 8):
            for mode in range(len(dims)):
                seen = np.zeros(dims, dtype=int)
                for r in range(world):
                    off, ext = shard.shard_box(dims, world, r, mode)
                    assert all(e == n for m, (e, n) in enumerate(zip(ext, dims)) if m != mode)
                    if ext[mode] == 0:
                        continue
                    sl = tuple(slice(o, o + e) for o, e in zip(off, ext))
                    seen[sl] += 1
                assert (seen == 1).all()


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tr = W.toy_tree()
    dims = [6, 5, 4, 5, 4, 5]
    n = len(tr[0])
    t = Tree(tr[0], tr[1], dims, [3] * n, [2] * n, tr[2])
    T, _ = W.exact_ttn(tr, dims, [2] * n, 5, noise=1e-3)
    drm = O.Drm(t, 21, "f64")
    off, ext = shard.shard_box(dims, world, rank, mode=0)
    sl = tuple(slice(o, o + e) for o, e in zip(off, ext))
    part = np.zeros(dims)
    part[sl] = T[sl]
    Om, Ps, Pr = O.sketch_ttnn(part, t, drm)
    keys = sorted(Om)
    flat = np.concatenate([Om[v].ravel() for v in keys] + [Ps[v].ravel() for v in keys] + [Pr.ravel()])
    buf = torch.from_numpy(flat.copy())
    shard.allreduce_(buf)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), buf.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_sketches_allreduce_to_whole_tensor_sketch(tmp_path, world):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    tr = W.toy_tree()
    dims = [6, 5, 4, 5, 4, 5]
    n = len(tr[0])
    t = Tree(tr[0], tr[1], dims, [3] * n, [2] * n, tr[2])
    T, _ = W.exact_ttn(tr, dims, [2] * n, 5, noise=1e-3)
    Om, Ps, Pr = O.sketch_ttnn(T, t, O.Drm(t, 21, "f64"))
    keys = sorted(Om)
    want = np.concatenate([Om[v].ravel() for v in keys] + [Ps[v].ravel() for v in keys] + [Pr.ravel()])
    outs = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    for o in outs:
        assert np.array_equal(o, outs[0])               # every rank holds the same sum
        assert np.abs(o - want).max() <= 1e-12 * np.abs(want).max()
    # recovery from the reduced sketch equals the single-process recovery
    got = {}
    off = 0
    for v in keys:
        got[v] = outs[0][off:off + Om[v].size].reshape(Om[v].shape)
        off += Om[v].size
    gps = {}
    for v in keys:
        gps[v] = outs[0][off:off + Ps[v].size].reshape(Ps[v].shape)
        off += Ps[v].size
    gpr = outs[0][off:].reshape(Pr.shape)
    A = O.reconstruct(t, O.recover(t, got, gps, gpr)[0])
    B = O.reconstruct(t, O.recover(t, Om, Ps, Pr)[0])
    assert np.linalg.norm(A - B) <= 1e-10 * np.linalg.norm(B)


def _bench_rank_main(rank, world, port, out_dir):
    """One CPU rank of the bench's launch bookkeeping: _dist() joins the
    process group from the torchrun environment variables (gloo without a
    GPU), _barrier() and _max_over_ranks() give every rank the slowest rank's
    time, as the timed region of the multi-GPU bench does."""
    # CPU ranks even on a machine with a GPU (no two ranks on one device)
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, ws = bench._dist()
    assert (r, ws) == (rank, world)
    assert dist.get_backend() == "gloo"
    bench._barrier(ws)
    ms = 1.0 + 0.25 * rank                      # each rank's own step time
    got = bench._max_over_ranks(ms, ws)
    np.save(os.path.join(out_dir, f"bench{rank}.npy"), np.array([got]))
    bench._barrier(ws)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_bench_timing_takes_the_slowest_rank(tmp_path, world):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_bench_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        assert np.load(tmp_path / f"bench{r}.npy")[0] == 1.0 + 0.25 * (world - 1)
