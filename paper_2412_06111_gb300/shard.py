"""Multi-GPU sharding of the sketch phase (Sec. 4: the sketches are linear in
the tensor).  One process per GPU owns a slab of the tensor along one mode,
folds it into its own state with a box update, and one sum all-reduce of the
states gives every rank the sketch of the whole tensor; recovery then runs on
any rank.  The DRMs are regenerated from the seed on every rank, so nothing
else is exchanged.  Argument marshalling and the collective only: the
sketch arithmetic runs in the library's kernels."""
from . import api


def shard_box(dims, world, rank, mode=0):
    """(offset, extent) of `rank`'s slab: contiguous along `mode`, sizes differ
    by at most one; the slabs of ranks 0..world-1 partition the tensor.  An
    extent of 0 on `mode` means the rank owns nothing."""
    n = int(dims[mode])
    lo, hi = rank * n // world, (rank + 1) * n // world
    off = [0] * len(dims)
    ext = [int(x) for x in dims]
    off[mode], ext[mode] = lo, hi - lo
    return off, ext


class _DeviceArray:
    """__cuda_array_interface__ view of a raw device buffer."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def state_tensor(plan, state):
    """A torch CUDA tensor aliasing the state's accumulator buffer (binary64
    for TTNN_F64 plans, binary32 otherwise): writes go to the state."""
    import torch
    ptr, n = api.ttnn_state_buffer(state)
    eb = api.ttnn_plan_sizes(plan)[1]
    typestr = "<f8" if eb == 8 else "<f4"
    return torch.as_tensor(_DeviceArray(ptr, n, typestr), device="cuda")


def allreduce_(tensor, group=None):
    """Sum of every rank's tensor, in place (NCCL for CUDA tensors, gloo for
    host tensors)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor


def allreduce_state_(plan, state, stream=None, group=None):
    """Sums the states of all ranks in place (one collective per step)."""
    import torch
    t = state_tensor(plan, state)
    if stream is not None:
        with torch.cuda.stream(stream):
            return allreduce_(t, group)
    return allreduce_(t, group)
