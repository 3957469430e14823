"""Python binding of the C ABI in include/ttnn.h: the same entry-point names,
argument marshalling only.  Device buffers are passed as torch CUDA tensors
(their data pointers), host arrays as Python sequences, streams as
torch.cuda.Stream or None (the current stream).  Every call runs in
libttnn.so; a failing status raises TtnnError with the library's message.
There is no fallback: without the compiled library or a GPU the calls fail.
"""
import ctypes as C

from . import _native, _sigs
from ._sigs import TtnnNodeInfo, TtnnOpts, TtnnTree

F64, F32, BF16, E4M3, BF16X2 = 0, 1, 2, 3, 4
VARIANT_TTNN, VARIANT_STTNN = 0, 1
FLAG_NO_SIDE_CACHE, FLAG_SIMT_PASS, FLAG_CLUSTER_REDUCE, FLAG_STRUCTURED_ONLY = 1, 2, 4, 8
FLAG_DUMP_PROGRAM, FLAG_WAIT_TEST, FLAG_RESERVE_SMS, FLAG_DENSE_DRM, FLAG_TRUNCATE = 16, 32, 64, 128, 256
KIND_X, KIND_Y, KIND_XT = 1, 2, 3


class TtnnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ttnn status {status}: {msg}")
        self.status = status


def _lib():
    return _native.load()


def _check(status):
    if status != 0:
        lib = _lib()
        buf = C.create_string_buffer(512)
        lib.ttnn_last_error(buf, 512)
        raise TtnnError(status, lib.ttnn_status_string(status).decode() + ": " + buf.value.decode())


def last_error_message():
    """The calling thread's last library error message."""
    buf = C.create_string_buffer(512)
    _lib().ttnn_last_error(buf, 512)
    return buf.value.decode()


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _arr(ctype, xs):
    xs = list(xs)
    return (ctype * max(len(xs), 1))(*xs)


class Tree:
    """A ttnn_tree with the host arrays it points to kept alive."""

    def __init__(self, parent, leaf_modes, identity=None):
        self.parent = _arr(C.c_int32, parent)
        ptr, modes = [0], []
        for lm in leaf_modes:
            modes.extend(int(m) for m in lm)
            ptr.append(len(modes))
        self.ptr = _arr(C.c_int32, ptr)
        self.modes = _arr(C.c_int32, modes)
        self.ident = None if identity is None else _arr(C.c_uint8, [1 if x else 0 for x in identity])
        self.c = TtnnTree(len(parent), self.parent, self.ptr, self.modes,
                          None if self.ident is None else C.cast(self.ident, C.POINTER(C.c_uint8)))


def ttnn_debug_fail_alloc(nth):
    """Testing: the nth device allocation of the library from now on fails
    (TTNN_ENOMEM); 0 disarms."""
    _check(_lib().ttnn_debug_fail_alloc(int(nth)))


def ttnn_philox_gaussian(seed, kind, ident, rows, cols, round_dtype, dst, stream=None):
    _check(_lib().ttnn_philox_gaussian(seed, kind, ident, rows, cols, round_dtype, _ptr(dst),
                                       _stream(stream)))


def ttnn_plan_create(tree, dims, ranks, oversample, seed, variant=VARIANT_TTNN, sketch_dtype=F32,
                     eps_factor=10.0, unit_roundoff=2.0 ** -52, flags=0, stream=None):
    """tree: a Tree or a (parent, leaf_modes, identity) tuple."""
    if not isinstance(tree, Tree):
        tree = Tree(*tree)
    opts = TtnnOpts(variant, sketch_dtype, eps_factor, unit_roundoff, flags)
    out = C.c_void_p()
    _check(_lib().ttnn_plan_create(C.byref(tree.c), len(dims), _arr(C.c_int64, dims),
                                   _arr(C.c_int32, ranks), _arr(C.c_int32, oversample),
                                   C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), C.byref(opts),
                                   _stream(stream), C.byref(out)))
    return out


def ttnn_plan_destroy(plan):
    _lib().ttnn_plan_destroy(plan)


def ttnn_plan_device_bytes(plan):
    """(total device bytes held by the plan, its workspace bytes)."""
    t, w = C.c_int64(), C.c_int64()
    _check(_lib().ttnn_plan_device_bytes(plan, C.byref(t), C.byref(w)))
    return t.value, w.value


def ttnn_plan_sizes(plan):
    se, eb, ce, nn = C.c_int64(), C.c_int32(), C.c_int64(), C.c_int32()
    _check(_lib().ttnn_plan_sizes(plan, C.byref(se), C.byref(eb), C.byref(ce), C.byref(nn)))
    return se.value, eb.value, ce.value, nn.value


def ttnn_plan_node(plan, user_index):
    info = TtnnNodeInfo()
    _check(_lib().ttnn_plan_node(plan, user_index, C.byref(info)))
    d = {k: getattr(info, k) for k, _ in TtnnNodeInfo._fields_}
    d["psi_shape"] = list(info.psi_shape)[:info.psi_ndim]
    d["core_shape"] = list(info.core_shape)[:info.core_ndim]
    return d


def ttnn_plan_factor(plan, which, mode, dst=None, stream=None):
    """Returns (rows, cols); copies the factor into dst (f64 CUDA tensor) if given."""
    rows, cols = C.c_int64(), C.c_int64()
    _check(_lib().ttnn_plan_factor(plan, which, mode, _ptr(dst), C.byref(rows), C.byref(cols),
                                   _stream(stream)))
    return rows.value, cols.value


def ttnn_state_create(plan, stream=None):
    out = C.c_void_p()
    _check(_lib().ttnn_state_create(plan, _stream(stream), C.byref(out)))
    return out


def ttnn_state_destroy(state):
    _lib().ttnn_state_destroy(state)


def ttnn_state_zero(state, stream=None):
    _check(_lib().ttnn_state_zero(state, _stream(stream)))


def ttnn_state_buffer(state):
    p, n = C.c_void_p(), C.c_int64()
    _check(_lib().ttnn_state_buffer(state, C.byref(p), C.byref(n)))
    return p.value, n.value


def ttnn_state_axpy(dst, src, alpha, stream=None):
    _check(_lib().ttnn_state_axpy(dst, src, C.c_double(alpha), _stream(stream)))


def ttnn_state_save(state, host_buf, stream=None):
    """host_buf: a writable contiguous numpy array of the state's size."""
    _check(_lib().ttnn_state_save(state, C.c_void_p(host_buf.ctypes.data), host_buf.nbytes,
                                  _stream(stream)))


def ttnn_state_load(state, host_buf, stream=None):
    _check(_lib().ttnn_state_load(state, C.c_void_p(host_buf.ctypes.data), host_buf.nbytes,
                                  _stream(stream)))


def ttnn_update_dense(state, data, offset=None, extent=None, tile_scale=None, lam=1.0, stream=None):
    off = None if offset is None else _arr(C.c_int64, offset)
    ext = None if extent is None else _arr(C.c_int64, extent)
    _check(_lib().ttnn_update_dense(state, _ptr(data), off, ext, _ptr(tile_scale),
                                    C.c_double(lam), _stream(stream)))


def ttnn_update_dense_static(state, data, offset=None, extent=None, tile_scale=None, lam=1.0,
                             stream=None):
    """ttnn_update_dense without device allocation: its scratch is a fixed
    32 MiB block of static device memory (one per device), so concurrent calls
    race and larger updates raise TtnnError (EINVAL)."""
    off = None if offset is None else _arr(C.c_int64, offset)
    ext = None if extent is None else _arr(C.c_int64, extent)
    _check(_lib().ttnn_update_dense_static(state, _ptr(data), off, ext, _ptr(tile_scale),
                                           C.c_double(lam), _stream(stream)))


def ttnn_update_cp(state, weights, factors, lam=1.0, stream=None):
    """weights: host sequence (cp_rank); factors: list of d f64 CUDA tensors n_mu x cp_rank."""
    fp = _arr(C.c_void_p, [f.data_ptr() for f in factors])
    _check(_lib().ttnn_update_cp(state, len(weights), _arr(C.c_double, weights), fp,
                                 C.c_double(lam), _stream(stream)))


def ttnn_update_ttn(state, cores_in, ranks_in, lam=1.0, stream=None):
    """cores_in: list (per user node) of f64 CUDA tensors; ranks_in: per node."""
    cp = _arr(C.c_void_p, [c.data_ptr() for c in cores_in])
    _check(_lib().ttnn_update_ttn(state, cp, _arr(C.c_int32, ranks_in), C.c_double(lam),
                                  _stream(stream)))


def ttnn_recover(state, cores, stream=None):
    _check(_lib().ttnn_recover(state, _ptr(cores), _stream(stream)))


def ttnn_recover_async(state, cores, stream=None):
    _check(_lib().ttnn_recover_async(state, _ptr(cores), _stream(stream)))


def ttnn_plan_sync(plan):
    _check(_lib().ttnn_plan_sync(plan))


def sttnn_run(plan, dense, cores, tile_scale=None, stream=None):
    _check(_lib().sttnn_run(plan, _ptr(dense), _ptr(tile_scale), _ptr(cores), _stream(stream)))


def ttnn_hmt(plan, dense, cores, stream=None):
    _check(_lib().ttnn_hmt(plan, _ptr(dense), _ptr(cores), _stream(stream)))


def ttnn_round(plan, cores_in, ranks_in, cores, stream=None):
    cp = _arr(C.c_void_p, [c.data_ptr() for c in cores_in])
    _check(_lib().ttnn_round(plan, cp, _arr(C.c_int32, ranks_in), _ptr(cores), _stream(stream)))


def ttnn_fp8_quantize(plan, src, dst, scales, extent=None, stream=None):
    """src: f32 CUDA tensor (whole tensor or box extents); dst: uint8 CUDA
    tensor of the same element count; scales: f32 CUDA tensor with one entry
    per 128 x 128 tile of the pass matrix."""
    ext = None if extent is None else _arr(C.c_int64, extent)
    _check(_lib().ttnn_fp8_quantize(plan, _ptr(src), ext, _ptr(dst), _ptr(scales), _stream(stream)))


def ttnn_profile(plan, enable=True):
    _check(_lib().ttnn_profile(plan, 1 if enable else 0))


def ttnn_profile_read(plan, phase):
    """(summed milliseconds, number of intervals) of a phase since the last read."""
    ms, n = C.c_double(), C.c_int32()
    _check(_lib().ttnn_profile_read(plan, phase, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def ttnn_kernel_launches():
    n = C.c_int64()
    _check(_lib().ttnn_kernel_launches(C.byref(n)))
    return n.value


def ttnn_plan_pass_counts(plan):
    """(tensor-core passes, SIMT passes) run by this plan."""
    a, b = C.c_int64(), C.c_int64()
    _check(_lib().ttnn_plan_pass_counts(plan, C.byref(a), C.byref(b)))
    return a.value, b.value


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
def ttnn_server_create(hbm_budget_bytes, max_batch=0, queue_capacity=0, workers=0,
                       stream_queue_capacity=0):
    out = C.c_void_p()
    opts = _sigs.TtnnServerOpts(int(hbm_budget_bytes), int(max_batch), int(queue_capacity),
                                int(workers), int(stream_queue_capacity))
    _check(_lib().ttnn_server_create(C.byref(opts), C.byref(out)))
    return out


def ttnn_server_destroy(server):
    _lib().ttnn_server_destroy(server)


def ttnn_server_open(server, tree, dims, ranks, oversample, seed, variant=VARIANT_TTNN,
                     sketch_dtype=F32, eps_factor=10.0, unit_roundoff=2.0 ** -52, flags=0):
    if not isinstance(tree, Tree):
        tree = Tree(*tree)
    opts = TtnnOpts(variant, sketch_dtype, eps_factor, unit_roundoff, flags)
    sid = C.c_int32()
    _check(_lib().ttnn_server_open(server, C.byref(tree.c), len(dims), _arr(C.c_int64, dims),
                                   _arr(C.c_int32, ranks), _arr(C.c_int32, oversample),
                                   C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), C.byref(opts),
                                   C.byref(sid)))
    return sid.value


def ttnn_server_close(server, stream_id, timeout_us=10_000_000):
    _check(_lib().ttnn_server_close(server, stream_id, int(timeout_us)))


def ttnn_server_submit(server, stream_id, data, offset=None, extent=None, tile_scale=None, lam=1.0):
    off = None if offset is None else _arr(C.c_int64, offset)
    ext = None if extent is None else _arr(C.c_int64, extent)
    t = C.c_uint64()
    _check(_lib().ttnn_server_submit(server, stream_id, _ptr(data), off, ext, _ptr(tile_scale),
                                     C.c_double(lam), C.byref(t)))
    return t.value


def ttnn_server_recover(server, stream_id, cores):
    t = C.c_uint64()
    _check(_lib().ttnn_server_recover(server, stream_id, _ptr(cores), C.byref(t)))
    return t.value


def ttnn_server_wait(server, ticket, timeout_us=10_000_000):
    """Returns the request's status (0 = OK); raises TtnnError on ETIMEOUT / EINVAL."""
    res = C.c_int32()
    _check(_lib().ttnn_server_wait(server, C.c_uint64(ticket), int(timeout_us), C.byref(res)))
    return res.value


def ttnn_server_stream_state(server, stream_id):
    out = C.c_void_p()
    _check(_lib().ttnn_server_stream_state(server, stream_id, C.byref(out)))
    return out


def ttnn_server_stats(server, reset=False):
    rep = _sigs.TtnnServerReport()
    _check(_lib().ttnn_server_stats(server, 1 if reset else 0, C.byref(rep)))
    return {k: getattr(rep, k) for k, _ in _sigs.TtnnServerReport._fields_}
