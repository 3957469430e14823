"""ctypes signatures of include/ttnn.h (argument marshalling only)."""
import ctypes as C

c_i32, c_i64, c_u64, c_dbl, c_vp, c_sz = C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_void_p, C.c_size_t


class TtnnTree(C.Structure):
    _fields_ = [("n_nodes", c_i32), ("parent", C.POINTER(c_i32)),
                ("leaf_mode_ptr", C.POINTER(c_i32)), ("leaf_modes", C.POINTER(c_i32)),
                ("identity", C.POINTER(C.c_uint8))]


class TtnnOpts(C.Structure):
    _fields_ = [("variant", c_i32), ("sketch_dtype", c_i32), ("eps_factor", c_dbl),
                ("unit_roundoff", c_dbl), ("flags", C.c_uint32)]


class TtnnNodeInfo(C.Structure):
    _fields_ = [("user_index", c_i32), ("lex_index", c_i32), ("level", c_i32), ("parent", c_i32),
                ("n_children", c_i32), ("mode_lo", c_i32), ("mode_hi", c_i32), ("is_leaf", c_i32),
                ("identity", c_i32), ("r", c_i32), ("p", c_i32), ("s", c_i32), ("n", c_i64),
                ("omega_offset", c_i64), ("omega_elems", c_i64), ("psi_offset", c_i64),
                ("psi_elems", c_i64), ("psi_ndim", c_i32), ("psi_shape", c_i64 * 10),
                ("core_offset", c_i64), ("core_elems", c_i64), ("core_ndim", c_i32),
                ("core_shape", c_i64 * 10), ("kept_rank", c_i32),
                ("jacobi_sweeps", c_i32)]


class TtnnServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", c_i64), ("max_batch", c_i32), ("queue_capacity", c_i32),
                ("workers", c_i32), ("stream_queue_capacity", c_i32)]


class TtnnServerReport(C.Structure):
    _fields_ = [("completed_updates", c_i64), ("completed_recoveries", c_i64), ("failed", c_i64),
                ("batches", c_i64), ("update_bytes", c_i64), ("p50_us", c_dbl), ("p99_us", c_dbl),
                ("max_us", c_dbl), ("seconds", c_dbl), ("device_bytes", c_i64),
                ("open_streams", c_i32), ("queued", c_i64), ("worker_host_s", c_dbl)]


SIGS = {
    "ttnn_status_string": (C.c_char_p, [c_i32]),
    "ttnn_last_error": (c_i32, [C.c_char_p, c_sz]),
    "ttnn_debug_fail_alloc": (c_i32, [c_i32]),
    "ttnn_philox_gaussian": (c_i32, [c_u64, c_i32, c_i32, c_i64, c_i64, c_i32, c_vp, c_vp]),
    "ttnn_plan_create": (c_i32, [C.POINTER(TtnnTree), c_i32, C.POINTER(c_i64), C.POINTER(c_i32),
                                 C.POINTER(c_i32), c_u64, C.POINTER(TtnnOpts), c_vp, C.POINTER(c_vp)]),
    "ttnn_plan_destroy": (None, [c_vp]),
    "ttnn_plan_device_bytes": (c_i32, [c_vp, C.POINTER(c_i64), C.POINTER(c_i64)]),
    "ttnn_plan_sizes": (c_i32, [c_vp, C.POINTER(c_i64), C.POINTER(c_i32), C.POINTER(c_i64),
                                C.POINTER(c_i32)]),
    "ttnn_plan_node": (c_i32, [c_vp, c_i32, C.POINTER(TtnnNodeInfo)]),
    "ttnn_plan_factor": (c_i32, [c_vp, c_i32, c_i32, c_vp, C.POINTER(c_i64), C.POINTER(c_i64), c_vp]),
    "ttnn_state_create": (c_i32, [c_vp, c_vp, C.POINTER(c_vp)]),
    "ttnn_state_destroy": (None, [c_vp]),
    "ttnn_state_zero": (c_i32, [c_vp, c_vp]),
    "ttnn_state_buffer": (c_i32, [c_vp, C.POINTER(c_vp), C.POINTER(c_i64)]),
    "ttnn_state_axpy": (c_i32, [c_vp, c_vp, c_dbl, c_vp]),
    "ttnn_state_save": (c_i32, [c_vp, c_vp, c_sz, c_vp]),
    "ttnn_state_load": (c_i32, [c_vp, c_vp, c_sz, c_vp]),
    "ttnn_update_dense": (c_i32, [c_vp, c_vp, C.POINTER(c_i64), C.POINTER(c_i64), c_vp, c_dbl, c_vp]),
    "ttnn_update_dense_static": (c_i32, [c_vp, c_vp, C.POINTER(c_i64), C.POINTER(c_i64), c_vp, c_dbl,
                                         c_vp]),
    "ttnn_update_cp": (c_i32, [c_vp, c_i32, C.POINTER(c_dbl), C.POINTER(c_vp), c_dbl, c_vp]),
    "ttnn_update_ttn": (c_i32, [c_vp, C.POINTER(c_vp), C.POINTER(c_i32), c_dbl, c_vp]),
    "ttnn_recover": (c_i32, [c_vp, c_vp, c_vp]),
    "ttnn_recover_async": (c_i32, [c_vp, c_vp, c_vp]),
    "ttnn_plan_sync": (c_i32, [c_vp]),
    "sttnn_run": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "ttnn_hmt": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "ttnn_round": (c_i32, [c_vp, C.POINTER(c_vp), C.POINTER(c_i32), c_vp, c_vp]),
    "ttnn_fp8_quantize": (c_i32, [c_vp, c_vp, C.POINTER(c_i64), c_vp, c_vp, c_vp]),
    "ttnn_profile": (c_i32, [c_vp, c_i32]),
    "ttnn_profile_read": (c_i32, [c_vp, c_i32, C.POINTER(c_dbl), C.POINTER(c_i32)]),
    "ttnn_kernel_launches": (c_i32, [C.POINTER(c_i64)]),
    "ttnn_plan_pass_counts": (c_i32, [c_vp, C.POINTER(c_i64), C.POINTER(c_i64)]),
    "ttnn_server_create": (c_i32, [C.POINTER(TtnnServerOpts), C.POINTER(c_vp)]),
    "ttnn_server_destroy": (None, [c_vp]),
    "ttnn_server_open": (c_i32, [c_vp, C.POINTER(TtnnTree), c_i32, C.POINTER(c_i64),
                                 C.POINTER(c_i32), C.POINTER(c_i32), c_u64, C.POINTER(TtnnOpts),
                                 C.POINTER(c_i32)]),
    "ttnn_server_close": (c_i32, [c_vp, c_i32, c_i64]),
    "ttnn_server_submit": (c_i32, [c_vp, c_i32, c_vp, C.POINTER(c_i64), C.POINTER(c_i64), c_vp,
                                   c_dbl, C.POINTER(c_u64)]),
    "ttnn_server_recover": (c_i32, [c_vp, c_i32, c_vp, C.POINTER(c_u64)]),
    "ttnn_server_wait": (c_i32, [c_vp, c_u64, c_i64, C.POINTER(c_i32)]),
    "ttnn_server_stream_state": (c_i32, [c_vp, c_i32, C.POINTER(c_vp)]),
    "ttnn_server_stats": (c_i32, [c_vp, c_i32, C.POINTER(TtnnServerReport)]),
}


def declare(lib):
    for name, (res, args) in SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
