"""ctypes binding of libmaskgs (``include/maskgs.h``).

Argument marshalling only: every function here has the name of the C entry
point it calls and forwards plain pointers and sizes.  Device pointers may be
given as ints or as torch tensors (their ``data_ptr()``).  Importing this
module loads the library and raises if it is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

(MG_OK, MG_ERR_INVALID_ARG, MG_ERR_CUDA, MG_ERR_CAPACITY, MG_ERR_TIMEOUT, MG_ERR_UNSUPPORTED,
 MG_ERR_BOUNDS) = range(7)
MG_MASK_GUMBEL, MG_MASK_ALL_ONES, MG_MASK_GIVEN, MG_MASK_STE = 0, 1, 2, 3
MG_APPLY_RASTER, MG_APPLY_OPACITY = 0, 1
MG_MASK_LOSS_L2, MG_MASK_LOSS_L1 = 0, 1
MG_BIN_FILTERED, MG_BIN_RECT = 0, 1
MG_DTYPE_F32, MG_DTYPE_BF16, MG_DTYPE_F16 = 0, 1, 2
MG_MAX_VIEWS = 64
MG_RECORD_FLOATS = 12
MG_GRAD2D_FLOATS = 12

EXPORTED = ("mg_preprocess", "mg_depth_order", "mg_depth_order_workspace_bytes", "mg_bin",
            "mg_bin_noalloc", "mg_bin_workspace_bytes", "mg_sort",
            "mg_sort_workspace_bytes", "mg_sort_by_tile", "mg_sort_by_tile_workspace_bytes", "mg_tile_bits", "mg_total_tiles", "mg_render", "mg_render_l1", "mg_render_l1_reset2d",
            "mg_l1_loss_grad", "mg_render_backward", "mg_render_backward_accumulate",
            "mg_preprocess_backward",
            "mg_mask_loss", "mg_advance_iteration", "mg_prune_sample", "mg_compact", "mg_compact_workspace_bytes",
            "mg_render_inference", "mg_tile_order", "mg_read_status", "mg_status_string",
            "mg_version", "mg_selftest_wait_timeout", "mg_selftest_warp_wait_timeout",
            "mg_validate_lists")


class MaskgsError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} failed: {status_string(status)} ({status})")


class mg_status_word(C.Structure):
    _fields_ = [("status", C.c_int32), ("detail", C.c_int32), ("required", C.c_uint64)]


class mg_gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("dtype", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("mask_logits", C.c_void_p)]


class mg_camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("viewmat", C.c_float * 12), ("cam_pos", C.c_float * 3),
                ("near_plane", C.c_float)]


class mg_view(C.Structure):
    _fields_ = [("cam", mg_camera), ("gaussian_offset", C.c_int64),
                ("gaussian_count", C.c_int64)]


class mg_raster_cfg(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("bg", C.c_float * 3),
                ("tau", C.c_float), ("seed", C.c_uint64), ("iteration", C.c_uint64),
                ("mask_mode", C.c_int32), ("mask_apply", C.c_int32), ("given_mask", C.c_void_p),
                ("lambda_m", C.c_float), ("mask_loss", C.c_int32), ("ste_logit", C.c_float),
                ("bin_mode", C.c_int32), ("render_batch", C.c_int32),
                ("render_batch_bwd", C.c_int32), ("iteration_dev", C.c_void_p)]


class mg_splats(C.Structure):
    _fields_ = [("record", C.c_void_p), ("tiles_touched", C.c_void_p), ("radius", C.c_void_p),
                ("clamp", C.c_void_p), ("bin_record", C.c_void_p), ("mask", C.c_void_p),
                ("mask_soft", C.c_void_p), ("mask_count", C.c_void_p), ("depth_key", C.c_void_p)]


class mg_gaussian_arrays(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("mask_logits", C.c_void_p)]


class mg_param_grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("mask_logits", C.c_void_p)]


_P = C.POINTER
_lib = None


def debug_library() -> bool:
    """MASKGS_LIBRARY=debug selects the build with the in-kernel bounds checks."""
    return os.environ.get("MASKGS_LIBRARY", "") == "debug"


def lib_path() -> str:
    return _build.DEBUG_LIB if debug_library() else _build.LIB


def load(build_if_missing: bool = True):
    """Load libmaskgs.so, or libmaskgs_debug.so under MASKGS_LIBRARY=debug
    (building it first when absent and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing:
        path = _build.build(debug=debug_library())
    if not os.path.exists(path):
        raise RuntimeError(f"libmaskgs not found at {path}; run paper_2412_20522_gb300/build.py")
    lib = C.CDLL(path)
    st = C.c_int
    vp = C.c_void_p
    sig = {
        "mg_preprocess": (st, [_P(mg_gaussians), _P(mg_view), C.c_int32, _P(mg_raster_cfg),
                               _P(mg_splats), vp, vp]),
        "mg_depth_order": (st, [_P(mg_splats), _P(mg_view), C.c_int32, _P(mg_raster_cfg), vp,
                                vp, vp, vp, vp, C.c_size_t, vp, vp]),
        "mg_depth_order_workspace_bytes": (C.c_size_t, [C.c_int64]),
        "mg_bin": (st, [_P(mg_splats), _P(mg_view), C.c_int32, _P(mg_raster_cfg), vp, vp, vp, vp,
                        C.c_uint64, vp, vp, C.c_size_t, vp, vp]),
        "mg_bin_noalloc": (st, [_P(mg_splats), _P(mg_view), C.c_int32, _P(mg_raster_cfg), vp,
                                vp, vp, vp, C.c_uint64, vp, vp, vp]),
        "mg_bin_workspace_bytes": (C.c_size_t, [C.c_int64]),
        "mg_sort": (st, [vp, vp, vp, vp, vp, C.c_uint64, C.c_int32, vp, C.c_int64, vp,
                         C.c_size_t, _P(C.c_int32), vp, vp, vp]),
        "mg_sort_workspace_bytes": (C.c_size_t, [C.c_uint64, C.c_int32]),
        "mg_sort_by_tile": (st, [vp, vp, vp, vp, C.c_uint64, C.c_int64, vp, vp, vp,
                                 C.c_size_t, vp, vp, vp]),
        "mg_sort_by_tile_workspace_bytes": (C.c_size_t, [C.c_uint64, C.c_int64]),
        "mg_tile_bits": (C.c_int32, [_P(mg_view), C.c_int32, _P(mg_raster_cfg)]),
        "mg_total_tiles": (C.c_int64, [_P(mg_view), C.c_int32, _P(mg_raster_cfg)]),
        "mg_render": (st, [_P(mg_splats), vp, vp, vp, _P(mg_view), C.c_int32,
                           _P(mg_raster_cfg), vp, vp, vp, vp, vp]),
        "mg_render_l1": (st, [_P(mg_splats), vp, vp, vp, _P(mg_view), C.c_int32,
                              _P(mg_raster_cfg), vp, vp, vp, vp, vp, vp, vp]),
        "mg_render_l1_reset2d": (st, [_P(mg_splats), vp, vp, vp, _P(mg_view), C.c_int32,
                                      _P(mg_raster_cfg), vp, vp, vp, vp, vp, vp, vp, vp]),
        "mg_tile_order": (st, [vp, C.c_int64, vp, vp]),
        "mg_l1_loss_grad": (st, [vp, vp, _P(mg_view), C.c_int32, vp, vp, vp]),
        "mg_render_backward": (st, [_P(mg_splats), vp, vp, vp, _P(mg_view), C.c_int32,
                                    _P(mg_raster_cfg), vp, vp, vp, vp, vp, vp]),
        "mg_render_backward_accumulate": (st, [_P(mg_splats), vp, vp, vp, _P(mg_view),
                                               C.c_int32, _P(mg_raster_cfg), vp, vp, vp, vp, vp,
                                               vp]),
        "mg_preprocess_backward": (st, [_P(mg_gaussians), _P(mg_view), C.c_int32,
                                        _P(mg_raster_cfg), _P(mg_splats), vp,
                                        _P(mg_param_grads), vp]),
        "mg_mask_loss": (st, [_P(mg_splats), _P(mg_view), C.c_int32, _P(mg_raster_cfg), vp, vp]),
        "mg_advance_iteration": (st, [vp, C.c_uint64, vp]),
        "mg_prune_sample": (st, [_P(mg_gaussians), C.c_uint64, C.c_uint64, C.c_int32, vp, vp]),
        "mg_compact": (st, [_P(mg_gaussians), vp, _P(mg_gaussian_arrays), vp, vp, vp, C.c_size_t,
                            vp, vp]),
        "mg_compact_workspace_bytes": (C.c_size_t, [C.c_int64]),
        "mg_render_inference": (st, [_P(mg_splats), vp, vp, vp, _P(mg_view), C.c_int32,
                                     _P(mg_raster_cfg), vp, vp]),
        "mg_read_status": (st, [vp, _P(mg_status_word), vp]),
        "mg_status_string": (C.c_char_p, [C.c_int32]),
        "mg_version": (C.c_char_p, []),
        "mg_selftest_wait_timeout": (st, [C.c_int32, vp, vp]),
        "mg_selftest_warp_wait_timeout": (st, [C.c_int32, vp, vp]),
        "mg_validate_lists": (st, [vp, vp, C.c_int64, vp, C.c_uint64, C.c_int64, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def ptr(x) -> int | None:
    """Device address of a tensor (or an int / None passed through)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _check(fn, status):
    if status != MG_OK:
        raise MaskgsError(fn, status)


def status_string(status: int) -> str:
    return load().mg_status_string(int(status)).decode()


def version() -> str:
    return load().mg_version().decode()


def mg_preprocess(g, views, n_views, cfg, out, d_status, stream):
    _check("mg_preprocess", load().mg_preprocess(C.byref(g), views, n_views, C.byref(cfg),
                                                 C.byref(out), ptr(d_status), stream))


def mg_depth_order(splats, views, n_views, cfg, order, order_alt, keys, keys_alt, workspace,
                   workspace_bytes, d_status, stream):
    _check("mg_depth_order", load().mg_depth_order(
        C.byref(splats), views, n_views, C.byref(cfg), ptr(order), ptr(order_alt), ptr(keys),
        ptr(keys_alt), ptr(workspace), workspace_bytes, ptr(d_status), stream))


def mg_depth_order_workspace_bytes(n_records) -> int:
    return int(load().mg_depth_order_workspace_bytes(n_records))


def mg_bin(splats, views, n_views, cfg, order, offsets, keys, vals, capacity, d_num_instances,
           workspace, workspace_bytes, d_status, stream):
    _check("mg_bin", load().mg_bin(C.byref(splats), views, n_views, C.byref(cfg), ptr(order),
                                   ptr(offsets), ptr(keys), ptr(vals), capacity,
                                   ptr(d_num_instances), ptr(workspace), workspace_bytes,
                                   ptr(d_status), stream))


def mg_bin_noalloc(splats, views, n_views, cfg, order, offsets, keys, vals, capacity,
                   d_num_instances, d_status, stream):
    """mg_bin for callers that cannot allocate: its scratch is a fixed array
    inside the library (at most 2^24 records; concurrent calls race)."""
    _check("mg_bin_noalloc", load().mg_bin_noalloc(C.byref(splats), views, n_views, C.byref(cfg),
                                                   ptr(order), ptr(offsets), ptr(keys), ptr(vals),
                                                   capacity, ptr(d_num_instances), ptr(d_status),
                                                   stream))


def mg_bin_workspace_bytes(n_records) -> int:
    return int(load().mg_bin_workspace_bytes(n_records))


def mg_sort(keys, vals, keys_alt, vals_alt, d_num_instances, capacity, key_bits, ranges,
            n_tiles_total, workspace, workspace_bytes, d_num_sorted, d_status, stream) -> int:
    alt = C.c_int32(0)
    _check("mg_sort", load().mg_sort(ptr(keys), ptr(vals), ptr(keys_alt), ptr(vals_alt),
                                     ptr(d_num_instances), capacity, key_bits, ptr(ranges),
                                     n_tiles_total, ptr(workspace), workspace_bytes,
                                     C.byref(alt), ptr(d_num_sorted), ptr(d_status), stream))
    return int(alt.value)


def mg_sort_workspace_bytes(capacity, key_bits) -> int:
    return int(load().mg_sort_workspace_bytes(capacity, key_bits))


def mg_sort_by_tile(keys, vals, depth_key, d_num_instances, capacity, n_tiles_total,
                    sorted_vals, ranges, workspace, workspace_bytes, d_num_sorted, d_status,
                    stream):
    _check("mg_sort_by_tile", load().mg_sort_by_tile(
        ptr(keys), ptr(vals), ptr(depth_key), ptr(d_num_instances), capacity, n_tiles_total,
        ptr(sorted_vals), ptr(ranges), ptr(workspace), workspace_bytes,
        ptr(d_num_sorted), ptr(d_status), stream))


def mg_sort_by_tile_workspace_bytes(capacity, n_tiles_total) -> int:
    return int(load().mg_sort_by_tile_workspace_bytes(capacity, n_tiles_total))


def mg_tile_bits(views, n_views, cfg) -> int:
    return int(load().mg_tile_bits(views, n_views, C.byref(cfg)))


def mg_total_tiles(views, n_views, cfg) -> int:
    return int(load().mg_total_tiles(views, n_views, C.byref(cfg)))


def mg_tile_order(ranges, n_tiles_total, tile_order, stream):
    _check("mg_tile_order", load().mg_tile_order(ptr(ranges), n_tiles_total, ptr(tile_order),
                                                 stream))


def mg_render(splats, sorted_vals, ranges, tile_order, views, n_views, cfg, image, final_T,
              n_contrib, frag_count, stream):
    _check("mg_render", load().mg_render(C.byref(splats), ptr(sorted_vals), ptr(ranges),
                                         ptr(tile_order), views, n_views, C.byref(cfg),
                                         ptr(image), ptr(final_T), ptr(n_contrib),
                                         ptr(frag_count), stream))


def mg_render_l1(splats, sorted_vals, ranges, tile_order, views, n_views, cfg, image, final_T,
                 n_contrib, target, dL_dimage, loss, stream):
    _check("mg_render_l1", load().mg_render_l1(
        C.byref(splats), ptr(sorted_vals), ptr(ranges), ptr(tile_order), views, n_views,
        C.byref(cfg), ptr(image), ptr(final_T), ptr(n_contrib), ptr(target), ptr(dL_dimage),
        ptr(loss), stream))


def mg_render_l1_reset2d(splats, sorted_vals, ranges, tile_order, views, n_views, cfg, image,
                         final_T, n_contrib, target, dL_dimage, loss, grad2d, stream):
    """mg_render_l1 that also zeroes grad2d for mg_render_backward_accumulate."""
    _check("mg_render_l1_reset2d", load().mg_render_l1_reset2d(
        C.byref(splats), ptr(sorted_vals), ptr(ranges), ptr(tile_order), views, n_views,
        C.byref(cfg), ptr(image), ptr(final_T), ptr(n_contrib), ptr(target), ptr(dL_dimage),
        ptr(loss), ptr(grad2d), stream))


def mg_l1_loss_grad(image, target, views, n_views, dL_dimage, loss, stream):
    _check("mg_l1_loss_grad", load().mg_l1_loss_grad(ptr(image), ptr(target), views, n_views,
                                                     ptr(dL_dimage), ptr(loss), stream))


def mg_render_backward(splats, sorted_vals, ranges, tile_order, views, n_views, cfg, final_T,
                       n_contrib, dL_dimage, grad2d, counters, stream):
    _check("mg_render_backward", load().mg_render_backward(
        C.byref(splats), ptr(sorted_vals), ptr(ranges), ptr(tile_order), views, n_views,
        C.byref(cfg),
        ptr(final_T), ptr(n_contrib), ptr(dL_dimage), ptr(grad2d), ptr(counters), stream))


def mg_render_backward_accumulate(splats, sorted_vals, ranges, tile_order, views, n_views, cfg,
                                  final_T, n_contrib, dL_dimage, grad2d, counters, stream):
    """mg_render_backward adding into grad2d, which the caller has zeroed."""
    _check("mg_render_backward_accumulate", load().mg_render_backward_accumulate(
        C.byref(splats), ptr(sorted_vals), ptr(ranges), ptr(tile_order), views, n_views,
        C.byref(cfg),
        ptr(final_T), ptr(n_contrib), ptr(dL_dimage), ptr(grad2d), ptr(counters), stream))


def mg_preprocess_backward(g, views, n_views, cfg, splats, grad2d, out, stream):
    _check("mg_preprocess_backward", load().mg_preprocess_backward(
        C.byref(g), views, n_views, C.byref(cfg), C.byref(splats), ptr(grad2d), C.byref(out),
        stream))


def mg_mask_loss(splats, views, n_views, cfg, loss, stream):
    _check("mg_mask_loss", load().mg_mask_loss(C.byref(splats), views, n_views, C.byref(cfg),
                                               ptr(loss), stream))


def mg_advance_iteration(iteration_dev, by, stream):
    """*iteration_dev += by on the stream (the mask sample's device-side
    iteration, read through mg_raster_cfg.iteration_dev)."""
    _check("mg_advance_iteration", load().mg_advance_iteration(ptr(iteration_dev), by, stream))


def mg_prune_sample(g, seed, iteration, n_draws, keep, stream):
    _check("mg_prune_sample", load().mg_prune_sample(C.byref(g), seed, iteration, n_draws,
                                                     ptr(keep), stream))


def mg_compact(src, keep, dst, new_index, d_n_kept, workspace, workspace_bytes, d_status, stream):
    _check("mg_compact", load().mg_compact(C.byref(src), ptr(keep), C.byref(dst), ptr(new_index),
                                           ptr(d_n_kept), ptr(workspace), workspace_bytes,
                                           ptr(d_status), stream))


def mg_compact_workspace_bytes(n) -> int:
    return int(load().mg_compact_workspace_bytes(n))


def mg_render_inference(splats, sorted_vals, ranges, tile_order, views, n_views, cfg, image,
                        stream):
    _check("mg_render_inference", load().mg_render_inference(
        C.byref(splats), ptr(sorted_vals), ptr(ranges), ptr(tile_order), views, n_views,
        C.byref(cfg), ptr(image), stream))


def mg_selftest_wait_timeout(max_polls, d_status, stream):
    _check("mg_selftest_wait_timeout", load().mg_selftest_wait_timeout(max_polls, ptr(d_status),
                                                                       stream))


def mg_selftest_warp_wait_timeout(max_polls, d_status, stream):
    _check("mg_selftest_warp_wait_timeout",
           load().mg_selftest_warp_wait_timeout(max_polls, ptr(d_status), stream))


def mg_read_status(d_status, stream) -> mg_status_word:
    h = mg_status_word()
    _check("mg_read_status", load().mg_read_status(ptr(d_status), C.byref(h), stream))
    return h


def mg_validate_lists(sorted_vals, ranges, n_tiles_total, d_num_sorted, capacity, n_records,
                      d_status, stream):
    _check("mg_validate_lists", load().mg_validate_lists(
        ptr(sorted_vals), ptr(ranges), n_tiles_total, ptr(d_num_sorted), capacity, n_records,
        ptr(d_status), stream))
