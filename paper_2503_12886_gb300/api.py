"""Thin ctypes binding of librgba (include/rgba.h): the same entry points, argument marshalling
only. Every step of the rasterizer runs in the CUDA library; if the library is missing this
module raises instead of falling back to anything else."""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librgba.so")

RGBA_OK = 0
RGBA_ERR_INVALID_ARG = 1
RGBA_ERR_CAPACITY = 2
RGBA_ERR_CUDA = 3
RGBA_ERR_TIMEOUT = 4
RGBA_ERR_UNSUPPORTED = 5
RGBA_LOSS_L1 = 1
RGBA_LOSS_L2 = 2
RGBA_FP_STRIDE = 20
RGBA_NCH = 14

# every symbol include/rgba.h declares
EXPORTS = ("rgba_last_error", "rgba_create", "rgba_destroy", "rgba_workspace_size",
           "rgba_workspace_layout", "rgba_blend", "rgba_preprocess", "rgba_bin_sort",
           "rgba_render_fwd", "rgba_render_bwd", "rgba_step", "rgba_step_async",
           "rgba_profile_enable", "rgba_profile_read", "rgba_render_fwd_noalloc", "rgba_adam",
           "rgba_step_adam_async", "rgba_step_capture", "rgba_step_replay", "rgba_graph_destroy",
           "rgba_debug_keys", "rgba_color_init", "rgba_debug_render_stats")
RGBA_N_STAGES = 9
STAGES = ("upload", "preprocess", "scan", "scatter", "sort", "render_fwd", "render_bwd",
          "gauss_bwd", "dpsi_reduce")


class RgbaModel(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_pad", C.c_int32), ("k", C.c_int32), ("mask", C.c_uint32),
                ("g0", C.c_void_p), ("dg", C.c_void_p), ("grad_g0", C.c_void_p),
                ("grad_dg", C.c_void_p), ("n_faces", C.c_int32), ("n_verts", C.c_int32),
                ("faces", C.c_void_p), ("face_uv", C.c_void_p), ("face_of", C.c_void_p),
                ("bary", C.c_void_p)]


class RgbaFrame(C.Structure):
    _fields_ = [("model", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("verts", C.c_void_p)]


class RgbaBatch(C.Structure):
    _fields_ = [("n_models", C.c_int32), ("models", C.POINTER(RgbaModel)),
                ("n_frames", C.c_int32), ("frames", C.POINTER(RgbaFrame)),
                ("k_stride", C.c_int32), ("psi", C.c_void_p), ("fparams", C.c_void_p),
                ("grad_psi", C.c_void_p), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("smem_batch", C.c_int32), ("loss_frames", C.c_int32)]


class RgbaStepOut(C.Structure):
    _fields_ = [("loss", C.c_double), ("pairs", C.c_int64), ("pair_capacity", C.c_int64),
                ("pairs_needed", C.c_int64), ("overflow", C.c_uint32),
                ("device_error", C.c_uint32)]


class RgbaWsLayout(C.Structure):
    _fields_ = [("counters", C.c_size_t), ("records", C.c_size_t), ("rects", C.c_size_t),
                ("tile_start", C.c_size_t), ("sorted", C.c_size_t), ("grad2d", C.c_size_t),
                ("pix_T", C.c_size_t), ("pix_n", C.c_size_t), ("pix_dl", C.c_size_t),
                ("pix_img", C.c_size_t), ("total_bytes", C.c_size_t), ("records_total", C.c_int64),
                ("tiles_total", C.c_int64), ("pair_capacity", C.c_int64)]


class RgbaAdamCfg(C.Structure):
    _fields_ = [("lr", C.c_float * RGBA_NCH), ("lr_delta", C.c_float * RGBA_NCH),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class RgbaAdamState(C.Structure):
    _fields_ = [("m_g0", C.c_void_p), ("v_g0", C.c_void_p), ("m_dg", C.c_void_p),
                ("v_dg", C.c_void_p)]


class RgbaRenderStats(C.Structure):
    _fields_ = [("fwd_staged", C.c_int64), ("fwd_hits", C.c_int64), ("fwd_visits", C.c_int64),
                ("fwd_blends", C.c_int64), ("bwd_staged", C.c_int64), ("bwd_hits", C.c_int64),
                ("bwd_visits", C.c_int64), ("bwd_pairs", C.c_int64)]


class RgbaProfile(C.Structure):
    _fields_ = [("ms", C.c_float * RGBA_N_STAGES), ("launches", C.c_int32), ("pad_", C.c_int32)]


class RgbaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rgba error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib() -> C.CDLL:
    """Load librgba.so from the package directory (built by build.py / __graft_entry__.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"librgba.so not built at {LIB_PATH}; run the package build")
            L = C.CDLL(LIB_PATH)
            P, i32, i64, sz = C.c_void_p, C.c_int, C.c_int64, C.c_size_t
            Bp = C.POINTER(RgbaBatch)
            L.rgba_last_error.restype = C.c_char_p
            L.rgba_create.argtypes = [i32, C.POINTER(P)]
            L.rgba_destroy.argtypes = [P]
            L.rgba_destroy.restype = None
            L.rgba_workspace_size.argtypes = [Bp, i64, C.POINTER(sz)]
            L.rgba_workspace_layout.argtypes = [Bp, sz, C.POINTER(RgbaWsLayout)]
            L.rgba_blend.argtypes = [P, Bp, P, P]
            L.rgba_preprocess.argtypes = [P, Bp, P, sz, P]
            L.rgba_bin_sort.argtypes = [P, Bp, P, sz, P]
            L.rgba_render_fwd.argtypes = [P, Bp, P, sz, P, P, P, P]
            L.rgba_render_bwd.argtypes = [P, Bp, P, sz, P, P, P, P, P]
            L.rgba_step.argtypes = [P, Bp, P, sz, P, i32, P, C.POINTER(RgbaStepOut), P]
            L.rgba_step_async.argtypes = [P, Bp, P, sz, P, i32, P, P]
            L.rgba_adam.argtypes = [P, Bp, C.POINTER(RgbaAdamCfg), C.POINTER(RgbaAdamState), i32, P, P]
            L.rgba_adam.restype = i32
            L.rgba_step_adam_async.argtypes = [P, Bp, P, sz, P, i32, P, C.POINTER(RgbaAdamCfg),
                                               C.POINTER(RgbaAdamState), i32, P, P]
            L.rgba_step_adam_async.restype = i32
            L.rgba_step_capture.argtypes = [P, Bp, P, sz, P, i32, P, C.POINTER(RgbaAdamCfg),
                                            C.POINTER(RgbaAdamState), P, P, C.POINTER(P)]
            L.rgba_step_capture.restype = i32
            L.rgba_step_replay.argtypes = [P, C.POINTER(RgbaStepOut)]
            L.rgba_step_replay.restype = i32
            L.rgba_graph_destroy.argtypes = [P]
            L.rgba_graph_destroy.restype = None
            L.rgba_debug_keys.argtypes = [P, Bp, P, sz, P, P, sz, C.POINTER(i64), P]
            L.rgba_debug_keys.restype = i32
            L.rgba_debug_render_stats.argtypes = [P, Bp, P, sz, C.POINTER(RgbaRenderStats), P]
            L.rgba_debug_render_stats.restype = i32
            L.rgba_render_fwd_noalloc.argtypes = [P, Bp, P, P, P, C.POINTER(RgbaStepOut), P]
            L.rgba_color_init.argtypes = [P, Bp, P, sz, P, C.c_float, C.POINTER(P),
                                          C.POINTER(RgbaStepOut), P]
            L.rgba_render_fwd_noalloc.restype = i32
            L.rgba_profile_enable.argtypes = [P, i32]
            L.rgba_profile_read.argtypes = [P, C.POINTER(RgbaProfile)]
            for name in ("rgba_profile_enable", "rgba_profile_read", "rgba_create", "rgba_workspace_size", "rgba_workspace_layout",
                         "rgba_blend", "rgba_preprocess", "rgba_bin_sort", "rgba_render_fwd",
                         "rgba_render_bwd", "rgba_step", "rgba_step_async"):
                getattr(L, name).restype = i32
            _lib = L
    return _lib


def last_error() -> str:
    return lib().rgba_last_error().decode()


def check(rc: int) -> int:
    if rc != RGBA_OK:
        raise RgbaError(rc, last_error())
    return rc


def rgba_create(device: int = 0) -> int:
    h = C.c_void_p()
    check(lib().rgba_create(device, C.byref(h)))
    return h.value


def rgba_destroy(ctx: int) -> None:
    lib().rgba_destroy(ctx)


def rgba_workspace_size(batch: RgbaBatch, pair_capacity: int) -> int:
    n = C.c_size_t()
    check(lib().rgba_workspace_size(C.byref(batch), pair_capacity, C.byref(n)))
    return n.value


def rgba_workspace_layout(batch: RgbaBatch, ws_bytes: int) -> RgbaWsLayout:
    out = RgbaWsLayout()
    check(lib().rgba_workspace_layout(C.byref(batch), ws_bytes, C.byref(out)))
    return out


def rgba_blend(ctx, batch, out_ptr, stream) -> int:
    return check(lib().rgba_blend(ctx, C.byref(batch), out_ptr, stream))


def rgba_preprocess(ctx, batch, ws, ws_bytes, stream) -> int:
    return check(lib().rgba_preprocess(ctx, C.byref(batch), ws, ws_bytes, stream))


def rgba_bin_sort(ctx, batch, ws, ws_bytes, stream) -> int:
    return check(lib().rgba_bin_sort(ctx, C.byref(batch), ws, ws_bytes, stream))


def rgba_render_fwd(ctx, batch, ws, ws_bytes, img, T_final, n_contrib, stream) -> int:
    return check(lib().rgba_render_fwd(ctx, C.byref(batch), ws, ws_bytes, img, T_final,
                                       n_contrib, stream))


def rgba_render_bwd(ctx, batch, ws, ws_bytes, dL_dimg, T_final, n_contrib, grad_blended,
                    stream) -> int:
    """grad_blended: device pointer for the per-frame dL/dG^psi_b (layout of rgba_blend's
    out), or None."""
    return check(lib().rgba_render_bwd(ctx, C.byref(batch), ws, ws_bytes, dL_dimg, T_final,
                                       n_contrib, grad_blended, stream))


def rgba_step(ctx, batch, ws, ws_bytes, target, loss_kind, img, stream) -> tuple[int, RgbaStepOut]:
    """Returns (status, out); RGBA_ERR_CAPACITY is returned, not raised, so callers can grow
    the workspace and retry."""
    out = RgbaStepOut()
    rc = lib().rgba_step(ctx, C.byref(batch), ws, ws_bytes, target, loss_kind, img,
                         C.byref(out), stream)
    if rc not in (RGBA_OK, RGBA_ERR_CAPACITY):
        check(rc)
    return rc, out


def rgba_color_init(ctx, batch, ws, ws_bytes, target, delta, done, stream) -> tuple[int, RgbaStepOut]:
    """done: per model a device pointer (uint8[n]) or None. Returns (status, out) like
    rgba_step (RGBA_ERR_CAPACITY returned, not raised)."""
    arr = (C.c_void_p * max(1, len(done)))(*done)
    out = RgbaStepOut()
    rc = lib().rgba_color_init(ctx, C.byref(batch), ws, ws_bytes, target, delta, arr,
                               C.byref(out), stream)
    if rc not in (RGBA_OK, RGBA_ERR_CAPACITY):
        check(rc)
    return rc, out


def rgba_step_async(ctx, batch, ws, ws_bytes, target, loss_kind, img, stream) -> int:
    return check(lib().rgba_step_async(ctx, C.byref(batch), ws, ws_bytes, target, loss_kind,
                                       img, stream))


def rgba_profile_enable(ctx, on) -> int:
    """on: False / 0 off, True / 1 stage timing, 2 stage timing and compositing statistics."""
    return check(lib().rgba_profile_enable(ctx, int(on)))


def rgba_debug_render_stats(ctx, batch, ws, ws_bytes, stream) -> dict:
    """The compositing statistics counted on this workspace (profiling mode 2)."""
    out = RgbaRenderStats()
    check(lib().rgba_debug_render_stats(ctx, C.byref(batch), ws, ws_bytes, C.byref(out), stream))
    return {name: int(getattr(out, name)) for name, _ in RgbaRenderStats._fields_}


def rgba_profile_read(ctx) -> dict:
    out = RgbaProfile()
    check(lib().rgba_profile_read(ctx, C.byref(out)))
    d = {name: float(out.ms[i]) for i, name in enumerate(STAGES)}
    d["launches"] = int(out.launches)
    return d


def rgba_render_fwd_noalloc(ctx, batch, img, T_final, n_contrib, stream) -> tuple[int, RgbaStepOut]:
    """Forward render with the library's fixed scratch block (no device allocation). Returns
    (status, out); RGBA_ERR_CAPACITY is returned, not raised."""
    out = RgbaStepOut()
    rc = lib().rgba_render_fwd_noalloc(ctx, C.byref(batch), img, T_final, n_contrib,
                                       C.byref(out), stream)
    if rc not in (RGBA_OK, RGBA_ERR_CAPACITY):
        check(rc)
    return rc, out


def rgba_step_adam_async(ctx, batch, ws, ws_bytes, target, loss_kind, img, cfg: RgbaAdamCfg, states,
                         step: int, step_dev, stream) -> int:
    """rgba_step_async + rgba_adam with the update fused into the backward (see rgba.h)."""
    return check(lib().rgba_step_adam_async(ctx, C.byref(batch), ws, ws_bytes, target, loss_kind, img,
                                            C.byref(cfg), states, step, step_dev, stream))


def rgba_step_capture(ctx, batch, ws, ws_bytes, target, loss_kind, img, cfg, states, step_dev,
                      stream):
    """Captures a training step (and the Adam update when cfg is not None) as a CUDA graph;
    returns the graph handle. See rgba.h."""
    g = C.c_void_p()
    check(lib().rgba_step_capture(ctx, C.byref(batch), ws, ws_bytes, target, loss_kind, img,
                                  C.byref(cfg) if cfg is not None else None, states, step_dev,
                                  stream, C.byref(g)))
    return g


def rgba_step_replay(graph) -> tuple[int, RgbaStepOut]:
    """One replay and its host synchronisation: (status, out); RGBA_ERR_CAPACITY is returned,
    not raised."""
    out = RgbaStepOut()
    rc = lib().rgba_step_replay(graph, C.byref(out))
    if rc not in (RGBA_OK, RGBA_ERR_CAPACITY):
        check(rc)
    return rc, out


def rgba_graph_destroy(graph) -> None:
    lib().rgba_graph_destroy(graph)


def rgba_debug_keys(ctx, batch, ws, ws_bytes, tile_start, sorted_, sorted_cap, stream) -> int:
    """Copies the last binning's tile starts and sorted lists (device pointers, or None);
    returns the pair count."""
    n = C.c_int64()
    check(lib().rgba_debug_keys(ctx, C.byref(batch), ws, ws_bytes, tile_start, sorted_, sorted_cap,
                                C.byref(n), stream))
    return int(n.value)


def rgba_adam(ctx, batch, cfg: RgbaAdamCfg, states, step: int, step_dev, stream) -> int:
    """states: ctypes array of RgbaAdamState, one per model of the batch; step_dev: device
    int32 pointer (completed steps, advanced on the device) or None to use `step`."""
    return check(lib().rgba_adam(ctx, C.byref(batch), C.byref(cfg), states, step, step_dev,
                                 stream))
