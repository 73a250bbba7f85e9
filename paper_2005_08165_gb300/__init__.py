"""Python binding of libtfn (include/tfn.h): Three-Filters-to-Normal on GB300.

The functions ``tfn_*`` mirror the C ABI one to one (ctypes); ``Context``
adds argument marshalling for torch tensors (device pointers, pitches, the
current CUDA stream).  Every step of the estimator runs in the library's CUDA
kernels; nothing here computes normals, and importing fails loudly if the
library has not been built.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtfn.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libtfn.so not found at {LIB_PATH}: build it first "
                      "(python -c 'import __graft_entry__ as g; g.build()' or python -m paper_2005_08165_gb300.build)")

_lib = ctypes.CDLL(LIB_PATH)

# ---- enums (tfn.h) ------------------------------------------------------------------------
TFN_OK, TFN_ERR_INVALID_ARG, TFN_ERR_UNSUPPORTED, TFN_ERR_MISALIGNED, TFN_ERR_OUT_OF_MEMORY, TFN_ERR_CUDA, \
    TFN_ERR_TIMEOUT, TFN_ERR_CANCELLED, TFN_ERR_BUSY, TFN_ERR_DEVICE, TFN_ERR_IO = range(11)
TFN_DEPTH_F32, TFN_DEPTH_F16, TFN_DISP_U16, TFN_DISP_F32 = range(4)
TFN_GRAD_FD, TFN_GRAD_SOBEL, TFN_GRAD_SCHARR, TFN_GRAD_PREWITT, TFN_GRAD_WEIGHTED, TFN_GRAD_SEP5, TFN_GRAD_FD5, \
    TFN_GRAD_SOBEL5, TFN_GRAD_PREWITT5 = range(9)
TFN_PHI_MEAN, TFN_PHI_MEDIAN = range(2)
TFN_EST_3F2N, TFN_EST_PLANEPCA = range(2)
TFN_OUT_F32, TFN_OUT_F16, TFN_OUT_BF16, TFN_OUT_F16X4, TFN_OUT_BF16X4, TFN_OUT_OCT16 = range(6)
TFN_FLAG_REFINE_ALL = 1
TFN_FLAG_TEST_WAIT_TIMEOUT = 2
TFN_FLAG_FULL_BOUND = 4
TFN_REQ_HOST = 1
TFN_REQ_TEST_WAIT_TIMEOUT = 2
TFN_SERVER_NO_GRAPHS = 1

GRADS = {"fd": TFN_GRAD_FD, "sobel": TFN_GRAD_SOBEL, "scharr": TFN_GRAD_SCHARR, "prewitt": TFN_GRAD_PREWITT,
         "weighted": TFN_GRAD_WEIGHTED, "sep5": TFN_GRAD_SEP5, "fd5": TFN_GRAD_FD5, "sobel5": TFN_GRAD_SOBEL5,
         "prewitt5": TFN_GRAD_PREWITT5}
PHIS = {"mean": TFN_PHI_MEAN, "median": TFN_PHI_MEDIAN}
OUTPUTS = {"f32": TFN_OUT_F32, "f16": TFN_OUT_F16, "bf16": TFN_OUT_BF16, "f16x4": TFN_OUT_F16X4,
           "bf16x4": TFN_OUT_BF16X4, "oct16": TFN_OUT_OCT16}


class tfn_camera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("u0", ctypes.c_float), ("v0", ctypes.c_float),
                ("baseline", ctypes.c_float)]


class tfn_frame(ctypes.Structure):
    _fields_ = [("input", ctypes.c_void_p), ("input_pitch", ctypes.c_int64),
                ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("input_type", ctypes.c_int32), ("disp_scale", ctypes.c_float),
                ("cam", tfn_camera),
                ("normals", ctypes.c_void_p), ("normals_pitch", ctypes.c_int64),
                ("normals_plane_stride", ctypes.c_int64),
                ("mask", ctypes.c_void_p), ("mask_pitch", ctypes.c_int64),
                ("points", ctypes.c_void_p), ("points_pitch", ctypes.c_int64),
                ("points_plane_stride", ctypes.c_int64)]


class tfn_method(ctypes.Structure):
    _fields_ = [("grad", ctypes.c_int32), ("phi", ctypes.c_int32), ("output", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("weights", ctypes.c_float * 5), ("estimator", ctypes.c_int32)]


class tfn_server_opts(ctypes.Structure):
    _fields_ = [("method", tfn_method), ("mem_budget_bytes", ctypes.c_size_t), ("max_batch_frames", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("max_delay_us", ctypes.c_int32), ("pipelines", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class tfn_serving_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("rejected", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("pixels", ctypes.c_uint64), ("elapsed_s", ctypes.c_double), ("frames_per_s", ctypes.c_double),
                ("mean_batch_frames", ctypes.c_double), ("latency_p50_us", ctypes.c_double),
                ("latency_p99_us", ctypes.c_double), ("latency_max_us", ctypes.c_double),
                ("latency_samples", ctypes.c_uint64), ("queued", ctypes.c_int32), ("in_flight", ctypes.c_int32),
                ("staging_bytes_in_use", ctypes.c_size_t), ("staging_bytes_capacity", ctypes.c_size_t),
                ("graph_launches", ctypes.c_uint64), ("max_batches_in_flight", ctypes.c_uint64),
                ("admitted_while_busy", ctypes.c_uint64), ("device_overlaps", ctypes.c_uint64),
                ("graph_captures", ctypes.c_uint64)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_lib.tfn_status_string.restype = ctypes.c_char_p
_lib.tfn_status_string.argtypes = [_I]
_lib.tfn_version.restype = ctypes.c_char_p
_lib.tfn_last_cuda_error.restype = ctypes.c_char_p
_lib.tfn_create.argtypes = [ctypes.POINTER(_P), _I, ctypes.c_size_t]
_lib.tfn_destroy.argtypes = [_P]
_lib.tfn_normals.argtypes = [_P, ctypes.POINTER(tfn_frame), ctypes.POINTER(tfn_method), _P]
_lib.tfn_normals_batch.argtypes = [_P, ctypes.POINTER(tfn_frame), _I, ctypes.POINTER(tfn_method), _P]
_lib.tfn_normals_batch_host.argtypes = [_P, ctypes.POINTER(tfn_frame), _I, ctypes.POINTER(tfn_method), _P]
_lib.tfn_device_status.argtypes = [_P, ctypes.POINTER(ctypes.c_uint32), _P]
_lib.tfn_tile_shape_count.restype = _I
_lib.tfn_tile_shape_info.argtypes = [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
_lib.tfn_tile_shape_info.restype = _I
_lib.tfn_tile_shape_warps.argtypes = [_I, ctypes.POINTER(_I), ctypes.POINTER(_I)]
_lib.tfn_tile_shape_warps.restype = _I
_lib.tfn_set_tile_shape.argtypes = [_P, _I]
_lib.tfn_set_tile_shape.restype = _I
_lib.tfn_plan_create.argtypes = [_P, ctypes.POINTER(tfn_frame), _I, ctypes.POINTER(tfn_method), ctypes.POINTER(_P)]
_lib.tfn_plan_launch.argtypes = [_P, _P]
_lib.tfn_plan_destroy.argtypes = [_P]
_lib.tfn_plan_kernels.argtypes = [_P, ctypes.POINTER(_I)]
_lib.tfn_plan_kernel_name.argtypes = [_P, _I, ctypes.POINTER(ctypes.c_char_p)]
_lib.tfn_refined_pixels.argtypes = [_P, ctypes.POINTER(ctypes.c_uint64), _P]
_lib.tfn_normals_noalloc.argtypes = [ctypes.POINTER(tfn_frame), _I, ctypes.POINTER(tfn_method), _P]
_lib.tfn_autotune.argtypes = [_P, ctypes.POINTER(tfn_frame), _I, ctypes.POINTER(tfn_method), _I, _P,
                              ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)]
_lib.tfn_tuned_shape.argtypes = [_P, _I, ctypes.POINTER(tfn_method), ctypes.POINTER(_I)]
_lib.tfn_tune_cache_save.argtypes = [_P, ctypes.c_char_p]
_lib.tfn_tune_cache_load.argtypes = [_P, ctypes.c_char_p]
_lib.tfn_server_create.argtypes = [_P, ctypes.POINTER(tfn_server_opts), ctypes.POINTER(_P)]
_lib.tfn_submit.argtypes = [_P, ctypes.POINTER(tfn_frame), _I, ctypes.POINTER(ctypes.c_uint64)]
_lib.tfn_wait.argtypes = [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(_I)]
_lib.tfn_server_stats.argtypes = [_P, ctypes.POINTER(tfn_serving_stats), _I]
_lib.tfn_server_destroy.argtypes = [_P]
for _f in ("tfn_create", "tfn_destroy", "tfn_normals", "tfn_normals_batch", "tfn_normals_batch_host",
           "tfn_device_status", "tfn_refined_pixels", "tfn_normals_noalloc", "tfn_plan_create", "tfn_plan_launch",
           "tfn_plan_destroy", "tfn_plan_kernels", "tfn_plan_kernel_name", "tfn_autotune", "tfn_tuned_shape", "tfn_tune_cache_save", "tfn_tune_cache_load",
           "tfn_server_create", "tfn_submit", "tfn_wait", "tfn_server_stats", "tfn_server_destroy"):
    getattr(_lib, _f).restype = _I

# The C entry points under their own names.
tfn_status_string = _lib.tfn_status_string
tfn_version = _lib.tfn_version
tfn_last_cuda_error = _lib.tfn_last_cuda_error
tfn_create = _lib.tfn_create
tfn_destroy = _lib.tfn_destroy
tfn_normals = _lib.tfn_normals
tfn_normals_batch = _lib.tfn_normals_batch
tfn_normals_batch_host = _lib.tfn_normals_batch_host
tfn_device_status = _lib.tfn_device_status
tfn_refined_pixels = _lib.tfn_refined_pixels
tfn_tile_shape_count = _lib.tfn_tile_shape_count
tfn_tile_shape_info = _lib.tfn_tile_shape_info
tfn_tile_shape_warps = _lib.tfn_tile_shape_warps
tfn_set_tile_shape = _lib.tfn_set_tile_shape
tfn_plan_create = _lib.tfn_plan_create
tfn_plan_launch = _lib.tfn_plan_launch
tfn_plan_destroy = _lib.tfn_plan_destroy
tfn_plan_kernels = _lib.tfn_plan_kernels
tfn_plan_kernel_name = _lib.tfn_plan_kernel_name
tfn_autotune = _lib.tfn_autotune
tfn_tuned_shape = _lib.tfn_tuned_shape
tfn_tune_cache_save = _lib.tfn_tune_cache_save
tfn_tune_cache_load = _lib.tfn_tune_cache_load
tfn_server_create = _lib.tfn_server_create
tfn_submit = _lib.tfn_submit
tfn_wait = _lib.tfn_wait
tfn_server_stats = _lib.tfn_server_stats
tfn_server_destroy = _lib.tfn_server_destroy
# For callers that may not allocate device memory (see include/tfn.h).
tfn_normals_noalloc = _lib.tfn_normals_noalloc
TFN_NOALLOC_MAX_FRAMES = 64

EXPORTED = ["tfn_status_string", "tfn_version", "tfn_last_cuda_error", "tfn_create", "tfn_destroy", "tfn_normals",
            "tfn_normals_batch", "tfn_normals_batch_host", "tfn_device_status", "tfn_refined_pixels",
            "tfn_normals_noalloc", "tfn_plan_create", "tfn_plan_launch", "tfn_plan_destroy", "tfn_plan_kernels",
            "tfn_plan_kernel_name",
            "tfn_tile_shape_count",
            "tfn_tile_shape_info", "tfn_tile_shape_warps", "tfn_set_tile_shape", "tfn_autotune", "tfn_tuned_shape", "tfn_tune_cache_save",
            "tfn_tune_cache_load", "tfn_server_create", "tfn_submit", "tfn_wait", "tfn_server_stats",
            "tfn_server_destroy"]


# Objects that own library handles, closed at interpreter exit (servers first, then plans, then contexts)
# so that no handle outlives the CUDA runtime's own teardown.
_LIVE = {"server": weakref.WeakSet(), "plan": weakref.WeakSet(), "ctx": weakref.WeakSet()}


@atexit.register
def _close_all():
    for kind in ("server", "plan", "ctx"):
        for obj in list(_LIVE[kind]):
            try:
                obj.close()
            except Exception:
                pass


class TfnError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        msg = tfn_status_string(status).decode()
        if status == TFN_ERR_CUDA:
            msg += f" ({tfn_last_cuda_error().decode()})"
        super().__init__(f"{what}: {msg}" if what else msg)
        self.status = status


def check(status: int, what: str = ""):
    if status != TFN_OK:
        raise TfnError(status, what)


# ---- tensor marshalling -----------------------------------------------------------------

def _torch():
    import torch
    return torch


def _input_type(t, disparity: bool) -> int:
    torch = _torch()
    if disparity:
        if t.dtype in (getattr(torch, "uint16", None), torch.int16):  # int16: raw u16 bits
            return TFN_DISP_U16
        if t.dtype == torch.float32:
            return TFN_DISP_F32
    else:
        if t.dtype == torch.float32:
            return TFN_DEPTH_F32
        if t.dtype == torch.float16:
            return TFN_DEPTH_F16
    raise TypeError(f"unsupported input dtype {t.dtype} (disparity={disparity})")


def padded_width(width: int, elem_bytes: int) -> int:
    """Smallest row length (elements) >= width whose byte size is a multiple of 16."""
    per = 16 // elem_bytes
    return (width + per - 1) // per * per


def empty_image(shape, dtype, device="cuda"):
    """(..., H, W) tensor whose rows start on 16-byte boundaries (a view of a padded buffer)."""
    torch = _torch()
    *lead, H, W = shape
    es = torch.empty((), dtype=dtype).element_size()
    Wp = padded_width(W, es)
    buf = torch.empty((*lead, H, Wp), dtype=dtype, device=device)
    return buf[..., :W]


def empty_normals(H, W, output="f32", device="cuda", lead=()):
    """Output buffer for one layout: planar (..., 3, H, W), packed (..., H, W, 4), or octahedral
    codes (..., H, W, 2) int16."""
    torch = _torch()
    fmt = OUTPUTS[output] if isinstance(output, str) else output
    if fmt == TFN_OUT_OCT16:
        buf = torch.empty((*lead, H, padded_width(W, 4), 2), dtype=torch.int16, device=device)
        return buf[..., :W, :]
    if fmt in (TFN_OUT_F32, TFN_OUT_F16, TFN_OUT_BF16):
        dt = {TFN_OUT_F32: torch.float32, TFN_OUT_F16: torch.float16, TFN_OUT_BF16: torch.bfloat16}[fmt]
        return empty_image((*lead, 3, H, W), dt, device)
    dt = torch.float16 if fmt == TFN_OUT_F16X4 else torch.bfloat16
    es = 8
    Wp = padded_width(W, es)
    buf = torch.empty((*lead, H, Wp, 4), dtype=dt, device=device)
    return buf[..., :W, :]


def empty_points(H, W, device="cuda", lead=()):
    """Point-cloud buffer: three float32 planes (..., 3, H, W) of X, Y, Z."""
    return empty_image((*lead, 3, H, W), _torch().float32, device)


def make_frame(inp, normals, mask, cam, disparity=False, disp_scale=1.0 / 16, output="f32",
               points=None) -> tfn_frame:
    """tfn_frame describing torch tensors `inp` (H, W), `normals`, `mask` (H, W) and optional `points`
    (3, H, W)."""
    fmt = OUTPUTS[output] if isinstance(output, str) else output
    H, W = inp.shape
    f = tfn_frame()
    f.input = inp.data_ptr()
    f.input_pitch = inp.stride(0) * inp.element_size()
    f.height, f.width = H, W
    f.input_type = _input_type(inp, disparity)
    f.disp_scale = disp_scale
    f.cam = tfn_camera(cam["fx"], cam["fy"], cam["u0"], cam["v0"], cam.get("baseline", 1.0))
    f.normals = normals.data_ptr()
    if fmt in (TFN_OUT_F32, TFN_OUT_F16, TFN_OUT_BF16):
        f.normals_pitch = normals.stride(1) * normals.element_size()
        f.normals_plane_stride = normals.stride(0) * normals.element_size()
    else:
        f.normals_pitch = normals.stride(0) * normals.element_size()
        f.normals_plane_stride = 0
    f.mask = mask.data_ptr()
    f.mask_pitch = mask.stride(0) * mask.element_size()
    if points is not None:
        f.points = points.data_ptr()
        f.points_pitch = points.stride(1) * points.element_size()
        f.points_plane_stride = points.stride(0) * points.element_size()
    return f


def _stacked(t, ndim: int) -> bool:
    return t is not None and hasattr(t, "data_ptr") and t.dim() == ndim + 1


def make_frames(inputs, normals, masks, cams, disparity=False, disp_scale=1.0 / 16, output="f32", points=None):
    """The tfn_frame array of a batch, as (keep-alive object, length, pointer to the first frame).

    Lists of per-frame tensors take one make_frame per frame.  Stacks (inputs (N, H, W), normals and
    masks with the same leading N, points too if given) are described in one pass instead: frame 0's
    descriptor is replicated into numpy records that have the C struct's layout, and the data
    pointers advance by each stack's leading stride, which saves the per-frame Python work of a
    large batch (about 4 us a frame)."""
    n = len(inputs)
    single = isinstance(cams, dict)
    # (every output layout has 3 dimensions per frame: (3, H, W), (H, W, 4) or (H, W, 2))
    if (n >= 2 and _stacked(inputs, 2) and _stacked(normals, 3) and _stacked(masks, 2)
            and (points is None or _stacked(points, 3))
            and normals.shape[0] == n and masks.shape[0] == n and (points is None or points.shape[0] == n)):
        import numpy as np
        f0 = make_frame(inputs[0], normals[0], masks[0], cams if single else cams[0], disparity, disp_scale, output,
                        points[0] if points is not None else None)
        dt = np.dtype(tfn_frame)
        arr = np.repeat(np.frombuffer(bytes(f0), dtype=dt), n)
        k = np.arange(n, dtype=np.uint64)
        for name, t in (("input", inputs), ("normals", normals), ("mask", masks), ("points", points)):
            if t is not None:
                arr[name] += k * np.uint64(t.stride(0) * t.element_size())
        if not single:
            for key in ("fx", "fy", "u0", "v0"):
                arr["cam"][key] = [c[key] for c in cams]
            arr["cam"]["baseline"] = [c.get("baseline", 1.0) for c in cams]
        return arr, n, arr.ctypes.data_as(ctypes.POINTER(tfn_frame))
    if single:
        cams = [cams] * n
    frames = (tfn_frame * n)(*[make_frame(inputs[k], normals[k], masks[k], cams[k], disparity, disp_scale, output,
                                          points[k] if points is not None else None) for k in range(n)])
    return frames, n, frames


def make_method(grad="fd", phi="mean", output="f32", flags=0, weights=None) -> tfn_method:
    """grad="weighted" takes the row weights (w0, w1, w2) of the gradient filter in `weights`; grad="sep5" takes
    the 5x5 profiles (d1, d2, s0, s1, s2); grad="planepca" selects the PlanePCA estimator (TFN_EST_PLANEPCA,
    which has no gradient filter and no Phi)."""
    m = tfn_method()
    if grad == "planepca":
        m.estimator, grad = TFN_EST_PLANEPCA, "fd"
    m.grad = GRADS[grad] if isinstance(grad, str) else grad
    m.phi = PHIS[phi] if isinstance(phi, str) else phi
    m.output = OUTPUTS[output] if isinstance(output, str) else output
    m.flags = flags
    if weights is not None:
        if len(weights) > 5:
            raise ValueError("at most 5 weights")
        m.weights = (ctypes.c_float * 5)(*weights)
    return m


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A libtfn context on one CUDA device (argument marshalling only)."""

    def __init__(self, device: int = -1, mem_budget: int = 0):
        h = ctypes.c_void_p()
        check(tfn_create(ctypes.byref(h), device, mem_budget), "tfn_create")
        self.handle = h
        _LIVE["ctx"].add(self)

    def close(self):
        if self.handle:
            tfn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def normals(self, inp, cam, *, grad="fd", phi="mean", output="f32", disparity=False, disp_scale=1.0 / 16,
                normals=None, mask=None, points=None, stream=None, flags=0, weights=None):
        """Normals of one (H, W) device image -> (normals, mask); `points` (3, H, W) also receives the
        back-projected point cloud."""
        H, W = inp.shape
        if normals is None:
            normals = empty_normals(H, W, output, inp.device)
        if mask is None:
            mask = empty_image((H, W), _torch().uint8, inp.device)
        f = make_frame(inp, normals, mask, cam, disparity, disp_scale, output, points)
        m = make_method(grad, phi, output, flags, weights)
        check(tfn_normals(self.handle, ctypes.byref(f), ctypes.byref(m), _stream_handle(stream)), "tfn_normals")
        return normals, mask

    def normals_batch(self, inputs, cams, *, grad="fd", phi="mean", output="f32", disparity=False,
                      disp_scale=1.0 / 16, normals=None, masks=None, points=None, stream=None, flags=0, weights=None):
        """Normals of a list of (H_i, W_i) device images (or an (N, H, W) stack) in one launch."""
        if normals is None:
            normals = [empty_normals(x.shape[0], x.shape[1], output, x.device) for x in inputs]
        if masks is None:
            masks = [empty_image(tuple(x.shape), _torch().uint8, x.device) for x in inputs]
        keep, n, frames = make_frames(inputs, normals, masks, cams, disparity, disp_scale, output, points)
        m = make_method(grad, phi, output, flags, weights)
        check(tfn_normals_batch(self.handle, frames, n, ctypes.byref(m), _stream_handle(stream)), "tfn_normals_batch")
        return normals, masks

    def normals_batch_host(self, inputs, cams, normals, masks, *, grad="fd", phi="mean", output="f32",
                           disparity=False, disp_scale=1.0 / 16, points=None, stream=None, flags=0, weights=None):
        """Like normals_batch, with every tensor in host memory (pinned is fastest); synchronous.  The tensors
        may be lists of per-frame tensors or stacks with a leading frame dimension (see make_frames)."""
        keep, n, frames = make_frames(inputs, normals, masks, cams, disparity, disp_scale, output, points)
        m = make_method(grad, phi, output, flags, weights)
        check(tfn_normals_batch_host(self.handle, frames, n, ctypes.byref(m), _stream_handle(stream)),
              "tfn_normals_batch_host")
        return normals, masks

    def plan(self, inputs, cams, *, grad="fd", phi="mean", output="f32", disparity=False, disp_scale=1.0 / 16,
             normals=None, masks=None, points=None, flags=0, weights=None):
        """Freezes a batch into a Plan (descriptors uploaded once, launches captured in a CUDA graph)."""
        if normals is None:
            normals = [empty_normals(x.shape[0], x.shape[1], output, x.device) for x in inputs]
        if masks is None:
            masks = [empty_image(tuple(x.shape), _torch().uint8, x.device) for x in inputs]
        keep, n, frames = make_frames(inputs, normals, masks, cams, disparity, disp_scale, output, points)
        m = make_method(grad, phi, output, flags, weights)
        h = ctypes.c_void_p()
        check(tfn_plan_create(self.handle, frames, n, ctypes.byref(m), ctypes.byref(h)), "tfn_plan_create")
        return Plan(h, inputs, normals, masks)

    def set_tile_shape(self, index: int):
        """Force tile shape `index`; -1 returns to the tune table."""
        check(tfn_set_tile_shape(self.handle, index), "tfn_set_tile_shape")

    def autotune(self, inputs, cams, *, grad="fd", phi="mean", output="f32", disparity=False, disp_scale=1.0 / 16,
                 normals=None, masks=None, reps=10, stream=None, weights=None):
        """Times every tile shape on this batch; returns (best index, [ms per run of each shape])."""
        if normals is None:
            normals = [empty_normals(x.shape[0], x.shape[1], output, x.device) for x in inputs]
        if masks is None:
            masks = [empty_image(tuple(x.shape), _torch().uint8, x.device) for x in inputs]
        keep, n, frames = make_frames(inputs, normals, masks, cams, disparity, disp_scale, output)
        m = make_method(grad, phi, output, 0, weights)
        best = ctypes.c_int()
        ms = (ctypes.c_float * tfn_tile_shape_count())()
        check(tfn_autotune(self.handle, frames, n, ctypes.byref(m), reps, _stream_handle(stream), ctypes.byref(best),
                           ms), "tfn_autotune")
        return best.value, list(ms)

    def tuned_shape(self, input_type: int, *, grad="fd", phi="mean", output="f32") -> int:
        """The tune table's shape for this combination, or -1."""
        m = make_method(grad, phi, output)
        idx = ctypes.c_int()
        check(tfn_tuned_shape(self.handle, input_type, ctypes.byref(m), ctypes.byref(idx)), "tfn_tuned_shape")
        return idx.value

    def save_tune_cache(self, path: str):
        check(tfn_tune_cache_save(self.handle, os.fsencode(path)), "tfn_tune_cache_save")

    def load_tune_cache(self, path: str):
        check(tfn_tune_cache_load(self.handle, os.fsencode(path)), "tfn_tune_cache_load")

    def refined_pixels(self, stream=None) -> int:
        """Pixels sent to the double-float path since the last call (diagnostics)."""
        n = ctypes.c_uint64()
        check(tfn_refined_pixels(self.handle, ctypes.byref(n), _stream_handle(stream)), "tfn_refined_pixels")
        return n.value

    def device_status(self, stream=None) -> int:
        bits = ctypes.c_uint32()
        check(tfn_device_status(self.handle, ctypes.byref(bits), _stream_handle(stream)), "tfn_device_status")
        return bits.value


def tile_shapes():
    """[(tile_w, tile_h, rows_per_thread)] for every compiled tile shape."""
    out = []
    for i in range(tfn_tile_shape_count()):
        w, h, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(tfn_tile_shape_info(i, ctypes.byref(w), ctypes.byref(h), ctypes.byref(r)), "tfn_tile_shape_info")
        out.append((w.value, h.value, r.value))
    return out


def tile_shape_warps():
    """[(warps per CTA for the 3x3 filters, for the 5x5 filters and PlanePCA)] for every compiled tile shape."""
    out = []
    for i in range(tfn_tile_shape_count()):
        a, b = ctypes.c_int(), ctypes.c_int()
        check(tfn_tile_shape_warps(i, ctypes.byref(a), ctypes.byref(b)), "tfn_tile_shape_warps")
        out.append((a.value, b.value))
    return out


class Plan:
    """A frozen batch; launch() replays its CUDA graph on a stream."""

    def __init__(self, handle, inputs, normals, masks):
        self.handle = handle
        _LIVE["plan"].add(self)
        self.inputs, self.normals, self.masks = inputs, normals, masks  # keep the buffers alive

    def launch(self, stream=None):
        check(tfn_plan_launch(self.handle, _stream_handle(stream)), "tfn_plan_launch")
        return self.normals, self.masks

    def kernels(self) -> int:
        """Kernel launches one replay runs."""
        n = _I()
        check(tfn_plan_kernels(self.handle, ctypes.byref(n)), "tfn_plan_kernels")
        return n.value

    def kernel_names(self) -> list:
        """The (mangled) names of the kernels one replay runs."""
        out = []
        for i in range(self.kernels()):
            nm = ctypes.c_char_p()
            check(tfn_plan_kernel_name(self.handle, i, ctypes.byref(nm)), "tfn_plan_kernel_name")
            out.append(nm.value.decode())
        return out

    def close(self):
        if self.handle:
            tfn_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A libtfn request server (continuous batching); see tfn_server_create in include/tfn.h.

    submit() takes torch tensors on the device, or in host memory with host=True; the tensors are kept
    alive until wait() returns for their ticket."""

    def __init__(self, ctx: Context, *, grad="fd", phi="mean", output="f32", flags=0, mem_budget=0,
                 max_batch=0, max_queue=0, max_delay_us=0, pipelines=0, weights=None, graphs=True):
        o = tfn_server_opts()
        o.method = make_method(grad, phi, output, flags, weights)
        o.mem_budget_bytes = mem_budget
        o.max_batch_frames, o.max_queue, o.max_delay_us, o.pipelines = max_batch, max_queue, max_delay_us, pipelines
        o.flags = 0 if graphs else TFN_SERVER_NO_GRAPHS
        h = ctypes.c_void_p()
        check(tfn_server_create(ctx.handle, ctypes.byref(o), ctypes.byref(h)), "tfn_server_create")
        self.handle = h
        _LIVE["server"].add(self)
        self.output = output
        self._keep = {}

    def submit(self, inp, cam, normals, mask, *, host=False, disparity=False, disp_scale=1.0 / 16,
               points=None, flags=0) -> int:
        """Queues one frame; returns its ticket (raises TfnError, e.g. TFN_ERR_BUSY).  `flags` adds
        TFN_REQ_* flags to the one `host` sets."""
        f = make_frame(inp, normals, mask, cam, disparity, disp_scale, self.output, points)
        t = ctypes.c_uint64()
        fl = (TFN_REQ_HOST if host else 0) | flags
        check(tfn_submit(self.handle, ctypes.byref(f), fl, ctypes.byref(t)), "tfn_submit")
        self._keep[t.value] = (inp, normals, mask, points)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 10000) -> int:
        """The request's status once done; raises TfnError(TFN_ERR_TIMEOUT) if not done in time."""
        r = ctypes.c_int()
        check(tfn_wait(self.handle, ticket, timeout_ms, ctypes.byref(r)), "tfn_wait")
        self._keep.pop(ticket, None)
        return r.value

    def stats(self, reset=False) -> dict:
        st = tfn_serving_stats()
        check(tfn_server_stats(self.handle, ctypes.byref(st), 1 if reset else 0), "tfn_server_stats")
        return {k: getattr(st, k) for k, _ in tfn_serving_stats._fields_}

    def close(self):
        if self.handle:
            tfn_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
