"""ctypes binding of libnam (include/nam.h): the same entry points, argument
marshalling only.  Every computation runs in libnam's CUDA kernels; there is
no Python or CPU fallback.  Importing this module fails loudly if the shared
library has not been built (``__graft_entry__.build()``).

Device arrays are passed as torch CUDA tensors (or raw integer pointers);
host arrays as numpy arrays (or torch CPU tensors).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import LIB as _LIB_PATH

NAM_OK = 0
NAM_ERR_INVALID_ARG, NAM_ERR_OOM, NAM_ERR_BUDGET, NAM_ERR_NOT_FOUND = -1, -2, -3, -4
NAM_ERR_BUSY, NAM_ERR_TIMEOUT, NAM_ERR_CUDA, NAM_ERR_DEVICE_ASSERT = -5, -6, -7, -8
NAM_ERR_UNSUPPORTED, NAM_ERR_CANCELLED = -9, -10
NAM_LATENT_F32, NAM_LATENT_F16 = 0, 1
NAM_PREC_F32, NAM_PREC_F16, NAM_PREC_FP8 = 0, 1, 2
NAM_FILTER_TRILINEAR, NAM_FILTER_STOCHASTIC = 0, 1
NAM_ADDRESS_WRAP, NAM_ADDRESS_CLAMP = 0, 1
NAM_HOST_STAGED = 1 << 8
NAM_FRAME_DEVICE = 1 << 9
NAM_OUT_COSINE = 1
NAM_FAULT_NONE, NAM_FAULT_ALLOC, NAM_FAULT_LAUNCH, NAM_FAULT_STALL = 0, 1, 2, 3
NAM_MAX_LEVELS, NAM_MAX_LAYERS = 16, 8
NAM_FRAME_MLP, NAM_FRAME_PAPER = 0, 1
NAM_ENCODER_HIDDEN, NAM_ENCODER_MAX_INPUTS = 32, 16

QUERY_FIELDS = ("u", "v", "lod", "wix", "wiy", "wiz", "wox", "woy", "woz", "xi")


class nam_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("serve_streams", C.c_int32), ("serve_queue_depth", C.c_int32),
                ("reserved0", C.c_int32), ("hbm_budget_bytes", C.c_uint64), ("wait_timeout_ns", C.c_uint64)]


class nam_material_desc(C.Structure):
    _fields_ = [("base_w", C.c_int32), ("base_h", C.c_int32), ("levels", C.c_int32), ("channels", C.c_int32),
                ("latent_dtype", C.c_int32), ("params_on_device", C.c_int32), ("pyramid", C.c_void_p),
                ("frame_hidden", C.c_int32), ("n_layers", C.c_int32), ("frame_weights", C.c_void_p),
                ("widths", C.c_int32 * (NAM_MAX_LAYERS + 1)), ("decoder_weights", C.c_void_p),
                ("precision", C.c_int32), ("filter", C.c_int32), ("address", C.c_int32), ("trainable", C.c_int32),
                ("fp8_act_scale", C.c_void_p), ("sampler_hidden", C.c_int32), ("sampler_weights", C.c_void_p),
                ("frame_form", C.c_int32), ("encoder_inputs", C.c_int32), ("encoder_weights", C.c_void_p)]


class nam_material_info(C.Structure):
    _fields_ = [("resident_bytes", C.c_uint64), ("texels", C.c_int64), ("n_params", C.c_int64),
                ("precision", C.c_int32), ("filter", C.c_int32), ("address", C.c_int32), ("levels", C.c_int32),
                ("fp8_weight_scale", C.c_float * NAM_MAX_LAYERS)]


class nam_queries(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in QUERY_FIELDS]


class nam_work_item(C.Structure):
    _fields_ = [("start", C.c_int64), ("count", C.c_int32), ("material", C.c_int32)]


class nam_adam(C.Structure):
    _fields_ = [("lr_params", C.c_float), ("lr_pyramid", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("step", C.c_int32)]


class nam_sphere(C.Structure):
    _fields_ = [("center", C.c_float * 3), ("radius", C.c_float), ("material", C.c_int32)]


class nam_scene(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("eye", C.c_float * 3), ("target", C.c_float * 3),
                ("up", C.c_float * 3), ("fov_y", C.c_float), ("ground_y", C.c_float), ("ground_material", C.c_int32),
                ("ground_uv_scale", C.c_float), ("spheres", C.c_void_p), ("n_spheres", C.c_int32),
                ("sky_radiance", C.c_float)]


class nam_gbuffer(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("material", "t", "u", "v", "lod", "frame", "view")]


NAM_SCENE_MAX_SPHERES = 64


def make_scene(width, height, eye, target, up, fov_y, spheres, ground_y=0.0, ground_material=-1,
               ground_uv_scale=1.0, sky_radiance=1.0):
    """nam_scene (and the sphere array it points to, kept on the object);
    spheres: list of (cx, cy, cz, radius, material)."""
    arr = (nam_sphere * max(1, len(spheres)))()
    for k, (cx, cy, cz, r, m) in enumerate(spheres):
        arr[k] = nam_sphere((C.c_float * 3)(cx, cy, cz), r, m)
    sc = nam_scene(width=width, height=height, eye=(C.c_float * 3)(*eye), target=(C.c_float * 3)(*target),
                   up=(C.c_float * 3)(*up), fov_y=fov_y, ground_y=ground_y, ground_material=ground_material,
                   ground_uv_scale=ground_uv_scale, spheres=C.addressof(arr), n_spheres=len(spheres),
                   sky_radiance=sky_radiance)
    sc._spheres = arr
    return sc


class nam_frame(C.Structure):
    _fields_ = [("n_queries", C.c_int64), ("q", nam_queries), ("items", C.c_void_p), ("n_items", C.c_int32),
                ("n_materials", C.c_int32), ("materials", C.c_void_p), ("rgb_out", C.c_void_p),
                ("flags", C.c_uint32), ("reserved0", C.c_int32), ("arrival_s", C.c_double)]


class nam_frame_stats(C.Structure):
    _fields_ = [("arrival_s", C.c_double), ("admit_s", C.c_double), ("start_s", C.c_double),
                ("finish_s", C.c_double), ("n_queries", C.c_int64), ("status", C.c_int32), ("slot", C.c_int32),
                ("submit_s", C.c_double), ("enqueued_s", C.c_double), ("gpu_begin_s", C.c_double),
                ("gpu_kernel_begin_s", C.c_double), ("gpu_kernel_end_s", C.c_double), ("gpu_end_s", C.c_double),
                ("in_flight_at_admit", C.c_int32), ("reserved1", C.c_int32)]


class nam_stats(C.Structure):
    _fields_ = [("resident_bytes", C.c_uint64), ("budget_bytes", C.c_uint64), ("queued", C.c_int64),
                ("in_flight", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("queries_completed", C.c_int64), ("p50_latency_ms", C.c_double),
                ("p99_latency_ms", C.c_double), ("evals_per_s", C.c_double)]


#: every symbol include/nam.h declares
EXPORTS = ("nam_status_string", "nam_last_error_message", "nam_init", "nam_shutdown", "nam_check_device_error",
           "nam_create_material", "nam_destroy_material", "nam_material_get_info", "nam_material_params",
           "nam_eval", "nam_eval_host", "nam_eval_multi", "nam_eval_binned", "nam_eval_select", "nam_fp8_calibrate", "nam_sample", "nam_sample_pdf", "nam_backward", "nam_train_step", "nam_eval_albedo", "nam_train_step_albedo",
           "nam_train_step_noalloc", "nam_encode", "nam_encoder_bake", "nam_backward_encoded",
           "nam_train_step_encoded", "nam_material_encoder", "nam_scene_gbuffer", "nam_scene_render_direct",
           "nam_scene_render_paths",
           "nam_now",
           "nam_submit", "nam_poll", "nam_wait", "nam_cancel", "nam_get_stats", "nam_inject_fault")


class NamError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} [status {status}]")
        self.status = status


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libnam.so is not built ({_LIB_PATH}); run __graft_entry__.build() first")
    lib = C.CDLL(_LIB_PATH)
    p, i32, i64, u32, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
    sig = {
        "nam_status_string": (C.c_char_p, [i32]),
        "nam_last_error_message": (C.c_char_p, []),
        "nam_init": (i32, [p, p]),
        "nam_shutdown": (i32, [p]),
        "nam_check_device_error": (i32, [p]),
        "nam_create_material": (i32, [p, p, p]),
        "nam_destroy_material": (i32, [p, p]),
        "nam_material_get_info": (i32, [p, p, p]),
        "nam_material_params": (i32, [p, p, p, p]),
        "nam_eval": (i32, [p, p, p, i64, p, p, u32]),
        "nam_eval_host": (i32, [p, p, p, i64, p, p, u32]),
        "nam_eval_multi": (i32, [p, p, i32, p, p, i32, p, p, u32]),
        "nam_eval_binned": (i32, [p, p, i32, p, p, i64, p, p, u32]),
        "nam_eval_select": (i32, [p, p, i32, p, p, i64, p, p, u32]),
        "nam_backward": (i32, [p, p, p, i64, p, p, p, p, u32]),
        "nam_train_step": (i32, [p, p, p, p, i64, p, p, p, u32]),
        "nam_eval_albedo": (i32, [p, p, p, i64, p, p, p, u32]),
        "nam_train_step_albedo": (i32, [p, p, p, p, p, i64, p, p, p, u32]),
        "nam_train_step_noalloc": (i32, [p, p, p, p, i64, p, p, p, u32]),
        "nam_encode": (i32, [p, p, p, i64, p, p]),
        "nam_encoder_bake": (i32, [p, p, p, p]),
        "nam_backward_encoded": (i32, [p, p, p, p, i64, p, p, p, p, u32]),
        "nam_train_step_encoded": (i32, [p, p, p, p, p, i64, p, p, p, u32]),
        "nam_material_encoder": (i32, [p, p, p]),
        "nam_scene_gbuffer": (i32, [p, p, i32, p, p]),
        "nam_scene_render_direct": (i32, [p, p, p, i32, p, p, p]),
        "nam_scene_render_paths": (i32, [p, p, p, i32, i32, p, p, p]),
        "nam_fp8_calibrate": (i32, [p, p, p, i64, p, p]),
        "nam_sample": (i32, [p, p, p, i64, p, p, p, p]),
        "nam_sample_pdf": (i32, [p, p, p, i64, p, p]),
        "nam_now": (C.c_double, []),
        "nam_submit": (i32, [p, p, p]),
        "nam_poll": (i32, [p, u64, p, p]),
        "nam_wait": (i32, [p, u64, u64, p]),
        "nam_cancel": (i32, [p, u64]),
        "nam_get_stats": (i32, [p, p]),
        "nam_inject_fault": (i32, [p, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


def _check(status, what):
    if status != NAM_OK:
        msg = _lib.nam_last_error_message().decode()
        raise NamError(status, f"{what}: {msg or _lib.nam_status_string(status).decode()}")


def ptr(x):
    """Address of a torch tensor, numpy array, ctypes object or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return C.addressof(x)


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def make_queries(q) -> nam_queries:
    """nam_queries from a dict of arrays/tensors keyed by QUERY_FIELDS."""
    s = nam_queries()
    for k in QUERY_FIELDS:
        setattr(s, k, ptr(q.get(k)))
    return s


# ----------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ----------------------------------------------------------------------------
def nam_status_string(s):
    return _lib.nam_status_string(s).decode()


def nam_last_error_message():
    return _lib.nam_last_error_message().decode()


def nam_init(device=0, hbm_budget_bytes=0, wait_timeout_ns=0, serve_streams=0, serve_queue_depth=0):
    cfg = nam_config(device=device, serve_streams=serve_streams, serve_queue_depth=serve_queue_depth,
                     hbm_budget_bytes=hbm_budget_bytes, wait_timeout_ns=wait_timeout_ns)
    h = C.c_void_p()
    _check(_lib.nam_init(C.byref(h), C.byref(cfg)), "nam_init")
    return h.value


def nam_shutdown(ctx):
    _check(_lib.nam_shutdown(ctx), "nam_shutdown")


def nam_check_device_error(ctx):
    _check(_lib.nam_check_device_error(ctx), "nam_check_device_error")


def nam_create_material(ctx, desc: nam_material_desc):
    h = C.c_void_p()
    _check(_lib.nam_create_material(ctx, C.byref(desc), C.byref(h)), "nam_create_material")
    return h.value


def nam_destroy_material(ctx, mat):
    _check(_lib.nam_destroy_material(ctx, mat), "nam_destroy_material")


def nam_material_get_info(ctx, mat) -> nam_material_info:
    info = nam_material_info()
    _check(_lib.nam_material_get_info(ctx, mat, C.byref(info)), "nam_material_get_info")
    return info


def nam_material_params(ctx, mat):
    pp, py = C.c_void_p(), C.c_void_p()
    _check(_lib.nam_material_params(ctx, mat, C.byref(pp), C.byref(py)), "nam_material_params")
    return pp.value, py.value


def nam_eval(ctx, mat, q, n, rgb_out, stream=None, flags=0):
    qs = make_queries(q)
    _check(_lib.nam_eval(ctx, mat, C.byref(qs), int(n), ptr(rgb_out), _stream(stream), flags), "nam_eval")


def nam_eval_albedo(ctx, mat, q, n, rgb_out, albedo_out, stream=None, flags=0):
    """RGB and the albedo head's directional albedo, both device [n][3]."""
    qs = make_queries(q)
    _check(_lib.nam_eval_albedo(ctx, mat, C.byref(qs), int(n), ptr(rgb_out), ptr(albedo_out), _stream(stream),
                                flags), "nam_eval_albedo")


def nam_fp8_calibrate(ctx, mat, q, n, stream=None):
    """Static per-layer FP8 activation scales (max |layer input| / 448) of
    material `mat` over n device queries; returns a float32 numpy array."""
    qs = make_queries(q)
    out = np.zeros(NAM_MAX_LAYERS, dtype=np.float32)
    _check(_lib.nam_fp8_calibrate(ctx, mat, C.byref(qs), int(n), out.ctypes.data, _stream(stream)),
           "nam_fp8_calibrate")
    return out


def nam_sample(ctx, mat, q, n, u, wo_out, pdf_out=None, stream=None):
    """Importance-sample one outgoing direction per query (device arrays)."""
    qs = make_queries(q)
    _check(_lib.nam_sample(ctx, mat, C.byref(qs), int(n), ptr(u), ptr(wo_out), ptr(pdf_out), _stream(stream)),
           "nam_sample")


def nam_sample_pdf(ctx, mat, q, n, pdf_out, stream=None):
    """Proxy density of each query's wo given its wi (device arrays)."""
    qs = make_queries(q)
    _check(_lib.nam_sample_pdf(ctx, mat, C.byref(qs), int(n), ptr(pdf_out), _stream(stream)), "nam_sample_pdf")


def nam_eval_host(ctx, mat, q, n, rgb_out, stream=None, flags=0):
    qs = make_queries(q)
    _check(_lib.nam_eval_host(ctx, mat, C.byref(qs), int(n), ptr(rgb_out), _stream(stream), flags),
           "nam_eval_host")


def nam_eval_multi(ctx, mats, q, items, rgb_out, stream=None, flags=0):
    """mats: list of material handles; items: list of (start, count, material)."""
    arr = (C.c_void_p * len(mats))(*mats)
    it = (nam_work_item * len(items))(*[nam_work_item(int(s), int(c), int(m)) for s, c, m in items])
    qs = make_queries(q)
    _check(_lib.nam_eval_multi(ctx, arr, len(mats), C.byref(qs), it, len(items), ptr(rgb_out), _stream(stream),
                               flags), "nam_eval_multi")


NAM_MAX_BIN_MATERIALS = 4096
NAM_SELECT_MAX_PASSES = 1


def nam_eval_binned(ctx, mats, q, material_ids, n, rgb_out, stream=None, flags=0):
    """mats: list of material handles; material_ids: device int32 [n]."""
    arr = (C.c_void_p * len(mats))(*mats)
    qs = make_queries(q)
    _check(_lib.nam_eval_binned(ctx, arr, len(mats), C.byref(qs), ptr(material_ids), int(n), ptr(rgb_out),
                                _stream(stream), flags), "nam_eval_binned")


def nam_eval_select(ctx, mats, q, material_ids, n, rgb_out, stream=None, flags=0):
    """Per-tile code-path selection (masked passes or binning); arguments as nam_eval_binned."""
    arr = (C.c_void_p * len(mats))(*mats)
    qs = make_queries(q)
    _check(_lib.nam_eval_select(ctx, arr, len(mats), C.byref(qs), ptr(material_ids), int(n), ptr(rgb_out),
                                _stream(stream), flags), "nam_eval_select")


def nam_backward(ctx, mat, q, n, grad_rgb, grad_params, grad_pyramid, stream=None, flags=0):
    qs = make_queries(q)
    _check(_lib.nam_backward(ctx, mat, C.byref(qs), int(n), ptr(grad_rgb), ptr(grad_params), ptr(grad_pyramid),
                             _stream(stream), flags), "nam_backward")


def nam_train_step(ctx, mat, q, target_rgb, n, lr_params=1e-3, lr_pyramid=1e-2, beta1=0.9, beta2=0.999, eps=1e-8,
                   step=1, stream=None, flags=0, want_loss=True):
    """One fused training step; returns the batch loss (which synchronises
    the stream), or None without synchronising if want_loss is False."""
    opt = nam_adam(lr_params, lr_pyramid, beta1, beta2, eps, step)
    loss = C.c_float(0.0)
    qs = make_queries(q)
    _check(_lib.nam_train_step(ctx, mat, C.byref(qs), ptr(target_rgb), int(n), C.byref(opt),
                               C.byref(loss) if want_loss else None, _stream(stream), flags), "nam_train_step")
    return loss.value if want_loss else None


def nam_train_step_albedo(ctx, mat, q, target_rgb, target_albedo, n, lr_params=1e-3, lr_pyramid=1e-2, beta1=0.9,
                          beta2=0.999, eps=1e-8, step=1, stream=None, flags=0, want_loss=True):
    """nam_train_step with the albedo head's L2 term; returns the summed loss."""
    opt = nam_adam(lr_params, lr_pyramid, beta1, beta2, eps, step)
    loss = C.c_float(0.0)
    qs = make_queries(q)
    _check(_lib.nam_train_step_albedo(ctx, mat, C.byref(qs), ptr(target_rgb), ptr(target_albedo), int(n),
                                      C.byref(opt), C.byref(loss) if want_loss else None, _stream(stream), flags),
           "nam_train_step_albedo")
    return loss.value if want_loss else None


NAM_NOALLOC_TRAIN_MAX_QUERIES = 65536


def nam_train_step_noalloc(ctx, mat, q, target_rgb, n, lr_params=1e-3, lr_pyramid=1e-2, beta1=0.9, beta2=0.999,
                           eps=1e-8, step=1, stream=None, flags=0):
    """nam_train_step with its per-batch buffers in the library's static
    device array (no device allocation; n <= NAM_NOALLOC_TRAIN_MAX_QUERIES)."""
    opt = nam_adam(lr_params, lr_pyramid, beta1, beta2, eps, step)
    loss = C.c_float(0.0)
    qs = make_queries(q)
    _check(_lib.nam_train_step_noalloc(ctx, mat, C.byref(qs), ptr(target_rgb), int(n), C.byref(opt), C.byref(loss),
                                       _stream(stream), flags), "nam_train_step_noalloc")
    return loss.value


def encoder_param_count(k_inputs):
    """Parameters of the K -> 32 -> 32 -> 8 encoder (Sec. 5.1)."""
    return 32 * k_inputs + 32 + 32 * 32 + 32 + 8 * 32 + 8


def nam_encode(ctx, mat, attrs, n, z_out, stream=None):
    _check(_lib.nam_encode(ctx, mat, ptr(attrs), int(n), ptr(z_out), _stream(stream)), "nam_encode")


def nam_encoder_bake(ctx, mat, texel_attrs, stream=None):
    _check(_lib.nam_encoder_bake(ctx, mat, ptr(texel_attrs), _stream(stream)), "nam_encoder_bake")


def nam_backward_encoded(ctx, mat, q, attrs, n, grad_rgb, grad_params, grad_encoder, stream=None, flags=0):
    qs = make_queries(q)
    _check(_lib.nam_backward_encoded(ctx, mat, C.byref(qs), ptr(attrs), int(n), ptr(grad_rgb), ptr(grad_params),
                                     ptr(grad_encoder), _stream(stream), flags), "nam_backward_encoded")


def nam_train_step_encoded(ctx, mat, q, attrs, target_rgb, n, lr_params=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                           step=1, stream=None, flags=0, want_loss=True):
    """One step of the encoder phase; returns the batch loss (synchronising
    the stream) or None if want_loss is False."""
    opt = nam_adam(lr_params, 0.0, beta1, beta2, eps, step)
    loss = C.c_float(0.0)
    qs = make_queries(q)
    _check(_lib.nam_train_step_encoded(ctx, mat, C.byref(qs), ptr(attrs), ptr(target_rgb), int(n), C.byref(opt),
                                       C.byref(loss) if want_loss else None, _stream(stream), flags),
           "nam_train_step_encoded")
    return loss.value if want_loss else None


def nam_material_encoder(ctx, mat):
    pe = C.c_void_p()
    _check(_lib.nam_material_encoder(ctx, mat, C.byref(pe)), "nam_material_encoder")
    return pe.value


def nam_scene_gbuffer(ctx, scene, lod_base_width, out, stream=None):
    """out: dict of device tensors material (int32), t, u, v, lod [pixels], frame [pixels][9], view [pixels][3]."""
    g = nam_gbuffer(**{k: ptr(out[k]) for k in ("material", "t", "u", "v", "lod", "frame", "view")})
    _check(_lib.nam_scene_gbuffer(ctx, C.byref(scene), int(lod_base_width), C.byref(g), _stream(stream)),
           "nam_scene_gbuffer")


def nam_scene_render_direct(ctx, scene, mats, variates, image, stream=None):
    arr = (C.c_void_p * len(mats))(*mats)
    _check(_lib.nam_scene_render_direct(ctx, C.byref(scene), arr, len(mats), ptr(variates), ptr(image),
                                        _stream(stream)), "nam_scene_render_direct")


NAM_SCENE_MAX_BOUNCES = 16


def nam_scene_render_paths(ctx, scene, mats, bounces, variates, image, stream=None):
    """variates: device [bounces][pixels][5]."""
    arr = (C.c_void_p * len(mats))(*mats)
    _check(_lib.nam_scene_render_paths(ctx, C.byref(scene), arr, len(mats), int(bounces), ptr(variates), ptr(image),
                                       _stream(stream)), "nam_scene_render_paths")


def nam_now():
    return _lib.nam_now()


def nam_submit(ctx, frame: nam_frame):
    t = C.c_uint64()
    _check(_lib.nam_submit(ctx, C.byref(frame), C.byref(t)), "nam_submit")
    return t.value


def nam_poll(ctx, ticket):
    done = C.c_int32()
    st = nam_frame_stats()
    _check(_lib.nam_poll(ctx, ticket, C.byref(done), C.byref(st)), "nam_poll")
    return bool(done.value), st


def nam_wait(ctx, ticket, timeout_ns=0):
    st = nam_frame_stats()
    status = _lib.nam_wait(ctx, ticket, timeout_ns, C.byref(st))
    return status, st


def nam_cancel(ctx, ticket):
    return _lib.nam_cancel(ctx, ticket)


def nam_get_stats(ctx) -> nam_stats:
    st = nam_stats()
    _check(_lib.nam_get_stats(ctx, C.byref(st)), "nam_get_stats")
    return st


def nam_inject_fault(ctx, fault):
    _check(_lib.nam_inject_fault(ctx, fault), "nam_inject_fault")

