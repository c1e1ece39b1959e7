"""Thin ctypes binding of the C ABI in include/mppi.h (argument marshalling only).

Array arguments may be numpy arrays (host pointers, must be C-contiguous
float32 / uint32 / uint16), torch tensors (their data_ptr(), host or device),
raw integer addresses, or None for a NULL pointer.  Every call that returns
a negative status raises MppiError with the library's message.
"""
import ctypes
import os

from numpy import ndarray as _np_ndarray

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmppi_gb300.so")

MPPI_OK = 0
MPPI_E_INVALID = -1
MPPI_E_OOM = -2
MPPI_E_CUDA = -3
MPPI_E_TIMEOUT = -4
MPPI_E_NOT_READY = -5
MPPI_E_UNSUPPORTED = -6
MPPI_E_ADMISSION = -7
MPPI_PENDING = 1

MPPI_SDF_ANALYTIC = 0
MPPI_SDF_MLP_FP32 = 1
MPPI_SDF_MLP_BF16 = 2
MPPI_SDF_MLP_FP16 = 3
MPPI_SDF_MLP_FP8 = 4

MPPI_COST_CONFIGURED = 0
MPPI_COST_PAPER = 1
MPPI_DYN_CTBR = 0
MPPI_DYN_ROTOR = 1
MPPI_STATE_MAX = 17
MPPI_MAX_PE_LEVELS = 6

MPPI_BUF_NOISE = 0
MPPI_BUF_POSITIONS = 1
MPPI_BUF_COST_PARTS = 2
MPPI_BUF_SDF = 3
MPPI_BUF_WEIGHTS = 4
MPPI_BUF_COSTS = 5
MPPI_DIAG_STORE_SDF = 1
MPPI_DIAG_SDF_SINGLE_CTA = 2
MPPI_LATENT_DIM = 64
MPPI_HIDDEN = 128
MPPI_TRAIN_GEMM_FP32 = 0
MPPI_TRAIN_GEMM_BF16 = 1

LATENT_DIM = 64
HIDDEN = 128

# every symbol include/mppi.h declares
EXPORTS = [
    "mppi_config_default", "mppi_state_dim", "mppi_create", "mppi_destroy", "mppi_last_error", "mppi_set_gates",
    "mppi_set_sdf_weights", "mppi_step", "mppi_step_async", "mppi_sync", "mppi_get_nominal",
    "mppi_get_state", "mppi_set_step_counter", "mppi_get_step_counter", "mppi_read_buffer",
    "mppi_read_noise_words", "mppi_debug_inject_timeout", "mppi_set_diagnostics", "mppi_set_timing", "mppi_get_kernel_times", "mppi_kernels_per_step",
    "mppi_selftest_tc_gemm", "mppi_softmax_update_noalloc",
    "mppi_server_config_default", "mppi_server_create", "mppi_server_destroy", "mppi_server_last_error",
    "mppi_server_set_sdf_weights", "mppi_server_submit", "mppi_server_poll", "mppi_server_next_result",
    "mppi_server_get_stats",
    "mppi_train_config_default", "mppi_train_create", "mppi_train_destroy", "mppi_train_last_error",
    "mppi_train_step", "mppi_train_set_lr", "mppi_train_set_gemm_precision", "mppi_train_loss_grads", "mppi_train_get_weights", "mppi_train_evaluate",
    "mppi_train_read_points", "mppi_train_num_params",
    "mppi_depth_camera_default", "mppi_render_depth", "mppi_sample_sdf_queries",
    "mppi_encoder_create", "mppi_encoder_destroy", "mppi_encoder_last_error", "mppi_encode_depth",
    "mppi_encoder_get_weights", "mppi_encoder_set_conv_path", "mppi_encoder_check",
    "mppi_encoder_debug_inject_timeout", "mppi_encoder_train_create", "mppi_encoder_train_destroy",
    "mppi_encoder_train_last_error", "mppi_encoder_train_loss_grads", "mppi_encoder_train_step",
    "mppi_encoder_train_get_decoder", "mppi_encoder_train_set_sdf", "mppi_encoder_train_loss_grads_sdf",
    "mppi_encoder_train_step_sdf", "mppi_encoder_train_get_sdf_decoder",
]


class MppiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mppi error {code}: {msg}")
        self.code = code


class MppiConfig(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32), ("H", ctypes.c_int32), ("max_gates", ctypes.c_int32), ("sdf_mode", ctypes.c_int32),
        ("dt", ctypes.c_float), ("mass", ctypes.c_float), ("gravity", ctypes.c_float),
        ("thrust_min", ctypes.c_float), ("thrust_max", ctypes.c_float), ("rate_max", ctypes.c_float),
        ("sigma_thrust", ctypes.c_float), ("sigma_rate", ctypes.c_float), ("lam", ctypes.c_float),
        ("w_col", ctypes.c_float), ("d_safe", ctypes.c_float), ("w_u", ctypes.c_float),
        ("gate_inner_half", ctypes.c_float), ("gate_outer_half", ctypes.c_float), ("gate_half_depth", ctypes.c_float),
        ("softplus_beta", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("drone_id", ctypes.c_uint32), ("cost_mode", ctypes.c_int32),
        ("q_gate", ctypes.c_float), ("q_vis", ctypes.c_float), ("q_sdf", ctypes.c_float),
        ("guide_tan_alpha", ctypes.c_float),
        ("dynamics_mode", ctypes.c_int32), ("tdot_max", ctypes.c_float), ("rotor_thrust_max", ctypes.c_float),
        ("sigma_tdot", ctypes.c_float), ("arm_length", ctypes.c_float), ("torque_coeff", ctypes.c_float),
        ("inertia_x", ctypes.c_float), ("inertia_y", ctypes.c_float), ("inertia_z", ctypes.c_float),
        ("pe_levels", ctypes.c_int32),
    ]


class MppiServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32), ("sdf_mode", ctypes.c_int32),
                ("batching", ctypes.c_int32), ("sdf_single_cta", ctypes.c_int32)]


class MppiServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("inflight", ctypes.c_uint64), ("evictions", ctypes.c_uint64), ("restores", ctypes.c_uint64),
                ("device_bytes", ctypes.c_size_t), ("peak_device_bytes", ctypes.c_size_t), ("batches", ctypes.c_uint64)]


class MppiTrainConfig(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("n_points", ctypes.c_int32), ("n_holdout", ctypes.c_int32),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("eikonal_weight", ctypes.c_float), ("softplus_beta", ctypes.c_float),
                ("near_surface_fraction", ctypes.c_float), ("near_surface_sigma", ctypes.c_float),
                ("cube_half", ctypes.c_float), ("gate_inner_half", ctypes.c_float),
                ("gate_outer_half", ctypes.c_float), ("gate_half_depth", ctypes.c_float), ("seed", ctypes.c_uint64)]


class MppiDepthCamera(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
        ("max_range", ctypes.c_float),
        ("gate_inner_half", ctypes.c_float), ("gate_outer_half", ctypes.c_float), ("gate_half_depth", ctypes.c_float),
        ("noise_depth_coeff", ctypes.c_float), ("dropout", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("frame", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
    ]


_vp = ctypes.c_void_p
_SIGS = {
    "mppi_config_default": (None, [ctypes.POINTER(MppiConfig)]),
    "mppi_state_dim": (ctypes.c_int, [ctypes.POINTER(MppiConfig)]),
    "mppi_create": (ctypes.c_int, [ctypes.POINTER(MppiConfig), _vp, ctypes.POINTER(_vp)]),
    "mppi_destroy": (None, [_vp]),
    "mppi_last_error": (ctypes.c_char_p, [_vp]),
    "mppi_set_gates": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "mppi_set_sdf_weights": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "mppi_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mppi_step_async": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mppi_sync": (ctypes.c_int, [_vp]),
    "mppi_get_nominal": (ctypes.c_int, [_vp, _vp]),
    "mppi_get_state": (ctypes.c_int, [_vp, _vp]),
    "mppi_set_step_counter": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "mppi_get_step_counter": (ctypes.c_uint64, [_vp]),
    "mppi_read_buffer": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t]),
    "mppi_read_noise_words": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "mppi_debug_inject_timeout": (ctypes.c_int, [_vp]),
    "mppi_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "mppi_set_diagnostics": (ctypes.c_int, [_vp, ctypes.c_int]),
    "mppi_get_kernel_times": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float),
                                             ctypes.c_int]),
    "mppi_kernels_per_step": (ctypes.c_int, [_vp]),
    "mppi_selftest_tc_gemm": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mppi_softmax_update_noalloc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                                   ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp]),
    "mppi_server_config_default": (None, [ctypes.POINTER(MppiServerConfig)]),
    "mppi_server_create": (ctypes.c_int, [ctypes.POINTER(MppiServerConfig), ctypes.POINTER(_vp)]),
    "mppi_server_destroy": (None, [_vp]),
    "mppi_server_last_error": (ctypes.c_char_p, [_vp]),
    "mppi_server_set_sdf_weights": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "mppi_server_submit": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(MppiConfig), _vp, ctypes.c_int, _vp, _vp,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "mppi_server_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, ctypes.POINTER(ctypes.c_double)]),
    "mppi_server_next_result": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64), _vp, ctypes.c_size_t,
                                               ctypes.POINTER(ctypes.c_double)]),
    "mppi_server_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(MppiServerStats)]),
    "mppi_train_config_default": (None, [ctypes.POINTER(MppiTrainConfig)]),
    "mppi_train_create": (ctypes.c_int, [ctypes.POINTER(MppiTrainConfig), ctypes.POINTER(_vp), _vp,
                                         ctypes.POINTER(_vp)]),
    "mppi_train_destroy": (None, [_vp]),
    "mppi_train_last_error": (ctypes.c_char_p, [_vp]),
    "mppi_train_step": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
    "mppi_train_set_lr": (ctypes.c_int, [_vp, ctypes.c_float]),
    "mppi_train_set_gemm_precision": (ctypes.c_int, [_vp, ctypes.c_int]),
    "mppi_train_loss_grads": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float), _vp]),
    "mppi_train_get_weights": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "mppi_train_evaluate": (ctypes.c_int, [_vp] + [ctypes.POINTER(ctypes.c_float)] * 4),
    "mppi_train_read_points": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t]),
    "mppi_train_num_params": (ctypes.c_int, []),
    "mppi_depth_camera_default": (None, [ctypes.POINTER(MppiDepthCamera)]),
    "mppi_sample_sdf_queries": (ctypes.c_int, [ctypes.POINTER(MppiDepthCamera), ctypes.c_int, _vp, ctypes.c_int, _vp,
                                               ctypes.c_int, ctypes.c_float, _vp, _vp, _vp]),
    "mppi_encoder_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp), ctypes.c_int,
                                           _vp, ctypes.POINTER(_vp)]),
    "mppi_encoder_destroy": (None, [_vp]),
    "mppi_encoder_last_error": (ctypes.c_char_p, [_vp]),
    "mppi_encode_depth": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_float, _vp]),
    "mppi_encoder_get_weights": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "mppi_encoder_set_conv_path": (ctypes.c_int, [_vp, ctypes.c_int]),
    "mppi_encoder_check": (ctypes.c_int, [_vp]),
    "mppi_encoder_debug_inject_timeout": (ctypes.c_int, [_vp]),
    "mppi_encoder_train_create": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_float, _vp, _vp, ctypes.POINTER(_vp)]),
    "mppi_encoder_train_destroy": (None, [_vp]),
    "mppi_encoder_train_last_error": (ctypes.c_char_p, [_vp]),
    "mppi_encoder_train_loss_grads": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_float,
                                                     ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_vp)]),
    "mppi_encoder_train_step": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_float,
                                               ctypes.POINTER(ctypes.c_float)]),
    "mppi_encoder_train_get_decoder": (ctypes.c_int, [_vp, _vp, _vp]),
    "mppi_encoder_train_set_sdf": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_float,
                                                  ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_int]),
    "mppi_encoder_train_get_sdf_decoder": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "mppi_encoder_train_loss_grads_sdf": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_float, _vp, _vp,
                                                         ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "mppi_encoder_train_step_sdf": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_float, _vp, _vp,
                                                   ctypes.c_int, _vp]),
    "mppi_render_depth": (ctypes.c_int, [ctypes.POINTER(MppiDepthCamera), ctypes.c_int, _vp, ctypes.c_int, _vp, _vp,
                                         _vp]),
}

_lib = None


def load(path=LIB_PATH):
    """Load the CUDA library (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2603_07199_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(x):
    """Address of a buffer: None, an int, a NumPy array (C-contiguous) or a tensor with
    data_ptr() (contiguous).  NumPy arrays are tested first by type: a host-buffer step passes
    two of them per call, and the attribute probes cost more than the call's own marshalling."""
    if x is None:
        return None
    if type(x) is _np_ndarray:
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(rc, ctx=None):
    if rc < 0:
        msg = load().mppi_last_error(ctx)
        raise MppiError(rc, msg.decode() if msg else "")
    return rc


def mppi_config_default():
    cfg = MppiConfig()
    load().mppi_config_default(ctypes.byref(cfg))
    return cfg


def mppi_state_dim(cfg):
    return load().mppi_state_dim(ctypes.byref(cfg))


def mppi_create(cfg, stream=None):
    ctx = _vp()
    _check(load().mppi_create(ctypes.byref(cfg), stream, ctypes.byref(ctx)))
    return ctx


def mppi_destroy(ctx):
    load().mppi_destroy(ctx)


def mppi_last_error(ctx=None):
    m = load().mppi_last_error(ctx)
    return m.decode() if m else ""


def mppi_set_gates(ctx, n_gates, poses, latents=None):
    return _check(load().mppi_set_gates(ctx, n_gates, _ptr(poses), _ptr(latents)), ctx)


def mppi_set_sdf_weights(ctx, layers, fp8_scales=None):
    """layers: [W1, b1, W2, b2, W3, b3, W4, b4, W5, b5] as float32 arrays (kept alive by the caller);
    fp8_scales: None or 3 float32 activation scales for MPPI_SDF_MLP_FP8."""
    arr = (_vp * len(layers))(*[_ptr(a) for a in layers])
    return _check(load().mppi_set_sdf_weights(ctx, arr, len(layers), _ptr(fp8_scales)), ctx)


def mppi_step(ctx, state, gate_poses, latents, nominal, new_controls, weights=None, costs=None):
    return _check(load().mppi_step(ctx, _ptr(state), _ptr(gate_poses), _ptr(latents), _ptr(nominal),
                                   _ptr(new_controls), _ptr(weights), _ptr(costs)), ctx)


def mppi_step_async(ctx, d_state, d_gate_poses, d_latents, d_nominal, d_new_controls, d_weights=None, d_costs=None):
    return _check(load().mppi_step_async(ctx, _ptr(d_state), _ptr(d_gate_poses), _ptr(d_latents), _ptr(d_nominal),
                                         _ptr(d_new_controls), _ptr(d_weights), _ptr(d_costs)), ctx)


def mppi_sync(ctx):
    return _check(load().mppi_sync(ctx), ctx)


def mppi_get_nominal(ctx, out):
    return _check(load().mppi_get_nominal(ctx, _ptr(out)), ctx)


def mppi_get_state(ctx, out):
    return _check(load().mppi_get_state(ctx, _ptr(out)), ctx)


def mppi_set_step_counter(ctx, step):
    return _check(load().mppi_set_step_counter(ctx, step), ctx)


def mppi_get_step_counter(ctx):
    return load().mppi_get_step_counter(ctx)


def mppi_read_buffer(ctx, which, out):
    return _check(load().mppi_read_buffer(ctx, which, _ptr(out), out.size if hasattr(out, "size") and
                                          not callable(out.size) else out.numel()), ctx)


def mppi_read_noise_words(ctx, out):
    return _check(load().mppi_read_noise_words(ctx, _ptr(out), out.size), ctx)


def mppi_debug_inject_timeout(ctx):
    return _check(load().mppi_debug_inject_timeout(ctx), ctx)


def mppi_set_diagnostics(ctx, flags):
    return _check(load().mppi_set_diagnostics(ctx, int(flags)), ctx)


def mppi_set_timing(ctx, enable):
    return _check(load().mppi_set_timing(ctx, 1 if enable else 0), ctx)


def mppi_get_kernel_times(ctx, cap=16):
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_float * cap)()
    n = _check(load().mppi_get_kernel_times(ctx, names, ms, cap), ctx)
    return [(names[i].decode(), ms[i]) for i in range(n)]


def mppi_kernels_per_step(ctx):
    return load().mppi_kernels_per_step(ctx)


MPPI_NOALLOC_MAX_K = 131072


def mppi_softmax_update_noalloc(d_costs, d_noise, d_nominal, K, H, lam, thrust_min, thrust_max, rate_max,
                                d_new_controls, d_weights=None, stream=None):
    """Allocation-free weights + update on caller-owned device buffers (see include/mppi.h)."""
    return _check(load().mppi_softmax_update_noalloc(_ptr(d_costs), _ptr(d_noise), _ptr(d_nominal), K, H, lam,
                                                     thrust_min, thrust_max, rate_max, _ptr(d_new_controls),
                                                     _ptr(d_weights), stream))


def mppi_selftest_tc_gemm(d_A, d_B, d_D, stream=None):
    return _check(load().mppi_selftest_tc_gemm(_ptr(d_A), _ptr(d_B), _ptr(d_D), stream))


# ------------------------------------------------------------------ serving
def _scheck(rc, server=None):
    if rc < 0:
        msg = load().mppi_server_last_error(server)
        raise MppiError(rc, msg.decode() if msg else "")
    return rc


def mppi_server_config_default():
    cfg = MppiServerConfig()
    load().mppi_server_config_default(ctypes.byref(cfg))
    return cfg


def mppi_server_create(cfg):
    srv = _vp()
    _scheck(load().mppi_server_create(ctypes.byref(cfg), ctypes.byref(srv)))
    return srv


def mppi_server_destroy(server):
    load().mppi_server_destroy(server)


def mppi_server_last_error(server=None):
    m = load().mppi_server_last_error(server)
    return m.decode() if m else ""


def mppi_server_set_sdf_weights(server, layers, fp8_scales=None):
    arr = (_vp * len(layers))(*[_ptr(a) for a in layers])
    return _scheck(load().mppi_server_set_sdf_weights(server, arr, len(layers), _ptr(fp8_scales)), server)


def mppi_server_submit(server, drone_id, cfg, state, n_gates, poses, latents):
    """Queue one control step; returns its ticket."""
    t = ctypes.c_uint64()
    _scheck(load().mppi_server_submit(server, drone_id, ctypes.byref(cfg), _ptr(state), n_gates, _ptr(poses),
                                      _ptr(latents), ctypes.byref(t)), server)
    return t.value


def mppi_server_poll(server, ticket, new_controls):
    """Returns (status, latency_us): status MPPI_PENDING while queued or running; raises on a request error."""
    lat = ctypes.c_double()
    rc = _scheck(load().mppi_server_poll(server, ticket, _ptr(new_controls), ctypes.byref(lat)), server)
    return rc, lat.value


def mppi_server_next_result(server, new_controls):
    """Returns (status, ticket, latency_us) of any finished request, or (MPPI_PENDING, 0, 0.0)."""
    t = ctypes.c_uint64()
    lat = ctypes.c_double()
    cap = 0 if new_controls is None else new_controls.size
    rc = _scheck(load().mppi_server_next_result(server, ctypes.byref(t), _ptr(new_controls), cap,
                                                ctypes.byref(lat)), server)
    return rc, t.value, lat.value


def mppi_server_get_stats(server):
    st = MppiServerStats()
    _scheck(load().mppi_server_get_stats(server, ctypes.byref(st)), server)
    return {f: getattr(st, f) for f, _ in MppiServerStats._fields_}


# ------------------------------------------------------------------ learned part (distillation)
def _tcheck(rc, trainer=None):
    if rc < 0:
        msg = load().mppi_train_last_error(trainer)
        raise MppiError(rc, msg.decode() if msg else "")
    return rc


def mppi_train_config_default():
    cfg = MppiTrainConfig()
    load().mppi_train_config_default(ctypes.byref(cfg))
    return cfg


def mppi_train_create(cfg, init_layers, latent):
    """init_layers: [W1, b1, ..., w5, b5] float32 arrays; latent: 64 float32."""
    arr = (_vp * len(init_layers))(*[_ptr(a) for a in init_layers])
    tr = _vp()
    _tcheck(load().mppi_train_create(ctypes.byref(cfg), arr, _ptr(latent), ctypes.byref(tr)))
    return tr


def mppi_train_destroy(trainer):
    load().mppi_train_destroy(trainer)


def mppi_train_set_lr(trainer, lr):
    return _tcheck(load().mppi_train_set_lr(trainer, ctypes.c_float(lr)), trainer)


def mppi_train_set_gemm_precision(trainer, precision):
    return _tcheck(load().mppi_train_set_gemm_precision(trainer, int(precision)), trainer)


def mppi_train_step(trainer, n_steps):
    loss = ctypes.c_float()
    _tcheck(load().mppi_train_step(trainer, n_steps, ctypes.byref(loss)), trainer)
    return loss.value


def mppi_train_num_params():
    return load().mppi_train_num_params()


def mppi_train_loss_grads(trainer, points, grads):
    loss = ctypes.c_float()
    _tcheck(load().mppi_train_loss_grads(trainer, _ptr(points), points.shape[0], ctypes.byref(loss), _ptr(grads)),
            trainer)
    return loss.value


def mppi_train_get_weights(trainer, layers_out):
    arr = (_vp * len(layers_out))(*[_ptr(a) for a in layers_out])
    return _tcheck(load().mppi_train_get_weights(trainer, arr), trainer)


def mppi_train_evaluate(trainer):
    """Held-out error against the exact SDF (metres): dict of mae, p99, max, near_p99."""
    v = [ctypes.c_float() for _ in range(4)]
    _tcheck(load().mppi_train_evaluate(trainer, *[ctypes.byref(x) for x in v]), trainer)
    return dict(mae=v[0].value, p99=v[1].value, max=v[2].value, near_p99=v[3].value)


def mppi_train_read_points(trainer, which, out):
    return _tcheck(load().mppi_train_read_points(trainer, which, _ptr(out), out.size), trainer)


# ------------------------------------------------------------------ vision front end (depth images)
MPPI_MAX_IMAGE_SIDE = 8192
MPPI_MAX_RENDER_GATES = 64


def mppi_depth_camera_default():
    cam = MppiDepthCamera()
    load().mppi_depth_camera_default(ctypes.byref(cam))
    return cam


def mppi_sample_sdf_queries(cam, n_views, d_cam_poses, n_gates, d_gate_poses, n_points, near_frac, d_points,
                            d_labels, stream=None):
    """Enqueue camera-frame training queries and their exact SDF labels (device pointers)."""
    return _check(load().mppi_sample_sdf_queries(ctypes.byref(cam), n_views, _ptr(d_cam_poses), n_gates,
                                                 _ptr(d_gate_poses), n_points, near_frac, _ptr(d_points),
                                                 _ptr(d_labels), _ptr(stream)))


def mppi_render_depth(cam, n_views, d_cam_poses, n_gates, d_gate_poses, d_depth, stream=None):
    """Enqueue n_views depth images [n_views, height, width] into d_depth (device pointers)."""
    return _check(load().mppi_render_depth(ctypes.byref(cam), n_views, _ptr(d_cam_poses), n_gates,
                                           _ptr(d_gate_poses), _ptr(d_depth), _ptr(stream)))


# ------------------------------------------------------------------ vision front end (depth encoder)
MPPI_ENCODER_LAYERS = 5
MPPI_ENC_CONV_FP32 = 0
MPPI_ENC_CONV_TC = 1


def _echeck(rc, enc=None):
    if rc < 0:
        msg = load().mppi_encoder_last_error(enc)
        raise MppiError(rc, msg.decode() if msg else "")
    return rc


def mppi_encoder_create(height, width, max_images, layers, stream=None):
    """layers: [W1, b1, ..., W4, b4, W5, b5] float32 host arrays (see include/mppi.h)."""
    arr = (_vp * len(layers))(*[_ptr(a) for a in layers])
    enc = _vp()
    _echeck(load().mppi_encoder_create(height, width, max_images, arr, len(layers), _ptr(stream), ctypes.byref(enc)))
    return enc


def mppi_encoder_destroy(enc):
    load().mppi_encoder_destroy(enc)


def mppi_encode_depth(enc, n_images, d_depth, max_range, d_latents):
    return _echeck(load().mppi_encode_depth(enc, n_images, _ptr(d_depth), max_range, _ptr(d_latents)), enc)


def mppi_encoder_set_conv_path(enc, path):
    return _echeck(load().mppi_encoder_set_conv_path(enc, path), enc)


def mppi_encoder_check(enc):
    return _echeck(load().mppi_encoder_check(enc), enc)


def mppi_encoder_debug_inject_timeout(enc):
    return _echeck(load().mppi_encoder_debug_inject_timeout(enc), enc)


def mppi_encoder_get_weights(enc, layers_out):
    arr = (_vp * len(layers_out))(*[_ptr(a) for a in layers_out])
    return _echeck(load().mppi_encoder_get_weights(enc, arr), enc)


# ------------------------------------------------------------------ vision front end (encoder training)
def _etcheck(rc, trainer=None):
    if rc < 0:
        msg = load().mppi_encoder_train_last_error(trainer)
        raise MppiError(rc, msg.decode() if msg else "")
    return rc


def mppi_encoder_train_create(enc, batch, lr, dec_W, dec_b):
    tr = _vp()
    _etcheck(load().mppi_encoder_train_create(enc, batch, lr, _ptr(dec_W), _ptr(dec_b), ctypes.byref(tr)))
    return tr


def mppi_encoder_train_destroy(trainer):
    load().mppi_encoder_train_destroy(trainer)


def mppi_encoder_train_loss_grads(trainer, n, d_noisy, d_clean, max_range, grads_out=None):
    """Returns the batch loss; fills the 12 host gradient arrays of grads_out when given."""
    loss = ctypes.c_float()
    arr = None if grads_out is None else (_vp * len(grads_out))(*[_ptr(a) for a in grads_out])
    _etcheck(load().mppi_encoder_train_loss_grads(trainer, n, _ptr(d_noisy), _ptr(d_clean), max_range,
                                                  ctypes.byref(loss), arr), trainer)
    return loss.value


def mppi_encoder_train_step(trainer, n, d_noisy, d_clean, max_range, want_loss=True):
    loss = ctypes.c_float()
    _etcheck(load().mppi_encoder_train_step(trainer, n, _ptr(d_noisy), _ptr(d_clean), max_range,
                                            ctypes.byref(loss) if want_loss else None), trainer)
    return loss.value if want_loss else None


def mppi_encoder_train_get_decoder(trainer, W, b):
    return _etcheck(load().mppi_encoder_train_get_decoder(trainer, _ptr(W), _ptr(b)), trainer)


def mppi_encoder_train_set_sdf(trainer, layers, pe_levels, softplus_beta, lambda_recon, lambda_sdf,
                               max_points_per_image, train_decoder=False):
    arr = (_vp * len(layers))(*[_ptr(a) for a in layers])
    return _etcheck(load().mppi_encoder_train_set_sdf(trainer, arr, pe_levels, softplus_beta, lambda_recon,
                                                      lambda_sdf, max_points_per_image, int(train_decoder)), trainer)


def mppi_encoder_train_get_sdf_decoder(trainer, layers_out):
    arr = (_vp * len(layers_out))(*[_ptr(a) for a in layers_out])
    return _etcheck(load().mppi_encoder_train_get_sdf_decoder(trainer, arr), trainer)


def mppi_encoder_train_loss_grads_sdf(trainer, n, d_noisy, d_clean, max_range, d_points, d_labels, n_points,
                                      grads_out=None):
    """Returns (total, reconstruction, SDF) losses; fills the 12 host gradient arrays when given."""
    import numpy as _np
    losses = _np.zeros(3, _np.float32)
    arr = None if grads_out is None else (_vp * len(grads_out))(*[_ptr(a) for a in grads_out])
    _etcheck(load().mppi_encoder_train_loss_grads_sdf(trainer, n, _ptr(d_noisy), _ptr(d_clean), max_range,
                                                      _ptr(d_points), _ptr(d_labels), n_points, _ptr(losses), arr),
             trainer)
    return tuple(float(x) for x in losses)


def mppi_encoder_train_step_sdf(trainer, n, d_noisy, d_clean, max_range, d_points, d_labels, n_points,
                                want_loss=True):
    import numpy as _np
    losses = _np.zeros(3, _np.float32)
    _etcheck(load().mppi_encoder_train_step_sdf(trainer, n, _ptr(d_noisy), _ptr(d_clean), max_range, _ptr(d_points),
                                                _ptr(d_labels), n_points, _ptr(losses) if want_loss else None),
             trainer)
    return tuple(float(x) for x in losses) if want_loss else None
