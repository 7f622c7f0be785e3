"""Thin Python binding of the C ABI in include/lidar.h (argument marshalling
only). Every step of the computation runs in the sm_103a library
``liblidar_gb300.so``; there is no other code path. Loading fails loudly if
the library has not been built.

Functions keep the C names (lidar_create, lidar_simulate, ...). ``Lidar`` is a
small convenience wrapper that owns a handle and allocates outputs as torch
CUDA tensors (PyTorch provides device memory and streams only).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblidar_gb300.so")

LIDAR_OK, LIDAR_EINVAL, LIDAR_ENOMEM, LIDAR_ECUDA, LIDAR_ETIMEOUT, LIDAR_ENUMERIC = range(6)
LIDAR_PROFILE_RADIAL, LIDAR_PROFILE_TABLE, LIDAR_PROFILE_SEPARABLE = 0, 1, 2
ECHO_CLIPPED_START, ECHO_CLIPPED_END, ECHO_NEAR_THRESHOLD = 1, 2, 4


class lidar_profile_t(C.Structure):
    _fields_ = [("kind", C.c_int32), ("sigma_deg", C.c_double), ("tail_amp", C.c_double),
                ("tail_core_deg", C.c_double), ("tail_pow", C.c_double), ("trunc_deg", C.c_double),
                ("table_w", C.c_int32), ("table_h", C.c_int32), ("pitch_deg", C.c_double),
                ("table", C.POINTER(C.c_float))]


class lidar_pattern_t(C.Structure):
    _fields_ = [("n_beams", C.c_int32), ("dirs", C.POINTER(C.c_float))]


class lidar_pulse_t(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("dt_s", C.c_double), ("t0_s", C.c_double), ("fwhm_s", C.c_double),
                ("trunc_sigmas", C.c_double)]


class lidar_calib_t(C.Structure):
    _fields_ = [("threshold", C.c_double), ("ambient_scale", C.c_double), ("max_echoes", C.c_int32),
                ("fit_epw", C.c_int32), ("epw_coef", C.c_double * 3)]


class lidar_gbuffer_t(C.Structure):
    _fields_ = [("U", C.c_int32), ("V", C.c_int32), ("az0", C.c_double), ("el0", C.c_double),
                ("daz", C.c_double), ("del_", C.c_double)] + [
        (n, C.c_void_p) for n in ("range", "nx", "ny", "nz", "rho_d", "retro", "ambient")]


class lidar_pose_t(C.Structure):
    _fields_ = [("R", C.c_float * 9)]


class lidar_echo_t(C.Structure):
    _fields_ = [("range_m", C.c_float), ("epw_m", C.c_float), ("intensity", C.c_float), ("peak", C.c_float),
                ("bin_peak", C.c_int32), ("bin_start", C.c_int32), ("bin_end", C.c_int32), ("flags", C.c_uint32)]


class lidar_echoes_t(C.Structure):
    _fields_ = [("echoes", C.c_void_p), ("counts", C.c_void_p)]


class lidar_stack_params_t(C.Structure):
    _fields_ = [("kh", C.c_int32), ("kw", C.c_int32), ("kernel", C.POINTER(C.c_float)), ("threshold", C.c_double),
                ("dr", C.c_double), ("r_max", C.c_double)]


class lidar_pinhole_t(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("R", C.c_double * 9), ("depth_is_z", C.c_int32),
                ("range", C.c_void_p), ("nx", C.c_void_p), ("ny", C.c_void_p), ("nz", C.c_void_p),
                ("rho_d", C.c_void_p), ("retro", C.c_void_p), ("ambient", C.c_void_p)]


class lidar_stack_sep_params_t(C.Structure):
    _fields_ = [("kh", C.c_int32), ("kw", C.c_int32), ("col", C.POINTER(C.c_float)), ("row", C.POINTER(C.c_float)),
                ("threshold", C.c_double), ("dr", C.c_double), ("r_max", C.c_double)]


class lidar_frame_t(C.Structure):
    _fields_ = [("sensor", C.c_void_p), ("gbuffer", lidar_gbuffer_t), ("pose", lidar_pose_t),
                ("out_waveforms", C.c_void_p), ("out_echoes", lidar_echoes_t)]


ECHO_DTYPE = np.dtype([("range_m", "f4"), ("epw_m", "f4"), ("intensity", "f4"), ("peak", "f4"),
                       ("bin_peak", "i4"), ("bin_start", "i4"), ("bin_end", "i4"), ("flags", "u4")])
assert ECHO_DTYPE.itemsize == C.sizeof(lidar_echo_t) == 32

# exported symbols (every function declared in include/lidar.h)
SYMBOLS = ("lidar_create", "lidar_simulate", "lidar_simulate_echoes", "lidar_reproject_pinhole", "lidar_simulate_host",
           "lidar_simulate_host_frames", "lidar_simulate_noalloc",
           "lidar_sync",
           "lidar_simulate_batch", "lidar_autotune_batch", "lidar_batch_config", "lidar_get_info",
           "lidar_launches_per_simulate", "lidar_set_deposit", "lidar_set_echo_mode", "lidar_hold_echo_slots",
           "lidar_profile_enable",
           "lidar_profile_read", "lidar_last_error",
           "lidar_destroy")
# include/lidar_tail.h
TAIL_SYMBOLS = ("lidar_tail_configure", "lidar_tail_features", "lidar_tail_exact", "lidar_simulate_split",
                "lidar_tailnet_create", "lidar_tailnet_destroy", "lidar_tailnet_last_error", "lidar_tailnet_num_params",
                "lidar_tailnet_get_params", "lidar_tailnet_set_params", "lidar_tailnet_predict",
                "lidar_tailnet_train_step", "lidar_tailnet_grads", "lidar_tailnet_save", "lidar_tailnet_load",
                "lidar_simulate_surrogate", "lidar_tailnet_profile_enable", "lidar_tailnet_profile_read",
                "lidar_tailnet_set_dense", "lidar_tailnet_sync")
# include/lidar_stack.h
STACK_SYMBOLS = ("lidar_stack_create", "lidar_stack_create_separable", "lidar_range_stack", "lidar_stack_last_error",
                 "lidar_stack_destroy")
KERNELS = ("setup", "footprint_wave")
TAIL_INPUT_CELLS = 5440

_lib = None


class LidarError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lidar status {status}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Loads the CUDA library; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2512_05932_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.POINTER
    lib.lidar_create.restype = C.c_int
    lib.lidar_create.argtypes = [P(lidar_profile_t), P(lidar_pattern_t), P(lidar_pulse_t), P(lidar_calib_t),
                                 P(C.c_void_p)]
    lib.lidar_simulate.restype = C.c_int
    lib.lidar_simulate.argtypes = [C.c_void_p, P(lidar_gbuffer_t), P(lidar_pose_t), C.c_void_p,
                                   P(lidar_echoes_t), C.c_void_p]
    lib.lidar_reproject_pinhole.restype = C.c_int
    lib.lidar_reproject_pinhole.argtypes = [P(lidar_pinhole_t), P(lidar_gbuffer_t), C.c_void_p]
    lib.lidar_simulate_echoes.restype = C.c_int
    lib.lidar_simulate_echoes.argtypes = [C.c_void_p, P(lidar_gbuffer_t), P(lidar_pose_t), P(lidar_echoes_t),
                                          C.c_void_p]
    lib.lidar_simulate_host.restype = C.c_int
    lib.lidar_simulate_host.argtypes = [C.c_void_p, P(lidar_gbuffer_t), P(lidar_pose_t), C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
    lib.lidar_simulate_host_frames.restype = C.c_int
    lib.lidar_simulate_host_frames.argtypes = [C.c_void_p, C.c_int, P(lidar_gbuffer_t), P(lidar_pose_t), C.c_void_p,
                                               C.c_void_p, C.c_void_p, C.c_void_p]
    lib.lidar_simulate_noalloc.restype = C.c_int
    lib.lidar_simulate_noalloc.argtypes = [C.c_void_p, P(lidar_gbuffer_t), P(lidar_pose_t), C.c_void_p,
                                           P(lidar_echoes_t), C.c_void_p]
    lib.lidar_simulate_batch.restype = C.c_int
    lib.lidar_simulate_batch.argtypes = [C.c_void_p, P(lidar_frame_t), C.c_int32, C.c_void_p]
    lib.lidar_autotune_batch.restype = C.c_int
    lib.lidar_autotune_batch.argtypes = [C.c_void_p, P(lidar_frame_t), C.c_int32, C.c_void_p]
    lib.lidar_batch_config.restype = C.c_int
    lib.lidar_batch_config.argtypes = [C.c_void_p, P(C.c_int32), P(C.c_int32)]
    lib.lidar_sync.restype = C.c_int
    lib.lidar_sync.argtypes = [C.c_void_p, C.c_void_p]
    lib.lidar_get_info.restype = C.c_int
    lib.lidar_get_info.argtypes = [C.c_void_p, P(C.c_int32), P(C.c_int32), P(C.c_int32), P(C.c_double),
                                   P(C.c_double)]
    lib.lidar_launches_per_simulate.restype = C.c_int32
    lib.lidar_launches_per_simulate.argtypes = [C.c_void_p]
    lib.lidar_set_deposit.restype = C.c_int
    lib.lidar_set_deposit.argtypes = [C.c_void_p, C.c_int32]
    lib.lidar_set_echo_mode.restype = C.c_int
    lib.lidar_set_echo_mode.argtypes = [C.c_void_p, C.c_int32]
    lib.lidar_hold_echo_slots.restype = C.c_int
    lib.lidar_hold_echo_slots.argtypes = [C.c_void_p, C.c_int32]
    lib.lidar_profile_enable.restype = C.c_int
    lib.lidar_profile_enable.argtypes = [C.c_void_p, C.c_int32]
    lib.lidar_profile_read.restype = C.c_int
    lib.lidar_profile_read.argtypes = [C.c_void_p, P(C.c_double), P(C.c_int32)]
    lib.lidar_last_error.restype = C.c_char_p
    lib.lidar_last_error.argtypes = [C.c_void_p]
    lib.lidar_destroy.restype = None
    lib.lidar_destroy.argtypes = [C.c_void_p]
    lib.lidar_tail_configure.restype = C.c_int
    lib.lidar_tail_configure.argtypes = [C.c_void_p, C.c_double, C.c_int32]
    lib.lidar_tail_features.restype = C.c_int
    lib.lidar_tail_features.argtypes = [C.c_void_p, P(lidar_gbuffer_t), P(lidar_pose_t), C.c_void_p, C.c_void_p,
                                        C.c_void_p]
    lib.lidar_tail_exact.restype = C.c_int
    lib.lidar_tail_exact.argtypes = [C.c_void_p, P(lidar_gbuffer_t), P(lidar_pose_t), C.c_void_p, C.c_void_p]
    lib.lidar_simulate_split.restype = C.c_int
    lib.lidar_simulate_split.argtypes = [C.c_void_p, P(lidar_gbuffer_t), P(lidar_pose_t), C.c_void_p, C.c_void_p,
                                         P(lidar_echoes_t), P(C.c_int32), C.c_void_p]
    lib.lidar_tailnet_create.restype = C.c_int
    lib.lidar_tailnet_create.argtypes = [C.c_int32, C.c_uint64, P(C.c_void_p)]
    lib.lidar_tailnet_destroy.restype = None
    lib.lidar_tailnet_destroy.argtypes = [C.c_void_p]
    lib.lidar_tailnet_last_error.restype = C.c_char_p
    lib.lidar_tailnet_last_error.argtypes = [C.c_void_p]
    lib.lidar_tailnet_num_params.restype = C.c_int64
    lib.lidar_tailnet_num_params.argtypes = [C.c_void_p]
    lib.lidar_tailnet_get_params.restype = C.c_int
    lib.lidar_tailnet_get_params.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    lib.lidar_tailnet_set_params.restype = C.c_int
    lib.lidar_tailnet_set_params.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    lib.lidar_tailnet_predict.restype = C.c_int
    lib.lidar_tailnet_predict.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
    lib.lidar_tailnet_train_step.restype = C.c_int
    lib.lidar_tailnet_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float,
                                             P(C.c_float), C.c_void_p]
    lib.lidar_tailnet_grads.restype = C.c_int
    lib.lidar_tailnet_grads.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                        P(C.c_float), C.c_void_p]
    lib.lidar_tailnet_save.restype = C.c_int
    lib.lidar_tailnet_save.argtypes = [C.c_void_p, C.c_char_p, C.c_int32]
    lib.lidar_tailnet_load.restype = C.c_int
    lib.lidar_tailnet_load.argtypes = [C.c_void_p, C.c_char_p]
    lib.lidar_tailnet_profile_enable.restype = C.c_int
    lib.lidar_tailnet_profile_enable.argtypes = [C.c_void_p, C.c_int32]
    lib.lidar_tailnet_profile_read.restype = C.c_int
    lib.lidar_tailnet_profile_read.argtypes = [C.c_void_p, P(C.c_double), P(C.c_int32)]
    lib.lidar_tailnet_set_dense.restype = C.c_int
    lib.lidar_tailnet_set_dense.argtypes = [C.c_void_p, C.c_int32]
    lib.lidar_tailnet_sync.restype = C.c_int
    lib.lidar_tailnet_sync.argtypes = [C.c_void_p, C.c_void_p]
    lib.lidar_stack_create.restype = C.c_int
    lib.lidar_stack_create.argtypes = [P(lidar_stack_params_t), P(C.c_void_p)]
    lib.lidar_stack_create_separable.restype = C.c_int
    lib.lidar_stack_create_separable.argtypes = [P(lidar_stack_sep_params_t), P(C.c_void_p)]
    lib.lidar_range_stack.restype = C.c_int
    lib.lidar_range_stack.argtypes = [C.c_void_p, P(lidar_gbuffer_t), C.c_void_p, C.c_void_p, C.c_void_p]
    lib.lidar_stack_last_error.restype = C.c_char_p
    lib.lidar_stack_last_error.argtypes = [C.c_void_p]
    lib.lidar_stack_destroy.restype = None
    lib.lidar_stack_destroy.argtypes = [C.c_void_p]
    lib.lidar_simulate_surrogate.restype = C.c_int
    lib.lidar_simulate_surrogate.argtypes = [C.c_void_p, C.c_void_p, P(lidar_gbuffer_t), P(lidar_pose_t), C.c_void_p,
                                             P(lidar_echoes_t), P(C.c_int32), C.c_void_p]
    _lib = lib
    return lib


# --------------------------------------------------------------------------
# struct builders from the plain dicts of the input generators
# --------------------------------------------------------------------------


def make_profile(prof: dict, keep: list) -> lidar_profile_t:
    p = lidar_profile_t()
    p.kind = int(prof["kind"])
    if p.kind == LIDAR_PROFILE_RADIAL:
        for k in ("sigma_deg", "tail_amp", "tail_core_deg", "tail_pow", "trunc_deg"):
            setattr(p, k, float(prof[k]))
    elif p.kind == LIDAR_PROFILE_SEPARABLE:
        h = np.ascontiguousarray(prof["h"], dtype=np.float32)
        v = np.ascontiguousarray(prof["v"], dtype=np.float32)
        t = np.ascontiguousarray(np.concatenate([h, v]), dtype=np.float32)
        keep.append(t)
        p.table_w, p.table_h = len(h), len(v)
        p.pitch_deg = float(prof["pitch_deg"])
        p.table = t.ctypes.data_as(C.POINTER(C.c_float))
    else:
        t = np.ascontiguousarray(prof["table"], dtype=np.float32)
        keep.append(t)
        p.table_w, p.table_h = t.shape[1], t.shape[0]
        p.pitch_deg = float(prof["pitch_deg"])
        p.table = t.ctypes.data_as(C.POINTER(C.c_float))
    return p


def make_pattern(dirs, keep: list) -> lidar_pattern_t:
    d = np.ascontiguousarray(dirs, dtype=np.float32).reshape(-1, 3)
    keep.append(d)
    return lidar_pattern_t(len(d), d.ctypes.data_as(C.POINTER(C.c_float)))


def make_pulse(pu: dict) -> lidar_pulse_t:
    return lidar_pulse_t(int(pu["n_bins"]), float(pu["dt_s"]), float(pu["t0_s"]), float(pu["fwhm_s"]),
                         float(pu["trunc_sigmas"]))


def make_calib(ca: dict) -> lidar_calib_t:
    c = lidar_calib_t()
    c.threshold = float(ca["threshold"])
    c.ambient_scale = float(ca["ambient_scale"])
    c.max_echoes = int(ca["max_echoes"])
    c.fit_epw = int(ca["fit_epw"])
    for i, v in enumerate(ca.get("epw_coef", (0.0, 0.0, 0.0))):
        c.epw_coef[i] = float(v)
    return c


def make_gbuffer(geom, planes) -> lidar_gbuffer_t:
    """geom: object with U, V, az0, el0, daz, dele; planes: 7 pointers (ints)."""
    g = lidar_gbuffer_t()
    g.U, g.V = int(geom.U), int(geom.V)
    g.az0, g.el0, g.daz, g.del_ = float(geom.az0), float(geom.el0), float(geom.daz), float(geom.dele)
    for name, ptr in zip(("range", "nx", "ny", "nz", "rho_d", "retro", "ambient"), planes):
        setattr(g, name, ptr)
    return g


def make_pose(R) -> lidar_pose_t:
    p = lidar_pose_t()
    R = np.asarray(R, dtype=np.float32).ravel()
    for i in range(9):
        p.R[i] = float(R[i])
    return p


# --------------------------------------------------------------------------
# C-named functions
# --------------------------------------------------------------------------


def lidar_last_error(handle=None) -> str:
    return load().lidar_last_error(handle).decode()


def _check(st, handle=None):
    if st != LIDAR_OK:
        raise LidarError(st, lidar_last_error(handle))


def lidar_create(profile: dict, dirs, pulse: dict, calib: dict) -> int:
    keep = []
    lib = load()
    out = C.c_void_p()
    st = lib.lidar_create(C.byref(make_profile(profile, keep)), C.byref(make_pattern(dirs, keep)),
                          C.byref(make_pulse(pulse)), C.byref(make_calib(calib)), C.byref(out))
    _check(st)
    return out.value


def lidar_simulate(handle, gbuffer: lidar_gbuffer_t, pose: lidar_pose_t, out_waveforms: int,
                   out_echoes: int, out_counts: int, stream: int = 0) -> None:
    e = lidar_echoes_t(out_echoes, out_counts)
    st = load().lidar_simulate(handle, C.byref(gbuffer), C.byref(pose), out_waveforms, C.byref(e), stream)
    _check(st, handle)


def make_pinhole(ph, ptrs) -> lidar_pinhole_t:
    """lidar_pinhole_t of a scenes.PinholeGBuffer with device plane pointers
    (range, nx, ny, nz, rho_d, retro, ambient)."""
    s = lidar_pinhole_t()
    s.W, s.H = int(ph.W), int(ph.H)
    s.fx, s.fy, s.cx, s.cy = float(ph.fx), float(ph.fy), float(ph.cx), float(ph.cy)
    for i, x in enumerate(np.asarray(ph.R, np.float64).ravel()):
        s.R[i] = float(x)
    s.depth_is_z = int(bool(ph.depth_is_z))
    s.range, s.nx, s.ny, s.nz, s.rho_d, s.retro, s.ambient = [int(p) for p in ptrs]
    return s


def lidar_reproject_pinhole(src: lidar_pinhole_t, dst: lidar_gbuffer_t, stream: int = 0) -> None:
    _check(load().lidar_reproject_pinhole(C.byref(src), C.byref(dst), stream), None)


def lidar_simulate_echoes(handle, gbuffer: lidar_gbuffer_t, pose: lidar_pose_t, out_echoes: int, out_counts: int,
                          stream: int = 0) -> None:
    e = lidar_echoes_t(out_echoes, out_counts)
    st = load().lidar_simulate_echoes(handle, C.byref(gbuffer), C.byref(pose), C.byref(e), stream)
    _check(st, handle)


def lidar_simulate_host(handle, gbuffer: lidar_gbuffer_t, pose: lidar_pose_t, out_waveforms: int,
                        out_echoes: int, out_counts: int, stream: int = 0) -> None:
    st = load().lidar_simulate_host(handle, C.byref(gbuffer), C.byref(pose), out_waveforms, out_echoes,
                                    out_counts, stream)
    _check(st, handle)


def lidar_simulate_host_frames(handle, gbuffers, poses, out_waveforms, out_echoes, out_counts,
                               stream: int = 0) -> None:
    """gbuffers, poses: sequences of lidar_gbuffer_t / lidar_pose_t; out_*:
    sequences of host addresses, one per frame (out_waveforms None: echo-only)."""
    n = len(gbuffers)
    if not (len(poses) == len(out_echoes) == len(out_counts) == n) or (
            out_waveforms is not None and len(out_waveforms) != n):
        raise ValueError("one pose and one output set per frame")
    garr = (lidar_gbuffer_t * max(n, 1))(*gbuffers)
    parr = (lidar_pose_t * max(n, 1))(*poses)
    ptrs = lambda xs: (C.c_void_p * max(n, 1))(*xs)
    st = load().lidar_simulate_host_frames(handle, n, garr, parr,
                                           None if out_waveforms is None else ptrs(out_waveforms),
                                           ptrs(out_echoes), ptrs(out_counts), stream)
    _check(st, handle)


def lidar_simulate_noalloc(handle, gbuffer: lidar_gbuffer_t, pose: lidar_pose_t, out_waveforms: int,
                           out_echoes: int, out_counts: int, stream: int = 0) -> None:
    """lidar_simulate without any device allocation inside the call (fixed
    32 MiB scratch, G-buffers up to 2^20 pixels; see include/lidar.h)."""
    e = lidar_echoes_t(out_echoes, out_counts)
    st = load().lidar_simulate_noalloc(handle, C.byref(gbuffer), C.byref(pose), out_waveforms, C.byref(e), stream)
    _check(st, handle)


def lidar_tail_configure(handle, core_deg: float, n_coarse: int) -> None:
    """Core/tail split of a radial profile (include/lidar_tail.h)."""
    _check(load().lidar_tail_configure(handle, float(core_deg), int(n_coarse)), handle)


def lidar_tail_features(handle, gbuffer: lidar_gbuffer_t, pose: lidar_pose_t, rows: int, inputs: int = 0,
                        stream: int = 0) -> None:
    st = load().lidar_tail_features(handle, C.byref(gbuffer), C.byref(pose), rows, inputs or None, stream)
    _check(st, handle)


def lidar_tail_exact(handle, gbuffer: lidar_gbuffer_t, pose: lidar_pose_t, rows: int, stream: int = 0) -> None:
    _check(load().lidar_tail_exact(handle, C.byref(gbuffer), C.byref(pose), rows, stream), handle)


def lidar_simulate_split(handle, gbuffer: lidar_gbuffer_t, pose: lidar_pose_t, tail: int, out_waveforms: int,
                         out_echoes: int, out_counts: int, stream: int = 0) -> int:
    """Returns the number of beams re-run with the exact profile."""
    e = lidar_echoes_t(out_echoes, out_counts)
    n = C.c_int32(-1)
    st = load().lidar_simulate_split(handle, C.byref(gbuffer), C.byref(pose), tail, out_waveforms, C.byref(e),
                                     C.byref(n), stream)
    _check(st, handle)
    return n.value


def lidar_simulate_surrogate(handle, net, gbuffer: lidar_gbuffer_t, pose: lidar_pose_t, out_waveforms: int,
                             out_echoes: int, out_counts: int, stream: int = 0) -> int:
    """Tail features, network prediction (net None: the physics prior) and the
    split simulation; returns the number of beams re-run exactly."""
    e = lidar_echoes_t(out_echoes, out_counts)
    n = C.c_int32(-1)
    st = load().lidar_simulate_surrogate(handle, net or None, C.byref(gbuffer), C.byref(pose), out_waveforms,
                                         C.byref(e), C.byref(n), stream)
    _check(st, handle)
    return n.value


class TailNet:
    """The learned tail estimator (include/lidar_tail.h): thin wrapper over
    the lidar_tailnet_* functions; device arrays are torch CUDA tensors."""

    def __init__(self, n_coarse: int = 256, seed: int = 0):
        lib = load()
        h = C.c_void_p()
        st = lib.lidar_tailnet_create(int(n_coarse), int(seed), C.byref(h))
        if st != 0:
            raise LidarError(st, lib.lidar_tailnet_last_error(None).decode())
        self.handle = h.value
        self.n_coarse = n_coarse

    def _check(self, st):
        if st != 0:
            raise LidarError(st, load().lidar_tailnet_last_error(self.handle).decode())

    @property
    def num_params(self) -> int:
        return int(load().lidar_tailnet_num_params(self.handle))

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.num_params, np.float32)
        self._check(load().lidar_tailnet_get_params(self.handle, p.ctypes.data, p.size))
        return p

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, np.float32)
        self._check(load().lidar_tailnet_set_params(self.handle, p.ctypes.data, p.size))

    def predict(self, inputs, rows, out, stream: int = 0) -> None:
        self._check(load().lidar_tailnet_predict(self.handle, inputs.data_ptr(), rows.data_ptr(), rows.shape[0],
                                                 out.data_ptr(), stream))

    def train_step(self, inputs, rows, target, lr: float, want_loss: bool = True, stream: int = 0):
        loss = C.c_float(float("nan"))
        self._check(load().lidar_tailnet_train_step(self.handle, inputs.data_ptr(), rows.data_ptr(), target.data_ptr(),
                                                    rows.shape[0], float(lr), C.byref(loss) if want_loss else None,
                                                    stream))
        return loss.value if want_loss else None

    def grads(self, inputs, rows, target, stream: int = 0):
        g = np.zeros(self.num_params, np.float32)
        loss = C.c_float(0.0)
        self._check(load().lidar_tailnet_grads(self.handle, inputs.data_ptr(), rows.data_ptr(), target.data_ptr(),
                                               rows.shape[0], g.ctypes.data, C.byref(loss), stream))
        return float(loss.value), g

    DENSE_TCGEN05 = 0
    DENSE_MMA_SYNC = 1

    def set_dense(self, mode: int) -> None:
        """Kernel of the forward GEMMs: DENSE_TCGEN05 (default) or DENSE_MMA_SYNC."""
        self._check(load().lidar_tailnet_set_dense(self.handle, int(mode)))

    def sync(self, stream: int = 0) -> None:
        """Synchronises `stream`; raises on an asynchronous error or a GEMM wait that gave up."""
        self._check(load().lidar_tailnet_sync(self.handle, stream))

    def profile_enable(self, enable: bool) -> None:
        self._check(load().lidar_tailnet_profile_enable(self.handle, int(bool(enable))))

    def profile_read(self) -> dict:
        t = (C.c_double * 2)()
        n = (C.c_int32 * 2)()
        self._check(load().lidar_tailnet_profile_read(self.handle, t, n))
        return {"conv": (t[0], n[0]), "dense": (t[1], n[1])}

    def save(self, path: str, with_state: bool = True) -> None:
        self._check(load().lidar_tailnet_save(self.handle, os.fsencode(path), int(bool(with_state))))

    def load(self, path: str) -> None:
        self._check(load().lidar_tailnet_load(self.handle, os.fsencode(path)))

    def close(self):
        if self.handle:
            load().lidar_tailnet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RangeStack:
    """Range stacking (include/lidar_stack.h): nearest slice above threshold per pixel."""

    def __init__(self, kernel, threshold: float, dr: float, r_max: float, separable=None):
        """kernel: [kh][kw] array, or None with separable = (col[kh], row[kw])
        for K = col row^T (lidar_stack_create_separable)."""
        h = C.c_void_p()
        lib = load()
        if separable is not None:
            col = np.ascontiguousarray(separable[0], np.float32)
            row = np.ascontiguousarray(separable[1], np.float32)
            self._k = (col, row)
            p = lidar_stack_sep_params_t(len(col), len(row), col.ctypes.data_as(C.POINTER(C.c_float)),
                                         row.ctypes.data_as(C.POINTER(C.c_float)), float(threshold), float(dr),
                                         float(r_max))
            st = lib.lidar_stack_create_separable(C.byref(p), C.byref(h))
        else:
            k = np.ascontiguousarray(kernel, np.float32)
            self._k = k
            p = lidar_stack_params_t(k.shape[0], k.shape[1], k.ctypes.data_as(C.POINTER(C.c_float)),
                                     float(threshold), float(dr), float(r_max))
            st = lib.lidar_stack_create(C.byref(p), C.byref(h))
        if st != 0:
            raise LidarError(st, lib.lidar_stack_last_error(None).decode())
        self.handle = h.value
        self.s_max = int(np.floor(r_max / dr))

    def run(self, gbuffer: lidar_gbuffer_t, out_slice: int, out_intensity: int, stream: int = 0) -> None:
        st = load().lidar_range_stack(self.handle, C.byref(gbuffer), out_slice, out_intensity, stream)
        if st != 0:
            raise LidarError(st, load().lidar_stack_last_error(self.handle).decode())

    def close(self):
        if self.handle:
            load().lidar_stack_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_frames(items) -> "C.Array":
    """items: list of (sensor handle, gbuffer struct, pose struct, waveforms ptr,
    echoes ptr, counts ptr)."""
    arr = (lidar_frame_t * len(items))()
    for i, (h, g, p, w, e, c) in enumerate(items):
        arr[i].sensor = h
        arr[i].gbuffer = g
        arr[i].pose = p
        arr[i].out_waveforms = w
        arr[i].out_echoes = lidar_echoes_t(e, c)
    return arr


def lidar_simulate_batch(executor, frames, stream: int = 0) -> None:
    _check(load().lidar_simulate_batch(executor, frames, len(frames), stream), executor)


def lidar_autotune_batch(executor, frames, stream: int = 0) -> None:
    _check(load().lidar_autotune_batch(executor, frames, len(frames), stream), executor)


def lidar_batch_config(executor) -> tuple:
    g, c = C.c_int32(), C.c_int32()
    _check(load().lidar_batch_config(executor, C.byref(g), C.byref(c)), executor)
    return g.value, c.value


def lidar_sync(handle, stream: int = 0) -> None:
    _check(load().lidar_sync(handle, stream), handle)


def lidar_get_info(handle) -> dict:
    nb, nbin, me = C.c_int32(), C.c_int32(), C.c_int32()
    Z = C.c_double()
    coef = (C.c_double * 3)()
    _check(load().lidar_get_info(handle, C.byref(nb), C.byref(nbin), C.byref(me), C.byref(Z), coef), handle)
    return dict(n_beams=nb.value, n_bins=nbin.value, max_echoes=me.value, profile_norm=Z.value,
                epw_coef=np.array(coef[:]))


def lidar_launches_per_simulate(handle) -> int:
    return int(load().lidar_launches_per_simulate(handle))


DEPOSIT_ATOMIC, DEPOSIT_TC_SPLIT, DEPOSIT_TC_BF16, DEPOSIT_TCGEN05_BF16, DEPOSIT_TCGEN05_FP16 = 0, 1, 2, 3, 4


def lidar_set_deposit(handle, mode: int) -> None:
    _check(load().lidar_set_deposit(handle, int(mode)), handle)


ECHOES_NEAREST, ECHOES_STRONGEST = 0, 1


def lidar_set_echo_mode(handle, mode: int) -> None:
    _check(load().lidar_set_echo_mode(handle, int(mode)), handle)


def lidar_hold_echo_slots(handle, held: bool) -> None:
    _check(load().lidar_hold_echo_slots(handle, int(bool(held))), handle)


def lidar_profile_enable(handle, enable: bool) -> None:
    _check(load().lidar_profile_enable(handle, int(bool(enable))), handle)


def lidar_profile_read(handle) -> dict:
    """{kernel name: (total ms, launches)} accumulated since the last read."""
    t = (C.c_double * 2)()
    n = (C.c_int32 * 2)()
    _check(load().lidar_profile_read(handle, t, n), handle)
    return {k: (t[i], n[i]) for i, k in enumerate(KERNELS)}


def lidar_destroy(handle) -> None:
    if handle:
        load().lidar_destroy(handle)


# --------------------------------------------------------------------------
# convenience wrapper over torch CUDA tensors
# --------------------------------------------------------------------------


def gbuffer_to_device(gb, device="cuda"):
    """Copies the 7 float32 planes of a scenes.GBuffer to torch CUDA tensors."""
    import torch
    return [torch.from_numpy(np.ascontiguousarray(p, dtype=np.float32)).to(device) for p in gb.planes()]


class Lidar:
    def __init__(self, profile, dirs, pulse, calib):
        self.handle = lidar_create(profile, dirs, pulse, calib)
        info = lidar_get_info(self.handle)
        self.n_beams, self.n_bins, self.max_echoes = info["n_beams"], info["n_bins"], info["max_echoes"]
        self.profile_norm, self.epw_coef = info["profile_norm"], info["epw_coef"]

    def alloc_outputs(self, device="cuda"):
        import torch
        wave = torch.empty((self.n_beams, self.n_bins), dtype=torch.float32, device=device)
        echoes = torch.empty((self.n_beams, self.max_echoes, 8), dtype=torch.int32, device=device)
        counts = torch.empty((self.n_beams,), dtype=torch.int32, device=device)
        return wave, echoes, counts

    def simulate(self, geom, planes, pose=None, outputs=None, stream=None):
        """planes: 7 CUDA tensors [V, U] float32. Returns (waveforms, echoes, counts)
        as torch tensors; echoes is int32 [n_beams, max_echoes, 8] holding
        lidar_echo_t records (view with ECHO_DTYPE after .cpu().numpy())."""
        import torch
        if outputs is None:
            outputs = self.alloc_outputs(planes[0].device)
        wave, echoes, counts = outputs
        for p in planes:
            assert p.is_cuda and p.dtype == torch.float32 and p.is_contiguous()
        g = make_gbuffer(geom, [p.data_ptr() for p in planes])
        s = (stream or torch.cuda.current_stream()).cuda_stream
        lidar_simulate(self.handle, g, make_pose(np.eye(3) if pose is None else pose), wave.data_ptr(),
                       echoes.data_ptr(), counts.data_ptr(), s)
        return wave, echoes, counts

    def simulate_echoes(self, geom, planes, pose=None, outputs=None, stream=None):
        """Echo-only form (lidar_simulate_echoes): returns (echoes, counts)."""
        import torch
        echoes, counts = outputs if outputs is not None else self._alloc_echoes(planes[0].device)
        g = make_gbuffer(geom, [p.data_ptr() for p in planes])
        s = (stream or torch.cuda.current_stream()).cuda_stream
        lidar_simulate_echoes(self.handle, g, make_pose(np.eye(3) if pose is None else pose), echoes.data_ptr(),
                              counts.data_ptr(), s)
        return echoes, counts

    def _alloc_echoes(self, device):
        import torch
        return (torch.empty((self.n_beams, self.max_echoes, 8), dtype=torch.int32, device=device),
                torch.empty((self.n_beams,), dtype=torch.int32, device=device))

    def simulate_host(self, geom, host_planes, pose=None, outputs=None, stream=None, echo_only=False):
        """Host-memory entry point: planes and outputs are (pinned) CPU tensors.
        echo_only: no waveforms (outputs = (None, echoes, counts) or allocated)."""
        import torch
        if outputs is None:
            outputs = (None if echo_only else
                       torch.empty((self.n_beams, self.n_bins), dtype=torch.float32, pin_memory=True),
                       torch.empty((self.n_beams, self.max_echoes, 8), dtype=torch.int32, pin_memory=True),
                       torch.empty((self.n_beams,), dtype=torch.int32, pin_memory=True))
        wave, echoes, counts = outputs
        g = make_gbuffer(geom, [p.data_ptr() for p in host_planes])
        s = (stream or torch.cuda.current_stream()).cuda_stream
        lidar_simulate_host(self.handle, g, make_pose(np.eye(3) if pose is None else pose),
                            wave.data_ptr() if wave is not None else None, echoes.data_ptr(), counts.data_ptr(), s)
        return wave, echoes, counts

    def simulate_host_frames(self, geoms, host_planes, poses=None, outputs=None, stream=None, echo_only=False):
        """A sequence of frames from host memory (lidar_simulate_host_frames):
        geoms[f], host_planes[f] (pinned CPU tensors) and poses[f] describe frame
        f; outputs[f] = (waveforms or None, echoes, counts) receives its results.
        Consecutive frames must not share output tensors."""
        import torch
        n = len(geoms)
        poses = [np.eye(3)] * n if poses is None else poses
        if outputs is None:
            outputs = [(None if echo_only else
                        torch.empty((self.n_beams, self.n_bins), dtype=torch.float32, pin_memory=True),
                        torch.empty((self.n_beams, self.max_echoes, 8), dtype=torch.int32, pin_memory=True),
                        torch.empty((self.n_beams,), dtype=torch.int32, pin_memory=True)) for _ in range(n)]
        gs = [make_gbuffer(geom, [p.data_ptr() for p in planes]) for geom, planes in zip(geoms, host_planes)]
        ps = [make_pose(p) for p in poses]
        s = (stream or torch.cuda.current_stream()).cuda_stream
        lidar_simulate_host_frames(self.handle, gs, ps, None if echo_only else [o[0].data_ptr() for o in outputs],
                                   [o[1].data_ptr() for o in outputs], [o[2].data_ptr() for o in outputs], s)
        return outputs

    def close(self):
        if self.handle:
            lidar_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def echoes_numpy(echoes_tensor) -> np.ndarray:
    a = echoes_tensor.detach().cpu().numpy()
    return np.ascontiguousarray(a).view(ECHO_DTYPE).reshape(a.shape[:-1])
