"""Python side of the FP64 CPU oracle (ctypes over ``lidar_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use this module to state what the beam model computes. It
shares no code with the CUDA library and never imports it.

Inputs are the same float32 arrays the GPU path receives (G-buffer planes,
beam directions, pose, profile table), promoted to float64 inside the C code.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lidar_oracle.c")
LIB = os.path.join(HERE, "liblidar_oracle.so")

CLIPPED_START, CLIPPED_END, NEAR_THRESHOLD, PEAK_AMBIGUOUS = 1, 2, 4, 8
C_LIGHT = 299_792_458.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE arithmetic)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


class _Profile(C.Structure):
    _fields_ = [("kind", C.c_int32), ("sigma_deg", C.c_double), ("tail_amp", C.c_double),
                ("tail_core_deg", C.c_double), ("tail_pow", C.c_double), ("trunc_deg", C.c_double),
                ("tw", C.c_int32), ("th", C.c_int32), ("pitch_deg", C.c_double),
                ("table", C.POINTER(C.c_float))]


class _GBuffer(C.Structure):
    _fields_ = [("U", C.c_int32), ("V", C.c_int32), ("az0", C.c_double), ("el0", C.c_double),
                ("daz", C.c_double), ("dele", C.c_double)] + [
        (n, C.POINTER(C.c_float)) for n in ("range", "nx", "ny", "nz", "rho", "retro", "amb")]


class _Pulse(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("dt", C.c_double), ("t0", C.c_double),
                ("fwhm", C.c_double), ("trunc_sigmas", C.c_double)]


class _Calib(C.Structure):
    _fields_ = [("T", C.c_double), ("s_amb", C.c_double), ("c0", C.c_double), ("c1", C.c_double),
                ("c2", C.c_double)]


class _Echo(C.Structure):
    _fields_ = [("range_m", C.c_double), ("epw_m", C.c_double), ("intensity", C.c_double),
                ("peak", C.c_double), ("r0", C.c_double), ("r1", C.c_double), ("x_peak", C.c_double),
                ("bin_peak", C.c_int32), ("bin_start", C.c_int32), ("bin_end", C.c_int32),
                ("flags", C.c_uint32)]


ECHO_DTYPE = np.dtype([("range_m", "f8"), ("epw_m", "f8"), ("intensity", "f8"), ("peak", "f8"),
                       ("r0", "f8"), ("r1", "f8"), ("x_peak", "f8"), ("bin_peak", "i4"),
                       ("bin_start", "i4"), ("bin_end", "i4"), ("flags", "u4")])
assert ECHO_DTYPE.itemsize == C.sizeof(_Echo)

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, p = C.c_double, C.c_int, C.c_void_p
        _lib.orc_profile_raw.restype = d
        _lib.orc_profile_raw.argtypes = [C.POINTER(_Profile), d, d]
        _lib.orc_profile_norm.restype = d
        _lib.orc_profile_norm.argtypes = [C.POINTER(_Profile)]
        _lib.orc_profile_support_deg.restype = d
        _lib.orc_profile_support_deg.argtypes = [C.POINTER(_Profile)]
        _lib.orc_deposit_weight.restype = d
        _lib.orc_deposit_weight.argtypes = [d, d, i]
        _lib.orc_pulse_taps.restype = i
        _lib.orc_pulse_taps.argtypes = [C.POINTER(_Pulse), p, i]
        _lib.orc_convolve.restype = None
        _lib.orc_convolve.argtypes = [p, i, p, i, d, p]
        _lib.orc_extract_echoes.restype = i
        _lib.orc_extract_echoes.argtypes = [p, i, C.POINTER(_Pulse), C.POINTER(_Calib), p, i]
        _lib.orc_fit_epw.restype = i
        _lib.orc_fit_epw.argtypes = [C.POINTER(_Pulse), d, p]
        _lib.orc_simulate.restype = i
        _lib.orc_simulate.argtypes = [C.POINTER(_GBuffer), C.POINTER(_Profile), d, p, p, p, i,
                                      C.POINTER(_Pulse), C.POINTER(_Calib), i, p, p, p, p, p, i]
        _lib.orc_pixels.restype = None
        _lib.orc_pixels.argtypes = [C.POINTER(_GBuffer), p, p, p, p, p]
        _lib.orc_offsets.restype = None
        _lib.orc_offsets.argtypes = [p, p, p, i, p, p, p]
        _lib.orc_stack_inputs.argtypes = [C.POINTER(_GBuffer), d, p, p]
        _lib.orc_range_stack.argtypes = [i, i, p, p, i, i, p, d, i, p, p]
        _lib.orc_range_stack_at.restype = None
        _lib.orc_range_stack_at.argtypes = [i, i, p, p, i, i, p, d, i, i, p, p, p, p, p]
        _lib.orc_pixel.restype = i
    return _lib


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _profile(prof, keep):
    s = _Profile()
    s.kind = int(prof["kind"])
    if s.kind == 0:
        for k in ("sigma_deg", "tail_amp", "tail_core_deg", "tail_pow", "trunc_deg"):
            setattr(s, k, float(prof[k]))
    elif s.kind == 2:
        h = np.ascontiguousarray(prof["h"], dtype=np.float32)
        v = np.ascontiguousarray(prof["v"], dtype=np.float32)
        t = np.ascontiguousarray(np.concatenate([h, v]), dtype=np.float32)
        keep.append(t)
        s.tw, s.th = len(h), len(v)
        s.pitch_deg = float(prof["pitch_deg"])
        s.table = _fptr(t)
    else:
        t = np.ascontiguousarray(prof["table"], dtype=np.float32)
        keep.append(t)
        s.tw, s.th = t.shape[1], t.shape[0]
        s.pitch_deg = float(prof["pitch_deg"])
        s.table = _fptr(t)
    return s


def _gbuffer(gb, keep):
    s = _GBuffer()
    s.U, s.V = int(gb.U), int(gb.V)
    s.az0, s.el0, s.daz, s.dele = float(gb.az0), float(gb.el0), float(gb.daz), float(gb.dele)
    for name, arr in zip(("range", "nx", "ny", "nz", "rho", "retro", "amb"), gb.planes()):
        a = np.ascontiguousarray(arr, dtype=np.float32)
        keep.append(a)
        setattr(s, name, _fptr(a))
    return s


def _pulse(pu):
    return _Pulse(int(pu["n_bins"]), float(pu["dt_s"]), float(pu["t0_s"]), float(pu["fwhm_s"]),
                  float(pu["trunc_sigmas"]))


def calib_coef(pu, cal):
    """EPW->intensity coefficients: fitted (Sec. II-C) or as given."""
    if cal.get("fit_epw", 0):
        return fit_epw(pu, cal["threshold"])
    return np.asarray(cal["epw_coef"], np.float64)


def _calib(pu, cal):
    c = calib_coef(pu, cal)
    return _Calib(float(cal["threshold"]), float(cal["ambient_scale"]), float(c[0]), float(c[1]),
                  float(c[2]))


# --------------------------------------------------------------------------
# thin wrappers
# --------------------------------------------------------------------------


def profile_raw(prof, u, v):
    keep = []
    s = _profile(prof, keep)
    u = np.atleast_1d(np.asarray(u, np.float64))
    v = np.broadcast_to(np.asarray(v, np.float64), u.shape)
    return np.array([lib().orc_profile_raw(C.byref(s), float(a), float(b)) for a, b in zip(u.ravel(), v.ravel())]
                    ).reshape(u.shape)


def profile_norm(prof) -> float:
    keep = []
    return lib().orc_profile_norm(C.byref(_profile(prof, keep)))


def profile_support_deg(prof) -> float:
    keep = []
    return lib().orc_profile_support_deg(C.byref(_profile(prof, keep)))


def deposit_weight(X0, X1, k) -> float:
    return lib().orc_deposit_weight(float(X0), float(X1), int(k))


def pulse_taps(pu) -> np.ndarray:
    buf = np.zeros(16384, np.float64)
    M = lib().orc_pulse_taps(C.byref(_pulse(pu)), buf.ctypes.data, 16384)
    assert M >= 0
    return buf[: 2 * M + 1].copy()


def convolve(h, taps, amb_level=0.0):
    h = np.ascontiguousarray(h, np.float64)
    taps = np.ascontiguousarray(taps, np.float64)
    out = np.zeros_like(h)
    lib().orc_convolve(h.ctypes.data, len(h), taps.ctypes.data, (len(taps) - 1) // 2, float(amb_level),
                       out.ctypes.data)
    return out


def extract_echoes(xi, pu, threshold, coef=(0.0, 0.0, 0.0), max_out=64):
    xi = np.ascontiguousarray(xi, np.float64)
    out = np.zeros(max_out, ECHO_DTYPE)
    cal = _Calib(float(threshold), 0.0, float(coef[0]), float(coef[1]), float(coef[2]))
    n = lib().orc_extract_echoes(xi.ctypes.data, len(xi), C.byref(_pulse(pu)), C.byref(cal),
                                 out.ctypes.data, max_out)
    return out[:n]


def strongest_echo(echoes):
    """The single-return selection (LIDAR_ECHOES_STRONGEST): of all echoes of a
    waveform (extract_echoes, nearest first), the one of largest intensity,
    the nearest of equal ones; empty if there is none."""
    if len(echoes) == 0:
        return echoes[:0]
    k = int(np.argmax(echoes["intensity"]))  # first maximum: the nearest on ties
    return echoes[k:k + 1]


def fit_epw(pu, threshold) -> np.ndarray:
    coef = np.zeros(3, np.float64)
    used = lib().orc_fit_epw(C.byref(_pulse(pu)), float(threshold), coef.ctypes.data)
    assert used > 16
    return coef


def pixels(gb):
    keep = []
    s = _gbuffer(gb, keep)
    n = gb.U * gb.V
    w, t0, t1, a = (np.zeros(n) for _ in range(4))
    hit = np.zeros(n, np.int32)
    lib().orc_pixels(C.byref(s), w.ctypes.data, t0.ctypes.data, t1.ctypes.data, a.ctypes.data,
                     hit.ctypes.data)
    sh = (gb.V, gb.U)
    return dict(w=w.reshape(sh), t0=t0.reshape(sh), t1=t1.reshape(sh), a=a.reshape(sh),
                hit=hit.reshape(sh).astype(bool))


def offsets(R, beam_dir, dirs3):
    R = np.ascontiguousarray(R, np.float32).ravel()
    bd = np.ascontiguousarray(beam_dir, np.float32).ravel()
    d = np.ascontiguousarray(dirs3, np.float64).reshape(-1, 3)
    n = len(d)
    u, v = np.zeros(n), np.zeros(n)
    front = np.zeros(n, np.int32)
    lib().orc_offsets(R.ctypes.data, bd.ctypes.data, d.ctypes.data, n, u.ctypes.data, v.ctypes.data,
                      front.ctypes.data)
    return u, v, front.astype(bool)


def simulate(gb, dirs, profile, pu, cal, pose=None, beams=None, nthreads=1, max_out=16, Z=None):
    """Run the oracle on the selected beams. Returns a dict with h (histogram
    before the pulse), amb (ambient sum A_b), xi (waveform), echoes
    ([n_sel, max_out] structured, all runs nearest first) and counts."""
    keep = []
    g = _gbuffer(gb, keep)
    p = _profile(profile, keep)
    if Z is None:
        Z = lib().orc_profile_norm(C.byref(p))
    R = np.ascontiguousarray(np.eye(3) if pose is None else pose, np.float32).ravel()
    dirs = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
    if beams is None:
        beams = np.arange(len(dirs), dtype=np.int32)
    beams = np.ascontiguousarray(beams, np.int32)
    ns, nb = len(beams), int(pu["n_bins"])
    h = np.zeros((ns, nb))
    xi = np.zeros((ns, nb))
    amb = np.zeros(ns)
    ech = np.zeros((ns, max_out), ECHO_DTYPE)
    cnt = np.zeros(ns, np.int32)
    pul = _pulse(pu)
    ca = _calib(pu, cal)
    rc = lib().orc_simulate(C.byref(g), C.byref(p), float(Z), R.ctypes.data, dirs.ctypes.data,
                            beams.ctypes.data, ns, C.byref(pul), C.byref(ca), int(nthreads),
                            h.ctypes.data, amb.ctypes.data, xi.ctypes.data, ech.ctypes.data,
                            cnt.ctypes.data, int(max_out))
    assert rc == 0
    return dict(h=h, amb=amb, xi=xi, echoes=ech, counts=cnt, Z=Z,
                coef=np.array([ca.c0, ca.c1, ca.c2]))


def simulate_workload(wl, beams=None, nthreads=1, max_out=16):
    return simulate(wl.gbuffer, wl.dirs, wl.profile, wl.pulse, wl.calib, wl.pose, beams, nthreads,
                    max_out)


def stack_inputs(gb, dr):
    """Per-pixel intensity and range index of Alg. 2 (range stacking)."""
    keep = []
    g = _gbuffer(gb, keep)
    I = np.zeros((gb.V, gb.U))
    rbar = np.zeros((gb.V, gb.U), np.int32)
    lib().orc_stack_inputs(C.byref(g), float(dr), I.ctypes.data, rbar.ctypes.data)
    return I, rbar


def range_stack_at(I, rbar, kernel, threshold, s_max, v, u):
    """Alg. 2 at the output pixels (v[q], u[q]) only: the values range_stack
    gives there, plus how near each decision came to flipping (min over the
    slices up to the answer of |sum - threshold| / threshold)."""
    I = np.ascontiguousarray(I, np.float64)
    rbar = np.ascontiguousarray(rbar, np.int32)
    K = np.ascontiguousarray(kernel, np.float64)
    v = np.ascontiguousarray(v, np.int32)
    u = np.ascontiguousarray(u, np.int32)
    V, U = I.shape
    n = len(v)
    S = np.zeros(n, np.int32)
    X = np.zeros(n)
    close = np.zeros(n)
    lib().orc_range_stack_at(U, V, I.ctypes.data, rbar.ctypes.data, K.shape[0], K.shape[1], K.ctypes.data,
                             float(threshold), int(s_max), n, v.ctypes.data, u.ctypes.data, S.ctypes.data,
                             X.ctypes.data, close.ctypes.data)
    return S, X, close


def range_stack(I, rbar, kernel, threshold, s_max):
    """Alg. 2: nearest slice index and intensity per pixel (FP64)."""
    I = np.ascontiguousarray(I, np.float64)
    rbar = np.ascontiguousarray(rbar, np.int32)
    K = np.ascontiguousarray(kernel, np.float64)
    V, U = I.shape
    S = np.zeros((V, U), np.int32)
    X = np.zeros((V, U))
    lib().orc_range_stack(U, V, I.ctypes.data, rbar.ctypes.data, K.shape[0], K.shape[1], K.ctypes.data,
                          float(threshold), int(s_max), S.ctypes.data, X.ctypes.data)
    return S, X
