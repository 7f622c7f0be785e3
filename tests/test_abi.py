"""CPU-side checks of the C ABI: the library loads, exports every function
declared in include/lidar.h, and rejects invalid arguments before touching
the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2512_05932_gb300 import build as B
from paper_2512_05932_gb300 import lidar, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lidar.load()


def declared_functions(header=None):
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h") or (header and h != header):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(lidar_[a-z_]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_binding_symbols():
    assert declared_functions("lidar.h") == sorted(lidar.SYMBOLS)
    assert declared_functions("lidar_tail.h") == sorted(lidar.TAIL_SYMBOLS)
    assert declared_functions("lidar_stack.h") == sorted(lidar.STACK_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_sizes_match_header(lib):
    # sizes of the ABI structs as laid out by the C compiler
    assert C.sizeof(lidar.lidar_echo_t) == 32
    assert C.sizeof(lidar.lidar_pose_t) == 36
    assert C.sizeof(lidar.lidar_echoes_t) == 16


def _args():
    w = scenes.tiny_case()
    return w.profile, w.dirs, w.pulse, w.calib


@pytest.mark.parametrize("mutate,match", [
    (lambda p, d, pu, c: pu.update(n_bins=100), "multiple of 32"),
    (lambda p, d, pu, c: pu.update(n_bins=0), "multiple of 32"),
    (lambda p, d, pu, c: pu.update(dt_s=0.0), "dt_s"),
    (lambda p, d, pu, c: pu.update(fwhm_s=-1.0), "fwhm_s"),
    (lambda p, d, pu, c: c.update(max_echoes=4), "max_echoes"),
    (lambda p, d, pu, c: c.update(threshold=0.0), "threshold"),
    (lambda p, d, pu, c: p.update(trunc_deg=20.0), "trunc_deg"),
    (lambda p, d, pu, c: p.update(sigma_deg=float("nan")), "sigma_deg"),
    (lambda p, d, pu, c: d.__setitem__(slice(0, 1), 0.0), "dirs"),
])
def test_create_rejects_invalid(lib, mutate, match):
    p, d, pu, c = _args()
    p, d, pu, c = dict(p), d.copy(), dict(pu), dict(c)
    mutate(p, d, pu, c)
    with pytest.raises(lidar.LidarError, match=match) as ei:
        lidar.lidar_create(p, d, pu, c)
    assert ei.value.status == lidar.LIDAR_EINVAL


def test_create_rejects_bad_table(lib):
    p, d, pu, c = _args()
    t = np.ones((5, 5), np.float32)
    t[2, 2] = -1
    with pytest.raises(lidar.LidarError, match="negative"):
        lidar.lidar_create(scenes.table_profile(t, 0.1), d, pu, c)
    with pytest.raises(lidar.LidarError, match="10 degrees"):
        lidar.lidar_create(scenes.table_profile(np.ones((5, 5), np.float32), 5.0), d, pu, c)


def test_empty_pattern_rejected(lib):
    p, d, pu, c = _args()
    with pytest.raises(lidar.LidarError, match="n_beams"):
        lidar.lidar_create(p, np.zeros((0, 3), np.float32), pu, c)


def test_simulate_rejects_null_handle(lib):
    g = lidar.lidar_gbuffer_t()
    with pytest.raises(lidar.LidarError):
        lidar.lidar_simulate(None, g, lidar.make_pose(np.eye(3)), 0, 0, 0, 0)


def test_no_fallback_when_library_missing(tmp_path):
    saved = lidar._lib
    lidar._lib = None
    try:
        with pytest.raises(RuntimeError, match="missing"):
            lidar.load(str(tmp_path / "nope.so"))
    finally:
        lidar._lib = saved


def test_new_entry_points_reject_null(lib):
    with pytest.raises(lidar.LidarError):
        lidar.lidar_set_deposit(None, 1)
    with pytest.raises(lidar.LidarError):
        lidar.lidar_batch_config(None)
    arr = lidar.make_frames([])
    with pytest.raises(lidar.LidarError):
        lidar.lidar_simulate_batch(None, arr, 0)
    g = lidar.lidar_gbuffer_t()
    with pytest.raises(lidar.LidarError):
        lidar.lidar_simulate_noalloc(None, g, lidar.make_pose(np.eye(3)), 0, 0, 0, 0)
    with pytest.raises(lidar.LidarError):
        lidar.lidar_simulate_echoes(None, g, lidar.make_pose(np.eye(3)), 0, 0, 0)


def test_host_frames_rejects_null_handle_and_mismatched_lists(lib):
    """The frame-sequence call: a NULL handle is rejected by the library before
    any CUDA call; per-frame lists of different lengths are rejected by the
    binding before the library is called."""
    g, pose = lidar.lidar_gbuffer_t(), lidar.make_pose(np.eye(3))
    with pytest.raises(lidar.LidarError):
        lidar.lidar_simulate_host_frames(None, [g], [pose], None, [0], [0], 0)
    with pytest.raises(lidar.LidarError):
        lidar.lidar_simulate_host(None, g, pose, 0, 0, 0, 0)
    with pytest.raises(ValueError):
        lidar.lidar_simulate_host_frames(None, [g, g], [pose], None, [0, 0], [0, 0], 0)
    with pytest.raises(ValueError):
        lidar.lidar_simulate_host_frames(None, [g], [pose], [0, 0], [0], [0], 0)


def test_frame_struct_layout(lib):
    # lidar_frame_t: sensor pointer, gbuffer, pose, waveforms pointer, echoes
    assert C.sizeof(lidar.lidar_frame_t) == 8 + C.sizeof(lidar.lidar_gbuffer_t) + 36 + 4 + 8 + 16


@pytest.mark.parametrize("kh,kw,thr,dr,rmax,match", [
    (4, 5, 1.0, 0.1, 10.0, "odd"),
    (131, 5, 1.0, 0.1, 10.0, "odd"),
    (3, 3, 0.0, 0.1, 10.0, "threshold"),
    (3, 3, 1.0, -0.1, 10.0, "dr"),
    (3, 3, 1.0, 0.1, 0.05, "r_max / dr"),
    (3, 3, 1.0, 1e-6, 1.0, "r_max / dr"),
])
def test_range_stack_rejects_bad_parameters(lib, kh, kw, thr, dr, rmax, match):
    with pytest.raises(lidar.LidarError, match=match):
        lidar.RangeStack(np.ones((kh, kw), np.float32), thr, dr, rmax)


def test_range_stack_rejects_negative_kernel(lib):
    k = np.ones((3, 3), np.float32)
    k[1, 1] = -1
    with pytest.raises(lidar.LidarError, match="negative"):
        lidar.RangeStack(k, 1.0, 0.1, 10.0)
