"""Pinhole G-buffer input (lidar_reproject_pinhole) against the FP64 oracle
(oracle/reproject.py), alone and followed by the beam model.

Bar: the chosen source cell bit-exact (materials equal) except for target
rays whose image point lies within 1e-6 pixel of a cell edge; ranges within
1e-6 relative (both compute the geometry in FP64); the simulated waveforms and
echoes meet the parity bar of tests/test_parity_gpu.py."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle import reproject as RP
from paper_2512_05932_gb300 import lidar
from paper_2512_05932_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEG = math.pi / 180
NTHREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def gpu_reproject(ph, grid):
    src = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in ph.planes()]
    dst = [torch.full((grid.V, grid.U), float("nan"), dtype=torch.float32, device="cuda") for _ in range(7)]
    lidar.lidar_reproject_pinhole(lidar.make_pinhole(ph, [p.data_ptr() for p in src]),
                                  lidar.make_gbuffer(grid, [p.data_ptr() for p in dst]),
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return dst, [p.cpu().numpy() for p in dst]


def box_scene_pinhole():
    g = S.rng(21)
    rects = [S.Plane(np.array([0.0, 0.0, 1.0]), -2.0, 0.2, 0.0)]
    boxes = []
    for _ in range(6):
        c = np.array([g.uniform(6, 20), g.uniform(-5, 5), g.uniform(-1.5, 0.5)])
        retro = [100.0 if g.uniform() < 0.3 else 0.0 for _ in range(6)]
        boxes += S.box_rects(c, g.uniform(0.4, 1.5, size=3), g.uniform(0, math.pi), g.uniform(0.05, 0.9), retro)
    scene = S.Scene(planes=rects, rects=boxes, ambient="sun", ambient_level=1e3)
    R = S.camera_looking_along(2 * DEG, -4 * DEG)
    ph = S.raycast_pinhole(scene, 256, 192, 400.0, 400.0, 128.0, 96.0, R)
    pitch = 0.1 * DEG
    grid = S.GBuffer(440, 300, 2 * DEG - 220 * pitch, -4 * DEG - 150 * pitch, pitch, pitch, *[None] * 7)
    return ph, grid


def assert_planes_match(ph, grid):
    _, got = gpu_reproject(ph, grid)
    ref, edge = RP.reproject_pinhole(ph, grid)
    sure = edge > 1e-6
    for k, g in zip(S.GBuffer.PLANES, got):
        r = getattr(ref, k)
        if k == "range":
            fin = sure & np.isfinite(r)
            np.testing.assert_allclose(g[fin], r[fin], rtol=1e-6)
            assert (np.isinf(g[sure & ~np.isfinite(r)])).all()
        else:
            np.testing.assert_array_equal(g[sure], r[sure], err_msg=k)
    return ref, sure


@pytest.mark.parametrize("depth_is_z", [False, True])
def test_reprojection_plane_retro(depth_is_z):
    ph, grid = S.pinhole_plane_retro(depth_is_z=depth_is_z)
    ref, sure = assert_planes_match(ph, grid)
    assert (ref.retro > 0).sum() > 1000


def test_reprojection_boxes_wide_angle_partial_cover():
    ph, grid = box_scene_pinhole()
    ref, sure = assert_planes_match(ph, grid)
    assert np.isinf(ref.range).any() and np.isfinite(ref.range).mean() > 0.3


def test_reprojected_frame_meets_parity():
    """Pinhole rendering -> reprojection -> beam model on the GPU against the
    same chain in the oracle."""
    from tests.test_parity_gpu import ambiguous_ok, compare
    ph, grid = S.pinhole_plane_retro()
    planes, _ = gpu_reproject(ph, grid)
    ref_gb, _ = RP.reproject_pinhole(ph, grid)
    dirs = S.grid_pattern(24, 16, 7.0 * DEG, 4.8 * DEG, az_c=0.5 * DEG, el_c=0.2 * DEG)
    w = S.Workload("pinhole_plane_retro", ref_gb, dirs, S.radial_profile(), S.pulse(1024, 0.1e-9),
                   S.calib(1e-5, 1e-4, 3, True))
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    wave, ech, cnt = L.simulate(grid, planes, w.pose)
    torch.cuda.synchronize()
    lidar.lidar_sync(L.handle, 0)
    beams = np.arange(len(dirs), dtype=np.int32)
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    st = compare(ref, wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech), cnt.cpu().numpy(), beams,
                 w.calib["threshold"], w.calib["max_echoes"], w.pulse)
    assert st["echoes"] >= 300 and ambiguous_ok(st), st
    L.close()


def test_reprojection_rejects_bad_arguments():
    ph, grid = S.pinhole_plane_retro(W=8, H=6, f=50.0)
    src = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in ph.planes()]
    dst = [torch.empty((grid.V, grid.U), dtype=torch.float32, device="cuda") for _ in range(7)]
    s = lidar.make_pinhole(ph, [p.data_ptr() for p in src])
    s.R[0] = 2.0
    with pytest.raises(lidar.LidarError, match="orthonormal"):
        lidar.lidar_reproject_pinhole(s, lidar.make_gbuffer(grid, [p.data_ptr() for p in dst]))
    s = lidar.make_pinhole(ph, [p.data_ptr() for p in src])
    s.fx = 0.0
    with pytest.raises(lidar.LidarError, match="fx"):
        lidar.lidar_reproject_pinhole(s, lidar.make_gbuffer(grid, [p.data_ptr() for p in dst]))
    s = lidar.make_pinhole(ph, [p.data_ptr() for p in src])
    with pytest.raises(lidar.LidarError, match="target plane"):
        lidar.lidar_reproject_pinhole(s, lidar.make_gbuffer(grid, [0] * 7))


def test_bench_frame_reprojection_every_pixel():
    """The benchmark's pinhole frame (2048x1024 rendering of the boxes scene,
    60 deg field of view) onto its 2048x1024 grid: every target pixel against
    the FP64 reprojection."""
    ph, grid, _ = S.pinhole_boxes_frame()
    ref, sure = assert_planes_match(ph, grid)
    assert sure.mean() > 0.999 and np.isfinite(ref.range).mean() > 0.5
