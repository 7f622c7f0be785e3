"""Pins of the FP64 reprojection statement (oracle/reproject.py) to things
other than itself: the exact range of a plane along every target ray, z-depth
input, the cell choice against a brute-force search, and agreement with a
direct spherical rendering of the same scene."""
import math

import numpy as np

from oracle import reproject as RP
from paper_2512_05932_gb300 import scenes as S

DEG = math.pi / 180


def tilted_plane_scene():
    n = np.array([-0.8, 0.36, 0.48])
    n = n / np.linalg.norm(n)
    return S.Scene(planes=[S.Plane(n, -9.0, 0.4, 0.0)], ambient="uniform", ambient_level=0.02), n, -9.0


def small_setup(depth_is_z=False, W=64, H=48, f=500.0):
    scene, n, d = tilted_plane_scene()
    R = S.camera_looking_along(3 * DEG, -2 * DEG)
    ph = S.raycast_pinhole(scene, W, H, f, f, W / 2 + 0.3, H / 2 - 0.2, R, depth_is_z)
    pitch = 0.05 * DEG
    grid = S.GBuffer(90, 60, 3 * DEG - 45 * pitch, -2 * DEG - 30 * pitch, pitch, pitch, *[None] * 7)
    return ph, grid, n, d


def test_plane_range_is_exact_along_every_target_ray():
    # r_corr = (p.n)/(v.n) r_p = d/(v.n) for a plane {x : x.n = d}: the
    # reprojected range is the true distance along the target ray (a swapped
    # ratio or the wrong direction would be off by the angle between them)
    ph, grid, n, d = small_setup()
    gb, _ = RP.reproject_pinhole(ph, grid)
    v = RP.target_dirs(grid)
    exact = d / (v @ n)
    ok = np.isfinite(gb.range)
    assert ok.mean() > 0.5
    np.testing.assert_allclose(gb.range[ok], exact[ok], rtol=2e-7)
    # the uncorrected source range differs by far more than that
    px, py, _ = RP.image_points(ph, grid)
    raw = ph.range[np.clip(np.floor(py).astype(int), 0, ph.H - 1), np.clip(np.floor(px).astype(int), 0, ph.W - 1)]
    assert np.abs(raw[ok] / exact[ok] - 1).max() > 1e-5


def test_z_depth_input_gives_the_same_ranges():
    ph, grid, _, _ = small_setup()
    phz, _, _, _ = small_setup(depth_is_z=True)
    assert not np.allclose(phz.range, ph.range)
    a, _ = RP.reproject_pinhole(ph, grid)
    b, _ = RP.reproject_pinhole(phz, grid)
    ok = np.isfinite(a.range)
    np.testing.assert_allclose(b.range[ok], a.range[ok], rtol=3e-7)


def test_cell_choice_matches_brute_force_nearest_centre():
    # the cell containing an image point is the pixel whose centre is nearest
    # in the max-norm: search every pixel for it
    W, H = 7, 5
    ph = S.PinholeGBuffer(W, H, 40.0, 35.0, 3.3, 2.6, S.camera_looking_along(0.0, 0.0), False,
                          *[np.zeros((H, W), np.float32) for _ in range(7)])
    ph.range[:] = 10.0
    ph.nx[:] = -1.0
    ph.rho_d[:] = np.arange(W * H, dtype=np.float32).reshape(H, W)
    pitch = 0.35 * DEG
    grid = S.GBuffer(31, 23, -15.5 * pitch, -11.5 * pitch, pitch, pitch, *[None] * 7)
    gb, edge = RP.reproject_pinhole(ph, grid)
    px, py, front = RP.image_points(ph, grid)
    cx_, cy_ = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    n_in = 0
    for a in range(grid.V):
        for b in range(grid.U):
            dist = np.maximum(np.abs(px[a, b] - cx_), np.abs(py[a, b] - cy_))
            k = np.unravel_index(np.argmin(dist), dist.shape)
            inside = front[a, b] and dist[k] < 0.5
            if not inside:
                assert gb.range[a, b] == np.inf and gb.rho_d[a, b] == 0
                continue
            if edge[a, b] < 1e-9:
                continue
            n_in += 1
            assert gb.rho_d[a, b] == ph.rho_d[k], (a, b)
    assert n_in > 200


def test_reprojection_agrees_with_direct_spherical_rendering():
    # plane + retro patch seen through the pinhole, reprojected, against the
    # same scene ray-cast directly on the spherical grid: equal ranges on the
    # plane, equal materials except near the patch edges (one source pixel)
    ph, grid = S.pinhole_plane_retro(W=200, H=150, f=1250.0)
    gb, _ = RP.reproject_pinhole(ph, grid)
    g = S.rng(6)
    jit = g.uniform(-1e-3, 1e-3, size=2)
    decal = S.Rect(np.array([10.0, jit[0], jit[1]]), np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]),
                   0.25, 0.25, rho_d=0.5, retro=100.0)
    scene = S.Scene(planes=[S.Plane(np.array([1.0, 0.0, 0.0]), 10.0, 0.5, 0.0, decal)], ambient="uniform",
                    ambient_level=0.01)
    direct = S.raycast(scene, grid.U, grid.V, grid.az0, grid.el0, grid.daz, grid.dele)
    ok = np.isfinite(gb.range)
    assert ok.all()
    np.testing.assert_allclose(gb.range, direct.range, rtol=2e-7)
    same = gb.retro == direct.retro
    assert same.mean() > 0.99
    assert (gb.retro > 0).sum() > 1000
