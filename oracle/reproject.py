"""FP64 statement of the reprojection of a pinhole G-buffer onto the spherical
grid of the beam model (lidar_reproject_pinhole).

TEST INFRASTRUCTURE ONLY: the GPU tests compare the library's reprojection
kernel against this function. It shares no code with the CUDA library.

What it computes (Sec. II-C: pinhole renderings can be used through a
reprojection of the rendered images; Sec. II-D: a pixel's range is
extrapolated to another direction along the surface with the normal,
r_corr = (p . n) / (v . n) r, instead of interpolating ranges between pixels):
for every target pixel with centre direction v,
  1. v in camera coordinates: c = R^T v; no source if c_z <= 0;
  2. its image point (px, py) = (cx + fx c_x / c_z, cy + fy c_y / c_z); the
     source pixel is the cell (floor(px), floor(py)), none outside the image;
  3. normal, reflectance, retro gain and ambient radiance are the source's;
  4. the source range r is measured along the source's centre direction p
     (z depth times |(X, Y, 1)| if the source holds z depth); the target range
     is (p . n) / (v . n) r, or r where |v . n| < 1e-3 or v . n and p . n
     differ in sign; a source without a hit keeps its range.
Pixels without a source: range +inf, everything else 0.
"""
from __future__ import annotations

import numpy as np

from paper_2512_05932_gb300.scenes import GBuffer


def target_dirs(grid):
    """Unit directions of the target pixel centres, [V, U, 3]."""
    az = grid.az0 + (np.arange(grid.U) + 0.5) * grid.daz
    el = grid.el0 + (np.arange(grid.V) + 0.5) * grid.dele
    ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
    ca, sa = np.cos(az)[None, :], np.sin(az)[None, :]
    return np.stack([ce * ca, ce * sa, np.broadcast_to(se, (grid.V, grid.U))], axis=-1)


def image_points(ph, grid):
    """Image coordinates (px, py) of every target direction and whether it lies
    in front of the camera."""
    R = np.asarray(ph.R, np.float64).reshape(3, 3)
    c = target_dirs(grid) @ R  # c_k = sum_r v_r R[r][k]
    front = c[..., 2] > 0
    cz = np.where(front, c[..., 2], 1.0)
    return ph.cx + ph.fx * c[..., 0] / cz, ph.cy + ph.fy * c[..., 1] / cz, front


def reproject_pinhole(ph, grid):
    """Returns (GBuffer on the target grid, boundary distance): the latter is
    the distance (pixels) of each target's image point from the nearest cell
    edge, for callers that must treat near-ties of the cell choice apart."""
    U, V = grid.U, grid.V
    v = target_dirs(grid)
    px, py, front = image_points(ph, grid)
    fi, fj = np.floor(px), np.floor(py)
    ok = front & (fi >= 0) & (fi < ph.W) & (fj >= 0) & (fj < ph.H)
    i = np.where(ok, fi, 0).astype(np.int64)
    j = np.where(ok, fj, 0).astype(np.int64)
    src = {k: np.asarray(getattr(ph, k), np.float64)[j, i] for k in GBuffer.PLANES}
    n = np.stack([src["nx"], src["ny"], src["nz"]], axis=-1)
    R = np.asarray(ph.R, np.float64).reshape(3, 3)
    X = (i + 0.5 - ph.cx) / ph.fx
    Y = (j + 0.5 - ph.cy) / ph.fy
    norm = np.sqrt(X * X + Y * Y + 1.0)
    p = np.stack([X, Y, np.ones_like(X)], axis=-1) @ R.T / norm[..., None]
    r = src["range"]
    hit = np.isfinite(r) & (r > 0)
    rp = np.where(hit, r * norm if ph.depth_is_z else r, r)
    pn = (p * n).sum(-1)
    vn = (v * n).sum(-1)
    use = hit & (np.abs(vn) >= 1e-3) & (vn * pn > 0)
    with np.errstate(invalid="ignore", divide="ignore"):  # rays without a hit are masked
        rc = np.where(use, pn / np.where(use, vn, 1.0) * rp, rp)
    out = {"range": np.where(ok, rc, np.inf)}
    for k in ("nx", "ny", "nz", "rho_d", "retro", "ambient"):
        out[k] = np.where(ok, src[k], 0.0)
    gb = GBuffer(U, V, grid.az0, grid.el0, grid.daz, grid.dele,
                 *[np.ascontiguousarray(out[k], dtype=np.float32) for k in GBuffer.PLANES])
    edge = np.minimum(np.minimum(px - fi, fi + 1 - px), np.minimum(py - fj, fj + 1 - py))
    return gb, np.where(front, edge, np.inf)
