"""Seeded synthetic inputs: scenes ray-cast into a spherical NIR G-buffer, beam
patterns, tabulated beam profiles and the named workload presets.

This module is the only code shared by the CUDA path and the FP64 oracle. It
plays the part of the renderer of Sec. II (the rasterised or ray-traced image
that the beam model consumes) and of the lab measurements of Sec. III (the
tabulated kappa*eta profile). It holds none of the beam model's arithmetic:
no profile weighting, no radiometry of the return, no range intervals, no
histogramming, no pulse convolution and no echo extraction.

G-buffer convention (equirectangular, sensor frame x forward, y left, z up):
pixel (u, v) with 0 <= u < U (azimuth) and 0 <= v < V (elevation) has its
centre at az = az0 + (u + 1/2) daz, el = el0 + (v + 1/2) del and direction
(cos el cos az, cos el sin az, sin el). Planes are float32 arrays of shape
[V, U] (row v contiguous in u). A pixel without a hit has range +inf.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299_792_458.0  # m/s

# ----------------------------------------------------------------------------
# seeded generator (splitmix64 seeding of numpy's PCG64)
# ----------------------------------------------------------------------------


def _splitmix64(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(_splitmix64(int(seed))))


# ----------------------------------------------------------------------------
# G-buffer container
# ----------------------------------------------------------------------------


@dataclass
class GBuffer:
    U: int
    V: int
    az0: float  # rad, left edge of column 0
    el0: float  # rad, lower edge of row 0
    daz: float  # rad per column
    dele: float  # rad per row
    range: np.ndarray  # [V, U] float32, m (+inf = no hit)
    nx: np.ndarray
    ny: np.ndarray
    nz: np.ndarray
    rho_d: np.ndarray  # NIR diffuse reflectance
    retro: np.ndarray  # retro gain (sr^-1), 0 if none
    ambient: np.ndarray  # ambient radiance, relative units

    PLANES = ("range", "nx", "ny", "nz", "rho_d", "retro", "ambient")

    def planes(self):
        return [getattr(self, p) for p in self.PLANES]

    def pixel_dirs(self) -> np.ndarray:
        """Unit directions of the pixel centres, float64 [V, U, 3]."""
        az = self.az0 + (np.arange(self.U) + 0.5) * self.daz
        el = self.el0 + (np.arange(self.V) + 0.5) * self.dele
        ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
        ca, sa = np.cos(az)[None, :], np.sin(az)[None, :]
        return np.stack([ce * ca, ce * sa, np.broadcast_to(se, (self.V, self.U))], axis=-1)


def _empty_planes(V, U):
    inf = np.full((V, U), np.inf, np.float64)
    z = np.zeros((V, U), np.float64)
    return dict(range=inf, nx=z.copy(), ny=z.copy(), nz=z.copy(), rho_d=z.copy(),
                retro=z.copy(), ambient=z.copy())


# ----------------------------------------------------------------------------
# scene primitives and the analytic ray-caster
# ----------------------------------------------------------------------------


@dataclass
class Rect:
    """Finite planar rectangle: centre c, in-plane unit axes e1, e2, half sizes."""
    c: np.ndarray
    e1: np.ndarray
    e2: np.ndarray
    h1: float
    h2: float
    rho_d: float
    retro: float = 0.0

    @property
    def n(self):
        return np.cross(self.e1, self.e2)


@dataclass
class Plane:
    """Infinite plane {x : x . n = d} with unit normal n."""
    n: np.ndarray
    d: float
    rho_d: float
    retro: float = 0.0
    # optional rectangular decal region (in-plane) with its own material
    decal: Rect | None = None


@dataclass
class Scene:
    planes: list = field(default_factory=list)
    rects: list = field(default_factory=list)
    ambient: str = "uniform"  # "uniform" | "sun" | "none"
    ambient_level: float = 0.0


def _hit_plane(dirs, n, d):
    dn = dirs @ n
    with np.errstate(divide="ignore", invalid="ignore"):
        t = d / dn
    t = np.where((np.abs(dn) > 1e-12) & (t > 0), t, np.inf)
    return t


def raycast(scene: Scene, U, V, az0, el0, daz, dele) -> GBuffer:
    """Nearest-hit ray cast of all primitives through every pixel centre."""
    gb = GBuffer(U, V, az0, el0, daz, dele, *[None] * 7)
    P = _empty_planes(V, U)
    dirs = gb.pixel_dirs()
    az = az0 + (np.arange(U) + 0.5) * daz
    el = el0 + (np.arange(V) + 0.5) * dele

    def commit(sel_v, sel_u, t, n, rho, retro):
        cur = P["range"][sel_v, sel_u]
        better = t < cur
        if not np.any(better):
            return
        for key, val in (("range", t), ("nx", n[..., 0]), ("ny", n[..., 1]), ("nz", n[..., 2]),
                         ("rho_d", rho), ("retro", retro)):
            blk = P[key][sel_v, sel_u]
            blk[better] = np.broadcast_to(val, better.shape)[better]
            P[key][sel_v, sel_u] = blk

    full_v, full_u = slice(0, V), slice(0, U)
    for pl in scene.planes:
        t = _hit_plane(dirs, pl.n, pl.d)
        n = np.broadcast_to(pl.n, dirs.shape)
        rho = np.full(t.shape, pl.rho_d)
        retro = np.full(t.shape, pl.retro)
        if pl.decal is not None:
            q = dirs * t[..., None]
            dq = q - pl.decal.c
            inside = (np.abs(dq @ pl.decal.e1) <= pl.decal.h1) & (np.abs(dq @ pl.decal.e2) <= pl.decal.h2)
            inside &= np.isfinite(t)
            rho = np.where(inside, pl.decal.rho_d, rho)
            retro = np.where(inside, pl.decal.retro, retro)
        commit(full_v, full_u, t, n, rho, retro)

    for r in scene.rects:
        # angular culling by the bounding sphere of the rectangle
        cn = np.linalg.norm(r.c)
        rad = math.hypot(r.h1, r.h2)
        if cn > rad * 1.0001:
            ang = math.asin(min(1.0, rad / cn)) + 2 * max(daz, dele)
            caz = math.atan2(r.c[1], r.c[0])
            cel = math.asin(r.c[2] / cn)
            vlo = max(0, int(math.floor((cel - ang - el0) / dele)))
            vhi = min(V, int(math.ceil((cel + ang - el0) / dele)) + 1)
            ce = max(1e-6, math.cos(min(math.pi / 2 - 1e-6, abs(cel) + ang)))
            aaz = min(math.pi, ang / ce + 2 * daz)
            ulo = max(0, int(math.floor((caz - aaz - az0) / daz)))
            uhi = min(U, int(math.ceil((caz + aaz - az0) / daz)) + 1)
            if vlo >= vhi or ulo >= uhi:
                continue
            sv, su = slice(vlo, vhi), slice(ulo, uhi)
        else:
            sv, su = full_v, full_u
        d = dirs[sv, su]
        n = r.n
        t = _hit_plane(d, n, float(n @ r.c))
        q = d * np.where(np.isfinite(t), t, 0.0)[..., None]
        dq = q - r.c
        inside = (np.abs(dq @ r.e1) <= r.h1) & (np.abs(dq @ r.e2) <= r.h2) & np.isfinite(t)
        t = np.where(inside, t, np.inf)
        commit(sv, su, t, np.broadcast_to(n, d.shape), np.full(t.shape, r.rho_d),
               np.full(t.shape, r.retro))

    hit = np.isfinite(P["range"])
    if scene.ambient == "uniform":
        P["ambient"][:] = scene.ambient_level
    elif scene.ambient == "sun":
        # sun straight overhead: radiance of a Lambertian surface lit from +z
        up = np.maximum(0.0, P["nz"])
        P["ambient"] = np.where(hit, scene.ambient_level * P["rho_d"] / math.pi * up, 0.0)
    for k in ("nx", "ny", "nz", "rho_d", "retro"):
        P[k] = np.where(hit, P[k], 0.0)
    for k in GBuffer.PLANES:
        setattr(gb, k, np.ascontiguousarray(P[k], dtype=np.float32))
    return gb


@dataclass
class PinholeGBuffer:
    """A pinhole rendering (include/lidar.h lidar_pinhole_t): pixel (i, j) looks
    along camera-frame (X, Y, 1), X = (i + 1/2 - cx) / fx, Y = (j + 1/2 - cy) / fy;
    R maps camera-frame vectors to the sensor frame. Planes [H, W] float32 as for
    GBuffer (range along the pixel-centre ray, or z depth if depth_is_z)."""
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray
    depth_is_z: bool
    range: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    nz: np.ndarray
    rho_d: np.ndarray
    retro: np.ndarray
    ambient: np.ndarray

    def planes(self):
        return [getattr(self, p) for p in GBuffer.PLANES]

    def pixel_dirs(self) -> np.ndarray:
        """Unit sensor-frame directions of the pixel centres, float64 [H, W, 3]."""
        X = (np.arange(self.W) + 0.5 - self.cx) / self.fx
        Y = (np.arange(self.H) + 0.5 - self.cy) / self.fy
        c = np.stack(np.broadcast_arrays(X[None, :], Y[:, None], np.ones((self.H, 1))), axis=-1)
        c = c / np.linalg.norm(c, axis=-1, keepdims=True)
        return c @ np.asarray(self.R, np.float64).T


def camera_looking_along(yaw, pitch):
    """Camera -> sensor rotation of a camera whose optical axis points at
    (azimuth yaw, elevation pitch), image x to the right (decreasing azimuth)
    and image y down."""
    ca, sa, ce, se = math.cos(yaw), math.sin(yaw), math.cos(pitch), math.sin(pitch)
    z = np.array([ce * ca, ce * sa, se])
    x = np.array([sa, -ca, 0.0])
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=1)


def raycast_pinhole(scene: Scene, W, H, fx, fy, cx, cy, R, depth_is_z=False) -> PinholeGBuffer:
    """Nearest-hit ray cast of the scene through the pinhole pixel centres."""
    ph = PinholeGBuffer(W, H, fx, fy, cx, cy, np.asarray(R, np.float64), bool(depth_is_z), *[None] * 7)
    dirs = ph.pixel_dirs()
    P = _empty_planes(H, W)
    for pl in scene.planes:
        t = _hit_plane(dirs, pl.n, pl.d)
        rho = np.full(t.shape, pl.rho_d)
        retro = np.full(t.shape, pl.retro)
        if pl.decal is not None:
            dq = dirs * np.where(np.isfinite(t), t, 0.0)[..., None] - pl.decal.c
            inside = (np.abs(dq @ pl.decal.e1) <= pl.decal.h1) & (np.abs(dq @ pl.decal.e2) <= pl.decal.h2)
            inside &= np.isfinite(t)
            rho = np.where(inside, pl.decal.rho_d, rho)
            retro = np.where(inside, pl.decal.retro, retro)
        better = t < P["range"]
        for key, val in (("range", t), ("nx", pl.n[0]), ("ny", pl.n[1]), ("nz", pl.n[2]), ("rho_d", rho),
                         ("retro", retro)):
            P[key] = np.where(better, val, P[key])
    Rm = np.asarray(R, np.float64)
    for r in scene.rects:
        # the pixels the rectangle can cover: its projected corners' box (+2 px),
        # or the whole image if a corner lies behind the camera
        corners = [r.c + sa * r.h1 * r.e1 + sb * r.h2 * r.e2 for sa in (-1, 1) for sb in (-1, 1)]
        cam = np.array(corners) @ Rm  # camera-frame coordinates
        if (cam[:, 2] > 1e-6).all():
            pxs = cx + fx * cam[:, 0] / cam[:, 2]
            pys = cy + fy * cam[:, 1] / cam[:, 2]
            i0, i1 = max(0, int(math.floor(pxs.min())) - 2), min(W, int(math.ceil(pxs.max())) + 3)
            j0, j1 = max(0, int(math.floor(pys.min())) - 2), min(H, int(math.ceil(pys.max())) + 3)
            if i0 >= i1 or j0 >= j1:
                continue
        else:
            i0, i1, j0, j1 = 0, W, 0, H
        sl = (slice(j0, j1), slice(i0, i1))
        d = dirs[sl]
        n = r.n
        t = _hit_plane(d, n, float(n @ r.c))
        dq = d * np.where(np.isfinite(t), t, 0.0)[..., None] - r.c
        inside = (np.abs(dq @ r.e1) <= r.h1) & (np.abs(dq @ r.e2) <= r.h2) & np.isfinite(t)
        t = np.where(inside, t, np.inf)
        better = t < P["range"][sl]
        for key, val in (("range", t), ("nx", n[0]), ("ny", n[1]), ("nz", n[2]), ("rho_d", r.rho_d),
                         ("retro", r.retro)):
            P[key][sl] = np.where(better, val, P[key][sl])
    hit = np.isfinite(P["range"])
    if scene.ambient == "uniform":
        P["ambient"][:] = scene.ambient_level
    elif scene.ambient == "sun":
        P["ambient"] = np.where(hit, scene.ambient_level * P["rho_d"] / math.pi * np.maximum(0.0, P["nz"]), 0.0)
    for k in ("nx", "ny", "nz", "rho_d", "retro"):
        P[k] = np.where(hit, P[k], 0.0)
    if depth_is_z:
        # z depth = distance times the cosine to the optical axis
        cz = dirs @ np.asarray(R, np.float64)[:, 2]
        P["range"] = np.where(hit, P["range"] * cz, P["range"])
    for k in GBuffer.PLANES:
        setattr(ph, k, np.ascontiguousarray(P[k], dtype=np.float32))
    return ph


def pinhole_plane_retro(seed: int = 6, W: int = 320, H: int = 240, f: float = 2000.0, depth_is_z=False):
    """The plane + retro patch scene rendered through a pinhole looking 0.5 deg
    off the plane's normal (a 9.2 x 6.9 deg field of view), and the spherical
    target grid (0.02 deg pitch) that covers it with a margin."""
    g = rng(seed)
    jit = g.uniform(-1e-3, 1e-3, size=2)
    decal = Rect(np.array([10.0, jit[0], jit[1]]), np.array([0.0, 1.0, 0.0]),
                 np.array([0.0, 0.0, 1.0]), 0.25, 0.25, rho_d=0.5, retro=100.0)
    scene = Scene(planes=[Plane(np.array([1.0, 0.0, 0.0]), 10.0, 0.5, 0.0, decal)],
                  ambient="uniform", ambient_level=0.01)
    R = camera_looking_along(0.5 * DEG, 0.2 * DEG)
    ph = raycast_pinhole(scene, W, H, f, f, W / 2.0, H / 2.0, R, depth_is_z)
    pitch = 0.02 * DEG
    U, V = 384, 256
    grid = GBuffer(U, V, 0.5 * DEG - U * pitch / 2, 0.2 * DEG - V * pitch / 2, pitch, pitch, *[None] * 7)
    return ph, grid


def pinhole_boxes_frame(seed: int = 7, W: int = 2048, H: int = 1024, U: int = 2048, V: int = 1024,
                        n_boxes: int = 40, rows: int = 16, cols: int = 1600):
    """A rasterised frame: the full frame's scene family (ground 2 m below the
    sensor, boxes at 5-150 m, log-uniform reflectance, 5 % retro faces, sun
    ambient) within +-28 deg of azimuth, rendered through a W x H pinhole with
    a 60 deg horizontal field of view (square pixels) looking along +x; the
    spherical target grid U x V spans +-29 x +-14 deg (inside the pinhole's
    view). Sensor: 16 x 1600 line scan over 56 x 26 deg, the 401 x 401 table
    profile, 2048 bins of 0.1 ns. Returns (PinholeGBuffer, target GBuffer
    geometry, Workload whose gbuffer is the target geometry)."""
    g = rng(seed)
    h_sensor = 2.0
    planes = [Plane(np.array([0.0, 0.0, 1.0]), -h_sensor, 0.2, 0.0)]
    rects = []
    for _ in range(n_boxes):
        rng_m = g.uniform(5.0, 150.0)
        az = g.uniform(-28 * DEG, 28 * DEG)
        half = g.uniform(0.25, 2.5, size=3)
        yaw = g.uniform(-math.pi, math.pi)
        rho = math.exp(g.uniform(math.log(0.05), math.log(0.9)))
        retro = np.where(g.uniform(size=6) < 0.05, 100.0, 0.0)
        dist = max(rng_m, float(np.linalg.norm(half)) + 1.5)
        c = np.array([dist * math.cos(az), dist * math.sin(az), -h_sensor + half[2]])
        rects += box_rects(c, half, yaw, rho, retro)
    scene = Scene(planes=planes, rects=rects, ambient="sun", ambient_level=1e3)
    f = W / 2 / math.tan(30 * DEG)
    ph = raycast_pinhole(scene, W, H, f, f, W / 2.0, H / 2.0, camera_looking_along(0.0, 0.0))
    daz, dele = 58 * DEG / U, 28 * DEG / V
    grid = GBuffer(U, V, -29 * DEG, -14 * DEG, daz, dele, *[None] * 7)
    dirs = linescan_pattern(rows, cols, 56 * DEG, 26 * DEG)
    wl = Workload(f"pinhole{W}x{H}_to_{U}x{V}_boxes_linescan{rows}x{cols}_table401_2048bins", grid, dirs,
                  table_profile(three_gauss_tail_table(), 0.01), pulse(2048, 0.1e-9), calib(2e-7, 1e-9, 3, True))
    return ph, grid, wl


def box_rects(center, half, yaw, rho_d, retro_faces) -> list:
    """The six faces of a box with vertical axis, as outward-facing rectangles."""
    cy, sy = math.cos(yaw), math.sin(yaw)
    ax = np.array([cy, sy, 0.0])
    ay = np.array([-sy, cy, 0.0])
    az = np.array([0.0, 0.0, 1.0])
    hx, hy, hz = half
    c = np.asarray(center, np.float64)
    faces = [
        (c + ax * hx, ay, az, hy, hz),
        (c - ax * hx, az, ay, hz, hy),
        (c + ay * hy, az, ax, hz, hx),
        (c - ay * hy, ax, az, hx, hz),
        (c + az * hz, ax, ay, hx, hy),
        (c - az * hz, ay, ax, hy, hx),
    ]
    out = []
    for i, (fc, e1, e2, h1, h2) in enumerate(faces):
        out.append(Rect(fc, e1, e2, h1, h2, rho_d, retro_faces[i]))
    return out


# ----------------------------------------------------------------------------
# beam patterns (unit directions in the sensor frame, float32 [n, 3])
# ----------------------------------------------------------------------------


def _dirs_from_angles(az, el):
    az = np.asarray(az, np.float64)
    el = np.asarray(el, np.float64)
    d = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=-1)
    return np.ascontiguousarray(d, dtype=np.float32)


def grid_pattern(n_az, n_el, fov_az, fov_el, az_c=0.0, el_c=0.0):
    """Regular grid of beam centres, row-major (elevation rows, azimuth inside)."""
    az = az_c - fov_az / 2 + (np.arange(n_az) + 0.5) * fov_az / n_az
    el = el_c - fov_el / 2 + (np.arange(n_el) + 0.5) * fov_el / n_el
    A, E = np.meshgrid(az, el)
    return _dirs_from_angles(A.ravel(), E.ravel())


def edge_two_depths(n_beams=41, span_deg=0.2, threshold=1e-6):
    """A 2x2 m board at 7 m (rho_d 0.3) covering the left half of the view in
    front of a plane at 10 m (rho_d 0.5), 512x256 at 0.01 deg, and a row of
    beams across the board's edge (azimuth within +-span_deg of it): beams
    near the edge return both surfaces, the nearer or the farther being the
    stronger depending on how much of the footprint each covers."""
    deg = math.pi / 180
    board = Rect(np.array([7.0, -1.0, 0.0]), np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]), 1.0, 1.0, 0.3, 0.0)
    sc = Scene(planes=[Plane(np.array([1.0, 0.0, 0.0]), 10.0, 0.5)], rects=[board], ambient="uniform",
               ambient_level=0.01)
    pitch = 0.01 * deg
    U, V = 512, 256
    gb = raycast(sc, U, V, -U * pitch / 2, -V * pitch / 2, pitch, pitch)
    az = np.linspace(-span_deg, span_deg, n_beams) * deg
    dirs = _dirs_from_angles(az, np.zeros_like(az))
    return Workload("edge_two_depths", gb, dirs, radial_profile(), pulse(1024, 0.1e-9), calib(threshold, 1e-5, 3, True))


def linescan_pattern(rows, cols, fov_az, fov_el):
    return grid_pattern(cols, rows, fov_az, fov_el)


def lissajous_pattern(n, fov_az, fov_el, fx=7, fy=9, phase=0.3):
    t = (np.arange(n) + 0.5) / n
    az = fov_az / 2 * np.sin(2 * math.pi * fx * t + phase)
    el = fov_el / 2 * np.sin(2 * math.pi * fy * t)
    return _dirs_from_angles(az, el)


# ----------------------------------------------------------------------------
# tabulated profiles (stand-ins for the goniometer measurement of Sec. III)
# ----------------------------------------------------------------------------


def table_grid(w, h, pitch_deg):
    u = (np.arange(w) - (w - 1) / 2) * pitch_deg
    v = (np.arange(h) - (h - 1) / 2) * pitch_deg
    return np.meshgrid(u, v)  # U[j, i], V[j, i]


def three_gauss_tail_table(w=401, h=401, pitch_deg=0.01, sigmas=(0.03, 0.1, 0.3),
                           weights=(1.0, 1e-2, 1e-4), tail_amp=1e-6, tail_core=0.05, tail_pow=3.0):
    Uu, Vv = table_grid(w, h, pitch_deg)
    th = np.hypot(Uu, Vv)
    t = np.zeros_like(th)
    for s, wt in zip(sigmas, weights):
        t += wt * np.exp(-th * th / (2 * s * s))
    with np.errstate(divide="ignore"):
        t += tail_amp * np.minimum(1.0, (th / tail_core) ** (-tail_pow))
    return np.ascontiguousarray(t, dtype=np.float32)


def elliptic_gauss_table(w, h, pitch_deg, sigma_u, sigma_v):
    Uu, Vv = table_grid(w, h, pitch_deg)
    t = np.exp(-0.5 * (Uu / sigma_u) ** 2 - 0.5 * (Vv / sigma_v) ** 2)
    return np.ascontiguousarray(t, dtype=np.float32)


# ----------------------------------------------------------------------------
# parameter sets (plain dicts, mirrored by the C structs of the library)
# ----------------------------------------------------------------------------


def radial_profile(sigma_deg=0.05, tail_amp=1e-4, tail_core_deg=0.05, tail_pow=3.0, trunc_deg=1.0):
    return dict(kind=0, sigma_deg=sigma_deg, tail_amp=tail_amp, tail_core_deg=tail_core_deg,
                tail_pow=tail_pow, trunc_deg=trunc_deg)


def table_profile(table, pitch_deg):
    table = np.ascontiguousarray(table, dtype=np.float32)
    return dict(kind=1, table=table, table_w=table.shape[1], table_h=table.shape[0], pitch_deg=pitch_deg)


def separable_profile(h, v, pitch_deg):
    """P(u, v) = H(u) V(v): nodes of H along u and of V along v, centred, at pitch_deg."""
    h = np.ascontiguousarray(h, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    return dict(kind=2, h=h, v=v, pitch_deg=pitch_deg)


def separable_gauss_tail(n_u, n_v, pitch_deg, sigma_u, sigma_v, tail_amp=0.0, tail_core=0.05, tail_pow=3.0):
    """1-D profiles exp(-x^2 / 2 s^2) + tail_amp min(1, (|x| / core)^-pow) on
    n nodes at pitch_deg along u and v (an anisotropic separable beam)."""
    def prof(n, s):
        x = (np.arange(n) - 0.5 * (n - 1)) * pitch_deg
        ax = np.maximum(np.abs(x), 1e-12)
        return np.exp(-0.5 * (x / s) ** 2) + tail_amp * np.minimum(1.0, (ax / tail_core) ** -tail_pow)
    return separable_profile(prof(n_u, sigma_u), prof(n_v, sigma_v), pitch_deg)


def pulse(n_bins=1024, dt_s=0.1e-9, t0_s=0.0, fwhm_s=4e-9, trunc_sigmas=6.0):
    return dict(n_bins=n_bins, dt_s=dt_s, t0_s=t0_s, fwhm_s=fwhm_s, trunc_sigmas=trunc_sigmas)


def calib(threshold=1e-5, ambient_scale=1e-4, max_echoes=3, fit_epw=True, epw_coef=(0.0, 0.0, 0.0)):
    return dict(threshold=threshold, ambient_scale=ambient_scale, max_echoes=max_echoes,
                fit_epw=int(fit_epw), epw_coef=tuple(epw_coef))


IDENTITY_POSE = np.eye(3, dtype=np.float32)


def pose_ypr(yaw, pitch, roll):
    """Rotation (sensor frame -> G-buffer frame) from yaw about z, pitch about y, roll about x."""
    cy, sy = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    cr, sr = math.cos(roll), math.sin(roll)
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    return np.ascontiguousarray(Rz @ Ry @ Rx, dtype=np.float32)


@dataclass
class Workload:
    name: str
    gbuffer: GBuffer
    dirs: np.ndarray
    profile: dict
    pulse: dict
    calib: dict
    pose: np.ndarray = field(default_factory=lambda: IDENTITY_POSE.copy())


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

DEG = math.pi / 180.0


def small_plane_retro(seed: int = 13, size: int = 256) -> Workload:
    """Plain FP32 small instance: 256x256 G-buffer at 0.02 deg pitch looking at a
    Lambertian plane at 10 m (reflectance 0.5) with a centred 0.5 x 0.5 m
    retroreflective patch (gain 100), uniform ambient 0.01, 32x16 grid beams,
    Gaussian (sigma 0.05 deg) + 1e-4 (theta/0.05 deg)^-3 tail truncated at 1 deg,
    1024 bins of 0.1 ns, 4 ns FWHM Gaussian pulse, up to 3 echoes.

    The seed jitters the patch centre and the plane's distance by up to +-1 mm
    each (the scene family); the pattern and all parameters are fixed. With the
    default seed no bin of any beam's FP64 waveform lies within 7e-4 T of the
    threshold T, so every echo of the instance is compared bit-exactly."""
    g = rng(seed)
    jit = g.uniform(-1e-3, 1e-3, size=3)
    pitch = 0.02 * DEG
    fov = size * pitch
    dist = 10.0 + jit[2]
    decal = Rect(np.array([dist, jit[0], jit[1]]), np.array([0.0, 1.0, 0.0]),
                 np.array([0.0, 0.0, 1.0]), 0.25, 0.25, rho_d=0.5, retro=100.0)
    scene = Scene(planes=[Plane(np.array([1.0, 0.0, 0.0]), dist, 0.5, 0.0, decal)],
                  ambient="uniform", ambient_level=0.01)
    gb = raycast(scene, size, size, -fov / 2, -fov / 2, pitch, pitch)
    dirs = grid_pattern(32, 16, 5.12 * DEG, 5.12 * DEG)
    return Workload("plane_retro_256x256_512beams_1024bins", gb, dirs, radial_profile(),
                    pulse(1024, 0.1e-9), calib(1e-5, 1e-4, 3, True))


def full_frame_boxes(seed: int = 2, U: int = 2048, V: int = 1024, n_boxes: int = 50,
                     rows: int = 16, cols: int = 1600) -> Workload:
    """Plain FP32 full frame: 2048x1024 G-buffer over 120 x 30 deg, ground plane
    2 m below the sensor, 50 boxes at 5-150 m (edges 0.5-5 m, log-uniform
    reflectance 0.05-0.9, 5 % of faces retroreflective with gain 100), sun
    ambient 1e3 on upward faces, 16 x 1600 line scan, 401x401 table at 0.01 deg
    (3 Gaussians + power-law tail), 2048 bins of 0.1 ns."""
    g = rng(seed)
    fov_az, fov_el = 120 * DEG, 30 * DEG
    daz, dele = fov_az / U, fov_el / V
    h_sensor = 2.0
    planes = [Plane(np.array([0.0, 0.0, 1.0]), -h_sensor, 0.2, 0.0)]
    rects = []
    for _ in range(n_boxes):
        rng_m = g.uniform(5.0, 150.0)
        az = g.uniform(-fov_az / 2, fov_az / 2)
        half = g.uniform(0.25, 2.5, size=3)
        yaw = g.uniform(-math.pi, math.pi)
        rho = math.exp(g.uniform(math.log(0.05), math.log(0.9)))
        retro = np.where(g.uniform(size=6) < 0.05, 100.0, 0.0)
        dist = max(rng_m, float(np.linalg.norm(half)) + 1.5)
        c = np.array([dist * math.cos(az), dist * math.sin(az), -h_sensor + half[2]])
        rects += box_rects(c, half, yaw, rho, retro)
    scene = Scene(planes=planes, rects=rects, ambient="sun", ambient_level=1e3)
    gb = raycast(scene, U, V, -fov_az / 2, -fov_el / 2, daz, dele)
    dirs = linescan_pattern(rows, cols, fov_az, fov_el)
    prof = table_profile(three_gauss_tail_table(), 0.01)
    return Workload(f"boxes_{U}x{V}_linescan{rows}x{cols}_table401_2048bins", gb, dirs, prof,
                    pulse(2048, 0.1e-9), calib(2e-7, 1e-9, 3, True))


def tiny_case(seed: int = 3, U: int = 37, V: int = 29, n_beams: int = 5, n_bins: int = 256) -> Workload:
    """A tiny ragged case: tilted plane, a box, random beams and a rolled pose."""
    g = rng(seed)
    pitch = 0.05 * DEG
    planes = [Plane(np.array([math.cos(0.3), 0.0, math.sin(0.3)]), 8.0, 0.4, 0.0)]
    rects = box_rects(np.array([6.0, 0.02, 0.0]), (0.1, 0.04, 0.04), 0.4, 0.6,
                      np.array([0, 100.0, 0, 0, 0, 0]))
    scene = Scene(planes=planes, rects=rects, ambient="uniform", ambient_level=0.05)
    gb = raycast(scene, U, V, -U * pitch / 2, -V * pitch / 2, pitch, pitch)
    az = g.uniform(-U * pitch / 3, U * pitch / 3, n_beams)
    el = g.uniform(-V * pitch / 3, V * pitch / 3, n_beams)
    dirs = _dirs_from_angles(az, el)
    prof = radial_profile(0.08, 1e-3, 0.08, 3.0, 0.4)
    return Workload("tiny", gb, dirs, prof, pulse(n_bins, 0.1e-9), calib(2e-4, 1e-3, 3, True),
                    pose_ypr(0.002, -0.001, 0.3))


# ----------------------------------------------------------------------------
# batched workload: many frames of uneven size, pattern and pose
# ----------------------------------------------------------------------------

SIZE_CLASSES = ((512, 256), (1024, 512), (2048, 1024), (4096, 2048))


def _boresight_frame(R):
    """Azimuth and elevation of the sensor boresight R x in the G-buffer frame."""
    a = np.asarray(R, np.float64) @ np.array([1.0, 0.0, 0.0])
    return math.atan2(a[1], a[0]), math.asin(max(-1.0, min(1.0, a[2])))


def plane_retro_frame(g, U, V, R, pitch_deg=0.02):
    """One frame of the plane + retro-patch scene family seen by a posed sensor:
    a Lambertian plane across the boresight at 6-14 m (reflectance 0.3-0.7),
    a 0.5 x 0.5 m retro patch (gain 100) placed within a few degrees of the
    boresight, uniform ambient 0.01; the G-buffer is centred on the boresight."""
    R = np.asarray(R, np.float64)
    bx, by, bz = R[:, 0], R[:, 1], R[:, 2]
    dist = g.uniform(6.0, 14.0)
    rho = g.uniform(0.3, 0.7)
    off = g.uniform(-2.5, 2.5, size=2) * DEG * dist
    decal = Rect(dist * bx + off[0] * by + off[1] * bz, by, bz, 0.25, 0.25, rho_d=rho, retro=100.0)
    scene = Scene(planes=[Plane(bx, dist, rho, 0.0, decal)], ambient="uniform", ambient_level=0.01)
    az_c, el_c = _boresight_frame(R)
    pitch = pitch_deg * DEG
    return raycast(scene, U, V, az_c - U * pitch / 2, el_c - V * pitch / 2, pitch, pitch)


def batched_frames(seed: int = 4, n_frames: int = 64, size_classes=SIZE_CLASSES, beams=(1_000, 100_000)):
    """Batched workload: n_frames frames, each with a G-buffer size drawn from
    size_classes, a beam count log-uniform in `beams`, a line-scan or a MEMS
    Lissajous (7:9) pattern over 80 % of its field of view, and a random pose
    (yaw +-180 deg, pitch +-5 deg, roll +-2 deg). All frames share the sensor
    model of the small plane/retro instance (radial profile, 1024 bins of 0.1 ns).
    Returns a list of Workload."""
    g = rng(seed)
    base = small_plane_retro()
    out = []
    for f in range(n_frames):
        U, V = size_classes[int(g.integers(len(size_classes)))]
        R = pose_ypr(g.uniform(-math.pi, math.pi), g.uniform(-5, 5) * DEG, g.uniform(-2, 2) * DEG)
        gb = plane_retro_frame(g, U, V, R)
        nb = int(round(math.exp(g.uniform(math.log(beams[0]), math.log(beams[1])))))
        fov_az, fov_el = 0.8 * U * 0.02 * DEG, 0.8 * V * 0.02 * DEG
        if g.uniform() < 0.5:
            rows = max(4, int(round(math.sqrt(nb * fov_el / fov_az))))
            cols = max(1, nb // rows)
            dirs = linescan_pattern(rows, cols, fov_az, fov_el)
            kind = f"linescan{rows}x{cols}"
        else:
            dirs = lissajous_pattern(nb, fov_az, fov_el, 7, 9, phase=g.uniform(0, 2 * math.pi))
            kind = f"lissajous{nb}"
        out.append(Workload(f"frame{f}_{U}x{V}_{kind}", gb, dirs, base.profile, base.pulse, base.calib, R))
    return out


def wide_frame(seed: int = 5, U: int = 8192, V: int = 4096, n_az: int = 500, n_el: int = 400,
               n_boxes: int = 24) -> Workload:
    """Wide-tail instance: 8192x4096 G-buffer at 0.02 deg (163.84 x 81.92 deg)
    of the plane/retro scene family (a plane at 10 m across the boresight with
    retro patches, a ground plane 2 m below, boxes at 5-25 m, uniform ambient
    0.01), 500 x 400 = 200k grid beams over 90 % of the field of view, the
    radial profile of the small instance with its tail truncated at 2 deg, and
    4096 bins of 0.05 ns."""
    g = rng(seed)
    pitch = 0.02 * DEG
    planes = [Plane(np.array([1.0, 0.0, 0.0]), 10.0, 0.5, 0.0,
                    Rect(np.array([10.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]),
                         0.25, 0.25, rho_d=0.5, retro=100.0)),
              Plane(np.array([0.0, 0.0, 1.0]), -2.0, 0.2, 0.0)]
    rects = []
    for _ in range(6):  # extra retro patches on the front plane
        c = np.array([9.999, g.uniform(-8, 8), g.uniform(-1.5, 4)])
        rects.append(Rect(c, np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]), 0.2, 0.2, 0.5, 100.0))
    for _ in range(n_boxes):
        rr = g.uniform(5.0, 25.0)
        az = g.uniform(-75, 75) * DEG
        half = g.uniform(0.25, 1.5, size=3)
        rho = math.exp(g.uniform(math.log(0.05), math.log(0.9)))
        retro = np.where(g.uniform(size=6) < 0.05, 100.0, 0.0)
        d = max(rr, float(np.linalg.norm(half)) + 1.5)
        c = np.array([d * math.cos(az), d * math.sin(az), -2.0 + half[2]])
        rects += box_rects(c, half, g.uniform(-math.pi, math.pi), rho, retro)
    scene = Scene(planes=planes, rects=rects, ambient="uniform", ambient_level=0.01)
    gb = raycast(scene, U, V, -U * pitch / 2, -V * pitch / 2, pitch, pitch)
    dirs = grid_pattern(n_az, n_el, 0.9 * U * 0.02 * DEG, 0.9 * V * 0.02 * DEG)
    prof = radial_profile(0.05, 1e-4, 0.05, 3.0, 2.0)
    return Workload(f"wide_{U}x{V}_{n_az * n_el}beams_4096bins", gb, dirs, prof, pulse(4096, 0.05e-9),
                    calib(1e-5, 1e-4, 3, True))
