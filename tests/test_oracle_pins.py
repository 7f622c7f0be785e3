"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these checks re-derives the oracle's own formula: each one compares
against a closed form, an invariant, an independent library routine or a
brute-force evaluation, chosen so that a dropped term, a wrong sign or index
or a transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from paper_2512_05932_gb300 import scenes as S

C = 299_792_458.0
DEG = math.pi / 180
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gauss_profile(sigma_deg, trunc_deg):
    return S.radial_profile(sigma_deg, 0.0, sigma_deg, 3.0, trunc_deg)


def plane_gbuffer(normal, dist, rho=0.5, retro=0.0, U=256, V=256, pitch_deg=0.02, az_c=0.0, el_c=0.0,
                  amb=0.0, decal=None, rects=()):
    pitch = pitch_deg * DEG
    sc = S.Scene(planes=[S.Plane(np.asarray(normal, float), dist, rho, retro, decal)] if normal is not None else [],
                 rects=list(rects), ambient="uniform", ambient_level=amb)
    return S.raycast(sc, U, V, az_c - U * pitch / 2, el_c - V * pitch / 2, pitch, pitch)


def boresight():
    return np.array([[1.0, 0.0, 0.0]], np.float32)


# --------------------------------------------------------------------------
# profile (Eq. centered kernel) and its normalisation
# --------------------------------------------------------------------------


def test_radial_gaussian_norm_closed_form(orc):
    # int_0^Theta exp(-t^2/2s^2) sin t dt: closed form in the small-angle limit
    # plus scipy quadrature of the exact spherical integrand
    for sig, tr in ((0.05, 1.0), (0.3, 2.0), (1.0, 3.0)):
        Z = orc.profile_norm(gauss_profile(sig, tr))
        s, T = sig * DEG, tr * DEG
        exact = 2 * math.pi * integrate.quad(lambda t: math.exp(-t * t / (2 * s * s)) * math.sin(t), 0, T,
                                             epsabs=0, epsrel=1e-13, limit=200)[0]
        planar = 2 * math.pi * s * s * (1 - math.exp(-T * T / (2 * s * s)))
        assert Z == pytest.approx(exact, rel=1e-9)
        assert Z == pytest.approx(planar, rel=2 * s * s)


def test_radial_profile_values(orc):
    p = S.radial_profile(0.05, 1e-4, 0.05, 3.0, 1.0)
    assert orc.profile_raw(p, 0.0, 0.0)[0] == pytest.approx(1 + 1e-4, rel=1e-15)
    # at theta = sigma the Gaussian is exp(-1/2) and the tail is at its core
    assert orc.profile_raw(p, 0.03, 0.04)[0] == pytest.approx(math.exp(-0.5) + 1e-4, rel=1e-12)
    # at 0.5 deg: tail 1e-4 (10)^-3 plus a negligible Gaussian
    assert orc.profile_raw(p, 0.0, -0.5)[0] == pytest.approx(1e-7 + math.exp(-50), rel=1e-12)
    assert orc.profile_raw(p, 1.0001, 0.0)[0] == 0.0


def test_table_profile_nodes_and_orientation(orc):
    # an asymmetric table: values at nodes must come back exactly, with the
    # column index along u and the row index along v
    t = np.arange(5 * 7, dtype=np.float32).reshape(5, 7) + 1.0  # [h=5][w=7]
    p = S.table_profile(t, 0.1)
    for j in range(5):
        for i in range(7):
            u, v = (i - 3) * 0.1, (j - 2) * 0.1
            assert orc.profile_raw(p, u, v)[0] == pytest.approx(t[j, i], rel=1e-12)
    # cell centre = mean of 4 corners; beyond the zero ring it is 0
    assert orc.profile_raw(p, 0.05, 0.05)[0] == pytest.approx(t[2:4, 3:5].mean(), rel=1e-12)
    assert orc.profile_raw(p, 0.35, 0.0)[0] == pytest.approx(0.5 * t[2, 6], rel=1e-12)
    assert orc.profile_raw(p, 0.41, 0.0)[0] == 0.0


def test_table_norm_closed_form(orc):
    # bilinear interpolant of a sampled Gaussian integrates like the
    # trapezoid rule, which is spectrally accurate: 2 pi su sv (small angles)
    for su, sv in ((0.05, 0.05), (0.05, 0.1)):
        tab = S.elliptic_gauss_table(121, 161, 0.01, su, sv)
        Z = orc.profile_norm(S.table_profile(tab, 0.01))
        assert Z == pytest.approx(2 * math.pi * su * sv * DEG * DEG, rel=2e-6)


def test_separable_profile_is_the_outer_product_table(orc):
    # H(u) V(v) with 1-D linear interpolation must equal the bilinear table of
    # the outer product V[j] H[i] everywhere (nodes, cell interiors, the zero
    # ring and beyond), and integrate to the same Z
    g = np.random.default_rng(11)
    h = g.uniform(0.1, 2.0, 7).astype(np.float32)
    v = g.uniform(0.1, 2.0, 5).astype(np.float32)
    sep = S.separable_profile(h, v, 0.1)
    tab = S.table_profile(np.outer(v.astype(np.float64), h.astype(np.float64)), 0.1)
    for j in range(5):
        for i in range(7):
            u_, v_ = (i - 3) * 0.1, (j - 2) * 0.1
            assert orc.profile_raw(sep, u_, v_)[0] == pytest.approx(float(h[i]) * float(v[j]), rel=1e-12)
    uu = g.uniform(-0.5, 0.5, 200)
    vv = g.uniform(-0.4, 0.4, 200)
    np.testing.assert_allclose(orc.profile_raw(sep, uu, vv), orc.profile_raw(tab, uu, vv), rtol=1e-6, atol=1e-12)
    assert orc.profile_raw(sep, 0.41, 0.0)[0] == 0.0 and orc.profile_raw(sep, 0.0, 0.31)[0] == 0.0
    # u runs along H, v along V: swapping the tables must change the value
    assert orc.profile_raw(sep, 0.3, 0.0)[0] != pytest.approx(orc.profile_raw(
        S.separable_profile(v, h, 0.1), 0.3, 0.0)[0], rel=1e-3)
    assert orc.profile_norm(sep) == pytest.approx(orc.profile_norm(tab), rel=1e-6)


def test_separable_gauss_norm_closed_form(orc):
    # a product of sampled 1-D Gaussians integrates to 2 pi su sv (small angles)
    for su, sv in ((0.05, 0.05), (0.05, 0.1)):
        prof = S.separable_gauss_tail(121, 161, 0.01, su, sv)
        assert orc.profile_norm(prof) == pytest.approx(2 * math.pi * su * sv * DEG * DEG, rel=2e-6)


# --------------------------------------------------------------------------
# beam frame and local offsets
# --------------------------------------------------------------------------


def _dir(az, el):
    return np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])


def test_offsets_meridian_and_great_circle(orc):
    I = np.eye(3)
    for az_b, el_b in ((0.0, 0.0), (0.7, 0.3), (-2.0, -1.2)):
        # the beam direction is a float32 input: use the angles it really has
        a = _dir(az_b, el_b).astype(np.float32).astype(np.float64)
        a /= np.linalg.norm(a)
        az_b, el_b = math.atan2(a[1], a[0]), math.asin(a[2])
        # along the meridian: pure +v, magnitude = elevation step
        d = _dir(az_b, el_b + 0.01)
        u, v, f = orc.offsets(I, a, d[None])
        assert f[0] and abs(u[0]) < 1e-12 and v[0] == pytest.approx(0.01 / DEG, rel=1e-10)
        # along the east great circle (rotation about the north axis): pure +u
        e1 = np.array([-math.sin(az_b), math.cos(az_b), 0.0])
        d = math.cos(0.02) * a + math.sin(0.02) * e1
        u, v, f = orc.offsets(I, a, d[None])
        assert u[0] == pytest.approx(0.02 / DEG, rel=1e-10) and abs(v[0]) < 1e-10
        # |(u, v)| equals the great-circle angle (spherical law of cosines)
        rng = S.rng(5)
        dd = np.array([_dir(az_b + x, el_b + y) for x, y in rng.uniform(-0.03, 0.03, (20, 2))])
        u, v, f = orc.offsets(I, a, dd)
        ang = np.arccos(np.clip(dd @ a, -1, 1)) / DEG
        np.testing.assert_allclose(np.hypot(u, v), ang, rtol=1e-8)
    # back hemisphere is outside
    _, _, f = orc.offsets(I, _dir(0, 0), _dir(math.pi, 0)[None])
    assert not f[0]


def test_offsets_pose_invariance(orc):
    rng = S.rng(11)
    a = _dir(0.2, 0.1)
    dd = np.array([_dir(0.2 + x, 0.1 + y) for x, y in rng.uniform(-0.02, 0.02, (30, 2))])
    u0, v0, _ = orc.offsets(np.eye(3), a, dd)
    R = S.pose_ypr(0.4, -0.2, 0.7).astype(np.float64)
    u1, v1, _ = orc.offsets(R.astype(np.float32), a, dd @ R.astype(np.float32).astype(np.float64).T)
    np.testing.assert_allclose(u1, u0, atol=1e-5)
    np.testing.assert_allclose(v1, v0, atol=1e-5)


# --------------------------------------------------------------------------
# per-pixel return, solid angle and range interval
# --------------------------------------------------------------------------


def _sphere_gbuffer(normal, dist, rho, retro, pitch_deg=0.25, amb=0.0):
    U, V = int(round(360 / pitch_deg)), int(round(180 / pitch_deg))
    pitch = pitch_deg * DEG
    sc = S.Scene(planes=[S.Plane(np.asarray(normal, float), dist, rho, retro)], ambient="uniform",
                 ambient_level=amb)
    return S.raycast(sc, U, V, -math.pi, -math.pi / 2, pitch, pitch)


@pytest.mark.parametrize("normal", [(1, 0, 0), (0.3, -0.5, 0.81), (0, 0, 1)])
def test_range_equation_over_sphere(orc, normal):
    # sum_p rho_hat d omega over the whole sphere for an infinite Lambertian
    # plane at distance d0: (rho/pi) int_hemisphere cos^3 d omega / d0^2
    # = rho / (2 d0^2), whatever the orientation; a retro gain g adds
    # g pi / (2 d0^2); every pixel's ambient sums to L * 4 pi
    n = np.asarray(normal, float)
    n /= np.linalg.norm(n)
    gb = _sphere_gbuffer(n, 3.0, 0.4, 0.0, amb=0.75)
    px = orc.pixels(gb)
    assert px["w"].sum() == pytest.approx(0.4 / (2 * 9.0), rel=2e-5)
    assert px["a"].sum() == pytest.approx(0.75 * 4 * math.pi, rel=1e-12)
    gb = _sphere_gbuffer(n, 3.0, 0.0, 50.0)
    assert orc.pixels(gb)["w"].sum() == pytest.approx(50.0 * math.pi / (2 * 9.0), rel=2e-5)


def test_solid_angle_telescopes(orc):
    gb = plane_gbuffer(None, 0, U=40, V=30, pitch_deg=0.7, el_c=0.4, amb=1.0)
    px = orc.pixels(gb)
    el_lo, el_hi = gb.el0, gb.el0 + gb.V * gb.dele
    assert px["a"].sum() == pytest.approx(gb.U * gb.daz * (math.sin(el_hi) - math.sin(el_lo)), rel=1e-12)
    assert not px["hit"].any() and (px["w"] == 0).all()


def test_range_interval_is_plane_extrapolation(orc):
    # for a plane the interval is spanned by the exact ranges of the four
    # corner rays and the centre ray (range correction of Sec. II-D)
    n = np.array([math.cos(1.2), math.sin(1.2) * 0.6, math.sin(1.2) * 0.8])
    # non-square pixels so that the azimuth and elevation half-widths differ
    sc = S.Scene(planes=[S.Plane(n, 6.0, 0.5)], ambient="none")
    gb = S.raycast(sc, 24, 18, -12 * 0.3 * DEG, -9 * 0.17 * DEG, 0.3 * DEG, 0.17 * DEG)
    px = orc.pixels(gb)
    for v in range(0, gb.V, 5):
        for u in range(0, gb.U, 7):
            az = gb.az0 + (u + 0.5) * gb.daz
            el = gb.el0 + (v + 0.5) * gb.dele
            rs = [6.0 / (_dir(az + i * gb.daz / 2, el + j * gb.dele / 2) @ n)
                  for i in (-1, 0, 1) for j in (-1, 0, 1) if (i == 0) == (j == 0)]
            assert px["t0"][v, u] == pytest.approx(2 * min(rs) / C, rel=1e-6)
            assert px["t1"][v, u] == pytest.approx(2 * max(rs) / C, rel=1e-6)


def test_range_interval_grazing_clamp(orc):
    # a plane seen edge-on by one corner ray: that corner is clamped to
    # |d.n| = 1e-3, giving r = range * mu_p / 1e-3
    az = 0.0
    gb = plane_gbuffer(np.array([0.0, 0.0, 1.0]), -1.0, U=3, V=3, pitch_deg=1.0, el_c=-1.0 * DEG - 0.5 * DEG)
    px = orc.pixels(gb)
    v, u = 2, 1  # top row: its upper corner ray is at el = 0, parallel to the plane
    el = gb.el0 + 2.5 * gb.dele
    rr = float(gb.range[v, u])
    mu_p = abs(math.sin(el))
    assert px["t1"][v, u] == pytest.approx(2 * rr * mu_p / 1e-3 / C, rel=1e-5)


def test_no_hit_and_nan(orc):
    gb = plane_gbuffer(np.array([1.0, 0, 0]), 5.0, U=8, V=8, pitch_deg=0.1)
    gb.range[0, 0] = np.nan
    gb.range[1, 1] = 0.0
    gb.range[2, 2] = -3.0
    px = orc.pixels(gb)
    assert not px["hit"][0, 0] and not px["hit"][1, 1] and not px["hit"][2, 2]
    assert px["hit"].sum() == 61


# --------------------------------------------------------------------------
# deposit over the range interval
# --------------------------------------------------------------------------


def test_deposit_weight_against_quadrature(orc):
    rng = S.rng(21)
    hat = lambda x: max(0.0, 1 - abs(x))
    for _ in range(200):
        X0 = rng.uniform(-3, 30)
        W = rng.choice([0.0, 1e-9, 0.3, 1.0, 2.7, 9.4])
        X1 = X0 + W
        ws = [orc.deposit_weight(X0, X1, k) for k in range(-6, 45)]
        if W == 0:
            ref = [hat(X0 - k) for k in range(-6, 45)]
        else:
            ref = [integrate.quad(lambda x: hat(x - k), X0, X1, points=[k - 1, k, k + 1], epsabs=1e-15,
                                  limit=100)[0] / W for k in range(-6, 45)]
        np.testing.assert_allclose(ws, ref, atol=1e-11 if W > 1e-6 else 1e-8)
        # partition of unity and first moment (centre of mass kept)
        assert sum(ws) == pytest.approx(1.0, abs=1e-12)
        assert sum(k * w for k, w in zip(range(-6, 45), ws)) == pytest.approx(X0 + W / 2, abs=1e-9)


# --------------------------------------------------------------------------
# pulse and convolution
# --------------------------------------------------------------------------


def test_pulse_taps(orc):
    pu = S.pulse(1024, 0.1e-9, 0.0, 4e-9, 6.0)
    taps = orc.pulse_taps(pu)
    M = (len(taps) - 1) // 2
    sig = 4e-9 / (2 * math.sqrt(2 * math.log(2))) / 0.1e-9
    assert M == math.ceil(6 * sig) == 102
    assert taps.sum() == pytest.approx(1.0, abs=1e-14)
    # half maximum at +-FWHM/2 = +-20 bins; symmetric; discrete variance = sigma^2
    assert taps[M + 20] / taps[M] == pytest.approx(0.5, rel=1e-12)
    assert taps[M - 20] == taps[M + 20]
    m = np.arange(-M, M + 1)
    assert (taps * m * m).sum() == pytest.approx(sig * sig, rel=1e-6)


def test_convolve_matches_numpy(orc):
    rng = S.rng(3)
    h = rng.uniform(0, 1, 300) * (rng.uniform(size=300) < 0.1)
    taps = orc.pulse_taps(S.pulse(300, 0.1e-9, 0, 2e-9, 4))
    M = (len(taps) - 1) // 2
    ref = np.convolve(h, taps)[M:M + 300] + 0.25
    np.testing.assert_allclose(orc.convolve(h, taps, 0.25), ref, rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------
# echoes: threshold intervals, crossings, peaks (Sec. II-C)
# --------------------------------------------------------------------------


PU = S.pulse(64, 0.1e-9, 0.0, 4e-9, 6.0)


def rng_of(x):
    return 0.5 * C * (x + 0.5) * 0.1e-9


def test_threshold_is_strict_and_runs_ordered(orc):
    xi = np.zeros(64)
    xi[5:9] = 1.0  # exactly at T: no echo
    xi[20:23] = [1.5, 2.0, 1.5]
    xi[40:42] = [3.0, 3.0]  # tie: lowest index wins
    xi[63] = 2.0  # clipped at the end
    e = orc.extract_echoes(xi, PU, 1.0)
    assert [(x["bin_start"], x["bin_end"], x["bin_peak"]) for x in e] == [(20, 22, 21), (40, 41, 40), (63, 63, 63)]
    assert e[2]["flags"] & 2 and not e[0]["flags"] & 3
    assert e[1]["flags"] & 8  # peak ambiguous
    xi2 = np.zeros(64)
    xi2[0:3] = 2.0
    assert orc.extract_echoes(xi2, PU, 1.0)[0]["flags"] & 1


def test_crossings_linear_interpolation(orc):
    xi = np.zeros(64)
    xi[10:20] = np.arange(1, 11)  # ramp 1..10 from bin 10, then drops to 0
    e = orc.extract_echoes(xi, PU, 2.5)[0]
    assert e["bin_start"] == 12 and e["bin_end"] == 19
    assert e["r0"] == pytest.approx(rng_of(11.5), rel=1e-14)
    assert e["r1"] == pytest.approx(rng_of(19 + 7.5 / 10), rel=1e-14)
    assert e["epw_m"] == pytest.approx(e["r1"] - e["r0"], rel=1e-14)


def test_log_parabola_recovers_gaussian_centre(orc):
    for mu in (30.0, 30.3, 30.5, 31.77):
        k = np.arange(64)
        xi = 5 * np.exp(-0.5 * ((k - mu) / 2.3) ** 2)
        e = orc.extract_echoes(xi, PU, 0.1)[0]
        assert e["x_peak"] == pytest.approx(mu, abs=1e-10)
        assert e["range_m"] == pytest.approx(rng_of(mu), rel=1e-12)


def test_intensity_from_coefficients(orc):
    xi = np.zeros(64)
    xi[10:13] = [2, 3, 2]
    e = orc.extract_echoes(xi, PU, 1.0, coef=(0.1, 2.0, -0.5))[0]
    E = e["epw_m"]
    assert e["intensity"] == pytest.approx(math.exp(0.1 + 2 * E * E - 0.5 * E ** 4), rel=1e-14)


# --------------------------------------------------------------------------
# EPW law for a perpendicular target (Sec. II-C) and its calibration fit
# --------------------------------------------------------------------------


def test_epw_law_and_fit(orc):
    pu = S.pulse(1024, 0.1e-9, 0.0, 4e-9, 6.0)
    T = 1e-5
    taps = orc.pulse_taps(pu)
    M = (len(taps) - 1) // 2
    sig = 4e-9 / (2 * math.sqrt(2 * math.log(2))) / 0.1e-9
    Zg = np.exp(-0.5 * (np.arange(-M, M + 1) / sig) ** 2).sum()
    sig_r = sig * 0.1e-9 * C / 2
    for a in (1e-3, 3e-2, 2.0):
        h = np.zeros(1024)
        h[500] = a  # point target at a bin centre
        xi = orc.convolve(h, taps)
        e = orc.extract_echoes(xi, pu, T)
        assert len(e) == 1
        law = 2 * sig_r * math.sqrt(2 * math.log(a / (T * Zg)))
        assert e[0]["epw_m"] == pytest.approx(law, abs=2e-3)
    coef = orc.fit_epw(pu, T)
    assert coef[1] == pytest.approx(1 / (8 * sig_r ** 2), rel=5e-3)
    assert coef[0] == pytest.approx(math.log(T * Zg), abs=0.02)
    assert abs(coef[2]) < 1e-3


# --------------------------------------------------------------------------
# whole beam model
# --------------------------------------------------------------------------

P1 = S.radial_profile(0.05, 1e-4, 0.05, 3.0, 1.0)
PU1 = S.pulse(1024, 0.1e-9, 0.0, 4e-9, 6.0)
CAL1 = S.calib(1e-5, 1e-4, 3, True)


def test_range_equation_perpendicular_and_tilted(orc):
    for R in (10.0, 5.0):
        gb = plane_gbuffer(np.array([1.0, 0, 0]), R, rho=0.5, amb=0.01)
        r = orc.simulate(gb, boresight(), P1, PU1, CAL1)
        E = r["h"][0].sum()
        assert E == pytest.approx(0.5 / (math.pi * R * R), rel=5e-5)
        # energy conservation through pulse and ambient
        assert r["xi"][0].sum() - 1024 * r["amb"][0] * 1e-4 == pytest.approx(E, rel=1e-11)
        assert r["amb"][0] == pytest.approx(0.01, rel=1e-5)
    th0 = 40 * DEG
    n = np.array([math.cos(th0), math.sin(th0), 0.0])
    gb = plane_gbuffer(n, 10.0 * math.cos(th0), rho=0.5)
    r = orc.simulate(gb, boresight(), P1, PU1, CAL1)
    assert r["h"][0].sum() == pytest.approx(0.5 / (math.pi * 100) * math.cos(th0), rel=2e-4)


def test_echo_time_two_r_over_c(orc):
    rng = S.rng(8)
    cal = S.calib(1e-5, 0.0, 3, True)
    for R in rng.uniform(1.5, 14.0, 6):
        gb = plane_gbuffer(np.array([1.0, 0, 0]), R, rho=0.5)
        r = orc.simulate(gb, boresight(), P1, PU1, cal)
        assert r["counts"][0] == 1
        e = r["echoes"][0][0]
        assert abs(e["range_m"] - R) < 1e-3
        X = 2 * R / C / 0.1e-9 - 0.5
        if abs(X - round(X)) < 0.45:
            assert e["bin_peak"] == int(math.floor(2 * R / C / 0.1e-9))


def _edge_scene(x_edge_az=None, el_edge=None, U=200, V=200, pitch_deg=0.02):
    """Plane at 10 m on one side of an edge, plane at 12 m elsewhere."""
    pitch = pitch_deg * DEG
    az0, el0 = -U * pitch / 2, -V * pitch / 2
    if x_edge_az is not None:
        ye = 10 * math.tan(x_edge_az)
        rect = S.Rect(np.array([10.0, ye - 50, 0.0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0]), 50, 50, 0.5)
    else:
        ze = 10 * math.tan(el_edge)
        rect = S.Rect(np.array([10.0, 0.0, ze - 50]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0]), 50, 50, 0.5)
    sc = S.Scene(planes=[S.Plane(np.array([1.0, 0, 0]), 12.0, 0.5)], rects=[rect], ambient="none")
    return S.raycast(sc, U, V, az0, el0, pitch, pitch)


def _split(r):
    h = r["h"][0]
    k12 = int(2 * 12 / C / 0.1e-9)
    EA, EB = h[: k12 - 30].sum(), h[k12 - 30:].sum()
    a, b = EA * 100, EB * 144  # undo 1/R^2 of each plane
    return a / (a + b)


@pytest.mark.parametrize("x0_sig", [0.0, 0.5, 1.0, -1.3])
def test_erf_split_at_depth_edge(orc, x0_sig):
    sig = 0.05
    prof = gauss_profile(sig, 0.6)
    pitch = 0.02 * DEG
    az_e = -100 * pitch + 100 * pitch  # pixel boundary at column 100
    gb = _edge_scene(x_edge_az=az_e)
    az_b = az_e - x0_sig * sig * DEG
    r = orc.simulate(gb, S._dirs_from_angles([az_b], [0.0]), prof, PU1, CAL1)
    # midpoint rule on the half line (-inf, x0]: sum = Phi(x0) - h^2/24 f'(x0)
    x0 = x0_sig * sig
    h = 0.02
    fprime = -x0 / sig ** 2 * math.exp(-0.5 * (x0 / sig) ** 2) / (sig * math.sqrt(2 * math.pi))
    expect = 0.5 * (1 + special.erf(x0 / (sig * math.sqrt(2)))) - h * h / 24 * fprime
    assert _split(r) == pytest.approx(expect, abs=3e-5)


def test_anisotropic_table_axes_and_roll(orc):
    # sigma_u along azimuth, sigma_v along elevation; a 90 deg roll swaps them
    su, sv = 0.05, 0.1
    tab = S.elliptic_gauss_table(81, 161, 0.01, su, sv)
    prof = S.table_profile(tab, 0.01)
    x0 = 0.04
    gba = _edge_scene(x_edge_az=0.0)
    gbe = _edge_scene(el_edge=0.0)
    Phi = lambda x, s: 0.5 * (1 + special.erf(x / (s * math.sqrt(2))))
    ra = orc.simulate(gba, S._dirs_from_angles([-x0 * DEG], [0.0]), prof, PU1, CAL1)
    re = orc.simulate(gbe, S._dirs_from_angles([0.0], [-x0 * DEG]), prof, PU1, CAL1)
    assert _split(ra) == pytest.approx(Phi(x0, su), abs=2e-3)
    assert _split(re) == pytest.approx(Phi(x0, sv), abs=2e-3)
    roll = S.pose_ypr(0.0, 0.0, math.pi / 2)
    ra2 = orc.simulate(gba, S._dirs_from_angles([0.0], [x0 * DEG]), prof, PU1, CAL1, pose=roll)
    # the sensor-frame elevation offset becomes a G-buffer azimuth offset
    assert _split(ra2) == pytest.approx(Phi(x0, sv), abs=2e-3)


def test_anisotropic_separable_axes_and_roll(orc):
    # the separable form of the same anisotropic Gaussian: sigma_u along
    # azimuth, sigma_v along elevation, swapped by a 90 deg roll
    su, sv = 0.05, 0.1
    prof = S.separable_gauss_tail(81, 161, 0.01, su, sv)
    x0 = 0.04
    gba = _edge_scene(x_edge_az=0.0)
    gbe = _edge_scene(el_edge=0.0)
    Phi = lambda x, s: 0.5 * (1 + special.erf(x / (s * math.sqrt(2))))
    ra = orc.simulate(gba, S._dirs_from_angles([-x0 * DEG], [0.0]), prof, PU1, CAL1)
    re = orc.simulate(gbe, S._dirs_from_angles([0.0], [-x0 * DEG]), prof, PU1, CAL1)
    assert _split(ra) == pytest.approx(Phi(x0, su), abs=2e-3)
    assert _split(re) == pytest.approx(Phi(x0, sv), abs=2e-3)
    roll = S.pose_ypr(0.0, 0.0, math.pi / 2)
    ra2 = orc.simulate(gba, S._dirs_from_angles([0.0], [x0 * DEG]), prof, PU1, CAL1, pose=roll)
    assert _split(ra2) == pytest.approx(Phi(x0, sv), abs=2e-3)


def test_ambient_only_sky(orc):
    gb = plane_gbuffer(None, 0, amb=2.0)
    r = orc.simulate(gb, boresight(), P1, PU1, S.calib(1e-5, 1e-6, 3, True))
    assert r["amb"][0] == pytest.approx(2.0, rel=1e-5)
    np.testing.assert_allclose(r["xi"][0], r["amb"][0] * 1e-6, rtol=1e-14)
    assert r["counts"][0] == 0 and r["h"][0].sum() == 0
    # ambient above the threshold: one run over the whole window, clipped both sides
    r = orc.simulate(gb, boresight(), P1, PU1, S.calib(1e-5, 1e-4, 3, True))
    e = r["echoes"][0][0]
    assert r["counts"][0] == 1 and e["bin_start"] == 0 and e["bin_end"] == 1023 and e["flags"] & 3 == 3


def test_pose_yaw_invariance(orc):
    w = S.small_plane_retro()
    k = 7
    psi = k * w.gbuffer.daz
    dirs = S._dirs_from_angles([0.003 - psi], [0.001])
    r0 = orc.simulate(w.gbuffer, S._dirs_from_angles([0.003], [0.001]), P1, PU1, CAL1)
    r1 = orc.simulate(w.gbuffer, dirs, P1, PU1, CAL1, pose=S.pose_ypr(psi, 0, 0))
    np.testing.assert_allclose(r1["h"], r0["h"], rtol=1e-5, atol=1e-12 * r0["h"].max())


def test_two_depths_give_two_echoes_nearest_first(orc):
    gb = _edge_scene(x_edge_az=0.0)
    r = orc.simulate(gb, boresight(), S.radial_profile(0.05, 1e-4, 0.05, 3, 1.0), PU1,
                     S.calib(1e-6, 0.0, 3, True))
    assert r["counts"][0] == 2
    e = r["echoes"][0]
    assert abs(e[0]["range_m"] - 10.0) < 2e-3 and abs(e[1]["range_m"] - 12.0) < 2e-3


def test_blooming_tail_reaches_retro(orc):
    # a retro patch 1 m in front of a plane; the beam core is 0.3 deg outside
    # the patch edge; the patch's echo energy equals the profile tail
    # integrated over the patch (scipy dblquad of the radial tail)
    g = 100.0
    patch = S.Rect(np.array([9.0, 0.0, 0.0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0]), 0.25, 0.25, 0.5, g)
    pitch = 0.02 * DEG
    U = 400
    sc = S.Scene(planes=[S.Plane(np.array([1.0, 0, 0]), 10.0, 0.5)], rects=[patch], ambient="none")
    gb = S.raycast(sc, U, U, -U * pitch / 2, -U * pitch / 2, pitch, pitch)
    edge = math.atan(0.25 / 9.0)
    az_b = edge + 0.3 * DEG
    r = orc.simulate(gb, S._dirs_from_angles([az_b], [0.0]), P1, PU1, CAL1)
    h = r["h"][0]
    k9, k10 = int(2 * 9 / C / 0.1e-9), int(2 * 10 / C / 0.1e-9)
    E_patch = h[: (k9 + k10) // 2].sum()
    Z = orc.profile_norm(P1) / (DEG * DEG)
    tail = lambda v, u: (1e-4 * min(1.0, (math.hypot(u, v) / 0.05) ** -3)
                         + math.exp(-0.5 * (u * u + v * v) / 0.05 ** 2)) if math.hypot(u, v) <= 1.0 else 0.0
    half = math.atan(0.25 / 9.0) / DEG
    integral = integrate.dblquad(tail, -2 * half - 0.3, -0.3, -half, half, epsrel=1e-6)[0]
    expect = (0.5 / math.pi + g) / 81.0 * integral / Z
    assert E_patch == pytest.approx(expect, rel=0.05)
    assert E_patch > 1e-3 * h.sum()  # blooming is visible


def test_brute_force_tiny(orc):
    # tiny G-buffer, a few beams: deposit by 20000-point supersampling of each
    # pixel's interval, pulse by numpy.convolve
    w = S.tiny_case()
    gb = w.gbuffer
    r = orc.simulate_workload(w)
    px = orc.pixels(gb)
    Z = orc.profile_norm(w.profile)
    dirs_px = gb.pixel_dirs().reshape(-1, 3)
    nb = w.pulse["n_bins"]
    taps = orc.pulse_taps(w.pulse)
    M = (len(taps) - 1) // 2
    ns = 20000
    frac = (np.arange(ns) + 0.5) / ns
    for b in range(len(w.dirs)):
        u, v, f = orc.offsets(w.pose, w.dirs[b], dirs_px)
        P = np.array([orc.profile_raw(w.profile, a, c)[0] if ok else 0.0 for a, c, ok in zip(u, v, f)]) / Z
        h = np.zeros(nb)
        A = 0.0
        for i in np.nonzero(P > 0)[0]:
            vv, uu = divmod(i, gb.U)
            A += P[i] * px["a"][vv, uu]
            if not px["hit"][vv, uu]:
                continue
            X0 = px["t0"][vv, uu] / 0.1e-9 - 0.5
            X1 = px["t1"][vv, uu] / 0.1e-9 - 0.5
            xs = X0 + (X1 - X0) * frac
            k0 = int(math.floor(X0)) - 1
            for k in range(max(0, k0), min(nb, int(math.ceil(X1)) + 2)):
                h[k] += P[i] * px["w"][vv, uu] * np.maximum(0, 1 - np.abs(xs - k)).mean()
        np.testing.assert_allclose(r["h"][b], h, rtol=1e-6, atol=1e-9 * h.max())
        assert r["amb"][b] == pytest.approx(A, rel=1e-12)
        xi = np.convolve(h, taps)[M:M + nb] + A * w.calib["ambient_scale"]
        np.testing.assert_allclose(r["xi"][b], xi, rtol=1e-6, atol=1e-9 * xi.max())


def test_golden_closed_forms(orc):
    """Constants derived by hand from the paper's equations (tests/golden)."""
    with open(os.path.join(GOLDEN, "closed_forms.json")) as f:
        g = json.load(f)
    gb = plane_gbuffer(np.array([1.0, 0, 0]), 10.0, rho=0.5)
    r = orc.simulate(gb, boresight(), P1, PU1, S.calib(1e-5, 0.0, 3, True))
    assert r["h"][0].sum() == pytest.approx(g["plane10m_rho05_energy"]["value"], rel=5e-5)
    e = r["echoes"][0][0]
    t_peak = 2 * e["range_m"] / C
    assert t_peak == pytest.approx(g["plane10m_echo_time_s"]["value"], abs=6e-12)
    assert orc.fit_epw(PU1, 1e-5)[1] == pytest.approx(g["epw_c1_per_m2"]["value"], rel=5e-3)
    taps = orc.pulse_taps(PU1)
    assert len(taps) == g["pulse_taps_4ns_0p1ns"]["value"]


def test_strongest_echo_selection(orc):
    """The single-return selection (LIDAR_ECHOES_STRONGEST): of three point
    targets the calibrated intensities follow the amplitudes (the EPW law), so
    the strongest echo is the largest target's; of two equal targets, the
    nearer one; no echo, no selection."""
    pu = S.pulse(1024, 0.1e-9, 0.0, 4e-9, 6.0)
    T = 1e-5
    taps, coef = orc.pulse_taps(pu), orc.fit_epw(pu, T)
    h = np.zeros(1024)
    h[200], h[500], h[800] = 3e-3, 2e-2, 8e-3
    e = orc.extract_echoes(orc.convolve(h, taps), pu, T, coef)
    assert [x["bin_peak"] for x in e] == [200, 500, 800]
    assert e[1]["intensity"] > e[2]["intensity"] > e[0]["intensity"]
    s = orc.strongest_echo(e)
    assert len(s) == 1 and s[0]["bin_peak"] == 500 and s[0]["intensity"] == e[1]["intensity"]
    # equal intensities: the nearer echo
    e2 = np.zeros(3, e.dtype)
    e2["bin_peak"] = [100, 300, 700]
    e2["intensity"] = [0.5, 2.0, 2.0]
    assert orc.strongest_echo(e2)[0]["bin_peak"] == 300
    assert len(orc.strongest_echo(orc.extract_echoes(np.zeros(64), PU, 1.0))) == 0
