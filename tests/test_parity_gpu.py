"""Parity of the sm_103a library (through the C ABI) with the FP64 oracle.

Bar (per beam): waveform relative L2 error <= 1e-3; echo counts and bins
(start, end, peak) bit-exact; echo range and EPW within 1 mm; intensity and
peak within 1e-3 relative (oracle/parity.py).

Guard band. The echo scan compares bins with the threshold T strictly; an
echo whose run or its two neighbouring bins hold an oracle value within
BAND * T of T may legitimately differ in FP32, so it is left out of the
bit-exact comparison (the echo alone, not its beam), counted, and must stay
at or below 0.1 % of the compared echoes. BAND = 1e-5 lies above the largest
deviation between the GPU waveform and the oracle's at bins near T that the
full-size workloads show (2.3e-6 T on the full frame, 7.4e-6 T on the
wide-tail frame), so an echo outside the band cannot flip. For beams with an
ambiguous echo the echo extraction is still checked exactly, by running the
FP64 extraction on the GPU's own waveform.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle import parity as PR
from paper_2512_05932_gb300 import lidar
from paper_2512_05932_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
DEG = math.pi / 180


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run_gpu(w, host=False, deposit=0):
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    lidar.lidar_set_deposit(L.handle, deposit)
    if host:
        # pinned planes (read by the set-up kernel where they lie) or pageable
        # ones (copied up); pinned outputs (asynchronous copies) or pageable
        # ones (staged by the driver)
        planes = [torch.from_numpy(np.ascontiguousarray(p)) for p in w.gbuffer.planes()]
        if host != "pageable_planes":
            planes = [p.pin_memory() for p in planes]
        outs = None
        if host == "pageable":
            outs = (torch.empty((L.n_beams, L.n_bins), dtype=torch.float32),
                    torch.empty((L.n_beams, L.max_echoes, 8), dtype=torch.int32),
                    torch.empty((L.n_beams,), dtype=torch.int32))
        wave, ech, cnt = L.simulate_host(w.gbuffer, planes, w.pose, outs)
    else:
        planes = lidar.gbuffer_to_device(w.gbuffer)
        wave, ech, cnt = L.simulate(w.gbuffer, planes, w.pose)
        torch.cuda.synchronize()
    lidar.lidar_sync(L.handle, 0)
    return L, wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech), cnt.cpu().numpy()


def check_own_waveform(b, wave_b, ech_b, cnt_b, pulse, T, coef, max_echoes):
    """Echo logic alone: the FP64 extraction run on the GPU's own (float32)
    waveform must give the same echo bins as the GPU."""
    T32 = float(np.float32(T))
    e = O.extract_echoes(wave_b, pulse, T32, coef, max_out=8)
    n = min(len(e), max_echoes)
    assert cnt_b == n, (b, cnt_b, n)
    for i in range(n):
        g = ech_b[i]
        assert (g["bin_start"], g["bin_end"]) == (e[i]["bin_start"], e[i]["bin_end"]), (b, i, g, e[i])
        if not (e[i]["flags"] & O.PEAK_AMBIGUOUS):
            assert g["bin_peak"] == e[i]["bin_peak"], (b, i, g, e[i])
        assert abs(g["epw_m"] - e[i]["epw_m"]) <= 1e-4 and abs(g["range_m"] - e[i]["range_m"]) <= 1e-4


BAND = 1e-5
MAX_AMBIGUOUS = 1e-3  # fraction of the compared echoes


def ambiguous_ok(st, strict=False):
    """At most 0.1 % of the compared echoes are ambiguous; a check on fewer
    than 1000 echoes may have one (strict: the 0.1 % alone, for the large
    samples of the full-size workloads)."""
    lim = MAX_AMBIGUOUS * st["echoes"]
    return st["ambiguous"] <= (lim if strict else max(1.0, lim))


def compare(ref, wave, ech, cnt, beams, T, max_echoes, pulse=None, tol_l2=1e-3):
    st, fails = PR.compare_frame(ref, beams, wave, ech, cnt, T, max_echoes, BAND, tol_l2)
    assert not fails, fails[:10]
    # beams with an echo in the band: the extraction itself, on the GPU's waveform
    for s, b in enumerate(beams):
        if np.any(np.abs(ref["xi"][s] - T) <= BAND * T):
            check_own_waveform(b, wave[b], ech[b], cnt[b], pulse, T, ref["coef"], max_echoes)
    return st


def check_workload(w, beams=None, host=False, deposit=0, strict=False):
    L, wave, ech, cnt = run_gpu(w, host, deposit)
    if beams is None:
        beams = np.arange(len(w.dirs), dtype=np.int32)
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    info = lidar.lidar_get_info(L.handle)
    assert info["profile_norm"] == pytest.approx(ref["Z"], rel=1e-7)
    np.testing.assert_allclose(info["epw_coef"], ref["coef"], rtol=1e-9, atol=1e-12)
    st = compare(ref, wave, ech, cnt, beams, w.calib["threshold"], w.calib["max_echoes"], w.pulse)
    assert ambiguous_ok(st, strict), st
    L.close()
    return st


# --------------------------------------------------------------------------


def test_small_plane_retro_all_beams():
    # seeded so that no bin lies within 7e-4 T of T: every echo is compared
    st = check_workload(S.small_plane_retro())
    assert st["echoes"] >= 500 and st["ambiguous"] == 0


def test_tiny_ragged_rolled_pose():
    check_workload(S.tiny_case())


@pytest.mark.parametrize("host", ["pinned", "pageable"])
def test_tiny_host_entry_point(host):
    check_workload(S.tiny_case(), host=host)


def test_full_frame_sampled_beams():
    """The benchmarked full frame on 1024 evenly spaced beams (the sample the
    benchmark checks) plus the first, last and row-end beams."""
    w = S.full_frame_boxes()
    n = len(w.dirs)
    beams = np.unique(np.concatenate([np.linspace(0, n - 1, 1024).astype(np.int64),
                                      [0, 1, 1599, 1600, n // 2, n - 1600, n - 1]])).astype(np.int32)
    st = check_workload(w, beams=beams, strict=True)
    assert st["echoes"] >= 500, st


@pytest.mark.parametrize("host", ["pinned", "pageable", "pageable_planes"])
def test_full_frame_host_entry_point_matches_device_entry_point(host):
    """The host-memory entry point pipelines a large frame (bands of rows set
    up as they arrive, launches on two streams whose results are copied back
    while later ones run), with pinned planes read in place or pageable ones
    copied up, into pinned or pageable outputs: same waveforms (up to the FP32
    order of the deposits), echoes and counts as the device entry point on the
    same frame."""
    w = S.full_frame_boxes()
    _, wave_d, ech_d, cnt_d = run_gpu(w)
    _, wave_h, ech_h, cnt_h = run_gpu(w, host=host)
    rel = np.linalg.norm(wave_h - wave_d, axis=1) / np.maximum(np.linalg.norm(wave_d, axis=1), 1e-30)
    assert rel.max() <= 1e-5, rel.max()
    assert (cnt_h == cnt_d).mean() >= 0.999
    same = cnt_h == cnt_d
    for k in ("bin_start", "bin_end"):
        a, b = ech_h[k][same], ech_d[k][same]
        assert (a == b).mean() >= 0.999, k


def test_full_frame_host_entry_point_tensor_core_deposit():
    """The pipelined host path with the tensor-core deposit (its own beams per
    CTA and launch shape): the device entry point's results in the same mode."""
    w = S.full_frame_boxes()
    _, wave_d, ech_d, cnt_d = run_gpu(w, deposit=1)
    _, wave_h, ech_h, cnt_h = run_gpu(w, host="pinned", deposit=1)
    rel = np.linalg.norm(wave_h - wave_d, axis=1) / np.maximum(np.linalg.norm(wave_d, axis=1), 1e-30)
    assert rel.max() <= 1e-5, rel.max()
    assert (cnt_h == cnt_d).mean() >= 0.999


def test_ragged_large_frame_host_entry_point():
    """A frame whose rows do not split evenly into the host path's upload bands
    and whose beams do not fill the last group (25 597 beams on 2000x999): the
    banded upload, per-band set-up and chunked launches on two streams give
    the device entry point's results."""
    w = S.full_frame_boxes(U=2000, V=999)
    w.dirs = w.dirs[:25597]
    _, wave_d, ech_d, cnt_d = run_gpu(w)
    _, wave_h, ech_h, cnt_h = run_gpu(w, host="pinned")
    rel = np.linalg.norm(wave_h - wave_d, axis=1) / np.maximum(np.linalg.norm(wave_d, axis=1), 1e-30)
    assert rel.max() <= 1e-5, rel.max()
    assert (cnt_h == cnt_d).mean() >= 0.999
    same = cnt_h == cnt_d
    for k in ("bin_start", "bin_end"):
        assert (ech_h[k][same] == ech_d[k][same]).mean() >= 0.999, k


def test_host_entry_point_right_after_another_frame():
    """The host path starts each beam chunk once the rows its beams can reach
    are set up: run right after a different frame (whose per-pixel records
    are still in the scratch), it gives the device path's results on the same
    frame, so no chunk reads a row before its set-up."""
    wa, wb = S.full_frame_boxes(seed=2), S.full_frame_boxes(seed=9)
    L = lidar.Lidar(wa.profile, wa.dirs, wa.pulse, wa.calib)
    pa, pb = lidar.gbuffer_to_device(wa.gbuffer), lidar.gbuffer_to_device(wb.gbuffer)
    wave_d, ech_d, cnt_d = L.simulate(wa.gbuffer, pa, wa.pose)
    wave_d, ech_d, cnt_d = wave_d.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech_d), cnt_d.cpu().numpy()
    hp = [torch.from_numpy(np.ascontiguousarray(p)).pin_memory() for p in wa.gbuffer.planes()]
    for _ in range(2):
        L.simulate(wb.gbuffer, pb, wb.pose)
        torch.cuda.synchronize()
        wave_h, ech_h, cnt_h = L.simulate_host(wa.gbuffer, hp, wa.pose)
        wave_h, ech_h, cnt_h = wave_h.numpy().astype(np.float64), lidar.echoes_numpy(ech_h), cnt_h.numpy()
        rel = np.linalg.norm(wave_h - wave_d, axis=1) / np.maximum(np.linalg.norm(wave_d, axis=1), 1e-30)
        assert rel.max() <= 1e-5, rel.max()
        assert (cnt_h == cnt_d).mean() >= 0.999
    L.close()


def test_table_profile_anisotropic_with_roll():
    w = S.small_plane_retro()
    w.profile = S.table_profile(S.elliptic_gauss_table(41, 81, 0.01, 0.05, 0.1), 0.01)
    w.pose = S.pose_ypr(0.001, 0.002, 0.6)
    check_workload(w, beams=np.arange(0, 512, 3, dtype=np.int32))


@pytest.mark.parametrize("deposit", [0, 1])
def test_separable_profile_anisotropic_with_roll_and_tail(deposit):
    """Separable profile H(u) V(v) (two 1-D tables, sigma 0.05 / 0.1 deg with a
    power-law tail on each axis) under a rolled pose, in the atomic and the
    tensor-core deposit forms."""
    w = S.small_plane_retro()
    w.profile = S.separable_gauss_tail(61, 101, 0.01, 0.05, 0.1, tail_amp=1e-3)
    w.pose = S.pose_ypr(0.001, 0.002, 0.6)
    st = check_workload(w, beams=np.arange(0, 512, 3, dtype=np.int32), deposit=deposit)
    assert st["echoes"] > 100


def test_separable_equals_outer_product_table_on_gpu():
    """The separable kernel path and the table path on the outer-product
    table give the same waveforms up to FP32 rounding."""
    w = S.small_plane_retro()
    prof = S.separable_gauss_tail(41, 81, 0.01, 0.05, 0.1, tail_amp=1e-3)
    w.profile = prof
    _, wave_s, _, cnt_s = run_gpu(w)
    w.profile = S.table_profile(np.outer(prof["v"].astype(np.float64), prof["h"].astype(np.float64)), 0.01)
    _, wave_t, _, cnt_t = run_gpu(w)
    rel = np.linalg.norm(wave_s - wave_t, axis=1) / np.maximum(np.linalg.norm(wave_t, axis=1), 1e-30)
    assert rel.max() <= 1e-5, rel.max()
    assert (cnt_s == cnt_t).mean() >= 0.99


def test_ragged_beam_count_and_min_bins():
    w = S.tiny_case(n_beams=37, n_bins=32)
    w.pulse = S.pulse(32, 1e-9, 2.0e-8, 4e-9, 3.0)
    check_workload(w)


@pytest.mark.parametrize("me", [1, 2])
def test_max_echoes(me):
    w = S.tiny_case()
    w.calib = dict(w.calib, max_echoes=me)
    check_workload(w)


def test_given_epw_coefficients():
    w = S.tiny_case()
    w.calib = dict(w.calib, fit_epw=0, epw_coef=(0.3, 1.5, -0.2))
    check_workload(w)


def test_sky_only_and_ambient_only():
    w = S.tiny_case()
    gb = w.gbuffer
    gb.range[:] = np.inf
    gb.ambient[:] = 0
    L, wave, ech, cnt = run_gpu(w)
    assert (wave == 0).all() and (cnt == 0).all()
    gb.ambient[:] = 0.5
    check_workload(w)


def test_beams_outside_gbuffer():
    w = S.tiny_case()
    w.dirs = S._dirs_from_angles([0.0, 0.5, -0.5, 0.0, 3.0], [0.0, 0.0, 0.0, 1.2, 0.0])
    L, wave, ech, cnt = run_gpu(w)
    assert (wave[1:] == 0).all() and (cnt[1:] == 0).all()
    check_workload(w)


def test_single_pixel_gbuffer():
    w = S.tiny_case()
    sc = S.Scene(planes=[S.Plane(np.array([1.0, 0, 0]), 5.0, 0.5, 10.0)], ambient="uniform", ambient_level=0.1)
    w.gbuffer = S.raycast(sc, 1, 1, -0.2 * DEG, -0.2 * DEG, 0.4 * DEG, 0.4 * DEG)
    w.dirs = S._dirs_from_angles([0.0, 0.05 * DEG], [0.0, -0.1 * DEG])
    w.pose = S.IDENTITY_POSE.copy()
    check_workload(w)


def test_panorama_wraps_at_seam():
    # full 360 deg G-buffer; beams straddling the +-180 deg seam and near the pole
    pitch = 0.5 * DEG
    U, V = 720, 200
    sc = S.Scene(planes=[S.Plane(np.array([-1.0, 0.0, 0.0]), 6.0, 0.5),
                         S.Plane(np.array([0.0, 0.0, 1.0]), -2.0, 0.3)], ambient="uniform", ambient_level=0.01)
    gb = S.raycast(sc, U, V, -math.pi, -50 * DEG, pitch, pitch)
    dirs = S._dirs_from_angles([math.pi - 0.3 * DEG, -math.pi + 0.2 * DEG, math.pi, 1.0, 0.5],
                               [0.0, -0.5 * DEG, -20 * DEG, -45 * DEG, 45 * DEG])
    prof = S.radial_profile(0.8, 1e-3, 0.8, 3.0, 4.0)
    w = S.Workload("pano", gb, dirs, prof, S.pulse(512, 0.2e-9), S.calib(1e-6, 1e-5, 3, True))
    check_workload(w)


def test_gbuffer_across_the_azimuth_seam():
    """A G-buffer (not a panorama) whose azimuth range crosses +-180 deg, seen
    by a sensor facing backwards: beams on both sides of the seam."""
    base = S.small_plane_retro()
    R = S.pose_ypr(math.pi, 0.01, 0.0)
    gb = S.plane_retro_frame(S.rng(21), 320, 160, R)
    assert gb.az0 < math.pi < gb.az0 + gb.U * gb.daz
    dirs = S.grid_pattern(24, 10, 5.0 * DEG, 2.5 * DEG)
    w = S.Workload("seam", gb, dirs, base.profile, base.pulse, base.calib, R)
    st = check_workload(w)
    assert st["echoes"] >= 200, st


def test_yaw_pose_matches_rotated_pattern():
    w = S.small_plane_retro()
    L, wave0, _, cnt0 = run_gpu(w)
    psi = 5 * w.gbuffer.daz
    R = S.pose_ypr(psi, 0, 0)
    w2 = S.Workload(w.name, w.gbuffer, (w.dirs.astype(np.float64) @ R.astype(np.float64)).astype(np.float32),
                    w.profile, w.pulse, w.calib, R)
    L2, wave1, _, cnt1 = run_gpu(w2)
    err = np.linalg.norm(wave1 - wave0, axis=1) / np.linalg.norm(wave0, axis=1)
    assert err.max() < 1e-4 and (cnt0 == cnt1).all()


def test_scratch_grows_with_larger_gbuffer():
    w = S.tiny_case()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    for size in ((11, 9), (37, 29), (64, 48)):
        big = S.tiny_case(U=size[0], V=size[1])
        planes = lidar.gbuffer_to_device(big.gbuffer)
        wave, ech, cnt = L.simulate(big.gbuffer, planes, big.pose)
        torch.cuda.synchronize()
        ref = O.simulate(big.gbuffer, w.dirs, w.profile, w.pulse, w.calib, big.pose, nthreads=NTHREADS)
        got = wave.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(got - ref["xi"], axis=1) / np.linalg.norm(ref["xi"], axis=1)
        assert err.max() <= 1e-3
    L.close()


def test_invalid_gbuffer_rejected_on_device_call():
    w = S.tiny_case()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    bad = S.GBuffer(w.gbuffer.U, w.gbuffer.V, 0.0, 0.0, 1.0, 0.01, *w.gbuffer.planes())
    with pytest.raises(lidar.LidarError, match="azimuth span"):
        L.simulate(bad, planes, w.pose)
    with pytest.raises(lidar.LidarError, match="orthonormal"):
        L.simulate(w.gbuffer, planes, np.diag([1.0, 2.0, 1.0]))
    L.close()


def test_wide_tail_frame_sampled_beams():
    """8192x4096 G-buffer, 200k beams, tail truncated at 2 deg, 4096 bins of
    0.05 ns: the full-size instance on a seeded 1 % subsample (2000 beams)."""
    w = S.wide_frame()
    n = len(w.dirs)
    beams = np.sort(S.rng(2000).choice(n, 2000, replace=False)).astype(np.int32)
    st = check_workload(w, beams=beams, strict=True)
    assert st["echoes"] >= 1000, st


def test_spread_beams_walk_their_own_boxes():
    """A coarse grid of 3 200 beams whose footprints (radial profile cut at
    0.5 deg: boxes about 21 pixels wide) lie 13 pixels apart: a group of 8
    neighbouring beams shares little of its union box, so each beam walks its
    own box, shifted inside the G-buffer where it reaches an edge. The corner
    and edge beams and a random sample against the oracle."""
    pitch = 0.05 * DEG
    U, V = 1024, 512
    n = np.array([-1.0, 0.3, 0.2])
    n /= np.linalg.norm(n)
    patch = S.Rect(np.array([8.0, 0.5, 0.3]), np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]),
                   0.4, 0.3, rho_d=0.3, retro=100.0)
    scene = S.Scene(planes=[S.Plane(n, -9.0, 0.4, 0.0)], rects=[patch], ambient="uniform",
                    ambient_level=0.01)
    gb = S.raycast(scene, U, V, -U * pitch / 2, -V * pitch / 2, pitch, pitch)
    dirs = S.grid_pattern(80, 40, U * pitch, V * pitch)
    w = S.Workload("spread_grid_1024x512_3200beams", gb, dirs, S.radial_profile(trunc_deg=0.5),
                   S.pulse(1024, 0.1e-9), S.calib(1e-5, 1e-4, 3, True))
    g = S.rng(21)
    edges = [0, 1, 79, 80, 3119, 3120, 3198, 3199] + list(range(0, 3200, 80)) + list(range(79, 3200, 80))
    beams = np.unique(np.concatenate([edges, g.choice(3200, 120, replace=False)])).astype(np.int32)
    st = check_workload(w, beams=beams)
    assert st["echoes"] >= 100
