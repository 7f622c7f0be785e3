"""Pins of the FP64 statement of Alg. 2 (range stacking; oracle/lidar_oracle.c
orc_range_stack) against SciPy's 2-D convolution, closed forms for single
pixels, the nearest-slice rule and the per-pixel inputs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_05932_gb300 import scenes as S

signal = pytest.importorskip("scipy.signal")


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def test_single_pixel_reproduces_the_kernel():
    I = np.zeros((9, 11))
    I[4, 5] = 2.0
    rb = np.full((9, 11), -1, np.int32)
    rb[4, 5] = 3
    K = np.arange(15, dtype=float).reshape(3, 5) + 1
    S_, X = O.range_stack(I, rb, K, 6.0, 10)
    expect = np.zeros((9, 11))
    expect[3:6, 3:8] = 2 * K                      # impulse response = the kernel
    above = expect >= 6.0                          # ">=": the value 6 itself counts
    assert above.sum() == 13
    np.testing.assert_array_equal(S_, np.where(above, 3, 10))
    np.testing.assert_allclose(X, np.where(above, expect, 0.0), rtol=0, atol=0)


def test_nearest_slice_wins_where_it_reaches_the_threshold():
    I = np.zeros((7, 20))
    rb = np.full((7, 20), -1, np.int32)
    I[3, 6], rb[3, 6] = 1.0, 8      # far surface
    I[3, 9], rb[3, 9] = 1.0, 2      # near surface, 3 px to the right
    K = np.ones((3, 7))             # reaches +-3 columns
    S_, X = O.range_stack(I, rb, K, 0.5, 12)
    # columns 6..12 are within reach of the near pixel -> slice 2
    assert (S_[2:5, 6:13] == 2).all() and (X[2:5, 6:13] == 1.0).all()
    # columns 3..5 only see the far pixel -> slice 8
    assert (S_[2:5, 3:6] == 8).all()
    # nothing else
    assert (S_[:, :3] == 12).all() and (S_[:, 13:] == 12).all() and (X[0] == 0).all()


@pytest.mark.parametrize("seed", [0, 1])
def test_matches_scipy_convolution_per_slice(seed):
    g = np.random.default_rng(seed)
    V, U, s_max = 13, 17, 6
    I = g.uniform(0, 1, (V, U))
    rb = g.integers(-1, s_max + 2, (V, U)).astype(np.int32)  # includes slices 0 and > s_max (never used)
    K = g.uniform(0, 1, (5, 3))
    thr = 1.2
    S_, X = O.range_stack(I, rb, K, thr, s_max)
    S_ref = np.full((V, U), s_max, np.int32)
    X_ref = np.zeros((V, U))
    for s in range(s_max, 0, -1):
        conv = signal.convolve2d(np.where(rb == s, I, 0.0), K, mode="same")
        hit = conv >= thr
        S_ref[hit] = s
        X_ref[hit] = conv[hit]
    np.testing.assert_array_equal(S_, S_ref)
    np.testing.assert_allclose(X, X_ref, rtol=1e-12, atol=1e-15)


def test_inputs_are_pixel_power_and_floor_range():
    w = S.tiny_case()
    dr = 0.05
    I, rb = O.stack_inputs(w.gbuffer, dr)
    px = O.pixels(w.gbuffer)
    hit = px["hit"].astype(bool)
    np.testing.assert_allclose(I[hit], px["w"][hit], rtol=0)
    assert (I[~hit] == 0).all() and (rb[~hit] == -1).all()
    r = w.gbuffer.range.astype(np.float64)
    np.testing.assert_array_equal(rb[hit], np.floor(r[hit] / dr).astype(np.int32))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_pixel_entry_equals_whole_image_sweep(seed):
    """range_stack_at (one output pixel at a time, for sampled checks at full
    size) gives exactly range_stack's slice and value at every pixel, with the
    nearest-to-threshold distance consistent with the answer."""
    g = np.random.default_rng(10 + seed)
    V, U, s_max = 11, 14, 7
    I = g.uniform(0, 1, (V, U))
    rb = g.integers(-1, s_max + 2, (V, U)).astype(np.int32)
    K = g.uniform(0, 1, (5, 7))
    thr = 1.1
    S_, X = O.range_stack(I, rb, K, thr, s_max)
    vv, uu = np.meshgrid(np.arange(V), np.arange(U), indexing="ij")
    S1, X1, close = O.range_stack_at(I, rb, K, thr, s_max, vv.ravel(), uu.ravel())
    np.testing.assert_array_equal(S1.reshape(V, U), S_)
    np.testing.assert_array_equal(X1.reshape(V, U), X)
    hit = X1 > 0
    assert (close[hit] <= np.abs(X1[hit] / thr - 1) + 1e-15).all()


def test_alg2_nearest_slice_equals_alg1_nearest_bin_for_a_pixel_centred_beam():
    """Alg. 1 and Alg. 2 agree within floating-point limits (Sec. II-C) where
    they compute the same thing: a beam through a pixel centre, range slices
    equal to the histogram's bins (slice = floor(R / dr), dr = c dt / 2), every
    pixel's return confined to one bin (surfaces facing the sensor at bin-centre
    ranges, so the ToF interval is a point up to the corner rays' 1e-5 bins),
    and the Alg. 2 kernel equal to the beam's profile weights at the pixels. Then
    Alg. 2's nearest slice at the beam's pixel, for any threshold, is Alg. 1's
    nearest histogram bin at or above it, and its value is that bin's value."""
    C_LIGHT = 299_792_458.0
    pitch = 0.02 * np.pi / 180
    n = 61
    c0 = n // 2
    pu = S.pulse(1024, 0.1e-9)
    dr = 0.5 * C_LIGHT * pu["dt_s"]
    gb = S.GBuffer(n, n, -n * pitch / 2, -n * pitch / 2, pitch, pitch, *[None] * 7)
    d = gb.pixel_dirs()
    vv, uu = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    # three surfaces at the centres of bins 500, 600 and 700 (a near strip to
    # the left of the beam, a far block below it, the middle elsewhere) and a
    # few pixels without a hit
    k = np.full((n, n), 600)
    k[:, :c0 - 8] = 500
    k[:c0 - 5, c0 - 8:] = 700
    rng_m = (k + 0.5) * dr
    rng_m[(vv - c0) ** 2 + (uu - c0 - 12) ** 2 < 9] = np.inf
    gb.range = rng_m.astype(np.float32)
    gb.nx, gb.ny, gb.nz = (d[..., i].astype(np.float32) for i in range(3))
    gb.rho_d = np.full((n, n), 0.5, np.float32)
    gb.retro = np.zeros((n, n), np.float32)
    gb.ambient = np.zeros((n, n), np.float32)
    prof = S.radial_profile(0.1, 1e-3, 0.1, 3.0, 0.6)
    beam = d[c0, c0][None, :].astype(np.float32)
    cal = S.calib(1e-5, 0.0, 3, True)
    h = O.simulate(gb, beam, prof, pu, cal)["h"][0]
    # the Alg. 2 kernel: the beam's weight at pixel (c0 - i, c0 - j) is K[m + i][n + j]
    u, v, front = O.offsets(np.eye(3), beam[0], d.reshape(-1, 3))
    Pb = np.where(front, O.profile_raw(prof, u, v), 0.0).reshape(n, n) / O.profile_norm(prof)
    K = Pb[::-1, ::-1].copy()
    I, rb = O.stack_inputs(gb, dr)
    assert set(np.unique(rb[rb >= 0])) == {500, 600, 700}
    s_max = 1000
    bins = [500, 600, 700]
    assert all(h[b] > 0 for b in bins)
    levels = sorted(h[b] for b in bins)
    thrs = [0.5 * levels[0]] + [0.5 * (a + b) for a, b in zip(levels, levels[1:])] + [2.0 * levels[-1]]
    for thr in thrs:
        S1, X1, _ = O.range_stack_at(I, rb, K, thr, s_max, np.array([c0]), np.array([c0]))
        above = np.nonzero(h[1:s_max + 1] >= thr)[0]
        if len(above) == 0:
            assert S1[0] == s_max and X1[0] == 0.0
        else:
            kk = 1 + int(above[0])
            assert S1[0] == kk, (thr, S1[0], kk)
            assert X1[0] == pytest.approx(h[kk], rel=1e-4)
