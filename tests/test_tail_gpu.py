"""Core/tail split (include/lidar_tail.h) against the FP64 oracle.

The oracle's tail of a beam is its full histogram minus the histogram of the
same profile cut at the core radius (same normalisation Z). The split path must
(1) reproduce that tail exactly when asked for it (lidar_tail_exact), (2) bound
it from above (the acceptance test relies on that bound), and (3) with any
tail estimate that respects the bound, give waveforms and echoes that meet the
parity bar of the plain path, because beams that cannot be guaranteed are
re-run exactly."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_05932_gb300 import lidar
from paper_2512_05932_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


class Split:
    def __init__(self, w, core_deg, n_coarse):
        self.w = w
        self.L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
        lidar.lidar_tail_configure(self.L.handle, core_deg, n_coarse)
        self.nc = n_coarse
        self.planes = lidar.gbuffer_to_device(w.gbuffer)
        self.g = lidar.make_gbuffer(w.gbuffer, [p.data_ptr() for p in self.planes])
        self.pose = lidar.make_pose(w.pose)
        self.s = torch.cuda.current_stream().cuda_stream

    def rows(self):
        return torch.zeros((self.L.n_beams, self.nc + 4), dtype=torch.float32, device="cuda")

    def features(self, inputs=False):
        r = self.rows()
        x = None
        if inputs:
            x = torch.empty((self.L.n_beams, lidar.TAIL_INPUT_CELLS, 2), dtype=torch.float16, device="cuda")
        lidar.lidar_tail_features(self.L.handle, self.g, self.pose, r.data_ptr(), x.data_ptr() if x is not None else 0,
                                  self.s)
        torch.cuda.synchronize()
        return r, x

    def exact(self):
        r = self.rows()
        lidar.lidar_tail_exact(self.L.handle, self.g, self.pose, r.data_ptr(), self.s)
        torch.cuda.synchronize()
        return r

    def split(self, tail):
        wave, ech, cnt = self.L.alloc_outputs()
        wave.fill_(float("nan"))
        cnt.fill_(-1)
        n = lidar.lidar_simulate_split(self.L.handle, self.g, self.pose, tail.data_ptr(), wave.data_ptr(),
                                       ech.data_ptr(), cnt.data_ptr(), self.s)
        torch.cuda.synchronize()
        lidar.lidar_sync(self.L.handle, 0)
        return n, (wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech), cnt.cpu().numpy())

    def close(self):
        self.L.close()


def oracle_tail(w, core_deg, beams):
    """FP64 tail histogram and ambient tail of the selected beams."""
    full = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    core_prof = dict(w.profile, trunc_deg=core_deg)
    core = O.simulate(w.gbuffer, w.dirs, core_prof, w.pulse, w.calib, w.pose, beams, NTHREADS, 8, Z=full["Z"])
    return full, full["h"] - core["h"], full["amb"] - core["amb"]


def coarse(h, nc):
    return h.reshape(h.shape[0], nc, -1).sum(axis=2)


def parity(w, res, beams):
    from tests.test_parity_gpu import ambiguous_ok, compare
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    wave, ech, cnt = res
    st = compare(ref, wave, ech, cnt, beams, w.calib["threshold"], w.calib["max_echoes"], w.pulse)
    assert ambiguous_ok(st), st
    return st


CORE_SMALL = 0.3


def test_exact_tail_and_bounds_small_instance():
    w = S.small_plane_retro()
    sp = Split(w, CORE_SMALL, 256)
    beams = np.arange(len(w.dirs), dtype=np.int32)
    full, th, ta = oracle_tail(w, CORE_SMALL, beams)
    ex = sp.exact().cpu().numpy().astype(np.float64)
    tc = coarse(th, 256)
    tot = th.sum(axis=1)
    assert (tot > 0).all()
    # exact tail: coarse bins and total within FP32 accumulation noise
    err = np.abs(ex[:, :256] - tc).sum(axis=1) / tot
    assert err.max() <= 2e-4, err.max()
    np.testing.assert_allclose(ex[:, 256], ta, rtol=2e-4)
    np.testing.assert_allclose(ex[:, 259], tot, rtol=2e-4)
    # the bounds of the features hold for every beam
    fr, _ = sp.features()
    fr = fr.cpu().numpy().astype(np.float64)
    assert (fr[:, 257] >= tot).all(), np.min(fr[:, 257] / tot)
    assert (np.abs(fr[:, 256] - ta) <= fr[:, 258] * (1 + 1e-6) + 1e-30).all()
    # the prior is a tail estimate: non-negative, within the bound, mass within a factor 2
    assert (fr[:, :256] >= 0).all() and (fr[:, 259] <= fr[:, 257] * (1 + 1e-6)).all()
    ratio = fr[:, 259] / tot
    assert 0.5 <= np.median(ratio) <= 2.0, np.median(ratio)
    sp.close()


def test_split_with_prior_meets_parity_small_instance():
    w = S.small_plane_retro()
    sp = Split(w, CORE_SMALL, 256)
    fr, _ = sp.features()
    n, res = sp.split(fr)
    st = parity(w, res, np.arange(len(w.dirs), dtype=np.int32))
    assert st["echoes"] >= 500
    assert 0 <= n < len(w.dirs)
    sp.close()


@pytest.mark.parametrize("kind", ["zero", "misplaced"])
def test_split_with_wrong_tail_still_meets_parity(kind):
    """Tails that respect the bound but are wrong (none, or all mass in one
    far coarse bin) must still give oracle-exact results: the acceptance test
    re-runs every beam it cannot guarantee."""
    w = S.small_plane_retro()
    sp = Split(w, CORE_SMALL, 256)
    fr, _ = sp.features()
    t = fr.clone()
    t[:, :256] = 0
    if kind == "misplaced":
        g = torch.Generator(device="cpu").manual_seed(5)
        col = torch.randint(0, 256, (len(w.dirs),), generator=g).cuda()
        t[torch.arange(len(w.dirs), device="cuda"), col] = 0.99 * fr[:, 257]
    t[:, 259] = t[:, :256].sum(dim=1)
    n, res = sp.split(t)
    parity(w, res, np.arange(len(w.dirs), dtype=np.int32))
    sp.close()


def test_split_tiny_rolled_ragged():
    w = S.tiny_case(n_beams=37, n_bins=256)
    sp = Split(w, 0.15, 64)
    fr, x = sp.features(inputs=True)
    assert torch.isfinite(x.float()).all()
    n, res = sp.split(fr)
    parity(w, res, np.arange(len(w.dirs), dtype=np.int32))
    sp.close()


def test_split_wide_frame_sampled():
    """The 8192x4096 wide-tail frame (200k beams, tails truncated at 2 deg)
    with a 0.3 deg exact core: the bound holds for every beam against the
    exact tail, and sampled beams meet the parity bar."""
    w = S.wide_frame()
    sp = Split(w, 0.3, 256)
    fr, _ = sp.features()
    ex = sp.exact()
    tot = ex[:, 259]
    assert bool((fr[:, 257] >= tot).all())
    n, res = sp.split(fr)
    assert n < 0.5 * len(w.dirs), n
    g = S.rng(31)
    nb = len(w.dirs)
    beams = np.unique(np.concatenate([[0, nb - 1], g.choice(nb, 40, replace=False)])).astype(np.int32)
    parity(w, res, beams)
    sp.close()


def test_split_rejects_table_profile_and_bad_sizes():
    w = S.full_frame_boxes(U=256, V=128, n_boxes=5, rows=2, cols=10)
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    with pytest.raises(lidar.LidarError, match="radial"):
        lidar.lidar_tail_configure(L.handle, 0.2, 256)
    L.close()
    w = S.tiny_case()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    with pytest.raises(lidar.LidarError, match="n_coarse"):
        lidar.lidar_tail_configure(L.handle, 0.15, 100)
    with pytest.raises(lidar.LidarError, match="core_deg"):
        lidar.lidar_tail_configure(L.handle, 1.0, 64)
    with pytest.raises(lidar.LidarError, match="configure"):
        lidar.lidar_tail_features(L.handle, lidar.make_gbuffer(w.gbuffer, [1] * 7), lidar.make_pose(w.pose), 1)
    L.close()
