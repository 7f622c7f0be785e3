"""Batched execution (lidar_simulate_batch): many frames of uneven size,
pattern and pose in one persistent launch replayed from a CUDA graph.

Each frame's result must equal the single-frame path's within FP32
accumulation-order noise, and sampled beams must match the FP64 oracle with
the same bar as the single-frame parity tests."""
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


class Batch:
    """Device buffers and sensors for a list of Workload frames."""

    def __init__(self, frames):
        self.frames = frames
        self.sensors = [lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib) for w in frames]
        self.planes = [lidar.gbuffer_to_device(w.gbuffer) for w in frames]
        self.outs = [s.alloc_outputs() for s in self.sensors]
        self.executor = self.sensors[0]
        self.arr = lidar.make_frames([
            (s.handle, lidar.make_gbuffer(w.gbuffer, [p.data_ptr() for p in pl]), lidar.make_pose(w.pose),
             o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr())
            for s, w, pl, o in zip(self.sensors, frames, self.planes, self.outs)])

    def run(self, tune=False):
        for o in self.outs:
            o[0].fill_(float("nan"))
            o[2].fill_(-1)
        s = torch.cuda.current_stream().cuda_stream
        if tune:
            lidar.lidar_autotune_batch(self.executor.handle, self.arr, s)
        lidar.lidar_simulate_batch(self.executor.handle, self.arr, s)
        torch.cuda.synchronize()
        lidar.lidar_sync(self.executor.handle, 0)
        return [(o[0].cpu().numpy().astype(np.float64), lidar.echoes_numpy(o[1]), o[2].cpu().numpy())
                for o in self.outs]

    def single(self, f):
        w = self.frames[f]
        wave, ech, cnt = self.sensors[f].simulate(w.gbuffer, self.planes[f], w.pose)
        torch.cuda.synchronize()
        return wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech), cnt.cpu().numpy()

    def close(self):
        for s in self.sensors:
            s.close()


def assert_same(a, b, tol=1e-5):
    wa, ea, ca = a
    wb, eb, cb = b
    nrm = np.maximum(np.linalg.norm(wb, axis=1), 1e-30)
    assert (np.linalg.norm(wa - wb, axis=1) / nrm).max() <= tol
    sure = (eb["flags"] & lidar.ECHO_NEAR_THRESHOLD).sum(axis=1) == 0
    assert (ca[sure] == cb[sure]).all()
    m = np.arange(ea.shape[1])[None, :] < cb[:, None]
    m &= sure[:, None]
    assert (ea["bin_start"][m] == eb["bin_start"][m]).all() and (ea["bin_end"][m] == eb["bin_end"][m]).all()


def oracle_check(w, wave, ech, cnt, beams):
    from tests.test_parity_gpu import ambiguous_ok, compare
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    st = compare(ref, wave, ech, cnt, beams, w.calib["threshold"], w.calib["max_echoes"], w.pulse)
    assert ambiguous_ok(st), st
    return st


def test_small_batch_matches_single_frame_and_oracle():
    frames = S.batched_frames(seed=11, n_frames=7, size_classes=((128, 96), (256, 128), (333, 77)),
                              beams=(37, 3000))
    B = Batch(frames)
    res = B.run()
    g = S.rng(5)
    for f in range(len(frames)):
        assert_same(res[f], B.single(f))
        beams = np.unique(g.choice(len(frames[f].dirs), min(6, len(frames[f].dirs)), replace=False)).astype(np.int32)
        oracle_check(frames[f], *res[f], beams)
    # replay of the captured graph, then a new batch shape
    res2 = B.run()
    for f in range(len(frames)):
        assert_same(res2[f], res[f])
    B.close()
    B2 = Batch(frames[:3])
    res3 = B2.run(tune=True)
    for f in range(3):
        assert_same(res3[f], res[f])
    G, cps = lidar.lidar_batch_config(B2.executor.handle)
    assert G in (2, 4, 8, 16) and cps in (1, 2)
    B2.close()


def test_batch_rejects_other_sensor_model():
    a = S.tiny_case()
    b = S.tiny_case()
    b.calib = dict(b.calib, threshold=3e-4)
    B = Batch([a])
    other = lidar.Lidar(b.profile, b.dirs, b.pulse, b.calib)
    arr = lidar.make_frames([(other.handle, lidar.make_gbuffer(b.gbuffer, [p.data_ptr() for p in B.planes[0]]),
                              lidar.make_pose(b.pose), B.outs[0][0].data_ptr(), B.outs[0][1].data_ptr(),
                              B.outs[0][2].data_ptr())])
    with pytest.raises(lidar.LidarError, match="sensor model"):
        lidar.lidar_simulate_batch(B.executor.handle, arr, 0)
    other.close()
    B.close()


def test_full_batched_workload_sampled():
    """64 frames, 512x256 .. 4096x2048, 1k .. 100k beams, autotuned: 16
    sampled beams of every frame (about 1000 echoes) against the oracle, the
    ambiguous echoes counted over the whole batch."""
    from oracle import parity as PR
    from tests.test_parity_gpu import BAND, ambiguous_ok, check_own_waveform
    frames = S.batched_frames()
    B = Batch(frames)
    res = B.run(tune=True)
    g = S.rng(9)
    tot = PR.Stats()
    for f in range(len(frames)):
        w = frames[f]
        n = len(w.dirs)
        beams = np.unique(np.concatenate([[0, n - 1], g.choice(n, 14, replace=False)])).astype(np.int32)
        wave, ech, cnt = res[f]
        ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
        T = w.calib["threshold"]
        st, fails = PR.compare_frame(ref, beams, wave, ech, cnt, T, w.calib["max_echoes"], BAND)
        assert not fails, (w.name, fails[:5])
        for s_, b in enumerate(beams):
            if np.any(np.abs(ref["xi"][s_] - T) <= BAND * T):
                check_own_waveform(b, wave[b], ech[b], cnt[b], w.pulse, T, ref["coef"], w.calib["max_echoes"])
        tot.merge(st)
    assert tot["echoes"] >= 900 and ambiguous_ok(tot, strict=True), dict(tot)
    # every frame's echo counts must be sane and waveforms finite
    for wave, ech, cnt in res:
        assert np.isfinite(wave).all() and (cnt >= 0).all()
    B.close()
