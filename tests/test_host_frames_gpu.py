"""lidar_simulate_host_frames: a sequence of frames from host memory, with
consecutive frames overlapped on two sets of device buffers (frame f + 1 set
up while frame f runs). Each frame's results must be those of the device
entry point on the same frame (which the parity tests pin to the FP64
oracle), and a few sampled beams of one frame are checked against the oracle
directly.
"""
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


def _pinned(w):
    return [torch.from_numpy(np.ascontiguousarray(p)).pin_memory() for p in w.gbuffer.planes()]


def _device(L, w):
    wave, ech, cnt = L.simulate(w.gbuffer, lidar.gbuffer_to_device(w.gbuffer), w.pose)
    torch.cuda.synchronize()
    return wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech), cnt.cpu().numpy()


def _same(got, ref):
    wave_h, ech_h, cnt_h = got
    wave_d, ech_d, cnt_d = ref
    if wave_h is not None:
        rel = np.linalg.norm(wave_h - wave_d, axis=1) / np.maximum(np.linalg.norm(wave_d, axis=1), 1e-30)
        assert rel.max() <= 1e-5, rel.max()
    assert (cnt_h == cnt_d).mean() >= 0.999
    same = cnt_h == cnt_d
    for k in ("bin_start", "bin_end"):
        assert (ech_h[k][same] == ech_d[k][same]).mean() >= 0.999, k


def _frames():
    """Five large frames: two scenes, a ragged-size frame (rows not a multiple
    of the upload bands) and a repeat with another pose, so that each buffer
    set sees frames of different content and size."""
    wa, wb = S.full_frame_boxes(seed=2), S.full_frame_boxes(seed=9)
    wc = S.full_frame_boxes(seed=4, U=2000, V=999)
    wd = S.full_frame_boxes(seed=2)
    wd.pose = S.pose_ypr(0.01, -0.004, 0.002)
    return wa, [wa, wb, wc, wd, wb]


def test_host_frames_match_device_entry_point():
    wa, ws = _frames()
    L = lidar.Lidar(wa.profile, wa.dirs, wa.pulse, wa.calib)
    refs = [_device(L, w) for w in ws]
    outs = L.simulate_host_frames([w.gbuffer for w in ws], [_pinned(w) for w in ws], [w.pose for w in ws])
    for f, (o, ref) in enumerate(zip(outs, refs)):
        got = (o[0].numpy().astype(np.float64), lidar.echoes_numpy(o[1]), o[2].numpy())
        _same(got, ref)
    # frame 2 (the ragged one) against the oracle on sampled beams
    w = ws[2]
    g = S.rng(31)
    beams = np.unique(np.concatenate([[0, len(w.dirs) - 1], g.choice(len(w.dirs), 24, replace=False)])).astype(np.int32)
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    wave = outs[2][0].numpy().astype(np.float64)
    for s, b in enumerate(beams):
        x = ref["xi"][s]
        nrm = np.linalg.norm(x)
        err = np.linalg.norm(wave[b] - x) / nrm if nrm > 0 else np.abs(wave[b]).max()
        assert err <= 1e-3, (b, err)
    L.close()


def test_host_frames_alternating_outputs():
    """Frames f and f + 2 may share outputs: with two output sets for four
    frames, each set holds the last frame written to it."""
    wa, ws = _frames()
    ws = ws[:4]
    L = lidar.Lidar(wa.profile, wa.dirs, wa.pulse, wa.calib)
    sets = [(torch.empty((L.n_beams, L.n_bins), dtype=torch.float32, pin_memory=True),
             torch.empty((L.n_beams, L.max_echoes, 8), dtype=torch.int32, pin_memory=True),
             torch.empty((L.n_beams,), dtype=torch.int32, pin_memory=True)) for _ in range(2)]
    L.simulate_host_frames([w.gbuffer for w in ws], [_pinned(w) for w in ws], [w.pose for w in ws],
                           outputs=[sets[f & 1] for f in range(4)])
    for p in range(2):
        o = sets[p]
        got = (o[0].numpy().astype(np.float64), lidar.echoes_numpy(o[1]), o[2].numpy())
        _same(got, _device(L, ws[2 + p]))
    L.close()


def test_host_frames_echo_only():
    """No waveform outputs: the echo-only form for every frame of the
    sequence (waveforms in the slot pool), same echoes and counts."""
    wa, ws = _frames()
    ws = ws[:3]
    L = lidar.Lidar(wa.profile, wa.dirs, wa.pulse, wa.calib)
    refs = [_device(L, w) for w in ws]
    outs = L.simulate_host_frames([w.gbuffer for w in ws], [_pinned(w) for w in ws], [w.pose for w in ws],
                                  echo_only=True)
    lidar.lidar_sync(L.handle, 0)
    for o, ref in zip(outs, refs):
        _same((None, lidar.echoes_numpy(o[1]), o[2].numpy()), ref)
    L.close()


def test_host_frames_small_and_empty():
    """Small frames run one after the other through lidar_simulate_host; an
    empty sequence does nothing; a NULL output pointer is rejected before
    anything is enqueued."""
    w = S.tiny_case()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    ref = _device(L, w)
    outs = L.simulate_host_frames([w.gbuffer] * 3, [_pinned(w)] * 3, [w.pose] * 3)
    for o in outs:
        _same((o[0].numpy().astype(np.float64), lidar.echoes_numpy(o[1]), o[2].numpy()), ref)
    lidar.lidar_simulate_host_frames(L.handle, [], [], None, [], [], 0)
    g = lidar.make_gbuffer(w.gbuffer, [p.data_ptr() for p in _pinned(w)])
    with pytest.raises(RuntimeError):
        lidar.lidar_simulate_host_frames(L.handle, [g], [lidar.make_pose(w.pose)], None, [None],
                                         [outs[0][2].data_ptr()], 0)
    L.close()
