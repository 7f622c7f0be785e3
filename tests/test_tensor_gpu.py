"""Tensor-core deposit forms (lidar_set_deposit).

LIDAR_DEPOSIT_TC_SPLIT (BF16 hi/lo split, FP32 accumulation) must meet the
same parity bar as the FP32 atomic form. LIDAR_DEPOSIT_TC_BF16 (plain BF16
products) is a reduced-precision form: its waveform error against the FP64
oracle is measured and bounded at 5e-3 (relative L2 per beam)."""
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


def run(w, mode):
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    lidar.lidar_set_deposit(L.handle, mode)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    wave, ech, cnt = L.simulate(w.gbuffer, planes, w.pose)
    torch.cuda.synchronize()
    lidar.lidar_sync(L.handle, 0)
    out = wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech), cnt.cpu().numpy()
    L.close()
    return out


def parity(w, beams=None):
    from tests.test_parity_gpu import ambiguous_ok, compare
    wave, ech, cnt = run(w, lidar.DEPOSIT_TC_SPLIT)
    if beams is None:
        beams = np.arange(len(w.dirs), dtype=np.int32)
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    st = compare(ref, wave, ech, cnt, beams, w.calib["threshold"], w.calib["max_echoes"], w.pulse)
    assert ambiguous_ok(st), st
    return st


def test_tc_split_small_instance():
    st = parity(S.small_plane_retro())
    assert st["echoes"] >= 500


def test_tc_split_tiny_rolled_and_ragged():
    parity(S.tiny_case())
    w = S.tiny_case(n_beams=37, n_bins=32)
    w.pulse = S.pulse(32, 1e-9, 2.0e-8, 4e-9, 3.0)
    parity(w)


def test_tc_split_full_frame_sampled():
    w = S.full_frame_boxes()
    g = S.rng(78)
    n = len(w.dirs)
    beams = np.unique(np.concatenate([[0, 1600, n - 1], g.choice(n, 40, replace=False)])).astype(np.int32)
    parity(w, beams)


def test_tc_split_matches_atomic_form():
    w = S.full_frame_boxes()
    a = run(w, lidar.DEPOSIT_ATOMIC)
    b = run(w, lidar.DEPOSIT_TC_SPLIT)
    nrm = np.maximum(np.linalg.norm(a[0], axis=1), 1e-30)
    assert (np.linalg.norm(a[0] - b[0], axis=1) / nrm).max() <= 1e-4


def test_tc_bf16_error_is_bounded():
    w = S.small_plane_retro()
    wave, ech, cnt = run(w, lidar.DEPOSIT_TC_BF16)
    ref = O.simulate_workload(w, nthreads=NTHREADS, max_out=8)
    err = np.linalg.norm(wave - ref["xi"], axis=1) / np.linalg.norm(ref["xi"], axis=1)
    assert err.max() <= 5e-3, err.max()


def test_tc_split_in_batch():
    from tests.test_batch_gpu import Batch, assert_same
    frames = S.batched_frames(seed=12, n_frames=4, size_classes=((128, 96), (256, 128)), beams=(50, 2000))
    B = Batch(frames)
    for s in B.sensors:
        lidar.lidar_set_deposit(s.handle, lidar.DEPOSIT_TC_SPLIT)
    res = B.run()
    for f in range(len(frames)):
        assert_same(res[f], B.single(f))
    B.close()
