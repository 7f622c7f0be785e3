"""The deposit on the 5th-generation tensor cores (LIDAR_DEPOSIT_TCGEN05_BF16 /
_FP16): 16 beams per CTA with their histograms in tensor memory, (bins x
pixels) hat weights times (pixels x beams) profile weights per 64-pixel tile.

The products are 16-bit, so the error against the FP64 oracle is stated per
result rather than held to the FP32 bar everywhere:
  - FP16 (power-of-two scaled) on the small instance and on the batch meets
    the parity bar of the FP32 path (waveform L2 <= 1e-3, echo bins exact
    outside the guard band, range within 1 mm);
  - BF16 (8-bit significand) on the wide-tail frame's 1 % subsample: waveform
    L2 <= 5e-3, ranges of the matching echoes within 1 mm, at most 5 % of
    echoes with a bin, intensity or peak outside the FP32 bar.
"""
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
BAND = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run(w, mode):
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    lidar.lidar_set_deposit(L.handle, mode)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    wave, ech, cnt = L.alloc_outputs()
    cnt.fill_(-1)
    L.simulate(w.gbuffer, planes, w.pose, (wave, ech, cnt))
    torch.cuda.synchronize()
    lidar.lidar_sync(L.handle, 0)
    L.close()
    return wave, lidar.echoes_numpy(ech), cnt.cpu().numpy()


def judge(w, beams, wave, ech, cnt, tol_l2):
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    bi = torch.as_tensor(beams, device=wave.device, dtype=torch.long)
    rows = {int(b): r for b, r in zip(beams, wave[bi].cpu().numpy().astype(np.float64))}
    st, fails = PR.compare_frame(ref, beams, rows, ech, cnt, w.calib["threshold"], w.calib["max_echoes"], BAND,
                                 tol_l2)
    assert (cnt[beams] >= 0).all(), "beams not written"
    return st, fails


def test_fp16_small_instance_meets_the_parity_bar():
    w = S.small_plane_retro()
    wave, ech, cnt = run(w, lidar.DEPOSIT_TCGEN05_FP16)
    st, fails = judge(w, np.arange(len(w.dirs), dtype=np.int32), wave, ech, cnt, 1e-3)
    assert not fails, fails[:5]
    assert st["echoes"] >= 500 and st["ambiguous"] == 0 and st["max_dr"] <= 1e-3, st


def test_bf16_small_instance_error_bound():
    w = S.small_plane_retro()
    wave, ech, cnt = run(w, lidar.DEPOSIT_TCGEN05_BF16)
    st, fails = judge(w, np.arange(len(w.dirs), dtype=np.int32), wave, ech, cnt, 5e-3)
    assert not [f for f in fails if "L2" in f[1]], fails[:5]
    assert st["mismatched"] <= 0.05 * st["echoes"] and st["max_dr"] <= 1e-3, st


@pytest.mark.parametrize("mode", ["bf16", "fp16"])
def test_wide_tail_frame_one_percent_subsample(mode):
    """8192x4096, 200k beams, 4096 bins of 0.05 ns: the BF16 form the wide
    frame's tensor-core configuration names (and the FP16 one) against the
    oracle on the seeded 2000-beam subsample."""
    w = S.wide_frame()
    m = lidar.DEPOSIT_TCGEN05_BF16 if mode == "bf16" else lidar.DEPOSIT_TCGEN05_FP16
    wave, ech, cnt = run(w, m)
    beams = np.sort(S.rng(2000).choice(len(w.dirs), 2000, replace=False)).astype(np.int32)
    st, fails = judge(w, beams, wave, ech, cnt, 5e-3 if mode == "bf16" else 1e-3)
    assert not [f for f in fails if "L2" in f[1]], fails[:5]
    assert st["echoes"] >= 1000 and st["max_dr"] <= 1e-3, st
    assert st["mismatched"] <= (0.05 if mode == "bf16" else 0.005) * st["echoes"], st


def test_fp16_batch_against_the_oracle():
    """The 64-frame batch through the persistent tcgen05 kernel with FP16
    operands: 16 sampled beams of every frame at the parity bar."""
    from tests.test_batch_gpu import Batch
    frames = S.batched_frames()
    B = Batch(frames)
    for s in B.sensors:
        lidar.lidar_set_deposit(s.handle, lidar.DEPOSIT_TCGEN05_FP16)
    res = B.run()
    g = S.rng(9)
    tot = PR.Stats()
    for f, w in enumerate(frames):
        n = len(w.dirs)
        beams = np.unique(np.concatenate([[0, n - 1], g.choice(n, 14, replace=False)])).astype(np.int32)
        wave, ech, cnt = res[f]
        ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
        st, fails = PR.compare_frame(ref, beams, wave, ech, cnt, w.calib["threshold"], w.calib["max_echoes"], BAND)
        assert not fails, (w.name, fails[:5])
        tot.merge(st)
    assert tot["echoes"] >= 900 and tot["ambiguous"] <= 1e-3 * tot["echoes"], dict(tot)
    # a replay of the captured graph gives the same result
    res2 = B.run()
    for f in range(len(frames)):
        np.testing.assert_array_equal(res2[f][2], res[f][2])
    B.close()


def test_entry_points_without_a_tcgen05_form_reject_it():
    w = S.tiny_case()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    lidar.lidar_set_deposit(L.handle, lidar.DEPOSIT_TCGEN05_BF16)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    with pytest.raises(lidar.LidarError, match="echo-only") as ei:
        L.simulate_echoes(w.gbuffer, planes, w.pose)
    assert ei.value.status == lidar.LIDAR_EINVAL
    hp = [torch.from_numpy(np.ascontiguousarray(p)).pin_memory() for p in w.gbuffer.planes()]
    with pytest.raises(lidar.LidarError, match="host entry points"):
        L.simulate_host(w.gbuffer, hp, w.pose)
    L.close()
    wide = S.tiny_case(n_bins=8192)
    L = lidar.Lidar(wide.profile, wide.dirs, wide.pulse, wide.calib)
    with pytest.raises(lidar.LidarError, match="n_bins <= 4096"):
        lidar.lidar_set_deposit(L.handle, lidar.DEPOSIT_TCGEN05_FP16)
    L.close()
