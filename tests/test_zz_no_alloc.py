"""lidar_simulate_noalloc: the entry point for callers that cannot let the
library allocate device memory during a call (a host whose memory pool has
already reserved the GPU, a real-time loop that must not allocate once
running). It keeps its per-pixel scratch in a fixed 32 MiB device array.

Checked through the C ABI: the first two calls on a fresh handle leave the
device's free memory unchanged and each match the regular lidar_simulate
within the parity tolerance, and a G-buffer larger than the array must be
rejected. This file is collected last so that, if it fails, a
run that stops at the first failure has already run every other test; it
also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2512_05932_gb300 import lidar
from paper_2512_05932_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _run(L, w, planes, fn, outputs=None):
    wave, ech, cnt = outputs if outputs is not None else L.alloc_outputs()
    wave.fill_(float("nan"))
    cnt.fill_(-1)
    g = lidar.make_gbuffer(w.gbuffer, [p.data_ptr() for p in planes])
    fn(L.handle, g, lidar.make_pose(w.pose), wave.data_ptr(), ech.data_ptr(), cnt.data_ptr(),
       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech), cnt.cpu().numpy()


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_noalloc_matches_regular_entry_point_twice():
    """The first two calls on a fresh handle are no-allocation calls: device
    free memory must not change across them (the regular entry point, run on
    a second fresh handle, does allocate its records), and each must match the
    regular entry point's results."""
    w = S.small_plane_retro()
    planes = lidar.gbuffer_to_device(w.gbuffer)
    # load the kernels' modules once, on a handle of its own
    warm = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    _run(warm, w, planes, lidar.lidar_simulate)
    warm.close()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    outs = [L.alloc_outputs() for _ in range(2)]
    got = []
    free0 = _free_bytes()
    for o in outs:
        got.append(_run(L, w, planes, lidar.lidar_simulate_noalloc, o))
    assert _free_bytes() == free0, "a no-allocation call changed the device's free memory"
    R = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    ro = R.alloc_outputs()
    free1 = _free_bytes()
    ref_wave, ref_ech, ref_cnt = _run(R, w, planes, lidar.lidar_simulate, ro)
    # the check above can see an allocation: the regular call's records (2 MB)
    assert _free_bytes() < free1
    for wave, ech, cnt in got:
        err = np.linalg.norm(wave - ref_wave, axis=1) / np.linalg.norm(ref_wave, axis=1)
        assert err.max() <= 1e-3, err.max()
        sure = (ref_ech["flags"] & lidar.ECHO_NEAR_THRESHOLD).sum(axis=1) == 0
        assert (cnt[sure] == ref_cnt[sure]).all()
        for b in np.nonzero(sure)[0]:
            for i in range(cnt[b]):
                assert ech[b, i]["bin_start"] == ref_ech[b, i]["bin_start"]
                assert ech[b, i]["bin_end"] == ref_ech[b, i]["bin_end"]
                assert abs(ech[b, i]["range_m"] - ref_ech[b, i]["range_m"]) <= 1e-3
    L.close()
    R.close()


def test_noalloc_rejects_gbuffer_beyond_its_scratch():
    w = S.tiny_case()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    wave, ech, cnt = L.alloc_outputs()
    big = S.GBuffer(1025, 1024, -0.1, -0.1, 1e-4, 1e-4, *([None] * 7))
    dummy = torch.zeros(1, device="cuda")
    g = lidar.make_gbuffer(big, [dummy.data_ptr()] * 7)
    with pytest.raises(lidar.LidarError, match="at most") as ei:
        lidar.lidar_simulate_noalloc(L.handle, g, lidar.make_pose(np.eye(3)), wave.data_ptr(), ech.data_ptr(),
                                     cnt.data_ptr(), 0)
    assert ei.value.status == lidar.LIDAR_EINVAL
    L.close()
