"""Echo-only simulation (lidar_simulate_echoes): the waveforms stay in a
pooled, L2-sized slot per CTA instead of the caller's memory. The echoes must
be lidar_simulate's: counts and bins equal, ranges, EPW, intensities and
peaks equal up to FP32 noise (the deposits are FP32 shared-memory atomics, so
the last bits of a waveform depend on the order of the additions, in either
entry point), and the parity bar against the FP64 oracle met."""
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


def both(L, w, planes, calls=2):
    """lidar_simulate once, then lidar_simulate_echoes `calls` times (outputs
    pre-filled with garbage so that unwritten entries show)."""
    wave, ech, cnt = L.simulate(w.gbuffer, planes, w.pose)
    torch.cuda.synchronize()
    lidar.lidar_sync(L.handle, 0)
    runs = []
    for _ in range(calls):
        e2 = torch.full_like(ech, -5)
        c2 = torch.full_like(cnt, -5)
        L.simulate_echoes(w.gbuffer, planes, w.pose, outputs=(e2, c2))
        torch.cuda.synchronize()
        lidar.lidar_sync(L.handle, 0)
        runs.append((e2.cpu().numpy(), c2.cpu().numpy()))
    return wave, ech.cpu().numpy(), cnt.cpu().numpy(), runs


def assert_identical(ech, cnt, runs):
    """Counts and echo bins equal (except echoes flagged near the threshold,
    whose crossings FP32 noise may move); float fields within 1e-5."""
    a = lidar.echoes_numpy(torch.from_numpy(ech))
    for e2, c2 in runs:
        np.testing.assert_array_equal(c2, cnt)
        b = lidar.echoes_numpy(torch.from_numpy(e2))
        for bi in range(len(cnt)):
            for k in range(cnt[bi]):
                x, y = a[bi][k], b[bi][k]
                if (x["flags"] | y["flags"]) & 4:
                    continue
                assert (x["bin_start"], x["bin_end"], x["bin_peak"], x["flags"]) == \
                       (y["bin_start"], y["bin_end"], y["bin_peak"], y["flags"]), (bi, k, x, y)
                assert abs(x["range_m"] - y["range_m"]) <= 1e-4 and abs(x["epw_m"] - y["epw_m"]) <= 1e-4, (bi, k)
                assert y["intensity"] == pytest.approx(x["intensity"], rel=1e-4), (bi, k)
                assert y["peak"] == pytest.approx(x["peak"], rel=1e-5), (bi, k)
            for k in range(cnt[bi], e2.shape[1]):
                assert (e2[bi, k] == 0).all(), (bi, k)


@pytest.mark.parametrize("deposit", [0, 1])
def test_echoes_identical_to_full_simulation_and_oracle(deposit):
    w = S.small_plane_retro()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    lidar.lidar_set_deposit(L.handle, deposit)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    wave, ech, cnt, runs = both(L, w, planes)
    assert_identical(ech, cnt, runs)
    from tests.test_parity_gpu import compare
    beams = np.arange(len(w.dirs), dtype=np.int32)
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    e2, c2 = runs[-1]
    st = compare(ref, wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(torch.from_numpy(e2)), c2, beams,
                 w.calib["threshold"], w.calib["max_echoes"], w.pulse)
    assert st["echoes"] >= 500
    L.close()


def test_ragged_group_and_interleaved_calls():
    """37 beams (a partial last group), calls alternating with the full
    simulation and with a second sensor that shares nothing."""
    w = S.tiny_case(n_beams=37, n_bins=256)
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    wave, ech, cnt, runs = both(L, w, planes, calls=1)
    assert_identical(ech, cnt, runs)
    w2 = S.small_plane_retro()
    L2 = lidar.Lidar(w2.profile, w2.dirs, w2.pulse, w2.calib)
    p2 = lidar.gbuffer_to_device(w2.gbuffer)
    _, ech2, cnt2, runs2 = both(L2, w2, p2, calls=1)
    assert_identical(ech2, cnt2, runs2)
    _, ech3, cnt3, runs3 = both(L, w, planes, calls=2)
    assert_identical(ech, cnt, runs3)
    L.close()
    L2.close()


def test_full_frame_identical():
    """The full-frame scene family (table profile, 2048 bins) on a
    1024x512 G-buffer: every beam's echoes identical to lidar_simulate's."""
    w = S.full_frame_boxes(U=1024, V=512, n_boxes=20, rows=8, cols=400)
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    wave, ech, cnt, runs = both(L, w, planes)
    assert_identical(ech, cnt, runs)
    assert cnt.sum() > 0
    L.close()


def test_rejects_null_outputs():
    w = S.tiny_case()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    g = lidar.make_gbuffer(w.gbuffer, [1] * 7)
    with pytest.raises(lidar.LidarError, match="NULL"):
        lidar.lidar_simulate_echoes(L.handle, g, lidar.make_pose(w.pose), 0, 0)
    L.close()


@pytest.mark.parametrize("echo_only", [False, True])
def test_strongest_echo_mode(echo_only):
    """LIDAR_ECHOES_STRONGEST on beams across a board's edge in front of a
    plane (two echoes near the edge, the farther one the stronger for half of
    them): every beam reports the oracle's strongest echo alone (count 0 or 1,
    the other entries zero), in the waveform and the echo-only forms. A beam
    with a waveform bin in the guard band, or whose two strongest oracle echoes
    are within 1e-3 in intensity, only has to report one of its echoes."""
    w = S.edge_two_depths()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    lidar.lidar_set_echo_mode(L.handle, lidar.ECHOES_STRONGEST)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    if echo_only:
        ech, cnt = L.simulate_echoes(w.gbuffer, planes, w.pose)
    else:
        _, ech, cnt = L.simulate(w.gbuffer, planes, w.pose)
    torch.cuda.synchronize()
    lidar.lidar_sync(L.handle, 0)
    ech, cnt = lidar.echoes_numpy(ech), cnt.cpu().numpy()
    beams = np.arange(len(w.dirs), dtype=np.int32)
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=64)
    T = w.calib["threshold"]
    assert set(np.unique(cnt)) <= {0, 1}
    assert (ech[:, 1:]["bin_end"] == 0).all() and (ech[:, 1:]["flags"] == 0).all()
    far_wins = 0
    for b in beams:
        oe = ref["echoes"][b][:int(ref["counts"][b])]
        assert cnt[b] == (1 if len(oe) else 0), b
        if not len(oe):
            continue
        g = ech[b, 0]
        ambiguous = np.any(np.abs(ref["xi"][b] - T) <= 1e-4 * T)
        top = np.sort(oe["intensity"])[::-1]
        if ambiguous or (len(oe) > 1 and top[1] >= top[0] * (1 - 1e-3)):
            assert any((g["bin_start"], g["bin_end"]) == (o["bin_start"], o["bin_end"]) for o in oe), b
            continue
        o = O.strongest_echo(oe)[0]
        far_wins += int(o["bin_start"] != oe[0]["bin_start"])
        assert (g["bin_start"], g["bin_end"]) == (o["bin_start"], o["bin_end"]), (b, g, o)
        assert g["intensity"] == pytest.approx(o["intensity"], rel=1e-3)
        assert abs(g["range_m"] - o["range_m"]) <= 1e-3
    assert far_wins >= 5
    # the default (nearest first) on the same frame meets the parity bar
    lidar.lidar_set_echo_mode(L.handle, lidar.ECHOES_NEAREST)
    wave, ech2, cnt2 = L.simulate(w.gbuffer, planes, w.pose)
    torch.cuda.synchronize()
    from tests.test_parity_gpu import compare
    st = compare(ref, wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech2), cnt2.cpu().numpy(), beams, T,
                 w.calib["max_echoes"], w.pulse)
    assert st["echoes"] >= 60
    L.close()


def test_echo_mode_rejects_unknown_values():
    w = S.tiny_case()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    with pytest.raises(lidar.LidarError, match="echo mode"):
        lidar.lidar_set_echo_mode(L.handle, 2)
    L.close()


@pytest.mark.parametrize("case", ["tiny", "full_frame"])
def test_host_entry_point_echo_only(case):
    """lidar_simulate_host with no waveform output (the echo-only form through
    the host entry point; the full frame takes the pipelined path): the echoes
    and counts of lidar_simulate_echoes on the same frame, pinned or pageable
    planes."""
    w = S.tiny_case() if case == "tiny" else S.full_frame_boxes()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    ech_d, cnt_d = L.simulate_echoes(w.gbuffer, planes, w.pose)
    torch.cuda.synchronize()
    lidar.lidar_sync(L.handle, 0)
    ech_d, cnt_d = ech_d.cpu().numpy(), cnt_d.cpu().numpy()
    for pin in (True, False):
        hp = [torch.from_numpy(np.ascontiguousarray(p)) for p in w.gbuffer.planes()]
        if pin:
            hp = [p.pin_memory() for p in hp]
        outs = (None, torch.full((L.n_beams, L.max_echoes, 8), -5, dtype=torch.int32, pin_memory=True),
                torch.full((L.n_beams,), -5, dtype=torch.int32, pin_memory=True))
        wave, ech_h, cnt_h = L.simulate_host(w.gbuffer, hp, w.pose, outs, echo_only=True)
        assert wave is None
        assert_identical(ech_d, cnt_d, [(ech_h.numpy(), cnt_h.numpy())])
    L.close()


def test_slot_claim_gives_up_and_reports_timeout():
    """The bounded wait of the echo-only form: with every waveform slot held
    (lidar_hold_echo_slots), the CTAs give up their claim after a bounded
    number of polls, write nothing, and lidar_sync reports LIDAR_ETIMEOUT;
    once the slots are free again the same call gives the normal result."""
    w = S.small_plane_retro()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    ech0, cnt0 = L.simulate_echoes(w.gbuffer, planes, w.pose)
    lidar.lidar_sync(L.handle, 0)
    ref_e, ref_c = lidar.echoes_numpy(ech0), cnt0.cpu().numpy()
    assert ref_c.sum() >= 500
    lidar.lidar_hold_echo_slots(L.handle, True)
    ech, cnt = L._alloc_echoes("cuda")
    cnt.fill_(-7)
    L.simulate_echoes(w.gbuffer, planes, w.pose, (ech, cnt))
    with pytest.raises(lidar.LidarError) as ei:
        lidar.lidar_sync(L.handle, 0)
    assert ei.value.status == lidar.LIDAR_ETIMEOUT
    assert (cnt.cpu().numpy() == -7).all()  # nothing was written
    lidar.lidar_sync(L.handle, 0)  # the error word was cleared by the report
    lidar.lidar_hold_echo_slots(L.handle, False)
    L.simulate_echoes(w.gbuffer, planes, w.pose, (ech, cnt))
    lidar.lidar_sync(L.handle, 0)
    assert (cnt.cpu().numpy() == ref_c).all()
    e = lidar.echoes_numpy(ech)
    for b in range(len(ref_c)):
        for i in range(ref_c[b]):
            assert e[b, i]["bin_start"] == ref_e[b, i]["bin_start"] and e[b, i]["bin_end"] == ref_e[b, i]["bin_end"]
    L.close()
