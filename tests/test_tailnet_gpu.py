"""The FP16 tail-network kernels (training and inference) against the FP64
NumPy statement of the network (oracle/tailnet.py), checkpoint round trips,
and the surrogate simulation against the FP64 beam oracle."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle import tailnet as TN
from paper_2512_05932_gb300 import lidar
from paper_2512_05932_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
NC = 64


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def random_batch(seed, B, nc=NC, slack=1e3):
    g = np.random.default_rng(seed)
    x = g.uniform(-1, 1.5, size=(B, lidar.TAIL_INPUT_CELLS, 2)).astype(np.float16)
    rows = np.zeros((B, nc + 4), np.float32)
    rows[:, :nc] = g.uniform(0, 1, size=(B, nc)) ** 3
    rows[:, nc + 3] = rows[:, :nc].sum(1)
    rows[:, nc + 1] = rows[:, nc + 3] * slack
    rows[:, nc] = g.uniform(0, 1, size=B)
    rows[:, nc + 2] = 0.01
    target = np.zeros_like(rows)
    target[:, :nc] = np.roll(rows[:, :nc], 1, axis=1) * g.uniform(0.5, 1.5, size=(B, 1))
    return x, rows, target


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def randomize(net, seed):
    """Random weights in every layer (a new network's output layer is zero,
    which would hide the layers before it)."""
    lay, n = TN.layout(net.n_coarse)
    g = np.random.default_rng(seed)
    P = TN.unpack(np.zeros(n), net.n_coarse)
    for k, v in P.items():
        fan = v.shape[1] if v.ndim == 2 else 1
        v[...] = g.uniform(-1, 1, size=v.shape) * np.sqrt(3.0 / fan) * (0.2 if v.ndim == 1 else 1.0)
    P["w1"][:, 18:] = 0
    P["w2"][:, 306:] = 0
    P["w3"][:, 306:] = 0
    P["f2"] *= 0.3
    net.set_params(TN.pack(P, net.n_coarse).astype(np.float32))


def clip_to_bound(tail, rows, nc):
    """A prediction whose mass exceeds the row's bound E is scaled down to E
    (the documented output of lidar_tailnet_predict); a random network with
    many coarse bins often predicts more than E."""
    E = np.asarray(rows, np.float64)[:, nc + 1]
    m = tail.sum(axis=1)
    f = np.where(m > E, E / np.where(m > 0, m, 1), 1.0)
    return tail * f[:, None]


def test_predict_matches_fp64_network():
    net = lidar.TailNet(NC, seed=7)
    randomize(net, 7)
    x, rows, _ = random_batch(1, 6)
    out = torch.zeros((6, NC + 4), dtype=torch.float32, device="cuda")
    net.predict(dev(x), dev(rows), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref, _ = TN.forward(net.get_params().astype(np.float64), x.astype(np.float64), rows, NC)
    err = np.abs(got[:, :NC] - ref) / np.abs(ref).max(axis=1, keepdims=True)
    assert err.max() <= 2e-2, err.max()
    np.testing.assert_allclose(got[:, NC], rows[:, NC])
    np.testing.assert_allclose(got[:, NC + 1], rows[:, NC + 1])
    np.testing.assert_allclose(got[:, NC + 3], got[:, :NC].sum(1), rtol=1e-5)
    net.close()


DENSE = {"tcgen05": lidar.TailNet.DENSE_TCGEN05, "mma_sync": lidar.TailNet.DENSE_MMA_SYNC}


@pytest.mark.parametrize("dense", sorted(DENSE))
@pytest.mark.parametrize("nc,B", [(256, 300), (64, 161), (40, 130)])
def test_predict_many_beams_matches_fp64_network(nc, B, dense):
    """More beams than one persistent pass of the fused convolutions covers,
    several row tiles of the dense layers with a ragged last tile, in both
    GEMM modes (40 bins: the output layer is not a multiple of 16 wide, so it
    runs on mma.sync in either mode)."""
    net = lidar.TailNet(nc, seed=13)
    net.set_dense(DENSE[dense])
    randomize(net, 13)
    x, rows, _ = random_batch(6, B, nc=nc)
    out = torch.zeros((B, nc + 4), dtype=torch.float32, device="cuda")
    net.predict(dev(x), dev(rows), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ref, _ = TN.forward(net.get_params().astype(np.float64), x.astype(np.float64), rows, nc)
    ref = clip_to_bound(ref, rows, nc)
    err = np.abs(got[:, :nc] - ref) / np.abs(ref).max(axis=1, keepdims=True)
    bad = np.argwhere(err.max(axis=1) > 2e-2).ravel()
    assert err.max() <= 2e-2, (err.max(), bad[:20], len(bad))
    np.testing.assert_allclose(got[:, nc + 3], got[:, :nc].sum(1), rtol=1e-5)
    assert (got[:, nc + 3] <= rows[:, nc + 1] * (1 + 1e-6)).all()
    net.sync()
    net.close()


def test_predict_clips_to_the_bound():
    net = lidar.TailNet(NC, seed=8)
    randomize(net, 8)
    x, rows, _ = random_batch(2, 9, slack=0.5)  # bound below the prior's mass
    out = torch.zeros((9, NC + 4), dtype=torch.float32, device="cuda")
    net.predict(dev(x), dev(rows), out)
    got = out.cpu().numpy()
    assert (got[:, :NC] >= 0).all()
    assert (got[:, :NC].sum(1) <= rows[:, NC + 1] * (1 + 1e-5)).all()
    net.close()


@pytest.mark.parametrize("dense", sorted(DENSE))
def test_gradient_matches_fp64_backprop(dense):
    net = lidar.TailNet(NC, seed=9)
    net.set_dense(DENSE[dense])
    randomize(net, 9)
    x, rows, target = random_batch(3, 8)
    loss, g = net.grads(dev(x), dev(rows), dev(target))
    p = net.get_params().astype(np.float64)
    ref_loss, ref_g = TN.loss_and_grad(p, x.astype(np.float64), rows.astype(np.float64), target.astype(np.float64), NC)
    assert loss == pytest.approx(ref_loss, rel=2e-2)
    lay, _ = TN.layout(NC)
    for name, (o, s) in lay.items():
        n = int(np.prod(s))
        a, b = g[o:o + n].astype(np.float64), ref_g[o:o + n]
        nrm = np.linalg.norm(b)
        if nrm == 0:
            assert np.abs(a).max() <= 1e-6, name
            continue
        rel = np.linalg.norm(a - b) / nrm
        assert rel <= 5e-2, (name, rel)
    net.close()


def test_new_network_predicts_the_prior():
    net = lidar.TailNet(NC, seed=3)
    x, rows, _ = random_batch(5, 7)
    out = torch.zeros((7, NC + 4), dtype=torch.float32, device="cuda")
    net.predict(dev(x), dev(rows), out)
    np.testing.assert_allclose(out.cpu().numpy()[:, :NC], rows[:, :NC], rtol=1e-6)
    net.close()


def test_training_reduces_the_loss_and_checkpoints_resume(tmp_path):
    net = lidar.TailNet(NC, seed=10)
    x, rows, target = random_batch(4, 256, slack=1.5)
    X, Rw, T = dev(x), dev(rows), dev(target)
    first = net.train_step(X, Rw, T, 1e-3)
    for _ in range(300):
        last = net.train_step(X, Rw, T, 1e-3)
    assert last < 0.7 * first, (first, last)
    path = str(tmp_path / "net.bin")
    net.save(path, with_state=True)
    other = lidar.TailNet(NC, seed=11)
    other.load(path)
    np.testing.assert_array_equal(other.get_params(), net.get_params())
    # one more step from the same state gives the same weights (up to the
    # order of FP32 atomic additions)
    net.train_step(X, Rw, T, 1e-3, want_loss=False)
    other.train_step(X, Rw, T, 1e-3, want_loss=False)
    np.testing.assert_allclose(other.get_params(), net.get_params(), rtol=1e-4, atol=1e-6)
    # weights-only file: same parameters, fresh optimiser
    net.save(path, with_state=False)
    other.load(path)
    np.testing.assert_array_equal(other.get_params(), net.get_params())
    net.close()
    other.close()


def test_dense_mode_rejects_unknown_values():
    net = lidar.TailNet(NC, seed=1)
    with pytest.raises(lidar.LidarError, match="dense mode"):
        net.set_dense(7)
    net.close()


def test_load_rejects_other_shapes_and_garbage(tmp_path):
    a = lidar.TailNet(64, seed=1)
    b = lidar.TailNet(128, seed=1)
    path = str(tmp_path / "a.bin")
    a.save(path)
    with pytest.raises(lidar.LidarError, match="shape"):
        b.load(path)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a network")
    with pytest.raises(lidar.LidarError, match="not a tail network"):
        a.load(str(bad))
    a.close()
    b.close()


def test_surrogate_simulation_meets_parity():
    """Whatever the network predicts, the acceptance test keeps the result
    within the parity bar of the plain path."""
    w = S.small_plane_retro()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    lidar.lidar_tail_configure(L.handle, 0.3, 256)
    net = lidar.TailNet(256, seed=12)
    randomize(net, 12)  # an untrained network: arbitrary tails within the bound
    planes = lidar.gbuffer_to_device(w.gbuffer)
    g = lidar.make_gbuffer(w.gbuffer, [p.data_ptr() for p in planes])
    wave, ech, cnt = L.alloc_outputs()
    n = lidar.lidar_simulate_surrogate(L.handle, net.handle, g, lidar.make_pose(w.pose), wave.data_ptr(),
                                       ech.data_ptr(), cnt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert 0 <= n <= len(w.dirs)
    from tests.test_parity_gpu import ambiguous_ok, compare
    beams = np.arange(len(w.dirs), dtype=np.int32)
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    st = compare(ref, wave.cpu().numpy().astype(np.float64), lidar.echoes_numpy(ech), cnt.cpu().numpy(), beams,
                 w.calib["threshold"], w.calib["max_echoes"], w.pulse)
    assert ambiguous_ok(st), st
    net.close()
    L.close()


def test_committed_network_on_the_wide_frame():
    """The learned surrogate as shipped: the trained weights
    (weights/tailnet_wide.bin) on the 8192x4096 wide-tail frame with 200k
    beams, exact core 0.3 deg; the gated result on a seeded 1 % subsample
    (2000 beams) against the oracle, at the parity bar."""
    path = os.path.join(os.path.dirname(lidar.__file__), "weights", "tailnet_wide.bin")
    w = S.wide_frame()
    L = lidar.Lidar(w.profile, w.dirs, w.pulse, w.calib)
    lidar.lidar_tail_configure(L.handle, 0.3, 256)
    net = lidar.TailNet(256)
    net.load(path)
    planes = lidar.gbuffer_to_device(w.gbuffer)
    g = lidar.make_gbuffer(w.gbuffer, [p.data_ptr() for p in planes])
    wave, ech, cnt = L.alloc_outputs()
    n = lidar.lidar_simulate_surrogate(L.handle, net.handle, g, lidar.make_pose(w.pose), wave.data_ptr(),
                                       ech.data_ptr(), cnt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    lidar.lidar_sync(L.handle, 0)
    net.sync(0)
    # most beams keep the network's tail; the re-run ones are a few percent
    assert 0 < n < 0.05 * len(w.dirs), n
    from tests.test_parity_gpu import ambiguous_ok, compare
    beams = np.sort(S.rng(2000).choice(len(w.dirs), 2000, replace=False)).astype(np.int32)
    ref = O.simulate_workload(w, beams=beams, nthreads=NTHREADS, max_out=8)
    bi = torch.as_tensor(beams, device="cuda", dtype=torch.long)
    rows = {int(b): r for b, r in zip(beams, wave[bi].cpu().numpy().astype(np.float64))}
    st = compare(ref, rows, lidar.echoes_numpy(ech), cnt.cpu().numpy(), beams, w.calib["threshold"],
                 w.calib["max_echoes"], w.pulse)
    assert st["echoes"] >= 1000 and ambiguous_ok(st, strict=True), st
    net.close()
    L.close()
