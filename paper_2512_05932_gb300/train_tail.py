"""Training of the learned tail estimator (lidar_tailnet_*) on footprints
generated by the library's own exact path.

Data: seeded frames of the plane/retro scene family with the wide-tail sensor
(radial profile sigma 0.05 deg + 1e-4 (theta / 0.05 deg)^-3 tail truncated
at 2 deg, 4096 bins of 0.05 ns): 4096x2048 frames of the wide-frame scene
(a plane at 10 m with retro patches, ground, boxes at 5-25 m; 250x200 grid
beams each) and 1024x1024 frames of a plane with a retro patch near the
boresight (100x100 grid beams each). Per beam the sample is the network input
and the physics prior (lidar_tail_features) and, as the target, the exact
coarse tail (lidar_tail_exact), everything kept in device memory.

  python -m paper_2512_05932_gb300.train_tail --out weights.bin [--wide 16 --plane 20 --epochs 6]

Writes the FP32 weights (and, with --checkpoint, a resumable checkpoint with
the Adam state) and prints a JSON summary with the held-out L1 error of the
prior and of the network relative to the exact tail's mass.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lidar
from . import scenes as S

CORE_DEG = 0.3
N_COARSE = 256


def wide_sensor():
    """Profile, pulse and calibration of the wide-tail frame."""
    return (S.radial_profile(0.05, 1e-4, 0.05, 3.0, 2.0), S.pulse(4096, 0.05e-9), S.calib(1e-5, 1e-4, 3, True))


def training_frames(seed, n_wide, n_plane):
    """Yields (name, GBuffer, dirs) of the training frames."""
    for i in range(n_wide):
        w = S.wide_frame(seed=seed + i, U=4096, V=2048, n_az=250, n_el=200)
        yield f"wide{i}", w.gbuffer, w.dirs
    g = S.rng(seed + 10_000)
    for i in range(n_plane):
        gb = S.plane_retro_frame(g, 1024, 1024, np.eye(3))
        dirs = S.grid_pattern(100, 100, 0.9 * 1024 * 0.02 * S.DEG, 0.9 * 1024 * 0.02 * S.DEG)
        yield f"plane{i}", gb, dirs


def collect(frames, device="cuda"):
    """Network inputs, prior rows and exact-tail rows of every beam of the frames."""
    import torch
    prof, pulse, cal = wide_sensor()
    X, R, T = [], [], []
    for _, gb, dirs in frames:
        L = lidar.Lidar(prof, dirs, pulse, cal)
        lidar.lidar_tail_configure(L.handle, CORE_DEG, N_COARSE)
        planes = lidar.gbuffer_to_device(gb, device)
        g = lidar.make_gbuffer(gb, [p.data_ptr() for p in planes])
        pose = lidar.make_pose(np.eye(3))
        n = len(dirs)
        x = torch.empty((n, lidar.TAIL_INPUT_CELLS, 2), dtype=torch.float16, device=device)
        r = torch.zeros((n, N_COARSE + 4), dtype=torch.float32, device=device)
        t = torch.zeros_like(r)
        s = torch.cuda.current_stream().cuda_stream
        lidar.lidar_tail_features(L.handle, g, pose, r.data_ptr(), x.data_ptr(), s)
        lidar.lidar_tail_exact(L.handle, g, pose, t.data_ptr(), s)
        torch.cuda.synchronize()
        lidar.lidar_sync(L.handle, 0)
        L.close()
        keep = (r[:, N_COARSE + 1] > 0)  # beams with a tail at all
        X.append(x[keep]); R.append(r[keep]); T.append(t[keep])
        del planes
    return torch.cat(X), torch.cat(R), torch.cat(T)


def rel_l1(pred, target):
    """Per-beam sum |pred - target| / sum target over the coarse bins (beams with a tail)."""
    p, t = pred[:, :N_COARSE].double(), target[:, :N_COARSE].double()
    m = t.sum(1)
    ok = m > 0
    return ((p - t).abs().sum(1)[ok] / m[ok]).cpu().numpy()


def evaluate(net, X, R, T, chunk=65536):
    import torch
    out = torch.zeros_like(R)
    for i in range(0, len(R), chunk):
        net.predict(X[i:i + chunk], R[i:i + chunk], out[i:i + chunk])
    torch.cuda.synchronize()
    e_net, e_prior = rel_l1(out, T), rel_l1(R, T)
    def q(a):
        return {"p50": float(np.median(a)), "p90": float(np.quantile(a, 0.9)), "mean": float(a.mean())}
    return {"net": q(e_net), "prior": q(e_prior), "beams": int(len(e_net))}


def train(net, X, R, T, epochs, batch, lr, seed, log=None):
    import torch
    n = len(R)
    g = torch.Generator(device="cpu").manual_seed(seed)
    steps = epochs * (n // batch)
    hist = []
    k = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        for i in range(n // batch):
            idx = perm[i * batch:(i + 1) * batch]
            lr_k = lr * 0.5 * (1 + math.cos(math.pi * k / max(1, steps)))
            want = (k % 200 == 0) or k == steps - 1
            loss = net.train_step(X[idx], R[idx], T[idx], lr_k, want_loss=want)
            if want:
                hist.append((k, float(loss)))
                if log:
                    log(f"step {k}/{steps} epoch {ep} loss {loss:.5f} ({time.perf_counter() - t0:.1f} s)")
            k += 1
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--resume", default=None)
    ap.add_argument("--wide", type=int, default=16)
    ap.add_argument("--plane", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=2024)
    a = ap.parse_args(argv)
    lidar.load()
    t0 = time.perf_counter()
    X, R, T = collect(training_frames(a.seed, a.wide, a.plane))
    Xv, Rv, Tv = collect(training_frames(a.seed + 500, 1, 2))
    t_data = time.perf_counter() - t0
    net = lidar.TailNet(N_COARSE, seed=a.seed)
    if a.resume:
        net.load(a.resume)
    before = evaluate(net, Xv, Rv, Tv)
    hist, t_train = train(net, X, R, T, a.epochs, a.batch, a.lr, a.seed, log=lambda s: print(s, flush=True))
    after = evaluate(net, Xv, Rv, Tv)
    net.save(a.out, with_state=False)
    if a.checkpoint:
        net.save(a.checkpoint, with_state=True)
    summary = {"train_beams": int(len(R)), "val_beams": int(len(Rv)), "data_s": t_data, "train_s": t_train,
               "epochs": a.epochs, "batch": a.batch, "lr": a.lr, "seed": a.seed, "loss_first_last": [hist[0], hist[-1]],
               "val_rel_l1_before": before, "val_rel_l1_after": after, "params": net.num_params}
    print(json.dumps(summary), flush=True)
    net.close()
    return summary


if __name__ == "__main__":
    main()
