"""Trains the learned-gamma MLP on the GPU with the library's own kernels.

Data: seeded synthetic volumes (blobs + value noise, 256^3 uint16 by default)
split into a K-brick decomposition, several orbit views each; per (PE, 16 x 16
tile) the features (vdi_tile_features) and the label from the per-ray
bisection search (vdi_choose_gamma + vdi_tile_labels).  Training: Adam on the
mean squared error of log2 gamma (vdi_mlp_train_step), mini-batches drawn from
a seeded permutation.  The gamma offset is then calibrated on held-out volumes:
the smallest offset whose supersegment-count error against the search is at
most --target-error.  Writes the checkpoint and a JSON report beside it.

    python -m paper_2206_14503_gb300.train_gamma --volumes 2000 --views 8
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_CKPT = os.path.join(HERE, "models", "gamma_ns32_k16.ckpt")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--volumes", type=int, default=2000)
    ap.add_argument("--views", type=int, default=8)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--res", type=int, default=512)
    ap.add_argument("--n-s", type=int, default=32)
    ap.add_argument("--grid", type=int, nargs=3, default=(4, 2, 2))
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--holdout", type=float, default=0.02)
    ap.add_argument("--target-error", type=float, default=0.04)
    ap.add_argument("--out", default=DEFAULT_CKPT)
    return ap.parse_args(argv)


def volume_seed(v):
    return 0x5EED0000 + v


def blob_count(v):
    return 32 + (v * 37) % 129


def make_dataset(vdi, torch, args, vols, lut_d, boxes):
    """Features, labels and validity of every (PE, tile) of the given volumes' views."""
    import synth
    from synth import gpu_volume

    S = args.size
    dims = (S, S, S)
    k = len(boxes)
    R = args.res
    tiles = ((R + 15) // 16) ** 2
    npix = R * R
    outs = [vdi.Compact(npix, 1) for _ in range(k)]
    ws = vdi.Workspace(vdi.vdi_generate_workspace(k, R, R))
    params = vdi.make_params()
    F = torch.zeros((k, tiles, 40), dtype=torch.float32, device="cuda")
    FV = torch.zeros((k, tiles), dtype=torch.uint8, device="cuda")
    L = torch.zeros((k, tiles), dtype=torch.float32, device="cuda")
    LV = torch.zeros((k, tiles), dtype=torch.uint8, device="cuda")
    xs, ys = [], []
    bricks = None
    for v in vols:
        vol = gpu_volume.volume(dims, blob_count(v), 3 + v % 2, volume_seed(v))
        if bricks is None:
            bricks = vdi.Bricks(vol, dims, boxes)
        else:
            bricks.rebuild(vol)
        for cam in synth.orbit(dims, args.views, R, R, 0xCAFE00 + v):
            c = vdi.make_camera(cam)
            vdi.check(vdi.vdi_choose_gamma(bricks.bricks, lut_d.data_ptr(), c, args.n_s, vdi.VDI_GAMMA_SEARCH,
                                           [o.struct() for o in outs], params, ws.ptr, ws.nbytes), "search")
            vdi.check(vdi.vdi_tile_labels([o.struct() for o in outs], R, R, L.data_ptr(), LV.data_ptr()), "labels")
            vdi.check(vdi.vdi_tile_features(bricks.bricks, lut_d.data_ptr(), c, args.n_s, params, F.data_ptr(),
                                            FV.data_ptr()), "features")
            keep = (FV & LV).reshape(-1).bool()
            xs.append(F.reshape(-1, 40)[keep].clone())
            ys.append(L.reshape(-1)[keep].clone())
    return torch.cat(xs), torch.cat(ys)


def count_error(vdi, torch, args, model, offset, vols, lut_d, boxes):
    """Supersegment-count error of learned generation against the search, and the fallback fraction."""
    import synth
    from synth import gpu_volume

    S, R = args.size, args.res
    dims = (S, S, S)
    k = len(boxes)
    npix = R * R
    search = [vdi.Compact(npix, 1) for _ in range(k)]
    learned = [vdi.Compact(npix, 1) for _ in range(k)]
    ws = vdi.Workspace(vdi.vdi_generate_workspace(k, R, R))
    lws = vdi.Workspace(vdi.vdi_learned_workspace(k, R, R))
    census = vdi.make_params(flags=vdi.VDI_FLAG_CENSUS)
    extra = lws.nbytes - vdi.vdi_generate_workspace(k, R, R)
    diff = tot = fell = rays = 0
    bricks = None
    for v in vols:
        vol = gpu_volume.volume(dims, blob_count(v), 3 + v % 2, volume_seed(v))
        if bricks is None:
            bricks = vdi.Bricks(vol, dims, boxes)
        else:
            bricks.rebuild(vol)
        for cam in synth.orbit(dims, args.views, R, R, 0xCAFE00 + v):
            c = vdi.make_camera(cam)
            vdi.check(vdi.vdi_choose_gamma(bricks.bricks, lut_d.data_ptr(), c, args.n_s, vdi.VDI_GAMMA_SEARCH,
                                           [o.struct() for o in search], vdi.make_params(), ws.ptr, ws.nbytes), "s")
            vdi.check(vdi.vdi_choose_gamma_learned(bricks.bricks, lut_d.data_ptr(), c, args.n_s, model.data_ptr(),
                                                   offset, [o.struct() for o in learned], census, lws.ptr,
                                                   lws.nbytes), "l")
            ctr = vdi.vdi_workspace_counters(lws.ptr + extra)
            cs = torch.stack([o.counts for o in search]).long()
            cl = torch.stack([o.counts for o in learned]).long()
            nz = cs > 0
            diff += int((cl - cs).abs()[nz].sum())
            tot += int(cs[nz].sum())
            fell += ctr[4]
            rays += ctr[3]
    return diff / max(tot, 1), fell / max(rays, 1)


def main(argv=None):
    args = parse(argv)
    import torch

    import paper_2206_14503_gb300 as vdi
    import synth

    torch.cuda.init()
    t0 = time.time()
    lut_d = torch.from_numpy(synth.transfer_function(synth.SEED_TF)).cuda()
    boxes = vdi.vdi_split_boxes((args.size,) * 3, tuple(args.grid))
    n_hold = max(1, int(round(args.volumes * args.holdout)))
    train_vols = list(range(args.volumes - n_hold))
    hold_vols = list(range(args.volumes - n_hold, args.volumes))
    X, Y = make_dataset(vdi, torch, args, train_vols, lut_d, boxes)
    t_data = time.time() - t0
    n = X.shape[0]
    model = torch.zeros(vdi.vdi_model_bytes(), dtype=torch.uint8, device="cuda")
    vdi.check(vdi.vdi_model_init(model.data_ptr(), args.seed), "init")
    batch = min(args.batch, n)
    ws = vdi.Workspace(vdi.vdi_mlp_train_workspace(batch))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ones = torch.ones(batch, dtype=torch.uint8, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed)
    perm = torch.randperm(n, device="cuda", generator=gen)
    pos = 0
    losses = []
    t1 = time.time()
    for s in range(args.steps):
        if pos + batch > n:
            perm = torch.randperm(n, device="cuda", generator=gen)
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        xb = X[idx].contiguous()
        yb = Y[idx].contiguous()
        lr = args.lr if s < args.steps * 0.6 else args.lr * 0.2
        vdi.check(vdi.vdi_mlp_train_step(model.data_ptr(), xb.data_ptr(), yb.data_ptr(), ones.data_ptr(), batch, lr,
                                         loss.data_ptr(), ws.ptr, ws.nbytes), "train")
        if s % 100 == 0 or s == args.steps - 1:
            losses.append((s, float(loss.item())))
    t_train = time.time() - t1
    # calibrate the offset on held-out volumes
    calib = []
    offset = None
    for off in [0.0, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.0]:
        err, fb = count_error(vdi, torch, args, model, off, hold_vols, lut_d, boxes)
        calib.append({"offset": off, "count_error": err, "fallback": fb})
        if err <= args.target_error:
            offset = off
            break
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    vdi.check(vdi.vdi_model_save(model.data_ptr(), args.out), "save")
    report = {"volumes": args.volumes, "views": args.views, "size": args.size, "res": args.res, "n_s": args.n_s,
              "grid": list(args.grid), "train_rows": n, "holdout_volumes": len(hold_vols), "steps": args.steps,
              "batch": batch, "lr": args.lr, "seed": args.seed, "losses": losses, "offset": offset,
              "calibration": calib, "seconds_data": t_data, "seconds_train": t_train}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps({k: report[k] for k in ("train_rows", "offset", "seconds_data", "seconds_train")}))
    print("final loss", losses[-1], "calibration", calib[-1])


if __name__ == "__main__":
    main()
