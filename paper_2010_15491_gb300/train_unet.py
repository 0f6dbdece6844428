"""Trains the warm-start U-Net (the library's own forward and backward
kernels) on synthetic pairs and saves its parameters.

Pairs: the 256^3 headline recipe at 128^3 (200 ellipsoids plus a smooth
field, Gaussian PSF sigma 1.5, decimation 2x2x2, 40 dB), input the Tikhonov
solution (tau 1e-2, nearest-neighbour prior), target ADMM-TV (lambda 5e-4,
rho 1e-2) after --ref-iters iterations from it.  Training pair j uses phantom
seed 50000 + j and validation pair j seed 90000 + j.

    python -m paper_2010_15491_gb300.train_unet --pairs 2000 --epochs 10 --out weights.npy
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--val", type=int, default=16)
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--ref-iters", type=int, default=300)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=2e-5)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--init-seed", type=int, default=7)
    ap.add_argument("--out", required=True, help="parameter file (.npy, float32)")
    args = ap.parse_args(argv)

    from . import warmstart as W
    pool = W.phantom_pool(args.workers)  # host workers start before the first GPU call
    from . import UNet
    rec = W.PairRecipe(size=args.size, ref_iters=args.ref_iters)
    t0 = time.time()
    Xv, Tv = W.make_pairs(rec, [90000 + j for j in range(args.val)], pool=pool, log=None)
    X, T = W.make_pairs(rec, [50000 + j for j in range(args.pairs)], pool=pool)
    t_pairs = time.time() - t0
    pool.shutdown()
    net = UNet()
    net.set_params(W.init_params(args.init_seed))
    base = W.evaluate(net, Xv, Tv)
    print(f"pairs ready in {t_pairs:.1f} s; validation MSE of the identity (Tikhonov input) {base:.4e}", flush=True)
    t1 = time.time()
    hist = W.train(net, X, T, args.epochs, lr=args.lr, lr_final=args.lr_final, X_val=Xv, T_val=Tv)
    t_train = time.time() - t1
    theta = net.get_params()
    np.save(args.out, theta)
    meta = {"pairs": args.pairs, "val": args.val, "size": args.size, "ref_iters": args.ref_iters,
            "epochs": args.epochs, "lr": args.lr, "lr_final": args.lr_final, "identity_val_mse": base,
            "history": hist, "pair_seconds": t_pairs, "train_seconds": t_train}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps({k: v for k, v in meta.items() if k != "history"}), flush=True)


if __name__ == "__main__":
    main()
