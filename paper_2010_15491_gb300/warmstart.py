"""Learned warm start for ADMM-TV (not in the paper).

The paper's ADMM-TV (Algorithm 1) starts from the Tikhonov solution of Eq. 12.
Here a 3D U-Net (the library's UNet, BF16 tensor-core kernels) maps that
Tikhonov estimate x_tik to a starting point x0 close to the ADMM-TV solution,
and the dual starts consistent with x0 (Plan.dual_init):

    x_tik = Tikhonov(y; tau, nearest-neighbour prior)      (Eq. 12)
    x0    = UNet(x_tik)
    d0_j  = t g_j / max(||g_j||, t),  g = L x0,  t = lambda / rho
    x     = ADMM-TV from (x0, u0 = L x0, d0) until both relative residuals < tol

Training pairs are (x_tik, x_ref) with x_ref = ADMM-TV after a fixed number of
iterations from the Tikhonov start; every pair is computed by the library's
own kernels on the GPU, and the network is trained by its own forward and
backward kernels (UNet.train_step, Adam).

Phantoms come from the seeded synthetic generator (`synth`), on host worker
processes; everything after the phantom runs on the GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import time
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import Plan, UNet


def warm_start(plan: Plan, net: UNet, y, lam: float, rho: float, tau: float, dual: bool = True):
    """x0 = UNet(Tikhonov(y)) and the dual consistent with it (None with
    dual=False: ADMM then starts from d0 = 0); returns (x0, d0)."""
    x_tik = plan.tikhonov(y, tau, xbar="nearest")
    x0 = net.forward(x_tik)
    d0 = plan.dual_init(x0, lam, rho) if dual else None
    return x0, d0


def solve(plan: Plan, y, lam: float, rho: float, tau: float, tol: float, max_iters: int,
          eval_every: int = 5, net: Optional[UNet] = None, dual: bool = True):
    """ADMM-TV to tolerance, cold (Tikhonov start, d0 = 0) or warm (net given;
    dual=False keeps d0 = 0).  Returns (x, statistics)."""
    if net is None:
        x = plan.empty_hr()
        st = plan.admm_tv(y, x, lam, rho, max_iters, tol=tol, tau_init=tau, eval_every=eval_every)
    else:
        x, d = warm_start(plan, net, y, lam, rho, tau, dual)
        st = plan.admm_tv(y, x, lam, rho, max_iters, d=d, tol=tol, eval_every=eval_every)
    return x, st


# ---------------------------------------------------------------------------
# training data and training
# ---------------------------------------------------------------------------

@dataclass
class PairRecipe:
    """How training pairs are made (the 256^3 headline recipe at another size)."""
    size: int = 128
    dec: tuple = (2, 2, 2)
    sigma: float = 1.5
    n_ellipsoids: int = 200
    field: float = 0.1
    snr_db: float = 40.0
    tau: float = 1e-2
    lam: float = 5e-4
    mu: float = 1e-2
    ref_iters: int = 300


def _phantom(args):
    import synth
    size, n_ell, seed, field = args
    return synth.ellipsoid_phantom((size, size, size), n_ell, seed, field).astype(np.float32)


def phantom_pool(workers: int):
    """A host process pool for phantoms; create it before the first GPU call."""
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def observe(plan: Plan, x_true, snr_db: float, seed: int):
    """y = D H x + n with the seeded noise field of `seed` at `snr_db`."""
    import torch
    import synth
    y = plan.forward(x_true)
    sig = synth.noise_sigma(y.double().cpu().numpy(), snr_db)
    return y + torch.tensor(sig * synth.noise_field(tuple(y.shape), seed), dtype=torch.float32, device=y.device)


def make_pairs(recipe: PairRecipe, seeds, pool=None, log=print):
    """Tikhonov inputs and ADMM-TV targets for each seed, resident on the GPU
    as two (P, s, n, m) FP32 tensors."""
    import torch
    import synth
    r = recipe
    psf = synth.gaussian_psf((r.sigma,) * 3)
    plan = Plan((r.size,) * 3, r.dec, psf, "f32")
    P = len(seeds)
    X = torch.empty((P,) + plan.hr_shape, dtype=torch.float32, device="cuda")
    T = torch.empty_like(X)
    jobs = [(r.size, r.n_ellipsoids, int(s), r.field) for s in seeds]
    it = pool.map(_phantom, jobs, chunksize=1) if pool is not None else map(_phantom, jobs)
    t0 = time.time()
    for i, (ph, seed) in enumerate(zip(it, seeds)):
        x_true = torch.from_numpy(ph).cuda()
        y = observe(plan, x_true, r.snr_db, int(seed))
        plan.tikhonov(y, r.tau, x=X[i], xbar="nearest")
        T[i].copy_(X[i])
        plan.admm_tv(y, T[i], r.lam, r.mu, r.ref_iters)
        if log and (i + 1) % max(1, P // 10) == 0:
            log(f"pairs {i + 1}/{P}  {time.time() - t0:.1f} s")
    torch.cuda.synchronize()
    plan.close()
    return X, T


def init_params(seed: int = 7) -> np.ndarray:
    """He-scaled normal weights (std sqrt(2 / (27 c_in))), zero biases and a
    zero head, so that the untrained network is the identity."""
    import synth
    from . import load
    n = int(load().sr3d_unet_param_count())
    z = synth.normal(seed, 0, n)
    theta = np.zeros(n)
    o = 0
    for co, ci in UNET_LAYERS:
        nw = co * 27 * ci
        theta[o:o + nw] = z[o:o + nw] * np.sqrt(2.0 / (27 * ci))
        o += nw + co
    return theta.astype(np.float32)


# (c_out, c_in) of the ten 3x3x3 layers, in parameter order
UNET_LAYERS = [(16, 1), (16, 16), (32, 16), (32, 32), (64, 32), (64, 64), (32, 96), (32, 32), (16, 48), (16, 16)]


def train(net: UNet, X, T, epochs: int, lr: float = 1e-3, lr_final: float = 1e-4, seed: int = 11,
          X_val=None, T_val=None, log=print):
    """Adam over the pairs (one volume per step, shuffled each epoch), learning
    rate decaying geometrically from lr to lr_final; returns the history."""
    import synth
    P = X.shape[0]
    steps = epochs * P
    hist = {"train": [], "val": []}
    k = 0
    t0 = time.time()
    for ep in range(epochs):
        order = np.argsort(synth.uniform(seed, ep, P))
        tot = 0.0
        for i in order:
            rate = lr * (lr_final / lr) ** (k / max(1, steps - 1))
            loss, _ = net.train_step(X[i], T[i], lr=rate)
            tot += loss
            k += 1
        hist["train"].append(tot / P)
        if X_val is not None:
            hist["val"].append(evaluate(net, X_val, T_val))
        if log:
            log(f"epoch {ep + 1}/{epochs}  train {hist['train'][-1]:.4e}"
                + (f"  val {hist['val'][-1]:.4e}" if hist["val"] else "") + f"  {time.time() - t0:.1f} s")
    return hist


def evaluate(net: UNet, X, T) -> float:
    """Mean squared error of the network over pairs."""
    import torch
    tot = 0.0
    for i in range(X.shape[0]):
        out = net.forward(X[i])
        tot += float(torch.mean((out - T[i]) ** 2))
    return tot / X.shape[0]
