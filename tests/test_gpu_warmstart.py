"""What the trained warm-start network gains over the plain method.

On held-out phantoms of the training recipe (128^3, seeds 90000 + j, never
used for training), ADMM-TV (Algorithm 1) is run to relative primal and dual
residuals below 1e-4 from three starts:
  cold      the paper's start: Tikhonov (eq. 12), d0 = 0;
  identity  the same Tikhonov start with the consistent dual (an untrained,
            all-zero network is the identity map);
  warm      Tikhonov -> trained U-Net -> consistent dual.
The warm start must reach the same tolerance, at the same objective value, in
fewer iterations than both others and in less wall-clock time than cold,
the network's inference included.  Cold-start ADMM stays the reference solution.
"""
import os
import time

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2010_15491_gb300",
                       "weights", "unet_warmstart.npy")


def test_trained_warm_start_converges_in_fewer_iterations_and_less_time(lib):
    import torch
    import synth
    from paper_2010_15491_gb300 import warmstart as W
    r = W.PairRecipe()
    plan = lib.Plan((r.size,) * 3, r.dec, synth.gaussian_psf((r.sigma,) * 3), "f32")
    net = lib.UNet()
    net.set_params(np.load(WEIGHTS))
    ident = lib.UNet()  # all parameters zero: the identity map
    tol, every, cap = 1e-4, 10, 5000

    def run(y, model):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, st = W.solve(plan, y, r.lam, r.mu, r.tau, tol, cap, eval_every=every, net=model)
        torch.cuda.synchronize()
        return st, time.perf_counter() - t0

    report = []
    for seed in (90000, 90001, 90002):
        x_true = torch.from_numpy(W._phantom((r.size, r.n_ellipsoids, seed, r.field))).cuda()
        y = W.observe(plan, x_true, r.snr_db, seed)
        for model in (None, net, ident):  # load every kernel and graph once
            run(y, model)
        cold, t_cold = min((run(y, None) for _ in range(2)), key=lambda v: v[1])
        warm, t_warm = min((run(y, net) for _ in range(2)), key=lambda v: v[1])
        idn, _ = run(y, ident)
        report.append((seed, cold["iters"], warm["iters"], idn["iters"], 1e3 * t_cold, 1e3 * t_warm))
        assert cold["converged"] and warm["converged"] and idn["converged"], report[-1]
        assert warm["primal_rel"] < tol and warm["dual_rel"] < tol
        assert warm["iters"] < cold["iters"] and warm["iters"] < idn["iters"], report[-1]
        assert abs(warm["objective"] - cold["objective"]) <= 1e-3 * cold["objective"], (warm, cold)
        assert t_warm < t_cold, report[-1]
    print("seed, cold iters, warm iters, identity iters, cold ms, warm ms:", report)
    plan.close()
    net.close()
    ident.close()
