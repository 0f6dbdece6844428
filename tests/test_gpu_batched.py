"""The batched solve (many volumes of uneven size and decimation in one CUDA
graph) against single-volume solves and the oracle."""
import numpy as np
import pytest

import oracle as O
from tests._problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu

VOLUMES = [((64, 64, 64), (2, 2, 2), 1e-2), ((96, 96, 64), (2, 2, 1), 3e-3), ((64, 32, 32), (1, 1, 4), 5e-2),
           ((32, 32, 16), (2, 2, 2), 1e-3), ((96, 24, 12), (2, 1, 3), 2e-2)]


def test_batched_equals_single_volume_solves(lib):
    import torch
    plans, ys, xs, probs = [], [], [], []
    for k, (dims, dec, tau) in enumerate(VOLUMES):
        psf, xt, y = make_problem(dims, dec, sigma=(1.0, 0.9, 1.1), seed=40 + k)
        p = lib.Plan(dims, dec, psf, "f32", stream=torch.cuda.Stream())
        plans.append(p)
        ys.append(torch.tensor(y, dtype=torch.float32, device="cuda"))
        xs.append(p.empty_hr())
        probs.append((psf, y, dec, tau))
    lams = [1e-3 * (1 + k) for k in range(len(plans))]
    rhos = [1e-2] * len(plans)
    taus = [v[2] for v in VOLUMES]
    for rep in range(2):  # the second call replays the cached graph
        lib.admm_tv_batched(plans, ys, xs, lams, rhos, taus, 7)
        for k, p in enumerate(plans):
            single = p.empty_hr()
            p.admm_tv(ys[k], single, lams[k], rhos[k], 7, tau_init=taus[k])
            assert torch.equal(single, xs[k]), (rep, k)
    for k in (0, 2, 4):
        psf, y, dec, tau = probs[k]
        x0 = O.tikhonov(y, psf, dec, tau, O.nearest_neighbour(y, dec))
        ref = O.admm_tv(y, psf, dec, lams[k], rhos[k], 7, x0)["x"]
        assert rel_l2(xs[k].cpu().numpy(), ref) < 1e-5
    for p in plans:
        p.close()


def test_batched_rejects_repeated_plans(lib):
    import torch
    psf, xt, y = make_problem((32, 32, 16), (2, 2, 2), seed=50)
    p = lib.Plan((32, 32, 16), (2, 2, 2), psf, "f32", stream=torch.cuda.Stream())
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.Sr3dError):
        lib.admm_tv_batched([p, p], [yd, yd], [p.empty_hr(), p.empty_hr()], [1e-3] * 2, [1e-2] * 2, [1e-2] * 2, 4)
    p.close()


def test_autotuned_plans_keep_parity(lib):
    import torch
    dims, dec = (128, 64, 32), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=60)
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, 1e-3, 1e-2, 6, x0)["x"]
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    for _ in range(2):  # the second plan applies the cached schedule
        p = lib.Plan(dims, dec, psf, "f32", stream=torch.cuda.Stream())
        p.autotune(2)
        x = p.empty_hr()
        p.admm_tv(yd, x, 1e-3, 1e-2, 6, tau_init=1e-2)
        assert rel_l2(x.cpu().numpy(), ref) < 1e-5
        xs = [p.empty_hr()]
        lib.admm_tv_batched([p], [yd], xs, [1e-3], [1e-2], [1e-2], 6)
        assert torch.equal(xs[0], x)
        p.close()
