"""Parity of whole benchmark workloads with the FP64 oracle, through the C ABI.

  * 32^3 in FP64 (12 ellipsoids, sigma 1 on 7^3 taps, d = 2x2x2, 40 dB):
    Tikhonov start (tau 1e-2, nearest-neighbour prior, eq. 12) and all 20
    ADMM-TV iterations (lambda 1e-3, mu 1e-2, Algorithm 1), every iterate
    within 1e-12 of the oracle.
  * 256^3 in FP32 (the benchmark, 100 iterations) and the anisotropic
    CBCT-like recipe (d = 1x1x4, sigma (1, 1, 2) on 7x7x13 taps, 35 dB, 200
    iterations) at 512 x 512 x 32: the FP32 iterate against the oracle's
    after k iterations, on a seeded sample of 4096 voxels, within 1e-5
    relative L2, together with the GPU's FP64 objective.  The oracle needs
    minutes for these runs, so tests/golden/make_long_runs.py stored its
    sampled iterates once; each test first re-runs the oracle here for the
    start and two iterations and checks that the stored values reproduce.
"""
import os

import numpy as np
import pytest

import oracle as O
from tests._problems import rel_l2

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def T(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype={"f32": torch.float32, "f64": torch.float64}[dtype],
                        device="cuda")


def H(t):
    return t.detach().cpu().numpy().astype(np.float64)


def test_config_32cubed_fp64_every_iterate(lib, request):
    import synth
    import torch
    w = synth.SMALL_FP64
    psf = w.psf()
    clean = O.forward(w.phantom(), psf, w.dec)
    y = clean + synth.noise_sigma(clean, w.snr_db) * w.noise()
    x0 = O.tikhonov(y, psf, w.dec, w.tau, O.nearest_neighbour(y, w.dec))
    iters = {}
    ref = O.admm_tv(y, psf, w.dec, w.lam, w.mu, w.iters, x0, record=True,
                    callback=lambda i, xi, u, d: iters.__setitem__(i + 1, xi.copy()))
    plan = lib.Plan(w.dims, w.dec, psf, "f64")
    yd = T(y, "f64")
    tol = 1e-12
    name = request.node.name
    xk = plan.tikhonov(yd, w.tau, xbar="nearest")
    assert rel_l2(H(xk), x0, f"{name}:x0") < tol
    for k in range(1, w.iters + 1):
        xg = plan.empty_hr()
        plan.admm_tv(yd, xg, w.lam, w.mu, k, tau_init=w.tau)
        assert rel_l2(H(xg), iters[k], f"{name}:x{k}") < tol, k
    xg = plan.empty_hr()
    d = torch.zeros((3,) + plan.hr_shape, dtype=torch.float64, device="cuda")
    st = plan.admm_tv(yd, xg, w.lam, w.mu, w.iters, d=d, tau_init=w.tau, eval_every=1, hist_len=w.iters)
    assert rel_l2(H(xg), ref["x"], f"{name}:x_stats") < tol
    assert rel_l2(H(d), ref["d"], f"{name}:d") < tol
    hist = np.array(st["objective_hist"])
    assert rel_l2(hist, np.array(ref["hist"]["objective"]), f"{name}:objective") < tol
    plan.close()


def _long_run(lib, name, request, autotune=True):
    from tests.golden.make_long_runs import workloads, problem, sample_indices
    w, _ = workloads()[name]
    g = np.load(os.path.join(GOLDEN, f"admm_{name}.npz"))
    assert tuple(g["dims"]) == w.dims and tuple(g["dec"]) == w.dec
    psf, y = problem(w)
    idx = sample_indices(w)
    assert np.array_equal(idx, g["idx"])
    # the stored oracle values reproduce on this host: start and two iterations
    x0 = O.tikhonov(y, psf, w.dec, w.tau, O.nearest_neighbour(y, w.dec))
    live = {0: x0.ravel()[idx].copy()}
    O.admm_tv(y, psf, w.dec, w.lam, w.mu, 2, x0,
              callback=lambda i, xi, u, d: live.__setitem__(i + 1, xi.ravel()[idx].copy()))
    ks = list(g["ks"])
    for k in (0, 1, 2):
        assert rel_l2(g["x"][ks.index(k)], live[k]) < 1e-10, k
    plan = lib.Plan(w.dims, w.dec, psf, "f32")
    if autotune:
        plan.autotune()
    yd = T(y, "f32")
    errs = {}
    for j, k in enumerate(ks):
        xg = plan.empty_hr()
        plan.admm_tv(yd, xg, w.lam, w.mu, int(k), tau_init=w.tau)
        got = H(xg).ravel()
        errs[int(k)] = rel_l2(got[idx], g["x"][j], f"{request.node.name}:x{k}")
        assert np.isclose(np.linalg.norm(got), g["norm"][j], rtol=1e-5, atol=0), k
    assert max(errs.values()) < 1e-5, errs
    # the FP64 objective of the GPU's statistics after the last iteration
    k = int(ks[-1])
    xg = plan.empty_hr()
    st = plan.admm_tv(yd, xg, w.lam, w.mu, k, tau_init=w.tau, eval_every=0)
    assert st["iters"] == k
    assert np.isclose(st["objective"], g["objective"][-1], rtol=1e-5, atol=0), (st["objective"], g["objective"][-1])
    assert rel_l2(H(xg).ravel()[idx], g["x"][-1]) < 1e-5
    plan.close()
    return errs


@pytest.mark.slow
def test_headline_256_error_curve_over_100_iterations(lib, request):
    """FP32 error against the FP64 oracle after 0 (Tikhonov), 1, 2, 5, 10, 25,
    50 and 100 iterations of the benchmark workload, in the benchmark's launch
    configuration (autotuned schedule, no statistics)."""
    _long_run(lib, "hr256_d2", request)


@pytest.mark.slow
def test_aniso_512x512x32_d114_over_200_iterations(lib, request):
    """The anisotropic CBCT-like recipe (d = 1x1x4) with 512-point transforms
    along m and n: FP32 iterates after up to 200 iterations."""
    _long_run(lib, "aniso512x512x32_d114", request)
