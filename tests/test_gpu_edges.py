"""Edge cases on the GPU against the oracle: the largest supported length on
each axis, the smallest s extent, a delta PSF (no blur), a zero TV weight and
a non-power-of-two length at the limits of the plans."""
import numpy as np
import pytest

import oracle as O
from tests._problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


def T(a, dtype="f32"):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype={"f32": torch.float32, "f64": torch.float64}[dtype],
                        device="cuda")


def H(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dims,dec", [((2048, 8, 4), (2, 1, 1)), ((32, 2048, 4), (1, 2, 1)),
                                      ((32, 8, 2048), (1, 1, 4)), ((1536, 16, 8), (2, 2, 2))])
def test_longest_axes(lib, dims, dec):
    psf, xt, y = make_problem(dims, dec, sigma=(1.0, 1.0, 1.0), seed=121, n_ell=4)
    plan = lib.Plan(dims, dec, psf, "f32")
    x = plan.tikhonov(T(y), 1e-2, xbar="nearest")
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    assert rel_l2(H(x), x0) < 1e-5
    xa = plan.empty_hr()
    plan.admm_tv(T(y), xa, 1e-3, 1e-2, 3, tau_init=1e-2)
    assert rel_l2(H(xa), O.admm_tv(y, psf, dec, 1e-3, 1e-2, 3, x0)["x"]) < 1e-5
    plan.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_delta_psf_and_smallest_s(lib, dtype):
    """A 1x1x1 PSF (H = I) on the smallest s extent (4 planes): Tikhonov has
    the voxelwise closed form of the oracle, and ADMM follows the oracle."""
    dims, dec = (64, 16, 4), (2, 2, 2)
    psf = np.ones((1, 1, 1))
    _, xt, _ = make_problem(dims, dec, seed=122)
    y = O.forward(xt, psf, dec) + 0.01 * np.random.default_rng(123).standard_normal((2, 8, 32))
    plan = lib.Plan(dims, dec, psf, dtype)
    tol = 1e-5 if dtype == "f32" else 1e-12
    for prior in (None, "nearest"):
        x = plan.tikhonov(T(y, dtype), 0.3, xbar=prior)
        xb = None if prior is None else O.nearest_neighbour(y, dec)
        assert rel_l2(H(x), O.tikhonov(y, psf, dec, 0.3, xb)) < tol
    xa = plan.empty_hr()
    plan.admm_tv(T(y, dtype), xa, 2e-3, 1e-1, 5, tau_init=0.3)
    x0 = O.tikhonov(y, psf, dec, 0.3, O.nearest_neighbour(y, dec))
    assert rel_l2(H(xa), O.admm_tv(y, psf, dec, 2e-3, 1e-1, 5, x0)["x"]) < tol
    plan.close()


def test_zero_tv_weight(lib):
    """lambda = 0: the u-step keeps nu (no shrink), and the iterates still
    follow the oracle."""
    dims, dec = (128, 32, 16), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=124)
    plan = lib.Plan(dims, dec, psf, "f64")
    x = plan.empty_hr()
    plan.admm_tv(T(y, "f64"), x, 0.0, 1e-2, 6, tau_init=1e-2)
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    assert rel_l2(H(x), O.admm_tv(y, psf, dec, 0.0, 1e-2, 6, x0)["x"]) < 1e-12
    plan.close()
