"""The allocation-free Tikhonov entry point (sr3d_tikhonov_noalloc) against
the planned one (sr3d_tikhonov), through the C ABI.

It serves callers that cannot allocate device memory while running (fixed
memory budgets, code inside CUDA stream capture); its work memory is one
fixed device array inside the library, reused by every call.  This file is
collected last so that a failure here never hides the other tests.
"""
import numpy as np
import pytest

from tests._problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("f64", 1e-11)])
def test_noalloc_matches_planned_tikhonov_on_consecutive_calls(lib, dtype, tol):
    import torch
    td = {"f32": torch.float32, "f64": torch.float64}[dtype]
    dims, dec = (64, 32, 32), (2, 2, 2)
    plan = None
    for call, (seed, tau, prior) in enumerate([(31, 1e-2, "nearest"), (32, 0.3, None)]):
        psf, _, y = make_problem(dims, dec, sigma=(1.0, 0.8, 1.2), seed=seed, asym=True)
        yd = torch.tensor(y, dtype=td, device="cuda")
        plan = lib.Plan(dims, dec, psf, dtype)
        ref = plan.tikhonov(yd, tau, xbar=prior)
        plan.close()
        got = torch.full_like(ref, float("nan"))
        lib.tikhonov_noalloc(dims, dec, psf, yd, tau, got, xbar=prior, dtype=dtype)
        err = rel_l2(got.cpu().numpy(), ref.cpu().numpy())
        assert err < tol, (call, err)


def test_noalloc_rejects_volumes_beyond_its_scratch(lib):
    import torch
    dims, dec = (256, 256, 64), (2, 2, 2)
    psf = np.ones((3, 3, 3)) / 27.0
    y = torch.zeros((32, 128, 128), dtype=torch.float32, device="cuda")
    x = torch.zeros((64, 256, 256), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.Sr3dError) as e:
        lib.tikhonov_noalloc(dims, dec, psf, y, 1e-2, x)
    assert e.value.name == "UNSUPPORTED_SIZE" and "sr3d_plan" in str(e.value)
