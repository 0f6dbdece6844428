"""The allocation-free Tikhonov entry point (sr3d_tikhonov_noalloc) against
the planned one (sr3d_tikhonov) and the FP64 oracle, through the C ABI.

It serves callers that may not allocate device memory once running (a
device-memory budget fixed at start-up, or a host application that owns the
device's memory pool); its work memory is one fixed device array inside the
library, reused by every call.  Each case makes two calls in a row, so the
second one runs on the scratch contents the first left behind.  This file is
collected last so that a failure here never hides the other tests.
"""
import numpy as np
import pytest

import oracle as O
from tests._problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-12}


@pytest.mark.parametrize("side_stream", [False, True], ids=["legacy_stream", "side_stream"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_planned_tikhonov_on_consecutive_calls(lib, dtype, side_stream):
    import torch
    td = {"f32": torch.float32, "f64": torch.float64}[dtype]
    dims, dec = (64, 32, 32), (2, 2, 2)
    stream = torch.cuda.Stream() if side_stream else None
    for call, (seed, tau, prior) in enumerate([(31, 1e-2, "nearest"), (32, 0.3, None), (33, 5e-2, "user")]):
        psf, xt, y = make_problem(dims, dec, sigma=(1.0, 0.8, 1.2), seed=seed, asym=True)
        yd = torch.tensor(y, dtype=td, device="cuda")
        if prior == "user":
            xbar_np = 0.5 * xt + 0.1 * np.random.default_rng(seed).standard_normal(xt.shape)
            xbar_o, xbar_g = xbar_np, torch.tensor(xbar_np, dtype=td, device="cuda")
        elif prior == "nearest":
            xbar_o, xbar_g = O.nearest_neighbour(y, dec), "nearest"
        else:
            xbar_o, xbar_g = None, None
        plan = lib.Plan(dims, dec, psf, dtype)
        ref = plan.tikhonov(yd, tau, xbar=xbar_g)
        plan.close()
        got = torch.full_like(ref, float("nan"))
        torch.cuda.synchronize()
        if stream is not None:
            with torch.cuda.stream(stream):
                lib.tikhonov_noalloc(dims, dec, psf, yd, tau, got, xbar=xbar_g, dtype=dtype, stream=stream)
        else:
            lib.tikhonov_noalloc(dims, dec, psf, yd, tau, got, xbar=xbar_g, dtype=dtype)
        g = got.cpu().numpy()
        assert rel_l2(g, ref.cpu().numpy()) < TOL[dtype], (call, prior)
        assert rel_l2(g, O.tikhonov(y, psf, dec, tau, xbar_o)) < TOL[dtype], (call, prior)


def test_noalloc_rejects_volumes_beyond_its_scratch(lib):
    import torch
    dims, dec = (256, 256, 64), (2, 2, 2)
    psf = np.ones((3, 3, 3)) / 27.0
    y = torch.zeros((32, 128, 128), dtype=torch.float32, device="cuda")
    x = torch.zeros((64, 256, 256), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.Sr3dError) as e:
        lib.tikhonov_noalloc(dims, dec, psf, y, 1e-2, x)
    assert e.value.name == "UNSUPPORTED_SIZE" and "sr3d_plan" in str(e.value)
