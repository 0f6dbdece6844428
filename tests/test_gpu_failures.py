"""Failure paths, made on the host or with a bounded wait that nothing
completes; none of them faults the GPU.

  * NaN in the observation: the FP64 reductions flag it and sr3d_admm_tv
    returns SR3D_ERR_NUMERIC; the plan then solves a clean problem correctly.
  * Out of memory: a per-plan device-memory cap set from the host makes
    sr3d_plan fail with SR3D_ERR_OOM and free what it had allocated, and makes
    the lazy buffers of the first ADMM call fail the same way with the plan
    staying usable.
  * Device wait limit: the bounded completion wait of the tensor-core
    convolution, shortened, runs out on a barrier that nothing arrives on (no
    MMA issued); the call returns SR3D_ERR_TIMEOUT and the network, its tensor
    memory freed, computes correctly afterwards.
"""
import numpy as np
import pytest

import oracle as O
from tests._problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


def T(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype={"f32": torch.float32, "f64": torch.float64}[dtype],
                        device="cuda")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_nan_in_y_returns_numeric_and_the_plan_stays_usable(lib, dtype):
    dims, dec = (64, 32, 16), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=141)
    plan = lib.Plan(dims, dec, psf, dtype)
    bad = y.copy()
    bad[1, 2, 3] = np.nan
    for kw in (dict(eval_every=1), dict(eval_every=0), dict(tol=1e-4, eval_every=2)):
        with pytest.raises(lib.Sr3dError) as e:
            plan.admm_tv(T(bad, dtype), plan.empty_hr(), 1e-3, 1e-2, 6, tau_init=1e-2, **kw)
        assert e.value.name == "NUMERIC", kw
    bad[1, 2, 3] = np.inf
    with pytest.raises(lib.Sr3dError) as e:
        plan.admm_tv(T(bad, dtype), plan.empty_hr(), 1e-3, 1e-2, 4, tau_init=1e-2, eval_every=1)
    assert e.value.name == "NUMERIC"
    x = plan.empty_hr()
    plan.admm_tv(T(y, dtype), x, 1e-3, 1e-2, 6, tau_init=1e-2, eval_every=1)
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, 1e-3, 1e-2, 6, x0)
    assert rel_l2(x.cpu().numpy(), ref["x"]) < (1e-5 if dtype == "f32" else 1e-12)
    plan.close()


def test_plan_memory_cap_gives_oom_and_leaves_nothing_allocated(lib):
    import torch
    dims, dec = (256, 128, 64), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=142)
    plan = lib.Plan(dims, dec, psf, "f32")
    need = plan.info()["bytes"]
    plan.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        lib.set_plan_memory_limit(need // 2)
        for _ in range(3):
            with pytest.raises(lib.Sr3dError) as e:
                lib.Plan(dims, dec, psf, "f32")
            assert e.value.name == "OOM" and "limit" in str(e.value)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        # the failed plans held about need/2 each before failing: nothing is left
        assert free1 >= free0 - (4 << 20), (free0, free1, need)
        # a plan that fits, whose first ADMM call cannot get its dual buffers
        lib.set_plan_memory_limit(need)
        plan = lib.Plan(dims, dec, psf, "f32")
        yd = T(y, "f32")
        x = plan.empty_hr()
        with pytest.raises(lib.Sr3dError) as e:
            plan.admm_tv(yd, x, 1e-3, 1e-2, 3, tau_init=1e-2)
        assert e.value.name == "OOM"
        xt_ = plan.tikhonov(yd, 1e-2, xbar="nearest")  # needs no new buffer
        assert rel_l2(xt_.cpu().numpy(), O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))) < 1e-5
    finally:
        lib.set_plan_memory_limit(0)
    plan.admm_tv(yd, x, 1e-3, 1e-2, 3, tau_init=1e-2)
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    assert rel_l2(x.cpu().numpy(), O.admm_tv(y, psf, dec, 1e-3, 1e-2, 3, x0)["x"]) < 1e-5
    plan.close()


def test_tensor_core_wait_timeout_is_reported_and_the_network_stays_usable(lib):
    import torch
    from paper_2010_15491_gb300 import warmstart as W
    net = lib.UNet()
    with pytest.raises(lib.Sr3dError) as e:
        net.wait_selftest(0)
    assert e.value.name == "INVALID_ARG"
    for _ in range(2):  # the flag is cleared after each report
        with pytest.raises(lib.Sr3dError) as e:
            net.wait_selftest(200_000)  # about 0.1 ms of SM clock
        assert e.value.name == "TIMEOUT"
    net.set_params(W.init_params(5))
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.rand((8, 8, 128), device="cuda", generator=g)
    net.set_path("tcgen05_all")
    out_tc = net.forward(x).clone()
    net.set_path("mma")
    out_mma = net.forward(x).clone()
    net.close()
    assert torch.isfinite(out_tc).all()
    assert rel_l2(out_tc.cpu().numpy(), out_mma.cpu().numpy()) < 1e-2
