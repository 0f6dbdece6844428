"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP32 plans must match the FP64 oracle within 1e-5 relative L2;
FP64 plans within 1e-12.  Inputs are seeded synthetic phantoms; every expected
value comes from oracle/.
"""
import numpy as np
import pytest

import oracle as O
from tests._problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-12}

# (dims (m, n, s), dec (dr, dc, ds), dtype): several tiles with ragged tails,
# mixed radix (96, 48, 24, 12), anisotropic and no decimation.
CASES = [
    ((32, 16, 8), (2, 2, 2), "f32"),
    ((96, 24, 12), (2, 1, 3), "f32"),
    ((64, 32, 32), (1, 1, 4), "f32"),
    ((64, 48, 16), (2, 2, 1), "f32"),
    ((128, 64, 32), (4, 2, 1), "f32"),
    ((32, 16, 8), (1, 1, 1), "f32"),
    ((32, 32, 32), (2, 2, 2), "f64"),
    ((96, 24, 12), (2, 1, 3), "f64"),
    # lengths with compile-time FFT plans: m half-length 128 / 256, n 256 / 512, s 256
    ((256, 256, 16), (2, 2, 2), "f32"),
    ((64, 16, 256), (2, 2, 2), "f32"),
    ((512, 32, 16), (1, 1, 4), "f32"),
    ((32, 512, 8), (1, 2, 1), "f32"),
    # compile-time plans of 3 * 2^a lengths (12 elements per thread): m half-lengths
    # 48 / 96 / 192, n 96 / 192, register-resident s passes of 96 and 192 points
    ((96, 96, 96), (2, 2, 2), "f32"),
    ((96, 96, 96), (2, 2, 1), "f32"),
    ((192, 32, 96), (1, 1, 4), "f32"),
    ((64, 192, 192), (2, 2, 2), "f32"),
    ((384, 16, 48), (4, 1, 1), "f32"),
]
IDS = [f"{d[0]}x{d[1]}x{d[2]}_d{c[0]}{c[1]}{c[2]}_{t}" for d, c, t in CASES]


def T(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype={"f32": torch.float32, "f64": torch.float64}[dtype],
                        device="cuda")


def H(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.fixture
def tag(request):
    """Name under which a test records its parity errors."""
    return lambda what: f"{request.node.name}:{what}"


@pytest.fixture(scope="module", params=list(range(len(CASES))), ids=IDS)
def case(request, lib):
    dims, dec, dtype = CASES[request.param]
    psf, x, y = make_problem(dims, dec, sigma=(1.0, 0.8, 1.2), seed=11 + request.param, asym=True)
    plan = lib.Plan(dims, dec, psf, dtype)
    yield dict(dims=dims, dec=dec, dtype=dtype, psf=psf, x=x, y=y, plan=plan)
    plan.close()


def test_otf(case, tag):
    m = case["dims"][0]
    ref = O.otf(case["psf"], case["x"].shape)[..., : m // 2 + 1]
    got = case["plan"].get_otf().cpu().numpy()
    assert rel_l2(got, ref, tag("otf")) < TOL[case["dtype"]]


def test_fft3(case, tag):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(case["x"].shape)
    m = case["dims"][0]
    got = case["plan"].fft3(T(x, case["dtype"])).cpu().numpy()
    assert rel_l2(got, np.fft.fftn(x)[..., : m // 2 + 1], tag("fft3")) < TOL[case["dtype"]]


def test_forward_model(case, tag):
    got = H(case["plan"].forward(T(case["x"], case["dtype"])))
    assert rel_l2(got, O.forward(case["x"], case["psf"], case["dec"]), tag("DHx")) < TOL[case["dtype"]]


@pytest.mark.parametrize("prior", ["zero", "nearest", "user"])
@pytest.mark.parametrize("tau", [1e-2, 0.5])
def test_tikhonov(case, prior, tau, tag):
    y, dec, dt = case["y"], case["dec"], case["dtype"]
    if prior == "zero":
        xbar_o, xbar_g = None, None
    elif prior == "nearest":
        xbar_o, xbar_g = O.nearest_neighbour(y, dec), "nearest"
    else:
        xbar_o = np.random.default_rng(5).standard_normal(case["x"].shape)
        xbar_g = T(xbar_o, dt)
    ref = O.tikhonov(y, case["psf"], dec, tau, xbar_o)
    got = H(case["plan"].tikhonov(T(y, dt), tau, xbar=xbar_g))
    assert rel_l2(got, ref, tag("x")) < TOL[dt]


def test_xstep(case, tag):
    rng = np.random.default_rng(6)
    shape = case["x"].shape
    rho = 0.05 * rng.standard_normal((3,) + shape)
    theta = O.grad_adj(rho)
    mu = 2e-2
    ref = O.admm_xstep(case["y"], O.otf(case["psf"], shape), theta, mu, case["dec"])
    got = H(case["plan"].xstep(T(case["y"], case["dtype"]), T(theta, case["dtype"]), mu))
    assert rel_l2(got, ref, tag("x")) < TOL[case["dtype"]]


def test_tv_step(case, tag):
    rng = np.random.default_rng(7)
    x, dt = case["x"], case["dtype"]
    d = 0.01 * rng.standard_normal((3,) + x.shape)
    lam, mu = 1e-3, 1e-2
    g = O.grad(x)
    u = O.shrink(g + d, lam / mu)
    d_new = d + g - u
    theta = O.grad_adj(u - d_new)
    d_got, th_got = case["plan"].tv_step(T(x, dt), T(d, dt), lam, mu)
    assert rel_l2(H(d_got), d_new, tag("d")) < TOL[dt]
    assert rel_l2(H(th_got), theta, tag("theta")) < TOL[dt]


def test_admm_iterates(case, tag):
    y, psf, dec, dt = case["y"], case["psf"], case["dec"], case["dtype"]
    lam, mu, tau0, iters = 1e-3, 1e-2, 1e-2, 10
    x0 = O.tikhonov(y, psf, dec, tau0, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, lam, mu, iters, x0, record=True)
    import torch
    x = T(np.zeros_like(x0), dt)
    d = torch.zeros((3,) + x0.shape, dtype=x.dtype, device="cuda")
    st = case["plan"].admm_tv(T(y, dt), x, lam, mu, iters, d=d, tau_init=tau0, eval_every=1, hist_len=iters)
    assert rel_l2(H(x), ref["x"], tag("x")) < TOL[dt]
    assert rel_l2(H(d), ref["d"], tag("d")) < (TOL[dt] * 10 if dt == "f32" else TOL[dt])
    rel_l2(hist_np := np.array(st["objective_hist"]), np.array(ref["hist"]["objective"]), tag("objective"))
    hist = np.array(st["objective_hist"])
    assert np.allclose(hist, ref["hist"]["objective"], rtol=TOL[dt] * 10, atol=0)
    assert st["iters"] == iters and st["evals"] == iters
    assert np.isclose(st["primal"], ref["hist"]["primal"][-1], rtol=1e-4)
    assert np.isclose(st["dual"], ref["hist"]["dual"][-1], rtol=1e-3)


def test_admm_from_given_x0_and_d0(case, tag):
    y, psf, dec, dt = case["y"], case["psf"], case["dec"], case["dtype"]
    rng = np.random.default_rng(8)
    x0 = case["x"] + 0.05 * rng.standard_normal(case["x"].shape)
    d0 = 0.02 * rng.standard_normal((3,) + x0.shape)
    ref = O.admm_tv(y, psf, dec, 2e-3, 5e-2, 4, x0, d0=d0)
    x = T(x0, dt)
    d = T(d0, dt)
    case["plan"].admm_tv(T(y, dt), x, 2e-3, 5e-2, 4, d=d, tau_init=0.0)
    assert rel_l2(H(x), ref["x"], tag("x")) < TOL[dt]
    assert rel_l2(H(d), ref["d"], tag("d")) < (TOL[dt] * 10 if dt == "f32" else TOL[dt])


def test_host_buffers_match_device_call(lib):
    import torch
    dims, dec = (64, 32, 16), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=21)
    plan = lib.Plan(dims, dec, psf, "f32")
    yd = T(y, "f32")
    xd = plan.empty_hr()
    plan.admm_tv(yd, xd, 1e-3, 1e-2, 5, tau_init=1e-2)
    yh = yd.cpu().pin_memory()
    xh = torch.empty(xd.shape, dtype=torch.float32).pin_memory()
    plan.admm_tv_host(yh, xh, 1e-3, 1e-2, 5, tau_init=1e-2)
    assert torch.equal(xh, xd.cpu())
    plan.close()


def test_tolerance_stop_and_zero_iterations(lib):
    dims, dec = (32, 32, 32), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=22)
    plan = lib.Plan(dims, dec, psf, "f64")
    x = plan.empty_hr()
    st = plan.admm_tv(T(y, "f64"), x, 1e-3, 1e-2, 400, tol=1e-3, tau_init=1e-2, eval_every=5)
    assert st["converged"] and st["iters"] % 5 == 0 and st["iters"] < 400
    assert st["primal_rel"] < 1e-3 and st["dual_rel"] < 1e-3
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, 1e-3, 1e-2, st["iters"], x0, record=True)
    assert rel_l2(H(x), ref["x"]) < TOL["f64"]
    rel_p = ref["hist"]["primal"][-1] / max(ref["hist"]["norm_Lx"][-1], ref["hist"]["norm_u"][-1])
    assert np.isclose(st["primal_rel"], rel_p, rtol=1e-6)
    # zero iterations returns the Tikhonov start
    x2 = plan.empty_hr()
    plan.admm_tv(T(y, "f64"), x2, 1e-3, 1e-2, 0, tau_init=1e-2)
    assert rel_l2(H(x2), x0) < TOL["f64"]
    plan.close()


def test_errors(lib):
    import torch
    dims, dec = (32, 16, 8), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=23)
    plan = lib.Plan(dims, dec, psf, "f32")
    yd = T(y, "f32")
    with pytest.raises(lib.Sr3dError) as e:
        plan.tikhonov(yd, 0.0)
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(lib.Sr3dError):
        plan.admm_tv(yd, plan.empty_hr(), 1e-3, -1.0, 3)
    plan.close()
    zero = np.zeros((3, 3, 3))
    zero[1, 1, 0], zero[1, 1, 2] = 1.0, -1.0  # taps summing to zero
    p2 = lib.Plan(dims, dec, zero, "f32")
    with pytest.raises(lib.Sr3dError) as e:
        p2.admm_tv(yd, p2.empty_hr(), 1e-3, 1e-2, 3)
    assert e.value.name == "SINGULAR"
    p2.close()
    with pytest.raises(ValueError):
        lib.Plan(dims, dec, psf, "f32").tikhonov(torch.zeros(3, device="cuda"), 1.0)


def test_headline_size_against_oracle(lib, tag):
    """256^3, d = 2x2x2, sigma 1.5, the benchmark's launch configuration:
    Tikhonov start plus two ADMM-TV iterations, compared element by element."""
    from synth import HEADLINE_256 as W
    psf = W.psf()
    x = W.phantom()
    clean = O.forward(x, psf, W.dec)
    from synth import noise_sigma
    y = clean + noise_sigma(clean, W.snr_db) * W.noise()
    plan = lib.Plan(W.dims, W.dec, psf, "f32")
    x0 = O.tikhonov(y, psf, W.dec, W.tau, O.nearest_neighbour(y, W.dec))
    xg = plan.empty_hr()
    plan.tikhonov(T(y, "f32"), W.tau, xg, xbar="nearest")
    assert rel_l2(H(xg), x0, tag("tikhonov")) < TOL["f32"]
    ref = O.admm_tv(y, psf, W.dec, W.lam, W.mu, 2, x0)
    plan.admm_tv(T(y, "f32"), xg, W.lam, W.mu, 2, tau_init=W.tau)
    assert rel_l2(H(xg), ref["x"], tag("admm2")) < TOL["f32"]
    plan.close()


def test_graph_replay_across_calls(lib, tag):
    """Fixed-iteration solves replay a captured two-iteration graph; a change of
    buffers or parameters re-captures it.  Every call must still match the oracle."""
    import torch
    dims, dec = (128, 64, 32), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=24)
    plan = lib.Plan(dims, dec, psf, "f32")
    yd = T(y, "f32")
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    for call, (lam, mu, iters) in enumerate([(1e-3, 1e-2, 7), (1e-3, 1e-2, 8), (3e-3, 2e-2, 9)]):
        x = plan.empty_hr() if call != 1 else x  # call 1 reuses the buffer of call 0
        plan.admm_tv(yd, x, lam, mu, iters, tau_init=1e-2)
        ref = O.admm_tv(y, psf, dec, lam, mu, iters, x0)["x"]
        assert rel_l2(H(x), ref, tag(f"call{call}")) < TOL["f32"]
    plan.close()


@pytest.mark.parametrize("every,dtype", [(4, "f32"), (3, "f32"), (1, "f64"), (5, "f64")])
def test_statistics_blocks_replayed_as_graphs_match_eager(lib, every, dtype):
    """With statistics, whole evaluation blocks are replayed as CUDA graphs
    (odd blocks alternate the dual buffers); profiling forces every launch to
    run eagerly.  Both give the same iterates, dual, residuals and objective
    history bit for bit, with and without a tolerance stop."""
    import torch
    dims, dec = (128, 32, 16), (2, 2, 1)
    psf, xt, y = make_problem(dims, dec, seed=31)
    plan = lib.Plan(dims, dec, psf, dtype)
    yd = T(y, dtype)
    runs = []
    for prof in (False, True):
        plan.profile(prof)
        x = plan.empty_hr()
        d = torch.zeros((3,) + plan.hr_shape, dtype=plan.tdtype, device="cuda")
        st = plan.admm_tv(yd, x, 2e-3, 1e-2, 23, d=d, tau_init=1e-2, eval_every=every, hist_len=64)
        x2 = plan.empty_hr()
        st2 = plan.admm_tv(yd, x2, 2e-3, 1e-2, 400, tol=3e-3, tau_init=1e-2, eval_every=every, hist_len=64)
        runs.append((x, d, st, x2, st2))
    plan.profile(False)
    (xa, da, sa, xa2, sa2), (xb, db, sb, xb2, sb2) = runs
    assert torch.equal(xa, xb) and torch.equal(da, db) and torch.equal(xa2, xb2)
    for k in ("iters", "evals", "objective", "primal_rel", "dual_rel", "objective_hist"):
        assert sa[k] == sb[k], k
        assert sa2[k] == sb2[k], k
    assert sa["evals"] == 23 // every + (1 if 23 % every else 0)
    assert sa2["converged"] and sa2["iters"] % every == 0
    # the history equals the oracle's objective at the evaluated iterations
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, 2e-3, 1e-2, 23, x0, record=True)
    its = [k for k in range(1, 24) if k % every == 0 or k == 23]
    tol = 1e-5 if dtype == "f32" else 1e-12
    assert np.allclose(sa["objective_hist"], [ref["hist"]["objective"][k - 1] for k in its], rtol=tol)
    plan.close()


@pytest.mark.parametrize("every", [2, 3])
def test_device_tolerance_loop_edges_match_eager(lib, every):
    """With tol > 0 one graph loops over the evaluation blocks and makes the
    stopping test (Algorithm 1, step 5) on the device.  Its edges against the
    eager, host-tested path, bit for bit: a tolerance met at the first
    evaluation (the loop runs no block), a budget spent without convergence
    with iterations left over after the last whole block, and the same run
    repeated (the cached graph, the history index reset).  Launch accounting:
    the same kernels of every kind but "other", where the device loop adds
    one gate ahead of the loop and one per block."""
    import torch
    dims, dec = (128, 32, 16), (2, 2, 1)
    psf, xt, y = make_problem(dims, dec, seed=33)
    plan = lib.Plan(dims, dec, psf, "f64")
    yd = T(y, "f64")
    cases = [(1.0, 40), (1e-14, 4 * every + 1), (1e-14, 4 * every + 1)]
    runs = []
    for prof in (False, True):
        out = []
        for tol, iters in cases:
            plan.profile(prof)
            x = plan.empty_hr()
            d = torch.zeros((3,) + plan.hr_shape, dtype=plan.tdtype, device="cuda")
            st = plan.admm_tv(yd, x, 2e-3, 1e-2, iters, d=d, tol=tol, tau_init=1e-2, eval_every=every, hist_len=64)
            out.append((x, d, st, plan.profile_read()))
        runs.append(out)
    plan.profile(False)
    for (xa, da, sa, na), (xb, db, sb, nb), (tol, iters) in zip(runs[0], runs[1], cases):
        assert torch.equal(xa, xb) and torch.equal(da, db), (tol, iters)
        for k in ("iters", "evals", "converged", "objective", "primal_rel", "dual_rel", "objective_hist"):
            assert sa[k] == sb[k], (k, tol, iters)
        for kind in na:
            if kind != "other":
                assert na[kind][1] == nb[kind][1], (kind, na[kind], nb[kind])
        if tol == 1.0:
            assert sa["converged"] and sa["iters"] == every and sa["evals"] == 1
            assert na["other"][1] == nb["other"][1] + 1  # the gate ahead of the loop only
        else:
            assert not sa["converged"] and sa["iters"] == iters and sa["evals"] == 5
            assert na["other"][1] == nb["other"][1] + 1 + 3  # the first block is eager: 3 loop blocks
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, 2e-3, 1e-2, 4 * every + 1, x0, record=True)
    assert rel_l2(H(runs[0][1][0]), ref["x"]) < TOL["f64"]
    assert rel_l2(H(runs[0][1][1]), ref["d"]) < TOL["f64"]  # the caller's dual buffer, returned by the loop
    its = [every * j for j in range(1, 5)] + [4 * every + 1]
    assert np.allclose(runs[0][1][2]["objective_hist"], [ref["hist"]["objective"][k - 1] for k in its], rtol=1e-12)
    plan.close()


def _separable_asym_psf(shape, seed):
    """Outer product of three asymmetric positive 1-D factors (complex Lambda)."""
    rng = np.random.default_rng(seed)
    f = [rng.uniform(0.2, 1.0, n) for n in shape]  # (p_s, p_n, p_m)
    psf = f[0][:, None, None] * f[1][None, :, None] * f[2][None, None, :]
    return psf / psf.sum()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_separable_psf_path(lib, dtype):
    """A separable PSF is detected and the class solve then forms Lambda from
    three 1-D DFTs; Tikhonov, the forward model and ADMM agree with the stored
    3-D Lambda to rounding and with the oracle.  A non-separable PSF keeps the
    stored Lambda."""
    import torch
    dims, dec = (64, 32, 16), (2, 2, 2)
    psf = _separable_asym_psf((5, 3, 7), 81)
    _, xt, _ = make_problem(dims, dec, seed=82)
    clean = O.forward(xt, psf, dec)
    import synth
    y = clean + synth.noise_sigma(clean, 40.0) * synth.noise_field(clean.shape, 83)
    plan = lib.Plan(dims, dec, psf, dtype)
    assert plan.separable()
    yd = T(y, dtype)
    outs = {}
    for use in (True, False):
        assert plan.separable(use) == use
        xk = plan.tikhonov(yd, 1e-2, xbar="nearest")
        fw = plan.forward(T(xt, dtype))
        xa = plan.empty_hr()
        d = torch.zeros((3,) + plan.hr_shape, dtype=plan.tdtype, device="cuda")
        plan.admm_tv(yd, xa, 2e-3, 1e-2, 6, d=d, tau_init=1e-2)
        outs[use] = (H(xk), H(fw), H(xa), H(d))
    agree = 1e-6 if dtype == "f32" else 1e-13
    for a, b in zip(outs[True], outs[False]):
        assert rel_l2(a, b) < agree
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, 2e-3, 1e-2, 6, x0)
    tol = TOL[dtype]
    assert rel_l2(outs[True][0], x0) < tol
    assert rel_l2(outs[True][1], clean) < tol
    assert rel_l2(outs[True][2], ref["x"]) < tol
    plan.separable(True)
    plan.close()
    # non-separable: detected as such
    psf_ns = psf * (1.0 + 0.3 * np.linspace(0, 1, psf.size).reshape(psf.shape))
    plan = lib.Plan(dims, dec, psf_ns / psf_ns.sum(), dtype)
    assert not plan.separable()
    plan.close()


@pytest.mark.parametrize("dims,dec", [((96, 48, 192), (2, 2, 2)), ((384, 16, 96), (2, 2, 1)),
                                      ((192, 96, 96), (1, 1, 4))])
def test_separable_psf_3x2a_compile_time_plans(lib, dims, dec):
    """The separable-PSF class solve on the compile-time plans of 3 * 2^a
    lengths (12 elements per thread): m half-lengths 48, 192 and 96 through
    the register real-FFT split (d_r 2, 2, 1), n lengths 48 and 96, and the
    register-resident s pass at 192 and 96 points for the three class shapes
    (Lambda formed from the three 1-D factors inside the solve).  Tikhonov and
    six ADMM-TV iterates against the oracle in FP32."""
    import torch
    psf = _separable_asym_psf((5, 3, 7), 91)
    _, xt, _ = make_problem(dims, dec, seed=92)
    clean = O.forward(xt, psf, dec)
    import synth
    y = clean + synth.noise_sigma(clean, 40.0) * synth.noise_field(clean.shape, 93)
    plan = lib.Plan(dims, dec, psf, "f32")
    assert plan.separable()
    yd = T(y, "f32")
    xk = plan.tikhonov(yd, 1e-2, xbar="nearest")
    xa = plan.empty_hr()
    d = torch.zeros((3,) + plan.hr_shape, dtype=plan.tdtype, device="cuda")
    plan.admm_tv(yd, xa, 2e-3, 1e-2, 6, d=d, tau_init=1e-2)
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, 2e-3, 1e-2, 6, x0)
    assert rel_l2(H(xk), x0) < TOL["f32"]
    assert rel_l2(H(xa), ref["x"]) < TOL["f32"]
    plan.close()


# ---------------------------------------------------------------------------
# other regularisers through the same x-update
# ---------------------------------------------------------------------------

def test_tikhonov_grad(case, tag):
    y, psf, dec, dt = case["y"], case["psf"], case["dec"], case["dtype"]
    for tau in (3e-2, 0.7):
        x = case["plan"].tikhonov_grad(T(y, dt), tau)
        ref = O.tikhonov_grad(y, psf, dec, tau)
        assert rel_l2(H(x), ref, tag(f"x_tau{tau}")) < TOL[dt]


def test_admm_anisotropic_tv_iterates(case, tag):
    import torch
    y, psf, dec, dt = case["y"], case["psf"], case["dec"], case["dtype"]
    plan = case["plan"]
    lam, mu, tau0, iters = 1e-3, 1e-2, 1e-2, 10
    x0 = O.tikhonov(y, psf, dec, tau0, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, lam, mu, iters, x0, record=True, aniso=True)
    plan.set_tv("anisotropic")
    try:
        x = T(np.zeros_like(x0), dt)
        d = torch.zeros((3,) + x0.shape, dtype=x.dtype, device="cuda")
        st = plan.admm_tv(T(y, dt), x, lam, mu, iters, d=d, tau_init=tau0, eval_every=1, hist_len=iters)
    finally:
        plan.set_tv("isotropic")
    assert rel_l2(H(x), ref["x"], tag("x")) < TOL[dt]
    assert rel_l2(H(d), ref["d"], tag("d")) < (TOL[dt] * 10 if dt == "f32" else TOL[dt])
    assert np.allclose(st["objective_hist"], ref["hist"]["objective"], rtol=TOL[dt] * 10, atol=0)
    assert np.isclose(st["primal"], ref["hist"]["primal"][-1], rtol=1e-4)


def test_switching_the_tv_recaptures_the_loop_graphs(lib):
    """Fixed-iteration solves replay a cached graph; switching the TV must
    re-capture it: isotropic, anisotropic, isotropic again with the same
    buffers gives the first result bit for bit and a different second one."""
    dims, dec = (128, 32, 16), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=91)
    plan = lib.Plan(dims, dec, psf, "f32")
    yd = T(y, "f32")
    x = plan.empty_hr()
    outs = []
    for kind in ("isotropic", "anisotropic", "isotropic"):
        plan.set_tv(kind)
        plan.admm_tv(yd, x, 3e-3, 1e-2, 9, tau_init=1e-2)
        outs.append(x.clone())
    import torch
    assert torch.equal(outs[0], outs[2])
    assert not torch.equal(outs[0], outs[1])
    x0 = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    ref = O.admm_tv(y, psf, dec, 3e-3, 1e-2, 9, x0, aniso=True)
    assert rel_l2(H(outs[1]), ref["x"]) < TOL["f32"]
    plan.close()


# ---------------------------------------------------------------------------
# the iterative comparator (conjugate gradients on eq. 6)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prior", ["zero", "nearest", "user"])
def test_cg_iterates_match_oracle(case, tag, prior):
    y, psf, dec, dt = case["y"], case["psf"], case["dec"], case["dtype"]
    plan = case["plan"]
    tau, iters = 2e-2, 8
    xbar_np = {"zero": None, "nearest": O.nearest_neighbour(y, dec), "user": case["x"] * 0.5}[prior]
    xbar = {"zero": None, "nearest": "nearest", "user": T(case["x"] * 0.5, dt)}[prior]
    x, k, rel, ok = plan.tikhonov_cg(T(y, dt), tau, xbar=xbar, max_iters=iters)
    ref = O.tikhonov_cg(y, psf, dec, tau, xbar_np, iters=iters)
    assert k == iters and ok
    assert rel_l2(H(x), ref["x"], tag("x")) < (1e-4 if dt == "f32" else 1e-10)
    assert np.isclose(rel, ref["residuals"][-1] / ref["residuals"][0], rtol=1e-2 if dt == "f32" else 1e-8)


@pytest.mark.parametrize("dtype,tol,agree", [("f64", 1e-9, 1e-7), ("f32", 1e-5, 2e-4)])
def test_cg_converges_to_the_closed_form(lib, dtype, tol, agree):
    """Run to tolerance, the comparator reaches the solution of eq. 12."""
    dims, dec = (64, 32, 16), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=95)
    plan = lib.Plan(dims, dec, psf, dtype)
    yd = T(y, dtype)
    x, k, rel, ok = plan.tikhonov_cg(yd, 1e-2, xbar="nearest", tol=tol, max_iters=2000)
    assert ok and rel <= tol and 1 < k < 2000
    closed = plan.tikhonov(yd, 1e-2, xbar="nearest")
    ref = O.tikhonov(y, psf, dec, 1e-2, O.nearest_neighbour(y, dec))
    assert rel_l2(H(x), ref) < agree
    assert rel_l2(H(x), H(closed)) < agree
    _, k, rel, ok = plan.tikhonov_cg(yd, 1e-2, tol=1e-30, max_iters=3)  # NOT_CONVERGED: x still written
    assert not ok and k == 3 and rel > 1e-30
    plan.close()


# ---------------------------------------------------------------------------
# PSF replacement and the Gaussian PSF fit
# ---------------------------------------------------------------------------

def test_set_psf_equals_a_fresh_plan(lib):
    """sr3d_set_psf recomputes Lambda in place: the same results, bit for bit,
    as a plan created with that PSF (separable and non-separable PSFs)."""
    import torch
    dims, dec = (64, 32, 16), (2, 2, 2)
    psf_a, xt, y = make_problem(dims, dec, sigma=(1.0, 1.0, 1.0), seed=111)
    psf_b, _, _ = make_problem(dims, dec, sigma=(1.4, 0.7, 1.1), seed=112, asym=True)
    plan = lib.Plan(dims, dec, psf_a, "f32")
    yd = T(y, "f32")
    plan.admm_tv(yd, plan.empty_hr(), 2e-3, 1e-2, 4, tau_init=1e-2)  # leaves graphs captured
    for psf in (psf_b, psf_a):
        plan.set_psf(psf)
        fresh = lib.Plan(dims, dec, psf, "f32")
        assert plan.separable() == fresh.separable()
        assert torch.equal(plan.get_otf(), fresh.get_otf())
        xa, xb = plan.empty_hr(), fresh.empty_hr()
        plan.admm_tv(yd, xa, 2e-3, 1e-2, 4, tau_init=1e-2)
        fresh.admm_tv(yd, xb, 2e-3, 1e-2, 4, tau_init=1e-2)
        assert torch.equal(xa, xb)
        fresh.close()
    plan.close()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_psf_fit_moments_equal_the_sums_of_the_oracle_forward_model(lib, dtype, tol):
    """sr3d_psf_fit_moments: the five FP64 sums of the gain/offset least
    squares, with yh = DHx formed in the library, against the oracle's DHx."""
    dims, dec = (64, 32, 16), (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=114, asym=True)
    plan = lib.Plan(dims, dec, psf, dtype)
    got = np.array(plan.psf_fit_moments(T(xt, dtype), T(y, dtype)))
    yv = H(T(y, dtype))  # the observation as the GPU holds it
    yh = O.forward(xt if dtype == "f64" else H(T(xt, dtype)), psf, dec)
    ref = np.array([yh.sum(), (yh * yh).sum(), yv.sum(), (yv * yv).sum(), (yh * yv).sum()])
    assert np.allclose(got, ref, rtol=tol, atol=tol * np.abs(ref).max()), (got, ref)
    plan.close()


def test_gaussian_psf_fit(lib):
    """The fit's objective equals the oracle's at the same sigma, and on
    noise-free data made with a known Gaussian, gain and offset it recovers
    them."""
    import torch
    from paper_2010_15491_gb300 import psf_fit
    dims, dec = (64, 64, 32), (2, 2, 2)
    _, xt, _ = make_problem(dims, dec, seed=113, n_ell=20)
    size = psf_fit.support((3.0, 3.0, 3.0), dims)
    s_true = (1.3, 0.9, 1.7)
    y = 2.0 * O.forward(xt, O.gaussian_psf_taps(s_true, size), dec) + 0.1
    plan = lib.Plan(dims, dec, O.gaussian_psf_taps((1.0, 1.0, 1.0), size), "f64")
    xd, yd = T(xt, "f64"), T(y, "f64")
    for s in [(1.0, 1.0, 1.0), (2.0, 0.7, 1.2)]:
        r, a, b = psf_fit.objective(plan, xd, yd, s, size)
        ro, ao, bo = O.psf_fit_objective(s, size, xt, y, dec)
        assert np.isclose(r, ro, rtol=1e-8) and np.isclose(a, ao, rtol=1e-10) and np.isclose(b, bo, rtol=1e-8, atol=1e-12)
    res = psf_fit.fit_gaussian_psf(plan, xd, yd, sigma0=(1.0, 1.0, 1.0), bounds=(0.3, 3.0))
    assert np.allclose(res["sigma"], s_true, rtol=1e-3), res
    assert np.isclose(res["gain"], 2.0, rtol=1e-4) and np.isclose(res["offset"], 0.1, rtol=1e-3)
    plan.close()


@pytest.mark.slow
def test_aniso512_tikhonov_optimality(lib):
    """512 x 512 x 256, d = 1x1x4, sigma (1, 1, 2) (the anisotropic CBCT-like
    workload at full size): the GPU Tikhonov solution satisfies the normal
    equations of eq. 6, H^T D^T (D H x - y) + tau (x - xbar) = 0, evaluated
    with the oracle's FP64 operators, to FP32 accuracy."""
    import synth
    W = synth.ANISO_512
    psf = W.psf()
    m, n, s = W.dims
    lr = (s // W.dec[2], n // W.dec[1], m // W.dec[0])
    # the property holds for any observation: a seeded smooth-plus-noise y
    # instead of the 500-ellipsoid phantom keeps the host work to a few FFTs
    y = 0.5 + 0.1 * synth.normal(W.seed, 5, int(np.prod(lr))).reshape(lr)
    lam = O.otf(psf, (s, n, m))
    plan = lib.Plan(W.dims, W.dec, psf, "f32")
    xg = H(plan.tikhonov(T(y, "f32"), W.tau, xbar="nearest"))
    plan.close()
    xbar = O.nearest_neighbour(y, W.dec)
    Ht = lambda v: np.real(np.fft.ifftn(np.conj(lam) * np.fft.fftn(v)))  # noqa: E731
    rhs = Ht(O.zero_fill(y, W.dec)) + W.tau * xbar
    r = Ht(O.zero_fill(O.forward(xg, psf, W.dec), W.dec)) + W.tau * xg - rhs
    assert np.linalg.norm(r) <= 1e-5 * np.linalg.norm(rhs)
