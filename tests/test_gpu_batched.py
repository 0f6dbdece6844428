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


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("dims", [(128, 64, 48), (256, 32, 64)])
def test_schedules_leave_results_unchanged(lib, dtype, dims):
    """Every tile width of the n and s passes, every TV plane count and every
    m-pass lines-per-CTA count the plan accepts (sr3d_schedule), including
    widths that do not divide the m-slot count, plane counts that do not
    divide S and line counts that do not divide N x S, splits the same
    per-element work differently: the iterate is bit-identical and the
    statistics agree to reduction order.  (256, 32, 64) has the 130 m-slots
    of a 256-long m axis at d_r = 2 and a compile-time s pass.  After a
    schedule change the statistics sum only the CTAs of the new grids."""
    import torch
    dec = (2, 2, 2)
    psf, xt, y = make_problem(dims, dec, seed=61)
    td = torch.float32 if dtype == "f32" else torch.float64
    yd = torch.tensor(y, dtype=td, device="cuda")
    p = lib.Plan(dims, dec, psf, dtype)
    base = p.schedule()
    assert base["tv_planes"] >= 4

    def run():
        x = p.empty_hr()
        st = p.admm_tv(yd, x, 1e-3, 1e-2, 12, tau_init=1e-2, eval_every=3, hist_len=8)
        return x, st

    x0, st0 = run()

    # The FP32 TV kernel sums a thread's planes in compensated FP32 (error
    # below 2u of the partial, u = 2^-24) before the FP64 reduction, so its
    # statistics move with the plane count by a few u of the (positive) sums;
    # FP64 statistics move by reduction order only.
    rtol = 4 * 2.0 ** -24 if dtype == "f32" else 1e-12

    def same(tag):
        x, st = run()
        assert torch.equal(x, x0), tag
        assert st["evals"] == st0["evals"]
        for a, b in zip(st["objective_hist"], st0["objective_hist"]):
            assert abs(a - b) <= rtol * abs(b), tag
        for k in ("objective", "data_term", "tv_term", "primal", "dual"):
            assert abs(st[k] - st0[k]) <= rtol * abs(st0[k]) + 1e-300, (tag, k)

    accepted = {}
    for arg, widths in (("n_pass_slots", (2, 6, 10, 12, 16, 22, 32, 34)),
                        ("s_pass_slots", (2, 4, 6, 8, 10, 12, 22)),
                        ("tv_planes", (4, 5, 7, 37, 64)),
                        ("m_fwd_lines", (3, 4, 8, 12, 16, 24, 40, 64)),
                        ("m_inv_lines", (3, 4, 8, 12, 16, 24, 40, 64))):
        accepted[arg] = []
        for w in widths:
            prev = p.schedule()
            try:
                sch = p.schedule(**{arg: w})
            except lib.Sr3dError:
                assert p.schedule() == prev  # a rejected value changes nothing
                continue
            assert sch[arg] == w
            accepted[arg].append(w)
            same((arg, w))
        p.schedule(**base)
    assert p.schedule() == base
    assert len(accepted["n_pass_slots"]) >= 4 and len(accepted["s_pass_slots"]) >= 3, accepted
    assert len(accepted["tv_planes"]) == 5 and len(accepted["m_fwd_lines"]) >= 3, accepted
    assert accepted["m_inv_lines"] == accepted["m_fwd_lines"], accepted
    same("restored")
    # the autotuner may change every schedule; statistics still match a fresh plan
    p.autotune(2)
    x = p.empty_hr()
    st = p.admm_tv(yd, x, 1e-3, 1e-2, 12, tau_init=1e-2, eval_every=3)
    assert torch.equal(x, x0)
    for k in ("objective", "data_term", "tv_term", "primal", "dual"):
        assert abs(st[k] - st0[k]) <= rtol * abs(st0[k]) + 1e-300, k
    before = p.schedule()
    for bad in ({"tv_planes": 3}, {"s_pass_slots": 3}, {"n_pass_slots": 3}, {"n_pass_slots": 1000},
                {"m_fwd_lines": 3}, {"m_inv_lines": 1000}):
        with pytest.raises(lib.Sr3dError):
            p.schedule(**bad)
        assert p.schedule() == before
    p.close()


# volumes that share a geometry, lambda and rho are solved as groups (one
# launch per pass over the group's volumes); each keeps its own PSF and tau
GROUPED = [((64, 64, 32), (2, 2, 2), 1.0, 1e-2), ((64, 64, 32), (2, 2, 2), 1.4, 3e-2),
           ((64, 64, 32), (2, 2, 2), 0.8, 5e-3), ((96, 96, 64), (2, 2, 1), 1.2, 2e-2),
           ((96, 96, 64), (2, 2, 1), 0.9, 1e-2), ((64, 32, 96), (2, 2, 2), 1.1, 1e-2),
           ((64, 32, 96), (2, 2, 2), 1.6, 4e-2), ((128, 64, 64), (1, 1, 4), 1.0, 1e-2)]


def test_grouped_volumes_equal_single_volume_solves(lib):
    """Three groups (64x64x32 d222: 32-point s pass with the shared-tile
    solve, 64-wide TV tiles; 96x96x64 d221: register-resident 64-point s pass,
    96-wide TV tiles, 48- and 96-point m and n plans; 64x32x96 d222:
    register-resident 96-point s pass) and a single volume: every volume
    equals its own single-plan solve bit for bit on six calls, three with an
    odd and three with an even iteration count (the first call of a grouping
    runs its set-up eagerly, the next captures the set-up graph, with the
    first iteration when the count is odd, and the iteration graph, the last
    replays both), and a sample matches the oracle."""
    import torch
    plans, ys, xs, probs = [], [], [], []
    for k, (dims, dec, sg, tau) in enumerate(GROUPED):
        psf, xt, y = make_problem(dims, dec, sigma=(sg, 0.9 * sg, 1.1 * sg), seed=70 + k)
        p = lib.Plan(dims, dec, psf, "f32", stream=torch.cuda.Stream())
        assert p.separable()
        plans.append(p)
        ys.append(torch.tensor(y, dtype=torch.float32, device="cuda"))
        xs.append(p.empty_hr())
        probs.append((psf, y, dec, tau))
    lams, rhos = [2e-3] * len(plans), [1e-2] * len(plans)
    taus = [v[3] for v in GROUPED]
    for rep, iters in enumerate((9, 9, 9, 10, 10, 10)):
        for x in xs:
            x.fill_(float("nan"))
        lib.admm_tv_batched(plans, ys, xs, lams, rhos, taus, iters)
        for k, p in enumerate(plans):
            single = p.empty_hr()
            p.admm_tv(ys[k], single, lams[k], rhos[k], iters, tau_init=taus[k])
            assert torch.equal(single, xs[k]), (rep, k)
        if iters == 9:
            x9 = [x.clone() for x in xs]
    for k in (1, 4, 6):
        psf, y, dec, tau = probs[k]
        x0 = O.tikhonov(y, psf, dec, tau, O.nearest_neighbour(y, dec))
        ref = O.admm_tv(y, psf, dec, lams[k], rhos[k], 9, x0)["x"]
        assert rel_l2(x9[k].cpu().numpy(), ref) < 1e-5, k
    for p in plans:
        p.close()


def test_batched_one_and_zero_iterations_through_the_setup_graph(lib):
    """Iteration counts 1 and 0 after a grouping has run once: the set-up
    graph then carries the only iteration (count 1) or none (count 0) and no
    iteration graph is replayed; counts 2 and 3 follow on the same grouping.
    Every call equals the single-plan solves bit for bit (0 iterations: the
    Tikhonov start), and the 0-iteration result matches the oracle's eq. 12."""
    import torch
    vols = GROUPED[:5]  # a group of three 64x64x32 d222 volumes and a group of two 96x96x64 d221
    plans, ys, xs, probs = [], [], [], []
    for k, (dims, dec, sg, tau) in enumerate(vols):
        psf, xt, y = make_problem(dims, dec, sigma=(sg, 0.9 * sg, 1.1 * sg), seed=170 + k)
        p = lib.Plan(dims, dec, psf, "f32", stream=torch.cuda.Stream())
        plans.append(p)
        ys.append(torch.tensor(y, dtype=torch.float32, device="cuda"))
        xs.append(p.empty_hr())
        probs.append((psf, y, dec, tau))
    lams, rhos, taus = [2e-3] * len(plans), [1e-2] * len(plans), [v[3] for v in vols]
    for rep, iters in enumerate((3, 1, 1, 1, 0, 0, 2, 2, 3, 3)):
        for x in xs:
            x.fill_(float("nan"))
        lib.admm_tv_batched(plans, ys, xs, lams, rhos, taus, iters)
        for k, p in enumerate(plans):
            single = p.empty_hr()
            p.admm_tv(ys[k], single, lams[k], rhos[k], iters, tau_init=taus[k])
            assert torch.equal(single, xs[k]), (rep, iters, k)
        if iters == 0:
            x_tik = [x.clone() for x in xs]
    for k in (0, 3):
        psf, y, dec, tau = probs[k]
        assert rel_l2(x_tik[k].cpu().numpy(), O.tikhonov(y, psf, dec, tau, O.nearest_neighbour(y, dec))) < 1e-5, k
    for p in plans:
        p.close()


@pytest.mark.slow
def test_full_ragged_batch_against_single_solves(lib):
    """The 64-volume ragged draw of the batch benchmark (sizes 64^3,
    96x96x64, 128^3, 128x128x96; d in 2x2x2, 2x2x1, 1x1x4; tau log-uniform,
    sigma uniform; 50 iterations) on seeded smooth observations: every volume
    equals its single-plan solve bit for bit, and three small volumes match
    the oracle."""
    import torch
    import synth
    ws = synth.batch_workloads()
    plans, ys, xs, yh = [], [], [], []
    for w in ws:
        p = lib.Plan(w.dims, w.dec, w.psf(), "f32", stream=torch.cuda.Stream())
        p.autotune(2)
        m, n, s = w.lr_dims
        y = 0.5 + 0.1 * synth.normal(w.seed, 5, m * n * s).reshape((s, n, m))
        yh.append(y)
        plans.append(p)
        ys.append(torch.tensor(y, dtype=torch.float32, device="cuda"))
        xs.append(p.empty_hr())
    lams, rhos, taus = [w.lam for w in ws], [w.mu for w in ws], [w.tau for w in ws]
    lib.admm_tv_batched(plans, ys, xs, lams, rhos, taus, ws[0].iters)
    for k, p in enumerate(plans):
        single = p.empty_hr()
        p.admm_tv(ys[k], single, lams[k], rhos[k], ws[k].iters, tau_init=taus[k])
        assert torch.equal(single, xs[k]), k
    small = [k for k, w in enumerate(ws) if w.dims == (64, 64, 64)][:3]
    for k in small:
        w = ws[k]
        psf = w.psf()
        x0 = O.tikhonov(yh[k], psf, w.dec, w.tau, O.nearest_neighbour(yh[k], w.dec))
        ref = O.admm_tv(yh[k], psf, w.dec, w.lam, w.mu, w.iters, x0)["x"]
        assert rel_l2(xs[k].cpu().numpy(), ref) < 1e-5, k
    for p in plans:
        p.close()
