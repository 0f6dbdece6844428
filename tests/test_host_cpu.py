"""Host-side logic that needs no GPU: the PSF-fit helpers, the warm-start
parameter initialisation and the U-Net cost figure used by bench.py."""
import numpy as np

import oracle as O
import oracle.unet_oracle as U


def test_psf_fit_gaussian_matches_the_oracle_taps():
    from paper_2010_15491_gb300 import psf_fit
    for s, size in [((1.3, 0.9, 1.7), (9, 7, 11)), ((0.5, 2.0, 1.0), (5, 13, 7))]:
        assert np.allclose(psf_fit.gaussian_psf(s, size), O.gaussian_psf_taps(s, size), rtol=1e-14, atol=0)


def test_psf_fit_support_rule():
    from paper_2010_15491_gb300 import psf_fit
    assert psf_fit.support((1.0, 1.5, 3.0), (64, 64, 64)) == (7, 11, 19)
    # clipped to the volume, kept odd
    assert psf_fit.support((6.0, 6.0, 6.0), (64, 32, 16)) == (37, 31, 15)


def test_golden_section_fit_on_a_host_objective(monkeypatch):
    """The search finds the minimum of a smooth objective with a known minimiser
    (the GPU objective replaced by a host function)."""
    from paper_2010_15491_gb300 import psf_fit
    target = (1.7, 0.6, 2.4)

    def fake(plan, x_ref, y, sigma, size):
        r = sum((np.log(s) - np.log(t)) ** 2 for s, t in zip(sigma, target))
        return r, 1.0, 0.0

    monkeypatch.setattr(psf_fit, "objective", fake)

    class P:
        dims = (64, 64, 64)

    res = psf_fit.fit_gaussian_psf(P(), None, None, sigma0=(1.0, 1.0, 1.0), bounds=(0.3, 6.0))
    assert np.allclose(res["sigma"], target, rtol=1e-3)


def test_init_params_is_the_identity_network():
    from paper_2010_15491_gb300 import warmstart as W
    theta = W.init_params(7).astype(np.float64)
    assert theta.size == U.param_count()
    assert W.UNET_LAYERS == U.layer_shapes()
    assert np.all(theta[-17:] == 0)  # zero head: out = x
    x = np.random.default_rng(0).standard_normal((4, 8, 8))
    assert np.array_equal(U.forward(theta, x), x)
    o = 0
    for co, ci in U.layer_shapes():
        nw = co * 27 * ci
        w = theta[o:o + nw]
        assert abs(w.std() - np.sqrt(2.0 / (27 * ci))) < 0.15 * np.sqrt(2.0 / (27 * ci))
        assert np.all(theta[o + nw:o + nw + co] == 0)
        o += nw + co


def test_bench_unet_cost_counts_every_layer():
    import bench
    c1, c2, c3 = 16, 32, 64
    density = [1, 1, 1 / 8, 1 / 8, 1 / 64, 1 / 64, 1 / 8, 1 / 8, 1, 1]
    macs = sum(27 * co * ci * f for (co, ci), f in zip(U.layer_shapes((c1, c2, c3)), density)) + c1
    assert bench.UNET_MACS == macs


def test_bench_recorded_traffic_follows_sources_and_schedule():
    """bench.py reports a kernel's recorded DRAM traffic only while the plan
    runs the kernel's schedule entry of the capture and the kernel's sources
    hash to the recorded value."""
    import bench
    for kind, (nbytes, sched, files, digest) in bench.NCU_TRAFFIC.items():
        full = {"n_pass_slots": 0, "s_pass_slots": 0, "tv_planes": 0, "m_fwd_lines": 0, "m_inv_lines": 0}
        full.update(sched)
        other = dict(full)
        key = next(iter(sched))
        other[key] = sched[key] + 1
        got = bench.ncu_traffic(kind, full)
        assert got in (nbytes, None)  # None once the sources changed
        assert bench.ncu_traffic(kind, other) is None
    assert bench.ncu_traffic("tv", None) == bench.ncu_traffic("tv", {"tv_planes": 37})
    assert bench.ncu_traffic("no_such_kernel") is None
