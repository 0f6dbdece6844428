"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: explicit DFT
matrices, dense circulant matrices built tap by tap, closed-form special cases,
exact rational solves (tests/golden), an independent primal-dual solver and
invariants of ADMM.  No GPU is needed.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import oracle.dense as D
from synth import gaussian_psf

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rand_psf(rng, shape):
    p = rng.random(shape) + 0.05
    return p / p.sum()


def dft_matrix(n):
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n)


# ---------------------------------------------------------------------------
# FFT primitive
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(4, 6, 5), (3, 8, 6), (2, 2, 12), (5, 3, 7)])
def test_fft_is_the_unnormalised_dft(shape):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Fs, Fn, Fm = (dft_matrix(n) for n in shape)
    ref = np.einsum("ai,bj,ck,ijk->abc", Fs, Fn, Fm, x)
    assert np.allclose(O.fftn(x), ref, atol=1e-11)
    assert np.allclose(O.ifftn(ref), x, atol=1e-12)
    # the real-input path the oracle takes for volumes
    assert np.allclose(O.fftn(x.real), np.einsum("ai,bj,ck,ijk->abc", Fs, Fn, Fm, x.real), atol=1e-11)
    # Parseval for the unnormalised transform
    assert np.isclose((np.abs(ref) ** 2).sum(), x.size * (np.abs(x) ** 2).sum())


# ---------------------------------------------------------------------------
# eq. (8): F D_ F^H is a Kronecker product of scaled all-ones blocks
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,dec", [((4, 6, 8), (2, 3, 2)), ((6, 2, 4), (1, 1, 3)), ((4, 4, 2), (2, 2, 4))])
def test_aliasing_lemma_eq8(shape, dec):
    s, n, m = shape
    dr, dc, ds = dec
    F = np.kron(np.kron(dft_matrix(s), dft_matrix(n)), dft_matrix(m)) / np.sqrt(s * n * m)  # unitary
    Dm = D.decimation_matrix(shape, dec)
    lhs = F @ (Dm.T @ Dm) @ F.conj().T

    def blk(dd, nl):
        return np.kron(np.ones((dd, dd)), np.eye(nl)) / dd

    rhs = np.kron(np.kron(blk(ds, s // ds), blk(dc, n // dc)), blk(dr, m // dr))
    assert np.abs(lhs - rhs).max() < 1e-13
    # the folding matrix below eq. (9) is what oracle.fold applies
    fold_mat = np.kron(np.kron(np.kron(np.ones((1, ds)), np.eye(s // ds)),
                               np.kron(np.ones((1, dc)), np.eye(n // dc))),
                       np.kron(np.ones((1, dr)), np.eye(m // dr)))
    rng = np.random.default_rng(2)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    assert np.allclose(O.fold(z, dec).ravel(), fold_mat @ z.ravel(), atol=1e-13)
    w = rng.standard_normal(O.fold(z, dec).shape)
    assert np.allclose(O.replicate(w, dec).ravel(), fold_mat.T @ w.ravel(), atol=1e-13)


# ---------------------------------------------------------------------------
# degradation model eq. (1)-(2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,dec,pshape", [((4, 6, 8), (2, 3, 2), (3, 3, 3)),
                                               ((8, 4, 4), (1, 2, 4), (5, 1, 3)),
                                               ((3, 5, 6), (1, 1, 1), (2, 4, 3))])
def test_forward_model_matches_spatial_convolution(shape, dec, pshape):
    rng = np.random.default_rng(3)
    psf = rand_psf(rng, pshape)  # asymmetric, even sizes included
    x = rng.standard_normal(shape)
    A = D.decimation_matrix(shape, dec) @ D.blur_matrix(psf, shape)
    assert np.abs(O.forward(x, psf, dec).ravel() - A @ x.ravel()).max() < 1e-13
    # Lambda holds the eigenvalues of the circulant H: H v_k = Lambda_k v_k
    Hm = D.blur_matrix(psf, shape)
    lam = O.otf(psf, shape)
    k = (1, 2, 3 % shape[2])
    idx = np.indices(shape)
    v = np.exp(2j * np.pi * sum(k[a] * idx[a] / shape[a] for a in range(3))).ravel()
    assert np.allclose(Hm @ v, lam[k] * v, atol=1e-12)


def test_zero_fill_is_adjoint_of_decimation():
    rng = np.random.default_rng(4)
    z = rng.standard_normal((4, 6, 8))
    y = rng.standard_normal((2, 2, 4))
    dec = (2, 3, 2)
    assert np.isclose((O.decimate(z, dec) * y).sum(), (z * O.zero_fill(y, dec)).sum())
    assert np.array_equal(O.decimate(O.zero_fill(y, dec), dec), y)  # D D^H = I


# ---------------------------------------------------------------------------
# Tikhonov, eq. (5)-(12)
# ---------------------------------------------------------------------------

TIK_CASES = [((4, 6, 8), (2, 3, 2), (3, 3, 3), "rand"),
             ((8, 4, 4), (1, 1, 4), (5, 3, 3), "none"),
             ((4, 4, 6), (2, 2, 2), (3, 2, 3), "nn"),
             ((6, 4, 4), (2, 1, 1), (1, 3, 3), "rand")]


@pytest.mark.parametrize("shape,dec,pshape,prior", TIK_CASES)
def test_tikhonov_matches_dense_normal_equations(shape, dec, pshape, prior):
    rng = np.random.default_rng(5)
    psf = rand_psf(rng, pshape)
    lr = tuple(a // b for a, b in zip(shape, dec[::-1]))
    y = rng.standard_normal(lr)
    xbar = {"none": None, "rand": rng.standard_normal(shape), "nn": O.nearest_neighbour(y, dec)}[prior]
    for tau in (1e-2, 0.3, 5.0):
        x = O.tikhonov(y, psf, dec, tau, xbar)
        xd, M, rhs = D.tikhonov_dense(y, psf, dec, tau, xbar)
        assert np.abs(x - xd).max() < 1e-10 * max(1.0, np.abs(xd).max())
        assert np.abs(M @ x.ravel() - rhs).max() < 1e-10  # normal-equation residual


def test_tikhonov_no_decimation_is_wiener():
    rng = np.random.default_rng(6)
    shape = (6, 8, 10)
    psf = rand_psf(rng, (3, 5, 3))
    y = rng.standard_normal(shape)
    xbar = rng.standard_normal(shape)
    tau = 0.05
    lam = O.otf(psf, shape)
    X = (np.conj(lam) * np.fft.fftn(y) + tau * np.fft.fftn(xbar)) / (np.abs(lam) ** 2 + tau)
    assert np.allclose(O.tikhonov(y, psf, (1, 1, 1), tau, xbar), np.real(np.fft.ifftn(X)), atol=1e-12)


def test_tikhonov_delta_psf_is_voxelwise():
    rng = np.random.default_rng(7)
    dec = (2, 2, 2)
    y = rng.standard_normal((3, 4, 2))
    shape = (6, 8, 4)
    xbar = rng.standard_normal(shape)
    tau = 0.4
    x = O.tikhonov(y, np.ones((1, 1, 1)), dec, tau, xbar)
    expect = xbar.copy()
    expect[::2, ::2, ::2] = (y + tau * xbar[::2, ::2, ::2]) / (1.0 + tau)
    assert np.allclose(x, expect, atol=1e-13)


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *rest = line.split()
            vals[key] = rest
    shp = lambda k: tuple(int(v) for v in vals[k])  # noqa: E731
    frac = lambda k: np.array([float(Fraction(v)) for v in vals[k]])  # noqa: E731
    out = dict(lr=shp("lr_shape"), dec=shp("dec"), pshape=shp("psf_shape"), tau=float(Fraction(vals["tau"][0])))
    out["y"] = frac("y").reshape(out["lr"])
    out["psf"] = frac("psf").reshape(out["pshape"])
    dr, dc, ds = out["dec"]
    shape = (out["lr"][0] * ds, out["lr"][1] * dc, out["lr"][2] * dr)
    out["xbar"] = frac("xbar").reshape(shape) if "xbar" in vals else None
    out["x"] = frac("x").reshape(shape)
    return out


@pytest.mark.parametrize("name", ["tik_1d_m8_d2.txt", "tik_3d_4x4x2_d221_asym.txt"])
def test_tikhonov_golden_exact(name):
    g = _read_golden(name)
    x = O.tikhonov(g["y"], g["psf"], g["dec"], g["tau"], g["xbar"])
    assert np.abs(x - g["x"]).max() < 1e-13


# ---------------------------------------------------------------------------
# ADMM-TV, Algorithm 1
# ---------------------------------------------------------------------------

def test_grad_and_adjoint_match_dense_operator():
    rng = np.random.default_rng(8)
    shape = (3, 4, 5)
    L = D.grad_matrix(shape)
    x = rng.standard_normal(shape)
    p = rng.standard_normal((3,) + shape)
    assert np.allclose(O.grad(x).ravel(), L @ x.ravel(), atol=1e-14)
    assert np.allclose(O.grad_adj(p).ravel(), L.T @ p.ravel(), atol=1e-14)
    # L^T L is diagonalised by the DFT with the symbol of Algorithm 1 step 4
    e = np.zeros(shape)
    e[0, 0, 0] = 1.0
    assert np.allclose(np.fft.fftn(O.grad_adj(O.grad(e))), O.laplacian_symbol(shape), atol=1e-13)


def test_shrink_edge_cases_and_prox_optimality():
    t = 0.5
    nu = np.zeros((3, 4, 1, 1))
    nu[:, 1, 0, 0] = [0.3, 0.4, 0.0]       # norm exactly t: ties go to zero
    nu[:, 2, 0, 0] = [3.0, 0.0, 4.0]       # norm 5
    nu[:, 3, 0, 0] = [1e-3, 0.0, 0.0]
    u = O.shrink(nu, t)
    assert np.all(u[:, 0] == 0) and np.all(u[:, 1] == 0) and np.all(u[:, 3] == 0)
    assert np.allclose(u[:, 2, 0, 0], np.array([3.0, 0.0, 4.0]) * 4.5 / 5.0)
    # u minimises t ||u|| + 1/2 ||u - nu||^2 per voxel: compare with a dense search
    rng = np.random.default_rng(9)
    for _ in range(5):
        v = rng.standard_normal(3)
        best = O.shrink(v.reshape(3, 1, 1, 1), t).ravel()
        f = lambda w: t * np.linalg.norm(w) + 0.5 * np.sum((w - v) ** 2)  # noqa: E731
        cand = rng.standard_normal((20000, 3)) * 0.3 + best
        assert f(best) <= min(f(c) for c in cand) + 1e-12


@pytest.mark.parametrize("shape,dec,pshape", [((4, 4, 4), (2, 2, 2), (3, 3, 3)),
                                               ((8, 4, 2), (1, 1, 4), (3, 3, 1)),
                                               ((4, 6, 4), (2, 3, 1), (2, 3, 3)),
                                               ((4, 4, 8), (2, 1, 1), (3, 3, 3))])
def test_admm_xstep_is_exact_minimiser(shape, dec, pshape):
    rng = np.random.default_rng(10)
    psf = rand_psf(rng, pshape)
    lr = (shape[0] // dec[2], shape[1] // dec[1], shape[2] // dec[0])
    y = rng.standard_normal(lr)
    rho = rng.standard_normal((3,) + shape)
    lam = O.otf(psf, shape)
    for mu in (1e-2, 0.7):
        x = O.admm_xstep(y, lam, O.grad_adj(rho), mu, dec)
        xd, M, rhs = D.admm_xstep_dense(y, psf, dec, mu, rho, shape)
        assert np.abs(x - xd).max() < 1e-9 * max(1.0, np.abs(xd).max())
        assert np.abs(M @ x.ravel() - rhs).max() < 1e-10 * max(1.0, np.abs(rhs).max())


def _small_problem(seed=11, shape=(4, 4, 4), dec=(2, 2, 2)):
    rng = np.random.default_rng(seed)
    psf = gaussian_psf((0.8, 0.8, 0.8), (3, 3, 3))
    xt = (rng.random(shape) > 0.5).astype(float)
    lr = (shape[0] // dec[2], shape[1] // dec[1], shape[2] // dec[0])
    y = O.forward(xt, psf, dec) + 0.01 * rng.standard_normal(lr)
    return psf, y, xt


def test_admm_steps_do_not_increase_augmented_lagrangian():
    psf, y, _ = _small_problem()
    dec, lam_tv, mu = (2, 2, 2), 0.05, 0.3
    shape = (4, 4, 4)
    lam = O.otf(psf, shape)
    x = O.tikhonov(y, psf, dec, 0.1, O.nearest_neighbour(y, dec))
    u = O.grad(x)
    dv = np.zeros((3,) + shape)
    for _ in range(15):
        L0 = O.augmented_lagrangian(x, u, dv, y, psf, dec, lam_tv, mu)
        x = O.admm_xstep(y, lam, O.grad_adj(u - dv), mu, dec)
        L1 = O.augmented_lagrangian(x, u, dv, y, psf, dec, lam_tv, mu)
        u = O.shrink(O.grad(x) + dv, lam_tv / mu)
        L2 = O.augmented_lagrangian(x, u, dv, y, psf, dec, lam_tv, mu)
        assert L1 <= L0 + 1e-12 and L2 <= L1 + 1e-12
        dv = dv + O.grad(x) - u
    # and the loop in admm_tv performs exactly these steps
    r = O.admm_tv(y, psf, dec, lam_tv, mu, 15, O.tikhonov(y, psf, dec, 0.1, O.nearest_neighbour(y, dec)))
    assert np.allclose(r["x"], x, atol=1e-13) and np.allclose(r["d"], dv, atol=1e-13)


@pytest.mark.slow
def test_admm_reaches_the_primal_dual_optimum():
    shape, dec = (4, 4, 8), (2, 2, 2)
    psf, y, _ = _small_problem(12, shape, dec)
    lam_tv = 0.02
    x0 = O.tikhonov(y, psf, dec, 0.1, O.nearest_neighbour(y, dec))
    r = O.admm_tv(y, psf, dec, lam_tv, 0.05, 3000, x0)
    f_admm = O.objective(r["x"], y, psf, dec, lam_tv)
    _, f_cp = D.chambolle_pock_tv(y, psf, dec, lam_tv, shape, iters=40000, x0=r["x"] * 0)
    assert abs(f_admm - f_cp) <= 1e-6 * f_cp


def test_admm_large_lambda_gives_constant():
    shape, dec = (4, 4, 4), (2, 2, 2)
    psf, y, _ = _small_problem(13, shape, dec)
    x0 = O.tikhonov(y, psf, dec, 0.1, O.nearest_neighbour(y, dec))
    r = O.admm_tv(y, psf, dec, 1e4, 1.0, 300, x0)
    assert np.allclose(r["x"], y.mean() / psf.sum(), atol=1e-6)


def test_data_term_by_parseval_over_aliasing_classes():
    """||y - DHx||^2 = (1/N_l) sum_i |Y_i - (1/d) sum_p Lambda_p X_p|^2: the data
    term of the objective needs only the fold of eq. (8), no extra transform."""
    rng = np.random.default_rng(14)
    shape, dec = (4, 6, 8), (2, 3, 2)
    psf = rand_psf(rng, (3, 3, 3))
    x = rng.standard_normal(shape)
    y = rng.standard_normal((2, 2, 4))
    lam = O.otf(psf, shape)
    direct = ((y - O.forward(x, psf, dec)) ** 2).sum()
    R = np.fft.fftn(y) - O.fold(lam * np.fft.fftn(x), dec) / np.prod(dec)
    # fold of an unnormalised HR DFT, /d, is the LR DFT of the decimated volume
    assert np.isclose(direct, (np.abs(R) ** 2).sum() / y.size)


# ---------------------------------------------------------------------------
# other regularisers through the same x-step
# ---------------------------------------------------------------------------

def test_shrink_aniso_is_the_prox_of_the_l1_norm():
    """u = shrink_aniso(nu, t) satisfies 0 in u - nu + t d|u| componentwise,
    and differs from the isotropic shrink unless one component is nonzero."""
    rng = np.random.default_rng(21)
    nu = rng.standard_normal((3, 50))
    t = 0.4
    u = O.shrink_aniso(nu, t)
    nz = u != 0
    assert np.allclose((u - nu + t * np.sign(u))[nz], 0.0)
    assert np.all(np.abs(nu[~nz]) <= t)
    one = np.zeros((3, 4))
    one[1] = [-2.0, -0.1, 0.3, 5.0]
    assert np.allclose(O.shrink_aniso(one, t), O.shrink(one, t))
    assert not np.allclose(u, O.shrink(nu, t))


def test_admm_aniso_reaches_the_primal_dual_optimum():
    shape, dec = (4, 4, 8), (2, 2, 2)
    psf, y, _ = _small_problem(22, shape, dec)
    lam_tv = 0.005  # small enough that the solution is not constant
    x0 = O.tikhonov(y, psf, dec, 0.1, O.nearest_neighbour(y, dec))
    r = O.admm_tv(y, psf, dec, lam_tv, 0.05, 3000, x0, aniso=True)
    assert (np.abs(O.grad(r["x"])) > 1e-6).sum() > 10
    f_admm = O.objective(r["x"], y, psf, dec, lam_tv, aniso=True)
    _, f_cp = D.chambolle_pock_tv(y, psf, dec, lam_tv, shape, iters=40000, aniso=True)
    assert abs(f_admm - f_cp) <= 1e-6 * f_cp
    # and it is a different problem from the isotropic one
    f_iso = O.objective(O.admm_tv(y, psf, dec, lam_tv, 0.05, 3000, x0)["x"], y, psf, dec, lam_tv, aniso=True)
    assert f_iso > f_admm * (1 + 1e-2)


def test_tikhonov_grad_equals_dense_normal_equations():
    rng = np.random.default_rng(23)
    for shape, dec in [((4, 6, 8), (2, 3, 2)), ((6, 4, 4), (1, 2, 2))]:
        psf = rand_psf(rng, (3, 3, 3))  # asymmetric: complex Lambda
        lr = (shape[0] // dec[2], shape[1] // dec[1], shape[2] // dec[0])
        y = rng.standard_normal(lr)
        x = O.tikhonov_grad(y, psf, dec, 0.07)
        xd, M = D.tikhonov_grad_dense(y, psf, dec, 0.07)
        assert np.allclose(x, xd, atol=1e-10)
        # the residual of the dense system, not only agreement
        A = D.decimation_matrix(shape, dec) @ D.blur_matrix(psf, shape)
        assert np.linalg.norm(M @ x.ravel() - A.T @ y.ravel()) <= 1e-10 * np.linalg.norm(A.T @ y.ravel())


# ---------------------------------------------------------------------------
# the iterative comparator (conjugate gradients on eq. 6)
# ---------------------------------------------------------------------------

def _cg_problem(seed):
    rng = np.random.default_rng(seed)
    shape, dec = (4, 6, 8), (2, 3, 2)
    psf = rand_psf(rng, (3, 3, 3))
    y = rng.standard_normal((2, 2, 4))
    xbar = rng.standard_normal(shape)
    return shape, dec, psf, y, xbar


def test_cg_first_step_is_the_steepest_descent_step():
    """From x = 0: x_1 = (b.b / b.Ab) b (textbook closed form)."""
    shape, dec, psf, y, xbar = _cg_problem(31)
    tau = 0.3
    x1 = O.tikhonov_cg(y, psf, dec, tau, xbar, iters=1)["x"]
    _, M, rhs = D.tikhonov_dense(y, psf, dec, tau, xbar)
    alpha = (rhs @ rhs) / (rhs @ (M @ rhs))
    assert np.allclose(x1.ravel(), alpha * rhs, rtol=1e-12, atol=1e-14)


def test_cg_converges_to_the_dense_solution_and_error_decreases():
    shape, dec, psf, y, xbar = _cg_problem(32)
    tau = 0.05
    xd, M, _ = D.tikhonov_dense(y, psf, dec, tau, xbar)
    errs = []
    for k in (2, 5, 10, 20, 40):
        xk = O.tikhonov_cg(y, psf, dec, tau, xbar, iters=k)["x"]
        e = (xk - xd).ravel()
        errs.append(float(e @ (M @ e)))  # A-norm error: non-increasing in k
    assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:]))
    r = O.tikhonov_cg(y, psf, dec, tau, xbar, iters=500, tol=1e-13)
    assert r["iters"] < 500
    assert np.allclose(r["x"], xd, atol=1e-10)
    # and it matches the closed form of eq. 12 used by the fast path
    assert np.allclose(r["x"], O.tikhonov(y, psf, dec, tau, xbar), atol=1e-10)


# ---------------------------------------------------------------------------
# Gaussian PSF fit objective
# ---------------------------------------------------------------------------

def test_gaussian_taps_match_the_input_generator():
    from synth import gaussian_psf
    s, size = (1.3, 0.9, 1.7), (9, 7, 11)
    assert np.allclose(O.gaussian_psf_taps(s, size), gaussian_psf(s, size), rtol=1e-14, atol=0)


def test_psf_fit_objective_is_zero_at_the_truth_and_grows_away():
    rng = np.random.default_rng(41)
    shape, dec = (8, 16, 16), (2, 2, 2)
    x = rng.random(shape)
    size, s_true = (9, 9, 7), (1.2, 0.8, 1.5)
    y = 2.0 * O.forward(x, O.gaussian_psf_taps(s_true, size), dec) + 0.1
    r0, a, b = O.psf_fit_objective(s_true, size, x, y, dec)
    assert r0 <= 1e-24 * (y ** 2).sum() and np.isclose(a, 2.0) and np.isclose(b, 0.1)
    for ax in range(3):
        for f in (0.9, 1.1):
            s = list(s_true)
            s[ax] *= f
            assert O.psf_fit_objective(s, size, x, y, dec)[0] > 1e3 * max(r0, 1e-30)


# ---------------------------------------------------------------------------
# the nearest-neighbour prior of eq. (5): every HR voxel copies the LR voxel of
# its dr x dc x ds block, checked voxel by voxel (a swap of two axes' factors
# must fail the check)
# ---------------------------------------------------------------------------

def _nearest_agrees(fn):
    dec = (2, 1, 3)  # (dr, dc, ds) on (m, n, s): three different factors
    y = np.random.default_rng(14).standard_normal((2, 3, 4))  # LR (s, n, m)
    dr, dc, ds = dec
    ref = np.zeros((2 * ds, 3 * dc, 4 * dr))
    for s in range(ref.shape[0]):
        for n in range(ref.shape[1]):
            for m in range(ref.shape[2]):
                ref[s, n, m] = y[s // ds, n // dc, m // dr]
    got = fn(y, dec)
    return got.shape == ref.shape and np.array_equal(got, ref)


def test_nearest_neighbour_prior_copies_each_lr_voxel_to_its_block():
    assert _nearest_agrees(O.nearest_neighbour)


def test_nearest_neighbour_checker_rejects_planted_mistakes():
    def swap_m_s(y, dec):
        dr, dc, ds = dec
        return O.nearest_neighbour(y, (ds, dc, dr))

    def tiled(y, dec):
        dr, dc, ds = dec
        return np.tile(y, (ds, dc, dr))

    assert not _nearest_agrees(swap_m_s)
    assert not _nearest_agrees(tiled)
