"""FP64 CPU oracle for the fast 3D single-image super-resolution method
(Tuador, Pham, Michetti, Basarab, Kouame, "A Novel Fast 3D Single Image
Super-Resolution Algorithm", arXiv:2010.15491).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import this module.  The CUDA library never
imports, links or calls it, and this module shares no code with it.

It is deliberately plain: numpy arrays in float64 / complex128, scipy's FFT
(pocketfft, threaded over the host's cores) as a library primitive (pinned
against an explicit DFT in the tests), and the paper's formulas written out in
the paper's order.  Nothing is fused, tiled or reordered.

Conventions (readings of the paper where it is silent):
  * A volume with HR sizes (m_h, n_h, s_h) is an array of shape (s_h, n_h, m_h);
    m is the fastest axis ("lexicographic" ordering, Sec. II-A).
  * dec = (dr, dc, ds) decimates the m, n and s axes; r in eq. 9, 12 and
    Algorithm 1 is d = dr*dc*ds.
  * The DFT is the unnormalised forward transform (fftn).  Every formula below is
    invariant under the choice between it and the paper's unitary F.
  * Lambda is the DFT of the PSF zero-padded to HR size with its centre tap
    (index floor(p/2)) moved to the origin: the eigenvalues of the circulant H.
  * D keeps sample 0 of every dr x dc x ds block; D^H fills zeros.
  * The Tikhonov weight is tau = 2*lambda of eq. 5.
  * L stacks periodic forward differences along m, n, s (components in that
    order); L^T is the matching periodic backward difference, negated.
  * TV is isotropic: sum_j ||(Lx)_j||_2, as the per-voxel shrinkage of
    Algorithm 1 step 5b implies.
  * Gamma = (sum_a Sigma_a^H Sigma_a)^-1 of Algorithm 1 step 4 is singular at
    the zero frequency; the aliasing class holding the zero frequency is solved
    exactly instead (a dense d x d solve of the class block).
  * ADMM starts from u0 = L x0 and d0 = 0 unless given (Algorithm 1 leaves the
    choice open).
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as _sfft

__all__ = [
    "otf", "blur", "decimate", "zero_fill", "forward", "nearest_neighbour",
    "fold", "replicate", "tikhonov", "grad", "grad_adj", "laplacian_symbol",
    "shrink", "shrink_aniso", "tv_term", "admm_xstep", "admm_tv", "objective", "augmented_lagrangian",
    "tikhonov_grad", "tikhonov_cg", "gaussian_psf_taps", "psf_fit_objective",
    "psnr", "fftn", "ifftn", "FFT_WORKERS",
]

# threads of the FFT primitive (the host's cores); the rest of the oracle is
# single-threaded numpy
FFT_WORKERS = os.cpu_count() or 1


def fftn(a: np.ndarray) -> np.ndarray:
    """Unnormalised forward 3D DFT X[k] = sum_n a[n] exp(-2 pi i k.n / N) (library primitive)."""
    return _sfft.fftn(a, workers=FFT_WORKERS)


def ifftn(a: np.ndarray) -> np.ndarray:
    """Inverse of fftn: the conjugate-exponent sum scaled by 1/N (library primitive)."""
    return _sfft.ifftn(a, workers=FFT_WORKERS)


def _lr_shape(shape, dec):
    s, n, m = shape
    dr, dc, ds = dec
    if m % dr or n % dc or s % ds:
        raise ValueError("HR sizes must be multiples of the decimation factors")
    return (s // ds, n // dc, m // dr)


def _hr_shape(lr_shape, dec):
    s, n, m = lr_shape
    dr, dc, ds = dec
    return (s * ds, n * dc, m * dr)


# ---------------------------------------------------------------------------
# Degradation model, Sec. II-A, eq. (1)-(2)
# ---------------------------------------------------------------------------

def otf(psf: np.ndarray, shape) -> np.ndarray:
    """Lambda of eq. (2): DFT of the PSF zero-padded to `shape` (the first column of H).

    psf has shape (p_s, p_n, p_m); its centre tap floor(p/2) goes to index 0.
    """
    big = np.zeros(shape, dtype=np.float64)
    ps, pn, pm = psf.shape
    if ps > shape[0] or pn > shape[1] or pm > shape[2]:
        raise ValueError("PSF larger than the volume")
    big[:ps, :pn, :pm] = psf
    big = np.roll(big, (-(ps // 2), -(pn // 2), -(pm // 2)), axis=(0, 1, 2))
    return fftn(big)


def blur(x: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """H x = F^H Lambda F x (eq. 2): cyclic convolution."""
    return np.real(ifftn(lam * fftn(x)))


def decimate(z: np.ndarray, dec) -> np.ndarray:
    """D z: keep sample 0 of every dr x dc x ds block."""
    dr, dc, ds = dec
    return z[::ds, ::dc, ::dr].copy()


def zero_fill(y: np.ndarray, dec) -> np.ndarray:
    """D^H y: interpolate with zeros (so D D^H = I)."""
    dr, dc, ds = dec
    s, n, m = y.shape
    out = np.zeros((s * ds, n * dc, m * dr), dtype=np.float64)
    out[::ds, ::dc, ::dr] = y
    return out


def forward(x: np.ndarray, psf: np.ndarray, dec) -> np.ndarray:
    """D H x, the noiseless part of eq. (1)."""
    return decimate(blur(x, otf(psf, x.shape)), dec)


def nearest_neighbour(y: np.ndarray, dec) -> np.ndarray:
    """Nearest-neighbour replication of the LR volume: a choice of the prior x-bar of eq. (5)."""
    dr, dc, ds = dec
    return np.repeat(np.repeat(np.repeat(y, ds, axis=0), dc, axis=1), dr, axis=2)


# ---------------------------------------------------------------------------
# Aliasing structure, eq. (8) and the folded Lambda below eq. (9)
# ---------------------------------------------------------------------------

def fold(Z: np.ndarray, dec) -> np.ndarray:
    """[(1_ds^T (x) I_sl) (x) (1_dc^T (x) I_nl) (x) (1_dr^T (x) I_ml)] Z.

    HR frequency (i_s + p_s s_l, i_n + p_n n_l, i_m + p_m m_l) is summed into LR
    frequency (i_s, i_n, i_m): an explicit loop over the d aliased blocks.
    """
    sl, nl, ml = _lr_shape(Z.shape, dec)
    dr, dc, ds = dec
    out = np.zeros((sl, nl, ml), dtype=Z.dtype)
    for ps in range(ds):
        for pn in range(dc):
            for pm in range(dr):
                out += Z[ps * sl:(ps + 1) * sl, pn * nl:(pn + 1) * nl, pm * ml:(pm + 1) * ml]
    return out


def replicate(Zl: np.ndarray, dec) -> np.ndarray:
    """Adjoint of fold: copy each LR frequency to the d HR frequencies of its class."""
    dr, dc, ds = dec
    return np.tile(Zl, (ds, dc, dr))


# ---------------------------------------------------------------------------
# Tikhonov regularisation, Sec. III-A, eq. (5)-(12): 3D-FSR-l2-l2
# ---------------------------------------------------------------------------

def tikhonov(y: np.ndarray, psf: np.ndarray, dec, tau: float, xbar=None) -> np.ndarray:
    """Minimiser of 1/2 ||y - DHx||^2 + tau/2 ||x - xbar||^2 by eq. (12) with 2*lambda = tau.

    xbar=None means xbar = 0.
    """
    if tau <= 0:
        raise ValueError("tau must be positive")
    dr, dc, ds = dec
    shape = (y.shape[0] * ds, y.shape[1] * dc, y.shape[2] * dr)
    d = dr * dc * ds
    lam = otf(psf, shape)
    # F k with k = H^H D^H y + 2 lambda xbar (eq. 7)
    Fk = np.conj(lam) * fftn(zero_fill(y, dec))
    if xbar is not None:
        Fk = Fk + tau * fftn(xbar)
    # eq. (12): x = k/(2l) - 1/(2l) F^H Lam_^H (2l r I + Lam_ Lam_^H)^-1 Lam_ F k
    inner = fold(lam * Fk, dec) / (tau * d + fold(np.abs(lam) ** 2, dec))
    X = Fk / tau - np.conj(lam) * replicate(inner, dec) / tau
    return np.real(ifftn(X))


# ---------------------------------------------------------------------------
# Total variation by ADMM, Sec. III-B, Algorithm 1: 3D-FSR-l2-TV
# ---------------------------------------------------------------------------

def grad(x: np.ndarray) -> np.ndarray:
    """L x = [D_m x; D_n x; D_s x]: periodic forward differences, shape (3,) + x.shape."""
    return np.stack([np.roll(x, -1, axis=2) - x,
                     np.roll(x, -1, axis=1) - x,
                     np.roll(x, -1, axis=0) - x])


def grad_adj(p: np.ndarray) -> np.ndarray:
    """L^T p = sum_a D_a^T p_a with (D_a^T q)[j] = q[j - e_a] - q[j]."""
    return ((np.roll(p[0], 1, axis=2) - p[0])
            + (np.roll(p[1], 1, axis=1) - p[1])
            + (np.roll(p[2], 1, axis=0) - p[2]))


def laplacian_symbol(shape) -> np.ndarray:
    """Sigma_h^H Sigma_h + Sigma_v^H Sigma_v + Sigma_s^H Sigma_s (Algorithm 1 steps 3-4):
    |exp(2 pi i k_a / N_a) - 1|^2 = 4 sin^2(pi k_a / N_a) summed over the three axes."""
    s, n, m = shape
    ks = 4.0 * np.sin(np.pi * np.arange(s) / s) ** 2
    kn = 4.0 * np.sin(np.pi * np.arange(n) / n) ** 2
    km = 4.0 * np.sin(np.pi * np.arange(m) / m) ** 2
    return ks[:, None, None] + kn[None, :, None] + km[None, None, :]


def shrink(nu: np.ndarray, t: float) -> np.ndarray:
    """Isotropic soft threshold of Algorithm 1 step 5b; u = 0 where ||nu_j|| <= t."""
    nrm = np.sqrt((nu ** 2).sum(axis=0))
    scale = np.zeros_like(nrm)
    big = nrm > t
    scale[big] = (nrm[big] - t) / nrm[big]
    return nu * scale[None]


def shrink_aniso(nu: np.ndarray, t: float) -> np.ndarray:
    """Anisotropic soft threshold: the prox of t * sum_a |nu_a| (the u-step of
    Algorithm 1 step 5b when phi is the anisotropic TV sum_j sum_a |(D_a x)_j|,
    one of the other regularisers the conclusion of the paper points to):
    each component shrinks towards 0 by t, u_a = 0 where |nu_a| <= t."""
    return np.sign(nu) * np.maximum(np.abs(nu) - t, 0.0)


def tv_term(g: np.ndarray, aniso: bool = False) -> float:
    """sum_j ||g_j||_2 (isotropic TV) or sum_j sum_a |g_a,j| (anisotropic)."""
    if aniso:
        return float(np.abs(g).sum())
    return float(np.sqrt((g ** 2).sum(axis=0)).sum())


def dc_class_indices(shape, dec):
    """HR frequencies aliased onto the LR zero frequency (eq. 8), member (0,0,0) first."""
    sl, nl, ml = _lr_shape(shape, dec)
    dr, dc, ds = dec
    return [(ps * sl, pn * nl, pm * ml) for ps in range(ds) for pn in range(dc) for pm in range(dr)]


def admm_xstep(y: np.ndarray, lam: np.ndarray, theta: np.ndarray, mu: float, dec) -> np.ndarray:
    """x-update of Algorithm 1 step 5a: the minimiser of
    1/2 ||y - DHx||^2 + mu/2 ||Lx - (u - d)||^2, given Theta = L^T (u - d)."""
    shape = theta.shape
    dr, dc, ds = dec
    d = dr * dc * ds
    # F k = Lambda^H F D^H y + mu F Theta
    Fk = np.conj(lam) * fftn(zero_fill(y, dec)) + mu * fftn(theta)
    sym = laplacian_symbol(shape)
    gamma = np.zeros_like(sym)
    nz = sym > 0
    gamma[nz] = 1.0 / sym[nz]
    # x_f = Gamma Lam_^H (mu r I + Lam_ Gamma Lam_^H)^-1 Lam_ Gamma F k
    inner = fold(lam * gamma * Fk, dec) / (mu * d + fold(np.abs(lam) ** 2 * gamma, dec))
    xf = gamma * np.conj(lam) * replicate(inner, dec)
    # x = 1/mu (F^H Gamma F k - F^H x_f), assembled in the Fourier domain
    X = (gamma * Fk - xf) / mu
    # Gamma is singular at the zero frequency: solve that aliasing class exactly.
    # Its block of (Lambda^H F D_ F^H Lambda + mu Sigma^H Sigma) is
    # mu diag(s_p) + (1/d) conj(Lambda_p) Lambda_q  (eq. 8).
    idx = dc_class_indices(shape, dec)
    lv = np.array([lam[i] for i in idx])
    sv = np.array([sym[i] for i in idx])
    A = mu * np.diag(sv) + np.outer(np.conj(lv), lv) / d
    sol = np.linalg.solve(A, np.array([Fk[i] for i in idx]))
    for i, v in zip(idx, sol):
        X[i] = v
    return np.real(ifftn(X))


def objective(x: np.ndarray, y: np.ndarray, psf: np.ndarray, dec, lam_tv: float, aniso: bool = False) -> float:
    """1/2 ||y - DHx||^2 + lambda phi(Lx) (eq. 3), phi the isotropic TV (or the
    anisotropic one with aniso=True)."""
    r = y - forward(x, psf, dec)
    return 0.5 * float((r ** 2).sum()) + lam_tv * tv_term(grad(x), aniso)


def tikhonov_grad(y: np.ndarray, psf: np.ndarray, dec, tau: float) -> np.ndarray:
    """Minimiser of 1/2 ||y - DHx||^2 + tau/2 ||Lx||^2 (Tikhonov on the
    gradient, another regulariser for the same Fourier-domain solve): its
    normal equations (H^T D^T D H + tau L^T L) x = H^T D^T y are those of the
    ADMM x-subproblem of Algorithm 1 step 5a with u - d = 0 and mu = tau."""
    return admm_xstep(y, otf(psf, _hr_shape(y.shape, dec)), np.zeros(_hr_shape(y.shape, dec)), tau, dec)


def augmented_lagrangian(x, u, dvar, y, psf, dec, lam_tv, mu) -> float:
    """L(x, u, d) = 1/2||y - DHx||^2 + lambda phi(u) + mu/2 ||Lx - (u - d)||^2 (Sec. III-B)."""
    r = y - forward(x, psf, dec)
    tv = float(np.sqrt((u ** 2).sum(axis=0)).sum())
    c = grad(x) - (u - dvar)
    return 0.5 * float((r ** 2).sum()) + lam_tv * tv + 0.5 * mu * float((c ** 2).sum())


def gaussian_psf_taps(sigma, size) -> np.ndarray:
    """Separable Gaussian of standard deviations sigma = (sigma_m, sigma_n,
    sigma_s) on an odd support size = (p_m, p_n, p_s), centre tap p // 2,
    normalised to sum 1 after truncation; shape (p_s, p_n, p_m)."""
    g = [np.exp(-0.5 * ((np.arange(p) - p // 2) / s) ** 2) for s, p in zip(sigma, size)]
    psf = np.einsum("i,j,k->ijk", g[2], g[1], g[0])
    return psf / psf.sum()


def psf_fit_objective(sigma, size, x_ref: np.ndarray, y: np.ndarray, dec):
    """Objective of the Gaussian PSF fit (Sec. IV estimates its PSF as a 3D
    Gaussian with the HR reference volume at hand): the least-squares misfit
    min_{a,b} ||y - a D H_sigma x_ref - b||^2 and its minimisers (a, b)."""
    yh = forward(x_ref, gaussian_psf_taps(sigma, size), dec).ravel()
    A = np.stack([yh, np.ones_like(yh)], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, y.ravel(), rcond=None)
    r = y.ravel() - a * yh - b
    return float(r @ r), float(a), float(b)


def tikhonov_cg(y: np.ndarray, psf: np.ndarray, dec, tau: float, xbar=None, iters: int = 100,
                tol: float = 0.0) -> dict:
    """The iterative comparator of Sec. IV (Table 1 solves eq. 5 both by eq. 12
    and iteratively): conjugate gradients on the normal equations of eq. 6,
    (H^T D^T D H + tau I) x = H^T D^T y + tau xbar, from x = 0.  Every operator
    application is spatial: H by its DFT diagonalisation (eq. 2), D^T D as the
    sampling mask.  Stops after `iters` iterations or when ||r|| <= tol ||b||.
    Returns x, the iterations run and the residual norms ||r_k||."""
    lam = otf(psf, _hr_shape(y.shape, dec))
    H = lambda v: np.real(ifftn(lam * fftn(v)))  # noqa: E731
    Ht = lambda v: np.real(ifftn(np.conj(lam) * fftn(v)))  # noqa: E731
    A = lambda v: Ht(zero_fill(decimate(H(v), dec), dec)) + tau * v  # noqa: E731
    b = Ht(zero_fill(y, dec))
    if xbar is not None:
        b = b + tau * xbar
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float((r * r).sum())
    bnorm = np.sqrt(float((b * b).sum()))
    res = [np.sqrt(rr)]
    k = 0
    while k < iters and not (tol > 0 and np.sqrt(rr) <= tol * bnorm):
        Ap = A(p)
        alpha = rr / float((p * Ap).sum())
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float((r * r).sum())
        p = r + (rr_new / rr) * p
        rr = rr_new
        res.append(np.sqrt(rr))
        k += 1
    return {"x": x, "iters": k, "residuals": res}


def admm_tv(y: np.ndarray, psf: np.ndarray, dec, lam_tv: float, mu: float, iters: int,
            x0: np.ndarray, d0=None, u0=None, record: bool = False, callback=None, aniso: bool = False) -> dict:
    """Algorithm 1 (3D-FSR-l2-TV) for `iters` iterations from x0.

    u0 defaults to L x0 and d0 to zero.  Returns x, u, d after the last
    iteration and, with record=True, per-iteration history: objective,
    primal residual ||Lx - u||, dual residual mu ||L^T (u - u_prev)||, and the
    norms ||Lx||, ||u||, mu ||L^T d|| used by relative stopping tests.
    `callback(i, x, u, d)` is called after every iteration.  aniso=True
    uses the anisotropic TV (shrink_aniso in the u-step, its objective).
    """
    if mu <= 0:
        raise ValueError("mu must be positive")
    shape = x0.shape
    lam = otf(psf, shape)
    x = np.array(x0, dtype=np.float64)
    u = grad(x) if u0 is None else np.array(u0, dtype=np.float64)
    dvar = np.zeros((3,) + shape) if d0 is None else np.array(d0, dtype=np.float64)
    hist = {"objective": [], "primal": [], "dual": [], "norm_Lx": [], "norm_u": [], "norm_LTd": []}
    for i in range(iters):
        # step 5a: rho = u - d, Theta = L^T rho, x from eq. (12) with Gamma
        theta = grad_adj(u - dvar)
        x = admm_xstep(y, lam, theta, mu, dec)
        # step 5b: u from the isotropic soft threshold of nu = Lx + d
        g = grad(x)
        u_prev = u
        u = (shrink_aniso if aniso else shrink)(g + dvar, lam_tv / mu)
        # step 5c: d = d + (Lx - u)
        dvar = dvar + (g - u)
        if record:
            hist["objective"].append(objective(x, y, psf, dec, lam_tv, aniso))
            hist["primal"].append(float(np.sqrt(((g - u) ** 2).sum())))
            hist["dual"].append(mu * float(np.sqrt((grad_adj(u - u_prev) ** 2).sum())))
            hist["norm_Lx"].append(float(np.sqrt((g ** 2).sum())))
            hist["norm_u"].append(float(np.sqrt((u ** 2).sum())))
            hist["norm_LTd"].append(mu * float(np.sqrt((grad_adj(dvar) ** 2).sum())))
        if callback is not None:
            callback(i, x, u, dvar)
    return {"x": x, "u": u, "d": dvar, "hist": hist}


def psnr(x: np.ndarray, x_true: np.ndarray) -> float:
    """10 log10(max(x_true)^2 / MSE) over HR voxels (the paper's PSNR, Sec. IV)."""
    mse = float(((x - x_true) ** 2).mean())
    return 10.0 * np.log10(float(x_true.max()) ** 2 / mse)
