"""Gaussian PSF fit from data.

Sec. IV estimates the PSF of its CBCT volume by approximating it with a 3D
Gaussian (a method the paper cites but does not state), with the matching
micro-CT volume as the high-resolution reference.  The estimator here: for an
HR reference x_ref and an LR observation y of the same object,

    sigma_hat = argmin_sigma  min_{a, b} || y - a D H_sigma x_ref - b ||^2,

with H_sigma the cyclic convolution by the normalised separable Gaussian of
standard deviations sigma = (sigma_m, sigma_n, sigma_s) on a fixed support, D
the decimation of the plan, and a gain a and offset b (the two scanners'
intensity scales differ) solved in closed form for each sigma.  sigma is
searched by cyclic golden-section line searches over log sigma, one axis at a
time.  Each objective evaluation replaces the plan's PSF (sr3d_set_psf) and
runs the forward model D H x and the sums of the gain/offset least squares
(sr3d_psf_fit_moments) on the GPU.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np


def gaussian_psf(sigma: Sequence[float], size: Sequence[int]) -> np.ndarray:
    """Separable Gaussian taps of shape (p_s, p_n, p_m) for sigma = (sigma_m,
    sigma_n, sigma_s) and size = (p_m, p_n, p_s) (odd), centre tap p // 2,
    normalised to sum 1 after truncation."""
    f = []
    for sg, p in zip(sigma, size):
        r = np.arange(p) - p // 2
        f.append(np.exp(-0.5 * (r / sg) ** 2))
    psf = f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    return psf / psf.sum()


def support(sigma_max: Sequence[float], dims: Sequence[int]) -> tuple:
    """Odd support 2 ceil(3 sigma) + 1 per axis, clipped to the volume."""
    return tuple(min(2 * int(math.ceil(3.0 * s)) + 1, d - (1 - d % 2)) for s, d in zip(sigma_max, dims))


def objective(plan, x_ref, y, sigma, size):
    """min over (a, b) of ||y - a D H_sigma x_ref - b||^2 and the minimising (a, b).
    The forward model and the five FP64 sums run in the library
    (sr3d_set_psf, sr3d_psf_fit_moments); only the 2x2 solve is here."""
    plan.set_psf(gaussian_psf(sigma, size))
    s1, s2, t1, t2, c = plan.psf_fit_moments(x_ref, y)
    n = int(np.prod(plan.lr_shape))
    det = n * s2 - s1 * s1
    if det <= 0:
        return float("inf"), 1.0, 0.0
    a = (n * c - s1 * t1) / det
    b = (t1 - a * s1) / n
    r = t2 + a * a * s2 + n * b * b - 2 * a * c - 2 * b * t1 + 2 * a * b * s1
    return max(r, 0.0), a, b


def fit_gaussian_psf(plan, x_ref, y, sigma0=(1.0, 1.0, 1.0), bounds=(0.3, 6.0), sweeps: int = 4,
                     tol: float = 1e-4) -> dict:
    """Cyclic golden-section search of sigma (per axis, in log sigma within
    bounds); the support is fixed by the upper bound.  Leaves the fitted PSF in
    the plan.  Returns sigma, gain a, offset b, the residual and the number of
    objective evaluations."""
    dims = plan.dims
    size = support((bounds[1],) * 3, dims)
    sig = [float(v) for v in sigma0]
    evals = 0
    gr = (math.sqrt(5.0) - 1.0) / 2.0

    def f(s):
        nonlocal evals
        evals += 1
        return objective(plan, x_ref, y, s, size)[0]

    lo0, hi0 = math.log(bounds[0]), math.log(bounds[1])
    for _ in range(sweeps):
        moved = 0.0
        for ax in range(3):
            lo, hi = lo0, hi0
            def g(t):
                s = list(sig)
                s[ax] = math.exp(t)
                return f(s)
            c = hi - gr * (hi - lo)
            d = lo + gr * (hi - lo)
            fc, fd = g(c), g(d)
            while hi - lo > tol:
                if fc < fd:
                    hi, d, fd = d, c, fc
                    c = hi - gr * (hi - lo)
                    fc = g(c)
                else:
                    lo, c, fc = c, d, fd
                    d = lo + gr * (hi - lo)
                    fd = g(d)
            new = math.exp(0.5 * (lo + hi))
            moved = max(moved, abs(math.log(new) - math.log(sig[ax])))
            sig[ax] = new
        if moved < 10 * tol:
            break
    r, a, b = objective(plan, x_ref, y, sig, size)
    return {"sigma": tuple(sig), "gain": a, "offset": b, "residual": r, "evaluations": evals + 1, "size": size}
