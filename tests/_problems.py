"""Seeded test problems shared by the parity tests (inputs only; expected
values always come from the oracle)."""
import numpy as np

import oracle as O
from synth import ellipsoid_phantom, gaussian_psf, noise_field, noise_sigma


def make_problem(dims, dec, sigma=(1.0, 1.0, 1.0), n_ell=8, seed=7, snr_db=40.0, field=0.0, psf_size=None,
                 asym=False):
    """HR phantom, PSF and noisy LR observation y = DHx + n (oracle forward model, FP64).
    The PSF support is 2*ceil(3 sigma)+1 per axis, clipped to the volume (odd)."""
    if psf_size is None:
        psf_size = tuple(min(2 * int(np.ceil(3.0 * sg)) + 1, dm - (1 - dm % 2)) for sg, dm in zip(sigma, dims))
    psf = gaussian_psf(sigma, psf_size)
    if asym:  # break the PSF symmetry so that conj(Lambda) != Lambda
        psf = psf * (1.0 + 0.3 * np.linspace(0, 1, psf.size).reshape(psf.shape))
        psf = psf / psf.sum()
    x = ellipsoid_phantom(dims, n_ell, seed, field)
    clean = O.forward(x, psf, dec)
    y = clean + noise_sigma(clean, snr_db) * noise_field(clean.shape, seed)
    return psf, x, y


REPORT = {}


def rel_l2(a, b, name=None):
    """Relative L2 distance ||a - b|| / ||b|| (complex-aware); recorded under `name`."""
    a = np.asarray(a)
    b = np.asarray(b)
    a = a.astype(np.complex128) if np.iscomplexobj(a) or np.iscomplexobj(b) else a.astype(np.float64)
    b = b.astype(a.dtype)
    err = float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
    if name is not None:
        REPORT[name] = err
    return err
