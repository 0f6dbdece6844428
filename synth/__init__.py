"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the super-resolution method itself: it draws
random numbers and builds the inputs the method consumes (a ground-truth
phantom, Gaussian PSF taps, standard-normal noise fields and the noise scale
that gives a requested SNR).  Applying the degradation model y = DHx + n
(Sec. II-A, eq. 1) is left to the caller, which uses either the oracle or the
CUDA library for it.

The phantoms stand in for the dental micro-CT / CBCT tooth volumes the paper
measures on (Sec. IV), which are not available: piecewise-constant random
ellipsoids, optionally with a smooth periodic low-frequency field.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value i of stream k under seed s is mix64(s * 2^32 + k * 2^52 + (i + 1) * gamma)
so every draw is addressable and reproducible on any machine.  Normals use the
Box-Muller transform.

Array layout everywhere: a volume with HR sizes (m, n, s) is a C-ordered numpy
array of shape (s, n, m) -- m is the fastest (contiguous) axis.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n raw 64-bit draws of stream `stream` under `seed`, starting at counter `offset`."""
    base = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) + (np.uint64(stream & 0xFFF) << np.uint64(52))
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(base + i * _GAMMA)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in [0, 1) with 53-bit resolution."""
    return (splitmix64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller over pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


# ---------------------------------------------------------------------------
# phantom
# ---------------------------------------------------------------------------

def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def ellipsoid_phantom(dims: Tuple[int, int, int], n_ellipsoids: int, seed: int,
                      field_amplitude: float = 0.0) -> np.ndarray:
    """Piecewise-constant phantom of random rotated ellipsoids, shape (s, n, m), float64.

    dims = (m, n, s).  Each ellipsoid has centre U[0,1)^3 * dims, semi-axes
    U[0.05, 0.25] * min(dims), a uniformly random rotation (normalised Gaussian
    quaternion) and value U[0, 1); ellipsoids are painted in order, later ones
    overwrite earlier ones, on a background of 0.  With field_amplitude > 0 a
    smooth field (four periodic cosines of integer frequency <= 2 cycles per
    axis, random phase) scaled to max |field| = field_amplitude is added.
    """
    m, n, s = dims
    vol = np.zeros((s, n, m), dtype=np.float64)
    per = 3 + 3 + 4 + 1  # centre, semi-axes, quaternion (normal), value
    u = uniform(seed, 0, n_ellipsoids * per)
    g = normal(seed, 1, n_ellipsoids * 4)
    dmin = float(min(dims))
    for e in range(n_ellipsoids):
        p = u[e * per:(e + 1) * per]
        c = np.array([p[0] * m, p[1] * n, p[2] * s])
        ax = (0.05 + 0.20 * p[3:6]) * dmin
        rot = _quat_to_rot(g[4 * e:4 * e + 4])
        val = p[10]
        r = float(ax.max())
        lo = np.maximum(np.floor(c - r).astype(int), 0)
        hi = np.minimum(np.ceil(c + r).astype(int) + 1, np.array([m, n, s]))
        if np.any(hi <= lo):
            continue
        zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]),
                                 np.arange(lo[0], hi[0]), indexing="ij")
        rel = np.stack([xx - c[0], yy - c[1], zz - c[2]], axis=-1) @ rot  # body frame
        inside = ((rel / ax) ** 2).sum(axis=-1) <= 1.0
        sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[inside] = val
    if field_amplitude > 0.0:
        uf = uniform(seed, 2, 4 * 4)
        zz = np.arange(s)[:, None, None] / s
        yy = np.arange(n)[None, :, None] / n
        xx = np.arange(m)[None, None, :] / m
        field = np.zeros_like(vol)
        for k in range(4):
            f = np.floor(uf[4 * k:4 * k + 3] * 5.0) - 2.0  # integer frequency in {-2..2}
            ph = 2.0 * np.pi * uf[4 * k + 3]
            field += np.cos(2.0 * np.pi * (f[0] * xx + f[1] * yy + f[2] * zz) + ph)
        mx = np.abs(field).max()
        if mx > 0:
            vol += field * (field_amplitude / mx)
    return vol


# ---------------------------------------------------------------------------
# PSF and noise
# ---------------------------------------------------------------------------

def gaussian_psf(sigma: Tuple[float, float, float],
                 size: Optional[Tuple[int, int, int]] = None) -> np.ndarray:
    """Separable Gaussian taps, shape (p_s, p_n, p_m), centre at floor(p/2), sum 1.

    sigma = (sigma_m, sigma_n, sigma_s); size = (p_m, p_n, p_s), default
    2*ceil(3*sigma)+1 per axis.  The taps are normalised after truncation.
    """
    if size is None:
        size = tuple(2 * int(math.ceil(3.0 * sg)) + 1 for sg in sigma)
    axes = []
    for sg, p in zip(sigma, size):
        i = np.arange(p) - (p // 2)
        axes.append(np.exp(-(i * i) / (2.0 * sg * sg)))
    h = axes[2][:, None, None] * axes[1][None, :, None] * axes[0][None, None, :]
    return h / h.sum()


def noise_sigma(clean_lr: np.ndarray, snr_db: float) -> float:
    """Noise standard deviation giving `snr_db` against the noiseless LR volume:
    sigma^2 = var(clean) * 10^(-snr/10) (population variance)."""
    return float(math.sqrt(np.var(np.asarray(clean_lr, dtype=np.float64)) * 10.0 ** (-snr_db / 10.0)))


def noise_field(shape: Tuple[int, ...], seed: int) -> np.ndarray:
    """Standard-normal field of the given array shape (stream 3 of `seed`)."""
    return normal(seed, 3, int(np.prod(shape))).reshape(shape)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic super-resolution problem: sizes, PSF, noise and solver parameters."""
    name: str
    dims: Tuple[int, int, int]          # HR (m, n, s)
    dec: Tuple[int, int, int]           # (dr, dc, ds)
    sigma: Tuple[float, float, float]   # PSF sigma per axis (m, n, s)
    n_ellipsoids: int
    field: float
    snr_db: float
    tau: float                          # Tikhonov weight (tau = 2*lambda of eq. 5)
    lam: float                          # TV weight
    mu: float                           # ADMM penalty
    iters: int
    seed: int
    dtype: str = "f32"
    psf_size: Optional[Tuple[int, int, int]] = None

    @property
    def lr_dims(self) -> Tuple[int, int, int]:
        return tuple(a // b for a, b in zip(self.dims, self.dec))

    @property
    def voxels(self) -> int:
        return int(np.prod(self.dims))

    def psf(self) -> np.ndarray:
        return gaussian_psf(self.sigma, self.psf_size)

    def phantom(self) -> np.ndarray:
        return ellipsoid_phantom(self.dims, self.n_ellipsoids, self.seed, self.field)

    def noise(self) -> np.ndarray:
        m, n, s = self.lr_dims
        return noise_field((s, n, m), self.seed)


# The five workloads: 32^3 FP64, 256^3 FP32 (headline), the anisotropic
# 512x512x256 CBCT-like volume, and the ingredients of the batched and
# learned-warm-start workloads.
SMALL_FP64 = Workload("hr32_d2_fp64", (32, 32, 32), (2, 2, 2), (1.0, 1.0, 1.0), 12, 0.0, 40.0,
                      1e-2, 1e-3, 1e-2, 20, 1001, "f64")
HEADLINE_256 = Workload("hr256_d2_fp32", (256, 256, 256), (2, 2, 2), (1.5, 1.5, 1.5), 200, 0.1, 40.0,
                        1e-2, 5e-4, 1e-2, 100, 1002, "f32")
ANISO_512 = Workload("hr512x512x256_d114_fp32", (512, 512, 256), (1, 1, 4), (1.0, 1.0, 2.0), 500, 0.0, 35.0,
                     5e-3, 5e-4, 1e-2, 200, 1003, "f32")

BATCH_SIZES = ((64, 64, 64), (96, 96, 64), (128, 128, 128), (128, 128, 96))
BATCH_DECS = ((2, 2, 2), (2, 2, 1), (1, 1, 4))


def batch_workloads(count: int = 64, seed: int = 1004, iters: int = 50) -> list:
    """The ragged batch: sizes and decimations uniform over the sets above,
    tau log-uniform in [1e-3, 1e-1], isotropic sigma U[0.8, 2]; volume i uses seed + i."""
    u = uniform(seed, 7, 4 * count)
    out = []
    for i in range(count):
        dims = BATCH_SIZES[int(u[4 * i] * len(BATCH_SIZES))]
        dec = BATCH_DECS[int(u[4 * i + 1] * len(BATCH_DECS))]
        tau = 10.0 ** (-3.0 + 2.0 * u[4 * i + 2])
        sg = 0.8 + 1.2 * u[4 * i + 3]
        out.append(Workload(f"batch{i}", dims, dec, (sg, sg, sg), 40, 0.0, 40.0,
                            tau, 5e-4, 1e-2, iters, seed + i, "f32"))
    return out


def scaled(w: Workload, dims: Tuple[int, int, int], name: Optional[str] = None, **kw) -> Workload:
    """Same recipe at other sizes (used for small parity cases)."""
    return dataclasses.replace(w, name=name or f"{w.name}@{dims}", dims=dims, **kw)
