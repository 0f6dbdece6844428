"""Writes the sampled FP64 oracle iterates of the two long ADMM-TV runs used by
the GPU parity tests (tests/test_gpu_long_runs.py).

The oracle needs minutes per run at these sizes, too long for a test, so this
script runs it once and stores, for a seeded sample of HR voxels, the iterate
x^k of Algorithm 1 (Sec. III-B) at a few iteration counts k, together with the
full-volume norm ||x^k|| and the objective 1/2||y - DHx^k||^2 + lambda TV(x^k).
It calls only oracle/ (the method) and synth/ (seeded inputs):

  hr256_d2: the 256^3 benchmark workload (200 ellipsoids + field, Gaussian
            PSF sigma 1.5 on 11^3 taps, d = 2x2x2, 40 dB), Tikhonov start
            (tau 1e-2, nearest-neighbour prior), 100 iterations, lambda 5e-4,
            mu 1e-2; samples at k = 0 (the start), 1, 2, 5, 10, 25, 50, 100.
  aniso512x512x32_d114: the anisotropic CBCT-like recipe (500 ellipsoids,
            sigma (1, 1, 2) on 7x7x13 taps, d = 1x1x4, 35 dB, tau 5e-3) with
            the s extent cut from 256 to 32 so that the oracle finishes, which
            keeps the 512-point transforms along m and n; 200 iterations,
            lambda 5e-4, mu 1e-2; samples at k = 0, 1, 2, 5, 10, 50, 100, 200.

Run from the repository root:  python tests/golden/make_long_runs.py [name ...]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle as O  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SAMPLES = 4096
SAMPLE_STREAM = 9  # synth stream of the sampled voxel indices


def workloads():
    """name -> (workload, iteration counts to record)."""
    aniso = synth.scaled(synth.ANISO_512, (512, 512, 32), name="aniso512x512x32_d114")
    return {
        "hr256_d2": (synth.HEADLINE_256, (1, 2, 5, 10, 25, 50, 100)),
        "aniso512x512x32_d114": (aniso, (1, 2, 5, 10, 50, 100, 200)),
    }


def problem(w):
    """Seeded phantom, PSF and y = DHx + n by the oracle's forward model."""
    psf = w.psf()
    x = w.phantom()
    clean = O.forward(x, psf, w.dec)
    y = clean + synth.noise_sigma(clean, w.snr_db) * w.noise()
    return psf, y


def sample_indices(w):
    return np.floor(synth.uniform(w.seed, SAMPLE_STREAM, SAMPLES) * w.voxels).astype(np.int64)


def run(name, w, ks):
    t0 = time.time()
    psf, y = problem(w)
    idx = sample_indices(w)
    x0 = O.tikhonov(y, psf, w.dec, w.tau, O.nearest_neighbour(y, w.dec))
    rec = {0: (x0.ravel()[idx].copy(), float(np.linalg.norm(x0)), O.objective(x0, y, psf, w.dec, w.lam))}

    def cb(i, xi, u, d):
        k = i + 1
        if k in ks:
            rec[k] = (xi.ravel()[idx].copy(), float(np.linalg.norm(xi)), O.objective(xi, y, psf, w.dec, w.lam))
            print(f"{name}: k = {k}  {time.time() - t0:.0f} s", flush=True)

    O.admm_tv(y, psf, w.dec, w.lam, w.mu, max(ks), x0, callback=cb)
    order = [0] + list(ks)
    np.savez_compressed(
        os.path.join(HERE, f"admm_{name}.npz"),
        dims=np.array(w.dims), dec=np.array(w.dec), tau=w.tau, lam=w.lam, mu=w.mu, seed=w.seed,
        ks=np.array(order), idx=idx, x=np.stack([rec[k][0] for k in order]),
        norm=np.array([rec[k][1] for k in order]), objective=np.array([rec[k][2] for k in order]))
    print(f"{name}: written in {time.time() - t0:.0f} s", flush=True)


def main():
    names = sys.argv[1:] or list(workloads())
    for name in names:
        w, ks = workloads()[name]
        run(name, w, ks)


if __name__ == "__main__":
    main()
