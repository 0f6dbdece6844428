"""Writes the exact-rational Tikhonov fixtures in this folder.

Each case is the normal-equation solve of eq. (6) of the paper (Sec. III-A),
(H^T D^T D H + tau I) x = H^T D^T y + tau xbar, carried out in exact rational
arithmetic by oracle.dense.tikhonov_exact (dense circulant H built tap by tap,
no FFT).  Run from the repository root:  python tests/golden/make_golden.py
"""
from fractions import Fraction as Fr
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.dense import tikhonov_exact  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    # 1-D along m: HR 8 -> LR 4 (dr = 2), symmetric 3-tap PSF, zero prior.
    "tik_1d_m8_d2": dict(
        y=[[[Fr(1), Fr(2), Fr(0), Fr(-1)]]],
        psf=[[[Fr(1, 4), Fr(1, 2), Fr(1, 4)]]],
        dec=(2, 1, 1), tau=Fr(1, 2), xbar=None),
    # 3-D: HR (m, n, s) = (4, 4, 2) -> LR (2, 2, 2) with d = 2x2x1, an asymmetric
    # 3x3x1 PSF (pins conj(Lambda) against Lambda) and a non-zero prior.
    "tik_3d_4x4x2_d221_asym": dict(
        y=[[[Fr(1), Fr(-2)], [Fr(3), Fr(0)]], [[Fr(2), Fr(1)], [Fr(-1), Fr(4)]]],
        psf=[[[Fr(1, 14), Fr(2, 14), Fr(0)], [Fr(3, 14), Fr(4, 14), Fr(1, 14)], [Fr(0), Fr(1, 14), Fr(2, 14)]]],
        dec=(2, 2, 1), tau=Fr(1, 3),
        xbar=[[[Fr((i * 7 + j * 3 + k) % 5 - 2, 3) for k in range(4)] for j in range(4)] for i in range(2)]),
}


def fmt(v):
    return " ".join(f"{q.numerator}/{q.denominator}" for q in v)


def main():
    for name, c in CASES.items():
        x = tikhonov_exact(c["y"], c["psf"], c["dec"], c["tau"], c["xbar"])
        y = [q for a in c["y"] for b in a for q in b]
        psf = [q for a in c["psf"] for b in a for q in b]
        sl, nl, ml = len(c["y"]), len(c["y"][0]), len(c["y"][0][0])
        ps, pn, pm = len(c["psf"]), len(c["psf"][0]), len(c["psf"][0][0])
        with open(os.path.join(HERE, name + ".txt"), "w") as f:
            f.write(f"# Exact solution of eq. (6), Sec. III-A (tau = 2*lambda); written by make_golden.py\n")
            f.write(f"# arrays are C-ordered (s, n, m); rationals p/q\n")
            f.write(f"lr_shape {sl} {nl} {ml}\n")
            f.write(f"dec {c['dec'][0]} {c['dec'][1]} {c['dec'][2]}\n")
            f.write(f"psf_shape {ps} {pn} {pm}\n")
            f.write(f"tau {c['tau'].numerator}/{c['tau'].denominator}\n")
            f.write(f"y {fmt(y)}\n")
            f.write(f"psf {fmt(psf)}\n")
            if c["xbar"] is not None:
                xb = [q for a in c["xbar"] for b in a for q in b]
                f.write(f"xbar {fmt(xb)}\n")
            f.write(f"x {fmt(x)}\n")


if __name__ == "__main__":
    main()
