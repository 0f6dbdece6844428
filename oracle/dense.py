"""Dense-matrix and independent solvers that pin the FP64 oracle on tiny volumes.

TEST INFRASTRUCTURE ONLY (same rule as sr3d_oracle: imported by tests and by
the committed script that writes tests/golden/, never by the CUDA library).

Everything here avoids the FFT: H is built tap by tap as a circulant
convolution matrix, D as a row selection, L as explicit periodic differences.
The dense normal equations of eq. (6) and of the ADMM x-subproblem
(Sec. III-B) are then solved with numpy.linalg, and the TV problem is solved a
second, independent way by Chambolle-Pock primal-dual iterations.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _flat(shape, i, j, k):
    s, n, m = shape
    return ((i % s) * n + (j % n)) * m + (k % m)


def blur_matrix(psf: np.ndarray, shape) -> np.ndarray:
    """Circulant H of eq. (1): (Hx)[i] = sum_t psf[t] x[i - (t - centre)], periodic."""
    s, n, m = shape
    nh = s * n * m
    ps, pn, pm = psf.shape
    cs, cn, cm = ps // 2, pn // 2, pm // 2
    H = np.zeros((nh, nh))
    ii, jj, kk = np.meshgrid(np.arange(s), np.arange(n), np.arange(m), indexing="ij")
    rows = _flat(shape, ii, jj, kk).ravel()
    for a in range(ps):
        for b in range(pn):
            for c in range(pm):
                cols = _flat(shape, ii - (a - cs), jj - (b - cn), kk - (c - cm)).ravel()
                np.add.at(H, (rows, cols), psf[a, b, c])
    return H


def decimation_matrix(shape, dec) -> np.ndarray:
    """D: keeps voxel (ds*i, dc*j, dr*k) of the HR volume as LR voxel (i, j, k)."""
    s, n, m = shape
    dr, dc, ds = dec
    sl, nl, ml = s // ds, n // dc, m // dr
    D = np.zeros((sl * nl * ml, s * n * m))
    r = 0
    for i in range(sl):
        for j in range(nl):
            for k in range(ml):
                D[r, _flat(shape, ds * i, dc * j, dr * k)] = 1.0
                r += 1
    return D


def grad_matrix(shape) -> np.ndarray:
    """L = [D_m; D_n; D_s] with periodic forward differences, (3 N_h) x N_h."""
    s, n, m = shape
    nh = s * n * m
    L = np.zeros((3 * nh, nh))
    for i in range(s):
        for j in range(n):
            for k in range(m):
                r = _flat(shape, i, j, k)
                for a, (di, dj, dk) in enumerate(((0, 0, 1), (0, 1, 0), (1, 0, 0))):
                    L[a * nh + r, _flat(shape, i + di, j + dj, k + dk)] += 1.0
                    L[a * nh + r, r] -= 1.0
    return L


def tikhonov_dense(y, psf, dec, tau, xbar=None):
    """Solve (H^T D^T D H + tau I) x = H^T D^T y + tau xbar (eq. 6, tau = 2 lambda)."""
    dr, dc, ds = dec
    shape = (y.shape[0] * ds, y.shape[1] * dc, y.shape[2] * dr)
    A = decimation_matrix(shape, dec) @ blur_matrix(psf, shape)
    rhs = A.T @ y.ravel()
    if xbar is not None:
        rhs = rhs + tau * xbar.ravel()
    M = A.T @ A + tau * np.eye(A.shape[1])
    return np.linalg.solve(M, rhs).reshape(shape), M, rhs


def admm_xstep_dense(y, psf, dec, mu, rho, shape):
    """Solve (H^T D^T D H + mu L^T L) x = H^T D^T y + mu L^T rho, the ADMM x-subproblem
    (Sec. III-B) with rho = u - d of shape (3,) + shape."""
    A = decimation_matrix(shape, dec) @ blur_matrix(psf, shape)
    L = grad_matrix(shape)
    M = A.T @ A + mu * (L.T @ L)
    rhs = A.T @ y.ravel() + mu * (L.T @ rho.reshape(-1))
    return np.linalg.solve(M, rhs).reshape(shape), M, rhs


def tikhonov_grad_dense(y, psf, dec, tau):
    """Solve (H^T D^T D H + tau L^T L) x = H^T D^T y (Tikhonov on the gradient)."""
    dr, dc, ds = dec
    shape = (y.shape[0] * ds, y.shape[1] * dc, y.shape[2] * dr)
    A = decimation_matrix(shape, dec) @ blur_matrix(psf, shape)
    L = grad_matrix(shape)
    M = A.T @ A + tau * (L.T @ L)
    return np.linalg.solve(M, A.T @ y.ravel()).reshape(shape), M


def tv_objective_dense(x, y, A, L, lam_tv, aniso=False):
    g = (L @ x.ravel()).reshape(3, -1)
    r = y.ravel() - A @ x.ravel()
    tv = np.abs(g).sum() if aniso else np.sqrt((g ** 2).sum(axis=0)).sum()
    return 0.5 * float(r @ r) + lam_tv * float(tv)


def chambolle_pock_tv(y, psf, dec, lam_tv, shape, iters=20000, x0=None, aniso=False):
    """Independent solver for min_x 1/2||y - DHx||^2 + lambda sum_j ||(Lx)_j||:
    primal-dual hybrid gradient (Chambolle & Pock 2011) with K = [DH; L], G = 0,
    F(z1, z2) = 1/2||z1 - y||^2 + lambda ||z2||_{2,1}; every prox is closed form.
    aniso=True: lambda ||z2||_1 (the dual projection clips each component)."""
    A = decimation_matrix(shape, dec) @ blur_matrix(psf, shape)
    L = grad_matrix(shape)
    K = np.vstack([A, L])
    knorm2 = float(np.linalg.eigvalsh(K.T @ K).max())
    sig = tau = 0.99 / np.sqrt(knorm2)
    nl = A.shape[0]
    nh = A.shape[1]
    yv = y.ravel()
    x = np.zeros(nh) if x0 is None else np.array(x0, dtype=np.float64).ravel()
    xb = x.copy()
    p = np.zeros(K.shape[0])
    for _ in range(iters):
        p = p + sig * (K @ xb)
        p[:nl] = (p[:nl] - sig * yv) / (1.0 + sig)
        q = p[nl:].reshape(3, nh)
        if aniso:
            q = np.clip(q, -lam_tv, lam_tv)
        else:
            nrm = np.sqrt((q ** 2).sum(axis=0))
            q /= np.maximum(1.0, nrm / lam_tv)[None]
        p[nl:] = q.ravel()
        xn = x - tau * (K.T @ p)
        xb = 2.0 * xn - x
        x = xn
    return x.reshape(shape), tv_objective_dense(x, y, A, L, lam_tv, aniso)


# ---------------------------------------------------------------------------
# exact rational arithmetic (writes the hand-checkable fixtures in tests/golden)
# ---------------------------------------------------------------------------

def _solve_fraction(M, b):
    n = len(b)
    A = [row[:] + [b[i]] for i, row in enumerate(M)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        pv = A[c][c]
        A[c] = [v / pv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [vr - f * vc for vr, vc in zip(A[r], A[c])]
    return [A[i][n] for i in range(n)]


def tikhonov_exact(y, psf, dec, tau, xbar=None):
    """eq. (6) solved in exact rational arithmetic; y, psf, tau, xbar hold Fractions/ints.

    y: nested lists [s][n][m]; psf: nested lists [p_s][p_n][p_m].  Returns a flat
    list of Fractions in (s, n, m) C order.
    """
    dr, dc, ds = dec
    sl, nl, ml = len(y), len(y[0]), len(y[0][0])
    shape = (sl * ds, nl * dc, ml * dr)
    s, n, m = shape
    nh = s * n * m
    ps, pn, pm = len(psf), len(psf[0]), len(psf[0][0])
    H = [[Fraction(0)] * nh for _ in range(nh)]
    for i in range(s):
        for j in range(n):
            for k in range(m):
                r = _flat(shape, i, j, k)
                for a in range(ps):
                    for b in range(pn):
                        for c in range(pm):
                            col = _flat(shape, i - (a - ps // 2), j - (b - pn // 2), k - (c - pm // 2))
                            H[r][col] += Fraction(psf[a][b][c])
    rows = [_flat(shape, ds * i, dc * j, dr * k) for i in range(sl) for j in range(nl) for k in range(ml)]
    A = [H[r] for r in rows]
    yv = [Fraction(y[i][j][k]) for i in range(sl) for j in range(nl) for k in range(ml)]
    tau = Fraction(tau)
    M = [[sum((A[q][a] * A[q][b] for q in range(len(A))), Fraction(0)) + (tau if a == b else 0)
          for b in range(nh)] for a in range(nh)]
    rhs = [sum((A[q][a] * yv[q] for q in range(len(A))), Fraction(0)) for a in range(nh)]
    if xbar is not None:
        xv = [Fraction(v) for v in np.asarray(xbar, dtype=object).ravel()]
        rhs = [r + tau * v for r, v in zip(rhs, xv)]
    return _solve_fraction(M, rhs)
