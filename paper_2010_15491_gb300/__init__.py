"""GB300-native fast 3D single-image super-resolution (Tuador et al., arXiv:2010.15491).

Thin Python binding of the C-ABI library libsr3d.so (include/sr3d.h).  It only
marshals arguments: every step of the method runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors (PyTorch provides device memory
and streams); layouts follow the header: a volume with HR sizes (m, n, s) is a
contiguous tensor of shape (s, n, m), the ADMM dual d has shape (3, s, n, m).

Importing the package does not load the library; the first call does, and it
raises if libsr3d.so has not been built (paper_2010_15491_gb300.build.build()).
There is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsr3d.so")

SR3D_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "NOT_DIVISIBLE", -3: "UNSUPPORTED_SIZE", -4: "SINGULAR", -5: "CUDA",
    -6: "OOM", -7: "TIMEOUT", -8: "NUMERIC", -9: "NOT_CONVERGED",
}
XBAR_NEAREST = ctypes.c_void_p(1)

EXPORTED = [
    "sr3d_plan", "sr3d_destroy", "sr3d_forward", "sr3d_tikhonov", "sr3d_admm_tv", "sr3d_admm_tv_host",
    "sr3d_last_error", "sr3d_get_otf", "sr3d_fft3", "sr3d_xstep", "sr3d_tv_step", "sr3d_plan_info",
    "sr3d_profile", "sr3d_profile_read", "sr3d_tikhonov_noalloc", "sr3d_admm_tv_batched", "sr3d_autotune",
    "sr3d_schedule",
    "sr3d_separable", "sr3d_set_tv", "sr3d_tikhonov_grad", "sr3d_tikhonov_cg", "sr3d_set_psf",
    "sr3d_dual_init", "sr3d_unet_param_count", "sr3d_unet_create", "sr3d_unet_destroy", "sr3d_unet_set_params",
    "sr3d_unet_get_params", "sr3d_unet_forward", "sr3d_unet_train_step", "sr3d_unet_read", "sr3d_unet_set_path",
    "sr3d_set_plan_memory_limit", "sr3d_unet_wait_selftest", "sr3d_psf_fit_moments",
]
KINDS = ["tv", "rfft_m_fwd", "fft_n_fwd", "fft_s", "fft_n_inv", "rfft_m_inv", "other", "setup"]


class Sr3dError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class Desc(ctypes.Structure):
    _fields_ = [("m_h", ctypes.c_int), ("n_h", ctypes.c_int), ("s_h", ctypes.c_int),
                ("dr", ctypes.c_int), ("dc", ctypes.c_int), ("ds", ctypes.c_int),
                ("psf", ctypes.POINTER(ctypes.c_double)),
                ("p_m", ctypes.c_int), ("p_n", ctypes.c_int), ("p_s", ctypes.c_int),
                ("dtype", ctypes.c_int), ("stream", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("eval_every", ctypes.c_int), ("objective_hist", ctypes.POINTER(ctypes.c_double)),
                ("hist_len", ctypes.c_int), ("iters", ctypes.c_int), ("evals", ctypes.c_int),
                ("objective", ctypes.c_double), ("data_term", ctypes.c_double), ("tv_term", ctypes.c_double),
                ("primal", ctypes.c_double), ("dual", ctypes.c_double),
                ("primal_rel", ctypes.c_double), ("dual_rel", ctypes.c_double)]


_lib = None


def load() -> ctypes.CDLL:
    """Loads libsr3d.so once; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: run paper_2010_15491_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "sr3d_plan": (i, [ctypes.POINTER(vp), ctypes.POINTER(Desc)]),
        "sr3d_destroy": (i, [vp]),
        "sr3d_forward": (i, [vp, vp, vp]),
        "sr3d_tikhonov": (i, [vp, vp, vp, d, vp]),
        "sr3d_admm_tv": (i, [vp, vp, vp, vp, d, d, i, d, d, ctypes.POINTER(Stats)]),
        "sr3d_admm_tv_host": (i, [vp, vp, vp, d, d, i, d, d, ctypes.POINTER(Stats)]),
        "sr3d_last_error": (ctypes.c_char_p, []),
        "sr3d_get_otf": (i, [vp, vp]),
        "sr3d_fft3": (i, [vp, vp, vp]),
        "sr3d_xstep": (i, [vp, vp, vp, d, vp]),
        "sr3d_tv_step": (i, [vp, vp, vp, vp, d, d, vp]),
        "sr3d_plan_info": (i, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]),
        "sr3d_profile": (i, [vp, i]),
        "sr3d_profile_read": (i, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
        "sr3d_tikhonov_noalloc": (i, [ctypes.POINTER(Desc), vp, vp, d, vp]),
        "sr3d_autotune": (i, [vp, i]),
        "sr3d_schedule": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "sr3d_admm_tv_batched": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d), i]),
        "sr3d_dual_init": (i, [vp, vp, d, d, vp]),
        "sr3d_separable": (i, [vp, i, ctypes.POINTER(i)]),
        "sr3d_set_tv": (i, [vp, i]),
        "sr3d_set_psf": (i, [vp, ctypes.POINTER(d), i, i, i]),
        "sr3d_tikhonov_grad": (i, [vp, vp, d, vp]),
        "sr3d_tikhonov_cg": (i, [vp, vp, vp, d, d, i, vp, ctypes.POINTER(i), ctypes.POINTER(d)]),
        "sr3d_unet_param_count": (ctypes.c_longlong, []),
        "sr3d_unet_create": (i, [ctypes.POINTER(vp), vp]),
        "sr3d_unet_destroy": (i, [vp]),
        "sr3d_unet_set_params": (i, [vp, vp, ctypes.c_longlong]),
        "sr3d_unet_get_params": (i, [vp, vp, ctypes.c_longlong]),
        "sr3d_unet_forward": (i, [vp, i, i, i, vp, vp]),
        "sr3d_unet_train_step": (i, [vp, i, i, i, vp, vp, d, ctypes.POINTER(d), vp, i]),
        "sr3d_unet_read": (i, [vp, i, vp, ctypes.c_longlong]),
        "sr3d_unet_set_path": (i, [vp, i]),
        "sr3d_set_plan_memory_limit": (i, [ctypes.c_longlong]),
        "sr3d_unet_wait_selftest": (i, [vp, ctypes.c_longlong]),
        "sr3d_psf_fit_moments": (i, [vp, vp, vp, ctypes.POINTER(d)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc: int, allow=()):
    if rc != SR3D_OK and rc not in allow:
        raise Sr3dError(rc, load().sr3d_last_error().decode())
    return rc


def _ptr(t, dtype=None, shape: Optional[Sequence[int]] = None, device: bool = True) -> int:
    """Device (or host) address of a contiguous torch tensor after checks."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if device and not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not device and t.is_cuda:
        raise ValueError("expected a host tensor")
    return t.data_ptr()


class Plan:
    """One problem geometry: HR sizes dims = (m, n, s), decimation dec = (dr, dc, ds),
    PSF taps psf of shape (p_s, p_n, p_m).  dtype "f32" or "f64"."""

    def __init__(self, dims, dec, psf, dtype: str = "f32", stream=None):
        import torch
        self._torch = torch
        L = load()
        psf = np.ascontiguousarray(psf, dtype=np.float64)
        if psf.ndim != 3:
            raise ValueError("psf must be 3-D (p_s, p_n, p_m)")
        self.dims = tuple(int(v) for v in dims)
        self.dec = tuple(int(v) for v in dec)
        self.dtype_name = dtype
        self.tdtype = {"f32": torch.float32, "f64": torch.float64}[dtype]
        m, n, s = self.dims
        dr, dc, ds = self.dec
        self.hr_shape = (s, n, m)
        self.lr_shape = (s // ds, n // dc, m // dr)
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        desc = Desc(m, n, s, dr, dc, ds, psf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    psf.shape[2], psf.shape[1], psf.shape[0], 0 if dtype == "f32" else 1,
                    ctypes.c_void_p(handle) if handle else None)
        self._psf_keep = psf
        h = ctypes.c_void_p()
        _check(L.sr3d_plan(ctypes.byref(h), ctypes.byref(desc)))
        self._h = h

    # -- helpers
    def _hr(self, t):
        return _ptr(t, self.tdtype, self.hr_shape)

    def _lr(self, t):
        return _ptr(t, self.tdtype, self.lr_shape)

    def empty_hr(self):
        return self._torch.empty(self.hr_shape, dtype=self.tdtype, device="cuda")

    def empty_lr(self):
        return self._torch.empty(self.lr_shape, dtype=self.tdtype, device="cuda")

    def info(self):
        sizes = (ctypes.c_int * 9)()
        b = ctypes.c_longlong()
        _check(load().sr3d_plan_info(self._h, sizes, ctypes.byref(b)))
        keys = ["m_h", "n_h", "s_h", "m_l", "n_l", "s_l", "m_slots", "m_pitch", "dtype"]
        out = dict(zip(keys, list(sizes)))
        out["bytes"] = b.value
        return out

    def set_psf(self, psf):
        """Replaces the PSF (taps of shape (p_s, p_n, p_m)) and recomputes Lambda (sr3d_set_psf)."""
        psf = np.ascontiguousarray(psf, dtype=np.float64)
        if psf.ndim != 3:
            raise ValueError("psf must be 3-D (p_s, p_n, p_m)")
        _check(load().sr3d_set_psf(self._h, psf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   psf.shape[2], psf.shape[1], psf.shape[0]))
        self._psf_keep = psf

    def set_tv(self, kind: str):
        """TV of admm_tv on this plan: "isotropic" (default) or "anisotropic" (sr3d_set_tv)."""
        _check(load().sr3d_set_tv(self._h, {"isotropic": 0, "anisotropic": 1}[kind]))

    def tikhonov_grad(self, y, tau: float, x=None):
        """argmin 1/2 ||y - DHx||^2 + tau/2 ||Lx||^2 (sr3d_tikhonov_grad)."""
        x = self.empty_hr() if x is None else x
        _check(load().sr3d_tikhonov_grad(self._h, self._lr(y), float(tau), self._hr(x)))
        return x

    def tikhonov_cg(self, y, tau: float, xbar=None, tol: float = 0.0, max_iters: int = 100, x=None):
        """eq. (5) solved iteratively by conjugate gradients (sr3d_tikhonov_cg);
        returns (x, iterations, ||r|| / ||b||, converged)."""
        x = self.empty_hr() if x is None else x
        if isinstance(xbar, str):
            if xbar != "nearest":
                raise ValueError("xbar must be None, 'nearest' or a tensor")
            xb = XBAR_NEAREST
        else:
            xb = self._hr(xbar) if xbar is not None else None
        it = ctypes.c_int()
        rel = ctypes.c_double()
        rc = load().sr3d_tikhonov_cg(self._h, self._lr(y), xb, float(tau), float(tol), int(max_iters),
                                     self._hr(x), ctypes.byref(it), ctypes.byref(rel))
        _check(rc, allow=(-9,))
        return x, it.value, rel.value, rc == SR3D_OK

    def separable(self, use: Optional[bool] = None) -> bool:
        """Separable-PSF fast path (sr3d_separable): enable / disable it, or
        only query with use=None; returns whether it is in use."""
        act = ctypes.c_int()
        _check(load().sr3d_separable(self._h, -1 if use is None else int(bool(use)), ctypes.byref(act)))
        return bool(act.value)

    def autotune(self, reps: int = 10):
        """Times candidate tile schedules (reps launches each) and keeps the
        fastest (cached per geometry)."""
        _check(load().sr3d_autotune(self._h, int(reps)))

    def schedule(self, n_pass_slots: int = 0, s_pass_slots: int = 0, tv_planes: int = 0, m_fwd_lines: int = 0,
                 m_inv_lines: int = 0) -> dict:
        """The tile schedule the plan launches (sr3d_schedule); positive
        arguments first set the n-pass and s-pass tile widths (m-slots per
        CTA), the TV kernel's s planes per CTA and the m passes' lines per CTA."""
        v = (ctypes.c_int * 5)()
        req = (int(n_pass_slots), int(s_pass_slots), int(tv_planes), int(m_fwd_lines), int(m_inv_lines))
        setv = (ctypes.c_int * 5)(*req) if any(r > 0 for r in req) else None
        _check(load().sr3d_schedule(self._h, setv, v))
        return {"n_pass_slots": v[0], "s_pass_slots": v[1], "tv_planes": v[2], "m_fwd_lines": v[3],
                "m_inv_lines": v[4]}

    def profile(self, on: bool = True):
        """Resets the per-kernel accounting; with on=True also times every launch."""
        _check(load().sr3d_profile(self._h, 1 if on else 0))

    def profile_read(self):
        """{kind: (milliseconds, launches)} since the last profile() call."""
        ms = (ctypes.c_double * len(KINDS))()
        n = (ctypes.c_longlong * len(KINDS))()
        _check(load().sr3d_profile_read(self._h, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(KINDS)}

    # -- entry points
    def forward(self, x, y=None):
        """y = D H x (eq. 1 without noise)."""
        y = self.empty_lr() if y is None else y
        _check(load().sr3d_forward(self._h, self._hr(x), self._lr(y)))
        return y

    def tikhonov(self, y, tau: float, x=None, xbar=None):
        """eq. (12); xbar None (zero prior), "nearest" or an HR tensor."""
        x = self.empty_hr() if x is None else x
        if isinstance(xbar, str):
            if xbar != "nearest":
                raise ValueError("xbar must be None, 'nearest' or a tensor")
            xb = XBAR_NEAREST
        else:
            xb = self._hr(xbar) if xbar is not None else None
        _check(load().sr3d_tikhonov(self._h, self._lr(y), xb, float(tau), self._hr(x)))
        return x

    def admm_tv(self, y, x, lam: float, rho: float, iters: int, d=None, tol: float = 0.0,
                tau_init: float = 0.0, eval_every: int = -1, hist_len: int = 0):
        """Algorithm 1.  Returns a dict of statistics when eval_every >= 0 or tol > 0, else None."""
        st, hist = self._stats(eval_every, hist_len, tol)
        dptr = _ptr(d, self.tdtype, (3,) + self.hr_shape) if d is not None else None
        rc = load().sr3d_admm_tv(self._h, self._lr(y), self._hr(x), dptr, float(lam), float(rho), int(iters),
                                 float(tol), float(tau_init), ctypes.byref(st) if st is not None else None)
        _check(rc, allow=(-9,))
        return self._stats_dict(st, hist, rc)

    def admm_tv_host(self, y_host, x_host, lam: float, rho: float, iters: int, tol: float = 0.0,
                     tau_init: float = 0.0, eval_every: int = -1, hist_len: int = 0):
        """Algorithm 1 on host tensors (pinned for asynchronous copies)."""
        st, hist = self._stats(eval_every, hist_len, tol)
        rc = load().sr3d_admm_tv_host(self._h, _ptr(y_host, self.tdtype, self.lr_shape, device=False),
                                      _ptr(x_host, self.tdtype, self.hr_shape, device=False), float(lam),
                                      float(rho), int(iters), float(tol), float(tau_init),
                                      ctypes.byref(st) if st is not None else None)
        _check(rc, allow=(-9,))
        return self._stats_dict(st, hist, rc)

    def psf_fit_moments(self, x, y):
        """(sum yh, sum yh^2, sum y, sum y^2, sum yh y) in FP64 with yh = D H x (sr3d_psf_fit_moments)."""
        m = (ctypes.c_double * 5)()
        _check(load().sr3d_psf_fit_moments(self._h, self._hr(x), self._lr(y), m))
        return tuple(m)

    def get_otf(self):
        """Lambda in natural half-spectrum layout, complex tensor (s, n, m/2+1)."""
        s, n, m = self.hr_shape
        out = self._torch.empty((s, n, m // 2 + 1, 2), dtype=self.tdtype, device="cuda")
        _check(load().sr3d_get_otf(self._h, out.data_ptr()))
        return self._torch.view_as_complex(out)

    def fft3(self, x):
        s, n, m = self.hr_shape
        out = self._torch.empty((s, n, m // 2 + 1, 2), dtype=self.tdtype, device="cuda")
        _check(load().sr3d_fft3(self._h, self._hr(x), out.data_ptr()))
        return self._torch.view_as_complex(out)

    def xstep(self, y, theta, rho: float, x=None):
        x = self.empty_hr() if x is None else x
        _check(load().sr3d_xstep(self._h, self._lr(y), self._hr(theta), float(rho), self._hr(x)))
        return x

    def tv_step(self, x, d_in, lam: float, rho: float, d_out=None, theta=None):
        d_out = self._torch.empty_like(d_in) if d_out is None else d_out
        theta = self.empty_hr() if theta is None else theta
        shp = (3,) + self.hr_shape
        _check(load().sr3d_tv_step(self._h, self._hr(x), _ptr(d_in, self.tdtype, shp),
                                   _ptr(d_out, self.tdtype, shp), float(lam), float(rho), self._hr(theta)))
        return d_out, theta

    def dual_init(self, x, lam: float, rho: float, d=None):
        """KKT-consistent initial dual for ADMM started at x (sr3d_dual_init)."""
        d = self._torch.empty((3,) + self.hr_shape, dtype=self.tdtype, device=x.device) if d is None else d
        _check(load().sr3d_dual_init(self._h, self._hr(x), float(lam), float(rho),
                                     _ptr(d, self.tdtype, (3,) + self.hr_shape)))
        return d

    def close(self):
        if getattr(self, "_h", None):
            load().sr3d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- statistics marshalling
    @staticmethod
    def _stats(eval_every, hist_len, tol):
        if eval_every < 0 and tol <= 0:
            return None, None
        hist = (ctypes.c_double * max(hist_len, 1))()
        st = Stats(max(eval_every, 0), hist if hist_len > 0 else None, hist_len)
        return st, hist

    @staticmethod
    def _stats_dict(st, hist, rc):
        if st is None:
            return None
        out = {k: getattr(st, k) for k in ("iters", "evals", "objective", "data_term", "tv_term", "primal",
                                             "dual", "primal_rel", "dual_rel")}
        out["converged"] = rc == SR3D_OK
        if st.hist_len > 0:
            out["objective_hist"] = [hist[i] for i in range(min(st.evals, st.hist_len))]
        return out


def tikhonov_noalloc(dims, dec, psf, y, tau: float, x, xbar=None, dtype: str = "f32", stream=None):
    """Allocation-free Tikhonov solve (sr3d_tikhonov_noalloc): same result as
    Plan(dims, dec, psf, dtype).tikhonov(y, tau, x, xbar) but all device work
    memory comes from the library's fixed scratch array; y and x are the
    caller's CUDA tensors.  Calls that overlap on the GPU race."""
    import torch
    L = load()
    psf = np.ascontiguousarray(psf, dtype=np.float64)
    m, n, s = (int(v) for v in dims)
    dr, dc, ds = (int(v) for v in dec)
    td = {"f32": torch.float32, "f64": torch.float64}[dtype]
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    desc = Desc(m, n, s, dr, dc, ds, psf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                psf.shape[2], psf.shape[1], psf.shape[0], 0 if dtype == "f32" else 1,
                ctypes.c_void_p(handle) if handle else None)
    if isinstance(xbar, str):
        if xbar != "nearest":
            raise ValueError("xbar must be None, 'nearest' or a tensor")
        xb = XBAR_NEAREST
    else:
        xb = _ptr(xbar, td, (s, n, m)) if xbar is not None else None
    _check(L.sr3d_tikhonov_noalloc(ctypes.byref(desc), _ptr(y, td, (s // ds, n // dc, m // dr)), xb, float(tau),
                                   _ptr(x, td, (s, n, m))))
    return x


def set_plan_memory_limit(nbytes: int):
    """Cap on the device bytes any one plan may hold (sr3d_set_plan_memory_limit; 0 = none)."""
    _check(load().sr3d_set_plan_memory_limit(int(nbytes)))


def admm_tv_batched(plans, ys, xs, lams, rhos, taus, iters: int):
    """sr3d_admm_tv_batched: ADMM-TV on many volumes (one plan each, each plan
    created with its own stream), iterations of all volumes in one CUDA graph."""
    n = len(plans)
    if not (len(ys) == len(xs) == len(lams) == len(rhos) == len(taus) == n):
        raise ValueError("one y, x, lambda, rho and tau per plan")
    vp = ctypes.c_void_p
    P = (vp * n)(*[p._h.value for p in plans])
    Y = (vp * n)(*[p._lr(t) for p, t in zip(plans, ys)])
    X = (vp * n)(*[p._hr(t) for p, t in zip(plans, xs)])
    dd = ctypes.c_double * n
    _check(load().sr3d_admm_tv_batched(n, P, Y, X, dd(*lams), dd(*rhos), dd(*taus), int(iters)))
    return xs


class UNet:
    """The learned warm-start network of the library (sr3d_unet_*): a 3D U-Net
    with channels 16 / 32 / 64 on BF16 tensor-core kernels.  Volumes are FP32
    CUDA tensors of shape (s, n, m), each size a multiple of 4.  A new network
    has all parameters zero (the identity map)."""

    def __init__(self, stream=None):
        import torch
        self._torch = torch
        L = load()
        self.n_params = int(L.sr3d_unet_param_count())
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self._h = ctypes.c_void_p()
        _check(L.sr3d_unet_create(ctypes.byref(self._h), ctypes.c_void_p(handle) if handle else None))

    def _vol(self, t):
        if t.dim() != 3:
            raise ValueError("expected an (s, n, m) volume")
        return _ptr(t, self._torch.float32)

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _check(load().sr3d_unet_set_params(self._h, a.ctypes.data, a.size))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.n_params, dtype=np.float32)
        _check(load().sr3d_unet_get_params(self._h, a.ctypes.data, a.size))
        return a

    def forward(self, x, out=None):
        out = self._torch.empty_like(x) if out is None else out
        s, n, m = x.shape
        _check(load().sr3d_unet_forward(self._h, m, n, s, self._vol(x), self._vol(out)))
        return out

    def train_step(self, x, target, lr: float = 1e-3, update: bool = True, want_grad: bool = False):
        """One step; returns (loss, gradient or None)."""
        s, n, m = x.shape
        if tuple(target.shape) != tuple(x.shape):
            raise ValueError("target must have the shape of x")
        loss = ctypes.c_double()
        g = np.empty(self.n_params, dtype=np.float32) if want_grad else None
        _check(load().sr3d_unet_train_step(self._h, m, n, s, self._vol(x), self._vol(target), float(lr),
                                           ctypes.byref(loss), g.ctypes.data if g is not None else None,
                                           int(bool(update))))
        return loss.value, g

    def set_path(self, path: str):
        """Convolution kernels (sr3d_unet_set_path): "tcgen05" (default: tcgen05 where it is the
        faster kernel), "mma" (mma.sync everywhere) or "tcgen05_all" (tcgen05 wherever it applies)."""
        _check(load().sr3d_unet_set_path(self._h, {"tcgen05": 0, "mma": 1, "tcgen05_all": 2}[path]))

    def wait_selftest(self, limit_cycles: int):
        """Makes the bounded tensor-core wait run out on a barrier nothing
        arrives on (sr3d_unet_wait_selftest); raises Sr3dError TIMEOUT."""
        _check(load().sr3d_unet_wait_selftest(self._h, int(limit_cycles)))

    ACTIVATIONS = ["x", "e1a", "e1", "p1", "e2a", "e2", "p2", "e3a", "e3", "d2a", "d2", "d1a", "d1", "out"]

    def read(self, name: str, shape) -> np.ndarray:
        """An activation of the last forward pass (sr3d_unet_read) as float32
        of shape (s, n, m, channels) at its level ((s, n, m) for x and out)."""
        which = self.ACTIVATIONS.index(name)
        count = int(np.prod(shape))
        if which == 13:
            a = np.empty(count, dtype=np.float32)
            _check(load().sr3d_unet_read(self._h, which, a.ctypes.data, a.nbytes))
            return a.reshape(shape)
        raw = np.empty(count, dtype=np.uint16)
        _check(load().sr3d_unet_read(self._h, which, raw.ctypes.data, raw.nbytes))
        return (raw.astype(np.uint32) << 16).view(np.float32).reshape(shape)

    def close(self):
        if getattr(self, "_h", None):
            load().sr3d_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
