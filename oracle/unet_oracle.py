"""FP64 CPU oracle of the learned warm-start network (a 3D U-Net) and of the
KKT-consistent initial dual used with it.

TEST INFRASTRUCTURE ONLY (same rule as sr3d_oracle).  The paper has no learned
component; this module fixes the network the library implements so that its
forward pass and gradients can be checked:

  volumes are arrays (s, n, m, C) (channels last); zero padding;
  conv3(X; W, b)[v, co] = b[co] + sum_{tap, ci} W[co, tap, ci] X[v + off(tap), ci]
      with tap = (ks*3 + kn)*3 + km and off(tap) = (ks-1, kn-1, km-1) in (s, n, m);
  maxpool: 2x2x2 blocks, the first maximum in (s, n, m) order wins ties;
  up: nearest-neighbour 2x upsampling;
  network (channels 16 / 32 / 64 by default):
    e1a = relu(conv3(x)),        e1 = relu(conv3(e1a))            full size
    e2a = relu(conv3(pool(e1))), e2 = relu(conv3(e2a))            1/2
    e3a = relu(conv3(pool(e2))), e3 = relu(conv3(e3a))            1/4
    d2a = relu(conv3([up(e3), e2])), d2 = relu(conv3(d2a))        1/2
    d1a = relu(conv3([up(d2), e1])), d1 = relu(conv3(d1a))        full size
    out = sum_c w_h[c] d1[..., c] + b_h + x                        (residual head)
  loss = mean((out - target)^2).

Parameters are one flat vector: for each of the ten 3x3x3 layers in the order
above W (co, tap, ci) then b (co); then w_h (C1) and b_h.

Max pooling decides an integer (the argmax) from floating-point values.  A
network that stores its activations in a lower precision takes that decision
on the stored values, so forward() and grad() accept `quant`, a rounding
applied to every stored activation (bf16_round for BF16 storage); the
arithmetic stays FP64 and quant=None is the exact network.
"""
from __future__ import annotations

import numpy as np

def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even) through FP32: the FP32
    bit pattern keeps its upper 16 bits after adding 0x7FFF plus the lowest
    kept bit (finite inputs)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


TAPS = [(ks - 1, kn - 1, km - 1) for ks in range(3) for kn in range(3) for km in range(3)]


def conv3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """3x3x3 convolution (correlation) with zero padding; x (s, n, m, ci), W (co, 27, ci)."""
    s, n, m, ci = x.shape
    xp = np.zeros((s + 2, n + 2, m + 2, ci))
    xp[1:-1, 1:-1, 1:-1] = x
    out = np.zeros((s, n, m, W.shape[0])) + b
    for t, (ds, dn, dm) in enumerate(TAPS):
        sh = xp[1 + ds:1 + ds + s, 1 + dn:1 + dn + n, 1 + dm:1 + dm + m]
        out += sh @ W[:, t, :].T
    return out


def conv3_grads(x: np.ndarray, W: np.ndarray, g: np.ndarray):
    """Gradients of sum(g * conv3(x; W, b)) with respect to x, W and b."""
    s, n, m, ci = x.shape
    xp = np.zeros((s + 2, n + 2, m + 2, ci))
    xp[1:-1, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for t, (ds, dn, dm) in enumerate(TAPS):
        sl = (slice(1 + ds, 1 + ds + s), slice(1 + dn, 1 + dn + n), slice(1 + dm, 1 + dm + m))
        gW[:, t, :] = np.einsum("snmo,snmi->oi", g, xp[sl])
        gxp[sl] += g @ W[:, t, :]
    return gxp[1:-1, 1:-1, 1:-1], gW, g.sum(axis=(0, 1, 2))


def maxpool(x: np.ndarray):
    """2x2x2 max pooling; returns the pooled volume and the argmax (0..7, (s, n, m) order)."""
    s, n, m, c = x.shape
    blocks = x.reshape(s // 2, 2, n // 2, 2, m // 2, 2, c).transpose(0, 2, 4, 1, 3, 5, 6).reshape(
        s // 2, n // 2, m // 2, 8, c)
    idx = blocks.argmax(axis=3)
    return np.take_along_axis(blocks, idx[:, :, :, None, :], axis=3)[:, :, :, 0, :], idx


def unpool(g: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Adjoint of maxpool: each pooled gradient goes to its argmax."""
    s, n, m, c = g.shape
    blocks = np.zeros((s, n, m, 8, c))
    np.put_along_axis(blocks, idx[:, :, :, None, :], g[:, :, :, None, :], axis=3)
    return blocks.reshape(s, n, m, 2, 2, 2, c).transpose(0, 3, 1, 4, 2, 5, 6).reshape(2 * s, 2 * n, 2 * m, c)


def up(x: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(np.repeat(x, 2, axis=0), 2, axis=1), 2, axis=2)


def up_adj(g: np.ndarray) -> np.ndarray:
    s, n, m, c = g.shape
    return g.reshape(s // 2, 2, n // 2, 2, m // 2, 2, c).sum(axis=(1, 3, 5))


def layer_shapes(c=(16, 32, 64)):
    c1, c2, c3 = c
    return [(c1, 1), (c1, c1), (c2, c1), (c2, c2), (c3, c2), (c3, c3), (c2, c3 + c2), (c2, c2), (c1, c2 + c1),
            (c1, c1)]


def param_count(c=(16, 32, 64)) -> int:
    return sum(co * 27 * ci + co for co, ci in layer_shapes(c)) + c[0] + 1


def unpack(theta: np.ndarray, c=(16, 32, 64)):
    layers, o = [], 0
    for co, ci in layer_shapes(c):
        W = theta[o:o + co * 27 * ci].reshape(co, 27, ci)
        o += co * 27 * ci
        b = theta[o:o + co]
        o += co
        layers.append((W, b))
    wh = theta[o:o + c[0]]
    bh = theta[o + c[0]]
    return layers, wh, bh


def forward(theta: np.ndarray, x: np.ndarray, c=(16, 32, 64), keep=False, quant=None):
    """x: (s, n, m) -> out (s, n, m); keep=True also returns the activations.
    quant (optional) rounds every stored activation (see the module notes)."""
    L, wh, bh = unpack(theta, c)
    q = (lambda z: z) if quant is None else quant  # noqa: E731
    relu = lambda z: q(np.maximum(z, 0.0))  # noqa: E731
    a = {"x": q(x)[..., None]}
    a["e1a"] = relu(conv3(a["x"], *L[0]))
    a["e1"] = relu(conv3(a["e1a"], *L[1]))
    a["p1"], a["i1"] = maxpool(a["e1"])
    a["e2a"] = relu(conv3(a["p1"], *L[2]))
    a["e2"] = relu(conv3(a["e2a"], *L[3]))
    a["p2"], a["i2"] = maxpool(a["e2"])
    a["e3a"] = relu(conv3(a["p2"], *L[4]))
    a["e3"] = relu(conv3(a["e3a"], *L[5]))
    a["c2"] = np.concatenate([up(a["e3"]), a["e2"]], axis=-1)
    a["d2a"] = relu(conv3(a["c2"], *L[6]))
    a["d2"] = relu(conv3(a["d2a"], *L[7]))
    a["c1"] = np.concatenate([up(a["d2"]), a["e1"]], axis=-1)
    a["d1a"] = relu(conv3(a["c1"], *L[8]))
    a["d1"] = relu(conv3(a["d1a"], *L[9]))
    out = a["d1"] @ wh + bh + x
    return (out, a) if keep else out


def loss(theta, x, target, c=(16, 32, 64)) -> float:
    return float(((forward(theta, x, c) - target) ** 2).mean())


def grad(theta, x, target, c=(16, 32, 64), quant=None):
    """Loss and its gradient with respect to the flat parameter vector (the
    activations rounded by quant, if given, as in forward)."""
    out, a = forward(theta, x, c, keep=True, quant=quant)
    L, wh, bh = unpack(theta, c)
    r = out - target
    lval = float((r ** 2).mean())
    g_out = 2.0 * r / r.size
    grads = [None] * 10
    g_wh = np.einsum("snmc,snm->c", a["d1"], g_out)
    g_bh = float(g_out.sum())

    def back(i, inp, outp, g):
        g = g * (a[outp] > 0)
        gx, gW, gb = conv3_grads(a[inp], L[i][0], g)
        grads[i] = (gW, gb)
        return gx

    c1, c2, c3 = c
    g = g_out[..., None] * wh
    g = back(9, "d1a", "d1", g)
    g = back(8, "c1", "d1a", g)
    g_e1 = g[..., c2:]
    g = up_adj(g[..., :c2])
    g = back(7, "d2a", "d2", g)
    g = back(6, "c2", "d2a", g)
    g_e2 = g[..., c3:]
    g = up_adj(g[..., :c3])
    g = back(5, "e3a", "e3", g)
    g = back(4, "p2", "e3a", g)
    g = unpool(g, a["i2"]) + g_e2
    g = back(3, "e2a", "e2", g)
    g = back(2, "p1", "e2a", g)
    g = unpool(g, a["i1"]) + g_e1
    g = back(1, "e1a", "e1", g)
    back(0, "x", "e1a", g)
    flat = []
    for gW, gb in grads:
        flat += [gW.ravel(), gb.ravel()]
    flat += [g_wh, np.array([g_bh])]
    return lval, np.concatenate(flat)


def dual_from_x(x: np.ndarray, lam: float, mu: float) -> np.ndarray:
    """KKT-consistent initial dual for ADMM started at x: with g = Lx,
    d_j = (lam/mu) g_j / max(||g_j||, lam/mu), the dual of the u-step at u = shrink(g + d)
    (the scaled dual lies in the ball of radius lam/mu and is aligned with Lx)."""
    from .sr3d_oracle import grad as Lgrad
    g = Lgrad(x)
    t = lam / mu
    nrm = np.sqrt((g ** 2).sum(axis=0))
    return t * g / np.maximum(nrm, t)[None]
