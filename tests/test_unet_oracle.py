"""Pins of the U-Net oracle: the convolution is an explicit sum over taps
(brute force), its gradients are adjoints (dot-product tests), the network
gradient matches central finite differences, and the pooling / upsampling
pairs are adjoint."""
import numpy as np
import pytest

import oracle.unet_oracle as U


def test_conv3_is_the_explicit_sum_over_taps():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5, 2))
    W = rng.standard_normal((3, 27, 2))
    b = rng.standard_normal(3)
    y = U.conv3(x, W, b)
    v = (1, 2, 0)  # a voxel next to the m boundary
    expect = b.copy()
    for t, (ds, dn, dm) in enumerate(U.TAPS):
        q = (v[0] + ds, v[1] + dn, v[2] + dm)
        if all(0 <= q[i] < x.shape[i] for i in range(3)):
            expect += W[:, t, :] @ x[q]
    assert np.allclose(y[v], expect)


def test_conv3_gradients_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 4, 6, 3))
    W = rng.standard_normal((5, 27, 3))
    g = rng.standard_normal((4, 4, 6, 5))
    gx, gW, gb = U.conv3_grads(x, W, g)
    dx = rng.standard_normal(x.shape)
    dW = rng.standard_normal(W.shape)
    zero = np.zeros(5)
    assert np.isclose((g * U.conv3(dx, W, zero)).sum(), (gx * dx).sum())
    assert np.isclose((g * U.conv3(x, dW, zero)).sum(), (gW * dW).sum())
    assert np.allclose(gb, g.sum(axis=(0, 1, 2)))


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 6, 8, 3))
    p, idx = U.maxpool(x)
    g = rng.standard_normal(p.shape)
    back = U.unpool(g, idx)
    # the gradient lands exactly on the maxima
    assert np.isclose((back * x).sum(), (g * p).sum())
    z = rng.standard_normal((2, 3, 4, 3))
    w = rng.standard_normal((4, 6, 8, 3))
    assert np.isclose((U.up(z) * w).sum(), (z * U.up_adj(w)).sum())


@pytest.mark.slow
def test_network_gradient_matches_finite_differences():
    c = (4, 4, 4)
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(U.param_count(c)) * 0.3
    x = rng.standard_normal((8, 8, 8))
    t = rng.standard_normal((8, 8, 8))
    lval, g = U.grad(theta, x, t, c)
    assert np.isclose(lval, U.loss(theta, x, t, c))
    idx = rng.choice(theta.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (U.loss(theta + e, x, t, c) - U.loss(theta - e, x, t, c)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_head_is_identity():
    c = (4, 4, 4)
    theta = np.random.default_rng(4).standard_normal(U.param_count(c))
    theta[-(c[0] + 1):] = 0.0
    x = np.random.default_rng(5).standard_normal((8, 8, 8))
    assert np.array_equal(U.forward(theta, x, c), x)


def test_dual_from_x_lies_in_the_ball_and_is_aligned():
    import oracle as O
    x = np.random.default_rng(6).standard_normal((4, 6, 8))
    d = U.dual_from_x(x, 1e-2, 1e-1)
    nrm = np.sqrt((d ** 2).sum(axis=0))
    assert nrm.max() <= 1e-1 + 1e-12
    g = O.grad(x)
    gn = np.sqrt((g ** 2).sum(axis=0))
    assert np.allclose(d * gn[None], g * nrm[None])  # parallel to Lx


def test_bf16_round_is_round_to_nearest_even():
    import torch
    rng = np.random.default_rng(7)
    a = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-20, 20, 10000),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 65504.0]])
    a32 = a.astype(np.float32)
    ref = torch.tensor(a32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(a32), ref)
    # halfway cases go to the even neighbour
    assert U.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert U.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_quantised_network_rounds_only_the_stored_activations():
    c = (4, 4, 4)
    rng = np.random.default_rng(8)
    theta = rng.standard_normal(U.param_count(c)) * 0.3
    x = rng.standard_normal((8, 8, 8))
    exact = U.forward(theta, x, c)
    _, a = U.forward(theta, x, c, keep=True, quant=U.bf16_round)
    for k in ("e1a", "e1", "e2", "e3", "d2", "d1"):
        assert np.array_equal(U.bf16_round(a[k]), a[k]), k
    out = U.forward(theta, x, c, quant=U.bf16_round)
    # 2^-9 relative per rounding through ten layers
    assert np.linalg.norm(out - exact) <= 5e-2 * np.linalg.norm(exact - x)
    assert np.array_equal(U.forward(theta, x, c, quant=None), exact)


# ---------------------------------------------------------------------------
# Pins of the selection rules themselves (the adjoint identities above hold
# for any selection, so they cannot see a wrong one).  Each checker is run on
# the oracle and on planted mistakes of it, which it must reject.
# ---------------------------------------------------------------------------

def _maxpool_by_loops(x):
    """2x2x2 pooling by explicit loops: the block maximum, and the offset of its
    first occurrence when the 8 members are visited in (s, n, m) order."""
    s, n, m, c = x.shape
    val = np.zeros((s // 2, n // 2, m // 2, c))
    arg = np.zeros((s // 2, n // 2, m // 2, c), dtype=int)
    for i in range(s // 2):
        for j in range(n // 2):
            for k in range(m // 2):
                for ch in range(c):
                    best, where = None, -1
                    for t in range(8):
                        a, b, e = t // 4, (t // 2) % 2, t % 2
                        v = x[2 * i + a, 2 * j + b, 2 * k + e, ch]
                        if best is None or v > best:
                            best, where = v, t
                    val[i, j, k, ch], arg[i, j, k, ch] = best, where
    return val, arg


def _maxpool_agrees(fn):
    rng = np.random.default_rng(12)
    # small integers: many ties inside a block
    x = rng.integers(0, 3, size=(4, 6, 4, 3)).astype(np.float64)
    # a hand-built block: maxima 5 at members 3 (s0 n1 m1) and 6 (s1 n1 m0)
    x[0:2, 0:2, 0:2, 0] = np.array([[[1, 2], [0, 5]], [[4, 3], [5, -1]]])
    got_v, got_i = fn(x)
    ref_v, ref_i = _maxpool_by_loops(x)
    return got_v.shape == ref_v.shape and np.array_equal(got_v, ref_v) and np.array_equal(got_i, ref_i)


def test_maxpool_takes_the_block_maximum_and_the_first_tie():
    assert _maxpool_by_loops(np.array([[[1, 2], [0, 5]], [[4, 3], [5, -1]]], float)[..., None])[1][0, 0, 0, 0] == 3
    assert _maxpool_agrees(U.maxpool)


def _blocks(x):
    s, n, m, c = x.shape
    return x.reshape(s // 2, 2, n // 2, 2, m // 2, 2, c).transpose(0, 2, 4, 1, 3, 5, 6).reshape(
        s // 2, n // 2, m // 2, 8, c)


def _pool_min(x):
    b = _blocks(x)
    i = b.argmin(axis=3)
    return np.take_along_axis(b, i[:, :, :, None, :], axis=3)[:, :, :, 0, :], i


def _pool_last_tie(x):
    b = _blocks(x)[:, :, :, ::-1, :]
    i = 7 - b.argmax(axis=3)
    return b.max(axis=3), i


def _pool_m_major(x):  # members numbered in (m, n, s) order
    s, n, m, c = x.shape
    b = x.reshape(s // 2, 2, n // 2, 2, m // 2, 2, c).transpose(0, 2, 4, 5, 3, 1, 6).reshape(
        s // 2, n // 2, m // 2, 8, c)
    i = b.argmax(axis=3)
    return b.max(axis=3), i


@pytest.mark.parametrize("mutant", [_pool_min, _pool_last_tie, _pool_m_major])
def test_maxpool_checker_rejects_planted_mistakes(mutant):
    assert not _maxpool_agrees(mutant)


def _up_agrees(up, up_adj):
    rng = np.random.default_rng(13)
    z = rng.standard_normal((2, 3, 4, 2))
    u = up(z)
    if u.shape != (4, 6, 8, 2):
        return False
    ok = all(u[s, n, m, c] == z[s // 2, n // 2, m // 2, c]
             for s in range(4) for n in range(6) for m in range(8) for c in range(2))
    w = rng.standard_normal((4, 6, 8, 2))
    a = up_adj(w)
    ref = np.zeros_like(z)
    for s in range(4):
        for n in range(6):
            for m in range(8):
                ref[s // 2, n // 2, m // 2] += w[s, n, m]
    return ok and a.shape == ref.shape and np.allclose(a, ref, rtol=0, atol=1e-14)


def test_upsampling_copies_each_voxel_to_its_block():
    assert _up_agrees(U.up, U.up_adj)
    # planted mistakes: a tiled (not repeated) upsampling; an averaging adjoint
    assert not _up_agrees(lambda z: np.tile(z, (2, 2, 2, 1)), U.up_adj)
    assert not _up_agrees(U.up, lambda g: U.up_adj(g) / 8.0)


def _dual_agrees(fn):
    """Closed form on a hand-built volume: x is zero except x[j0] = v.  Then
    (Lx)_{j0} = (-v, -v, -v) (norm sqrt(3)|v|) and (Lx)_{j0 - e_a} = v e_a
    (norm |v|); every other g is zero.  With t = lam/mu between |v| and
    sqrt(3)|v|, d_{j0} = t (-1, -1, -1)/sqrt(3) (outside the ball: scaled to
    its surface) and d_{j0 - e_a} = v e_a (inside: unchanged)."""
    shape = (5, 4, 6)
    j0 = (2, 1, 3)
    v, lam, mu = 1.0, 1.2e-3, 1e-3
    t = lam / mu
    x = np.zeros(shape)
    x[j0] = v
    ref = np.zeros((3,) + shape)
    ref[(slice(None),) + j0] = -t / np.sqrt(3.0)
    ref[(0, j0[0], j0[1], j0[2] - 1)] = v  # m component at j0 - e_m
    ref[(1, j0[0], j0[1] - 1, j0[2])] = v  # n component at j0 - e_n
    ref[(2, j0[0] - 1, j0[1], j0[2])] = v  # s component at j0 - e_s
    got = fn(x, lam, mu)
    # on the sphere: t = |v| exactly keeps the neighbours unchanged
    got2 = fn(x, 1e-3, 1e-3)
    ref2 = ref.copy()
    ref2[(slice(None),) + j0] = -1.0 / np.sqrt(3.0)
    return (got.shape == ref.shape and np.allclose(got, ref, rtol=0, atol=1e-15)
            and np.allclose(got2, ref2, rtol=0, atol=1e-15))


def test_dual_from_x_equals_its_closed_form_on_both_sides_of_the_ball():
    assert _dual_agrees(U.dual_from_x)


def test_dual_checker_rejects_planted_mistakes():
    import oracle as O

    def half(x, lam, mu):
        return 0.5 * U.dual_from_x(x, lam, mu)

    def always_scaled(x, lam, mu):  # t g/||g|| everywhere (wrong inside the ball)
        g = O.grad(x)
        n = np.sqrt((g ** 2).sum(axis=0))
        return (lam / mu) * g / np.maximum(n, 1e-300)[None]

    def min_not_max(x, lam, mu):
        g = O.grad(x)
        n = np.sqrt((g ** 2).sum(axis=0))
        t = lam / mu
        return t * g / np.maximum(np.minimum(n, t), 1e-300)[None]

    for f in (half, always_scaled, min_not_max):
        assert not _dual_agrees(f)
