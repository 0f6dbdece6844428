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
