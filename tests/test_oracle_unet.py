"""Pins of the FP64 U-Net oracle: brute-force convolution on tiny grids,
adjointness of the pooling / upsampling backward maps, and central finite
differences of the loss against the analytical gradient."""
import numpy as np

from oracle import unet as U


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 5))
    w = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    got = U.conv(x, w, b)
    ref = np.zeros_like(got)
    C, D, H, W = x.shape
    for o in range(3):
        for z in range(D):
            for y in range(H):
                for xx in range(W):
                    s = b[o]
                    t = 0
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                zz, yy, x2 = z + dz, y + dy, xx + dx
                                if 0 <= zz < D and 0 <= yy < H and 0 <= x2 < W:
                                    s += sum(w[o, c, t] * x[c, zz, yy, x2] for c in range(C))
                                t += 1
                    ref[o, z, y, xx] = s
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_pool_and_upsample_backward_are_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 4, 6, 8))
    y = rng.standard_normal((2, 2, 3, 4))
    assert abs(np.sum(U.pool(x) * y) - np.sum(x * U.pool_backward(y))) < 1e-12
    assert abs(np.sum(U.upsample(y) * x) - np.sum(y * U.upsample_backward(x))) < 1e-12


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    dims = (3, 4, 5, 2)
    theta = 0.3 * rng.standard_normal(U.n_params(*dims))
    x = rng.standard_normal((3, 4, 4, 6))
    t = rng.standard_normal((2, 4, 4, 6))
    loss, g = U.loss_and_grad(theta, x, t, dims)
    idx = rng.choice(theta.size, 40, replace=False)
    eps = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd = (U.loss_and_grad(tp, x, t, dims)[0] - U.loss_and_grad(tm, x, t, dims)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding_is_nearest_even():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159265])
    r = U.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0            # tie to even
    assert r[2] == 1.0 + 2 ** -7                  # above the tie rounds up
    assert r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12
