"""Pins of the FP64 U-Net oracle: brute-force convolution on tiny grids,
adjointness of the pooling / upsampling backward maps, central finite
differences of the exact network's loss against its analytical gradient, the
placement of the BF16 rounding points, and round-to-nearest-even BF16."""
import numpy as np

from oracle import unet as U


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 5))
    w = rng.standard_normal((27, 3, 2))      # [taps][Cout][Cin]
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
                                    s += sum(w[t, o, c] * x[c, zz, yy, x2] for c in range(C))
                                t += 1
                    ref[o, z, y, xx] = s
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_conv_backward_is_the_adjoint_and_the_weight_derivative():
    rng = np.random.default_rng(6)
    x = rng.standard_normal((3, 4, 3, 5))
    w = rng.standard_normal((27, 2, 3))
    g = rng.standard_normal((2, 4, 3, 5))
    gx, gw, gb = U.conv_backward(x, w, g)
    # <g, conv(x) - b> = <gx, x> (linear in x) and = <gw, w> (linear in w)
    lin = np.sum(g * (U.conv(x, w, np.zeros(2))))
    assert abs(lin - np.sum(gx * x)) <= 1e-11 * abs(lin)
    assert abs(lin - np.sum(gw * w)) <= 1e-11 * abs(lin)
    np.testing.assert_allclose(gb, g.sum(axis=(1, 2, 3)), rtol=1e-13)


def test_pool_and_upsample_backward_are_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 4, 6, 8))
    y = rng.standard_normal((2, 2, 3, 4))
    assert abs(np.sum(U.pool(x) * y) - np.sum(x * U.pool_backward(y))) < 1e-12
    assert abs(np.sum(U.upsample(y) * x) - np.sum(y * U.upsample_backward(x))) < 1e-12


def test_parameter_count_and_layout():
    # widths 16-32-48-64 with 8 input and 2 output channels
    n = U.n_params(8, 2)
    expect = 27 * (8 * 16 + 16 * 16 + 16 * 32 + 32 * 32 + 32 * 48 + 48 * 48 + 48 * 64 + 64 * 64 + 112 * 48
                   + 48 * 48 + 80 * 32 + 32 * 32 + 48 * 16 + 16 * 16) + 16 * 2
    expect += 16 + 16 + 32 + 32 + 48 + 48 + 64 + 64 + 48 + 48 + 32 + 32 + 16 + 16 + 2
    assert n == expect
    theta = np.arange(n, dtype=np.float64)
    layers = U.unpack(theta, 8, 2)
    assert layers[0][0].shape == (27, 16, 8) and layers[8][0].shape == (27, 48, 112)
    assert layers[14][0].shape == (1, 2, 16)
    assert layers[1][0][0, 0, 0] == layers[0][1][-1] + 1       # weights follow the previous biases


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    widths = (3, 4, 5, 6)
    cin, cout = 2, 2
    theta = 0.3 * rng.standard_normal(U.n_params(cin, cout, widths))
    x = rng.standard_normal((cin, 8, 8, 8))
    t = rng.standard_normal((cout, 8, 8, 8))
    loss, g = U.loss_and_grad(theta, x, t, cin, cout, widths, bf16=False)
    idx = rng.choice(theta.size, 40, replace=False)
    eps = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd = (U.loss_and_grad(tp, x, t, cin, cout, widths, bf16=False)[0] -
              U.loss_and_grad(tm, x, t, cin, cout, widths, bf16=False)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_network_rounds_only_at_its_stated_points():
    """With weights and input already on the BF16 grid, the mixed network
    differs from the exact one only through rounded activations: its output
    is close (BF16 relative error compounds mildly over 15 layers) but not
    identical, and its stored activations are all BF16 numbers."""
    rng = np.random.default_rng(7)
    widths = (4, 4, 4, 4)
    theta = U.bf16_round(0.3 * rng.standard_normal(U.n_params(2, 2, widths)))
    x = U.bf16_round(rng.standard_normal((2, 8, 8, 8)))
    y1, (act, _) = U.forward(theta, x, 2, 2, widths, bf16=True)
    y0, _ = U.forward(theta, x, 2, 2, widths, bf16=False)
    rel = np.linalg.norm(y1 - y0) / np.linalg.norm(y0)
    assert 0 < rel < 5e-2
    for k in ("a0", "e1", "p1", "a7", "d1"):
        np.testing.assert_array_equal(act[k], U.bf16_round(act[k]))


def test_bf16_rounding_is_nearest_even():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159265])
    r = U.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0            # tie to even
    assert r[2] == 1.0 + 2 ** -7                  # above the tie rounds up
    assert r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12
