"""The CUDA U-Net (forward, loss gradient, Adam) against the FP64 oracle with
the same BF16-rounded weights.  Tolerances: FP32 accumulation over at most a
few thousand terms, relative 1e-4 (forward) and 2e-3 (gradients)."""
import ctypes

import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu
DIMS = (4, 16, 32, 2)


def _net(torch):
    from paper_2103_00081_gb300 import _lib as L
    lib = L.lib()
    h = ctypes.c_void_p()
    assert lib.ht_unet_create(ctypes.byref(h), 4, 2, 0, None) == 0
    return lib, h


def test_forward_and_gradient_match_oracle(built_lib):
    torch = pytest.importorskip("torch")
    lib, h = _net(torch)
    n = lib.ht_unet_num_params(h)
    assert n == U.n_params(*DIMS)
    rng = np.random.default_rng(4)
    theta = (0.2 * rng.standard_normal(n)).astype(np.float32)
    assert lib.ht_unet_set_params(h, theta.ctypes.data_as(ctypes.c_void_p)) == 0
    # the oracle sees the BF16-rounded weights and the FP32 biases
    th = theta.astype(np.float64)
    o = 0
    for co, ci, k in U.layer_shapes(*DIMS):
        th[o:o + co * ci * k] = U.bf16_round(th[o:o + co * ci * k])
        o += co * ci * k + co
    D, H, W = 6, 8, 10
    x = rng.standard_normal((4, D, H, W)).astype(np.float32)
    t = rng.standard_normal((2, D, H, W)).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    td = torch.tensor(t, device="cuda")
    yd = torch.empty((2, D, H, W), device="cuda")
    assert lib.ht_unet_forward(h, ctypes.c_void_p(xd.data_ptr()), D, H, W, ctypes.c_void_p(yd.data_ptr())) == 0
    torch.cuda.synchronize()
    yref, _ = U.forward(th, x.astype(np.float64), DIMS)
    got = yd.cpu().numpy()
    assert np.linalg.norm(got - yref) / np.linalg.norm(yref) <= 1e-4
    loss = ctypes.c_double()
    g = np.empty(n, dtype=np.float32)
    assert lib.ht_unet_loss_grad(h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(td.data_ptr()), D, H, W,
                                 ctypes.byref(loss), g.ctypes.data_as(ctypes.c_void_p)) == 0
    lref, gref = U.loss_and_grad(th, x.astype(np.float64), t.astype(np.float64), DIMS)
    assert abs(loss.value - lref) <= 1e-4 * abs(lref)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 2e-3
    lib.ht_unet_destroy(h)


def test_adam_training_reduces_the_loss(built_lib):
    torch = pytest.importorskip("torch")
    lib, h = _net(torch)
    n = lib.ht_unet_num_params(h)
    rng = np.random.default_rng(5)
    theta = (0.1 * rng.standard_normal(n)).astype(np.float32)
    lib.ht_unet_set_params(h, theta.ctypes.data_as(ctypes.c_void_p))
    D, H, W = 8, 8, 8
    x = rng.standard_normal((4, D, H, W)).astype(np.float32)
    t = np.stack([x[0] + 0.5 * x[1], x[2] - x[3]]).astype(np.float32)   # a learnable local map
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    loss = ctypes.c_double()
    losses = []
    for it in range(300):
        assert lib.ht_unet_train_step(h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(td.data_ptr()), D, H, W,
                                      ctypes.c_float(3e-3), ctypes.byref(loss)) == 0
        losses.append(loss.value)
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
    lib.ht_unet_destroy(h)
