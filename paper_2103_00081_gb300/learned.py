"""Training and use of the U-Net warm start (thin driver over the C ABI).

The network (include/ht.h, ht_unet_*) predicts the next step's increments of
temperature and head from the last two increments of both fields, the Darcy
flux and the heat sources; the solver gates the prediction against the
initial guess it would take without it: the field at t^n, or its
extrapolation in time (ht_set_learned_guess, HT_GUESS_EXTRAPOLATE).
Samples come from trajectories the simulator itself generates
(ht_learned_sample); all arithmetic runs in the library's kernels and torch
only provides device buffers.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int, c_void_p

import numpy as np

from . import _lib as L


FEATURES = 8      # [dT1, dT2, dh1, dh2, F_T, q_x, q_y, q_z] (see include/ht.h)


def layer_shapes(cin: int = FEATURES, cout: int = 2):
    """(Cin, Cout, taps) of the 15 convolutions of the library's U-Net, in the
    order of its parameter vector (widths 16-32-48-64)."""
    c1, c2, c3, c4 = 16, 32, 48, 64
    return [(cin, c1, 27), (c1, c1, 27), (c1, c2, 27), (c2, c2, 27), (c2, c3, 27), (c3, c3, 27),
            (c3, c4, 27), (c4, c4, 27), (c4 + c3, c3, 27), (c3, c3, 27), (c3 + c2, c2, 27), (c2, c2, 27),
            (c2 + c1, c1, 27), (c1, c1, 27), (c1, cout, 1)]


class UNet:
    def __init__(self, device: int = 0, seed: int = 0, cin: int = FEATURES):
        self._lib = L.lib()
        h = c_void_p()
        rc = self._lib.ht_unet_create(byref(h), int(cin), 2, int(device), None)
        if rc != L.HT_OK:
            raise RuntimeError(f"ht_unet_create failed ({rc})")
        self._h = h
        self.cin = cin
        self.n_params = self._lib.ht_unet_num_params(h)
        self.set_params(self.initial_params(seed))

    def initial_params(self, seed: int) -> np.ndarray:
        """He-uniform weights (the last layer scaled by 1/10), zero biases; the
        layout is per layer weights [taps][Cout][Cin] then biases [Cout]."""
        rng = np.random.default_rng(seed)
        shapes = layer_shapes(self.cin)
        out = []
        for li, (ci, co, k) in enumerate(shapes):
            bound = np.sqrt(6.0 / (ci * k)) * (0.1 if li == len(shapes) - 1 else 1.0)
            out.append(rng.uniform(-bound, bound, k * co * ci))
            out.append(np.zeros(co))
        theta = np.concatenate(out).astype(np.float32)
        assert theta.size == self.n_params
        return theta

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        rc = self._lib.ht_unet_set_params(self._h, theta.ctypes.data_as(c_void_p))
        if rc != L.HT_OK:
            raise RuntimeError(self._lib.ht_unet_last_error(self._h).decode())

    def get_params(self) -> np.ndarray:
        theta = np.empty(self.n_params, dtype=np.float32)
        self._lib.ht_unet_get_params(self._h, theta.ctypes.data_as(c_void_p))
        return theta

    def train_step(self, x, t, lr: float) -> float:
        D, H, W = x.shape[1:]
        loss = c_double()
        rc = self._lib.ht_unet_train_step(self._h, c_void_p(x.data_ptr()), c_void_p(t.data_ptr()), D, H, W,
                                          ctypes.c_float(lr), byref(loss))
        if rc != L.HT_OK:
            raise RuntimeError(self._lib.ht_unet_last_error(self._h).decode())
        return loss.value

    def loss(self, x, t) -> float:
        D, H, W = x.shape[1:]
        loss = c_double()
        self._lib.ht_unet_loss_grad(self._h, c_void_p(x.data_ptr()), c_void_p(t.data_ptr()), D, H, W,
                                    byref(loss), None)
        return loss.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ht_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def attach(sim, net, record: bool = False):
    rc = sim._lib.ht_set_learned_guess(sim._h, net._h if net is not None else None, int(record))
    if rc != L.HT_OK:
        raise RuntimeError("ht_set_learned_guess failed")


def collect_samples(sim, dt: float, n_steps: int):
    """Step `sim` n_steps times with recording on; return the (features,
    targets) pairs of every step that had two earlier increments."""
    import torch
    attach(sim, None, record=True)
    samples = []
    dims = (c_int * 3)()
    for _ in range(n_steps):
        sim.step(dt)
        Dp, Hp, Wp = ((sim.dims[2] + 7) // 8 * 8, (sim.dims[1] + 7) // 8 * 8, (sim.dims[0] + 7) // 8 * 8)
        f = torch.empty((FEATURES, Dp, Hp, Wp), dtype=torch.float32, device="cuda")
        t = torch.empty((2, Dp, Hp, Wp), dtype=torch.float32, device="cuda")
        rc = sim._lib.ht_learned_sample(sim._h, c_void_p(f.data_ptr()), c_void_p(t.data_ptr()), dims)
        if rc == L.HT_OK:
            samples.append((f, t))
    attach(sim, None, record=False)
    return samples


def train(net: UNet, samples, epochs: int = 20, lr: float = 1e-3, seed: int = 0):
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(epochs):
        ep = []
        for i in rng.permutation(len(samples)):
            x, t = samples[i]
            ep.append(net.train_step(x, t, lr))
        losses.append(float(np.mean(ep)))
    return losses
