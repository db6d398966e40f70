"""The learned warm start end to end: samples from simulator trajectories,
training with the library's kernels, and the gain on an unseen scenario --
Krylov iterations with the gated learned guess against the same run without
it, with the same solutions to the solver tolerance."""
import numpy as np
import pytest

import scenarios as S

pytestmark = pytest.mark.gpu


def _scenario(seed):
    return S.config3(nx=32, ny=32, nz=16, seed=seed, extent=(400.0, 400.0, 50.0), n_piles=(6, 6))


@pytest.mark.parametrize("mixed", [False, True])
def test_learned_guess_trains_and_cuts_iterations(built_lib, mixed):
    pytest.importorskip("torch")
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro, learned
    # against the previous-step guess, the fallback the learned guess replaces
    opts = dict(tol=1e-10, precision=L.HT_MIXED if mixed else L.HT_FP64, guess=L.HT_GUESS_PREVIOUS)
    train_sc = _scenario(11)
    sim = hydro.Simulator.from_scenario(train_sc, **opts)
    samples = learned.collect_samples(sim, train_sc.dt, 40)
    assert len(samples) == 38
    net = learned.UNet(seed=1)
    losses = learned.train(net, samples, epochs=25, lr=1e-3)
    assert losses[-1] < 0.5 * losses[0], losses

    test_sc = _scenario(12)
    runs = {}
    for use in (False, True):
        s = hydro.Simulator.from_scenario(test_sc, **opts)
        if use:
            learned.attach(s, net)
        its, wins = 0, 0
        for k in range(20):
            st = s.step(test_sc.dt)
            if k >= 3:
                its += st["iters_head"] + st["iters_heat"]
                wins += (st["guess_head"] == 1) + (st["guess_heat"] == 1)
        runs[use] = (its, wins, s.get_field(S.HEAD), s.get_field(S.TEMP))
        s.close()
    its0, _, h0, T0 = runs[False]
    its1, wins1, h1, T1 = runs[True]
    assert wins1 > 0
    assert its1 < its0, (its0, its1)
    # both runs stop at relative residual 1e-10; their difference is bounded
    # by about 2 kappa tol with kappa ~ 1e3 on this mesh
    assert np.linalg.norm(h1 - h0) / np.linalg.norm(h0) < 1e-7
    assert np.linalg.norm(T1 - T0) / np.linalg.norm(T0) < 1e-7
    print(f"[{'mixed' if mixed else 'fp64'}] iterations without / with the learned guess: "
          f"{its0} / {its1}; gate wins {wins1}")
