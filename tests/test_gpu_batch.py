"""Batched steps (ht_batch_step) against the oracle and against the
single-problem path: problems of different sizes in one batch."""
import numpy as np
import pytest

import scenarios as S
from oracle import fem

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("mode", [0, 1], ids=["concurrent", "shared_launches"])
@pytest.mark.parametrize("order", [1, 2])
def test_batched_steps_match_oracle_and_single_path(built_lib, order, mode):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sizes = [(7, 5, 4), (12, 9, 6), (3, 3, 2)] if order == 2 else [(13, 9, 7), (20, 17, 9), (5, 4, 3)]
    scs = [S.random_small(40 + i, nx, ny, nz, order, n_wells=1) for i, (nx, ny, nz) in enumerate(sizes)]
    opts = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4)
    sims = [hydro.Simulator.from_scenario(sc, **opts) for sc in scs]
    singles = [hydro.Simulator.from_scenario(sc, **opts) for sc in scs]
    oracles = [fem.OracleSim(sc) for sc in scs]
    batch = hydro.Batch(sims, mode=mode)
    for step in range(2):
        stats = batch.step(scs[0].dt)
        for sim, single, o, st in zip(sims, singles, oracles, stats):
            single.step(o.sc.dt)
            o.step(o.sc.dt)
            assert st["res_head"] <= 1e-12 and st["iters_head"] > 0
            h, T = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
            assert _rel(h, o.h) <= 1e-9 and _rel(T, o.T) <= 1e-9
            assert _rel(h, single.get_field(S.HEAD)) <= 1e-9
            assert abs(sim.time - (step + 1) * o.sc.dt) < 1e-6
    batch.close()


def test_batch_rejects_wrong_solver_options(built_lib):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sc = S.random_small(50, 4, 4, 3, 1)
    sim = hydro.Simulator.from_scenario(sc)            # plain FP64: not batchable
    batch = hydro.Batch([sim])
    with pytest.raises(hydro.HTError):
        hydro.Batch([sim], mode=7)
    with pytest.raises(hydro.HTError) as e:
        batch.step(sc.dt)
    assert e.value.code == L.HT_EINVAL
    batch.close()
