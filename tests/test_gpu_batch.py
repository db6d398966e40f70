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


@pytest.mark.parametrize("planes", [0, 3])
def test_persistent_batch_matches_oracle_and_single_path(built_lib, planes):
    """One cooperative launch per outer pass runs the inner CG of all
    problems: meshes of one to several tiles, z chunks of 3 planes (several
    chunks per problem) and the automatic choice."""
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sizes = [(13, 9, 7), (61, 45, 11), (5, 4, 3), (30, 41, 9)]
    scs = [S.random_small(60 + i, nx, ny, nz, 1, n_wells=1) for i, (nx, ny, nz) in enumerate(sizes)]
    opts = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4)
    sims = [hydro.Simulator.from_scenario(sc, **opts) for sc in scs]
    singles = [hydro.Simulator.from_scenario(sc, **opts) for sc in scs]
    oracles = [fem.OracleSim(sc) for sc in scs]
    batch = hydro.Batch(sims, mode=L.HT_BATCH_PERSISTENT)
    batch.set_persistent(planes=planes)
    for step in range(2):
        stats = batch.step(scs[0].dt)
        info = batch.persistent_info()
        assert info["err_cta"] == -1 and info["grid"] >= 1 and info["items"] >= len(sims)
        if planes:
            assert info["planes"] == planes
        for sim, single, o, st in zip(sims, singles, oracles, stats):
            single.step(o.sc.dt)
            o.step(o.sc.dt)
            assert st["res_head"] <= 1e-12 and st["iters_head"] > 0
            h, T = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
            assert _rel(h, o.h) <= 1e-9 and _rel(T, o.T) <= 1e-9
            assert _rel(h, single.get_field(S.HEAD)) <= 1e-9
            assert abs(sim.time - (step + 1) * o.sc.dt) < 1e-6
    batch.close()


def test_persistent_barrier_wait_runs_out_and_returns_timeout(built_lib):
    """Failure injection on the host: one CTA of the cooperative launch skips
    its first barrier arrival, so the other CTAs' waits (bounded at 1 ms)
    run out; the step returns HT_ETIMEOUT, leaves the problems' times and
    fields as they were, and the same step then succeeds."""
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sizes = [(61, 45, 11), (30, 41, 9)]
    scs = [S.random_small(70 + i, nx, ny, nz, 1, n_wells=1) for i, (nx, ny, nz) in enumerate(sizes)]
    opts = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4)
    sims = [hydro.Simulator.from_scenario(sc, **opts) for sc in scs]
    oracles = [fem.OracleSim(sc) for sc in scs]
    h0 = [s.get_field(S.HEAD) for s in sims]
    batch = hydro.Batch(sims, mode=L.HT_BATCH_PERSISTENT)
    batch.set_persistent(planes=2, wait_ms=1.0, drop_cta=1)
    with pytest.raises(hydro.HTError) as e:
        batch.step(scs[0].dt)
    assert e.value.code == L.HT_ETIMEOUT
    info = batch.persistent_info()
    assert info["grid"] >= 2 and info["err_cta"] >= 0 and info["err_cta"] != 1
    for sim, h in zip(sims, h0):
        assert sim.time == 0.0
        np.testing.assert_array_equal(sim.get_field(S.HEAD), h)
    batch.set_persistent(planes=2, wait_ms=2000.0, drop_cta=-1)
    batch.step(scs[0].dt)
    for sim, o in zip(sims, oracles):
        o.step(o.sc.dt)
        assert _rel(sim.get_field(S.HEAD), o.h) <= 1e-9 and _rel(sim.get_field(S.TEMP), o.T) <= 1e-9
    batch.close()


def test_persistent_mode_needs_q1_single_pass(built_lib):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sc = S.random_small(80, 4, 4, 3, 2)
    sim = hydro.Simulator.from_scenario(sc, precision=L.HT_MIXED)
    with pytest.raises(hydro.HTError) as e:
        hydro.Batch([sim], mode=L.HT_BATCH_PERSISTENT)
    assert e.value.code == L.HT_EINVAL
    sc1 = S.random_small(81, 4, 4, 3, 1)
    sim1 = hydro.Simulator.from_scenario(sc1, precision=L.HT_MIXED)
    b = hydro.Batch([sim1], mode=L.HT_BATCH_PERSISTENT)
    for bad in [dict(planes=-1), dict(wait_ms=0.0), dict(wait_ms=1e9), dict(drop_cta=-2)]:
        with pytest.raises(hydro.HTError):
            b.set_persistent(**bad)
    b.close()
