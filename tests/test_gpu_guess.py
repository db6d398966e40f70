"""Initial guesses extrapolated in time (HT_GUESS_EXTRAPOLATE, the default):
each step may start its two Krylov solves from the Lagrange extrapolation to
t^{n+1} of the last two or three fields instead of the field at t^n, when
the extrapolation has the smaller residual.  The guess changes the number of
iterations, not the solution: the fields match the oracle at the parity
tolerances, also with step sizes that vary from step to step, and match the
run that starts every solve from the previous field."""
import numpy as np
import pytest

import scenarios as S
from oracle import fem

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _scenario(p):
    if p == 1:
        return S.config3(nx=24, ny=24, nz=8, seed=21, extent=(300.0, 300.0, 40.0), n_piles=(4, 4))
    return S.config2(nx=10, ny=10, nz=4)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("mixed", [False, True])
def test_extrapolated_guess_matches_oracle_and_cuts_iterations(built_lib, p, mixed):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sc = _scenario(p)
    o = fem.OracleSim(sc)
    base = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4) if mixed else dict(tol=1e-13)
    sims = {g: hydro.Simulator.from_scenario(sc, guess=g, max_iter=100000, **base)
            for g in (L.HT_GUESS_PREVIOUS, L.HT_GUESS_EXTRAPOLATE)}
    its = {g: 0 for g in sims}
    chosen = []
    try:
        for k in range(8):
            o.step(sc.dt)
            for g, sim in sims.items():
                st = sim.step(sc.dt)
                if k >= 3:
                    its[g] += st["iters_head"] + st["iters_heat"]
                if g == L.HT_GUESS_EXTRAPOLATE:
                    chosen.append((st["guess_head"], st["guess_heat"]))
                    if k == 0:   # no past field yet: no gate ran
                        assert st["guess_res_head"] == -1.0 and st["guess_res_heat"] == -1.0
                h, T = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
                assert _rel(h, o.h) <= 1e-9 and _rel(T, o.T) <= 1e-9, (g, k, _rel(h, o.h), _rel(T, o.T))
    finally:
        for sim in sims.values():
            sim.close()
    assert chosen[0] == (0, 0)
    # from the third step on the quadratic extrapolation is available; the
    # smooth seasonal loads make it the better start for most solves
    assert sum(c[0] == 2 for c in chosen[2:]) + sum(c[1] == 2 for c in chosen[2:]) >= 6, chosen
    print(f"[p={p} mixed={mixed}] iterations of steps 4-8, previous / extrapolated: "
          f"{its[L.HT_GUESS_PREVIOUS]} / {its[L.HT_GUESS_EXTRAPOLATE]}; choices {chosen}")
    assert its[L.HT_GUESS_EXTRAPOLATE] < its[L.HT_GUESS_PREVIOUS], its


def test_extrapolation_with_varying_steps_and_restart_from_a_state(built_lib):
    """Step sizes of 1, 0.5, 2, 1 and 3 days (the Lagrange weights use the
    actual times); ht_set_state forgets the past fields, so the step after it
    starts from the set field again."""
    from paper_2103_00081_gb300 import hydro
    sc = _scenario(1)
    o = fem.OracleSim(sc)
    sim = hydro.Simulator.from_scenario(sc, tol=1e-13, max_iter=100000)
    try:
        for d in (1.0, 0.5, 2.0, 1.0, 3.0):
            dt = d * S.DAY
            o.step(dt)
            sim.step(dt)
            assert _rel(sim.get_field(S.HEAD), o.h) <= 1e-9 and _rel(sim.get_field(S.TEMP), o.T) <= 1e-9
        assert abs(sim.time - o.t) <= 1e-9 * o.t
        sim.set_state(o.h, o.T, o.t)
        st = sim.step(S.DAY)
        o.step(S.DAY)
        assert (st["guess_head"], st["guess_heat"]) == (0, 0)
        assert st["guess_res_head"] == -1.0
        assert _rel(sim.get_field(S.HEAD), o.h) <= 1e-9 and _rel(sim.get_field(S.TEMP), o.T) <= 1e-9
    finally:
        sim.close()


def test_unknown_guess_is_rejected(built_lib):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sc = _scenario(1)
    sim = hydro.Simulator.from_scenario(sc)
    try:
        with pytest.raises(hydro.HTError) as e:
            sim.set_solver(guess=7)
        assert e.value.code == L.HT_EINVAL
    finally:
        sim.close()
