"""Pile surfaces at a prescribed temperature and seasonal Dirichlet faces
(Section 3.3) in the library, against the oracle's definitions
(oracle/fem.py: pile_surface_nodes, pile_temperature, seasonal_value).

The pile nodes inside the mesh are Dirichlet rows of the heat system that no
face mask describes; a pile that reaches the top face puts some of its nodes
on the seasonal face, where the pile's value wins.  Tolerances as in
test_gpu_parity: operator, diagonal and right-hand side 1e-12, steps solved
to 1e-12 relative residual 1e-9."""
import math

import numpy as np
import pytest

import scenarios as S
from oracle import fem

pytestmark = pytest.mark.gpu

YEAR = 365 * S.DAY


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _close(got, ref, tol=1e-12):
    assert _rel(got, ref) <= tol, _rel(got, ref)
    assert np.max(np.abs(got - ref)) <= tol * max(np.max(np.abs(ref)), 1e-300)


def _scenario(p, n, nz, seed, faces=True, seasonal=True):
    """n x n x nz cells over 12 x 12 x 6 m, lognormal K, a head gradient in
    x, three piles (one from the top face down, two buried) with different
    phases, fixed temperatures on x = 0 and x = 12 and a seasonal top face."""
    rng = np.random.default_rng(seed)
    sc = S.random_small(seed, n, n, nz, p, n_piles=2, n_wells=0, extent=(12.0, 12.0, 6.0), dt=30 * S.DAY)
    rows = [[6.0, 6.0, 6.0, 2.0, 0.8, 288.55, 13.0, YEAR, 0.0],
            [3.1, 8.9, 4.5, 1.0, 0.7, 290.0, 5.0, YEAR, 1.0],
            [9.0, 3.0, 5.0, 0.5, 1e-3, 286.0, 8.0, 0.5 * YEAR, 2.5]]   # thinner than a node spacing
    sc.pile_temps = np.asarray(rows, dtype=np.float64)
    sc.T0 = 288.0 + rng.standard_normal(sc.n_nodes)
    tb = {0: (S.DIRICHLET, 287.0), 1: (S.DIRICHLET, 289.0)} if faces else {}
    sc.bc = {S.HEAD: dict(sc.bc.get(S.HEAD, {})), S.TEMP: tb}
    if seasonal and faces:
        sc.bc_seasonal = {S.TEMP: {5: (287.45, 8.0, YEAR, 0.3)}}
    return sc


CASES = [(1, 24, 8, 1), (2, 9, 4, 2), (1, 33, 20, 3)]


def _ids(c):
    return f"q{c[0]}_{c[1]}x{c[1]}x{c[2]}"


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_operator_diag_rhs_with_pile_rows_match_oracle(built_lib, case):
    from paper_2103_00081_gb300 import hydro
    p, n, nz, seed = case
    sc = _scenario(p, n, nz, seed)
    o = fem.OracleSim(sc)
    sim = hydro.Simulator.from_scenario(sc)
    assert sum(len(v) for v in o.pile_nodes) > 0
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(sc.n_nodes)
    dt = sc.dt
    _close(sim.apply(S.TEMP, dt, x), o.apply_heat(x, o.h, dt))
    _close(sim.diag(S.TEMP, dt), o.diag_heat(o.h, dt))
    _close(sim.rhs(S.TEMP, dt), o.heat_rhs(dt, dt, o.h))
    _close(sim.rhs(S.HEAD, dt), o.head_rhs(dt, dt))
    # the emulated residual of such a context is formed in FP64: it agrees
    # with the FP64 one
    b = o.heat_rhs(dt, dt, o.h)
    assert abs(sim.residual(S.TEMP, dt, x, b, emulated=True) - sim.residual(S.TEMP, dt, x, b)) <= \
        1e-12 * sim.residual(S.TEMP, dt, x, b)


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("mixed", [False, True])
def test_steps_with_pile_and_seasonal_temperatures_match_oracle(built_lib, case, mixed):
    """Five 30-day steps: the third pile (half-year period) switches its
    square wave after 91 days.  The pile nodes hold their square-wave values
    and the rest of the top face its seasonal value at every step's end
    time."""
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    p, n, nz, seed = case
    sc = _scenario(p, n, nz, seed)
    o = fem.OracleSim(sc)
    opts = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4) if mixed else dict(tol=1e-13)
    sim = hydro.Simulator.from_scenario(sc, **opts)
    top = o.mesh.face_nodes(5)
    held = set(np.concatenate(o.pile_nodes).tolist())
    seasonal_only = np.array([i for i in top if i not in held])
    for k in range(1, 6):
        sim.step(sc.dt)
        o.step(sc.dt)
        h, T = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
        assert _rel(h, o.h) <= 1e-9 and _rel(T, o.T) <= 1e-9, (_rel(h, o.h), _rel(T, o.T))
        t1 = k * sc.dt
        for row, nodes in zip(sc.pile_temps, o.pile_nodes):
            np.testing.assert_allclose(T[nodes], fem.pile_temperature(row, t1), rtol=1e-13, atol=0)
        ts = fem.seasonal_value((287.45, 8.0, YEAR, 0.3), t1)
        np.testing.assert_allclose(T[seasonal_only], ts, rtol=1e-13, atol=0)


@pytest.mark.parametrize("p", [1, 2])
def test_insulated_block_with_a_pile_surface_matches_oracle(built_lib, p):
    """No Dirichlet face in the heat system: the pile nodes are its only
    Dirichlet rows."""
    from paper_2103_00081_gb300 import hydro
    sc = _scenario(p, 10, 5, 7, faces=False, seasonal=False)
    o = fem.OracleSim(sc)
    sim = hydro.Simulator.from_scenario(sc, tol=1e-13)
    for _ in range(3):
        sim.step(sc.dt)
        o.step(sc.dt)
        assert _rel(sim.get_field(S.TEMP), o.T) <= 1e-9
        assert _rel(sim.get_field(S.HEAD), o.h) <= 1e-9


def test_pile_surface_nodes_match_the_oracle_selection(built_lib):
    """The library's node selection (radius, depth range, nearest column for
    a pile thinner than the node spacing) is the oracle's: the held rows of
    the diagonal are exactly the oracle's pile nodes."""
    from paper_2103_00081_gb300 import hydro
    sc = _scenario(1, 12, 6, 11, faces=False, seasonal=False)
    o = fem.OracleSim(sc)
    sim = hydro.Simulator.from_scenario(sc)
    d = sim.diag(S.TEMP, sc.dt)
    held = np.zeros(sc.n_nodes, dtype=bool)
    held[np.concatenate(o.pile_nodes)] = True
    assert np.all(d[held] == 1.0)
    assert np.all(d[~held] != 1.0)


def test_invalid_pile_temperatures_and_seasonal_faces_are_rejected(built_lib):
    from paper_2103_00081_gb300 import hydro
    sc = S.random_small(5, 4, 4, 3, 1, extent=(12.0, 12.0, 6.0))
    sim = hydro.Simulator.from_scenario(sc)
    good = [6.0, 6.0, 6.0, 2.0, 0.8, 288.55, 13.0, YEAR, 0.0]
    for bad in ([*good[:4], -1.0, *good[5:]], [*good[:7], 0.0, 0.0], [*good[:5], math.nan, *good[6:]],
                [6.0, 6.0, 20.0, 10.0, 0.8, 288.0, 1.0, YEAR, 0.0]):
        with pytest.raises(hydro.HTError):
            sim.set_pile_temperatures([bad])
    with pytest.raises(hydro.HTError):
        sim.set_seasonal_face(S.TEMP, 6, 1.0, 1.0, YEAR)
    with pytest.raises(hydro.HTError):
        sim.set_seasonal_face(S.TEMP, 5, 1.0, 1.0, 0.0)
    sim.set_pile_temperatures(np.zeros((0, 9)))
    sim.close()
