"""The hot-water injection benchmark of Section 2 (Fig. 2, Table 1) in the
library: a quarter of the 20 m x 300 m cylinder around the wellbore on a
graded box mesh, injection flux Q_b through the wellbore surface (a quarter
of the well's rate as a line source on the axis) and T_b on the wellbore
nodes (interior Dirichlet rows), Table 1's materials, the geotherm, and
K = 1e-6 / 1e-10 m/s in the aquifer / confining layers.

* Coarse meshes: operator, diagonal and right-hand side of both systems at
  1e-12, and three daily steps in FP64 and mixed precision at 1e-9 against
  the oracle (the tolerances of test_gpu_parity).
* The default mesh (266 x 266 x 90 cells, 6,487,299 nodes, cell Peclet
  number <= 2 outside the wellbore): sampled operator rows and right-hand
  side rows of the row-wise oracle, and one daily mixed-precision step whose
  solution satisfies the oracle's rows to the solver tolerance; the step
  keeps the wellbore at T_b and the fields mirror-symmetric in x <-> y, and
  the temperature stays within the initial range (no Galerkin overshoot).
"""
import numpy as np
import pytest

import scenarios as S
from oracle import fem

pytestmark = pytest.mark.gpu

TB = S.ATES_TABLE1["T_b"]


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _close(got, ref, tol=1e-12):
    assert _rel(got, ref) <= tol, _rel(got, ref)
    assert np.max(np.abs(got - ref)) <= tol * max(np.max(np.abs(ref)), 1e-300)


COARSE = [(4, 12, 4, 3), (6, 20, 6, 4)]


def _coarse(case):
    nb, no, na, ncf = case
    return S.ates_table1(n_bore=nb, n_out=no, nz_aquifer=na, nz_confining=ncf)


def _ids(c):
    return f"bore{c[0]}_out{c[1]}_aq{c[2]}_conf{c[3]}"


@pytest.mark.parametrize("case", COARSE, ids=_ids)
def test_ates_operators_and_rhs_match_oracle(built_lib, case):
    from paper_2103_00081_gb300 import hydro
    sc = _coarse(case)
    o = fem.OracleSim(sc)
    sim = hydro.Simulator.from_scenario(sc)
    try:
        rng = np.random.default_rng(7)
        # a head with the injection's gradients, so that the heat operator
        # carries the strong advection next to the wellbore
        dt = sc.dt
        A = fem.constrain(o.head_matrix(dt), o.dmask[S.HEAD])
        h1 = fem.solve(A, o.head_rhs(dt, dt), "direct", 1e-14)
        T = sc.T0 + rng.standard_normal(sc.n_nodes)
        sim.set_state(h1, T, 0.0)
        o.h, o.T = h1.copy(), T.copy()
        x = rng.standard_normal(sc.n_nodes)
        _close(sim.apply(S.HEAD, dt, x), o.apply_head(x, dt))
        _close(sim.apply(S.TEMP, dt, x), o.apply_heat(x, h1, dt))
        _close(sim.diag(S.HEAD, dt), o.diag_head(dt))
        _close(sim.diag(S.TEMP, dt), o.diag_heat(h1, dt))
        _close(sim.rhs(S.HEAD, dt), o.head_rhs(dt, dt))
        _close(sim.rhs(S.TEMP, dt), o.heat_rhs(dt, dt, h1))
    finally:
        sim.close()


@pytest.mark.parametrize("case", COARSE, ids=_ids)
@pytest.mark.parametrize("mixed", [False, True])
def test_ates_daily_steps_match_oracle(built_lib, case, mixed):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sc = _coarse(case)
    o = fem.OracleSim(sc)
    opts = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4, max_iter=200000) if mixed else \
        dict(tol=1e-13, max_iter=200000)
    sim = hydro.Simulator.from_scenario(sc, **opts)
    try:
        for _ in range(3):
            sim.step(sc.dt)
            o.step(sc.dt)
            h, T = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
            assert _rel(h, o.h) <= 1e-9 and _rel(T, o.T) <= 1e-9, (_rel(h, o.h), _rel(T, o.T))
            np.testing.assert_allclose(T[o.pile_nodes[0]], TB, rtol=1e-13, atol=0)
    finally:
        sim.close()


TOL = 1e-10


@pytest.fixture(scope="module")
def full(built_lib):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sc = S.ates_table1()
    ro = fem.RowOracle(sc)
    sim = hydro.Simulator.from_scenario(sc, tol=TOL, precision=L.HT_MIXED, inner_tol=1e-5,
                                        inner_tol_heat=1e-4, max_iter=400000)
    yield sc, ro, sim, _rows(sc, ro)
    sim.close()


def _rows(sc, ro, n_random=96):
    """Random nodes, the wellbore rim and axis, the layer interfaces, the
    outer faces and the corners of the quarter mesh."""
    m = ro.mesh
    Nx, Ny, Nz = m.N
    rng = np.random.default_rng(0)
    rows = {int(i) for i in rng.integers(0, m.n_nodes, n_random)}
    x, _, z = sc.node_coords()
    k_aq = [int(np.argmin(np.abs(z - v))) for v in (100.0, 150.0, 200.0)]
    i_rim = int(np.searchsorted(x, 0.1))       # first node column outside r_w on an axis
    for k in k_aq + [k_aq[0] - 1, k_aq[2] + 1, 0, Nz - 1]:
        for i, j in ((0, 0), (i_rim - 1, 0), (i_rim, 0), (i_rim, i_rim), (Nx // 2, Ny // 3),
                     (Nx - 1, Ny // 2), (Nx // 2, Ny - 1), (Nx - 1, Ny - 1)):
            rows.add(int(m.node_index(i, j, k)))
    return sorted(rows)


def _check(got, ref, scale, what, tol=1e-12):
    bound = tol * np.maximum(scale, np.max(np.abs(ref)))
    bad = np.abs(got - ref) > bound
    assert not bad.any(), f"{what}: {int(bad.sum())} rows off, worst {np.max(np.abs(got - ref) / bound):.2e}"


def test_ates_full_size_operator_and_rhs_rows_match_oracle(full):
    sc, ro, sim, rows = full
    rng = np.random.default_rng(3)
    h = sc.h0 + 50.0 * rng.standard_normal(sc.n_nodes)
    T = sc.T0 + rng.standard_normal(sc.n_nodes)
    sim.set_state(h, T, 0.0)
    x = rng.standard_normal(sc.n_nodes)
    y, a = ro.apply_rows(S.HEAD, sc.dt, x, rows)
    _check(sim.apply(S.HEAD, sc.dt, x)[rows], y, a, "head apply")
    y, a = ro.apply_rows(S.TEMP, sc.dt, x, rows, h=h)
    _check(sim.apply(S.TEMP, sc.dt, x)[rows], y, a, "heat apply")
    b, a = ro.rhs_rows(S.HEAD, sc.dt, sc.dt, h, rows)
    _check(sim.rhs(S.HEAD, sc.dt)[rows], b, a, "head rhs", tol=1e-11)
    b, a = ro.rhs_rows(S.TEMP, sc.dt, sc.dt, T, rows, h=h)
    _check(sim.rhs(S.TEMP, sc.dt)[rows], b, a, "heat rhs", tol=1e-11)


def test_ates_full_size_daily_step(full):
    """One mixed-precision daily step from the initial state: the oracle's
    rows hold at the GPU solution, the wellbore is at T_b, both fields are
    symmetric about the plane x = y, and with the cell Peclet number at most
    2 the temperature stays within the geotherm's range and T_b."""
    sc, ro, sim, rows = full
    sim.set_state(sc.h0, sc.T0, 0.0)
    bh_norm = np.linalg.norm(sim.rhs(S.HEAD, sc.dt))
    st = sim.step(sc.dt)
    assert st["status"] == 0
    assert st["res_head"] <= TOL * 1.001 and st["res_heat"] <= TOL * 1.001
    h1, T1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
    b, ba = ro.rhs_rows(S.HEAD, sc.dt, sc.dt, sc.h0, rows)
    y, ya = ro.apply_rows(S.HEAD, sc.dt, h1, rows)
    assert np.all(np.abs(b - y) <= 1.01 * TOL * bh_norm + 1e-12 * (ba + ya))
    sim.set_state(h1, sc.T0, 0.0)
    bT_norm = np.linalg.norm(sim.rhs(S.TEMP, sc.dt))
    b, ba = ro.rhs_rows(S.TEMP, sc.dt, sc.dt, sc.T0, rows, h=h1)
    y, ya = ro.apply_rows(S.TEMP, sc.dt, T1, rows, h=h1)
    assert np.all(np.abs(b - y) <= 1.01 * TOL * bT_norm + 1e-12 * (ba + ya))

    np.testing.assert_allclose(T1[ro.pile_nodes[0]], TB, rtol=1e-13, atol=0)
    Nx, Ny, Nz = sc.node_dims
    for f, name in ((h1, "head"), (T1, "temperature")):
        F = f.reshape(Nz, Ny, Nx)
        # both solves stop at 1e-10 of right-hand sides dominated by the
        # storage of the whole field: the mirror image agrees to that level
        assert _rel(F.transpose(0, 2, 1), F) <= 1e-8, name
    lo, hi = sc.T0.min(), max(sc.T0.max(), TB)
    assert T1.min() >= lo - 1e-3 and T1.max() <= hi + 1e-3, (T1.min(), T1.max())
    # the injection raises the head at the wellbore rim above hydrostatic
    x, _, z = sc.node_coords()
    k = int(np.argmin(np.abs(z - 150.0)))
    i_rim = int(np.searchsorted(x, 0.1))
    assert h1.reshape(Nz, Ny, Nx)[k, 0, i_rim] > sc.h0[0] + 100.0
