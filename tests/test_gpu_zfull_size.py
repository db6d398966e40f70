"""Parity at the full sizes of the step benchmark's workloads, with the
solver options the benchmark times (mixed precision; on Q1 the single-pass
head CG, on Q2 the two-pass fused kernels; BiCGStab for heat):

* city_q1: 512 x 512 x 96 Q1 (25,527,393 nodes per field), layered + GRF lnK,
  20,000 piles and 50 box heat sources -- the benchmark's default workload;
* pile_q1: 256 x 256 x 64 Q1 (4,293,185 nodes), GRF lnK, 1000 piles;
* ates_q2: 128 x 128 x 32 Q2 (4,293,185 nodes), lognormal layers, two wells.

The oracle cannot assemble these meshes, so it computes sampled rows one by
one (``fem.RowOracle``, itself checked against the assembled oracle at every
row of small meshes).  The samples cover random nodes, every face and the
layer next to it (Dirichlet rows and lifted rows), the corners, the K layer
interfaces, nodes carrying pile, box or well loads, and the nodes of largest
load.

* FP64 operator rows (the tiled kernels of the plain FP64 leg): |diff| <=
  1e-12 times the larger of the row's sum of absolute terms and the largest
  sampled value (FP64 rounding of <= 125 terms summed in another order).
* Right-hand-side rows (float-float for cells without Dirichlet nodes):
  the same with 1e-11.
* One mixed-precision step: the solver stops at ||b - A x||_2 <= tol ||b||_2,
  so every row of the oracle's residual at the GPU solution obeys
  |r_i| <= tol ||b||_2, up to the float-float residual's 1e-13 and rounding.
"""
import numpy as np
import pytest

import scenarios as S
from oracle import fem

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _layer_planes(sc):
    """Node planes at and beside the cell-layer interfaces of the K layering."""
    if sc.name.startswith("ates"):
        nb = int(round(sc.nz * 10 / 32))
        return [nb, sc.nz - nb]
    if sc.name.startswith("city"):
        zc = (np.arange(sc.nz) + 0.5) / sc.nz
        bounds = np.cumsum([f for _, f, _ in S.CITY_LAYERS])
        lay = np.searchsorted(bounds, zc, side="right")
        return [int(k) for k in np.nonzero(np.diff(lay))[0] + 1]
    return [sc.nz // 2]


def _rows(sc, ro, n_random=96, seed=0):
    m = ro.mesh
    Nx, Ny, Nz = m.N
    rng = np.random.default_rng(seed)
    rows = {int(i) for i in rng.integers(0, m.n_nodes, n_random)}
    mid = (Nx // 2, Ny // 2, Nz // 2)
    for axis, last in ((0, Nx - 1), (1, Ny - 1), (2, Nz - 1)):
        for v in (0, 1, last - 1, last):
            ijk = list(mid)
            ijk[axis] = v
            rows.add(int(m.node_index(*ijk)))
    for i in (0, Nx - 1):
        for j in (0, Ny - 1):
            for k in (0, Nz - 1):
                rows.add(int(m.node_index(i, j, k)))
    for kc in _layer_planes(sc):
        for k in (m.p * kc - 1, m.p * kc, m.p * kc + 1):
            rows.add(int(m.node_index(Nx // 3, 2 * Ny // 3, k)))
    # nodes of the first piles and boxes, the wells and the largest head loads
    for w in ro.pile_w[:4] + ro.box_w[:2]:
        keys = sorted(w)
        rows.update(int(keys[i]) for i in rng.integers(0, len(keys), min(6, len(keys))))
    rows.update(int(i) for i in np.argsort(ro.d_well)[-8:])
    rows.update(int(i) for i in np.argsort(np.abs(ro.F_static[fem.HEAD]))[-8:])
    return sorted(rows)


WORKLOADS = {"city_q1": S.config5, "pile_q1": S.config3, "ates_q2": S.config2}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def full(request, built_lib):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sc = WORKLOADS[request.param]()
    ro = fem.RowOracle(sc)
    variant = L.HT_APPLY_SINGLE_PASS if sc.order == 1 else L.HT_APPLY_TWO_PASS
    sim = hydro.Simulator.from_scenario(
        sc, tol=TOL, precision=L.HT_MIXED, inner_tol=1e-5, inner_tol_heat=1e-4, max_iter=200000,
        apply_variant=variant, krylov=L.HT_KRYLOV_BICGSTAB, precond=L.HT_PREC_JACOBI)
    yield sc, ro, sim, _rows(sc, ro)
    sim.close()


def _check(got, ref, scale, what, tol=1e-12):
    """|diff| <= tol times the larger of the row's sum of absolute terms and
    the largest sampled |ref| (the bound of the small-mesh parity tests)."""
    bound = tol * np.maximum(scale, np.max(np.abs(ref)))
    bad = np.abs(got - ref) > bound
    assert not bad.any(), f"{what}: {int(bad.sum())} rows off, worst {np.max(np.abs(got - ref) / bound):.2e} of the bound"


def _test_state(sc):
    """A head with gradients everywhere (so that the heat operator carries
    advection in every cell) and a perturbed temperature."""
    rng = np.random.default_rng(3)
    return 0.5 * rng.standard_normal(sc.n_nodes), sc.T0 + rng.standard_normal(sc.n_nodes)


def test_full_size_operator_rows_match_oracle(full):
    """FP64 operator applies in the launch configuration of the benchmark's
    plain FP64 leg (the tiled kernels)."""
    from paper_2103_00081_gb300 import hydro
    sc, ro, _, rows = full
    h, T = _test_state(sc)
    sim64 = hydro.Simulator.from_scenario(sc, tol=TOL)
    try:
        sim64.set_state(h, T, 0.0)
        x = np.random.default_rng(1).standard_normal(sc.n_nodes)
        y, a = ro.apply_rows(S.HEAD, sc.dt, x, rows)
        _check(sim64.apply(S.HEAD, sc.dt, x)[rows], y, a, "head apply")
        y, a = ro.apply_rows(S.TEMP, sc.dt, x, rows, h=h)
        _check(sim64.apply(S.TEMP, sc.dt, x)[rows], y, a, "heat apply")
    finally:
        sim64.close()


def test_full_size_rhs_rows_match_oracle(full):
    """Right-hand sides as the benchmark's step forms them: cells without
    Dirichlet nodes in float-float (48-bit significands), so the bound is
    1e-11 (about 216 float-float operations per row, each within 2^-47)."""
    sc, ro, sim, rows = full
    h, T = _test_state(sc)
    sim.set_state(h, T, 0.0)
    b, a = ro.rhs_rows(S.HEAD, sc.dt, sc.dt, h, rows)
    _check(sim.rhs(S.HEAD, sc.dt)[rows], b, a, "head rhs", tol=1e-11)
    b, a = ro.rhs_rows(S.TEMP, sc.dt, sc.dt, T, rows, h=h)
    _check(sim.rhs(S.TEMP, sc.dt)[rows], b, a, "heat rhs", tol=1e-11)


def test_full_size_mixed_step_solves_the_oracle_rows(full):
    """The benchmark's step (FP32 fused inner solves, FP64 / float-float outer
    loop): the GPU solution satisfies the oracle's rows of both systems to the
    solver tolerance."""
    sc, ro, sim, rows = full
    sim.set_state(sc.h0, sc.T0, 0.0)
    bh_norm = np.linalg.norm(sim.rhs(S.HEAD, sc.dt))
    st = sim.step(sc.dt)
    assert st["status"] == 0
    assert st["res_head"] <= TOL * 1.001 and st["res_heat"] <= TOL * 1.001
    h1, T1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
    b, ba = ro.rhs_rows(S.HEAD, sc.dt, sc.dt, sc.h0, rows)
    y, ya = ro.apply_rows(S.HEAD, sc.dt, h1, rows)
    r = np.abs(b - y)
    assert np.all(r <= 1.01 * TOL * bh_norm + 1e-12 * (ba + ya)), np.max(r) / bh_norm
    # heat: the system of the step, with the Darcy flux of the GPU's h^{n+1}
    sim.set_state(h1, sc.T0, 0.0)
    bT_norm = np.linalg.norm(sim.rhs(S.TEMP, sc.dt))
    b, ba = ro.rhs_rows(S.TEMP, sc.dt, sc.dt, sc.T0, rows, h=h1)
    y, ya = ro.apply_rows(S.TEMP, sc.dt, T1, rows, h=h1)
    r = np.abs(b - y)
    assert np.all(r <= 1.01 * TOL * bT_norm + 1e-12 * (ba + ya)), np.max(r) / bT_norm
