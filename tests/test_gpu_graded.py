"""Graded tensor-product meshes (Fig. 10b) in the library, against the
oracle's graded mesh (`fem.Mesh(..., spacing=...)`): every geometric
quantity per cell.  Tolerances as in test_gpu_parity: operator, diagonal and
right-hand side 1e-12, steps solved to 1e-13 (FP64) or 1e-12 (mixed)
relative residual 1e-9."""
import math

import numpy as np
import pytest

import scenarios as S
from oracle import fem

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _close(got, ref, tol=1e-12):
    assert _rel(got, ref) <= tol, _rel(got, ref)
    assert np.max(np.abs(got - ref)) <= tol * max(np.max(np.abs(ref)), 1e-300)


def _graded(p, n, seed, stretch=(0.8, -0.6, 1.1), boxes=1, per_cell=True):
    """A random small problem on a graded mesh: widths from a smooth map
    (cells finer at one end), lognormal K, piles, spread and line wells, a
    box heat source and per-cell thermal data."""
    nx, ny, nz = n
    sc = S.random_small(seed, nx, ny, nz, p, n_wells=2, per_cell_thermal=per_cell, n_boxes=boxes,
                        extent=(40.0, 30.0, 20.0))
    sc.spacing = tuple(S.graded_widths(m, L, a) for m, L, a in zip(n, sc.extent, stretch))
    return sc


CASES = [(1, (13, 9, 7), 21), (2, (7, 5, 4), 22), (1, (30, 17, 9), 23)]


def _ids(c):
    return f"q{c[0]}_{c[1][0]}x{c[1][1]}x{c[1][2]}"


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_graded_operator_diag_rhs_match_oracle(built_lib, case):
    from paper_2103_00081_gb300 import hydro
    p, n, seed = case
    sc = _graded(p, n, seed)
    o = fem.OracleSim(sc)
    sim = hydro.Simulator.from_scenario(sc)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(sc.n_nodes)
    dt = sc.dt
    _close(sim.apply(S.HEAD, dt, x), o.apply_head(x, dt))
    _close(sim.apply(S.TEMP, dt, x), o.apply_heat(x, o.h, dt))
    _close(sim.diag(S.HEAD, dt), o.diag_head(dt))
    _close(sim.diag(S.TEMP, dt), o.diag_heat(o.h, dt))
    _close(sim.rhs(S.HEAD, dt), o.head_rhs(dt, dt))
    _close(sim.rhs(S.TEMP, dt), o.heat_rhs(dt, dt, o.h))
    for comp, field in enumerate((S.HEAD + 2, S.HEAD + 3, S.HEAD + 4)):
        _close(sim.get_field(field), o.cell_flux()[comp])


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("mixed", [False, True])
def test_graded_steps_match_oracle(built_lib, case, mixed):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    p, n, seed = case
    sc = _graded(p, n, seed)
    o = fem.OracleSim(sc)
    opts = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4) if mixed else dict(tol=1e-13)
    sim = hydro.Simulator.from_scenario(sc, **opts)
    for _ in range(3):
        sim.step(sc.dt)
        o.step(sc.dt)
        assert _rel(sim.get_field(S.HEAD), o.h) <= 1e-9
        assert _rel(sim.get_field(S.TEMP), o.T) <= 1e-9


def test_equal_widths_reproduce_the_uniform_mesh(built_lib):
    """Widths all equal to the uniform cell size: the graded kernels give the
    uniform kernels' operator and step."""
    from paper_2103_00081_gb300 import hydro
    sc = S.random_small(31, 11, 8, 6, 2, n_wells=1, extent=(40.0, 30.0, 20.0))
    uni = hydro.Simulator.from_scenario(sc, tol=1e-13)
    sc.spacing = tuple(np.full(m, L / m) for m, L in zip((11, 8, 6), sc.extent))
    gr = hydro.Simulator.from_scenario(sc, tol=1e-13)
    x = np.random.default_rng(3).standard_normal(sc.n_nodes)
    _close(gr.apply(S.HEAD, sc.dt, x), uni.apply(S.HEAD, sc.dt, x))
    _close(gr.apply(S.TEMP, sc.dt, x), uni.apply(S.TEMP, sc.dt, x))
    gr.step(sc.dt)
    uni.step(sc.dt)
    assert _rel(gr.get_field(S.TEMP), uni.get_field(S.TEMP)) <= 1e-10


def _mms(p, n, stretch=(0.7, -0.7, 0.5)):
    """The steady head problem of the oracle's graded manufactured-solution
    pin: -div(K grad h) = f with h = sin(x) cos(0.7 y) exp(0.3 z) as per-node
    Dirichlet data on all faces (storage 1e-12 in place of zero, which the
    library rejects), and its quadrature for the L2 error."""
    L = (1.0, 1.2, 0.9)
    sc = S.config1(nx=n, ny=n, nz=n, order=p)
    sc.extent = L
    sc.spacing = tuple(S.graded_widths(n, Ld, a) for Ld, a in zip(L, stretch))
    sc.piles = np.zeros((0, 8))
    Kh = 2e-5
    sc.K = np.full(sc.n_cells, Kh)
    sc.Ss = 1e-12
    m = fem.Mesh(n, n, n, p, (0, 0, 0), L, sc.spacing)
    X, Y, Z = m.node_xyz()

    def u(x, y, z):
        return np.sin(x) * np.cos(0.7 * y) * np.exp(0.3 * z)
    lap = -1.0 - 0.49 + 0.09
    sc.bc = {S.HEAD: {f: (S.DIRICHLET, u(X, Y, Z)[m.face_nodes(f)]) for f in range(6)}, S.TEMP: {}}
    sc.h0 = np.zeros(m.n_nodes)
    sc.T0 = np.zeros(m.n_nodes)
    xq, _ = fem.gauss01(5)
    F = np.zeros(m.n_nodes)
    hw = m.cell_widths()
    Nq, _, W1 = fem.reference_element(p, (1.0, 1.0, 1.0), nq=5)
    quad = []
    for c in range(m.n_cells):
        cx, cy, cz = c % n, (c // n) % n, c // (n * n)
        Wq = W1 * np.prod(hw[c])
        lo = (m.faces[0][cx], m.faces[1][cy], m.faces[2][cz])
        P_ = np.array([(lo[0] + hw[c, 0] * xq[qx], lo[1] + hw[c, 1] * xq[qy], lo[2] + hw[c, 2] * xq[qz])
                       for qz in range(5) for qy in range(5) for qx in range(5)])
        fq = -Kh * lap * u(P_[:, 0], P_[:, 1], P_[:, 2])
        F[m.conn[c]] += np.einsum("q,ql,q->l", Wq, Nq, fq)
        quad.append((c, Nq, Wq, u(P_[:, 0], P_[:, 1], P_[:, 2])))

    def err(h):
        return math.sqrt(sum(np.sum(Wq * (Nq @ h[m.conn[c]] - uq) ** 2) for c, Nq, Wq, uq in quad))
    return sc, F, err


@pytest.mark.parametrize("p", [1, 2])
def test_graded_manufactured_solution_matches_oracle_and_converges(built_lib, p):
    """The graded MMS meshes of the oracle pin: the GPU solution equals the
    oracle's to 1e-9 at two refinements of the same smooth graded map, and
    its L2 error falls at order p + 1."""
    from paper_2103_00081_gb300 import hydro
    errs = []
    for n in (3, 6):
        sc, F, err = _mms(p, n)
        o = fem.OracleSim(sc)
        o.extra[S.HEAD] = F
        o.step(sc.dt)
        sim = hydro.Simulator.from_scenario(sc, tol=1e-13)
        sim.set_extra_rhs(S.HEAD, F)
        sim.step(sc.dt)
        h = sim.get_field(S.HEAD)
        assert _rel(h, o.h) <= 1e-9, _rel(h, o.h)
        errs.append(err(h))
    order = math.log(errs[0] / errs[1]) / math.log(2.0)
    assert order > p + 1 - 0.35, (errs, order)


def test_graded_mesh_rejects_bad_spacing_and_uniform_only_modes(built_lib):
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro
    sc = _graded(1, (6, 5, 4), 41, boxes=0, per_cell=False)
    sim = hydro.Simulator.from_scenario(sc, precision=L.HT_MIXED)
    for axis, w in [(3, np.ones(6)), (0, np.ones(5)), (0, np.r_[np.ones(5), -1.0]), (1, np.r_[np.ones(4), 0.0])]:
        with pytest.raises(hydro.HTError):
            sim.set_spacing(axis, w)
    with pytest.raises(hydro.HTError):
        hydro.Batch([sim], mode=L.HT_BATCH_PERSISTENT)
    b = hydro.Batch([sim], mode=L.HT_BATCH_SHARED_LAUNCHES)
    with pytest.raises(hydro.HTError):
        b.step(sc.dt)
    b.close()
