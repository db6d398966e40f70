"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle on
the same seeded inputs.

Tolerances:
* operator apply / diagonal / right-hand side: relative L2 <= 1e-12 and
  max |diff| <= 1e-12 * max |y| (FP64 rounding of sums of <= 27*8 terms);
* solutions of steps solved to relative residual 1e-13: relative L2 <= 1e-9;
* FP32-inner / FP64-outer mixed precision solved to 1e-12: relative L2
  <= 1e-9 as well (the outer loop is FP64);
* Darcy flux at cell centres: 1e-12 relative;
* on meshes of one or two cells, where most rows are Dirichlet identity
  rows, the forward error of a solve at relative residual tol is bounded only
  by amp * tol (amp = ||A0^-1|| ||A0 x|| / ||x||, up to 1e9 there): those
  checks take that bound from the oracle's matrices and add a backward-error
  check of the GPU solution in the oracle's system.
Mesh sizes span several CTA tiles with ragged tails (Q1 tiles own 15 x 15
node columns, Q2 tiles 30 x 30) and several z chunks.
"""
import numpy as np
import pytest

import scenarios as S
from oracle import fem

pytestmark = pytest.mark.gpu

CASES = [
    (1, 33, 20, 7, 11),
    (2, 17, 9, 5, 12),
    (1, 1, 1, 1, 13),
    (2, 1, 1, 1, 14),
    (2, 3, 1, 2, 15),
    (1, 16, 16, 16, 16),
]


def _ids(c):
    return f"q{c[0]}_{c[1]}x{c[2]}x{c[3]}"


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _fwd_tol(o, dt, res_tol, floor=1e-9, max_nodes=1000):
    """Forward-error tolerances (head, heat) for solutions whose relative
    residual is at most res_tol, after o.step(dt).  The forward error is
    bounded by amp * res_tol with amp = ||A0^-1|| ||A0 x|| / ||x||; on the
    regular parity meshes amp is small and the floor 1e-9 applies, but on a
    mesh of one or two cells where most rows are Dirichlet identity rows amp
    reaches 1e9, so small systems take the bound computed from the oracle's
    own matrices (dense, hence the size limit)."""
    out = []
    for A, x in ((fem.constrain(o.head_matrix(dt), o.dmask[fem.HEAD]), o.h),
                 (fem.constrain(o.heat_matrix(dt, o.h), o.dmask[fem.TEMP]), o.T)):
        if A.shape[0] > max_nodes:
            out.append(floor)
            continue
        Ad = A.toarray()
        amp = np.linalg.norm(np.linalg.inv(Ad), 2) * np.linalg.norm(Ad @ x) / np.linalg.norm(x)
        out.append(max(floor, 2.0 * amp * res_tol))
    return out


def _backward(o, dt, t1, h_prev, T_prev, h1, T1):
    """Relative residuals (head, heat) of the GPU solutions h1, T1 in the
    oracle's systems of the step, built from the GPU's own previous state
    (h_prev, T_prev) and, for heat, the GPU's h1."""
    h_now, T_now = o.h, o.T
    o.h, o.T = h_prev, T_prev
    bh = o.head_rhs(dt, t1)
    bT = o.heat_rhs(dt, t1, h1)
    o.h, o.T = h_now, T_now
    rh = np.linalg.norm(bh - o.apply_head(h1, dt)) / np.linalg.norm(bh)
    rT = np.linalg.norm(bT - o.apply_heat(T1, h1, dt)) / np.linalg.norm(bT)
    return rh, rT


def _close(got, ref, tol=1e-12):
    assert _rel(got, ref) <= tol, _rel(got, ref)
    assert np.max(np.abs(got - ref)) <= tol * max(np.max(np.abs(ref)), 1e-300)


@pytest.fixture(scope="module")
def Sim(built_lib):
    from paper_2103_00081_gb300 import hydro
    return hydro.Simulator


def _scenario(case, per_cell=False, wells=2, piles=3):
    p, nx, ny, nz, seed = case
    return S.random_small(seed, nx, ny, nz, p, n_piles=piles, n_wells=wells,
                          per_cell_thermal=per_cell)


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("per_cell", [False, True])
def test_operator_apply_diag_rhs_match_oracle(Sim, case, per_cell):
    sc = _scenario(case, per_cell)
    o = fem.OracleSim(sc)
    sim = Sim.from_scenario(sc)
    rng = np.random.default_rng(100 + case[-1])
    dt = sc.dt
    x = rng.standard_normal(sc.n_nodes)
    _close(sim.apply(S.HEAD, dt, x), o.apply_head(x, dt))
    _close(sim.apply(S.TEMP, dt, x), o.apply_heat(x, o.h, dt))
    _close(sim.diag(S.HEAD, dt), o.diag_head(dt))
    _close(sim.diag(S.TEMP, dt), o.diag_heat(o.h, dt))
    _close(sim.rhs(S.HEAD, dt), o.head_rhs(dt, dt))
    _close(sim.rhs(S.TEMP, dt), o.heat_rhs(dt, dt, o.h))
    for comp, field in enumerate((S.HEAD + 2, S.HEAD + 3, S.HEAD + 4)):
        _close(sim.get_field(field), o.cell_flux()[comp])


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_two_pass_apply_variant_matches_oracle(Sim, case):
    """Operator applies through the two-pass (element buffer + node gather) kernels."""
    from paper_2103_00081_gb300 import _lib as L
    sc = _scenario(case, per_cell=True)
    o = fem.OracleSim(sc)
    sim = Sim.from_scenario(sc, apply_variant=L.HT_APPLY_TWO_PASS)
    x = np.random.default_rng(5).standard_normal(sc.n_nodes)
    _close(sim.apply(S.HEAD, sc.dt, x), o.apply_head(x, sc.dt))
    _close(sim.apply(S.TEMP, sc.dt, x), o.apply_heat(x, o.h, sc.dt))


@pytest.mark.parametrize("case", [(1, 20, 17, 9, 21), (2, 9, 16, 7, 22)], ids=_ids)
@pytest.mark.parametrize("chunks", [1, 2, 3])
def test_multi_layer_z_chunks_match_oracle(Sim, case, chunks):
    """Tiles that march through several cell layers (1-3 z chunks)."""
    sc = _scenario(case, per_cell=True)
    o = fem.OracleSim(sc)
    sim = Sim.from_scenario(sc, z_chunks=chunks)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(sc.n_nodes)
    _close(sim.apply(S.HEAD, sc.dt, x), o.apply_head(x, sc.dt))
    _close(sim.apply(S.TEMP, sc.dt, x), o.apply_heat(x, o.h, sc.dt))
    _close(sim.diag(S.TEMP, sc.dt), o.diag_heat(o.h, sc.dt))
    _close(sim.rhs(S.TEMP, sc.dt), o.heat_rhs(sc.dt, sc.dt, o.h))


@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_steps_match_oracle_fp64(Sim, case):
    sc = _scenario(case)
    o = fem.OracleSim(sc)
    sim = Sim.from_scenario(sc, tol=1e-13, max_iter=50000)
    for _ in range(3):
        st = sim.step(sc.dt)
        o.step(sc.dt)
        assert st["res_head"] <= 1.001e-13 and st["res_heat"] <= 1.001e-13
        assert _rel(sim.get_field(S.HEAD), o.h) <= 1e-9
        assert _rel(sim.get_field(S.TEMP), o.T) <= 1e-9
    assert abs(sim.time - 3 * sc.dt) < 1e-6


@pytest.mark.parametrize("case", [CASES[0], CASES[1]], ids=_ids)
def test_bicgstab_heat_solver_matches_oracle(Sim, case):
    from paper_2103_00081_gb300 import _lib as L
    sc = _scenario(case)
    o = fem.OracleSim(sc)
    sim = Sim.from_scenario(sc, tol=1e-13, krylov=L.HT_KRYLOV_BICGSTAB)
    for _ in range(2):
        sim.step(sc.dt)
        o.step(sc.dt)
    assert _rel(sim.get_field(S.TEMP), o.T) <= 1e-9


@pytest.mark.parametrize("case", [CASES[0], CASES[1]], ids=_ids)
@pytest.mark.parametrize("restart", [2, 5, 40])
def test_gmres_restart_lengths_match_oracle(Sim, case, restart):
    sc = _scenario(case)
    o = fem.OracleSim(sc)
    sim = Sim.from_scenario(sc, tol=1e-13, restart=restart, max_iter=100000)
    sim.step(sc.dt)
    o.step(sc.dt)
    assert _rel(sim.get_field(S.TEMP), o.T) <= 1e-9


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4]], ids=_ids)
@pytest.mark.parametrize("degree", [1, 3, 6])
@pytest.mark.parametrize("mixed", [False, True])
def test_chebyshev_preconditioned_cg_matches_oracle(Sim, case, degree, mixed):
    """Head CG with the Chebyshev-Jacobi polynomial preconditioner."""
    from paper_2103_00081_gb300 import _lib as L
    sc = _scenario(case)
    o = fem.OracleSim(sc)
    sim = Sim.from_scenario(sc, tol=1e-12, precond=L.HT_PREC_CHEBYSHEV, cheb_degree=degree,
                            precision=L.HT_MIXED if mixed else L.HT_FP64)
    for _ in range(2):
        st = sim.step(sc.dt)
        o.step(sc.dt)
        assert st["res_head"] <= 1e-12
        assert _rel(sim.get_field(S.HEAD), o.h) <= 1e-9
        assert _rel(sim.get_field(S.TEMP), o.T) <= 1e-9


@pytest.mark.parametrize("case", [CASES[0], CASES[1]], ids=_ids)
def test_mixed_precision_matches_oracle(Sim, case):
    sc = _scenario(case)
    o = fem.OracleSim(sc)
    from paper_2103_00081_gb300 import _lib as L
    sim = Sim.from_scenario(sc, tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4)
    for _ in range(2):
        st = sim.step(sc.dt)
        o.step(sc.dt)
        assert st["outer_head"] >= 1
        assert _rel(sim.get_field(S.HEAD), o.h) <= 1e-9
        assert _rel(sim.get_field(S.TEMP), o.T) <= 1e-9


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("mixed", [False, True])
def test_fused_two_pass_cg_steps_match_oracle(Sim, case, mixed):
    """Head CG fused into the two-pass kernels (two launches per iteration):
    the same answer as the oracle, and in FP64 the same iteration count as the
    unfused CG over the tiled apply, up to rounding (2 iterations or 2%)."""
    from paper_2103_00081_gb300 import _lib as L
    sc = _scenario(case)
    o = fem.OracleSim(sc)
    prec = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4) if mixed else dict(tol=1e-13)
    sim = Sim.from_scenario(sc, apply_variant=L.HT_APPLY_TWO_PASS, max_iter=50000, **prec)
    ref = None if mixed else Sim.from_scenario(sc, apply_variant=L.HT_APPLY_TILED, max_iter=50000, **prec)
    for _ in range(3):
        h_prev, T_prev, t1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP), o.t + sc.dt
        st = sim.step(sc.dt)
        o.step(sc.dt)
        h1, T1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
        tol_h, tol_T = _fwd_tol(o, sc.dt, prec["tol"])
        assert st["res_head"] <= prec["tol"] * 1.001
        assert _rel(h1, o.h) <= tol_h
        assert _rel(T1, o.T) <= tol_T
        rh, rT = _backward(o, sc.dt, t1, h_prev, T_prev, h1, T1)
        assert rh <= 10 * prec["tol"] and rT <= 10 * prec["tol"], (rh, rT)
        if ref is not None:
            st_ref = ref.step(sc.dt)
            assert abs(st["iters_head"] - st_ref["iters_head"]) <= max(2, 0.02 * st_ref["iters_head"])


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("mixed", [False, True])
def test_fused_two_pass_bicgstab_steps_match_oracle(Sim, case, mixed):
    """Heat BiCGStab fused into the two-pass kernels (five launches per
    iteration, wells added in the node passes): the same answer as the
    oracle, and in FP64 an iteration count close to the unfused BiCGStab over
    the tiled apply (rounding differs, so within 2 iterations or 10%)."""
    from paper_2103_00081_gb300 import _lib as L
    sc = _scenario(case)
    o = fem.OracleSim(sc)
    prec = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4) if mixed else dict(tol=1e-13)
    common = dict(krylov=L.HT_KRYLOV_BICGSTAB, max_iter=50000, **prec)
    sim = Sim.from_scenario(sc, apply_variant=L.HT_APPLY_TWO_PASS, **common)
    ref = None if mixed else Sim.from_scenario(sc, apply_variant=L.HT_APPLY_TILED, **common)
    for _ in range(2):
        h_prev, T_prev, t1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP), o.t + sc.dt
        st = sim.step(sc.dt)
        o.step(sc.dt)
        h1, T1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
        tol_h, tol_T = _fwd_tol(o, sc.dt, prec["tol"])
        assert st["res_heat"] <= prec["tol"] * 1.001
        assert _rel(h1, o.h) <= tol_h
        assert _rel(T1, o.T) <= tol_T
        rh, rT = _backward(o, sc.dt, t1, h_prev, T_prev, h1, T1)
        assert rh <= 10 * prec["tol"] and rT <= 10 * prec["tol"], (rh, rT)
        if ref is not None:
            st_ref = ref.step(sc.dt)
            assert abs(st["iters_heat"] - st_ref["iters_heat"]) <= max(2, 0.1 * st_ref["iters_heat"])


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4], CASES[5]], ids=_ids)
def test_box_heat_sources_match_oracle(Sim, case):
    """Box heat sources (flux over horizontal rectangles snapped to cell
    faces, on interior planes and on the natural top and bottom faces): the
    heat right-hand side to 1e-12 and three steps to the forward-error bound."""
    p, nx, ny, nz, seed = case
    sc = S.random_small(seed, nx, ny, nz, p, n_piles=2, n_wells=1, n_boxes=4, faces_temp=(0, 1, 2))
    o = fem.OracleSim(sc)
    tol = 1e-13
    sim = Sim.from_scenario(sc, tol=tol, max_iter=50000)
    _close(sim.rhs(S.TEMP, sc.dt), o.heat_rhs(sc.dt, sc.dt, o.h))
    for _ in range(3):
        h_prev, T_prev, t1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP), o.t + sc.dt
        st = sim.step(sc.dt)
        o.step(sc.dt)
        h1, T1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
        tol_h, tol_T = _fwd_tol(o, sc.dt, tol)
        assert st["res_heat"] <= tol * 1.001
        assert _rel(h1, o.h) <= tol_h
        assert _rel(T1, o.T) <= tol_T
        rh, rT = _backward(o, sc.dt, t1, h_prev, T_prev, h1, T1)
        assert rh <= 10 * tol and rT <= 10 * tol, (rh, rT)


def _nodal_bc_scenario(case):
    """random_small with boundary data that vary along the faces: per-node
    Dirichlet heads on x faces and a per-node recharge flux at the bottom;
    per-node Dirichlet temperatures on the x = x0 face and the top, and a
    per-node heat flux at the bottom."""
    p, nx, ny, nz, seed = case
    sc = S.random_small(seed, nx, ny, nz, p, n_piles=2, n_wells=1)
    m = fem.Mesh(sc.nx, sc.ny, sc.nz, p, sc.origin, sc.extent)
    rng = np.random.default_rng(500 + seed)

    def vals(face, lo, hi):
        return rng.uniform(lo, hi, m.face_nodes(face).size)
    sc.bc = {S.HEAD: {0: (S.DIRICHLET, vals(0, -0.3, 0.3)), 1: (S.DIRICHLET, vals(1, -0.3, 0.3)),
                      4: (S.FLUX, vals(4, -1e-7, 1e-7))},
             S.TEMP: {0: (S.DIRICHLET, vals(0, 14.0, 16.0)), 5: (S.DIRICHLET, vals(5, 10.0, 20.0)),
                      4: (S.FLUX, vals(4, 0.5, 1.5))}}
    return sc


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4]], ids=_ids)
def test_nodal_boundary_values_match_oracle(Sim, case):
    """Per-face-node Dirichlet values and interpolated per-node fluxes:
    right-hand sides to 1e-12 and three steps to the forward-error bound."""
    sc = _nodal_bc_scenario(case)
    o = fem.OracleSim(sc)
    tol = 1e-13
    sim = Sim.from_scenario(sc, tol=tol, max_iter=50000)
    _close(sim.rhs(S.HEAD, sc.dt), o.head_rhs(sc.dt, sc.dt))
    _close(sim.rhs(S.TEMP, sc.dt), o.heat_rhs(sc.dt, sc.dt, o.h))
    for _ in range(3):
        h_prev, T_prev, t1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP), o.t + sc.dt
        sim.step(sc.dt)
        o.step(sc.dt)
        h1, T1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
        tol_h, tol_T = _fwd_tol(o, sc.dt, tol)
        assert _rel(h1, o.h) <= tol_h
        assert _rel(T1, o.T) <= tol_T
        rh, rT = _backward(o, sc.dt, t1, h_prev, T_prev, h1, T1)
        assert rh <= 10 * tol and rT <= 10 * tol, (rh, rT)
    # ht_set_bc on a face drops its per-node values
    sim.set_bc(S.TEMP, 5, S.DIRICHLET, 12.0)
    T = sim.get_field(S.TEMP)
    o.sc.bc[S.TEMP][5] = (S.DIRICHLET, 12.0)
    o2 = fem.OracleSim(o.sc)
    o2.h, o2.T, o2.t = sim.get_field(S.HEAD), T, sim.time
    _close(sim.rhs(S.TEMP, sc.dt), o2.heat_rhs(sc.dt, o2.t + sc.dt, o2.h))


def test_invalid_nodal_boundary_values_are_rejected(Sim):
    from paper_2103_00081_gb300 import _lib as L
    sc = _scenario(CASES[1])
    sim = Sim.from_scenario(sc)
    Nx, Ny, Nz = sc.node_dims
    assert [sim.face_nodes(f) for f in range(6)] == [Ny * Nz] * 2 + [Nx * Nz] * 2 + [Nx * Ny] * 2
    for args in [(S.HEAD, 0, S.DIRICHLET, np.zeros(Ny * Nz - 1)),        # wrong count
                 (S.HEAD, 2, S.DIRICHLET, np.zeros(Ny * Nz)),            # count of another face
                 (S.TEMP, 4, S.NONE, np.zeros(Nx * Ny)),                 # no values for "none"
                 (S.TEMP, 4, S.FLUX, np.full(Nx * Ny, np.inf))]:         # non-finite
        with pytest.raises(RuntimeError) as e:
            sim.set_bc(*args)
        assert e.value.code == L.HT_EINVAL
    assert sim.set_bc(S.TEMP, 4, S.FLUX, np.ones(Nx * Ny)) == L.HT_OK


def test_invalid_box_sources_are_rejected(Sim):
    from paper_2103_00081_gb300 import _lib as L
    sc = _scenario(CASES[0])
    sim = Sim.from_scenario(sc)
    H = sc.extent[0] / sc.nx
    good = [0.0, 3 * H, 0.0, 5.0, 0.0, 1.0, 0.5, 1e6, 0.0]
    bad = [
        [3 * H, 0.0] + good[2:],                                  # x1 <= x0
        [1.1 * H, 1.3 * H] + good[2:],                            # both edges snap to face 1
        good[:4] + [sc.extent[2] + 1.0] + good[5:],               # plane above the box
        good[:7] + [0.0, 0.0],                                    # period 0
        good[:5] + [float("nan")] + good[6:],                     # non-finite flux
    ]
    for row in bad:
        with pytest.raises(RuntimeError) as e:
            sim.add_box_sources([row])
        assert e.value.code == L.HT_EINVAL
    assert sim.add_box_sources([good]) == L.HT_OK


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[5]], ids=_ids)
def test_float_float_outer_residual_matches_fp64(Sim, case):
    """The mixed form computes its outer residuals b - A x with the operator
    in float-float arithmetic (about 48 bits).  On the systems of a step and
    the solutions returned, that residual must equal the FP64 one to 1e-13
    relative to ||b||, equal the residual the step reported, and the FP64
    residual must meet the tolerance to within that margin; the solutions
    agree with the FP64-residual variant and the oracle."""
    from paper_2103_00081_gb300 import _lib as L
    sc = _scenario(case)
    o = fem.OracleSim(sc)
    tol = 1e-12
    common = dict(tol=tol, precision=L.HT_MIXED, inner_tol=1e-4)
    sim = Sim.from_scenario(sc, **common)
    ref = Sim.from_scenario(sc, outer_fp64=1, **common)
    dt = sc.dt
    for _ in range(2):
        t0 = sim.time
        T0 = sim.get_field(S.TEMP)
        bh = sim.rhs(S.HEAD, dt)
        st = sim.step(dt)
        ref.step(dt)
        o.step(dt)
        h1, T1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
        sim.set_state(h1, T0, t0)          # heat system of this step: T^n with h^{n+1}
        bT = sim.rhs(S.TEMP, dt)
        for field, x, b, rep in ((S.HEAD, h1, bh, st["res_head"]), (S.TEMP, T1, bT, st["res_heat"])):
            r_df = sim.residual(field, dt, x, b, emulated=True)
            r_64 = sim.residual(field, dt, x, b, emulated=False)
            assert abs(r_df - r_64) <= 1e-13, (field, r_df, r_64)
            assert abs(r_df - rep) <= 1e-15, (field, r_df, rep)
            assert r_64 <= tol + 1e-13, (field, r_64)
        sim.set_state(h1, T1, t0 + dt)
        assert _rel(h1, o.h) <= 1e-9 and _rel(T1, o.T) <= 1e-9
        assert _rel(h1, ref.get_field(S.HEAD)) <= 1e-9 and _rel(T1, ref.get_field(S.TEMP)) <= 1e-9


def test_config1_plain_workload_matches_oracle(Sim):
    """The plain FP64 workload: 16^3 Q1 cube, line source, 10 days."""
    sc = S.config1()
    o = fem.OracleSim(sc)
    sim = Sim.from_scenario(sc, tol=1e-13)
    for _ in range(sc.n_steps):
        sim.step(sc.dt)
        o.step(sc.dt)
    assert _rel(sim.get_field(S.HEAD), o.h) <= 1e-9
    assert _rel(sim.get_field(S.TEMP), o.T) <= 1e-9


def test_bitwise_reproducible(Sim):
    sc = _scenario(CASES[1])
    out = []
    for _ in range(2):
        sim = Sim.from_scenario(sc, tol=1e-10)
        for _ in range(2):
            sim.step(sc.dt)
        out.append((sim.get_field(S.HEAD), sim.get_field(S.TEMP)))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_error_codes(Sim):
    from paper_2103_00081_gb300 import hydro
    from paper_2103_00081_gb300 import _lib as L
    sc = _scenario(CASES[2])
    sim = Sim.from_scenario(sc)
    with pytest.raises(hydro.HTError) as e:
        sim.set_cells(np.zeros(sc.n_cells))
    assert e.value.code == L.HT_EINVAL
    with pytest.raises(hydro.HTError) as e:
        sim.add_line_sources([[1e6, 0, 1, 0, 1, 0, 1, 0]])
    assert e.value.code == L.HT_EINVAL
    sc2 = _scenario(CASES[0])
    sim2 = Sim.from_scenario(sc2, tol=1e-14, max_iter=1)
    st = sim2.step(sc2.dt, check=False)
    assert st["rc"] == L.HT_ENOCONV


Q1_SINGLE = [(1, 33, 20, 7, 41), (1, 57, 44, 9, 42), (1, 1, 1, 1, 43), (1, 16, 16, 16, 44), (1, 29, 21, 5, 45)]


@pytest.mark.parametrize("case", Q1_SINGLE, ids=_ids)
@pytest.mark.parametrize("faces", [(0, 1), (0, 1, 2, 3, 4, 5), (4,)])
@pytest.mark.parametrize("chunks", [0, 1, 3])
def test_single_pass_q1_cg_steps_match_oracle(Sim, case, faces, chunks):
    """The single-pass Q1 head CG (one tiled launch per iteration, the
    single-reduction form of CG with the Jacobi diagonal formed from the
    cell conductivities): mixed-precision steps match the oracle, the GPU
    solution solves the oracle's system of the step, and the inner iteration
    count stays within rounding of classical PCG over the tiled apply.  The
    tiles own at most 28 x 20 node columns, so these meshes give several
    tiles with ragged tails; chunks 0 lets the library split the planes (one
    plane per chunk on these small meshes), 1 and 3 force multi-plane chunks.
    The face sets put Dirichlet rows on x, on every face, or on the bottom."""
    from paper_2103_00081_gb300 import _lib as L
    p, nx, ny, nz, seed = case
    sc = S.random_small(seed, nx, ny, nz, p, n_piles=3, n_wells=2, faces_head=faces)
    o = fem.OracleSim(sc)
    prec = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4, max_iter=50000, z_chunks=chunks)
    sim = Sim.from_scenario(sc, apply_variant=L.HT_APPLY_SINGLE_PASS, **prec)
    ref = Sim.from_scenario(sc, apply_variant=L.HT_APPLY_TILED, **prec)
    for _ in range(3):
        h_prev, T_prev, t1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP), o.t + sc.dt
        st = sim.step(sc.dt)
        o.step(sc.dt)
        h1, T1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
        tol_h, tol_T = _fwd_tol(o, sc.dt, prec["tol"])
        assert st["res_head"] <= prec["tol"] * 1.001
        assert _rel(h1, o.h) <= tol_h
        assert _rel(T1, o.T) <= tol_T
        rh, rT = _backward(o, sc.dt, t1, h_prev, T_prev, h1, T1)
        assert rh <= 10 * prec["tol"] and rT <= 10 * prec["tol"], (rh, rT)
        st_ref = ref.step(sc.dt)
        assert abs(st["iters_head"] - st_ref["iters_head"]) <= max(3, 0.05 * st_ref["iters_head"]), \
            (st["iters_head"], st_ref["iters_head"])
    sim.close()
    ref.close()


def test_single_pass_q1_cg_reports_non_convergence(Sim):
    """An iteration limit below what the solve needs ends the single-pass CG
    with HT_ENOCONV, through the same device flags as the other solvers."""
    from paper_2103_00081_gb300 import _lib as L
    sc = S.random_small(46, 20, 18, 9, 1)
    sim = Sim.from_scenario(sc, tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4, max_iter=3,
                            apply_variant=L.HT_APPLY_SINGLE_PASS)
    st = sim.step(sc.dt, check=False)
    assert st["rc"] == L.HT_ENOCONV
    sim.close()


@pytest.mark.parametrize("case", Q1_SINGLE[:4], ids=_ids)
@pytest.mark.parametrize("per_cell", [False, True])
@pytest.mark.parametrize("chunks", [0, 2])
def test_single_pass_q1_bicgstab_steps_match_oracle(Sim, case, per_cell, chunks):
    """The single-pass Q1 heat BiCGStab (two tiled heat applies with the
    advection formed from the head at the Gauss points, then the pointwise
    update): mixed-precision steps with wells (the lumped injection term),
    piles, box heat sources and optionally per-cell lambda and c_T match the
    oracle, the GPU solution solves the oracle's heat system of the step, and
    the tiled unfused BiCGStab reaches the same solution."""
    from paper_2103_00081_gb300 import _lib as L
    p, nx, ny, nz, seed = case
    sc = S.random_small(seed, nx, ny, nz, p, n_piles=3, n_wells=2, per_cell_thermal=per_cell,
                        n_boxes=2 if nx > 1 else 0)
    # both wells spread laterally over a few cells: a line-source injection
    # well makes the Galerkin heat operator indefinite next to its axis, where
    # FP32 BiCGStab (any kernel) may stagnate or break down
    sc.wells[:, 6] = np.maximum(sc.wells[:, 6], 2.0 * max(sc.extent[0] / nx, sc.extent[1] / ny))
    o = fem.OracleSim(sc)
    prec = dict(tol=1e-12, precision=L.HT_MIXED, inner_tol=1e-4, inner_tol_heat=1e-4, max_iter=50000,
                krylov=L.HT_KRYLOV_BICGSTAB, z_chunks=chunks)
    sim = Sim.from_scenario(sc, apply_variant=L.HT_APPLY_SINGLE_PASS, **prec)
    ref = Sim.from_scenario(sc, apply_variant=L.HT_APPLY_TILED, **prec)
    for _ in range(3):
        h_prev, T_prev, t1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP), o.t + sc.dt
        st = sim.step(sc.dt)
        o.step(sc.dt)
        h1, T1 = sim.get_field(S.HEAD), sim.get_field(S.TEMP)
        tol_h, tol_T = _fwd_tol(o, sc.dt, prec["tol"])
        assert st["res_heat"] <= prec["tol"] * 1.001
        assert _rel(h1, o.h) <= tol_h
        assert _rel(T1, o.T) <= tol_T
        rh, rT = _backward(o, sc.dt, t1, h_prev, T_prev, h1, T1)
        assert rh <= 10 * prec["tol"] and rT <= 10 * prec["tol"], (rh, rT)
        # the tiled unfused BiCGStab reaches the same solution (its iteration
        # count is not compared: near the wells these heat systems are far from
        # normal, and BiCGStab's count there depends on rounding)
        ref.step(sc.dt)
        assert _rel(ref.get_field(S.TEMP), T1) <= 2 * tol_T
    sim.close()
    ref.close()
