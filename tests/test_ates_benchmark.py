"""The hot-water injection benchmark of Section 2 (Fig. 2, Table 1) as a
box-mesh workload (scenarios.ates_table1), pinned on the CPU oracle by what
the physics fixes for it:

* the generator keeps the cell Peclet number c_w |q| H / lambda <= 2 outside
  the wellbore, where the plain Galerkin heat operator of Eq. 4 needs no
  stabilisation;
* the steady head around the wellbore is Thiem's logarithm,
  h(r1) - h(r2) = Q / (2 pi K b) ln(r2 / r1), with Q = Q_b 2 pi r_w b the whole
  well's rate (the quarter mesh carries a quarter of it on the axis);
* the early transient head is Theis' well function,
  s(r, t) = Q / (4 pi K b) E1(r^2 S_s / (4 K t)), which pins S_s = rho_w g / B_poro
  of Eq. 1 and the time stepping;
* the quarter problem is mirror-symmetric in x <-> y, and the wellbore
  nodes hold T_b.

COMSOL's curves (Figs. 3-6) are figure-only; these closed forms replace
them."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spl
from scipy.special import exp1

import scenarios as S
from oracle import fem

T1 = S.ATES_TABLE1
B = 100.0            # aquifer thickness of the generator's default layering
Q_WELL = T1["Q_b"] * 2.0 * math.pi * 0.1 * B
TRANS = 1.0e-6 * B   # transmissivity K b


def _midplane(sc, h):
    x, _, z = sc.node_coords()
    Nx, Ny, Nz = sc.node_dims
    k = int(np.argmin(np.abs(z - 150.0)))
    return x, h.reshape(Nz, Ny, Nx)[k]


def test_default_mesh_keeps_the_cell_peclet_number_at_most_two():
    sc = S.ates_table1()
    wx, wy, wz = sc.spacing
    assert np.allclose(wx, wy) and abs(wx.sum() - 20.0) < 1e-9 and abs(wz.sum() - 300.0) < 1e-9
    x = np.concatenate([[0.0], np.cumsum(wx)])
    xc = 0.5 * (x[1:] + x[:-1])
    r = np.hypot(xc[:, None], xc[None, :])
    H = np.maximum(wx[:, None], wx[None, :])
    out = r > 0.1
    q = T1["Q_b"] * 0.1 / r[out]          # radial flux outside the wellbore
    Pe = T1["c_w"] * q * H[out] / T1["lam"]
    assert Pe.max() <= 2.0
    # the wellbore row covers the aquifer and its radius, the well a quarter rate
    assert sc.pile_temps.shape == (1, 9) and sc.pile_temps[0, 4] == 0.1
    assert sc.wells[0, 4] == pytest.approx(Q_WELL / 4.0, rel=1e-15)
    # K: 1e-6 in the aquifer (100 < z < 200), 1e-10 above and below
    zf = np.concatenate([[0.0], np.cumsum(wz)])
    zc = 0.5 * (zf[1:] + zf[:-1])
    Kz = sc.K.reshape(sc.nz, sc.ny, sc.nx)[:, 0, 0]
    np.testing.assert_array_equal(Kz, np.where((zc > 100) & (zc < 200), 1e-6, 1e-10))


@pytest.mark.parametrize("n_bore,n_out,tol", [(4, 20, 4e-3), (6, 30, 2e-3), (8, 40, 1e-3)])
def test_steady_head_follows_thiem(n_bore, n_out, tol):
    """One step of 1e13 s leaves the storage term negligible: the head in
    the aquifer is the steady radial flow of the well.  The outer square at
    20 m adds a harmonic term of fourfold symmetry, O((r/R)^4) at r <= 5 m."""
    sc = S.ates_table1(n_bore=n_bore, n_out=n_out, nz_aquifer=2, nz_confining=2)
    o = fem.OracleSim(sc)
    dt = 1e13
    A = fem.constrain(o.head_matrix(dt), o.dmask[S.HEAD])
    h = fem.solve(A, o.head_rhs(dt, dt), "direct", 1e-14)
    x, H = _midplane(sc, h)
    i1, i2 = int(np.argmin(np.abs(x - 0.5))), int(np.argmin(np.abs(x - 5.0)))
    thiem = Q_WELL / (2 * math.pi * TRANS) * math.log(x[i2] / x[i1])
    assert abs((H[0, i1] - H[0, i2]) / thiem - 1.0) <= tol
    # the same along the diagonal
    j1 = int(np.argmin(np.abs(x - 0.5 / math.sqrt(2))))
    j2 = int(np.argmin(np.abs(x - 5.0 / math.sqrt(2))))
    thiem_d = Q_WELL / (2 * math.pi * TRANS) * math.log(x[j2] / x[j1])
    assert abs((H[j1, j1] - H[j2, j2]) / thiem_d - 1.0) <= 1.5 * tol
    assert np.max(np.abs(H - H.T)) <= 1e-12 * np.max(np.abs(H))


def test_early_head_follows_theis():
    """Half a day in 48 backward Euler steps: the head rise at 0.5 m and 0.9 m
    from the axis is Theis' E1 within 1 %.  A wrong storage coefficient, a
    full rate on the quarter mesh or a step that drops the storage term of
    Eq. 3 misses it by tens of percent."""
    sc = S.ates_table1(n_bore=6, n_out=30, nz_aquifer=2, nz_confining=2)
    o = fem.OracleSim(sc)
    n, tend = 48, 0.5 * S.DAY
    dt = tend / n
    lu = spl.splu(fem.constrain(o.head_matrix(dt), o.dmask[S.HEAD]).tocsc())
    for k in range(n):
        o.h = lu.solve(o.head_rhs(dt, (k + 1) * dt))
    x, H = _midplane(sc, o.h)
    Ss = S.RHO_W * S.G_ACC / T1["B_poro"]
    for r in (0.5, 0.9):
        i = int(np.argmin(np.abs(x - r)))
        theis = Q_WELL / (4 * math.pi * TRANS) * exp1(x[i] ** 2 * Ss * B / (4 * TRANS * tend))
        assert abs((H[0, i] - sc.h0[0]) / theis - 1.0) <= 0.01, (r, (H[0, i] - sc.h0[0]) / theis)


def test_daily_steps_are_symmetric_and_hold_the_wellbore_at_t_b():
    sc = S.ates_table1(n_bore=4, n_out=12, nz_aquifer=4, nz_confining=3)
    o = fem.OracleSim(sc)
    bore = o.pile_nodes[0]
    x, y, z = sc.node_coords()
    Nx, Ny, Nz = sc.node_dims
    X = np.tile(x, Ny * Nz)
    Y = np.tile(np.repeat(y, Nx), Nz)
    Z = np.repeat(z, Nx * Ny)
    sel = np.hypot(X, Y) <= 0.1 + 1e-9
    np.testing.assert_array_equal(np.sort(bore), np.nonzero(sel & (Z >= 100 - 1e-9) & (Z <= 200 + 1e-9))[0])
    for _ in range(2):
        o.step(sc.dt)
        np.testing.assert_allclose(o.T[bore], T1["T_b"], rtol=1e-14)
        for f in (o.h, o.T):
            F = f.reshape(Nz, Ny, Nx)
            assert np.max(np.abs(F - F.transpose(0, 2, 1))) <= 1e-11 * np.max(np.abs(F))
    # injection raises the head around the well above its hydrostatic value
    _, H = _midplane(sc, o.h)
    assert H[0, 1] > sc.h0[0] + 10.0
