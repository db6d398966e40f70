"""Pins of the CPU oracle against mathematics it does not contain.

Each test checks the oracle (``oracle.fem``) against something fixed outside
it: textbook 1D element matrices, exact symbolic integrals, discrete
eigen-solutions, exact reproduction of linear heads, conservation, and the
erfc / Ogata-Banks analytic solutions.  A dropped term, a wrong sign, a wrong
index order or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import closed_forms as cf
from oracle import fem
import scenarios as S


def _lam(sc):
    """Bulk thermal conductivity of a scenario (the oracle's mixture rule)."""
    return fem.bulk_properties(sc)[0]


def _cT(sc):
    """Bulk volumetric heat capacity of a scenario (the oracle's mixture rule)."""
    return fem.bulk_properties(sc)[1]


def test_mixture_rules_and_storage_match_hand_values():
    """The Section 2 mixture rules for the sand of the workloads (phi 0.3,
    lambda_s 2.5, lambda_w 0.6, c_s 2e6, c_w 4.18e6) worked by hand:
    0.7 * 2.5 + 0.3 * 0.6 = 1.93 and 0.7 * 2e6 + 0.3 * 4.18e6 = 2.654e6; the
    storage of Eq. 1 with Table 1's B_poro: 1000 * 9.81 / 1e5 = 0.0981."""
    lam, cT = fem.mixture(0.3, 2.5, 0.6, 2.0e6, 4.18e6)
    assert abs(lam - 1.93) < 1e-14 and abs(cT - 2.654e6) < 1e-8
    assert fem.mixture(0.0, 2.5, 0.6, 2.0e6, 4.18e6) == (2.5, 2.0e6)       # no pores: the solid
    assert fem.mixture(1.0, 2.5, 0.6, 2.0e6, 4.18e6) == (0.6, 4.18e6)      # all water
    assert abs(fem.specific_storage(1.0e5) - 0.0981) < 1e-16
    sc = S.config1(nx=2)
    assert fem.bulk_properties(sc)[:3] == (*fem.mixture(0.3, 2.5, 0.6, 2.0e6, 4.18e6), 4.18e6)
    sc.lam, sc.cT, sc.Ss = 2.2, 2.5e6, 0.0           # bulk values given directly win
    assert fem.bulk_properties(sc) == (2.2, 2.5e6, 4.18e6, 0.0)

def _kron3(Ax, Ay, Az):
    # local node l = a + n*(b + n*c): x fastest -> kron(z, kron(y, x))
    return np.kron(Az, np.kron(Ay, Ax))


def _m1(p, H):
    if p == 1:
        return H / 6.0 * np.array([[2, 1], [1, 2]], dtype=float)
    return H / 30.0 * np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]], dtype=float)


def _k1(p, H):
    if p == 1:
        return 1.0 / H * np.array([[1, -1], [-1, 1]], dtype=float)
    return 1.0 / (3.0 * H) * np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]], dtype=float)


@pytest.mark.parametrize("p", [1, 2])
def test_element_matrices_are_tensor_products_of_textbook_1d(p):
    """Reference mass / stiffness equal the tensor products of the standard
    1D Lagrange element matrices (Q1: H/6[2 1;1 2], 1/H[1 -1;-1 1];
    Q2: H/30[4 2 -1;2 16 2;-1 2 4], 1/(3H)[7 -8 1;-8 16 -8;1 -8 7])."""
    H = (1.3, 0.7, 2.1)
    N, G, W = fem.reference_element(p, H)
    Me = fem.element_mass(N, W)
    Ke = fem.element_stiffness(G, W)
    Mx, My, Mz = (_m1(p, h) for h in H)
    Kx, Ky, Kz = (_k1(p, h) for h in H)
    np.testing.assert_allclose(Me, _kron3(Mx, My, Mz), rtol=1e-13, atol=1e-15)
    Kref = _kron3(Kx, My, Mz) + _kron3(Mx, Ky, Mz) + _kron3(Mx, My, Kz)
    np.testing.assert_allclose(Ke, Kref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2])
def test_advection_element_matches_symbolic_integral(p):
    """C_lm = c_w int N_l (q . grad N_m), q = -K grad h, integrated exactly by
    sympy on one cell.  For Q1 (any h) and Q2 with a trilinear h the Gauss
    rule of the oracle is exact, so the two must agree to rounding."""
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    H = (1.5, 0.8, 1.1)
    n = p + 1
    nodes = [sympy.Rational(i, p) for i in range(n)]

    def lag(a, s):
        e = sympy.Integer(1)
        for m in range(n):
            if m != a:
                e *= (s - nodes[m]) / (nodes[a] - nodes[m])
        return e

    rng = np.random.default_rng(7)
    # h trilinear in physical coordinates
    hc = [sympy.Rational(int(v), 64) for v in rng.integers(-64, 64, 8)]
    H = tuple(sympy.Rational(v).limit_denominator(100) for v in H)
    X, Y, Z = x * H[0], y * H[1], z * H[2]
    h_expr = (hc[0] + hc[1] * X + hc[2] * Y + hc[3] * Z + hc[4] * X * Y + hc[5] * Y * Z
              + hc[6] * X * Z + hc[7] * X * Y * Z)
    Kc, cw = sympy.Rational(23, 100000), 4180000
    gh = [sympy.diff(h_expr, v) / H[i] for i, v in enumerate((x, y, z))]
    q = [-Kc * g for g in gh]
    shapes = []
    for c in range(n):
        for b in range(n):
            for a in range(n):
                shapes.append(lag(a, x) * lag(b, y) * lag(c, z))
    Hf = tuple(float(v) for v in H)
    N, G, W = fem.reference_element(p, Hf)
    mesh = fem.Mesh(1, 1, 1, p, (0, 0, 0), Hf)
    # nodal h: evaluate h at the element nodes
    xs = [float(v) for v in nodes]
    hn = np.zeros(n ** 3)
    for c in range(n):
        for b in range(n):
            for a in range(n):
                hn[a + n * (b + n * c)] = float(h_expr.subs({x: xs[a], y: xs[b], z: xs[c]}))
    qf = fem.darcy_at_qp(mesh, np.array([float(Kc)]), G, hn)
    Ce = fem.advection_elements(N, G, W, qf, float(cw))[0]
    vol = H[0] * H[1] * H[2]
    stride_l, stride_m = (3, 2) if p == 1 else (7, 9)
    for l in range(0, n ** 3, stride_l):
        for m in range(1, n ** 3, stride_m):
            dN = [sympy.diff(shapes[m], v) / H[i] for i, v in enumerate((x, y, z))]
            integrand = cw * shapes[l] * sum(qq * d for qq, d in zip(q, dN)) * vol
            exact = float(sympy.integrate(integrand, (x, 0, 1), (y, 0, 1), (z, 0, 1)))
            assert abs(Ce[l, m] - exact) <= 1e-10 * max(1.0, abs(exact)), (l, m, Ce[l, m], exact)


@pytest.mark.parametrize("p", [1, 2])
def test_row_sums_symmetry_and_definiteness(p):
    sc = S.random_small(3, 3, 2, 2, p, n_piles=0, n_wells=0)
    o = fem.OracleSim(sc)
    one = np.ones(o.mesh.n_nodes)
    # constants lie in the kernel of stiffness and advection
    assert np.max(np.abs(o.KK @ one)) < 1e-12 * np.max(np.abs(o.KK.data))
    qf = fem.darcy_at_qp(o.mesh, o.K, o.G, o.h)
    C = fem.assemble(o.mesh, np.ones(o.mesh.n_cells),
                     fem.advection_elements(o.N, o.G, o.W, qf, o.cw))
    assert np.max(np.abs(C @ one)) < 1e-10 * np.max(np.abs(C.data))
    # mass integrates the constant exactly: sum of entries = volume
    vol = np.prod(sc.extent)
    assert abs(o.M.sum() - vol) < 1e-11 * vol
    # head operator symmetric positive definite (constrained form too)
    A = fem.constrain(o.head_matrix(S.DAY), o.dmask[S.HEAD]).toarray()
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("layered", [False, True])
def test_linear_head_is_reproduced_exactly(p, layered):
    """Q1/Q2 contain linear functions: with K uniform, or varying only in z,
    and a head gradient along x fixed on the x faces, the discrete head stays
    exactly linear and q_x = -K(z) dh/dx (Darcy's law, Section 2)."""
    sc = S.config1(nx=4, ny=3, nz=5, order=p, n_steps=2)
    sc.piles = np.zeros((0, 8))
    if layered:
        kz = np.exp(np.linspace(-12, -8, sc.nz))
        sc.K = np.repeat(kz, sc.nx * sc.ny)
    o = fem.OracleSim(sc)
    x, _, _ = o.mesh.node_xyz()
    exact = 0.2 - 0.01 * x
    o.h[:] = exact + 0.0   # start on the linear solution
    for _ in range(2):
        o.step(sc.dt)
        np.testing.assert_allclose(o.h, exact, rtol=0, atol=1e-12)
    q = o.cell_flux()
    np.testing.assert_allclose(q[0], 0.01 * sc.K, rtol=1e-10)
    np.testing.assert_allclose(q[1:], 0.0, atol=1e-15)


def _all_dirichlet(value):
    return {f: (S.DIRICHLET, value) for f in range(6)}


@pytest.mark.parametrize("field", ["heat", "head"])
def test_discrete_sine_mode_decays_by_closed_form_factor(field):
    """Q1, homogeneous Dirichlet on all faces, no flow: the sine mode is a
    discrete eigenvector, T^n = T^0 / (1 + dt a sum_d mu_d)^n exactly, with
    a = lambda / c_T (heat) or K / S_s (head)."""
    sc = S.config1(nx=6, ny=5, nz=4, order=1)
    sc.extent = (12.0, 7.0, 5.0)
    sc.piles = np.zeros((0, 8))
    o_mesh = fem.Mesh(sc.nx, sc.ny, sc.nz, 1, sc.origin, sc.extent)
    i, j, k = o_mesh.node_ijk()
    mode = (np.sin(np.pi * i / sc.nx) * np.sin(np.pi * j / sc.ny) * np.sin(np.pi * k / sc.nz))
    if field == "heat":
        sc.bc = {S.HEAD: {}, S.TEMP: _all_dirichlet(0.0)}
        sc.h0 = np.zeros_like(mode)
        sc.T0 = mode.copy()
        lam, cT, _, _ = fem.bulk_properties(sc)
        diff = lam / cT
    else:
        sc.bc = {S.HEAD: _all_dirichlet(0.0), S.TEMP: {}}
        sc.h0 = mode.copy()
        sc.T0 = np.zeros_like(mode)
        diff = sc.K[0] / fem.bulk_properties(sc)[3]
    o = fem.OracleSim(sc)
    dt = 0.3 * S.DAY if field == "heat" else 20.0
    fac = cf.q1_mode_factor(dt, diff, o.mesh.H, sc.extent)
    for n in range(1, 4):
        o.step(dt)
        got = o.T if field == "heat" else o.h
        np.testing.assert_allclose(got, mode * fac ** n, rtol=0, atol=1e-12)


def test_energy_balance_with_pile_flux_face_and_injection_well():
    """Closed box, no flow, consistent loads: the stored heat sum_i
    [M_cT (T^{n+1} - T^n)]_i equals dt * (q_l(t) * pile length + flux * face
    area + injected c_w Q_in (T_in - T))."""
    for p in (1, 2):
        sc = S.random_small(5, 4, 3, 3, p, n_piles=2, n_wells=0)
        sc.bc = {S.HEAD: {}, S.TEMP: {4: (S.FLUX, 0.89)}}
        sc.h0 = np.full_like(sc.h0, 0.1)
        o = fem.OracleSim(sc)
        T0 = o.T.copy()
        dt = sc.dt
        o.step(dt)
        stored = (o.McT @ (o.T - T0)).sum()
        t1 = dt
        expect = sum(fem.pile_amplitude(pl, t1) * abs(pl[2] - pl[3]) for pl in sc.piles)
        expect += 0.89 * sc.extent[0] * sc.extent[1]
        assert abs(stored - dt * expect) <= 1e-11 * abs(dt * expect)


def test_energy_balance_with_injection_well_implicit_term():
    sc = S.random_small(6, 4, 4, 3, 1, n_piles=0, n_wells=1)
    sc.bc = {S.HEAD: {}, S.TEMP: {}}
    o = fem.OracleSim(sc)
    T0 = o.T.copy()
    o.step(sc.dt)
    stored = (o.McT @ (o.T - T0)).sum()
    # advective term sum_i (C T)_i is not zero in general with a source of
    # water; the identity is sum_i [C T]_i = sum_cells int c_w q . grad T
    qf = fem.darcy_at_qp(o.mesh, o.K, o.G, o.h)
    C = fem.assemble(o.mesh, np.ones(o.mesh.n_cells), fem.advection_elements(o.N, o.G, o.W, qf, o.cw))
    wl = sc.wells[0]
    L = wl[2] - wl[3]
    injected = sc.cw * wl[4] / L * sum(w * (wl[5] - o.T[nd]) for nd, w in
                                       fem.line_weights(o.mesh, wl[0], wl[1], wl[2], wl[3]).items())
    adv = (C @ o.T).sum()
    assert abs(stored - sc.dt * (injected - adv)) <= 1e-10 * abs(sc.dt * injected)


def _slab(p, nx, L, dt, steps, bc_temp, bc_head=None, h0=None, K=1e-4):
    sc = S.config1(nx=nx, ny=1, nz=1, order=p, n_steps=steps)
    sc.extent = (L, 1.0, 1.0)
    sc.piles = np.zeros((0, 8))
    sc.K = np.full(sc.n_cells, K)
    sc.bc = {S.HEAD: bc_head or {}, S.TEMP: bc_temp}
    Nn = sc.n_nodes
    sc.h0 = np.zeros(Nn) if h0 is None else h0
    sc.T0 = np.zeros(Nn)
    sc.dt = dt
    return sc


@pytest.mark.parametrize("p", [1, 2])
def test_erfc_conduction_converges(p):
    """Step change T = 1 at x = 0 into a cold slab: error against
    erfc(x / (2 sqrt(a t))) shrinks as H and dt are refined."""
    errs = []
    for nx, nsteps in ((40 // p, 10), (80 // p, 40)):
        t_end = 5 * S.DAY
        sc = _slab(p, nx, 6.0, t_end / nsteps, nsteps, {0: (S.DIRICHLET, 1.0)})
        o = fem.OracleSim(sc)
        for _ in range(nsteps):
            o.step(sc.dt)
        x, _, _ = o.mesh.node_xyz()
        ex = cf.erfc_1d(x, t_end, _lam(sc) / _cT(sc), 1.0)
        errs.append(np.max(np.abs(o.T - ex)))
    assert errs[0] < 0.02
    assert errs[1] < errs[0] / 2.5, errs


def test_ogata_banks_advection_diffusion_converges():
    """Uniform Darcy flux from a linear head: heat front against the Ogata-
    Banks solution with v = c_w q / c_T, D = lambda / c_T."""
    errs = []
    for nx, nsteps in ((40, 20), (80, 80)):
        L = 4.0
        grad = 0.05
        p = 1
        Nn = (nx + 1) * 2 * 2
        sc = _slab(p, nx, L, 1.0, nsteps, {0: (S.DIRICHLET, 1.0)},
                   bc_head={0: (S.DIRICHLET, grad * L), 1: (S.DIRICHLET, 0.0)})
        o_mesh = fem.Mesh(nx, 1, 1, 1, (0, 0, 0), (L, 1, 1))
        x, _, _ = o_mesh.node_xyz()
        sc.h0 = grad * (L - x)
        K = 1e-4
        q = K * grad
        v = sc.cw * q / _cT(sc)
        D = _lam(sc) / _cT(sc)
        t_end = 0.4 * L / v
        sc.dt = t_end / nsteps
        o = fem.OracleSim(sc)
        for _ in range(nsteps):
            o.step(sc.dt)
        ex = cf.ogata_banks(x, t_end, v, D, 1.0)
        errs.append(np.max(np.abs(o.T - ex)))
    assert errs[0] < 0.08, errs
    assert errs[1] < errs[0] / 2.5, errs


def _mms_error(p, n, with_advection):
    """One backward Euler step of a manufactured problem whose exact solution
    u = sin(x) cos(0.7 y) exp(0.3 z) satisfies c u - dt div(k grad u) + dt
    c_w q . grad u = f exactly; returns the L2 error of the discrete solution."""
    L = (1.0, 1.2, 0.9)
    sc = S.config1(nx=n, ny=n, nz=n, order=p)
    sc.extent = L
    sc.piles = np.zeros((0, 8))
    Kh = 2e-5
    sc.K = np.full(sc.n_cells, Kh)
    grad = 0.1
    m = fem.Mesh(n, n, n, p, (0, 0, 0), L)
    X, Y, Z = m.node_xyz()

    def u(x, y, z):
        return np.sin(x) * np.cos(0.7 * y) * np.exp(0.3 * z)

    lap = (-1.0 - 0.49 + 0.09)
    dt = 1000.0
    qx = Kh * grad if with_advection else 0.0
    lam, cT, cw, _ = fem.bulk_properties(sc)

    def f(x, y, z):
        uu = u(x, y, z)
        ux = np.cos(x) * np.cos(0.7 * y) * np.exp(0.3 * z)
        return -dt * lam * lap * uu + dt * cw * qx * ux

    sc.bc = {S.HEAD: {0: (S.DIRICHLET, grad * L[0]), 1: (S.DIRICHLET, 0.0)} if with_advection else {},
             S.TEMP: _all_dirichlet(0.0)}
    sc.h0 = grad * (L[0] - X) if with_advection else np.zeros_like(X)
    sc.T0 = np.zeros_like(X)
    o = fem.OracleSim(sc)
    # Dirichlet data = exact solution on the boundary
    mask = o.dmask[S.TEMP]
    o.gval[S.TEMP] = np.where(mask, u(X, Y, Z), 0.0)
    # load: (f, N_i) / dt + mass term of the exact solution, 5-point Gauss
    Nq, Gq, Wq = fem.reference_element(p, m.H, nq=5)
    xq, _ = fem.gauss01(5)
    F = np.zeros(m.n_nodes)
    errsq = 0.0
    n1 = p + 1
    for c in range(m.n_cells):
        cx, cy, cz = c % n, (c // n) % n, c // (n * n)
        for qz in range(5):
            for qy in range(5):
                for qx_ in range(5):
                    qi = qx_ + 5 * (qy + 5 * qz)
                    px = (cx + xq[qx_]) * m.H[0]
                    py = (cy + xq[qy]) * m.H[1]
                    pz = (cz + xq[qz]) * m.H[2]
                    F[m.conn[c]] += Wq[qi] * Nq[qi] * (f(px, py, pz) + cT * u(px, py, pz)) / dt
    o.extra[S.TEMP] = F
    o.T[:] = 0.0
    # remove the mass term of T^n (= 0) -- the load already carries c_T u
    o.step(dt)
    for c in range(m.n_cells):
        cx, cy, cz = c % n, (c // n) % n, c // (n * n)
        uh = Nq @ o.T[m.conn[c]]
        for qi in range(125):
            qx_, qy, qz = qi % 5, (qi // 5) % 5, qi // 25
            px = (cx + xq[qx_]) * m.H[0]
            py = (cy + xq[qy]) * m.H[1]
            pz = (cz + xq[qz]) * m.H[2]
            errsq += Wq[qi] * (uh[qi] - u(px, py, pz)) ** 2
    return math.sqrt(errsq)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("adv", [False, True])
def test_manufactured_solution_convergence_order(p, adv):
    e1 = _mms_error(p, 3, adv)
    e2 = _mms_error(p, 6, adv)
    order = math.log(e1 / e2) / math.log(2.0)
    assert order > p + 1 - 0.35, (e1, e2, order)


def test_mirror_symmetry_between_identical_piles():
    """Two identical piles placed symmetrically in still water give a
    temperature field symmetric about the midline (Section 3.5)."""
    sc = S.config1(nx=8, ny=4, nz=4, order=1)
    sc.extent = (16.0, 8.0, 8.0)
    sc.piles = np.array([[5.0, 4.0, 8.0, 2.0, 10.0, 0.0, 1e9, 0.0],
                         [11.0, 4.0, 8.0, 2.0, 10.0, 0.0, 1e9, 0.0]])
    sc.bc = {S.HEAD: {}, S.TEMP: {0: (S.DIRICHLET, 15.0), 1: (S.DIRICHLET, 15.0), 5: (S.DIRICHLET, 15.0)}}
    sc.h0 = np.zeros(sc.n_nodes)
    o = fem.OracleSim(sc)
    for _ in range(3):
        o.step(sc.dt)
    T = o.T.reshape(sc.node_dims[::-1])
    np.testing.assert_allclose(T, T[:, :, ::-1], rtol=0, atol=1e-12)


def test_gaussian_well_integrals_match_erf_closed_forms():
    """The lateral cell integrals of a spread well: summed over the local basis
    they give the probability mass of the cell (partition of unity), and the
    first moment sum_a x_a I_a equals int x g dx (linear reproduction), both
    in closed form with erf."""
    from scipy import special
    for p in (1, 2):
        m = fem.Mesh(20, 3, 2, p, (0.0, 0.0, 0.0), (30.0, 3.0, 2.0))
        mu, sg = 13.7, 1.3
        I = fem.gaussian_cell_integrals(m, 0, mu, sg)
        H = m.H[0]
        for c in range(m.nx):
            a0, a1 = c * H, (c + 1) * H
            if not any((c, a) in I for a in range(p + 1)):
                continue
            za, zb = (a0 - mu) / sg, (a1 - mu) / sg
            mass = 0.5 * (special.erf(zb / math.sqrt(2)) - special.erf(za / math.sqrt(2)))
            dens = lambda z: math.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
            first = mu * mass - sg * (dens(zb) - dens(za))
            got_mass = sum(I[(c, a)] for a in range(p + 1))
            got_first = sum(I[(c, a)] * (a0 + a * H / p) for a in range(p + 1))
            assert abs(got_mass - mass) < 1e-13
            assert abs(got_first - first) < 1e-12
        # a well spread inside the box injects exactly Q (weights sum to L)
        sc = S.random_small(3, 6, 6, 3, p, n_piles=0, n_wells=0)
        wl = np.array([sc.extent[0] / 2, sc.extent[1] / 2, 15.0, 5.0, 1e-3, 20.0, 2.0])
        w = fem.well_weights(fem.Mesh(sc.nx, sc.ny, sc.nz, p, sc.origin, sc.extent), wl)
        assert abs(sum(w.values()) - 10.0) < 1e-9


def test_box_source_weights_closed_forms():
    """Box heat sources: the weights integrate 1, x, y and x*y over the snapped
    rectangle exactly (area, first moments and the mixed moment in closed
    form), every weight sits on the snapped node plane, and edges that lie
    within 0.3 cells of a face snap to that face."""
    for p in (1, 2):
        m = fem.Mesh(7, 5, 4, p, (1.0, -2.0, 0.5), (14.0, 10.0, 8.0))
        Hx, Hy, Hz = m.H
        box = [1.0 + 2 * Hx + 0.29 * Hx, 1.0 + 6 * Hx - 0.21 * Hx, -2.0 + 1 * Hy - 0.3 * Hy,
               -2.0 + 4 * Hy + 0.1 * Hy, 0.5 + 3 * Hz + 0.2 * Hz, 1.0, 0.0, 1.0, 0.0]
        assert fem.box_snap(m, box) == (2, 6, 1, 4, 3)
        xa, xb, ya, yb = 1.0 + 2 * Hx, 1.0 + 6 * Hx, -2.0 + Hy, -2.0 + 4 * Hy
        w = fem.box_weights(m, box)
        x, y, z = m.node_xyz()
        idx = np.array(list(w.keys()))
        val = np.array(list(w.values()))
        assert np.allclose(z[idx], 0.5 + 3 * Hz, rtol=0, atol=1e-12)
        area = (xb - xa) * (yb - ya)
        assert abs(val.sum() - area) <= 1e-12 * area
        assert abs((val * x[idx]).sum() - 0.5 * (xb ** 2 - xa ** 2) * (yb - ya)) <= 1e-11 * area * 15
        assert abs((val * y[idx]).sum() - 0.5 * (yb ** 2 - ya ** 2) * (xb - xa)) <= 1e-11 * area * 15
        mixed = 0.25 * (xb ** 2 - xa ** 2) * (yb ** 2 - ya ** 2)
        assert abs((val * x[idx] * y[idx]).sum() - mixed) <= 1e-11 * abs(mixed)
        if p == 2:   # Q2 also integrates x^2 exactly
            sq = (xb ** 3 - xa ** 3) / 3 * (yb - ya)
            assert abs((val * x[idx] ** 2).sum() - sq) <= 1e-11 * sq
        # edges outside the mesh are clamped to it
        assert fem.box_snap(m, [-50.0, 100.0, -50.0, 100.0, 99.0, 0, 0, 1, 0]) == (0, 7, 0, 5, 4)


def test_box_source_over_the_top_face_equals_the_face_flux():
    """A box covering the whole top face with a constant flux gives the same
    nodal load as a Neumann flux on that face."""
    for p in (1, 2):
        m = fem.Mesh(4, 3, 2, p, (0.0, 0.0, 0.0), (8.0, 6.0, 4.0))
        box = [0.0, 8.0, 0.0, 6.0, 4.0, 0.89, 0.0, 1.0, 0.0]
        F = np.zeros(m.n_nodes)
        for nd, wv in fem.box_weights(m, box).items():
            F[nd] += fem.box_flux(box, 0.0) * wv
        np.testing.assert_allclose(F, fem.face_load(m, 5, 0.89), rtol=0, atol=1e-14)


def test_energy_balance_with_box_sources():
    """Insulated box, still water: the stored heat of one step is dt times the
    sum over boxes of q(t^{n+1}) times the snapped area (Eq. 4 with the
    conduction term summing to zero over all rows)."""
    for p in (1, 2):
        sc = S.random_small(8, 5, 4, 3, p, n_piles=0, n_wells=0, n_boxes=3)
        sc.bc = {S.HEAD: {}, S.TEMP: {}}
        sc.h0 = np.zeros_like(sc.h0)
        o = fem.OracleSim(sc)
        T0 = o.T.copy()
        o.step(sc.dt)
        assert np.abs(o.h).max() == 0.0
        stored = (o.McT @ (o.T - T0)).sum()
        expect = 0.0
        for bx in sc.boxes:
            i0, i1, j0, j1, _ = fem.box_snap(o.mesh, bx)
            expect += fem.box_flux(bx, sc.dt) * (i1 - i0) * o.mesh.H[0] * (j1 - j0) * o.mesh.H[1]
        assert abs(expect) > 0
        assert abs(stored - sc.dt * expect) <= 1e-10 * abs(sc.dt * expect)


def test_nodal_face_flux_closed_forms():
    """A normal flux given per face node: a constant reduces to the uniform
    face load, and a flux linear along the face integrates to the closed-form
    total and first moment (the face basis reproduces linear functions)."""
    for p in (1, 2):
        m = fem.Mesh(4, 3, 5, p, (1.0, 2.0, -3.0), (8.0, 6.0, 5.0))
        x, y, z = m.node_xyz()
        for face in range(6):
            nodes = m.face_nodes(face)
            np.testing.assert_allclose(fem.face_load_nodal(m, face, np.full(nodes.size, 0.7)),
                                       fem.face_load(m, face, 0.7), rtol=0, atol=1e-13)
        face = 2                                   # y = y0; tangential axes x (fastest), z
        nodes = m.face_nodes(face)
        q = 0.5 + 0.25 * x[nodes] - 0.4 * z[nodes]
        F = fem.face_load_nodal(m, face, q)
        xa, xb, za, zb = 1.0, 9.0, -3.0, 2.0
        total = 0.5 * (xb - xa) * (zb - za) + 0.25 * 0.5 * (xb ** 2 - xa ** 2) * (zb - za) \
            - 0.4 * 0.5 * (zb ** 2 - za ** 2) * (xb - xa)
        first = 0.5 * 0.5 * (xb ** 2 - xa ** 2) * (zb - za) + 0.25 * (xb ** 3 - xa ** 3) / 3 * (zb - za) \
            - 0.4 * 0.25 * (xb ** 2 - xa ** 2) * (zb ** 2 - za ** 2)
        assert abs(F.sum() - total) <= 1e-12 * abs(total)
        assert abs((F * x).sum() - first) <= 1e-12 * abs(first)
        assert np.all(F[np.setdiff1d(np.arange(m.n_nodes), nodes)] == 0.0)


def test_linear_head_from_nodal_dirichlet_faces_is_exact():
    """Per-node Dirichlet values on all six faces equal to a linear head,
    uniform K and no storage: the discrete solution is that linear head at
    every node, which fails if face values land on the wrong nodes."""
    for p in (1, 2):
        sc = S.random_small(9, 4, 3, 5, p, n_piles=0, n_wells=0)
        sc.K = np.full(sc.n_cells, 2e-5)
        sc.Ss = 0.0
        m = fem.Mesh(sc.nx, sc.ny, sc.nz, p, sc.origin, sc.extent)
        x, y, z = m.node_xyz()
        h_lin = 0.3 + 0.02 * x - 0.05 * y + 0.07 * z
        sc.bc = {S.HEAD: {f: (S.DIRICHLET, h_lin[m.face_nodes(f)]) for f in range(6)}, S.TEMP: {}}
        o = fem.OracleSim(sc)
        o.step(sc.dt)
        np.testing.assert_allclose(o.h, h_lin, rtol=0, atol=1e-12)


@pytest.mark.parametrize("case", [(1, 5, 4, 3, 11), (2, 3, 4, 2, 12)])
@pytest.mark.parametrize("nodal", [False, True])
def test_row_oracle_equals_the_assembled_oracle_at_every_row(case, nodal):
    """The row-wise oracle (used to check meshes too large to assemble) gives
    the assembled oracle's A0 x and lifted b at every row: piles, wells, box
    sources, per-cell thermal coefficients, and optionally per-node
    boundary data."""
    p, nx, ny, nz, seed = case
    sc = S.random_small(seed, nx, ny, nz, p, n_piles=2, n_wells=2, n_boxes=2, per_cell_thermal=True,
                        faces_temp=(0, 2, 5))
    if nodal:
        m = fem.Mesh(nx, ny, nz, p, sc.origin, sc.extent)
        rng = np.random.default_rng(seed)
        sc.bc[S.HEAD][1] = (S.DIRICHLET, rng.uniform(-1, 1, m.face_nodes(1).size))
        sc.bc[S.TEMP][4] = (S.FLUX, rng.uniform(0, 2, m.face_nodes(4).size))
    o = fem.OracleSim(sc)
    r = fem.RowOracle(sc)
    rows = list(range(sc.n_nodes))
    x = np.random.default_rng(1).standard_normal(sc.n_nodes)
    h = np.random.default_rng(2).standard_normal(sc.n_nodes)
    dt, t1 = sc.dt, 1.7 * sc.dt
    for (got, scale), ref in [(r.apply_rows(S.HEAD, dt, x, rows), o.apply_head(x, dt)),
                              (r.apply_rows(S.TEMP, dt, x, rows, h), o.apply_heat(x, h, dt)),
                              (r.rhs_rows(S.HEAD, dt, t1, o.h, rows), o.head_rhs(dt, t1)),
                              (r.rhs_rows(S.TEMP, dt, t1, o.T, rows, h), o.heat_rhs(dt, t1, h))]:
        assert np.all(np.abs(got - ref) <= 1e-13 * scale + 1e-300)
        assert np.all(scale >= np.abs(ref) * (1 - 1e-12))


def test_cells_of_node_lists_each_holding_cell_once():
    for p in (1, 2):
        m = fem.Mesh(3, 2, 2, p, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        seen = {}
        for c in range(m.n_cells):
            for l, nd in enumerate(m.conn[c]):
                seen.setdefault(int(nd), set()).add((c, l))
        for nd in range(m.n_nodes):
            got = fem.cells_of_node(m, nd)
            assert len(got) == len(set(got)) and set(got) == seen[nd]


def _line_source_run(n, steps, t_end, L=20.0, Lz=2.0, ql=10.0):
    """A full-height line source of q_l W/m on the axis of an L x L x Lz
    block of Q1 cells, insulated top and bottom (so the problem is the 2D
    infinite line), T = 0 on the far lateral faces, still water.  Returns the
    radii and temperatures along a ray from the source at the bottom plane."""
    sc = S.config1(nx=n, ny=n, nz=1, order=1, n_steps=steps)
    sc.extent = (L, L, Lz)
    sc.K = np.full(sc.n_cells, 1e-4)
    sc.h0 = np.zeros(sc.n_nodes)
    sc.T0 = np.zeros(sc.n_nodes)
    sc.bc = {S.HEAD: {}, S.TEMP: {f: (S.DIRICHLET, 0.0) for f in (0, 1, 2, 3)}}
    sc.piles = np.array([[L / 2, L / 2, Lz, 0.0, ql, 0.0, 1e9, 0.0]])
    sc.dt = t_end / steps
    o = fem.OracleSim(sc)
    for _ in range(steps):
        o.step(sc.dt)
    x, y, z = o.mesh.node_xyz()
    ray = (np.abs(y - L / 2) < 1e-9) & (z == 0.0) & (x > L / 2)
    return x[ray] - L / 2, o.T[ray], sc


def test_infinite_line_source_converges_to_the_e1_solution():
    """The continuous line source dT = q_l/(4 pi lambda) E1(r^2/(4 a t)),
    a = lambda / c_T, at t = 30 d (diffusion length 3.1 m, far field 10 m
    away): the error at r = 2, 3, 4 m is below 5% on 0.5 m cells and falls
    by more than 2.5x from 1 m cells (second order in H, first in dt)."""
    t_end = 30 * 86400.0
    errs = []
    for n, steps in ((20, 10), (40, 20)):
        r, T, sc = _line_source_run(n, steps, t_end)
        keep = np.isin(np.round(r, 9), [2.0, 3.0, 4.0])
        ex = cf.line_source_e1(r[keep], t_end, 10.0, _lam(sc), _lam(sc) / _cT(sc))
        errs.append(np.abs(T[keep] - ex) / ex)
    assert errs[0].size == errs[1].size == 3
    assert np.all(errs[1] < 0.05), errs[1]
    assert np.all(errs[0] > 2.5 * errs[1]), errs


def test_response_decays_monotonically_with_distance_from_a_pile():
    """Section 3.5: the temperature rise falls off monotonically with the
    distance from an energy pile."""
    r, T, _ = _line_source_run(40, 20, 30 * 86400.0)
    assert np.all(np.diff(T) < 0.0)
    assert T[0] > 0.0


def test_moving_line_source_closed_form_limits():
    """The moving-line-source integral reduces to E1 without flow and to the
    steady K0 form at long times."""
    lam, cT, U = 1.93, 2.654e6, 1.575e-6
    a = lam / cT
    x, y = np.array([2.0, -3.0, 0.0, 1.0]), np.array([0.5, 1.0, 2.0, -1.5])
    t = 30 * 86400.0
    np.testing.assert_allclose(cf.moving_line_source(x, y, t, 10.0, lam, a, 0.0),
                               cf.line_source_e1(np.hypot(x, y), t, 10.0, lam, a), rtol=1e-10)
    np.testing.assert_allclose(cf.moving_line_source(x, y, 1e14, 10.0, lam, a, U),
                               cf.moving_line_source_steady(x, y, 10.0, lam, a, U), rtol=1e-8)


def test_line_source_in_uniform_flow_converges_to_the_moving_line_source():
    """A full-height line source of 10 W/m in a uniform Darcy flux
    q = 1e-6 m/s along x (a linear head, which Q1 reproduces exactly), 30 d:
    the oracle approaches the moving-line-source solution, U = c_w q / c_T,
    downstream and to the side, with the error falling as H and dt halve;
    the plume is carried downstream."""
    L, Lz, grad, K = 30.0, 2.0, 0.01, 1e-4
    t_end = 30 * 86400.0
    pts = [(2.0, 0.0), (3.0, 0.0), (4.0, 0.0), (0.0, 2.0)]
    errs, temps = [], []
    for n, steps in ((30, 10), (60, 20)):
        sc = S.config1(nx=n, ny=n, nz=1, order=1, n_steps=steps)
        sc.extent = (L, L, Lz)
        sc.K = np.full(sc.n_cells, K)
        sc.h0 = np.zeros(sc.n_nodes)
        sc.T0 = np.zeros(sc.n_nodes)
        sc.bc = {S.HEAD: {0: (S.DIRICHLET, grad * L), 1: (S.DIRICHLET, 0.0)},
                 S.TEMP: {f: (S.DIRICHLET, 0.0) for f in (0, 1, 2, 3)}}
        sc.piles = np.array([[L / 2, L / 2, Lz, 0.0, 10.0, 0.0, 1e9, 0.0]])
        sc.dt = t_end / steps
        o = fem.OracleSim(sc)
        for _ in range(steps):
            o.step(sc.dt)
        x, y, z = o.mesh.node_xyz()
        U = sc.cw * K * grad / _cT(sc)
        a = _lam(sc) / _cT(sc)
        got = []
        for px, py in pts + [(-2.0, 0.0)]:
            got.append(o.T[np.nonzero((np.abs(x - L / 2 - px) < 1e-9) & (np.abs(y - L / 2 - py) < 1e-9)
                                      & (z == 0.0))[0][0]])
        ex = cf.moving_line_source([p[0] for p in pts], [p[1] for p in pts], t_end, 10.0, _lam(sc), a, U)
        errs.append(np.abs(np.array(got[:-1]) - ex) / ex)
        temps.append(got)
    assert np.all(errs[1][:3] < 0.05) and errs[1][3] < 0.15, errs[1]
    assert np.all(errs[0] > 1.6 * errs[1]), errs
    assert temps[1][0] > 10.0 * temps[1][-1]     # downstream of the pile >> upstream


@pytest.mark.parametrize("p", [1, 2])
def test_dirichlet_lift_satisfies_the_unconstrained_free_rows_and_reactions_close_the_balance(p):
    """After a step with Dirichlet faces, the free rows of the unconstrained
    systems hold exactly: R = A u^{n+1} - c M u^n - dt F vanishes off the
    Dirichlet nodes (so lifting b = F - A g_D was done right), u^{n+1} = g on
    them, and the boundary reactions R_D close the balance: with 1^T K = 0,
    S_s 1^T M (h^{n+1} - h^n) = dt 1^T F_h + sum_D R_D for the head."""
    sc = S.random_small(21, 4, 3, 3, p, n_piles=2, n_wells=2)
    o = fem.OracleSim(sc)
    h0, T0 = o.h.copy(), o.T.copy()
    t1 = sc.dt
    o.step(sc.dt)
    for field, u0, u1, A, cM in ((S.HEAD, h0, o.h, o.head_matrix(sc.dt), o.Ss * o.M),
                                 (S.TEMP, T0, o.T, o.heat_matrix(sc.dt, o.h), o.McT)):
        F = o.head_load(t1) if field == S.HEAD else o.heat_load(t1)
        R = A @ u1 - cM @ u0 - sc.dt * F
        mask = o.dmask[field]
        scale = np.abs(A) @ np.abs(u1) + np.abs(cM) @ np.abs(u0) + sc.dt * np.abs(F)
        assert np.all(np.abs(R[~mask]) <= 1e-12 * scale[~mask])
        np.testing.assert_allclose(u1[mask], o.gval[field][mask], rtol=1e-14, atol=0)
    R = o.head_matrix(sc.dt) @ o.h - o.Ss * (o.M @ h0) - sc.dt * o.head_load(t1)
    stored = o.Ss * (o.M @ (o.h - h0)).sum()
    rhs = sc.dt * o.head_load(t1).sum() + R[o.dmask[S.HEAD]].sum()
    assert abs(stored - rhs) <= 1e-10 * (abs(stored) + abs(rhs))


def _graded(sc, stretch=(0.8, -0.6, 1.2)):
    sc.spacing = tuple(S.graded_widths(n, L, a) for n, L, a in zip((sc.nx, sc.ny, sc.nz), sc.extent, stretch))
    return sc


@pytest.mark.parametrize("p", [1, 2])
def test_graded_mesh_with_equal_widths_is_the_uniform_mesh(p):
    """Graded spacing with all widths equal reduces to the uniform mesh."""
    sc = S.random_small(31, 4, 3, 2, p, n_piles=2, n_wells=2, n_boxes=2, per_cell_thermal=True)
    o = fem.OracleSim(sc)
    sg = S.random_small(31, 4, 3, 2, p, n_piles=2, n_wells=2, n_boxes=2, per_cell_thermal=True)
    sg.spacing = tuple(np.full(n, L / n) for n, L in zip((sg.nx, sg.ny, sg.nz), sg.extent))
    og = fem.OracleSim(sg)
    assert og.mesh.H is None
    x = np.random.default_rng(2).standard_normal(sc.n_nodes)
    for a, b in [(o.apply_head(x, sc.dt), og.apply_head(x, sc.dt)),
                 (o.apply_heat(x, o.h, sc.dt), og.apply_heat(x, og.h, sc.dt)),
                 (o.head_rhs(sc.dt, sc.dt), og.head_rhs(sc.dt, sc.dt)),
                 (o.heat_rhs(sc.dt, sc.dt, o.h), og.heat_rhs(sc.dt, sc.dt, og.h)),
                 (o.cell_flux(), og.cell_flux())]:
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-13 * np.abs(a).max())


@pytest.mark.parametrize("p", [1, 2])
def test_graded_mesh_integrates_constants_and_reproduces_linear_heads(p):
    """On a graded mesh the mass matrix integrates 1 to the volume, constants
    lie in the kernel of the stiffness and advection matrices, the head
    operator is symmetric, the row-wise oracle equals the assembled one, and
    per-node Dirichlet faces carrying a linear head with uniform K and no
    storage give that head exactly."""
    sc = _graded(S.random_small(32, 4, 3, 3, p, n_piles=1, n_wells=1, n_boxes=1))
    o = fem.OracleSim(sc)
    m = o.mesh
    one = np.ones(m.n_nodes)
    assert abs(o.M.sum() - np.prod(sc.extent)) <= 1e-12 * np.prod(sc.extent)
    assert np.abs(o.KK @ one).max() <= 1e-12 * np.abs(o.KK.data).max()
    qf = fem.darcy_at_qp(m, o.K, o.G, o.h)
    C = fem.assemble(m, np.ones(m.n_cells), fem.advection_elements(o.N, o.G, o.W, qf, o.cw))
    assert np.abs(C @ one).max() <= 1e-10 * np.abs(C.data).max()
    A = o.head_matrix(sc.dt).toarray()
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    r = fem.RowOracle(sc)
    rows = list(range(m.n_nodes))
    x = np.random.default_rng(4).standard_normal(m.n_nodes)
    np.testing.assert_allclose(r.apply_rows(S.TEMP, sc.dt, x, rows, h=o.h)[0], o.apply_heat(x, o.h, sc.dt),
                               rtol=0, atol=1e-13 * np.abs(o.apply_heat(x, o.h, sc.dt)).max())
    np.testing.assert_allclose(r.rhs_rows(S.TEMP, sc.dt, sc.dt, o.T, rows, h=o.h)[0],
                               o.heat_rhs(sc.dt, sc.dt, o.h), rtol=0,
                               atol=1e-13 * np.abs(o.heat_rhs(sc.dt, sc.dt, o.h)).max())
    sc2 = _graded(S.random_small(33, 4, 3, 3, p, n_piles=0, n_wells=0))
    sc2.K = np.full(sc2.n_cells, 2e-5)
    sc2.Ss = 0.0
    m2 = fem.Mesh(sc2.nx, sc2.ny, sc2.nz, p, sc2.origin, sc2.extent, sc2.spacing)
    X, Y, Z = m2.node_xyz()
    h_lin = 0.3 + 0.02 * X - 0.05 * Y + 0.07 * Z
    sc2.bc = {S.HEAD: {f: (S.DIRICHLET, h_lin[m2.face_nodes(f)]) for f in range(6)}, S.TEMP: {}}
    o2 = fem.OracleSim(sc2)
    o2.step(sc2.dt)
    np.testing.assert_allclose(o2.h, h_lin, rtol=0, atol=1e-12)


def _graded_mms_error(p, n, stretch=(0.7, -0.7, 0.5)):
    """Steady head problem -div(K grad h) = f on a graded mesh with the exact
    solution h = sin(x) cos(0.7 y) exp(0.3 z) as per-node Dirichlet data on
    all faces; returns the L2 error by 5-point Gauss per cell."""
    L = (1.0, 1.2, 0.9)
    sc = S.config1(nx=n, ny=n, nz=n, order=p)
    sc.extent = L
    sc.spacing = tuple(S.graded_widths(n, Ld, a) for Ld, a in zip(L, stretch))
    sc.piles = np.zeros((0, 8))
    Kh = 2e-5
    sc.K = np.full(sc.n_cells, Kh)
    sc.Ss = 0.0
    m = fem.Mesh(n, n, n, p, (0, 0, 0), L, sc.spacing)
    X, Y, Z = m.node_xyz()

    def u(x, y, z):
        return np.sin(x) * np.cos(0.7 * y) * np.exp(0.3 * z)
    lap = -1.0 - 0.49 + 0.09
    sc.bc = {S.HEAD: {f: (S.DIRICHLET, u(X, Y, Z)[m.face_nodes(f)]) for f in range(6)}, S.TEMP: {}}
    sc.h0 = np.zeros(m.n_nodes)
    sc.T0 = np.zeros(m.n_nodes)
    o = fem.OracleSim(sc)
    xq, _ = fem.gauss01(5)
    F = np.zeros(m.n_nodes)
    hw = m.cell_widths()
    Nq, _, W1 = fem.reference_element(p, (1.0, 1.0, 1.0), nq=5)
    quad = []
    for c in range(m.n_cells):
        cx, cy, cz = c % n, (c // n) % n, c // (n * n)
        Wq = W1 * np.prod(hw[c])
        lo = (m.faces[0][cx], m.faces[1][cy], m.faces[2][cz])
        pts = [(lo[0] + hw[c, 0] * xq[qx], lo[1] + hw[c, 1] * xq[qy], lo[2] + hw[c, 2] * xq[qz])
               for qz in range(5) for qy in range(5) for qx in range(5)]
        P = np.array(pts)
        fq = -Kh * lap * u(P[:, 0], P[:, 1], P[:, 2])
        F[m.conn[c]] += np.einsum("q,ql,q->l", Wq, Nq, fq)
        quad.append((c, Nq, Wq, u(P[:, 0], P[:, 1], P[:, 2])))
    o.extra[S.HEAD] = F
    o.step(sc.dt)
    err = 0.0
    for c, Nq, Wq, uq in quad:
        err += np.sum(Wq * (Nq @ o.h[m.conn[c]] - uq) ** 2)
    return math.sqrt(err)


@pytest.mark.parametrize("p", [1, 2])
def test_graded_mesh_manufactured_solution_converges_at_order_p_plus_1(p):
    """Refining the same smooth graded map halves every width: the L2 error
    falls at order 2 (Q1) and 3 (Q2)."""
    e1, e2 = _graded_mms_error(p, 3), _graded_mms_error(p, 6)
    order = math.log(e1 / e2) / math.log(2.0)
    assert order > p + 1 - 0.35, (e1, e2, order)


def _pile_temp_scenario(p, rows, n=6, nz=3, insulated=False):
    sc = S.config1(nx=n, ny=n, nz=nz, order=p)
    sc.extent = (12.0, 12.0, 6.0)
    sc.piles = np.zeros((0, 8))
    sc.h0 = np.zeros(sc.n_nodes)
    sc.T0 = np.full(sc.n_nodes, 15.0)
    sc.bc = {S.HEAD: {}, S.TEMP: {} if insulated else {0: (S.DIRICHLET, 15.0), 1: (S.DIRICHLET, 15.0)}}
    sc.pile_temps = np.asarray(rows, dtype=np.float64).reshape(-1, 9)
    return sc


@pytest.mark.parametrize("p", [1, 2])
def test_pile_surface_temperature_is_held_and_drives_an_insulated_box_to_it(p):
    """Pile surfaces held at a square wave (Section 3.3: 288.55 K +- 13 K, six
    months each way): the pile nodes take T_p(t^{n+1}) exactly at every step,
    the wave flips after half a period, and with insulated outer faces one
    very long step brings the whole block to the pile temperature."""
    year = 365 * S.DAY
    row = [6.0, 6.0, 6.0, 1.0, 0.8, 288.55, 13.0, year, 0.0]
    sc = _pile_temp_scenario(p, [row])
    o = fem.OracleSim(sc)
    nodes = o.pile_nodes[0]
    X, Y, Z = o.mesh.node_xyz()
    assert nodes.size > 0 and np.all((X[nodes] - 6) ** 2 + (Y[nodes] - 6) ** 2 <= 0.64 + 1e-9)
    dt = 60 * S.DAY
    for k in range(1, 8):
        o.step(dt)
        expect = 301.55 if math.sin(2 * math.pi * k * dt / year) >= 0 else 275.55
        np.testing.assert_array_equal(o.T[nodes], expect)
    # a radius below the node spacing takes the nearest node column
    thin = fem.pile_surface_nodes(o.mesh, [6.1, 5.9, 6.0, 1.0, 1e-3, 0, 0, 1, 0])
    assert np.all(X[thin] == 6.0) and np.all(Y[thin] == 6.0)
    si = _pile_temp_scenario(p, [[6.0, 6.0, 6.0, 0.0, 0.8, 290.0, 0.0, year, 0.0]], insulated=True)
    oi = fem.OracleSim(si)
    oi.step(1e19)       # the block's diffusion time is ~2e8 s: storage is negligible
    np.testing.assert_allclose(oi.T, 290.0, rtol=0, atol=1e-7)


def test_two_identical_pile_surfaces_give_a_mirror_symmetric_field():
    year = 365 * S.DAY
    rows = [[3.0, 6.0, 6.0, 1.0, 0.8, 288.55, 13.0, year, 0.0],
            [9.0, 6.0, 6.0, 1.0, 0.8, 288.55, 13.0, year, 0.0]]
    sc = _pile_temp_scenario(1, rows, n=12)
    o = fem.OracleSim(sc)
    for _ in range(3):
        o.step(30 * S.DAY)
    T = o.T.reshape(sc.node_dims[::-1])
    np.testing.assert_allclose(T, T[:, :, ::-1], rtol=0, atol=1e-9)


@pytest.mark.parametrize("p", [1, 2])
def test_seasonal_surface_temperature_follows_its_record_and_the_lift_holds(p):
    """A seasonal top-face temperature (the monthly surface record of
    Section 3.3 as a sinusoid): the top nodes take T_s(t^{n+1}) at every
    step, the x = x1 face (static Dirichlet, lower index) loses the shared
    edge to it, the free rows of the unconstrained heat system hold, and the
    row-wise oracle agrees with the assembled one."""
    year = 365 * S.DAY
    sc = _pile_temp_scenario(p, [[6.0, 6.0, 6.0, 3.0, 0.8, 288.55, 13.0, year, 0.0]])
    sc.bc[S.TEMP][5] = (S.DIRICHLET, 0.0)
    sc.bc_seasonal = {S.TEMP: {5: (287.45, 8.0, year, 0.3)}}
    o = fem.OracleSim(sc)
    r = fem.RowOracle(sc)
    top = o.mesh.face_nodes(5)
    dt = 20 * S.DAY
    for k in range(1, 4):
        T0 = o.T.copy()
        t1 = k * dt
        b_rows = r.rhs_rows(S.TEMP, dt, t1, T0, list(range(sc.n_nodes)), h=o.h)[0]
        np.testing.assert_allclose(b_rows, o.heat_rhs(dt, t1, o.h), rtol=0,
                                   atol=1e-12 * np.abs(o.heat_rhs(dt, t1, o.h)).max())
        o.step(dt)
        ts = 287.45 + 8.0 * math.sin(2 * math.pi * t1 / year + 0.3)
        pile = set(o.pile_nodes[0].tolist())
        top_free_of_pile = np.array([i for i in top if i not in pile])
        np.testing.assert_allclose(o.T[top_free_of_pile], ts, rtol=0, atol=1e-9)
        A = o.heat_matrix(dt, o.h)
        R = A @ o.T - o.McT @ T0 - dt * o.heat_load(t1)
        mask = o.dmask[S.TEMP]
        scale = np.abs(A) @ np.abs(o.T) + np.abs(o.McT) @ np.abs(T0) + dt * np.abs(o.heat_load(t1))
        assert np.all(np.abs(R[~mask]) <= 1e-12 * scale[~mask])


def test_iterative_oracle_solves_agree_with_the_direct_solve():
    """The Jacobi-PCG / BiCGStab path the CPU baseline times reaches the
    direct solution to the forward-error bound of its tolerance."""
    sc = S.random_small(40, 8, 6, 4, 2, n_piles=2, n_wells=2)
    od = fem.OracleSim(sc, solver="direct")
    oi = fem.OracleSim(sc, solver="iterative", tol=1e-13)
    for _ in range(2):
        od.step(sc.dt)
        oi.step(sc.dt)
    for a, b in ((oi.h, od.h), (oi.T, od.T)):
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
