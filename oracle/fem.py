"""CPU FP64 oracle for the coupled head / heat finite element step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import or call this module; only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` use it.  It shares no code with the CUDA path: it consumes the
same seeded inputs (``scenarios``) and nothing else.

What it computes, written out the plain way (global sparse matrices assembled
cell by cell from shape functions evaluated directly at every Gauss point, no
sum factorisation, no blocking, then a sparse direct solve):

* Head (Eq. 1 in hydraulic-head form, discretised as in Eq. 3 with backward
  Euler): (S_s M + dt K_K) h^{n+1} = S_s M h^n + dt F_h, where
  M_ij = int N_i N_j and K_K,ij = sum_c K_c int_c grad N_i . grad N_j.
  With p = rho_w g (h - z) the gravity term of Eq. 1 / Eq. 3 vanishes.
* Heat (Eq. 2 in energy form, discretised as in Eq. 4):
  (M_cT + dt L_lambda + dt C(q) + dt D_w) T^{n+1} = M_cT T^n + dt F_T, with
  C_ij = sum_qp w c_w N_i (q . grad N_j) and q = -K_c grad h^{n+1} evaluated at
  the same Gauss points (Darcy's law, Section 2, q = -k (grad p + rho_w g)).
  D_w is the lumped term of an injection well, c_w (Q/L) int N_i s dV with s
  the well's lateral profile (a line, or a normal density of width sigma).
* Loads F_T: Neumann faces and box sources (heat flux q(t) over a horizontal
  rectangle snapped to cell faces, the building heat of Section 1) as
  int q N_i dS; energy piles (Section 3.2) as int q_l N_i dz.
* Quadrature: (p+1)-point Gauss-Legendre per direction for order p.
* Dirichlet nodes: rows replaced by the identity and the prescribed values
  moved to the right-hand side (columns eliminated, so the head operator stays
  symmetric).  Free rows see no Dirichlet columns.

Parity pins (tests/test_oracle_pins.py) tie this code to closed forms: the 1D
Q1/Q2 mass and stiffness matrices, exact symbolic integrals on one cell,
discrete eigenmode decay, exactness for linear heads, energy balance, the
erfc and Ogata-Banks 1D solutions, manufactured-solution convergence
orders, and the moments of the box-source and per-node face loads.  On the
ATES benchmark of Section 2 (tests/test_ates_benchmark.py) the head follows
Thiem's steady logarithm and Theis' transient well function.

Meshes are uniform along each axis, or graded with tensor-product cell
widths (the fine-near-the-piles meshes of Section 3.3, Fig. 10b); a graded
mesh takes every geometric quantity per cell.

RowOracle evaluates the same definitions row by row (cell by cell over the
cells holding a node) for meshes too large to assemble, forming a graded
cell's element matrices when a row first needs them; it is pinned to the
assembled form at every row of small meshes.
"""
from __future__ import annotations

import math
from typing import Dict, Optional, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

HEAD, TEMP = 0, 1
NONE, DIRICHLET, FLUX = 0, 1, 2


# ---------------------------------------------------------------------------
# 1D ingredients
# ---------------------------------------------------------------------------
def gauss01(n: int):
    """n-point Gauss-Legendre rule mapped to [0, 1]."""
    xi, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (xi + 1.0), 0.5 * w


def lagrange_nodes(p: int) -> np.ndarray:
    return np.linspace(0.0, 1.0, p + 1)


def lagrange_value(p: int, a: int, xi: float) -> float:
    """phi_a(xi) for equispaced Lagrange nodes on [0, 1], product formula."""
    nodes = lagrange_nodes(p)
    v = 1.0
    for m in range(p + 1):
        if m != a:
            v *= (xi - nodes[m]) / (nodes[a] - nodes[m])
    return v


def lagrange_deriv(p: int, a: int, xi: float) -> float:
    """phi_a'(xi) by differentiating the product formula term by term."""
    nodes = lagrange_nodes(p)
    s = 0.0
    for m in range(p + 1):
        if m == a:
            continue
        term = 1.0 / (nodes[a] - nodes[m])
        for k in range(p + 1):
            if k != a and k != m:
                term *= (xi - nodes[k]) / (nodes[a] - nodes[k])
        s += term
    return s


# ---------------------------------------------------------------------------
# Mesh
# ---------------------------------------------------------------------------
def mixture(phi, lam_s, lam_w, c_s, c_w):
    """Bulk thermal conductivity and volumetric heat capacity of the saturated
    medium: volume-fraction averages of the solid and water values, the
    mixture rules given with Eq. 2 (Section 2)."""
    return (1.0 - phi) * lam_s + phi * lam_w, (1.0 - phi) * c_s + phi * c_w


def specific_storage(B_poro, rho_w=1000.0, g=9.81):
    """Specific storage of the head form: Eq. 1's storage coefficient 1/B_poro
    times rho_w g, from p = rho_w g (h - z) (Section 2)."""
    return rho_w * g / B_poro


def bulk_properties(sc):
    """(lambda, c_T, c_w, S_s) of a scenario: its directly given bulk values
    where present, else the mixture rules and the storage of Eq. 1 applied to
    its raw material properties."""
    m = sc.material
    lam, cT = mixture(m.phi, m.lam_s, m.lam_w, m.c_s, m.c_w)
    Ss = specific_storage(m.B_poro, m.rho_w, m.g)
    return (sc.lam if sc.lam is not None else lam, sc.cT if sc.cT is not None else cT, m.c_w,
            sc.Ss if sc.Ss is not None else Ss)


class Mesh:
    """Structured box of nx*ny*nz Lagrange hexahedra of order p.

    Cells are uniform along each axis (H = extent / n), or graded with a
    tensor-product spacing: spacing = (widths along x, along y, along z),
    one positive width per cell layer, summing to the extent.  A graded mesh
    has H = None, and every geometric quantity is taken per cell.
    """

    def __init__(self, nx, ny, nz, p, origin, extent, spacing=None):
        self.nx, self.ny, self.nz, self.p = nx, ny, nz, p
        self.origin = tuple(float(v) for v in origin)
        ncs = (nx, ny, nz)
        if spacing is None:
            self.extent = tuple(float(v) for v in extent)
            self.H = (self.extent[0] / nx, self.extent[1] / ny, self.extent[2] / nz)
            self.widths = tuple(np.full(ncs[d], self.H[d]) for d in range(3))
            self.faces = tuple(self.origin[d] + np.arange(ncs[d] + 1) * self.H[d] for d in range(3))
        else:
            self.widths = tuple(np.asarray(spacing[d], dtype=np.float64).reshape(-1) for d in range(3))
            for d in range(3):
                if self.widths[d].size != ncs[d] or not np.all(self.widths[d] > 0):
                    raise ValueError(f"spacing along axis {d} needs {ncs[d]} positive widths")
            self.extent = tuple(float(self.widths[d].sum()) for d in range(3))
            self.H = None
            self.faces = tuple(self.origin[d] + np.concatenate([[0.0], np.cumsum(self.widths[d])])
                               for d in range(3))
        self.N = (p * nx + 1, p * ny + 1, p * nz + 1)
        self.n_nodes = self.N[0] * self.N[1] * self.N[2]
        self.n_cells = nx * ny * nz
        n1 = p + 1
        self.nl = n1 ** 3
        cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        cx, cy, cz = cx.reshape(-1), cy.reshape(-1), cz.reshape(-1)
        conn = np.empty((self.n_cells, self.nl), dtype=np.int64)
        for c in range(n1):
            for b in range(n1):
                for a in range(n1):
                    l = a + n1 * (b + n1 * c)
                    conn[:, l] = self.node_index(p * cx + a, p * cy + b, p * cz + c)
        self.conn = conn

    def node_index(self, i, j, k):
        return i + self.N[0] * (j + self.N[1] * k)

    def node_ijk(self):
        idx = np.arange(self.n_nodes)
        i = idx % self.N[0]
        j = (idx // self.N[0]) % self.N[1]
        k = idx // (self.N[0] * self.N[1])
        return i, j, k

    def node_xyz(self):
        i, j, k = self.node_ijk()
        if self.H is not None:
            hx, hy, hz = (self.H[d] / self.p for d in range(3))
            return (self.origin[0] + i * hx, self.origin[1] + j * hy, self.origin[2] + k * hz)
        out = []
        for d, idx in enumerate((i, j, k)):
            c = np.minimum(idx // self.p, self.widths[d].size - 1)
            out.append(self.faces[d][c] + (idx - self.p * c) * self.widths[d][c] / self.p)
        return tuple(out)

    def width(self, d: int, c: int) -> float:
        """Width of cell layer c along axis d."""
        return self.H[d] if self.H is not None else float(self.widths[d][c])

    def locate(self, d: int, v: float):
        """Cell layer along axis d that holds coordinate v (clamped to the
        mesh) and the local coordinate of v in it."""
        n = self.widths[d].size
        if self.H is not None:
            s = (v - self.origin[d]) / self.H[d]
            c = int(min(max(math.floor(s), 0), n - 1))
            return c, s - c
        c = int(min(max(np.searchsorted(self.faces[d], v, side="right") - 1, 0), n - 1))
        return c, (v - self.faces[d][c]) / self.widths[d][c]

    def cell_widths(self):
        """(hx, hy, hz) of every cell: [cells, 3]."""
        cz, cy, cx = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx), indexing="ij")
        return np.stack([self.widths[0][cx.reshape(-1)], self.widths[1][cy.reshape(-1)],
                         self.widths[2][cz.reshape(-1)]], axis=1)

    def face_nodes(self, face: int) -> np.ndarray:
        i, j, k = self.node_ijk()
        axis, side = face // 2, face % 2
        coord = (i, j, k)[axis]
        last = self.N[axis] - 1
        return np.nonzero(coord == (last if side else 0))[0]


# ---------------------------------------------------------------------------
# Reference element, evaluated directly at the Gauss points
# ---------------------------------------------------------------------------
def reference_element(p: int, H, nq: Optional[int] = None):
    """Shape values N[q, l], physical gradients G[q, l, d] and weights W[q]
    (including the cell volume) at the nq^3 tensor Gauss points of a cell of
    size H = (Hx, Hy, Hz).  Local node l = a + n*(b + n*c)."""
    n = p + 1
    nq = n if nq is None else nq
    xi, w = gauss01(nq)
    nl = n ** 3
    N = np.zeros((nq ** 3, nl))
    G = np.zeros((nq ** 3, nl, 3))
    W = np.zeros(nq ** 3)
    vol = H[0] * H[1] * H[2]
    for qz in range(nq):
        for qy in range(nq):
            for qx in range(nq):
                q = qx + nq * (qy + nq * qz)
                W[q] = w[qx] * w[qy] * w[qz] * vol
                for c in range(n):
                    for b in range(n):
                        for a in range(n):
                            l = a + n * (b + n * c)
                            vx, vy, vz = (lagrange_value(p, a, xi[qx]), lagrange_value(p, b, xi[qy]),
                                          lagrange_value(p, c, xi[qz]))
                            dx, dy, dz = (lagrange_deriv(p, a, xi[qx]), lagrange_deriv(p, b, xi[qy]),
                                          lagrange_deriv(p, c, xi[qz]))
                            N[q, l] = vx * vy * vz
                            G[q, l, 0] = dx * vy * vz / H[0]
                            G[q, l, 1] = vx * dy * vz / H[1]
                            G[q, l, 2] = vx * vy * dz / H[2]
    return N, G, W


def element_mass(N, W):
    return np.einsum("q,ql,qm->lm", W, N, N)


def element_stiffness(G, W):
    return np.einsum("q,qld,qmd->lm", W, G, G)


def assemble(mesh: Mesh, coef: np.ndarray, Ke: np.ndarray) -> sp.csr_matrix:
    """Global matrix sum_c coef[c] * Ke (Ke either [nl, nl] or [cells, nl, nl])."""
    nl = mesh.nl
    rows = np.repeat(mesh.conn[:, :, None], nl, axis=2)
    cols = np.repeat(mesh.conn[:, None, :], nl, axis=1)
    if Ke.ndim == 2:
        data = coef[:, None, None] * Ke[None, :, :]
    else:
        data = coef[:, None, None] * Ke
    A = sp.coo_matrix((data.reshape(-1), (rows.reshape(-1), cols.reshape(-1))),
                      shape=(mesh.n_nodes, mesh.n_nodes))
    return A.tocsr()


def darcy_at_qp(mesh: Mesh, K: np.ndarray, G: np.ndarray, h: np.ndarray) -> np.ndarray:
    """q = -K_c grad h at every Gauss point of every cell: [cells, q, 3].
    G is [q, l, d] (one cell size) or [cells, q, l, d] (graded)."""
    he = h[mesh.conn]                                   # [c, l]
    gh = np.einsum("cl,qld->cqd", he, G) if G.ndim == 3 else np.einsum("cl,cqld->cqd", he, G)
    return -K[:, None, None] * gh


def advection_elements(N, G, W, qf: np.ndarray, cw: float) -> np.ndarray:
    """C_e[c, l, m] = sum_q W_q c_w N_l(q) (q_c(q) . grad N_m(q)); G, W per
    cell ([cells, q, l, d], [cells, q]) on graded meshes."""
    if G.ndim == 3:
        qg = np.einsum("cqd,qmd->cqm", qf, G)           # q . grad N_m
        return cw * np.einsum("q,ql,cqm->clm", W, N, qg)
    qg = np.einsum("cqd,cqmd->cqm", qf, G)
    return cw * np.einsum("cq,ql,cqm->clm", W, N, qg)


def cell_geometry(mesh: Mesh, p: int, cells=None):
    """Shape values and per-cell gradients, weights, mass and stiffness
    element matrices: N [q, l] and G, W, Me, Ke for one cell size, or with a
    leading cell axis on a graded mesh (reference_element of each cell; of
    the cells listed in `cells` only, when given)."""
    if mesh.H is not None:
        N, G, W = reference_element(p, mesh.H)
        return N, G, W, element_mass(N, W), element_stiffness(G, W)
    hw = mesh.cell_widths()
    if cells is not None:
        hw = hw[np.asarray(cells, dtype=np.int64)]
    # reference_element of a cell of widths (hx, hy, hz): the unit cell's
    # gradients divided by the widths and its weights times the volume
    N, G1, W1 = reference_element(p, (1.0, 1.0, 1.0))
    G = G1[None, :, :, :] / hw[:, None, None, :]
    W = W1[None, :] * np.prod(hw, axis=1)[:, None]
    Me = np.einsum("cq,ql,qm->clm", W, N, N)
    Ke = np.einsum("cq,cqld,cqmd->clm", W, G, G)
    return N, G, W, Me, Ke


# ---------------------------------------------------------------------------
# Loads
# ---------------------------------------------------------------------------
def _column_weights(mesh: Mesh, x: float, y: float):
    """Cell column containing (x, y) and the x / y shape factors there."""
    p = mesh.p
    out = []
    for d, v in ((0, x), (1, y)):
        c, xi = mesh.locate(d, v)
        out.append((c, [lagrange_value(p, a, xi) for a in range(p + 1)]))
    return out


def line_weights(mesh: Mesh, x: float, y: float, z_top: float, z_bot: float) -> Dict[int, float]:
    """w_i = int_{z_bot}^{z_top} N_i(x, y, z) dz for a vertical segment."""
    p = mesh.p
    (cx, fx), (cy, fy) = _column_weights(mesh, x, y)
    z0 = mesh.origin[2]
    lo, hi = max(min(z_bot, z_top), z0), min(max(z_bot, z_top), z0 + mesh.extent[2])
    w: Dict[int, float] = {}
    if hi <= lo:
        return w
    xg, wg = gauss01(3)
    for cz in range(mesh.nz):
        a0, a1, Hz = mesh.faces[2][cz], mesh.faces[2][cz + 1], mesh.width(2, cz)
        s0, s1 = max(a0, lo), min(a1, hi)
        if s1 <= s0:
            continue
        # exact integral of phi_c over [s0, s1] in cell-local coordinates
        for c in range(p + 1):
            Iz = 0.0
            for g in range(3):
                zz = s0 + (s1 - s0) * xg[g]
                Iz += wg[g] * (s1 - s0) * lagrange_value(p, c, (zz - a0) / Hz)
            for b in range(p + 1):
                for a in range(p + 1):
                    node = mesh.node_index(p * cx + a, p * cy + b, p * cz + c)
                    w[node] = w.get(node, 0.0) + fx[a] * fy[b] * Iz
    return w


def gaussian_cell_integrals(mesh: Mesh, axis: int, centre: float, sigma: float, nq: int = 10):
    """I[(c, a)] = int_cell phi_a(x) g(x) dx with g the normal density of mean
    `centre` and standard deviation `sigma` along `axis`, by an nq-point Gauss
    rule on every cell within 10 sigma of the centre."""
    p = mesh.p
    xg, wg = gauss01(nq)
    n = (mesh.nx, mesh.ny, mesh.nz)[axis]
    out = {}
    for c in range(n):
        a0, H = mesh.faces[axis][c], mesh.width(axis, c)
        if a0 > centre + 10 * sigma or a0 + H < centre - 10 * sigma:
            continue
        for a in range(p + 1):
            s = 0.0
            for g in range(nq):
                xx = a0 + H * xg[g]
                dens = math.exp(-0.5 * ((xx - centre) / sigma) ** 2) / (math.sqrt(2 * math.pi) * sigma)
                s += wg[g] * H * lagrange_value(p, a, xg[g]) * dens
            out[(c, a)] = s
    return out


def segment_z_integrals(mesh: Mesh, z_top: float, z_bot: float):
    """J[(cz, c)] = int over [z_bot, z_top] of phi_c on cell layer cz."""
    p = mesh.p
    z0 = mesh.origin[2]
    lo, hi = max(min(z_bot, z_top), z0), min(max(z_bot, z_top), z0 + mesh.extent[2])
    xg, wg = gauss01(3)
    out = {}
    for cz in range(mesh.nz):
        a0, a1, Hz = mesh.faces[2][cz], mesh.faces[2][cz + 1], mesh.width(2, cz)
        s0, s1 = max(a0, lo), min(a1, hi)
        if s1 <= s0:
            continue
        for c in range(p + 1):
            out[(cz, c)] = sum(wg[g] * (s1 - s0) * lagrange_value(p, c, (s0 + (s1 - s0) * xg[g] - a0) / Hz)
                               for g in range(3))
    return out


def well_weights(mesh: Mesh, wl) -> Dict[int, float]:
    """Source weights of a well: w_i = int N_i(x, y, z) s(x, y) dz dx dy over
    the screen, with s a line (sigma = 0) or a lateral normal density of
    standard deviation sigma (the well's spread), so that sum_i w_i equals the
    screen length inside the box."""
    sigma = float(wl[6]) if len(wl) > 6 else 0.0
    if sigma <= 0.0:
        return line_weights(mesh, wl[0], wl[1], wl[2], wl[3])
    p = mesh.p
    Ix = gaussian_cell_integrals(mesh, 0, wl[0], sigma)
    Iy = gaussian_cell_integrals(mesh, 1, wl[1], sigma)
    Jz = segment_z_integrals(mesh, wl[2], wl[3])
    out: Dict[int, float] = {}
    for (cz, c), vz in Jz.items():
        for (cy, b), vy in Iy.items():
            for (cx, a), vx in Ix.items():
                nd = mesh.node_index(p * cx + a, p * cy + b, p * cz + c)
                out[nd] = out.get(nd, 0.0) + vx * vy * vz
    return out


def face_load(mesh: Mesh, face: int, value: float) -> np.ndarray:
    """F_i = value * int_face N_i dS for a uniform normal flux into the domain."""
    p = mesh.p
    F = np.zeros(mesh.n_nodes)
    axis = face // 2
    t1, t2 = [d for d in range(3) if d != axis]
    xg, wg = gauss01(p + 1)
    i1 = [sum(wg[g] * lagrange_value(p, a, xg[g]) for g in range(p + 1)) for a in range(p + 1)]
    n1, n2 = (mesh.nx, mesh.ny, mesh.nz)[t1], (mesh.nx, mesh.ny, mesh.nz)[t2]
    fixed = 0 if face % 2 == 0 else mesh.N[axis] - 1
    for c2 in range(n2):
        for c1 in range(n1):
            for b in range(p + 1):
                for a in range(p + 1):
                    ijk = [0, 0, 0]
                    ijk[axis] = fixed
                    ijk[t1] = p * c1 + a
                    ijk[t2] = p * c2 + b
                    F[mesh.node_index(*ijk)] += value * i1[a] * mesh.width(t1, c1) * i1[b] * mesh.width(t2, c2)
    return F


def box_snap(mesh: Mesh, box):
    """Cell-face indices (i0, i1, j0, j1, k) of a box source's rectangle.

    Each edge x0, x1, y0, y1 moves to the nearest cell face (ties upwards)
    and is clamped to the mesh; z moves to the nearest plane of horizontal
    cell faces.  The rectangle covers cells i0 <= cx < i1, j0 <= cy < j1 on
    the node plane p * k.
    """
    def nearest(v, d, n):
        if mesh.H is not None:
            return int(min(max(math.floor((v - mesh.origin[d]) / mesh.H[d] + 0.5), 0), n))
        dist = np.abs(mesh.faces[d] - v)
        return int(np.nonzero(dist == dist.min())[0][-1])
    i0, i1 = nearest(box[0], 0, mesh.nx), nearest(box[1], 0, mesh.nx)
    j0, j1 = nearest(box[2], 1, mesh.ny), nearest(box[3], 1, mesh.ny)
    k = nearest(box[4], 2, mesh.nz)
    return i0, i1, j0, j1, k


def box_weights(mesh: Mesh, box) -> Dict[int, float]:
    """w_i = int_R N_i dS over the snapped horizontal rectangle R of a box
    source, by (p+1) x (p+1) Gauss points on every cell face inside R."""
    p = mesh.p
    i0, i1, j0, j1, k = box_snap(mesh, box)
    xg, wg = gauss01(p + 1)
    w: Dict[int, float] = {}
    for cy in range(j0, j1):
        for cx in range(i0, i1):
            Hx, Hy = mesh.width(0, cx), mesh.width(1, cy)
            for gy in range(p + 1):
                for gx in range(p + 1):
                    dS = wg[gx] * Hx * wg[gy] * Hy
                    for b in range(p + 1):
                        for a in range(p + 1):
                            node = mesh.node_index(p * cx + a, p * cy + b, p * k)
                            w[node] = w.get(node, 0.0) + dS * lagrange_value(p, a, xg[gx]) * \
                                lagrange_value(p, b, xg[gy])
    return w


def box_flux(box, t: float) -> float:
    """q(t) = mean + amp sin(2 pi t / period + phase), W/m^2 into the domain."""
    return box[5] + box[6] * math.sin(2.0 * math.pi * t / box[7] + box[8])


def face_load_nodal(mesh: Mesh, face: int, q: np.ndarray) -> np.ndarray:
    """F_i = int_face N_i q_h dS for a normal flux given at the face nodes
    (ascending node order) and interpolated by the face's shape functions,
    q_h = sum_j q_j N_j, integrated by (p+1)^2 Gauss points per cell face."""
    p = mesh.p
    F = np.zeros(mesh.n_nodes)
    axis = face // 2
    t1, t2 = [d for d in range(3) if d != axis]
    nodes = mesh.face_nodes(face)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    if q.size != nodes.size:
        raise ValueError(f"face {face} has {nodes.size} nodes, got {q.size} values")
    qn = np.zeros(mesh.n_nodes)
    qn[nodes] = q
    xg, wg = gauss01(p + 1)
    ncs = (mesh.nx, mesh.ny, mesh.nz)
    fixed = 0 if face % 2 == 0 else mesh.N[axis] - 1
    for c2 in range(ncs[t2]):
        for c1 in range(ncs[t1]):
            dA = mesh.width(t1, c1) * mesh.width(t2, c2)
            local = []
            for b in range(p + 1):
                for a in range(p + 1):
                    ijk = [0, 0, 0]
                    ijk[axis] = fixed
                    ijk[t1] = p * c1 + a
                    ijk[t2] = p * c2 + b
                    local.append((a, b, mesh.node_index(*ijk)))
            for g2 in range(p + 1):
                for g1 in range(p + 1):
                    Ng = [lagrange_value(p, a, xg[g1]) * lagrange_value(p, b, xg[g2]) for a, b, _ in local]
                    qg = sum(n * qn[nd] for n, (_, _, nd) in zip(Ng, local))
                    for n, (_, _, nd) in zip(Ng, local):
                        F[nd] += wg[g1] * wg[g2] * dA * n * qg
    return F


def pile_amplitude(pile, t: float) -> float:
    """q_l(t) = mean + amp sin(2 pi t / period + phase), W/m."""
    return pile[4] + pile[5] * math.sin(2.0 * math.pi * t / pile[6] + pile[7])


# ---------------------------------------------------------------------------
# Dirichlet handling and solves
# ---------------------------------------------------------------------------
def dirichlet_data(mesh: Mesh, bc: Dict[int, Tuple[int, float]]):
    """Mask and values of Dirichlet nodes; later faces override earlier ones
    on shared edges.  A face's value is a scalar or one value per face node
    in ascending node order (the lower tangential axis fastest)."""
    mask = np.zeros(mesh.n_nodes, dtype=bool)
    g = np.zeros(mesh.n_nodes)
    for face in range(6):
        if face in bc and bc[face][0] == DIRICHLET:
            nodes = mesh.face_nodes(face)
            mask[nodes] = True
            g[nodes] = bc[face][1]
    return mask, g


def pile_surface_nodes(mesh: Mesh, row) -> np.ndarray:
    """Nodes held at a pile's temperature: those within `radius` of the pile
    axis (x, y) and between z_bot and z_top, or, when no node lies within the
    radius, the node column nearest the axis (lowest index on ties).
    row = (x, y, z_top, z_bot, radius, T_mean, T_amp, period, phase)."""
    X, Y, Z = mesh.node_xyz()
    eps = 1e-9 * max(mesh.extent)
    inz = (Z >= min(row[2], row[3]) - eps) & (Z <= max(row[2], row[3]) + eps)
    lat = (X - row[0]) ** 2 + (Y - row[1]) ** 2
    sel = inz & (lat <= row[4] ** 2 + eps)
    if not sel.any():
        cand = np.nonzero(inz)[0]
        if cand.size == 0:
            raise ValueError("pile lies outside the mesh")
        best = cand[np.argmin(lat[cand])]
        sel = inz & (X == X[best]) & (Y == Y[best])
    return np.nonzero(sel)[0]


def pile_temperature(row, t: float) -> float:
    """Square wave T_mean + T_amp sign(sin(2 pi t / period + phase)), with
    sign(0) = +1: the warm half first (Section 3.3: 301.55 K for six months,
    then 275.55 K)."""
    return row[5] + row[6] * (1.0 if math.sin(2.0 * math.pi * t / row[7] + row[8]) >= 0.0 else -1.0)


def seasonal_value(v, t: float) -> float:
    """mean + amp sin(2 pi t / period + phase) for v = (mean, amp, period, phase)."""
    return v[0] + v[1] * math.sin(2.0 * math.pi * t / v[2] + v[3])


def constrain(A: sp.csr_matrix, mask: np.ndarray) -> sp.csr_matrix:
    """A0 = P A P + (I - P), P = projector on free nodes."""
    free = (~mask).astype(np.float64)
    P = sp.diags(free)
    return (P @ A @ P + sp.diags(mask.astype(np.float64))).tocsr()


def lifted_rhs(A: sp.csr_matrix, rhs: np.ndarray, mask: np.ndarray, g: np.ndarray) -> np.ndarray:
    gD = np.where(mask, g, 0.0)
    b = rhs - A @ gD
    return np.where(mask, g, b)


def solve(A0: sp.csr_matrix, b: np.ndarray, method: str = "direct", tol: float = 1e-14,
          x0: Optional[np.ndarray] = None, maxiter: int = 100000):
    if not np.any(b):
        return np.zeros_like(b)
    if method == "direct":
        return spla.spsolve(A0.tocsc(), b)
    M = sp.diags(1.0 / A0.diagonal())
    if method == "cg":
        x, info = spla.cg(A0, b, x0=x0, rtol=tol, atol=0.0, M=M, maxiter=maxiter)
    else:
        x, info = spla.bicgstab(A0, b, x0=x0, rtol=tol, atol=0.0, M=M, maxiter=maxiter)
    if info != 0:
        raise RuntimeError(f"oracle iterative solve did not converge (info={info})")
    return x


# ---------------------------------------------------------------------------
# The simulator
# ---------------------------------------------------------------------------
class _TimeDirichlet:
    """Dirichlet values that change with time: faces with a seasonal value
    (mean, amp, period, phase), re-evaluated at each step's t^{n+1}, and pile
    surfaces held at a square-wave temperature.  Faces keep their order on
    shared edges (the higher face index wins); pile nodes override faces."""

    def _init_time_dirichlet(self, sc):
        m = self.mesh
        self.seasonal = {f: dict(d) for f, d in (getattr(sc, "bc_seasonal", None) or {}).items()}
        for f, faces in self.seasonal.items():
            bc_mask = dict(sc.bc.get(f, {}))
            for face in faces:
                bc_mask[face] = (DIRICHLET, 0.0)
            self.dmask[f], self.gval[f] = dirichlet_data(m, bc_mask)
        self.pile_temps = np.asarray(getattr(sc, "pile_temps", np.zeros((0, 9))), dtype=np.float64).reshape(-1, 9)
        self.pile_nodes = [pile_surface_nodes(m, row) for row in self.pile_temps]
        for nodes in self.pile_nodes:
            self.dmask[TEMP][nodes] = True

    def g_at(self, field: int, t: float) -> np.ndarray:
        """Dirichlet values of `field` at time t."""
        seas = self.seasonal.get(field, {})
        if not seas and (field != TEMP or not self.pile_nodes):
            return self.gval[field]
        bc_t = dict(self.sc.bc.get(field, {}))
        for face, v in seas.items():
            bc_t[face] = (DIRICHLET, seasonal_value(v, t))
        _, g = dirichlet_data(self.mesh, bc_t)
        if field == TEMP:
            for row, nodes in zip(self.pile_temps, self.pile_nodes):
                g[nodes] = pile_temperature(row, t)
        return g


class OracleSim(_TimeDirichlet):
    """Plain FP64 reference of one coupled step (head, then heat)."""

    def __init__(self, sc, solver: str = "direct", tol: float = 1e-14):
        self.sc = sc
        self.mesh = Mesh(sc.nx, sc.ny, sc.nz, sc.order, sc.origin, sc.extent, getattr(sc, "spacing", None))
        m = self.mesh
        self.N, self.G, self.W, self.Me, self.Ke = cell_geometry(m, sc.order)
        nc = m.n_cells
        self.K = np.asarray(sc.K, dtype=np.float64)
        lam, cT, self.cw, self.Ss = bulk_properties(sc)
        self.lam_c = np.asarray(sc.lam_cells if sc.lam_cells is not None else np.full(nc, lam))
        self.cT_c = np.asarray(sc.cT_cells if sc.cT_cells is not None else np.full(nc, cT))
        self.M = assemble(m, np.ones(nc), self.Me)
        self.KK = assemble(m, self.K, self.Ke)
        self.McT = assemble(m, self.cT_c, self.Me)
        self.Llam = assemble(m, self.lam_c, self.Ke)
        self.dmask = {}
        self.gval = {}
        for f in (HEAD, TEMP):
            self.dmask[f], self.gval[f] = dirichlet_data(m, sc.bc.get(f, {}))
        self._init_time_dirichlet(sc)
        # static loads: Neumann faces
        self.F_static = {HEAD: np.zeros(m.n_nodes), TEMP: np.zeros(m.n_nodes)}
        for f in (HEAD, TEMP):
            for face, (typ, val) in sc.bc.get(f, {}).items():
                if typ == FLUX:
                    self.F_static[f] += face_load(m, face, val) if np.ndim(val) == 0 else \
                        face_load_nodal(m, face, val)
        # wells: head source and lumped heat injection term
        self.d_well = np.zeros(m.n_nodes)
        self.Tin_well = np.zeros(m.n_nodes)       # sum d*T_in
        wells = np.asarray(sc.wells, dtype=np.float64)
        wells = wells.reshape(-1, wells.shape[-1] if wells.size else 7)
        for wl in wells:
            L = abs(wl[2] - wl[3])
            if L <= 0:
                continue
            wts = well_weights(m, wl)
            for node, wv in wts.items():
                self.F_static[HEAD][node] += wl[4] / L * wv
                if wl[4] > 0:
                    self.d_well[node] += self.cw * wl[4] / L * wv
                    self.Tin_well[node] += self.cw * wl[4] / L * wv * wl[5]
        self.pile_w = [line_weights(m, pl[0], pl[1], pl[2], pl[3])
                       for pl in np.asarray(sc.piles).reshape(-1, 8)]
        self.boxes = np.asarray(getattr(sc, "boxes", np.zeros((0, 9))), dtype=np.float64).reshape(-1, 9)
        self.box_w = [box_weights(m, bx) for bx in self.boxes]
        self.extra = {HEAD: np.zeros(m.n_nodes), TEMP: np.zeros(m.n_nodes)}
        self.h = np.array(sc.h0, dtype=np.float64)
        self.T = np.array(sc.T0, dtype=np.float64)
        self.t = 0.0
        self.solver = solver
        self.tol = tol

    # -- operators (constrained, as the solver sees them) -------------------
    def head_matrix(self, dt):
        return self.Ss * self.M + dt * self.KK

    def heat_matrix(self, dt, h):
        qf = darcy_at_qp(self.mesh, self.K, self.G, h)
        Ce = advection_elements(self.N, self.G, self.W, qf, self.cw)
        C = assemble(self.mesh, np.ones(self.mesh.n_cells), Ce)
        return self.McT + dt * self.Llam + dt * C + dt * sp.diags(self.d_well)

    def apply_head(self, x, dt):
        return constrain(self.head_matrix(dt), self.dmask[HEAD]) @ x

    def apply_heat(self, x, h, dt):
        return constrain(self.heat_matrix(dt, h), self.dmask[TEMP]) @ x

    def diag_head(self, dt):
        return constrain(self.head_matrix(dt), self.dmask[HEAD]).diagonal()

    def diag_heat(self, h, dt):
        return constrain(self.heat_matrix(dt, h), self.dmask[TEMP]).diagonal()

    # -- loads ----------------------------------------------------------------
    def head_load(self, t):
        return self.F_static[HEAD] + self.extra[HEAD]

    def heat_load(self, t):
        F = self.F_static[TEMP] + self.extra[TEMP] + self.Tin_well
        for pl, wts in zip(np.asarray(self.sc.piles).reshape(-1, 8), self.pile_w):
            a = pile_amplitude(pl, t)
            for node, wv in wts.items():
                F[node] += a * wv
        for bx, wts in zip(self.boxes, self.box_w):
            a = box_flux(bx, t)
            for node, wv in wts.items():
                F[node] += a * wv
        return F

    def head_rhs(self, dt, t1):
        A = self.head_matrix(dt)
        rhs = self.Ss * (self.M @ self.h) + dt * self.head_load(t1)
        return lifted_rhs(A, rhs, self.dmask[HEAD], self.g_at(HEAD, t1))

    def heat_rhs(self, dt, t1, h1):
        A = self.heat_matrix(dt, h1)
        rhs = self.McT @ self.T + dt * self.heat_load(t1)
        return lifted_rhs(A, rhs, self.dmask[TEMP], self.g_at(TEMP, t1))

    # -- one backward Euler step: head first, then heat with q(h^{n+1}) -------
    def step(self, dt):
        t1 = self.t + dt
        Ah = self.head_matrix(dt)
        bh = lifted_rhs(Ah, self.Ss * (self.M @ self.h) + dt * self.head_load(t1),
                        self.dmask[HEAD], self.g_at(HEAD, t1))
        h1 = solve(constrain(Ah, self.dmask[HEAD]), bh, self.solver if self.solver == "direct" else "cg",
                   self.tol, x0=self.h)
        AT = self.heat_matrix(dt, h1)
        bT = lifted_rhs(AT, self.McT @ self.T + dt * self.heat_load(t1),
                        self.dmask[TEMP], self.g_at(TEMP, t1))
        T1 = solve(constrain(AT, self.dmask[TEMP]), bT,
                   self.solver if self.solver == "direct" else "bicgstab", self.tol, x0=self.T)
        self.h, self.T, self.t = h1, T1, t1
        return h1, T1

    # -- outputs ----------------------------------------------------------------
    def cell_flux(self, h=None):
        """Darcy flux q = -K_c grad h at each cell centre: [3, cells]."""
        h = self.h if h is None else h
        m = self.mesh
        p = m.p
        n = p + 1
        he = h[m.conn]
        hw = m.cell_widths()
        g = np.zeros((m.n_cells, 3))
        for c in range(n):
            for b in range(n):
                for a in range(n):
                    l = a + n * (b + n * c)
                    vx, vy, vz = (lagrange_value(p, a, 0.5), lagrange_value(p, b, 0.5),
                                  lagrange_value(p, c, 0.5))
                    dx, dy, dz = (lagrange_deriv(p, a, 0.5), lagrange_deriv(p, b, 0.5),
                                  lagrange_deriv(p, c, 0.5))
                    g[:, 0] += he[:, l] * dx * vy * vz / hw[:, 0]
                    g[:, 1] += he[:, l] * vx * dy * vz / hw[:, 1]
                    g[:, 2] += he[:, l] * vx * vy * dz / hw[:, 2]
        return (-self.K[:, None] * g).T.copy()


# ---------------------------------------------------------------------------
# Selected rows at any mesh size
# ---------------------------------------------------------------------------
def cells_of_node(mesh: Mesh, node: int):
    """(cell, local index) for every cell that holds the node."""
    p = mesh.p
    n1 = p + 1
    ijk = (node % mesh.N[0], (node // mesh.N[0]) % mesh.N[1], node // (mesh.N[0] * mesh.N[1]))
    per_axis = []
    for d, nc in enumerate((mesh.nx, mesh.ny, mesh.nz)):
        opts = []
        for c in range(max(0, ijk[d] // p - 1), min(nc - 1, ijk[d] // p) + 1):
            a = ijk[d] - p * c
            if 0 <= a <= p:
                opts.append((c, a))
        per_axis.append(opts)
    out = []
    for cz, c3 in per_axis[2]:
        for cy, b in per_axis[1]:
            for cx, a in per_axis[0]:
                out.append((cx + mesh.nx * (cy + mesh.ny * cz), a + n1 * (b + n1 * c3)))
    return out


class RowOracle(_TimeDirichlet):
    """Rows of the constrained operators A0 and of the lifted right-hand
    sides b of one step at selected nodes, for meshes too large to assemble.

    The definitions are those of OracleSim (the same element matrices from
    shape functions at the Gauss points, the same loads, Dirichlet rows as
    identity rows and Dirichlet columns moved to the right-hand side), but
    each requested row is summed cell by cell over the cells that hold its
    node.  Every row also returns the sum of the absolute values of its
    terms, the scale of its rounding error.
    """

    def __init__(self, sc):
        self.sc = sc
        m = Mesh(sc.nx, sc.ny, sc.nz, sc.order, sc.origin, sc.extent, getattr(sc, "spacing", None))
        self.mesh = m
        # on a graded mesh the element matrices of a cell are formed when a
        # row first needs them (the same cell_geometry, one cell at a time)
        self.graded = m.H is None
        self._geo_cache = {}
        if self.graded:
            self.N = cell_geometry(m, sc.order, cells=[0])[0]
        else:
            self.N, self.G, self.W, self.Me, self.Ke = cell_geometry(m, sc.order)
        nc = m.n_cells
        self.K = np.asarray(sc.K, dtype=np.float64)
        lam, cT, self.cw, self.Ss = bulk_properties(sc)
        self.lam_c = np.asarray(sc.lam_cells if sc.lam_cells is not None else np.full(nc, lam))
        self.cT_c = np.asarray(sc.cT_cells if sc.cT_cells is not None else np.full(nc, cT))
        self.dmask, self.gval, self.F_static = {}, {}, {}
        for f in (HEAD, TEMP):
            self.dmask[f], self.gval[f] = dirichlet_data(m, sc.bc.get(f, {}))
            F = np.zeros(m.n_nodes)
            for face, (typ, val) in sc.bc.get(f, {}).items():
                if typ == FLUX:
                    F += face_load(m, face, val) if np.ndim(val) == 0 else face_load_nodal(m, face, val)
            self.F_static[f] = F
        self._init_time_dirichlet(sc)
        self.d_well = np.zeros(m.n_nodes)
        self.Tin_well = np.zeros(m.n_nodes)
        wells = np.asarray(sc.wells, dtype=np.float64)
        for wl in wells.reshape(-1, wells.shape[-1] if wells.size else 7):
            L = abs(wl[2] - wl[3])
            if L <= 0:
                continue
            for node, wv in well_weights(m, wl).items():
                self.F_static[HEAD][node] += wl[4] / L * wv
                if wl[4] > 0:
                    self.d_well[node] += self.cw * wl[4] / L * wv
                    self.Tin_well[node] += self.cw * wl[4] / L * wv * wl[5]
        self.piles = np.asarray(sc.piles, dtype=np.float64).reshape(-1, 8)
        self.pile_w = [line_weights(m, pl[0], pl[1], pl[2], pl[3]) for pl in self.piles]
        self.boxes = np.asarray(getattr(sc, "boxes", np.zeros((0, 9))), dtype=np.float64).reshape(-1, 9)
        self.box_w = [box_weights(m, bx) for bx in self.boxes]

    # -- element matrices of one cell ------------------------------------------
    def _geo(self, c):
        """G, W, Me, Ke of cell c."""
        if not self.graded:
            return self.G, self.W, self.Me, self.Ke
        if c not in self._geo_cache:
            _, G, W, Me, Ke = cell_geometry(self.mesh, self.mesh.p, cells=[c])
            self._geo_cache[c] = (G[0], W[0], Me[0], Ke[0])
        return self._geo_cache[c]

    def _advection(self, c, h):
        G, W, _, _ = self._geo(c)
        qf = -self.K[c] * np.einsum("l,qld->qd", h[self.mesh.conn[c]], G)
        qg = np.einsum("qd,qmd->qm", qf, G)
        return self.cw * np.einsum("q,ql,qm->lm", W, self.N, qg)

    def _cell_matrix(self, field, c, dt, h=None, mass_only=False):
        _, _, Me, Ke = self._geo(c)
        if field == HEAD:
            return self.Ss * Me if mass_only else self.Ss * Me + dt * self.K[c] * Ke
        if mass_only:
            return self.cT_c[c] * Me
        return self.cT_c[c] * Me + dt * self.lam_c[c] * Ke + dt * self._advection(c, h)

    def _row(self, field, i, dt, x, cols, h=None, mass_only=False):
        """sum_j A_ij x_j over the columns j selected by cols ('all', 'free'
        or 'dirichlet'), with the sum of |A_ij x_j|."""
        mask = self.dmask[field]
        s = a = 0.0
        for c, l in cells_of_node(self.mesh, i):
            nodes = self.mesh.conn[c]
            keep = np.ones(nodes.size, dtype=bool) if cols == "all" else \
                (~mask[nodes] if cols == "free" else mask[nodes])
            terms = self._cell_matrix(field, c, dt, h, mass_only)[l] * x[nodes] * keep
            s += terms.sum()
            a += np.abs(terms).sum()
        if field == TEMP and not mass_only and (cols == "all" or (cols == "free") != mask[i]):
            t = dt * self.d_well[i] * x[i]
            s += t
            a += abs(t)
        return s, a

    # -- rows of A0 x and of b ----------------------------------------------------
    def apply_rows(self, field, dt, x, rows, h=None):
        """(A0 x)_i: x_i on Dirichlet rows, the free-column sum elsewhere.
        The heat operator takes the Darcy flux of the head h."""
        x = np.asarray(x, dtype=np.float64)
        y, a = np.zeros(len(rows)), np.zeros(len(rows))
        for k, i in enumerate(rows):
            if self.dmask[field][i]:
                y[k], a[k] = x[i], abs(x[i])
            else:
                y[k], a[k] = self._row(field, i, dt, x, "free", h)
        return y, a

    def load(self, field, t, i):
        """F_i(t): face fluxes, wells, and for heat the piles and boxes."""
        F = self.F_static[field][i]
        if field == TEMP:
            F += self.Tin_well[i]
            for pl, wts in zip(self.piles, self.pile_w):
                F += pile_amplitude(pl, t) * wts.get(i, 0.0)
            for bx, wts in zip(self.boxes, self.box_w):
                F += box_flux(bx, t) * wts.get(i, 0.0)
        return F

    def rhs_rows(self, field, dt, t1, state, rows, h=None):
        """b_i of the step from the state (h^n or T^n) to t1: g_i on
        Dirichlet rows, else (c M state)_i + dt F_i(t1) - sum_{j in D} A_ij g_j
        (c = S_s for head, c_T for heat; the heat operator at the head h)."""
        state = np.asarray(state, dtype=np.float64)
        g = self.g_at(field, t1)
        b, a = np.zeros(len(rows)), np.zeros(len(rows))
        for k, i in enumerate(rows):
            if self.dmask[field][i]:
                b[k], a[k] = g[i], abs(g[i])
                continue
            ms, ma = self._row(field, i, dt, state, "all", mass_only=True)
            ls, la = self._row(field, i, dt, g, "dirichlet", h)
            F = dt * self.load(field, t1, i)
            b[k] = ms + F - ls
            a[k] = ma + abs(F) + la
        return b, a
