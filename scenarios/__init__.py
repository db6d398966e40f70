"""Seeded synthetic input generators for the hydrothermal solver.

This module only *draws inputs*: mesh sizes, per-cell hydraulic conductivity
fields, material constants, boundary-condition choices, pile / well tables and
initial fields.  It holds none of the finite element arithmetic (no shape
functions, no quadrature, no operators, no loads), so both the CUDA path and
the CPU oracle can consume the same inputs without sharing any method code.

Material values are handed over raw: porosity, solid and water thermal
conductivities and heat capacities, and the bulk modulus B_poro of Table 1.
The bulk coefficients that the method derives from them (the mixture rules
below Eq. 2 and the specific storage of Eq. 1) are computed by each consumer
on its own side: the oracle in oracle/fem.py, the library by ht_mixture and
ht_specific_storage.  A scenario may instead carry bulk values directly
(lam, cT, Ss), as the Table 3 layers are given.  The synthetic workloads
(sizes, layering, random fields, pile and well layouts) stand in for the
paper's ATES benchmark (Section 2) and Treasure Island energy-pile case
(Section 3), whose site data exist only in figures.

Conventions
-----------
* Structured box [x0, x0+Lx] x [y0, y0+Ly] x [z0, z0+Lz], z up, nx*ny*nz
  hexahedral cells of order p (1 = trilinear Q1, 2 = triquadratic Q2).
* Cell index  c = cx + nx*(cy + ny*cz); node index n = i + Nx*(j + Ny*k),
  Nx = p*nx + 1 (x fastest).
* Faces: 0 x-min, 1 x-max, 2 y-min, 3 y-max, 4 z-min (bottom), 5 z-max (top).
* Piles (line heat sources): rows [x, y, z_top, z_bot, mean, amp, period, phase]
  giving q_l(t) = mean + amp*sin(2*pi*t/period + phase) in W/m.
* Wells: rows [x, y, z_top, z_bot, Q, T_in, sigma]; Q in m^3/s (+ injection)
  spread uniformly along the screen and laterally either on the well axis
  (sigma = 0, a line source) or as a normal density of standard deviation
  sigma (m); injected water enters at temperature T_in.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional, Tuple

import numpy as np

DAY = 86400.0
RHO_W = 1000.0
G_ACC = 9.81

HEAD, TEMP = 0, 1
NONE, DIRICHLET, FLUX = 0, 1, 2


@dataclasses.dataclass
class Scenario:
    """One hydrothermal problem: mesh, coefficients, boundary data, loads."""
    name: str
    nx: int
    ny: int
    nz: int
    order: int
    origin: Tuple[float, float, float]
    extent: Tuple[float, float, float]
    K: np.ndarray                      # [cells] hydraulic conductivity, m/s
    material: "Material"               # raw phase properties (bulk values derived by the consumer)
    bc: Dict[int, Dict[int, Tuple[int, float]]]   # field -> face -> (type, value)
    piles: np.ndarray                  # [n, 8]
    wells: np.ndarray                  # [n, 7]
    h0: np.ndarray                     # [nodes] initial head, m
    T0: np.ndarray                     # [nodes] initial temperature
    dt: float                          # time step, s
    n_steps: int
    lam_cells: Optional[np.ndarray] = None   # optional per-cell lambda
    cT_cells: Optional[np.ndarray] = None    # optional per-cell c_T
    # horizontal heat-flux rectangles [n, 9]: x0, x1, y0, y1, z, mean, amp,
    # period, phase (W/m^2 into the domain), edges snapped to cell faces
    boxes: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 9)))
    # optional graded mesh: cell widths along x, y and z (tensor-product
    # spacing summing to the extent); None for uniform cells
    spacing: Optional[Tuple[np.ndarray, np.ndarray, np.ndarray]] = None
    # optional pile surfaces held at a square-wave temperature [n, 9]: x, y,
    # z_top, z_bot, radius, T_mean, T_amp, period, phase
    pile_temps: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 9)))
    # optional Dirichlet faces whose value follows a seasonal sinusoid:
    # field -> face -> (mean, amp, period, phase)
    bc_seasonal: Dict[int, Dict[int, Tuple[float, float, float, float]]] = \
        dataclasses.field(default_factory=dict)
    # optional bulk values given directly (None: derived from `material` by
    # the consumer): thermal conductivity W/(m K), heat capacity J/(m^3 K),
    # specific storage 1/m
    lam: Optional[float] = None
    cT: Optional[float] = None
    Ss: Optional[float] = None

    @property
    def cw(self) -> float:
        """Volumetric heat capacity of water, J/(m^3 K) (a raw property)."""
        return self.material.c_w

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def node_dims(self) -> Tuple[int, int, int]:
        p = self.order
        return (p * self.nx + 1, p * self.ny + 1, p * self.nz + 1)

    @property
    def n_nodes(self) -> int:
        a, b, c = self.node_dims
        return a * b * c

    def node_coords(self):
        """Node coordinate axes (1D arrays along x, y, z)."""
        Nx, Ny, Nz = self.node_dims
        x0, y0, z0 = self.origin
        Lx, Ly, Lz = self.extent
        if self.spacing is None:
            return (x0 + Lx * np.arange(Nx) / (Nx - 1),
                    y0 + Ly * np.arange(Ny) / (Ny - 1),
                    z0 + Lz * np.arange(Nz) / (Nz - 1))
        out = []
        for o, w in zip(self.origin, self.spacing):
            w = np.asarray(w, dtype=np.float64)
            faces = o + np.concatenate([[0.0], np.cumsum(w)])
            sub = [faces[:-1, None] + w[:, None] * np.arange(self.order)[None, :] / self.order]
            out.append(np.concatenate([np.concatenate(sub, axis=1).reshape(-1), faces[-1:]]))
        return tuple(out)

    def cell_centres(self):
        x0, y0, z0 = self.origin
        Lx, Ly, Lz = self.extent
        return (x0 + Lx * (np.arange(self.nx) + 0.5) / self.nx,
                y0 + Ly * (np.arange(self.ny) + 0.5) / self.ny,
                z0 + Lz * (np.arange(self.nz) + 0.5) / self.nz)


@dataclasses.dataclass(frozen=True)
class Material:
    """Raw properties of the saturated porous medium (Section 2 symbols):
    porosity phi, solid and water thermal conductivities lam_s, lam_w
    (W/(m K)), solid and water volumetric heat capacities c_s, c_w
    (J/(m^3 K)), bulk modulus B_poro (Pa), water density rho_w and gravity g."""
    phi: float
    lam_s: float
    lam_w: float
    c_s: float
    c_w: float
    B_poro: float
    rho_w: float = RHO_W
    g: float = G_ACC


# Sand / water values shared by the synthetic workloads; B_poro from Table 1.
B_PORO_TABLE1 = 1.0e5
SAND = Material(phi=0.3, lam_s=2.5, lam_w=0.6, c_s=2.0e6, c_w=4.18e6, B_poro=B_PORO_TABLE1)


def _linear_x(sc_dims, origin, extent, order, a, b, nx, ny, nz):
    """Nodal field a + b*x (used for initial heads)."""
    p = order
    Nx, Ny, Nz = p * nx + 1, p * ny + 1, p * nz + 1
    x = origin[0] + extent[0] * np.arange(Nx) / (Nx - 1)
    f = np.broadcast_to((a + b * x)[None, None, :], (Nz, Ny, Nx))
    return np.ascontiguousarray(f).reshape(-1).astype(np.float64)


def gaussian_field_fft(shape, spacing, corr_len, sigma, rng):
    """Stationary zero-mean Gaussian field on a periodic grid, covariance
    sigma^2 exp(-r^2 / (2 l^2)), by spectral (FFT) filtering of white noise.

    shape = (nz, ny, nx) cell counts, spacing = (hz, hy, hx).
    """
    nz, ny, nx = shape
    hz, hy, hx = spacing
    noise = rng.standard_normal(shape)
    kz = 2 * np.pi * np.fft.fftfreq(nz, d=hz)
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=hy)
    kx = 2 * np.pi * np.fft.rfftfreq(nx, d=hx)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    amp = np.exp(-0.25 * k2 * corr_len ** 2)          # sqrt of Gaussian spectrum
    f = np.fft.irfftn(np.fft.rfftn(noise) * amp, s=shape, axes=(0, 1, 2))
    std = f.std()
    return sigma * f / (std if std > 0 else 1.0)


def _bc(head: Dict[int, Tuple[int, float]], temp: Dict[int, Tuple[int, float]]):
    return {HEAD: dict(head), TEMP: dict(temp)}


def config1(nx: int = 16, ny: Optional[int] = None, nz: Optional[int] = None,
            order: int = 1, n_steps: int = 10) -> Scenario:
    """Plain workload: 20 m cube, homogeneous sand K = 1e-4 m/s, head gradient
    0.01 along x, T0 = 15, 10 W/m line source on the central vertical axis,
    backward Euler with dt = 1 day."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    L = 20.0
    K = np.full(nx * ny * nz, 1.0e-4)
    h0 = _linear_x(None, (0, 0, 0), (L, L, L), order, 0.2, -0.01, nx, ny, nz)
    Nn = h0.size
    T0 = np.full(Nn, 15.0)
    piles = np.array([[L / 2, L / 2, L, 0.0, 10.0, 0.0, 365 * DAY, 0.0]])
    bc = _bc({0: (DIRICHLET, 0.2), 1: (DIRICHLET, 0.2 - 0.01 * L)},
             {0: (DIRICHLET, 15.0), 1: (DIRICHLET, 15.0), 2: (DIRICHLET, 15.0),
              3: (DIRICHLET, 15.0), 5: (DIRICHLET, 15.0)})
    return Scenario("plain_q1_cube", nx, ny, nz, order, (0.0, 0.0, 0.0), (L, L, L),
                    K, SAND, bc, piles, np.zeros((0, 7)), h0, T0,
                    1.0 * DAY, n_steps)


def config2(nx: int = 128, ny: int = 128, nz: int = 32, seed: int = 2,
            n_steps: int = 180, order: int = 2, well_sigma: float = 1.5) -> Scenario:
    """ATES-like layered aquifer: 200 m x 200 m x 50 m, Q2 cells, three
    horizontal layers (10/12/10 of 32 cell layers, scaled with nz) with iid
    lognormal K per cell (geometric means 1e-6 / 1e-4 / 1e-6 m/s, sigma_lnK =
    0.5), an injection well (+5 L/s at T0 + 10) and an extraction well
    (-5 L/s) 60 m apart, both screened over the aquifer layer; dt = 0.5 day."""
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = 200.0, 200.0, 50.0
    nb = int(round(nz * 10 / 32))
    nt = int(round(nz * 10 / 32))
    nm = nz - nb - nt
    layer_mean = np.concatenate([np.full(nb, 1e-6), np.full(nm, 1e-4), np.full(nt, 1e-6)])
    lnK = np.log(layer_mean)[:, None, None] + 0.5 * rng.standard_normal((nz, ny, nx))
    K = np.exp(lnK).reshape(-1)
    Hz = Lz / nz
    z_lo, z_hi = nb * Hz, (nb + nm) * Hz
    T_amb = 15.0
    # wells snapped to the nearest node column
    p = order
    hx, hy = Lx / (p * nx), Ly / (p * ny)
    def snap(v, h):
        return round(v / h) * h
    # lateral spread of 1.5 m (about one cell of the 128 x 128 mesh): a line
    # source makes the advective Galerkin heat system indefinite near the
    # well (local Courant number ~40 at the Gauss points next to the axis)
    wells = np.array([
        [snap(70.0, hx), snap(100.0, hy), z_hi, z_lo, +5.0e-3, T_amb + 10.0, well_sigma],
        [snap(130.0, hx), snap(100.0, hy), z_hi, z_lo, -5.0e-3, T_amb + 10.0, well_sigma],
    ])
    Nn = (p * nx + 1) * (p * ny + 1) * (p * nz + 1)
    h0 = np.zeros(Nn)
    T0 = np.full(Nn, T_amb)
    bc = _bc({0: (DIRICHLET, 0.0), 1: (DIRICHLET, 0.0), 2: (DIRICHLET, 0.0), 3: (DIRICHLET, 0.0)},
             {0: (DIRICHLET, T_amb), 1: (DIRICHLET, T_amb), 2: (DIRICHLET, T_amb),
              3: (DIRICHLET, T_amb), 5: (DIRICHLET, T_amb)})
    return Scenario("ates_layered_q2", nx, ny, nz, order, (0.0, 0.0, 0.0), (Lx, Ly, Lz),
                    K, SAND, bc, np.zeros((0, 8)), wells, h0, T0,
                    0.5 * DAY, n_steps)


def config3(nx: int = 256, ny: int = 256, nz: int = 64, seed: int = 3,
            n_steps: int = 365, n_piles: Tuple[int, int] = (40, 25),
            extent=(2000.0, 2000.0, 100.0), order: int = 1) -> Scenario:
    """Energy-pile field: 2 km x 2 km x 100 m, Q1 cells, Gaussian random lnK
    (mean ln 1e-5, sigma 1, correlation length 50 m), piles on a 50 m grid
    with +-10 m jitter, 30 m long from the top, q_l = 40 sin(2 pi t / 1 yr +
    phase) W/m with random phases; head gradient 5.1e-4 along x (5 Pa/m,
    Section 3.3); dt = 1 day."""
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = extent
    lnK = math.log(1e-5) + gaussian_field_fft((nz, ny, nx), (Lz / nz, Ly / ny, Lx / nx),
                                              50.0, 1.0, rng)
    K = np.exp(lnK).reshape(-1)
    gx, gy = n_piles
    cx0 = Lx / 2 - 50.0 * (gx - 1) / 2
    cy0 = Ly / 2 - 50.0 * (gy - 1) / 2
    px = cx0 + 50.0 * np.arange(gx)
    py = cy0 + 50.0 * np.arange(gy)
    PX, PY = np.meshgrid(px, py, indexing="ij")
    n = PX.size
    jit = rng.uniform(-10.0, 10.0, size=(n, 2))
    X = np.clip(PX.reshape(-1) + jit[:, 0], 0.0, Lx)
    Y = np.clip(PY.reshape(-1) + jit[:, 1], 0.0, Ly)
    phase = rng.uniform(0.0, 2 * np.pi, size=n)
    piles = np.stack([X, Y, np.full(n, Lz), np.full(n, max(Lz - 30.0, 0.0)),
                      np.zeros(n), np.full(n, 40.0), np.full(n, 365 * DAY), phase], axis=1)
    grad = 5.0 / (RHO_W * G_ACC)
    h0 = _linear_x(None, (0, 0, 0), extent, order, grad * Lx, -grad, nx, ny, nz)
    T0 = np.full(h0.size, 15.0)
    bc = _bc({0: (DIRICHLET, grad * Lx), 1: (DIRICHLET, 0.0)},
             {0: (DIRICHLET, 15.0), 1: (DIRICHLET, 15.0), 2: (DIRICHLET, 15.0),
              3: (DIRICHLET, 15.0), 5: (DIRICHLET, 15.0)})
    return Scenario("pile_field_q1", nx, ny, nz, order, (0.0, 0.0, 0.0), extent,
                    K, SAND, bc, piles, np.zeros((0, 7)), h0, T0,
                    1.0 * DAY, n_steps)


# Layered profile of the city-scale workload, bottom to top: (name, thickness
# as a fraction of the depth, geometric-mean K in m/s).  The conductivities
# are those of Table 3 (Section 3.3); the order and proportions follow its
# description of the profile (bedrock from about 75 % of the depth down, the
# two bay muds above it, a thin shoal and the fill at the top), stretched to
# the workload's depth.
CITY_LAYERS = (("franciscan_bedrock", 0.25, 1.0e-6),
               ("old_bay_mud", 0.35, 1.7e-9),
               ("young_bay_mud", 0.25, 1.7e-9),
               ("shoal", 0.05, 3.5e-5),
               ("fill", 0.10, 1.1e-5))


def config5(nx: int = 512, ny: int = 512, nz: int = 96, seed: int = 5,
            n_steps: int = 365, pile_grid: Tuple[int, int] = (160, 125),
            n_boxes: int = 50, extent=(10000.0, 10000.0, 200.0)) -> Scenario:
    """City-scale workload: 10 km x 10 km x 200 m, Q1 cells, layered lnK
    (the five Table 3 soils, CITY_LAYERS) plus a Gaussian random field
    (sigma 1, correlation length 50 m), 20,000 piles (a 160 x 125 grid at
    50 m spacing with +-10 m jitter, 30 m long from the top, q_l = 40 sin(2 pi
    t / 1 yr + phase) W/m with random phases), and 50 basement / subway heat
    sources: horizontal rectangles 100-600 m (and at least 1.5 cells) on a
    side at 4-20 m below the surface, 5-20 W/m^2 into the ground with a seasonal part of up to a
    quarter of that.  Head gradient 5.1e-4 along x (5 Pa/m, Section 3.3);
    T = 15 on the lateral faces and the top; dt = 1 day."""
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = extent
    # layer of each cell layer (by the depth of its centre)
    zc = (np.arange(nz) + 0.5) / nz
    bounds = np.cumsum([f for _, f, _ in CITY_LAYERS])
    lay = np.minimum(np.searchsorted(bounds, zc, side="right"), len(CITY_LAYERS) - 1)
    ln_mean = np.log(np.array([k for _, _, k in CITY_LAYERS]))[lay]
    lnK = ln_mean[:, None, None] + gaussian_field_fft((nz, ny, nx), (Lz / nz, Ly / ny, Lx / nx),
                                                      50.0, 1.0, rng)
    K = np.exp(lnK).reshape(-1)
    gx, gy = pile_grid
    px = Lx / 2 - 50.0 * (gx - 1) / 2 + 50.0 * np.arange(gx)
    py = Ly / 2 - 50.0 * (gy - 1) / 2 + 50.0 * np.arange(gy)
    PX, PY = np.meshgrid(px, py, indexing="ij")
    n = PX.size
    jit = rng.uniform(-10.0, 10.0, size=(n, 2))
    X = np.clip(PX.reshape(-1) + jit[:, 0], 0.0, Lx)
    Y = np.clip(PY.reshape(-1) + jit[:, 1], 0.0, Ly)
    phase = rng.uniform(0.0, 2 * np.pi, size=n)
    piles = np.stack([X, Y, np.full(n, Lz), np.full(n, Lz - 30.0),
                      np.zeros(n), np.full(n, 40.0), np.full(n, 365 * DAY), phase], axis=1)
    # at least 1.5 cells on a side, so that no box snaps to an empty rectangle
    # on the coarser meshes of the same generator
    wx = np.maximum(rng.uniform(100.0, 600.0, n_boxes), 1.5 * Lx / nx)
    wy = np.maximum(rng.uniform(100.0, 600.0, n_boxes), 1.5 * Ly / ny)
    bx0 = rng.uniform(0.0, Lx - wx)
    by0 = rng.uniform(0.0, Ly - wy)
    bz = Lz - rng.uniform(4.0, 20.0, n_boxes)
    flux = rng.uniform(5.0, 20.0, n_boxes)
    boxes = np.stack([bx0, bx0 + wx, by0, by0 + wy, bz, flux,
                      flux * rng.uniform(0.0, 0.25, n_boxes), np.full(n_boxes, 365 * DAY),
                      rng.uniform(0.0, 2 * np.pi, n_boxes)], axis=1)
    grad = 5.0 / (RHO_W * G_ACC)
    h0 = _linear_x(None, (0, 0, 0), extent, 1, grad * Lx, -grad, nx, ny, nz)
    T0 = np.full(h0.size, 15.0)
    bc = _bc({0: (DIRICHLET, grad * Lx), 1: (DIRICHLET, 0.0)},
             {0: (DIRICHLET, 15.0), 1: (DIRICHLET, 15.0), 2: (DIRICHLET, 15.0),
              3: (DIRICHLET, 15.0), 5: (DIRICHLET, 15.0)})
    sc = Scenario("city_q1", nx, ny, nz, 1, (0.0, 0.0, 0.0), extent,
                  K, SAND, bc, piles, np.zeros((0, 7)), h0, T0, 1.0 * DAY, n_steps)
    sc.boxes = boxes
    return sc


def random_small(seed: int, nx: int, ny: int, nz: int, order: int,
                 n_piles: int = 3, n_wells: int = 2, sigma_lnK: float = 1.0,
                 faces_head=(0, 1), faces_temp=(0, 1, 2, 3, 5),
                 extent=(40.0, 30.0, 20.0), dt: float = 0.5 * DAY,
                 per_cell_thermal: bool = False, n_boxes: int = 0) -> Scenario:
    """Small random problem for parity tests: iid lognormal K, random piles
    and wells at arbitrary (off-node) positions, random initial fields, and
    optionally box heat sources whose edges lie within 0.3 cells of a cell
    face (so that snapping is exercised but never ambiguous)."""
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = extent
    nc = nx * ny * nz
    K = np.exp(math.log(3e-5) + sigma_lnK * rng.standard_normal(nc))
    p = order
    Nn = (p * nx + 1) * (p * ny + 1) * (p * nz + 1)
    h0 = rng.uniform(-0.5, 0.5, Nn)
    T0 = 15.0 + rng.uniform(-1.0, 1.0, Nn)
    piles = np.stack([rng.uniform(0, Lx, n_piles), rng.uniform(0, Ly, n_piles),
                      rng.uniform(0.6 * Lz, Lz, n_piles), rng.uniform(0.0, 0.4 * Lz, n_piles),
                      rng.uniform(-20, 20, n_piles), rng.uniform(0, 40, n_piles),
                      np.full(n_piles, 30 * DAY), rng.uniform(0, 2 * np.pi, n_piles)], axis=1) \
        if n_piles else np.zeros((0, 8))
    # even wells are line sources, odd wells spread laterally
    wells = np.stack([rng.uniform(0, Lx, n_wells), rng.uniform(0, Ly, n_wells),
                      rng.uniform(0.5 * Lz, Lz, n_wells), rng.uniform(0.0, 0.5 * Lz, n_wells),
                      np.where(np.arange(n_wells) % 2 == 0, 2e-3, -2e-3),
                      np.full(n_wells, 25.0),
                      np.where(np.arange(n_wells) % 2 == 0, 0.0, rng.uniform(0.5, 3.0, n_wells))],
                     axis=1) if n_wells else np.zeros((0, 7))
    bc = {HEAD: {f: (DIRICHLET, float(rng.uniform(-0.3, 0.3))) for f in faces_head},
          TEMP: {f: (DIRICHLET, float(rng.uniform(14, 16))) for f in faces_temp}}
    sc = Scenario(f"random_q{order}_{nx}x{ny}x{nz}_s{seed}", nx, ny, nz, order,
                  (0.0, 0.0, 0.0), extent, K, SAND, bc, piles, wells,
                  h0, T0, dt, 3)
    if per_cell_thermal:
        # lognormal about the sand's bulk values (1.93 W/(m K), 2.654e6 J/(m^3 K))
        sc.lam_cells = 1.93 * np.exp(0.3 * rng.standard_normal(nc))
        sc.cT_cells = 2.654e6 * np.exp(0.2 * rng.standard_normal(nc))
    if n_boxes:
        sc.boxes = random_boxes(rng, n_boxes, (nx, ny, nz), extent)
    return sc


def graded_widths(n: int, length: float, stretch: float) -> np.ndarray:
    """n cell widths of a graded spacing along one axis: faces at
    length * expm1(stretch * s) / expm1(stretch) for s = 0, 1/n, ..., 1, so
    that refining n refines the same smooth map (stretch 0: uniform)."""
    s = np.arange(n + 1, dtype=np.float64) / n
    x = length * s if stretch == 0.0 else length * np.expm1(stretch * s) / math.expm1(stretch)
    return np.diff(x)


def random_boxes(rng, n: int, cells: Tuple[int, int, int], extent, period: float = 30 * DAY) -> np.ndarray:
    """n box heat sources [n, 9]: a random non-empty run of cell faces per
    axis, each edge (and the plane z) jittered by up to 0.3 cells, fluxes of
    -20..20 W/m^2 with seasonal amplitude 0..15 W/m^2."""
    nx, ny, nz = cells
    Hx, Hy, Hz = extent[0] / nx, extent[1] / ny, extent[2] / nz
    rows = []
    for _ in range(n):
        i0 = int(rng.integers(0, nx)); i1 = int(rng.integers(i0 + 1, nx + 1))
        j0 = int(rng.integers(0, ny)); j1 = int(rng.integers(j0 + 1, ny + 1))
        k = int(rng.integers(0, nz + 1))
        jit = rng.uniform(-0.3, 0.3, 5)
        z = min(max((k + jit[4]) * Hz, 0.0), extent[2])
        rows.append([(i0 + jit[0]) * Hx, (i1 + jit[1]) * Hx, (j0 + jit[2]) * Hy, (j1 + jit[3]) * Hy, z,
                     rng.uniform(-20, 20), rng.uniform(0, 15), period, rng.uniform(0, 2 * np.pi)])
    return np.asarray(rows, dtype=np.float64).reshape(-1, 9)


def config4(n_problems: int = 64, seed0: int = 1000, n_steps: int = 30,
            size_range=(16, 48), extent=(400.0, 400.0, 100.0)) -> list:
    """Batched scenarios: independent Q1 problems with nz ~ U{16..48} and
    nx = ny = 2 nz cells (32x32x16 .. 96x96x48) over the same box, each with
    its own Gaussian-random lnK (sigma_lnK ~ U(0.5, 1.5), correlation length
    50 m) and 10-200 piles with random seasonal loads; dt = 1 day."""
    out = []
    for i in range(n_problems):
        rng = np.random.default_rng(seed0 + i)
        nz = int(rng.integers(size_range[0], size_range[1] + 1))
        nx = ny = 2 * nz
        Lx, Ly, Lz = extent
        sig = float(rng.uniform(0.5, 1.5))
        lnK = math.log(1e-5) + gaussian_field_fft((nz, ny, nx), (Lz / nz, Ly / ny, Lx / nx), 50.0, sig, rng)
        K = np.exp(lnK).reshape(-1)
        npl = int(rng.integers(10, 201))
        piles = np.stack([rng.uniform(0.1 * Lx, 0.9 * Lx, npl), rng.uniform(0.1 * Ly, 0.9 * Ly, npl),
                          np.full(npl, Lz), np.full(npl, Lz - 30.0), rng.uniform(-5, 5, npl),
                          rng.uniform(10, 40, npl), np.full(npl, 365 * DAY),
                          rng.uniform(0, 2 * np.pi, npl)], axis=1)
        grad = 5.0 / (RHO_W * G_ACC)
        h0 = _linear_x(None, (0, 0, 0), extent, 1, grad * Lx, -grad, nx, ny, nz)
        T0 = np.full(h0.size, 15.0)
        bc = _bc({0: (DIRICHLET, grad * Lx), 1: (DIRICHLET, 0.0)},
                 {0: (DIRICHLET, 15.0), 1: (DIRICHLET, 15.0), 2: (DIRICHLET, 15.0),
                  3: (DIRICHLET, 15.0), 5: (DIRICHLET, 15.0)})
        out.append(Scenario(f"batch_q1_{nx}x{ny}x{nz}_s{seed0 + i}", nx, ny, nz, 1, (0.0, 0.0, 0.0), extent,
                            K, SAND, bc, piles, np.zeros((0, 7)), h0, T0, 1.0 * DAY, n_steps))
    return out


def geometric_widths(first: float, n: int, length: float) -> np.ndarray:
    """n cell widths growing by a constant ratio from `first`, summing to
    `length` (the ratio is found by bisection; n * first = length gives
    uniform cells, and a larger n * first shrinks the cells instead)."""
    if n == 1:
        return np.array([float(length)])
    def total(r):
        return first * n if abs(r - 1.0) < 1e-14 else first * (r ** n - 1.0) / (r - 1.0)
    lo, hi = (1.0, 2.0) if first * n <= length else (1e-6, 1.0)
    while total(hi) < length:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < length:
            lo = mid
        else:
            hi = mid
    w = first * (0.5 * (lo + hi)) ** np.arange(n)
    return w * (length / w.sum())


# Table 1 (Section 2): the ATES benchmark's material values, shared by all
# three formations, and its boundary data.
ATES_TABLE1 = dict(cT=1.2e6, lam=1.2, B_poro=1.0e5, T_top=278.15, T_b=288.15, P0=1.0e5,
                   Q_b=1.0e-3, c_w=1.0e6, dTdz=0.05)


def ates_table1(n_bore: int = 42, n_out: int = 224, nz_aquifer: int = 50, nz_confining: int = 20,
                radius: float = 20.0, depth: float = 300.0, r_w: float = 0.1,
                layers=(100.0, 100.0, 100.0), K_aquifer: float = 1.0e-6,
                K_confining: float = 1.0e-10, n_steps: int = 180, dt: float = DAY,
                first_dz: float = 1.0) -> Scenario:
    """Hot-water injection benchmark of Section 2 (Fig. 2, Table 1) on a box
    mesh: one quarter of the 20 m x 300 m cylinder around the wellbore, cut
    by its two symmetry planes x = 0 and y = 0 (no-flow, insulated), the
    wellbore axis on their common edge.

    Formations, bottom to top: basement rock, aquifer, caprock (`layers`, m;
    the thicknesses are not printed, equal thirds are taken), K = 1e-6 m/s in
    the aquifer and 1e-10 m/s in the confining layers.  Table 1 gives c_T,
    lambda, B_poro (S_s = rho_w g / B_poro), c_w, T_top, the geothermal
    gradient dT, the initial pressure P0 and the wellbore data Q_b and T_b.

    * Wellbore (radius r_w, not printed; 0.1 m taken), over the aquifer:
      injection flux Q_b through its surface, i.e. Q = Q_b 2 pi r_w b for the
      whole well and a quarter of it here, as a line source on the axis
      (`wells`), and temperature T_b on every node within r_w of the axis
      (`pile_temps`, constant).
    * Head: hydrostatic initial state from P0 at the top, h = P0/(rho_w g) +
      z_top everywhere, held on the outer faces x = R and y = R.
    * Temperature: the geotherm T_top + dT (z_top - z) initially, T_top on
      the top face, the geothermal flux lambda dT into the bottom face,
      natural (outflow) conditions on the outer faces.
    * Cells: n_bore equal cells across [0, r_w] and n_out cells growing
      geometrically from the same width to R; in z, nz_aquifer equal cells in
      the aquifer and nz_confining cells in each confining layer growing from
      `first_dz` at the aquifer.  The defaults keep the cell Peclet number
      c_w |q| H / lambda at or below 2 everywhere outside the wellbore (|q|
      <= Q_b r_w / r), so that the plain Galerkin heat operator of Eq. 4 needs
      no stabilisation.

    180 daily steps give the six months of Section 2."""
    t = ATES_TABLE1
    h_b = r_w / n_bore
    wx = np.concatenate([np.full(n_bore, h_b), geometric_widths(h_b, n_out, radius - r_w)])
    d_bas, d_aq, d_cap = layers
    assert abs(d_bas + d_aq + d_cap - depth) < 1e-9 * depth
    wz = np.concatenate([geometric_widths(first_dz, nz_confining, d_bas)[::-1],
                         np.full(nz_aquifer, d_aq / nz_aquifer),
                         geometric_widths(first_dz, nz_confining, d_cap)])
    nx = ny = wx.size
    nz = wz.size
    z_lo, z_hi = d_bas, d_bas + d_aq
    zc = np.concatenate([[0.0], np.cumsum(wz)])
    zc = 0.5 * (zc[:-1] + zc[1:])
    in_aq = (zc > z_lo) & (zc < z_hi)
    K = np.where(in_aq, K_aquifer, K_confining)[:, None, None] * np.ones((1, ny, nx))
    K = K.reshape(-1)
    mat = Material(phi=0.0, lam_s=t["lam"], lam_w=t["lam"], c_s=t["cT"], c_w=t["c_w"],
                   B_poro=t["B_poro"])
    Q = t["Q_b"] * 2.0 * math.pi * r_w * d_aq
    wells = np.array([[0.0, 0.0, z_hi, z_lo, Q / 4.0, t["T_b"], 0.0]])
    bore = np.array([[0.0, 0.0, z_hi, z_lo, r_w, t["T_b"], 0.0, 365 * DAY, 0.0]])
    h_top = t["P0"] / (RHO_W * G_ACC) + depth
    sc = Scenario("ates_table1_q1", nx, ny, nz, 1, (0.0, 0.0, 0.0), (radius, radius, depth),
                  K, mat, {}, np.zeros((0, 8)), wells, np.zeros(1), np.zeros(1), dt, n_steps)
    sc.spacing = (wx, wx.copy(), wz)
    _, _, zn = sc.node_coords()
    Nx, Ny, Nz = sc.node_dims
    sc.h0 = np.full(sc.n_nodes, h_top)
    sc.T0 = np.repeat(t["T_top"] + t["dTdz"] * (depth - zn), Nx * Ny)
    sc.bc = _bc({1: (DIRICHLET, h_top), 3: (DIRICHLET, h_top)},
                {5: (DIRICHLET, t["T_top"]), 4: (FLUX, t["lam"] * t["dTdz"])})
    sc.pile_temps = bore
    sc.lam, sc.cT = t["lam"], t["cT"]
    return sc
