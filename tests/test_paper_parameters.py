"""Paper-printed parameters (tests/golden/, cited there) exercised through the
oracle: storage from Table 1, and the layer-diffusivity ordering of Table 3
that Section 3.5 uses to explain why clay layers barely follow the surface
temperature."""
import os

import numpy as np

from oracle import fem
import scenarios as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[parts[0]] = [float(v) for v in parts[1:3]] if len(parts) > 3 else float(parts[1])
            if len(parts) > 3:
                rows[parts[0]] = [float(v) for v in parts[1:4]]
    return rows


def test_table1_specific_storage():
    t1 = _table("table1_ates_parameters.txt")
    # S_s = rho_w g / B_poro with B_poro from Table 1
    assert abs(fem.specific_storage(t1["B_poro"]) - 0.0981) < 1e-15


def test_table3_low_diffusivity_layer_responds_least_to_surface_forcing():
    """A surface temperature step penetrates a Table 3 clay column less than a
    fill/shoal column over the same time (Section 3.5 observation)."""
    t3 = _table("table3_treasure_island.txt")
    out = {}
    for layer in ("fill", "young_bay_mud"):
        K, cT, lam = t3[layer]
        sc = S.config1(nx=1, ny=1, nz=40, order=1)
        sc.extent = (1.0, 1.0, 20.0)
        sc.piles = np.zeros((0, 8))
        sc.K = np.full(sc.n_cells, K)
        sc.lam, sc.cT = lam, cT
        sc.bc = {S.HEAD: {}, S.TEMP: {5: (S.DIRICHLET, 25.0)}}
        sc.h0 = np.zeros(sc.n_nodes)
        sc.T0 = np.full(sc.n_nodes, 15.0)
        o = fem.OracleSim(sc)
        for _ in range(30):
            o.step(S.DAY)
        T = o.T.reshape(sc.node_dims[::-1])[:, 0, 0]
        out[layer] = T[-9]          # 4 m below the surface
    assert out["fill"] - 15.0 > 1.2 * (out["young_bay_mud"] - 15.0) > 0
