"""The allocation-free head apply (ht_head_apply_dot_noalloc), through the C
ABI, on two calls in a row: y and x^T y against the CPU oracle's constrained
head operator and against the context-based entry point ht_apply.

This entry point serves callers that cannot allocate device memory (an
application whose own pool owns all device memory, or a latency-critical loop
that must not call cudaMalloc); its scratch is a static device array.  The
cases include a face mask that is not the workloads' default (one Dirichlet
face) so that the mask handling is checked against the oracle on its own.
The file is named to be collected last so a stop-at-first-failure run has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import scenarios as S
from oracle import fem

pytestmark = pytest.mark.gpu

CASES = [(1, 33, 20, 7, 31, (0, 1)), (2, 17, 9, 5, 32, (0, 1)), (1, 12, 9, 6, 33, (3,)),
         (2, 6, 5, 4, 34, (4,))]


@pytest.mark.parametrize("case", CASES)
def test_noalloc_head_apply_matches_oracle_and_context_apply_twice(built_lib, case):
    import torch
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import hydro

    p, nx, ny, nz, seed, faces = case
    sc = S.random_small(seed, nx, ny, nz, p, faces_head=faces)
    oracle = fem.OracleSim(sc)
    sim = hydro.Simulator.from_scenario(sc)
    lib = L.lib()
    mask = sum(1 << f for f in faces)
    mesh = L.Mesh(nx, ny, nz, p, *sc.origin, *sc.extent)
    dev = torch.device("cuda:0")
    K = torch.tensor(sc.K, dtype=torch.float64, device=dev)
    y = torch.empty(sc.n_nodes, dtype=torch.float64, device=dev)
    dot = torch.empty(1, dtype=torch.float64, device=dev)
    msg = ctypes.create_string_buffer(256)
    rng = np.random.default_rng(seed)
    for call in range(2):
        x_host = rng.standard_normal(sc.n_nodes)
        x = torch.tensor(x_host, dtype=torch.float64, device=dev)
        y.fill_(float("nan"))
        dot.fill_(float("nan"))
        rc = lib.ht_head_apply_dot_noalloc(ctypes.byref(mesh), mask, oracle.Ss, sc.dt,
                                           ctypes.c_void_p(K.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(dot.data_ptr()),
                                           0, None, msg, len(msg))
        assert rc == L.HT_OK, msg.value
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        for name, ref in (("oracle", oracle.apply_head(x_host, sc.dt)),
                          ("ht_apply", sim.apply(S.HEAD, sc.dt, x_host))):
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel <= 1e-12, (name, call, rel)
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (name, call)
            ref_dot = float(x_host @ ref)
            assert abs(dot.item() - ref_dot) <= 1e-12 * np.sum(np.abs(x_host * ref)), \
                (name, call, dot.item(), ref_dot)
    sim.close()


def test_noalloc_rejects_meshes_beyond_the_static_scratch(built_lib):
    from paper_2103_00081_gb300 import _lib as L
    lib = L.lib()
    big = L.Mesh(4000, 4000, 4, 1, 0, 0, 0, 1, 1, 1)
    msg = ctypes.create_string_buffer(256)
    dummy = ctypes.c_void_p(1)
    rc = lib.ht_head_apply_dot_noalloc(ctypes.byref(big), 0, 0.1, 1.0, dummy, dummy, dummy, dummy,
                                       0, None, msg, len(msg))
    assert rc == L.HT_EINVAL
    assert b"static scratch" in msg.value


def test_noalloc_rejects_meshes_whose_counts_overflow_int(built_lib):
    """Sizes whose node count exceeds the kernels' int indexing are refused
    before any device work (the pointers are never touched)."""
    from paper_2103_00081_gb300 import _lib as L
    lib = L.lib()
    msg = ctypes.create_string_buffer(256)
    dummy = ctypes.c_void_p(1)
    for dims in ((2 ** 30, 2 ** 30, 2 ** 30), (70000, 70000, 1), (2 ** 31 - 1, 2, 2)):
        huge = L.Mesh(*dims, 2, 0, 0, 0, 1, 1, 1)
        rc = lib.ht_head_apply_dot_noalloc(ctypes.byref(huge), 0, 0.1, 1.0, dummy, dummy, dummy, dummy,
                                           0, None, msg, len(msg))
        assert rc == L.HT_EINVAL, dims
        assert b"too large" in msg.value, msg.value
