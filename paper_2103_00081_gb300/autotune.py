"""Autotuner for the kernel and solver choices of one workload.

Candidates are tuples of solver options (operator-apply variant, z chunks of
the tiled kernel, heat Krylov method, Chebyshev degree).  Each candidate is
timed on fresh simulators built by the caller's factory over a few steps of
the real workload (the first step is discarded); the fastest is cached in a
JSON file keyed by a signature of the workload (order, mesh, precision), so a
later run with the same signature reuses it without timing.

Only the library's own timers (CUDA events inside ht_step) are used; the
tuning steps are never part of a measurement.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, List, Optional, Tuple

from . import _lib as L

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_2103_00081_gb300", "autotune.json")


def signature(nx: int, ny: int, nz: int, order: int, precision: int) -> str:
    return f"q{order}-{nx}x{ny}x{nz}-prec{precision}"


def default_candidates(precision: int, order: int = 2) -> List[Dict]:
    """Operator-kernel and solver choices worth timing for a mesh of this
    order: on Q1 the single-pass head CG against the two-pass and tiled
    kernels; on Q2 the two-pass and tiled kernels, the heat Krylov method
    and a Chebyshev preconditioner."""
    out = []
    if order == 1:
        for krylov in (L.HT_KRYLOV_BICGSTAB, L.HT_KRYLOV_GMRES):
            out.append(dict(apply_variant=L.HT_APPLY_SINGLE_PASS, krylov=krylov, precond=L.HT_PREC_JACOBI))
        out.append(dict(apply_variant=L.HT_APPLY_TWO_PASS, krylov=L.HT_KRYLOV_BICGSTAB, precond=L.HT_PREC_JACOBI))
        out.append(dict(apply_variant=L.HT_APPLY_TILED, krylov=L.HT_KRYLOV_BICGSTAB, precond=L.HT_PREC_JACOBI))
        return out
    variants = [L.HT_APPLY_TWO_PASS, L.HT_APPLY_TILED]
    for v in variants:
        for krylov in (L.HT_KRYLOV_BICGSTAB, L.HT_KRYLOV_GMRES):
            out.append(dict(apply_variant=v, krylov=krylov, precond=L.HT_PREC_JACOBI))
    out.append(dict(apply_variant=L.HT_APPLY_TWO_PASS, krylov=L.HT_KRYLOV_BICGSTAB,
                    precond=L.HT_PREC_CHEBYSHEV, cheb_degree=4))
    out.append(dict(apply_variant=L.HT_APPLY_TILED, krylov=L.HT_KRYLOV_BICGSTAB, z_chunks=8))
    return out


def _load(path: str) -> Dict:
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(path: str, data: Dict) -> None:
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except Exception:
        pass


def tune(factory: Callable[[Dict], object], dt: float, sig: str, candidates: Optional[Iterable[Dict]] = None,
         steps: int = 2, cache: Optional[str] = DEFAULT_CACHE, force: bool = False) -> Tuple[Dict, List]:
    """Return (best options, table of (options, ms per step, status)).

    factory(opts) must build a fresh Simulator configured with ``opts``.
    """
    if cache and not force:
        hit = _load(cache).get(sig)
        if hit:
            return hit["opts"], hit.get("table", [])
    cands = list(candidates) if candidates is not None else default_candidates(0)
    table = []
    best, best_ms = None, float("inf")
    for opts in cands:
        sim = None
        try:
            sim = factory(opts)
            ms = []
            for k in range(steps + 1):
                st = sim.step(dt, check=False)
                if st["rc"] != L.HT_OK:
                    raise RuntimeError(f"rc {st['rc']}")
                if k > 0:
                    ms.append(st["ms_total"])
            t = sum(ms) / len(ms)
            table.append((opts, t, "ok"))
            if t < best_ms:
                best, best_ms = opts, t
        except Exception as e:  # a candidate that fails is skipped
            table.append((opts, None, f"failed: {e}"))
        finally:
            if sim is not None:
                sim.close()
    if best is None:
        raise RuntimeError("no autotuning candidate succeeded")
    if cache:
        data = _load(cache)
        data[sig] = {"opts": best, "ms": best_ms, "table": table}
        _store(cache, data)
    return best, table


def default_batch_candidates() -> List[Dict]:
    """Batched-step choices worth timing: the persistent mode with the
    automatic z chunking and with fixed node planes per work item (the tile
    shape of the persistent launch along z), and the concurrent mode."""
    out = [dict(mode=L.HT_BATCH_PERSISTENT, planes=p) for p in (0, 4, 8, 12, 16, 24, 32)]
    out.append(dict(mode=L.HT_BATCH_CONCURRENT))
    return out


class _TimedBatch:
    """Adapter that gives a batch the step() of a simulator for tune(): the
    batched step returns only after its work on the device is complete, so
    the host clock around it is the step's time."""

    def __init__(self, batch):
        self.batch = batch

    def step(self, dt, check=True):
        import time
        t0 = time.perf_counter()
        stats = self.batch.step(dt, check=False)
        ms = (time.perf_counter() - t0) * 1e3
        rc = next((st["rc"] for st in stats if st["rc"] != L.HT_OK), L.HT_OK)
        return {"rc": rc, "ms_total": ms}

    def close(self):
        self.batch.close()


def tune_batch(factory: Callable[[Dict], object], dt: float, sig: str,
               candidates: Optional[Iterable[Dict]] = None, steps: int = 2,
               cache: Optional[str] = DEFAULT_CACHE, force: bool = False) -> Tuple[Dict, List]:
    """tune() for batched steps: factory(opts) must build a fresh batch (over
    fresh simulators) configured with ``opts`` (mode, planes)."""
    cands = list(candidates) if candidates is not None else default_batch_candidates()
    return tune(lambda o: _TimedBatch(factory(o)), dt, sig, cands, steps=steps, cache=cache, force=force)
