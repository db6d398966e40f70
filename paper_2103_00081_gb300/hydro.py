"""Thin Python wrapper of the C ABI: one ``Simulator`` per ``ht_ctx``.

Only argument marshalling happens here: every arithmetic step of the solver
runs in the CUDA library.  Host arrays are numpy float64; device arrays may be
torch CUDA float64 tensors (passed by data pointer with on_device=1).
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int, c_size_t, c_void_p

import numpy as np

from . import _lib as L


class HTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{L.ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(a, on_device):
    if a is None:
        return None, 0
    if on_device:
        return c_void_p(a.data_ptr()), 1
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data_as(c_void_p), 0


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


class Simulator:
    def __init__(self, nx, ny, nz, order, origin=(0.0, 0.0, 0.0), extent=(1.0, 1.0, 1.0),
                 device=0, stream=None):
        self._lib = L.lib()
        m = L.Mesh(nx, ny, nz, order, *[float(v) for v in origin], *[float(v) for v in extent])
        h = c_void_p()
        rc = self._lib.ht_create(byref(h), byref(m), int(device), c_void_p(stream) if stream else None)
        if rc != L.HT_OK:
            raise HTError(rc, self._lib.ht_last_error(None).decode())
        self._h = h
        nn, nc = c_size_t(), c_size_t()
        self._lib.ht_sizes(self._h, byref(nn), byref(nc))
        self.n_nodes, self.n_cells = nn.value, nc.value
        self.dims = (order * nx + 1, order * ny + 1, order * nz + 1)

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.ht_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc):
        if rc != L.HT_OK:
            raise HTError(rc, self._lib.ht_last_error(self._h).decode())
        return rc

    # -- set-up ---------------------------------------------------------------
    def set_cells(self, K, lam=None, cT=None, lam_u=0.0, cT_u=0.0, cw=4.18e6, Ss=0.0981):
        K = np.ascontiguousarray(K, dtype=np.float64)
        lp = np.ascontiguousarray(lam, dtype=np.float64) if lam is not None else None
        cp = np.ascontiguousarray(cT, dtype=np.float64) if cT is not None else None
        for a in (K, lp, cp):
            if a is not None and a.size != self.n_cells:
                raise ValueError("per-cell arrays need one value per cell")
        return self._check(self._lib.ht_set_cells(
            self._h, K.ctypes.data_as(c_void_p),
            lp.ctypes.data_as(c_void_p) if lp is not None else None,
            cp.ctypes.data_as(c_void_p) if cp is not None else None,
            float(lam_u), float(cT_u), float(cw), float(Ss)))

    def set_bc(self, field, face, typ, value=0.0):
        """Boundary condition on a face: a scalar value, or one value per face
        node in ascending node order (the lower tangential axis fastest)."""
        if np.ndim(value) == 0:
            return self._check(self._lib.ht_set_bc(self._h, int(field), int(face), int(typ), float(value)))
        v = np.ascontiguousarray(value, dtype=np.float64).reshape(-1)
        return self._check(self._lib.ht_set_bc_values(self._h, int(field), int(face), int(typ),
                                                      v.ctypes.data, v.size))

    def set_spacing(self, axis, widths):
        """Cell widths along one axis of a graded tensor-product mesh."""
        w = np.ascontiguousarray(widths, dtype=np.float64).reshape(-1)
        return self._check(self._lib.ht_set_spacing(self._h, int(axis), w.ctypes.data, int(w.size)))

    def set_seasonal_face(self, field, face, mean, amp, period, phase=0.0):
        """Dirichlet face whose value is mean + amp sin(2 pi t / period + phase)
        at each step's end time."""
        return self._check(self._lib.ht_set_seasonal_face(self._h, int(field), int(face), float(mean), float(amp),
                                                          float(period), float(phase)))

    def set_pile_temperatures(self, rows):
        """Pile surfaces held at a square-wave temperature; rows [n][9] =
        (x, y, z_top, z_bot, radius, T_mean, T_amp, period, phase)."""
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.float64).reshape(-1, 9))
        return self._check(self._lib.ht_set_pile_temperatures(self._h, r.shape[0], r.ctypes.data if r.size else None))

    def face_nodes(self, face):
        n = ctypes.c_size_t()
        self._check(self._lib.ht_face_nodes(self._h, int(face), ctypes.byref(n)))
        return n.value

    def set_state(self, h=None, T=None, t=0.0):
        dev = _is_torch_cuda(h) or _is_torch_cuda(T)
        hp, _ = _ptr(h, dev)
        tp, _ = _ptr(T, dev)
        keep = (np.ascontiguousarray(h, dtype=np.float64) if (h is not None and not dev) else None,
                np.ascontiguousarray(T, dtype=np.float64) if (T is not None and not dev) else None)
        if not dev:
            hp = keep[0].ctypes.data_as(c_void_p) if keep[0] is not None else None
            tp = keep[1].ctypes.data_as(c_void_p) if keep[1] is not None else None
        return self._check(self._lib.ht_set_state(self._h, hp, tp, float(t), int(dev)))

    def add_box_sources(self, rows):
        """Rows of (x0, x1, y0, y1, z, mean, amp, period, phase): heat flux in
        W/m^2 over a horizontal rectangle snapped to cell faces."""
        rows = np.asarray(rows, dtype=np.float64).reshape(-1, 9)
        if rows.shape[0] == 0:
            return L.HT_OK
        arr = (L.BoxSrc * rows.shape[0])(*[L.BoxSrc(*map(float, r)) for r in rows])
        return self._check(self._lib.ht_add_box_sources(self._h, rows.shape[0], arr))

    def add_line_sources(self, rows):
        rows = np.asarray(rows, dtype=np.float64).reshape(-1, 8)
        if rows.shape[0] == 0:
            return L.HT_OK
        arr = (L.LineSrc * rows.shape[0])(*[L.LineSrc(*map(float, r)) for r in rows])
        return self._check(self._lib.ht_add_line_sources(self._h, rows.shape[0], arr))

    def add_wells(self, rows):
        rows = np.asarray(rows, dtype=np.float64)
        if rows.size == 0:
            return L.HT_OK
        rows = rows.reshape(-1, rows.shape[-1])
        if rows.shape[1] == 6:
            rows = np.concatenate([rows, np.zeros((rows.shape[0], 1))], axis=1)
        arr = (L.Well * rows.shape[0])(*[L.Well(*map(float, r)) for r in rows])
        return self._check(self._lib.ht_add_wells(self._h, rows.shape[0], arr))

    def set_extra_rhs(self, field, F):
        if F is None:
            return self._check(self._lib.ht_set_extra_rhs(self._h, int(field), None, 0))
        dev = _is_torch_cuda(F)
        if dev:
            return self._check(self._lib.ht_set_extra_rhs(self._h, int(field), c_void_p(F.data_ptr()), 1))
        F = np.ascontiguousarray(F, dtype=np.float64)
        return self._check(self._lib.ht_set_extra_rhs(self._h, int(field), F.ctypes.data_as(c_void_p), 0))

    def set_solver(self, **kw):
        o = L.SolverOpts()
        self._lib.ht_default_solver(byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        return self._check(self._lib.ht_set_solver(self._h, byref(o)))

    # -- stepping -------------------------------------------------------------
    def step(self, dt, check=True):
        st = L.StepStats()
        rc = self._lib.ht_step(self._h, float(dt), byref(st))
        if check:
            self._check(rc)
        d = st.as_dict()
        d["rc"] = rc
        return d

    @property
    def time(self):
        t = c_double()
        self._check(self._lib.ht_get_time(self._h, byref(t)))
        return t.value

    # -- outputs / parity hooks -------------------------------------------------
    def get_field(self, field, out=None):
        n = self.n_nodes if field in (L.HT_HEAD, L.HT_TEMP) else self.n_cells
        if out is not None and _is_torch_cuda(out):
            self._check(self._lib.ht_get_field(self._h, int(field), c_void_p(out.data_ptr()), n, 1))
            return out
        a = np.empty(n, dtype=np.float64)
        self._check(self._lib.ht_get_field(self._h, int(field), a.ctypes.data_as(c_void_p), n, 0))
        return a

    def _vec_call(self, fn, field, dt, x=None):
        y = np.empty(self.n_nodes, dtype=np.float64)
        if x is None:
            self._check(fn(self._h, int(field), float(dt), y.ctypes.data_as(c_void_p), 0))
        else:
            x = np.ascontiguousarray(x, dtype=np.float64)
            self._check(fn(self._h, int(field), float(dt), x.ctypes.data_as(c_void_p),
                           y.ctypes.data_as(c_void_p), 0))
        return y

    def apply(self, field, dt, x):
        return self._vec_call(self._lib.ht_apply, field, dt, x)

    def residual(self, field, dt, x, b, emulated=False):
        """||b - A x|| / ||b|| with A x in FP64 or in float-float (emulated)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        rel = c_double()
        self._check(self._lib.ht_residual(self._h, int(field), float(dt), x.ctypes.data_as(c_void_p),
                                          b.ctypes.data_as(c_void_p), int(bool(emulated)), 0, byref(rel)))
        return rel.value

    def diag(self, field, dt):
        return self._vec_call(self._lib.ht_diag, field, dt)

    def rhs(self, field, dt):
        return self._vec_call(self._lib.ht_rhs, field, dt)

    # -- profiling -------------------------------------------------------------
    def profile(self, on=True):
        return self._check(self._lib.ht_profile(self._h, int(on)))

    def profile_read(self):
        st = L.ProfileStats()
        self._check(self._lib.ht_profile_read(self._h, byref(st)))
        return st.as_dict()

    # -- scenario helper -----------------------------------------------------------
    def bulk_properties(self, m):
        """(lambda, c_T, S_s) from raw material properties by the library's
        ht_mixture and ht_specific_storage."""
        lam, cT = c_double(), c_double()
        self._check(self._lib.ht_mixture(m.phi, m.lam_s, m.lam_w, m.c_s, m.c_w, byref(lam), byref(cT)))
        return lam.value, cT.value, self._lib.ht_specific_storage(m.B_poro, m.rho_w, m.g)

    @classmethod
    def from_scenario(cls, sc, device=0, stream=None, **solver):
        s = cls(sc.nx, sc.ny, sc.nz, sc.order, sc.origin, sc.extent, device=device, stream=stream)
        if getattr(sc, "spacing", None) is not None:
            for axis, w in enumerate(sc.spacing):
                s.set_spacing(axis, w)
        lam, cT, Ss = s.bulk_properties(sc.material)
        s.set_cells(sc.K, sc.lam_cells, sc.cT_cells, sc.lam if sc.lam is not None else lam,
                    sc.cT if sc.cT is not None else cT, sc.material.c_w, sc.Ss if sc.Ss is not None else Ss)
        for field, faces in sc.bc.items():
            for face, (typ, val) in faces.items():
                s.set_bc(field, face, typ, val)
        for field, faces in (getattr(sc, "bc_seasonal", None) or {}).items():
            for face, (mean, amp, period, phase) in faces.items():
                s.set_seasonal_face(field, face, mean, amp, period, phase)
        s.set_pile_temperatures(getattr(sc, "pile_temps", np.zeros((0, 9))))
        s.add_line_sources(sc.piles)
        s.add_wells(sc.wells)
        s.add_box_sources(getattr(sc, "boxes", np.zeros((0, 9))))
        s.set_state(sc.h0, sc.T0, 0.0)
        if solver:
            s.set_solver(**solver)
        return s


class Batch:
    """Batched steps of several Simulators (ht_batch_*).  mode
    HT_BATCH_CONCURRENT (the library default) steps the problems concurrently
    on their own streams; HT_BATCH_SHARED_LAUNCHES runs the inner FP32 head CG
    of all problems in shared launches captured in a CUDA graph."""

    def __init__(self, sims, mode=None):
        self._lib = L.lib()
        self.sims = list(sims)
        arr = (c_void_p * len(self.sims))(*[s._h.value for s in self.sims])
        h = c_void_p()
        rc = self._lib.ht_batch_create(byref(h), len(self.sims), arr)
        if rc != L.HT_OK:
            raise HTError(rc, "ht_batch_create failed")
        self._h = h
        if mode is not None:
            rc = self._lib.ht_batch_set_mode(self._h, int(mode))
            if rc != L.HT_OK:
                raise HTError(rc, self._lib.ht_batch_last_error(self._h).decode())

    def set_persistent(self, planes: int = 0, wait_ms: float = 2000.0, drop_cta: int = -1):
        """Options of the persistent mode (see ht_batch_set_persistent)."""
        rc = self._lib.ht_batch_set_persistent(self._h, int(planes), float(wait_ms), int(drop_cta))
        if rc != L.HT_OK:
            raise HTError(rc, self._lib.ht_batch_last_error(self._h).decode())

    def persistent_info(self) -> dict:
        v = [c_int() for _ in range(4)]
        self._lib.ht_batch_persistent_info(self._h, *[byref(x) for x in v])
        return dict(zip(("planes", "items", "grid", "err_cta"), (x.value for x in v)))

    def step(self, dt, check=True):
        n = len(self.sims)
        stats = (L.StepStats * n)()
        rc = self._lib.ht_batch_step(self._h, float(dt), ctypes.cast(stats, c_void_p))
        if check and rc != L.HT_OK:
            raise HTError(rc, self._lib.ht_batch_last_error(self._h).decode())
        out = [s.as_dict() for s in stats]
        for d in out:
            d["rc"] = rc
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ht_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
