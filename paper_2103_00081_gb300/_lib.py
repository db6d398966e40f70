"""ctypes declarations of the C ABI in include/ht.h (argument marshalling only).

The shared library is built in-tree by ``paper_2103_00081_gb300.build``.  If it
is missing, importing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libht.so")

HT_OK, HT_EINVAL, HT_ENOMEM, HT_ECUDA, HT_ENOCONV, HT_EBREAKDOWN, HT_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
HT_HEAD, HT_TEMP, HT_QX, HT_QY, HT_QZ = 0, 1, 2, 3, 4
HT_BC_NONE, HT_BC_DIRICHLET, HT_BC_FLUX = 0, 1, 2
HT_FP64, HT_MIXED = 0, 1
HT_KRYLOV_BICGSTAB, HT_KRYLOV_GMRES = 0, 1
HT_PREC_JACOBI, HT_PREC_CHEBYSHEV = 0, 1
HT_APPLY_AUTO, HT_APPLY_TILED, HT_APPLY_TWO_PASS, HT_APPLY_SINGLE_PASS = 0, 1, 2, 3
HT_BATCH_CONCURRENT, HT_BATCH_SHARED_LAUNCHES, HT_BATCH_PERSISTENT = 0, 1, 2
HT_GUESS_PREVIOUS, HT_GUESS_EXTRAPOLATE = 0, 1

ERROR_NAMES = {0: "HT_OK", -1: "HT_EINVAL", -2: "HT_ENOMEM", -3: "HT_ECUDA", -4: "HT_ENOCONV",
               -5: "HT_EBREAKDOWN", -6: "HT_ETIMEOUT"}


class Mesh(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("order", c_int),
                ("x0", c_double), ("y0", c_double), ("z0", c_double),
                ("Lx", c_double), ("Ly", c_double), ("Lz", c_double)]


class SolverOpts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_iter", c_int), ("krylov", c_int), ("restart", c_int),
                ("precond", c_int),
                ("cheb_degree", c_int), ("precision", c_int), ("inner_tol", c_double),
                ("max_outer", c_int), ("check_every", c_int), ("use_graphs", c_int),
                ("z_chunks", c_int), ("apply_variant", c_int), ("inner_tol_heat", c_double),
                ("outer_fp64", c_int), ("guess", c_int)]


class LineSrc(ctypes.Structure):
    _fields_ = [(n, c_double) for n in ("x", "y", "z_top", "z_bot", "mean", "amp", "period", "phase")]


class BoxSrc(ctypes.Structure):
    _fields_ = [(n, c_double) for n in ("x0", "x1", "y0", "y1", "z", "mean", "amp", "period", "phase")]


class Well(ctypes.Structure):
    _fields_ = [(n, c_double) for n in ("x", "y", "z_top", "z_bot", "Q", "T_in", "sigma")]


class StepStats(ctypes.Structure):
    _fields_ = [("iters_head", c_int), ("iters_heat", c_int), ("outer_head", c_int),
                ("outer_heat", c_int), ("res_head", c_double), ("res_heat", c_double),
                ("t", c_double), ("ms_loads", c_double), ("ms_head", c_double),
                ("ms_heat", c_double), ("ms_total", c_double), ("status", c_int),
                ("guess_head", c_int), ("guess_heat", c_int), ("guess_res_head", c_double),
                ("guess_res_heat", c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class ProfileStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("head_applies", ctypes.c_longlong),
                ("heat_applies", ctypes.c_longlong), ("head_apply_ms", c_double),
                ("heat_apply_ms", c_double), ("head_applies_fp32", ctypes.c_longlong),
                ("heat_applies_fp32", ctypes.c_longlong), ("head_apply_ms_fp32", c_double),
                ("heat_apply_ms_fp32", c_double), ("cg_iters", ctypes.c_longlong),
                ("bicgstab_iters", ctypes.c_longlong), ("cg_iter_ms", c_double),
                ("bicgstab_iter_ms", c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


# name -> (restype, argtypes); every function declared in include/ht.h
SIGNATURES = {
    "ht_default_solver": (c_int, [POINTER(SolverOpts)]),
    "ht_create": (c_int, [POINTER(c_void_p), POINTER(Mesh), c_int, c_void_p]),
    "ht_destroy": (None, [c_void_p]),
    "ht_last_error": (ctypes.c_char_p, [c_void_p]),
    "ht_sizes": (c_int, [c_void_p, POINTER(c_size_t), POINTER(c_size_t)]),
    "ht_set_cells": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_double, c_double, c_double]),
    "ht_set_bc": (c_int, [c_void_p, c_int, c_int, c_int, c_double]),
    "ht_set_bc_values": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_size_t]),
    "ht_face_nodes": (c_int, [c_void_p, c_int, POINTER(c_size_t)]),
    "ht_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int]),
    "ht_add_line_sources": (c_int, [c_void_p, c_int, POINTER(LineSrc)]),
    "ht_add_wells": (c_int, [c_void_p, c_int, POINTER(Well)]),
    "ht_add_box_sources": (c_int, [c_void_p, c_int, POINTER(BoxSrc)]),
    "ht_set_extra_rhs": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "ht_set_solver": (c_int, [c_void_p, POINTER(SolverOpts)]),
    "ht_step": (c_int, [c_void_p, c_double, POINTER(StepStats)]),
    "ht_get_field": (c_int, [c_void_p, c_int, c_void_p, c_size_t, c_int]),
    "ht_get_time": (c_int, [c_void_p, POINTER(c_double)]),
    "ht_apply": (c_int, [c_void_p, c_int, c_double, c_void_p, c_void_p, c_int]),
    "ht_residual": (c_int, [c_void_p, c_int, c_double, c_void_p, c_void_p, c_int, c_int, POINTER(c_double)]),
    "ht_diag": (c_int, [c_void_p, c_int, c_double, c_void_p, c_int]),
    "ht_rhs": (c_int, [c_void_p, c_int, c_double, c_void_p, c_int]),
    "ht_set_spacing": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "ht_set_seasonal_face": (c_int, [c_void_p, c_int, c_int, c_double, c_double, c_double, c_double]),
    "ht_set_pile_temperatures": (c_int, [c_void_p, c_int, c_void_p]),
    "ht_batch_create": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p)]),
    "ht_batch_destroy": (None, [c_void_p]),
    "ht_batch_step": (c_int, [c_void_p, c_double, c_void_p]),
    "ht_batch_set_mode": (c_int, [c_void_p, c_int]),
    "ht_batch_set_persistent": (c_int, [c_void_p, c_int, c_double, c_int]),
    "ht_batch_persistent_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "ht_batch_last_error": (ctypes.c_char_p, [c_void_p]),
    "ht_unet_create": (c_int, [POINTER(c_void_p), c_int, c_int, c_int, c_void_p]),
    "ht_unet_destroy": (None, [c_void_p]),
    "ht_unet_num_params": (c_int, [c_void_p]),
    "ht_unet_last_error": (ctypes.c_char_p, [c_void_p]),
    "ht_unet_set_params": (c_int, [c_void_p, c_void_p]),
    "ht_unet_get_params": (c_int, [c_void_p, c_void_p]),
    "ht_unet_forward": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "ht_unet_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, POINTER(c_double), c_void_p]),
    "ht_unet_train_step": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, ctypes.c_float,
                                   POINTER(c_double)]),
    "ht_set_learned_guess": (c_int, [c_void_p, c_void_p, c_int]),
    "ht_learned_sample": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_int)]),
    "ht_profile": (c_int, [c_void_p, c_int]),
    "ht_profile_read": (c_int, [c_void_p, POINTER(ProfileStats)]),
    "ht_head_apply_dot_noalloc": (c_int, [POINTER(Mesh), c_int, c_double, c_double, c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_int, c_void_p, ctypes.c_char_p, c_size_t]),
    "ht_mixture": (c_int, [c_double, c_double, c_double, c_double, c_double, POINTER(c_double), POINTER(c_double)]),
    "ht_specific_storage": (c_double, [c_double, c_double, c_double]),
    "ht_fma_peak": (c_int, [c_int, c_int, POINTER(c_double)]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2103_00081_gb300.build` "
                          "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB
