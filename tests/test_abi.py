"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
function declared in include/ht.h, and its pure host helpers behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "ht.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ht_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib(built_lib):
    from paper_2103_00081_gb300 import _lib
    return _lib.load(built_lib)


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2103_00081_gb300 import _lib
    names = _declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"{n} has no ctypes signature"


def test_host_helpers(lib):
    from paper_2103_00081_gb300 import _lib
    o = _lib.SolverOpts()
    assert lib.ht_default_solver(ctypes.byref(o)) == 0
    assert o.tol == 1e-10 and o.precision == _lib.HT_FP64
    lam, cT = ctypes.c_double(), ctypes.c_double()
    assert lib.ht_mixture(0.3, 2.5, 0.6, 2.0e6, 4.18e6, ctypes.byref(lam), ctypes.byref(cT)) == 0
    assert abs(lam.value - 1.93) < 1e-14 and abs(cT.value - 2.654e6) < 1e-6
    assert abs(lib.ht_specific_storage(1e5, 1000.0, 9.81) - 0.0981) < 1e-16
    assert lib.ht_mixture(1.5, 1, 1, 1, 1, ctypes.byref(lam), ctypes.byref(cT)) == _lib.HT_EINVAL


def test_invalid_mesh_is_rejected_before_touching_the_device(lib):
    from paper_2103_00081_gb300 import _lib
    h = ctypes.c_void_p()
    bad = _lib.Mesh(4, 4, 4, 3, 0, 0, 0, 1, 1, 1)
    assert lib.ht_create(ctypes.byref(h), ctypes.byref(bad), 0, None) == _lib.HT_EINVAL
    assert b"order" in lib.ht_last_error(None)
    bad = _lib.Mesh(0, 4, 4, 1, 0, 0, 0, 1, 1, 1)
    assert lib.ht_create(ctypes.byref(h), ctypes.byref(bad), 0, None) == _lib.HT_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: loading a library that is not there raises."""
    from paper_2103_00081_gb300 import _lib
    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "libht.so"))


def test_struct_layouts_match_the_header():
    """The ctypes structures have the field counts and sizes of include/ht.h."""
    from paper_2103_00081_gb300 import _lib
    txt = open(os.path.join(ROOT, "include", "ht.h")).read()

    def fields(name):
        m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", txt)
        body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
        n = 0
        for decl in body.split(";"):
            decl = decl.strip()
            if decl:
                n += len(decl.split(None, 1)[1].split(","))
        return n
    for cname, cls in (("ht_mesh", _lib.Mesh), ("ht_line_src", _lib.LineSrc), ("ht_well", _lib.Well),
                       ("ht_box_src", _lib.BoxSrc), ("ht_solver_opts", _lib.SolverOpts),
                       ("ht_step_stats", _lib.StepStats), ("ht_profile_stats", _lib.ProfileStats)):
        assert fields(cname) == len(cls._fields_), cname
    assert ctypes.sizeof(_lib.BoxSrc) == 9 * 8 and ctypes.sizeof(_lib.LineSrc) == 8 * 8

