"""The C-ABI library builds for sm_103a, loads, and exports every entry point the header declares.

No compute call is made here (these tests run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stokes_vanka.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(stokes_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2401_06277_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("stokes_hierarchy_create", "stokes_vcycle_apply", "stokes_fgmres_solve",
                     "stokes_vanka_sweep", "stokes_restrict", "stokes_prolong_add", "stokes_coarse_solve",
                     "stokes_apply_operator", "stokes_residual", "stokes_last_error"):
        assert required in names, required


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_exactly_the_header(lib_path):
    from paper_2401_06277_gb300 import stokes
    stokes._load()
    assert sorted(stokes.exported_symbols()) == header_functions()


def test_library_is_built_for_sm_103a(lib_path):
    from paper_2401_06277_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.getsize(lib_path) > 0


def test_default_params_and_argument_errors_need_no_gpu(lib_path):
    """Argument validation happens on the host before any device work."""
    from paper_2401_06277_gb300 import stokes
    p = stokes.default_params()
    assert (p.nu1, p.nu2, p.coarse_n, p.restart, p.maxit) == (2, 2, 4, 30, 1000)
    assert abs(p.omega - 0.7) < 1e-15 and abs(p.rtol - 1e-8) < 1e-20
    lib = stokes._load()
    out = ctypes.c_void_p()
    for n in (12, 6, 3):      # not coarse_n * 2^k
        st = lib.stokes_hierarchy_create(n, 1.0, ctypes.byref(p), None, ctypes.byref(out))
        assert st == stokes.STOKES_ERR_ARG
        assert b"coarse_n" in lib.stokes_last_error()
    st = lib.stokes_hierarchy_create(16, -1.0, ctypes.byref(p), None, ctypes.byref(out))
    assert st == stokes.STOKES_ERR_ARG
    bad = stokes.default_params()
    bad.restart = 0
    assert lib.stokes_hierarchy_create(16, 1.0, ctypes.byref(bad), None, ctypes.byref(out)) == stokes.STOKES_ERR_ARG
    assert lib.stokes_vcycle_apply(None, None, None) == stokes.STOKES_ERR_ARG
    assert lib.stokes_hierarchy_destroy(None) == stokes.STOKES_OK


def test_product_code_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2401_06277_gb300")
    pat = re.compile(r"^\s*(from\s+oracle|import\s+oracle|from\s+\.+oracle)", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                assert not pat.search(open(os.path.join(dirpath, f)).read()), f


def _header_struct_fields(name):
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    # enum-typed fields (stokes_precision) are ints
    fields = re.findall(r"^\s*(int|double|long long|stokes_[a-z]+)\s+([a-z0-9_]+)\s*;", m.group(1), flags=re.M)
    return [("int" if t.startswith("stokes_") else t, f) for t, f in fields]


@pytest.mark.parametrize("name", ["stokes_params", "stokes_stats"])
def test_binding_structs_match_the_header(name):
    """The ctypes mirrors of the header's structs have the same fields, in the same order, of the same types."""
    import ctypes as C
    from paper_2401_06277_gb300 import stokes
    ctype = {"int": C.c_int, "double": C.c_double, "long long": C.c_longlong}
    want = [(f, C.sizeof(ctype[t]), t == "double") for t, f in _header_struct_fields(name)]
    got = [(f, C.sizeof(t), t is C.c_double) for f, t in getattr(stokes, name)._fields_]
    assert got == want


def test_orth_parameter_default_and_range(lib_path):
    from paper_2401_06277_gb300 import stokes
    p = stokes.default_params()
    assert p.orth == 0
    lib = stokes._load()
    out = ctypes.c_void_p()
    p.orth = 3
    assert lib.stokes_hierarchy_create(16, 1.0, ctypes.byref(p), None, ctypes.byref(out)) == stokes.STOKES_ERR_ARG
    assert b"orth" in lib.stokes_last_error()
