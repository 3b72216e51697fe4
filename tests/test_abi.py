"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/vie.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_1903_07884_gb300 import build, vie

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vie.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][A-Za-z_0-9]*\s*\**\s+)+\**(vie_[a-z_0-9]+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("vie_plan_create", "vie_set_permittivity", "vie_build_preconditioner", "vie_matvec",
                 "vie_precond_apply", "vie_solve", "vie_solve_batch", "vie_server_submit", "vie_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the Python binding wraps every declared entry point under the same name
    assert set(declared_functions()) <= set(vie.exported_symbols())


def test_default_opts_and_estimate_without_gpu():
    o = vie.default_opts()
    assert o.restart == 50 and o.precision == vie.VIE_MIXED and o.homog == vie.VIE_HOM_REALMEAN
    assert abs(o.reduce_tol - 1e-3) < 1e-18
    est = vie.vie_estimate_bytes(1024, 16, 8, o)
    assert 1e8 < est < 2e10


def _header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/vie.h, in order."""
    text = open(os.path.join(ROOT, "include", "vie.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "int x0, y0, z0" or "const vie_box* boxes"
        head, *rest = [s.strip() for s in decl.split(",")]
        fields.append(re.findall(r"[A-Za-z_][A-Za-z_0-9]*", head)[-1])
        fields.extend(re.findall(r"[A-Za-z_][A-Za-z_0-9]*", r)[-1] for r in rest)
    return fields


def test_ctypes_structs_match_the_header():
    """The binding's structs list the header's fields in the same order (a
    field added on one side only would shift every later field)."""
    for cls in (vie.vie_box, vie.vie_opts, vie.vie_info):
        assert [f for f, _ in cls._fields_] == _header_struct_fields(cls.__name__), cls.__name__


def test_box_tuples_of_six_or_seven_values():
    """A 6-tuple box is a 1-level box (levels 0); the 7th value selects the level."""
    b6 = vie.vie_box(*(1, 2, 3, 4, 5, 6))
    b7 = vie.vie_box(*(1, 2, 3, 4, 5, 6, 2))
    assert (b6.nz, b6.levels) == (6, 0) and b7.levels == 2
