"""The C ABI library loads and exports every entry point its headers declare (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mrp_[a-z_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2512_08555_gb300 import build
    build.build()
    from paper_2512_08555_gb300 import mrp
    return mrp.load_library()


def test_headers_declare_the_boundary():
    d = _declared()
    for name in ("mrp_create", "mrp_solve", "mrp_solve_adjoint", "mrp_destroy", "mrp_error_string"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    from paper_2512_08555_gb300 import mrp
    assert set(mrp.EXPORTED) == _declared()


def test_error_strings(lib):
    assert lib.mrp_error_string(0) == b"ok"
    assert lib.mrp_error_string(2) == b"invalid forest"


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2512_08555_gb300 import mrp
    h = ctypes.c_void_p()
    assert lib.mrp_create(None, None, 1, None) == 1
    assert lib.mrp_create(ctypes.byref(h), None, 1, None) == 1
    assert lib.mrp_destroy(None) == 0
    st = mrp.Stats()
    assert lib.mrp_solve(None, None, None, None, ctypes.byref(st)) == 1
    assert lib.mrp_solve_graph(None, None, None, None, ctypes.byref(st)) == 1
    assert lib.mrp_solve_host(None, None, None, None, ctypes.byref(st)) == 1
    assert lib.mrp_solve_adjoint(None, None, None, None, ctypes.byref(st)) == 1


def test_option_and_stats_structs_match_the_header():
    """The binding's ctypes structs have the header's field order (parsed from include/mrp.h)."""
    from paper_2512_08555_gb300 import mrp
    txt = open(os.path.join(ROOT, "include", "mrp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    for name, cls in (("mrp_options", mrp._Options), ("mrp_stats", mrp.Stats), ("mrp_forest", mrp._Forest)):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", txt).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            names = decl.split(None, 1)[1] if not decl.startswith("const") else decl.split("*", 1)[1]
            for nm in names.split(","):
                fields.append(re.sub(r"[\s*]|\[.*\]", "", nm))
        assert fields == [f for f, _ in cls._fields_], (name, fields)


def _forest_struct(nb0, n, lev, ijk):
    from paper_2512_08555_gb300 import mrp
    import numpy as np
    lev = np.ascontiguousarray(lev, np.int32)
    ijk = np.ascontiguousarray(ijk, np.int32)
    fd = mrp._Forest()
    fd.nb0[:] = nb0
    fd.n = n
    fd.origin[:] = [0.0, 0.0, 0.0]
    fd.h0 = 0.1
    fd.n_leaves = len(lev)
    fd.leaf_level = lev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    fd.leaf_ijk = ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    fd.ncomp = 1
    return fd, (lev, ijk)


def _opts(order=4):
    from paper_2512_08555_gb300 import mrp
    op = mrp._Options()
    op.order, op.tol, op.stop_rule, op.max_cycles, op.nu1, op.nu2 = order, 1e-10, 0, 10, 3, 3
    return op


@pytest.mark.parametrize("case", ["odd_n", "boundary_refined", "gap", "overlap", "unbalanced"])
def test_invalid_forest_rejected_on_host(lib, case):
    """mrp_create validates the forest before touching the device."""
    import numpy as np
    from paper_2512_08555_gb300 import synth
    desc = synth.adaptive_forest((4, 4, 4), 8, (0, 0, 0), 0.1, 1, lambda k, c: np.ones(len(c), bool))
    lev, ijk, n = desc.leaf_level.copy(), desc.leaf_ijk.copy(), 8
    if case == "odd_n":
        n = 9
    elif case == "boundary_refined":
        keep = ~((lev == 0) & np.all(ijk == 0, axis=1))
        kids = np.array([(o & 1, (o >> 1) & 1, (o >> 2) & 1) for o in range(8)])
        lev, ijk = np.concatenate([lev[keep], np.ones(8, int)]), np.concatenate([ijk[keep], kids])
    elif case == "gap":
        lev, ijk = lev[1:], ijk[1:]
    elif case == "overlap":
        lev, ijk = np.concatenate([lev, [0]]), np.concatenate([ijk, [[1, 1, 1]]])
    elif case == "unbalanced":
        l1 = np.nonzero(lev == 1)[0][0]
        c = ijk[l1]
        g = np.array([(2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + ((o >> 2) & 1)) for o in range(8)])
        lev = np.concatenate([np.delete(lev, l1), np.full(8, 2)])
        ijk = np.concatenate([np.delete(ijk, l1, axis=0), g])
    fd, keep = _forest_struct([4, 4, 4], n, lev, ijk)
    h = ctypes.c_void_p()
    rc = lib.mrp_create(ctypes.byref(h), ctypes.byref(fd), 1, ctypes.byref(_opts()))
    assert rc == 2 and not h


def test_bad_options_rejected(lib):
    from paper_2512_08555_gb300 import synth
    desc = synth.uniform_forest((2, 2, 2), 8, (0, 0, 0), 0.1)
    fd, keep = _forest_struct([2, 2, 2], 8, desc.leaf_level, desc.leaf_ijk)
    h = ctypes.c_void_p()
    op = _opts(order=3)
    assert lib.mrp_create(ctypes.byref(h), ctypes.byref(fd), 1, ctypes.byref(op)) == 1
    op = _opts()
    op.max_cycles = 0
    assert lib.mrp_create(ctypes.byref(h), ctypes.byref(fd), 1, ctypes.byref(op)) == 1


@pytest.mark.parametrize("launch", [100, 129, 512 | 4096, 4096, 128 | 8192, 64])
def test_bad_launch_choices_rejected(lib, launch):
    """mrp_options.launch takes 0, 128, 256 or 512, and 128 or 256 with MRP_LAUNCH_NOSTAGE (4096) only."""
    from paper_2512_08555_gb300 import synth
    desc = synth.uniform_forest((2, 2, 2), 8, (0, 0, 0), 0.1)
    fd, keep = _forest_struct([2, 2, 2], 8, desc.leaf_level, desc.leaf_ijk)
    h = ctypes.c_void_p()
    op = _opts()
    op.launch = launch
    assert lib.mrp_create(ctypes.byref(h), ctypes.byref(fd), 1, ctypes.byref(op)) == 1 and not h


def test_launch_flag_matches_the_header():
    from paper_2512_08555_gb300.mrp import MRP_LAUNCH_NOSTAGE
    hdr = open(os.path.join(ROOT, "include", "mrp.h")).read()
    assert f"MRP_LAUNCH_NOSTAGE = {MRP_LAUNCH_NOSTAGE}" in hdr
