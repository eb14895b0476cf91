"""The C-ABI library loads, exports every entry point include/doctors.h
declares, and its host-only logic (quadrature tables, argument validation)
behaves; no GPU work is issued here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest
from scipy import special

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1811_12391_gb300.build import build
    build()
    from paper_1811_12391_gb300 import _lib
    return _lib


def _declared():
    txt = open(os.path.join(ROOT, "include", "doctors.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(doctors_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("doctors_create_problem", "doctors_set_materials", "doctors_set_source", "doctors_solve",
              "doctors_dose", "doctors_adjoint_solve", "doctors_destroy", "doctors_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    for n in _declared():
        assert hasattr(L, n), n
    bound = {s[0] for s in lib.SIGNATURES}
    assert set(_declared()) <= bound


@pytest.mark.parametrize("N,L", [(2, 0), (4, 1), (6, 2), (8, 3), (12, 3), (16, 3)])
def test_library_quadrature_pins(lib, N, L):
    from paper_1811_12391_gb300.solver import quadrature
    dirs, w, R = quadrature(N, L)
    assert dirs.shape == (N * (N + 2), 3)
    assert np.all(w > 0)
    assert abs(w.sum() - 4 * math.pi) < 1e-12
    np.testing.assert_allclose(np.linalg.norm(dirs, axis=1), 1, atol=1e-6)
    # degree-2L products integrate exactly where the set allows (2L <= N-1)
    if 2 * L <= N - 1:
        ls = np.array([l for l in range(L + 1) for _ in range(2 * l + 1)])
        np.testing.assert_allclose((R * w[:, None]).T @ R, np.diag(4 * math.pi / (2 * ls + 1)), atol=1e-12)
    # addition theorem against scipy's Legendre polynomials
    cos = dirs @ dirs.T
    for l in range(L + 1):
        sl = slice(l * l, (l + 1) ** 2)
        np.testing.assert_allclose(R[:, sl] @ R[:, sl].T, special.eval_legendre(l, cos), atol=1e-12)


def test_quadrature_rejects_bad_orders(lib):
    n = ctypes.c_int()
    assert lib.doctors_quadrature(5, 1, None, None, None, ctypes.byref(n)) == lib.DOCTORS_ERR_INVALID_ARG
    assert "sn_order" in lib.last_error()
    assert lib.doctors_quadrature(8, 4, None, None, None, ctypes.byref(n)) == lib.DOCTORS_ERR_INVALID_ARG


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    C = lib
    mesh = C.doctors_mesh(0, 4, 4, 1.0, 1.0, 1.0, (ctypes.c_double * 3)(0, 0, 0))
    opt = C.doctors_options()
    opt.groups, opt.sn_order, opt.legendre, opt.tol, opt.max_iters = 4, 4, 1, 1e-6, 10
    h = ctypes.c_void_p()
    assert C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt), None, ctypes.byref(h)) == \
        C.DOCTORS_ERR_INVALID_ARG
    mesh.nx = 4
    opt.sn_order = 3
    assert C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt), None, ctypes.byref(h)) == \
        C.DOCTORS_ERR_INVALID_ARG
    opt.sn_order = 4
    opt.legendre = 5
    assert C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt), None, ctypes.byref(h)) == \
        C.DOCTORS_ERR_INVALID_ARG
    opt.legendre = 1
    opt.differencing = 2
    assert C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt), None, ctypes.byref(h)) == \
        C.DOCTORS_ERR_INVALID_ARG
    assert "differencing" in C.last_error()
    opt.differencing = C.DOCTORS_DIFF_DIAMOND
    # diamond differencing: dataflow kernels on whole octants only (S16 in blocks of 12 is refused)
    for kernel, sn, ab in ((1, 4, 0), (3, 4, 0), (5, 4, 0), (0, 16, 12)):
        opt.sweep_kernel, opt.sn_order, opt.angles_per_block = kernel, sn, ab
        assert C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt), None, ctypes.byref(h)) == \
            C.DOCTORS_ERR_INVALID_ARG
        assert "diamond" in C.last_error()
    opt.angles_per_block = 0
    opt.differencing = C.DOCTORS_DIFF_STEP
    for kernel in (1, 3):
        # whole S16 octants run on the dataflow kernels only
        opt.sweep_kernel, opt.sn_order, opt.angles_per_block = kernel, 16, 36
        assert C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt), None, ctypes.byref(h)) == \
            C.DOCTORS_ERR_INVALID_ARG
    opt.angles_per_block = 0
    for kernel in (2, 6):
        # taken out (both measured slower than the kernels kept), rejected before any device call
        opt.sweep_kernel = kernel
        assert C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt), None, ctypes.byref(h)) == \
            C.DOCTORS_ERR_INVALID_ARG
        assert "not offered" in C.last_error()
    for kernel in (-1, 9):
        opt.sweep_kernel = kernel
        assert C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt), None, ctypes.byref(h)) == \
            C.DOCTORS_ERR_INVALID_ARG
        assert "sweep_kernel" in C.last_error()
    opt.sweep_kernel, opt.sn_order = 0, 4
    opt.reserved[0] = 1
    assert C.doctors_create_problem(ctypes.byref(mesh), ctypes.byref(opt), None, ctypes.byref(h)) == \
        C.DOCTORS_ERR_INVALID_ARG
    assert h.value is None
    assert C.doctors_solve(None, None) == C.DOCTORS_ERR_INVALID_ARG
    C.doctors_destroy(None)


def test_ct_conversion_checks_tables_before_touching_the_device(lib):
    """doctors_ct_to_materials validates its calibration on the host and
    returns at once for an empty image (no device needed for either)."""
    import numpy as np
    from paper_1811_12391_gb300 import solver as S
    C = lib
    hu = np.zeros(4, np.float32)
    bad = [
        ([0.0, 0.0], [0, 1, 2], [0.0, 1.0], [1.0, 1.0], "ascending"),
        ([np.nan], [0, 1], [0.0, 1.0], [1.0, 1.0], "finite"),
        ([0.0], [0, 1], [1.0, 0.0], [1.0, 1.0], "ascending"),
        ([0.0], [0, 1], [0.0, 1.0], [1.0, -1.0], ">= 0"),
        ([0.0], [0, 1], [], [], "n_knots"),
        (list(range(32)), list(range(33)), [0.0], [1.0], "n_thresholds"),
    ]
    for t, b, hk, rk, word in bad:
        try:
            S.ct_to_materials(hu, t, b, hk, rk)
        except C.DoctorsError as e:
            assert e.code == C.DOCTORS_ERR_INVALID_ARG
            assert word in str(e)
        else:
            raise AssertionError(f"accepted {t} {hk} {rk}")
    m0, r0 = S.ct_to_materials(np.zeros(0, np.float32), [], [4], [0.0], [1.25])
    assert m0.size == 0 and r0.size == 0


def _c_struct_fields(header: str, name: str):
    """(field name, array length) in declaration order of `typedef struct name {...}`
    in the public header (comments stripped)."""
    import re
    m = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), header, re.S)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "type a, b[3], c": the first part ends with the first declarator
        parts = decl.split(",")
        tm = re.match(r"((?:const\s+)?(?:unsigned\s+)?(?:long\s+long|\w+))\s*(\**)", parts[0].strip())
        ctype = tm.group(1).replace("const ", "").strip() + ("*" if tm.group(2) else "")
        for part in parts:
            mm = re.search(r"\**\s*(\w+)\s*(?:\[(\d+)\])?\s*$", part.strip())
            assert mm, (name, part)
            out.append((mm.group(1), int(mm.group(2) or 1), ctype))
    return out


def test_ctypes_structs_mirror_the_header():
    """Every struct of include/doctors.h and its ctypes mirror in the binding
    have the same fields in the same order with the same array lengths (an
    inserted option field must move in both)."""
    import ctypes
    import os
    from paper_1811_12391_gb300 import _lib as C
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "doctors.h")).read()
    ctypes_of = {"int": ctypes.c_int, "double": ctypes.c_double, "long long": ctypes.c_longlong,
                 "float": ctypes.c_float, "double*": ctypes.POINTER(ctypes.c_double)}
    for name in ("doctors_mesh", "doctors_options", "doctors_source", "doctors_result", "doctors_tuning"):
        want = _c_struct_fields(hdr, name)
        got = []
        for fname, ftype in getattr(C, name)._fields_:
            n = getattr(ftype, "_length_", 1) if issubclass(ftype, ctypes.Array) else 1
            got.append((fname, n, ftype._type_ if n > 1 else ftype))
        assert [(f, n) for f, n, _ in got] == [(f, n) for f, n, _ in want], (name, got, want)
        for (f, n, t), (_, _, ct) in zip(got, want):
            assert ct in ctypes_of, (name, f, ct)
            assert ctypes.sizeof(t) == ctypes.sizeof(ctypes_of[ct]) and \
                (t is ctypes_of[ct] or getattr(t, "_type_", None) == getattr(ctypes_of[ct], "_type_", None)), (name, f, t, ct)
        assert ctypes.sizeof(getattr(C, name)) >= 1
