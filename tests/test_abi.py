"""The C ABI: the library loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gkb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gkb_geometry_create", "gkb_geometry_destroy", "projector_forward", "projector_back",
                     "projector_forward_adjoint", "projector_back_adjoint", "gkb_solve", "gkb_solve_batched"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2606_31153_b300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_argument_checks_without_gpu():
    import paper_2606_31153_b300 as gkb
    lib = gkb.load_library()
    assert lib.gkb_status_string(gkb.ERR_INVALID_ARG) == b"invalid argument"
    assert lib.gkb_version().decode().count(".") == 2
    # invalid descriptors are rejected on the host before any CUDA call
    out = ctypes.c_void_p()
    assert lib.gkb_geometry_create(None, ctypes.byref(out)) == gkb.ERR_INVALID_ARG
    ang = (ctypes.c_double * 1)(0.0)
    bad = gkb.GeometryDesc(gkb.PARALLEL, 0, 4, 1.0, 1, ang, 5, 1.0, 0.0, 0.0)
    assert lib.gkb_geometry_create(ctypes.byref(bad), ctypes.byref(out)) == gkb.ERR_INVALID_ARG
    fan_inside = gkb.GeometryDesc(gkb.FAN_FLAT, 64, 64, 1.0, 1, ang, 91, 1.0, 30.0, 60.0)
    assert lib.gkb_geometry_create(ctypes.byref(fan_inside), ctypes.byref(out)) == gkb.ERR_INVALID_ARG
    p = gkb.make_params(k_max=0)
    assert lib.gkb_solve(None, ctypes.byref(p), None, None, None, None) == gkb.ERR_INVALID_ARG
