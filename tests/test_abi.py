"""CPU checks of the C-ABI library: it builds, loads and exports every declared symbol.

No compute call is made here (there is no GPU in the CPU suite).
"""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for fn in sorted(os.listdir(HEADER_DIR)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(helm6_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1212_1397_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("helm6_create", "helm6_apply_A", "helm6_apply_Pinv", "helm6_solve",
                     "helm6_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_header_function(lib_path):
    from paper_1212_1397_gb300 import helm6 as H
    assert set(H.EXPORTS) == set(declared_functions())
    H.load(lib_path)


def test_status_strings_and_defaults(lib_path):
    """Host-only calls (no device work): status strings and default options."""
    from paper_1212_1397_gb300 import helm6 as H
    lib = H.load(lib_path)
    for code in H.STATUS:
        assert lib.helm6_status_string(code)
    o = H.Opts()
    lib.helm6_opts_default(ctypes.byref(o))
    assert o.precision == H.FP64 and o.method == H.GMRES and o.max_restart == 30
    assert o.xform_terms == 3 and abs(o.inner_tol - 1e-5) < 1e-20


def test_create_rejects_bad_arguments_before_touching_the_device(lib_path):
    from paper_1212_1397_gb300 import helm6 as H
    lib = H.load(lib_path)
    ctx = ctypes.c_void_p()
    k = H.C64(5.0, 0.0)
    faces_bad = (ctypes.c_int * 6)(2, 0, 0, 0, 0, 2)        # Sommerfeld-like on two axis pairs
    assert lib.helm6_create(ctypes.byref(ctx), 8, 0.0, k, faces_bad, None) == -1
    faces_bad = (ctypes.c_int * 6)(0, 0, 2, 2, 2, 0)
    assert lib.helm6_create(ctypes.byref(ctx), 8, 0.0, k, faces_bad, None) == -1
    faces = (ctypes.c_int * 6)(0, 0, 0, 0, 0, 0)
    assert lib.helm6_create(ctypes.byref(ctx), 0, 0.0, k, faces, None) == -1
    o = H.Opts()
    lib.helm6_opts_default(ctypes.byref(o))
    o.max_restart = 1000
    assert lib.helm6_create(ctypes.byref(ctx), 8, 0.0, k, faces, ctypes.byref(o)) == -1
    lib.helm6_opts_default(ctypes.byref(o))
    assert o.transform == H.XFORM_AUTO
    for bad in (-1, H.XFORM_TENSOR):   # TENSOR is a reported value, not an option
        o.transform = bad
        assert lib.helm6_create(ctypes.byref(ctx), 8, 0.0, k, faces, ctypes.byref(o)) == -1
    assert lib.helm6_transform(None, 0) == -1


def test_noalloc_binding_rejects_wrong_sizes_before_any_launch():
    """residual_noalloc checks F, u and r against the grid that n and faces imply before it
    touches the library or the device (a short r would be written out of bounds)."""
    torch = pytest.importorskip("torch")
    from paper_1212_1397_gb300 import helm6 as H
    n, faces = 6, "DDNNSS"            # 6 x 8 x 8 unknowns
    good = torch.zeros((8, 8, 6), dtype=torch.complex128)
    short = torch.zeros(8 * 8 * 6 - 1, dtype=torch.complex128)
    ss = torch.zeros(1, dtype=torch.float64)
    for F, u, r in ((short, good, good), (good, short, good), (good, good, short)):
        with pytest.raises(ValueError):
            H.residual_noalloc(n, 3.0, faces, F, u, r, ss)
    with pytest.raises(ValueError):
        H.residual_noalloc(n, 3.0, "DDNNS", good, good, good, ss)
    with pytest.raises(ValueError):
        H.residual_noalloc(n, 3.0, "DDNNSX", good, good, good, ss)
