"""The C-ABI library loads on the host and exports every declared entry point.

No device compute here: these run on machines without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gblb.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    return lb


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lb_create", "lb_destroy", "lb_upload_geometry", "lb_build_corrections",
                 "lb_load_corrections", "lb_apply_S", "lb_apply_Sp", "lb_apply_gradS", "lb_apply_A",
                 "lb_solve_lb", "lb_harmonic_fields"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lb_[A-Za-z0-9_]+)", out))
    assert set(_declared()) <= exported


def test_default_params_and_null_handling(lib):
    p = lib.default_params()
    assert p.tol == 1e-10 and p.max_iter == 100 and p.formulation == lib.LB_A3
    assert p.near_factor == 2.0 and p.eps_quad == 1e-12 and p.precision == lib.LB_FP64
    assert lib.lib.lb_destroy(None) == lib.LB_OK
    assert lib.lib.lb_default_params(None) == lib.LB_EINVAL
    assert lib.lib.lb_apply_S(None, 1, None, None) == lib.LB_EINVAL
    assert lib.lib.lb_upload_geometry(None, 1, 4, None, None, None, None, None) == lib.LB_EINVAL


def test_bad_params_rejected(lib):
    p = lib.default_params(near_factor=0.5)
    h = ctypes.c_void_p()
    rc = lib.lib.lb_create(ctypes.byref(h), 0, ctypes.byref(p))
    assert rc in (lib.LB_EINVAL, lib.LB_ECUDA)   # no device here gives LB_ECUDA first
    assert lib.lib.lb_last_error(None)


def test_no_device_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(lib.LBError) as e:
        lib.Context(0)
    assert e.value.code == lib.LB_ECUDA


def test_binding_covers_every_declared_entry_point():
    """Each declared function has a ctypes signature in the Python binding."""
    src = open(os.path.join(ROOT, "paper_2111_10743_gb300", "__init__.py")).read()
    missing = [n for n in _declared() if f'"{n}"' not in src and f"lib.{n}" not in src]
    assert not missing, missing
