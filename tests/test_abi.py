"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/sgp.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    with open(os.path.join(ROOT, "include", "sgp.h")) as f:
        txt = f.read()
    names = re.findall(r"^\s*(?:sgp_status|void|const \w+ \*)\s*\*?(sgp_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2410_04512_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("sgp_collision_graph", "sgp_friction_assemble", "sgp_max_spanning_tree",
                 "sgp_tree_factor", "sgp_pcg_solve", "sgp_create", "sgp_destroy", "sgp_spmv",
                 "sgp_tree_apply", "sgp_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (sgp_\w+)", out))
    assert set(declared()) <= exported


def test_binding_names_match_header():
    import paper_2410_04512_gb300 as sgp
    assert set(sgp.exported_symbols()) == set(declared())


def test_build_targets_sm103a_only():
    from paper_2410_04512_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.sgp_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sgp_version()


def test_create_fails_cleanly_without_device(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = ctypes.CDLL(libpath)
    p = ctypes.c_void_p()
    rc = lib.sgp_create(ctypes.byref(p), 0, None)
    assert rc != 0 and not p.value
