"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/og.h declares (no compute calls: this runs without a GPU)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

from paper_2609_17658_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(og_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("og_create", "og_tree_build", "og_tree_force", "og_tree_free", "og_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (og_[a-z0-9_]+)", out))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_resolves(libpath):
    L = ctypes.CDLL(libpath)
    for name in _declared():
        assert getattr(L, name) is not None
    L.og_last_error.restype = ctypes.c_char_p
    assert L.og_last_error() == b""


def test_binding_has_the_c_names():
    from paper_2609_17658_gb300 import og
    for name in _declared():
        if name in ("og_params_default",):
            continue
        assert hasattr(og, name), name


def test_build_targets_sm103a_only():
    # one -gencode, native sm_103a code and no PTX for run-time compilation
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.gpu
def test_device_code_is_sm103a(libpath):
    from paper_2609_17658_gb300 import og
    assert og.og_device_code_version() == 103


def test_failure_injection_arguments_without_gpu(libpath):
    from paper_2609_17658_gb300 import og
    L = og.lib()
    assert L.og_debug_fail_allocations(0, -1) == og.OG_ERR_ARG
    assert L.og_debug_fail_allocations(-1, 1) == og.OG_ERR_ARG
    assert L.og_debug_fail_allocations(0, 0) == og.OG_OK


def test_params_defaults_without_gpu(libpath):
    from paper_2609_17658_gb300 import og
    p = og.og_params()
    assert og.lib().og_params_default(ctypes.byref(p)) == 0
    assert p.box == 1.0 and p.theta == 0.5 and p.rcut_over_rs == 4.5 and p.group_max == 32
