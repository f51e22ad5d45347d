"""The C ABI library builds, loads, and exports every entry point cs.h declares.

CPU only: no compute call is made here (the host has no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2512_08465_gb300 import build as libbuild
from paper_2512_08465_gb300 import cs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cs_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    path = libbuild.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"cs_load_network", "cs_submit_contingencies", "cs_poll", "cs_risk_index"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(cs.EXPORTS) <= names


def test_binding_loads_and_defaults():
    L = cs.load_library()
    o = cs.default_options()
    assert abs(o.damping_min - 0.05) < 1e-15 and abs(o.opf_tol - 1e-8) < 1e-20 and o.opf_max_it == 50
    assert L.cs_last_error(None) == b"no context"


def test_library_is_built_for_sm103a_only():
    """The build compiles every translation unit for sm_103a and nothing else."""
    assert libbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(libbuild.LIB)
