"""The C ABI library builds, loads, and exports every entry point cs.h declares.

CPU only: no compute call is made here (the host has no GPU)."""
import ctypes
import os
import re
import shutil
import subprocess

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
    assert o.main_island == 0 and o.serve_slots == 3 and o.batch_cap == 4096 and o.autotune == 0
    assert cs.default_options(main_island=1, chunk=4096).main_island == 1
    with pytest.raises(TypeError):
        cs.default_options(main_islnd=1)                 # a misspelt option is an error, not ignored
    assert L.cs_last_error(None) == b"no context"


@pytest.mark.parametrize("cname,py", [("cs_options", cs.Options), ("cs_result", cs.Result),
                                      ("cs_network_desc", cs.NetworkDesc)])
def test_struct_layouts_match_the_header(cname, py, tmp_path):
    """Every field offset and the size of the binding's ctypes mirrors equal the C
    compiler's for include/cs.h (a C probe compiled with the host compiler)."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = [f'printf("size %zu\\n", sizeof({cname}));']
    lines += [f'printf("{f} %zu\\n", offsetof({cname}, {f}));' for f, _ in py._fields_]
    src = tmp_path / "probe.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"cs.h\"\nint main(void) {\n"
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    assert int(got["size"]) == ctypes.sizeof(py)
    for f, _ in py._fields_:
        assert int(got[f]) == getattr(py, f).offset, f


def test_library_is_built_for_sm103a_only():
    """The build compiles every translation unit for sm_103a and nothing else."""
    assert libbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(libbuild.LIB)
