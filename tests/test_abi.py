"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (no GPU needed: no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:long\s+long|int|void|char|double|float|size_t)\s*\*?\s*(\w+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2405_17696_gb300 import build
    return build.build()


def test_header_declares_the_path_entry_points():
    names = _declared()
    for n in ("helm_setup", "helm_solve", "helm_apply", "helm_vcycle", "helm_destroy", "helm_last_error",
              "helm_default_opts"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_default_opts_and_error_string(libpath):
    from paper_2405_17696_gb300 import native
    o = native.helm_default_opts()
    assert (o.restart, o.max_iter, o.mg_levels, o.pre, o.post) == (10, 300, 3, 2, 2)
    assert abs(o.sl_beta - 0.5) < 1e-7
    assert isinstance(native.last_error(), str)
