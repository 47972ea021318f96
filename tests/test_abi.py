"""The C ABI library builds, loads without a GPU, and exports every entry
point include/mcubes.h declares; host-side argument checks that need no
device."""
import ctypes
import os
import re

import pytest

from paper_2202_01753_gb300 import build, mcubes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mcubes_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mcubes.lib()


def test_exports_every_declared_symbol(lib):
    decl = declared_functions()
    assert len(decl) >= 18
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) <= set(mcubes.EXPORTED)


def test_defaults_and_strerror(lib):
    o = mcubes.mcubes_default_opts()
    assert (o.nbins, o.ita, o.g_override, o.alpha, o.seed, o.precision) == (500, -1, 0, 1.5, 0, 0)
    for st in range(8):
        assert lib.mcubes_strerror(st)
    assert lib.mcubes_strerror(99) == b"unknown status"


def test_null_arguments_rejected_without_device(lib):
    h = ctypes.c_void_p()
    assert lib.mcubes_create(None, 0, None) == mcubes.EINVAL
    bad = mcubes.make_opts(nbins=1)
    assert lib.mcubes_create(ctypes.byref(h), 0, ctypes.byref(bad)) == mcubes.EINVAL
    bad = mcubes.make_opts(lanes_per_cube=3)
    assert lib.mcubes_create(ctypes.byref(h), 0, ctypes.byref(bad)) == mcubes.EINVAL
    assert lib.mcubes_destroy(None) == mcubes.OK
    assert lib.mcubes_iterate(None, 1) == mcubes.EINVAL
    assert lib.mcubes_integrate(None, 0, None, 0, 1, None, None, 10, 1, 0.0, 0.0, None) == mcubes.EINVAL
