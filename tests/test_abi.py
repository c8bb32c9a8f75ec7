"""The C-ABI library loads and exports every symbol include/dpinn.h declares.

CPU only: no call here touches a GPU (creation is only exercised on a
configuration that fails host-side validation).
"""
import ctypes as C
import os
import re

import pytest

from paper_2602_15883_b300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dpinn.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dpinn_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS) == names


def test_config_default_is_host_only(lib):
    c = binding.Config()
    assert lib.dpinn_config_default(C.addressof(c)) == 0
    assert c.lr == 1e-3 and c.beta1 == 0.9 and c.beta2 == 0.999 and c.eps == 1e-8
    assert c.width == 32 and c.depth == 4 and list(c.splits) == [1, 1, 1, 1]


@pytest.mark.parametrize("field,value", [("width", 48), ("width", 100), ("width", 225), ("depth", 0),
                                         ("d_space", 4), ("activation", 2),
                                         ("precision", 2), ("precision", 1),
                                         ("beta1", 1.0), ("beta2", -0.1), ("beta2", float("nan"))])
def test_create_rejects_bad_configs_before_touching_a_device(lib, field, value):
    c = binding.Config()
    lib.dpinn_config_default(C.addressof(c))
    setattr(c, field, value)
    h = C.c_void_p()
    rc = lib.dpinn_create(C.addressof(c), C.addressof(h))
    assert rc == -1 and not h.value
    assert lib.dpinn_last_error(None)


def test_tf32x3_needs_width_128(lib):
    c = binding.Config()
    lib.dpinn_config_default(C.addressof(c))
    c.precision = 1
    c.width = 64
    h = C.c_void_p()
    assert lib.dpinn_create(C.addressof(c), C.addressof(h)) == -1
    assert b"width 128" in lib.dpinn_last_error(None)


def test_create_rejects_anchor_outside_domain(lib):
    c = binding.Config()
    lib.dpinn_config_default(C.addressof(c))
    c.anchor_x[0] = 2.0
    h = C.c_void_p()
    assert lib.dpinn_create(C.addressof(c), C.addressof(h)) == -1
    assert b"anchor" in lib.dpinn_last_error(None)


def test_struct_layout_matches_header():
    # dpinn_config: 2 ints, 8 doubles, 4 ints, 3 ints, ... as declared
    c = binding.Config
    assert c.lo.offset == 8 and c.hi.offset == 40 and c.splits.offset == 72
    assert c.nu.offset == 104 and c.seed.offset % 8 == 0
    assert C.sizeof(binding.Layout) == 24
