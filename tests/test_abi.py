"""The C-ABI library loads and exports every entry point include/rpd.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import paper_2403_18761_gb300 as pkg
from paper_2403_18761_gb300 import rpd


def test_library_exports_every_declared_symbol():
    lib = pkg.load()
    syms = pkg.header_symbols()
    assert "rpd_build" in syms and "rpd_euler" in syms and "rpd_components" in syms
    assert "rpd_contractible" in syms and "rpd_pieces" in syms
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_option_defaults_without_gpu():
    lib = pkg.load()
    o = rpd.rpd_options()
    lib.rpd_default_options(ctypes.byref(o))
    assert (o.precision, o.k, o.grid_bits, o.debug_checks, o.edge_lengths) == (rpd.RPD_FP32_FILTERED, 16, 20, 0, 0)


def test_build_rejects_bad_sizes_before_touching_the_device():
    lib = pkg.load()
    out = ctypes.c_void_p()
    st = lib.rpd_build(None, 0, None, 0, None, None, 0, None, None, ctypes.byref(out))
    assert st == rpd.RPD_E_INVALID and not out.value
    assert lib.rpd_build_error().decode()


def test_struct_layouts_match_header():
    text = open(rpd.HEADER).read()
    opt = re.search(r"typedef struct \{(.*?)\} rpd_options;", text, re.S).group(1)
    assert [n for n in re.findall(r"int32_t\s+(\w+);", opt)] == [f for f, _ in rpd.rpd_options._fields_]
    assert ctypes.sizeof(rpd.rpd_stats) == 8 * (2 + 4 + 4 + 5 + 3 + 8 + 8) + 4 * 10 + 8


def test_no_cpu_fallback_in_the_package():
    here = os.path.dirname(pkg.__file__)
    for name in os.listdir(here):
        if name.endswith(".py"):
            src = open(os.path.join(here, name)).read()
            assert "import oracle" not in src and "from oracle" not in src
