"""The C-ABI library builds, loads and exports every symbol include/*.h declares (CPU only)."""
import glob
import os
import re

import pytest

from paper_2308_09782_gb300 import build as B
from paper_2308_09782_gb300 import vgtb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(vgtb_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return vgtb.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vgtb_create", "vgtb_set_field", "vgtb_propagate", "vgtb_observables",
                     "vgtb_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_exports():
    assert set(declared_functions()) <= set(vgtb.EXPORTS)


def test_struct_layout_matches_header(lib):
    import ctypes as C
    # default options round-trip through the library (no GPU needed)
    o = vgtb.VgtbOptions()
    lib.vgtb_default_options(C.byref(o))
    assert o.precision == vgtb.FP64 and o.init == vgtb.INIT_GROUND
    assert o.obs_stride == 1 and o.graph_steps == 32 and o.scc_max_iter == 200
    assert abs(o.scc_tol - 1e-11) < 1e-25 and o.timeout_ns == 2_000_000_000
    # the trailing fields: a layout mismatch would misplace these
    assert o.integrator == vgtb.LEAPFROG and o.cn_iter == 12 and abs(o.cn_tol - 1e-10) < 1e-24
    assert list(o.tile_variant) == [-1, -1]


def test_destroy_is_null_safe(lib):
    lib.vgtb_destroy(None)


def test_create_rejects_null_output(lib):
    import ctypes as C
    rc = lib.vgtb_create(None, None, None)
    assert rc == -1
    assert b"NULL" in lib.vgtb_last_error(None)


def test_library_has_no_oracle_dependency():
    """The product path never imports the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2308_09782_gb300")
    for f in glob.glob(os.path.join(pkg, "*.py")):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src, f
