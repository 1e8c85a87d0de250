"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point that include/pd.h declares.  No compute calls."""
import ctypes
import os
import re
import sys

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2506_05362_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["pd_create", "pd_build_bonds", "pd_step", "pd_damage", "pd_bulk_stress",
                     "pd_forces", "pd_get_state", "pd_set_state", "pd_mlp_forward", "pd_mlp_train_step"]:
        assert required in names


def test_pack_broken_layout():
    """Bit c % 32 of word c // 32 for slot c, as pd_get_state_packed writes it."""
    sys.path.insert(0, ROOT)
    from paper_2506_05362_gb300 import pd
    b = np.zeros(70, np.uint8)
    b[[0, 31, 32, 69]] = 1
    w = pd.pack_broken(b)
    assert w.dtype == np.uint32 and len(w) == 3
    assert w.tolist() == [(1 << 0) | (1 << 31), 1 << 0, 1 << 5]


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, f"not exported: {missing}"


def test_default_options_without_gpu(libpath):
    from paper_2506_05362_gb300 import pd
    o = pd.pd_default_options()
    assert o.precision == pd.PD_MIXED and o.contact == 1 and o.graph_chunk == 64
    assert o.lanes_per_node == 0 and not o.alloc


def test_oracle_and_library_share_no_code():
    """The oracle never includes or loads the CUDA sources and vice versa."""
    csrc = os.path.join(ROOT, "paper_2506_05362_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read()
    for f in ["pd_oracle.c", "__init__.py", "mlp.py"]:
        txt = open(os.path.join(ROOT, "oracle", f)).read()
        assert "paper_2506_05362_gb300" not in txt and "libpd" not in txt


def test_binding_fails_loudly_without_the_library():
    """No CPU fallback: with the library missing, the binding raises at its first
    call instead of computing anything another way."""
    import subprocess
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2506_05362_gb300 import pd\n"
            "pd.LIB_PATH = %r\n"
            "try:\n"
            "    pd.lib()\n"
            "except RuntimeError as e:\n"
            "    print('raised:', 'not built' in str(e))\n" % (ROOT, os.path.join(ROOT, "no_such_dir", "libpd.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-1000:]
    assert r.stdout.strip() == "raised: True"


def test_binding_has_no_library_override():
    """The binding always loads the in-tree build: no environment variable can
    point the tests or the benchmark at another library."""
    txt = open(os.path.join(ROOT, "paper_2506_05362_gb300", "pd.py")).read()
    assert "environ" not in txt


def test_product_package_never_imports_the_oracle():
    """The package (binding, scenarios, surrogate) has no path into oracle/."""
    pkg = os.path.join(ROOT, "paper_2506_05362_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            txt = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in txt and "from oracle" not in txt, f
