"""The C-ABI library loads without a GPU and exports every function that
include/*.h declares; the Python binding declares a signature for each."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^[A-Za-z_][\w\s\*]*?\b(scuc_\w+)\s*\(", re.M)


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)      # comments
        text = re.sub(r"typedef[^;]*;", "", text, flags=re.S)   # struct and enum typedefs
        names.update(m.group(1) for m in DECL.finditer(text))
    return names


@pytest.fixture(scope="module")
def so():
    from paper_2510_10891_b300 import build
    return ctypes.CDLL(build.build())


def test_headers_declare_the_expected_entry_points():
    names = _declared()
    for must in ("scuc_lp_create", "scuc_lp_solve", "scuc_lp_solve_batch", "scuc_fix_and_propagate",
                 "scuc_ws_train", "scuc_ws_predict", "scuc_ws_assemble", "scuc_lp_solve_warm",
                 "scuc_lp_destroy", "scuc_last_error", "scuc_lp_kkt_noalloc"):
        assert must in names, must


def test_library_exports_every_declared_function(so):
    missing = [n for n in sorted(_declared()) if not hasattr(so, n)]
    assert not missing, missing


def test_binding_has_a_signature_for_every_declared_function():
    from paper_2510_10891_b300 import _lib
    assert _declared() == set(_lib._SIGS), (_declared() ^ set(_lib._SIGS))


def test_last_error_is_callable_without_a_gpu(so):
    so.scuc_last_error.restype = ctypes.c_char_p
    assert isinstance(so.scuc_last_error(), bytes)


def test_library_leaves_none_of_its_own_symbols_undefined(so):
    """Every function of the library is defined in it (a template used by
    one file and defined in another must be instantiated there), so loading
    with immediate binding succeeds on a machine without a GPU."""
    import subprocess
    from paper_2510_10891_b300 import build
    out = subprocess.run(["nm", "-D", "-C", "--undefined-only", build.SO], capture_output=True, text=True,
                         check=True).stdout
    own = [line for line in out.splitlines() if "scuc::" in line or " scuc_" in line]
    assert not own, own
    ctypes.CDLL(build.SO, mode=ctypes.RTLD_GLOBAL | os.RTLD_NOW)
