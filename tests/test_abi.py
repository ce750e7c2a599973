"""CPU checks of the C ABI boundary: the library builds, loads without a GPU
and exports every function include/*.h declares."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(", src, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2107_08119_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert "nep_compute_efv" in names and "nep_md_step" in names and "nep_heat_current" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep
    assert set(_declared()) <= set(nep.exported_symbols())


def test_error_paths_need_no_gpu():
    """Argument checks fail with status codes before touching the device."""
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep as N
    import numpy as np
    h = N.Hyper(n_max_A=3)
    z = np.zeros(h.n_par, np.float32)
    try:
        N.NEP(z, h)
        raise AssertionError("expected NEP_ERR_UNSUPPORTED")
    except N.NepError as e:
        assert e.code == -8
    h = N.Hyper()
    try:
        N.NEP(np.zeros(h.n_par - 1, np.float32), h)
        raise AssertionError("expected NEP_ERR_ARG")
    except N.NepError as e:
        assert e.code == -1
