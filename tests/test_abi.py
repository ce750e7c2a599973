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


def test_analysis_entry_points_reject_bad_arguments_without_a_gpu():
    """The spectral and HNEMD analysis calls check their arguments on the host
    (NULL buffers, empty lengths, a non-finite x per omega) and return
    NEP_ERR_ARG with a message, before any device work."""
    import ctypes as C
    import math

    from paper_2107_08119_gb300 import build
    build.build()
    lib = C.CDLL(build.LIB)
    lib.nep_last_error.restype = C.c_char_p
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    lib.nep_hnemd_kappa.argtypes = [vp, i, d, vp, vp]
    lib.nep_shc_quantum.argtypes = [vp, i, d, vp, vp]
    lib.nep_shc_spectrum.argtypes = [vp, i, d, i, vp, d, i, vp, vp]
    lib.nep_hnemd_kappa_si.argtypes = [vp, i, d, d, d, vp, vp]
    lib.nep_kappa_spectrum.argtypes = [vp, i, d, vp, i, d, d, d, i, i, vp, vp]
    fake = vp(64)  # never dereferenced: every call below fails its checks first
    cases = [
        lambda: lib.nep_hnemd_kappa(None, 5, 1.0, fake, None),
        lambda: lib.nep_hnemd_kappa(fake, 0, 1.0, fake, None),
        lambda: lib.nep_hnemd_kappa(fake, 5, 1.0, None, None),
        lambda: lib.nep_shc_quantum(None, 4, 1.0, fake, None),
        lambda: lib.nep_shc_quantum(fake, 0, 1.0, fake, None),
        lambda: lib.nep_shc_quantum(fake, 4, math.nan, fake, None),
        lambda: lib.nep_shc_quantum(fake, 4, math.inf, fake, None),
        lambda: lib.nep_shc_spectrum(fake, 0, 1.0, 3, fake, 1.0, 0, fake, None),
        lambda: lib.nep_shc_spectrum(fake, 8, 0.0, 3, fake, 1.0, 0, fake, None),
        lambda: lib.nep_hnemd_kappa_si(fake, 5, 0.0, 1.0, 1.0, fake, None),
        lambda: lib.nep_hnemd_kappa_si(fake, 5, 300.0, -1.0, 1.0, fake, None),
        lambda: lib.nep_hnemd_kappa_si(fake, 5, 300.0, 1.0, 0.0, fake, None),
        lambda: lib.nep_hnemd_kappa_si(fake, 5, 300.0, 1.0, math.inf, fake, None),
        lambda: lib.nep_hnemd_kappa_si(None, 5, 300.0, 1.0, 1.0, fake, None),
        lambda: lib.nep_kappa_spectrum(fake, 8, 2.0, fake, 4, 300.0, 1.0, 0.0, 1, 0, fake, None),
        lambda: lib.nep_kappa_spectrum(fake, 8, 0.0, fake, 4, 300.0, 1.0, 1e-4, 1, 0, fake, None),
        lambda: lib.nep_kappa_spectrum(fake, 0, 2.0, fake, 4, 300.0, 1.0, 1e-4, 1, 0, fake, None),
        lambda: lib.nep_kappa_spectrum(fake, 8, 2.0, None, 4, 300.0, 1.0, 1e-4, 1, 0, fake, None),
        lambda: lib.nep_kappa_spectrum(fake, 8, 2.0, fake, 4, math.nan, 1.0, 1e-4, 1, 0, fake, None),
    ]
    for call in cases:
        assert call() == -1  # NEP_ERR_ARG
        assert lib.nep_last_error()


def test_cell_grid_stays_within_int_range_for_large_sparse_boxes():
    """The cell grid is counted in 64 bits and coarsened to at most 2^22
    cells: a 10,240 A cube with a 5 A list radius would otherwise need 2048^3
    cells, a product that wraps to 0 in 32-bit arithmetic.  Every cell edge
    stays at least the list radius (so the 27-cell stencil still holds every
    neighbour).  Host-only call: no GPU needed."""
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep as N
    import numpy as np
    cap = 1 << 22
    for L, r in [((10240.0,) * 3, 5.0), ((1e12, 50.0, 50.0), 6.0), ((3e5, 3e5, 20.0), 6.0),
                 ((135.75, 135.75, 135.75), 6.0), ((217.2, 217.2, 434.4), 6.0)]:
        nc = N.cell_grid(np.diag(L), r)
        assert all(c >= 3 for c in nc), (L, nc)
        assert int(np.prod(np.array(nc, dtype=np.int64))) <= cap, (L, nc)
        assert all(L[d] / nc[d] >= r for d in range(3)), (L, nc)
    # an uncrowded grid is left as floor(L / r_list)
    assert N.cell_grid(np.diag([135.75] * 3), 6.0) == (22, 22, 22)
    assert N.cell_grid(np.diag([217.2, 217.2, 434.4]), 6.0) == (36, 36, 72)
    # edges under three list radii use the all-pairs search
    assert N.cell_grid(np.diag([10.86] * 3), 6.0) == (0, 0, 0)
    try:
        N.cell_grid(np.diag([10.0, 10.0, 10.0]), float("nan"))
        raise AssertionError("expected NEP_ERR_ARG")
    except N.NepError as e:
        assert e.code == -1


def test_status_decoding_of_device_error_bits():
    """The device-side error bits map to status codes on the host, including
    the timeout bit that the tensor-core kernel latches when a bounded wait
    gives up (that path is never forced on a GPU; its decoding is checked
    here).  Priority: overflow, asymmetric list, non-finite, timeout."""
    import ctypes as C

    from paper_2107_08119_gb300 import build
    build.build()
    lib = C.CDLL(build.LIB)
    lib.nep_status_from_bits.argtypes = [C.c_uint]
    lib.nep_last_error.restype = C.c_char_p
    OK, OVERFLOW, NONFINITE, TIMEOUT = 0, -4, -5, -6
    cases = {0: OK, 1: OVERFLOW, 4: OVERFLOW, 2: NONFINITE, 8: TIMEOUT, 1 | 8: OVERFLOW, 2 | 8: NONFINITE,
             4 | 2: OVERFLOW, 16: OK}
    for bits, want in cases.items():
        assert lib.nep_status_from_bits(bits) == want, bits
        if want != OK:
            assert lib.nep_last_error()
    assert b"timed out" in (lib.nep_status_from_bits(8), lib.nep_last_error())[1]
