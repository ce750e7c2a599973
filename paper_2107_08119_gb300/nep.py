"""Python binding of libnep.so (the C ABI in include/nep.h).

Argument marshalling only: every step of the NEP path runs in the library's
CUDA kernels.  PyTorch provides device memory (output tensors) and the
current CUDA stream.  There is no CPU fallback: importing this module raises
if the compiled library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnep.so")

NEP_OK = 0
STATUS = {
    0: "NEP_OK", -1: "NEP_ERR_ARG", -2: "NEP_ERR_OOM", -3: "NEP_ERR_CUDA", -4: "NEP_ERR_NEIGHBOR_OVERFLOW",
    -5: "NEP_ERR_NONFINITE", -6: "NEP_ERR_TIMEOUT", -7: "NEP_ERR_BOX", -8: "NEP_ERR_UNSUPPORTED",
}
THERMO_COLS = 8
LOSS_COLS = 6
PREC_FP32, PREC_BF16 = 0, 1


class NepError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


class _Hyper(C.Structure):
    _fields_ = [("n_max_R", C.c_int), ("n_max_A", C.c_int), ("l_max", C.c_int), ("n_neu", C.c_int),
                ("rc_R", C.c_double), ("rc_A", C.c_double), ("skin", C.c_double), ("max_neighbors", C.c_int)]


_vp = C.c_void_p
_SIGNATURES = {
    "nep_create": (C.c_int, [C.POINTER(_Hyper), _vp, C.c_int, C.POINTER(_vp)]),
    "nep_set_parameters": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "nep_destroy": (C.c_int, [_vp]),
    "nep_compute_efv": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nep_compute_efv_plain": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nep_sync_status": (C.c_int, [_vp, _vp]),
    "nep_heat_current": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp]),
    "nep_get_neighbors": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "nep_cell_grid": (C.c_int, [_vp, C.c_double, _vp]),
    "nep_status_from_bits": (C.c_int, [C.c_uint]),
    "nep_md_create": (C.c_int, [_vp, C.c_int, _vp, C.c_double, C.POINTER(_vp)]),
    "nep_md_destroy": (C.c_int, [_vp]),
    "nep_md_step": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, _vp, _vp, _vp]),
    "nep_md_invalidate": (C.c_int, [_vp]),
    "nep_md_set_thermostat": (C.c_int, [_vp, C.c_double, C.c_double]),
    "nep_md_set_hnemd": (C.c_int, [_vp, _vp]),
    "nep_md_set_force_form": (C.c_int, [_vp, C.c_int]),
    "nep_md_rebuild_count": (C.c_int, [_vp, C.POINTER(C.c_longlong), _vp]),
    "nep_md_forces": (_vp, [_vp]),
    "nep_profile_enable": (C.c_int, [_vp, C.c_int]),
    "nep_profile_read": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "nep_dataset_create": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(_vp)]),
    "nep_dataset_destroy": (C.c_int, [_vp]),
    "nep_dataset_info": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "nep_dataset_descriptors": (C.c_int, [_vp, _vp, _vp]),
    "nep_dataset_counts": (C.c_int, [_vp, _vp]),
    "snes_evaluate_population": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp]),
    "nep_force_loss": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "nep_force_loss_backward": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "snes_create": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_ulonglong, C.POINTER(_vp)]),
    "snes_destroy": (C.c_int, [_vp]),
    "snes_step": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp, _vp]),
    "snes_get_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "snes_run": (C.c_int, [_vp, _vp, C.c_int, _vp, C.c_int, _vp, _vp]),
    "nep_md_set_shc": (C.c_int, [_vp, C.c_int, C.c_int]),
    "nep_set_species": (C.c_int, [_vp, C.c_int, _vp]),
    "nep_dataset_create_species": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(_vp)]),
    "nep_md_get_shc": (C.c_int, [_vp, _vp, C.POINTER(C.c_longlong), _vp]),
    "nep_shc_spectrum": (C.c_int, [_vp, C.c_int, C.c_double, C.c_int, _vp, C.c_double, C.c_int, _vp, _vp]),
    "nep_shc_quantum": (C.c_int, [_vp, C.c_int, C.c_double, _vp, _vp]),
    "nep_hnemd_kappa": (C.c_int, [_vp, C.c_int, C.c_double, _vp, _vp]),
    "nep_hnemd_kappa_si": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double, C.c_double, _vp, _vp]),
    "nep_kappa_spectrum": (C.c_int, [_vp, C.c_int, C.c_double, _vp, C.c_int, C.c_double, C.c_double, C.c_double,
                                     C.c_int, C.c_int, _vp, _vp]),
    "nep_dataset_set_shape": (C.c_int, [_vp, _vp]),
    "nep_dataset_get_shape": (C.c_int, [_vp, _vp]),
    "nep_dataset_tune": (C.c_int, [_vp, _vp, C.c_int, C.c_int, C.c_int, _vp, C.POINTER(C.c_float), _vp]),
    "nep_compute_efv_static": (C.c_int, [C.POINTER(_Hyper), _vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                                         _vp, _vp, _vp]),
    "nep_tc_selftest": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp]),
    "nep_last_error": (C.c_char_p, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libnep.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def exported_symbols():
    return list(_SIGNATURES)


def _check(code: int, where: str):
    if code != NEP_OK:
        raise NepError(code, where, _lib.nep_last_error().decode())


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _box9(box):
    b = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(9))
    return b, b.ctypes.data_as(_vp)


def _soa_f64(t, n=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.dim() == 2
            and t.shape[0] == 3 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float64 tensor of shape (3, n)")
    if n is not None and t.shape[1] != n:
        raise ValueError(f"expected {n} atoms, got {t.shape[1]}")
    return t


@dataclass(frozen=True)
class Hyper:
    n_max_R: int = 7
    n_max_A: int = 5
    l_max: int = 4
    n_neu: int = 30
    rc_R: float = 5.0
    rc_A: float = 4.0
    skin: float = 1.0
    max_neighbors: int = 96

    @property
    def n_des(self) -> int:
        return (self.n_max_R + 1) + (self.n_max_A + 1) * self.l_max

    @property
    def n_par(self) -> int:
        return (self.n_des + 2) * self.n_neu + 1

    def c(self) -> _Hyper:
        return _Hyper(self.n_max_R, self.n_max_A, self.l_max, self.n_neu, self.rc_R, self.rc_A, self.skin,
                      self.max_neighbors)


class NEP:
    """A NEP model on the GPU (handle of nep_create)."""

    def __init__(self, z, hyper: Hyper = Hyper()):
        self.hyper = hyper
        zf = np.ascontiguousarray(np.asarray(z, dtype=np.float32).reshape(-1))
        h = hyper.c()
        out = _vp()
        _check(_lib.nep_create(C.byref(h), zf.ctypes.data_as(_vp), zf.size, C.byref(out)), "nep_create")
        self._h = out

    def close(self):
        if getattr(self, "_h", None):
            _lib.nep_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_parameters(self, z, stream=None):
        zf = np.ascontiguousarray(np.asarray(z, dtype=np.float32).reshape(-1))
        _check(_lib.nep_set_parameters(self._h, zf.ctypes.data_as(_vp), zf.size, _stream(stream)),
               "nep_set_parameters")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def compute(self, pos, box, *, e_total=True, e_atom=True, force=True, virial_atom=True, virial_total=True,
                sync=True, stream=None, plain=False):
        """pos: CUDA float64 (3, n).  Returns a dict of device tensors.
        plain=True runs nep_compute_efv_plain (the plain FP32 comparator)."""
        pos = _soa_f64(pos)
        n = pos.shape[1]
        dev = pos.device
        out = {
            "e_total": torch.empty(1, dtype=torch.float64, device=dev) if e_total else None,
            "e_atom": torch.empty(n, dtype=torch.float64, device=dev) if e_atom else None,
            "force": torch.empty(3, n, dtype=torch.float32, device=dev) if force else None,
            "virial_atom": torch.empty(9, n, dtype=torch.float32, device=dev) if virial_atom else None,
            "virial_total": torch.empty(9, dtype=torch.float64, device=dev) if virial_total else None,
        }
        b, bp = _box9(box)
        fn, name = ((_lib.nep_compute_efv_plain, "nep_compute_efv_plain") if plain
                    else (_lib.nep_compute_efv, "nep_compute_efv"))
        _check(fn(self._h, n, bp, _ptr(pos), _ptr(out["e_total"]), _ptr(out["e_atom"]), _ptr(out["force"]),
                  _ptr(out["virial_atom"]), _ptr(out["virial_total"]), _stream(stream)), name)
        if sync:
            self.sync_status(stream)
        return {k: v for k, v in out.items() if v is not None}

    def sync_status(self, stream=None):
        _check(_lib.nep_sync_status(self._h, _stream(stream)), "nep_sync_status")

    def neighbors(self, n: int, stream=None):
        """(count[n], nbr[max_neighbors, n]) of the last compute() call."""
        dev = torch.device("cuda")
        cnt = torch.empty(n, dtype=torch.int32, device=dev)
        nbr = torch.empty(self.hyper.max_neighbors, n, dtype=torch.int32, device=dev)
        _check(_lib.nep_get_neighbors(self._h, n, _ptr(cnt), _ptr(nbr), _stream(stream)), "nep_get_neighbors")
        return cnt, nbr

    def set_species(self, z_atom=None):
        """Per-atom species numbers (atomic numbers) for the multicomponent
        weighting f_c -> f_c sqrt(Z_i Z_j); None: one species."""
        if z_atom is None:
            _check(_lib.nep_set_species(self._h, 0, None), "nep_set_species")
            return
        zs = _host(z_atom, np.float64, (-1,))
        _check(_lib.nep_set_species(self._h, zs.size, zs.ctypes.data_as(_vp)), "nep_set_species")

    def profile(self, on: bool = True):
        _check(_lib.nep_profile_enable(self._h, 1 if on else 0), "nep_profile_enable")

    def profile_read(self):
        """Summed ms and bracket counts per phase since the last read:
        {"site": (ms, n), "assemble": ..., "neighbor": ..., "step": ...}."""
        ms = (C.c_double * 4)()
        cnt = (C.c_longlong * 4)()
        _check(_lib.nep_profile_read(self._h, ms, cnt), "nep_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(("site", "assemble", "neighbor", "step"))}

    def heat_current(self, virial_atom, vel, stream=None):
        vel = _soa_f64(vel)
        n = vel.shape[1]
        if not (virial_atom.is_cuda and virial_atom.dtype == torch.float32 and tuple(virial_atom.shape) == (9, n)
                and virial_atom.is_contiguous()):
            raise ValueError("virial_atom must be a contiguous CUDA float32 tensor of shape (9, n)")
        J = torch.empty(3, dtype=torch.float64, device=vel.device)
        _check(_lib.nep_heat_current(self._h, n, _ptr(virial_atom), _ptr(vel), _ptr(J), _stream(stream)),
               "nep_heat_current")
        return J


def tc_selftest(A, B, stream=None):
    """D = A B^T through the library's tcgen05 BF16 path (A: 128 x 32, B: N x 32,
    CUDA bfloat16).  Returns (D, error bits)."""
    if not (A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.is_cuda and B.is_cuda
            and tuple(A.shape) == (128, 32) and B.dim() == 2 and B.shape[1] == 32):
        raise ValueError("A must be CUDA bf16 (128, 32) and B CUDA bf16 (N, 32)")
    A = A.contiguous()
    B = B.contiguous()
    D = torch.empty(128, B.shape[0], dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(_lib.nep_tc_selftest(_ptr(A), _ptr(B), B.shape[0], _ptr(D), _ptr(err), _stream(stream)), "nep_tc_selftest")
    return D, err


STATIC_MAX_ATOMS = 4096
STATIC_MAX_NEIGHBORS = 96


def cell_grid(box, r_list: float):
    """Cells per direction of the neighbour-list build for `box` and list
    radius `r_list` (host only; (0, 0, 0) means the all-pairs search)."""
    nc = (C.c_int * 3)()
    _, bp = _box9(box)
    _check(_lib.nep_cell_grid(bp, float(r_list), nc), "nep_cell_grid")
    return tuple(nc)


def compute_efv_static(z_dev, pos, box, hyper: Hyper = Hyper(max_neighbors=STATIC_MAX_NEIGHBORS), stream=None):
    """nep_compute_efv_static: the force path without any device allocation
    inside the call (scratch in a fixed-size array in the library).  z_dev is
    a CUDA float32 tensor of the n_par parameters.  Output tensors are
    allocated here by PyTorch, as the caller's memory.  Returns a dict of
    device tensors including "err" (device-side error bits)."""
    pos = _soa_f64(pos)
    n = pos.shape[1]
    dev = pos.device
    out = {"e_total": torch.empty(1, dtype=torch.float64, device=dev),
           "e_atom": torch.empty(n, dtype=torch.float64, device=dev),
           "force": torch.empty(3, n, dtype=torch.float32, device=dev),
           "virial_atom": torch.empty(9, n, dtype=torch.float32, device=dev),
           "virial_total": torch.empty(9, dtype=torch.float64, device=dev),
           "err": torch.empty(1, dtype=torch.int32, device=dev)}
    b, bp = _box9(box)
    h = hyper.c()
    _check(_lib.nep_compute_efv_static(C.byref(h), _ptr(z_dev), int(z_dev.numel()), n, bp, _ptr(pos),
                                       _ptr(out["e_total"]), _ptr(out["e_atom"]), _ptr(out["force"]),
                                       _ptr(out["virial_atom"]), _ptr(out["virial_total"]), _ptr(out["err"]),
                                       _stream(stream)), "nep_compute_efv_static")
    return out


class MD:
    """Velocity-Verlet integrator on a NEP model (handle of nep_md_create):
    NVE, optionally with a Berendsen thermostat and HNEMD driving."""

    def __init__(self, model: NEP, n: int, box, mass: float):
        self.model = model
        self.n = n
        b, bp = _box9(box)
        out = _vp()
        _check(_lib.nep_md_create(model._h, n, bp, float(mass), C.byref(out)), "nep_md_create")
        self._h = out
        self._shc_lags = 0

    def close(self):
        if getattr(self, "_h", None):
            _lib.nep_md_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, pos, vel, n_steps: int, dt: float, thermo=None, heat=None, stream=None):
        """Advance in place.  thermo: CUDA float64 (n_steps, 8) or None;
        heat: CUDA float64 (n_steps, 3) or None."""
        pos = _soa_f64(pos, self.n)
        vel = _soa_f64(vel, self.n)
        for t, cols in ((thermo, THERMO_COLS), (heat, 3)):
            if t is not None and not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                                      and t.numel() >= n_steps * cols):
                raise ValueError("thermo/heat buffers must be contiguous CUDA float64 with room for every step")
        _check(_lib.nep_md_step(self._h, _ptr(pos), _ptr(vel), int(n_steps), float(dt), _ptr(thermo), _ptr(heat),
                                _stream(stream)), "nep_md_step")

    def invalidate(self):
        _check(_lib.nep_md_invalidate(self._h), "nep_md_invalidate")

    def set_thermostat(self, t0: float, tau: float):
        """Berendsen rescaling towards t0 K with coupling time tau fs (tau <= 0: off)."""
        _check(_lib.nep_md_set_thermostat(self._h, float(t0), float(tau)), "nep_md_set_thermostat")

    def set_force_form(self, plain: bool):
        """Force pass of the MD steps: the optimised form (False) or the plain
        FP32 comparator (True, literal O(M^2) Eq. 13, unfused)."""
        _check(_lib.nep_md_set_force_form(self._h, 1 if plain else 0), "nep_md_set_force_form")

    def set_hnemd(self, fe):
        """HNEMD driving force parameter F_e (1/A, three values), or None: off."""
        arr = None if fe is None else _host(fe, np.float64, (3,))
        _check(_lib.nep_md_set_hnemd(self._h, None if arr is None else arr.ctypes.data_as(_vp)),
               "nep_md_set_hnemd")

    def set_shc(self, n_lags: int, every: int = 1):
        """Accumulate the virial-velocity correlation K(t) over n_lags lags,
        sampling every `every` steps (0 lags: off).  Resets the sums."""
        _check(_lib.nep_md_set_shc(self._h, int(n_lags), int(every)), "nep_md_set_shc")
        self._shc_lags = int(n_lags)

    def shc(self, stream=None):
        """(K, n_samples): K a CUDA float64 (n_lags, 3) tensor, the correlation
        averaged over its time origins (eV A/fs)."""
        K = torch.empty(self._shc_lags, 3, dtype=torch.float64, device="cuda")
        ns = C.c_longlong()
        _check(_lib.nep_md_get_shc(self._h, _ptr(K), C.byref(ns), _stream(stream)), "nep_md_get_shc")
        return K, ns.value

    def rebuild_count(self, stream=None) -> int:
        c = C.c_longlong()
        _check(_lib.nep_md_rebuild_count(self._h, C.byref(c), _stream(stream)), "nep_md_rebuild_count")
        return c.value

    def sync_status(self, stream=None):
        self.model.sync_status(stream)


def _host(a, dtype, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if shape is not None:
        a = a.reshape(shape)
    return a


class Dataset:
    """A training set on the device (handle of nep_dataset_create).
    structures: list of {"pos": (n, 3), "box": (3, 3)}; e_tar per structure,
    f_tar (N, 3) concatenated, w_tar (n_struct, 6) in the order xx yy zz xy yz zx."""

    def __init__(self, model: NEP, structures, e_tar, f_tar, w_tar, species=None):
        """species: per-atom species numbers of the concatenated structures
        (multicomponent weighting), or None for one species."""
        self.model = model
        n_atoms = _host([len(s["pos"]) for s in structures], np.int32)
        boxes = _host(np.stack([np.asarray(s["box"], np.float64).reshape(3, 3) for s in structures]), np.float64)
        pos = _host(np.concatenate([np.asarray(s["pos"], np.float64).reshape(-1, 3) for s in structures]),
                    np.float64)
        e = _host(e_tar, np.float64)
        f = _host(f_tar, np.float64, (-1, 3))
        w = _host(w_tar, np.float64, (-1, 6))
        out = _vp()
        zs = None if species is None else _host(species, np.float64, (-1,))
        _check(_lib.nep_dataset_create_species(model._h, len(structures), n_atoms.ctypes.data_as(_vp),
                                               boxes.ctypes.data_as(_vp), pos.ctypes.data_as(_vp),
                                               None if zs is None else zs.ctypes.data_as(_vp), e.ctypes.data_as(_vp),
                                               f.ctypes.data_as(_vp), w.ctypes.data_as(_vp), C.byref(out)),
               "nep_dataset_create")
        self._h = out
        self.n_struct = len(structures)
        self._default_shape = self.shape()

    def close(self):
        if getattr(self, "_h", None):
            _lib.nep_dataset_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        na, npairs, nb = C.c_int(), C.c_longlong(), C.c_longlong()
        _check(_lib.nep_dataset_info(self._h, C.byref(na), C.byref(npairs), C.byref(nb)), "nep_dataset_info")
        return {"atoms": na.value, "pairs": npairs.value, "device_bytes": nb.value}

    def counts(self):
        """atoms, pairs, angular pairs, structures, atoms of the largest structure"""
        a = np.zeros(5, np.int64)
        _check(_lib.nep_dataset_counts(self._h, a.ctypes.data_as(_vp)), "nep_dataset_counts")
        return dict(zip(("atoms", "pairs", "angular_pairs", "structures", "largest_structure"), (int(v) for v in a)))

    def descriptors(self, stream=None):
        n = self.info()["atoms"]
        q = torch.empty(n, self.model.hyper.n_des, dtype=torch.float32, device="cuda")
        _check(_lib.nep_dataset_descriptors(self._h, _ptr(q), _stream(stream)), "nep_dataset_descriptors")
        return q

    SHAPE_KEYS = ("waves", "owner_warps", "discard", "mlp_threads", "recv_unroll", "fused", "owner_tc", "pop_pipe")

    def shape(self):
        """Launch shape of the population evaluation (nep_dataset_get_shape)."""
        a = np.zeros(len(self.SHAPE_KEYS), np.int32)
        _check(_lib.nep_dataset_get_shape(self._h, a.ctypes.data_as(_vp)), "nep_dataset_get_shape")
        return dict(zip(self.SHAPE_KEYS, (int(v) for v in a)))

    def set_shape(self, **shape):
        """Set the launch shape; keys not given take the dataset's default
        (the shape it had when created)."""
        bad = set(shape) - set(self.SHAPE_KEYS)
        if bad:
            raise ValueError(f"unknown shape keys {sorted(bad)}")
        full = dict(self._default_shape, **shape)
        a = np.asarray([full[k] for k in self.SHAPE_KEYS], np.int32)
        _check(_lib.nep_dataset_set_shape(self._h, a.ctypes.data_as(_vp)), "nep_dataset_set_shape")

    def default_shape(self):
        return dict(self._default_shape)

    def tune(self, n_pop, precision=PREC_FP32, reps=5, stream=None):
        """Autotune the launch shape (nep_dataset_tune); returns (shape, ms per evaluation)."""
        a = np.zeros(len(self.SHAPE_KEYS), np.int32)
        ms = C.c_float()
        _check(_lib.nep_dataset_tune(self.model._h, self._h, int(n_pop), int(precision), int(reps),
                                     a.ctypes.data_as(_vp), C.byref(ms), _stream(stream)), "nep_dataset_tune")
        return dict(zip(self.SHAPE_KEYS, (int(v) for v in a))), ms.value

    def evaluate(self, z_pop, precision=PREC_FP32, lambdas=None, stream=None):
        """z_pop: CUDA float32 (n_pop, n_par).  Returns CUDA float64 (n_pop, 6)."""
        if not (z_pop.is_cuda and z_pop.dtype == torch.float32 and z_pop.is_contiguous() and z_pop.dim() == 2):
            raise ValueError("z_pop must be a contiguous CUDA float32 (n_pop, n_par) tensor")
        loss = torch.empty(z_pop.shape[0], LOSS_COLS, dtype=torch.float64, device=z_pop.device)
        lam = None if lambdas is None else _host(lambdas, np.float64, (5,))
        _check(_lib.snes_evaluate_population(self.model._h, self._h, _ptr(z_pop), z_pop.shape[0], int(precision),
                                             None if lam is None else lam.ctypes.data_as(_vp), _ptr(loss),
                                             _stream(stream)), "snes_evaluate_population")
        return loss

    def force_loss(self, z, stream=None):
        """L_f of Eq. 30 for one parameter vector (CUDA float32 (n_par,)).
        Returns a CUDA float64 (1,) tensor; the dataset keeps what
        force_loss_backward needs."""
        z = _param_vector(z, self.model.hyper.n_par)
        out = torch.empty(1, dtype=torch.float64, device=z.device)
        _check(_lib.nep_force_loss(self.model._h, self._h, _ptr(z), _ptr(out), _stream(stream)), "nep_force_loss")
        return out

    def force_loss_backward(self, seed=None, stream=None):
        """seed * dL_f/dz at the z of the last force_loss (CUDA float64 (n_par,));
        seed: CUDA float64 scalar tensor or None for 1."""
        grad = torch.empty(self.model.hyper.n_par, dtype=torch.float64, device="cuda")
        if seed is not None:
            seed = seed.detach().to(device="cuda", dtype=torch.float64).reshape(1).contiguous()
        _check(_lib.nep_force_loss_backward(self.model._h, self._h, None if seed is None else _ptr(seed), _ptr(grad),
                                            _stream(stream)), "nep_force_loss_backward")
        return grad


def _param_vector(z, n_par):
    if not (z.is_cuda and z.dtype == torch.float32 and z.is_contiguous() and z.numel() == n_par):
        raise ValueError(f"z must be a contiguous CUDA float32 tensor of {n_par} parameters")
    return z


class ForceLoss(torch.autograd.Function):
    """Differentiable L_f(z) on a training set: forward = nep_force_loss,
    backward = nep_force_loss_backward (hand-written adjoint, descriptors
    recomputed).  Use as ForceLoss.apply(z, dataset); z is CUDA float32.
    The dataset holds the state of its latest forward, so run each backward
    before the next forward on the same dataset."""

    @staticmethod
    def forward(ctx, z, dataset):
        ctx.dataset = dataset
        return dataset.force_loss(z.detach().contiguous()).reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.dataset.force_loss_backward(seed=grad_out)
        return g.to(torch.float32), None


def force_loss(z, dataset):
    """L_f(z) on `dataset` as a differentiable torch scalar (float64)."""
    return ForceLoss.apply(z, dataset)


def shc_spectrum(K, dt_lag: float, omega, scale: float = 1.0, window: bool = False, stream=None):
    """The transform of Sec. II.B on the device: scale * 2 * trapezoid of
    K(t) cos(w t) over the lags (K even in t).  K: CUDA float64 (n_lags, 3);
    omega: CUDA float64 (n_omega,) in rad per unit of dt_lag."""
    if not (K.is_cuda and K.dtype == torch.float64 and K.is_contiguous() and omega.is_cuda
            and omega.dtype == torch.float64 and omega.is_contiguous()):
        raise ValueError("K and omega must be contiguous CUDA float64 tensors")
    out = torch.empty(omega.numel(), 3, dtype=torch.float64, device="cuda")
    _check(_lib.nep_shc_spectrum(_ptr(K), K.shape[0], float(dt_lag), omega.numel(), _ptr(omega), float(scale),
                                 1 if window else 0, _ptr(out), _stream(stream)), "nep_shc_spectrum")
    return out


def shc_quantum(spec, omega, x_per_omega: float, stream=None):
    """Quantum correction of Sec. IV.C on the device, in place: spec[k] *=
    x^2 e^x / (e^x - 1)^2 with x = x_per_omega * omega[k].  spec: CUDA
    float64 (n_omega, 3); omega: CUDA float64 (n_omega,).  Returns spec."""
    if not (spec.is_cuda and spec.dtype == torch.float64 and spec.is_contiguous() and omega.is_cuda
            and omega.dtype == torch.float64 and omega.is_contiguous() and spec.shape == (omega.numel(), 3)):
        raise ValueError("spec (n, 3) and omega (n,) must be contiguous CUDA float64 tensors")
    _check(_lib.nep_shc_quantum(_ptr(omega), omega.numel(), float(x_per_omega), _ptr(spec), _stream(stream)),
           "nep_shc_quantum")
    return spec


def hnemd_kappa(J, temperature: float, volume: float, fe: float, scale: float = None, stream=None):
    """Running HNEMD conductivity estimate on the device (Sec. II.B):
    kappa(t) = <J>_{0..t} / (T V F_e) in W / (m K) for J in eV A/fs (the heat
    series of MD.step), T in K, V in A^3 and the driving force fe (1/A) along
    the component of interest (nep_hnemd_kappa_si); `scale` instead gives the
    factor of nep_hnemd_kappa directly.  J: CUDA float64 (n, 3).  Returns (n, 3)."""
    if not (J.is_cuda and J.dtype == torch.float64 and J.is_contiguous() and J.dim() == 2 and J.shape[1] == 3):
        raise ValueError("J must be a contiguous CUDA float64 (n, 3) tensor")
    out = torch.empty_like(J)
    if scale is None:
        _check(_lib.nep_hnemd_kappa_si(_ptr(J), J.shape[0], float(temperature), float(volume), float(fe), _ptr(out),
                                       _stream(stream)), "nep_hnemd_kappa_si")
    else:
        _check(_lib.nep_hnemd_kappa(_ptr(J), J.shape[0], float(scale), _ptr(out), _stream(stream)),
               "nep_hnemd_kappa")
    return out


def kappa_spectrum(K, dt_lag_fs: float, nu_thz, temperature: float, volume: float, fe: float, window: bool = True,
                   quantum: bool = False, stream=None):
    """Spectral thermal conductivity kappa(nu) in W / (m K THz) at frequencies
    nu (THz, CUDA float64) from K in eV A/fs at lags dt_lag_fs apart, for a
    driving force fe (1/A) along the direction of interest, temperature (K)
    and volume (A^3) (nep_kappa_spectrum): kappa(w) = (2 / (T V F_e)) int K
    e^{iwt} dt, with int kappa(nu) dnu the HNEMD conductivity.  quantum=True
    applies the correction factor of Sec. IV.C at that temperature."""
    if not (K.is_cuda and K.dtype == torch.float64 and K.is_contiguous() and nu_thz.is_cuda
            and nu_thz.dtype == torch.float64 and nu_thz.is_contiguous()):
        raise ValueError("K and nu_thz must be contiguous CUDA float64 tensors")
    out = torch.empty(nu_thz.numel(), 3, dtype=torch.float64, device="cuda")
    _check(_lib.nep_kappa_spectrum(_ptr(K), K.shape[0], float(dt_lag_fs), _ptr(nu_thz), nu_thz.numel(),
                                   float(temperature), float(volume), float(fe), 1 if window else 0,
                                   1 if quantum else 0, _ptr(out), _stream(stream)), "nep_kappa_spectrum")
    return out


class SNES:
    """Separable natural evolution strategy on the device (handle of snes_create)."""

    def __init__(self, model: NEP, n_pop: int, mean0, sigma0, seed: int):
        self.model = model
        self.n_pop = n_pop
        m0 = _host(mean0, np.float32, (-1,))
        s0 = _host(sigma0, np.float32, (-1,))
        out = _vp()
        _check(_lib.snes_create(model._h, n_pop, m0.ctypes.data_as(_vp), s0.ctypes.data_as(_vp), int(seed),
                                C.byref(out)), "snes_create")
        self._h = out

    def close(self):
        if getattr(self, "_h", None):
            _lib.snes_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, ds: Dataset, precision=PREC_FP32, lambdas=None, r=None, loss=None, stream=None):
        lam = None if lambdas is None else _host(lambdas, np.float64, (5,))
        _check(_lib.snes_step(self._h, ds._h, int(precision), None if lam is None else lam.ctypes.data_as(_vp),
                              _ptr(r), _ptr(loss), _stream(stream)), "snes_step")

    def run(self, ds: Dataset, n_gen: int, precision=PREC_FP32, lambdas=None, history=False, stream=None):
        """n_gen generations replayed from a captured CUDA graph (snes_run).
        Returns the CUDA float64 (n_gen, n_pop, 6) loss history, or None."""
        lam = None if lambdas is None else _host(lambdas, np.float64, (5,))
        hist = (torch.empty(max(n_gen, 1), self.n_pop, LOSS_COLS, dtype=torch.float64, device="cuda")
                if history else None)
        _check(_lib.snes_run(self._h, ds._h, int(precision), None if lam is None else lam.ctypes.data_as(_vp),
                             int(n_gen), _ptr(hist), _stream(stream)), "snes_run")
        return None if hist is None else hist[:n_gen]

    def state(self, stream=None):
        npar = self.model.hyper.n_par
        m = torch.empty(npar, dtype=torch.float32, device="cuda")
        s = torch.empty(npar, dtype=torch.float32, device="cuda")
        r = torch.empty(self.n_pop, npar, dtype=torch.float32, device="cuda")
        order = torch.empty(self.n_pop, dtype=torch.int32, device="cuda")
        _check(_lib.snes_get_state(self._h, _ptr(m), _ptr(s), _ptr(r), _ptr(order), _stream(stream)),
               "snes_get_state")
        return m, s, r, order
