"""ctypes binding of the FP64 CPU oracle (``nep_oracle.c``).

Test infrastructure only: used by ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg, never by the CUDA product path.

Arrays are numpy float64 in AoS layout: positions (n, 3), forces (n, 3),
per-atom virials (n, 3, 3) with W[i, a, b] = sum_j r_ij^a (dU_j/dr_ji)^b
(Eq. 6 of the paper), boxes (3, 3) with rows = lattice vectors.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nep_oracle.c")
# NEP_ORACLE_LIB names a prebuilt copy of the library to load instead (the
# planted-mistake test compiles altered copies and runs the pins on them)
_PREBUILT = os.environ.get("NEP_ORACLE_LIB")
_LIB_PATH = _PREBUILT or os.path.join(_HERE, "liboracle.so")
GCC_FLAGS = ["-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, strict IEEE: no fast-math)."""
    if _PREBUILT:
        return _LIB_PATH
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "nep_oracle.h")))
        if force or stale:
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            cmd = ["gcc"] + GCC_FLAGS + [_SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Hyper(C.Structure):
    _fields_ = [("n_max_R", C.c_int), ("n_max_A", C.c_int), ("l_max", C.c_int), ("n_neu", C.c_int),
                ("rc_R", C.c_double), ("rc_A", C.c_double)]


@dataclass(frozen=True)
class NepHyper:
    """Descriptor and network sizes (Table I of the paper names these)."""
    n_max_R: int = 7
    n_max_A: int = 5
    l_max: int = 4
    n_neu: int = 30
    rc_R: float = 5.0
    rc_A: float = 4.0

    def c(self) -> Hyper:
        return Hyper(self.n_max_R, self.n_max_A, self.l_max, self.n_neu, self.rc_R, self.rc_A)


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_U32 = C.POINTER(C.c_uint32)
_H = C.POINTER(Hyper)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB_PATH)
        sig = {
            "orc_n_des": (C.c_int, [_H]),
            "orc_n_par": (C.c_int, [_H]),
            "orc_chebyshev": (None, [C.c_double, C.c_int, _D, _D]),
            "orc_cutoff": (C.c_double, [C.c_double, C.c_double, _D]),
            "orc_radial": (None, [C.c_double, C.c_double, C.c_int, _D, _D]),
            "orc_legendre": (C.c_double, [C.c_int, C.c_double, _D]),
            "orc_neighbors": (C.c_int, [C.c_int, _D, _D, C.c_double, C.c_int, C.c_int, _I, _I, _D]),
            "orc_descriptors": (C.c_int, [_H, C.c_int, _D, _D, _D]),
            "orc_efv": (C.c_int, [_H, _D, C.c_int, _D, _D, _D, _D, _D]),
            "orc_efv_brute": (C.c_int, [_H, _D, C.c_int, _D, _D, _D, _D, _D]),
            "orc_site": (C.c_int, [_H, _D, C.c_int, _D, _D, _D, _D, _D]),
            "orc_efv_sample": (C.c_int, [_H, _D, C.c_int, _D, _D, C.c_int, _I, _D, _D, _D]),
            "orc_heat_current": (None, [C.c_int, _D, _D, _D]),
            "orc_md": (C.c_int, [_H, _D, C.c_int, _D, _D, _D, C.c_double, C.c_double, C.c_int, _D, _D]),
            "orc_md_ext": (C.c_int, [_H, _D, C.c_int, _D, _D, _D, C.c_double, C.c_double, C.c_int, C.c_double,
                                     C.c_double, _D, _D, _D]),
            "orc_md_record": (C.c_int, [_H, _D, C.c_int, _D, _D, _D, C.c_double, C.c_double, C.c_int,
                                        C.c_double, C.c_double, _D, _D, _D, _D, _D, _D]),
            "orc_descriptors_z": (C.c_int, [_H, C.c_int, _D, _D, _D, _D]),
            "orc_efv_z": (C.c_int, [_H, _D, C.c_int, _D, _D, _D, _D, _D, _D]),
            "orc_loss_z": (C.c_int, [_H, _D, C.c_int, _I, _D, _D, _D, _D, _D, _D, _D, _D]),
            "orc_force_loss_grad_z": (C.c_int, [_H, _D, C.c_int, _I, _D, _D, _D, _D, _D, _D]),
            "orc_shc": (None, [C.c_int, C.c_int, C.c_int, _D, _D, _D]),
            "orc_shc_spectrum": (None, [C.c_int, _D, C.c_double, C.c_int, _D, C.c_double, C.c_int, _D]),
            "orc_shc_quantum": (None, [C.c_int, _D, C.c_double, _D]),
            "orc_hnemd_kappa": (None, [C.c_int, _D, C.c_double, _D]),
            "orc_loss": (C.c_int, [_H, _D, C.c_int, _I, _D, _D, _D, _D, _D, _D, _D]),
            "orc_force_loss_grad": (C.c_int, [_H, _D, C.c_int, _I, _D, _D, _D, _D, _D]),
            "orc_snes_utilities": (None, [C.c_int, _D]),
            "orc_snes_eta_s": (C.c_double, [C.c_int]),
            "orc_snes_update": (C.c_int, [C.c_int, C.c_int, _D, _D, _D, _D, C.c_double, C.c_double, _I]),
            "orc_philox4x32_10": (None, [_U32, _U32, _U32]),
            "orc_gaussian": (None, [C.c_uint64, C.c_uint32, C.c_long, _D]),
            "orc_num_threads": (C.c_int, []),
            "orc_set_num_threads": (None, [C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(code, what):
    if code != 0:
        raise RuntimeError(f"oracle {what} failed with status {code}")


def n_des(h: NepHyper) -> int:
    return _load().orc_n_des(C.byref(h.c()))


def n_par(h: NepHyper) -> int:
    return _load().orc_n_par(C.byref(h.c()))


def chebyshev(x: float, n: int):
    T = np.zeros(n + 1)
    U = np.zeros(n + 1)
    _load().orc_chebyshev(float(x), n, _d(T), _d(U))
    return T, U


def cutoff(r: float, rc: float):
    d = C.c_double()
    f = _load().orc_cutoff(float(r), float(rc), C.byref(d))
    return f, d.value


def radial(r: float, rc: float, nmax: int):
    g = np.zeros(nmax + 1)
    dg = np.zeros(nmax + 1)
    _load().orc_radial(float(r), float(rc), nmax, _d(g), _d(dg))
    return g, dg


def legendre(l: int, t: float):
    d = C.c_double()
    p = _load().orc_legendre(l, float(t), C.byref(d))
    return p, d.value


def neighbors(pos, box, rc: float, method: int = 2, cap: int = 512):
    """Per-atom neighbour lists: (count[n], j[n, cap], r_ij[n, cap, 3]).
    method 0 = brute force over images, 1/2 = cell list."""
    pos = _f64(pos, (-1, 3))
    box = _f64(box, (3, 3))
    n = pos.shape[0]
    cnt = np.zeros(n, dtype=np.int32)
    js = np.zeros((n, cap), dtype=np.int32)
    rs = np.zeros((n, cap, 3))
    code = _load().orc_neighbors(n, _d(box), _d(pos), float(rc), method, cap, cnt.ctypes.data_as(_I),
                                 js.ctypes.data_as(_I), _d(rs))
    _check(code, "neighbors")
    return cnt, js, rs


def _zat(Z, n):
    """Per-atom atomic numbers (multicomponent weighting), or None."""
    return None if Z is None else _f64(Z, (n,))


def descriptors(h: NepHyper, pos, box, Z=None):
    """q (n, N_des); Z: the atomic number of every atom (multicomponent
    weighting f_c -> f_c sqrt(Z_i Z_j)) or None for one species."""
    pos = _f64(pos, (-1, 3))
    box = _f64(box, (3, 3))
    q = np.zeros((pos.shape[0], n_des(h)))
    Za = _zat(Z, pos.shape[0])
    _check(_load().orc_descriptors_z(C.byref(h.c()), pos.shape[0], _d(box), _d(pos), _d(Za), _d(q)), "descriptors")
    return q


def efv(h: NepHyper, z, pos, box, brute: bool = False, Z=None):
    """Site energies U (n), forces F (n, 3), per-atom virials W (n, 3, 3);
    Z: per-atom atomic numbers (multicomponent weighting) or None."""
    z = _f64(z)
    assert z.size == n_par(h)
    pos = _f64(pos, (-1, 3))
    box = _f64(box, (3, 3))
    n = pos.shape[0]
    U = np.zeros(n)
    F = np.zeros((n, 3))
    W = np.zeros((n, 3, 3))
    if Z is not None:
        assert not brute
        Za = _zat(Z, n)
        _check(_load().orc_efv_z(C.byref(h.c()), _d(z), n, _d(box), _d(pos), _d(Za), _d(U), _d(F), _d(W)), "efv")
        return U, F, W
    fn = _load().orc_efv_brute if brute else _load().orc_efv
    _check(fn(C.byref(h.c()), _d(z), n, _d(box), _d(pos), _d(U), _d(F), _d(W)), "efv")
    return U, F, W


def efv_sample(h: NepHyper, z, pos, box, idx):
    """U, F, W of the atoms in idx only (same definitions as efv)."""
    z = _f64(z)
    pos = _f64(pos, (-1, 3))
    box = _f64(box, (3, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    k = idx.size
    U = np.zeros(k)
    F = np.zeros((k, 3))
    W = np.zeros((k, 3, 3))
    _check(_load().orc_efv_sample(C.byref(h.c()), _d(z), pos.shape[0], _d(box), _d(pos), k, idx.ctypes.data_as(_I),
                                  _d(U), _d(F), _d(W)), "efv_sample")
    return U, F, W


def site(h: NepHyper, z, pos, box):
    """Descriptors q (n, N_des), dU/dq G (n, N_des), hidden states x (n, n_neu)."""
    z = _f64(z)
    pos = _f64(pos, (-1, 3))
    box = _f64(box, (3, 3))
    n = pos.shape[0]
    q = np.zeros((n, n_des(h)))
    G = np.zeros((n, n_des(h)))
    x = np.zeros((n, h.n_neu))
    _check(_load().orc_site(C.byref(h.c()), _d(z), n, _d(box), _d(pos), _d(q), _d(G), _d(x)), "site")
    return q, G, x


def heat_current(W, v):
    W = _f64(W, (-1, 3, 3))
    v = _f64(v, (-1, 3))
    J = np.zeros(3)
    _load().orc_heat_current(W.shape[0], _d(W), _d(v), _d(J))
    return J


def md(h: NepHyper, z, pos, vel, box, mass: float, dt: float, n_steps: int):
    """Velocity-Verlet NVE; returns (pos, vel, thermo[n_steps, 2] = (E_pot, E_kin), J[n_steps, 3])."""
    z = _f64(z)
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    box = _f64(box, (3, 3))
    thermo = np.zeros((n_steps, 2))
    J = np.zeros((n_steps, 3))
    _check(_load().orc_md(C.byref(h.c()), _d(z), pos.shape[0], _d(box), _d(pos), _d(vel), float(mass), float(dt),
                          n_steps, _d(thermo), _d(J)), "md")
    return pos, vel, thermo, J


def md_ext(h: NepHyper, z, pos, vel, box, mass: float, dt: float, n_steps: int, t0: float = 0.0,
           tau: float = 0.0, fe=None):
    """Velocity Verlet with an optional Berendsen thermostat (target t0 K,
    coupling time tau fs; tau <= 0 off) and HNEMD driving force F_e (1/A;
    None off).  Returns (pos, vel, thermo[n_steps, 2], J[n_steps, 3]) with
    E_kin after the thermostat and J before it."""
    z = _f64(z)
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    box = _f64(box, (3, 3))
    thermo = np.zeros((n_steps, 2))
    J = np.zeros((n_steps, 3))
    fe_arr = None if fe is None else _f64(fe, (3,))
    _check(_load().orc_md_ext(C.byref(h.c()), _d(z), pos.shape[0], _d(box), _d(pos), _d(vel), float(mass),
                              float(dt), n_steps, float(t0), float(tau), None if fe_arr is None else _d(fe_arr),
                              _d(thermo), _d(J)), "md_ext")
    return pos, vel, thermo, J


def md_record(h: NepHyper, z, pos, vel, box, mass: float, dt: float, n_steps: int, t0: float = 0.0,
              tau: float = 0.0, fe=None, Z=None):
    """md_ext that also returns, per step, the per-atom virials W_i
    (n_steps, n, 3, 3) and velocities (n_steps, n, 3) from which J is taken."""
    z = _f64(z)
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    box = _f64(box, (3, 3))
    n = pos.shape[0]
    thermo = np.zeros((n_steps, 2))
    J = np.zeros((n_steps, 3))
    Wh = np.zeros((n_steps, n, 9))
    vh = np.zeros((n_steps, n, 3))
    fe_arr = None if fe is None else _f64(fe, (3,))
    _check(_load().orc_md_record(C.byref(h.c()), _d(z), n, _d(box), _d(pos), _d(vel), float(mass), float(dt),
                                 n_steps, float(t0), float(tau), None if fe_arr is None else _d(fe_arr),
                                 _d(_zat(Z, n)), _d(thermo), _d(J), _d(Wh), _d(vh)), "md_record")
    return pos, vel, thermo, J, Wh.reshape(n_steps, n, 3, 3), vh


def shc(W_hist, v_hist, n_lags: int):
    """Sums over time origins of the virial-velocity correlation,
    K_sum[tau] = sum_{s0} sum_i W_i(s0) . v_i(s0 + tau), for the samples given
    (W_hist (S, n, 3, 3), v_hist (S, n, 3)); the average is K_sum[tau] / (S - tau)."""
    W = _f64(W_hist)
    v = _f64(v_hist)
    S, n = v.shape[0], v.shape[1]
    K = np.zeros((n_lags, 3))
    _load().orc_shc(n, S, n_lags, _d(W), _d(v), _d(K))
    return K


def shc_spectrum(K, dt_s: float, omega, scale: float = 1.0, window: bool = False):
    """scale * 2 int_0^T K(t) cos(w t) dt (trapezoid, K even in t) for each
    omega; K (n_lags, 3) at lags t = tau dt_s."""
    K = _f64(K, (-1, 3))
    om = _f64(omega, (-1,))
    out = np.zeros((om.shape[0], 3))
    _load().orc_shc_spectrum(K.shape[0], _d(K), float(dt_s), om.shape[0], _d(om), float(scale), 1 if window else 0,
                             _d(out))
    return out


def shc_quantum(spec, omega, x_per_omega: float):
    """The quantum-corrected spectrum kappa(w) x^2 e^x / (e^x - 1)^2,
    x = x_per_omega * w (Sec. IV.C): spec (n_omega, 3) at the frequencies
    omega; returns a new array."""
    out = _f64(spec, (-1, 3)).copy()
    om = _f64(omega, (-1,))
    _load().orc_shc_quantum(om.shape[0], _d(om), float(x_per_omega), _d(out))
    return out


def hnemd_kappa(J, scale: float):
    """Running HNEMD conductivity estimate (Sec. II.B): scale times the mean
    of the heat current J (n, 3) over steps 0..t, for every t."""
    J = _f64(J, (-1, 3))
    out = np.zeros_like(J)
    _load().orc_hnemd_kappa(J.shape[0], _d(J), float(scale), _d(out))
    return out


def _dataset_arrays(structures):
    n_atoms = np.array([s["pos"].shape[0] for s in structures], dtype=np.int32)
    boxes = np.ascontiguousarray(np.stack([np.asarray(s["box"], np.float64).reshape(3, 3) for s in structures]))
    pos = np.ascontiguousarray(np.concatenate([np.asarray(s["pos"], np.float64).reshape(-1, 3) for s in structures]))
    return n_atoms, boxes, pos


def loss(h: NepHyper, z, structures, e_tar, f_tar, w_tar, lambdas=(1.0, 1.0, 1.0, 0.05, 0.05), Z=None):
    """(L, L_e, L_f, L_v, L_1, L_2) of Eqs. 29-34 over a list of structures
    (dicts with "pos" (n, 3) and "box" (3, 3)); e_tar per structure, f_tar
    concatenated (N, 3), w_tar (n_struct, 6) in the order xx yy zz xy yz zx."""
    z = _f64(z)
    n_atoms, boxes, pos = _dataset_arrays(structures)
    e_tar = _f64(e_tar)
    f_tar = _f64(f_tar, (-1, 3))
    w_tar = _f64(w_tar, (-1, 6))
    lam = _f64(lambdas)
    out = np.zeros(6)
    Za = _zat(Z, pos.shape[0])
    _check(_load().orc_loss_z(C.byref(h.c()), _d(z), len(structures), n_atoms.ctypes.data_as(_I), _d(boxes),
                              _d(pos), _d(Za), _d(e_tar), _d(f_tar), _d(w_tar), _d(lam), _d(out)), "loss")
    return out


def force_loss_grad(h: NepHyper, z, structures, f_tar, Z=None):
    """(dL_f/dz, L_f) by the analytic chain rule through the partial forces."""
    z = _f64(z)
    n_atoms, boxes, pos = _dataset_arrays(structures)
    f_tar = _f64(f_tar, (-1, 3))
    grad = np.zeros(z.size)
    lf = C.c_double()
    Za = _zat(Z, pos.shape[0])
    _check(_load().orc_force_loss_grad_z(C.byref(h.c()), _d(z), len(structures), n_atoms.ctypes.data_as(_I),
                                         _d(boxes), _d(pos), _d(Za), _d(f_tar), _d(grad), C.byref(lf)),
           "force_loss_grad")
    return grad, lf.value


def snes_utilities(npop: int):
    u = np.zeros(npop)
    _load().orc_snes_utilities(npop, _d(u))
    return u


def snes_eta_s(npar: int) -> float:
    return _load().orc_snes_eta_s(npar)


def snes_update(loss_values, r, m, s, eta_m: float = 1.0, eta_s: float | None = None):
    """Returns (m', s', order) after one SNES update (Eqs. 36-39)."""
    loss_values = _f64(loss_values)
    npop = loss_values.size
    r = _f64(r, (npop, -1))
    npar = r.shape[1]
    m = _f64(m).copy()
    s = _f64(s).copy()
    if eta_s is None:
        eta_s = snes_eta_s(npar)
    order = np.zeros(npop, dtype=np.int32)
    _check(_load().orc_snes_update(npar, npop, _d(loss_values), _d(r), _d(m), _d(s), float(eta_m), float(eta_s),
                                   order.ctypes.data_as(_I)), "snes_update")
    return m, s, order


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32))
    return out


def gaussian(seed: int, gen: int, count: int):
    out = np.zeros(count)
    _load().orc_gaussian(int(seed), int(gen), int(count), _d(out))
    return out


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(t: int) -> None:
    _load().orc_set_num_threads(int(t))
