"""ctypes binding of the C oracle (lb_oracle.c).  Test infrastructure only.

Array conventions: scalar fields are float64 arrays of shape (nz, ny, nx), C
order, so that the flat index is x + nx*(y + ny*z); vector fields have shape
(3, nz, ny, nx).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIB = os.path.join(_HERE, "liblb_oracle.so")
_lock = threading.Lock()
_lib = None

FORCE_NONE, FORCE_CONST, FORCE_ABC, FORCE_LINEAR = 0, 1, 2, 3

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile lb_oracle.c into liblb_oracle.so (FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-std=c99", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_create.restype = ctypes.c_void_p
            lib.orc_create.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [
                ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_int]
            lib.orc_destroy.argtypes = [ctypes.c_void_p]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_init.argtypes = [ctypes.c_void_p, _dp, _dp]
            lib.orc_init.restype = ctypes.c_int
            lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_set_density.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 4
            lib.orc_set_gravity.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double]
            lib.orc_set_phase_solver.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_weno5_face.argtypes = [_dp]
            lib.orc_weno5_face.restype = ctypes.c_double
            lib.orc_step.restype = ctypes.c_int
            lib.orc_moments.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
            lib.orc_diagnostics.argtypes = [ctypes.c_void_p, _dp]
            lib.orc_time.argtypes = [ctypes.c_void_p]
            lib.orc_time.restype = ctypes.c_longlong
            lib.orc_get_populations.argtypes = [ctypes.c_void_p, _dp, _dp]
            lib.orc_set_populations.argtypes = [ctypes.c_void_p, _dp, _dp]
            lib.orc_get_phase.argtypes = [ctypes.c_void_p, _dp]
            lib.orc_set_phase.argtypes = [ctypes.c_void_p, _dp]
            lib.orc_last_force.argtypes = [ctypes.c_void_p, _dp]
            lib.orc_lattice27.argtypes = [ctypes.POINTER(ctypes.c_int), _dp]
            lib.orc_lattice7.argtypes = [ctypes.POINTER(ctypes.c_int), _dp]
            lib.orc_gradient.argtypes = [ctypes.c_int] * 3 + [_dp, _dp]
            lib.orc_equilibrium.argtypes = [ctypes.c_double, _dp, _dp]
            lib.orc_guo_source.argtypes = [_dp, _dp, _dp]
            lib.orc_regularized_neq.argtypes = [_dp, _dp]
            lib.orc_phase_equilibrium.argtypes = [ctypes.c_double, _dp, _dp, ctypes.c_double, _dp]
            lib.orc_interface.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_dp] * 5
            lib.orc_interface.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def threads() -> int:
    return int(_load().orc_threads())


def lattice27():
    """(c, w): the oracle's D3Q27 velocities (27, 3) and weights (27,)."""
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    _load().orc_lattice27(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(w))
    return c, w


def lattice7():
    c = np.zeros((7, 3), dtype=np.int32)
    w = np.zeros(7)
    _load().orc_lattice7(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(w))
    return c, w


def gradient(psi: np.ndarray) -> np.ndarray:
    """Lattice gradient (Sec. 2.3) of a periodic field of shape (nz, ny, nx)."""
    psi = _f64(psi)
    nz, ny, nx = psi.shape
    out = np.zeros((3,) + psi.shape)
    _load().orc_gradient(nx, ny, nz, _ptr(psi), _ptr(out))
    return out


def interface(phi: np.ndarray, W: float, sigma: float):
    """(grad phi, n, kappa, F^s) of a periodic phase field, by the step's own stages."""
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    grad = np.zeros((3,) + phi.shape)
    nrm = np.zeros((3,) + phi.shape)
    kappa = np.zeros(phi.shape)
    Fs = np.zeros((3,) + phi.shape)
    rc = _load().orc_interface(nx, ny, nz, float(W), float(sigma), _ptr(phi), _ptr(grad),
                               _ptr(nrm), _ptr(kappa), _ptr(Fs))
    if rc != 0:
        raise ValueError("orc_interface rejected the parameters")
    return grad, nrm, kappa, Fs


def weno5_face(v) -> float:
    """WENO-5 face value (Jiang and Shu) from five values along the flow; the face
    lies between v[2] and v[3]."""
    a = _f64(v)
    assert a.shape == (5,)
    return float(_load().orc_weno5_face(_ptr(a)))


def equilibrium(p: float, u) -> np.ndarray:
    out = np.zeros(27)
    _load().orc_equilibrium(float(p), _ptr(_f64(u)), _ptr(out))
    return out


def guo_source(u, F) -> np.ndarray:
    out = np.zeros(27)
    _load().orc_guo_source(_ptr(_f64(u)), _ptr(_f64(F)), _ptr(out))
    return out


def regularized_neq(a2) -> np.ndarray:
    """a2 in order xx, yy, zz, xy, xz, yz."""
    out = np.zeros(27)
    _load().orc_regularized_neq(_ptr(_f64(a2)), _ptr(out))
    return out


def phase_equilibrium(phi: float, u, n, sharp: float) -> np.ndarray:
    out = np.zeros(7)
    _load().orc_phase_equilibrium(float(phi), _ptr(_f64(u)), _ptr(_f64(n)), float(sharp), _ptr(out))
    return out


class Oracle:
    """One periodic box advanced by the FP64 oracle."""

    def __init__(self, nx, ny, nz, tau, M, W, sigma, force_kind=FORCE_NONE, g=(0.0, 0.0, 0.0),
                 A_abc=0.0, kf=0.0, K_target=0.0, T_relax=100.0, regularize=True):
        self._lib = _load()
        self.shape = (int(nz), int(ny), int(nx))
        gc = _f64(g)
        h = self._lib.orc_create(int(nx), int(ny), int(nz), float(tau), float(M), float(W),
                                 float(sigma), int(force_kind), _ptr(gc), float(A_abc), float(kf),
                                 float(K_target), float(T_relax), 1 if regularize else 0)
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def N(self) -> int:
        nz, ny, nx = self.shape
        return nx * ny * nz

    def init(self, phi, u):
        phi = _f64(phi).reshape(self.shape)
        u = _f64(u).reshape((3,) + self.shape)
        if self._lib.orc_init(self._h, _ptr(phi), _ptr(u)) != 0:
            raise RuntimeError("orc_init failed")

    def set_density(self, rho_l, rho_g, tau_l, tau_g):
        """Variable density and viscosity (Sec. 2.3): rho and tau of the phi = 1 and
        phi = 0 phases, linear in phi in between."""
        if self._lib.orc_set_density(self._h, float(rho_l), float(rho_g), float(tau_l), float(tau_g)) != 0:
            raise ValueError("oracle rejected the density parameters")

    def set_phase_solver(self, solver: str):
        """"lb" (the D3Q7 model) or "weno5" (Eq. 4 by finite differences); before init."""
        code = {"lb": 0, "weno5": 1}[solver]
        if self._lib.orc_set_phase_solver(self._h, code) != 0:
            raise ValueError("oracle rejected the phase solver")

    def set_gravity(self, g, rho_ref):
        """Buoyancy (rho(phi) - rho_ref) g (needs set_density first)."""
        gv = _f64(g)
        if self._lib.orc_set_gravity(self._h, _ptr(gv), float(rho_ref)) != 0:
            raise ValueError("oracle rejected the gravity parameters")

    def step(self, n: int = 1):
        if self._lib.orc_step(self._h, int(n)) != 0:
            raise RuntimeError("orc_step failed")

    @property
    def time(self) -> int:
        return int(self._lib.orc_time(self._h))

    def moments(self):
        """(rho, u, phi) at the current time: rho = p*, u the forced velocity."""
        rho = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        phi = np.zeros(self.shape)
        self._lib.orc_moments(self._h, _ptr(rho), _ptr(u), _ptr(phi))
        return rho, u, phi

    def diagnostics(self) -> np.ndarray:
        """[Phi, K, eps, max|u|, A_next] reduced during the last step."""
        out = np.zeros(5)
        self._lib.orc_diagnostics(self._h, _ptr(out))
        return out

    def populations(self):
        f = np.zeros((27,) + self.shape)
        g = np.zeros((7,) + self.shape)
        self._lib.orc_get_populations(self._h, _ptr(f), _ptr(g))
        return f, g

    def set_populations(self, f, g):
        """f (27 planes) and g (7 planes); either may be None to keep it."""
        self._lib.orc_set_populations(self._h, None if f is None else _ptr(_f64(f)),
                                      None if g is None else _ptr(_f64(g)))

    def phase_field(self) -> np.ndarray:
        """The stored phi of the WENO-5 phase solver (the state that solver steps)."""
        phi = np.zeros(self.shape)
        if self._lib.orc_get_phase(self._h, _ptr(phi)) != 0:
            raise RuntimeError("phase_field: the WENO-5 phase solver is not selected")
        return phi

    def set_phase_field(self, phi):
        if self._lib.orc_set_phase(self._h, _ptr(_f64(phi))) != 0:
            raise RuntimeError("set_phase_field: the WENO-5 phase solver is not selected")

    def last_force(self) -> np.ndarray:
        F = np.zeros((3,) + self.shape)
        self._lib.orc_last_force(self._h, _ptr(F))
        return F
