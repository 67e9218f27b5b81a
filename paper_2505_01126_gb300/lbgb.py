"""Thin ctypes binding of the CUDA library (C ABI in include/lbgb.h).

Argument marshalling only: every step of the time step runs in the library's
kernels.  Fields may be torch CUDA tensors (passed by device pointer), CPU
torch tensors or numpy arrays (passed by host pointer); scalar fields have
shape (nz, ny, nx) and vector fields (3, nz, ny, nx), float32, contiguous.
Importing this module loads csrc/liblbgb.so and raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "csrc", "liblbgb.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_ENONFINITE, LB_ESTATE = 0, -1, -2, -3, -4, -5
LB_F32, LB_F16_SHIFTED, LB_BF16_SHIFTED, LB_F32_MOMENTS = 0, 1, 2, 3
LB_F16_SHIFTED_G16, LB_BF16_SHIFTED_G16 = 4, 5
LB_FORCE_NONE, LB_FORCE_CONST, LB_FORCE_ABC, LB_FORCE_LINEAR = 0, 1, 2, 3

STORAGE = {"f32": LB_F32, "f16": LB_F16_SHIFTED, "bf16": LB_BF16_SHIFTED, "moments": LB_F32_MOMENTS,
           "f16g": LB_F16_SHIFTED_G16, "bf16g": LB_BF16_SHIFTED_G16}


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class lb_force(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("g", ctypes.c_double * 3), ("A", ctypes.c_double),
                ("kf", ctypes.c_double), ("K_target", ctypes.c_double), ("T_relax", ctypes.c_double)]


EXPORTS = ["lb_create", "lb_set_stream", "lb_init", "lb_step", "lb_moments", "lb_diagnostics",
           "lb_sync", "lb_time", "lb_set_tile", "lb_get_tile", "lb_tune", "lb_bytes_per_site",
           "lb_destroy", "lb_last_error", "lb_launch_count", "lb_set_timing", "lb_kernel_time",
           "lb_field_stats_static", "lb_batch_create", "lb_batch_set_stream", "lb_batch_init",
           "lb_batch_step", "lb_batch_moments", "lb_batch_diagnostics", "lb_batch_set_tile", "lb_batch_get_tile",
           "lb_batch_tune", "lb_batch_sites", "lb_batch_time", "lb_batch_destroy", "lb_velocity_statistics",
           "lb_spectrum", "lb_state_bytes", "lb_save", "lb_load", "lb_set_density", "lb_set_gravity",
           "lb_set_phase_solver", "lb_measure_fp32_peak", "lb_set_pairing", "lb_get_pairing", "lb_batch_set_density",
           "lb_batch_set_pairing", "lb_batch_get_pairing"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2505_01126_gb300.build.build() first")
    try:  # make the CUDA runtime that torch loaded visible first (same soname)
        import torch  # noqa: F401
    except Exception:
        pass
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.lb_create.argtypes = [i, i, i, d, d, d, d, ctypes.POINTER(lb_force), i, ctypes.POINTER(vp)]
    lib.lb_set_stream.argtypes = [vp, vp]
    lib.lb_init.argtypes = [vp, vp, vp]
    lib.lb_step.argtypes = [vp, i]
    lib.lb_moments.argtypes = [vp, vp, vp, vp]
    lib.lb_diagnostics.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.lb_sync.argtypes = [vp]
    lib.lb_time.argtypes = [vp]
    lib.lb_time.restype = ctypes.c_longlong
    lib.lb_set_tile.argtypes = [vp, i, i]
    lib.lb_get_tile.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.lb_tune.argtypes = [vp, i]
    lib.lb_bytes_per_site.argtypes = [vp]
    lib.lb_bytes_per_site.restype = d
    lib.lb_destroy.argtypes = [vp]
    lib.lb_destroy.restype = None
    lib.lb_last_error.restype = ctypes.c_char_p
    lib.lb_launch_count.argtypes = [vp]
    lib.lb_launch_count.restype = ctypes.c_longlong
    lib.lb_set_timing.argtypes = [vp, i]
    lib.lb_kernel_time.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]
    lib.lb_field_stats_static.argtypes = [vp, vp, i, i, i, vp, ctypes.POINTER(d)]
    dp_ = ctypes.POINTER(d)
    lib.lb_batch_create.argtypes = [i, ctypes.POINTER(i), dp_, dp_, dp_, dp_, i, ctypes.POINTER(vp)]
    lib.lb_batch_set_stream.argtypes = [vp, vp]
    lib.lb_batch_init.argtypes = [vp, i, vp, vp]
    lib.lb_batch_step.argtypes = [vp, i]
    lib.lb_batch_moments.argtypes = [vp, i, vp, vp, vp]
    lib.lb_batch_diagnostics.argtypes = [vp, i, dp_]
    lib.lb_batch_set_tile.argtypes = [vp, i, i]
    lib.lb_batch_get_tile.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.lb_batch_tune.argtypes = [vp, i]
    lib.lb_batch_sites.argtypes = [vp]
    lib.lb_batch_sites.restype = ctypes.c_longlong
    lib.lb_batch_time.argtypes = [vp]
    lib.lb_batch_time.restype = ctypes.c_longlong
    lib.lb_batch_destroy.argtypes = [vp]
    lib.lb_batch_destroy.restype = None
    lib.lb_velocity_statistics.argtypes = [vp, i, i, i, i, i, d, d, vp, dp_, ctypes.POINTER(ctypes.c_ulonglong)]
    lib.lb_spectrum.argtypes = [vp, i, i, i, vp, dp_]
    lib.lb_state_bytes.argtypes = [vp]
    lib.lb_state_bytes.restype = ctypes.c_size_t
    lib.lb_save.argtypes = [vp, vp, ctypes.c_size_t]
    lib.lb_set_density.argtypes = [vp, d, d, d, d]
    lib.lb_set_gravity.argtypes = [vp, d, d, d, d]
    lib.lb_set_phase_solver.argtypes = [vp, i]
    lib.lb_load.argtypes = [vp, vp, ctypes.c_size_t]
    lib.lb_measure_fp32_peak.argtypes = [vp, dp_]
    lib.lb_batch_set_density.argtypes = [vp, dp_, dp_, dp_, dp_]
    lib.lb_batch_set_pairing.argtypes = [vp, i]
    lib.lb_batch_get_pairing.argtypes = [vp, ctypes.POINTER(i)]
    lib.lb_set_pairing.argtypes = [vp, i]
    lib.lb_get_pairing.argtypes = [vp, ctypes.POINTER(i)]
    return lib


_lib = _load()


def lib():
    return _lib


def _check(rc: int):
    if rc != LB_OK:
        raise LBError(rc, _lib.lb_last_error().decode())


def _ptr(a, n_expected: int, writable: bool = False):
    """Pointer of a contiguous float32 torch tensor (CUDA or CPU) or numpy array."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            if writable:
                raise ValueError("output arrays must be contiguous float32")
            a = np.ascontiguousarray(a, dtype=np.float32)
        if a.size != n_expected:
            raise ValueError(f"expected {n_expected} floats, got {a.size}")
        return ctypes.c_void_p(a.ctypes.data), a
    import torch

    if not isinstance(a, torch.Tensor):
        raise TypeError("fields must be torch tensors or numpy arrays")
    if a.dtype != torch.float32 or not a.is_contiguous():
        if writable:
            raise ValueError("output tensors must be contiguous float32")
        a = a.contiguous().float()
    if a.numel() != n_expected:
        raise ValueError(f"expected {n_expected} floats, got {a.numel()}")
    return ctypes.c_void_p(a.data_ptr()), a


def field_stats_static(phi, u, stream=None) -> np.ndarray:
    """FP64 {Phi, K, 0, max|u|, 0} of device fields phi (nz, ny, nx) and u (3, nz, ny, nx)
    through lb_field_stats_static, which allocates no device memory (for callers
    that must not call cudaMalloc); the result is returned in host memory."""
    import torch

    nz, ny, nx = (int(v) for v in phi.shape)
    p, _a = _ptr(phi, nx * ny * nz)
    q, _b = _ptr(u, 3 * nx * ny * nz)
    handle = getattr(stream, "cuda_stream", stream)
    out = (ctypes.c_double * 5)()
    with torch.cuda.device(phi.device):  # the library runs on the current device
        rc = _lib.lb_field_stats_static(p, q, nx, ny, nz, ctypes.c_void_p(int(handle) if handle else 0), out)
    if rc == LB_ENONFINITE:
        raise LBError(rc, _lib.lb_last_error().decode())
    _check(rc)
    return np.array(list(out))


def measure_fp32_peak(stream=None) -> dict:
    """The device's measured FP32 FMA throughput (lb_measure_fp32_peak)."""
    handle = getattr(stream, "cuda_stream", stream)
    out = (ctypes.c_double * 6)()
    _check(_lib.lb_measure_fp32_peak(ctypes.c_void_p(int(handle) if handle else 0), out))
    return {"fp32_flops": out[0], "warp_inst_per_s": out[1], "ms": out[2], "sm_mhz": out[3],
            "fp32_flops_paired": out[4], "paired_warp_inst_per_s": out[5]}


def velocity_statistics(u, rmax: int = 0, nbins: int = 0, range_: float = 8.0, scale: float = 0.0, stream=None):
    """Turbulence statistics of a device velocity field u (3, nz, ny, nx) through
    lb_velocity_statistics: a dict with M2, M3, M4, skewness S, flatness F, the
    structure functions S2, S3 (r = 1 .. rmax) and, with nbins > 0, the histogram
    counts of g / scale (bins, then below and above the range)."""
    _, nz, ny, nx = (int(v) for v in u.shape)
    q, _a = _ptr(u, 3 * nx * ny * nz)
    handle = getattr(stream, "cuda_stream", stream)
    out = (ctypes.c_double * (5 + 2 * rmax))()
    hist = (ctypes.c_ulonglong * (nbins + 2))() if nbins > 0 else None
    _check(_lib.lb_velocity_statistics(q, nx, ny, nz, int(rmax), int(nbins), float(range_), float(scale),
                                       ctypes.c_void_p(int(handle) if handle else 0), out, hist))
    o = np.array(list(out))
    res = {"M2": o[0], "M3": o[1], "M4": o[2], "S": o[3], "F": o[4], "S2": o[5:5 + rmax], "S3": o[5 + rmax:]}
    if nbins > 0:
        res["hist"] = np.array(list(hist), dtype=np.int64)
    return res


def spectrum(f, kmax: int, stream=None) -> np.ndarray:
    """Shell spectrum E(0 .. kmax) of a device field f of shape (ncomp, n, n, n)
    (or (n, n, n) for one component) through lb_spectrum."""
    shape = tuple(int(v) for v in f.shape)
    ncomp = 1 if len(shape) == 3 else shape[0]
    n = shape[-1]
    q, _a = _ptr(f, ncomp * n ** 3)
    handle = getattr(stream, "cuda_stream", stream)
    out = (ctypes.c_double * (kmax + 1))()
    _check(_lib.lb_spectrum(q, ncomp, n, int(kmax), ctypes.c_void_p(int(handle) if handle else 0), out))
    return np.array(list(out))


@dataclass
class Force:
    kind: int = LB_FORCE_NONE
    g: tuple = (0.0, 0.0, 0.0)
    A: float = 0.0
    kf: float = 0.0
    K_target: float = 0.0
    T_relax: float = 100.0

    def to_c(self) -> lb_force:
        f = lb_force()
        f.kind = int(self.kind)
        for k in range(3):
            f.g[k] = float(self.g[k])
        f.A, f.kf = float(self.A), float(self.kf)
        f.K_target, f.T_relax = float(self.K_target), float(self.T_relax)
        return f


class Box:
    """One periodic box: lb_create / lb_init / lb_step / lb_moments / lb_diagnostics."""

    def __init__(self, nx, ny, nz, tau, M, W, sigma, force: Force | None = None, storage="f32",
                 stream=None):
        self._h = None
        self.shape = (int(nz), int(ny), int(nx))
        self.N = int(nx) * int(ny) * int(nz)
        st = STORAGE[storage] if isinstance(storage, str) else int(storage)
        h = ctypes.c_void_p()
        fc = (force or Force()).to_c()
        _check(_lib.lb_create(int(nx), int(ny), int(nz), float(tau), float(M), float(W), float(sigma),
                              ctypes.byref(fc), st, ctypes.byref(h)))
        self._h = h
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an integer cudaStream_t or None."""
        handle = getattr(stream, "cuda_stream", stream)
        _check(_lib.lb_set_stream(self._h, ctypes.c_void_p(int(handle) if handle else 0)))

    def init(self, phi, u):
        p, _k1 = _ptr(phi, self.N)
        q, _k2 = _ptr(u, 3 * self.N)
        _check(_lib.lb_init(self._h, p, q))

    def step(self, n: int = 1):
        _check(_lib.lb_step(self._h, int(n)))

    def set_phase_solver(self, solver: str):
        """"lb" (the D3Q7 model) or "weno5" (Eq. 4 by finite differences); before init."""
        _check(_lib.lb_set_phase_solver(self._h, {"lb": 0, "weno5": 1}[solver]))

    def set_density(self, rho_l: float, rho_g: float, tau_l: float, tau_g: float):
        """Density and viscosity contrasts (lb_set_density): rho and tau of the
        phi = 1 and phi = 0 phases, linear in phi in between."""
        _check(_lib.lb_set_density(self._h, float(rho_l), float(rho_g), float(tau_l), float(tau_g)))

    def set_gravity(self, g, rho_ref: float):
        """Buoyancy (rho(phi) - rho_ref) g (lb_set_gravity); needs set_density first."""
        gx, gy, gz = (float(v) for v in g)
        _check(_lib.lb_set_gravity(self._h, gx, gy, gz, float(rho_ref)))

    def moments(self, rho=None, u=None, phi=None):
        """Fill caller buffers (any may be None) with p*, u (forced velocity) and phi."""
        r, _a = _ptr(rho, self.N, True)
        v, _b = _ptr(u, 3 * self.N, True)
        p, _c = _ptr(phi, self.N, True)
        _check(_lib.lb_moments(self._h, r, v, p))

    def moments_numpy(self):
        rho = np.zeros(self.shape, np.float32)
        u = np.zeros((3,) + self.shape, np.float32)
        phi = np.zeros(self.shape, np.float32)
        self.moments(rho, u, phi)
        return rho, u, phi

    def diagnostics(self, allow_nonfinite: bool = False) -> np.ndarray:
        out = (ctypes.c_double * 5)()
        rc = _lib.lb_diagnostics(self._h, out)
        if rc != LB_OK and not (allow_nonfinite and rc == LB_ENONFINITE):
            _check(rc)
        return np.array(list(out))

    def sync(self):
        _check(_lib.lb_sync(self._h))

    @property
    def time(self) -> int:
        return int(_lib.lb_time(self._h))

    def set_tile(self, ty: int, zc: int):
        _check(_lib.lb_set_tile(self._h, int(ty), int(zc)))

    def tile(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(_lib.lb_get_tile(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def tune(self, steps: int = 3):
        _check(_lib.lb_tune(self._h, int(steps)))
        return self.tile()

    def set_pairing(self, on: bool):
        """The paired step kernel (two sites per thread) for FP16/BF16 storage (lb_set_pairing)."""
        _check(_lib.lb_set_pairing(self._h, 1 if on else 0))

    @property
    def paired(self) -> bool:
        v = ctypes.c_int()
        _check(_lib.lb_get_pairing(self._h, ctypes.byref(v)))
        return bool(v.value)

    @property
    def bytes_per_site(self) -> float:
        return float(_lib.lb_bytes_per_site(self._h))

    @property
    def launches(self) -> int:
        return int(_lib.lb_launch_count(self._h))

    def set_timing(self, on: bool = True):
        _check(_lib.lb_set_timing(self._h, 1 if on else 0))

    def kernel_time(self):
        """(summed fused-kernel milliseconds, timed launches) since timing was switched on."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        _check(_lib.lb_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def save(self) -> np.ndarray:
        """Checkpoint of the current state (lb_save) as a uint8 array."""
        buf = np.empty(int(_lib.lb_state_bytes(self._h)), dtype=np.uint8)
        _check(_lib.lb_save(self._h, ctypes.c_void_p(buf.ctypes.data), buf.nbytes))
        return buf

    def load(self, buf: np.ndarray):
        """Restore a checkpoint written by save() (lb_load)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(_lib.lb_load(self._h, ctypes.c_void_p(buf.ctypes.data), buf.nbytes))

    def close(self):
        if self._h is not None and self._h.value:
            _lib.lb_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Independent periodic boxes advanced together by one persistent launch per
    step (lb_batch_*).  dims: list of (nx, ny, nz); tau, M, W, sigma: per box."""

    def __init__(self, dims, tau, M, W, sigma, storage="f32", stream=None):
        self._h = None
        self.dims = [tuple(int(v) for v in d) for d in dims]
        n = len(self.dims)
        flat = (ctypes.c_int * (3 * n))(*[v for d in self.dims for v in d])

        def arr(x):
            x = list(x) if hasattr(x, "__len__") else [x] * n
            return (ctypes.c_double * n)(*[float(v) for v in x])

        st = STORAGE[storage] if isinstance(storage, str) else int(storage)
        h = ctypes.c_void_p()
        _check(_lib.lb_batch_create(n, flat, arr(tau), arr(M), arr(W), arr(sigma), st, ctypes.byref(h)))
        self._h = h
        if stream is not None:
            handle = getattr(stream, "cuda_stream", stream)
            _check(_lib.lb_batch_set_stream(self._h, ctypes.c_void_p(int(handle) if handle else 0)))

    def _N(self, box):
        nx, ny, nz = self.dims[box]
        return nx * ny * nz

    def set_density(self, rho_l, rho_g, tau_l, tau_g):
        """Density and viscosity contrasts per box (lb_batch_set_density); scalars apply to every box."""
        n = len(self.dims)

        def arr(x):
            x = list(x) if hasattr(x, "__len__") else [x] * n
            return (ctypes.c_double * n)(*[float(v) for v in x])

        _check(_lib.lb_batch_set_density(self._h, arr(rho_l), arr(rho_g), arr(tau_l), arr(tau_g)))

    def set_pairing(self, on):
        """The paired tile body for FP16/BF16 storage (lb_batch_set_pairing):
        False/0, True (64 sites wide), or the tile width 64 or 32."""
        _check(_lib.lb_batch_set_pairing(self._h, int(on)))

    @property
    def pair_width(self) -> int:
        """Width of the paired tiles, 0 when one site per thread runs."""
        v = ctypes.c_int()
        _check(_lib.lb_batch_get_pairing(self._h, ctypes.byref(v)))
        return v.value

    @property
    def paired(self) -> bool:
        return self.pair_width != 0

    def init(self, box, phi, u):
        p, _a = _ptr(phi, self._N(box))
        q, _b = _ptr(u, 3 * self._N(box))
        _check(_lib.lb_batch_init(self._h, int(box), p, q))

    def step(self, n=1):
        _check(_lib.lb_batch_step(self._h, int(n)))

    def moments_numpy(self, box):
        nx, ny, nz = self.dims[box]
        rho = np.zeros((nz, ny, nx), np.float32)
        u = np.zeros((3, nz, ny, nx), np.float32)
        phi = np.zeros((nz, ny, nx), np.float32)
        _check(_lib.lb_batch_moments(self._h, int(box), ctypes.c_void_p(rho.ctypes.data),
                                     ctypes.c_void_p(u.ctypes.data), ctypes.c_void_p(phi.ctypes.data)))
        return rho, u, phi

    def diagnostics(self, box) -> np.ndarray:
        out = (ctypes.c_double * 5)()
        _check(_lib.lb_batch_diagnostics(self._h, int(box), out))
        return np.array(list(out))

    def set_tile(self, ty, zc):
        _check(_lib.lb_batch_set_tile(self._h, int(ty), int(zc)))

    def tile(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(_lib.lb_batch_get_tile(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def tune(self, steps=3):
        _check(_lib.lb_batch_tune(self._h, int(steps)))
        return self.tile()

    @property
    def sites(self) -> int:
        return int(_lib.lb_batch_sites(self._h))

    @property
    def time(self) -> int:
        return int(_lib.lb_batch_time(self._h))

    def close(self):
        if self._h is not None and self._h.value:
            _lib.lb_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
