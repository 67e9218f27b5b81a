"""Seeded synthetic inputs for the two-phase lattice Boltzmann step.

This module holds no arithmetic of the method itself: it only builds initial
fields (phase field phi and velocity u) from a seed.  Both the CUDA library's
tests/benchmark and the FP64 oracle take their inputs from here.

Random numbers come from splitmix64 (Steele, Lea and Flood 2014; the
finaliser constants are Vigna's published ones), written here from that
definition; normal deviates use the Box-Muller transform.

Field conventions: scalar fields have shape (nz, ny, nx), vector fields
(3, nz, ny, nx), C order, so the flat site index is x + nx*(y + ny*z).
Workloads stand in for the paper's bubble-laden homogeneous isotropic
turbulence at 512^3 (Sec. 5.2): random solenoidal velocity from Fourier modes
1 <= |k| <= 4, seeded non-overlapping bubbles with the equilibrium tanh
interface profile.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator: state += golden gamma, then a 3-step finaliser."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK
        self._spare = None

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self) -> float:
        """Standard normal deviate (Box-Muller, both outputs used in turn)."""
        if self._spare is not None:
            v, self._spare = self._spare, None
            return v
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        self._spare = r * math.sin(2.0 * math.pi * u2)
        return r * math.cos(2.0 * math.pi * u2)


def tanh_profile(d: np.ndarray, R: float, W: float) -> np.ndarray:
    """Interface profile of a sphere of radius R, phi = 1 inside:
    1/2 - 1/2 tanh(2 (d - R) / W) in the Euclidean distance d (the equilibrium
    profile of the conservative Allen-Cahn equation with interface width W)."""
    return 0.5 - 0.5 * np.tanh(2.0 * (d - R) / W)


def _min_image(delta: np.ndarray, n: int) -> np.ndarray:
    return delta - n * np.round(delta / n)


def droplet(nx: int, ny: int, nz: int, R: float, W: float, center=None) -> np.ndarray:
    """A single sphere; default centre is ((nx-1)/2, (ny-1)/2, (nz-1)/2), which keeps the
    box's mirror symmetries.  Distances use the minimum image."""
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dx = _min_image(x - center[0], nx)
    dy = _min_image(y - center[1], ny)
    dz = _min_image(z - center[2], nz)
    d = np.sqrt(dx * dx + dy * dy + dz * dz)
    return tanh_profile(d, R, W)


def bubble_centers(n: tuple, count: int, R: float, W: float, rng: SplitMix64,
                   max_tries: int = 1_000_000) -> np.ndarray:
    """Uniform centres, a draw rejected when its minimum-image distance to an
    accepted centre is below 2R + 2W.  n = (nx, ny, nz)."""
    nx, ny, nz = n
    dmin = 2.0 * R + 2.0 * W
    centers = []
    tries = 0
    while len(centers) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place the bubbles without overlap")
        c = (rng.uniform() * nx, rng.uniform() * ny, rng.uniform() * nz)
        ok = True
        for p in centers:
            dx = _min_image(np.float64(c[0] - p[0]), nx)
            dy = _min_image(np.float64(c[1] - p[1]), ny)
            dz = _min_image(np.float64(c[2] - p[2]), nz)
            if dx * dx + dy * dy + dz * dz < dmin * dmin:
                ok = False
                break
        if ok:
            centers.append(c)
    return np.array(centers, dtype=np.float64).reshape(-1, 3)


def bubbles(n: tuple, centers: np.ndarray, R: float, W: float, margin: float | None = None) -> np.ndarray:
    """phi = max over bubbles of the tanh profile.  Each bubble is evaluated on a
    box of half-width R + margin around its centre (default margin 8W, where
    the profile is below 1e-13); phi is 0 elsewhere."""
    nx, ny, nz = n
    if margin is None:
        margin = 8.0 * W
    phi = np.zeros((nz, ny, nx), dtype=np.float64)
    h = int(math.ceil(R + margin))
    for c in centers:
        ix = np.arange(int(math.floor(c[0])) - h, int(math.floor(c[0])) + h + 2)
        iy = np.arange(int(math.floor(c[1])) - h, int(math.floor(c[1])) + h + 2)
        iz = np.arange(int(math.floor(c[2])) - h, int(math.floor(c[2])) + h + 2)
        # the local box may wrap; keep each periodic site once
        ix = np.unique(np.mod(ix, nx))
        iy = np.unique(np.mod(iy, ny))
        iz = np.unique(np.mod(iz, nz))
        dx = _min_image(ix - c[0], nx)
        dy = _min_image(iy - c[1], ny)
        dz = _min_image(iz - c[2], nz)
        d = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        local = tanh_profile(d, R, W)
        sub = phi[np.ix_(iz, iy, ix)]
        phi[np.ix_(iz, iy, ix)] = np.maximum(sub, local)
    return phi


def fourier_modes(kmin: float, kmax: float):
    """Integer wave vectors k with kmin <= |k| <= kmax, in a fixed order
    (kz, then ky, then kx, each ascending)."""
    K = int(math.floor(kmax))
    ks = []
    for kz in range(-K, K + 1):
        for ky in range(-K, K + 1):
            for kx in range(-K, K + 1):
                k2 = kx * kx + ky * ky + kz * kz
                if kmin * kmin <= k2 <= kmax * kmax:
                    ks.append((kx, ky, kz))
    return np.array(ks, dtype=np.int64)


def solenoidal_amplitudes(rng: SplitMix64, ks: np.ndarray) -> np.ndarray:
    """Complex amplitude per mode: 3 complex N(0,1) components (re, im drawn in
    turn), with the part along k removed so each mode is divergence-free."""
    amp = np.zeros((len(ks), 3), dtype=np.complex128)
    for m, k in enumerate(ks):
        a = np.array([complex(rng.normal(), rng.normal()) for _ in range(3)])
        kk = k.astype(np.float64)
        a = a - kk * (np.dot(a, kk) / np.dot(kk, kk))
        amp[m] = a
    return amp


def solenoidal_velocity(nx: int, ny: int, nz: int, u_rms: float, seed: int,
                        kmin: float = 1.0, kmax: float = 4.0) -> np.ndarray:
    """u(x) = sum_k Re(a_k exp(2 pi i (kx x/nx + ky y/ny + kz z/nz))), rescaled so that
    sqrt(<|u|^2>/3) = u_rms over the grid.  Evaluated by inverse FFT."""
    rng = SplitMix64(seed)
    ks = fourier_modes(kmin, kmax)
    amp = solenoidal_amplitudes(rng, ks)
    u = np.zeros((3, nz, ny, nx), dtype=np.float64)
    N = nx * ny * nz
    for comp in range(3):
        spec = np.zeros((nz, ny, nx), dtype=np.complex128)
        for m, k in enumerate(ks):
            spec[k[2] % nz, k[1] % ny, k[0] % nx] += amp[m, comp]
        u[comp] = np.real(np.fft.ifftn(spec)) * N
    rms = math.sqrt(float(np.mean(np.sum(u * u, axis=0))) / 3.0)
    if rms > 0:
        u *= u_rms / rms
    return u


def taylor_green(nx: int, ny: int, nz: int, U: float) -> np.ndarray:
    """2D Taylor-Green vortex in the x-y plane (one period per box edge):
    u = U sin(kx x) cos(ky y), v = -U (kx/ky) cos(kx x) sin(ky y), w = 0."""
    kx = 2 * math.pi / nx
    ky = 2 * math.pi / ny
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    u[0] = U * np.sin(kx * x) * np.cos(ky * y)
    u[1] = -U * (kx / ky) * np.cos(kx * x) * np.sin(ky * y)
    return u


def slab(nx: int, ny: int, nz: int, W: float, x0: float, x1: float) -> np.ndarray:
    """Planar slab phi = 1 for x0 < x < x1 (periodic in x): the tanh profile in the
    minimum-image distance from the mid-plane, half-thickness (x1 - x0)/2."""
    x = np.arange(nx, dtype=np.float64)
    d = np.abs(_min_image(x - 0.5 * (x0 + x1), nx))
    p = tanh_profile(d, 0.5 * (x1 - x0), W)
    return np.broadcast_to(p[None, None, :], (nz, ny, nx)).copy()


def to_f32(a: np.ndarray) -> np.ndarray:
    """Round an FP64 field to FP32 (both implementations take the same FP32 values)."""
    return np.ascontiguousarray(a, dtype=np.float32)


@dataclass
class Workload:
    name: str
    n: tuple            # (nx, ny, nz)
    tau: float
    M: float
    W: float
    sigma: float
    force_kind: int     # 0 none, 1 const, 2 ABC, 3 linear
    phi: np.ndarray     # FP32, (nz, ny, nx)
    u: np.ndarray       # FP32, (3, nz, ny, nx)
    T_relax: float = 100.0


def static_droplet(edge: int = 32, R: float = 8.0, W: float = 3.0, sigma: float = 0.01,
                   tau: float = 1.0, M: float = 0.1) -> Workload:
    """Periodic edge^3 box, one droplet of radius R at the centre, zero velocity."""
    phi = droplet(edge, edge, edge, R, W)
    u = np.zeros((3, edge, edge, edge))
    return Workload(f"droplet{edge}", (edge, edge, edge), tau, M, W, sigma, 0, to_f32(phi), to_f32(u))


def bubbly_hit(edge: int, n_bubbles: int, R: float, seed: int, tau: float = 0.51,
               u_rms: float = 0.02, W: float = 3.0, sigma: float = 0.01, M: float = 0.1,
               force_kind: int = 3) -> Workload:
    """Forced homogeneous isotropic turbulence with bubbles: solenoidal velocity from modes
    1 <= |k| <= 4 scaled to u_rms, n_bubbles bubbles of radius R at seeded
    non-overlapping positions, linear forcing (force_kind 3) by default."""
    rng = SplitMix64(seed)
    centers = bubble_centers((edge, edge, edge), n_bubbles, R, W, rng)
    phi = bubbles((edge, edge, edge), centers, R, W)
    u = solenoidal_velocity(edge, edge, edge, u_rms, seed=seed + 0x5EED)
    return Workload(f"hit{edge}_b{n_bubbles}", (edge, edge, edge), tau, M, W, sigma, force_kind,
                    to_f32(phi), to_f32(u))


def ensemble_specs(count: int, seed: int, edges=(24, 32, 48, 64, 96)):
    """Box specs for a batched ensemble: edge uniform in `edges`, droplet radius
    0.25 edge (1 + U[-0.2, 0.2]), sigma uniform in [0.005, 0.02]; tau=1, M=0.1, W=3."""
    rng = SplitMix64(seed)
    specs = []
    for _ in range(count):
        e = edges[min(int(rng.uniform() * len(edges)), len(edges) - 1)]
        R = 0.25 * e * (1.0 + (rng.uniform() * 0.4 - 0.2))
        sigma = 0.005 + 0.015 * rng.uniform()
        specs.append({"edge": e, "R": R, "sigma": sigma, "tau": 1.0, "M": 0.1, "W": 3.0})
    return specs


def bubbly_hit_device(edge: int, n_bubbles: int, R: float, seed: int, tau: float = 0.51, u_rms: float = 0.02,
                      W: float = 3.0, sigma: float = 0.01, M: float = 0.1, force_kind: int = 3, device="cuda"):
    """bubbly_hit built on a CUDA device, for boxes too large for host FFTs (512^3 and
    up): the same splitmix64 draws, spectrum, bubble centres and profile, evaluated in
    FP64 with torch's FFT on the device and rounded to FP32.  Returns a Workload whose
    phi and u are device tensors."""
    import torch

    n = edge
    rng = SplitMix64(seed)
    centers = bubble_centers((n, n, n), n_bubbles, R, W, rng)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device=device)
    h = int(math.ceil(R + 8.0 * W))
    for c in centers:
        idx = []
        dist = []
        for ax in range(3):
            i = np.unique(np.mod(np.arange(int(math.floor(c[ax])) - h, int(math.floor(c[ax])) + h + 2), n))
            idx.append(torch.from_numpy(i).to(device))
            dist.append(torch.from_numpy(_min_image(i - c[ax], n)).to(device))
        d = torch.sqrt(dist[2][:, None, None] ** 2 + dist[1][None, :, None] ** 2 + dist[0][None, None, :] ** 2)
        local = 0.5 - 0.5 * torch.tanh(2.0 * (d - R) / W)
        iz, iy, ix = idx[2][:, None, None], idx[1][None, :, None], idx[0][None, None, :]
        phi[iz, iy, ix] = torch.maximum(phi[iz, iy, ix], local)
    rng_u = SplitMix64(seed + 0x5EED)
    ks = fourier_modes(1.0, 4.0)
    amp = solenoidal_amplitudes(rng_u, ks)
    u = torch.empty((3, n, n, n), dtype=torch.float32, device=device)
    sq = torch.zeros((), dtype=torch.float64, device=device)
    for comp in range(3):
        spec = torch.zeros((n, n, n), dtype=torch.complex128, device=device)
        for m, k in enumerate(ks):
            spec[k[2] % n, k[1] % n, k[0] % n] += complex(amp[m, comp])
        uc = torch.fft.ifftn(spec).real * float(n ** 3)
        del spec
        sq += (uc * uc).sum()
        u[comp] = uc.to(torch.float32)
        del uc
    rms = math.sqrt(float(sq) / n ** 3 / 3.0)
    # rescale in FP64 before the final rounding, as bubbly_hit does
    u64_scale = u_rms / rms if rms > 0 else 1.0
    for comp in range(3):
        spec = torch.zeros((n, n, n), dtype=torch.complex128, device=device)
        for m, k in enumerate(ks):
            spec[k[2] % n, k[1] % n, k[0] % n] += complex(amp[m, comp])
        u[comp] = (torch.fft.ifftn(spec).real * float(n ** 3) * u64_scale).to(torch.float32)
        del spec
    return Workload(f"hit{edge}_b{n_bubbles}", (n, n, n), tau, M, W, sigma, force_kind,
                    phi.to(torch.float32), u)
