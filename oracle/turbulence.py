"""FP64 oracle of the velocity statistics of homogeneous isotropic turbulence
(Sec. 5.1: the PDF of the longitudinal velocity gradient with its skewness S
and flatness F, the second- and third-order structure functions, and the
energy and pressure spectra).

TEST INFRASTRUCTURE, like the rest of this package: plain numpy, written out
from the definitions, sharing nothing with the CUDA library.

Definitions (readings of Sec. 5.1, which defines S, F, S_2 and S_3 but not
the discretisation or the sampling):
- Longitudinal gradient samples: g = d_a u_a for a = x, y, z at every site
  (3N samples of a periodic nx*ny*nz field), with the lattice gradient of
  Sec. 2.3, (1/cs^2) sum_i w_i c_ia psi(x + c_i), in FP64.  Using the
  factorisation of the D3Q27 weights this is (1/72) sum over the two
  transverse offsets of k(c) k(c') [psi(+1) - psi(-1)], k = (1, 4, 1).
- Moments M_n = mean of g^n (n = 2, 3, 4); S = M3 / M2^(3/2), F = M4 / M2^2.
- Histogram of g / scale over nbins equal bins on [-range, range): sample g
  falls in bin floor((g / scale + range) * nbins / (2 range)), with counts
  below and above the range; all in FP64.
- Longitudinal structure functions S_n(r) = mean over a and sites of
  (u_a(x + r e_a) - u_a(x))^n, n = 2, 3, periodic.
"""
from __future__ import annotations

import numpy as np

# array axes of a (nz, ny, nx) field for the Cartesian directions x, y, z
_AX = {0: 2, 1: 1, 2: 0}


def _shift(f: np.ndarray, axis: int, c: int) -> np.ndarray:
    """psi(x + c e_axis) on the periodic grid."""
    return np.roll(f, -c, axis=axis)


def _stencil_terms(u: np.ndarray):
    """For each direction a: the nine differences d(c1, c2) = u_a(x + e_a + c1 e_t1
    + c2 e_t2) - u_a(x - e_a + c1 e_t1 + c2 e_t2) (t1, t2 the transverse
    directions) with their weights k(c1) k(c2), k = (1, 4, 1)."""
    u = np.asarray(u, dtype=np.float64)
    k = {-1: 1.0, 0: 4.0, 1: 1.0}
    for a in range(3):
        ax = _AX[a]
        t1, t2 = [_AX[t] for t in range(3) if t != a]
        d = _shift(u[a], ax, 1) - _shift(u[a], ax, -1)
        yield a, [(k[c1] * k[c2], _shift(_shift(d, t1, c1), t2, c2)) for c1 in (-1, 0, 1) for c2 in (-1, 0, 1)]


def longitudinal_gradients(u: np.ndarray) -> np.ndarray:
    """d_a u_a for a = x, y, z: array (3, nz, ny, nx), FP64,
    g = (1/72) sum_{c1, c2} k(c1) k(c2) d(c1, c2)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.empty_like(u)
    for a, terms in _stencil_terms(u):
        out[a] = sum(w * d for w, d in terms) / 72.0
    return out


def stencil_magnitude(u: np.ndarray) -> np.ndarray:
    """(1/72) sum_{c1, c2} k(c1) k(c2) |d(c1, c2)| per sample, shape (3, nz, ny, nx):
    the scale of the rounding error of any evaluation of the gradient that
    rounds each of its operations (an FP32 evaluation is off by at most a few
    2^-24 of it)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.empty_like(u)
    for a, terms in _stencil_terms(u):
        out[a] = sum(w * np.abs(d) for w, d in terms) / 72.0
    return out


def gradient_moments(u: np.ndarray) -> dict:
    g = longitudinal_gradients(u).ravel()
    g2 = g * g
    m2, m3, m4 = g2.mean(), (g2 * g).mean(), (g2 * g2).mean()
    return {"M2": m2, "M3": m3, "M4": m4, "S": m3 / m2 ** 1.5, "F": m4 / (m2 * m2), "samples": g.size}


def gradient_histogram(u: np.ndarray, nbins: int, rng: float, scale: float) -> np.ndarray:
    """Counts (nbins + 2 integers): the nbins bins, then below and above."""
    g = longitudinal_gradients(u).ravel()
    b = np.floor((g / scale + rng) * (nbins / (2.0 * rng)))
    out = np.zeros(nbins + 2, dtype=np.int64)
    inside = (b >= 0) & (b < nbins)
    np.add.at(out, b[inside].astype(np.int64), 1)
    out[nbins] = int((b < 0).sum())
    out[nbins + 1] = int((b >= nbins).sum())
    return out


def structure_functions(u: np.ndarray, rmax: int) -> tuple[np.ndarray, np.ndarray]:
    """(S_2(r), S_3(r)) for r = 1 .. rmax."""
    u = np.asarray(u, dtype=np.float64)
    s2 = np.zeros(rmax)
    s3 = np.zeros(rmax)
    for r in range(1, rmax + 1):
        acc2 = acc3 = 0.0
        for a in range(3):
            d = _shift(u[a], _AX[a], r) - u[a]
            acc2 += (d * d).sum()
            acc3 += (d * d * d).sum()
        s2[r - 1] = acc2 / (3 * u[0].size)
        s3[r - 1] = acc3 / (3 * u[0].size)
    return s2, s3


def spectrum(f: np.ndarray, kmax: int) -> np.ndarray:
    """Shell spectrum E(k), k = 0 .. kmax, of a periodic cubic field f of shape
    (ncomp, n, n, n): E(k) = 1/2 sum over the components and over the integer
    wavevectors m with round(|m|) = k of |f_hat(m)|^2, f_hat = FFT(f) / N.
    For a velocity field this is the energy spectrum, with sum_k E(k) = mean
    |u|^2 / 2 when kmax covers every shell (Parseval); for the pressure, 1/2
    |p_hat|^2 per shell."""
    f = np.asarray(f, dtype=np.float64)
    n = f.shape[-1]
    assert f.shape[-3:] == (n, n, n)
    N = n ** 3
    m = np.fft.fftfreq(n, 1.0 / n)  # signed integer wavenumbers
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    k = np.floor(np.sqrt(mx * mx + my * my + mz * mz) + 0.5).astype(np.int64)
    p = np.zeros(k.shape)
    for c in range(f.shape[0]):
        fh = np.fft.fftn(f[c]) / N
        p += 0.5 * (fh.real ** 2 + fh.imag ** 2)
    out = np.zeros(kmax + 1)
    sel = k <= kmax
    np.add.at(out, k[sel], p[sel])
    return out
