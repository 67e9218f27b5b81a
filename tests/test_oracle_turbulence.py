"""Pins of the turbulence-statistics oracle (oracle/turbulence.py, Sec. 5.1)
against closed forms and brute force, independent of the oracle's own code.

Closed forms: for u_a = A_a sin(k_a x_a + p_a) (each component a function of
its own coordinate) with k_a = 2 pi m_a / n_a, the lattice gradient is
d_a u_a = A_a sin(k_a) cos(k_a x_a + p_a) exactly, so over the 3N samples
M2 = (1/3) sum_a A_a^2 sin^2(k_a) / 2, M3 = 0, M4 = (1/3) sum_a A_a^4 sin^4(k_a) 3/8
(full periods, 4 m_a not a multiple of n_a), and
S_2(r) = (1/3) sum_a A_a^2 (1 - cos k_a r), S_3(r) = 0.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import turbulence as T


def mode_field(n, m, A, p):
    nz, ny, nx = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coords = (x, y, z)
    ns = (nx, ny, nz)
    u = np.zeros((3,) + n)
    for a in range(3):
        u[a] = A[a] * np.sin(2 * math.pi * m[a] / ns[a] * coords[a] + p[a])
    return u


@pytest.mark.parametrize("n,m", [((24, 20, 16), (3, 2, 5)), ((9, 14, 11), (1, 3, 2))])
def test_single_mode_closed_forms(n, m):
    nz, ny, nx = n
    ns = (nx, ny, nz)
    A, p = (0.02, 0.013, 0.007), (0.3, 1.1, -0.7)
    u = mode_field(n, m, A, p)
    k = [2 * math.pi * m[a] / ns[a] for a in range(3)]
    mo = T.gradient_moments(u)
    m2 = sum(A[a] ** 2 * math.sin(k[a]) ** 2 / 2 for a in range(3)) / 3
    m4 = sum(A[a] ** 4 * math.sin(k[a]) ** 4 * 3 / 8 for a in range(3)) / 3
    assert mo["M2"] == pytest.approx(m2, rel=1e-12)
    assert mo["M4"] == pytest.approx(m4, rel=1e-12)
    assert abs(mo["M3"]) < 1e-12 * m2 ** 1.5
    s2, s3 = T.structure_functions(u, 6)
    for r in range(1, 7):
        want = sum(A[a] ** 2 * (1 - math.cos(k[a] * r)) for a in range(3)) / 3
        assert s2[r - 1] == pytest.approx(want, rel=1e-12, abs=1e-18)
        assert abs(s3[r - 1]) < 1e-12 * max(want, 1e-12) ** 1.5


def test_gradient_is_the_lattice_stencil_by_brute_force():
    """(1/cs^2) sum over the 27 D3Q27 directions of w_i c_ia u_a(x + c_i), looped."""
    rng = np.random.default_rng(5)
    n = (4, 5, 6)
    u = rng.standard_normal((3,) + n)
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    g = T.longitudinal_gradients(u)
    nz, ny, nx = n
    for a in range(3):
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            acc = 0.0
            for cx, cy, cz in itertools.product((-1, 0, 1), repeat=3):
                c = (cx, cy, cz)
                acc += w1[cx] * w1[cy] * w1[cz] * c[a] * u[a][(z + cz) % nz, (y + cy) % ny, (x + cx) % nx]
            assert g[a, z, y, x] == pytest.approx(3.0 * acc, abs=1e-14)


def test_structure_functions_by_brute_force():
    rng = np.random.default_rng(6)
    n = (5, 4, 7)
    u = rng.standard_normal((3,) + n)
    s2, s3 = T.structure_functions(u, 4)
    nz, ny, nx = n
    ns = (nx, ny, nz)
    for r in range(1, 5):
        a2 = a3 = 0.0
        for a in range(3):
            for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
                q = [x, y, z]
                q[a] = (q[a] + r) % ns[a]
                d = u[a][q[2], q[1], q[0]] - u[a][z, y, x]
                a2 += d ** 2
                a3 += d ** 3
        assert s2[r - 1] == pytest.approx(a2 / (3 * u[0].size), rel=1e-12)
        assert s3[r - 1] == pytest.approx(a3 / (3 * u[0].size), rel=1e-10, abs=1e-14)


def test_histogram_counts():
    u = np.zeros((3, 6, 5, 4))
    h = T.gradient_histogram(u, 10, 5.0, 1.0)
    assert h.sum() == 3 * u[0].size
    assert h[5] == 3 * u[0].size  # g = 0 falls in bin floor(5 * 10 / 10) = 5
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3, 6, 5, 4))
    g = T.longitudinal_gradients(u).ravel()
    sig = float(np.sqrt((g * g).mean()))
    h = T.gradient_histogram(u, 8, 1.0, sig)
    assert h.sum() == g.size
    assert h[8] == int((g / sig < -1.0).sum()) and h[9] == int((g / sig >= 1.0).sum())
    # bin b holds -1 + b/4 <= g/sig < -1 + (b+1)/4
    for b in range(8):
        assert h[b] == int(((g / sig >= -1 + b / 4) & (g / sig < -1 + (b + 1) / 4)).sum())


def test_stencil_magnitude_bounds_the_gradient():
    """|g| <= the stencil magnitude, with equality when every difference has one
    sign (a linear field along its own axis), and the magnitude is, by brute
    force, (1/cs^2) sum over the D3Q27 directions c with c_a = +1 of
    w_c |u_a(x + c) - u_a(x + c - 2 e_a)| (each difference taken across the
    site at one transverse offset, as the factorised stencil takes it)."""
    rng = np.random.default_rng(8)
    n = (7, 6, 5)
    u = rng.standard_normal((3,) + n)
    g = T.longitudinal_gradients(u)
    m = T.stencil_magnitude(u)
    assert np.all(np.abs(g) <= m * (1 + 1e-12))
    nz, ny, nx = n
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    for a in range(3):
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            acc = 0.0
            for c in itertools.product((-1, 0, 1), repeat=3):  # c = (cx, cy, cz)
                if c[a] != 1:
                    continue
                w = w1[c[0]] * w1[c[1]] * w1[c[2]]
                p = [(x + c[0]) % nx, (y + c[1]) % ny, (z + c[2]) % nz]
                cq = [c[b] - 2 * (b == a) for b in range(3)]
                q = [(x + cq[0]) % nx, (y + cq[1]) % ny, (z + cq[2]) % nz]
                acc += 3 * w * abs(u[a, p[2], p[1], p[0]] - u[a, q[2], q[1], q[0]])
            assert m[a, z, y, x] == pytest.approx(acc, rel=1e-12)
    # a linear field along its own axis: every difference has one sign away
    # from the periodic seam, so |g| equals the magnitude there
    z, y, x = np.meshgrid(*[np.arange(8)] * 3, indexing="ij")
    lin = np.stack([0.003 * x, 0.002 * y, 0.001 * z]).astype(np.float64)
    g, m = T.longitudinal_gradients(lin), T.stencil_magnitude(lin)
    inner = (slice(1, -1),) * 3
    for a, slope in enumerate((0.003, 0.002, 0.001)):
        np.testing.assert_allclose(g[a][inner], slope, rtol=1e-12)
        np.testing.assert_allclose(m[a][inner], slope, rtol=1e-12)


def test_spectrum_single_modes_and_parseval():
    """A cosine mode A cos(2 pi m.x / n) puts A^2/4 in shell round(|m|); any
    field's shells sum to mean |f|^2 / 2 (Parseval)."""
    n = 16
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = 0.02 * np.cos(2 * math.pi * (3 * x + 4 * z) / n + 0.4)   # |m| = 5
    u[2] = 0.01 * np.cos(2 * math.pi * (1 * y) / n)                 # |m| = 1
    E = T.spectrum(u, 14)
    want = np.zeros(15)
    want[5] = 0.02 ** 2 / 4
    want[1] = 0.01 ** 2 / 4
    np.testing.assert_allclose(E, want, atol=1e-18)
    rng = np.random.default_rng(9)
    f = rng.standard_normal((3, 8, 8, 8))
    E = T.spectrum(f, 7)  # 7 > sqrt(3)*4 = 6.93: every shell
    assert E.sum() == pytest.approx(0.5 * (f * f).sum(axis=0).mean(), rel=1e-12)
    # brute-force DFT of one scalar field, one shell
    g = rng.standard_normal((1, 4, 4, 4))
    E = T.spectrum(g, 3)
    acc = 0.0
    for mz, my, mx in itertools.product(range(4), repeat=3):
        sm = [v if v < 2 else v - 4 for v in (mx, my, mz)]
        if int(math.floor(math.sqrt(sum(v * v for v in sm)) + 0.5)) != 1:
            continue
        c = 0j
        for zz, yy, xx in itertools.product(range(4), repeat=3):
            c += g[0, zz, yy, xx] * np.exp(-2j * math.pi * (mx * xx + my * yy + mz * zz) / 4)
        acc += 0.5 * abs(c / 64) ** 2
    assert E[1] == pytest.approx(acc, rel=1e-12)
