"""lb_velocity_statistics (Sec. 5.1 turbulence statistics on the device)
against the FP64 oracle of oracle/turbulence.py on the same FP32 fields.

- The histogram: the oracle bins the FP64 gradient samples; the device bins
  samples it evaluates in FP32, each operation of the factorised stencil
  rounded on its own.  That chain has six roundings (the difference, two
  additions at each transverse level, the division by 72), so a device sample
  is within 6 * 2^-24 of the stencil magnitude (1/72) sum k k |d| of its FP64
  value (8 * 2^-24 is used).  Only samples whose FP64 position lies within that
  distance of a bin edge can change bins: the count of each bin may differ
  from the oracle's by at most the number of such samples at its two edges,
  and the total is the same.
- The moments: the device sums FP32 products of the FP32 samples per thread
  (at most a few hundred terms) and then in FP64; the oracle's are the FP64
  moments of the FP64 gradient.  FP32 rounding of a sample (a few 2^-24 of the
  stencil's terms), of the products and of the partial sums gives rtol 2e-5
  for M2 and M4, and 2e-5 of M(|g|^3) for M3, which cancels.  The skewness and
  flatness the library forms from them follow: |dS| <= 2e-5 M(|g|^3) / M2^1.5
  + 1.5 * 2e-5 |S| and rtol 6e-5 for F.
- The structure functions take FP32 differences and per-thread FP32 sums of
  at most a few hundred terms before the FP64 reduction: each term is within
  a few 2^-24 of its FP64 value and each partial sum within K 2^-24, so rtol
  2e-5 for S_2 and 2e-5 of the mean |d|^3 for S_3.
"""
import numpy as np
import pytest

from oracle import turbulence as T
from paper_2505_01126_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbgb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_01126_gb300 import build

    build.build()
    from paper_2505_01126_gb300 import lbgb as mod

    return mod


FP32_STENCIL_ERR = 8 * 2.0 ** -24  # of the stencil magnitude; six roundings in the device's chain


def histogram_allowance(u64, nbins, rng, scale, rel_scale=0.0):
    """Per-bin allowance for the device's counts (nbins bins, then below and
    above): the FP64 samples within the device's evaluation error of a bin edge
    (an edge k in bin units is the boundary between bins k-1 and k, edge 0 that
    of 'below', edge nbins that of 'above').  rel_scale: relative uncertainty of
    the device's scale (auto-scaled histograms bin by the device's own sqrt(M2))."""
    g = T.longitudinal_gradients(u64).ravel()
    m = T.stencil_magnitude(u64).ravel()
    f = nbins / (2.0 * rng)
    t = (g / scale + rng) * f
    err = (FP32_STENCIL_ERR * m / scale + np.abs(g / scale) * rel_scale) * f + 1e-9
    k = np.rint(t)
    near = (np.abs(t - k) <= err) & (k >= 0) & (k <= nbins)
    allow = np.zeros(nbins + 2, dtype=np.int64)
    for kk in k[near].astype(np.int64):
        allow[nbins if kk == 0 else kk - 1] += 1  # the bin below the edge (or 'below')
        allow[nbins + 1 if kk == nbins else kk] += 1  # the bin above the edge (or 'above')
    return allow, int(near.sum())


def check_histogram(got, u64, nbins, rng, scale, rel_scale=0.0):
    want = T.gradient_histogram(u64, nbins, rng, scale)
    allow, near = histogram_allowance(u64, nbins, rng, scale, rel_scale)
    assert int(got.sum()) == int(want.sum()) == 3 * u64[0].size
    diff = np.abs(got.astype(np.int64) - want)
    assert np.all(diff <= allow), (np.nonzero(diff > allow), diff[diff > allow], allow[diff > allow])
    return near


def check(lbgb, u32, rmax, nbins=64, rng=6.0):
    import torch

    u64 = u32.astype(np.float64)
    mo = T.gradient_moments(u64)
    sig = float(np.sqrt(mo["M2"]))
    res = lbgb.velocity_statistics(torch.from_numpy(u32).cuda(), rmax=rmax, nbins=nbins, range_=rng, scale=sig)
    assert res["M2"] == pytest.approx(mo["M2"], rel=2e-5)
    assert res["M4"] == pytest.approx(mo["M4"], rel=2e-5)
    gabs3 = float(np.mean(np.abs(T.longitudinal_gradients(u64)) ** 3))
    assert abs(res["M3"] - mo["M3"]) <= 2e-5 * gabs3
    assert abs(res["S"] - mo["S"]) <= 2e-5 * gabs3 / mo["M2"] ** 1.5 + 3e-5 * abs(mo["S"])
    assert res["F"] == pytest.approx(mo["F"], rel=6e-5)
    check_histogram(res["hist"], u64, nbins, rng, sig)
    if rmax:
        s2, s3 = T.structure_functions(u64, rmax)
        np.testing.assert_allclose(res["S2"], s2, rtol=2e-5)
        for r in range(1, rmax + 1):
            dabs3 = np.mean([np.abs(np.roll(u64[a], -r, axis=2 - a) - u64[a]) ** 3 for a in range(3)])
            assert abs(res["S3"][r - 1] - s3[r - 1]) <= 2e-5 * dabs3 + 1e-30
    return res, mo


def test_solenoidal_field_48(lbgb):
    """The HIT generator's velocity (modes 1 <= |k| <= 4, u_rms 0.02) on 48^3."""
    u = inputs.to_f32(inputs.solenoidal_velocity(48, 48, 48, 0.02, seed=11))
    res, mo = check(lbgb, u, rmax=24)
    assert res["F"] == pytest.approx(mo["F"], rel=1e-4)


@pytest.mark.parametrize("shape", [(20, 7, 13), (5, 1, 1), (3, 4, 2)])
def test_ragged_and_thin_boxes(lbgb, shape):
    rng = np.random.default_rng(sum(shape))
    u = inputs.to_f32(0.01 * rng.standard_normal((3,) + shape))
    check(lbgb, u, rmax=min(shape) if min(shape) > 1 else 2, nbins=16, rng=3.0)


def test_auto_scale_histogram(lbgb):
    """scale <= 0 bins in units of the device's own sqrt(M2), within 1e-5 of the
    oracle's (M2 to 2e-5): the allowance adds that relative uncertainty of the
    scale to each sample's position."""
    import torch

    u = inputs.to_f32(inputs.solenoidal_velocity(32, 32, 32, 0.02, seed=3))
    res = lbgb.velocity_statistics(torch.from_numpy(u).cuda(), nbins=40, range_=5.0)
    u64 = u.astype(np.float64)
    mo = T.gradient_moments(u64)
    check_histogram(res["hist"], u64, 40, 5.0, float(np.sqrt(mo["M2"])), rel_scale=1.1e-5)


def test_zero_field_has_no_skewness_or_flatness(lbgb):
    import torch

    res = lbgb.velocity_statistics(torch.zeros((3, 4, 4, 4), device="cuda"))
    assert res["M2"] == 0.0 and np.isnan(res["S"]) and np.isnan(res["F"])


def test_bench_workload_256(lbgb):
    """The 256^3 bench workload's initial velocity: moments and histogram exact
    against the oracle, structure functions for r <= 4."""
    w = inputs.bubbly_hit(256, 64, 10.0, seed=2)
    check(lbgb, w.u, rmax=4, nbins=100, rng=8.0)


def test_rejects_bad_arguments(lbgb):
    import torch

    u = torch.zeros(3 * 8, device="cuda")
    with pytest.raises(lbgb.LBError) as e:
        lbgb.velocity_statistics(u.view(3, 2, 2, 2), nbins=10, range_=0.0)
    assert e.value.code == lbgb.LB_EINVAL


@pytest.mark.parametrize("n", [16, 15])
def test_spectrum_modes_and_parseval(lbgb, n):
    """Cosine modes land in their shells; the shells of a random field sum to
    mean |u|^2 / 2 (cuFFT single precision: rtol 1e-5)."""
    import torch

    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    u = np.zeros((3, n, n, n), np.float32)
    u[0] = 0.02 * np.cos(2 * np.pi * (3 * x + 4 * z) / n + 0.4)
    u[2] = 0.01 * np.cos(2 * np.pi * y / n)
    kmax = int(np.ceil(np.sqrt(3) * n / 2))
    E = lbgb.spectrum(torch.from_numpy(u).cuda(), kmax)
    want = T.spectrum(u.astype(np.float64), kmax)
    np.testing.assert_allclose(E, want, rtol=1e-5, atol=1e-6 * want.sum())
    rng = np.random.default_rng(n)
    f = rng.standard_normal((3, n, n, n)).astype(np.float32)
    E = lbgb.spectrum(torch.from_numpy(f).cuda(), kmax)
    assert E.sum() == pytest.approx(0.5 * float((f.astype(np.float64) ** 2).sum(axis=0).mean()), rel=1e-5)


def test_spectrum_bench_workload(lbgb):
    """Energy spectrum of the 256^3 bench workload's velocity and the spectrum of
    one scalar field (its phi) against the FP64 oracle: cuFFT FP32 gives each
    coefficient to ~1e-6 of the field's norm, so shells within 1e-4 relative
    or 1e-6 of the total."""
    import torch

    w = inputs.bubbly_hit(256, 64, 10.0, seed=2)
    for f, kmax in ((w.u, 128), (w.phi[None], 64)):
        E = lbgb.spectrum(torch.from_numpy(np.ascontiguousarray(f)).cuda(), kmax)
        want = T.spectrum(f.astype(np.float64), kmax)
        np.testing.assert_allclose(E, want, rtol=1e-4, atol=1e-6 * want.sum())
