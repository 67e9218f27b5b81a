"""Moment-only storage (LB_F32_MOMENTS): each site keeps the ten FP32
coefficients of its post-collision population polynomial (Eq. 7, rebuilt from
p*, u, a2 and F as in the thread-safe scheme of Sec. 3) and the next step pulls
f_i(x) = w_i (1 + v_i(x - c_i)) from the neighbours' coefficients.

Every pulled value is formed by the same FP32 additions the AA storage uses
to evaluate the polynomial before storing it, so the two storages give the
same fields and reductions bit for bit; with the FP32 AA path's parity with
the FP64 oracle this carries the oracle parity over.  The oracle is also
compared directly.
"""
import math

import numpy as np
import pytest

from paper_2505_01126_gb300 import inputs
from test_gpu_parity import TOL, check_diagnostics, max_err, smooth_fields

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


FORCES = {
    "none": dict(kind=0),
    "const": dict(kind=1, g=(1e-5, -2e-5, 5e-6)),
    "abc": dict(kind=2, A=2e-5, kf=2 * math.pi / 12),
    "linear": dict(kind=3, T_relax=20.0),
}


def run(lbgb, storage, shape, phi, u, steps, force, tile=None, sample=()):
    nz, ny, nx = shape
    b = lbgb.Box(nx, ny, nz, 0.6, 0.1, 3.0, 0.01, force=lbgb.Force(**force), storage=storage)
    if tile is not None:
        b.set_tile(*tile)
    b.init(phi, u)
    out = []
    done = 0
    for t in sorted(set(sample) | {steps}):
        b.step(t - done)
        done = t
        out.append((b.moments_numpy(), b.diagnostics()))
    b.close()
    return out


@pytest.mark.parametrize("force", sorted(FORCES))
@pytest.mark.parametrize("shape", [(20, 16, 32), (21, 19, 44), (13, 9, 45), (7, 5, 3)])
def test_moment_storage_equals_f32_bit_for_bit(lbgb, shape, force):
    """Ragged and float4 tiles (nx = 44 vs 45), thin boxes, every forcing kind;
    fields and FP64 reductions compared at t = 0, 1, 2, 5 and 9 (the first step
    evaluates the equilibrium coefficients lb_init stored, the later ones pull;
    pairs of steps run as CUDA graphs)."""
    phi, u = smooth_fields(shape, sum(shape))
    a = run(lbgb, "f32", shape, phi, u, 9, FORCES[force], sample=(0, 1, 2, 5))
    m = run(lbgb, "moments", shape, phi, u, 9, FORCES[force], sample=(0, 1, 2, 5))
    for (fa, da), (fm, dm) in zip(a, m):
        for x, y in zip(fa, fm):
            assert np.array_equal(x, y)
        assert np.array_equal(da, dm)


@pytest.mark.parametrize("tile", [(4, 8), (8, 16), (8, 5), (4, 1), (4, 64)])
def test_moment_storage_tile_shapes(lbgb, tile):
    """Every launch shape (z-chunks that split the box unevenly, one plane per
    chunk) gives the same fields as the FP32 AA storage."""
    shape = (23, 19, 44)
    phi, u = smooth_fields(shape, 4)
    a = run(lbgb, "f32", shape, phi, u, 6, FORCES["none"])
    m = run(lbgb, "moments", shape, phi, u, 6, FORCES["none"], tile=tile)
    for x, y in zip(a[0][0], m[0][0]):
        assert np.array_equal(x, y)


def test_moment_storage_hit_64_against_oracle(lbgb, orc):
    """64^3 forced HIT surrogate (two bubbles R = 10, tau = 0.51, linear forcing),
    50 steps, against the FP64 oracle with the FP32 parity tolerance."""
    w = inputs.bubbly_hit(64, 2, 10.0, seed=2)
    n = 64
    o = orc.Oracle(n, n, n, w.tau, w.M, w.W, w.sigma, force_kind=3, T_relax=w.T_relax)
    o.init(w.phi.astype(np.float64), w.u.astype(np.float64))
    o.step(50)
    b = lbgb.Box(n, n, n, w.tau, w.M, w.W, w.sigma, force=lbgb.Force(kind=3, T_relax=w.T_relax),
                 storage="moments")
    b.init(w.phi, w.u)
    b.step(50)
    e = max_err(b.moments_numpy(), o.moments())
    assert max(e) <= TOL, e
    check_diagnostics(b.diagnostics(), o.diagnostics(), n ** 3, field_err=max(e), tau=w.tau)


def test_moment_storage_full_size_256(lbgb):
    """The 256^3 benchmark workload in the launch shape the tuner picks for the
    moment-only storage: 5 steps equal the FP32 AA storage in the same launch
    shape bit for bit (the same shape, because the linear forcing amplitude
    follows from FP64 sums of per-block partials, whose grouping the shape sets)."""
    w = inputs.bubbly_hit(256, 64, 10.0, seed=2)
    n = 256
    res = []
    tile = None
    for st in ("moments", "f32"):
        b = lbgb.Box(n, n, n, w.tau, w.M, w.W, w.sigma, force=lbgb.Force(kind=3, T_relax=w.T_relax), storage=st)
        if tile is None:
            tile = b.tune(2)
        else:
            b.set_tile(*tile)
        b.init(w.phi, w.u)
        b.step(5)
        res.append((b.moments_numpy(), b.diagnostics()))
        b.close()
    for x, y in zip(res[0][0], res[1][0]):
        assert np.array_equal(x, y)
    assert np.array_equal(res[0][1], res[1][1])


def test_moment_storage_bytes_and_state(lbgb):
    b = lbgb.Box(16, 16, 16, 0.8, 0.1, 3.0, 0.01, storage="moments")
    assert b.bytes_per_site == 136.0
    with pytest.raises(lbgb.LBError) as e:
        b.step(1)
    assert e.value.code == lbgb.LB_ESTATE
    b.close()
