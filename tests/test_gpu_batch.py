"""Batched ensemble: many independent periodic boxes of uneven sizes advanced
by one persistent launch per step.

Every box is computed by the same per-tile code as a single box, so after any
number of steps its fields (and FP64 reductions) must equal, bit for bit,
those of the single-box path with the same tile shape.  Together with the
single-box parity tests against the FP64 oracle, this carries the oracle
parity over to every box of a batch; test_batch_boxes_match_the_oracle also
compares every box of a batch with its own oracle directly.
"""
import math

import numpy as np
import pytest

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


def box_fields(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    R = 0.25 * min(nx, ny, nz) * (1 + rng.uniform(-0.2, 0.2))
    c = (rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz))
    phi = inputs.droplet(nx, ny, nz, R, 3.0, center=c)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.stack([0.01 * np.sin(2 * np.pi * (y / ny + rng.uniform())),
                  0.01 * np.cos(2 * np.pi * (z / nz + rng.uniform())),
                  0.01 * np.sin(2 * np.pi * (x / nx + rng.uniform()))])
    return inputs.to_f32(phi), inputs.to_f32(u)


@pytest.mark.parametrize("dims", [
    [(32, 32, 32), (24, 24, 24), (48, 40, 36), (64, 16, 20), (8, 8, 8)],    # every nx % 4 == 0: float4 phase A
    [(32, 32, 32), (37, 13, 11), (24, 24, 24)],                              # a ragged nx: per-site phase A
])
@pytest.mark.parametrize("storage", ["f32", "f16", "moments"])
def test_batch_boxes_equal_single_boxes(lbgb, dims, storage):
    tau = [0.8, 1.0, 0.6, 0.9, 0.7][: len(dims)]
    sigma = [0.01, 0.005, 0.02, 0.015, 0.01][: len(dims)]
    fields = [box_fields(*d, seed=k) for k, d in enumerate(dims)]
    batch = lbgb.Batch(dims, tau, 0.1, 3.0, sigma, storage=storage)
    # FP16 with every nx % 4 == 0 runs the paired body by default
    paired = storage == "f16" and all(d[0] % 4 == 0 for d in dims)
    assert batch.paired == paired
    if storage == "f16" and not paired:
        with pytest.raises(lbgb.LBError):
            batch.set_pairing(True)
    with pytest.raises(lbgb.LBError):
        batch.set_pairing(16)  # widths are 64 and 32
    batch.set_tile(4, 16)
    for k, (phi, u) in enumerate(fields):
        batch.init(k, phi, u)
    batch.step(7)  # three graph pairs and one single step
    assert batch.time == 7
    for k, (d, (phi, u)) in enumerate(zip(dims, fields)):
        box = lbgb.Box(*d, tau[k], 0.1, 3.0, sigma[k], storage=storage)
        if storage in ("f16", "bf16"):
            box.set_pairing(paired)  # the same tile body as the batch
        box.set_tile(4, 16)
        box.init(phi, u)
        box.step(7)
        for a, b in zip(box.moments_numpy(), batch.moments_numpy(k)):
            assert np.array_equal(a, b), (k, d)
        np.testing.assert_array_equal(box.diagnostics()[:4], batch.diagnostics(k)[:4])
        box.close()
    batch.close()


@pytest.mark.parametrize("dims", [
    [(32, 24, 20), (24, 24, 24), (16, 40, 12), (8, 8, 8), (48, 16, 9)],     # every nx % 4 == 0: float4 phase A
    [(32, 24, 20), (37, 13, 11), (24, 24, 24), (13, 9, 30), (5, 7, 3)],     # ragged nx: per-site phase A
])
@pytest.mark.parametrize("storage", ["f32", "moments"])
def test_batch_boxes_match_the_oracle(lbgb, orc, dims, storage):
    """Five boxes of uneven sizes with their own tau and sigma, advanced 50 steps
    by the persistent batch kernel (graph pairs and a last single step), each
    against its own FP64 oracle: max|delta| <= 1e-5 in p*, u and phi, and the
    per-box FP64 reductions within the bounds the field error gives."""
    from test_gpu_parity import TOL, check_diagnostics, max_err

    tau = [0.8, 1.0, 0.6, 0.9, 0.7]
    sigma = [0.01, 0.005, 0.02, 0.015, 0.01]
    fields = [box_fields(*d, seed=20 + k) for k, d in enumerate(dims)]
    batch = lbgb.Batch(dims, tau, 0.1, 3.0, sigma, storage=storage)
    for k, (phi, u) in enumerate(fields):
        batch.init(k, phi, u)
    batch.step(49)
    batch.step(1)
    assert batch.time == 50
    for k, (d, (phi, u)) in enumerate(zip(dims, fields)):
        o = orc.Oracle(*d, tau[k], 0.1, 3.0, sigma[k])
        o.init(phi.astype(np.float64), u.astype(np.float64))
        o.step(50)
        e = max_err(batch.moments_numpy(k), o.moments())
        assert max(e) <= TOL, (k, d, e)
        dg, do = batch.diagnostics(k), o.diagnostics()
        check_diagnostics(dg, do, int(np.prod(d)), field_err=max(e), tau=tau[k])
        o.close()
    batch.close()


@pytest.mark.parametrize("storage", ["f32", "moments", "f16"])
def test_batch_with_density_contrasts_matches_the_oracle(lbgb, orc, storage):
    """Four boxes with their own density and viscosity contrasts (heavy droplets
    at ratios 10 and 100, a light one at 1/10, and ratio 1), one persistent
    launch per step, 50 steps: each box against its own FP64 oracle with the
    same contrasts within 1e-5, and its reductions within the derived bounds.
    FP16 runs the paired tile body with contrasts, within its 2e-4 bound."""
    from test_gpu_parity import TOL, check_diagnostics, max_err

    dims = [(32, 24, 20), (24, 24, 24), (16, 40, 12), (36, 12, 16)]
    tau = [0.8, 1.0, 0.6, 0.9]
    sigma = [0.01, 0.005, 0.02, 0.015]
    dens = [(10.0, 1.0, 0.6, 0.8), (100.0, 1.0, 0.8, 0.8), (1.0, 10.0, 1.0, 0.6), (1.0, 1.0, 0.7, 0.7)]
    fields = [box_fields(*d, seed=40 + k) for k, d in enumerate(dims)]
    batch = lbgb.Batch(dims, tau, 0.1, 3.0, sigma, storage=storage)
    batch.set_density(*[[dd[j] for dd in dens] for j in range(4)])
    assert batch.paired == (storage == "f16")
    for k, (phi, u) in enumerate(fields):
        batch.init(k, phi, u)
    batch.step(50)
    for k, (d, (phi, u)) in enumerate(zip(dims, fields)):
        o = orc.Oracle(*d, tau[k], 0.1, 3.0, sigma[k])
        o.set_density(*dens[k])
        o.init(phi.astype(np.float64), u.astype(np.float64))
        o.step(50)
        e = max_err(batch.moments_numpy(k), o.moments())
        if storage == "f16":
            assert max(e) <= 2e-4, (k, d, e)
            o.close()
            continue
        assert max(e) <= TOL, (k, d, e)
        check_diagnostics(batch.diagnostics(k), o.diagnostics(), int(np.prod(d)), field_err=max(e),
                          tau=dens[k][2:])
        o.close()
    with pytest.raises(lbgb.LBError) as ex:
        batch.set_density([1.0] * 4, [0.0] * 4, [1.0] * 4, [1.0] * 4)
    assert ex.value.code == lbgb.LB_EINVAL
    batch.close()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_batch_paired_matches_the_oracle(lbgb, orc, storage):
    """16-bit storages run the paired tile body (two sites per thread, tiles 64
    or 32 sites wide) in the persistent batch kernel: five boxes with nx % 4 == 0,
    one a single x tile of 8, one ragged at 36 and one two tiles wide at 100, 50
    steps, each against its own FP64 oracle within the 16-bit storage's bound
    (2e-4 FP16, 5e-3 BF16, as the single-box kernels), and within that bound of
    the one-site body's fields."""
    from test_gpu_pair import BOUND
    from test_gpu_parity import max_err

    dims = [(32, 24, 20), (8, 8, 8), (36, 12, 16), (100, 9, 7), (64, 16, 12)]
    tau = [0.8, 1.0, 0.6, 0.9, 0.7]
    sigma = [0.01, 0.005, 0.02, 0.015, 0.01]
    fields = [box_fields(*d, seed=60 + k) for k, d in enumerate(dims)]
    got = {}
    for pair in (64, 32, 0):
        batch = lbgb.Batch(dims, tau, 0.1, 3.0, sigma, storage=storage)
        batch.set_pairing(pair)
        batch.set_tile(4 if pair == 64 else 8, 16)
        assert batch.pair_width == pair
        for k, (phi, u) in enumerate(fields):
            batch.init(k, phi, u)
        batch.step(49)
        batch.step(1)
        got[pair] = [batch.moments_numpy(k) for k in range(len(dims))]
        batch.close()
    for k, (d, (phi, u)) in enumerate(zip(dims, fields)):
        o = orc.Oracle(*d, tau[k], 0.1, 3.0, sigma[k])
        o.init(phi.astype(np.float64), u.astype(np.float64))
        o.step(50)
        want = o.moments()
        es = max_err(got[0][k], want)
        for pw in (64, 32):
            ep = max_err(got[pw][k], want)
            assert max(ep) <= BOUND[storage], (pw, k, d, ep, es)
            dd = max_err(got[pw][k], [x.astype(np.float64) for x in got[0][k]])
            assert max(dd) <= BOUND[storage], (pw, k, d, dd)
        o.close()


def test_batch_call_order(lbgb):
    batch = lbgb.Batch([(16, 16, 16), (24, 8, 8)], 0.8, 0.1, 3.0, 0.01)
    phi, u = box_fields(16, 16, 16, 1)
    batch.init(0, phi, u)
    with pytest.raises(lbgb.LBError) as e:
        batch.step(1)
    assert e.value.code == lbgb.LB_ESTATE
    phi2, u2 = box_fields(24, 8, 8, 2)
    batch.init(1, phi2, u2)
    batch.step(1)
    with pytest.raises(lbgb.LBError) as e:
        batch.init(0, phi, u)
    assert e.value.code == lbgb.LB_ESTATE
    with pytest.raises(lbgb.LBError) as e:
        batch.tune(2)
    assert e.value.code == lbgb.LB_ESTATE


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_tune_then_run(lbgb, storage):
    dims = [(24, 24, 24), (32, 32, 32), (48, 48, 48)]
    batch = lbgb.Batch(dims, 1.0, 0.1, 3.0, 0.01, storage=storage)
    ty, zc = batch.tune(2)
    assert ty in (4, 8) and zc >= 1
    assert storage == "f16" or not batch.paired
    for k, d in enumerate(dims):
        batch.init(k, *box_fields(*d, seed=10 + k))
    batch.step(4)
    for k in range(len(dims)):
        rho, u, phi = batch.moments_numpy(k)
        assert np.isfinite(rho).all() and abs(rho.mean() - 1) < 1e-5


def test_ensemble_laplace_per_box(lbgb):
    """A small droplet ensemble drawn like the 512-box workload (edges 24-48, radius
    0.25 edge +-20%, sigma in [0.005, 0.02], tau = 1, M = 0.1, W = 3), 300 steps:
    every box holds a Laplace jump within 20% of 2 sigma / R (within 12% once R >= 8)."""
    specs = inputs.ensemble_specs(8, seed=4, edges=(24, 32, 48))
    dims = [(s["edge"],) * 3 for s in specs]
    batch = lbgb.Batch(dims, [s["tau"] for s in specs], [s["M"] for s in specs], [s["W"] for s in specs],
                       [s["sigma"] for s in specs])
    for k, s in enumerate(specs):
        e = s["edge"]
        batch.init(k, inputs.to_f32(inputs.droplet(e, e, e, s["R"], s["W"])), np.zeros((3, e, e, e), np.float32))
    batch.step(300)
    for k, s in enumerate(specs):
        e, R, W = s["edge"], s["R"], s["W"]
        rho, _, _ = batch.moments_numpy(k)
        c = (e - 1) / 2
        z, y, x = np.meshgrid(*[np.arange(e)] * 3, indexing="ij")
        d = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
        dp = (rho[d < max(R - 2 * W, 1.5)].mean() - rho[d > R + 2 * W].mean()) / 3
        rel = abs(dp / (2 * s["sigma"] / R) - 1)
        assert rel < (0.12 if R >= 8 else 0.20), (k, e, R, rel)
