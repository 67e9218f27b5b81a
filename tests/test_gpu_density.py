"""Parity of the CUDA path with density and viscosity contrasts (lb_set_density;
accLB Sec. 2.3: rho(phi), tau(phi), F^p, F^nu) with the FP64 oracle, through
the C ABI.

Bar: FP32 storage max|delta| <= 1e-5 in p*, u and phi after 50 steps, as for
the single-density step; the moment-only storage equals the FP32 populations
bit for bit; 16-bit storage states its error.  Cases: heavy and light droplets
with viscosity contrasts, ragged and degenerate boxes, the three forcing kinds,
forced turbulence with gas bubbles, the contrasts switched on mid-run (the
captured graph must be replaced), checkpoint/restart, the full 256^3 bubbly
workload, and layered shear against the 1D momentum equation.
"""
import math

import numpy as np
import pytest

from paper_2505_01126_gb300 import inputs

from test_gpu_parity import check_diagnostics, max_err, smooth_fields
from test_oracle_density import _phi_layers, _shear_reference

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def lbgb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_01126_gb300 import build

    build.build()
    from paper_2505_01126_gb300 import lbgb as mod

    return mod


def _lb_force(lbgb, force):
    return lbgb.Force(kind=force.get("force_kind", 0), g=force.get("g", (0, 0, 0)), A=force.get("A_abc", 0.0),
                      kf=force.get("kf", 0.0), K_target=force.get("K_target", 0.0),
                      T_relax=force.get("T_relax", 100.0))


def run_vd(lbgb, orc, shape, tau, M, W, sigma, phi, u, steps, dens, force=None, storage="f32", tile=None,
           oracle=True):
    """The same run on the GPU and (optionally) on the oracle: lb_set_density(dens)
    before lb_init, `steps` steps.  Returns (box, oracle, gpu fields, oracle fields)."""
    nz, ny, nx = shape
    force = force or {}
    b = lbgb.Box(nx, ny, nz, tau, M, W, sigma, force=_lb_force(lbgb, force), storage=storage)
    b.set_density(*dens)
    if tile is not None:
        b.set_tile(*tile)
    b.init(phi, u)
    b.step(steps)
    got = b.moments_numpy()
    o = want = None
    if oracle:
        o = orc.Oracle(nx, ny, nz, tau, M, W, sigma, **force)
        o.set_density(*dens)
        o.init(phi.astype(np.float64), u.astype(np.float64))
        o.step(steps)
        want = o.moments()
    return b, o, got, want


@pytest.mark.parametrize("dens", [(10.0, 1.0, 0.6, 1.0), (1.0, 10.0, 1.0, 0.6), (100.0, 1.0, 0.8, 0.8)])
def test_droplet_32_with_density_and_viscosity_contrast(lbgb, orc, dens):
    """32^3 droplet R = 8: heavy (ratio 10, tau 0.6 inside), light (ratio 1/10,
    tau 0.6 outside) and ratio 100; 50 steps."""
    w = inputs.static_droplet()
    b, o, got, want = run_vd(lbgb, orc, (32, 32, 32), w.tau, w.M, w.W, w.sigma, w.phi, w.u, 50, dens)
    e = max_err(got, want)
    assert max(e) <= TOL, e
    check_diagnostics(b.diagnostics(), o.diagnostics(), 32 ** 3, field_err=max(e), tau=dens[2:])


@pytest.mark.parametrize("shape", [(11, 13, 37), (5, 9, 70), (40, 3, 33), (2, 2, 2), (1, 1, 1), (3, 1, 5)])
def test_ragged_and_degenerate_boxes(lbgb, orc, shape):
    phi, u = smooth_fields(shape, sum(shape) + 5)
    b, o, got, want = run_vd(lbgb, orc, shape, 0.7, 0.1, 3.0, 0.02, phi, u, 50, (5.0, 1.0, 0.7, 0.9))
    e = max_err(got, want)
    assert max(e) <= TOL, e


@pytest.mark.parametrize("kind", ["const", "abc", "linear"])
def test_forcing_kinds(lbgb, orc, kind):
    """The external force is a force density (acceleration F/rho); with linear
    forcing the amplitude A follows eps summed over each site's own nu."""
    shape = (12, 20, 36)
    phi, u = smooth_fields(shape, 3)
    force = {"const": dict(force_kind=1, g=(1e-5, -2e-5, 5e-6)),
             "abc": dict(force_kind=2, A_abc=2e-5, kf=2 * math.pi / 12),
             "linear": dict(force_kind=3, T_relax=20.0)}[kind]
    b, o, got, want = run_vd(lbgb, orc, shape, 0.6, 0.1, 3.0, 0.01, phi, u, 50, (10.0, 1.0, 0.6, 0.8), force=force)
    e = max_err(got, want)
    assert max(e) <= TOL, e
    dg, do = b.diagnostics(), o.diagnostics()
    check_diagnostics(dg, do, int(np.prod(shape)), field_err=max(e), tau=(0.6, 0.8))
    if kind == "linear":
        assert abs(dg[4] - do[4]) <= 1e-5 * abs(do[4]) + 1e-9


def gas_bubbles(edge, n, R, seed):
    """Forced-turbulence surrogate with gas bubbles: the bubbly workload's phase
    field flipped (phi = 0 in the bubbles, the gas of Sec. 2.3's mixture law)."""
    w = inputs.bubbly_hit(edge, n, R, seed=seed)
    return w, inputs.to_f32(1.0 - w.phi.astype(np.float64))


def test_hit_64_heavy_droplets(lbgb, orc):
    """64^3 forced turbulence, two droplets R = 10 ten times denser than the
    carrier (tau 0.55 inside, 0.51 outside), linear forcing; 50 steps.  The bulk
    sits at phi = 0, so the full FP32 bar holds in every field."""
    w = inputs.bubbly_hit(64, 2, 10.0, seed=2)
    force = dict(force_kind=3, T_relax=w.T_relax)
    b, o, got, want = run_vd(lbgb, orc, (64, 64, 64), w.tau, w.M, w.W, w.sigma, w.phi, w.u, 50,
                             (10.0, 1.0, 0.55, 0.51), force=force)
    e = max_err(got, want)
    assert max(e) <= TOL, e
    check_diagnostics(b.diagnostics(), o.diagnostics(), 64 ** 3, field_err=max(e), tau=(0.55, 0.51))


def storage_rounded_oracle(orc, o):
    """One step of oracle `o` followed by rounding its state to what FP32
    storage keeps (f as the shifted population f/w - 1, g as is)."""
    _, wt = orc.lattice27()
    o.step(1)
    f, g = o.populations()
    w4 = wt[:, None, None, None]
    d = (f / w4 - 1.0).astype(np.float32).astype(np.float64)
    o.set_populations(w4 * (1.0 + d), g.astype(np.float32).astype(np.float64))


GAS_K = 4.0  # GPU error in phi at most GAS_K times the oracle's own storage-rounding spread


def test_hit_64_gas_bubbles(lbgb, orc):
    """64^3 forced turbulence (tau 0.51 in the liquid), two gas bubbles R = 10 at
    density ratio 10 and tau 0.55 in the gas (phi = 0 in the bubbles), linear
    forcing.  p* and u meet the FP32 bar after 50 steps; phi does after 10
    steps.  After 50 it does not: the liquid bulk sits at phi ~ 1, where FP32
    resolves phi to 6e-8 only, and on the nearly flat plateaus next to the bulk
    (phi (1 - phi) ~ 1e-2, |grad phi| ~ 1e-5) the normal grad phi / |grad phi|
    turns with that rounding, which the sharpening flux amplifies about 1.26x
    per step.  The bar for phi at 50 steps therefore comes from the method's
    own sensitivity: a second oracle run whose state is rounded to FP32 storage
    after every step (f as f/w - 1, g as is) departs from the plain oracle by a
    spread s; the GPU, which rounds its storage the same way and its arithmetic
    on top, must stay within GAS_K = 4 s of the plain oracle (measured: 2.1 s)."""
    w, phi = gas_bubbles(64, 2, 10.0, 2)
    force = dict(force_kind=3, T_relax=w.T_relax)
    dens = (1.0, 0.1, 0.51, 0.55)
    b, o, got, want = run_vd(lbgb, orc, (64, 64, 64), w.tau, w.M, w.W, w.sigma, phi, w.u, 10, dens, force=force)
    e = max_err(got, want)
    assert max(e) <= TOL, e
    b.step(40)
    o.step(40)
    got, want = b.moments_numpy(), o.moments()
    e = max_err(got, want)
    assert max(e[:2]) <= TOL, e
    check_diagnostics(b.diagnostics(), o.diagnostics(), 64 ** 3, delta=e[2], tau=dens[2:])
    r = orc.Oracle(64, 64, 64, w.tau, w.M, w.W, w.sigma, **force)
    r.set_density(*dens)
    r.init(phi.astype(np.float64), w.u.astype(np.float64))
    for _ in range(50):
        storage_rounded_oracle(orc, r)
    spread = max_err(r.moments(), want)
    r.close()
    assert 0.0 < spread[2] and e[2] <= GAS_K * spread[2], (e, spread)


@pytest.mark.parametrize("tile", [(4, 8), (8, 16), (8, 5)])
def test_moment_storage_equals_fp32_and_16bit_bounds(lbgb, orc, tile):
    """The moment-only storage rebuilds exactly the populations the FP32 storage
    stores, so with contrasts too the fields agree bit for bit (same tile); FP16
    and BF16 populations stay within their single-density error bounds."""
    shape = (20, 24, 44)
    phi, u = smooth_fields(shape, 11)
    dens = (10.0, 1.0, 0.6, 0.9)
    res = {}
    for st in ("f32", "moments", "f16", "bf16"):
        b, o, got, want = run_vd(lbgb, orc, shape, 0.7, 0.1, 3.0, 0.01, phi, u, 50, dens, storage=st, tile=tile,
                                 oracle=(st == "f32"))
        res[st] = got
        if st == "f32":
            ref = want
        b.close()
    for a, c in zip(res["f32"], res["moments"]):
        assert np.array_equal(a, c)
    assert max(max_err(res["f32"], ref)) <= TOL
    assert max(max_err(res["f16"], ref)) <= 2e-4, max_err(res["f16"], ref)
    assert max(max_err(res["bf16"], ref)) <= 5e-3, max_err(res["bf16"], ref)


def test_ratio_one_is_the_single_density_step(lbgb):
    """rho_l = rho_g = 1, tau_l = tau_g = tau: the contrast kernel computes the
    single-density step up to the rounding of omega (1/tau taken in FP32 on the
    device instead of FP64 on the host)."""
    shape = (16, 24, 40)
    phi, u = smooth_fields(shape, 4)
    out = []
    for vd in (False, True):
        b = lbgb.Box(40, 24, 16, 0.7, 0.1, 3.0, 0.01)
        if vd:
            b.set_density(1.0, 1.0, 0.7, 0.7)
        b.init(phi, u)
        b.step(30)
        out.append(b.moments_numpy())
        b.close()
    assert max(max_err(out[1], [x.astype(np.float64) for x in out[0]])) <= 1e-6


def test_contrast_switched_on_mid_run(lbgb, orc):
    """10 single-density steps (a captured graph), then lb_set_density and 20
    more: the new kernel must replace the captured launches."""
    shape = (12, 16, 40)
    phi, u = smooth_fields(shape, 8)
    b = lbgb.Box(40, 16, 12, 0.8, 0.1, 3.0, 0.01)
    b.init(phi, u)
    b.step(10)
    b.set_density(10.0, 1.0, 0.6, 0.8)
    b.step(20)
    got = b.moments_numpy()
    o = orc.Oracle(40, 16, 12, 0.8, 0.1, 3.0, 0.01)
    o.init(phi.astype(np.float64), u.astype(np.float64))
    o.step(10)
    o.set_density(10.0, 1.0, 0.6, 0.8)
    o.step(20)
    e = max_err(got, o.moments())
    assert max(e) <= TOL, e


@pytest.mark.parametrize("storage", ["f32", "moments"])
def test_checkpoint_restart_with_contrast(lbgb, storage):
    """A checkpoint holds the state; the loading context sets the same contrasts
    and then continues bit for bit as the uninterrupted run."""
    shape = (12, 16, 40)
    phi, u = smooth_fields(shape, 9)
    dens = (10.0, 1.0, 0.6, 0.8)
    a = lbgb.Box(40, 16, 12, 0.8, 0.1, 3.0, 0.01, storage=storage)
    a.set_density(*dens)
    a.init(phi, u)
    a.step(15)
    buf = a.save()
    a.step(20)
    want = a.moments_numpy()
    c = lbgb.Box(40, 16, 12, 0.8, 0.1, 3.0, 0.01, storage=storage)
    c.set_density(*dens)
    c.load(buf)
    c.step(20)
    for x, y in zip(c.moments_numpy(), want):
        assert np.array_equal(x, y)


def test_checkpoint_with_other_contrast_settings_is_rejected(lbgb):
    """A checkpoint records the density, viscosity and gravity settings it was
    stepped with; a context without them, or with other values, refuses it."""
    shape = (8, 8, 12)
    phi, u = smooth_fields(shape, 4)
    a = lbgb.Box(12, 8, 8, 0.8, 0.1, 3.0, 0.01)
    a.set_density(10.0, 1.0, 0.6, 0.8)
    a.set_gravity((0.0, 0.0, -1e-5), 2.0)
    a.init(phi, u)
    a.step(3)
    buf = a.save()
    plain = lbgb.Box(12, 8, 8, 0.8, 0.1, 3.0, 0.01)
    other = lbgb.Box(12, 8, 8, 0.8, 0.1, 3.0, 0.01)
    other.set_density(10.0, 1.0, 0.6, 0.8)  # no gravity
    for c in (plain, other):
        with pytest.raises(lbgb.LBError) as e:
            c.load(buf)
        assert e.value.code == lbgb.LB_EINVAL
    same = lbgb.Box(12, 8, 8, 0.8, 0.1, 3.0, 0.01)
    same.set_density(10.0, 1.0, 0.6, 0.8)
    same.set_gravity((0.0, 0.0, -1e-5), 2.0)
    same.load(buf)
    assert same.time == 3
    # a checkpoint without contrasts does not load into a context with them
    b = lbgb.Box(12, 8, 8, 0.8, 0.1, 3.0, 0.01)
    b.init(phi, u)
    with pytest.raises(lbgb.LBError) as e:
        same.load(b.save())
    assert e.value.code == lbgb.LB_EINVAL
    for x in (a, plain, other, same, b):
        x.close()


def test_set_density_rejects_bad_parameters(lbgb):
    b = lbgb.Box(8, 8, 8, 1.0, 0.1, 3.0, 0.01)
    for bad in ((0.0, 1.0, 1.0, 1.0), (1.0, -1.0, 1.0, 1.0), (1.0, 1.0, 0.5, 1.0), (1.0, 1.0, 1.0, 0.4),
                (float("nan"), 1.0, 1.0, 1.0), (float("inf"), 1.0, 1.0, 1.0)):
        with pytest.raises(lbgb.LBError) as e:
            b.set_density(*bad)
        assert e.value.code == lbgb.LB_EINVAL
    b.close()


def test_layered_shear_ratio_100(lbgb):
    """Layers at density ratio 100 under a uniform body force on the device follow
    rho dw/dt = d/dx(rho nu dw/dx) + g to the oracle's 4.1% (the model without
    F^nu is 2.4 off)."""
    nx, ny, W, x0, x1, g, T = 64, 4, 4.0, 16.0, 48.0, 1e-6, 3000
    ph = _phi_layers(np.arange(nx, dtype=np.float64), nx, W, x0, x1)
    phi = inputs.to_f32(np.broadcast_to(ph[None, None, :], (ny, ny, nx)))
    b = lbgb.Box(nx, ny, ny, 1.0, 0.1, W, 0.0, force=lbgb.Force(kind=1, g=(0.0, 0.0, g)))
    b.set_density(100.0, 1.0, 1.0, 1.0)
    b.init(phi, np.zeros((3, ny, ny, nx), np.float32))
    b.step(T)
    _, u, _ = b.moments_numpy()
    ref = _shear_reference(nx, W, x0, x1, 100.0, 1.0, 1.0, 1.0, g, T)
    err = np.abs(u[2, 0, 0].astype(np.float64) - ref).max() / np.abs(ref).max()
    assert err < 0.06, err
    assert np.abs(u[:2]).max() < 1e-9


def test_full_size_256_gas_bubbles_one_step_each_parity(lbgb, orc):
    """The benchmark's 256^3 bubbly workload with gas bubbles at density ratio 10
    (tau 0.51 liquid, 0.55 gas), in the benchmark's launch shape after lb_tune:
    2 steps, every site compared with the oracle."""
    w, phi = gas_bubbles(256, 64, 10.0, 2)
    n = 256
    b = lbgb.Box(n, n, n, w.tau, w.M, w.W, w.sigma, force=lbgb.Force(kind=3, T_relax=w.T_relax))
    b.set_density(1.0, 0.1, 0.51, 0.55)
    b.tune(2)
    b.init(phi, w.u)
    b.step(2)
    got = b.moments_numpy()
    dg = b.diagnostics()
    b.close()
    o = orc.Oracle(n, n, n, w.tau, w.M, w.W, w.sigma, force_kind=3, T_relax=w.T_relax)
    o.set_density(1.0, 0.1, 0.51, 0.55)
    o.init(phi.astype(np.float64), w.u.astype(np.float64))
    o.step(2)
    want = o.moments()
    do = o.diagnostics()
    o.close()
    e = max_err(got, want)
    assert max(e) <= TOL, e
    check_diagnostics(dg, do, n ** 3, field_err=max(e), tau=(0.51, 0.55))


def test_gas_bubbles_64_stay_finite_for_400_steps(lbgb):
    """Forced turbulence with gas bubbles at ratio 10 runs stably (no NaN or Inf,
    phase conserved to FP32 rounding) over 400 steps."""
    w, phi = gas_bubbles(64, 2, 10.0, 2)
    b = lbgb.Box(64, 64, 64, w.tau, w.M, w.W, w.sigma, force=lbgb.Force(kind=3, T_relax=w.T_relax))
    b.set_density(1.0, 0.1, 0.51, 0.55)
    b.init(phi, w.u)
    d0 = b.diagnostics()
    b.step(400)
    d = b.diagnostics()
    assert np.isfinite(d).all()
    assert abs(d[0] - d0[0]) <= 1e-4 * abs(d0[0])
    assert d[3] < 0.2


def test_paper_droplet_case_256_full_parity(lbgb, orc):
    """The paper's two-component benchmark recipe (one heavier droplet, density
    ratio 100, nu = 0.005 in both phases) at 256^3 with R = 64, in the tuned
    launch shape: 2 steps, every site compared with the oracle."""
    import bench

    n = 256
    w = bench.droplet_workload(n)
    dens = bench.DROPLET_DENSITY
    b = lbgb.Box(n, n, n, w.tau, w.M, w.W, w.sigma)
    b.set_density(*dens)
    b.tune(2)
    b.init(w.phi, w.u)
    b.step(2)
    got = b.moments_numpy()
    dg = b.diagnostics()
    b.close()
    o = orc.Oracle(n, n, n, w.tau, w.M, w.W, w.sigma)
    o.set_density(*dens)
    o.init(w.phi.astype(np.float64), w.u.astype(np.float64))
    o.step(2)
    want = o.moments()
    do = o.diagnostics()
    o.close()
    e = max_err(got, want)
    assert max(e) <= TOL, e
    check_diagnostics(dg, do, n ** 3, field_err=max(e), tau=dens[2:])


def test_paper_droplet_case_512_properties(lbgb):
    """The benchmark's own 512^3 box (R = 128) in the tuned launch shape, 20 steps:
    finite, phase mass conserved to FP32 rounding, and the droplet's mirror
    symmetries about the box centre kept to 1e-6 in every field (the tiles and
    z-chunks of the launch do not break them)."""
    import bench

    n = 512
    w = bench.droplet_workload(n)
    b = lbgb.Box(n, n, n, w.tau, w.M, w.W, w.sigma)
    b.set_density(*bench.DROPLET_DENSITY)
    b.tune(2)
    b.init(w.phi, w.u)
    d0 = b.diagnostics()
    b.step(20)
    d = b.diagnostics()
    rho, u, phi = b.moments_numpy()
    b.close()
    assert np.isfinite(d).all()
    assert abs(d[0] - d0[0]) <= 1e-6 * d0[0]
    for axis in range(3):
        assert np.abs(phi - np.flip(phi, axis)).max() <= 1e-6
        assert np.abs(rho - np.flip(rho, axis)).max() <= 1e-6
        # u is odd under the mirror along its own axis, even along the others
        for a in range(3):
            s = -1.0 if a == 2 - axis else 1.0
            assert np.abs(u[a] - s * np.flip(u[a], axis)).max() <= 1e-6


# ---------------------------------------------------------------- buoyancy
def _mean_rho(phi, rho_l, rho_g):
    return float(rho_g + (rho_l - rho_g) * phi.astype(np.float64).mean())


@pytest.mark.parametrize("storage", ["f32", "moments"])
def test_buoyant_droplet_32(lbgb, orc, storage):
    """A heavy droplet (ratio 10, tau 0.6 inside) sinking under gravity
    (0, 0, -1e-5) with rho_ref the mean density: 50 steps against the oracle."""
    w = inputs.static_droplet()
    dens = (10.0, 1.0, 0.6, 1.0)
    rr = _mean_rho(w.phi, 10.0, 1.0)
    b = lbgb.Box(32, 32, 32, w.tau, w.M, w.W, w.sigma, storage=storage)
    b.set_density(*dens)
    b.set_gravity((0.0, 0.0, -1e-5), rr)
    b.init(w.phi, w.u)
    b.step(50)
    got = b.moments_numpy()
    o = orc.Oracle(32, 32, 32, w.tau, w.M, w.W, w.sigma)
    o.set_density(*dens)
    o.set_gravity((0.0, 0.0, -1e-5), rr)
    o.init(w.phi.astype(np.float64), w.u.astype(np.float64))
    o.step(50)
    e = max_err(got, o.moments())
    assert max(e) <= TOL, e
    assert float(np.abs(got[1][2]).max()) > 1e-5  # the droplet does move
    check_diagnostics(b.diagnostics(), o.diagnostics(), 32 ** 3, field_err=max(e), tau=dens[2:])


def test_buoyant_turbulence_64_heavy_droplets(lbgb, orc):
    """64^3 forced turbulence with two heavy droplets (ratio 10) under gravity
    along -y, linear forcing; 50 steps."""
    w = inputs.bubbly_hit(64, 2, 10.0, seed=2)
    dens = (10.0, 1.0, 0.55, 0.51)
    rr = _mean_rho(w.phi, 10.0, 1.0)
    force = dict(force_kind=3, T_relax=w.T_relax)
    b = lbgb.Box(64, 64, 64, w.tau, w.M, w.W, w.sigma, force=_lb_force(lbgb, force))
    b.set_density(*dens)
    b.set_gravity((0.0, -2e-6, 0.0), rr)
    b.init(w.phi, w.u)
    b.step(50)
    o = orc.Oracle(64, 64, 64, w.tau, w.M, w.W, w.sigma, **force)
    o.set_density(*dens)
    o.set_gravity((0.0, -2e-6, 0.0), rr)
    o.init(w.phi.astype(np.float64), w.u.astype(np.float64))
    o.step(50)
    e = max_err(b.moments_numpy(), o.moments())
    assert max(e) <= TOL, e
    check_diagnostics(b.diagnostics(), o.diagnostics(), 64 ** 3, field_err=max(e), tau=dens[2:])


def test_gravity_switched_on_mid_run(lbgb, orc):
    shape = (12, 16, 40)
    phi, u = smooth_fields(shape, 21)
    dens = (10.0, 1.0, 0.7, 0.9)
    rr = _mean_rho(phi, 10.0, 1.0)
    b = lbgb.Box(40, 16, 12, 0.8, 0.1, 3.0, 0.01)
    b.set_density(*dens)
    b.init(phi, u)
    b.step(10)
    b.set_gravity((3e-6, 0.0, -1e-5), rr)
    b.step(20)
    o = orc.Oracle(40, 16, 12, 0.8, 0.1, 3.0, 0.01)
    o.set_density(*dens)
    o.init(phi.astype(np.float64), u.astype(np.float64))
    o.step(10)
    o.set_gravity((3e-6, 0.0, -1e-5), rr)
    o.step(20)
    e = max_err(b.moments_numpy(), o.moments())
    assert max(e) <= TOL, e


def test_counter_current_layers_on_the_device(lbgb):
    """Gravity along layers at ratio 100 on the device: within 7% of the 1D
    momentum equation with the force density (rho - rho_ref) g."""
    nx, ny, W, x0, x1, g, T = 64, 4, 4.0, 16.0, 48.0, -1e-6, 3000
    ph = _phi_layers(np.arange(nx, dtype=np.float64), nx, W, x0, x1)
    phi = inputs.to_f32(np.broadcast_to(ph[None, None, :], (ny, ny, nx)))
    rr = float((1.0 + ph * 99.0).mean())
    b = lbgb.Box(nx, ny, ny, 1.0, 0.1, W, 0.0)
    b.set_density(100.0, 1.0, 1.0, 1.0)
    b.set_gravity((0.0, 0.0, g), rr)
    b.init(phi, np.zeros((3, ny, ny, nx), np.float32))
    b.step(T)
    _, u, _ = b.moments_numpy()
    ref = _shear_reference(nx, W, x0, x1, 100.0, 1.0, 1.0, 1.0, 0.0, T, force=lambda r: (r - rr) * g)
    err = np.abs(u[2, 0, 0].astype(np.float64) - ref).max() / np.abs(ref).max()
    assert err < 0.07, err


def test_set_gravity_errors(lbgb):
    b = lbgb.Box(8, 8, 8, 1.0, 0.1, 3.0, 0.01)
    with pytest.raises(lbgb.LBError) as e:
        b.set_gravity((0.0, 0.0, -1e-5), 1.0)
    assert e.value.code == lbgb.LB_ESTATE
    b.set_density(2.0, 1.0, 1.0, 1.0)
    b.set_gravity((0.0, 0.0, -1e-5), 1.5)
    with pytest.raises(lbgb.LBError) as e:
        b.set_gravity((0.0, float("nan"), 0.0), 1.5)
    assert e.value.code == lbgb.LB_EINVAL
    b.close()
