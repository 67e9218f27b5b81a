#!/usr/bin/env python3
"""Benchmark of the fused two-phase lattice Boltzmann step on GB300.

Workload (default, preset hit512): 512^3 periodic bubble-laden forced
homogeneous isotropic turbulence with 256 bubbles of radius 12 (seed 3,
non-overlapping), interface width W = 3, sigma = 0.01, tau = 0.51, M = 0.1,
solenoidal initial velocity from Fourier modes 1 <= |k| <= 4 with
u_rms = 0.02, linear forcing holding the kinetic energy.  The box runs twice
in one invocation: with FP32 population storage (the line's value) and with
FP16 shifted storage (the line's storage16 object); the errors of both
storages against the FP64 oracle (kinetic energy, phase-mass drift, fields,
Laplace pressure jump) are measured on the 64^3 surrogate of the same recipe
and the 32^3 static droplet, whose oracle runs are the CPU baseline.  A
"step" is one full time step of the box (the fused kernel plus the FP64
reduction).  The metric is MLUPS (million lattice-site updates per second,
the paper's GLUPS x 1000) and the fraction of the measured HBM bandwidth
reached by the fused kernel.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--preset hit256|hit512|hit768|hit1024]
                       [--storage f32|f16|bf16|moments|f16g|bf16g] [--compare f16|bf16|f16g|bf16g|none]
                       [--workload hit|ensemble|droplet|abc] [--edge E]
                       [--density RHO_L RHO_G TAU_L TAU_G] [--gravity GX,GY,GZ]
                       [--phase lb|weno5]
--density runs the same box with density and viscosity contrasts (Sec. 2.3):
the bubbles become the gas (phi = 0 inside, phi flipped), the liquid phi = 1.
--gravity adds the buoyancy (rho(phi) - rho_ref) g with rho_ref the mean density.
--phase weno5 advances the phase field by finite differences (WENO-5, SSP-RK3).
Under torchrun (N > 1) every rank advances its own replica box (weak scaling,
no collective on the data path); value = sum of sites*steps over ranks divided
by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2505_01126_gb300 import inputs  # noqa: E402

METRIC = "two-phase MLUPS & % HBM roofline, FP32 vs 16-bit storage at stated error"
UNIT = "MLUPS"
# the oracle's sample for the CPU baseline of the workloads other than the
# bubbly HIT comparison: a 128^3 box of the same recipe, 10 steps
SAMPLE_EDGE, SAMPLE_STEPS = 128, 10
# the reference arm's per-step sample: 64^3 box of the same recipe (1 bubble)
REF_EDGE = 64
# the cases the storages' errors are stated on: the 64^3 surrogate of the bubbly
# HIT preset (K every 50 steps for 500 steps) and the 32^3 static droplet R = 8
# (Laplace pressure jump averaged over steps 220-400)
SURR_EDGE, SURR_STEPS, SURR_EVERY = 64, 500, 50
LAP_EDGE, LAP_R, LAP_SAMPLES = 32, 8.0, list(range(220, 401, 20))
# bytes per site and step when a stored FP32 phi field is also written and
# re-read (8 B/site); the f16g/bf16g kernels keep a 16-bit phi~ (4 B/site) of their own
PHI_STORED_BYTES = {"f32": 280.0, "f16": 172.0, "bf16": 172.0, "f16g": 144.0, "bf16g": 144.0}


# Presets of the bubbly forced HIT workload: edge, bubbles, radius, tau, seed.
PRESETS = {
    "hit256": (256, 64, 10.0, 0.51, 2),     # 256^3, 64 bubbles R = 10, FP32
    "hit512": (512, 256, 12.0, 0.51, 3),    # 512^3, 256 bubbles R = 12, FP32 and 16-bit (the default)
    "hit768": (768, 864, 12.0, 0.505, 5),   # FP32 comparison box for hit1024 (same bubble fraction)
    "hit1024": (1024, 2048, 12.0, 0.505, 5),  # 1024^3, 2048 bubbles R = 12, 16-bit storage
}
DEFAULT_PRESET = "hit512"


# The paper's two-component benchmark case (Sec. 4): one droplet of the heavier
# phase at density contrast 100 in a lighter carrier, kinematic viscosity 0.005
# (tau = 0.515) in both phases, 512^3 per GPU.  The radius, W, sigma and M are
# not given: R = edge/4, W = 3, sigma = 0.01, M = 0.1, zero initial velocity.
DROPLET_EDGE, DROPLET_TAU, DROPLET_DENSITY = 512, 0.515, (100.0, 1.0, 0.515, 0.515)


# Single-phase forced HIT (Sec. 5.1): ABC forcing, no interface (phi = 0
# everywhere, sigma = 0), 512^3, the seeded solenoidal start of the bubbly
# workload.  The paper gives neither the amplitude nor k_f: A = 2e-6,
# k_f = 2 pi / edge (one forcing period per box), tau = 0.51.
ABC_EDGE, ABC_TAU, ABC_A, ABC_SEED = 512, 0.51, 2e-6, 7


def abc_workload(edge: int):
    if edge >= 384:
        return inputs.bubbly_hit_device(edge, 0, 1.0, seed=ABC_SEED, tau=ABC_TAU, sigma=0.0, force_kind=2)
    return inputs.bubbly_hit(edge, 0, 1.0, seed=ABC_SEED, tau=ABC_TAU, sigma=0.0, force_kind=2)


def droplet_workload(edge: int):
    return inputs.static_droplet(edge=edge, R=edge / 4.0, tau=DROPLET_TAU)


def workload(edge: int, preset: str = DEFAULT_PRESET):
    """An edge^3 sample of a bubbly HIT preset: its generator, seed, radius and tau,
    with the bubble count scaled to the same volume fraction (at least one)."""
    full, nb_full, R, tau, seed = PRESETS[preset]
    nb = max(1, round(nb_full * (edge / full) ** 3))
    return inputs.bubbly_hit(edge, nb, R, seed=seed, tau=tau), nb


def preset_workload(name: str):
    """Workload and bubble count of a preset; large boxes are generated on the device."""
    edge, nb, R, tau, seed = PRESETS[name]
    if edge >= 384:
        return inputs.bubbly_hit_device(edge, nb, R, seed=seed, tau=tau), nb
    return inputs.bubbly_hit(edge, nb, R, seed=seed, tau=tau), nb


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def whole_job(ms_local: float, sites_per_rank: int, steps: int, world: int, dist=None):
    """Whole-job MLUPS over `world` replica ranks: the slowest rank's time (max over
    ranks, via an all-reduce when `dist` is a torch.distributed module with an
    initialised group) divides the sites all ranks updated.  Returns (MLUPS, t_max_ms)."""
    t_max = float(ms_local)
    if dist is not None and world > 1:
        import torch

        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([t_max], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return sites_per_rank * steps * world / (t_max * 1e-3) / 1e6, t_max


def measured_traffic(storage: str, n_sites: int, tile=None):
    """DRAM bytes per fused-kernel launch from the committed ncu record, scaled to
    n_sites, or None if the kernel sources changed since the capture or the
    capture was taken in another launch shape (tile width, height and
    z-chunk; a capture on a smaller box of the same shape scales by the sites)."""
    try:
        import hashlib

        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["kernel_sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != rec["kernel_sources_sha256"] or storage not in rec["captures"]:
            return None
        cap = rec["captures"][storage]
        if tile is not None and list(cap["tile"]) != list(tile):
            return None
        return cap["bytes_per_site"] * n_sites
    except Exception:
        return None


def measured_inst_per_site(storage: str, tile=None):
    """Warp-instructions per site of the fused kernel from the committed ncu
    record (same conditions as measured_traffic), or None."""
    try:
        import hashlib

        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["kernel_sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        cap = rec["captures"].get(storage)
        if h.hexdigest() != rec["kernel_sources_sha256"] or cap is None:
            return None
        if tile is not None and list(cap["tile"]) != list(tile):
            return None
        return cap.get("warp_inst_per_site")
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(n: int, kind: str = "hit", density=None, gravity=None, phase: str = "lb",
                  preset: str = DEFAULT_PRESET):
    """The oracle (as it stands) initialised on an n^3 sample of the benchmark's
    workload with its options, as the GPU arm builds it: the bubbly HIT recipe
    (its bubbles flipped to gas at phi = 0 when density contrasts are given),
    the two-component droplet, or the single-phase ABC HIT.  Returns the oracle
    and a description of the sample."""
    import oracle

    oracle.build()
    if kind == "abc":
        w = abc_workload(n)
        o = oracle.Oracle(n, n, n, w.tau, w.M, w.W, w.sigma, force_kind=oracle.FORCE_ABC, A_abc=ABC_A,
                          kf=2 * math.pi / n)
        desc = f"single phase, ABC forcing k_f = 2 pi/{n}"
    elif kind == "droplet":
        w = droplet_workload(n)
        o = oracle.Oracle(n, n, n, w.tau, w.M, w.W, w.sigma)
        density = DROPLET_DENSITY
        desc = f"droplet R={n / 4:g}, density ratio 100, tau 0.515"
    else:
        w, nb = workload(n, preset)
        o = oracle.Oracle(n, n, n, w.tau, w.M, w.W, w.sigma, force_kind=oracle.FORCE_LINEAR, T_relax=w.T_relax)
        desc = (f"{nb} bubble{'s' if nb != 1 else ''} R={PRESETS[preset][2]:g}, u_rms 0.02, tau {w.tau:g}, "
                f"linear forcing")
    phi = w.phi.astype(np.float64)
    o.set_phase_solver(phase)
    if density:
        o.set_density(*density)
        if kind != "droplet":
            phi = 1.0 - phi  # the gas at phi = 0, as the GPU arm does
        desc += ", density contrasts"
        if gravity:
            o.set_gravity(gravity, density[1] + (density[0] - density[1]) * float(phi.mean()))
            desc += ", buoyancy"
    if phase != "lb":
        desc += ", WENO-5 phase field"
    o.init(phi, w.u.astype(np.float64))
    return o, desc


def cpu_baseline_sample(kind: str = "hit", density=None, gravity=None, phase: str = "lb",
                        preset: str = DEFAULT_PRESET):
    """Time the oracle (as it stands) on a bounded sample of the workload:
    SAMPLE_STEPS steps of a SAMPLE_EDGE^3 box after one untimed step."""
    import oracle

    n = SAMPLE_EDGE
    o, desc = oracle_sample(n, kind, density, gravity, phase, preset)
    o.step(1)  # first touch of the arrays
    t0 = time.perf_counter()
    o.step(SAMPLE_STEPS)
    dt = time.perf_counter() - t0
    o.close()
    return {"value": n ** 3 * SAMPLE_STEPS / dt / 1e6, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{n}^3 box of the same recipe ({desc}), {SAMPLE_STEPS} FP64 oracle steps after 1 untimed "
                      f"step, {dt:.1f} s"}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, each step one oracle step of
    the REF_EDGE^3 (64^3) sample of the workload and options the GPU arm runs (the
    ensemble's arm times the bubbly sample)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    kind = getattr(args, "workload", "hit")
    kind = kind if kind in ("droplet", "abc") else "hit"
    n = REF_EDGE
    preset = getattr(args, "preset", DEFAULT_PRESET) or DEFAULT_PRESET
    o, desc = oracle_sample(n, kind, getattr(args, "density", None), getattr(args, "gravity", None),
                            getattr(args, "phase", "lb"), preset)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    o.close()
    value = n ** 3 * args.steps / dt / 1e6
    sample = f"{n}^3 box of the same recipe ({desc}), one FP64 oracle step per bench step"
    pe, pnb, pR, ptau, pseed = PRESETS[preset]
    full = {"hit": f"the {pe}^3 periodic bubbly forced HIT workload ({pnb} bubbles R={pR:g}, W=3, sigma=0.01, "
                   f"tau={ptau:g}, M=0.1, u_rms=0.02, linear forcing, seed {pseed})",
            "droplet": "the 512^3 two-component droplet case (density ratio 100, nu 0.005)",
            "abc": "the 512^3 single-phase ABC-forced HIT"}[kind]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{n}^3 sample of {full}: {desc}", "edge": n, "storage": "f64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ensemble(args):
    """512 independent periodic droplet boxes (edges uniform in {24,32,48,64,96},
    R = 0.25 edge (1 +- 20%), sigma in [0.005, 0.02], tau 1, M 0.1, W 3, u = 0),
    advanced by one persistent launch per step under a CUDA graph with tuned
    tiles.  Reports MLUPS over all boxes and the per-box Laplace error."""
    import torch

    from paper_2505_01126_gb300 import build

    build.build()
    from paper_2505_01126_gb300 import lbgb

    specs = inputs.ensemble_specs(args.boxes, seed=4)
    dims = [(sp["edge"],) * 3 for sp in specs]
    stream = torch.cuda.Stream()
    batch = lbgb.Batch(dims, [sp["tau"] for sp in specs], [sp["M"] for sp in specs], [sp["W"] for sp in specs],
                       [sp["sigma"] for sp in specs], storage=args.storage, stream=stream)
    if args.density:  # every box with the same contrasts: droplets of the phase at phi = 1
        batch.set_density(*args.density)
    if args.pair_width is not None:
        batch.set_pairing(args.pair_width)
    if args.tile:
        batch.set_tile(*args.tile)
        ty, zc = batch.tile()
    else:
        ty, zc = batch.tune(3)
    fields = {}
    for k, sp in enumerate(specs):
        e = sp["edge"]
        phi = inputs.to_f32(inputs.droplet(e, e, e, sp["R"], sp["W"]))
        fields[k] = phi
        batch.init(k, phi, np.zeros((3, e, e, e), np.float32))
    batch.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    time.sleep(0.3)
    e0.record(stream)
    batch.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    sites = batch.sites
    value = sites * args.steps / (ms * 1e-3) / 1e6
    bps = {"f32": 272.0, "f16": 164.0, "bf16": 164.0, "moments": 136.0}[args.storage]  # per site and step
    peak, peak_kind = peaks()
    achieved = bps * sites / (ms / args.steps * 1e-3) / 1e9
    errs = []
    for k, sp in enumerate(specs):
        e, R, W = sp["edge"], sp["R"], sp["W"]
        rho, _, phi = batch.moments_numpy(k)
        if args.density:  # p = (p* - 1) rho(phi) cs^2, the pressure of the contrast step
            rl, rg = args.density[0], args.density[1]
            rho = (rho.astype(np.float64) - 1.0) * (rg + (rl - rg) * phi.astype(np.float64))
        c = (e - 1) / 2
        ax = np.arange(e)
        d = np.sqrt((ax[None, None, :] - c) ** 2 + (ax[None, :, None] - c) ** 2 + (ax[:, None, None] - c) ** 2)
        dp = (rho[d < max(R - 2 * W, 1.5)].mean() - rho[d > R + 2 * W].mean()) / 3
        errs.append(abs(dp / (2 * sp["sigma"] / R) - 1))
    errs = np.array(errs)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(specs)} independent periodic droplet boxes, edges in {{24,32,48,64,96}}, "
                                   "R = 0.25 edge (1 +- 20%), sigma in [0.005, 0.02], tau 1, M 0.1, W 3; one "
                                   "persistent launch per step under a CUDA graph"
                                   + (", density and viscosity contrasts rho_l, rho_g, tau_l, tau_g = "
                                      + ", ".join(f"{v:g}" for v in args.density) if args.density else ""),
                       "boxes": len(specs), "sites": sites, "storage": args.storage,
                       "tile": [batch.pair_width or 32, ty, zc], "paired": batch.paired,
                       "l2": "populations larger than L2, no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "batch_step_kernel (step time incl. "
                         "the per-box reduction launch)", "peak_source": peak_kind},
            "laplace_relerr": {"median": float(np.median(errs)), "p90": float(np.quantile(errs, 0.9)),
                               "max": float(errs.max()), "after_steps": args.warmup + args.steps},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


def laplace_dp(rho, edge: int, R: float, W: float) -> float:
    """Pressure jump c_s^2 (<p*> inside r < R - 2W - <p*> outside r > R + 2W) of a
    centred droplet."""
    c = (edge - 1) / 2
    z, y, x = np.meshgrid(*[np.arange(edge)] * 3, indexing="ij")
    d = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    return float((rho[d < R - 2 * W].mean() - rho[d > R + 2 * W].mean()) / 3)


def error_cases(preset: str):
    """The two cases the storages' errors are stated on: the SURR_EDGE^3 surrogate
    of the preset's bubbly HIT (same generator, seed, tau, one bubble of the
    preset's radius, linear forcing; a periodic crop of the large box cannot be
    run) and the LAP_EDGE^3 static droplet of the Laplace law."""
    edge, nb, R, tau, seed = PRESETS[preset]
    return inputs.bubbly_hit(SURR_EDGE, 1, R, seed=seed, tau=tau), inputs.static_droplet(edge=LAP_EDGE, R=LAP_R)


def oracle_references(preset: str):
    """The oracle (as it stands) on the two error cases: K and Phi every
    SURR_EVERY steps over SURR_STEPS steps of the HIT surrogate, and the droplet's
    pressure jump averaged over LAP_SAMPLES.  Its stepping time is the CPU
    baseline (the surrogate is a bounded sample of the benchmark's recipe)."""
    import oracle

    oracle.build()
    w, d = error_cases(preset)
    n = SURR_EDGE
    o = oracle.Oracle(n, n, n, w.tau, w.M, w.W, w.sigma, force_kind=oracle.FORCE_LINEAR, T_relax=w.T_relax)
    o.init(w.phi.astype(np.float64), w.u.astype(np.float64))
    t_step, K, Phi = 0.0, [], []
    for _ in range(SURR_STEPS // SURR_EVERY):
        t0 = time.perf_counter()
        o.step(SURR_EVERY)
        t_step += time.perf_counter() - t0
        rho, u, phi = o.moments()
        K.append(0.5 * float((u * u).sum()))
        Phi.append(float(phi.sum()))
    final = (rho, u, phi)
    o.close()
    m = LAP_EDGE
    o = oracle.Oracle(m, m, m, d.tau, d.M, d.W, d.sigma)
    o.init(d.phi.astype(np.float64), d.u.astype(np.float64))
    dps, done = [], 0
    for t in LAP_SAMPLES:
        t0 = time.perf_counter()
        o.step(t - done)
        t_step += time.perf_counter() - t0
        done = t
        dps.append(laplace_dp(o.moments()[0], m, LAP_R, d.W))
    o.close()
    updates = n ** 3 * SURR_STEPS + m ** 3 * LAP_SAMPLES[-1]
    return {"K": K, "Phi": Phi, "Phi0": float(w.phi.astype(np.float64).sum()), "final": final,
            "dp": float(np.mean(dps)), "time_s": t_step, "updates": updates, "cores": oracle.threads()}


def storage_errors(lbgb, storage: str, preset: str, ref) -> dict:
    """Errors of one storage against the oracle references: the largest relative
    error of K over the surrogate's SURR_STEPS steps, the phase-mass drift
    |Phi(t)/Phi(0) - 1| at the end (the oracle's own drift alongside), max|delta|
    of p*, u, phi at the end, and the relative error of the droplet's Laplace
    pressure jump."""
    w, d = error_cases(preset)
    n = SURR_EDGE
    b = lbgb.Box(n, n, n, w.tau, w.M, w.W, w.sigma, force=lbgb.Force(kind=lbgb.LB_FORCE_LINEAR, T_relax=w.T_relax),
                 storage=storage)
    b.init(w.phi, w.u)
    kerr = 0.0
    for j in range(SURR_STEPS // SURR_EVERY):
        b.step(SURR_EVERY)
        rho, u, phi = b.moments_numpy()
        u64 = u.astype(np.float64)
        kerr = max(kerr, abs(0.5 * float((u64 * u64).sum()) / ref["K"][j] - 1))
    drift = abs(float(phi.astype(np.float64).sum()) / ref["Phi0"] - 1)
    fields = max(float(np.abs(g.astype(np.float64) - x).max()) for g, x in zip((rho, u, phi), ref["final"]))
    b.close()
    m = LAP_EDGE
    b = lbgb.Box(m, m, m, d.tau, d.M, d.W, d.sigma, storage=storage)
    b.init(d.phi, d.u)
    dps, done = [], 0
    for t in LAP_SAMPLES:
        b.step(t - done)
        done = t
        dps.append(laplace_dp(b.moments_numpy()[0].astype(np.float64), m, LAP_R, d.W))
    b.close()
    return {"K_max_relerr": kerr, "phase_mass_drift": drift,
            "phase_mass_drift_oracle": abs(ref["Phi"][-1] / ref["Phi0"] - 1),
            "fields_max_abs_diff": fields, "laplace_dp_relerr": abs(float(np.mean(dps)) / ref["dp"] - 1)}


def run_box(args, lbgb, torch, w, storage: str, force, rank: int, world: int, pg, barrier, alu=None):
    """Create, tune and initialise one box in `storage`, time args.steps steps
    on the device (CUDA events on the library's stream, the fused kernel's own
    event pairs), then the same run end to end through the C ABI with pinned host
    fields.  Returns the measurements; the box is freed."""
    n = w.n[0]
    N = n ** 3
    droplet = args.workload == "droplet"
    stream = torch.cuda.Stream()
    box = lbgb.Box(n, n, n, w.tau, w.M, w.W, w.sigma, force=force, storage=storage, stream=stream)
    if args.phase != "lb":
        box.set_phase_solver(args.phase)
    if args.density:
        box.set_density(*args.density)
    rho_ref = None
    if args.gravity:
        if not args.density:
            raise SystemExit("--gravity needs --density (or --workload droplet)")
        phim = float(w.phi.double().mean()) if torch.is_tensor(w.phi) else float(w.phi.astype(np.float64).mean())
        if not droplet:
            phim = 1.0 - phim  # the flipped field of the gas-bubble case
        rho_ref = args.density[1] + (args.density[0] - args.density[1]) * phim
        box.set_gravity(args.gravity, rho_ref)
    sixteen = storage in ("f16", "bf16", "f16g", "bf16g")
    if args.tile:
        if args.no_pair and sixteen:
            box.set_pairing(False)
        box.set_tile(*args.tile)
    elif not args.no_tune:
        box.tune(8)  # times the paired and the one-site kernel
    ty, zc = box.tile()
    paired = box.paired if sixteen else False
    phi_d = w.phi if torch.is_tensor(w.phi) else torch.from_numpy(w.phi).cuda()
    if args.density and not droplet:
        phi_d = 1.0 - phi_d  # gas bubbles: phi = 0 inside
    u_d = w.u if torch.is_tensor(w.u) else torch.from_numpy(w.u).cuda()
    box.init(phi_d, u_d)
    # clock sampling starts before the warm-up so it is running throughout the timed region
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    time.sleep(0.3)
    box.step(args.warmup)
    box.sync()

    # ---- device-resident timed region (kernel events on the library's stream)
    box.set_timing(True)
    launches0 = box.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    box.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    kern_ms, kern_n = box.kernel_time()
    launches = box.launches - launches0
    box.set_timing(False)
    diag = box.diagnostics(allow_nonfinite=True)
    value, t_max = whole_job(ms, N, args.steps, world, pg)

    # ---- end to end through the public API with pinned host buffers
    phi_h = phi_d.cpu().pin_memory()
    u_h = u_d.cpu().pin_memory()
    del phi_d, u_d
    rho_o = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    u_o = torch.empty((3, n, n, n), dtype=torch.float32).pin_memory()
    phi_o = torch.empty((n, n, n), dtype=torch.float32).pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    box.init(phi_h.numpy(), u_h.numpy())
    for _ in range(args.steps):
        box.step(1)
        box.diagnostics(allow_nonfinite=True)  # per-step result read back (40 bytes)
    box.moments(rho_o.numpy(), u_o.numpy(), phi_o.numpy())
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e_value, _ = whole_job(t_e2e * 1e3, N, args.steps, world, pg)
    bps = box.bytes_per_site
    box.close()
    del phi_h, u_h, rho_o, u_o, phi_o
    torch.cuda.empty_cache()
    peak, peak_kind = peaks()
    kern_avg_s = kern_ms / max(kern_n, 1) * 1e-3
    achieved = bps * N / kern_avg_s / 1e9
    key = storage + ("+density" if args.density else "") + ("+weno5" if args.phase != "lb" else "")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": measured_traffic(key + ("+paired" if paired else ""), N, [64 if paired else 32, ty, zc]),
            "kernel": "fused_step_kernel" + (" (VD)" if args.density else "") + (" (PF)" if args.phase != "lb" else "")
                      + (" (paired: two sites per thread)" if paired else ""),
            "bytes_per_site": bps, "kernel_ms_avg": kern_avg_s * 1e3, "peak_source": peak_kind}
    ips = measured_inst_per_site(key + ("+paired" if paired else ""), [64 if paired else 32, ty, zc])
    if ips is not None and alu:
        # the compute side: warp-instructions issued per second against the
        # device's measured FMA issue rate (one per scheduler and cycle)
        ach = ips * N / kern_avg_s
        roof["issue"] = {"warp_inst_per_site": ips, "achieved": ach, "peak": alu["warp_inst_per_s"],
                         "unit": "warp-instructions/s", "frac": ach / alu["warp_inst_per_s"],
                         "peak_source": "measured (lb_measure_fp32_peak)"}
    if args.phase == "lb" and not args.density and storage in PHI_STORED_BYTES:
        # the same kernel time against the count with a stored FP32 phi (written
        # and re-read; this kernel rebuilds phi on chip)
        roof["bytes_per_site_with_phi"] = PHI_STORED_BYTES[storage]
        roof["frac_with_phi"] = PHI_STORED_BYTES[storage] * N / kern_avg_s / 1e9 / peak
    if args.phase != "lb":
        # the three finite-difference stage kernels and the reduction, per step
        roof["other_kernels_ms_per_step"] = t_max / args.steps - kern_avg_s * 1e3
        roof["other_kernels_bytes_per_site"] = 3 * (4 + 12 + 4) + 2 * 4
    return {"storage": storage, "value": value, "ms_per_step": t_max / args.steps, "tile": [64 if paired else 32, ty, zc],
            "paired": paired,
            "roofline": roof, "clocks": clk, "gpu_launches": launches, "rho_ref": rho_ref,
            "l2": "inputs larger than L2 (populations %.2f GB), no flush" % (bps * N / 2 / 1e9),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * N * 4 / args.steps,
                    "d2h_bytes_per_step": 40 + 5 * N * 4 / args.steps,
                    "note": "lb_init from pinned host fields, K x (lb_step(1) + lb_diagnostics), "
                            "lb_moments to pinned host"},
            "diagnostics": {"Phi": diag[0], "K": diag[1], "eps": diag[2], "umax": diag[3], "A": diag[4]}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "moments", "f16g", "bf16g"],
                    help="population storage: FP32/FP16/BF16 AA populations, the moment-only coefficients, or "
                         "FP16/BF16 AA populations with 16-bit D3Q7 populations (f16g, bf16g)")
    ap.add_argument("--compare", default="f16,f16g",
                    help="16-bit storages (comma list of f16, bf16, f16g, bf16g, or none) run in the same invocation "
                         "next to FP32 storage (bubbly HIT only), each with its errors against the oracle; the first "
                         "is the line's storage16 object, the others follow under compare")
    ap.add_argument("--no-pair", action="store_true",
                    help="one site per thread for the 16-bit storages (the paired kernel is the default)")
    ap.add_argument("--pair-width", type=int, choices=[0, 32, 64], default=None,
                    help="ensemble: paired tile width of the 16-bit storages (0: one site per thread); with --tile "
                         "it skips the tuner")
    ap.add_argument("--edge", type=int, default=None, help="box edge of the droplet and ABC workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--tile", type=int, nargs=2, metavar=("TY", "ZC"), help="fixed launch shape (skips tuning)")
    ap.add_argument("--workload", default="hit", choices=["hit", "ensemble", "droplet", "abc"],
                    help="hit: one bubbly HIT box (preset, default hit512); ensemble: the 512-box droplet batch; "
                         "droplet: the paper's two-component benchmark (512^3, one droplet, density ratio 100); "
                         "abc: single-phase ABC-forced HIT (512^3)")
    ap.add_argument("--boxes", type=int, default=512)
    ap.add_argument("--preset", choices=sorted(PRESETS), default=DEFAULT_PRESET,
                    help="bubbly HIT preset (default hit512: 512^3, 256 bubbles R = 12)")
    ap.add_argument("--density", type=float, nargs=4, metavar=("RHO_L", "RHO_G", "TAU_L", "TAU_G"),
                    help="density and viscosity contrasts: gas bubbles (phi = 0) in the liquid (phi = 1)")
    ap.add_argument("--phase", default="lb", choices=["lb", "weno5"],
                    help="phase-field solver: the D3Q7 model (default) or WENO-5 finite differences")
    ap.add_argument("--gravity", type=lambda v: tuple(float(x) for x in v.split(",")), metavar="GX,GY,GZ",
                    help="buoyancy (rho(phi) - rho_ref) g, rho_ref the mean density (needs --density or droplet)")
    args = ap.parse_args()
    if args.gravity is not None and len(args.gravity) != 3:
        ap.error("--gravity takes three comma-separated components")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)

    rank, world, local = dist_env()
    import torch

    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    from paper_2505_01126_gb300 import build

    if rank == 0:
        build.build()
    barrier()
    from paper_2505_01126_gb300 import lbgb

    if not args.no_tune and not args.tile:
        os.environ.setdefault("LBGB_TUNE_CACHE", os.path.join(ROOT, "paper_2505_01126_gb300", "tune_cache.txt"))
    droplet = args.workload == "droplet"
    abc = args.workload == "abc"
    hit = not (droplet or abc)
    if abc:
        args.edge = args.edge or ABC_EDGE
        w, nb = abc_workload(args.edge), 0
        torch.cuda.empty_cache()
    elif droplet:
        args.edge = args.edge or DROPLET_EDGE
        args.density = DROPLET_DENSITY
        w, nb = droplet_workload(args.edge), 0
    else:
        w, nb = preset_workload(args.preset)
        args.edge = w.n[0]
        torch.cuda.empty_cache()  # the generator's FFT scratch goes back before the box is allocated
    n = args.edge
    if abc:
        force = lbgb.Force(kind=lbgb.LB_FORCE_ABC, A=ABC_A, kf=2 * math.pi / n)
    else:
        force = None if droplet else lbgb.Force(kind=lbgb.LB_FORCE_LINEAR, T_relax=w.T_relax)

    alu = lbgb.measure_fp32_peak() if rank == 0 else None  # the compute-side roofline's denominator
    main_run = run_box(args, lbgb, torch, w, args.storage, force, rank, world, pg, barrier, alu)
    compare = None
    compare_list = [] if args.compare == "none" else args.compare.split(",")
    for st in compare_list:
        if st not in ("f16", "bf16", "f16g", "bf16g"):
            raise SystemExit(f"--compare: unknown storage {st}")
    compares = []
    if hit and args.storage == "f32" and compare_list and not args.density and args.phase == "lb":
        compares = [run_box(args, lbgb, torch, w, st, force, rank, world, pg, barrier, alu) for st in compare_list]
        compare = compares[0]

    if rank == 0:
        cpu, errors = None, None
        if not args.no_cpu_baseline and world == 1:
            try:
                if compare is not None:
                    # the oracle on the error cases, timed: the CPU baseline and the
                    # reference the storages' errors are stated against
                    ref = oracle_references(args.preset)
                    cpu = {"value": ref["updates"] / ref["time_s"] / 1e6, "unit": UNIT, "cores": ref["cores"],
                           "kind": "oracle",
                           "sample": f"{SURR_EDGE}^3 surrogate of this workload (same generator, seed and tau, one "
                                     f"bubble R={PRESETS[args.preset][2]:g}, linear forcing) for {SURR_STEPS} FP64 "
                                     f"oracle steps, and the {LAP_EDGE}^3 static droplet R={LAP_R:g} for "
                                     f"{LAP_SAMPLES[-1]} steps; {ref['time_s']:.1f} s of stepping"}
                    errors = {st: storage_errors(lbgb, st, args.preset, ref) for st in ["f32"] + compare_list}
                    errors["how"] = (f"each storage on the GPU against the FP64 oracle: K = 1/2 sum |u|^2 every "
                                     f"{SURR_EVERY} steps for {SURR_STEPS} steps of the {SURR_EDGE}^3 surrogate "
                                     f"(largest relative error), phase mass sum(phi) drift and max|delta| of p*, u, "
                                     f"phi after {SURR_STEPS} steps; Laplace pressure jump of the {LAP_EDGE}^3 "
                                     f"droplet averaged over steps {LAP_SAMPLES[0]}-{LAP_SAMPLES[-1]} (relative "
                                     f"error); the same quantities tests/test_gpu_precision.py bounds")
                else:
                    cpu = cpu_baseline_sample("droplet" if droplet else ("abc" if abc else "hit"), args.density,
                                              args.gravity, args.phase, args.preset)
            except Exception as ex:  # report, do not fail the benchmark line
                cpu = {"error": str(ex)}
        R = PRESETS[args.preset][2]
        rho_ref = main_run["rho_ref"]
        workload_name = ((f"{n}^3 periodic single-phase forced HIT (phi = 0, sigma = 0), ABC forcing "
                          f"A = {ABC_A:g}, k_f = 2 pi/{n}, tau = {w.tau}, seeded solenoidal start u_rms = 0.02")
                         if abc else
                         (f"{n}^3 periodic box, one droplet R={n / 4:g} of the heavier phase, density ratio 100, "
                          f"nu=0.005 (tau={w.tau}) in both phases, W=3, sigma=0.01, M=0.1, zero initial velocity, "
                          f"no forcing (the paper's two-component benchmark case)") if droplet else
                         (f"{n}^3 periodic bubble-laden forced HIT, {nb} bubbles R={R:g} at seeded non-overlapping "
                          f"positions (seed {PRESETS[args.preset][4]}), W=3, sigma=0.01, tau={w.tau}, M=0.1, "
                          f"solenoidal start from modes 1 <= |k| <= 4 with u_rms=0.02, linear forcing holding K"
                          + (", gas bubbles (phi = 0) with rho_l, rho_g, tau_l, tau_g = "
                             + ", ".join(f"{v:g}" for v in args.density) if args.density else "")
                          + (f"; run with FP32 population storage (value) and {compare_list[0].upper()} shifted "
                             f"storage (storage16)"
                             + "".join(f", {st.upper()}" for st in compare_list[1:])
                             + (" (compare)" if compare_list[1:] else "")
                             + ", FP32 arithmetic, FP64 reductions" if compare else "")))
        workload_name += ((f", buoyancy g = ({', '.join(f'{v:g}' for v in args.gravity)}), "
                           f"rho_ref = {rho_ref:.6g} (mean density)" if args.gravity else "")
                          + (", phase field by WENO-5 finite differences (SSP-RK3)" if args.phase != "lb" else ""))
        line = {"metric": METRIC, "value": main_run["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": main_run["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name, "edge": n, "storage": args.storage, "tile": main_run["tile"],
                           "l2": main_run["l2"], "parallelism": f"replicas x{world}"},
                "roofline": main_run["roofline"], "cpu_baseline": cpu, "e2e": main_run["e2e"],
                "clocks": main_run["clocks"], "gpu_launches": main_run["gpu_launches"],
                "alu_peak": alu}
        if compare is not None:
            line["storage16"] = {k: compare[k] for k in ("storage", "value", "ms_per_step", "tile", "paired", "roofline",
                                                         "e2e", "clocks", "gpu_launches", "diagnostics")}
            line["storage16"]["speedup_vs_f32"] = compare["value"] / main_run["value"]
            line["storage16"]["errors"] = errors[compare_list[0]] if errors else None
            line["gpu_launches"] += compare["gpu_launches"]
            for st, c in zip(compare_list[1:], compares[1:]):
                o = {k: c[k] for k in ("storage", "value", "ms_per_step", "tile", "paired", "roofline", "e2e",
                                       "clocks", "gpu_launches", "diagnostics")}
                o["speedup_vs_f32"] = c["value"] / main_run["value"]
                o["errors"] = errors[st] if errors else None
                line.setdefault("compare", {})[st] = o
                line["gpu_launches"] += c["gpu_launches"]
            line["errors"] = errors
        if droplet:
            line["paper_context"] = {"value": 105480.0 / 64, "unit": "MLUPS per GPU",
                                     "what": "two-component weak scaling, 512^3 per GPU: 105.48 GLUPS on 64 A100 "
                                             "(Leonardo) divided by 64; derived, not printed"}
        if abc:
            line["paper_context"] = {"value": 154940.0 / 64, "unit": "MLUPS per GPU",
                                     "what": "single-component weak scaling, 512^3 per GPU: 154.94 GLUPS on 64 A100 "
                                             "(Leonardo) divided by 64; derived, not printed; that code has no "
                                             "phase field, this step still carries one (phi = 0)"}
        line["diagnostics"] = main_run["diagnostics"]
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
