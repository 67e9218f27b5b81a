"""The workloads against the values the paper prints (tests/golden/), and the
oracle's viscosity against the paper's relation nu = c_s^2 (tau - 1/2).

The benchmark's own recipes follow the configurations it is asked to measure
(a 512^3 box with 256 bubbles of radius 12, about 1.4% gas): where they depart
from the paper's printed values (the paper's 6% gas fraction), the departure
is asserted here and stated, not hidden."""
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_parameters.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("="))
                out[k] = float(v)
    return out


def test_droplet_workload_is_the_papers_two_component_case():
    import bench

    g = golden()
    rho_l, rho_g, tau_l, tau_g = bench.DROPLET_DENSITY
    assert rho_l / rho_g == g["two_component_density_contrast"]
    nu = g["viscosity_relation_cs2"] * (bench.DROPLET_TAU - 0.5)
    assert abs(nu - g["benchmark_kinematic_viscosity"]) < 1e-12
    assert tau_l == tau_g == bench.DROPLET_TAU  # the same viscosity in both phases
    assert bench.DROPLET_EDGE == g["benchmark_grid_per_gpu"]


def test_bubbly_hit_workload_against_the_papers_values():
    import bench
    from paper_2505_01126_gb300 import inputs

    g = golden()
    full, nb, R, tau, seed = bench.PRESETS[bench.DEFAULT_PRESET]
    assert full == g["hit_grid"]
    assert inputs.bubbly_hit(32, 1, 6.0, seed=seed).sigma == g["bubbly_surface_tension"]
    import inspect

    assert inspect.signature(inputs.bubbly_hit_device).parameters["sigma"].default == g["bubbly_surface_tension"]
    # the benchmark's gas fraction, stated against the paper's 6%
    frac = nb * 4.0 / 3.0 * math.pi * R ** 3 / full ** 3
    assert 0.01 < frac < g["bubble_volume_fraction"]


def test_oracle_viscosity_follows_the_papers_relation(orc):
    """A shear wave u_x = A sin(2 pi y / L) decays at exp(-nu k^2 t) with
    nu = c_s^2 (tau - 1/2); the rate measured on the oracle over 200 steps gives
    back the printed c_s^2 = 1/3 within 1%."""
    g = golden()
    L, tau, A, steps = 32, 0.8, 1e-4, 200
    y = np.arange(L)
    u = np.zeros((3, 1, L, 4))
    u[0] = (A * np.sin(2 * np.pi * y / L))[None, :, None]
    o = orc.Oracle(4, L, 1, tau, 0.1, float("inf"), 0.0)
    o.init(np.zeros((1, L, 4)), u)
    o.step(steps)
    amp = np.abs(o.moments()[1][0]).max()
    o.close()
    k = 2 * np.pi / L
    nu = -math.log(amp / A) / (k * k * steps)
    cs2 = nu / (tau - 0.5)
    assert abs(cs2 / g["viscosity_relation_cs2"] - 1) < 0.01, cs2
