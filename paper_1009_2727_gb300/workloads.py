"""Seeded, synthetic workload definitions shared by the tests, the oracle and the bench.

Pure data: every entry is a plain number (SI units). This module holds none of
the method's arithmetic; each consumer (the CUDA library through
``pic_init``/``pic_load_plasma``/``pic_inject_laser``, the CPU oracle)
derives its own numerical parameters (boosted cell, time step, weights) from
these inputs.

Shapes and parameter values follow the paper's workloads: the scaled 0.1 GeV
stage of Table Tablephyspar2d (n_e = 1e19 cm^-3, lambda = 0.8 um, dx = 0.65 um,
lambda/dz resolution, boosted frame gamma = 13) and the tunable-solver table
(Table CKcoefs). No public dataset is involved; every input is synthetic.
"""
from __future__ import annotations

import copy

import numpy as np

# Table CKcoefs: (alpha, beta, gamma) of the tunable solver, cubic-cell sets
SOLVERS = {
    "yee": (1.0, 0.0, 0.0),
    "ck": (7.0 / 12.0, 1.0 / 12.0, 1.0 / 48.0),
    "ck2": (19.0 / 24.0, 1.0 / 24.0, 1.0 / 96.0),
    "ck3": (11.0 / 12.0, 1.0 / 24.0, -1.0 / 48.0),
    "ck4": (3.0 / 4.0, 1.0 / 16.0, 0.0),
    "ck5": (5.0 / 8.0, 3.0 / 40.0, 3.0 / 160.0),
}

LAMBDA0 = 0.8e-6


def parity_2d() -> dict:
    """Plain FP64 parity workload: 2D 256 (z) x 64 (x) cells, gamma_boost = 5.

    dz = lambda0/16 in the lab (boosted dz* = (1+beta) gamma dz = 0.4949 um),
    dx = 1.98 um (four boosted cells), Courant 0.9, Yee coefficients, 8-cell
    PML, one bilinear pass (no compensation) on J and on the gathered fields,
    cubic shapes, n0 = 1e18 cm^-3 with a 10-cell linear entrance ramp, 2x2
    particles per cell, ions fixed in the lab; Gaussian laser a0 = 1,
    w0 = 8 um, tau = 30 fs (intensity FWHM), y-polarised.
    """
    return {
        "name": "parity_2d_256x64_g5",
        "nx": 64, "nz": 256,
        "dz_lab": LAMBDA0 / 16.0, "dx": 1.98e-6,
        "gamma_boost": 5.0, "courant": 0.9, "dt": 0.0,
        "solver": SOLVERS["yee"], "theta": 0.0,
        "pml_cells": 8, "pml_sigma_max": 4.0, "pml_delta": 5.0, "pml_power": 2.0, "pml_xi_exp": 1,
        "filter_passes": 1, "filter_stride": 1, "filter_compensate": 0, "filter_J": 1, "filter_gather": 1,
        "order": 3, "particle_guard": -1,
        "moving_window": 0, "window_beta": 0.0,
        "precision": "fp64",
        "plasma": {"n0": 1e24, "z_start_lab": 5.0 * 30.0e-6, "ramp_lab": 5.0 * 10 * 0.4949e-6,
                   "length_lab": 0.0, "ppc_x": 2, "ppc_z": 2, "ions": 1},
        "laser": {"lambda0": LAMBDA0, "a0": 1.0, "w0": 8e-6, "tau_fwhm": 30e-15, "t_peak": 27e-15,
                  "x_center": 32 * 1.98e-6, "phase": 0.0, "z_antenna": 18 * 0.4949e-6, "beta_s": 0.0},
        "steps": 500, "parity_steps": 100,
    }


def stage_2d(gamma_boost: float = 13.0) -> dict:
    """Mixed-precision 2D boosted-frame 0.1 GeV-class stage: 4096 (z) x 256 (x) cells.

    n0 = 1e19 cm^-3, 4x4 particles per cell, a0 = 2, w0 = 12 um, tau = 30 fs,
    gamma_boost = 13, lambda/dz = 64 in the lab, dx = 0.65 um, Cole-Karkkainen
    coefficients at Courant 0.99, 16-cell PML, Friedman theta = 0.1, four
    bilinear passes plus compensation, cubic shapes. The plasma fills the box
    and keeps entering through the +z plane (steady streaming state).
    """
    g = float(gamma_boost)
    dz_b = (1.0 + np.sqrt(1.0 - 1.0 / g ** 2)) * g * LAMBDA0 / 64.0 if g > 1 else LAMBDA0 / 64.0
    return {
        "name": f"stage_2d_4096x256_g{g:g}",
        "nx": 256, "nz": 4096,
        "dz_lab": LAMBDA0 / 64.0, "dx": 0.65e-6,
        "gamma_boost": g, "courant": 0.99, "dt": 0.0,
        "solver": SOLVERS["ck"], "theta": 0.1,
        "pml_cells": 16, "pml_sigma_max": 4.0, "pml_delta": 5.0, "pml_power": 2.0, "pml_xi_exp": 1,
        "filter_passes": 4, "filter_stride": 1, "filter_compensate": 1, "filter_J": 1, "filter_gather": 1,
        "order": 3, "particle_guard": -1,
        "moving_window": 0, "window_beta": 0.0,
        "precision": "mixed",
        "plasma": {"n0": 1e25, "z_start_lab": g * 40 * dz_b, "ramp_lab": 4e-6,
                   "length_lab": 0.0, "ppc_x": 4, "ppc_z": 4, "ions": 1},
        "laser": {"lambda0": LAMBDA0, "a0": 2.0, "w0": 12e-6, "tau_fwhm": 30e-15, "t_peak": 45e-15,
                  "x_center": 128 * 0.65e-6, "phase": 0.0, "z_antenna": 34 * dz_b, "beta_s": 0.0},
    }


def shrink(w: dict, nx: int, nz: int, **over) -> dict:
    """Same physics on a smaller box (parity cases the oracle finishes in seconds)."""
    v = copy.deepcopy(w)
    v["nx"], v["nz"] = nx, nz
    if v.get("laser"):
        v["laser"]["x_center"] = 0.5 * nx * v["dx"]
    v["name"] = f"{w['name']}_shrunk_{nz}x{nx}"
    for k, val in over.items():
        if isinstance(val, dict) and isinstance(v.get(k), dict):
            v[k].update(val)
        else:
            v[k] = val
    return v


def parity_3d() -> dict:
    """Plain FP64 parity workload in 3D: 64 (z) x 24 (y) x 24 (x) cells, gamma_boost = 5.

    dz = lambda0/16 in the lab (boosted 0.4949 um), dx = dy = 0.99 um (two boosted cells), Courant 0.9
    with the CK2 coefficients, 4-cell PML on every face, one bilinear pass (no compensation) on J and
    on the gathered fields, cubic shapes, n0 = 1e18 cm^-3 with a 4-cell ramp, 1 x 1 x 2 particles per
    cell, ions fixed in the lab; Gaussian laser a0 = 1, w0 = 4 um, tau = 20 fs, y-polarised.
    """
    dzb = 0.4949e-6
    return {
        "name": "parity_3d_64x24x24_g5", "dim": 3,
        "nx": 24, "ny": 24, "nz": 64,
        "dz_lab": LAMBDA0 / 16.0, "dx": 2 * dzb, "dy": 2 * dzb,
        "gamma_boost": 5.0, "courant": 0.9, "dt": 0.0,
        "solver": SOLVERS["ck2"], "theta": 0.0,
        "pml_cells": 4, "pml_sigma_max": 4.0, "pml_delta": 5.0, "pml_power": 2.0, "pml_xi_exp": 1,
        "filter_passes": 1, "filter_stride": 1, "filter_compensate": 0, "filter_J": 1, "filter_gather": 1,
        "order": 3, "particle_guard": -1,
        "moving_window": 0, "window_beta": 0.0,
        "precision": "fp64",
        "plasma": {"n0": 1e24, "z_start_lab": 5.0 * 22 * dzb, "ramp_lab": 5.0 * 4 * dzb,
                   "length_lab": 0.0, "ppc_x": 1, "ppc_y": 1, "ppc_z": 2, "ions": 1},
        "laser": {"lambda0": LAMBDA0, "a0": 1.0, "w0": 4e-6, "tau_fwhm": 20e-15, "t_peak": 20e-15,
                  "x_center": 12 * 2 * dzb, "y_center": 12 * 2 * dzb, "phase": 0.0, "z_antenna": 14 * dzb,
                  "beta_s": 0.0},
        "steps": 60,
    }


def stage_3d(gamma_boost: float = 30.0) -> dict:
    """Mixed-precision 3D boosted-frame stage: 1024 (z) x 128 (y) x 128 (x) cells.

    gamma_boost = 30, lambda/dz = 32 in the lab (boosted dz* = (1+beta) gamma lambda/32), dx = dy = 2 dz*
    (the transverse-to-longitudinal ratio of the paper's gamma = 130 runs), CK2 coefficients at the
    paper's low-instability step c dt = dz/sqrt(2), Friedman theta = 0.1, 16-cell PML, 4 passes +
    compensation, cubic shapes, n0 = 1e18 cm^-3, 1 x 1 x 2 particles per cell (ions fixed in the lab);
    Gaussian laser a0 = 1.5, w0 = 20 um, tau = 60 fs; the box is full of plasma that keeps streaming
    in through the +z plane.
    """
    g = float(gamma_boost)
    beta = np.sqrt(1.0 - 1.0 / g ** 2)
    dzb = (1.0 + beta) * g * LAMBDA0 / 32.0
    c = 299792458.0
    nx = ny = 128
    return {
        "name": f"stage_3d_1024x128x128_g{g:g}", "dim": 3,
        "nx": nx, "ny": ny, "nz": 1024,
        "dz_lab": LAMBDA0 / 32.0, "dx": 2 * dzb, "dy": 2 * dzb,
        "gamma_boost": g, "courant": 0.99, "dt": dzb / (np.sqrt(2.0) * c),
        "solver": SOLVERS["ck2"], "theta": 0.1,
        "pml_cells": 16, "pml_sigma_max": 4.0, "pml_delta": 5.0, "pml_power": 2.0, "pml_xi_exp": 1,
        "filter_passes": 4, "filter_stride": 1, "filter_compensate": 1, "filter_J": 1, "filter_gather": 1,
        "order": 3, "particle_guard": -1,
        "moving_window": 0, "window_beta": 0.0,
        "precision": "mixed",
        "plasma": {"n0": 1e24, "z_start_lab": 0.0, "ramp_lab": 0.0, "length_lab": 0.0,
                   "ppc_x": 1, "ppc_y": 1, "ppc_z": 2, "ions": 1},
        "laser": {"lambda0": LAMBDA0, "a0": 1.5, "w0": 20e-6, "tau_fwhm": 60e-15, "t_peak": 120e-15,
                  "x_center": 0.5 * nx * 2 * dzb, "y_center": 0.5 * ny * 2 * dzb, "phase": 0.0,
                  "z_antenna": 40 * dzb, "beta_s": 0.0},
    }


def shrink3(w: dict, nx: int, ny: int, nz: int, **over) -> dict:
    """the same 3D workload on a smaller box (laser recentred transversely)"""
    v = copy.deepcopy(w)
    v["nx"], v["ny"], v["nz"] = nx, ny, nz
    if v.get("laser"):
        v["laser"]["x_center"] = 0.5 * nx * v["dx"]
        v["laser"]["y_center"] = 0.5 * ny * v["dy"]
    v.update(over)
    return v


def lab_beam(n: int, seed: int, gamma_b: float, R_b: float, L_b: float, z_c: float, x_c: float,
             spread: float = 0.0):
    """Seeded lab-frame test beam (Table Tablephyspar2d profiles): transverse exp(-r^2/(8 R_b^2)),
    longitudinal exp(-z^2/(2 L_b^2)), momentum along z with an optional relative spread.

    Returns (x, z, ux, uy, uz) with u = gamma v in m/s.
    """
    rng = np.random.default_rng(seed)
    c = 299792458.0
    x = x_c + rng.normal(0.0, 2.0 * R_b, n)
    z = z_c + rng.normal(0.0, L_b, n)
    g = gamma_b * (1.0 + spread * rng.normal(0.0, 1.0, n))
    uz = np.sqrt(g * g - 1.0) * c
    return x, z, np.zeros(n), np.zeros(n), uz


def ensemble_2d(n: int = 64, seed: int = 4) -> list:
    """Uneven 2D boosted-frame runs sampled from a seeded generator: nz ~ U{512..4096} (multiples of
    64), nx ~ U{128..256} (multiples of 16), log10 n0 ~ U(23, 25) m^-3, a0 ~ U(0.5, 2.5),
    w0 ~ U(6, 25) um, tau ~ U(20, 60) fs, gamma_boost ~ U(5, 30), particles per cell 2x2 or 4x4 (the
    power-of-two counts of 4..16), mixed precision, the stage's solver and filter settings."""
    rng = np.random.default_rng(seed)
    runs = []
    for i in range(n):
        nz = int(rng.integers(8, 65)) * 64
        nx = int(rng.integers(8, 17)) * 16
        g = float(rng.uniform(5.0, 30.0))
        n0 = float(10.0 ** rng.uniform(23.0, 25.0))
        a0 = float(rng.uniform(0.5, 2.0))
        w0 = float(rng.uniform(6e-6, 25e-6))
        tau = float(rng.uniform(20e-15, 60e-15))
        ppc = int(rng.choice([2, 4]))
        dz_b = (1.0 + np.sqrt(1.0 - 1.0 / g ** 2)) * g * LAMBDA0 / 64.0
        dx = 0.65e-6
        runs.append({
            "name": f"ensemble_{i}_{nz}x{nx}_g{g:.1f}",
            "nx": nx, "nz": nz, "dz_lab": LAMBDA0 / 64.0, "dx": dx,
            "gamma_boost": g, "courant": 0.99, "dt": 0.0,
            "solver": SOLVERS["ck"], "theta": 0.1,
            "pml_cells": 16, "pml_sigma_max": 4.0, "pml_delta": 5.0, "pml_power": 2.0, "pml_xi_exp": 1,
            "filter_passes": 4, "filter_stride": 1, "filter_compensate": 1, "filter_J": 1, "filter_gather": 1,
            "order": 3, "particle_guard": -1, "moving_window": 0, "window_beta": 0.0, "precision": "mixed",
            "plasma": {"n0": n0, "z_start_lab": g * 40 * dz_b, "ramp_lab": 4e-6, "length_lab": 0.0,
                       "ppc_x": ppc, "ppc_z": ppc, "ions": 1},
            "laser": {"lambda0": LAMBDA0, "a0": a0, "w0": w0, "tau_fwhm": tau, "t_peak": 1.5 * tau,
                      "x_center": 0.5 * nx * dx, "phase": 0.0, "z_antenna": 34 * dz_b, "beta_s": 0.0},
        })
    return runs


def surrogate_runs(n: int, seed: int) -> list:
    """Stage runs for the surrogate's training and held-out sets, sampled from a seeded generator over
    (log10 n0 in [23.5, 25] m^-3, a0 in [0.5, 2], w0 in [8, 20] um, tau in [20, 40] fs,
    stage length L in [0.2, 0.8] mm (lab), gamma_boost in [4, 6]).

    Reduced resolution so that thousands of runs fit in minutes: lambda/dz = 16 in the lab, dx = 1.5 um
    (dz <= dx in the boosted frame up to gamma 7.5), 1600 (z) x 96 (x) cells, 2 x 2 particles per cell, CK
    at c dt = dz/sqrt(2) (the paper's low-instability step), theta = 0.1, four passes + compensation,
    cubic shapes, mixed precision, fixed grid. A 256-particle lab test beam at the wake's Lorentz factor
    starts half a plasma wavelength behind the laser peak and becomes active when it crosses the plasma
    entrance; the antenna, at rest, sits far enough from the lower z edge that this crossing (which the
    boost moves back by gamma beta lambda_p / 2) lies inside the box. The plasma of length L starts far
    enough beyond the antenna that the whole pulse has left the antenna before the plasma, streaming
    towards it, arrives (the antenna stays in vacuum while it emits). Each run carries its inputs under
    "inputs", its step count under "steps" (the laser's tail has then left the plasma's end) and under
    "emit_steps" the step at which the antenna has finished emitting."""
    rng = np.random.default_rng(seed)
    runs = []
    for i in range(n):
        ln0 = float(rng.uniform(23.5, 25.0))
        a0 = float(rng.uniform(0.5, 2.0))
        w0 = float(rng.uniform(8e-6, 20e-6))
        tau = float(rng.uniform(20e-15, 40e-15))
        L = float(rng.uniform(0.2e-3, 0.8e-3))
        g = float(rng.uniform(4.0, 6.0))
        runs.append(stage_run(ln0, a0, w0, tau, L, g, beam_seed=seed * 100003 + i, name=f"surrogate_{seed}_{i}"))
    return runs


def stage_run(ln0: float, a0: float, w0: float, tau: float, L: float, g: float, beam_seed: int, name: str,
              nz: int = 1600) -> dict:
    """One stage run of the surrogate_runs recipe for the given inputs (log10 n0 [m^-3], a0, w0 [m], tau [s],
    stage length L [m], gamma_boost): 1600 (z) x 96 (x) cells of lambda/16 (lab) by 1.5 um, 2 x 2 particles per
    cell with rigid ions, CK at c dt = dz/sqrt(2), theta = 0.1, 4 passes + compensation, cubic shapes, a
    256-particle lab test beam at gamma_w half a plasma wavelength behind the laser peak."""
    c = 299792458.0
    qe, me, eps0 = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12
    n0 = 10.0 ** ln0
    beta = np.sqrt(1.0 - 1.0 / g ** 2)
    dz_lab = LAMBDA0 / 16.0
    dz_b = (1.0 + beta) * g * dz_lab
    nx, dx = 96, 1.5e-6
    dt = dz_b / (np.sqrt(2.0) * c)
    t_peak = 1.6 * tau
    wp = np.sqrt(n0 * qe * qe / (eps0 * me))
    lam_p = 2 * np.pi * c / wp
    gw = (2 * np.pi * c / LAMBDA0) / wp
    z_ant = (48 + np.ceil(g * beta * (0.5 * lam_p + 4e-6) / dz_b)) * dz_b
    # the antenna at rest emits for (1 + beta) gamma 2 t_peak; the plasma closes in at beta c
    t_emit = (1.0 + beta) * g * 2.0 * t_peak
    gap = (np.ceil(beta * c * t_emit / dz_b) + 24) * dz_b
    z_start_lab = g * (z_ant + gap)
    # laser peak in the lab at t = 0 (emitted at t' = (1+beta) gamma t_peak by the antenna at rest)
    z_peak0 = z_ant / ((1.0 + beta) * g) - c * t_peak
    x, z, ux, uy, uz = lab_beam(256, seed=beam_seed, gamma_b=gw, R_b=1e-6, L_b=0.5e-6,
                                z_c=z_peak0 - 0.5 * lam_p, x_c=0.5 * nx * dx)
    # the pulse's tail leaves the antenna at t_emit; the plasma's end (gap + ramp + L/gamma beyond the
    # antenna at t = 0, moving at -beta c) then meets it after the closing distance / (1 + beta) c
    z_end = gap + (20e-6 + L) / g
    steps = int((t_emit + (z_end - beta * c * t_emit) / ((1.0 + beta) * c)) / dt) + 50
    return {
        "name": name, "inputs": [ln0, a0, w0 * 1e6, tau * 1e15, L * 1e3, g],
        "steps": steps, "emit_steps": int(t_emit / dt) + 1, "lambda_p": lam_p, "gamma_w": gw,
        "nx": nx, "nz": nz, "dz_lab": dz_lab, "dx": dx, "gamma_boost": g, "courant": 0.99, "dt": dt,
        "solver": SOLVERS["ck"], "theta": 0.1,
        "pml_cells": 16, "pml_sigma_max": 4.0, "pml_delta": 5.0, "pml_power": 2.0, "pml_xi_exp": 1,
        "filter_passes": 4, "filter_stride": 1, "filter_compensate": 1, "filter_J": 1, "filter_gather": 1,
        "order": 3, "particle_guard": -1, "moving_window": 0, "window_beta": 0.0, "precision": "mixed",
        "plasma": {"n0": n0, "z_start_lab": z_start_lab, "ramp_lab": 20e-6, "length_lab": L,
                   "ppc_x": 2, "ppc_z": 2, "ions": 1},
        "laser": {"lambda0": LAMBDA0, "a0": a0, "w0": w0, "tau_fwhm": tau, "t_peak": t_peak,
                  "x_center": 0.5 * nx * dx, "phase": 0.0, "z_antenna": z_ant, "beta_s": 0.0},
        "beam": {"x": x, "z": z, "ux": ux, "uy": uy, "uz": uz, "t_lab": 0.0, "z_plane_lab": z_start_lab},
    }


def scaled_stage(gamma_boost: float, solver: str = "ck", theta: float = 0.0, filter_strides=None) -> dict:
    """The scaled 0.1 GeV-class stage of Sec. 5.1 (n_e = 1e19 cm^-3, gamma_w = 13.2) in the frame boosted by
    gamma_boost, for the comparison of solvers, damping and smoothing against the frame (Sec. 5.1.2): a0 = 1.5,
    w0 = 12 um, tau = 30 fs, a 0.4 mm plasma behind a 20 um ramp, lambda/16 in the lab by 1.5 um cells, 2 x 2
    particles per cell with rigid ions, cubic shapes, the given solver and Friedman theta (the time step 0.99 of
    that solver's limit with the damping's factor, or the singular step c dt = dz/sqrt(2) for undamped CK),
    the stage's 4 passes + compensation, or a wide-band filter S(...) of one pass + compensation per stride;
    every variant has the particle domain of the widest filter. A 256-particle lab test beam at gamma_w rides
    half a plasma wavelength behind the laser peak. The geometry follows the frame: the antenna sits far enough
    up the box that the beam, which the boost holds nearly at rest when gamma_boost approaches gamma_w, starts
    inside it; the plasma starts beyond the emitted pulse; the run ends when the plasma's end has passed the
    beam and the laser's tail has left the plasma (the box grows along z to hold all of it)."""
    c = 299792458.0
    qe, me, eps0 = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12
    g = float(gamma_boost)
    n0, a0, w0, tau, L, ramp = 1e25, 1.5, 12e-6, 30e-15, 0.4e-3, 20e-6
    beta = np.sqrt(1.0 - 1.0 / g ** 2)
    dz_lab = LAMBDA0 / 16.0
    dz_b = (1.0 + beta) * g * dz_lab
    nx, dx = 96, 1.5e-6
    dt = dz_b / (np.sqrt(2.0) * c)
    t_peak = 1.6 * tau
    wp = np.sqrt(n0 * qe * qe / (eps0 * me))
    lam_p = 2 * np.pi * c / wp
    gw = (2 * np.pi * c / LAMBDA0) / wp
    guard = 19
    # the beam starts (t = 0, lab) half a plasma wavelength behind the laser peak, which is still c t_peak
    # behind the antenna's lab position: the antenna sits that far (boosted) above the particle domain's edge
    z_ant = (16 + guard + 8 + np.ceil((1.0 + beta) * g * (c * t_peak + 0.5 * lam_p + 2e-6) / dz_b)) * dz_b
    t_emit = (1.0 + beta) * g * 2.0 * t_peak
    gap = (np.ceil(beta * c * t_emit / dz_b) + 24) * dz_b
    z_start_lab = g * (z_ant + gap)
    z_peak0 = z_ant / ((1.0 + beta) * g) - c * t_peak
    z_beam0 = z_peak0 - 0.5 * lam_p
    x, z, ux, uy, uz = lab_beam(256, seed=7, gamma_b=gw, R_b=1e-6, L_b=0.5e-6, z_c=z_beam0, x_c=0.5 * nx * dx)
    # end: the laser's tail leaves the plasma's end, and the plasma's end passes the beam (lab worldlines
    # transformed: the beam crosses the lab plane z_start_lab + ramp + L at t = (plane - z_beam0) / v_b)
    vb = c * np.sqrt(1.0 - 1.0 / gw ** 2)
    z_end = gap + (ramp + L) / g
    t_laser = t_emit + (z_end - beta * c * t_emit) / ((1.0 + beta) * c)
    z_pl_end = z_start_lab + ramp + L
    t_beam = g * ((z_pl_end - z_beam0) / vb - beta * z_pl_end / c)
    steps = int(max(t_laser, t_beam) / dt) + 50
    nz = int(np.ceil((z_ant + gap + (ramp + L) / g) / dz_b + 16 + guard + 40) / 64.0) * 64
    r = {
        "name": f"scaled_stage_g{g:g}_{solver}_th{theta:g}", "inputs": [np.log10(n0), a0, w0 * 1e6, tau * 1e15, L * 1e3, g],
        "steps": steps, "emit_steps": int(t_emit / dt) + 1, "lambda_p": lam_p, "gamma_w": gw,
        "nx": nx, "nz": max(nz, 640), "dz_lab": dz_lab, "dx": dx, "gamma_boost": g, "courant": 0.99, "dt": dt,
        "solver": SOLVERS[solver], "theta": float(theta),
        "pml_cells": 16, "pml_sigma_max": 4.0, "pml_delta": 5.0, "pml_power": 2.0, "pml_xi_exp": 1,
        "filter_passes": 4, "filter_stride": 1, "filter_compensate": 1, "filter_J": 1, "filter_gather": 1,
        "order": 3, "particle_guard": guard, "moving_window": 0, "window_beta": 0.0, "precision": "mixed",
        "plasma": {"n0": n0, "z_start_lab": z_start_lab, "ramp_lab": ramp, "length_lab": L,
                   "ppc_x": 2, "ppc_z": 2, "ions": 1},
        "laser": {"lambda0": LAMBDA0, "a0": a0, "w0": w0, "tau_fwhm": tau, "t_peak": t_peak,
                  "x_center": 0.5 * nx * dx, "phase": 0.0, "z_antenna": z_ant, "beta_s": 0.0},
        "beam": {"x": x, "z": z, "ux": ux, "uy": uy, "uz": uz, "t_lab": 0.0, "z_plane_lab": z_start_lab},
    }
    if solver != "ck" or theta != 0.0:
        r["dt"] = 0.0        # the library's step: courant x the solver's limit (Friedman factor included)
    if filter_strides:
        r["filter_strides"] = list(filter_strides)
        r["filter_passes"] = 1
        r["filter_compensate"] = 1
        r["name"] += "_S(" + ":".join(str(v) for v in filter_strides) + ")"
    return r


def parity_1d(gamma_boost: float = 3.0) -> dict:
    """Plain FP64 parity workload in 1D: 400 cells, dz = lambda0/24 in the lab, Courant 0.9 with Friedman
    theta = 0.1, 10-cell PML at both ends, 2 passes + compensation on J and on the gathered fields, cubic
    shapes, n0 = 1e19 cm^-3 behind a 2 um ramp, 4 particles per cell, ions fixed in the lab, a0 = 0.5
    pulse of 10 fs."""
    lam = LAMBDA0
    beta = (1.0 - 1.0 / gamma_boost ** 2) ** 0.5
    dzb = (1.0 + beta) * gamma_boost * lam / 24.0
    return {
        "name": f"parity_1d_400_g{gamma_boost:g}", "dim": 1, "nz": 400, "dz_lab": lam / 24.0,
        "gamma_boost": gamma_boost, "courant": 0.9, "dt": 0.0, "theta": 0.1,
        "pml_cells": 10, "pml_sigma_max": 4.0, "pml_delta": 5.0, "pml_power": 2.0, "pml_xi_exp": 1,
        "filter_passes": 2, "filter_stride": 1, "filter_compensate": 1, "filter_J": 1, "filter_gather": 1,
        "order": 3, "particle_guard": -1, "moving_window": 0, "window_beta": 0.0, "precision": "fp64",
        "plasma": {"n0": 1e25, "z_start_lab": gamma_boost * 80 * dzb, "ramp_lab": 2e-6, "length_lab": 0.0,
                   "ppc_z": 4, "ions": 1},
        "laser": {"lambda0": lam, "a0": 0.5, "tau_fwhm": 10e-15, "t_peak": 12e-15, "phase": 0.0,
                  "z_antenna": 60 * dzb},
        "steps": 400,
    }


def app1_lwfa(filtered: bool = True) -> dict:
    """The 1D scaled laser-wakefield stage of App. I (Table Tablephyspar): 952 cells of lambda/24 in the lab
    frame with a moving window at c, c dt = dz (the CFL limit, where the odd-even Nyquist mode of Eq.
    1db-1de is undamped), cubic shapes, 10 particles per cell, n_e = 1e19 cm^-3 over 1.5 mm behind a 4 um
    ramp, a0 = 1 at 0.8 um with a 10.08 um (33.6 fs) long pulse; the current filtered by one bilinear pass
    without compensation, or not at all. The paper's half-sine ramp and sin(pi z/L) pulse envelope are
    replaced by a linear ramp and a Gaussian of the same FWHM (this path's antenna and plasma profiles);
    the beam of the table (1e14 cm^-3, a test population) is left out."""
    lam = LAMBDA0
    dz = lam / 24.0
    nz = 952
    tau = 10.08e-6 / 299792458.0
    return {
        "name": "app1_lwfa_952" + ("_filtered" if filtered else "_unfiltered"), "dim": 1, "nz": nz,
        "dz_lab": dz, "gamma_boost": 1.0, "courant": 1.0, "dt": 0.0, "theta": 0.0,
        "pml_cells": 16, "pml_sigma_max": 4.0, "pml_delta": 5.0, "pml_power": 2.0, "pml_xi_exp": 1,
        "filter_passes": 1 if filtered else 0, "filter_stride": 1, "filter_compensate": 0,
        "filter_J": int(filtered), "filter_gather": 0, "order": 3, "particle_guard": -1,
        "moving_window": 1, "window_beta": 1.0, "precision": "mixed",
        "plasma": {"n0": 1e25, "z_start_lab": (nz - 60) * dz, "ramp_lab": 4e-6, "length_lab": 1.5e-3,
                   "ppc_z": 10, "ions": 1},
        "laser": {"lambda0": lam, "a0": 1.0, "tau_fwhm": tau, "t_peak": 1.6 * tau, "phase": 0.0,
                  "z_antenna": (nz - 80) * dz},
        "steps": 20000,
    }
