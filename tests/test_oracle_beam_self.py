"""Self-consistent test beam in the 2-1/2D oracle (Sec. 3.1.1: the charge and current of the frozen and
active beam particles are accumulated so that the fields at the injection plane are consistent).

- the frozen beam's initial self-field (relativistic Poisson solve on the Yee mesh) satisfies the
  discrete Gauss law exactly;
- with the beam's current deposited, Gauss's law still holds after the beam has moved; without it, it
  does not;
- the self-field travels with the beam: after 100 steps it matches the self-field solved at the new
  positions, and the field energy is conserved (no radiation from a uniformly moving charge).
"""
import numpy as np
import pytest

from paper_1009_2727_gb300 import workloads as W

C, QE, EPS0 = 299792458.0, 1.602176634e-19, 8.8541878128e-12


def _beam_case(orc, beam_self=1, gamma_b=2.0):
    nx, nz = 64, 256
    w = {"nx": nx, "nz": nz, "dz_lab": 1e-6, "dx": 1e-6, "gamma_boost": 1.0, "courant": 0.95,
         "solver": W.SOLVERS["yee"], "theta": 0.0, "pml_cells": 0, "order": 3, "beam_self": beam_self}
    s = orc.Sim(w)
    rng = np.random.default_rng(7)
    n = 2000
    x = rng.normal(32e-6, 4e-6, n)
    z = rng.normal(80e-6, 4e-6, n)
    uz = np.full(n, np.sqrt(gamma_b ** 2 - 1) * C)
    s.set_beam(x, z, np.zeros(n), np.zeros(n), uz, 0.0, 1.0)      # the plane 1 m ahead: frozen throughout
    s.beam_weights(np.full(n, 1e-6 / (QE * n)))                   # 1 uC per metre along y
    s.add_beam_self_field()
    return s


def _div_e(s):
    ex, ez = s.field(0), s.field(2)
    return (ex[1:-1, 1:-1] - ex[:-2, 1:-1]) / s.dx + (ez[1:-1, 1:-1] - ez[1:-1, :-2]) / s.dz


def test_beam_self_field_satisfies_discrete_gauss(orc):
    s = _beam_case(orc)
    ref = s.beam_rho()[1:-1, 1:-1] / EPS0
    assert np.abs(_div_e(s) - ref).max() < 1e-10 * np.abs(ref).max()
    # B_y = v E_x / c^2 of a rigidly moving charge
    v = s.info()["beam_vbar"]
    assert v == pytest.approx(np.sqrt(3.0) / 2.0 * C, rel=1e-12)


def test_beam_deposit_keeps_gauss_and_the_field_travels_with_the_beam(orc):
    s = _beam_case(orc)
    e0 = s.diag()["field_energy"]
    s.step(100)
    ref = s.beam_rho()[1:-1, 1:-1] / EPS0
    assert np.abs(_div_e(s) - ref).max() < 1e-9 * np.abs(ref).max()
    moved = s.beam_self_field(0.0)
    ex = s.field(0)
    assert np.linalg.norm(ex - moved["Ex"]) / np.linalg.norm(moved["Ex"]) < 0.05
    assert s.diag()["field_energy"] == pytest.approx(e0, rel=0.05)


def test_without_the_beam_deposit_gauss_fails(orc):
    s = _beam_case(orc, beam_self=0)
    s.step(100)
    ref = s.beam_rho()[1:-1, 1:-1] / EPS0
    assert np.abs(_div_e(s) - ref).max() > 0.1 * np.abs(ref).max()


def _beam_case3(orc, beam_self=1, gamma_b=2.0):
    n3 = (32, 32, 96)
    w = {"dim": 3, "nx": n3[0], "ny": n3[1], "nz": n3[2], "dz_lab": 1e-6, "dx": 1e-6, "dy": 1e-6, "gamma_boost": 1.0,
         "courant": 0.95, "solver": W.SOLVERS["yee"], "theta": 0.0, "pml_cells": 0, "order": 3,
         "beam_self": beam_self}
    s = orc.Sim3(w)
    rng = np.random.default_rng(9)
    n = 1500
    x = rng.normal(16e-6, 2.5e-6, n)
    y = rng.normal(16e-6, 2.5e-6, n)
    z = rng.normal(35e-6, 2.5e-6, n)
    uz = np.full(n, np.sqrt(gamma_b ** 2 - 1) * C)
    zero = np.zeros(n)
    s.set_beam(x, y, z, zero, zero, uz, 0.0, 1.0)
    s.beam_weights(np.full(n, 1e-12 / (QE * n)))                  # 1 pC
    s.add_beam_self_field()
    return s


def _div_e3(s):
    ex, ey, ez = s.field(0), s.field(1), s.field(2)
    c = (slice(1, -1),) * 3
    return ((ex[c] - ex[:-2, 1:-1, 1:-1]) / s.dx + (ey[c] - ey[1:-1, :-2, 1:-1]) / s.dy
            + (ez[c] - ez[1:-1, 1:-1, :-2]) / s.dz)


def test_3d_beam_self_field_gauss_and_travel(orc):
    """the 3D frozen beam: its self-field satisfies the discrete Gauss law at the start and, with the
    deposit, after 60 steps; the field travels with the beam (E_x, E_y within 10%; measured 5%, against 73%
    with B reversed) and keeps its energy"""
    s = _beam_case3(orc)
    c = (slice(1, -1),) * 3
    ref = s.beam_rho()[c] / EPS0
    assert np.abs(_div_e3(s) - ref).max() < 1e-10 * np.abs(ref).max()
    e0 = s.diag()["field_energy"]
    s.step(60)
    ref = s.beam_rho()[c] / EPS0
    assert np.abs(_div_e3(s) - ref).max() < 1e-9 * np.abs(ref).max()
    moved = s.beam_self_field(0.0)
    for comp, k in ((0, "Ex"), (1, "Ey")):
        assert np.linalg.norm(s.field(comp) - moved[k]) / np.linalg.norm(moved[k]) < 0.10, k
    assert s.diag()["field_energy"] == pytest.approx(e0, rel=0.05)
    s2 = _beam_case3(orc, beam_self=0)
    s2.step(60)
    ref = s2.beam_rho()[c] / EPS0
    assert np.abs(_div_e3(s2) - ref).max() > 0.1 * np.abs(ref).max()
