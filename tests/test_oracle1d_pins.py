"""Pins of the 1D oracle (oracle/pic_oracle1d.c) against closed forms and exact identities.

- vacuum standing modes of Eq. 1db-1de (and of the (E_y, B_x) pair) advance by the root of
  sin(w dt/2) = (c dt/dz) sin(k dz/2), exact at c dt = dz (App. I);
- the 1D Esirkepov deposit conserves charge at every node and carries q w v in total;
- full steps with plasma, ions and the antenna keep Gauss's law (E_z from rho) at round-off, with the
  current filter on (div E against the filtered rho, PR-8);
- the linear wake of a Gaussian pulse in a cold plasma: amplitude (sqrt(pi)/4) a0^2 k_p sigma
  exp(-k_p^2 sigma^2/4) E0 and wavelength 2 pi c/w_p (exact theory in 1D), lab frame and boosted frame.
"""
import math

import numpy as np
import pytest

C = 299792458.0
QE = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12


def vac1(nz, courant=0.95, **kw):
    w = {"dim": 1, "nz": nz, "dz_lab": 1e-6, "gamma_boost": 1.0, "courant": courant, "theta": 0.0,
         "pml_cells": 0, "order": 3}
    w.update(kw)
    return w


@pytest.mark.parametrize("courant", [0.5, 0.9, 1.0])
@pytest.mark.parametrize("pol", ["x", "y"])
def test_1d_vacuum_standing_modes(orc, courant, pol):
    nz = 64
    s = orc.Sim1(vac1(nz, courant))
    dz, dt = s.dz, s.dt
    k = np.arange(nz + 1)
    for m in (3, 11, 30):
        K = math.pi * m / (nz * dz)
        om = 2.0 / dt * math.asin(C * dt / dz * math.sin(K * dz / 2))
        B0 = -(dt / dz) * math.sin(K * dz / 2) / math.sin(om * dt / 2)
        e = np.sin(K * k * dz)
        b = B0 * np.cos(K * (k + 0.5) * dz) * math.sin(-om * dt / 2)
        b[-1] = 0.0
        s2 = orc.Sim1(vac1(nz, courant))
        # (E_x, B_y): dBy/dt = -dEx/dz; (E_y, B_x): dBx/dt = +dEy/dz, so B_x takes the opposite sign
        s2.set_field(0 if pol == "x" else 1, e)
        s2.set_field(4 if pol == "x" else 3, b if pol == "x" else -b)
        n = 37
        s2.step(n)
        got = s2.field(0 if pol == "x" else 1)
        assert np.abs(got - e * math.cos(om * n * dt)).max() < 1e-11, m
    if courant == 1.0:
        # App. I: at c dt = dz the scheme has no dispersion, w = c k
        assert om == pytest.approx(C * math.pi * 30 / (nz * dz), rel=1e-12)


@pytest.mark.parametrize("order", [1, 3])
def test_1d_esirkepov_continuity_and_total_current(orc, order):
    rng = np.random.default_rng(3)
    for _ in range(20):
        s = orc.Sim1(vac1(40, order=order))
        dz, dt = s.dz, s.dt
        z0 = rng.uniform(15, 25) * dz
        z1 = z0 + rng.uniform(-0.9, 0.9) * dz
        vx, vy, qw = rng.normal(size=3)
        s.deposit_one(z0, z1, vx, vy, qw)
        jx, jy, jz = s.field(6), s.field(7), s.field(8)
        k = np.arange(41)
        S0 = np.array([orc.shape(order, z0 / dz - kk) for kk in k])
        S1 = np.array([orc.shape(order, z1 / dz - kk) for kk in k])
        drho = qw * (S1 - S0) / dz / dt
        div = (jz - np.concatenate(([0.0], jz[:-1]))) / dz
        assert np.abs(drho + div).max() < 1e-12 * np.abs(drho).max()
        assert jz.sum() * dz == pytest.approx(qw * (z1 - z0) / dt, rel=1e-12)
        assert jx.sum() * dz == pytest.approx(qw * vx, rel=1e-12)
        assert jy.sum() * dz == pytest.approx(qw * vy, rel=1e-12)


def _plasma_laser_1d(gamma, filt):
    lam = 0.8e-6
    w = {"dim": 1, "nz": 400, "dz_lab": lam / 24, "gamma_boost": gamma, "courant": 0.9, "theta": 0.1,
         "pml_cells": 10, "order": 3, "filter_passes": 2 if filt else 0, "filter_compensate": 1 if filt else 0,
         "filter_J": int(filt), "filter_gather": int(filt),
         "plasma": {"n0": 1e25, "z_start_lab": 0.0, "ramp_lab": 2e-6, "length_lab": 0.0, "ppc_z": 4, "ions": 1},
         "laser": {"lambda0": lam, "a0": 0.5, "tau_fwhm": 10e-15, "t_peak": 12e-15, "phase": 0.0,
                   "z_antenna": 60 * (1 + math.sqrt(1 - 1 / gamma ** 2)) * gamma * lam / 24}}
    return w


@pytest.mark.parametrize("gamma,filt", [(1.0, False), (3.0, True)])
def test_1d_gauss_law_through_full_steps(orc, gamma, filt):
    s = orc.Sim1(_plasma_laser_1d(gamma, filt))
    s.step(300)
    ez = s.field(2)
    rho = s.rho()
    if filt:
        rho = s.filter_field(6, rho)
    div = (ez[1:] - ez[:-1]) / s.dz               # at nodes 1..nz-1
    # the interior: particles that leave through the domain's ends take their charge with them
    info = s.info()
    lo, hi = int(info["gz_lo"]) + 6, int(info["gz_hi"]) - 6
    ref = rho[1:][lo:hi] / EPS0
    assert np.abs(ref).max() > 0
    assert np.abs(div[lo:hi] - ref).max() < 1e-9 * np.abs(ref).max()
    assert s.diag()["n_e"] > 1000
    assert np.abs(s.field(1)).max() > 1e10           # the laser is in


LW_N0, LW_A0, LW_LAM = 2e25, 0.1, 0.8e-6


def _linear_wake_1d(gamma, nz, start_cells, ant_cells):
    wp = math.sqrt(LW_N0 * QE * QE / (EPS0 * ME))
    kp = wp / C
    sig = math.sqrt(2.0) / kp
    tau = 2.0 * math.sqrt(math.log(2.0)) * sig / C
    dzl = LW_LAM / 24.0
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    dzb = (1.0 + beta) * gamma * dzl
    lab = gamma == 1.0
    w = {"dim": 1, "nz": nz, "dz_lab": dzl, "gamma_boost": gamma, "courant": 0.95, "theta": 0.0,
         "pml_cells": 8, "order": 1, "moving_window": int(lab), "window_beta": 1.0 if lab else 0.0,
         "plasma": {"n0": LW_N0, "z_start_lab": gamma * start_cells * dzb, "ramp_lab": 1e-6, "length_lab": 0.0,
                    "ppc_z": 2, "ions": 1},
         "laser": {"lambda0": LW_LAM, "a0": LW_A0, "tau_fwhm": tau,
                   "t_peak": 3.2 * tau / (2.0 * math.sqrt(math.log(2.0))), "phase": 0.0,
                   "z_antenna": ant_cells * dzb}}
    ez_lin = math.sqrt(math.pi) / 4 * LW_A0 ** 2 * kp * sig * math.exp(-(kp * sig) ** 2 / 4) * ME * C * wp / QE
    return w, ez_lin, 2 * math.pi / kp / dzl, sig / dzl


def _wake(s, lp_cells, sig_cells, gamma):
    ez, ey = s.field(2), s.field(1)
    kl = int(np.argmax(np.abs(ey)))
    dzb_over_dzl = s.dz / (LW_LAM / 24.0)
    lp_b, sig_b = lp_cells / dzb_over_dzl * gamma, sig_cells / dzb_over_dzl * gamma   # boosted-frame lengths
    a, b = max(kl - int(1.5 * lp_b), 20), kl - int(3 * sig_b)
    seg = ez[a:b]
    zc = [a + i + seg[i] / (seg[i] - seg[i + 1]) for i in range(len(seg) - 1) if seg[i] * seg[i + 1] < 0]
    return np.abs(seg).max(), zc, lp_b


def test_1d_linear_wake_lab_and_boosted(orc):
    w, ez_lin, lp, sg = _linear_wake_1d(1.0, 600, 540, 530)
    s = orc.Sim1(w)
    s.step(520)
    ez, zc, lpb = _wake(s, lp, sg, 1.0)
    assert ez == pytest.approx(ez_lin, rel=0.03)
    assert len(zc) >= 2 and np.diff(zc)[-1] == pytest.approx(lpb / 2, rel=0.03)
    # the same pulse and plasma in a frame boosted at gamma = 2: E_z is invariant under the boost
    w2, _, _, _ = _linear_wake_1d(2.0, 720, 340, 40)
    s2 = orc.Sim1(w2)
    s2.step(600)
    ez2, _, _ = _wake(s2, lp, sg, 2.0)
    assert ez2 == pytest.approx(ez_lin, rel=0.04)


def _g(s, a, k):
    return a + (1 - a) * np.cos(s * k)


@pytest.mark.parametrize("n,stride,comp,strides", [(1, 1, 0, None), (4, 1, 1, None), (2, 3, 1, None),
                                                   (4, 1, 1, (1, 2, 4))])
def test_1d_filter_gain_single_mode(orc, n, stride, comp, strides):
    """Sec. 4.1 in 1D: the filter multiplies an interior mode cos(k z) by the product of the pass gains
    g(s, 1/2, k)^n g(s, n/2 + 1, k) over its strides"""
    nz = 200
    w = vac1(nz, filter_passes=n, filter_stride=stride, filter_compensate=comp)
    if strides:
        w["filter_strides"] = list(strides)
    s = orc.Sim1(w)
    kk = np.arange(nz + 1)
    for m in (5, 17, 40):
        k = 2 * np.pi * m / nz
        f = np.cos(k * kk + 0.3)
        got = s.filter_field(1, f)
        gain = 1.0
        for st in (strides or (stride,)):
            gain *= _g(st, 0.5, k) ** n * (_g(st, n / 2 + 1, k) if comp else 1.0)
        H = (n + comp) * sum(strides or (stride,))
        sl = slice(H + 2, nz - H - 2)
        assert np.abs(got[sl] - gain * f[sl]).max() < 1e-12


def test_1d_momentum_conserving_gather_node_values(orc):
    """Sec. 5 in 1D: the node value of a half-staggered gather copy (E_z, B_x, B_y) is the mean of its two
    neighbours: a quadratic Z^2 at the half positions gains exactly 1/4 at the nodes"""
    nz = 60
    s = orc.Sim1(vac1(nz, gather="momentum"))
    K = np.arange(nz + 1, dtype=float)
    s.set_field(2, (K + 0.5) ** 2)            # E_z, curl free and static without current
    s.set_field(3, 2.0 * (K + 0.5) + 1.0)     # B_x: Faraday leaves it (E_y = 0)
    s.set_field(4, -(K + 0.5) ** 2)           # B_y: E_x = 0
    s.step(1)
    sl = slice(2, nz - 2)
    assert np.abs(s.gather_field(2)[sl] - (K ** 2 + 0.25)[sl]).max() < 1e-12 * (nz ** 2)
    assert np.abs(s.gather_field(3)[sl] - (2.0 * K + 1.0)[sl]).max() < 1e-12 * nz
    assert np.abs(s.gather_field(4)[sl] + (K ** 2 + 0.25)[sl]).max() < 1e-12 * (nz ** 2)


@pytest.mark.parametrize("scheme,extra", [("energy", 0.0), ("momentum", 0.25)])
def test_1d_gather_schemes_on_quadratic_field(orc, scheme, extra):
    """electrons at rest in a static E_z = Z^2 sampled at the half nodes: one Boris step gives
    u_z = (q/m) dt (Z^2 + 1/3 [cubic spline variance] + 1/4 [node interpolation, 'momentum conserving'])"""
    nz = 60
    w = vac1(nz, gather=scheme)
    w["plasma"] = {"n0": 1e10, "z_start_lab": 0.0, "ramp_lab": 0.0, "length_lab": 0.0, "ppc_z": 3, "ions": 0}
    s = orc.Sim1(w)
    K = np.arange(nz + 1, dtype=float)
    s.set_field(2, (K + 0.5) ** 2)
    s.step(1)
    p = s.particles(0)
    assert p["z"].size > 20
    # the position before the step: z moved by dt u_z / gamma
    g = np.sqrt(1 + (p["uz"] / C) ** 2)
    Z = (p["z"] - s.dt * p["uz"] / g) / s.dz
    ez = p["uz"] / (-QE / ME * s.dt)
    assert np.abs(ez - (Z ** 2 + 1.0 / 3.0 + extra)).max() < 1e-9 * np.abs(Z ** 2).max()


# ---------------------------------------------------------------------------
# PR-26: the 1D step is the 2-1/2D step with d/dx = 0. With x periodic (no layer along x) and fields
# independent of x, the 2D CK operator reduces to Yee's (alpha_2 + 2 beta_2 = 1, PR-3) and the split
# PML's x parts stay zero, so interior noise advanced through Friedman damping and the PML at both ends
# of z must equal the separately pinned 2D oracle, component by component.
def test_1d_matches_2d_with_x_independent_fields(orc):
    from paper_1009_2727_gb300 import workloads as W
    rng = np.random.default_rng(31)
    nz, nx, pml = 72, 4, 10
    w2 = {"nx": nx, "nz": nz, "dz_lab": 0.7e-6, "dx": 1.3e-6, "gamma_boost": 1.0, "courant": 0.9,
          "solver": W.SOLVERS["ck"], "theta": 0.25, "pml_cells": pml, "order": 3,
          "periodic_x": 1, "periodic_z": 0}
    s2 = orc.Sim(w2)
    s1 = orc.Sim1(vac1(nz, dz_lab=0.7e-6, theta=0.25, pml_cells=pml, dt=s2.dt))
    assert s1.dt == s2.dt and s1.dz == s2.dz
    f0 = {}
    for comp in range(6):
        f = np.zeros(nz + 1)
        f[pml + 2:nz - pml - 2] = rng.standard_normal(nz - 2 * pml - 4) * (1.0 if comp < 3 else 1.0 / C)
        f0[comp] = f
        s1.set_field(comp, f)
        s2.set_field(comp, np.repeat(f[None, :], nx + 1, axis=0))
    s1.step(90)
    s2.step(90)
    for comp in range(6):
        a1 = s1.field(comp)
        a2 = s2.field(comp)[:nx]
        assert np.abs(a2 - a1[None, :]).max() <= 1e-12 * max(np.abs(a1).max(), np.abs(f0[comp]).max()), comp
    # the transverse pairs reached the layers and lost energy there; E_z and B_z do not propagate in 1D
    for comp in (0, 1, 3, 4):
        assert np.sum(s1.field(comp) ** 2) < 0.5 * np.sum(f0[comp] ** 2), comp
    for comp in (2, 5):
        assert np.array_equal(s1.field(comp), f0[comp]), comp


# ---------------------------------------------------------------------------
# The 1D push through whole steps, in uniform fields far from the walls (weightless particles, so the
# fields stay uniform where the particle is): the E x B drift state of the relativistic Boris push moves
# at exactly v_d = E_x/B_y along z, and in a uniform B_z the momentum turns by 2 atan(q B dt/(2 gamma m))
# per step (an electron turns counter-clockwise about +z) with |u| and z unchanged.
def test_1d_push_through_full_steps_drift_and_gyration(orc):
    nz = 400
    s = orc.Sim1(vac1(nz, courant=0.95))
    Ex, By = 3e8, 2.0
    vd = Ex / By
    gd = 1 / math.sqrt(1 - (vd / C) ** 2)
    s.set_field(0, np.full(nz + 1, Ex))
    s.set_field(4, np.full(nz + 1, By))
    z0 = 200 * s.dz
    s.set_particles(0, [z0], [0.0], [0.0], [gd * vd], [0.0])
    N = 60                          # the walls' disturbance travels < 60 cells; the particle stays > 140 away
    s.step(N)
    p = s.particles(0)
    assert p["z"][0] == pytest.approx(z0 + vd * N * s.dt, abs=1e-9 * s.dz)
    assert abs(p["ux"][0]) < 1e-6 * gd * vd and p["uz"][0] == pytest.approx(gd * vd, rel=1e-9)

    s = orc.Sim1(vac1(nz, courant=0.95))
    B = 2.0
    s.set_field(5, np.full(nz + 1, B))
    u = np.array([0.6 * C, 0.3 * C, 0.0])
    g = math.sqrt(1 + (u @ u) / C ** 2)
    s.set_particles(0, [z0], [u[0]], [u[1]], [u[2]], [0.0])
    N = 300
    s.step(N)
    p = s.particles(0)
    assert p["z"][0] == z0
    assert math.hypot(p["ux"][0], p["uy"][0]) == pytest.approx(math.hypot(u[0], u[1]), rel=1e-13)
    turned = math.atan2(p["uy"][0], p["ux"][0]) - math.atan2(u[1], u[0])
    expect = N * 2 * math.atan(QE * B * s.dt / (2 * g * ME))
    assert abs((turned - expect + math.pi) % (2 * math.pi) - math.pi) < 1e-9
