"""Pins of the 3D FP64 oracle against what the paper and the mathematics fix.

Closed forms (the 3D numerical dispersion of Eq. num_disp, the filter gain per axis), exact invariants
(discrete charge conservation of the 3D Esirkepov scheme, Gauss's law over full steps with the antenna's
dual particle arrays) and reductions to the separately pinned 2-1/2D oracle (fields independent of y,
a deposit summed over y).
"""
import math

import numpy as np
import pytest

from paper_1009_2727_gb300 import workloads as W

C = 299792458.0
QE = 1.602176634e-19
EPS0 = 8.8541878128e-12


def vacuum3(nx, ny, nz, solver="yee", dx=1e-6, dy=1e-6, dz=1e-6, courant=0.95, theta=0.0, periodic=True, **kw):
    w = {"dim": 3, "nx": nx, "ny": ny, "nz": nz, "dz_lab": dz, "dx": dx, "dy": dy, "gamma_boost": 1.0,
         "courant": courant, "solver": W.SOLVERS[solver] if isinstance(solver, str) else solver,
         "theta": theta, "pml_cells": 0, "order": 3,
         "periodic_x": int(periodic), "periodic_y": int(periodic), "periodic_z": int(periodic)}
    w.update(kw)
    return w


# ---------------------------------------------------------------------------
# Eq. num_disp in 3D: a vacuum Fourier mode advances by the root of the dispersion relation. With
# K_a = 2 sin(k_a d_a/2)/d_a and C_a = alpha + 2 beta (c_b + c_c) + 4 gamma c_b c_c, the leapfrog
# eigenmode has E.K = 0, Omega = 2 sin(omega dt/2)/dt = c sqrt(sum C_a K_a^2) and B = (K* x E)/Omega,
# K* = (C_x K_x, C_y K_y, C_z K_z), each component sampled at its own Yee position.
ST = {0: (0.5, 0, 0), 1: (0, 0.5, 0), 2: (0, 0, 0.5), 3: (0, 0.5, 0.5), 4: (0.5, 0, 0.5), 5: (0.5, 0.5, 0)}


def _mode3(w, s, m, n, e_dir, om=None):
    a, b, g = w["solver"]
    nn = (w["nx"], w["ny"], w["nz"])
    d = (s.dx, s.dy, s.dz)
    k = [2 * np.pi * m[q] / (nn[q] * d[q]) for q in range(3)]
    K = np.array([2 * np.sin(k[q] * d[q] / 2) / d[q] for q in range(3)])
    cc = [np.cos(k[q] * d[q]) for q in range(3)]
    Cq = [a + 2 * b * (cc[(q + 1) % 3] + cc[(q + 2) % 3]) + 4 * g * cc[(q + 1) % 3] * cc[(q + 2) % 3]
          for q in range(3)]
    Ks = np.array([Cq[q] * K[q] for q in range(3)])
    Om = C * math.sqrt(float(np.sum(np.array(Cq) * K * K)))
    if om is None:
        om = 2 * math.asin(Om * s.dt / 2) / s.dt
    E = np.array(e_dir, dtype=float)
    E = E - K * (E @ K) / (K @ K)              # discrete transversality E.K = 0
    E /= np.abs(E).max()
    B = np.cross(Ks, E) / Om
    idx = np.meshgrid(*[np.arange(nn[q] + 1) for q in range(3)], indexing="ij")

    def wave(comp, t):
        ph = sum(k[q] * (idx[q] + ST[comp][q]) * d[q] for q in range(3))
        return np.cos(ph - om * t)
    out = {}
    for c in range(3):
        out[c] = E[c] * wave(c, n * s.dt)
        out[3 + c] = B[c] * wave(3 + c, (n - 0.5) * s.dt)
    return out


@pytest.mark.parametrize("name", ["yee", "ck", "ck2", "ck5"])
@pytest.mark.parametrize("dx,dy,dz", [(1e-6, 1e-6, 1e-6), (1.3e-6, 2.0e-6, 0.6e-6)])
def test_3d_vacuum_mode_follows_dispersion(orc, name, dx, dy, dz):
    w = vacuum3(10, 8, 12, name, dx=dx, dy=dy, dz=dz, courant=0.97)
    for m, e in (((1, 0, 0), (0, 1, 0)), ((0, 2, 3), (1, 0, 0)), ((2, 3, 5), (0.3, -1, 0.4)), ((4, 3, 5), (1, 1, 1))):
        s = orc.Sim3(w)
        f0 = _mode3(w, s, m, 0, e)
        for comp in range(6):
            s.set_field(comp, f0[comp])
        N = 30
        s.step(N)
        fN = _mode3(w, s, m, N, e)
        scale = max(np.abs(fN[c]).max() for c in range(3))
        for comp in range(6):
            got = s.field(comp)[:10, :8, :12]
            ref = fN[comp][:10, :8, :12]
            sc = scale if comp < 3 else max(np.abs(fN[c]).max() for c in range(3, 6))
            assert np.abs(got - ref).max() <= 1e-10 * sc, (name, m, comp)


def test_3d_fields_independent_of_y_match_2d(orc):
    """the enlarged 3D operator restricted to d/dy = 0 is the 2D operator of PR-3: a y-independent
    random state advances exactly like the 2-1/2D oracle (CK coefficients, Friedman damping)"""
    rng = np.random.default_rng(3)
    nx, nz = 12, 14
    common = dict(dx=1.1e-6, dz=0.8e-6, courant=0.9, theta=0.3)
    w2 = {"nx": nx, "nz": nz, "dz_lab": common["dz"], "dx": common["dx"], "gamma_boost": 1.0,
          "courant": 0.9, "solver": W.SOLVERS["ck"], "theta": 0.3, "pml_cells": 0, "order": 3,
          "periodic_x": 1, "periodic_z": 1}
    s2 = orc.Sim(w2)
    w3 = vacuum3(nx, 4, nz, "ck", dx=common["dx"], dy=1.7e-6, dz=common["dz"], courant=0.9, theta=0.3)
    w3["dt"] = s2.dt
    s3 = orc.Sim3(w3)
    for comp in range(6):
        f = np.zeros((nx + 1, nz + 1))
        f[:nx, :nz] = rng.standard_normal((nx, nz)) * (1.0 if comp < 3 else 1.0 / C)
        s2.set_field(comp, f)
        s3.set_field(comp, np.repeat(f[:, None, :], 5, axis=1))
    s2.step(25)
    s3.step(25)
    for comp in range(6):
        a2 = s2.field(comp)[:nx, :nz]
        a3 = s3.field(comp)[:nx, :4, :nz]
        assert np.abs(a3 - a2[:, None, :]).max() <= 1e-12 * np.abs(a2).max(), comp


# ---------------------------------------------------------------------------
# 3D filter: the gain of a periodic mode is the product of the 1D gains along x, y and z (Sec. 4.1)
@pytest.mark.parametrize("n,stride,comp", [(1, 1, 0), (4, 1, 1), (2, 2, 1)])
def test_3d_filter_gain_is_product_of_axis_gains(orc, n, stride, comp):
    w = vacuum3(16, 12, 20, filter_passes=n, filter_stride=stride, filter_compensate=comp)
    s = orc.Sim3(w)
    m = (3, 2, 5)
    k = [2 * np.pi * m[0] / 16, 2 * np.pi * m[1] / 12, 2 * np.pi * m[2] / 20]
    i, j, l = np.meshgrid(np.arange(17), np.arange(13), np.arange(21), indexing="ij")
    f = np.cos(k[0] * i + k[1] * j + k[2] * l + 0.4)

    def G(kk):
        g = (0.5 + 0.5 * np.cos(stride * kk)) ** n
        if comp:
            ac = n / 2 + 1
            g *= ac + (1 - ac) * np.cos(stride * kk)
        return g
    got = s.filter_field(1, f)[:16, :12, :20]
    assert np.abs(got - G(k[0]) * G(k[1]) * G(k[2]) * f[:16, :12, :20]).max() < 1e-13


# ---------------------------------------------------------------------------
# Esirkepov in 3D: discrete continuity d(rho)/dt + div J = 0 exactly, and the total current q v
def _rho1(orc, w, pos, qw):
    s = orc.Sim3(w)
    s.set_particles(0, [pos[0]], [pos[1]], [pos[2]], [0.0], [0.0], [0.0], [qw / -QE])
    return s.rho()


@pytest.mark.parametrize("order", [1, 3])
def test_3d_esirkepov_continuity_and_total_current(orc, order):
    w = vacuum3(16, 16, 16, dx=1.1e-6, dy=0.9e-6, dz=0.7e-6, periodic=False, order=order)
    rng = np.random.default_rng(5 + order)
    for _ in range(8):
        s = orc.Sim3(w)
        d = np.array([s.dx, s.dy, s.dz])
        p0 = rng.uniform(6, 9, 3) * d
        p1 = p0 + rng.uniform(-0.95, 0.95, 3) * d
        qw = -QE * 2.3e7
        Jx, Jy, Jz = s.deposit_one(p0, p1, qw)
        r0, r1 = _rho1(orc, w, p0, qw), _rho1(orc, w, p1, qw)
        div = np.zeros_like(r0)
        div[1:] += (Jx[1:] - Jx[:-1]) / s.dx
        div[0] += Jx[0] / s.dx
        div[:, 1:] += (Jy[:, 1:] - Jy[:, :-1]) / s.dy
        div[:, 0] += Jy[:, 0] / s.dy
        div[:, :, 1:] += (Jz[:, :, 1:] - Jz[:, :, :-1]) / s.dz
        div[:, :, 0] += Jz[:, :, 0] / s.dz
        res = (r1 - r0) / s.dt + div
        scale = np.abs(r1 - r0).max() / s.dt
        assert np.abs(res).max() <= 1e-12 * scale
        vol = s.dx * s.dy * s.dz
        for J, a in ((Jx, 0), (Jy, 1), (Jz, 2)):
            assert J.sum() * vol == pytest.approx(qw * (p1[a] - p0[a]) / s.dt, rel=1e-12)


def test_3d_deposit_summed_over_y_is_the_2d_deposit(orc):
    """a particle moving in the x-z plane: sum_j J3D dy equals the 2-1/2D Esirkepov current"""
    w3 = vacuum3(16, 10, 16, dx=1.1e-6, dy=0.9e-6, dz=0.7e-6, periodic=False)
    s3 = orc.Sim3(w3)
    w2 = {"nx": 16, "nz": 16, "dz_lab": 0.7e-6, "dx": 1.1e-6, "gamma_boost": 1.0, "courant": 0.9,
          "solver": W.SOLVERS["yee"], "theta": 0.0, "pml_cells": 0, "order": 3}
    s2 = orc.Sim(w2)
    w2["dt"] = s3.dt
    s2 = orc.Sim(w2)
    rng = np.random.default_rng(9)
    for _ in range(4):
        s3 = orc.Sim3(w3)
        x0, z0 = rng.uniform(6, 9) * s3.dx, rng.uniform(6, 9) * s3.dz
        x1, z1 = x0 + rng.uniform(-0.9, 0.9) * s3.dx, z0 + rng.uniform(-0.9, 0.9) * s3.dz
        y = 4.3 * s3.dy
        qw = -QE * 1e8
        J3 = s3.deposit_one((x0, y, z0), (x1, y, z1), qw)
        J2 = s2.deposit_one(x0, z0, x1, z1, 0.0, qw)
        for a in (0, 2):
            ref = J2[a]
            assert np.abs(J3[a].sum(axis=1) * s3.dy - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(J3[1]).max() == 0.0


# ---------------------------------------------------------------------------
# Gauss's law over full steps (Sec. 4.2.2 with PR-8 and the dual antenna arrays of Sec. 3.1.2):
# div E - F(rho)/eps0 stays at round-off in the interior, rho including the antenna pairs
@pytest.mark.slow
def test_3d_gauss_law_full_step_with_antenna(orc):
    w = W.shrink3(W.parity_3d(), 32, 32, 56)
    w["laser"]["z_antenna"] = 24 * 0.4949e-6
    s = orc.Sim3(w)
    info = s.info()
    s.step(24)
    Ex, Ey, Ez = s.field(0), s.field(1), s.field(2)
    div = np.zeros_like(Ex)
    div[1:] += (Ex[1:] - Ex[:-1]) / s.dx
    div[:, 1:] += (Ey[:, 1:] - Ey[:, :-1]) / s.dy
    div[:, :, 1:] += (Ez[:, :, 1:] - Ez[:, :, :-1]) / s.dz
    frho = s.filter_field(1, s.rho())
    G = div - frho / EPS0
    lo = [int(info[f"g{a}_lo"]) + 5 for a in "xyz"]
    hi = [int(info[f"g{a}_hi"]) - 5 for a in "xyz"]
    sl = (slice(lo[0], hi[0]), slice(lo[1], hi[1]), slice(lo[2], hi[2]))
    p = s.particles(0)
    n_e = np.abs(p["w"]).max() * 2 / (s.dx * s.dy * s.dz)
    scale = QE * n_e / EPS0
    assert np.abs(div[sl]).max() > 1e-7 * scale       # the laser and the antenna did separate charge
    assert np.abs(G[sl]).max() < 1e-11 * scale


def test_3d_wide_band_filter_gain(orc):
    """S(1:2) in 3D: the gain of a periodic mode is the product over the three axes and both strides of
    g(s, 1/2, k)^4 g(s, 3, k), the compensation pass at alpha_c = n/2 + 1 = 3 for n = 4"""
    w = vacuum3(16, 12, 20, filter_passes=4, filter_compensate=1, filter_strides=[1, 2])
    s = orc.Sim3(w)
    m = (3, 2, 5)
    k = [2 * np.pi * m[0] / 16, 2 * np.pi * m[1] / 12, 2 * np.pi * m[2] / 20]
    i, j, l = np.meshgrid(np.arange(17), np.arange(13), np.arange(21), indexing="ij")
    f = np.cos(k[0] * i + k[1] * j + k[2] * l + 0.4)

    def G(st, kk):
        return (0.5 + 0.5 * np.cos(st * kk)) ** 4 * (3 - 2 * np.cos(st * kk))
    gain = np.prod([G(st, kk) for st in (1, 2) for kk in k])
    got = s.filter_field(1, f)[:16, :12, :20]
    assert np.abs(got - gain * f[:16, :12, :20]).max() < 1e-13


def test_3d_momentum_conserving_gather_copies_at_the_nodes(orc):
    """Sec. 5, 'momentum conserving' gather in 3D: the node value of each gather copy is the mean of its
    nearest staggered values (two along one half-integer axis, four along two); a field quadratic along a
    half-integer axis gains exactly 1/4 per such axis, a linear one is exact"""
    n = (14, 12, 16)
    s = orc.Sim3(vacuum3(*n, periodic=False, gather="momentum"))
    I, J, K = np.meshgrid(*[np.arange(m + 1, dtype=float) for m in n], indexing="ij")
    # E_q depends only on its own coordinate (curl free); B is static (Faraday leaves it unchanged)
    s.set_field(0, (I + 0.5) ** 2 + (I + 0.5))
    s.set_field(1, 2.0 * (J + 0.5) ** 2)
    s.set_field(2, -(K + 0.5) ** 2 + 3.0)
    s.set_field(3, (J + 0.5) ** 2 + (K + 0.5) ** 2 + (J + 0.5) * (K + 0.5))
    s.set_field(4, (I + 0.5) * (K + 0.5) + 1.0)
    s.set_field(5, (I + 0.5) ** 2 - (J + 0.5))
    s.step(1)
    want = {0: I ** 2 + 0.25 + I, 1: 2.0 * (J ** 2 + 0.25), 2: -(K ** 2 + 0.25) + 3.0,
            3: J ** 2 + K ** 2 + J * K + 0.5, 4: I * K + 1.0, 5: I ** 2 + 0.25 - J}
    sl = tuple(slice(3, m - 2) for m in n)
    for c in range(6):
        got = s.gather_field(c)
        assert np.abs(got[sl] - want[c][sl]).max() < 1e-12 * np.abs(want[c][sl]).max(), c


@pytest.mark.parametrize("scheme,extra", [("energy", 0.0), ("momentum", 0.25)])
def test_3d_gather_schemes_on_quadratic_field(orc, scheme, extra):
    """electrons at rest in a static E_x = X^2 (X = x/dx; uniform in y and z): one Boris step gives
    u_x = (q/m) dt E_x at the particle. The cubic B-spline adds its variance 1/3 (times f''/2 = 1); the
    node-interpolated ('momentum conserving') gather adds 1/4 more, from averaging the staggered samples
    (i + 1/2)^2 to the nodes"""
    n = (16, 12, 14)
    w = vacuum3(*n, periodic=False, gather=scheme)
    w["plasma"] = {"n0": 1e10, "z_start_lab": 0.0, "ramp_lab": 0.0, "length_lab": 0.0, "ppc_x": 2, "ppc_y": 1,
                   "ppc_z": 1, "ions": 0}
    s = orc.Sim3(w)
    I = np.arange(n[0] + 1, dtype=float)[:, None, None] * np.ones((1, n[1] + 1, n[2] + 1))
    s.set_field(0, (I + 0.5) ** 2)
    s.step(1)
    p = s.particles(0)
    p = {k: v[p["alive"]] for k, v in p.items()}
    assert p["x"].size > 10
    X = p["x"] / s.dx
    qe, me = 1.602176634e-19, 9.1093837015e-31
    ex = p["ux"] / (-qe / me * s.dt)
    assert np.abs(ex - (X ** 2 + 1.0 / 3.0 + extra)).max() < 1e-9 * np.abs(X ** 2).max()


# ---------------------------------------------------------------------------
# App. II in 3D: the split-field PML. The 2-1/2D PML is pinned by its reflection of a Harris pulse;
# with y periodic (no layer along y) and fields independent of y, the 3D layers on the x and z faces
# must advance exactly like the 2D ones.
def _interior_noise(rng, shape, lo, scale):
    f = np.zeros(shape)
    sl = tuple(slice(lo, n - lo) for n in shape)
    f[sl] = rng.standard_normal(tuple(n - 2 * lo for n in shape)) * scale
    return f


def test_3d_pml_reduces_to_2d_when_y_is_periodic(orc):
    rng = np.random.default_rng(17)
    nx, nz, pml = 26, 30, 6
    w2 = {"nx": nx, "nz": nz, "dz_lab": 0.8e-6, "dx": 1.1e-6, "gamma_boost": 1.0, "courant": 0.9,
          "solver": W.SOLVERS["ck"], "theta": 0.2, "pml_cells": pml, "order": 3,
          "periodic_x": 0, "periodic_z": 0}
    s2 = orc.Sim(w2)
    w3 = vacuum3(nx, 4, nz, "ck", dx=1.1e-6, dy=1.7e-6, dz=0.8e-6, courant=0.9, theta=0.2,
                 periodic=False, pml_cells=pml, periodic_y=1)
    w3["dt"] = s2.dt
    s3 = orc.Sim3(w3)
    for comp in range(6):
        f = _interior_noise(rng, (nx + 1, nz + 1), pml + 2, 1.0 if comp < 3 else 1.0 / C)
        s2.set_field(comp, f)
        s3.set_field(comp, np.repeat(f[:, None, :], 5, axis=1))
    # long enough for the noise to cross the layers several times
    s2.step(60)
    s3.step(60)
    inside = 0.0
    for comp in range(6):
        a2 = s2.field(comp)
        a3 = s3.field(comp)[:, :4, :]
        assert np.abs(a3 - a2[:, None, :]).max() <= 1e-12 * np.abs(a2).max(), comp
        inside += float(np.sum(a2[:pml, :] ** 2) + np.sum(a2[:, :pml] ** 2)) * (1.0 if comp < 3 else C * C)
    assert inside > 0.0            # the layers took part


# x <-> y mirror symmetry with dx = dy and nx = ny: E is a polar vector, B an axial one, so the
# mirrored state (E'_x, E'_y, E'_z)(i, j) = (E_y, E_x, E_z)(j, i), B' = -(B_y, B_x, B_z)(j, i), with
# particles at (y, x, z) and momenta (u_y, u_x, u_z), must stay the mirror of the original under the
# CK solver, the PML on all six faces, Friedman damping, the filter, the cubic gather, the Boris push and
# the Esirkepov deposit. Every y-term of the 3D oracle is thereby tied to its x-term.
def _mirror(comp, a):
    src = {0: 1, 1: 0, 2: 2, 3: 4, 4: 3, 5: 5}[comp]
    sign = 1.0 if comp < 3 else -1.0
    return src, sign


@pytest.mark.parametrize("gather,order", [("energy", 3), ("momentum", 3), ("energy", 1)])
def test_3d_mirror_x_y_with_pml_particles_and_filter(orc, gather, order):
    rng = np.random.default_rng(23)
    n, nz, pml = 28, 26, 4
    w = vacuum3(n, n, nz, "ck", dx=0.9e-6, dy=0.9e-6, dz=0.7e-6, courant=0.9, theta=0.2, periodic=False,
                pml_cells=pml, filter_passes=2, filter_compensate=1, particle_guard=5, gather=gather, order=order)
    s1, s2 = orc.Sim3(w), orc.Sim3(w)
    F = [_interior_noise(rng, (n + 1, n + 1, nz + 1), pml + 2, 3e9 if c < 3 else 3e9 / C) for c in range(6)]
    for comp in range(6):
        src, sign = _mirror(comp, None)
        s1.set_field(comp, F[comp])
        s2.set_field(comp, sign * np.transpose(F[src], (1, 0, 2)))
    info = s1.info()
    npart = 40
    lo, hi = info["gx_lo"] + 1.5, info["gx_hi"] - 1.5
    x = rng.uniform(lo, hi, npart) * s1.dx
    y = rng.uniform(lo, hi, npart) * s1.dy
    z = rng.uniform(info["gz_lo"] + 1.5, info["gz_hi"] - 1.5, npart) * s1.dz
    u = rng.standard_normal((3, npart)) * 0.3 * C
    # weights of 1e8 make the deposit's field ~100x the initial noise, and the noise changes the momenta by
    # about 1% a step; at 1e9 the orbits grow chaotic and round-off differences grow past 1e-12
    wt = np.full(npart, 1e8)
    s1.set_particles(0, x, y, z, u[0], u[1], u[2], wt)
    s2.set_particles(0, y, x, z, u[1], u[0], u[2], wt)
    s1.step(30)
    s2.step(30)
    for comp in range(6):
        src, sign = _mirror(comp, None)
        a = s2.field(comp)
        b = sign * np.transpose(s1.field(src), (1, 0, 2))
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), comp
    assert np.abs(s1.field(1)).max() > 10 * np.abs(F[1]).max()       # the deposit shaped the fields
    p1, p2 = s1.particles(0), s2.particles(0)
    assert p1["alive"].sum() > npart // 2
    o1, o2 = np.argsort(p1["id"]), np.argsort(p2["id"])
    assert np.array_equal(p1["alive"][o1], p2["alive"][o2])
    live = p1["alive"][o1]
    for k1, k2, scale in (("x", "y", s1.dx), ("y", "x", s1.dy), ("z", "z", s1.dz),
                          ("ux", "uy", C), ("uy", "ux", C), ("uz", "uz", C)):
        assert np.abs(p2[k1][o2][live] - p1[k2][o1][live]).max() <= 1e-12 * scale, k1
    du = np.abs(p1["ux"][o1][live] - u[0][np.sort(p1["id"])][live])
    assert du.max() > 1e-3 * C                                       # the gather and push acted


# ---------------------------------------------------------------------------
# Sec. 3.2 in 3D: the lab stations. The 2-1/2D stations are pinned by the lab-frame identity and by a
# boosted laser seen in the lab with its lab amplitude and period; with fields independent of y the 3D
# rows (interpolation in z' and t', the transform of E_perp and B_perp to the lab) must equal them at every y.
def test_3d_lab_stations_reduce_to_2d(orc):
    rng = np.random.default_rng(29)
    nx, nz, g = 10, 40, 3.0
    beta = math.sqrt(1 - 1 / g ** 2)
    w2 = {"nx": nx, "nz": nz, "dz_lab": 0.3e-6, "dx": 1.2e-6, "gamma_boost": g, "courant": 0.9,
          "solver": W.SOLVERS["ck"], "theta": 0.1, "pml_cells": 0, "order": 3,
          "periodic_x": 1, "periodic_z": 1}
    s2 = orc.Sim(w2)
    w3 = vacuum3(nx, 4, nz, "ck", dx=1.2e-6, dy=2.0e-6, dz=0.3e-6, courant=0.9, theta=0.1, gamma_boost=g)
    w3["dz_lab"] = 0.3e-6
    w3["dt"] = s2.dt
    s3 = orc.Sim3(w3)
    assert s3.dz == s2.dz and s3.dt == s2.dt
    for comp in range(6):
        f = np.zeros((nx + 1, nz + 1))
        f[:nx, :nz] = rng.standard_normal((nx, nz)) * (1.0 if comp < 3 else 1.0 / C)
        s2.set_field(comp, f)
        s3.set_field(comp, np.repeat(f[:, None, :], 5, axis=1))
    # rows at boosted (z', t') inside the run, given as lab (z_L, t_L)
    nst = 12
    zp = rng.uniform(5, nz - 5, nst) * s2.dz
    tp = rng.uniform(3, 20, nst) * s2.dt
    zL = g * (zp + beta * C * tp)
    tL = g * (tp + beta * zp / C)
    s2.btd_set(zL, tL)
    s3.btd_set(zL, tL)
    s2.step(24)
    s3.step(24)
    o2, d2 = s2.btd_get()
    o3, d3 = s3.btd_get()
    assert d2.all() and np.array_equal(d2, d3)
    scale = np.abs(o2[:, :3]).max()
    for j in range(4):
        for comp in range(6):
            sc = scale if comp < 3 else scale / C
            assert np.abs(o3[:, comp, :nx, j] - o2[:, comp, :nx]).max() <= 1e-12 * sc, (j, comp)
    assert scale > 0.5                     # rows of the unit-variance noise, not empty rows


# ---------------------------------------------------------------------------
# Sec. 4.2.1 on cubic cells at each solver's Courant limit: Yee has no numerical dispersion along the
# 3D diagonal, CK none along the principal axes, CK3 none along the 2D diagonals. There the oracle's
# vacuum mode must travel at exactly c (omega = c|k|), while Yee along an axis lags.
@pytest.mark.parametrize("name,m,exact", [("ck", (3, 0, 0), True), ("ck", (0, 0, 4), True),
                                          ("yee", (3, 3, 3), True), ("ck3", (3, 3, 0), True),
                                          ("ck3", (0, 2, 2), True), ("yee", (3, 0, 0), False)])
def test_3d_dispersion_free_directions_at_the_courant_limit(orc, name, m, exact):
    n = 12
    w = vacuum3(n, n, n, name, courant=1.0)
    s = orc.Sim3(w)
    d = s.dx
    k = np.array([2 * np.pi * m[q] / (n * d) for q in range(3)])
    om_c = C * float(np.linalg.norm(k))
    e_dir = (0.0, 0.0, 1.0) if m[2] == 0 else (1.0, 0.0, 0.0)
    f0 = _mode3(w, s, m, 0, e_dir)
    for comp in range(6):
        s.set_field(comp, f0[comp])
    N = 40
    s.step(N)
    ref = _mode3(w, s, m, N, e_dir, om=om_c)
    scale = max(np.abs(ref[c]).max() for c in range(3))
    err = max(np.abs(s.field(c)[:n, :n, :n] - ref[c][:n, :n, :n]).max() for c in range(3)) / scale
    if exact:
        assert err < 1e-9
    else:
        assert err > 1e-2


# ---------------------------------------------------------------------------
# Sec. 4.3 on cubic cells near each solver's Courant limit: Yee-Friedman damps the short waves most
# along the 3D diagonal, CK-Friedman most along the axes. A vacuum mode of k dx = 3 pi/4 keeps its
# energy without damping and, at theta = 0.5, loses it in 20 steps in the direction that the paper names.
def _mode_energy_after(orc, name, m, theta, steps=20, n=8):
    w = vacuum3(n, n, n, name, courant=0.999, theta=theta)
    s = orc.Sim3(w)
    e_dir = (0.0, 0.0, 1.0) if m[2] == 0 else (1.0, -1.0, 0.0)
    f0 = _mode3(w, s, m, 0, e_dir)
    for comp in range(6):
        s.set_field(comp, f0[comp])

    def energy():
        return (sum(np.sum(s.field(c)[:n, :n, :n] ** 2) for c in range(3))
                + C * C * sum(np.sum(s.field(c)[:n, :n, :n] ** 2) for c in range(3, 6)))
    e0 = energy()
    s.step(steps)
    return energy() / e0


def test_3d_friedman_damping_directions(orc):
    axis, diag = (3, 0, 0), (3, 3, 3)
    for name in ("yee", "ck"):
        for m in (axis, diag):
            assert _mode_energy_after(orc, name, m, 0.0) == pytest.approx(1.0, abs=1e-3), (name, m)
    yf = {m: _mode_energy_after(orc, "yee", m, 0.5) for m in (axis, diag)}
    ckf = {m: _mode_energy_after(orc, "ck", m, 0.5) for m in (axis, diag)}
    assert yf[diag] < 0.1 * yf[axis]          # YF: strongest along the 3D diagonal
    assert ckf[axis] < 0.1 * ckf[diag]        # CKF: strongest along the axes


# ---------------------------------------------------------------------------
# The 3D push through whole steps in uniform periodic fields (weightless particles): the E x B drift
# state moves at exactly v_d = E_x/B_y along z; in a uniform B_y the momentum turns in the (z, x) plane by
# 2 atan(q B dt/(2 gamma m)) per step, with |u| and y unchanged.
def test_3d_push_through_full_steps_drift_and_gyration(orc):
    QEl, MEl = 1.602176634e-19, 9.1093837015e-31
    n, nz = 16, 40
    shape = (n + 1, n + 1, nz + 1)
    w = vacuum3(n, n, nz, "ck", courant=0.95)
    s = orc.Sim3(w)
    Ex, By = 6e7, 1.0
    vd = Ex / By                                   # 0.2 c
    gd = 1 / math.sqrt(1 - (vd / C) ** 2)
    s.set_field(0, np.full(shape, Ex))
    s.set_field(4, np.full(shape, By))
    x0, y0, z0 = 8.3 * s.dx, 7.6 * s.dy, 12.2 * s.dz
    s.set_particles(0, [x0], [y0], [z0], [0.0], [0.0], [gd * vd], [0.0])
    N = 60
    s.step(N)
    p = s.particles(0)
    assert p["alive"][0]
    assert p["z"][0] == pytest.approx(z0 + vd * N * s.dt, abs=1e-9 * s.dz)
    assert p["x"][0] == pytest.approx(x0, abs=1e-9 * s.dx) and p["y"][0] == y0
    assert p["uz"][0] == pytest.approx(gd * vd, rel=1e-9)

    s = orc.Sim3(w)
    B = 10.0                                       # gyration radius about one cell
    s.set_field(4, np.full(shape, B))
    u = np.array([0.005 * C, 0.0, 0.004 * C])
    g = math.sqrt(1 + (u @ u) / C ** 2)
    s.set_particles(0, [x0], [y0], [20.0 * s.dz], [u[0]], [u[1]], [u[2]], [0.0])
    N = 200
    s.step(N)
    p = s.particles(0)
    assert p["alive"][0] and p["y"][0] == y0
    assert math.hypot(p["ux"][0], p["uz"][0]) == pytest.approx(math.hypot(u[0], u[2]), rel=1e-13)
    # about +y the positive sense runs from z to x; an electron turns that way
    turned = math.atan2(p["ux"][0], p["uz"][0]) - math.atan2(u[0], u[2])
    expect = N * 2 * math.atan(QEl * B * s.dt / (2 * g * MEl))
    assert abs((turned - expect + math.pi) % (2 * math.pi) - math.pi) < 1e-9


# x <-> z mirror of the 3D step (dx = dz, nx = nz, gamma = 1): E'(i, j, k) = (E_z, E_y, E_x)(k, j, i),
# B' = -(B_z, B_y, B_x)(k, j, i), particles at (z, y, x) with (u_z, u_y, u_x); ties the 3D z-terms (the
# z layers, the z filter passes, the z deposit) to the x-terms. The particles stay in the middle of the box
# (the removal edge along z is one cell above the inflow plane).
def test_3d_mirror_x_z_with_pml_particles_and_filter(orc):
    rng = np.random.default_rng(37)
    n, ny, pml = 28, 28, 4
    w = vacuum3(n, ny, n, "ck", dx=0.8e-6, dy=1.1e-6, dz=0.8e-6, courant=0.9, theta=0.2, periodic=False,
                pml_cells=pml, filter_passes=2, filter_compensate=1, particle_guard=5)
    s1, s2, s0 = orc.Sim3(w), orc.Sim3(w), orc.Sim3(w)
    swap = {0: (2, 1.0), 1: (1, 1.0), 2: (0, 1.0), 3: (5, -1.0), 4: (4, -1.0), 5: (3, -1.0)}
    F = [_interior_noise(rng, (n + 1, ny + 1, n + 1), pml + 2, 3e9 if c < 3 else 3e9 / C) for c in range(6)]
    for comp in range(6):
        src, sign = swap[comp]
        s1.set_field(comp, F[comp])
        s0.set_field(comp, F[comp])
        s2.set_field(comp, sign * np.transpose(F[src], (2, 1, 0)))
    npart = 40
    x = rng.uniform(11.5, 16.5, npart) * s1.dx
    y = rng.uniform(11.5, 16.5, npart) * s1.dy
    z = rng.uniform(11.5, 16.5, npart) * s1.dz
    u = rng.standard_normal((3, npart)) * 0.05 * C
    wt = np.full(npart, 1e8)
    s1.set_particles(0, x, y, z, u[0], u[1], u[2], wt)
    s2.set_particles(0, z, y, x, u[2], u[1], u[0], wt)
    for s in (s0, s1, s2):
        s.step(30)
    for comp in range(6):
        src, sign = swap[comp]
        a = s2.field(comp)
        b = sign * np.transpose(s1.field(src), (2, 1, 0))
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), comp
    p1, p2 = s1.particles(0), s2.particles(0)
    assert len(p1["id"]) == npart and len(p2["id"]) == npart          # nobody left the particle domain
    o1, o2 = np.argsort(p1["id"]), np.argsort(p2["id"])
    for k1, k2, scale in (("x", "z", s1.dx), ("y", "y", s1.dy), ("z", "x", s1.dz),
                          ("ux", "uz", C), ("uy", "uy", C), ("uz", "ux", C)):
        assert np.abs(p2[k1][o2] - p1[k2][o1]).max() <= 1e-12 * scale, k1
    assert np.abs(p1["ux"][o1] - u[0]).max() > 1e-3 * C                  # the gather and push acted
    assert np.abs(s1.field(1) - s0.field(1)).max() > 0.1 * np.abs(s0.field(1)).max()   # the deposit acted
