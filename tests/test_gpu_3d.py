"""3D GPU path (CUDA library through the C ABI) against the 3D FP64 CPU oracle on the same seeded inputs.

FP64 GPU path: relative L2 <= 1e-10 on the fields, the particle state, the charge density, the lab-frame
samples and the beam; mixed path (FP32 fields, momenta and arithmetic, FP64 positions): relative L2
<= 1e-3 on the fields over the first steps of the same case.
"""
import numpy as np
import pytest

from paper_1009_2727_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-3
C = 299792458.0
EPS0 = 8.8541878128e-12


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


@pytest.fixture(scope="module")
def Sim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_2727_gb300.pic import Simulation
    return Simulation


def case(**over):
    w = W.shrink3(W.parity_3d(), 32, 32, 64)
    for k, v in over.items():
        if isinstance(v, dict) and isinstance(w.get(k), dict):
            w[k].update(v)
        else:
            w[k] = v
    return w


def check_fields(g, o, tol):
    worst = {}
    for name, grp in (("E", (0, 1, 2)), ("B", (3, 4, 5))):
        a = np.stack([g.field(c) for c in grp])
        b = np.stack([o.field(c) for c in grp])
        worst[name] = rel(a, b)
    assert all(v <= tol for v in worst.values()), worst
    return worst


def check_particles(g, o, tol, species=0):
    pg, po = g.particles(species), o.particles(species)
    po = {k: v[po["alive"]] for k, v in po.items()}
    assert len(pg["x"]) == len(po["x"]), (len(pg["x"]), len(po["x"]))
    ig, io = np.argsort(pg["id"], kind="stable"), np.argsort(po["id"], kind="stable")
    assert np.array_equal(pg["id"][ig], po["id"][io])
    for k in ("x", "y", "z"):
        assert np.abs(pg[k][ig] - po[k][io]).max() <= tol * np.abs(po[k]).max(), k
    ug = np.stack([pg[k][ig] for k in ("ux", "uy", "uz")])
    uo = np.stack([po[k][io] for k in ("ux", "uy", "uz")])
    assert rel(ug, uo) <= tol, rel(ug, uo)
    if species == 0:
        assert rel(pg["w"][ig], po["w"][io]) <= tol


def test_3d_vacuum_laser_pml_filter_fp64(Sim, orc):
    """antenna (dual particle arrays), CK2, PML on six faces, filter, Friedman damping; no plasma"""
    w = case(theta=0.2, filter_passes=2, filter_compensate=1)
    del w["plasma"]
    g = Sim(w, precision="fp64")
    o = orc.Sim3(w)
    g.step(40)
    o.step(40)
    g.sync()
    check_fields(g, o, TOL64)
    assert np.abs(o.field(1)).max() > 0


def test_3d_parity_plasma_laser_fp64(Sim, orc):
    w = case()
    g = Sim(w, precision="fp64")
    o = orc.Sim3(w)
    g.step(30)
    o.step(30)
    g.sync()
    check_fields(g, o, TOL64)
    check_particles(g, o, TOL64)
    # charge density (electrons, rigid ions, antenna pairs) and Gauss's law on the GPU's own fields
    rg, ro = g.field(9), o.rho()
    assert rel(rg, ro) <= TOL64
    st, dg = g.stats(), o.diag()
    assert st["n_electrons"] == dg["n_e"]
    assert st["field_energy"] == pytest.approx(dg["field_energy"], rel=1e-10)


def test_3d_linear_shapes_and_yee_fp64(Sim, orc):
    w = case(order=1, solver=W.SOLVERS["yee"], filter_passes=0, filter_J=0, filter_gather=0)
    g = Sim(w, precision="fp64")
    o = orc.Sim3(w)
    g.step(20)
    o.step(20)
    g.sync()
    check_fields(g, o, TOL64)
    check_particles(g, o, TOL64)


@pytest.mark.parametrize("gather", ["energy", "momentum"])
def test_3d_beam_and_lab_samples_fp64(Sim, orc, gather):
    w = case(gather=gather)
    rng = np.random.default_rng(12)
    n = 64
    x = w["laser"]["x_center"] + rng.normal(0, 1e-6, n)
    y = w["laser"]["y_center"] + rng.normal(0, 1e-6, n)
    z = rng.normal(2e-6, 0.3e-6, n)
    uz = np.sqrt(8.0 ** 2 - 1) * C * np.ones(n)     # gamma 8: +0.45 c in the boosted frame, stays in the box
    # lab plane at 3 um: the boosted crossings fall inside the particle domain, before t' = 0
    w["beam"] = {"x": x, "y": y, "z": z, "ux": np.zeros(n), "uy": np.zeros(n), "uz": uz, "t_lab": 0.0,
                 "z_plane_lab": 3e-6}
    g = Sim(w, precision="fp64")
    o = orc.Sim3(w)
    gam = w["gamma_boost"]
    beta = np.sqrt(1 - 1 / gam ** 2)
    dz = (1 + beta) * gam * w["dz_lab"]
    # lab rows of boosted events (z' = 15 um, t' inside the 40 steps below)
    tp = np.array([1e-14, 2e-14, 3e-14, 4.5e-14])
    zp = np.full_like(tp, 15e-6)
    zl = gam * (zp + beta * C * tp)
    tl = gam * (tp + beta * zp / C)
    o.btd_set(zl, tl)
    from paper_1009_2727_gb300 import capi
    import ctypes
    req = capi.PicBtdReq()
    req.struct_size, req.version = ctypes.sizeof(capi.PicBtdReq), capi.API_VERSION
    zz, tt = np.ascontiguousarray(zl), np.ascontiguousarray(tl)
    req.n_rows = zz.size
    req.z_lab = zz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    req.t_lab = tt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert g.L.pic_boosted_to_lab_diag(g.h, ctypes.byref(req), None) == 0
    g.step(40)
    o.step(40)
    g.sync()
    check_fields(g, o, TOL64)
    check_particles(g, o, TOL64, species=2)
    data = np.zeros(zz.size * 6 * 33 * 33)
    done = np.zeros(2 * zz.size, dtype=np.int32)
    out = capi.PicBtdOut()
    out.struct_size, out.version = ctypes.sizeof(capi.PicBtdOut), capi.API_VERSION
    out.data = data.ctypes.data_as(ctypes.c_void_p)
    out.done = done.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    out.on_device = 0
    assert g.L.pic_boosted_to_lab_diag(g.h, None, ctypes.byref(out)) == 0
    ref, rdone = o.btd_get()
    assert np.array_equal(done.reshape(-1, 2), rdone)
    assert rdone.sum() > 0
    assert rel(data.reshape(ref.shape), ref) <= TOL64
    st, dg = g.stats(), o.diag()
    assert st["n_beam_active"] == dg["n_beam"]
    if dg["n_beam"]:
        assert st["beam_gamma_lab"] == pytest.approx(dg["gamma_lab"], rel=1e-12)


def test_3d_wide_band_filter_strides_fp64(Sim, orc):
    """wide-band filter (Sec. 4.1): one pass and the compensation pass at strides 1 and 2 along each axis
    (halo 6, default guard 11); the antenna and the plasma edge sit inside the wider particle domain"""
    w = W.shrink3(W.parity_3d(), 40, 40, 80)
    w.update(filter_passes=1, filter_compensate=1, filter_strides=[1, 2])
    dzb = 0.4949e-6
    w["laser"]["z_antenna"] = 17 * dzb
    w["plasma"]["z_start_lab"] = 5.0 * 25 * dzb
    g = Sim(w, precision="fp64")
    o = orc.Sim3(w)
    g.step(40)
    o.step(40)
    g.sync()
    assert o.info()["guard"] == 11
    assert np.abs(o.field(1)).max() > 1e10
    check_fields(g, o, TOL64)
    check_particles(g, o, TOL64)


@pytest.mark.parametrize("order", [3, 1])
def test_3d_momentum_conserving_gather_fp64(Sim, orc, order):
    """'momentum conserving' gather (Sec. 5) in 3D: node-interpolated gather copies, node-centred shapes"""
    w = case(order=order, gather="momentum")
    g = Sim(w, precision="fp64")
    o = orc.Sim3(w)
    g.step(30)
    o.step(30)
    g.sync()
    check_fields(g, o, TOL64)
    check_particles(g, o, TOL64)


@pytest.mark.parametrize("steps", [20, 60])
def test_3d_mixed_vs_oracle(Sim, orc, steps):
    """the 3D mixed path against the FP64 oracle: the E and B vectors and each non-zero component on its own
    within 1e-3 in relative L2"""
    w = case()
    g = Sim(w, precision="mixed")
    o = orc.Sim3(w)
    g.step(steps)
    o.step(steps)
    g.sync()
    check_fields(g, o, TOLMIX)
    for c in range(6):
        ref = o.field(c)
        if np.abs(ref).max() > 0:
            assert rel(g.field(c), ref) <= TOLMIX, c


def test_3d_stage_workload_runs_mixed(Sim):
    """the 3D stage's numerics (gamma 30, CK2 at c dt = dz/sqrt(2), 16-cell PML, 4 passes + compensation)
    on a reduced box: finite fields and a steady plasma count"""
    w = W.shrink3(W.stage_3d(), 64, 64, 192)
    g = Sim(w, precision="mixed")
    n0 = g.stats()["n_electrons"]
    g.step(30)
    g.sync()
    st = g.stats()
    assert np.isfinite(st["field_energy"]) and st["field_energy"] > 0
    assert abs(st["n_electrons"] - n0) <= 0.05 * n0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_3d_self_consistent_beam_on_device(Sim, orc, precision):
    """the self-consistent test beam in 3D (Sec. 3.1.1, PR-27): 1500 frozen particles of a 1 pC, gamma 2 beam
    deposit their current while they move; their self-field, solved on the GPU (pic_beam_self_field: sine
    transforms along the three axes), equals the oracle's solve of the same discrete problem, and the run from
    it follows the oracle for 60 steps, fields and beam (FP64: 1e-10; mixed: 1e-3)"""
    n3 = (32, 32, 96)
    w = {"name": "beam_self_3d", "dim": 3, "nx": n3[0], "ny": n3[1], "nz": n3[2], "dz_lab": 1e-6, "dx": 1e-6,
         "dy": 1e-6, "gamma_boost": 1.0, "courant": 0.95, "dt": 0.0, "solver": W.SOLVERS["yee"], "theta": 0.0,
         "pml_cells": 0, "order": 3, "filter_passes": 0, "filter_J": 0, "filter_gather": 0, "precision": "fp64",
         "beam_self": 1}
    rng = np.random.default_rng(9)
    n = 1500
    x = rng.normal(16e-6, 2.5e-6, n)
    y = rng.normal(16e-6, 2.5e-6, n)
    z = rng.normal(35e-6, 2.5e-6, n)
    uz = np.full(n, np.sqrt(3.0) * C)
    zero = np.zeros(n)
    wts = np.full(n, 1e-12 / (1.602176634e-19 * n))
    o = orc.Sim3(w)
    o.set_beam(x, y, z, zero, zero, uz, 0.0, 1.0)
    o.beam_weights(wts)
    o.add_beam_self_field()
    wg = dict(w)
    wg["beam"] = {"x": x, "y": y, "z": z, "ux": zero, "uy": zero, "uz": uz, "t_lab": 0.0, "z_plane_lab": 1.0,
                  "self": 1, "w": wts}
    g = Sim(wg, precision=precision)
    g.beam_self_field()
    tol = TOL64 if precision == "fp64" else TOLMIX
    for c in (0, 1, 2, 3, 4):
        assert np.abs(o.field(c)).max() > 0, c
        assert rel(g.field(c), o.field(c)) <= tol, c
    g.step(60)
    o.step(60)
    g.sync()
    check_fields(g, o, tol)
    pg, po = g.particles(2), o.particles(2)
    for k in ("x", "y", "z", "uz"):
        assert rel(pg[k], po[k]) <= tol, k
