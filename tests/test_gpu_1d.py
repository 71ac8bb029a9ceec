"""1D path (CUDA library through the C ABI, pic_config.dim = 1) against the 1D FP64 CPU oracle on the same
inputs: FP64 at relative L2 <= 1e-10 on the fields, the electrons (matched by id), the charge density and
the diagnostics; the mixed path at 1e-3 on the fields."""
import numpy as np
import pytest

from paper_1009_2727_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-3


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


def run(Sim, orc, w, steps, precision="fp64"):
    g = Sim(w, precision=precision)
    o = orc.Sim1(w)
    g.step(steps)
    o.step(steps)
    g.sync()
    return g, o


def check_fields(g, o, tol):
    worst = {}
    for name, grp in (("E", (0, 1, 2)), ("B", (3, 4, 5))):
        worst[name] = rel(np.stack([g.field(c) for c in grp]), np.stack([o.field(c) for c in grp]))
    assert all(v <= tol for v in worst.values()), worst


def check_electrons(g, o, tol):
    pg, po = g.particles(0), o.particles(0)
    assert len(pg["z"]) == len(po["z"]), (len(pg["z"]), len(po["z"]))
    ig, io = np.argsort(pg["id"], kind="stable"), np.argsort(po["id"], kind="stable")
    assert np.array_equal(pg["id"][ig], po["id"][io])
    assert np.abs(pg["z"][ig] - po["z"][io]).max() <= tol * np.abs(po["z"]).max()
    ug = np.stack([pg[k][ig] for k in ("ux", "uy", "uz")])
    uo = np.stack([po[k][io] for k in ("ux", "uy", "uz")])
    assert rel(ug, uo) <= tol
    assert rel(pg["w"][ig], po["w"][io]) <= tol


def test_1d_vacuum_laser_pml_filter_fp64(Sim, orc):
    w = W.parity_1d()
    del w["plasma"]
    g, o = run(Sim, orc, w, 300)
    assert np.abs(o.field(1)).max() > 1e10
    check_fields(g, o, TOL64)


def test_1d_parity_plasma_laser_boosted_fp64(Sim, orc):
    w = W.parity_1d()
    g, o = run(Sim, orc, w, 300)
    check_fields(g, o, TOL64)
    check_electrons(g, o, TOL64)
    assert rel(g.field(9), o.rho()) <= TOL64
    st, dg = g.stats(), o.diag()
    assert st["n_electrons"] == dg["n_e"]
    assert st["field_energy"] == pytest.approx(dg["field_energy"], rel=1e-10)


def test_1d_linear_nodal_gather_wide_filter_fp64(Sim, orc):
    w = W.parity_1d(gamma_boost=2.0)
    w.update(order=1, gather="momentum", filter_passes=1, filter_compensate=1, filter_strides=[1, 2])
    g, o = run(Sim, orc, w, 250)
    check_fields(g, o, TOL64)
    check_electrons(g, o, TOL64)


def test_1d_lab_frame_moving_window_app1_fp64(Sim, orc):
    """App. I's scaled stage in the lab frame with the window moving at c and c dt = dz, over its first
    steps (the window has shifted and the plasma has entered), with and without the current filter"""
    for filtered in (True, False):
        w = W.app1_lwfa(filtered)
        w["precision"] = "fp64"
        g, o = run(Sim, orc, w, 700)
        assert o.info()["z0"] > 0
        assert o.diag()["n_e"] > 1000
        check_fields(g, o, TOL64)
        check_electrons(g, o, TOL64)
        assert g.stats()["z0"] == pytest.approx(o.info()["z0"], rel=1e-15)


def test_1d_mixed_vs_oracle(Sim, orc):
    w = W.parity_1d()
    g, o = run(Sim, orc, w, 300, precision="mixed")
    check_fields(g, o, TOLMIX)
