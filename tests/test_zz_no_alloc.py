"""pic_get_rho_noalloc: the charge density computed without any device allocation.

Callers that must not allocate device memory once their run is set up (an
application whose device memory belongs entirely to its own pool allocator, or a
real-time loop that cannot afford cudaMalloc's latency and implicit
synchronisation) read the density through this entry point. It must return
what pic_get_field(PIC_RHO) returns, call after call, although its scratch is
a static device array shared by every call.
"""
import ctypes

import numpy as np
import pytest

from paper_1009_2727_gb300 import capi
from paper_1009_2727_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rho_noalloc_matches_accessor_on_consecutive_calls(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_2727_gb300.pic import Simulation
    w = W.shrink(W.parity_2d(), 48, 160)
    sim = Simulation(w, precision=precision)
    sim.step(25)
    L = capi.load()
    out = torch.empty((sim.nx + 1, sim.nz + 1), dtype=torch.float64, device="cuda")
    ptr = ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double))
    # rho is the small difference of the electron and ion densities: round-off from the order of the
    # atomic additions is measured against one species' density e gamma n0
    scale = 1.602176634e-19 * w["gamma_boost"] * w["plasma"]["n0"]
    tol = 1e-10
    for call in range(2):
        ref = sim.field(capi.RHO)
        out.fill_(123.0)                      # stale contents must not leak into the result
        torch.cuda.synchronize()
        # the library allocates through torch's caching allocator (its allocator callback), and a direct
        # cudaMalloc would show in the device's free memory: neither may move during the call
        n_alloc = torch.cuda.memory_stats()["allocation.all.allocated"]
        free0, _ = torch.cuda.mem_get_info()
        r = L.pic_get_rho_noalloc(sim.h, ptr)
        assert r == capi.PIC_OK, sim.L.pic_last_error(sim.h)
        sim.sync()
        assert torch.cuda.memory_stats()["allocation.all.allocated"] == n_alloc
        assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy()
        assert np.abs(ref).max() > 0
        err = np.abs(got - ref).max() / scale
        assert err <= tol, (call, err)
        sim.step(3)
    sim.close()


def test_rho_noalloc_rejects_grid_above_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_2727_gb300.pic import Simulation
    w = {"nx": 16, "nz": capi.NOALLOC_MAX_NZ + 8, "dz_lab": 1e-7, "dx": 1e-6, "gamma_boost": 1.0,
         "solver": W.SOLVERS["yee"], "order": 1, "precision": "fp64"}
    sim = Simulation(w, precision="fp64")
    out = torch.empty((17, w["nz"] + 1), dtype=torch.float64, device="cuda")
    ptr = ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double))
    r = capi.load().pic_get_rho_noalloc(sim.h, ptr)
    assert r == capi.PIC_EINVAL
    assert b"PIC_NOALLOC_MAX_NZ" in sim.L.pic_last_error(sim.h)
    sim.close()
