"""Sec. 5, scan of the time step: on the 2D stage workload the gather from the Yee locations keeps the
high-k E_z power low up to the singular step c dt = dz/sqrt(2) and far lower than at 0.8, while the
node-interpolated ('momentum conserving') gather lets the instability grow by orders of magnitude more at
the same step (the paper: high at every step). Mixed path, one GB300."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_dt_scan_energy_vs_momentum_conserving_gather():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_2727_gb300 import stability
    ec = {r["c_dt_over_dz"]: r["high_k"][-1]
          for r in stability.dt_scan((0.7071, 0.8), schemes=("energy",), marks=(2400,))}
    mc = stability.dt_scan((0.7071,), schemes=("momentum",), marks=(2400,))[0]["high_k"][-1]
    assert all(np.isfinite(v) and v > 0 for v in ec.values())
    # measured: 2.7e22 at dz/sqrt(2) and 3.4e23 at 0.8 (energy conserving), 3.9e29 (momentum conserving)
    assert ec[0.8] > 3.0 * ec[0.7071]
    assert mc > 1e3 * ec[0.7071]
