"""App. I on the GPU: the 1D scaled laser-wakefield stage (Table Tablephyspar) at c dt = dz over 20000
steps. Without filtering of the current an instability grows at the grid Nyquist frequency (the odd-even
mode of Eq. 1db-1de, driven resonantly) and swamps the fields; one bilinear pass on the current, without
compensation, removes it and the laser keeps its amplitude. Mixed path, one GB300."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_app1_nyquist_instability_and_its_filter():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_2727_gb300 import stability
    runs = {r["filtered"]: r for r in stability.app1_runs(20000)}
    C, QE, ME = 299792458.0, 1.602176634e-19, 9.1093837015e-31
    e0 = 1.0 * ME * C * (2 * math.pi * C / 0.8e-6) / QE
    # measured: Nyquist share 0.999 and max |E_y| 7e15 V/m unfiltered; 0.0 and 4.0e12 filtered
    assert runs[False]["nyq_Ey"] > 0.9
    assert runs[False]["max_Ey"] > 100 * e0
    assert runs[True]["nyq_Ey"] < 1e-3
    assert runs[True]["max_Ey"] == pytest.approx(e0, rel=0.15)
    assert runs[True]["n_electrons"] > 8000
