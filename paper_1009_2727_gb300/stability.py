"""Time-step scan of the numerical instability for the two gather schemes (Sec. 5, 'Effects of time
step' and the scan repeated with the 'momentum conserving' gather).

The paper compares the spectrum of E_z averaged over the domain at a fixed time for c dt / dz between 0.5
and 1: with the gather from the Yee locations ('energy conserving') the instability is lowest at the
singular step c dt = dz / sqrt(2); with node-interpolated fields ('momentum conserving') it stays high at
every step. Here the same comparison runs on the 2D stage workload: each run is stepped to the same
physical times, E_z is read back and its power along z above k dz = pi/4 (far above the laser and the
wake, which sit below k dz = 0.1) measures the instability. Host-side analysis of the GPU runs only.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

C = 299792458.0


def high_k_power(ez: np.ndarray, margin: int, k_cut: float = np.pi / 4) -> tuple[float, float]:
    """power of E_z along z above and below k dz = k_cut, over the grid minus `margin` cells per side"""
    seg = ez[margin:-margin, margin:-margin]
    p = np.abs(np.fft.rfft(seg, axis=1)) ** 2
    kdz = np.arange(p.shape[1]) * 2 * np.pi / seg.shape[1]
    return float(p[:, kdz > k_cut].sum()), float(p[:, kdz <= k_cut].sum())


def dt_scan(ratios, schemes=("energy", "momentum"), marks=(1200, 1800, 2400), workload: dict | None = None,
            precision: str = "mixed") -> list[dict]:
    """Step the stage workload at c dt = r dz for each r and gather scheme to the physical times
    t_m = m (dz / sqrt(2)) / c, m in marks; return per run the high- and low-k power of E_z at each time."""
    from .pic import Simulation
    base = workload if workload is not None else W.stage_2d()
    g = base["gamma_boost"]
    dz = (1.0 + np.sqrt(1.0 - 1.0 / g ** 2)) * g * base["dz_lab"]
    times = [m * dz / (np.sqrt(2.0) * C) for m in marks]
    out = []
    for scheme in schemes:
        for r in ratios:
            w = dict(base)
            w["gather"] = scheme
            w["dt"] = r * dz / C
            s = Simulation(w, precision=precision)
            done = 0
            rec = {"gather": scheme, "c_dt_over_dz": r, "t": times, "steps": [], "high_k": [], "low_k": []}
            for t in times:
                n = int(round(t / w["dt"]))
                s.step(n - done)
                done = n
                hk, lk = high_k_power(s.field(2), w["pml_cells"] + 40)
                rec["steps"].append(n)
                rec["high_k"].append(hk)
                rec["low_k"].append(lk)
            s.close()
            out.append(rec)
    return out


def nyquist_fraction(f: np.ndarray, margin: int) -> float:
    """share of the one-sided power spectrum of a 1D field in its top quarter of wavenumbers (k dz > 3 pi/4),
    the band of the odd-even mode of App. I, over the grid minus `margin` cells per side"""
    seg = f[margin:-margin]
    p = np.abs(np.fft.rfft(seg)) ** 2
    kdz = np.arange(p.size) * 2 * np.pi / seg.size
    tot = p.sum()
    return float(p[kdz > 0.75 * np.pi].sum() / tot) if tot > 0 else 0.0


def app1_runs(steps: int = 20000, precision: str = "mixed", every: int = 0) -> list[dict]:
    """App. I's 1D scaled stage at c dt = dz with and without one bilinear pass on the current: per run
    the Nyquist-band share of E_y and of E_z at the end (and every `every` steps when > 0), the peak
    wake field and the electron count."""
    from .pic import Simulation
    out = []
    for filtered in (False, True):
        w = W.app1_lwfa(filtered)
        s = Simulation(w, precision=precision)
        rec = {"filtered": filtered, "steps": steps, "history": []}
        done = 0
        chunk = every if every > 0 else steps
        while done < steps:
            n = min(chunk, steps - done)
            s.step(n)
            done += n
            ey, ez = s.field(1), s.field(2)
            m = w["pml_cells"] + 10
            rec["history"].append({"step": done, "nyq_Ey": nyquist_fraction(ey, m), "nyq_Ez": nyquist_fraction(ez, m),
                                   "max_Ez": float(np.abs(ez[m:-m]).max()), "max_Ey": float(np.abs(ey[m:-m]).max())})
        st = s.stats()
        rec.update(rec["history"][-1])
        rec["n_electrons"] = st["n_electrons"]
        s.close()
        out.append(rec)
    return out
