"""Python-side handle of one library context (marshalling through capi.py).

``Simulation(workload)`` creates a context from a workload dict (see
workloads.py): pic_init + pic_load_plasma + pic_inject_laser, with device
memory from torch's caching allocator on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi

_D = ctypes.POINTER(ctypes.c_double)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


class PicError(RuntimeError):
    pass


def make_config(w: dict, precision: int, tile=None, sort_every: int = 0) -> capi.PicConfig:
    """pic_config from a workload dict (SI units)."""
    c = capi.PicConfig()
    c.struct_size = ctypes.sizeof(capi.PicConfig)
    c.version = capi.API_VERSION
    c.dim = int(w.get("dim", 2))
    c.nx, c.nz = int(w.get("nx", 0)), int(w["nz"])
    if c.dim == 3:
        c.ny, c.dy = int(w["ny"]), float(w["dy"])
    c.dz_lab, c.dx = float(w["dz_lab"]), float(w.get("dx", 0.0))
    c.gamma_boost = float(w.get("gamma_boost", 1.0))
    c.courant = float(w.get("courant", 0.9))
    c.dt = float(w.get("dt", 0.0) or 0.0)
    c.ck_alpha, c.ck_beta, c.ck_gamma = (float(v) for v in w.get("solver", (1.0, 0.0, 0.0)))
    c.theta = float(w.get("theta", 0.0))
    c.pml_cells = int(w.get("pml_cells", 0))
    c.pml_sigma_max = float(w.get("pml_sigma_max", 4.0))
    c.pml_delta = float(w.get("pml_delta", 5.0))
    c.pml_power = float(w.get("pml_power", 2.0))
    c.pml_xi_exp = int(w.get("pml_xi_exp", 1))
    c.filter_passes = int(w.get("filter_passes", 0))
    c.filter_stride = int(w.get("filter_stride", 1))
    c.filter_compensate = int(w.get("filter_compensate", 0))
    for q, v in enumerate(list(w.get("filter_strides", []))[:4]):
        c.filter_stride_set[q] = int(v)
    c.gather_scheme = {"energy": 0, "momentum": 1}[w.get("gather", "energy")]
    c.filter_J = int(w.get("filter_J", 0))
    c.filter_gather = int(w.get("filter_gather", 0))
    c.shape_order = int(w.get("order", 3))
    c.particle_guard = int(w.get("particle_guard", -1))
    c.precision = precision
    c.moving_window = int(w.get("moving_window", 0))
    c.window_beta = float(w.get("window_beta", 0.0))
    if tile:
        c.tile_x, c.tile_z = int(tile[0]), int(tile[1])
    c.sort_every = int(sort_every or w.get("sort_every", 0))
    return c


def make_plasma(p: dict | None, beam: dict | None, keep: list) -> capi.PicPlasma:
    """pic_plasma from a plasma dict and an optional lab-frame test beam (arrays kept alive in keep)."""
    pl = capi.PicPlasma()
    pl.struct_size = ctypes.sizeof(capi.PicPlasma)
    pl.version = capi.API_VERSION
    if p:
        pl.n0 = float(p["n0"])
        pl.z_start_lab = float(p.get("z_start_lab", 0.0))
        pl.ramp_lab = float(p.get("ramp_lab", 0.0))
        pl.length_lab = float(p.get("length_lab", 0.0))
        pl.ppc_x, pl.ppc_z = int(p.get("ppc_x", 1)), int(p["ppc_z"])
        pl.ppc_y = int(p.get("ppc_y", 0))
        pl.ions = int(p.get("ions", 1))
    else:
        pl.ppc_x = pl.ppc_z = 1
    if beam:
        arrs = [np.ascontiguousarray(beam[k], dtype=np.float64) for k in ("x", "z", "ux", "uy", "uz")]
        keep.append(arrs)
        pl.beam_n = arrs[0].size
        pl.beam_x, pl.beam_z, pl.beam_ux, pl.beam_uy, pl.beam_uz = (_p(a) for a in arrs)
        if "y" in beam:
            ya = np.ascontiguousarray(beam["y"], dtype=np.float64)
            keep.append(ya)
            pl.beam_y = _p(ya)
        pl.beam_t_lab = float(beam.get("t_lab", 0.0))
        pl.beam_z_plane_lab = float(beam["z_plane_lab"])
        if beam.get("self"):
            wa = np.ascontiguousarray(beam["w"], dtype=np.float64)
            keep.append(wa)
            pl.beam_self = 1
            pl.beam_w = _p(wa)
    return pl


def make_laser(l: dict, nx: int, dx: float, ny: int = 0, dy: float = 0.0) -> capi.PicLaser:
    la = capi.PicLaser()
    la.struct_size = ctypes.sizeof(capi.PicLaser)
    la.version = capi.API_VERSION
    la.lambda0, la.a0, la.w0 = float(l["lambda0"]), float(l["a0"]), float(l.get("w0", 0.0))
    la.tau_fwhm, la.t_peak = float(l["tau_fwhm"]), float(l.get("t_peak", 0.0))
    la.x_center = float(l.get("x_center", 0.5 * nx * dx))
    la.phase, la.z_antenna, la.beta_s = float(l.get("phase", 0.0)), float(l["z_antenna"]), float(l.get("beta_s", 0.0))
    la.y_center = float(l.get("y_center", 0.5 * ny * dy))
    return la


def torch_allocator(device_index: int):
    """allocator callbacks on PyTorch's caching allocator (keep the returned pair alive)"""
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device_index, stream)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    return capi.ALLOC_FN(_alloc), capi.FREE_FN(_free)


def autotune(w: dict, steps: int = 16, precision: str | None = None, stream=None, warm: int = 4) -> dict:
    """Tile shape and sort cadence for this workload, timed on `steps` steps after `warm` untimed ones
    (pic_autotune_window; the result is cached per run shape and window inside the library)."""
    import torch
    L = capi.load()
    prec = precision or w.get("precision", "fp64")
    c = make_config(w, capi.PIC_FP64 if prec == "fp64" else capi.PIC_MIXED)
    keep = []
    pl = make_plasma(w.get("plasma"), w.get("beam"), keep)
    la = make_laser(w["laser"], int(w["nx"]), float(w["dx"])) if w.get("laser") else None
    st = stream if stream is not None else torch.cuda.current_stream()
    acb, fcb = torch_allocator(torch.cuda.current_device())
    out = capi.PicTuneResult()
    out.struct_size = ctypes.sizeof(capi.PicTuneResult)
    r = L.pic_autotune_window(ctypes.byref(c), ctypes.byref(pl), ctypes.byref(la) if la is not None else None,
                              int(warm), int(steps), acb, fcb, None, ctypes.c_void_p(st.cuda_stream),
                              ctypes.byref(out))
    if r != 0:
        raise PicError(f"pic_autotune failed: {capi.STATUS_NAMES.get(r, r)}")
    n = out.n_trials
    return {"tile": (out.tile_x, out.tile_z), "sort_every": out.sort_every, "ms_per_step": out.ms_per_step,
            "cached": bool(out.cached),
            "trials": [((out.trial_tile_x[i], out.trial_tile_z[i]), out.trial_sort_every[i], out.trial_ms[i])
                       for i in range(n)]}


class Simulation:
    def __init__(self, w: dict, precision: str | None = None, stream=None, tile=None, sort_every: int = 0,
                 use_torch_allocator: bool = True, tune: bool = False, tune_window: tuple = (4, 16)):
        import torch
        if not torch.cuda.is_available():
            raise PicError("a CUDA device is required (the library has no CPU path)")
        self.L = capi.load()
        self.w = dict(w)
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        prec = precision or w.get("precision", "fp64")
        self.precision = capi.PIC_FP64 if prec == "fp64" else capi.PIC_MIXED
        self.nx, self.nz = int(w.get("nx", 0)), int(w["nz"])
        self.dim = int(w.get("dim", 2))
        self.ny = int(w["ny"]) if self.dim == 3 else 0
        self.shape = ((self.nx + 1, self.ny + 1, self.nz + 1) if self.dim == 3 else (self.nz + 1,) if self.dim == 1
                      else (self.nx + 1, self.nz + 1))
        if tune:
            # the layout tuned on `tune_window` = (untimed, timed) steps of this run
            t = autotune(w, precision=prec, stream=self.stream, warm=int(tune_window[0]), steps=int(tune_window[1]))
            tile, sort_every = t["tile"], t["sort_every"]
            self.tuned = t
        c = make_config(w, self.precision, tile, sort_every)
        self._cfg = c
        self._keep = []
        if use_torch_allocator:
            self._alloc_cb, self._free_cb = torch_allocator(self.device.index)
        else:
            self._alloc_cb = capi.ALLOC_FN()
            self._free_cb = capi.FREE_FN()
        h = ctypes.c_void_p()
        r = self.L.pic_init(ctypes.byref(c), self._alloc_cb, self._free_cb, None,
                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if r != 0:
            raise PicError(f"pic_init failed: {capi.STATUS_NAMES.get(r, r)}")
        self.h = h
        if w.get("plasma") or w.get("beam"):
            self.load_plasma(w.get("plasma"), w.get("beam"))
        if w.get("laser"):
            self.inject_laser(w["laser"])

    # ------------------------------------------------------------------
    def _check(self, r: int, what: str):
        if r != 0:
            msg = self.L.pic_last_error(self.h).decode()
            raise PicError(f"{what} failed: {capi.STATUS_NAMES.get(r, r)} {msg}")

    def load_plasma(self, p: dict | None, beam: dict | None = None):
        pl = make_plasma(p, beam, self._keep)
        self._check(self.L.pic_load_plasma(self.h, ctypes.byref(pl)), "pic_load_plasma")

    def inject_laser(self, l: dict):
        la = make_laser(l, self.nx, float(self.w.get("dx", 0.0)), self.ny, float(self.w.get("dy", 0.0)))
        self._check(self.L.pic_inject_laser(self.h, ctypes.byref(la)), "pic_inject_laser")

    def step(self, n: int = 1):
        self._check(self.L.pic_step(self.h, int(n)), "pic_step")

    def sync(self):
        self._check(self.L.pic_sync(self.h), "pic_sync")

    def field(self, comp: int) -> np.ndarray:
        out = np.zeros(int(np.prod(self.shape)))
        self._check(self.L.pic_get_field(self.h, comp, _p(out), 0), "pic_get_field")
        return out.reshape(self.shape)

    def field_device(self, comp: int):
        t = self.torch.empty(self.shape, dtype=self.torch.float64, device=self.device)
        ptr = ctypes.cast(ctypes.c_void_p(t.data_ptr()), _D)
        self._check(self.L.pic_get_field(self.h, comp, ptr, 1), "pic_get_field")
        return t

    def set_field(self, comp: int, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        self._check(self.L.pic_set_field(self.h, comp, _p(a)), "pic_set_field")

    def beam_self_field(self):
        """add the frozen test beam's self-field, solved on the device (pic_beam_self_field)"""
        self._check(self.L.pic_beam_self_field(self.h), "pic_beam_self_field")

    def particles(self, species: int = capi.ELECTRONS) -> dict:
        n = ctypes.c_int64(0)
        self._check(self.L.pic_get_particles(self.h, species, None, None, None, None, None, None, None, None,
                                             ctypes.byref(n)), "pic_get_particles")
        cnt = max(int(n.value), 1)
        a = {k: np.zeros(cnt) for k in ("x", "z", "ux", "uy", "uz", "w")}
        ids = np.zeros(cnt, dtype=np.uint32)
        fl = np.zeros(cnt, dtype=np.int32)
        n = ctypes.c_int64(cnt)
        self._check(self.L.pic_get_particles(self.h, species, *(_p(a[k]) for k in ("x", "z", "ux", "uy", "uz", "w")),
                                             ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                             fl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(n)),
                    "pic_get_particles")
        m = int(n.value)
        out = {k: v[:m] for k, v in a.items()}
        if getattr(self, "dim", 2) == 3:
            y = np.zeros(cnt)
            n = ctypes.c_int64(cnt)
            self._check(self.L.pic_get_particles_y(self.h, species, _p(y), ctypes.byref(n)), "pic_get_particles_y")
            out["y"] = y[:m]
        out["id"] = ids[:m]
        out["alive"] = (fl[:m] & 1) != 0
        out["active"] = (fl[:m] & 2) != 0
        return out

    def stats(self, trap_gamma_lab: float = 0.0) -> dict:
        """diagnostics; trap_gamma_lab > 0 replaces the default trapping threshold (twice gamma_w)"""
        s = capi.PicStats()
        s.struct_size = ctypes.sizeof(capi.PicStats)
        s.version = capi.API_VERSION
        s.trap_gamma_lab = float(trap_gamma_lab)
        self._check(self.L.pic_get_stats(self.h, ctypes.byref(s)), "pic_get_stats")
        return {k: getattr(s, k) for k, _ in capi.PicStats._fields_ if k not in ("struct_size", "version")}

    def btd_set(self, z_lab: np.ndarray, t_lab: np.ndarray):
        z = np.ascontiguousarray(z_lab, dtype=np.float64)
        t = np.ascontiguousarray(t_lab, dtype=np.float64)
        r = capi.PicBtdReq()
        r.struct_size = ctypes.sizeof(capi.PicBtdReq)
        r.version = capi.API_VERSION
        r.n_rows = z.size
        r.z_lab, r.t_lab = _p(z), _p(t)
        self._btd_rows = z.size
        self._check(self.L.pic_boosted_to_lab_diag(self.h, ctypes.byref(r), None), "pic_boosted_to_lab_diag")

    def btd_get(self):
        n = self._btd_rows
        dt = np.float64 if self.precision == capi.PIC_FP64 else np.float32
        data = np.zeros(n * 6 * (self.nx + 1), dtype=dt)
        done = np.zeros(2 * n, dtype=np.int32)
        o = capi.PicBtdOut()
        o.struct_size = ctypes.sizeof(capi.PicBtdOut)
        o.version = capi.API_VERSION
        o.data = data.ctypes.data_as(ctypes.c_void_p)
        o.done = done.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        o.on_device = 0
        self._check(self.L.pic_boosted_to_lab_diag(self.h, None, ctypes.byref(o)), "pic_boosted_to_lab_diag")
        return data.reshape(n, 6, self.nx + 1).astype(np.float64), done.reshape(n, 2)

    def launches(self) -> int:
        return int(self.L.pic_kernel_launches(self.h))

    def timing(self, enable: bool, which: int = 0):
        ms = ctypes.c_double(0.0)
        nl = ctypes.c_int64(0)
        self._check(self.L.pic_kernel_timing(self.h, int(enable), int(which), ctypes.byref(ms), ctypes.byref(nl)),
                    "pic_kernel_timing")
        return ms.value, nl.value

    def close(self):
        h = getattr(self, "h", None)
        if h:
            self.L.pic_free(h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Member(Simulation):
    """a run of an Ensemble: the accessors of Simulation on a context the ensemble owns"""

    def __init__(self, ens, h, w, precision):
        import torch
        self.L, self.h, self.w, self.torch = ens.L, h, dict(w), torch
        self.device = ens.device
        self.stream = None
        self.precision = precision
        self.nx, self.nz = int(w["nx"]), int(w["nz"])
        self.dim = int(w.get("dim", 2))
        self.ny = int(w["ny"]) if self.dim == 3 else 0
        self.shape = (self.nx + 1, self.ny + 1, self.nz + 1) if self.dim == 3 else (self.nx + 1, self.nz + 1)
        self._keep = []

    def step(self, n: int = 1):
        raise PicError("a member of an ensemble advances with the ensemble")

    def close(self):
        self.h = None     # owned by the ensemble


class Ensemble:
    """Independent runs of uneven size advanced together (pic_ensemble_*): in batched mode one launch per
    kernel class advances every run (replayed from a CUDA graph); otherwise each run has its own stream and
    the runs of one step execute concurrently."""

    def __init__(self, ws: list, precision: str | None = None, stream=None, tune=False):
        """tune: False (each run's own configuration), "runs" (each run's tile and sort cadence from
        pic_autotune, timed on that run alone) or "ensemble" (one layout for all runs from
        pic_ensemble_autotune, timed on the ensemble itself)"""
        import torch
        if not torch.cuda.is_available():
            raise PicError("a CUDA device is required (the library has no CPU path)")
        self.L = capi.load()
        self.device = torch.device("cuda", torch.cuda.current_device())
        st = stream if stream is not None else torch.cuda.current_stream()
        n = len(ws)
        precs = [(precision or w.get("precision", "fp64")) for w in ws]
        self._keep = []
        self.tuned = []
        layouts = [(None, 0)] * n
        if tune == "runs" or tune is True:
            for i, (w, p) in enumerate(zip(ws, precs)):
                t = autotune(w, steps=8, precision=p, stream=st)
                self.tuned.append(t)
                layouts[i] = (t["tile"], t["sort_every"])
        elif tune == "ensemble":
            c0 = (capi.PicConfig * n)(*[make_config(w, capi.PIC_FP64 if p == "fp64" else capi.PIC_MIXED)
                                        for w, p in zip(ws, precs)])
            p0 = (capi.PicPlasma * n)(*[make_plasma(w.get("plasma"), w.get("beam"), self._keep) for w in ws])
            l0 = (capi.PicLaser * n)()
            for i, w in enumerate(ws):
                if w.get("laser"):
                    l0[i] = make_laser(w["laser"], int(w["nx"]), float(w["dx"]), int(w.get("ny", 0)),
                                       float(w.get("dy", 0.0)))
            acb, fcb = torch_allocator(self.device.index)
            out = capi.PicTuneResult()
            out.struct_size = ctypes.sizeof(capi.PicTuneResult)
            r = self.L.pic_ensemble_autotune(n, c0, p0, l0, 8, acb, fcb, None, ctypes.c_void_p(st.cuda_stream),
                                             ctypes.byref(out))
            if r != 0:
                raise PicError(f"pic_ensemble_autotune failed: {capi.STATUS_NAMES.get(r, r)}")
            t = {"tile": (out.tile_x, out.tile_z), "sort_every": out.sort_every, "ms_per_step": out.ms_per_step,
                 "trials": [((out.trial_tile_x[i], out.trial_tile_z[i]), out.trial_sort_every[i], out.trial_ms[i])
                            for i in range(out.n_trials)]}
            self.tuned = [t] * n
            layouts = [(t["tile"], t["sort_every"])] * n
        cfgs = (capi.PicConfig * n)(*[make_config(w, capi.PIC_FP64 if p == "fp64" else capi.PIC_MIXED, tl, se)
                                      for w, p, (tl, se) in zip(ws, precs, layouts)])
        pls = (capi.PicPlasma * n)(*[make_plasma(w.get("plasma"), w.get("beam"), self._keep) for w in ws])
        las = (capi.PicLaser * n)()
        for i, w in enumerate(ws):
            if w.get("laser"):
                las[i] = make_laser(w["laser"], int(w["nx"]), float(w["dx"]), int(w.get("ny", 0)),
                                    float(w.get("dy", 0.0)))
        self._alloc_cb, self._free_cb = torch_allocator(self.device.index)
        h = ctypes.c_void_p()
        r = self.L.pic_ensemble_create(n, cfgs, pls, las, self._alloc_cb, self._free_cb, None,
                                       ctypes.c_void_p(st.cuda_stream), ctypes.byref(h))
        if r != 0:
            raise PicError(f"pic_ensemble_create failed: {capi.STATUS_NAMES.get(r, r)}")
        self.h = h
        self.members = [_Member(self, self.L.pic_ensemble_member(h, i), w,
                                capi.PIC_FP64 if p == "fp64" else capi.PIC_MIXED)
                        for i, (w, p) in enumerate(zip(ws, precs))]

    def step(self, n: int = 1):
        r = self.L.pic_ensemble_step(self.h, int(n))
        if r != 0:
            raise PicError(f"pic_ensemble_step failed: {capi.STATUS_NAMES.get(r, r)}")

    @property
    def batched(self) -> bool:
        """the runs step through the batched kernels (one launch per kernel class per ensemble step)"""
        return bool(self.L.pic_ensemble_batched(self.h))

    def use_graphs(self, enable: bool = True):
        """batched mode: replay every step from a CUDA graph (the default) or launch the kernels directly"""
        self.L.pic_ensemble_use_graphs(self.h, int(bool(enable)))

    def launches(self) -> int:
        return int(self.L.pic_ensemble_launches(self.h))

    def sync(self):
        r = self.L.pic_ensemble_sync(self.h)
        if r != 0:
            raise PicError(f"pic_ensemble_sync failed: {capi.STATUS_NAMES.get(r, r)}")

    def __len__(self):
        return len(self.members)

    def __getitem__(self, i):
        return self.members[i]

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None
            self.L.pic_ensemble_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
