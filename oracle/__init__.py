"""FP64 CPU oracle of the boosted-frame PIC step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package. The product path (the CUDA
library behind ``include/pic.h`` and its Python binding) never imports it, and
this package imports nothing from the product.

``pic_oracle.c`` (2-1/2D), ``pic_oracle3d.c`` (3D) and ``pic_oracle1d.c`` (1D) restate the method of
Vay et al., "Modeling laser wakefield accelerators in a Lorentz boosted frame"
(arXiv:1009.2727) in plain double precision loops; this module builds them
with gcc into one library and exposes it through ctypes.
``boost.py`` holds the paper's analytic frame/speed-up formulas (Sec. 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRCS = [os.path.join(_HERE, "pic_oracle.c"), os.path.join(_HERE, "pic_oracle3d.c"),
         os.path.join(_HERE, "pic_oracle1d.c")]
_lock = threading.Lock()
_lib = None

C = 299792458.0
QE = 1.602176634e-19
EPS0 = 8.8541878128e-12

# component ids used by the oracle: E, B, J
EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)
COMPONENTS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")


def build(force: bool = False) -> str:
    """Compile the oracle sources into oracle/_build/liboracle.so (plain gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(f) for f in _SRCS):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("nz", ctypes.c_int),
        ("dz_lab", ctypes.c_double), ("dx", ctypes.c_double), ("gamma_boost", ctypes.c_double),
        ("courant", ctypes.c_double), ("dt_override", ctypes.c_double),
        ("ck_alpha", ctypes.c_double), ("ck_beta", ctypes.c_double), ("ck_gamma", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("pml_cells", ctypes.c_int), ("pml_sigma_max", ctypes.c_double), ("pml_delta", ctypes.c_double),
        ("pml_power", ctypes.c_double), ("pml_xi_exp", ctypes.c_int),
        ("filter_passes", ctypes.c_int), ("filter_stride", ctypes.c_int), ("filter_compensate", ctypes.c_int),
        ("filter_J", ctypes.c_int), ("filter_gather", ctypes.c_int),
        ("order", ctypes.c_int), ("particle_guard", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("periodic_z", ctypes.c_int),
        ("moving_window", ctypes.c_int), ("window_beta", ctypes.c_double),
        ("filter_strides", ctypes.c_int * 4), ("gather_nodal", ctypes.c_int), ("beam_self", ctypes.c_int),
    ]


class _Plasma(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_double), ("z_start_lab", ctypes.c_double), ("ramp_lab", ctypes.c_double),
                ("length_lab", ctypes.c_double), ("ppc_x", ctypes.c_int), ("ppc_z", ctypes.c_int),
                ("ions", ctypes.c_int)]


class _Laser(ctypes.Structure):
    _fields_ = [("lambda0", ctypes.c_double), ("a0", ctypes.c_double), ("w0", ctypes.c_double),
                ("tau_fwhm", ctypes.c_double), ("t_peak", ctypes.c_double), ("x_center", ctypes.c_double),
                ("phase", ctypes.c_double), ("z_antenna", ctypes.c_double), ("beta_s", ctypes.c_double)]


class _Config3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dz_lab", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("gamma_boost", ctypes.c_double), ("courant", ctypes.c_double), ("dt_override", ctypes.c_double),
        ("ck_alpha", ctypes.c_double), ("ck_beta", ctypes.c_double), ("ck_gamma", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("pml_cells", ctypes.c_int), ("pml_sigma_max", ctypes.c_double), ("pml_delta", ctypes.c_double),
        ("pml_power", ctypes.c_double), ("pml_xi_exp", ctypes.c_int),
        ("filter_passes", ctypes.c_int), ("filter_stride", ctypes.c_int), ("filter_compensate", ctypes.c_int),
        ("filter_J", ctypes.c_int), ("filter_gather", ctypes.c_int),
        ("order", ctypes.c_int), ("particle_guard", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int), ("periodic_z", ctypes.c_int),
        ("filter_strides", ctypes.c_int * 4), ("gather_nodal", ctypes.c_int), ("beam_self", ctypes.c_int),
    ]


class _Plasma3(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_double), ("z_start_lab", ctypes.c_double), ("ramp_lab", ctypes.c_double),
                ("length_lab", ctypes.c_double), ("ppc_x", ctypes.c_int), ("ppc_y", ctypes.c_int),
                ("ppc_z", ctypes.c_int), ("ions", ctypes.c_int)]


class _Laser3(ctypes.Structure):
    _fields_ = [("lambda0", ctypes.c_double), ("a0", ctypes.c_double), ("w0", ctypes.c_double),
                ("tau_fwhm", ctypes.c_double), ("t_peak", ctypes.c_double), ("x_center", ctypes.c_double),
                ("y_center", ctypes.c_double), ("phase", ctypes.c_double), ("z_antenna", ctypes.c_double)]


class _Config1(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int), ("dz_lab", ctypes.c_double), ("gamma_boost", ctypes.c_double),
        ("courant", ctypes.c_double), ("dt_override", ctypes.c_double), ("theta", ctypes.c_double),
        ("pml_cells", ctypes.c_int), ("pml_sigma_max", ctypes.c_double), ("pml_delta", ctypes.c_double),
        ("pml_power", ctypes.c_double), ("pml_xi_exp", ctypes.c_int),
        ("filter_passes", ctypes.c_int), ("filter_stride", ctypes.c_int), ("filter_compensate", ctypes.c_int),
        ("filter_J", ctypes.c_int), ("filter_gather", ctypes.c_int),
        ("order", ctypes.c_int), ("particle_guard", ctypes.c_int),
        ("moving_window", ctypes.c_int), ("window_beta", ctypes.c_double),
        ("filter_strides", ctypes.c_int * 4), ("gather_nodal", ctypes.c_int),
    ]


class _Plasma1(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_double), ("z_start_lab", ctypes.c_double), ("ramp_lab", ctypes.c_double),
                ("length_lab", ctypes.c_double), ("ppc_z", ctypes.c_int), ("ions", ctypes.c_int)]


class _Laser1(ctypes.Structure):
    _fields_ = [("lambda0", ctypes.c_double), ("a0", ctypes.c_double), ("tau_fwhm", ctypes.c_double),
                ("t_peak", ctypes.c_double), ("phase", ctypes.c_double), ("z_antenna", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(_Config)]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_load_plasma.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Plasma)]
            L.orc_set_laser.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Laser)]
            L.orc_set_beam.argtypes = [ctypes.c_void_p, ctypes.c_long, _D, _D, _D, _D, _D,
                                       ctypes.c_double, ctypes.c_double]
            L.orc_info.argtypes = [ctypes.c_void_p, _D]
            for f in ("orc_get_field", "orc_set_field", "orc_get_gather_field"):
                getattr(L, f).argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
            L.orc_get_history.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D]
            L.orc_set_history.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D]
            L.orc_set_ext_current.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_int]
            L.orc_set_ext_profile.argtypes = [ctypes.c_void_p, ctypes.c_long, _D]
            L.orc_num_particles.restype = ctypes.c_long
            L.orc_num_particles.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_get_particles.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, _D, _D, _D, _D, _D,
                                            ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int)]
            L.orc_set_particles.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_long, _D, _D, _D, _D, _D, _D]
            L.orc_rho.argtypes = [ctypes.c_void_p, _D]
            L.orc_diag.argtypes = [ctypes.c_void_p, _D]
            L.orc_btd_set.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, _D]
            L.orc_btd_get.argtypes = [ctypes.c_void_p, _D, ctypes.POINTER(ctypes.c_int)]
            L.orc_filter_field.argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
            L.orc_deposit_one.argtypes = [ctypes.c_void_p, _D, _D, _D] + [ctypes.c_double] * 6
            L.orc_rho_one.argtypes = [ctypes.c_void_p, _D] + [ctypes.c_double] * 3
            L.orc_beam_weights.argtypes = [ctypes.c_void_p, _D]
            L.orc_shape.restype = ctypes.c_double
            L.orc_shape.argtypes = [ctypes.c_int, ctypes.c_double]
            L.orc_cfl_2d.restype = ctypes.c_double
            L.orc_cfl_2d.argtypes = [ctypes.c_double] * 6
            L.orc_cfl_3d.restype = ctypes.c_double
            L.orc_cfl_3d.argtypes = [ctypes.c_double] * 7
            L.orc_filter_line.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int]
            L.orc_boris.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            vp = ctypes.c_void_p
            L.o3_create.restype = vp
            L.o3_create.argtypes = [ctypes.POINTER(_Config3)]
            L.o3_destroy.argtypes = [vp]
            L.o3_step.argtypes = [vp, ctypes.c_int]
            L.o3_load_plasma.argtypes = [vp, ctypes.POINTER(_Plasma3)]
            L.o3_set_laser.argtypes = [vp, ctypes.POINTER(_Laser3)]
            L.o3_set_beam.argtypes = [vp, ctypes.c_long, _D, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double]
            L.o3_info.argtypes = [vp, _D]
            for f in ("o3_get_field", "o3_set_field", "o3_get_gather_field", "o3_filter_field"):
                getattr(L, f).argtypes = [vp, ctypes.c_int, _D]
            L.o3_num_particles.restype = ctypes.c_long
            L.o3_num_particles.argtypes = [vp, ctypes.c_int]
            L.o3_get_particles.argtypes = [vp, ctypes.c_int] + [_D] * 7 + [ctypes.POINTER(ctypes.c_uint32),
                                                                            ctypes.POINTER(ctypes.c_int)]
            L.o3_set_particles.argtypes = [vp, ctypes.c_int, ctypes.c_long] + [_D] * 7
            L.o3_rho.argtypes = [vp, _D]
            L.o3_diag.argtypes = [vp, _D]
            L.o3_btd_set.argtypes = [vp, ctypes.c_int, _D, _D]
            L.o3_btd_get.argtypes = [vp, _D, ctypes.POINTER(ctypes.c_int)]
            L.o3_deposit_one.argtypes = [vp] + [ctypes.c_double] * 7
            L.o3_beam_weights.argtypes = [vp, _D]
            L.o3_rho_one.argtypes = [vp, _D] + [ctypes.c_double] * 4
            L.o1_create.restype = vp
            L.o1_create.argtypes = [ctypes.POINTER(_Config1)]
            L.o1_destroy.argtypes = [vp]
            L.o1_step.argtypes = [vp, ctypes.c_int]
            L.o1_load_plasma.argtypes = [vp, ctypes.POINTER(_Plasma1)]
            L.o1_set_laser.argtypes = [vp, ctypes.POINTER(_Laser1)]
            L.o1_info.argtypes = [vp, _D]
            for f in ("o1_get_field", "o1_set_field", "o1_get_gather_field", "o1_filter_field"):
                getattr(L, f).argtypes = [vp, ctypes.c_int, _D]
            L.o1_num_particles.restype = ctypes.c_long
            L.o1_num_particles.argtypes = [vp, ctypes.c_int]
            L.o1_get_particles.argtypes = [vp, ctypes.c_int] + [_D] * 5 + [ctypes.POINTER(ctypes.c_uint32)]
            L.o1_set_particles.argtypes = [vp, ctypes.c_int, ctypes.c_long] + [_D] * 5
            L.o1_rho.argtypes = [vp, _D]
            L.o1_diag.argtypes = [vp, _D]
            L.o1_deposit_one.argtypes = [vp] + [ctypes.c_double] * 5
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
# single functions
def shape(order: int, s: float) -> float:
    return lib().orc_shape(order, s)


def cfl_2d(a, b, g, dx, dz, theta=0.0) -> float:
    """dt limit of the 2D tunable solver (Eq. cfl restricted to d/dy = 0), with Friedman factor."""
    return lib().orc_cfl_2d(a, b, g, dx, dz, theta)


def cfl_3d(a, b, g, dx, dy, dz, theta=0.0) -> float:
    return lib().orc_cfl_3d(a, b, g, dx, dy, dz, theta)


def filter_line(x: np.ndarray, stride: int, alpha: float, periodic: bool) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(a)
    lib().orc_filter_line(_p(a), _p(out), a.size, stride, alpha, int(periodic))
    return out


def boris(u, E, B, q, m, dt) -> np.ndarray:
    uu = np.array(u, dtype=np.float64)
    e = np.array(E, dtype=np.float64)
    b = np.array(B, dtype=np.float64)
    lib().orc_boris(_p(uu), _p(e), _p(b), q, m, dt)
    return uu


# ----------------------------------------------------------------------------
def _mk_config(w: dict) -> _Config:
    c = _Config()
    c.nx, c.nz = int(w["nx"]), int(w["nz"])
    c.dz_lab, c.dx = float(w["dz_lab"]), float(w["dx"])
    c.gamma_boost = float(w.get("gamma_boost", 1.0))
    c.courant = float(w.get("courant", 0.9))
    c.dt_override = float(w.get("dt", 0.0) or 0.0)
    a, b, g = w.get("solver", (1.0, 0.0, 0.0))
    c.ck_alpha, c.ck_beta, c.ck_gamma = float(a), float(b), float(g)
    c.theta = float(w.get("theta", 0.0))
    c.pml_cells = int(w.get("pml_cells", 0))
    c.pml_sigma_max = float(w.get("pml_sigma_max", 4.0))
    c.pml_delta = float(w.get("pml_delta", 5.0))
    c.pml_power = float(w.get("pml_power", 2.0))
    c.pml_xi_exp = int(w.get("pml_xi_exp", 1))
    c.filter_passes = int(w.get("filter_passes", 0))
    c.filter_stride = int(w.get("filter_stride", 1))
    c.filter_compensate = int(w.get("filter_compensate", 0))
    c.filter_J = int(w.get("filter_J", 0))
    c.filter_gather = int(w.get("filter_gather", 0))
    c.order = int(w.get("order", 3))
    c.particle_guard = int(w.get("particle_guard", -1))
    c.periodic_x = int(w.get("periodic_x", 0))
    c.periodic_z = int(w.get("periodic_z", 0))
    c.moving_window = int(w.get("moving_window", 0))
    c.window_beta = float(w.get("window_beta", 0.0))
    for q, v in enumerate(list(w.get("filter_strides", []))[:4]):
        c.filter_strides[q] = int(v)
    c.gather_nodal = 1 if w.get("gather", "energy") == "momentum" else 0
    c.beam_self = int(w.get("beam_self", 0))
    return c


class Sim:
    """One oracle simulation built from a workload dict (see paper_1009_2727_gb300.workloads)."""

    def __init__(self, w: dict):
        self.L = lib()
        self.w = dict(w)
        self._cfg = _mk_config(w)
        self.h = self.L.orc_create(ctypes.byref(self._cfg))
        info = self.info()
        self.nx, self.nz = int(w["nx"]), int(w["nz"])
        self.dx, self.dz, self.dt = info["dx"], info["dz"], info["dt"]
        if w.get("plasma"):
            p = w["plasma"]
            pl = _Plasma(float(p["n0"]), float(p.get("z_start_lab", 0.0)), float(p.get("ramp_lab", 0.0)),
                         float(p.get("length_lab", 0.0)), int(p["ppc_x"]), int(p["ppc_z"]), int(p.get("ions", 1)))
            self.L.orc_load_plasma(self.h, ctypes.byref(pl))
        if w.get("laser"):
            l = w["laser"]
            la = _Laser(float(l["lambda0"]), float(l["a0"]), float(l["w0"]), float(l["tau_fwhm"]),
                        float(l.get("t_peak", 0.0)), float(l.get("x_center", 0.5 * self.nx * self.dx)),
                        float(l.get("phase", 0.0)), float(l["z_antenna"]), float(l.get("beta_s", 0.0)))
            self.L.orc_set_laser(self.h, ctypes.byref(la))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    # -- state ------------------------------------------------------------
    def info(self) -> dict:
        o = np.zeros(14)
        self.L.orc_info(self.h, _p(o))
        keys = ("dx", "dz", "dt", "gamma", "beta", "z0", "step", "t", "guard", "gx_lo", "gx_hi", "gz_lo", "gz_hi",
                "beam_vbar")
        return dict(zip(keys, o.tolist()))

    def step(self, n: int = 1):
        self.L.orc_step(self.h, int(n))

    def field(self, comp: int) -> np.ndarray:
        out = np.zeros((self.nx + 1) * (self.nz + 1))
        self.L.orc_get_field(self.h, comp, _p(out))
        return out.reshape(self.nx + 1, self.nz + 1)

    def set_field(self, comp: int, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        self.L.orc_set_field(self.h, comp, _p(a))

    def gather_field(self, comp: int) -> np.ndarray:
        out = np.zeros((self.nx + 1) * (self.nz + 1))
        self.L.orc_get_gather_field(self.h, comp, _p(out))
        return out.reshape(self.nx + 1, self.nz + 1)

    def history(self, which: int, comp: int) -> np.ndarray:
        out = np.zeros((self.nx + 1) * (self.nz + 1))
        self.L.orc_get_history(self.h, which, comp, _p(out))
        return out.reshape(self.nx + 1, self.nz + 1)

    def set_history(self, which: int, comp: int, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        self.L.orc_set_history(self.h, which, comp, _p(a))

    def set_ext_current(self, comp: int, a: np.ndarray, alternate: bool = False):
        """comp 0..2 = Jx, Jy, Jz; added every step before the current filter."""
        self._ext = getattr(self, "_ext", {})
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        self._ext[comp] = a
        self.L.orc_set_ext_current(self.h, comp, _p(a), int(alternate))

    def set_ext_profile(self, prof: np.ndarray):
        """per-step multiplier of the external current (zero after the table ends)"""
        self._prof = np.ascontiguousarray(prof, dtype=np.float64)
        self.L.orc_set_ext_profile(self.h, self._prof.size, _p(self._prof))

    def filter_field(self, comp: int, a: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(a, dtype=np.float64).reshape(-1).copy()
        self.L.orc_filter_field(self.h, comp, _p(b))
        return b.reshape(self.nx + 1, self.nz + 1)

    def rho(self) -> np.ndarray:
        out = np.zeros((self.nx + 1) * (self.nz + 1))
        self.L.orc_rho(self.h, _p(out))
        return out.reshape(self.nx + 1, self.nz + 1)

    def particles(self, species: int = 0) -> dict:
        n = self.L.orc_num_particles(self.h, species)
        arrs = {k: np.zeros(n) for k in ("x", "z", "ux", "uy", "uz", "w")}
        ids = np.zeros(n, dtype=np.uint32)
        flag = np.zeros(n, dtype=np.int32)
        self.L.orc_get_particles(self.h, species, *(_p(arrs[k]) for k in ("x", "z", "ux", "uy", "uz", "w")),
                                 ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                 flag.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        arrs["id"] = ids
        arrs["alive"] = (flag & 1) != 0
        arrs["active"] = (flag & 2) != 0
        return arrs

    def set_particles(self, species: int, x, z, ux, uy, uz, w):
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, z, ux, uy, uz, w)]
        self.L.orc_set_particles(self.h, species, a[0].size, *(_p(v) for v in a))

    def set_beam(self, x, z, ux, uy, uz, t_lab: float, z_plane: float):
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, z, ux, uy, uz)]
        self.L.orc_set_beam(self.h, a[0].size, *(_p(v) for v in a), float(t_lab), float(z_plane))

    def beam_weights(self, w):
        """macro-particle weights of the test beam (per unit length along y), in the order it was given"""
        a = np.ascontiguousarray(w, dtype=np.float64)
        self._beam_w = a
        self.L.orc_beam_weights(self.h, _p(a))

    def beam_rho(self, shift: float = 0.0) -> np.ndarray:
        """charge density of the frozen beam particles inside the particle domain (the ones that deposit), their
        positions taken `shift` seconds from now"""
        info = self.info()
        v = info["beam_vbar"]
        xlo, xhi = info["gx_lo"] * self.dx, info["gx_hi"] * self.dx
        zlo, zhi = info["z0"] + info["gz_lo"] * self.dz, info["z0"] + (info["gz_hi"] + 1) * self.dz
        p = self.particles(2)
        rho = np.zeros((self.nx + 1) * (self.nz + 1))
        for j in range(len(p["x"])):
            x, z = p["x"][j], p["z"][j] + v * shift
            if p["alive"][j] and not p["active"][j] and xlo <= x < xhi and zlo <= z < zhi:
                self.L.orc_rho_one(self.h, _p(rho), x, z, -QE * p["w"][j])
        return rho.reshape(self.nx + 1, self.nz + 1)

    def beam_self_field(self, shift: float = 0.0) -> dict:
        """Self-field of the frozen beam (Sec. 3.1.1: the fields at the injection plane must be consistent
        with the beam): its charge moves rigidly at the mean velocity v along z, so in the computational frame
        phi solves d2phi/dx2 + d2phi/dz2 / gamma_v^2 = -rho/eps0 (zero on the grid edges, the PEC walls),
        E_x = -dphi/dx, E_z = -dphi/dz / gamma_v^2, B_y = v E_x / c^2. The discrete operators are those of
        the Yee mesh (second differences for phi, one-sided differences for E at its half positions), so the
        discrete Gauss law holds exactly; the DST-I diagonalises them. The beam's positions are taken
        `shift` seconds from now (frozen particles move at v). Returns Ex, Ez, By on the grid."""
        from scipy.fft import dstn, idstn
        v = self.info()["beam_vbar"]
        gv2 = 1.0 / (1.0 - (v / C) ** 2)
        rho = self.beam_rho(shift)
        nx, nz, dx, dz = self.nx, self.nz, self.dx, self.dz
        lx = -(2.0 - 2.0 * np.cos(np.pi * np.arange(1, nx) / nx)) / dx ** 2
        lz = -(2.0 - 2.0 * np.cos(np.pi * np.arange(1, nz) / nz)) / dz ** 2
        rh = dstn(rho[1:nx, 1:nz], type=1)
        ph = -rh / EPS0 / (lx[:, None] + lz[None, :] / gv2)
        phi = np.zeros((nx + 1, nz + 1))
        phi[1:nx, 1:nz] = idstn(ph, type=1)
        ex = np.zeros_like(phi)
        ez = np.zeros_like(phi)
        by = np.zeros_like(phi)
        ex[:nx, :] = -(phi[1:, :] - phi[:-1, :]) / dx                     # (i + 1/2, k)
        ez[:, :nz] = -(phi[:, 1:] - phi[:, :-1]) / dz / gv2               # (i, k + 1/2)
        by[:nx, :nz] = v / C ** 2 * 0.5 * (ex[:nx, :nz] + ex[:nx, 1:])     # (i + 1/2, k + 1/2)
        return {"Ex": ex, "Ez": ez, "By": by, "vbar": v}

    def add_beam_self_field(self):
        """add the frozen beam's self-field: E at the current time, B half a step earlier (B^{n-1/2})"""
        fe = self.beam_self_field(0.0)
        fb = self.beam_self_field(-0.5 * self.dt)
        self.set_field(EX, self.field(EX) + fe["Ex"])
        self.set_field(EZ, self.field(EZ) + fe["Ez"])
        self.set_field(BY, self.field(BY) + fb["By"])

    def diag(self) -> dict:
        o = np.zeros(5)
        self.L.orc_diag(self.h, _p(o))
        return dict(zip(("n_e", "n_beam", "gamma_lab", "spread", "field_energy"), o.tolist()))

    def btd_set(self, zL: np.ndarray, tL: np.ndarray):
        zL = np.ascontiguousarray(zL, dtype=np.float64)
        tL = np.ascontiguousarray(tL, dtype=np.float64)
        self._nrows = zL.size
        self.L.orc_btd_set(self.h, zL.size, _p(zL), _p(tL))

    def btd_get(self):
        out = np.zeros(self._nrows * 6 * (self.nx + 1))
        done = np.zeros(self._nrows * 2, dtype=np.int32)
        self.L.orc_btd_get(self.h, _p(out), done.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return out.reshape(self._nrows, 6, self.nx + 1), done.reshape(self._nrows, 2)

    def deposit_one(self, x0, z0, x1, z1, vy, qw):
        shp = (self.nx + 1) * (self.nz + 1)
        J = [np.zeros(shp) for _ in range(3)]
        self.L.orc_deposit_one(self.h, _p(J[0]), _p(J[1]), _p(J[2]), x0, z0, x1, z1, vy, qw)
        return [j.reshape(self.nx + 1, self.nz + 1) for j in J]

    def rho_one(self, x, z, qw):
        r = np.zeros((self.nx + 1) * (self.nz + 1))
        self.L.orc_rho_one(self.h, _p(r), x, z, qw)
        return r.reshape(self.nx + 1, self.nz + 1)


# ----------------------------------------------------------------------------
# 3D
def _mk_config3(w: dict) -> _Config3:
    c = _Config3()
    c.nx, c.ny, c.nz = int(w["nx"]), int(w["ny"]), int(w["nz"])
    c.dz_lab, c.dx, c.dy = float(w["dz_lab"]), float(w["dx"]), float(w["dy"])
    c.gamma_boost = float(w.get("gamma_boost", 1.0))
    c.courant = float(w.get("courant", 0.9))
    c.dt_override = float(w.get("dt", 0.0) or 0.0)
    a, b, g = w.get("solver", (1.0, 0.0, 0.0))
    c.ck_alpha, c.ck_beta, c.ck_gamma = float(a), float(b), float(g)
    c.theta = float(w.get("theta", 0.0))
    c.pml_cells = int(w.get("pml_cells", 0))
    c.pml_sigma_max = float(w.get("pml_sigma_max", 4.0))
    c.pml_delta = float(w.get("pml_delta", 5.0))
    c.pml_power = float(w.get("pml_power", 2.0))
    c.pml_xi_exp = int(w.get("pml_xi_exp", 1))
    c.filter_passes = int(w.get("filter_passes", 0))
    c.filter_stride = int(w.get("filter_stride", 1))
    c.filter_compensate = int(w.get("filter_compensate", 0))
    c.filter_J = int(w.get("filter_J", 0))
    c.filter_gather = int(w.get("filter_gather", 0))
    c.order = int(w.get("order", 3))
    c.particle_guard = int(w.get("particle_guard", -1))
    c.periodic_x = int(w.get("periodic_x", 0))
    c.periodic_y = int(w.get("periodic_y", 0))
    c.periodic_z = int(w.get("periodic_z", 0))
    for q, v in enumerate(list(w.get("filter_strides", []))[:4]):
        c.filter_strides[q] = int(v)
    c.gather_nodal = 1 if w.get("gather", "energy") == "momentum" else 0
    c.beam_self = int(w.get("beam_self", 0))
    return c


class Sim3:
    """One 3D oracle simulation built from a 3D workload dict (nx, ny, nz, dx, dy, ...)."""

    def __init__(self, w: dict):
        self.L = lib()
        self.w = dict(w)
        self._cfg = _mk_config3(w)
        self.h = self.L.o3_create(ctypes.byref(self._cfg))
        info = self.info()
        self.nx, self.ny, self.nz = int(w["nx"]), int(w["ny"]), int(w["nz"])
        self.shape = (self.nx + 1, self.ny + 1, self.nz + 1)
        self.dx, self.dy, self.dz, self.dt = info["dx"], info["dy"], info["dz"], info["dt"]
        if w.get("plasma"):
            p = w["plasma"]
            pl = _Plasma3(float(p["n0"]), float(p.get("z_start_lab", 0.0)), float(p.get("ramp_lab", 0.0)),
                          float(p.get("length_lab", 0.0)), int(p["ppc_x"]), int(p["ppc_y"]), int(p["ppc_z"]),
                          int(p.get("ions", 1)))
            self.L.o3_load_plasma(self.h, ctypes.byref(pl))
        if w.get("beam"):
            b = w["beam"]
            self.set_beam(b["x"], b["y"], b["z"], b["ux"], b["uy"], b["uz"], b["t_lab"], b["z_plane_lab"])
        if w.get("laser"):
            l = w["laser"]
            la = _Laser3(float(l["lambda0"]), float(l["a0"]), float(l["w0"]), float(l["tau_fwhm"]),
                         float(l.get("t_peak", 0.0)), float(l.get("x_center", 0.5 * self.nx * self.dx)),
                         float(l.get("y_center", 0.5 * self.ny * self.dy)), float(l.get("phase", 0.0)),
                         float(l["z_antenna"]))
            self.L.o3_set_laser(self.h, ctypes.byref(la))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.o3_destroy(h)
            self.h = None

    def info(self) -> dict:
        o = np.zeros(16)
        self.L.o3_info(self.h, _p(o))
        keys = ("dx", "dy", "dz", "dt", "gamma", "beta", "step", "t", "guard",
                "gx_lo", "gx_hi", "gy_lo", "gy_hi", "gz_lo", "gz_hi", "beam_vbar")
        return dict(zip(keys, o.tolist()))

    def step(self, n: int = 1):
        self.L.o3_step(self.h, int(n))

    def field(self, comp: int) -> np.ndarray:
        out = np.zeros(int(np.prod(self.shape)))
        self.L.o3_get_field(self.h, comp, _p(out))
        return out.reshape(self.shape)

    def set_field(self, comp: int, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        self.L.o3_set_field(self.h, comp, _p(a))

    def gather_field(self, comp: int) -> np.ndarray:
        out = np.zeros(int(np.prod(self.shape)))
        self.L.o3_get_gather_field(self.h, comp, _p(out))
        return out.reshape(self.shape)

    def filter_field(self, comp: int, a: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(a, dtype=np.float64).reshape(-1).copy()
        self.L.o3_filter_field(self.h, comp, _p(b))
        return b.reshape(self.shape)

    def rho(self) -> np.ndarray:
        out = np.zeros(int(np.prod(self.shape)))
        self.L.o3_rho(self.h, _p(out))
        return out.reshape(self.shape)

    def particles(self, species: int = 0) -> dict:
        n = self.L.o3_num_particles(self.h, species)
        keys = ("x", "y", "z", "ux", "uy", "uz", "w")
        arrs = {k: np.zeros(n) for k in keys}
        ids = np.zeros(n, dtype=np.uint32)
        flag = np.zeros(n, dtype=np.int32)
        self.L.o3_get_particles(self.h, species, *(_p(arrs[k]) for k in keys),
                                ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                flag.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        arrs["id"] = ids
        arrs["alive"] = (flag & 1) != 0
        arrs["active"] = (flag & 2) != 0
        return arrs

    def set_particles(self, species: int, x, y, z, ux, uy, uz, w):
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, z, ux, uy, uz, w)]
        self.L.o3_set_particles(self.h, species, a[0].size, *(_p(v) for v in a))

    def set_beam(self, x, y, z, ux, uy, uz, t_lab: float, z_plane: float):
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, y, z, ux, uy, uz)]
        self._beam = a
        self.L.o3_set_beam(self.h, a[0].size, *(_p(v) for v in a), float(t_lab), float(z_plane))

    def beam_weights(self, w):
        a = np.ascontiguousarray(w, dtype=np.float64)
        self._beam_w = a
        self.L.o3_beam_weights(self.h, _p(a))

    def beam_rho(self, shift: float = 0.0) -> np.ndarray:
        """charge density of the frozen beam particles inside the particle domain (the ones that deposit), their
        positions taken `shift` seconds from now"""
        info = self.info()
        v = info["beam_vbar"]
        d = (self.dx, self.dy, self.dz)
        lo = [info[k] * d[a] for a, k in enumerate(("gx_lo", "gy_lo", "gz_lo"))]
        hi = [info[k] * d[a] for a, k in enumerate(("gx_hi", "gy_hi", "gz_hi"))]
        hi[2] += self.dz
        p = self.particles(2)
        rho = np.zeros(int(np.prod(self.shape)))
        for j in range(len(p["x"])):
            r = (p["x"][j], p["y"][j], p["z"][j] + v * shift)
            if p["alive"][j] and not p["active"][j] and all(lo[a] <= r[a] < hi[a] for a in range(3)):
                self.L.o3_rho_one(self.h, _p(rho), r[0], r[1], r[2], -QE * p["w"][j])
        return rho.reshape(self.shape)

    def beam_self_field(self, shift: float = 0.0) -> dict:
        """3D self-field of the frozen beam moving rigidly at v along z (as the 2-1/2D Sim.beam_self_field):
        d2phi/dx2 + d2phi/dy2 + d2phi/dz2 / gamma_v^2 = -rho/eps0 with phi = 0 on the PEC walls (DST-I of
        the Yee second differences), E = -grad phi with E_z divided by gamma_v^2, B = v z x E / c^2
        (B_x = -v E_y / c^2, B_y = v E_x / c^2) at their Yee positions."""
        from scipy.fft import dstn, idstn
        v = self.info()["beam_vbar"]
        gv2 = 1.0 / (1.0 - (v / C) ** 2)
        rho = self.beam_rho(shift)
        nx, ny, nz = self.nx, self.ny, self.nz
        lam = [-(2.0 - 2.0 * np.cos(np.pi * np.arange(1, n) / n)) / d ** 2
               for n, d in ((nx, self.dx), (ny, self.dy), (nz, self.dz))]
        den = lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :] / gv2
        ph = -dstn(rho[1:nx, 1:ny, 1:nz], type=1) / EPS0 / den
        phi = np.zeros((nx + 1, ny + 1, nz + 1))
        phi[1:nx, 1:ny, 1:nz] = idstn(ph, type=1)
        ex, ey, ez = (np.zeros_like(phi) for _ in range(3))
        bx, by = np.zeros_like(phi), np.zeros_like(phi)
        ex[:nx] = -(phi[1:] - phi[:-1]) / self.dx                               # (i + 1/2, j, k)
        ey[:, :ny] = -(phi[:, 1:] - phi[:, :-1]) / self.dy                      # (i, j + 1/2, k)
        ez[:, :, :nz] = -(phi[:, :, 1:] - phi[:, :, :-1]) / self.dz / gv2       # (i, j, k + 1/2)
        bx[:, :ny, :nz] = -v / C ** 2 * 0.5 * (ey[:, :ny, :nz] + ey[:, :ny, 1:])   # (i, j + 1/2, k + 1/2)
        by[:nx, :, :nz] = v / C ** 2 * 0.5 * (ex[:nx, :, :nz] + ex[:nx, :, 1:])    # (i + 1/2, j, k + 1/2)
        return {"Ex": ex, "Ey": ey, "Ez": ez, "Bx": bx, "By": by, "vbar": v}

    def add_beam_self_field(self):
        """add the frozen beam's self-field: E now, B half a step earlier (B^{n-1/2})"""
        fe = self.beam_self_field(0.0)
        fb = self.beam_self_field(-0.5 * self.dt)
        for c, k in ((EX, "Ex"), (EY, "Ey"), (EZ, "Ez")):
            self.set_field(c, self.field(c) + fe[k])
        for c, k in ((BX, "Bx"), (BY, "By")):
            self.set_field(c, self.field(c) + fb[k])

    def diag(self) -> dict:
        o = np.zeros(5)
        self.L.o3_diag(self.h, _p(o))
        return dict(zip(("n_e", "n_beam", "gamma_lab", "spread", "field_energy"), o.tolist()))

    def btd_set(self, zL: np.ndarray, tL: np.ndarray):
        zL = np.ascontiguousarray(zL, dtype=np.float64)
        tL = np.ascontiguousarray(tL, dtype=np.float64)
        self._nrows = zL.size
        self.L.o3_btd_set(self.h, zL.size, _p(zL), _p(tL))

    def btd_get(self):
        out = np.zeros(self._nrows * 6 * (self.nx + 1) * (self.ny + 1))
        done = np.zeros(self._nrows * 2, dtype=np.int32)
        self.L.o3_btd_get(self.h, _p(out), done.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return out.reshape(self._nrows, 6, self.nx + 1, self.ny + 1), done.reshape(self._nrows, 2)

    def deposit_one(self, p0, p1, qw):
        """current of one particle moved from p0 to p1 (x, y, z), deposited into the (zeroed) J arrays"""
        self.L.o3_deposit_one(self.h, *[float(v) for v in p0], *[float(v) for v in p1], float(qw))
        return [self.field(JX + c) for c in range(3)]


def _mk_config1(w: dict) -> _Config1:
    c = _Config1()
    c.nz = int(w["nz"])
    c.dz_lab = float(w["dz_lab"])
    c.gamma_boost = float(w.get("gamma_boost", 1.0))
    c.courant = float(w.get("courant", 0.95))
    c.dt_override = float(w.get("dt", 0.0))
    c.theta = float(w.get("theta", 0.0))
    c.pml_cells = int(w.get("pml_cells", 0))
    c.pml_sigma_max = float(w.get("pml_sigma_max", 4.0))
    c.pml_delta = float(w.get("pml_delta", 5.0))
    c.pml_power = float(w.get("pml_power", 2.0))
    c.pml_xi_exp = int(w.get("pml_xi_exp", 1))
    c.filter_passes = int(w.get("filter_passes", 0))
    c.filter_stride = int(w.get("filter_stride", 1))
    c.filter_compensate = int(w.get("filter_compensate", 0))
    c.filter_J = int(w.get("filter_J", 0))
    c.filter_gather = int(w.get("filter_gather", 0))
    c.order = int(w.get("order", 3))
    c.particle_guard = int(w.get("particle_guard", -1))
    c.moving_window = int(w.get("moving_window", 0))
    c.window_beta = float(w.get("window_beta", 0.0))
    for q, v in enumerate(list(w.get("filter_strides", []))[:4]):
        c.filter_strides[q] = int(v)
    c.gather_nodal = 1 if w.get("gather", "energy") == "momentum" else 0
    return c


class Sim1:
    """One 1D oracle simulation (fields and positions along z only) built from a workload dict with
    dim = 1 (nz, dz_lab, ...; the plasma's ppc_z; the laser's lambda0, a0, tau_fwhm, t_peak, z_antenna)."""

    def __init__(self, w: dict):
        self.L = lib()
        self.w = dict(w)
        self._cfg = _mk_config1(w)
        self.h = self.L.o1_create(ctypes.byref(self._cfg))
        info = self.info()
        self.nz = int(w["nz"])
        self.dz, self.dt = info["dz"], info["dt"]
        if w.get("plasma"):
            p = w["plasma"]
            pl = _Plasma1(float(p["n0"]), float(p.get("z_start_lab", 0.0)), float(p.get("ramp_lab", 0.0)),
                          float(p.get("length_lab", 0.0)), int(p["ppc_z"]), int(p.get("ions", 1)))
            self.L.o1_load_plasma(self.h, ctypes.byref(pl))
        if w.get("laser"):
            l = w["laser"]
            la = _Laser1(float(l["lambda0"]), float(l["a0"]), float(l["tau_fwhm"]), float(l.get("t_peak", 0.0)),
                         float(l.get("phase", 0.0)), float(l["z_antenna"]))
            self.L.o1_set_laser(self.h, ctypes.byref(la))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.o1_destroy(h)
            self.h = None

    def info(self) -> dict:
        o = np.zeros(10)
        self.L.o1_info(self.h, _p(o))
        keys = ("dz", "dt", "gamma", "beta", "step", "t", "guard", "gz_lo", "gz_hi", "z0")
        return dict(zip(keys, o.tolist()))

    def step(self, n: int = 1):
        self.L.o1_step(self.h, int(n))

    def field(self, comp: int) -> np.ndarray:
        out = np.zeros(self.nz + 1)
        self.L.o1_get_field(self.h, comp, _p(out))
        return out

    def set_field(self, comp: int, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        self.L.o1_set_field(self.h, comp, _p(a))

    def gather_field(self, comp: int) -> np.ndarray:
        out = np.zeros(self.nz + 1)
        self.L.o1_get_gather_field(self.h, comp, _p(out))
        return out

    def filter_field(self, comp: int, a: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(a, dtype=np.float64).reshape(-1).copy()
        self.L.o1_filter_field(self.h, comp, _p(b))
        return b

    def rho(self) -> np.ndarray:
        out = np.zeros(self.nz + 1)
        self.L.o1_rho(self.h, _p(out))
        return out

    def deposit_one(self, z0: float, z1: float, vx: float, vy: float, qw: float):
        self.L.o1_deposit_one(self.h, z0, z1, vx, vy, qw)

    def particles(self, species: int = 0) -> dict:
        n = self.L.o1_num_particles(self.h, species)
        keys = ("z", "ux", "uy", "uz", "w")
        arrs = {k: np.zeros(n) for k in keys}
        ids = np.zeros(n, dtype=np.uint32)
        self.L.o1_get_particles(self.h, species, *(_p(arrs[k]) for k in keys),
                                ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        arrs["id"] = ids
        return arrs

    def set_particles(self, species: int, z, ux, uy, uz, w):
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (z, ux, uy, uz, w)]
        self.L.o1_set_particles(self.h, species, a[0].size, *(_p(v) for v in a))

    def diag(self) -> dict:
        o = np.zeros(2)
        self.L.o1_diag(self.h, _p(o))
        return {"n_e": o[0], "field_energy": o[1]}
