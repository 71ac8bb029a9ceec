"""Stage surrogate: a multilayer perceptron mapping stage parameters to stage outputs, trained on the
boosted-frame runs the library itself produces (argument marshalling and bookkeeping only: the network's
forward, backward and optimiser steps run in the library's pic_mlp_* kernels, the runs in pic_ensemble_*).

Inputs (6): log10 n0 [m^-3], a0, w0 [um], tau [fs], stage length L [mm], gamma_boost.
Outputs (4), measured on each run:
  gain        lab-frame energy gain of the test beam at the end of the stage [MeV]
  log_spread  log10(0.1 + relative rms energy spread of the test beam at the end [%]); the spread spans
              three decades, set mostly by dephasing at high density
  trapped     charge of the plasma electrons above the wake's Lorentz factor gamma_w [pC/um of y]
  depleted    fraction of the peak field energy (computational frame) gone by the end of the stage; the
              depletion length follows as L / depleted (depletion_length)
Runs that went numerically unstable are left out of the training set (stage_labels' valid mask).
Queries outside the training inputs' axis-aligned box are flagged for a PIC run instead.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi
from .pic import Ensemble, PicError, torch_allocator

ME_MEV = 0.51099895000
OUTPUTS = ("gain", "log_spread", "trapped", "depleted")


class MLP:
    """The library's BF16/FP32 multilayer perceptron (pic_mlp_*) on a CUDA stream."""

    def __init__(self, widths, seed: int = 0, stream=None):
        import torch
        self.torch = torch
        self.L = capi.load()
        self.widths = [int(w) for w in widths]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._acb, self._fcb = torch_allocator(torch.cuda.current_device())
        w = (ctypes.c_int * len(self.widths))(*self.widths)
        h = ctypes.c_void_p()
        r = self.L.pic_mlp_create(len(self.widths) - 1, w, ctypes.c_uint64(seed), self._acb, self._fcb, None,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if r != 0:
            raise PicError(f"pic_mlp_create failed: {capi.STATUS_NAMES.get(r, r)}")
        self.h = h
        self.n_params = int(self.L.pic_mlp_param_count(h))

    def _dev(self, a):
        t = self.torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()
        return t, ctypes.c_void_p(t.data_ptr())

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        self._check(self.L.pic_mlp_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.L.pic_mlp_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def use_tensor_cores(self, enable: bool = True):
        """serve with the fused tcgen05 kernel (default when every padded width <= 256) or the CUDA-core GEMMs"""
        self._check(self.L.pic_mlp_use_tensor_cores(self.h, int(bool(enable))))

    def use_graphs(self, enable: bool = True):
        """train by replaying one captured epoch (default) or by direct launches"""
        self._check(self.L.pic_mlp_use_graphs(self.h, int(bool(enable))))

    def forward(self, x) -> np.ndarray:
        xd, xp = self._dev(x)
        y = self.torch.empty((xd.shape[0], self.widths[-1]), dtype=self.torch.float32, device="cuda")
        self._check(self.L.pic_mlp_infer(self.h, xp, xd.shape[0], ctypes.c_void_p(y.data_ptr())))
        self._check(self.L.pic_mlp_status(self.h))
        return y.cpu().numpy()

    def forward_device(self, x_ptr: int, n: int, y_ptr: int):
        """outputs of n rows at device address x_ptr into device address y_ptr, on the MLP's stream"""
        self._check(self.L.pic_mlp_infer(self.h, ctypes.c_void_p(x_ptr), int(n), ctypes.c_void_p(y_ptr)))

    def grad(self, x, t):
        xd, xp = self._dev(x)
        td, tp = self._dev(t)
        loss = ctypes.c_float(0.0)
        g = np.zeros(self.n_params, dtype=np.float32)
        self._check(self.L.pic_mlp_grad(self.h, xp, tp, xd.shape[0], ctypes.byref(loss),
                                        g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return float(loss.value), g

    def train(self, x, t, epochs: int, batch: int, lr: float = 1e-3, weight_decay: float = 1e-4, seed: int = 0):
        xd, xp = self._dev(x)
        td, tp = self._dev(t)
        curve = np.zeros(max(epochs, 1), dtype=np.float32)
        self._check(self.L.pic_mlp_train(self.h, xp, tp, xd.shape[0], int(epochs), int(batch), float(lr),
                                         float(weight_decay), ctypes.c_uint64(seed),
                                         curve.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return curve[:epochs]

    def _check(self, r):
        if r != 0:
            raise PicError(f"pic_mlp call failed: {capi.STATUS_NAMES.get(r, r)}")

    def close(self):
        if getattr(self, "h", None):
            self.L.pic_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stage_labels(runs: list, batch: int = 64, every: int = 50):
    """Run the stage workloads (workloads.surrogate_runs) in ensembles of `batch` runs of similar length and
    measure the four outputs of each at its own step count. The field energy is sampled every `every`
    steps; the depletion is one minus the final field energy over the largest sample; the trapped charge
    counts the plasma electrons above the wake's Lorentz factor gamma_w.
    Returns (inputs n x 6, outputs n x 4, valid n): a run is valid when its test beam entered the plasma
    and its field energy did not grow after the antenna stopped emitting (at most twice the energy then:
    with no source left, a larger growth is a numerical instability, not physics)."""
    order = sorted(range(len(runs)), key=lambda i: runs[i]["steps"])
    X = np.zeros((len(runs), 6))
    Y = np.zeros((len(runs), len(OUTPUTS)))
    ok = np.zeros(len(runs), dtype=bool)
    for b0 in range(0, len(order), batch):
        ids = order[b0:b0 + batch]
        part = [runs[i] for i in ids]
        ens = Ensemble(part)
        marks = set(range(every, max(r["steps"] for r in part), every))
        marks |= {r["steps"] for r in part} | {r["emit_steps"] for r in part}
        wmax = np.zeros(len(part))
        w_emit = np.zeros(len(part))
        done = 0
        for t in sorted(marks):
            ens.step(t - done)
            done = t
            ens.sync()
            for j, (r, m) in enumerate(zip(part, ens.members)):
                if done > r["steps"]:
                    continue
                st = m.stats(trap_gamma_lab=r["gamma_w"])
                wmax[j] = max(wmax[j], st["field_energy"])
                if done == r["emit_steps"]:
                    w_emit[j] = st["field_energy"]
                if done == r["steps"]:
                    active = st["n_beam_active"] > 0
                    gain = (st["beam_gamma_lab"] - r["gamma_w"]) * ME_MEV if active else 0.0
                    dep = 1.0 - st["field_energy"] / wmax[j] if wmax[j] > 0 else 0.0
                    X[ids[j]] = r["inputs"]
                    spread = np.log10(0.1 + 100.0 * st["beam_spread"]) if active else -1.0
                    Y[ids[j]] = [gain, spread, st["trapped_charge"] * 1e6, dep]
                    ok[ids[j]] = bool(active and np.isfinite(Y[ids[j]]).all()
                                      and st["field_energy"] <= 2.0 * w_emit[j])
        ens.close()
    return X, Y, ok


def depletion_length(X, Y):
    """pump-depletion length [mm] implied by a depleted fraction over the stage length (linear in L)"""
    f = np.asarray(Y)[:, OUTPUTS.index("depleted")]
    return np.asarray(X)[:, 4] / np.maximum(f, 1e-6)


class Surrogate:
    """Standardised inputs and outputs around the library's MLP (6 -> 256 -> 256 -> 256 -> 4 by default)."""

    def __init__(self, hidden=(256, 256, 256), seed: int = 0):
        self.hidden = tuple(hidden)
        self.seed = seed
        self.net = None

    def fit(self, X, Y, epochs: int = 400, batch: int = 64, lr: float = 1e-3, weight_decay: float = 1e-4):
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        self.xm, self.xs = X.mean(0), X.std(0) + 1e-12
        self.ym, self.ys = Y.mean(0), Y.std(0) + 1e-12
        self.lo, self.hi = X.min(0), X.max(0)
        self.net = MLP([X.shape[1], *self.hidden, Y.shape[1]], seed=self.seed)
        return self.net.train((X - self.xm) / self.xs, (Y - self.ym) / self.ys, epochs, min(batch, len(X)), lr,
                              weight_decay, seed=self.seed)

    def inside(self, X) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        return np.all((X >= self.lo) & (X <= self.hi), axis=1)

    def predict(self, X):
        """outputs for every query and a mask of the queries inside the training box (the others need PIC)"""
        X = np.asarray(X, dtype=np.float64)
        y = self.net.forward((X - self.xm) / self.xs).astype(np.float64)
        return y * self.ys + self.ym, self.inside(X)
