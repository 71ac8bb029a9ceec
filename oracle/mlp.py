"""FP64 CPU reference of the surrogate's multilayer perceptron (test infrastructure only).

Plain restatement of the network that the library's pic_mlp_* kernels run: widths w0 -> ... -> wL,
GELU(z) = z Phi(z) (exact, erf form) after every layer but the last, mean squared error loss.
Parameter layout, as in include/pic.h: per layer the weight (w_l x w_{l-1}, row-major) then the bias.
Its analytic gradient is pinned by central finite differences in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def unpack(params, widths):
    """list of (W, b) per layer from the flat parameter vector"""
    out, o = [], 0
    for l in range(1, len(widths)):
        nw = widths[l] * widths[l - 1]
        W = params[o:o + nw].reshape(widths[l], widths[l - 1])
        o += nw
        b = params[o:o + widths[l]]
        o += widths[l]
        out.append((W, b))
    assert o == params.size
    return out


def forward(params, widths, x):
    """outputs and the per-layer (input, pre-activation) pairs"""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    layers = unpack(np.asarray(params, dtype=np.float64), widths)
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if l < len(layers) - 1 else z
    return h, cache


def loss_and_grad(params, widths, x, t):
    """mean squared error over all outputs and its gradient with respect to the flat parameters"""
    y, cache = forward(params, widths, x)
    t = np.asarray(t, dtype=np.float64)
    n_el = y.size
    loss = float(np.sum((y - t) ** 2) / n_el)
    dz = 2.0 * (y - t) / n_el
    layers = unpack(np.asarray(params, dtype=np.float64), widths)
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        h_in, _ = cache[l]
        grads.append((dz.T @ h_in, dz.sum(axis=0)))
        if l > 0:
            dz = (dz @ W) * gelu_prime(cache[l - 1][1])
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.reshape(-1))
        flat.append(gb)
    return loss, np.concatenate(flat)
