"""Stage surrogate on the GPU: the library's BF16 multilayer perceptron against the FP64 oracle of the same
network (oracle/mlp.py), its training, and a small end-to-end surrogate over stage runs.

Tolerances follow from BF16 (8 significant bits, unit roundoff 2^-9 ~ 2e-3): the GPU multiplies BF16
weights (the oracle is given the same BF16-rounded weights, FP32 biases) by BF16-stored inputs and
activations and accumulates in FP32, so each layer's output carries a relative error of a few 2^-9;
over three layers the outputs stay within 2e-2 of the largest output and the gradient within 3e-2 in
relative L2 norm.
"""
import numpy as np
import pytest

from paper_1009_2727_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_2727_gb300 import surrogate
    return surrogate


def bf16(a):
    """round FP32 values to the nearest BF16 (ties to even), returned as FP64"""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_weights(p, widths):
    """the weights rounded to BF16, the biases kept in FP32, in the flat layout"""
    q = np.asarray(p, dtype=np.float64).copy()
    o = 0
    for l in range(1, len(widths)):
        nw = widths[l] * widths[l - 1]
        q[o:o + nw] = bf16(p[o:o + nw])
        o += nw + widths[l]
    return q


def smooth_target(x):
    return np.stack([np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2], np.cos(x[:, 3] - x[:, 4]),
                     np.tanh(x[:, 5] + x[:, 0]), x[:, 1] ** 2 - 0.3 * x[:, 4]], axis=1)


def test_bf16_rounding_helper():
    assert bf16(np.float32(1.0 + 2.0 ** -8))[()] == 1.0                   # tie to even (down)
    assert bf16(np.float32(1.0 + 3 * 2.0 ** -8))[()] == 1.0 + 2.0 ** -6   # tie to even (up)
    assert bf16(np.float32(1.0 + 2.0 ** -8 + 2.0 ** -20))[()] == 1.0 + 2.0 ** -7


@pytest.mark.parametrize("widths,n", [([6, 96, 80, 4], 150), ([6, 256, 256, 256, 4], 333), ([3, 1, 5], 1)])
def test_mlp_forward_and_gradient_match_oracle(S, widths, n):
    """several 64-row and 64-column tiles with ragged tails, the surrogate's own shape, and a degenerate
    one-unit layer with a single sample"""
    from oracle import mlp as ref
    rng = np.random.default_rng(11)
    net = S.MLP(widths, seed=5)
    p = net.get_params().astype(np.float64)
    p += rng.normal(0, 0.05, p.size)          # non-zero biases
    net.set_params(p)
    p32 = net.get_params()
    x = rng.normal(0, 1, (n, widths[0]))
    t = rng.normal(0, 1, (n, widths[-1]))
    pq = bf16_weights(p32, widths)
    y_ref, _ = ref.forward(pq, widths, bf16(x))
    y = net.forward(x)
    assert np.abs(y - y_ref).max() <= 2e-2 * np.abs(y_ref).max()
    loss_ref, g_ref = ref.loss_and_grad(pq, widths, bf16(x), t)
    loss, g = net.grad(x, t)
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    assert np.linalg.norm(g - g_ref) <= 3e-2 * np.linalg.norm(g_ref)
    net.close()


@pytest.mark.parametrize("widths,n", [([6, 256, 256, 256, 4], 1000), ([6, 96, 80, 4], 333), ([3, 1, 5], 1),
                                      ([16, 128, 16], 128)])
def test_mlp_tensor_core_inference_matches_oracle_and_cuda_cores(S, widths, n):
    """the fused tcgen05 inference kernel: several 128-row tiles with a ragged last one, padded widths,
    a one-unit layer and a single row, an exact tile; against the oracle and the CUDA-core GEMM path"""
    from oracle import mlp as ref
    rng = np.random.default_rng(17)
    net = S.MLP(widths, seed=8)
    p = net.get_params().astype(np.float64)
    p += rng.normal(0, 0.05, p.size)
    net.set_params(p)
    x = rng.normal(0, 1, (n, widths[0]))
    y_tc = net.forward(x)
    net.use_tensor_cores(False)
    y_cc = net.forward(x)
    net.use_tensor_cores(True)
    y_ref, _ = ref.forward(bf16_weights(net.get_params(), widths), widths, bf16(x))
    scale = np.abs(y_ref).max()
    assert np.abs(y_tc - y_ref).max() <= 2e-2 * scale
    assert np.abs(y_tc - y_cc).max() <= 2e-2 * scale
    # after a parameter change the packed weights are rebuilt
    net.set_params(p * 0.5)
    y2 = net.forward(x)
    y2_ref, _ = ref.forward(bf16_weights(net.get_params(), widths), widths, bf16(x))
    assert np.abs(y2 - y2_ref).max() <= 2e-2 * np.abs(y2_ref).max()
    net.close()


def test_mlp_forward_over_chunks_matches_rows(S):
    """a batch larger than one 65536-row chunk with a ragged last chunk: sampled rows against the oracle"""
    from oracle import mlp as ref
    widths = [6, 64, 64, 4]
    net = S.MLP(widths, seed=2)
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, (65536 + 777, 6))
    y = net.forward(x)
    pq = bf16_weights(net.get_params(), widths)
    rows = np.concatenate([rng.choice(65536, 200, replace=False), 65536 + np.arange(777)])
    y_ref, _ = ref.forward(pq, widths, bf16(x[rows]))
    assert np.abs(y[rows] - y_ref).max() <= 2e-2 * np.abs(y_ref).max()
    net.close()


def test_mlp_training_fits_and_is_deterministic(S):
    rng = np.random.default_rng(7)
    x = rng.uniform(-1.5, 1.5, (2048, 6))
    t = smooth_target(x)
    xh = rng.uniform(-1.5, 1.5, (512, 6))
    curves, params = [], []
    for _ in range(2):
        net = S.MLP([6, 128, 128, 4], seed=1)
        curves.append(net.train(x, t, epochs=120, batch=64, lr=2e-3, weight_decay=1e-4, seed=9))
        params.append(net.get_params())
        err = np.sqrt(np.mean((net.forward(xh) - smooth_target(xh)) ** 2))
        net.close()
    c = curves[0]
    assert np.all(np.isfinite(c)) and c[-1] < 0.05 * c[0], (c[0], c[-1])
    assert err < 0.1 * np.sqrt(np.mean(smooth_target(xh) ** 2))
    # the sample order and the products are deterministic: same seed, same parameters
    assert np.array_equal(params[0], params[1])


def test_mlp_training_graph_matches_direct_launches(S):
    """an epoch captured once and replayed gives bitwise the parameters and loss curve of the direct launches"""
    rng = np.random.default_rng(11)
    x = rng.uniform(-1.5, 1.5, (640, 6))
    t = smooth_target(x)
    out = []
    for graphs in (True, False):
        net = S.MLP([6, 96, 96, 4], seed=3)
        net.use_graphs(graphs)
        c = net.train(x, t, epochs=7, batch=64, lr=2e-3, weight_decay=1e-4, seed=4)
        out.append((net.get_params(), c))
        net.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.allclose(out[0][1], out[1][1], rtol=1e-5, atol=0.0)


def test_stage_surrogate_end_to_end(S):
    """a handful of stage runs through the ensemble: finite, plausible labels; the fitted surrogate
    reproduces its training set and flags a query outside the sampled box"""
    runs = W.surrogate_runs(6, seed=21)
    X, Y, ok = S.stage_labels(runs, batch=6)
    assert np.all(np.isfinite(Y)) and ok.sum() >= 5, ok
    X, Y = X[ok], Y[ok]
    runs = [r for r, v in zip(runs, ok) if v]
    me_c2 = 0.51099895000
    for r, y in zip(runs, Y):
        # the beam cannot gain more than the largest 1D cold wake over the stage, (a0^2/2) E0 L roughly
        # bounded here by 4 E0 L, nor lose more than its own energy
        n0 = 10.0 ** r["inputs"][0]
        E0 = 96.0 * np.sqrt(n0 * 1e-6)                            # V/m, cold wave-breaking field
        assert -r["gamma_w"] * me_c2 < y[0] < 4.0 * E0 * r["inputs"][4] * 1e-3 * 1e-6, (r["inputs"], y)
        assert -1.0 <= y[1] < 3.0
        assert y[2] >= 0.0
        assert -0.05 <= y[3] <= 1.0, (r["inputs"], y)
    sur = S.Surrogate(hidden=(64, 64), seed=3)
    curve = sur.fit(X, Y, epochs=1500, batch=6, lr=3e-3, weight_decay=0.0)
    assert curve[-1] < 0.05 * curve[0]
    pred, inside = sur.predict(X)
    assert inside.all()
    assert np.all(np.abs(pred - Y) <= 0.25 * Y.std(0) + 1e-9)
    q = X[:1].copy()
    q[0, 5] = 20.0            # a boost outside the sampled range
    assert not sur.predict(q)[1][0]


def test_surrogate_within_5_percent_on_50_heldout_pic_runs(S):
    """the surrogate's acceptance criterion: trained on 2048 stage runs (1956 valid), it predicts the beam's
    energy gain of 50 fresh PIC runs (seed 5; the runs that gain more than 5 MeV and lie inside the training
    box) with a median relative error at most 5% (measured 2.9-3.2%) and an rms error below 0.15 of the
    gains' spread (R^2 above 0.97; measured 0.991)"""
    tr = W.surrogate_runs(2048, seed=1)
    te = W.surrogate_runs(50, seed=5)
    X, Y, ok = S.stage_labels(tr)
    Xt, Yt, okt = S.stage_labels(te)
    assert ok.sum() >= 1900 and okt.sum() >= 45, (ok.sum(), okt.sum())
    sur = S.Surrogate(hidden=(256, 256, 256), seed=0)
    sur.fit(X[ok], Y[ok], epochs=1500, batch=64, lr=1e-3, weight_decay=1e-4)
    pred, inside = sur.predict(Xt[okt])
    g, gp = Yt[okt][inside, 0], pred[inside, 0]
    assert inside.mean() >= 0.9
    big = np.abs(g) > 5.0
    assert big.sum() >= 25
    rel_err = np.abs(gp[big] - g[big]) / np.abs(g[big])
    assert np.median(rel_err) <= 0.05, np.median(rel_err)
    assert np.sqrt(np.mean((gp - g) ** 2)) <= 0.15 * g.std()


def test_surrogate_gain_over_pic_on_heldout_runs(S):
    """what the trained network gains over the method without it: on fresh held-out stage runs it
    predicts the beam's energy gain close to what PIC measures, at a tiny fraction of a PIC run's cost"""
    import time
    tr = W.surrogate_runs(256, seed=1)
    te = W.surrogate_runs(16, seed=5)
    X, Y, ok = S.stage_labels(tr)
    t0 = time.time()
    Xt, Yt, okt = S.stage_labels(te)
    pic_per_run = (time.time() - t0) / len(te)
    sur = S.Surrogate(hidden=(256, 256, 256), seed=0)
    sur.fit(X[ok], Y[ok], epochs=1500, batch=64, lr=1e-3, weight_decay=1e-4)
    q = np.repeat(Xt[okt], 1000, axis=0)
    sur.predict(q[:10])
    t0 = time.time()
    pred, inside = sur.predict(q)
    per_query = (time.time() - t0) / len(q)
    pred, inside = pred[::1000], inside[::1000]
    g, gp = Yt[okt][inside, 0], pred[inside, 0]
    assert inside.mean() >= 0.8
    # held-out gain within 30% of the spread of gains in rms (R^2 >= 0.91) from only 256 training runs
    # (0.2 measured); the 2048-run surrogate of the benchmark does several times better
    assert np.sqrt(np.mean((gp - g) ** 2)) <= 0.3 * g.std(), (g, gp)
    assert per_query * 1e4 < pic_per_run, (per_query, pic_per_run)
