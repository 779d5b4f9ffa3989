"""Pins of the FP64 learned-direction oracle (oracle/mlp.py) against things
other than itself: the C oracle's SplitMix64 stream, central finite
differences of the loss, closed-form loss values, the first Adam step's
closed form, and features of axis-aligned data whose components are known."""
import numpy as np
import pytest

import oracle
from oracle import mlp


def test_splitmix64_stream_matches_the_c_oracle():
    idx = [0, 1, 2, 77, 4095, 123456]
    for stream in (1, 101, 103):
        v = mlp.splitmix64_units(1234567, stream, idx)
        for i, x in zip(idx, v):
            assert x == oracle.splitmix64_unit(1234567, stream, i)


def test_init_bounds_and_zero_biases():
    P = mlp.init_params(16, seed=3)
    assert P["W1"].shape == (160, 256) and P["W3"].shape == (256, 64)
    assert np.abs(P["W1"]).max() <= np.sqrt(6.0 / 160) and np.abs(P["W2"]).max() <= np.sqrt(6.0 / 256)
    assert all(np.all(P[f"b{i}"] == 0) for i in (1, 2, 3))
    # values are FP32 numbers
    assert np.array_equal(P["W2"], P["W2"].astype(np.float32).astype(np.float64))


def _rand_problem(D=8, B=5, seed=0):
    rng = np.random.default_rng(seed)
    P = mlp.init_params(D, seed=seed)
    for k in P:  # non-zero biases exercise every term
        if k.startswith("b"):
            P[k] = rng.standard_normal(P[k].shape) * 0.1
    X = rng.standard_normal((B, 10 * D))
    W = rng.standard_normal((B, D))
    W /= np.linalg.norm(W, axis=1, keepdims=True)
    return P, X, W


def test_gradient_matches_central_differences():
    P, X, W = _rand_problem()
    G = mlp.backward(P, mlp.forward(P, X, W))
    rng = np.random.default_rng(1)
    h = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for i in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + h
            lp = mlp.forward(P, X, W)["loss_mean"]
            flat[i] = old - h
            lm = mlp.forward(P, X, W)["loss_mean"]
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = G[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-8, (k, i, fd, an)


def test_loss_closed_forms():
    # W1 = W2 = W3 = 0, b3 = the chosen raw outputs: z does not depend on x
    D = 8
    P = {k: np.zeros_like(v) for k, v in mlp.init_params(D, 0).items()}
    w = np.zeros(D)
    w[2] = 1.0
    X = np.ones((1, 10 * D))
    # every direction along w: c_j = 1, loss = 1 - (1/tau) log(4 e^tau) = -log(4)/tau
    P["b3"] = np.tile(3.0 * w, 4)
    f = mlp.forward(P, X, w[None, :])
    assert f["loss_mean"] == pytest.approx(-np.log(4) / mlp.TAU, abs=1e-15)
    # every direction orthogonal to w: loss = 1 - log(4)/tau
    e = np.zeros(D)
    e[5] = -2.0
    P["b3"] = np.tile(e, 4)
    f = mlp.forward(P, X, w[None, :])
    assert f["loss_mean"] == pytest.approx(1 - np.log(4) / mlp.TAU, abs=1e-15)
    # one aligned, three orthogonal: 1 - (1/tau) log(e^tau + 3)
    P["b3"] = np.concatenate([w, e, e, e])
    f = mlp.forward(P, X, w[None, :])
    assert f["loss_mean"] == pytest.approx(1 - np.log(np.exp(mlp.TAU) + 3) / mlp.TAU, abs=1e-15)
    # unit outputs whatever the raw scale
    assert np.allclose(np.linalg.norm(f["U"], axis=2), 1.0)


def test_first_adam_step_is_a_signed_step():
    # step 1: m_hat = g, v_hat = g^2, so p moves by lr g / (|g| + eps)
    P = {"a": np.array([1.0, -2.0, 0.5])}
    G = {"a": np.array([0.3, -1e-3, 0.0])}
    M = {"a": np.zeros(3)}
    V = {"a": np.zeros(3)}
    mlp.adam_step(P, M, V, G, lr=0.01, step=1)
    expect = np.array([1.0, -2.0, 0.5]) - 0.01 * G["a"] / (np.abs(G["a"]) + 1e-8)
    np.testing.assert_allclose(P["a"], expect, rtol=0, atol=1e-15)


def test_features_of_axis_aligned_sets():
    # independent coordinates with distinct variances: components are the axes
    rng = np.random.default_rng(0)
    D = 12
    sd = np.linspace(3.0, 0.5, D)
    A = (rng.standard_normal((4000, D)) * sd).astype(np.float32)
    B = (rng.standard_normal((4000, D)) * sd + 0.25).astype(np.float32)
    f = mlp.features(A, B)
    assert f.shape == (10 * D,)
    _, C = oracle.union_covariance(A, B)
    s2 = np.trace(C) / D
    np.testing.assert_allclose(f[9 * D:], np.diag(C) / s2, rtol=1e-12)
    dmu = B.astype(np.float64).mean(0) - A.astype(np.float64).mean(0)
    np.testing.assert_allclose(f[:D], dmu / np.sqrt(s2), rtol=1e-12)
    # component l: sqrt(lambda_l) e_l up to the rotation noise of the sample
    for l in range(8):
        v = f[(1 + l) * D:(2 + l) * D] * np.sqrt(s2)
        assert np.argmax(np.abs(v)) == l
        assert v[l] > 0


def test_flatten_roundtrip():
    P = mlp.init_params(8, 5)
    flat = mlp.flatten(P, 8)
    assert flat.size % 64 == 0
    Q = mlp.unflatten(flat, 8)
    for k in P:
        assert np.array_equal(P[k], Q[k])


def test_bf16_rounding():
    # exact BF16 values stay; halfway cases go to the even neighbour; the
    # result has at most 8 significant bits
    assert mlp.bf16_round(1.0) == 1.0
    assert mlp.bf16_round(1.0 + 2.0**-8) == 1.0            # halfway, even is 1.0
    assert mlp.bf16_round(1.0 + 3 * 2.0**-8) == 1.0 + 2.0**-6  # halfway, even is 1 + 2^-6
    assert mlp.bf16_round(1.0 + 2.0**-8 + 2.0**-12) == 1.0 + 2.0**-7
    assert mlp.bf16_round(-3.0) == -3.0
    rng = np.random.default_rng(0)
    x = rng.standard_normal(1000) * 10.0 ** rng.uniform(-5, 5, 1000)
    r = mlp.bf16_round(x)
    assert np.all(np.abs(r - x) <= 2.0**-8 * np.abs(x) * (1 + 1e-7))
    m, _ = np.frexp(r)
    assert np.all((m * 2**8) == np.round(m * 2**8))
    torch = pytest.importorskip("torch")
    t = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(r, t)


def test_bf16_gradient_matches_central_differences_of_the_bf16_forward_away_from_kinks():
    # with operands rounded the loss is piecewise smooth; the chain rule
    # still holds for the rounded forward in the sense that the FP64 form
    # (bf16 = False) and the rounded form differ by about the rounding
    P, X, W = _rand_problem(D=8, B=6, seed=3)
    f0 = mlp.forward(P, X, W)
    f1 = mlp.forward(P, X, W, bf16=True)
    assert abs(f1["loss_mean"] - f0["loss_mean"]) <= 2e-2 * abs(f0["loss_mean"]) + 1e-3
    G0 = mlp.backward(P, f0)
    G1 = mlp.backward(P, f1)
    for k in G0:
        assert np.linalg.norm(G1[k] - G0[k]) <= 0.2 * np.linalg.norm(G0[k]) + 1e-12, k
