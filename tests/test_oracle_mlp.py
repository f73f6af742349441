"""Pins of the FP64 proposal-network oracle (no GPU): finite differences, the Adam closed form,
bf16 rounding against torch's, SplitMix64's published first output, feature closed forms."""
import numpy as np
import pytest

import oracle
import oracle.mlp as om


def _data(n=32, seed=0):
    rng = np.random.default_rng(seed)
    X = om.bf16(rng.normal(size=(n, 64)) * 0.5)
    X[:, 51:] = 0.0
    T = rng.normal(size=(n, 3))
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    return X, T


def test_splitmix64_first_output():
    # SplitMix64 seeded with 0 yields 0xE220A8397B1DCDAF first
    assert om.splitmix64(0) == 0xE220A8397B1DCDAF


def test_gradient_matches_finite_differences():
    P = om.init(3)
    X, T = _data()
    _, G = om.loss_and_grads(P, X, T, round=False)
    rng = np.random.default_rng(1)
    offsets = np.cumsum([0] + [int(np.prod(s)) for _, s in om.SIZES])
    for t in range(len(om.SIZES)):
        for e in rng.integers(offsets[t], offsets[t + 1], 4):
            if t == 0 and (e % 64) >= 51:
                continue
            h = 1e-6
            Pp, Pm = P.copy(), P.copy()
            Pp[e] += h
            Pm[e] -= h
            fd = (om.loss_and_grads(Pp, X, T, round=False)[0] - om.loss_and_grads(Pm, X, T, round=False)[0]) / (2 * h)
            assert abs(G[e] - fd) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (e, G[e], fd)


def test_loss_is_sign_invariant_and_zero_at_target():
    P = om.init(4)
    X, T = _data()
    D, _ = om.forward(P, X)
    assert np.allclose(np.linalg.norm(D, axis=1), 1.0)
    l1, _ = om.loss_and_grads(P, X, T)
    l2, _ = om.loss_and_grads(P, X, -T)
    assert l1 == pytest.approx(l2, abs=1e-15)
    D0, _ = om.forward(P, X, round=False)
    l0, g0 = om.loss_and_grads(P, X, D0, round=False)
    assert l0 == pytest.approx(0.0, abs=1e-12)
    assert np.max(np.abs(g0)) < 1e-9


def test_adam_first_step_closed_form():
    P = np.array([1.0, -2.0, 0.5])
    G = np.array([0.3, -4.0, 1e-3])
    P1, M1, V1 = om.adam(P, G, np.zeros(3), np.zeros(3), 1, 1e-3)
    # first step: m_hat = g, v_hat = g^2, update = lr g / (|g| + eps)
    assert np.allclose(P1, P - 1e-3 * G / (np.abs(G) + 1e-8))
    assert np.allclose(M1, 0.1 * G) and np.allclose(V1, 0.001 * G * G)


def test_bf16_rounding_matches_torch():
    import torch
    x = np.random.default_rng(2).normal(size=10000) * np.exp(np.random.default_rng(3).normal(size=10000) * 4)
    ours = om.bf16(x)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)
    assert np.array_equal(om.from_bits(om.bf16_bits(x)), ref)


def test_init_range_and_padding():
    P = om.init(9)
    p = om.unpack(P)
    assert np.all(p["W1"][:, 51:] == 0.0)
    assert np.max(np.abs(p["W1"])) <= 1 / np.sqrt(51) and np.max(np.abs(p["W2"])) <= 1 / np.sqrt(256)
    assert np.array_equal(P, om.init(9)) and not np.array_equal(P, om.init(10))
    assert P.size == om.COUNT == 83203


def test_features_closed_form():
    """One point seen by one constant map: features are (sin 2t, cos 2t, C) for every feature view
    mapping to that view; the bounding-box centre maps to 0 and the extreme side to +-1."""
    cam = np.array([100.0, 100.0, 32.0, 32.0, 1, 0, 0, 0, -1, 0, 0, 0, -1, 0, 0, 3])
    theta, C = 0.4, 0.7
    ang = np.full((1, 64, 64), theta, np.float32)
    cf = np.full((1, 64, 64), C, np.float32)
    pts = np.array([[0.0, 0.0, 0.0], [0.2, -0.1, 0.05], [-0.2, 0.3, -0.05]])
    f = oracle.features(oracle.Scene(pts, cam[None], ang, cf, None))
    for m in range(16):   # V = 1: every feature view is view 0
        assert f[0, 3 * m] == pytest.approx(np.sin(2 * theta)) and f[0, 3 * m + 1] == pytest.approx(np.cos(2 * theta))
        assert f[0, 3 * m + 2] == pytest.approx(C, abs=1e-7)
    centre = (pts.min(0) + pts.max(0)) / 2
    half = 0.5 * np.max(pts.max(0) - pts.min(0))
    assert np.allclose(f[:, 48:51], (pts - centre) / half)
    assert np.max(np.abs(f[:, 48:51])) == pytest.approx(1.0)
    assert np.all(f[:, 51:] == 0.0)
