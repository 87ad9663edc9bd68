"""Pins for the oracle's fp64 learned-step MLP: gradients against central
finite differences, the forward pass against a plain numpy restatement of a
dense layer stack computed by matrix products, and Adam against its
closed-form first step."""
import numpy as np

import synth


def _params(seed, scale=0.3):
    import oracle
    rng = synth.SplitMix64(seed)
    return (rng.uniform(oracle.mlp_nparam()) * 2 - 1) * scale


def test_gradient_matches_central_differences(oracle_lib):
    rng = synth.SplitMix64(3)
    B = 7
    x = rng.uniform(B * 16).reshape(B, 16) * 2 - 1
    t = rng.uniform(B * 2).reshape(B, 2)
    p = _params(4)
    loss, g = oracle_lib.mlp_loss_grad(x, t, p)
    h = 1e-6
    idx = np.unique(np.concatenate([np.arange(0, p.size, 97), [0, 1023, 1024, 1087, 5375, 5377]]))
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle_lib.mlp_loss_grad(x, t, pp)[0] - oracle_lib.mlp_loss_grad(x, t, pm)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_is_a_relu_layer_stack(oracle_lib):
    rng = synth.SplitMix64(5)
    x = rng.uniform(33 * 16).reshape(33, 16) - 0.5
    p = _params(6)
    W1 = p[:1024].reshape(64, 16); b1 = p[1024:1088]
    W2 = p[1088:5184].reshape(64, 64); b2 = p[5184:5248]
    W3 = p[5248:5376].reshape(2, 64); b3 = p[5376:5378]
    ref = np.maximum(np.maximum(x @ W1.T + b1, 0) @ W2.T + b2, 0) @ W3.T + b3
    assert np.allclose(oracle_lib.mlp_forward(x, p), ref, rtol=1e-12, atol=1e-12)
    assert oracle_lib.mlp_nparam() == 5378


def test_adam_first_step_moves_each_weight_by_lr(oracle_lib):
    p = np.zeros(10)
    m = np.zeros(10)
    v = np.zeros(10)
    g = np.linspace(-2, 2, 10)
    g[5] = 0.0
    oracle_lib.adam_step(p, g, m, v, 1e-3, step=1)
    # first step: m_hat = g, v_hat = g^2 -> -lr * sign(g) (up to eps)
    assert np.allclose(p, -1e-3 * np.sign(g), atol=1e-9)
