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


def test_adam_steps_with_a_constant_gradient(oracle_lib):
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2 at every step, so K steps move each weight by K lr sign(g) (up to eps)."""
    g = np.array([-3.0, -0.5, 0.25, 2.0, 7.0])
    p, m, v = np.zeros(5), np.zeros(5), np.zeros(5)
    for k in range(1, 6):
        oracle_lib.adam_step(p, g, m, v, 1e-2, step=k)
        assert np.allclose(m, (1 - 0.9 ** k) * g, rtol=1e-14)
        assert np.allclose(v, (1 - 0.999 ** k) * g * g, rtol=1e-14)
    assert np.allclose(p, -5e-2 * np.sign(g), atol=1e-8)


# ---- the error bound of a reduced-precision network (the GPU's tolerance)
def _bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even)."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _split(p):
    return (p[:1024].reshape(64, 16), p[1024:1088], p[1088:5184].reshape(64, 64), p[5184:5248],
            p[5248:5376].reshape(2, 64), p[5376:5378])


def _emulate(x, t, p, mistake=None, flip_tiny=False):
    """A float32 computation of the network, loss and gradient that rounds the
    hidden activations and the weight-gradient operands to bfloat16 -- the
    model the bound is stated for -- written independently of the oracle.
    flip_tiny: an adversarial member of the model that inverts the first-layer
    ReLU decision wherever the pre-activation is within 1e-7 of its
    magnitude (the model allows either decision there)."""
    f = np.float32
    W1, b1, W2, b2, W3, b3 = (a.astype(f) for a in _split(p))
    x = x.astype(f)
    B = x.shape[0]
    z1 = x @ W1.T + b1
    h1 = _bf16(np.maximum(z1, 0))
    z2 = h1 @ W2.T + b2
    h2 = _bf16(np.maximum(z2, 0))
    y = h2 @ W3.T + b3
    e = y - t.astype(f)
    loss = f(np.sum(e * e, dtype=f) / f(B))
    dy = (f(2) * e) / f(B)
    if mistake == "no_two":  # dL/dy without the factor 2
        dy = e / f(B)
    g2 = dy @ W3
    dz2 = g2 if mistake == "no_mask2" else np.where(z2 > 0, g2, f(0))
    g1 = _bf16(dz2) @ W2
    on1 = z1 > 0
    if flip_tiny:
        m1 = np.abs(x) @ np.abs(W1).T + np.abs(b1)
        on1 = on1 ^ (np.abs(z1) < f(1e-7) * m1)
    dz1 = np.where(on1, g1, f(0))
    gW3 = _bf16(dy).T @ h2
    gW2 = _bf16(dz2).T @ (_bf16(z1) if mistake == "pre_relu" else h1)
    if mistake == "shift_sample":  # activations of the neighbouring sample
        gW2 = _bf16(dz2).T @ np.roll(h1, 1, axis=0)
    gW1 = _bf16(dz1).T @ x
    gb1, gb2, gb3 = dz1.sum(0), dz2.sum(0), dy.sum(0)
    if mistake == "transpose_W2":
        gW2 = gW2.T
    if mistake == "drop_b1":
        gb1 = np.zeros_like(gb1)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3]).astype(np.float64)
    return y.astype(np.float64), float(loss), g


def _case(seed, B, near_zero=False):
    rng = synth.SplitMix64(seed)
    x = _bf16(rng.uniform(B * 16).reshape(B, 16) * 2 - 1).astype(np.float64)
    t = rng.uniform(B * 2).reshape(B, 2) - 0.5
    p = _params(seed + 1).astype(np.float32)
    w = np.ones(p.size, bool)
    for off, cnt in ((1024, 64), (5184, 64), (5376, 2)):
        w[off:off + cnt] = False
    p[w] = _bf16(p[w])
    p = p.astype(np.float64)
    if near_zero:  # first-layer biases that put sample 0's pre-activations at 0
        W1 = p[:1024].reshape(64, 16)
        p[1024:1088] = (-(W1 @ x[0])).astype(np.float32)
    return x, t, p


def test_error_bound_covers_the_reduced_precision_model(oracle_lib):
    for seed, B, nz in ((31, 1, False), (32, 64, False), (33, 333, False), (34, 97, True), (36, 1, True)):
        x, t, p = _case(seed, B, nz)
        y0 = oracle_lib.mlp_forward(x, p)
        l0, g0 = oracle_lib.mlp_loss_grad(x, t, p)
        yb, gb, lb = oracle_lib.mlp_error_bound(x, t, p)
        y1, l1, g1 = _emulate(x, t, p)
        assert np.all(np.abs(y1 - y0) <= yb), seed
        assert abs(l1 - l0) <= lb, seed
        bad = np.abs(g1 - g0) > gb
        assert not np.any(bad), (seed, np.flatnonzero(bad)[:5])
        if nz:  # sample 0 sits on every first-layer ReLU edge
            _, _, g2 = _emulate(x, t, p, flip_tiny=True)
            assert np.any(g2 != g1), seed
            bad = np.abs(g2 - g0) > gb
            assert not np.any(bad), (seed, "flipped", np.flatnonzero(bad)[:5])
        # a worst-case bound, yet below the size of the values it bounds
        assert np.median(yb / np.abs(y0)) < 0.5, seed
        assert np.median(gb[g0 != 0] / np.abs(g0[g0 != 0])) < 1.0, seed


def test_error_bound_without_rounding_is_the_accumulation_error(oracle_lib):
    x, t, p = _case(41, 50)
    yb, gb, lb = oracle_lib.mlp_error_bound(x, t, p, u_act=0.0, u_grad=0.0)
    _, g0 = oracle_lib.mlp_loss_grad(x, t, p)
    y0 = oracle_lib.mlp_forward(x, p)
    assert np.max(yb) < 2e-3 * max(1.0, np.max(np.abs(y0)))  # 2^-23 (K + 1), times the weights' gain
    assert np.max(gb) < 2e-3 * np.max(np.abs(g0))
    yb8, gb8, _ = oracle_lib.mlp_error_bound(x, t, p)
    assert np.all(yb8 > 10 * yb) and np.median(gb8 / np.maximum(gb, 1e-300)) > 10


def test_error_bound_catches_planted_gradient_mistakes(oracle_lib):
    """A wrong slice or a wrong factor in the gradient -- a dropped bias vector,
    a transposed weight matrix, a missing ReLU mask, dL/dy without its factor
    2, pre-activations or the next sample's activations in a weight gradient --
    leaves the bound somewhere."""
    x, t, p = _case(51, 256)
    _, g0 = oracle_lib.mlp_loss_grad(x, t, p)
    _, gb, _ = oracle_lib.mlp_error_bound(x, t, p)
    for mk in ("drop_b1", "transpose_W2", "no_mask2", "no_two", "pre_relu", "shift_sample"):
        _, _, g1 = _emulate(x, t, p, mistake=mk)
        assert np.any(np.abs(g1 - g0) > gb), mk
