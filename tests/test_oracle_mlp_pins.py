"""Pins of the oracle's MLP surrogate (CPU only): backward pass against finite
differences (FP64, rounding off), special cases with closed forms (zero hidden
weights; the linear regime of SiLU against matrix products), one Adam step in
closed form, the counter generator against an independent splitmix64, and the
BF16 rounding against torch's bfloat16 conversion."""
import numpy as np
import pytest

import oracle
from paper_1910_12214_b300 import synth

OW1, OB1, OW2, OB2, OW3, OB3 = 0, 192, 256, 4352, 4416, 4608


def _params(seed=3):
    P = oracle.mlp_init(seed, 2)
    rng = np.random.default_rng(seed)
    P[OB1:OW2] = rng.normal(0, 0.3, 64)
    P[OB2:OW3] = rng.normal(0, 0.3, 64)
    P[OB3:] = rng.normal(0, 0.3, 3)
    return P


def test_backprop_matches_finite_differences():
    P = _params()
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, (8, 3))
    t = rng.normal(0, 0.5, (8, 3))
    g, loss = oracle.mlp_grad(P, x, t, exact=True)
    idx = np.concatenate([rng.choice(np.arange(0, OB1), 8), rng.choice(np.arange(OB1, OW2), 4),
                          rng.choice(np.arange(OW2, OB2), 16), rng.choice(np.arange(OB2, OW3), 4),
                          rng.choice(np.arange(OW3, OB3), 8), np.arange(OB3, 4611)])
    for k in idx:
        h = 1e-3 * max(1.0, abs(float(P[k])))
        Pp, Pm = P.astype(np.float64).copy(), P.astype(np.float64).copy()
        # FD in float32 parameters would be too coarse: evaluate the loss in FP64 by hand-shifting
        Pp[k] += h
        Pm[k] -= h
        lp = np.mean(np.sum((oracle.mlp_forward(Pp.astype(np.float32), x, exact=True) - t) ** 2, axis=1))
        lm = np.mean(np.sum((oracle.mlp_forward(Pm.astype(np.float32), x, exact=True) - t) ** 2, axis=1))
        hp = float(np.float32(P[k] + h)) - float(P[k])  # the step actually taken in float32
        hm = float(P[k]) - float(np.float32(P[k] - h))
        fd = (lp - lm) / (hp + hm)
        assert abs(fd - g[k]) <= 2e-4 * max(1e-3, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_zero_hidden_weights_give_the_output_bias():
    P = _params()
    P[OW2:OB2] = 0.0
    P[OB2:OW3] = 0.0  # h2 = SiLU(0) = 0
    x = np.random.default_rng(2).uniform(-1, 1, (5, 3))
    for exact in (True, False):
        out = oracle.mlp_forward(P, x, exact=exact)
        assert np.array_equal(out, np.tile(P[OB3:].astype(np.float64), (5, 1)))


def test_linear_regime_equals_matrix_products():
    """With large positive pre-activations SiLU(z) = z / (1 + e^-z) ~ z, so the
    network is the affine map W3 (W2 (W1 x + b1) + b2) + b3."""
    rng = np.random.default_rng(4)
    P = np.zeros(4611, np.float32)
    W1 = rng.uniform(-0.1, 0.1, (64, 3))
    W2 = rng.uniform(-0.01, 0.01, (64, 64))
    W3 = rng.uniform(-0.1, 0.1, (3, 64))
    P[OW1:OB1] = W1.ravel()
    P[OB1:OW2] = 40.0
    P[OW2:OB2] = W2.ravel()
    P[OB2:OW3] = 40.0
    P[OW3:OB3] = W3.ravel()
    P[OB3:] = [0.1, -0.2, 0.3]
    W1, W2, W3 = (P[a:b].astype(np.float64).reshape(s) for a, b, s in
                  ((OW1, OB1, (64, 3)), (OW2, OB2, (64, 64)), (OW3, OB3, (3, 64))))
    x = rng.uniform(-1, 1, (6, 3))
    ref = (W3 @ (W2 @ (W1 @ x.T + 40.0) + 40.0) + P[OB3:, None].astype(np.float64)).T
    out = oracle.mlp_forward(P, x, exact=True)
    assert np.max(np.abs(out - ref)) < 1e-12 * 1e4


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(5)
    w0 = rng.normal(size=50)
    g = rng.normal(size=50)
    w1, m, v = oracle.adam(w0, np.zeros(50), np.zeros(50), g, t=1, T=100, lr=1e-3)
    assert np.allclose(w1, w0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_counter_generator_is_splitmix64():
    m = (1 << 64) - 1
    for seed, a, b, k in [(1, 0, 0, 0), (7, 3, 12345, 99), (2 ** 40 + 3, 35, 0x5EED00000000, 4610)]:
        h = synth.splitmix64((synth.splitmix64((synth.splitmix64((seed + a) & m) + b) & m) + k) & m)
        assert oracle.counter_uniform(seed, a, b, k) == (h >> 40) / 2.0 ** 24
    u = np.array([oracle.counter_uniform(1, 0, 0, k) for k in range(4000)])
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.02


def test_bf16_rounding_is_round_to_nearest_even():
    import torch
    vals = np.random.default_rng(6).normal(0, 10, 2000).astype(np.float32)
    vals = np.concatenate([vals, np.float32([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0])])
    ref = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.bf16(v) for v in vals], np.float32)
    assert np.array_equal(got, ref)
