"""Pins of the oracle's conv-net preconditioner (oracle/convnet.py): the correlation against
an independent library routine, exact gradients against central finite differences, the
adjoint identity, the Jacobi special case, positive homogeneity and one Adam step written
from its published definition."""
import numpy as np
import pytest
from scipy import signal

from oracle import convnet as cn


def _case(h=9, w=7, seed=0, noise=0.3):
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((h, w))
    g = rng.uniform(0, 1, (h, w))
    d = rng.uniform(1, 5, (h, w))
    z = rng.standard_normal((h, w))
    W = [noise * rng.standard_normal(s) for s in cn.SHAPES]
    return r, g, d, z, W


def test_conv_is_zero_padded_cross_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 6, 5))
    w = rng.standard_normal((4, 3, 3, 3))
    y = cn.conv(x, w)
    for o in range(4):
        ref = sum(signal.correlate2d(x[c], w[o, c], mode="same", boundary="fill") for c in range(3))
        np.testing.assert_allclose(y[o], ref, atol=1e-12)


def test_conv_t_is_the_adjoint_of_conv():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((5, 7, 6))
    g = rng.standard_normal((3, 7, 6))
    w = rng.standard_normal((3, 5, 3, 3))
    lhs = np.sum(cn.conv(x, w) * g)
    rhs = np.sum(x * cn.conv_t(g, w))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_weight_gradients_match_central_differences(layer):
    r, g, d, z, W = _case()
    _, grads = cn.backward(r, g, d, z, W)
    rng = np.random.default_rng(3 + layer)
    idx = [tuple(rng.integers(0, s) for s in cn.SHAPES[layer]) for _ in range(12)]
    h = 1e-5          # truncation ~h^2, rounding ~1e-16 |loss| / h: both below 1e-9
    for ix in idx:
        Wp = [w.copy() for w in W]
        Wm = [w.copy() for w in W]
        Wp[layer][ix] += h
        Wm[layer][ix] -= h
        fd = (cn.loss(r, g, d, z, Wp) - cn.loss(r, g, d, z, Wm)) / (2 * h)
        an = grads[layer][ix]
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-9, (ix, fd, an)


def test_jacobi_weights_give_exactly_d_inverse():
    r, g, d, _, _ = _case(seed=4)
    T, _ = cn.forward(r, g, d, cn.jacobi_weights())
    np.testing.assert_allclose(T, r / d, rtol=1e-14, atol=1e-15)


def test_preconditioner_is_positively_homogeneous():
    r, g, d, _, W = _case(seed=5)
    T1, _ = cn.forward(r, g, d, W)
    T2, _ = cn.forward(3.5 * r, g, d, W)
    np.testing.assert_allclose(T2, 3.5 * T1, rtol=1e-12, atol=1e-14)


def test_adam_step_from_its_definition():
    w = [np.array([1.0, -2.0])]
    g = [np.array([0.5, 0.25])]
    m = [np.zeros(2)]
    v = [np.zeros(2)]
    W1, m1, v1 = cn.adam_step(w, g, m, v, t=1, lr=0.1)
    # first step: m_hat = g, v_hat = g^2, so each weight moves by lr * sign(g) (up to eps)
    np.testing.assert_allclose(W1[0], [0.9, -2.1], atol=1e-7)
    np.testing.assert_allclose(m1[0], 0.1 * g[0])
    np.testing.assert_allclose(v1[0], 0.001 * g[0] ** 2)


def test_adam_three_steps_hand_computed():
    """Three Adam steps on one weight with the gradients 1, -2, 0.5 (lr 0.1, beta1 0.9,
    beta2 0.999, eps 1e-8), worked out by hand from Kingma and Ba's update:
    m_t = 0.1, -0.11, -0.049;  v_t = 0.001, 0.004999, 0.005244001;
    bias-corrected m_t / (1 - 0.9^t) = 1, -0.578947..., -0.180812...;
    v_t / (1 - 0.999^t) = 1, 2.500750..., 1.749749...;
    w_t = 0.900000001, 0.936610353..., 0.950279419...  From the second step on, the
    corrections 1 - beta^t differ from their first-step values, so a dropped exponent
    fails here."""
    w, m, v = [np.array([1.0])], [np.zeros(1)], [np.zeros(1)]
    expect = [(0.1, 0.001, 0.900000001), (-0.11, 0.004999, 0.9366103534720751),
              (-0.049, 0.005244001, 0.9502794196738217)]
    for t, (g, (m_ref, v_ref, w_ref)) in enumerate(zip((1.0, -2.0, 0.5), expect), start=1):
        w, m, v = cn.adam_step(w, [np.array([g])], m, v, t=t, lr=0.1)
        np.testing.assert_allclose(m[0], [m_ref], rtol=1e-12)
        np.testing.assert_allclose(v[0], [v_ref], rtol=1e-12)
        np.testing.assert_allclose(w[0], [w_ref], rtol=1e-12)


def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient the bias corrections make m_hat = g and v_hat = g^2 at
    every step t (m_t = (1 - beta1^t) g, v_t = (1 - beta2^t) g^2), so each step moves every
    weight by lr * sign(g) up to eps, whatever t."""
    g = [np.array([0.3, -1.7, 4.0])]
    w, m, v = [np.zeros(3)], [np.zeros(3)], [np.zeros(3)]
    for t in range(1, 8):
        w_prev = w[0].copy()
        w, m, v = cn.adam_step(w, g, m, v, t=t, lr=0.05)
        np.testing.assert_allclose(w[0] - w_prev, -0.05 * np.sign(g[0]), rtol=1e-6)
