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
