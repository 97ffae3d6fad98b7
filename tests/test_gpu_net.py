"""The learned preconditioner on the GPU (bf_net: forward, backward, Adam) against the FP64
oracle of oracle/convnet.py, and flexible CG with it (Algorithm 2 with a nonlinear T)."""
import numpy as np
import pytest
import torch

from oracle import convnet as cn
from oracle import solvers
from tests.gpu_helpers import TOL_F32, bf, dev, host, image_case, make_pair, rel_l2

pytestmark = pytest.mark.gpu


def split(w):
    """Flat weight vector -> [W1, W2, W3] (float64)."""
    w = np.asarray(w, np.float64)
    out, o = [], 0
    for s in cn.SHAPES:
        k = int(np.prod(s))
        out.append(w[o:o + k].reshape(s))
        o += k
    return out


def setup(ny=37, nx=45, seed=3, noise=0.3, wseed=0):
    _, noisy = image_case(ny, nx, seed)
    G, O = make_pair(noisy, 3, 2.0, 0.08)
    d = host(bf().graph_degree(G)).reshape(ny, nx)
    W = [np.asarray(w, np.float32) for w in cn.jacobi_weights(noise=noise, seed=wseed)]
    net = bf().Net(W)
    Wq = split(net.weights(rounded=True))
    return G, O, noisy, d, net, Wq


def test_weights_are_stored_and_rounded_to_bf16():
    W = [np.asarray(w, np.float32) for w in cn.jacobi_weights(noise=0.3, seed=1)]
    net = bf().Net(W)
    flat = np.concatenate([w.ravel() for w in W])
    np.testing.assert_array_equal(net.weights(), flat)
    wq = net.weights(rounded=True)
    # round to nearest even on the top 16 bits
    bits = flat.view(np.uint32).astype(np.uint64)
    rb = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    np.testing.assert_array_equal(wq, rb.astype(np.uint32).view(np.float32))


@pytest.mark.parametrize("k", [1, 3, 6])
def test_forward_matches_oracle(k):
    G, O, noisy, d, net, Wq = setup()
    ny, nx = noisy.shape
    rng = np.random.default_rng(7)
    R = rng.standard_normal((ny * nx, k)).astype(np.float32)
    Z = host(net.apply(G, dev(R)))
    for j in range(k):
        ref, _ = cn.forward(R[:, j].reshape(ny, nx).astype(np.float64), noisy, d, Wq)
        assert rel_l2(Z[:, j], ref.ravel()) <= TOL_F32


def test_jacobi_weights_reproduce_d_inverse():
    _, noisy = image_case(33, 70, 5)
    G, O = make_pair(noisy, 3, 2.0, 0.08)
    net = bf().Net([np.asarray(w, np.float32) for w in cn.jacobi_weights()])
    r = np.random.default_rng(2).standard_normal(noisy.size).astype(np.float32)
    z = host(net.apply(G, dev(r)))
    d = host(bf().graph_degree(G))
    assert rel_l2(z, r / d) <= 1e-6


def test_gradient_and_loss_match_oracle():
    G, O, noisy, d, net, Wq = setup(ny=40, nx=67, seed=4)
    ny, nx = noisy.shape
    rng = np.random.default_rng(9)
    r = rng.standard_normal(ny * nx).astype(np.float32)
    z = rng.standard_normal(ny * nx).astype(np.float32)
    net.zero_grad()
    net.accumulate(G, dev(r), dev(z))
    g, loss = net.grad()
    ref_loss, ref = cn.backward(r.reshape(ny, nx).astype(np.float64), noisy, d,
                                z.reshape(ny, nx).astype(np.float64), Wq)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    gs = split(g)
    for layer in range(3):
        assert rel_l2(gs[layer], ref[layer]) <= 1e-4, layer


def test_gradient_accumulates_over_pairs():
    G, O, noisy, d, net, Wq = setup(ny=24, nx=35, seed=6)
    rng = np.random.default_rng(11)
    pairs = [(rng.standard_normal(noisy.size).astype(np.float32),
              rng.standard_normal(noisy.size).astype(np.float32)) for _ in range(3)]
    net.zero_grad()
    for r, z in pairs:
        net.accumulate(G, dev(r), dev(z))
    g, loss = net.grad()
    tot = [np.zeros(s) for s in cn.SHAPES]
    tl = 0.0
    for r, z in pairs:
        l, gr = cn.backward(r.reshape(noisy.shape).astype(np.float64), noisy, d,
                            z.reshape(noisy.shape).astype(np.float64), Wq)
        tl += l
        for i in range(3):
            tot[i] += gr[i]
    assert abs(loss - tl) <= 1e-5 * tl
    for layer, gl in enumerate(split(g)):
        assert rel_l2(gl, tot[layer]) <= 1e-4


def test_adam_steps_match_definition():
    """Three Adam steps (t = 1, 2, 3), each on the gradient of a different pair: the GPU
    weights follow the oracle's adam_step chained with the same moments.  From t = 2 on the
    bias corrections 1 - beta^t differ from their t = 1 values."""
    G, O, noisy, d, net, Wq = setup(ny=20, nx=33, seed=8)
    rng = np.random.default_rng(12)
    w_ref = net.weights().astype(np.float64)
    m = [np.zeros_like(w_ref)]
    v = [np.zeros_like(w_ref)]
    for t in (1, 2, 3):
        r = rng.standard_normal(noisy.size).astype(np.float32)
        z = rng.standard_normal(noisy.size).astype(np.float32)
        net.zero_grad()
        net.accumulate(G, dev(r), dev(z))
        net.accumulate(G, dev(z), dev(r))
        g, _ = net.grad()
        net.adam(lr=1e-2, scale=0.5)
        w_gpu = net.weights().astype(np.float64)
        W, m, v = cn.adam_step([w_ref], [0.5 * g.astype(np.float64)], m, v, t=t, lr=1e-2)
        np.testing.assert_allclose(w_gpu, W[0], rtol=1e-6, atol=1e-7)
        # continue from the GPU's FP32 weights so that rounding does not accumulate
        w_ref = w_gpu
    # the BF16 copy follows the master weights, and the accumulators were reset
    wq = net.weights(rounded=True)
    assert np.max(np.abs(wq - w_gpu) / np.maximum(np.abs(w_gpu), 1e-30)) <= 2.0 ** -8
    g2, l2 = net.grad()
    assert np.all(g2 == 0) and l2 == 0.0


@pytest.mark.parametrize("shift", [0.0, 1e-2])
def test_cg_with_jacobi_net_equals_jacobi_cg(shift):
    _, noisy = image_case(48, 52, 10)
    G, O = make_pair(noisy, 3, 2.0, 0.08)
    net = bf().Net([np.asarray(w, np.float32) for w in cn.jacobi_weights()])
    x0 = dev(noisy.ravel())
    xj, ij, hj = bf().cg_filter(G, x0, 15, precond="jacobi", shift=shift, hist=True)
    xn, inn, hn = bf().cg_filter(G, x0, 15, precond="net", net=net, shift=shift, hist=True)
    assert ij.iters == inn.iters == 15
    assert rel_l2(host(xn), host(xj)) <= TOL_F32
    np.testing.assert_allclose(host(hn), host(hj), rtol=1e-4)


def test_flexible_cg_with_net_matches_oracle():
    G, O, noisy, d, net, Wq = setup(ny=44, nx=41, seed=12, noise=0.05, wseed=3)
    ny, nx = noisy.shape
    T = lambda r: cn.forward(np.asarray(r).reshape(ny, nx), noisy, d, Wq)[0].ravel()
    shift = 1e-2
    ref = solvers.cg(O, noisy.ravel().astype(np.float64), 8, precond=T, shift=shift)
    x, info, h = bf().cg_filter(G, dev(noisy.ravel()), 8, precond="net", net=net, shift=shift, hist=True)
    assert info.iters == ref["iters"] == 8
    # measured: x within 7e-8 and alpha within 9e-8 of the oracle (the net's ReLUs do not
    # flip between the FP32 and the FP64 run on this input), so the FP32 bar holds
    assert rel_l2(host(x), ref["x"]) <= TOL_F32
    np.testing.assert_allclose(host(h).reshape(-1, 2)[:, 0], ref["alpha"], rtol=1e-5)


def test_net_rejected_where_unsupported():
    _, noisy = image_case(16, 16, 1)
    G64 = bf().bf_weights(dev(noisy, torch.float64), 3, 2.0, 0.08)
    net = bf().Net([np.asarray(w, np.float32) for w in cn.jacobi_weights()])
    with pytest.raises(bf().BFError):
        bf().cg_filter(G64, dev(noisy.ravel(), torch.float64), 3, precond="net", net=net)
    G32 = bf().bf_weights(dev(noisy), 3, 2.0, 0.08)
    with pytest.raises(bf().BFError):
        bf().cg_filter(G32, dev(noisy.ravel()), 3, precond="net", net=None)
    with pytest.raises(bf().BFError):
        bf().cg_filter_noalloc(G32, dev(noisy.ravel()), 3, precond="net")


def test_lobpcg_with_jacobi_net_equals_jacobi_lobpcg():
    from tests.gpu_helpers import TOL_RITZ_SMALL_F32
    from paper_1509_02468_gb300 import synth
    _, noisy = image_case(40, 44, 13)
    G, O = make_pair(noisy, 3, 2.0, 0.08)
    net = bf().Net([np.asarray(w, np.float32) for w in cn.jacobi_weights()])
    X0 = dev(synth.block_start(noisy.ravel(), 4, 13))
    for constrain in (False, True):
        a = bf().lobpcg_filter(G, X0, 8, precond="jacobi", constrain=constrain)
        b = bf().lobpcg_filter(G, X0, 8, precond="net", net=net, constrain=constrain)
        th_a, th_b = host(a["theta"]), host(b["theta"])
        scale = np.maximum(np.abs(th_a), 1e-3 * np.abs(th_a).max())
        assert np.max(np.abs(th_a - th_b) / scale) <= TOL_RITZ_SMALL_F32
        assert rel_l2(host(b["y"]), host(a["y"])) <= TOL_F32


def test_lobpcg_with_net_gives_valid_ritz_pairs():
    """With a nonlinear T the trajectory is not reproducible at FP32 level: Ritz-vector signs
    are arbitrary and T(-r) != -T(r), so the oracle's own run moves by ~1e-3 under a 6e-8
    perturbation of the start block.  What is unique is checked instead: X B-orthonormal,
    theta the Rayleigh quotients of X, theta above the exact eigenvalues of the pencil
    (Cauchy interlacing), and the reported residual norms those of X."""
    import scipy.linalg as sla
    from paper_1509_02468_gb300 import synth
    G, O, noisy, d, net, Wq = setup(ny=36, nx=40, seed=14, noise=0.05, wseed=5)
    k = 4
    X0 = synth.block_start(noisy.ravel(), k, 14)
    out = bf().lobpcg_filter(G, dev(X0), 6, precond="net", net=net)
    X, th, res = host(out["X"]), host(out["theta"]), host(out["resid"])
    L, D = O.L.toarray(), O.d
    np.testing.assert_allclose(X.T @ (D[:, None] * X), np.eye(k), atol=2e-5)
    rq = np.einsum("ij,ij->j", X, L @ X) / np.einsum("ij,ij->j", X, D[:, None] * X)
    scale = np.maximum(np.abs(rq), 1e-3 * np.abs(rq).max())
    assert np.max(np.abs(th - rq) / scale) <= 1e-4
    lam = sla.eigh(L, np.diag(D), eigvals_only=True)[:k]
    assert np.all(th >= lam - 1e-6 * np.abs(lam).max())
    R = L @ X - (D[:, None] * X) * th[None, :]
    rn = np.linalg.norm(R, axis=0) / np.linalg.norm(D[:, None] * X, axis=0)
    np.testing.assert_allclose(res, rn, rtol=2e-2, atol=1e-6)
