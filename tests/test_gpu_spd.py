"""The learned symmetric positive definite preconditioner T = D^-1/2 (I + K^T K) D^-1/2
(bf_spd) on the GPU against the oracle (oracle/precond_spd.py): its application, the
A-norm loss and gradient, Adam, CG (Algorithm 2) and LOBPCG (Algorithm 3) with it, and
what a K trained by the library's own kernels gains over Jacobi on the held-out
1024 x 1024 image of the shifted system."""
import json
import time

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl
import torch

from oracle import convnet, precond_spd as ps, solvers
from paper_1509_02468_gb300 import synth
from tests.gpu_helpers import TOL_F32, TOL_RITZ_SMALL_F32, bf, dev, host, image_case, make_pair, rel_l2

pytestmark = pytest.mark.gpu


def _kernel(half, seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal((2 * half + 1, 2 * half + 1))).astype(np.float32)


@pytest.mark.parametrize("half,k", [(1, 1), (3, 1), (3, 3), (4, 2)])
def test_apply_matches_oracle(half, k):
    """Z = T R on a ragged image (several 32 x 8 tiles, partial edge tiles), k columns."""
    _, g = image_case(45, 77, 31)
    G, O = make_pair(g, 3, 2.0, 0.08)
    K = _kernel(half, half + 10 * k)
    T = bf().Spd(half, K)
    R = np.random.default_rng(k).standard_normal((O.n, k))
    Rd = dev(R)
    Z = host(T.apply(G, Rd if k > 1 else Rd[:, 0]))
    ref = ps.apply(K.astype(np.float64), O.d, g.shape, host(Rd) if k > 1 else host(Rd)[:, 0])
    assert rel_l2(Z, ref) <= TOL_F32, rel_l2(Z, ref)
    # in place
    Zi = T.apply(G, Rd, out=Rd)
    assert rel_l2(host(Zi).reshape(ref.shape), ref) <= TOL_F32


def test_zero_kernel_is_jacobi():
    _, g = image_case(40, 33, 32)
    G, O = make_pair(g, 3, 2.0, 0.08)
    r = dev(np.random.default_rng(0).standard_normal(O.n))
    z = host(bf().Spd(3).apply(G, r))
    assert rel_l2(z, host(r) / O.d) <= 1e-6


def _pair(shape=(38, 53), seed=33, sigma=0.05):
    _, g = image_case(*shape, seed)
    G, O = make_pair(g, 3, 2.0, 0.08)
    A = (O.L + sigma * sp.identity(O.n, format="csr")).tocsr()
    r = np.random.default_rng(seed).standard_normal(O.n).astype(np.float32).astype(np.float64)
    z = spl.spsolve(A.tocsc(), r).astype(np.float32).astype(np.float64)
    return G, O, A, r, z, g.shape


@pytest.mark.parametrize("half", [2, 3])
def test_loss_and_gradient_match_oracle(half):
    """The A-norm loss of one pair and its gradient with respect to K; FP32 operator and
    stencil passes with FP64 sums: gradient to 1e-4 relative (the entries are sums of
    ~2000 products of FP32 values with cancellation between the two terms)."""
    G, O, A, r, z, shape = _pair()
    K = _kernel(half, 7 + half)
    T = bf().Spd(half, K)
    T.zero_grad()
    T.accumulate(G, 0.05, dev(r), dev(z))
    grad, loss = T.grad()
    ref_loss, ref_grad = ps.loss_grad(K.astype(np.float64), O.d, shape, A, r, z)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    assert np.linalg.norm(grad - ref_grad) <= 1e-4 * np.linalg.norm(ref_grad), (grad, ref_grad)
    # accumulation over pairs adds, and zero_grad resets
    T.accumulate(G, 0.05, dev(r), dev(z))
    grad2, loss2 = T.grad()
    np.testing.assert_allclose(grad2, 2 * grad, rtol=1e-12)
    assert loss2 == pytest.approx(2 * loss, rel=1e-12)
    T.zero_grad()
    g0, l0 = T.grad()
    assert l0 == 0.0 and not g0.any()


def test_three_adam_steps_match_oracle():
    """Three chained Adam steps on the mean gradient of two pairs, against Kingma and Ba's
    update (oracle/convnet.adam_step) applied to the GPU's own gradients."""
    G, O, A, r, z, shape = _pair()
    G2, O2, A2, r2, z2, shape2 = _pair((29, 41), 34)
    K = _kernel(3, 21)
    T = bf().Spd(3, K)
    W, m, v = [K.astype(np.float64)], [np.zeros_like(K, np.float64)], [np.zeros_like(K, np.float64)]
    for t in (1, 2, 3):
        T.zero_grad()
        T.accumulate(G, 0.05, dev(r), dev(z))
        T.accumulate(G2, 0.05, dev(r2), dev(z2))
        grad, _ = T.grad()
        T.adam(3e-3, 0.5)
        W, m, v = convnet.adam_step(W, [0.5 * grad], m, v, t, lr=3e-3)
        np.testing.assert_allclose(T.kernel(), W[0], rtol=1e-5, atol=1e-7)


def test_cg_with_spd_matches_oracle():
    """Algorithm 2 on the shifted system with T = the SPD preconditioner, fixed count, and
    the plain system: the FP32 GPU iterate against the oracle's CG with the same T."""
    _, g = image_case(64, 75, 35)
    G, O = make_pair(g, 3, 2.0, 0.08)
    K = _kernel(3, 36, 0.15)
    T = bf().Spd(3, K)
    Tref = lambda v: ps.apply(K.astype(np.float64), O.d, g.shape, v)
    x0 = dev(g.reshape(-1))
    for shift, iters in ((0.01, 30), (0.0, 15)):
        x, info, _ = bf().cg_filter(G, x0, iters, precond="spd", spd=T, shift=shift)
        ref = solvers.cg(O, host(x0), iters, precond=Tref, shift=shift)
        assert info.iters == ref["iters"] == iters
        assert rel_l2(host(x), ref["x"]) <= TOL_F32, rel_l2(host(x), ref["x"])


def test_lobpcg_with_spd_matches_oracle():
    """Algorithm 3 for the pencil (L, D) with T = the SPD preconditioner."""
    _, g = image_case(48, 53, 37)
    G, O = make_pair(g, 2, 2.0, 0.08)
    K = _kernel(2, 38, 0.15)
    T = bf().Spd(2, K)
    Tref = lambda V: ps.apply(K.astype(np.float64), O.d, g.shape, V)
    X0 = dev(synth.block_start(g.reshape(-1), 4, seed=3))
    out = bf().lobpcg_filter(G, X0, 12, precond="spd", spd=T)
    ref = solvers.lobpcg(O, host(X0), 12, precond=Tref)
    th, rt = host(out["theta"]), np.asarray(ref["theta"])
    err = np.max(np.abs(th - rt) / np.maximum(np.abs(rt), 1e-3 * np.abs(rt).max()))
    assert err <= TOL_RITZ_SMALL_F32, err
    assert rel_l2(host(out["y"]), ref["y"]) <= TOL_F32


def test_rejects_bad_arguments():
    _, g = image_case(20, 21, 39)
    G, _ = make_pair(g, 3, 2.0, 0.08)
    with pytest.raises(bf().BFError):
        bf().Spd(5)
    with pytest.raises(bf().BFError):
        bf().cg_filter(G, dev(g.reshape(-1)), 3, precond="spd")          # no bf_spd
    G64, _ = make_pair(g, 3, 2.0, 0.08, dtype=torch.float64)
    with pytest.raises(bf().BFError):
        bf().cg_filter(G64, dev(g.reshape(-1), torch.float64), 3, precond="spd", spd=bf().Spd(1))


def test_trained_spd_against_jacobi_on_held_out_1024():
    """K (7 x 7) trained by the library's kernels (A-norm loss, full-batch Adam, 36 pairs of
    six 128 x 128 images with white-noise residuals) on the shifted system of the held-out
    1024 x 1024 image (seed 5, sigma 1e-2), solved to a TRUE relative residual of 1e-5 by the
    library's refinement (FP64 residuals, FP32 inner CG to 1e-3): inner iterations and
    Mpix/s with T = Jacobi and with the trained T, both checked with the oracle's FP64
    matrices.  The trained T must need fewer iterations."""
    from oracle.graph import Graph
    from paper_1509_02468_gb300 import train
    pairs = train.make_random_pairs(range(1000, 1006), 128, 6)
    T = bf().Spd(3, train.spd_initial_kernel(3))
    hist = train.train_spd(T, pairs, epochs=200, lr=3e-3)
    assert hist[-1] < hist[0]
    _, noisy = synth.polygon_image(1024, 1024, 5)
    g32 = torch.as_tensor(noisy, device="cuda")
    G32 = bf().bf_weights(g32, train.RADIUS, train.SIGMA_S, train.SIGMA_R)
    G64 = bf().bf_weights(g32.double(), train.RADIUS, train.SIGMA_S, train.SIGMA_R)
    O = Graph(noisy.astype(np.float64), noisy.shape, train.RADIUS, train.SIGMA_S, train.SIGMA_R)
    A = (O.L + train.SIGMA * sp.identity(O.n, format="csr")).tocsr()
    b = train.SIGMA * noisy.reshape(-1).astype(np.float64)
    rec = {"loss_first_epoch": hist[0], "loss_last_epoch": hist[-1]}
    for name, kw in (("jacobi", dict(precond="jacobi")), ("spd", dict(precond="spd", spd=T))):
        train.refined_cg(G32, G64, g32.reshape(-1), train.SIGMA, 1e-5, **kw)          # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, rel, inner, outer = train.refined_cg(G32, G64, g32.reshape(-1), train.SIGMA, 1e-5, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        true = float(np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b))
        rec[name] = {"inner_iters": inner, "outer": outer, "seconds": dt, "mpix_s": noisy.size / dt / 1e6,
                     "reported_rel": rel, "oracle_rel": true}
        assert rel <= 1e-5 and true <= 1.01e-5, (name, rel, true)
    print("spd-vs-jacobi " + json.dumps(rec))
    assert rec["spd"]["inner_iters"] < 0.8 * rec["jacobi"]["inner_iters"], rec
