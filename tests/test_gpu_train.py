"""Training of the learned preconditioner with the library's own kernels: the pairs solve
(L + sigma I) z = r, and Adam on them lowers the loss from the Jacobi-equivalent start."""
import numpy as np
import pytest
import torch

from tests.gpu_helpers import bf

pytestmark = pytest.mark.gpu


def test_pairs_solve_the_shifted_system():
    from paper_1509_02468_gb300 import train
    pairs = train.make_pairs([1000, 1001], 48, picks=(0, 3))
    for G, r, z in pairs:
        Az = bf().bf_apply(G, "L", z).double() + train.SIGMA * z.double()
        rel = torch.linalg.vector_norm(Az - r.double()) / torch.linalg.vector_norm(r.double())
        assert rel <= 1e-4     # z solved to 1e-8 in FP64, then rounded to FP32 (amplified by cond)


def test_training_lowers_the_loss():
    from paper_1509_02468_gb300 import train
    pairs = train.make_pairs(range(1000, 1006), 64, picks=(0, 2, 5))
    net = bf().Net(train.initial_weights())
    before = train.mean_loss(net, pairs)
    hist = train.train(net, pairs, epochs=4, batch=6, lr=2e-3)
    after = train.mean_loss(net, pairs)
    assert np.isfinite(hist).all()
    assert after < before, (before, after)


def test_trained_net_against_jacobi_on_held_out_1024():
    """The shifted system on the held-out 1024 x 1024 image (seed 5, sigma 1e-2) solved to a
    TRUE relative residual of 1e-5 by the library's refinement (FP64 residuals, flexible
    FP32 CG inner solves to 1e-3) with T = Jacobi and with a net trained here on 32 pairs
    of 8 images (128 x 128).  Records inner iterations and Mpix/s of both; every run that
    reports convergence is checked with the oracle's FP64 matrices.  (The nets this
    training reaches are neither linear nor odd, so flexible CG may stall with them: the
    record says which.)"""
    import json
    import time

    import scipy.sparse as sp

    from oracle.graph import Graph
    from paper_1509_02468_gb300 import synth, train
    pairs = train.make_pairs(range(1000, 1008), 128, picks=(0, 2, 6, 13))
    net = bf().Net(train.initial_weights())
    train.train(net, pairs, epochs=3, batch=8, lr=2e-3)
    _, noisy = synth.polygon_image(1024, 1024, 5)
    g32 = torch.as_tensor(noisy, device="cuda")
    G32 = bf().bf_weights(g32, train.RADIUS, train.SIGMA_S, train.SIGMA_R)
    G64 = bf().bf_weights(g32.double(), train.RADIUS, train.SIGMA_S, train.SIGMA_R)
    O = Graph(noisy.astype(np.float64), noisy.shape, train.RADIUS, train.SIGMA_S, train.SIGMA_R)
    A = (O.L + train.SIGMA * sp.identity(O.n, format="csr")).tocsr()
    x0 = noisy.reshape(-1).astype(np.float64)
    b = train.SIGMA * x0
    rec = {}
    for name, kw in (("jacobi", dict(precond="jacobi")), ("net", dict(precond="net", net=net))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, rel, inner, outer = train.refined_cg(G32, G64, g32.reshape(-1), train.SIGMA, 1e-5, outer_max=12, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ok = bool(rel <= 1e-5)
        rec[name] = {"converged": ok, "inner_iters": inner, "outer": outer, "seconds": dt,
                     "mpix_s": noisy.size / dt / 1e6, "reported_rel": rel}
        if ok:
            true = float(np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b))
            rec[name]["oracle_rel"] = true
            assert true <= 1.01e-5, (name, true)
    print("learned-vs-jacobi " + json.dumps(rec))
    assert rec["jacobi"]["converged"]
