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
