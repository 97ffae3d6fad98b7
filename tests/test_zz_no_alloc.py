"""cg_filter_noalloc: the CG filter for callers that must not allocate device memory
while running (its scratch is a static array inside the library).  It must give what
cg_filter gives, on two calls in a row (the array keeps the previous call's contents),
and refuse problems larger than the array.  Collected last on purpose."""
import numpy as np
import pytest
import torch

from tests.gpu_helpers import TOL_F32, bf, dev, host, image_case, rel_l2

pytestmark = pytest.mark.gpu


def test_noalloc_cg_matches_cg_filter_twice():
    _, g = image_case(200, 160, 21)
    G = bf().bf_weights(dev(g), 3, 2.0, 0.08)
    x0 = dev(g.reshape(-1))
    ref, info_ref, _ = bf().cg_filter(G, x0, 30)
    # a second, different problem in between leaves other contents in the static array
    _, g2 = image_case(64, 96, 22)
    G2 = bf().bf_weights(dev(g2), 2, 1.5, 0.1)
    for G_, x_, r_, it_ in [(G, x0, ref, info_ref.iters), (G2, dev(g2.reshape(-1)), None, None),
                            (G, x0, ref, info_ref.iters)]:
        x, info = bf().cg_filter_noalloc(G_, x_, 30)
        if r_ is None:
            r_, _, _ = bf().cg_filter(G_, x_, 30)
        else:
            assert info.iters == it_
        assert rel_l2(host(x), host(r_)) <= TOL_F32


def test_noalloc_cg_shifted_with_tolerance():
    _, g = image_case(128, 128, 23)
    G = bf().bf_weights(dev(g), 3, 2.0, 0.08)
    x0 = dev(g.reshape(-1))
    ref, info_ref, _ = bf().cg_filter(G, x0, 400, shift=1e-2, tol=1e-5)
    for _ in range(2):
        x, info = bf().cg_filter_noalloc(G, x0, 400, shift=1e-2, tol=1e-5)
        assert info.status == info_ref.status == "converged"
        assert info.iters == info_ref.iters
        assert rel_l2(host(x), host(ref)) <= TOL_F32


def test_noalloc_cg_rejects_oversized_problems():
    g = np.random.default_rng(0).uniform(size=(513, 512)).astype(np.float32)
    G = bf().bf_weights(dev(g), 1, 1.0, 0.1)
    with pytest.raises(bf().BFError) as e:
        bf().cg_filter_noalloc(G, dev(g.reshape(-1)), 5)
    assert e.value.code == bf().BF_EINVAL
