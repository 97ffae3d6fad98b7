"""cg_filter_noalloc: the CG filter (Algorithm 2) for callers that must not allocate device
memory while running -- a memory budget owned by another allocator, or a loop that cannot
take the device-wide synchronisation of cudaMalloc/cudaFree.  Its scratch is a static
array inside the library, shared by every call and holding the previous call's contents.

It runs cg_filter's own code on that array, so its output must equal cg_filter's exactly,
and both must match the FP64 oracle: checked on two calls in a row (with another problem
in between), on FP32 and FP64 graphs, with weights on the fly and stored, with a shift and
a tolerance; problems larger than the array are refused.  Collected last on purpose."""
import numpy as np
import pytest
import torch

from oracle import solvers
from tests.gpu_helpers import TOL_F32, TOL_F64, bf, dev, host, image_case, make_pair, rel_l2

pytestmark = pytest.mark.gpu


def test_noalloc_cg_matches_cg_filter_and_oracle_twice():
    _, g = image_case(200, 160, 21)
    G, O = make_pair(g, 3, 2.0, 0.08)
    x0 = dev(g.reshape(-1))
    ref = solvers.cg(O, g.reshape(-1).astype(np.float64), 30)["x"]
    xc, info_c, _ = bf().cg_filter(G, x0, 30)
    # a second, different problem in between leaves other contents in the static array
    _, g2 = image_case(64, 96, 22)
    G2, O2 = make_pair(g2, 2, 1.5, 0.1)
    ref2 = solvers.cg(O2, g2.reshape(-1).astype(np.float64), 30)["x"]
    for G_, x_, r_ in [(G, x0, ref), (G2, dev(g2.reshape(-1)), ref2), (G, x0, ref)]:
        x, info = bf().cg_filter_noalloc(G_, x_, 30)
        assert info.iters == 30
        assert rel_l2(host(x), r_) <= TOL_F32
        if G_ is G:
            assert torch.equal(x, xc)


@pytest.mark.parametrize("mode", ["stored_f32", "stored_bf16"])
def test_noalloc_cg_stored_weights(mode):
    """Stored weights: the oracle's operator is built from the stored (rounded) values."""
    _, g = image_case(96, 110, 24)
    G, O = make_pair(g, 3, 2.0, 0.08, mode=mode)
    x0 = dev(g.reshape(-1))
    ref = solvers.cg(O, g.reshape(-1).astype(np.float64), 25)["x"]
    xc, _, _ = bf().cg_filter(G, x0, 25)
    for _ in range(2):
        x, _ = bf().cg_filter_noalloc(G, x0, 25)
        assert rel_l2(host(x), ref) <= TOL_F32
        assert torch.equal(x, xc)


def test_noalloc_cg_fp64_graph():
    _, g = image_case(70, 90, 25, dtype=np.float64)
    G, O = make_pair(g, 2, 2.0, 0.1, dtype=torch.float64)
    x0 = dev(g.reshape(-1), torch.float64)
    ref = solvers.cg(O, g.reshape(-1), 20)["x"]
    for _ in range(2):
        x, info = bf().cg_filter_noalloc(G, x0, 20)
        assert info.iters == 20
        assert rel_l2(host(x), ref) <= TOL_F64


def test_noalloc_cg_shifted_with_tolerance():
    _, g = image_case(128, 128, 23)
    G, O = make_pair(g, 3, 2.0, 0.08)
    x0 = dev(g.reshape(-1))
    ref = solvers.cg(O, g.reshape(-1).astype(np.float64), 400, shift=1e-2, tol=1e-5)
    xc, info_c, _ = bf().cg_filter(G, x0, 400, shift=1e-2, tol=1e-5)
    for _ in range(2):
        x, info = bf().cg_filter_noalloc(G, x0, 400, shift=1e-2, tol=1e-5)
        assert info.status == info_c.status == ref["status"] == "converged"
        assert info.iters == info_c.iters
        assert abs(info.iters - ref["iters"]) <= 1
        assert torch.equal(x, xc)
        assert rel_l2(host(x), ref["x"]) <= TOL_F32


def test_noalloc_cg_rejects_oversized_problems():
    g = np.random.default_rng(0).uniform(size=(513, 512)).astype(np.float32)
    G = bf().bf_weights(dev(g), 1, 1.0, 0.1)
    with pytest.raises(bf().BFError) as e:
        bf().cg_filter_noalloc(G, dev(g.reshape(-1)), 5)
    assert e.value.code == bf().BF_EINVAL
