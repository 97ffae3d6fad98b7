"""GPU parity of the CG filter (Algorithm 2, Section 5) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import solvers, spectral
from oracle.graph import Graph
from paper_1509_02468_gb300 import synth
from tests.gpu_helpers import bf, dev, host, image_case, make_pair, rel_l2, signal_case

pytestmark = pytest.mark.gpu


def test_cg_signal_1d_n4096_fp64():
    """1D piecewise-constant signal, n = 4096, window radius 5, sigma_s 3, sigma_r 0.1, FP64,
    20 iterations."""
    w = synth.SIGNAL_1D_4096
    _, g = synth.make_input(w)
    G, O = make_pair(g, w.radius, w.sigma_s, w.sigma_r, dtype=torch.float64)
    x, info, h = bf().cg_filter(G, dev(g, torch.float64), w.cg_iters, hist=True)
    ref = solvers.cg(O, g, w.cg_iters)
    assert info.iters == ref["iters"] == 20
    assert rel_l2(host(x), ref["x"]) < 1e-10
    hh = host(h).reshape(-1, 2)
    np.testing.assert_allclose(hh[:, 0], ref["alpha"], rtol=1e-9)
    np.testing.assert_allclose(hh[1:, 1], ref["beta"][1:], rtol=1e-8)


@pytest.mark.parametrize("mode", ["onthefly", "stored_f32"])
def test_cg_image_512_fp32(mode):
    """512 x 512 image, 7 x 7 window, sigma_s 2, sigma_r 0.08, 50 iterations, FP32 vectors:
    relative L2 error <= 1e-5 against the FP64 oracle."""
    w = synth.IMAGE_512
    _, g = synth.make_input(w)
    G, O = make_pair(g, w.radius, w.sigma_s, w.sigma_r, mode=mode)
    x, info, _ = bf().cg_filter(G, dev(g), w.cg_iters)
    ref = solvers.cg(O, g.reshape(-1).astype(np.float64), w.cg_iters)
    assert info.iters == 50
    err = rel_l2(host(x), ref["x"])
    assert err < 1e-5, err


def test_cg_bf16_weights_match_rounded_operator():
    _, g = image_case(96, 80, 7)
    G, O = make_pair(g, 3, 2.0, 0.08, mode="stored_bf16")
    x, _, _ = bf().cg_filter(G, dev(g), 30)
    ref = solvers.cg(O, g.reshape(-1).astype(np.float64), 30)
    assert rel_l2(host(x), ref["x"]) < 1e-5


@pytest.mark.parametrize("precond,beta", [("jacobi", "printed"), ("identity", "flexible"),
                                          ("identity", "printed")])
def test_cg_variants(precond, beta):
    _, g = image_case(64, 75, 8)
    G, O = make_pair(g, 2, 2.0, 0.1)
    x, info, _ = bf().cg_filter(G, dev(g), 15, precond=precond, beta=beta)
    ref = solvers.cg(O, g.reshape(-1).astype(np.float64), 15, precond=precond,
                     beta="sr" if beta == "flexible" else "ss")
    assert rel_l2(host(x), ref["x"]) < 1e-5


def test_cg_shifted_system_to_tolerance():
    """(L + sigma I) x = sigma x0 to ||r|| <= 1e-5 ||b||; iterations equal the oracle's."""
    _, g = image_case(128, 128, 9)
    G, O = make_pair(g, 3, 2.0, 0.08)
    x, info, _ = bf().cg_filter(G, dev(g), 500, shift=1e-2, tol=1e-5)
    ref = solvers.cg(O, g.reshape(-1).astype(np.float64), 500, shift=1e-2, tol=1e-5)
    assert info.status == "converged"
    assert abs(info.iters - ref["iters"]) <= 1
    assert info.rnorm <= 1e-5 * info.ref * 1.0001
    assert rel_l2(host(x), ref["x"]) < 1e-5


def test_cg_polynomial_form_on_gpu():
    """Section 5: the GPU's x_k equals chi_k(D^-1 L) x0 with chi_k built from the GPU's own
    alpha/beta, evaluated spectrally in FP64 (small image)."""
    _, g = image_case(14, 15, 11, dtype=np.float64)
    G, O = make_pair(g, 1, 1.0, 0.1, dtype=torch.float64)
    x, _, h = bf().cg_filter(G, dev(g, torch.float64), 8, hist=True)
    hh = host(h).reshape(-1, 2)
    ref, _ = spectral.spectral_filter(O, g.reshape(-1), lambda mu: spectral.cg_polynomial(hh[:, 0], hh[:, 1], mu))
    assert rel_l2(host(x), ref) < 1e-10


def test_cg_null_start_and_zero_iterations():
    _, g = image_case(20, 20, 12)
    G, _ = make_pair(g, 1, 1.0, 0.1)
    z = torch.zeros(g.size, device="cuda")
    x, info, _ = bf().cg_filter(G, z, 10)
    assert info.iters == 0 and info.status == "converged"
    assert torch.count_nonzero(x).item() == 0
    c = torch.full((g.size,), 0.25, device="cuda")
    x, info, _ = bf().cg_filter(G, c, 10)
    assert torch.all(x == 0.25)      # L e = 0 exactly in the difference form
    x, info, _ = bf().cg_filter(G, dev(g), 0)
    assert torch.equal(x, dev(g))


def test_cg_in_place_and_1d_ragged():
    _, g = signal_case(1777, 3, dtype=np.float32)
    G, O = make_pair(g, 5, 3.0, 0.1)
    x = dev(g)
    bf().cg_filter(G, x, 20, out=x)
    ref = solvers.cg(O, g.astype(np.float64), 20)
    assert rel_l2(host(x), ref["x"]) < 1e-5


def test_cg_fixed_count_captured_in_a_cuda_graph():
    """A fixed-count cg_filter (tol = 0, no info) only enqueues kernels -- its scalar state
    is set by a kernel -- so it can be captured once and replayed: every replay gives the
    uncaptured result exactly."""
    _, g = image_case(120, 136, 31)
    G, O = make_pair(g, 3, 2.0, 0.08)
    x0 = dev(g.reshape(-1))
    ref, _, _ = bf().cg_filter(G, x0, 20)            # uncaptured; sizes the workspace
    out = torch.empty_like(x0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        bf().cg_filter(G, x0, 20, out=out, sync=False)
    for _ in range(2):
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    assert rel_l2(host(out), solvers.cg(O, g.reshape(-1).astype(np.float64), 20)["x"]) < 1e-5


@pytest.mark.parametrize("mode", ["stored_f32", "stored_bf16"])
@pytest.mark.parametrize("shape", [(131, 160), (96, 123)])
def test_cg_stored_weights(mode, shape):
    """Stored weights through the strip kernels, an even and an odd width: the result equals
    the oracle of the stored operator."""
    _, g = image_case(*shape, 33)
    G, O = make_pair(g, 3, 2.0, 0.08, mode=mode)
    x, info, h = bf().cg_filter(G, dev(g), 25, hist=True)
    ref = solvers.cg(O, g.reshape(-1).astype(np.float64), 25)
    assert info.iters == 25
    assert rel_l2(host(x), ref["x"]) < 1e-5
    np.testing.assert_allclose(host(h).reshape(-1, 2)[:, 0], ref["alpha"], rtol=1e-5)
