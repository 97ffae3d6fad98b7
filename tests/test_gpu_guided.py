"""GPU parity of the guided filter's graph (Section 3: Algorithm 1, Eqs. 5-6) and of CG
(Algorithm 2) and LOBPCG (Algorithm 3) on it, against the FP64 oracle, through the C-ABI.
FP32 outputs are held to 1e-5 relative L2 (the difference form keeps L x accurate on
smooth vectors), FP64 ones to rounding level."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import guided, solvers
from paper_1509_02468_gb300 import synth
from tests.gpu_helpers import (TOL_RITZ_SMALL_F32, bf, dev, host, image_case, rel_l2, signal_case,
                               tol_for)

pytestmark = pytest.mark.gpu

EPS = 1e-2


def _case(kind):
    if kind == "1d":
        _, g = signal_case(700, 21)
        return g, 2
    if kind == "1d_r5":                          # radius at run time (1D)
        _, g = signal_case(900, 25)
        return g, 5
    if kind == "2d_r5":                          # radius at run time (2D)
        _, g = image_case(41, 70, 26)
        return g, 5
    if kind == "2d_r1":
        _, g = image_case(20, 33, 22)
        return g, 1
    _, g = image_case(45, 77, 23)
    return g, 2 if kind == "2d" else 3


def _pair(g, r, dtype, eps=EPS):
    gd = dev(g, dtype)
    G = bf().guided_graph(gd, r, eps)
    shape = (1, g.size) if g.ndim == 1 else g.shape
    O = guided.GuidedGraph(host(gd), shape, r, eps)
    return G, O, shape


def _oracle_op(O, op, X):
    if op == "W":
        return O.W @ X
    if op == "L":
        return O.L @ X
    if op == "DINV_W":
        return O.DINV_W @ X
    if op == "D":
        return O.D @ X
    dis = sp.diags(1.0 / np.sqrt(O.d))
    return dis @ (O.L @ (dis @ X))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("kind", ["1d", "1d_r5", "2d_r1", "2d", "2d_r3", "2d_r5"])
@pytest.mark.parametrize("k", [1, 3, 16])
def test_guided_apply(dtype, kind, k):
    """Y = op X for every operator of the guided graph; sizes span several tiles with a
    ragged edge, k not a multiple of the kernel's column pass (3) too."""
    g, r = _case(kind)
    G, O, _ = _pair(g, r, dtype)
    X = np.random.default_rng(k).standard_normal((O.n, k))
    Xd = dev(X, dtype)
    for op in ["W", "L", "DINV_W", "D", "NSYM"]:
        Y = host(bf().bf_apply(G, op, Xd))
        ref = _oracle_op(O, op, host(Xd).reshape(O.n, k))
        assert rel_l2(Y, ref) < tol_for(dtype), (op, rel_l2(Y, ref))


def test_guided_apply_smooth_vector_and_dots():
    """L on a smooth vector (L x << D x): the difference form keeps FP32 relative accuracy;
    the fused column dots x^T y."""
    g, r = _case("2d")
    G, O, shape = _pair(g, r, torch.float32)
    yy, xx = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    x = (1.0 + 0.001 * xx + 0.0005 * yy).reshape(-1, 1)
    y, dots = bf().bf_apply(G, "L", dev(x), dots=True)
    ref = O.L @ host(dev(x))
    assert rel_l2(host(y), ref) < 1e-5                          # measured 1.6e-7
    np.testing.assert_allclose(host(dots), [float(host(dev(x)).reshape(-1) @ ref.reshape(-1))], rtol=1e-5)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_guided_is_algorithm1_and_degree(dtype):
    """D^-1 W x equals Algorithm 1 (with another guide and self-guided); the degree is the
    window count."""
    g, r = _case("2d")
    G, O, shape = _pair(g, r, dtype)
    x = np.random.default_rng(7).uniform(0, 1, O.n)
    y = host(bf().bf_apply(G, "DINV_W", dev(x, dtype)))
    assert rel_l2(y, guided.guided_filter(host(dev(x, dtype)), O.guide, shape, r, EPS)) < tol_for(dtype)
    ys = host(bf().bf_apply(G, "DINV_W", dev(g.reshape(-1), dtype)))
    assert rel_l2(ys, guided.guided_filter(O.guide, O.guide, shape, r, EPS)) < tol_for(dtype)
    np.testing.assert_allclose(host(bf().graph_degree(G)), guided.window_count(shape, r))


@pytest.mark.parametrize("iters", [1, 5])
def test_guided_linear_and_nonlinear_iterations(iters):
    """Section 3's two ways of iterating the guided filter: fixed guide (bf_simple_filter)
    and re-guided by each result (bf_reguided_filter)."""
    g, r = _case("2d")
    G, O, shape = _pair(g, r, torch.float32)
    x = dev(g.reshape(-1))
    y = bf().bf_simple_filter(G, x, iters)
    assert rel_l2(host(y), solvers.simple_iteration(O, host(x), iters)) < 1e-5
    z = bf().reguided_filter(G, x, iters)
    ref = host(x).astype(np.float64)
    for _ in range(iters):
        ref = guided.guided_filter(ref, ref, shape, r, EPS)
    assert rel_l2(host(z), ref) < 1e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shift", [0.0, 0.05])
def test_guided_cg(dtype, shift):
    """Algorithm 2 on L = D - Wt (Jacobi T = D^-1), plain and shifted."""
    g, r = _case("2d")
    G, O, _ = _pair(g, r, dtype)
    x0 = dev(g.reshape(-1), dtype)
    x, info, _ = bf().cg_filter(G, x0, 20, shift=shift)
    ref = solvers.cg(O, host(x0), 20, shift=shift)
    assert rel_l2(host(x), ref["x"]) < (1e-10 if dtype == torch.float64 else 1e-5)
    assert info.iters == 20


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_guided_lobpcg(dtype):
    """Algorithm 3 for the pencil (L, D) of the guided graph: Ritz values and y."""
    _, g = image_case(30, 41, 24)
    G, O, _ = _pair(g, 2, dtype)
    X0 = synth.block_start(g.reshape(-1), 4, seed=1, dtype=np.float64)
    X0d = dev(X0, dtype)
    out = bf().lobpcg_filter(G, X0d, 10)
    ref = solvers.lobpcg(O, host(X0d), 10)
    th, rt = host(out["theta"]), np.asarray(ref["theta"])
    err = np.max(np.abs(th - rt) / np.maximum(np.abs(rt), 1e-3 * np.abs(rt).max()))
    assert err < (1e-9 if dtype == torch.float64 else TOL_RITZ_SMALL_F32), err
    assert rel_l2(host(out["y"]), ref["y"]) < (1e-9 if dtype == torch.float64 else 1e-5)   # FP32: 3.9e-7


def test_guided_graph_rejects_and_reports():
    g, r = _case("2d_r1")
    G, _, _ = _pair(g, r, torch.float32)
    with pytest.raises(bf().BFError) as e:
        bf().graph_export_weights(G)
    assert e.value.code == bf().BF_EINVAL
    with pytest.raises(bf().BFError) as e:
        bf().bf_apply(G, "NDIAGL", dev(g.reshape(-1)))
    assert e.value.code == bf().BF_EINVAL
    bad = g.copy()
    bad[3, 3] = np.nan
    with pytest.raises(bf().BFError) as e:
        bf().guided_graph(dev(bad), 1, EPS)
    assert e.value.code == bf().BF_ENONFINITE
    with pytest.raises(bf().BFError) as e:
        bf().guided_graph(dev(g), 1, 0.0)
    assert e.value.code == bf().BF_EINVAL
