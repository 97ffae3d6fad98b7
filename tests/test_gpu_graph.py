"""GPU parity of the graph (Eq. 2 weights, degree) and the matrix-free operator (Eqs. 1-4,
Section 4) against the FP64 oracle, through the C-ABI."""
import numpy as np
import pytest
import torch

from oracle import solvers
from oracle.graph import Graph
from tests.gpu_helpers import (TOL_F32, bf, dev, host, image_case, make_pair, rel_l2, signal_case,
                               tol_for)

pytestmark = pytest.mark.gpu

OPS = ["W", "L", "DINV_W", "D", "NSYM", "NDIAGL"]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("mode", ["onthefly", "stored_f32"])
@pytest.mark.parametrize("case", ["1d", "2d", "2d_cross"])
def test_degree_and_weights(dtype, mode, case):
    """Eq. 2 weights exported per tap and the degree d_i = sum_j w_ij against the oracle
    (stored FP32 weights: Eq. 2 rounded to float)."""
    if case == "1d":
        _, g = signal_case(1000, 1)
        r, ss, sr, win = 5, 3.0, 0.1, "square"
    else:
        _, g = image_case(45, 77, 2)
        r, ss, sr, win = (3, 2.0, 0.08, "square") if case == "2d" else (1, 2.0, 0.08, "cross")
    G = bf().bf_weights(dev(g, dtype), r, ss, sr, window=win, weight_mode=mode)
    shape = (1, g.size) if g.ndim == 1 else g.shape
    O = Graph(host(dev(g, dtype)), shape, r, ss, sr, window=win)
    exact = dtype == torch.float64 and mode == "onthefly"
    tol = 1e-12 if exact else 2e-6
    assert rel_l2(host(bf().graph_degree(G)), O.d) < tol
    taps = host(bf().graph_export_weights(G))
    assert taps.shape == O.taps.shape
    if exact:
        np.testing.assert_allclose(taps, O.taps, rtol=1e-12, atol=1e-300)
    else:
        # float path: w = exp2(a) with the argument a rounded to float (the squared
        # difference and the coefficient each carry a rounding), so the relative error
        # grows like a few 2^-24 |a| (times ln 2), plus 2 ulp of exp2; weights far below
        # the largest ones are compared absolutely.
        arg = np.abs(np.log2(np.maximum(O.taps, 1e-300)))
        bound = (4.0 + 4.0 * arg) * 2.0 ** -24
        ok = (np.abs(taps - O.taps) <= bound * O.taps) | (np.abs(taps - O.taps) <= 1e-12)
        assert ok.all(), np.argwhere(~ok)[:5]


def test_bf16_weights_are_rounded_oracle_weights():
    """Stored BF16 weights: each equals the FP64 weight to BF16 rounding (2^-8 relative)."""
    _, g = image_case(40, 50, 3)
    G = bf().bf_weights(dev(g), 3, 2.0, 0.08, weight_mode="stored_bf16")
    O = Graph(g.astype(np.float64), g.shape, 3, 2.0, 0.08)
    taps = host(bf().graph_export_weights(G))
    np.testing.assert_allclose(taps, O.taps, rtol=2 ** -8, atol=1e-30)
    # and the degree is the exact sum of the stored weights
    Ob = Graph.from_taps(taps, g.shape, 3)
    assert rel_l2(host(bf().graph_degree(G)), Ob.d) < 1e-6


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("mode", ["onthefly", "stored_f32", "stored_bf16"])
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("k", [1, 3, 4, 16])
def test_apply_2d(dtype, mode, op, k):
    if mode == "stored_bf16" and dtype == torch.float64:
        pytest.skip("bf16 weights need the float path")
    _, g = image_case(45, 70, 4)       # ragged against 32 x 8 tiles
    G, O = make_pair(g, 3, 2.0, 0.08, mode=mode, dtype=dtype)
    X = np.random.default_rng(k).standard_normal((g.size, k))
    if k > 1:
        X[:, 0] = g.reshape(-1)          # a smooth column too
    Xd = dev(X, dtype)
    Y = host(bf().bf_apply(G, op, Xd))
    ref = O.apply(op, host(Xd))
    assert rel_l2(Y, ref) < tol_for(dtype), (op, k, rel_l2(Y, ref))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("k", [1, 2, 4, 32])
def test_apply_1d(dtype, op, k):
    _, g = signal_case(1531, 5)         # ragged against 256-sample tiles
    G, O = make_pair(g, 5, 3.0, 0.1, dtype=dtype)
    X = np.random.default_rng(k).standard_normal((g.size, k))
    Xd = dev(X, dtype)
    Y = host(bf().bf_apply(G, op, Xd))
    assert rel_l2(Y, O.apply(op, host(Xd))) < tol_for(dtype)


@pytest.mark.parametrize("shape,radius", [((1, 1), 1), ((1, 9), 3), ((9, 1), 3), ((3, 3), 7),
                                          ((2, 300), 2), ((33, 9), 1)])
def test_apply_small_and_degenerate_images(shape, radius):
    """Images smaller than a tile, one pixel wide or tall, radius beyond the image."""
    g = np.random.default_rng(7).uniform(size=shape).astype(np.float32)
    G, O = make_pair(g, radius, 1.5, 0.2)
    X = np.random.default_rng(8).standard_normal((g.size, 4))
    Xd = dev(X)
    for op in OPS:
        Y = host(bf().bf_apply(G, op, Xd))
        ref = O.apply(op, host(Xd))
        if np.linalg.norm(ref) == 0:
            assert np.abs(Y).max() < 1e-6
        else:
            assert rel_l2(Y, ref) < 1e-5, op


def test_apply_strided_block_and_dots():
    """ld > k (a column slice of a wider block) and the fused column dot products."""
    _, g = image_case(37, 41, 6)
    G, O = make_pair(g, 2, 2.0, 0.1)
    big = dev(np.random.default_rng(9).standard_normal((g.size, 12)))
    Xv = big[:, 2:9]                     # k = 7, ld = 12, offset 2
    Y, d = bf().bf_apply(G, "L", Xv, dots=True)
    Xh = host(Xv)
    ref = O.apply("L", Xh)
    assert rel_l2(host(Y), ref) < 1e-5
    np.testing.assert_allclose(host(d), np.sum(Xh * ref, axis=0), rtol=1e-5)


def test_apply_rejects_bad_arguments():
    _, g = image_case(16, 16, 1)
    G, _ = make_pair(g, 1, 1.0, 0.1)
    X = dev(np.ones((g.size, 2)))
    with pytest.raises(bf().BFError) as e:
        bf().bf_apply(G, "L", X, Y=X)    # in place
    assert e.value.code == bf().BF_EINVAL


def test_nonfinite_guide_is_reported():
    g = np.ones((8, 8), np.float32)
    g[3, 4] = np.nan
    with pytest.raises(bf().BFError) as e:
        bf().bf_weights(dev(g), 1, 1.0, 0.1)
    assert e.value.code == bf().BF_ENONFINITE


@pytest.mark.parametrize("iters", [0, 1, 2, 7])
def test_simple_filter(iters):
    """x <- D^-1 W x repeated (Section 4); also in place."""
    _, g = image_case(30, 47, 10)
    G, O = make_pair(g, 3, 2.0, 0.08)
    x = dev(g.reshape(-1))
    y = bf().bf_simple_filter(G, x, iters)
    ref = solvers.simple_iteration(O, host(x), iters)
    assert rel_l2(host(y), ref) < 1e-5
    xin = x.clone()
    bf().bf_simple_filter(G, xin, iters, out=xin)
    assert rel_l2(host(xin), ref) < 1e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("case", ["1d", "2d"])
@pytest.mark.parametrize("iters", [0, 1, 3])
def test_reguided_filter(dtype, case, iters):
    """The nonlinear iteration of Section 2 (weights rebuilt from each iterate) against the
    oracle; in place too.  FP32: each re-guide moves the weights by about
    2 |g_i - g_j| / sigma_r^2 times the iterate's rounding (a few 1e-6 relative here), so
    three steps stay inside the FP32 bar."""
    if case == "1d":
        _, g = signal_case(1500, 4)
        r, ss, sr = 5, 3.0, 0.1
        shape = (1, g.size)
    else:
        _, g = image_case(37, 52, 11)
        r, ss, sr = 3, 2.0, 0.08
        shape = g.shape
    x = dev(g.reshape(-1) if case == "1d" else g, dtype)
    G = bf().bf_weights(x, r, ss, sr)
    xv = x.reshape(-1)
    y = bf().reguided_filter(G, xv, iters)
    ref = solvers.reguided_iteration(host(xv), shape, r, ss, sr, iters)
    assert rel_l2(host(y), ref) < tol_for(dtype)
    xin = xv.clone()
    bf().reguided_filter(G, xin, iters, out=xin)
    assert rel_l2(host(xin), ref) < tol_for(dtype)
    if iters >= 1:
        # g is left holding the graph of the last guide x_{iters-1}
        prev = solvers.reguided_iteration(host(xv), shape, r, ss, sr, iters - 1)
        O = Graph(prev, shape, r, ss, sr)
        assert rel_l2(host(bf().graph_degree(G)), O.d) < (1e-12 if dtype == torch.float64 else 1e-5)


@pytest.mark.parametrize("mode", ["stored_f32", "stored_bf16"])
def test_reguided_filter_stored_weights(mode):
    """With stored weights every step rebuilds them from the iterate (the graph of the last
    guide is left behind).  BF16 storage rounds each weight to 2^-9 relative, which moves a
    weighted average by at most that times the spread of the averaged values: against the
    exact oracle it is held to the bound the precision study uses for BF16 weights, 2^-6."""
    _, g = image_case(29, 40, 12)
    x = dev(g)
    G = bf().bf_weights(x, 3, 2.0, 0.08, weight_mode=mode)
    xv = x.reshape(-1)
    y = bf().reguided_filter(G, xv, 3)
    ref = solvers.reguided_iteration(host(xv), g.shape, 3, 2.0, 0.08, 3)
    assert rel_l2(host(y), ref) < (1e-5 if mode == "stored_f32" else 2.0 ** -6)


def test_reguided_filter_reports_nonfinite():
    _, g = image_case(16, 16, 3)
    x = dev(g)
    G = bf().bf_weights(x, 1, 1.0, 0.1)
    bad = x.reshape(-1).clone()
    bad[40] = float("inf")
    with pytest.raises(bf().BFError) as e:
        bf().reguided_filter(G, bad, 2)
    assert e.value.code == bf().BF_ENONFINITE


def test_full_size_image_apply_sampled():
    """The 512 x 512, 7 x 7 window operator at k = 16 (the block width LOBPCG uses on this
    image), checked on sampled rows computed one by one from the oracle's definition."""
    _, g = image_case(512, 512, 2)
    G = bf().bf_weights(dev(g), 3, 2.0, 0.08)
    X = np.random.default_rng(0).standard_normal((g.size, 16)).astype(np.float32)
    Y = host(bf().bf_apply(G, "L", dev(X)))
    rng = np.random.default_rng(1)
    rows = np.concatenate([rng.integers(0, g.size, 200), [0, 511, g.size - 1, g.size - 512]])
    gg = g.astype(np.float64)
    for i in rows:
        y, x = divmod(int(i), 512)
        acc = np.zeros(16)
        for dy in range(-3, 4):
            for dx in range(-3, 4):
                yy, xx = y + dy, x + dx
                if (dy or dx) and 0 <= yy < 512 and 0 <= xx < 512:
                    w = np.exp(-(dx * dx + dy * dy) / 8.0) * np.exp(-(gg[y, x] - gg[yy, xx]) ** 2 / (2 * 0.08 ** 2))
                    acc += w * (X[i].astype(np.float64) - X[yy * 512 + xx].astype(np.float64))
        assert rel_l2(Y[i], acc) < 1e-5


def _l_rows_from_definition(g, X, rows, radius, sigma_s, sigma_r):
    """(L X)[i] for the sampled pixels i: Eq. 2 weights over the square window, difference
    form sum_j w_ij (x_i - x_j), FP64."""
    ny, nx = g.shape
    gg = g.astype(np.float64)
    out = np.zeros((len(rows), X.shape[1]))
    for r, i in enumerate(rows):
        y, x = divmod(int(i), nx)
        for dy in range(-radius, radius + 1):
            for dx in range(-radius, radius + 1):
                yy, xx = y + dy, x + dx
                if (dy or dx) and 0 <= yy < ny and 0 <= xx < nx:
                    w = np.exp(-(dx * dx + dy * dy) / (2 * sigma_s ** 2)) * \
                        np.exp(-(gg[y, x] - gg[yy, xx]) ** 2 / (2 * sigma_r ** 2))
                    out[r] += w * (X[i].astype(np.float64) - X[yy * nx + xx].astype(np.float64))
    return out


@pytest.mark.parametrize("k,shape", [(4, (1100, 700)), (8, (1100, 700)), (16, (400, 450)),
                                     (32, (400, 450)), (48, (300, 333))])
def test_apply_l_block_widths_sampled(k, shape):
    """The 7 x 7 L operator with weights on the fly at each register-blocked block width, on
    images with more tiles than the GPU has SMs (several tiles per CTA, both halo buffers
    in use) and ragged right and bottom edges; sampled rows against the definition."""
    _, g = image_case(shape[0], shape[1], 11)
    G = bf().bf_weights(dev(g), 3, 2.0, 0.08)
    X = np.random.default_rng(k).standard_normal((g.size, k)).astype(np.float32)
    X[:, 0] = g.reshape(-1)
    Y = host(bf().bf_apply(G, "L", dev(X)))
    assert np.all(np.isfinite(Y))
    ny, nx = shape
    rng = np.random.default_rng(2)
    edge = [0, nx - 1, (ny - 1) * nx, g.size - 1, 31, 32, 33 * nx + 63, (ny - 2) * nx + nx // 2,
            (ny // 2) * nx + nx - 2, 15 * nx + 16, 16 * nx + 17, 63 * nx + 5, 64 * nx + 5]
    rows = np.concatenate([rng.integers(0, g.size, 150), edge])
    ref = _l_rows_from_definition(g, X, rows, 3, 2.0, 0.08)
    for r, i in enumerate(rows):
        assert rel_l2(Y[i], ref[r]) < 1e-5, (int(i), rel_l2(Y[i], ref[r]))


def test_apply_l_spatial_only_weights():
    """sigma_r = inf (range term off, pure spatial Gaussian) on the 7 x 7 window."""
    _, g = image_case(45, 70, 4)
    G, O = make_pair(g, 3, 2.0, np.inf)
    X = np.random.default_rng(3).standard_normal((g.size, 16))
    Xd = dev(X)
    Y = host(bf().bf_apply(G, "L", Xd))
    assert rel_l2(Y, O.apply("L", host(Xd))) < 1e-5


@pytest.mark.parametrize("offset", [4, 2])
def test_apply_l_strided_column_slice(offset):
    """A 16-column slice of a 24-column block (leading dimension 24): at offset 4 the slice
    is 16-byte aligned and takes the pipelined kernel, at offset 2 it is not and takes the
    tile-per-CTA one; both against sampled rows of the definition, on an image with more
    tiles than SMs."""
    _, g = image_case(420, 390, 12)
    G = bf().bf_weights(dev(g), 3, 2.0, 0.08)
    big = np.random.default_rng(offset).standard_normal((g.size, 24)).astype(np.float32)
    bigd = dev(big)
    Xv = bigd[:, offset:offset + 16]
    Y = host(bf().bf_apply(G, "L", Xv))
    rows = np.concatenate([np.random.default_rng(5).integers(0, g.size, 120), [0, g.size - 1, 389, 419 * 390]])
    ref = _l_rows_from_definition(g, big[:, offset:offset + 16], rows, 3, 2.0, 0.08)
    for r, i in enumerate(rows):
        assert rel_l2(Y[i], ref[r]) < 1e-5, (int(i), offset)


@pytest.mark.parametrize("mode", ["onthefly", "stored_bf16"])
def test_graph_update_equals_a_new_graph(mode):
    """bf_graph_update recomputes a graph in place for a new guide of the same shape: the
    operators, the degree and both filters give exactly what a newly built graph gives,
    also after the filters' workspaces were created on the old guide."""
    from paper_1509_02468_gb300 import synth
    _, g1 = image_case(45, 70, 4)
    _, g2 = image_case(45, 70, 9)
    G = bf().bf_weights(dev(g1), 3, 2.0, 0.08, weight_mode=mode)
    bf().cg_filter(G, dev(g1.reshape(-1)), 5)
    X0 = dev(synth.block_start(g2.reshape(-1), 4, 9))
    bf().lobpcg_filter(G, X0, 3)
    bf().graph_update(G, dev(g2))
    H = bf().bf_weights(dev(g2), 3, 2.0, 0.08, weight_mode=mode)
    X = dev(np.random.default_rng(2).standard_normal((g2.size, 16)))
    for op in OPS:
        assert torch.equal(bf().bf_apply(G, op, X), bf().bf_apply(H, op, X)), op
    assert torch.equal(bf().graph_degree(G), bf().graph_degree(H))
    xa = bf().cg_filter(G, dev(g2.reshape(-1)), 7)[0]
    xb = bf().cg_filter(H, dev(g2.reshape(-1)), 7)[0]
    assert torch.equal(xa, xb)
    la, lb = bf().lobpcg_filter(G, X0, 4), bf().lobpcg_filter(H, X0, 4)
    assert torch.equal(la["theta"], lb["theta"]) and torch.equal(la["y"], lb["y"])


def test_graph_update_rejects_and_reports():
    _, g = image_case(30, 40, 2)
    G = bf().bf_weights(dev(g), 3, 2.0, 0.08)
    with pytest.raises(ValueError):
        bf().graph_update(G, dev(g[:, :39]))                         # wrong shape
    with pytest.raises(ValueError):
        bf().graph_update(G, dev(g, torch.float64))                  # wrong dtype
    bad = g.copy()
    bad[3, 5] = np.nan
    with pytest.raises(bf().BFError) as ei:
        bf().graph_update(G, dev(bad))
    assert ei.value.code == bf().BF_ENONFINITE
    bf().graph_update(G, dev(g))                                     # a valid guide recovers it
    H = bf().bf_weights(dev(g), 3, 2.0, 0.08)
    assert torch.equal(bf().graph_degree(G), bf().graph_degree(H))


@pytest.mark.parametrize("shape", [(150, 163), (137, 168)])
@pytest.mark.parametrize("mode", ["onthefly", "stored_f32", "stored_bf16"])
@pytest.mark.parametrize("op", ["L", "NSYM", "NDIAGL"])
def test_apply_k1_interior_and_border_tiles(shape, mode, op):
    """One column on an image large enough for unmasked interior tiles (32 x 32 tiles with
    a radius-3 halo) next to ragged border tiles, with the fused dot x^T y; an odd and an
    even width."""
    _, g = image_case(*shape, 41)
    G, O = make_pair(g, 3, 2.0, 0.08, mode=mode)
    x = np.random.default_rng(3).standard_normal(g.size)
    xd = dev(x)
    Y, d = bf().bf_apply(G, op, xd, dots=True)
    ref = O.apply(op, host(xd))
    assert rel_l2(host(Y), ref) < TOL_F32
    assert abs(host(d)[0] - host(xd) @ ref) <= 1e-5 * np.abs(host(xd) * ref).sum()
