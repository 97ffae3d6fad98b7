"""Gram products on the tensor cores (tcgen05, BF16 and split-BF16 operands, FP32
accumulation) against FP64 products of the same FP32 blocks, with error bounds from the
operand rounding and the accumulation; and LOBPCG with each Gram precision mode, the
three-way split against the FP64 oracle at the FP32 bar."""
import numpy as np
import pytest
import torch

from tests.gpu_helpers import TOL_RITZ, bf, dev, host, image_case, make_pair

pytestmark = pytest.mark.gpu


def blocks(n, k, nblk, seed):
    rng = np.random.default_rng(seed)
    S = [rng.standard_normal((n, k)).astype(np.float32) * (1.0 + 9.0 * rng.random(k)).astype(np.float32)
         for _ in range(nblk)]
    AS = [rng.standard_normal((n, k)).astype(np.float32) for _ in range(nblk)]
    b = rng.uniform(1.0, 20.0, n).astype(np.float32)
    return S, AS, b


@pytest.mark.parametrize("n,k,nblk", [(5000, 16, 3), (4097, 8, 2), (300, 32, 3), (64, 4, 1), (131, 12, 3)])
@pytest.mark.parametrize("split", [False, True])
def test_tensor_core_gram_within_rounding_bounds(n, k, nblk, split):
    S, AS, b = blocks(n, k, nblk, seed=n + k)
    GA, GB = bf().gram_tc([dev(x) for x in S], [dev(x) for x in AS], dev(b), split=split)
    S64 = np.hstack(S).astype(np.float64)
    AS64 = np.hstack(AS).astype(np.float64)
    BS64 = b.astype(np.float64)[:, None] * S64
    refA, refB = S64.T @ AS64, S64.T @ BS64
    # per-entry scale: |s_i| . |t_j| (Cauchy-Schwarz bound of the product sums' size)
    sA = np.linalg.norm(S64, axis=0)[:, None] * np.linalg.norm(AS64, axis=0)[None, :]
    sB = np.linalg.norm(S64, axis=0)[:, None] * np.linalg.norm(BS64, axis=0)[None, :]
    # BF16 rounding of both factors: |rel| <= 2^-8 each; split: the dropped lo*lo term and
    # the rounding of lo give ~2^-16, FP32 accumulation adds up to ~2^-24 sqrt(n) per entry
    eps = (2.0 ** -16 + 2.0 ** -24 * np.sqrt(n)) if split else 2.0 ** -7
    assert np.max(np.abs(host(GA) - refA) / sA) <= 4 * eps
    assert np.max(np.abs(host(GB) - refB) / sB) <= 4 * eps


@pytest.mark.parametrize("n,k,nblk", [(64, 4, 1), (4097, 8, 2), (131, 12, 3), (5000, 16, 3), (70001, 16, 3)])
def test_three_way_split_gram_at_fp32_level(n, k, nblk):
    """BF_GRAM_BF16X6: x = hi + mid + lo carries all 24 bits of an FP32 value; the dropped
    products are below 2^-24 relative; every two chunks of 64 pixels are accumulated in
    FP32 in tensor memory by at most 40 MMA results (8 for hi*hi), then folded into
    double-float sums.  Bound: 32 * 2^-24 of the Cauchy-Schwarz scale |s_i| |t_j| per entry.  Widths
    in increasing order: each needs more shared memory than the one before."""
    S, AS, b = blocks(n, k, nblk, seed=n + 3 * k)
    GA, GB = bf().gram_tc([dev(x) for x in S], [dev(x) for x in AS], dev(b), mode="bf16x6")
    S64 = np.hstack(S).astype(np.float64)
    AS64 = np.hstack(AS).astype(np.float64)
    BS64 = b.astype(np.float64)[:, None] * S64
    refA, refB = S64.T @ AS64, S64.T @ BS64
    sA = np.linalg.norm(S64, axis=0)[:, None] * np.linalg.norm(AS64, axis=0)[None, :]
    sB = np.linalg.norm(S64, axis=0)[:, None] * np.linalg.norm(BS64, axis=0)[None, :]
    eps = 32 * 2.0 ** -24
    assert np.max(np.abs(host(GA) - refA) / sA) <= eps
    assert np.max(np.abs(host(GB) - refB) / sB) <= eps


def test_three_way_split_needs_narrow_bases():
    S, AS, b = blocks(300, 32, 3, seed=5)
    with pytest.raises(bf().BFError):
        bf().gram_tc([dev(x) for x in S], [dev(x) for x in AS], dev(b), mode="bf16x6")


def test_lobpcg_512_k16_three_way_split_gram_meets_fp32_bar():
    """The benchmark's LOBPCG (512 x 512 image, k = 16, 30 iterations) with its Gram
    products on the tensor cores in the three-way split: Ritz values within 1e-6 (reading
    A8) and the filtered signal within 1e-5 of the FP64 oracle."""
    from oracle import solvers
    from paper_1509_02468_gb300 import synth
    from tests.gpu_helpers import TOL_F32, rel_l2
    w = synth.IMAGE_512
    _, g = synth.make_input(w)
    G, O = make_pair(g, w.radius, w.sigma_s, w.sigma_r)
    X0 = dev(synth.block_start(g.reshape(-1), w.lobpcg_k, seed=w.seed))
    out = bf().lobpcg_filter(G, X0, w.lobpcg_iters, gram="bf16x6")
    ref = solvers.lobpcg(O, host(X0), w.lobpcg_iters)
    th, th_ref = host(out["theta"]), ref["theta"]
    err = np.max(np.abs(th - th_ref) / np.maximum(np.abs(th_ref), 1e-3 * np.abs(th_ref).max()))
    assert out["info"].iters == 30
    assert err <= TOL_RITZ, err
    assert rel_l2(host(out["y"]), ref["y"]) <= TOL_F32


@pytest.mark.parametrize("gram", ["bf16x3", "bf16"])
def test_lobpcg_with_tensor_core_gram(gram):
    from paper_1509_02468_gb300 import synth
    _, noisy = image_case(96, 112, 21)
    G, O = make_pair(noisy, 3, 2.0, 0.08)
    X0 = dev(synth.block_start(noisy.ravel(), 16, 21))
    ref = bf().lobpcg_filter(G, X0, 12)
    out = bf().lobpcg_filter(G, X0, 12, gram=gram)
    th_ref, th = host(ref["theta"]), host(out["theta"])
    err = np.max(np.abs(th - th_ref) / np.maximum(np.abs(th_ref), 1e-3 * np.abs(th_ref).max()))
    # split-BF16 reproduces the FP32 Gram's run to the FP32 tolerance; plain BF16 converges
    # to a nearby trajectory (its Gram carries ~4e-3 relative errors)
    assert err <= (10 * TOL_RITZ if gram == "bf16x3" else 0.2), err
    assert out["info"].status in ("ran", "converged")


def test_bounded_wait_gives_up_and_the_context_survives():
    """The bounded mbarrier wait of the tensor-core kernels: with nothing arriving it gives
    up after its poll limit and the call reports BF_ETIMEOUT; the context still runs work."""
    bf().wait_test(64, arrive=True)
    with pytest.raises(bf().BFError) as ei:
        bf().wait_test(256, arrive=False)
    assert ei.value.code == -5                      # BF_ETIMEOUT
    _, g = image_case(40, 45, 3)
    G, O = make_pair(g, 3, 2.0, 0.08)
    X = np.random.default_rng(1).standard_normal((g.size, 4))
    Xd = dev(X)
    Y = host(bf().bf_apply(G, "L", Xd))
    assert np.linalg.norm(Y - O.apply("L", host(Xd))) <= 1e-5 * np.linalg.norm(O.apply("L", host(Xd)))
    bf().wait_test(64, arrive=True)
