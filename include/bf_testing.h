/*
 * bf_testing.h -- extra entry points of libbf.so that expose internal steps of
 * lobpcg_filter and its bounded device waits for direct testing (see bf.h for the
 * conventions).
 */
#ifndef BF_TESTING_H_
#define BF_TESTING_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The Rayleigh-Ritz step of LOBPCG (Algorithm 3, Section 6: "use the Rayleigh-Ritz method
 * for the pencil L - lambda D on the trial subspace"), on the GPU in FP64, one CTA.
 * G (device, 2*m*m doubles): G_A = S^T L S then G_B = S^T B S, row-major, symmetric up
 * to rounding, G_B positive definite.  Finds the k smallest eigenpairs of
 * G_A c = theta G_B c:  C (device, m*k doubles, row-major [m][k]) with C^T G_B C = I,
 * theta (device, k doubles, ascending).  If a squared pivot of the Cholesky factor of the
 * unit-diagonal-scaled G_B is <= 1e-10 and 0 < m_nop < m, the problem is solved again on
 * the leading m_nop x m_nop blocks (rows m_nop.. of C are then 0).  Cp (device, m*k
 * doubles, may be NULL) receives the coefficients of the next search direction P: the
 * rows of C past the first k, minus C times C^T G_B (those rows), i.e. B-orthogonal to
 * the Ritz vectors.  flags (device, 2 ints) must hold {0, 0}; on return flags[0] is 2
 * for a dependent basis that dropping P does not cure, 3 for a non-finite Ritz value,
 * and flags[1] counts drops of P.  Needs 1 <= k <= m <= 96 and k <= 32.  Asynchronous. */
int bf_rayleigh_ritz(const double* G, int m, int k, int m_nop, double* C, double* Cp,
                     double* theta, int* flags, void* stream);

/* The tensor-core Gram products of the LOBPCG Rayleigh-Ritz step (Algorithm 3): with
 * S = [S0 S1 S2] and AS = [AS0 AS1 AS2] (the first nblk blocks, each n x k pixel-major
 * float) and B = diag(b) (b NULL: I), writes G[0] = S^T AS and G[1] = S^T B S (double,
 * [2][m][m], m = nblk k) computed by tcgen05 MMAs in mode BF_GRAM_BF16 (BF16 operands),
 * BF_GRAM_BF16X3 (hi + lo, hi*hi + hi*lo + lo*hi) or BF_GRAM_BF16X6 (hi + mid + lo, six
 * products, per-chunk folding into double-float sums; m <= 48), FP32 accumulation in
 * tensor memory.  Needs k % 4 == 0 and m <= 96.  Allocates scratch and synchronises the
 * stream. */
int bf_gram_tc_test(const float* S0, const float* S1, const float* S2, const float* AS0,
                    const float* AS1, const float* AS2, const float* b, int nblk, int k,
                    int64_t n, int mode, double* G, void* stream);

/* The bounded device wait used by the tensor-core Gram (an mbarrier wait that gives up
 * after a number of polls, so that a kernel whose producer never signals returns an error
 * instead of hanging), on a barrier of its own: one CTA of 32 threads waits for phase 0
 * of an mbarrier with arrival count 1, polling at most iters times (1 <= iters <= 2^20).
 * arrive != 0: thread 0 arrives first and the call returns BF_OK; arrive == 0: nothing
 * arrives, every wait gives up and the call returns BF_ETIMEOUT, with the CUDA context
 * intact.  Synchronises the stream. */
int bf_wait_test(int iters, int arrive, void* stream);

/* bf_batch_cg_persistent (Jacobi, flexible beta, no shift) with CTA 0 leaving before its
 * first grid barrier, so that every other CTA's bounded wait runs out: returns
 * BF_ETIMEOUT and leaves the context usable.  Needs the batch type from bf.h. */
struct bf_batch;
int bf_batch_barrier_test(struct bf_batch* b, const float* const* x0, float* const* x_out, int kmax,
                          void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BF_TESTING_H_ */
