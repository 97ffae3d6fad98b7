/*
 * bf.h -- C-ABI of libbf.so: the bilateral-filter graph operator and the Krylov filters
 * built on it, for NVIDIA GB300 (sm_103a).
 *
 * Method: A. Knyazev, A. Malyshev, "Accelerated graph-based spectral polynomial filters",
 * IEEE MLSP 2015.  Section 2 defines the graph (Eqs. 1-4), Section 4 the normalised
 * Laplacian and the simple iteration, Section 5 preconditioned CG for L x = 0
 * (Algorithm 2), Section 6 LOBPCG as a low-pass filter (Algorithm 3).
 *
 * Conventions (all entry points):
 *  - Every array argument is DEVICE memory owned by the caller unless stated otherwise;
 *    the library never frees it.  Element type is the graph's dtype (float for BF_F32,
 *    double for BF_F64), except FP64 scalar outputs, which are always double.
 *  - A signal/image has n = nx * ny samples, row-major (x fastest).  A block of k vectors
 *    is pixel-major: element (i, c) is at X[i * ld + c], ld >= k.  Block pointers must be
 *    16-byte aligned and ld a multiple of 16 / sizeof(element) when k is.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are ordered on
 *    that stream and return before the GPU finishes, except where a host output (an
 *    info struct, a status read) is requested: then the call synchronises the stream.
 *  - Return value: BF_OK (0) or a negative BF_E* code; bf_last_error() gives a message
 *    (thread-local, valid until the next call on that thread).
 *  - A bf_graph owns its device buffers and grow-only workspaces.  cg_filter,
 *    lobpcg_filter and bf_simple_filter each keep their own workspace, so calls of
 *    different families may run at the same time on different streams (they only read
 *    the graph); two calls of the same family on one graph must not overlap.
 */
#ifndef BF_H_
#define BF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define BF_OK             0
#define BF_EINVAL        -1   /* bad argument (sizes, alignment, enum values, NULL)      */
#define BF_ECUDA         -2   /* a CUDA runtime call failed                               */
#define BF_EBREAKDOWN    -3   /* CG: p^T q <= 0;  LOBPCG: dependent basis without P       */
#define BF_ENONFINITE    -4   /* NaN/Inf in the guide or in a solver scalar               */
#define BF_ETIMEOUT      -5   /* a bounded device wait gave up                            */
#define BF_ENOMEM        -6   /* device allocation failed                                 */

/* ---- enums ----------------------------------------------------------------------- */
#define BF_F32            0
#define BF_F64            1

#define BF_WINDOW_SQUARE  0   /* |dx| <= r and |dy| <= r (Section 2's window)             */
#define BF_WINDOW_CROSS   1   /* dx = 0 or dy = 0: the 5-point lattice of Section 7 at r=1 */

#define BF_W_ONTHEFLY     0   /* weights recomputed from the guide inside every apply     */
#define BF_W_STORED_F32   1   /* forward half-window weights stored once, float           */
#define BF_W_STORED_BF16  2   /* forward half-window weights stored once, bfloat16        */

#define BF_OP_W           0   /* Y = W X                                    (Eq. 2)       */
#define BF_OP_L           1   /* Y = (D - W) X                              (Eq. 4)       */
#define BF_OP_DINV_W      2   /* Y = D^-1 W X, one BF step                  (Eqs. 1, 3)   */
#define BF_OP_D           3   /* Y = D X                                    (Section 2)   */
#define BF_OP_NSYM        4   /* Y = D^-1/2 L D^-1/2 X                                    */
#define BF_OP_NDIAGL      5   /* Y = (diag L)^-1/2 L (diag L)^-1/2 X        (Section 4)   */

#define BF_PRECOND_JACOBI   0 /* T = D^-1 (Algorithm 2's preconditioner)                  */
#define BF_PRECOND_IDENTITY 1 /* T = I                                                    */
#define BF_PRECOND_NET      2 /* T = the learned conv net of a bf_net (FP32 graphs)        */
#define BF_PRECOND_SPD      3 /* T = D^-1/2 (I + K^T K) D^-1/2 of a bf_spd (FP32 graphs)    */

#define BF_BETA_FLEXIBLE  0   /* beta = s^T (r - r_old) / (s_old^T r_old)                 */
#define BF_BETA_PRINTED   1   /* beta = s^T (r - r_old) / (s_old^T s_old), as printed     */

#define BF_PENCIL_D       0   /* LOBPCG for L x = lambda D x (Algorithm 3)                */
#define BF_PENCIL_I       1   /* LOBPCG for L x = lambda x                                */

#define BF_GRAM_FP32      0   /* FP32 products in runs of 16 pixels, folded into FP64     */
#define BF_GRAM_BF16      1   /* tensor cores (tcgen05): BF16 operands, FP32 accumulation */
#define BF_GRAM_BF16X3    2   /* tensor cores: x = hi + lo in BF16, hi*hi + hi*lo + lo*hi */
#define BF_GRAM_BF16X6    3   /* tensor cores: x = hi + mid + lo in BF16 (24 bits), six   */
                              /* products, accumulators folded per 64 pixels into         */
                              /* double-float sums; bases of m = 3k <= 48 columns (k <= 16), */
                              /* wider ones use BF_GRAM_FP32                               */

#define BF_CG_CONVERGED   1   /* bf_info.status: stopped by s^T r = 0 or by tol           */
#define BF_CG_BREAKDOWN   2   /* bf_info.status: stopped by p^T q <= 0                    */

/* ---- structs ---------------------------------------------------------------------- */
typedef struct bf_params {
  int32_t ndim;          /* 1: signal (ny must be 1); 2: image                             */
  int32_t radius;        /* window radius r, 1..7 (2D) or 1..32 (1D)                        */
  int64_t nx, ny;        /* samples per row, rows                                           */
  int32_t window;        /* BF_WINDOW_*                                                     */
  int32_t weight_mode;   /* BF_W_*                                                          */
  int32_t dtype;         /* BF_F32 or BF_F64 (BF_W_STORED_BF16 needs BF_F32)                */
  int32_t reserved;      /* must be 0                                                       */
  double  sigma_s;       /* spatial width of Eq. 2 (> 0; +inf: factor 1)                    */
  double  sigma_r;       /* range width of Eq. 2   (> 0; +inf: factor 1)                    */
} bf_params;

/* The guided filter's graph (Section 3): window radius r (width rho = 2r + 1) and the
 * epsilon of Algorithm 1. */
typedef struct bf_guided_params {
  int32_t ndim;          /* 1: signal (ny must be 1); 2: image                             */
  int32_t radius;        /* window radius r, 1..8 (2D) or 1..32 (1D)                        */
  int64_t nx, ny;        /* samples per row, rows                                           */
  int32_t dtype;         /* BF_F32 or BF_F64                                                */
  int32_t reserved;      /* must be 0                                                       */
  double  eps;           /* epsilon of Algorithm 1 (> 0, finite)                            */
} bf_guided_params;

typedef struct bf_graph bf_graph;   /* opaque */
typedef struct bf_net bf_net;       /* opaque: the learned preconditioner (see below) */
typedef struct bf_spd bf_spd;       /* opaque: the learned SPD preconditioner (see below) */

typedef struct bf_info {
  int32_t iters;         /* iterations completed                                            */
  int32_t status;        /* 0 = ran all iterations, BF_CG_CONVERGED, BF_CG_BREAKDOWN        */
  int32_t restarts;      /* LOBPCG: iterations redone without P                             */
  int32_t reserved;
  double  rnorm;         /* CG: final ||r||_2;  LOBPCG: max relative residual               */
  double  ref;           /* CG: ||b||_2 (or ||r_0||_2 when b = 0)                           */
} bf_info;

typedef struct bf_cg_opts {
  int32_t precond;       /* BF_PRECOND_*                                                    */
  int32_t beta;          /* BF_BETA_*                                                       */
  double  shift;         /* sigma >= 0: solve (L + sigma I) x = sigma x0; 0 = L x = 0       */
  double  tol;           /* > 0: stop once ||r|| <= tol * ||b|| (||r_0|| if b = 0)          */
  double* hist;          /* optional device array [2 * kmax]: alpha_j, beta_j per iteration */
  const bf_net* net;     /* BF_PRECOND_NET: the preconditioner (else ignored)               */
  const bf_spd* spd;     /* BF_PRECOND_SPD: the preconditioner (else ignored)               */
} bf_cg_opts;

typedef struct bf_lobpcg_opts {
  int32_t pencil;        /* BF_PENCIL_*                                                     */
  int32_t precond;       /* BF_PRECOND_*                                                    */
  int32_t constrain_e;   /* 1: keep X B-orthogonal to the constant vector e (Section 6)     */
  int32_t gram;          /* BF_GRAM_*: precision of the Gram products S^T [A S, B S]        */
  double  tol;           /* > 0: stop once max_j ||L x_j - theta_j B x_j|| / ||B x_j|| <= tol */
  double* theta_hist;    /* optional device array [(kmax + 1) * k]: Ritz values per step    */
  const bf_net* net;     /* BF_PRECOND_NET: the preconditioner (else ignored)               */
  const bf_spd* spd;     /* BF_PRECOND_SPD: the preconditioner (else ignored)               */
} bf_lobpcg_opts;

/* ---- graph ------------------------------------------------------------------------ */

/* Build the graph of Section 2 from the guide g (device, n elements of dtype): the
 * degree d_i = sum_j w_ij (w_ii = 1 included), diag L_i = sum_{j != i} w_ij, and, in the
 * stored modes, the forward half-window weights w_ij = exp(-|p_i-p_j|^2 / 2 sigma_s^2) *
 * exp(-|g_i-g_j|^2 / 2 sigma_r^2) (Eq. 2).  Neighbours outside the image do not exist.
 * The guide is copied; *out receives a new graph (free with bf_graph_free).
 * Synchronises `stream` (it reports BF_ENONFINITE if the guide holds NaN or Inf). */
int bf_weights(const bf_params* params, const void* guide, bf_graph** out, void* stream);

/* Recompute a graph for a new guide of the same shape and dtype (device, n elements):
 * the same work as bf_weights (Eq. 2 weights, degree, scalings) into the graph's own
 * buffers, so no device memory is allocated and the filters' workspaces are kept (for a
 * stream of images of one size).  The guide is copied.  Synchronises `stream`; returns
 * BF_ENONFINITE if the guide holds NaN or Inf (the graph's values are then undefined
 * until the next successful update).  Must not overlap filter calls on the same graph. */
int bf_graph_update(bf_graph* g, const void* guide, void* stream);

/* The guided filter as a graph (Section 3: Algorithm 1 is the transform y = W(g) x of
 * Eq. 5 with W of Eq. 6).  Square windows (1D: intervals) of radius r are truncated at
 * the border: window k holds N_k in-image pixels with guide mean mu_k and variance
 * sigma_k^2, and the graph is
 *   Wt_ij = sum over windows k containing i and j of (1 + (g_i - mu_k)(g_j - mu_k) /
 *           (sigma_k^2 + eps)) / N_k,
 * whose rows sum to N_i (the in-image pixels of the window centred at i): D = diag(N),
 * L = D - Wt, and Algorithm 1 with truncated mean filters is exactly D^-1 Wt.  In the
 * interior N = |omega| and Wt / |omega| is Eq. 6 (the paper's D = I).  The returned graph
 * works with bf_apply (ops W, L, D^-1 W = Algorithm 1, D, D^-1/2 L D^-1/2; not the
 * (diag L) form), bf_simple_filter (the linear GF iteration), bf_reguided_filter (the
 * nonlinear GF iteration of Section 3), cg_filter (Jacobi or identity preconditioner)
 * and lobpcg_filter (pencil (L, D) or (L, I), Jacobi or identity preconditioner), and
 * with bf_graph_update / bf_graph_degree / bf_graph_free; not with the learned
 * preconditioner, the batched driver, cg_filter_noalloc or bf_graph_export_weights
 * (BF_EINVAL).  The guide (device, n elements of dtype) is copied.  Synchronises
 * `stream`; BF_ENONFINITE if the guide holds NaN or Inf; BF_EINVAL for a bad parameter. */
int bf_guided_graph(const bf_guided_params* params, const void* guide, bf_graph** out,
                    void* stream);

/* Release a graph and everything it owns (NULL is allowed). */
int bf_graph_free(bf_graph* g);

/* n, the number of window taps (centre included), and the dtype of a graph. */
int bf_graph_info(const bf_graph* g, int64_t* n, int32_t* taps, int32_t* dtype);

/* Copy the degree d (n elements, dtype) into d_out. */
int bf_graph_degree(const bf_graph* g, void* d_out, void* stream);

/* Write every weight of the window, w(i, i + offset_t), into taps_out[i * taps + t]
 * (dtype; 0 where the neighbour is outside the image).  Taps are ordered row-major by
 * (dy, dx), each from -r to r (dy = 0 only in 1D; only dx = 0 or dy = 0 for the cross).
 * In the stored modes these are the stored (rounded) values. */
int bf_graph_export_weights(const bf_graph* g, void* taps_out, void* stream);

/* ---- operator --------------------------------------------------------------------- */

/* Y = op X for a block of k >= 1 vectors (Eqs. 1-4, Section 4); op is BF_OP_*.  X and Y
 * are [n][ldx] and [n][ldy] and must not overlap.  If dots is not NULL (device, k
 * doubles) it receives the column dot products dots[c] = sum_i X[i,c] * Y[i,c]. */
int bf_apply(const bf_graph* g, int op, const void* X, int64_t ldx, int k, void* Y,
             int64_t ldy, double* dots, void* stream);

/* iters steps of the bilateral filter with fixed weights, x <- D^-1 W x (Section 2's
 * linear iteration; Section 4's simple iteration for L x = 0 with preconditioner D).
 * x0 and x_out hold n elements and may be the same array. */
int bf_simple_filter(const bf_graph* g, const void* x0, int iters, void* x_out,
                     void* stream);

/* iters steps of the nonlinear bilateral filter (Section 2, the first way of iterating
 * it): each step takes the current iterate as the guide of Eq. 2 and applies one step,
 * x_{t+1} = D(x_t)^-1 W(x_t) x_t.  g gives the shape, window, sigmas, dtype and weight
 * mode; its weights, degree and scalings are overwritten: after the call (iters > 0) it
 * is the graph of the guide x_{iters-1}.  x0 and x_out hold n elements of g's dtype
 * (device, element-aligned) and may be the same array; iters = 0 copies.  Uses g's
 * simple-iteration workspace (two n-vectors).  Errors: BF_EINVAL for NULL or misaligned
 * arguments or iters < 0, BF_ENONFINITE if an iterate held NaN or Inf (read after the
 * last step, which synchronises the stream). */
int bf_reguided_filter(bf_graph* g, const void* x0, int iters, void* x_out, void* stream);

/* ---- Krylov filters --------------------------------------------------------------- */

/* Algorithm 2 (Section 5): kmax iterations of preconditioned CG for A x = b, A = L +
 * shift * I, b = shift * x0 (shift = 0: L x = 0 as printed), started at x = x0.  beta is
 * the flexible formula (opts->beta).  Stops early when s^T r = 0, when p^T q <= 0
 * (breakdown: x keeps its last value) or, with tol > 0, once ||r|| <= tol * ||b||.
 * x0 and x_out hold n elements (may be the same array).  opts may be NULL (Jacobi,
 * flexible beta, shift 0, tol 0).  If info is not NULL the stream is synchronised and
 * info filled; a breakdown then returns BF_EBREAKDOWN.  With tol > 0 the call also reads
 * the solver status every 64 iterations (a stream synchronisation) and stops enqueueing
 * once the run has stopped.  With tol = 0 and info = NULL it only enqueues kernels (the
 * scalar state is initialised by a kernel, not copied from the host), so it can be
 * captured in a CUDA graph once an uncaptured call on the same graph has sized the
 * workspace (the first call, or one with a larger problem, may allocate it).
 * BF_PRECOND_NET takes T from opts->net, BF_PRECOND_SPD from opts->spd (both run s = T r
 * by kernels of their own after each update of x and r). */
int cg_filter(const bf_graph* g, const void* x0, int kmax, const bf_cg_opts* opts,
              void* x_out, bf_info* info, void* stream);

/* Algorithm 3 (Section 6) on a block of k vectors: kmax steps of LOBPCG for the pencil
 * (L, B), B = D or I, Rayleigh-Ritz on span{X, W, P}, W = T (L X - B X Theta); the small
 * Rayleigh-Ritz problems are solved in FP64 on the GPU.  X0 is [n][ldx0] (column 0 is
 * the signal x0 to filter).  Outputs (any may be NULL): X_out [n][k] B-orthonormal Ritz
 * vectors, theta_out [k] Ritz values (ascending, double), resid_out [k] relative
 * residual norms ||L x_j - theta_j B x_j|| / ||B x_j|| (double), y_out [n] the filtered
 * signal y = X X^T B x0 (with the constraint: e_bar e + X X^T B (x0 - e_bar e), e_bar the
 * B-mean of x0).  Needs 1 <= k and 3k <= n; k <= 32.  If info is not NULL the stream
 * is synchronised and info filled. */
int lobpcg_filter(const bf_graph* g, const void* X0, int64_t ldx0, int k, int kmax,
                  const bf_lobpcg_opts* opts, void* X_out, double* theta_out,
                  double* resid_out, void* y_out, bf_info* info, void* stream);

/* r_out = shift (x0 - x) - L x, the residual of the shifted system (L + shift I) x =
 * shift x0 of cg_filter (A9's Tikhonov filter; the learned preconditioner's training pairs
 * solve (L + shift I) z = r for such r).  n elements of the graph's dtype each; r_out must
 * not alias x0 or x.  Asynchronous. */
int bf_shifted_residual(const bf_graph* g, const void* x0, const void* x, double shift, void* r_out,
                        void* stream);

/* The shifted system (L + shift I) x = shift x0 of cg_filter solved to a TRUE relative
 * residual ||shift x0 - (L + shift I) x|| / ||shift x0|| <= tol by mixed-precision
 * refinement (the FP32 recurrence of Algorithm 2 alone stalls near eps_32 times the
 * condition number): each outer step forms the residual r in FP64 on g64 and solves
 * (L + shift I) e = r by cg_filter on g32 (started at r / shift, options `inner`: T,
 * beta, inner tolerance inner->tol (default 1e-3), learned net) for at most inner_kmax
 * iterations, then x += e.  g64 (BF_F64) and g32 (BF_F32) are graphs of the same guide
 * and shape.  x0, x_out: n doubles (may be the same array).  Stops after outer_max
 * corrections.  info (may be NULL): iters = inner iterations in total, restarts = outer
 * steps, rnorm = ||r||, ref = ||shift x0||, status = BF_CG_CONVERGED once tol is met.
 * Uses the CG workspaces of both graphs; synchronises the stream once per outer step.
 * Errors: BF_EINVAL (graphs, shift <= 0, tol <= 0), those of cg_filter for an inner solve
 * (BF_EBREAKDOWN, ...), BF_ENONFINITE for a non-finite residual. */
int cg_refine(const bf_graph* g64, const bf_graph* g32, const double* x0, double shift, double tol,
              const bf_cg_opts* inner, int inner_kmax, int outer_max, double* x_out, bf_info* info,
              void* stream);

/* cg_filter without any device allocation (the paper has no counterpart: this is a
 * deployment variant).  cg_filter keeps its vectors in the graph's workspace, which grows
 * with cudaMalloc -- and cudaFree, which synchronises the whole device -- when a larger
 * problem arrives.  Callers that must not allocate device memory once they are running
 * (a fixed memory budget owned by another allocator, a loop that cannot take the implicit
 * device synchronisation) call this instead.  Same arguments and the same algorithm as
 * cg_filter, run by the same code (the same kernels for the graph's window, the same
 * early stop with tol > 0), so the results equal cg_filter's; the scratch lives in a
 * static device array of the library, about 12.6 MB, which every GPU that loads the
 * library holds until the process exits.  Bilateral graphs (bf_weights) only, FP32 or
 * FP64, any weight mode; T = Jacobi or identity (BF_EINVAL otherwise).  Limits: n <=
 * 262144 samples and at most 65536 operator tiles; larger problems return BF_EINVAL.  The
 * caller still provides the graph (built beforehand with bf_weights), x0 and x_out.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.  Every call
 * shares the one array and starts by rewriting its scalar state, so calls whose GPU work
 * overlaps (other streams, other host threads) race and must be serialised by the
 * caller. */
int cg_filter_noalloc(const bf_graph* g, const void* x0, int kmax, const bf_cg_opts* opts,
                      void* x_out, bf_info* info, void* stream);

/* ---- the learned preconditioner ----------------------------------------------------
 * The preconditioner T of Algorithms 2 and 3 is left open by the paper (Section 5: the
 * flexible beta admits a variable, nonlinear T).  A bf_net is a three-layer 3 x 3 conv
 * net on the image-shaped residual r of a graph's grid (no bias, zero outside the image):
 *   C = [ (D^-1 r) / rho, g, 1/d ] with rho = rms(D^-1 r),
 *   A1 = conv(C, W1) (16 channels), A2 = conv(relu(A1), W2) (16), O = conv(relu(A2), W3),
 *   T(r) = rho O.
 * Weights w[bf_net_nweights()] = W1 [16][3][3][3], W2 [16][16][3][3], W3 [1][16][3][3]
 * (output channel, input channel, tap row, tap column), kept in FP32 and applied rounded
 * to BF16 with FP32 accumulation.  Training pairs (r, z) solve (L + sigma I) z = r; the
 * loss of a pair is ||T(r) - z||^2 / ||z||^2.  A bf_net owns its weights, Adam state and
 * workspace; calls that use one net must be ordered on one stream.  FP32 graphs only. */
int bf_net_nweights(void);
/* New net from host weights (copied); *out must be freed with bf_net_free. */
int bf_net_create(const float* w_host, bf_net** out);
int bf_net_free(bf_net* net);
/* Copy the FP32 master weights (rounded = 0) or the BF16-rounded ones (1) to the host. */
int bf_net_weights(const bf_net* net, float* w_host, int rounded);
/* Z[:, j] = T(R[:, j]) for k image-shaped columns on g's grid (pixel-major blocks). */
int bf_net_apply(const bf_net* net, const bf_graph* g, const float* R, int64_t ldr, int k,
                 float* Z, int64_t ldz, void* stream);
/* Reset the accumulated gradient and loss. */
int bf_net_zero_grad(bf_net* net, void* stream);
/* Add the gradient and the loss of the pair (r, z) (n floats each, on g's grid). */
int bf_net_accumulate(bf_net* net, const bf_graph* g, const float* r, const float* z,
                      void* stream);
/* Read the accumulated gradient [bf_net_nweights()] and loss to the host (either may be
 * NULL); synchronises the stream. */
int bf_net_grad(const bf_net* net, float* grad_host, double* loss_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on scale times
 * the accumulated gradient (scale = 1 / pairs for the mean); then resets the
 * accumulators. */
int bf_net_adam(bf_net* net, float lr, float scale, void* stream);

/* ---- the learned symmetric positive definite preconditioner ---------------------------
 * T of Algorithms 2 and 3 (left open by the paper, Section 5; Section 8 names better
 * preconditioners as future work), linear, symmetric and positive definite by
 * construction, so that CG keeps Section 5's A-norm optimality and LOBPCG's Ritz vectors
 * stay sign-free:
 *   T r = D^-1/2 (u + K^T K u),   u = D^-1/2 r,
 * K a (2h + 1) x (2h + 1) cross-correlation of the image-shaped u on the graph's grid
 * (row-major taps K[dy][dx], zero outside the image), K^T its adjoint (K turned by 180
 * degrees).  K = 0 is Jacobi.  Training pairs (r, z) solve A z = r, A = L + sigma I; the
 * loss of a pair is the A-norm error of T r relative to z,
 *   (z - T r)^T A (z - T r) / (z^T A z).
 * A bf_spd owns K (FP32), its Adam state, gradient accumulators and a grow-only workspace
 * (cudaMalloc on first use and when a larger image comes; the device is synchronised
 * before a regrowth); calls that use one bf_spd must be ordered on one stream.  FP32
 * bilateral graphs only; cg_filter_noalloc and the batched drivers do not take it. */
/* New preconditioner of half-width h (1..4, K (2h+1)^2 taps, copied from K_host, NULL:
 * zero); *out must be freed with bf_spd_free. */
int bf_spd_create(int half, const float* K_host, bf_spd** out);
int bf_spd_free(bf_spd* T);
/* Number of taps (2h+1)^2 (0 for NULL). */
int bf_spd_size(const bf_spd* T);
/* Copy K to the host (bf_spd_size floats). */
int bf_spd_weights(const bf_spd* T, float* K_host);
/* Z[:, j] = T R[:, j] for k image-shaped columns on g's grid (pixel-major, ld >= k);
 * Z may equal R. */
int bf_spd_apply(const bf_spd* T, const bf_graph* g, const float* R, int64_t ldr, int k,
                 float* Z, int64_t ldz, void* stream);
/* Reset the accumulated gradient and loss. */
int bf_spd_zero_grad(bf_spd* T, void* stream);
/* Add the loss and its gradient with respect to K of the pair (r, z) (n floats each on
 * g's grid, A z = r with A = L + shift I, shift >= 0). */
int bf_spd_accumulate(bf_spd* T, const bf_graph* g, double shift, const float* r,
                      const float* z, void* stream);
/* Read the accumulated gradient (bf_spd_size doubles) and loss to the host (either may
 * be NULL); synchronises the stream. */
int bf_spd_grad(const bf_spd* T, double* grad_host, double* loss_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on scale times
 * the accumulated gradient; then resets the accumulators. */
int bf_spd_adam(bf_spd* T, float lr, float scale, void* stream);

/* ---- batched CG -----------------------------------------------------------------------
 * Algorithm 2 on many instances (images and signals of uneven sizes) at once: every launch
 * covers the tiles of all instances (one work list per window shape), so small instances
 * still fill the GPU; per-instance FP64 scalars as in cg_filter.  The whole run of kmax
 * iterations is captured once as a CUDA graph and replayed by later calls with the same
 * kmax and options.  Graphs must be FP32 with on-the-fly weights and a 7 x 7 (images),
 * 11-tap (signals) or 5-point cross window; instances with the same window shape must
 * share sigma_s and sigma_r.  The batch keeps pointers to the graphs (which must outlive
 * it) and owns the per-instance vectors (5 n-vectors each). */
typedef struct bf_batch bf_batch;
int bf_batch_create(const bf_graph* const* graphs, int count, bf_batch** out);
int bf_batch_free(bf_batch* b);
/* x0[i], x_out[i]: HOST array of device pointers, n_i floats each (x_out[i] may equal
 * x0[i]).  opts as for cg_filter (Jacobi or identity; hist and net unused).  infos: NULL
 * or a host array of count bf_info, filled after synchronising the stream. */
int bf_batch_cg(bf_batch* b, const float* const* x0, float* const* x_out, int kmax,
                const bf_cg_opts* opts, bf_info* infos, void* stream);
/* The same run as bf_batch_cg in one persistent, cooperative launch: every CTA walks the
 * work lists of all instances phase by phase (start, then per iteration the direction and
 * the update jobs), the phases separated by a grid-wide barrier in device memory.  Same
 * jobs and reduction order as bf_batch_cg, so the results are identical.  Every barrier
 * wait is bounded (1 s): if one gives up, the kernel returns and the call reports
 * BF_ETIMEOUT (the instance vectors are then undefined).  Synchronises the stream. */
int bf_batch_cg_persistent(bf_batch* b, const float* const* x0, float* const* x_out, int kmax,
                           const bf_cg_opts* opts, bf_info* infos, void* stream);
/* Algorithm 3 (block LOBPCG, as lobpcg_filter) on every instance of the batch: instance i
 * runs on internal stream i % S (S = nstreams, 1..64), enqueued by S host threads, so the
 * Rayleigh-Ritz solves of different instances (one SM each) and their data-parallel
 * kernels run side by side.  X0: HOST array of device pointers, [n_i][k] floats each
 * (ld = k; column 0 the signal to filter); theta_out, y_out: NULL or HOST arrays of device
 * pointers (k doubles, n_i floats).  opts as for lobpcg_filter.  Needs 3k <= n_i.  The
 * work is ordered after the caller's stream and the caller's stream waits for it; with
 * infos (host array of count) every instance's call synchronises its stream and fills its
 * entry.  Each graph's LOBPCG workspace is used, so no other LOBPCG call may run on these
 * graphs meanwhile.  Errors: the first failing instance's code and message. */
int bf_batch_lobpcg(bf_batch* b, const float* const* X0, int k, int kmax, const bf_lobpcg_opts* opts,
                    double* const* theta_out, float* const* y_out, int nstreams, bf_info* infos, void* stream);
/* Autotuner: time `iters` iterations with each candidate tile shape of the image class
 * (32 x 8, 64 x 4, 16 x 16 pixels) on these vectors and keep the fastest; ms_out (host,
 * 3 floats) receives the timings.  Synchronises the stream. */
int bf_batch_tune(bf_batch* b, const float* const* x0, float* const* x_out, int iters,
                  float* ms_out, void* stream);
/* Total tiles of the work lists and the image-class tile shape in use (0, 1, 2 as above). */
int bf_batch_tiles(const bf_batch* b, int64_t* tiles_out, int* variant_out);

/* Message for the last error on the calling thread ("" if none). */
const char* bf_last_error(void);

/* Number of kernels this library has launched in the process so far (all threads). */
uint64_t bf_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* BF_H_ */
