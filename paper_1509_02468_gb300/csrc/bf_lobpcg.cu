// Algorithm 3 (Section 6) for a block of k vectors: LOBPCG as a low-pass filter for the
// pencil (L, B), B = D or I, with preconditioner T = D^-1 or I and the optional
// constraint x ⊥_B e.
//
// Device pipeline of one iteration (all state on the GPU, no host read-back):
//   [project W off e]  ->  AW = L W (matrix-free operator)  ->  Gram partials of
//   G_A = S^T (A S) and G_B = S^T (B S), S = [X W P], FP32 products with compensated
//   accumulation, FP64 across blocks  ->  one-CTA FP64 Rayleigh-Ritz (unit-diagonal
//   scaling, Cholesky of G_B with the drop-P restart, standard form, parallel cyclic
//   Jacobi, ascending sort)  ->  fused update X = S C_X, AX = AS C_X, P = [W P] C_{WP},
//   AP = [AW AP] C_{WP}, and the next residual W = T (AX - B X Theta) with its norms.
// Buffers ping-pong between two copies; the final kernels pick the current copy from the
// device-side iteration count, so an early stop (tolerance or breakdown) needs no sync.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "bf_internal.cuh"
#include "bf_rr.cuh"

int bf_apply_f32(const bf_graph* g, int op, const float* X, int64_t ldx, int k, float* Y,
                 int64_t ldy, double* dots, cudaStream_t s);
int bf_net_apply_f32(const bf_net* net, const bf_graph* g, const float* R, int64_t ldr, int k, float* Z,
                     int64_t ldz, cudaStream_t s, const int* stop);
int bf_spd_apply_f32(const bf_spd* T, const bf_graph* g, const float* R, int64_t ldr, int k, float* Z,
                     int64_t ldz, cudaStream_t s);
int bf_gram_tc(const float* const* S, const float* const* AS, const float* b, int nblk, int k, int64_t n,
               int mode, double* partials, int grid, double* G, const int* status, int* err, cudaStream_t s);
int bf_apply_f64(const bf_graph* g, int op, const double* X, int64_t ldx, int k, double* Y,
                 int64_t ldy, double* dots, cudaStream_t s);

#define LOB_KMAX 32

namespace {

enum { LOB_RUN = 0, LOB_CONV = 1, LOB_BREAK = 2, LOB_NONFINITE = 3, LOB_TIMEOUT = 4 };

struct LobState {
  double theta[LOB_KMAX];
  double resid[LOB_KMAX];
  double cw[LOB_KMAX];      // e^T B W / e^T B e (constraint projection coefficients)
  double ebe;               // e^T B e
  double tol;
  int status;
  int iter;                 // completed iterations
  int restarts;
  int pad;
  unsigned int counter;
  unsigned int pad2;
};

// ------------------------------------------------------------------ apply wrapper
template <typename T>
int apply_T(const bf_graph* g, int op, const T* X, int64_t ldx, int k, T* Y, int64_t ldy,
            cudaStream_t s);
template <>
int apply_T<float>(const bf_graph* g, int op, const float* X, int64_t ldx, int k, float* Y,
                   int64_t ldy, cudaStream_t s) {
  return bf_apply_f32(g, op, X, ldx, k, Y, ldy, nullptr, s);
}
template <>
int apply_T<double>(const bf_graph* g, int op, const double* X, int64_t ldx, int k, double* Y,
                    int64_t ldy, cudaStream_t s) {
  return bf_apply_f64(g, op, X, ldx, k, Y, ldy, nullptr, s);
}

// ------------------------------------------------------------------ runtime-width grid sums
// Each block adds its per-value sums into shared memory (sh[0..nv)); then the block writes
// them as partials and the last block to arrive sums all partials in block order.
// Returns true in every thread of the last block; `out` (nv doubles) is then valid.
__device__ bool grid_colsum_last(const double* sh, int nv, double* partials,
                                 unsigned int* counter, double* out, int* is_last_sh) {
  const unsigned nb = gridDim.x;
  __syncthreads();
  for (int j = threadIdx.x; j < nv; j += blockDim.x) partials[(size_t)blockIdx.x * nv + j] = sh[j];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *is_last_sh = (atomicAdd(counter, 1u) == nb - 1);
  __syncthreads();
  if (!*is_last_sh) return false;
  __threadfence();
  // one warp per value: lanes take blocks lane, lane + 32, ... in order, then a
  // fixed shuffle tree (deterministic)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < nv; j += nw) {
    double s = 0.0;
    for (unsigned b = lane; b < nb; b += 32) s += ((volatile double*)partials)[(size_t)b * nv + j];
    s = warp_sum(s);
    if (lane == 0) out[j] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// ------------------------------------------------------------------ small kernels
// Copy a block [n][ldx] -> [n][k] (contiguous).
template <typename T>
__global__ void k_copy_block(const T* __restrict__ X, int64_t ldx, int k, int64_t n, T* Y) {
  const int64_t tot = n * k;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / k;
    const int c = (int)(q - i * k);
    Y[q] = X[i * ldx + c];
  }
}

// Sums for the constraint: cs[c] = sum_i b_i V[i][c] (c < k), cs[k] = sum_i b_i.  The last
// block stores cw[c] = cs[c] / cs[k] and ebe = cs[k].  Thread t of a block owns column
// t % k of pixel lane t / k.
template <typename T>
__global__ void __launch_bounds__(256) k_bsums(const T* __restrict__ V, int k, int64_t n,
                                               const T* __restrict__ b, double* partials,
                                               LobState* st) {
  if (st->status != LOB_RUN) return;
  __shared__ double sh[LOB_KMAX + 1];
  __shared__ double out[LOB_KMAX + 1];
  __shared__ int last;
  for (int j = threadIdx.x; j <= k; j += blockDim.x) sh[j] = 0.0;
  __syncthreads();
  const int lanes = blockDim.x / k;
  const int pl = threadIdx.x / k, c = threadIdx.x - pl * k;
  T acc = T(0), accb = T(0);
  if (pl < lanes) {
    for (int64_t i = (int64_t)blockIdx.x * lanes + pl; i < n; i += (int64_t)gridDim.x * lanes) {
      const T bi = b ? b[i] : T(1);
      acc = fma(bi, V[i * k + c], acc);
      if (c == 0) accb += bi;
    }
    atomicAdd(&sh[c], (double)acc);
    if (c == 0) atomicAdd(&sh[k], (double)accb);
  }
  if (grid_colsum_last(sh, k + 1, partials, &st->counter, out, &last)) {
    if (threadIdx.x == 0) {
      st->ebe = out[k];
      for (int q = 0; q < k; ++q) st->cw[q] = out[q] / out[k];
    }
  }
}

// Reset the state before a run (kernel form, so the whole run can be captured in a graph).
__global__ void k_state_init(LobState* st, double tol) {
  if (threadIdx.x == 0) {
    st->status = LOB_RUN;
    st->iter = 0;
    st->restarts = 0;
    st->counter = 0u;
    st->tol = tol;
    st->ebe = 0.0;
  }
  if (threadIdx.x < LOB_KMAX) {
    st->theta[threadIdx.x] = 0.0;
    st->resid[threadIdx.x] = 0.0;
    st->cw[threadIdx.x] = 0.0;
  }
}

__global__ void k_state_iter0(LobState* st) {
  if (threadIdx.x == 0) st->iter = 0;
}

template <typename T>
struct XPair {
  const T* p[2];
};

// V[i][c] -= cw[c]  (B-orthogonal projection off e, coefficients from k_bsums/k_update).
template <typename T>
__global__ void k_project(T* V, int k, int64_t n, const LobState* st) {
  if (st->status != LOB_RUN) return;
  const int64_t tot = n * k;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q % k);
    V[q] -= (T)st->cw[c];
  }
}

// ------------------------------------------------------------------ Gram partials
// G_A = S^T (A S) and G_B = S^T (B S) for S = [X W P] (m = nblk k columns), split over the
// pixels: each block accumulates its share and writes one partial, summed in order by
// k_gram_reduce.  Both matrices are symmetric (L and B are), so only the upper-triangle
// 4 x 4 tiles (ta <= tb) are formed; k_gram_reduce mirrors them.  A thread owns one tile
// of both matrices (16 + 16 accumulators, the S values of the tile's rows are shared) and
// one pixel group of the staged chunk.  Float path: FP32 products summed over runs of 16
// pixels, then folded by TwoSum into (hi, lo) pairs; groups are combined by a tree of
// TwoSums, and the block partial hi + lo is written in FP64.
#define GRAM_T 512
// pixels per shared-memory chunk (two buffers of S and A S chunks, m4 <= 96 columns each):
// 128 in FP32 (193 KB), 64 in FP64; longer chunks mean fewer CTA barriers per pixel
template <typename T>
struct GramChunk {
  static constexpr int pxc = sizeof(T) == 4 ? 128 : 64;
  static constexpr int buf = pxc * 96;
};

template <typename T>
struct GramArgs {
  const T* S[3];
  const T* AS[3];
  const T* b;        // B diagonal (NULL: I)
  int nblk, k, m, m4;
  int64_t n;
  double* partials;  // [gridDim.x][2][m][m] (upper tiles only)
  const LobState* st;
};

// p[i] for i < 3 by selects (a runtime index into a kernel-parameter array makes the
// compiler copy the array to local memory)
template <typename P>
__device__ __forceinline__ P pick3(const P (&p)[3], int i) {
  return i == 0 ? p[0] : (i == 1 ? p[1] : p[2]);
}

// Two FP32 lanes in one 64-bit register (f32x2 arithmetic, round to nearest per lane).
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
  f2_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
  f2_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
  f2_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
  f2_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}
__device__ __forceinline__ void two_sum(double& hi, double& lo, double x) { hi += x; }

template <typename T>
__global__ void __launch_bounds__(GRAM_T) k_gram(const GramArgs<T> a) {
  bf_pdl_enter();
  if (a.st->status != LOB_RUN) return;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PXC = GramChunk<T>::pxc, BUF = GramChunk<T>::buf;
  const int m = a.m, m4 = a.m4, k = a.k;
  const int ta_n = m4 / 4;
  const int nt = ta_n * (ta_n + 1) / 2;
  const int ng = GRAM_T / nt;                         // pixel groups (>= 1)
  const int grp = threadIdx.x / nt, tile = threadIdx.x - grp * nt;
  const bool act = grp < ng;
  // tile -> (ta, tb), ta <= tb, row-major over the upper triangle
  int ta = 0, tb = 0;
  {
    int t = act ? tile : 0, row = 0;
    while (t >= ta_n - row) { t -= ta_n - row; ++row; }
    ta = row;
    tb = row + t;
  }
  T* sS = reinterpret_cast<T*>(smem);                 // [2][BUF]: chunk of S, [PXC][m4]
  T* sA = sS + 2 * BUF;                          // [2][BUF]: chunk of A S
  T* sb = sA + 2 * BUF;                          // [2][PXC]
  T cA[16], cB[16], hA[16], lA[16], hB[16], lB[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) cA[e] = cB[e] = hA[e] = lA[e] = hB[e] = lB[e] = T(0);
  int since_fold = 0;
  const int fold_every = 16;      // FP32 runs of 16 products (64 cost ~5e-7 in Ritz values on small images)
  const int64_t nchunks = (a.n + PXC - 1) / PXC;
  const bool vec = (k % 4 == 0);
  // FP32 blocks with k % 4 == 0: the next chunk is copied into the second shared-memory
  // buffer by cp.async while the current one is processed (zero-filled past n and m).
  const bool pipe = vec && sizeof(T) == 4;
  const int q4 = m4 / 4;
  auto issue = [&](int64_t ch, int buf) {
    const int64_t i0 = ch * PXC;
    T* dS = sS + (size_t)buf * BUF;
    T* dA = sA + (size_t)buf * BUF;
    T* db = sb + (size_t)buf * PXC;
    for (int q = threadIdx.x; q < PXC * q4; q += GRAM_T) {
      const int p = q / q4, c4 = q - p * q4;
      const int64_t i = i0 + p;
      const int col = c4 * 4, blk = col / k, c = col - blk * k;
      const bool ok = i < a.n && col < m;
      const T* gs = ok ? pick3(a.S, blk) + i * k + c : a.S[0];
      const T* ga = ok ? pick3(a.AS, blk) + i * k + c : a.AS[0];
      const unsigned nb = ok ? 16u : 0u;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dS + p * m4 + col)),
                   "l"(gs), "r"(nb) : "memory");
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dA + p * m4 + col)),
                   "l"(ga), "r"(nb) : "memory");
    }
    if (threadIdx.x < PXC) {
      const int64_t i = i0 + threadIdx.x;
      if (a.b) {
        const bool ok = i < a.n;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((unsigned)__cvta_generic_to_shared(db + threadIdx.x)),
                     "l"(ok ? a.b + i : a.b), "r"(ok ? 4u : 0u) : "memory");
      } else {
        db[threadIdx.x] = (i < a.n) ? T(1) : T(0);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (pipe && blockIdx.x < nchunks) issue(blockIdx.x, 0);
  int it_local = 0;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x, ++it_local) {
    const int64_t i0 = ch * PXC;
    const int cur = pipe ? (it_local & 1) : 0;
    __syncthreads();                       // the previous chunk's readers are done
    if (pipe) {
      if (ch + gridDim.x < nchunks) {
        issue(ch + gridDim.x, cur ^ 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncthreads();
    } else if (vec) {
      const int q4v = m4 / 4;
      for (int q = threadIdx.x; q < PXC * q4v; q += GRAM_T) {
        const int p = q / q4v, c4 = q - p * q4v;
        const int64_t i = i0 + p;
        const int col = c4 * 4, blk = col / k, c = col - blk * k;
        Vec<T, 4> vs, va;
        if (i < a.n && col < m) {
          vs = *reinterpret_cast<const Vec<T, 4>*>(pick3(a.S, blk) + i * k + c);
          va = *reinterpret_cast<const Vec<T, 4>*>(pick3(a.AS, blk) + i * k + c);
        } else {
          vs.v[0] = vs.v[1] = vs.v[2] = vs.v[3] = T(0);
          va = vs;
        }
        *reinterpret_cast<Vec<T, 4>*>(sS + p * m4 + col) = vs;
        *reinterpret_cast<Vec<T, 4>*>(sA + p * m4 + col) = va;
      }
      for (int p = threadIdx.x; p < PXC; p += GRAM_T) {
        const int64_t i = i0 + p;
        sb[p] = (i < a.n) ? (a.b ? a.b[i] : T(1)) : T(0);
      }
      __syncthreads();
    } else {
      for (int q = threadIdx.x; q < PXC * m4; q += GRAM_T) {
        const int p = q / m4, col = q - p * m4;
        const int64_t i = i0 + p;
        T vs = T(0), va = T(0);
        if (i < a.n && col < m) {
          const int blk = col / k, c = col - blk * k;
          vs = pick3(a.S, blk)[i * k + c];
          va = pick3(a.AS, blk)[i * k + c];
        }
        sS[q] = vs;
        sA[q] = va;
      }
      for (int p = threadIdx.x; p < PXC; p += GRAM_T) {
        const int64_t i = i0 + p;
        sb[p] = (i < a.n) ? (a.b ? a.b[i] : T(1)) : T(0);
      }
      __syncthreads();
    }
    const T* cS = sS + (size_t)cur * BUF;
    const T* cA_ = sA + (size_t)cur * BUF;
    const T* cb = sb + (size_t)cur * PXC;
    if (act) {
      for (int p = grp; p < PXC; p += ng) {
        const Vec<T, 4> xa = *reinterpret_cast<const Vec<T, 4>*>(cS + p * m4 + ta * 4);
        const Vec<T, 4> xb = *reinterpret_cast<const Vec<T, 4>*>(cS + p * m4 + tb * 4);
        const Vec<T, 4> yb = *reinterpret_cast<const Vec<T, 4>*>(cA_ + p * m4 + tb * 4);
        const T bp = cb[p];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const T bx = bp * xa.v[i];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            cA[i * 4 + j] = fma(xa.v[i], yb.v[j], cA[i * 4 + j]);
            cB[i * 4 + j] = fma(bx, xb.v[j], cB[i * 4 + j]);
          }
        }
        if (++since_fold == fold_every) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            two_sum(hA[e], lA[e], cA[e]);
            two_sum(hB[e], lB[e], cB[e]);
            cA[e] = cB[e] = T(0);
          }
          since_fold = 0;
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    two_sum(hA[e], lA[e], cA[e]);
    two_sum(hB[e], lB[e], cB[e]);
  }
  // tree over the pixel groups: the sender (odd multiple of stride) hands its (hi, lo)
  // pairs to the receiver stride groups below
  T* scr = reinterpret_cast<T*>(smem);               // [ng / 2 + 1][nt][64]
  for (int stride = 1; stride < ng; stride <<= 1) {
    __syncthreads();
    const bool sender = act && (grp % (2 * stride) == stride);
    if (sender) {
      T* dst = scr + ((size_t)((grp - stride) / (2 * stride)) * nt + tile) * 64;
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        dst[e] = hA[e];
        dst[16 + e] = lA[e];
        dst[32 + e] = hB[e];
        dst[48 + e] = lB[e];
      }
    }
    __syncthreads();
    const bool receiver = act && (grp % (2 * stride) == 0) && (grp + stride < ng);
    if (receiver) {
      const T* src = scr + ((size_t)(grp / (2 * stride)) * nt + tile) * 64;
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        two_sum(hA[e], lA[e], src[e]);
        lA[e] += src[16 + e];
        two_sum(hB[e], lB[e], src[32 + e]);
        lB[e] += src[48 + e];
      }
    }
  }
  if (act && grp == 0) {
    double* out = a.partials + (size_t)blockIdx.x * 2 * m * m;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = ta * 4 + i, c = tb * 4 + j;
        if (r < m && c < m && r <= c) {
          out[(size_t)r * m + c] = (double)hA[i * 4 + j] + (double)lA[i * 4 + j];
          out[(size_t)m * m + (size_t)r * m + c] = (double)hB[i * 4 + j] + (double)lB[i * 4 + j];
        }
      }
  }
}

// Sum the Gram partials over blocks (one warp per entry, each lane a strided share of the
// blocks, combined by shuffles) and write both triangles: G[2][m][m].
__global__ void k_gram_reduce(const double* __restrict__ partials, int nblocks, int m, double* G,
                              const LobState* st) {
  bf_pdl_enter();
  if (st->status != LOB_RUN) return;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = gtid >> 5, part = gtid & 31;
  const int nupper = m * (m + 1) / 2;
  const bool ok = e < 2 * nupper;
  int w = 0, r = 0, c = 0;
  if (ok) {
    w = e / nupper;
    int t = e - w * nupper;
    while (t >= m - r) { t -= m - r; ++r; }
    c = r + t;
  }
  double s = 0.0;
  if (ok) {
    const size_t off = (size_t)w * m * m + (size_t)r * m + c;
    for (int b = part; b < nblocks; b += 32) s += partials[(size_t)b * 2 * m * m + off];
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (ok && part == 0) {
    G[(size_t)w * m * m + (size_t)r * m + c] = s;
    G[(size_t)w * m * m + (size_t)c * m + r] = s;
  }
}

// ------------------------------------------------------------------ update
// For a tile of pixels and a group of CW columns per thread:
//   X' = S C[:, cols]  and  P' = S Cp[:, cols]  (Cp: the next P, B-orthogonal to X').
// A X' and A P' are not formed here: they are recomputed by the operator kernel, which
// keeps S^T A S consistent with S (linear combinations of [AX AW AP] cancel heavily once
// X is nearly converged).
template <typename T>
struct UpdArgs {
  const T* S[3];
  int nblk, k, m;
  int64_t n;
  const double* C;       // [m][k]
  const double* Cp;      // [m][k] or NULL
  T* Xn;
  T* Pn;                 // NULL when Cp is NULL
  const LobState* st;
};

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// FP32 update for a block width KT known at compile time: one pixel per thread, all KT
// columns, so that every coefficient load is the same address across the warp (a shared-
// memory broadcast); persistent, the coefficients staged once per CTA.  The arithmetic is
// that of k_update (double-float X-block part, FMA for the W and P terms) on packed column
// pairs, entry by entry in the same order, so the result is the same bit for bit.
template <int KT>
__global__ void __launch_bounds__(256, 2) k_update_f32(const UpdArgs<float> a) {
  bf_pdl_enter();
  if (a.st->status != LOB_RUN) return;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NV = KT / 4, NP = KT / 2;
  const int m = a.m;
  const bool with_p = a.Pn != nullptr;
  float* sC = reinterpret_cast<float*>(smem);     // [m][KT]
  float* sCp = sC + m * KT;                       // [m][KT]
  for (int q = threadIdx.x; q < m * KT; q += 256) {
    sC[q] = (float)a.C[q];
    sCp[q] = with_p ? (float)a.Cp[q] : 0.0f;
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * 256) {
    // the pixel's row of block blk + 1 is loaded while block blk is processed
    Vec<float, 4> sv[NV], sn[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) sv[c] = *reinterpret_cast<const Vec<float, 4>*>(a.S[0] + i * KT + 4 * c);
    f2_t x2[NP], xl2[NP], pp2[NP];
#pragma unroll
    for (int h = 0; h < NP; ++h) x2[h] = xl2[h] = pp2[h] = 0ull;
#pragma unroll
    for (int blk = 0; blk < 3; ++blk) {
      if (blk >= a.nblk) break;
      if (blk + 1 < a.nblk) {
        const float* row = pick3(a.S, blk + 1) + i * KT;
#pragma unroll
        for (int c = 0; c < NV; ++c) sn[c] = *reinterpret_cast<const Vec<float, 4>*>(row + 4 * c);
      }
#pragma unroll
      for (int c = 0; c < NV; ++c) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float sx = sv[c].v[u];
          const int r = blk * KT + 4 * c + u;
          const ulonglong2* cr = reinterpret_cast<const ulonglong2*>(sC + r * KT);
          const f2_t s2 = f2(sx, sx);
          if (blk == 0) {
            const f2_t ns2 = f2(-sx, -sx);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
              const ulonglong2 cv = cr[q];
#pragma unroll
              for (int l = 0; l < 2; ++l) {
                const int h = 2 * q + l;
                const f2_t c2 = l ? cv.y : cv.x;
                const f2_t pr = f2_mul(s2, c2);
                const f2_t pen = f2_fma(ns2, c2, pr);
                const f2_t t = f2_add(x2[h], pr);
                const f2_t bp = f2_sub(t, x2[h]);
                const f2_t lo = f2_add(f2_sub(x2[h], f2_sub(t, bp)), f2_sub(pr, bp));
                xl2[h] = f2_add(xl2[h], f2_sub(lo, pen));
                x2[h] = t;
              }
            }
          } else {
#pragma unroll
            for (int q = 0; q < NV; ++q) {
              const ulonglong2 cv = cr[q];
              xl2[2 * q] = f2_fma(s2, cv.x, xl2[2 * q]);
              xl2[2 * q + 1] = f2_fma(s2, cv.y, xl2[2 * q + 1]);
            }
          }
          if (with_p) {
            const ulonglong2* pr = reinterpret_cast<const ulonglong2*>(sCp + r * KT);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
              const ulonglong2 pv = pr[q];
              pp2[2 * q] = f2_fma(s2, pv.x, pp2[2 * q]);
              pp2[2 * q + 1] = f2_fma(s2, pv.y, pp2[2 * q + 1]);
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NV; ++c) sv[c] = sn[c];
    }
    ulonglong2* xo = reinterpret_cast<ulonglong2*>(a.Xn + i * KT);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      ulonglong2 o;
      o.x = f2_add(x2[2 * q], xl2[2 * q]);
      o.y = f2_add(x2[2 * q + 1], xl2[2 * q + 1]);
      xo[q] = o;
    }
    if (with_p) {
      ulonglong2* po = reinterpret_cast<ulonglong2*>(a.Pn + i * KT);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        ulonglong2 o;
        o.x = pp2[2 * q];
        o.y = pp2[2 * q + 1];
        po[q] = o;
      }
    }
  }
}

template <typename T, int CW>
__global__ void __launch_bounds__(256) k_update(const UpdArgs<T> a) {
  if (a.st->status != LOB_RUN) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = a.k, m = a.m;
  const int ngrp = k / CW;
  const bool with_p = a.Pn != nullptr;
  T* sC = reinterpret_cast<T*>(smem);         // [m][k]
  T* sCp = sC + m * k;                        // [m][k]
  for (int q = threadIdx.x; q < m * k; q += 256) {
    sC[q] = (T)a.C[q];
    sCp[q] = with_p ? (T)a.Cp[q] : T(0);
  }
  __syncthreads();
  const int64_t total = a.n * ngrp;
  for (int64_t q = (int64_t)blockIdx.x * 256 + threadIdx.x; q < total; q += (int64_t)gridDim.x * 256) {
    const int64_t i = q / ngrp;
    const int g = (int)(q - i * ngrp);
    // X' = X C_x + (W C_w + P C_p): the X-block part in double-float (each product exactly
    // by TwoProd, the running sum by TwoSum; an FP32 running sum over all 3k terms moved
    // the Ritz values of small problems by ~1e-6), the W and P terms, which carry the
    // step's correction, by FMA into the low part
    T x[CW], xl[CW], pp[CW];
#pragma unroll
    for (int e = 0; e < CW; ++e) x[e] = xl[e] = pp[e] = T(0);
    for (int blk = 0; blk < a.nblk; ++blk) {
      const T* row = pick3(a.S, blk) + i * k;
      for (int c0 = 0; c0 < k; c0 += CW) {
        Vec<T, CW> sv = *reinterpret_cast<const Vec<T, CW>*>(row + c0);
#pragma unroll
        for (int u = 0; u < CW; ++u) {
          const int r = blk * k + c0 + u;
          const Vec<T, CW> cv = *reinterpret_cast<const Vec<T, CW>*>(sC + r * k + g * CW);
          if (blk == 0) {
#pragma unroll
            for (int e = 0; e < CW; ++e) {
              const T pr = mul_rn(sv.v[u], cv.v[e]);    // not contracted into the add below
              const T pe = fma(sv.v[u], cv.v[e], -pr);
              const T t = x[e] + pr;
              const T bp = t - x[e];
              xl[e] += ((x[e] - (t - bp)) + (pr - bp)) + pe;
              x[e] = t;
            }
          } else {
#pragma unroll
            for (int e = 0; e < CW; ++e) xl[e] = fma(sv.v[u], cv.v[e], xl[e]);
          }
          if (with_p) {
            const Vec<T, CW> pv = *reinterpret_cast<const Vec<T, CW>*>(sCp + r * k + g * CW);
#pragma unroll
            for (int e = 0; e < CW; ++e) pp[e] = fma(sv.v[u], pv.v[e], pp[e]);
          }
        }
      }
    }
    Vec<T, CW> xo, po;
#pragma unroll
    for (int e = 0; e < CW; ++e) {
      xo.v[e] = x[e] + xl[e];
      po.v[e] = pp[e];
    }
    *reinterpret_cast<Vec<T, CW>*>(a.Xn + i * k + g * CW) = xo;
    if (with_p) *reinterpret_cast<Vec<T, CW>*>(a.Pn + i * k + g * CW) = po;
  }
}

// ------------------------------------------------------------------ residual
// R = AX - b X theta, W = t R (t = 1/d or 1), per-column block sums of R^2, (b X)^2 and
// b W (thread t of a block owns column t % k of pixel lane t / k); k_resid_cols and
// k_resid_tail turn them into the residual norms.
template <typename T>
__global__ void __launch_bounds__(256) k_resid(const T* __restrict__ X, const T* __restrict__ AX,
                                               int k, int64_t n, const T* __restrict__ b,
                                               const T* __restrict__ tinv, T* __restrict__ Wn,
                                               double* __restrict__ partials, const LobState* st) {
  bf_pdl_enter();
  if (st->status != LOB_RUN) return;
  __shared__ T sred[3][256];                  // the threads' sums (blockDim.x = 256)
  const int lanes = blockDim.x / k;
  const int pl = threadIdx.x / k, c = threadIdx.x - pl * k;
  T r2 = T(0), bx2 = T(0), bw = T(0);
  if (pl < lanes) {
    const T th = (T)st->theta[c];
#pragma unroll 4
    for (int64_t i = (int64_t)blockIdx.x * lanes + pl; i < n; i += (int64_t)gridDim.x * lanes) {
      const T bi = b ? b[i] : T(1);
      const T ti = tinv ? tinv[i] : T(1);
      const T bx = bi * X[i * k + c];
      const T rr = AX[i * k + c] - bx * th;
      const T w = ti * rr;
      Wn[i * k + c] = w;
      r2 = fma(rr, rr, r2);
      bx2 = fma(bx, bx, bx2);
      bw = fma(bi, w, bw);
    }
  }
  // block partials only, summed by the next kernels (a kernel boundary instead of a fence,
  // an arrival counter and a last block, which cost more than the pass itself); inside
  // the block the threads' sums go through shared memory and are added in FP64 in a
  // fixed order (no shared-memory FP64 atomics)
  const bool own = pl < lanes;
  sred[0][threadIdx.x] = own ? r2 : T(0);
  sred[1][threadIdx.x] = own ? bx2 : T(0);
  sred[2][threadIdx.x] = own ? bw : T(0);
  __syncthreads();
  for (int q = threadIdx.x; q < 3 * k; q += blockDim.x) {
    const int which = q / k, cc = q - which * k;
    double t = 0.0;
    for (int p = 0; p < lanes; ++p) t += (double)sred[which][p * k + cc];
    partials[(size_t)blockIdx.x * 3 * k + q] = t;
  }
}

// Column sums of k_resid's block partials: block j sums value j over all blocks (each
// thread a strided share, then a fixed-order block reduction) into cols[j].
__global__ void __launch_bounds__(256) k_resid_cols(const double* __restrict__ partials, int nb, int nv,
                                                    double* __restrict__ cols, const LobState* st) {
  bf_pdl_enter();
  if (st->status != LOB_RUN) return;
  __shared__ double red[256 / 32];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) acc += partials[(size_t)b * nv + j];
  double v[1] = {acc}, tot[1];
  block_sum<1, double>(v, red, tot);
  if (threadIdx.x == 0) cols[j] = tot[0];
}

// The relative residual norms, the constraint coefficients e^T B W / e^T B e, the step
// count and the tolerance test from the column sums of R^2, (b X)^2 and b W.
__global__ void k_resid_tail(const double* __restrict__ cols, int k, int constrain, LobState* st) {
  bf_pdl_enter();
  if (st->status != LOB_RUN) return;
  const int t = threadIdx.x;
  double r = 0.0;
  if (t < k) {
    r = sqrt(cols[t]) / sqrt(cols[k + t]);
    st->resid[t] = r;
    st->cw[t] = constrain ? cols[2 * k + t] / st->ebe : 0.0;
  }
  __syncwarp();
  if (t == 0) {
    st->iter += 1;
    double mx = 0.0;
    bool fin = true;
    for (int q = 0; q < k; ++q) {
      mx = fmax(mx, st->resid[q]);
      fin = fin && isfinite(st->resid[q]);
    }
    if (!fin) st->status = LOB_NONFINITE;
    else if (st->tol > 0.0 && mx <= st->tol) st->status = LOB_CONV;
  }
}

// y = X c + ebar (constrained) with c = X^T B (x0 - ebar e).  First the sums
// out[c] = sum b_i X_ic x0_i, out[k + c] = sum b_i X_ic, out[2k] = sum b_i x0_i,
// out[2k + 1] = sum b_i (column-lane mapping as in k_bsums), then the combination.
template <typename T>
__global__ void __launch_bounds__(256) k_ysums(const XPair<T> xs, int k, int64_t n,
                                               const T* __restrict__ x0, int64_t ldx0,
                                               const T* b, double* partials, LobState* st,
                                               double* out) {
  __shared__ double sh[2 * LOB_KMAX + 2];
  __shared__ int last;
  const T* X = xs.p[st->iter & 1];
  for (int j = threadIdx.x; j < 2 * k + 2; j += blockDim.x) sh[j] = 0.0;
  __syncthreads();
  const int lanes = blockDim.x / k;
  const int pl = threadIdx.x / k, c = threadIdx.x - pl * k;
  T a1 = T(0), a2 = T(0), a3 = T(0), a4 = T(0);
  if (pl < lanes) {
    for (int64_t i = (int64_t)blockIdx.x * lanes + pl; i < n; i += (int64_t)gridDim.x * lanes) {
      const T bi = b ? b[i] : T(1);
      const T xi = x0[i * ldx0];
      const T bx = bi * X[i * k + c];
      a1 = fma(bx, xi, a1);
      a2 += bx;
      if (c == 0) {
        a3 = fma(bi, xi, a3);
        a4 += bi;
      }
    }
    atomicAdd(&sh[c], (double)a1);
    atomicAdd(&sh[k + c], (double)a2);
    if (c == 0) {
      atomicAdd(&sh[2 * k], (double)a3);
      atomicAdd(&sh[2 * k + 1], (double)a4);
    }
  }
  grid_colsum_last(sh, 2 * k + 2, partials, &st->counter, out, &last);
}

template <typename T>
__global__ void k_yout(const XPair<T> xs, int k, int64_t n, const double* sums, int constrain,
                       const LobState* st, T* y) {
  const T* X = xs.p[st->iter & 1];
  __shared__ T cf[LOB_KMAX + 1];
  if (threadIdx.x == 0) {
    const double ebar = constrain ? sums[2 * k] / sums[2 * k + 1] : 0.0;
    for (int c = 0; c < k; ++c) cf[c] = (T)(sums[c] - ebar * sums[k + c]);
    cf[k] = (T)ebar;
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T acc = cf[k];
    for (int c = 0; c < k; ++c) acc = fma(X[i * k + c], cf[c], acc);
    y[i] = acc;
  }
}

template <typename T>
__global__ void k_xout(const XPair<T> xs, int k, int64_t n, const LobState* st, T* out) {
  const T* X = xs.p[st->iter & 1];
  const int64_t tot = n * k;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < tot;
       q += (int64_t)gridDim.x * blockDim.x)
    out[q] = X[q];
}

__global__ void k_theta_out(const LobState* st, int k, double* theta, double* resid) {
  const int c = threadIdx.x;
  if (c < k) {
    if (theta) theta[c] = st->theta[c];
    if (resid) resid[c] = st->resid[c];
  }
}

// ------------------------------------------------------------------ host driver
template <typename T>
struct LobBuffers {
  T* X[2];
  T* AX[2];
  T* P[2];
  T* AP[2];
  T* W[2];
  T* AW;
  double* gram_part;
  double* G;
  double* C;
  double* Cp;
  double* part;       // small reductions
  double* ysums;
  LobState* st;
};

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 132;
  }
  return n;
}

template <typename T>
static int run_gram(const GramArgs<T>& ga, int grid, cudaStream_t s) {
  const int ta_n = ga.m4 / 4;
  const int nt = ta_n * (ta_n + 1) / 2;
  if (nt > GRAM_T) return bf_fail(BF_EINVAL, "lobpcg_filter: block too wide");
  const int ng = GRAM_T / nt;
  size_t sm = (size_t)(4 * GramChunk<T>::buf + 2 * GramChunk<T>::pxc) * sizeof(T);
  sm = std::max(sm, (size_t)(ng / 2 + 1) * nt * 64 * sizeof(T));
  {
    const int rc_ = bf_smem_attr((const void*)k_gram<T>, 200 * 1024, "cudaFuncSetAttribute(k_gram)");
    if (rc_) return rc_;
  }
  BF_LAUNCH_PDL(k_gram<T>, grid, GRAM_T, sm, s, ga);
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

static void run_gram_reduce(const double* partials, int nblocks, int m, double* G,
                            const LobState* st, cudaStream_t s) {
  const int threads = 2 * (m * (m + 1) / 2) * 32;
  BF_LAUNCH_PDL(k_gram_reduce, (threads + 255) / 256, 256, 0, s, partials, nblocks, m, G, st);
}

template <typename T, int CW>
static void launch_update_cw(const UpdArgs<T>& ua, int grid, cudaStream_t s) {
  const size_t sm = (size_t)(2 * ua.m * ua.k) * sizeof(T);
  const int64_t work = ua.n * (ua.k / CW);
  grid = (int)std::min<int64_t>((work + 255) / 256, (int64_t)grid);
  // a failure here shows as a failed launch, which the caller's cudaGetLastError reports
  (void)bf_smem_attr((const void*)k_update<T, CW>, 200 * 1024, "cudaFuncSetAttribute(k_update)");
  BF_LAUNCH(k_update<T, CW><<<grid, 256, sm, s>>>(ua));
}

template <int KT>
static void launch_update_f32(const UpdArgs<float>& ua, cudaStream_t s) {
  const size_t sm = (size_t)(2 * ua.m * KT) * sizeof(float);
  (void)bf_smem_attr((const void*)k_update_f32<KT>, 200 * 1024, "cudaFuncSetAttribute(k_update_f32)");
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update_f32<KT>, 256, 2 * 3 * KT * KT * sizeof(float)) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  const int grid = (int)std::min<int64_t>((ua.n + 255) / 256, (int64_t)per_sm * sm_count());
  BF_LAUNCH(k_update_f32<KT><<<grid, 256, sm, s>>>(ua));
}

template <typename T>
static int run_update(const UpdArgs<T>& ua, int grid, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (ua.k == 16 || ua.k == 8) {
      if (ua.k == 16) launch_update_f32<16>(ua, s);
      else launch_update_f32<8>(ua, s);
      BF_CUDA(cudaGetLastError());
      return BF_OK;
    }
  }
  if (ua.k % 4 == 0) launch_update_cw<T, 4>(ua, grid, s);
  else launch_update_cw<T, 1>(ua, grid, s);
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

inline int net_T(const bf_net* net, const bf_graph* g, float* W, int k, cudaStream_t s, const int* stop) {
  return bf_net_apply_f32(net, g, W, k, k, W, k, s, stop);
}
inline int net_T(const bf_net*, const bf_graph*, double*, int, cudaStream_t, const int*) {
  return bf_fail(BF_EINVAL, "lobpcg_filter: the net preconditioner needs an FP32 graph");
}
inline int spd_T(const bf_spd* T, const bf_graph* g, float* W, int k, cudaStream_t s) {
  return bf_spd_apply_f32(T, g, W, k, k, W, k, s);
}
inline int spd_T(const bf_spd*, const bf_graph*, double*, int, cudaStream_t) {
  return bf_fail(BF_EINVAL, "lobpcg_filter: the SPD preconditioner needs an FP32 graph");
}

// A X = L X, then the residual kernel: W = T (A X - B X theta) and its norms.  With a
// learned preconditioner (the net or the SPD T) the kernel writes R = A X - B X theta, T
// maps it to W = T(R) in place and the constraint coefficients e^T B W / e^T B e are
// recomputed.
template <typename T>
static int run_resid(const bf_graph* g, const T* X, T* AX, int k, T* Wn, const T* bdiag,
                     const T* tinv, int constrain, double* part, LobState* st, int rgrid,
                     cudaStream_t s, const bf_net* net = nullptr, const bf_spd* spd = nullptr) {
  int rc = apply_T<T>(g, BF_OP_L, X, k, k, AX, k, s);
  if (rc) return rc;
  const int resgrid = 4 * rgrid;                // many blocks: enough loads in flight
  BF_LAUNCH_PDL(k_resid<T>, resgrid, 256, 0, s, X, AX, k, g->n, bdiag, (net || spd) ? nullptr : tinv, Wn, part, st);
  double* cols = part + (size_t)resgrid * 3 * k;
  BF_LAUNCH_PDL(k_resid_cols, 3 * k, 256, 0, s, part, resgrid, 3 * k, cols, st);
  BF_LAUNCH_PDL(k_resid_tail, 1, 32, 0, s, cols, k, constrain, st);
  BF_CUDA(cudaGetLastError());
  if (net || spd) {
    if (net) {
      if ((rc = net_T(net, g, Wn, k, s, &st->status))) return rc;
    } else if ((rc = spd_T(spd, g, Wn, k, s))) {
      return rc;
    }
    if (constrain) BF_LAUNCH(k_bsums<T><<<rgrid, 256, 0, s>>>(Wn, k, g->n, bdiag, part, st));
    BF_CUDA(cudaGetLastError());
  }
  return BF_OK;
}

// The Gram products: FP32 kernel, or (FP32 graphs, k % 4 == 0) the tensor-core kernel in
// BF16, two-way or three-way split BF16 (the latter for m <= 48; wider bases fall back to
// the FP32 kernel).
template <typename T>
static int gram_step(const GramArgs<T>& ga, int gram_mode, int ggrid, double* part, double* G, LobState* st,
                     cudaStream_t s) {
  if (sizeof(T) == 4 && gram_mode != BF_GRAM_FP32) {
    const int rc = bf_gram_tc(reinterpret_cast<const float* const*>(ga.S), reinterpret_cast<const float* const*>(ga.AS),
                              reinterpret_cast<const float*>(ga.b), ga.nblk, ga.k, ga.n, gram_mode, part, ggrid, G,
                              &st->status, &st->status, s);
    if (rc != BF_EINVAL) return rc;
  }
  const int rc = run_gram<T>(ga, ggrid, s);
  if (rc) return rc;
  run_gram_reduce(part, ggrid, ga.m, G, st, s);
  return BF_OK;
}

template <typename T>
int lob_run(const bf_graph* g, const T* X0, int64_t ldx0, int k, int kmax,
            const bf_lobpcg_opts& o, T* X_out, double* theta_out, double* resid_out, T* y_out,
            bf_info* info, cudaStream_t s) {
  bf_graph* gm = const_cast<bf_graph*>(g);
  const int64_t n = g->n;
  const int nsm = sm_count();
  const int ggrid = nsm;                       // Gram blocks
  const int ugrid = 64 * nsm;                  // update blocks (capped by the work)
  const int rgrid = 2 * nsm;                   // reduction blocks
  const size_t blk = (((size_t)n * k * sizeof(T)) + 255) & ~(size_t)255;
  const int m3 = 3 * k;
  const size_t gpb = (((size_t)ggrid * 2 * m3 * m3 * sizeof(double)) + 255) & ~(size_t)255;
  const size_t gb = ((2 * (size_t)m3 * m3 * sizeof(double)) + 255) & ~(size_t)255;
  const size_t cb = (((size_t)m3 * k * sizeof(double)) + 255) & ~(size_t)255;
  const size_t pb = (((size_t)std::max(ugrid, rgrid) * (3 * LOB_KMAX + 2) * sizeof(double)) + 255) & ~(size_t)255;
  const size_t yb = 256 * sizeof(double) * 2;
  const size_t rrb = (sizeof(RRScratch) + 255) & ~(size_t)255;
  const size_t total = 11 * blk + gpb + gb + 2 * cb + pb + yb + rrb + 1024;
  int rc = bf_ws_reserve(gm, BF_WS_LOB, total);
  if (rc) return rc;
  char* w = (char*)gm->ws[BF_WS_LOB];
  LobBuffers<T> B;
  for (int j = 0; j < 2; ++j) {
    B.X[j] = (T*)w; w += blk;
    B.AX[j] = (T*)w; w += blk;
    B.P[j] = (T*)w; w += blk;
    B.AP[j] = (T*)w; w += blk;
    B.W[j] = (T*)w; w += blk;
  }
  B.AW = (T*)w; w += blk;
  B.gram_part = (double*)w; w += gpb;
  B.G = (double*)w; w += gb;
  B.C = (double*)w; w += cb;
  B.Cp = (double*)w; w += cb;
  B.part = (double*)w; w += pb;
  B.ysums = (double*)w; w += yb;
  RRScratch* rr_scr = (RRScratch*)w; w += rrb;
  B.st = (LobState*)w; w += 1024;

  const T* bdiag = (o.pencil == BF_PENCIL_D) ? (const T*)g->d : nullptr;
  const T* tinv = (o.precond == BF_PRECOND_JACOBI) ? (const T*)g->dinv : nullptr;

  BF_LAUNCH(k_state_init<<<1, 64, 0, s>>>(B.st, o.tol));
  XPair<T> xs;
  xs.p[0] = B.X[0];
  xs.p[1] = B.X[1];

  const int egrid = (int)std::min<int64_t>((n * k + 255) / 256, 4 * nsm);
  // ---- start block: copy, constrain, A X
  BF_LAUNCH(k_copy_block<T><<<egrid, 256, 0, s>>>(X0, ldx0, k, n, B.X[1]));
  BF_LAUNCH(k_bsums<T><<<rgrid, 256, 0, s>>>(B.X[1], k, n, bdiag, B.part, B.st));
  if (o.constrain_e) BF_LAUNCH(k_project<T><<<egrid, 256, 0, s>>>(B.X[1], k, n, B.st));
  BF_CUDA(cudaGetLastError());
  rc = apply_T<T>(g, BF_OP_L, B.X[1], k, k, B.AX[1], k, s);
  if (rc) return rc;
  // Rayleigh-Ritz on span(X0)
  GramArgs<T> ga;
  memset(&ga, 0, sizeof(ga));
  ga.b = bdiag;
  ga.k = k;
  ga.n = n;
  ga.partials = B.gram_part;
  ga.st = B.st;
  ga.nblk = 1;
  ga.S[0] = B.X[1];
  ga.AS[0] = B.AX[1];
  ga.m = k;
  ga.m4 = (k + 3) & ~3;
  rc = gram_step<T>(ga, o.gram, ggrid, B.gram_part, B.G, B.st, s);
  if (rc) return rc;
  RRParams ra;
  ra.G = B.G;
  ra.C = B.C;
  ra.Cp = nullptr;
  ra.theta = B.st->theta;
  ra.status = &B.st->status;
  ra.restarts = &B.st->restarts;
  ra.k = k;
  ra.m = k;
  ra.m_nop = 0;
  ra.theta_hist = o.theta_hist;
  ra.scr = rr_scr;
  rc = bf_rr_launch(ra, s);
  if (rc) return rc;
  UpdArgs<T> ua;
  memset(&ua, 0, sizeof(ua));
  ua.k = k;
  ua.n = n;
  ua.C = B.C;
  ua.Cp = nullptr;
  ua.st = B.st;
  ua.nblk = 1;
  ua.m = k;
  ua.S[0] = B.X[1];
  ua.Xn = B.X[0];
  ua.Pn = nullptr;
  rc = run_update<T>(ua, ugrid, s);
  if (rc) return rc;
  const bf_net* net = (o.precond == BF_PRECOND_NET) ? o.net : nullptr;
  const bf_spd* spd = (o.precond == BF_PRECOND_SPD) ? o.spd : nullptr;
  rc = run_resid<T>(g, B.X[0], B.AX[0], k, B.W[0], bdiag, tinv, o.constrain_e, B.part, B.st, rgrid, s, net, spd);
  if (rc) return rc;
  // the start step counted as one residual evaluation: iterations count from 0 after it
  BF_LAUNCH(k_state_iter0<<<1, 32, 0, s>>>(B.st));
  // ---- iterations: current copy j = it & 1, next copy 1 - j
  for (int it = 0; it < kmax; ++it) {
    const int j = it & 1, nj = 1 - j;
    if (o.constrain_e) BF_LAUNCH(k_project<T><<<egrid, 256, 0, s>>>(B.W[j], k, n, B.st));
    rc = apply_T<T>(g, BF_OP_L, B.W[j], k, k, B.AW, k, s);
    if (rc) return rc;
    const int nblk = (it == 0) ? 2 : 3;
    ga.nblk = nblk;
    ga.m = nblk * k;
    ga.m4 = (ga.m + 3) & ~3;
    ga.S[0] = B.X[j];
    ga.AS[0] = B.AX[j];
    ga.S[1] = B.W[j];
    ga.AS[1] = B.AW;
    ga.S[2] = B.P[j];
    ga.AS[2] = B.AP[j];
    rc = gram_step<T>(ga, o.gram, ggrid, B.gram_part, B.G, B.st, s);
    if (rc) return rc;
    ra.m = ga.m;
    ra.m_nop = (nblk == 3) ? 2 * k : 0;
    ra.Cp = B.Cp;
    ra.theta_hist = o.theta_hist ? o.theta_hist + (size_t)(it + 1) * k : nullptr;
    rc = bf_rr_launch(ra, s);
    if (rc) return rc;
    ua.nblk = nblk;
    ua.m = ga.m;
    for (int b2 = 0; b2 < 3; ++b2) ua.S[b2] = ga.S[b2];
    ua.Cp = B.Cp;
    ua.Xn = B.X[nj];
    ua.Pn = B.P[nj];
    rc = run_update<T>(ua, ugrid, s);
    if (rc) return rc;
    rc = apply_T<T>(g, BF_OP_L, B.P[nj], k, k, B.AP[nj], k, s);
    if (rc) return rc;
    rc = run_resid<T>(g, B.X[nj], B.AX[nj], k, B.W[nj], bdiag, tinv, o.constrain_e, B.part, B.st, rgrid, s, net,
                      spd);
    if (rc) return rc;
  }
  // ---- outputs
  if (X_out) BF_LAUNCH(k_xout<T><<<egrid, 256, 0, s>>>(xs, k, n, B.st, X_out));
  if (theta_out || resid_out) BF_LAUNCH(k_theta_out<<<1, 32, 0, s>>>(B.st, k, theta_out, resid_out));
  if (y_out) {
    BF_LAUNCH(k_ysums<T><<<rgrid, 256, 0, s>>>(xs, k, n, X0, ldx0, bdiag, B.part, B.st, B.ysums));
    BF_LAUNCH(k_yout<T><<<egrid, 256, 0, s>>>(xs, k, n, B.ysums, o.constrain_e, B.st, y_out));
  }
  BF_CUDA(cudaGetLastError());
  if (info) {
    LobState h;
    BF_CUDA(cudaMemcpyAsync(&h, B.st, sizeof(h), cudaMemcpyDeviceToHost, s));
    BF_CUDA(cudaStreamSynchronize(s));
    info->iters = h.iter;
    info->status = h.status == LOB_CONV ? BF_CG_CONVERGED : (h.status == LOB_BREAK ? BF_CG_BREAKDOWN : 0);
    info->restarts = h.restarts;
    info->reserved = 0;
    double mx = 0.0;
    for (int c = 0; c < k; ++c) mx = std::max(mx, h.resid[c]);
    info->rnorm = mx;
    info->ref = 0.0;
    if (h.status == LOB_BREAK) return bf_fail(BF_EBREAKDOWN, "lobpcg_filter: dependent trial basis");
    if (h.status == LOB_NONFINITE) return bf_fail(BF_ENONFINITE, "lobpcg_filter: non-finite value");
    if (h.status == LOB_TIMEOUT) return bf_fail(BF_ETIMEOUT, "lobpcg_filter: a bounded wait of the Gram kernel gave up");
  }
  return BF_OK;
}

}  // namespace

extern "C" int lobpcg_filter(const bf_graph* g, const void* X0, int64_t ldx0, int k, int kmax,
                             const bf_lobpcg_opts* opts, void* X_out, double* theta_out,
                             double* resid_out, void* y_out, bf_info* info, void* stream) {
  if (!g || !X0) return bf_fail(BF_EINVAL, "lobpcg_filter: NULL argument");
  if (k < 1 || k > LOB_KMAX) return bf_fail(BF_EINVAL, "lobpcg_filter: need 1 <= k <= 32");
  if ((int64_t)3 * k > g->n) return bf_fail(BF_EINVAL, "lobpcg_filter: need 3k <= n");
  if (kmax < 0 || ldx0 < k) return bf_fail(BF_EINVAL, "lobpcg_filter: need kmax >= 0 and ldx0 >= k");
  bf_lobpcg_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.pencil != BF_PENCIL_D && o.pencil != BF_PENCIL_I) return bf_fail(BF_EINVAL, "lobpcg_filter: bad pencil");
  if (o.precond != BF_PRECOND_JACOBI && o.precond != BF_PRECOND_IDENTITY && o.precond != BF_PRECOND_NET &&
      o.precond != BF_PRECOND_SPD)
    return bf_fail(BF_EINVAL, "lobpcg_filter: bad precond");
  if (o.precond == BF_PRECOND_NET && (!o.net || g->esize != 4 || g->kind != BF_KIND_BILATERAL))
    return bf_fail(BF_EINVAL, "lobpcg_filter: BF_PRECOND_NET needs a net and an FP32 bilateral graph");
  if (o.precond == BF_PRECOND_SPD && (!o.spd || g->esize != 4 || g->kind != BF_KIND_BILATERAL))
    return bf_fail(BF_EINVAL, "lobpcg_filter: BF_PRECOND_SPD needs a bf_spd and an FP32 bilateral graph");
  if (!(o.tol >= 0.0)) return bf_fail(BF_EINVAL, "lobpcg_filter: tol must be >= 0");
  if (o.gram != BF_GRAM_FP32 && o.gram != BF_GRAM_BF16 && o.gram != BF_GRAM_BF16X3 && o.gram != BF_GRAM_BF16X6)
    return bf_fail(BF_EINVAL, "lobpcg_filter: bad gram mode");
  cudaStream_t s = (cudaStream_t)stream;
  if (g->esize == 4)
    return lob_run<float>(g, (const float*)X0, ldx0, k, kmax, o, (float*)X_out, theta_out, resid_out,
                          (float*)y_out, info, s);
  return lob_run<double>(g, (const double*)X0, ldx0, k, kmax, o, (double*)X_out, theta_out, resid_out,
                         (double*)y_out, info, s);
}
