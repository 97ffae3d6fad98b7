// The small Rayleigh-Ritz problem of block LOBPCG (Algorithm 3, Section 6): the k smallest
// eigenpairs of the pencil (G_A, G_B) of size m <= 96, solved by one CTA.
//
// On GB300 FP64 runs at about 2 FMA/clk per SM with a 64-cycle dependent latency, while
// FP32 runs at 128 FMA/clk with a 4-cycle latency.  The solver therefore keeps FP64 for
// the steps whose accuracy decides the result and does the O(m^3) eigen-decomposition in
// FP32, then restores FP64 accuracy with one residual correction:
//   1. symmetrise, scale to unit diag(G_B), right-looking Cholesky G_B = R R^T carrying
//      the forward solve Y = R^-1 G_A along (a squared pivot <= 1e-10 means a dependent
//      trial basis: retry on the leading m_nop block, i.e. without P, else breakdown);
//   2. standard form M = Y R^-T (FP64, lower triangle);
//   3. FP32 eigenpairs (lambda_i, v_i) of float(M): Householder reduction to tridiagonal
//      form, then one warp per eigenpair (a kernel of its own, so the eigenpairs run on
//      many SMs): its eigenvalue by multisection on Sturm counts, its eigenvector by
//      inverse iteration and back-transformation; modified Gram-Schmidt inside clusters;
//   4. X = the eigenvectors of the k smallest lambda and of the unwanted ones chained to
//      the k-th closer than the FP32 resolution 64 eps_32 |M| (kk <= 32 in all), Y = M X in
//      FP64, Rayleigh quotients theta_j and the FP64 residual r_j = y_j - theta_j x_j;
//   5. first-order correction x_j += sum_i v_i (v_i^T r_j) / (theta_j - lambda_i) over the
//      unwanted eigenpairs outside a 64 eps_32 |M| neighbourhood of theta_j (FP32 products
//      of FP64 data; the error of the corrected vectors is second order in the FP32 one);
//   6. symmetric orthonormalisation T = (X^T X)^-1/2 = I + D, D = -E/2 + 3E^2/8 for
//      X^T X = I + E, H = T (X^T M X) T in FP64, cyclic Jacobi on the kk x kk H in FP64,
//      the k smallest of its eigenvalues kept (so a cluster across the k-th eigenvalue is
//      split in FP64, not by the FP32 ordering);
//   7. C = R^-T X T Q with the scaling undone; with Cp requested, the coefficients of the
//      next P made B-orthogonal to the next X (see the driver).
// Reciprocals and square roots use an FP32 seed refined by two FP64 Newton steps
// (rounding-level accuracy), avoiding the long FP64 divide and square-root sequences.
#include <math.h>

#include "bf_internal.cuh"
#include "bf_rr.cuh"

#define RR_T 512
#define RR_KLD 33           // padded leading dimension of the m x k work matrices
#define DEP_TOL 1e-10

namespace {

// 1/x and 1/sqrt(x) from an FP32 seed (relative error < 2^-22) and two Newton steps, each
// of which squares the relative error; values outside the FP32 range take the exact path.
__device__ __forceinline__ double frcp(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ double frsqrt(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
  const double h = 0.5 * x;
  y = y * fma(-h, y * y, 1.5);
  return y * fma(-h, y * y, 1.5);
}

// Number of eigenvalues of the symmetric tridiagonal T (diagonal d, squared off-diagonal
// e2) smaller than x: negative pivots of the LDL^T factorisation of T - x I,
// q_0 = d_0 - x, q_i = (d_i - x) - e2_{i-1} / q_{i-1} (the ratio form of the Sturm
// sequence: no over- or underflow to rescale).  A pivot smaller than pivmin in magnitude
// is replaced by -pivmin.
__device__ int sturm_count_f(const float* d, const float* e2, int m, float x, float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = (q < 0.0f);
  float dn = (m > 1) ? d[1] : 0.0f, en = e2[0];   // operands of the next step, loaded ahead
  for (int i = 1; i < m; ++i) {
    const float di = dn, ei = en;
    if (i + 1 < m) {
      dn = d[i + 1];
      en = e2[i];
    }
    q = (di - x) - __fdividef(ei, q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += (q < 0.0f);
  }
  return cnt;
}

// Inverse iteration on T - lambda I (FP32): elimination with row interchanges (the
// working row, entries in columns i, i+1, i+2, against the next original row; the larger
// entry in column i pivots; zero pivots become `tiny`), then `reps` solves from the start
// vector b, each normalised by its largest entry.
// f, ri, u1, u2, sw: work arrays of m entries (shared memory).
__device__ void tri_inverse_iteration(const float* d, const float* e, int m, float lambda, float tiny,
                                      int reps, float* b, float* f, float* ri, float* u1, float* u2,
                                      unsigned char* sw) {
  float r0 = d[0] - lambda, r1 = (m > 1) ? e[0] : 0.0f, r2 = 0.0f;
  for (int i = 0; i < m - 1; ++i) {
    const float n0 = e[i], n1 = d[i + 1] - lambda, n2 = (i + 2 < m) ? e[i + 1] : 0.0f;
    const bool keep = fabsf(r0) >= fabsf(n0);
    float p0 = keep ? r0 : n0;
    const float p1 = keep ? r1 : n1, p2 = keep ? r2 : n2;
    const float o0 = keep ? n0 : r0, o1 = keep ? n1 : r1, o2 = keep ? n2 : r2;
    if (p0 == 0.0f) p0 = tiny;
    const float rp = __fdividef(1.0f, p0);
    const float fi = o0 * rp;
    f[i] = fi;
    sw[i] = keep ? 0 : 1;
    ri[i] = rp;
    u1[i] = p1;
    u2[i] = p2;
    r0 = fmaf(-fi, p1, o1);
    r1 = fmaf(-fi, p2, o2);
    r2 = 0.0f;
  }
  if (r0 == 0.0f) r0 = tiny;
  ri[m - 1] = __fdividef(1.0f, r0);
  u1[m - 1] = 0.0f;
  u2[m - 1] = 0.0f;
  for (int rep = 0; rep < reps; ++rep) {
    float rb = b[0];
    for (int i = 0; i < m - 1; ++i) {
      const float nb = b[i + 1];
      const float pb = sw[i] ? nb : rb, ob = sw[i] ? rb : nb;
      b[i] = pb;
      rb = fmaf(-f[i], pb, ob);
    }
    float x2 = rb * ri[m - 1], x1 = x2;              // b[i + 2], b[i + 1] carried in registers
    b[m - 1] = x2;
    if (m > 1) {
      x1 = fmaf(-u1[m - 2], x2, b[m - 2]) * ri[m - 2];
      b[m - 2] = x1;
    }
    for (int i = m - 3; i >= 0; --i) {
      const float x0 = fmaf(-u2[i], x2, fmaf(-u1[i], x1, b[i])) * ri[i];
      b[i] = x0;
      x2 = x1;
      x1 = x0;
    }
    float nrm = 0.0f;
    for (int i = 0; i < m; ++i) nrm = fmaxf(nrm, fabsf(b[i]));
    const float inv = (nrm > 0.0f && isfinite(nrm)) ? __fdividef(1.0f, nrm) : 1.0f;
    for (int i = 0; i < m; ++i) b[i] *= inv;
  }
}

// Round-robin pairing of np (even) indices: in step s (0 <= s < np - 1) pair i (i < np / 2)
// joins s + i and s - i (mod np - 1), pair 0 joins s with the fixed index np - 1.
__device__ __forceinline__ void jacobi_pair_k(int step, int i, int np, int& p, int& q) {
  const int n1 = np - 1;
  if (i == 0) {
    p = step;
    q = n1;
  } else {
    p = step + i;
    if (p >= n1) p -= n1;
    q = step - i;
    if (q < 0) q += n1;
  }
  if (p > q) { const int t = p; p = q; q = t; }
}

// q / d for q < 2^32 / d by a multiply-high with ceil(2^32 / d)
struct FastDiv {
  unsigned d, inv;
  __device__ explicit FastDiv(unsigned dd) : d(dd), inv(dd > 1 ? 0xFFFFFFFFu / dd + 1u : 0u) {}
  __device__ __forceinline__ unsigned div(unsigned q) const { return d > 1 ? __umulhi(q, inv) : q; }
};

// lower-stored symmetric matrix
__device__ __forceinline__ double symv(const double* A, int r, int c) {
  return (c <= r) ? A[r * RR_LD + c] : A[c * RR_LD + r];
}

// Lane layout for outputs with at most 32 columns: a warp covers 32 >> sh rows of 1 << sh
// columns (1 << sh >= ncol), so index arithmetic needs shifts and masks only.
struct Tiling {
  int sh, rows, lr, lc;
  __device__ Tiling(int ncol, int lane) {
    sh = (ncol <= 1) ? 0 : 32 - __clz(ncol - 1);
    rows = 32 >> sh;
    lr = lane >> sh;
    lc = lane & ((1 << sh) - 1);
  }
};
#define RR_NW (RR_T / 32)
// for (r, c) in [0, nrow) x [0, ncol) with the tiling t (warp w, RR_NW warps)
#define FOR_RC(t, nrow, ncol, w)                                            \
  for (int r0_ = (w) * (t).rows; r0_ < (nrow); r0_ += RR_NW * (t).rows)  \
    for (int r = r0_ + (t).lr, c = (t).lc; r < (nrow) && c < (ncol); r = (nrow))

// Y = M X (FP64), M lower-stored, X and Y [m][RR_KLD]
__device__ void mul_mx(const double* MA, const double* X, double* Y, int m, const Tiling& tk, int k,
                       int wid) {
  FOR_RC(tk, m, k, wid) {
    double s0 = 0.0, s1 = 0.0;
    int cc = 0;
    for (; cc + 1 <= r; cc += 2) {
      s0 = fma(MA[r * RR_LD + cc], X[cc * RR_KLD + c], s0);
      s1 = fma(MA[r * RR_LD + cc + 1], X[(cc + 1) * RR_KLD + c], s1);
    }
    for (; cc < m; ++cc) s0 = fma(MA[cc * RR_LD + r], X[cc * RR_KLD + c], s0);
    Y[r * RR_KLD + c] = s0 + s1;
  }
}

// Part 1 (one CTA): scaling, Cholesky with the forward solve, standard form, FP32
// tridiagonal reduction; hands M, R, T and the reflectors to the next kernels.
__global__ void __launch_bounds__(RR_T) k_rr_reduce(const RRParams a) {
  bf_pdl_enter();
  if (*a.status != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double* MA = reinterpret_cast<double*>(smem);           // [96][RR_LD]: A, Y, M (lower) + R^T (upper)
  double* RB = MA + RR_MMAX * RR_LD;                      // [96][RR_LD]: B, R (lower); then FP32 J, V
  double* XD = RB + RR_MMAX * RR_LD;                      // [96][RR_KLD]: X, X'
  double* YD = XD + RR_MMAX * RR_KLD;                     // [96][RR_KLD]: M X, M X', Z, C
  double* sc = YD + RR_MMAX * RR_KLD;                     // [96] unit-diagonal scaling
  double* rdg = sc + RR_MMAX;                             // [96] 1 / diag(R)
  double* fv = rdg + RR_MMAX;                             // [2][96] multipliers (by step parity)
  double* th = fv + 2 * RR_MMAX;                          // [32] Rayleigh quotients
  double* csd = th + RR_KMAX;                             // [16] k x k rotations
  double* snd = csd + RR_KMAX / 2;                        // [16]
  float* lam = reinterpret_cast<float*>(snd + RR_KMAX / 2);  // [96] FP32 eigenvalues of M
  float* dd32 = lam + RR_MMAX;                            // [96] tridiagonal: diagonal
  float* ee32 = dd32 + RR_MMAX;                           // [96] off-diagonal
  float* e2f = ee32 + RR_MMAX;                            // [96] squared off-diagonal
  float* bet32 = e2f + RR_MMAX;                           // [96] reflector scalars
  float* pv32 = bet32 + RR_MMAX;                          // [96] work vector
  int* sel = reinterpret_cast<int*>(pv32 + RR_MMAX);      // [32]
  int* perm = sel + RR_KMAX;                              // [32]
  int* rk = perm + RR_KMAX;                               // [96] rank of each FP32 eigenvalue
  int* pp = rk + RR_MMAX;                                 // [48] pairs of one Jacobi step
  int* qq = pp + RR_MMAX / 2;                             // [48]
  // lower triangle of order 96 in row-major order: entry (r, l), l <= r, packed r << 8 | l;
  // every smaller triangle is a prefix of it
  unsigned short* tri = reinterpret_cast<unsigned short*>(qq + RR_MMAX / 2);  // [4656]
  // FP32 view of the RB region once R has been moved out of it (37,248 B): float(M),
  // then T and the reflectors
  float* J = reinterpret_cast<float*>(RB);                // [96][RR_LDF]
  __shared__ int fail, dropped;
  __shared__ float shlo, shhi;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int k = a.k;
  const Tiling tk(k, lane);
  int m = a.m;
  if (tid == 0) dropped = 0;
  for (int r = wid; r < a.m; r += RR_NW)
    for (int l = lane; l <= r; l += 32) tri[r * (r + 1) / 2 + l] = (unsigned short)((r << 8) | l);

  // ------------------------------------------ 1-2. scale, Cholesky with the forward solve
  for (int attempt = 0; attempt < 2; ++attempt) {
    const FastDiv fdv(m);
    __syncthreads();
    for (int r = wid; r < m; r += RR_NW)
      for (int c = lane; c < m; c += 32) {
        MA[r * RR_LD + c] = 0.5 * (a.G[r * a.m + c] + a.G[c * a.m + r]);
        RB[r * RR_LD + c] = 0.5 * (a.G[a.m * a.m + r * a.m + c] + a.G[a.m * a.m + c * a.m + r]);
      }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int r = tid; r < m; r += RR_T) {
      const double dg = RB[r * RR_LD + r];
      if (!(dg > 0.0) || !isfinite(dg)) fail = 1;
      sc[r] = (dg > 0.0) ? frsqrt(dg) : 0.0;
    }
    __syncthreads();
    if (!fail) {
      for (int r = wid; r < m; r += RR_NW)
        for (int c = lane; c < m; c += 32) {
          const double s2 = sc[r] * sc[c];
          MA[r * RR_LD + c] *= s2;
          RB[r * RR_LD + c] *= s2;
        }
      __syncthreads();
      // Right-looking Cholesky B = R R^T with unscaled columns c (R(:, j) = c / sqrt(piv)),
      // carrying the forward solve Y = R^-1 A along: both updates use f_i = c_i / piv.
      // Look-ahead: in step j warp 0 updates column j + 1 and forms the multipliers of step
      // j + 1 (the serial reciprocal chain) while the other warps update the rest, so each
      // step ends in one barrier.  fv holds two multiplier buffers, by step parity.
      if (wid == 0 && RB[0] > DEP_TOL) {
        const double ip = frcp(RB[0]);
        for (int i = 1 + lane; i < m; i += 32) fv[i] = RB[i * RR_LD] * ip;
      }
      __syncthreads();
      for (int j = 0; j < m; ++j) {
        if (!(RB[j * RR_LD + j] > DEP_TOL)) break;       // same value in every thread
        const double* fj = fv + (j & 1) * RR_MMAX;
        const int t = m - j - 1;
        if (wid == 0) {
          if (t > 0) {                                   // column j + 1, then step j + 1's f
            for (int i = j + 1 + lane; i < m; i += 32)
              RB[i * RR_LD + j + 1] = fma(-fj[i], RB[(j + 1) * RR_LD + j], RB[i * RR_LD + j + 1]);
            __syncwarp();
            const double piv = RB[(j + 1) * RR_LD + j + 1];
            if (piv > DEP_TOL) {
              const double ip = frcp(piv);
              double* fn = fv + ((j + 1) & 1) * RR_MMAX;
              for (int i = j + 2 + lane; i < m; i += 32) fn[i] = RB[i * RR_LD + j + 1] * ip;
            }
          }
        } else {
          const int t2 = t - 1, nb = t2 > 0 ? t2 * (t2 + 1) / 2 : 0;
          for (int q = tid - 32; q < nb + t * m; q += RR_T - 32) {
            if (q < nb) {                                // trailing B: j + 1 < l <= i < m
              const int e = tri[q], i = j + 2 + (e >> 8), l = j + 2 + (e & 255);
              RB[i * RR_LD + l] = fma(-fj[i], RB[l * RR_LD + j], RB[i * RR_LD + l]);
            } else {                                     // rows i > j of Y
              const int q2 = q - nb, i1 = (int)fdv.div((unsigned)q2), c = q2 - i1 * m, i = j + 1 + i1;
              MA[i * RR_LD + c] = fma(-fj[i], MA[j * RR_LD + c], MA[i * RR_LD + c]);
            }
          }
        }
        __syncthreads();
      }
      for (int j = tid; j < m; j += RR_T) {
        const double piv = RB[j * RR_LD + j];
        if (!(piv > DEP_TOL)) fail = 1;
        rdg[j] = (piv > 0.0) ? frsqrt(piv) : 0.0;
      }
      __syncthreads();
    }
    if (!fail) break;
    if (attempt == 0 && a.m_nop > 0 && a.m_nop < a.m) {
      m = a.m_nop;
      if (tid == 0) dropped = 1;
      continue;
    }
    if (tid == 0) *a.status = 2;
    return;
  }
  for (int i = wid; i < m; i += RR_NW)              // R(i, c) = c_i rdg_c, Y(i, :) *= rdg_i
    for (int c = lane; c < m; c += 32) {
      if (c < i) RB[i * RR_LD + c] *= rdg[c];
      MA[i * RR_LD + c] *= rdg[i];
    }
  __syncthreads();

  // ------------------------------------------ 3. M = Y R^-T (lower triangle), columns in order
  // Look-ahead as in the Cholesky: in step i warp 0 updates and finalises column i + 1
  // (the multipliers of step i + 1) while the other warps update columns i + 2 ...
  if (wid == 0)
    for (int r = lane; r < m; r += 32) {
      const double v = MA[r * RR_LD] * rdg[0];      // final M(r, 0)
      MA[r * RR_LD] = v;
      fv[r] = v;
    }
  __syncthreads();
  for (int i = 0; i + 1 < m; ++i) {
    const double* fi = fv + (i & 1) * RR_MMAX;
    if (wid == 0) {
      double* fn = fv + ((i + 1) & 1) * RR_MMAX;
      const double rl = RB[(i + 1) * RR_LD + i];
      for (int r = i + 1 + lane; r < m; r += 32) {
        const double v = fma(-fi[r], rl, MA[r * RR_LD + i + 1]) * rdg[i + 1];   // final M(r, i + 1)
        MA[r * RR_LD + i + 1] = v;
        fn[r] = v;
      }
    } else {
      const int t2 = m - i - 2;
      for (int q = tid - 32; q < t2 * (t2 + 1) / 2; q += RR_T - 32) {   // i + 1 < l <= r < m
        const int e = tri[q], r = i + 2 + (e >> 8), l = i + 2 + (e & 255);
        MA[r * RR_LD + l] = fma(-fi[r], RB[l * RR_LD + i], MA[r * RR_LD + l]);
      }
    }
    __syncthreads();
  }
  for (int r = wid; r < m; r += RR_NW)              // strict upper of MA <- R^T
    for (int c = r + 1 + lane; c < m; c += 32) MA[r * RR_LD + c] = RB[c * RR_LD + r];
  __syncthreads();

  // ------------------------------------------ 4. FP32 eigen-decomposition of M
  // 4a. Householder reduction of float(M) (full storage in J) to a tridiagonal T; the
  //     reflector vectors stay below the subdiagonal of J.  Look-ahead: in step j warp 0
  //     updates column j + 1 first and forms the reflector of step j + 1 while the other
  //     warps update the rest of the trailing block; K = beta v^T p / 2 is summed by every
  //     warp itself (the same lanes and order, so the same value).  Two barriers per step.
  for (int r = wid; r < m; r += RR_NW)
    for (int c = lane; c < m; c += 32) J[r * RR_LDF + c] = (float)symv(MA, r, c);
  __syncthreads();
  // reflector of column j (warp 0): x = J(j+1:m, j) -> v = x - alpha e_1, beta = 2 / v^T v
  auto reflector = [&](int j) {
    const int n1 = m - j - 1;
    float* col = J + (j + 1) * RR_LDF + j;
    float s = 0.0f;
    for (int i = lane; i < n1; i += 32) s = fmaf(col[i * RR_LDF], col[i * RR_LDF], s);
    s = warp_sum(s);
    if (lane == 0) {
      const float x0 = col[0];
      const float tail = s - x0 * x0;
      float al = x0, be = 0.0f;
      if (tail > 0.0f) {
        const float nrm = sqrtf(s);
        al = (x0 >= 0.0f) ? -nrm : nrm;
        const float v0 = x0 - al;
        be = 2.0f / fmaf(v0, v0, tail);
        col[0] = v0;
      }
      dd32[j] = J[j * RR_LDF + j];
      ee32[j] = al;
      bet32[j] = be;
    }
  };
  if (m >= 3 && wid == 0) reflector(0);
  __syncthreads();
  for (int j = 0; j + 2 < m; ++j) {
    const int n1 = m - j - 1;
    const bool next = (j + 3 < m);
    const float beta = bet32[j];
    float* col = J + (j + 1) * RR_LDF + j;          // v_i = col[i * RR_LDF], i < n1
    float* A1 = J + (j + 1) * RR_LDF + (j + 1);      // trailing n1 x n1 block
    if (beta == 0.0f) {                              // nothing to reflect: next column as is
      if (next && wid == 0) reflector(j + 1);
      __syncthreads();
      continue;
    }
    // p = beta A1 v: a warp takes rows r, r + RR_NW, r + 2 RR_NW together, so that their
    // shuffle reductions are independent and overlap
    for (int r = wid; r < n1; r += 3 * RR_NW) {
      const int r1 = r + RR_NW, r2 = r + 2 * RR_NW;
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
      for (int c = lane; c < n1; c += 32) {
        const float vc = col[c * RR_LDF];
        s0 = fmaf(A1[r * RR_LDF + c], vc, s0);
        if (r1 < n1) s1 = fmaf(A1[r1 * RR_LDF + c], vc, s1);
        if (r2 < n1) s2 = fmaf(A1[r2 * RR_LDF + c], vc, s2);
      }
      s0 = warp_sum(s0);
      s1 = warp_sum(s1);
      s2 = warp_sum(s2);
      if (lane == 0) {
        pv32[r] = beta * s0;
        if (r1 < n1) pv32[r1] = beta * s1;
        if (r2 < n1) pv32[r2] = beta * s2;
      }
    }
    __syncthreads();
    float K = 0.0f;
    for (int i = lane; i < n1; i += 32) K = fmaf(col[i * RR_LDF], pv32[i], K);
    K = 0.5f * beta * warp_sum(K);
    if (wid == 0) {                                   // column j + 1 of J, then its reflector
      const float v0 = col[0], w0 = fmaf(-K, v0, pv32[0]);
      for (int r = lane; r < n1; r += 32) {
        const float vr = col[r * RR_LDF], wr = fmaf(-K, vr, pv32[r]);
        A1[r * RR_LDF] = fmaf(-vr, w0, fmaf(-wr, v0, A1[r * RR_LDF]));
      }
      __syncwarp();
      if (next) reflector(j + 1);
    } else {                                          // A1(1:, 1:) -= v w^T + w v^T, w = p - K v
      for (int r = wid; r < n1; r += RR_NW - 1) {     // rows 1 .. n1-1 over warps 1 .. RR_NW-1
        const float vr = col[r * RR_LDF], wr = fmaf(-K, vr, pv32[r]);
        for (int c = 1 + lane; c < n1; c += 32) {
          const float vc = col[c * RR_LDF], wc = fmaf(-K, vc, pv32[c]);
          A1[r * RR_LDF + c] = fmaf(-vr, wc, fmaf(-wr, vc, A1[r * RR_LDF + c]));
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      dd32[m - 2] = J[(m - 2) * RR_LDF + (m - 2)];
      ee32[m - 2] = J[(m - 1) * RR_LDF + (m - 2)];
      bet32[m - 2] = 0.0f;
    }
    dd32[m - 1] = J[(m - 1) * RR_LDF + (m - 1)];
    ee32[m - 1] = 0.0f;
    float lo = 3e38f, hi = -3e38f;                  // Gershgorin interval
    for (int i = 0; i < m; ++i) {
      const float rad = fabsf(ee32[i]) + (i > 0 ? fabsf(ee32[i - 1]) : 0.0f);
      lo = fminf(lo, dd32[i] - rad);
      hi = fmaxf(hi, dd32[i] + rad);
    }
    shlo = lo;
    shhi = hi;
  }
  __syncthreads();
  for (int i = tid; i < m; i += RR_T) e2f[i] = ee32[i] * ee32[i];
  __syncthreads();
  RRScratch* S = a.scr;
  for (int r = wid; r < m; r += RR_NW)
    for (int c = lane; c < m; c += 32) {
      S->MA[r * RR_LD + c] = MA[r * RR_LD + c];
      S->J[r * RR_LDF + c] = J[r * RR_LDF + c];
    }
  for (int i = tid; i < m; i += RR_T) {
    S->sc[i] = sc[i];
    S->rdg[i] = rdg[i];
    S->dd[i] = dd32[i];
    S->ee[i] = ee32[i];
    S->e2[i] = e2f[i];
    S->bet[i] = bet32[i];
  }
  if (tid == 0) {
    S->lo = shlo;
    S->hi = shhi;
    S->tn = fmaxf(fabsf(shlo), fabsf(shhi));
    S->m = m;
    S->dropped = dropped;
  }
}

// Part 2 (one warp per eigenpair j of T): the j-th eigenvalue by multisection on Sturm
// counts (32 points per round), its eigenvector by three steps of inverse iteration, then
// the back-transformation by the reflectors; writes column j of V.
__global__ void __launch_bounds__(32) k_rr_vectors(const RRParams a) {
  bf_pdl_enter();
  if (*a.status != 0) return;
  RRScratch* S = a.scr;
  const int m = S->m, j = blockIdx.x, lane = threadIdx.x;
  if (j >= m) return;
  __shared__ float dd[RR_MMAX], ee[RR_MMAX], e2[RR_MMAX], v[RR_MMAX], bet[RR_MMAX];
  __shared__ float f[RR_MMAX], ri[RR_MMAX], u1[RR_MMAX], u2[RR_MMAX];
  __shared__ unsigned char sw[RR_MMAX];
  // reflector vectors, transposed: Jt[c * RR_LDF + r] = J(r, c) for r > c + 1 (J(c + 1, c)
  // holds v_0); staged by all lanes with their loads in flight together, since J was
  // written by the previous kernel and every read of it from L2 costs hundreds of cycles
  __shared__ float Jt[(RR_MMAX - 2) * RR_LDF];
  for (int i = lane; i < m; i += 32) {
    dd[i] = S->dd[i];
    ee[i] = S->ee[i];
    e2[i] = S->e2[i];
    bet[i] = S->bet[i];
  }
  {
    const int tot = m * m;
    for (int q0 = 0; q0 < tot; q0 += 36 * 32) {      // m <= 48: two batches of loads
      float val[36];
#pragma unroll
      for (int u = 0; u < 36; ++u) {
        const int q = q0 + u * 32 + lane;
        const int r = q / m, c = q - r * m;
        val[u] = (q < tot && c + 1 <= r && c + 2 < m) ? S->J[r * RR_LDF + c] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 36; ++u) {
        const int q = q0 + u * 32 + lane;
        const int r = q / m, c = q - r * m;
        if (q < tot && c + 1 <= r && c + 2 < m) Jt[c * RR_LDF + r] = val[u];
      }
    }
  }
  __syncwarp();
  const float tn = S->tn;
  float lo = S->lo, hi = S->hi;
  lo -= 1e-6f * fabsf(lo) + 1e-30f;
  hi += 1e-6f * fabsf(hi) + 1e-30f;
  const float stop = 4.0f * 6e-8f * tn + 1e-30f;
  // pivots below this are replaced: |e2 / pivmin| stays finite for |T| < 2^12
  const float pivmin = 0x1p-100f * fmaxf(1.0f, tn * tn);
  for (int round = 0; round < 10 && hi - lo > stop; ++round) {
    const float w = (hi - lo) * (1.0f / 33.0f);
    const float x = lo + w * (float)(lane + 1);
    const unsigned above = __ballot_sync(0xffffffffu, sturm_count_f(dd, e2, m, x, pivmin) > j);
    const int first = above ? __ffs(above) - 1 : 32;     // first point with more than j below
    const float nlo = (first == 0) ? lo : lo + w * (float)first;
    const float nhi = (first == 32) ? hi : lo + w * (float)(first + 1);
    lo = nlo;
    hi = nhi;
  }
  const float lamj = 0.5f * (lo + hi);
  // start vectors differ per index, so a cluster's vectors span the cluster's subspace
  for (int i = lane; i < m; i += 32) v[i] = 1.0f + 0.25f * (float)(((i + 1) * (j + 3) * 7919) % 97) / 97.0f;
  __syncwarp();
  if (lane == 0) {
    S->lam[j] = lamj;
    tri_inverse_iteration(dd, ee, m, lamj, 4.0f * 6e-8f * tn + 1e-30f, 3, v, f, ri, u1, u2, sw);
  }
  __syncwarp();
  // back-transformation by the reflectors (last first): the vector stays in registers
  // (entry i in lane i % 32, slot i / 32) and the next reflector column is loaded ahead,
  // so each reflector costs one FMA, one shuffle reduction and one FMA on the chain
  float vr[3], cn[3];
#pragma unroll
  for (int s3 = 0; s3 < 3; ++s3) {
    const int i = lane + 32 * s3;
    vr[s3] = (i < m) ? v[i] : 0.0f;
    cn[s3] = (m >= 3 && i > m - 3 && i < m) ? Jt[(m - 3) * RR_LDF + i] : 0.0f;
  }
  for (int jj = m - 3; jj >= 0; --jj) {
    float cj[3];
#pragma unroll
    for (int s3 = 0; s3 < 3; ++s3) {
      cj[s3] = cn[s3];
      const int i = lane + 32 * s3;
      cn[s3] = (jj >= 1 && i > jj - 1 && i < m) ? Jt[(jj - 1) * RR_LDF + i] : 0.0f;
    }
    const float beta = bet[jj];
    if (beta == 0.0f) continue;
    float sum = 0.0f;
#pragma unroll
    for (int s3 = 0; s3 < 3; ++s3) sum = fmaf(cj[s3], vr[s3], sum);   // cj is 0 outside rows jj+1 .. m-1
    sum = beta * warp_sum(sum);
#pragma unroll
    for (int s3 = 0; s3 < 3; ++s3) vr[s3] = fmaf(-cj[s3], sum, vr[s3]);
  }
#pragma unroll
  for (int s3 = 0; s3 < 3; ++s3) {
    const int i = lane + 32 * s3;
    if (i < m) S->V[i * RR_LDF + j] = vr[s3];
  }
}

// Part 3 (one CTA): Gram-Schmidt inside clusters (on the back-transformed vectors, which
// is the same as before it: the transformation is orthogonal), the FP64 correction, the
// k x k Rayleigh-Ritz and the coefficients C (and Cp).
__global__ void __launch_bounds__(RR_T) k_rr(const RRParams a) {
  bf_pdl_enter();
  if (*a.status != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double* MA = reinterpret_cast<double*>(smem);           // [96][RR_LD]: A, Y, M (lower) + R^T (upper)
  double* RB = MA + RR_MMAX * RR_LD;                      // [96][RR_LD]: B, R (lower); then FP32 J, V
  double* XD = RB + RR_MMAX * RR_LD;                      // [96][RR_KLD]: X, X'
  double* YD = XD + RR_MMAX * RR_KLD;                     // [96][RR_KLD]: M X, M X', Z, C
  double* sc = YD + RR_MMAX * RR_KLD;                     // [96] unit-diagonal scaling
  double* rdg = sc + RR_MMAX;                             // [96] 1 / diag(R)
  double* fv = rdg + RR_MMAX;                             // [2][96] multipliers (by step parity)
  double* th = fv + 2 * RR_MMAX;                          // [32] Rayleigh quotients
  double* csd = th + RR_KMAX;                             // [16] k x k rotations
  double* snd = csd + RR_KMAX / 2;                        // [16]
  float* lam = reinterpret_cast<float*>(snd + RR_KMAX / 2);  // [96] FP32 eigenvalues of M
  float* dd32 = lam + RR_MMAX;                            // [96] tridiagonal: diagonal
  float* ee32 = dd32 + RR_MMAX;                           // [96] off-diagonal
  float* e2f = ee32 + RR_MMAX;                            // [96] squared off-diagonal
  float* bet32 = e2f + RR_MMAX;                           // [96] reflector scalars
  float* pv32 = bet32 + RR_MMAX;                          // [96] work vector
  int* sel = reinterpret_cast<int*>(pv32 + RR_MMAX);      // [32]
  int* perm = sel + RR_KMAX;                              // [32]
  int* rk = perm + RR_KMAX;                               // [96] rank of each FP32 eigenvalue
  int* pp = rk + RR_MMAX;                                 // [48] pairs of one Jacobi step
  int* qq = pp + RR_MMAX / 2;                             // [48]
  // lower triangle of order 96 in row-major order: entry (r, l), l <= r, packed r << 8 | l;
  // every smaller triangle is a prefix of it
  unsigned short* tri = reinterpret_cast<unsigned short*>(qq + RR_MMAX / 2);  // [4656]
  // FP32 views of the RB region once R has been moved out of it (J, V: 37,248 B each):
  // J holds float(M), then T and the reflectors; V the eigenvectors of M
  float* J = reinterpret_cast<float*>(RB);                // [96][RR_LDF]
  float* V = J + RR_MMAX * RR_LDF;                        // [96][RR_LDF]
  // after the FP32 sweeps: J's region holds R32 and CC, V's region the k x k work
  float* R32 = J;                                         // [96][RR_KLD] FP32 residual
  float* CC = J + RR_MMAX * RR_KLD;                       // [96][RR_KLD] correction coefficients
  double* H = reinterpret_cast<double*>(V);               // [32][RR_KLD]
  double* Vk = H + RR_KMAX * RR_KLD;                      // [32][RR_KLD]
  double* Wk = Vk + RR_KMAX * RR_KLD;                     // [32][RR_KLD]
  // k x k work of step 8 in the J region (R32 and CC are dead by then)
  double* D64 = reinterpret_cast<double*>(J);             // [32][RR_KLD]
  double* K64 = D64 + RR_KMAX * RR_KLD;                   // [32][RR_KLD]
  float* E32 = reinterpret_cast<float*>(K64 + RR_KMAX * RR_KLD);  // [32][RR_KLD]
  float* D32 = E32 + RR_KMAX * RR_KLD;                    // [32][RR_KLD]
  __shared__ int dropped;
  __shared__ int kext;
  __shared__ float lmax;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int k = a.k;
  const Tiling tk(k, lane);
  int m = a.m;
  if (tid == 0) dropped = 0;
  for (int r = wid; r < a.m; r += RR_NW)
    for (int l = lane; l <= r; l += 32) tri[r * (r + 1) / 2 + l] = (unsigned short)((r << 8) | l);

  {
    const RRScratch* S = a.scr;
    m = S->m;
    if (tid == 0) dropped = S->dropped;
    for (int r = wid; r < m; r += RR_NW)
      for (int c = lane; c < m; c += 32) {
        MA[r * RR_LD + c] = S->MA[r * RR_LD + c];
        V[r * RR_LDF + c] = S->V[r * RR_LDF + c];
      }
    for (int i = tid; i < m; i += RR_T) {
      sc[i] = S->sc[i];
      rdg[i] = S->rdg[i];
      lam[i] = S->lam[i];
    }
  }
  __syncthreads();
  const float clus = 1e-3f * a.scr->tn;             // eigenvalues closer than this: a cluster
  // 4d. orthonormalise within clusters, normalise the rest: classical Gram-Schmidt applied
  //     twice (orthogonal to working precision like the modified form); lane t forms the
  //     whole dot product with column j + t of the cluster, so no shuffle reduction is on
  //     the chain, and the projections are then removed row by row.  The coefficients go
  //     to the warp's slice of J's region (free until step 7).
  for (int j = wid; j < m; j += RR_NW) {
    if (j > 0 && lam[j] - lam[j - 1] < clus) continue;   // not the first of its cluster
    int e = j + 1;
    while (e < m && lam[e] - lam[e - 1] < clus) ++e;
    float* dsc = J + wid * RR_MMAX;
    for (int i = j; i < e; ++i) {
      for (int pass = 0; pass < 2 && i > j; ++pass) {
        for (int l = j + lane; l < i; l += 32) {
          float d0 = 0.0f, d1 = 0.0f;
          int r = 0;
          for (; r + 1 < m; r += 2) {
            d0 = fmaf(V[r * RR_LDF + l], V[r * RR_LDF + i], d0);
            d1 = fmaf(V[(r + 1) * RR_LDF + l], V[(r + 1) * RR_LDF + i], d1);
          }
          if (r < m) d0 = fmaf(V[r * RR_LDF + l], V[r * RR_LDF + i], d0);
          dsc[l - j] = d0 + d1;
        }
        __syncwarp();
        for (int r = lane; r < m; r += 32) {
          float x = V[r * RR_LDF + i];
          for (int l = j; l < i; ++l) x = fmaf(-dsc[l - j], V[r * RR_LDF + l], x);
          V[r * RR_LDF + i] = x;
        }
        __syncwarp();
      }
      float n2 = 0.0f;
      for (int r = lane; r < m; r += 32) n2 = fmaf(V[r * RR_LDF + i], V[r * RR_LDF + i], n2);
      n2 = warp_sum(n2);
      const float inv = (n2 > 0.0f) ? rsqrtf(n2) : 0.0f;
      for (int r = lane; r < m; r += 32) V[r * RR_LDF + i] *= inv;
      __syncwarp();
    }
  }
  __syncthreads();

  // ------------------------------------------ 5. the k smallest FP32 eigenpairs
  // (multisection returns the eigenvalues in ascending order), extended to kk >= k by the
  // unwanted eigenpairs chained to the k-th within the FP32 resolution: their FP32 vectors
  // are mixed with the wanted ones, which the correction below cannot separate (it skips
  // pairs that close), so the FP64 Rayleigh-Ritz of step 8 runs on all kk and the k
  // smallest are taken after it
  if (tid < m) rk[tid] = tid;
  if (tid == 0) {
    lmax = fmaxf(fabsf(lam[0]), fabsf(lam[m - 1]));
    const float dres = 64.0f * 6e-8f * lmax;
    int e = k;
    while (e < m && e < RR_KMAX && lam[e] - lam[e - 1] <= dres) ++e;
    kext = e;
  }
  __syncthreads();
  const int kk = kext;
  const Tiling tkk(kk, lane);
  if (tid < kk) sel[tid] = tid;
  __syncthreads();

  // ------------------------------------------ 6. X = V(:, sel) in FP64, Y = M X
  FOR_RC(tkk, m, kk, wid) XD[r * RR_KLD + c] = (double)V[r * RR_LDF + sel[c]];
  __syncthreads();
  mul_mx(MA, XD, YD, m, tkk, kk, wid);
  __syncthreads();

  // ------------------------------------------ 7. one correction of X from the FP64 residual
  for (int j = wid; j < kk; j += RR_NW) {
    double xy = 0.0, xx = 0.0;
    for (int r = lane; r < m; r += 32) {
      xy = fma(XD[r * RR_KLD + j], YD[r * RR_KLD + j], xy);
      xx = fma(XD[r * RR_KLD + j], XD[r * RR_KLD + j], xx);
    }
    xy = warp_sum(xy);
    xx = warp_sum(xx);
    if (lane == 0) th[j] = xy * frcp(xx);
  }
  __syncthreads();
  FOR_RC(tkk, m, kk, wid) R32[r * RR_KLD + c] = (float)fma(-th[c], XD[r * RR_KLD + c], YD[r * RR_KLD + c]);
  __syncthreads();
  {
    const float delta = 64.0f * 6e-8f * lmax;      // unwanted: beyond the FP32 resolution
    const float delta_w = 1e-3f * lmax;             // wanted pairs: well separated only
    FOR_RC(tkk, m, kk, wid) {                       // r: eigenpair i, c: column j
      float f0 = 0.0f, f1 = 0.0f;
      int q = 0;
      for (; q + 1 < m; q += 2) {
        f0 = fmaf(V[q * RR_LDF + r], R32[q * RR_KLD + c], f0);
        f1 = fmaf(V[(q + 1) * RR_LDF + r], R32[(q + 1) * RR_KLD + c], f1);
      }
      if (q < m) f0 = fmaf(V[q * RR_LDF + r], R32[q * RR_KLD + c], f0);
      const float gap = (float)th[c] - lam[r];
      // close wanted directions are mixed by the k x k Rayleigh-Ritz below; correcting
      // only well-separated ones keeps X'^T X' - I of order eps_32 |M| / delta_w
      CC[r * RR_KLD + c] = (fabsf(gap) > (rk[r] >= kk ? delta : delta_w)) ? (f0 + f1) / gap : 0.0f;
    }
  }
  __syncthreads();
  FOR_RC(tkk, m, kk, wid) {                         // X' = X + V CC
    float d0 = 0.0f, d1 = 0.0f;
    int i = 0;
    for (; i + 1 < m; i += 2) {
      d0 = fmaf(V[r * RR_LDF + i], CC[i * RR_KLD + c], d0);
      d1 = fmaf(V[r * RR_LDF + i + 1], CC[(i + 1) * RR_KLD + c], d1);
    }
    if (i < m) d0 = fmaf(V[r * RR_LDF + i], CC[i * RR_KLD + c], d0);
    XD[r * RR_KLD + c] += (double)(d0 + d1);
  }
  __syncthreads();
  mul_mx(MA, XD, YD, m, tkk, kk, wid);              // Y' = M X'
  __syncthreads();

  // ------------------------------------------ 8. orthonormalise, k x k Rayleigh-Ritz
  // G = X'^T X' = I + E with |E| <= 1e-4, so T = G^-1/2 = I + D with
  // D = -E/2 + 3/8 E^2 - 5/16 E^3 to O(|E|^4) (E^2, E^3 in FP32); H = T H' T with
  // H' = X'^T M X', in FP64.
  FOR_RC(tkk, 2 * kk, kk, wid) {
    const int which = (r >= kk), i = r - which * kk;
    if (which == 0 && c < i) continue;
    const double* B2 = which ? YD : XD;
    double s0 = 0.0, s1 = 0.0;
    int q = 0;
    for (; q + 1 < m; q += 2) {
      s0 = fma(XD[q * RR_KLD + i], B2[q * RR_KLD + c], s0);
      s1 = fma(XD[(q + 1) * RR_KLD + i], B2[(q + 1) * RR_KLD + c], s1);
    }
    if (q < m) s0 = fma(XD[q * RR_KLD + i], B2[q * RR_KLD + c], s0);
    const double v = s0 + s1;
    if (which) {
      H[i * RR_KLD + c] = v;
    } else {
      const double e = v - (i == c ? 1.0 : 0.0);
      D64[i * RR_KLD + c] = e;
      D64[c * RR_KLD + i] = e;
      E32[i * RR_KLD + c] = (float)e;
      E32[c * RR_KLD + i] = (float)e;
    }
  }
  __syncthreads();
  FOR_RC(tkk, kk, kk, wid) {                        // E^2 (FP32, into D32)
    float s = 0.0f;
    for (int l = 0; l < kk; ++l) s = fmaf(E32[r * RR_KLD + l], E32[l * RR_KLD + c], s);
    D32[r * RR_KLD + c] = s;
  }
  __syncthreads();
  FOR_RC(tkk, kk, kk, wid) {                        // D = -E/2 + 3/8 E^2 - 5/16 E^3
    float e3 = 0.0f;
    for (int l = 0; l < kk; ++l) e3 = fmaf(E32[r * RR_KLD + l], D32[l * RR_KLD + c], e3);
    K64[r * RR_KLD + c] = fma(-0.5, D64[r * RR_KLD + c], (double)fmaf(-0.3125f, e3, 0.375f * D32[r * RR_KLD + c]));
  }
  __syncthreads();
  FOR_RC(tkk, kk, kk, wid) {
    const double d = K64[r * RR_KLD + c];
    D64[r * RR_KLD + c] = d;
    D32[r * RR_KLD + c] = (float)d;
  }
  __syncthreads();
  FOR_RC(tkk, kk, kk, wid) {                        // K = H' D
    double s = 0.0;
    for (int l = 0; l < kk; ++l) s = fma(H[r * RR_KLD + l], D64[l * RR_KLD + c], s);
    K64[r * RR_KLD + c] = s;
  }
  __syncthreads();
  FOR_RC(tkk, kk, kk, wid) {                        // H = H' + K + D (H' + K)
    double s = K64[r * RR_KLD + c];
    for (int l = 0; l < kk; ++l) s = fma(D64[r * RR_KLD + l], H[l * RR_KLD + c] + K64[l * RR_KLD + c], s);
    Wk[r * RR_KLD + c] = H[r * RR_KLD + c] + s;
  }
  __syncthreads();
  const int kp = kk + (kk & 1);
  const int kh = kp / 2;
  for (int i = wid; i < kp; i += RR_NW)
    for (int j = lane; j < kp; j += 32) {
      double v;
      if (i < kk && j < kk) v = 0.5 * (Wk[i * RR_KLD + j] + Wk[j * RR_KLD + i]);
      else v = (i == j) ? 1e300 : 0.0;
      H[i * RR_KLD + j] = v;
      Vk[i * RR_KLD + j] = (i == j) ? 1.0 : 0.0;
    }
  __syncthreads();
  // Cyclic Jacobi in FP64: the angle is taken in FP32 (it only has to shrink the coupling),
  // the rotation itself is exactly orthogonal in FP64; couplings below 1e-13 of the
  // diagonal entries cannot change an eigenvalue beyond rounding and are left alone.
  if (kp > 1) {
    const FastDiv fkp(kp);
    const int nblk = kh * (kh + 1) / 2;
    for (int sweep = 0; sweep < 30; ++sweep) {
      // a sweep that would rotate nothing ends the iteration: every pair is tested at
      // once (one barrier) instead of round by round (kp - 1 barriers)
      int need = 0;
      for (int q2 = tid; q2 < kp * kp; q2 += RR_T) {
        const int p = (int)fkp.div((unsigned)q2), q = q2 - p * kp;
        if (p < q && fabsf((float)H[p * RR_KLD + q]) >
                         1e-13f * (fabsf((float)H[p * RR_KLD + p]) + fabsf((float)H[q * RR_KLD + q])) + 1e-37f)
          need = 1;
      }
      if (__syncthreads_or(need) == 0) break;
      int nrot = 0;
      for (int step = 0; step < kp - 1; ++step) {
        int rot = 0;
        if (tid < kh) {
          int p, q;
          jacobi_pair_k(step, tid, kp, p, q);
          pp[tid] = p;
          qq[tid] = q;
          const double apq = H[p * RR_KLD + q], app = H[p * RR_KLD + p], aqq = H[q * RR_KLD + q];
          double c = 1.0, s = 0.0;
          // the significance test in FP32 (short chain; couplings below 1e-13 of the
          // diagonal cannot move an eigenvalue beyond rounding)
          const float apq32 = (float)apq;
          if (fabsf(apq32) > 1e-13f * (fabsf((float)app) + fabsf((float)aqq)) + 1e-37f) {
            rot = 1;
            const float tau = __fdividef((float)(aqq - app), 2.0f * apq32);
            float t32;
            if (fabsf(tau) > 1e9f) {
              t32 = __fdividef(0.5f, tau);
            } else {
              const float u = fmaf(tau, tau, 1.0f);
              t32 = copysignf(__fdividef(1.0f, fabsf(tau) + u * rsqrtf(u)), tau);
            }
            // c = (1 + t^2)^-1/2 from the FP32 seed and one Newton step (relative error
            // ~2^-44: c^2 + s^2 = 1 to ~6e-14 per rotation, far below the FP32 blocks'
            // rounding after the ~30 rotations of a call)
            const double t = (double)t32;
            const double x = fma(t, t, 1.0);
            const double y0 = (double)rsqrtf((float)x);
            c = y0 * fma(-0.5 * x, y0 * y0, 1.5);
            s = t * c;
          }
          csd[tid] = c;
          snd[tid] = s;
        }
        const int nstep = __syncthreads_count(rot);
        nrot += nstep;
        if (nstep == 0) continue;
        // A warp-wide FP64 instruction holds an SMSP's FP64 pipe for ~64 cycles however
        // few lanes are active, so the work is packed into full warps spread over the SMSPs:
        // the first hw warps take the 2 x 2 blocks of H (ba <= bb) as two half-tasks on
        // lanes 2i, 2i + 1 (one output row of the block each), the other warps Vk.
        const int hw = (nblk + 15) / 16;
        if (wid < hw) {
          const int task = tid >> 1, h = tid & 1;
          int pa = 0, qa = 0, pb = 0, qb = 0;
          bool act = false, dg = false;
          double n0 = 0.0, n1 = 0.0;
          if (task < nblk) {
            const int e = tri[task], bb = e >> 8, ba = e & 255;
            const double sa = snd[ba], sb = snd[bb];
            act = !(sa == 0.0 && sb == 0.0);
            if (act) {
              pa = pp[ba], qa = qq[ba], pb = pp[bb], qb = qq[bb];
              dg = (bb == ba);
              const double ca = csd[ba], cb = csd[bb];
              const double j00 = H[pa * RR_KLD + pb], j01 = H[pa * RR_KLD + qb];
              const double j10 = H[qa * RR_KLD + pb], j11 = H[qa * RR_KLD + qb];
              double t0, t1;
              if (h == 0) {
                t0 = ca * j00 - sa * j10;
                t1 = ca * j01 - sa * j11;
              } else {
                t0 = sa * j00 + ca * j10;
                t1 = sa * j01 + ca * j11;
              }
              n0 = cb * t0 - sb * t1;
              n1 = sb * t0 + cb * t1;
            }
          }
          // diagonal blocks: n01 (lane h = 0) and n10 (lane h = 1) are averaged
          const double other = __shfl_xor_sync(0xffffffffu, h ? n0 : n1, 1);
          __syncwarp();                                  // every read of H before any write
          if (act) {
            const int ra = h ? qa : pa;
            if (dg) {
              const double off = h ? 0.5 * (other + n0) : 0.5 * (n1 + other);
              H[ra * RR_KLD + ra] = h ? n1 : n0;
              H[ra * RR_KLD + (h ? pa : qa)] = off;
            } else {
              H[ra * RR_KLD + pb] = n0;
              H[ra * RR_KLD + qb] = n1;
              H[pb * RR_KLD + ra] = n0;
              H[qb * RR_KLD + ra] = n1;
            }
          }
        } else {
          for (int q3 = tid - 32 * hw; q3 < kh * kp; q3 += RR_T - 32 * hw) {
            const int ba = (int)fkp.div((unsigned)q3), r = q3 - ba * kp;
            const double sa = snd[ba];
            if (sa == 0.0) continue;
            const double ca = csd[ba];
            const int pa = pp[ba], qa = qq[ba];
            const double vp = Vk[r * RR_KLD + pa], vq = Vk[r * RR_KLD + qa];
            Vk[r * RR_KLD + pa] = ca * vp - sa * vq;
            Vk[r * RR_KLD + qa] = sa * vp + ca * vq;
          }
        }
        __syncthreads();
      }
      if (nrot == 0) break;
    }
  }
  for (int i = tid; i < kk; i += RR_T) {             // ascending order of the kk values
    const double li = H[i * RR_KLD + i];
    int rank = 0;
    for (int j = 0; j < kk; ++j) {
      const double lj = H[j * RR_KLD + j];
      rank += (lj < li) || (lj == li && j < i);
    }
    perm[rank] = i;
  }
  __syncthreads();
  FOR_RC(tk, kk, k, wid) {                          // W = T Vk(:, perm) = Vk + D Vk (FP32 part),
    const int pj = perm[c];                         // the k smallest of the kk
    float s = 0.0f;
    for (int l = 0; l < kk; ++l) s = fmaf(D32[r * RR_KLD + l], (float)Vk[l * RR_KLD + pj], s);
    Wk[r * RR_KLD + c] = Vk[r * RR_KLD + pj] + (double)s;
  }
  __syncthreads();
  FOR_RC(tk, m, k, wid) {                           // Z = X' W
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < kk; i += 2) {
      s0 = fma(XD[r * RR_KLD + i], Wk[i * RR_KLD + c], s0);
      s1 = fma(XD[r * RR_KLD + i + 1], Wk[(i + 1) * RR_KLD + c], s1);
    }
    if (i < kk) s0 = fma(XD[r * RR_KLD + i], Wk[i * RR_KLD + c], s0);
    YD[r * RR_KLD + c] = s0 + s1;
  }
  __syncthreads();

  // ------------------------------------------ 9. C = R^-T Z (rows from the bottom), unscale
  // Look-ahead: in step i warp 0 updates row i - 1 and forms its multipliers while the
  // other warps update the rows above it; one barrier per row.
  if (wid == 0 && lane < k) fv[((m - 1) & 1) * RR_MMAX + lane] = YD[(m - 1) * RR_KLD + lane] * rdg[m - 1];
  __syncthreads();
  for (int i = m - 1; i >= 1; --i) {
    const double* fi = fv + (i & 1) * RR_MMAX;
    if (wid == 0) {
      if (lane < k) {
        const double y = fma(-MA[(i - 1) * RR_LD + i], fi[lane], YD[(i - 1) * RR_KLD + lane]);
        YD[(i - 1) * RR_KLD + lane] = y;
        fv[((i - 1) & 1) * RR_MMAX + lane] = y * rdg[i - 1];
      }
    } else {
      for (int r0 = (wid - 1) * tk.rows; r0 < i - 1; r0 += (RR_NW - 1) * tk.rows) {
        const int r = r0 + tk.lr, c = tk.lc;
        if (r < i - 1 && c < k) YD[r * RR_KLD + c] = fma(-MA[r * RR_LD + i], fi[c], YD[r * RR_KLD + c]);
      }
    }
    __syncthreads();
  }
  FOR_RC(tk, a.m, k, wid) a.C[r * k + c] = (r < m) ? YD[r * RR_KLD + c] * (rdg[r] * sc[r]) : 0.0;
  if (tid < k) {
    const double thv = H[perm[tid] * RR_KLD + perm[tid]];
    a.theta[tid] = thv;
    if (a.theta_hist) a.theta_hist[tid] = thv;
    if (!isfinite(thv)) *a.status = 3;
  }
  if (tid == 0 && dropped && a.restarts) *a.restarts += 1;
  if (!a.Cp) return;
  // ------------------------------------------ 10. coefficients of the next P, B-orthogonal
  // to the next X:  Cw = C with the X rows zeroed,  Z2 = C^T G_B Cw,  Cp = Cw - C Z2.
  __syncthreads();
  const int mm = a.m;
  double* Cs = MA;                   // [mm][k]
  double* T1 = MA + mm * k;          // [mm][k]
  double* Z2 = T1 + mm * k;          // [k][k]
  FOR_RC(tk, mm, k, wid) Cs[r * k + c] = a.C[r * k + c];
  __syncthreads();
  const double* GBg = a.G + (size_t)mm * mm;
  FOR_RC(tk, mm, k, wid) {
    double acc0 = 0.0, acc1 = 0.0;
    int b = k;
    for (; b + 1 < mm; b += 2) {
      acc0 = fma(GBg[r * mm + b], Cs[b * k + c], acc0);
      acc1 = fma(GBg[r * mm + b + 1], Cs[(b + 1) * k + c], acc1);
    }
    if (b < mm) acc0 = fma(GBg[r * mm + b], Cs[b * k + c], acc0);
    T1[r * k + c] = acc0 + acc1;
  }
  __syncthreads();
  FOR_RC(tk, k, k, wid) {
    double acc0 = 0.0, acc1 = 0.0;
    int q = 0;
    for (; q + 1 < mm; q += 2) {
      acc0 = fma(Cs[q * k + r], T1[q * k + c], acc0);
      acc1 = fma(Cs[(q + 1) * k + r], T1[(q + 1) * k + c], acc1);
    }
    if (q < mm) acc0 = fma(Cs[q * k + r], T1[q * k + c], acc0);
    Z2[r * k + c] = acc0 + acc1;
  }
  __syncthreads();
  FOR_RC(tk, mm, k, wid) {
    double acc = (r >= k) ? Cs[r * k + c] : 0.0;
    for (int i = 0; i < k; ++i) acc = fma(-Cs[r * k + i], Z2[i * k + c], acc);
    a.Cp[r * k + c] = acc;
  }
}

size_t rr_smem_bytes() {
  return (size_t)(2 * RR_MMAX * RR_LD + 2 * RR_MMAX * RR_KLD + 4 * RR_MMAX + RR_KMAX + RR_KMAX) *
             sizeof(double) +
         (size_t)(6 * RR_MMAX) * sizeof(float) +
         (2 * RR_KMAX + RR_MMAX + RR_MMAX) * sizeof(int) +
         (size_t)(RR_MMAX * (RR_MMAX + 1) / 2) * sizeof(unsigned short);
}

}  // namespace

int bf_rr_launch(const RRParams& a, cudaStream_t s) {
  const size_t sm = rr_smem_bytes();
  if (!a.scr) return bf_fail(BF_EINVAL, "Rayleigh-Ritz: no scratch area");
  int rc = bf_smem_attr((const void*)k_rr_reduce, (int)sm, "cudaFuncSetAttribute(k_rr_reduce)");
  if (!rc) rc = bf_smem_attr((const void*)k_rr, (int)sm, "cudaFuncSetAttribute(k_rr)");
  if (rc) return rc;
  // k_rr_vectors waits for the one-CTA reduction by a plain launch: launched early its m
  // CTAs would hold SMs the concurrent work of other streams can use meanwhile
  BF_LAUNCH_PDL(k_rr_reduce, 1, RR_T, sm, s, a);
  BF_LAUNCH(k_rr_vectors<<<a.m, 32, 0, s>>>(a));
  BF_LAUNCH_PDL(k_rr, 1, RR_T, sm, s, a);
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

extern "C" int bf_rayleigh_ritz(const double* G, int m, int k, int m_nop, double* C,
                                double* Cp, double* theta, int* flags, void* stream) {
  if (!G || !C || !theta || !flags) return bf_fail(BF_EINVAL, "bf_rayleigh_ritz: NULL argument");
  if (m < 1 || m > RR_MMAX || k < 1 || k > RR_KMAX || k > m || m_nop < 0 || m_nop > m)
    return bf_fail(BF_EINVAL, "bf_rayleigh_ritz: need 1 <= k <= m <= 96, k <= 32");
  RRParams a;
  a.G = G;
  a.m = m;
  a.k = k;
  a.m_nop = m_nop;
  a.C = C;
  a.Cp = Cp;
  a.theta = theta;
  a.theta_hist = nullptr;
  a.status = flags;
  a.restarts = flags + 1;
  // one scratch area per process and device for this test entry (kept until exit)
  static RRScratch* scr[64] = {nullptr};
  int dev = 0;
  BF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return bf_fail(BF_EINVAL, "bf_rayleigh_ritz: device index");
  if (!scr[dev]) BF_CUDA(cudaMalloc(&scr[dev], sizeof(RRScratch)));
  a.scr = scr[dev];
  return bf_rr_launch(a, (cudaStream_t)stream);
}
