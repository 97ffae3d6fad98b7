// The small Rayleigh-Ritz problem of block LOBPCG (Algorithm 3, Section 6), solved in
// FP64 by one CTA: the k smallest eigenpairs of the pencil (G_A, G_B) of size m <= 96.
//
// On GB300 a dependent FP64 FMA costs about 64 cycles, an FP64 divide about 640 and FP64
// throughput is about 1.7 FMA/clk per SM, so the solver keeps FP64 work near m^3 and, more
// importantly, keeps every dependent FP64 chain short:
//   1. symmetrise, scale to unit diag(G_B), right-looking Cholesky G_B = R R^T (a squared
//      pivot <= 1e-10 means a dependent trial basis: retry on the leading m_nop block,
//      i.e. without P, else report a breakdown);
//   2. standard form M = R^-1 G_A R^-T by two right-looking triangular solves;
//   3. Householder reduction M = Q T Q^T to a tridiagonal T (reflectors kept in M);
//   4. shifts near the k smallest eigenvalues of T from Sturm counts evaluated in FP32
//      at 32 points per warp (multisection), which is all the accuracy inverse iteration
//      needs: the final eigenvalues come from step 6;
//   5. one eigenvector per shift by four steps of FP64 inverse iteration on
//      T - lambda I (one tridiagonal factorisation with row interchanges, reused by
//      every step), all k in parallel;
//   6. Cholesky QR (twice) of those k vectors and a k x k Rayleigh-Ritz on T (cyclic
//      Jacobi; the matrix is diagonal up to rounding except inside clusters): FP64
//      eigenvalues and vectors;
//   7. back-transformation by the reflectors, C = R^-T Y and the unit-diagonal scaling
//      undone; with Cp requested, the coefficients of the next P made B-orthogonal to
//      the next X (see the driver).
// Reciprocals and square roots use an FP32 seed refined by two FP64 Newton steps
// (rounding-level accuracy), avoiding the long FP64 divide and square-root sequences.
#include <math.h>

#include "bf_internal.cuh"
#include "bf_rr.cuh"

#define RR_T 512
#define RR_LD 97            // padded leading dimension of the m x m work matrices
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
// e2) smaller than x, in FP32: sign changes along p_0 = 1, p_1 = d_0 - x,
// p_i = (d_{i-1} - x) p_{i-1} - e2_{i-2} p_{i-2}.  A zero p_i is counted as a sign change
// (as if it were a tiny number of the opposite sign); the pair (p_{i-1}, p_i) is rescaled
// by a power of two whenever p_i leaves [2^-60, 2^60].
__device__ int sturm_count_f(const float* d, const float* e2, int m, float x) {
  float p0 = 1.0f, p1 = d[0] - x;
  if (p1 == 0.0f) p1 = -0x1p-40f;
  int cnt = (p1 < 0.0f);
  for (int i = 1; i < m; ++i) {
    float p2 = (d[i] - x) * p1 - e2[i - 1] * p0;
    if (p2 == 0.0f) p2 = -p1 * 0x1p-40f;
    cnt += ((p2 < 0.0f) != (p1 < 0.0f));
    p0 = p1;
    p1 = p2;
    const float a = fabsf(p1);
    if (a > 0x1p60f || a < 0x1p-60f) {
      const float sc = scalbnf(1.0f, -ilogbf(p1));
      p0 *= sc;
      p1 *= sc;
    }
  }
  return cnt;
}

// Factor T - lambda I by elimination with row interchanges: the working row (entries in
// columns i, i+1, i+2) is compared with the next original row and the larger entry in
// column i is the pivot.  Kept per row i: the multiplier f[i], whether the rows were
// interchanged (sw[i]), the pivot reciprocal ri[i] and the two entries right of the
// pivot (u1, u2).  Zero pivots are replaced by `tiny`.
__device__ void tri_factor(const double* d, const double* e, int m, double lambda, double tiny,
                           double* f, unsigned char* sw, double* ri, double* u1, double* u2) {
  double r0 = d[0] - lambda, r1 = (m > 1) ? e[0] : 0.0, r2 = 0.0;
  for (int i = 0; i < m - 1; ++i) {
    const double n0 = e[i], n1 = d[i + 1] - lambda, n2 = (i + 2 < m) ? e[i + 1] : 0.0;
    const bool keep = fabs(r0) >= fabs(n0);
    double p0 = keep ? r0 : n0;
    const double p1 = keep ? r1 : n1, p2 = keep ? r2 : n2;
    const double o0 = keep ? n0 : r0, o1 = keep ? n1 : r1, o2 = keep ? n2 : r2;
    if (p0 == 0.0) p0 = tiny;
    const double rp = frcp(p0);
    const double fi = o0 * rp;
    f[i] = fi;
    sw[i] = keep ? 0 : 1;
    ri[i] = rp;
    u1[i] = p1;
    u2[i] = p2;
    r0 = fma(-fi, p1, o1);
    r1 = fma(-fi, p2, o2);
    r2 = 0.0;
  }
  if (r0 == 0.0) r0 = tiny;
  ri[m - 1] = frcp(r0);
  u1[m - 1] = 0.0;
  u2[m - 1] = 0.0;
}

// Solve with the factors of tri_factor, b -> x in place.
__device__ void tri_solve(int m, const double* f, const unsigned char* sw, const double* ri,
                          const double* u1, const double* u2, double* b) {
  double rb = b[0];
  for (int i = 0; i < m - 1; ++i) {
    const double nb = b[i + 1];
    const double pb = sw[i] ? nb : rb, ob = sw[i] ? rb : nb;
    b[i] = pb;
    rb = fma(-f[i], pb, ob);
  }
  b[m - 1] = rb * ri[m - 1];
  if (m > 1) b[m - 2] = fma(-u1[m - 2], b[m - 1], b[m - 2]) * ri[m - 2];
  for (int i = m - 3; i >= 0; --i) b[i] = fma(-u2[i], b[i + 2], fma(-u1[i], b[i + 1], b[i])) * ri[i];
}

__device__ __forceinline__ void jacobi_pair_k(int step, int i, int np, int& p, int& q) {
  const int n1 = np - 1;
  if (i == 0) {
    p = step % n1;
    q = n1;
  } else {
    p = (step + i) % n1;
    q = (step - i + n1) % n1;
  }
  if (p > q) { const int t = p; p = q; q = t; }
}

__global__ void __launch_bounds__(RR_T) k_rr(const RRParams a) {
  if (*a.status != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double* M = reinterpret_cast<double*>(smem);          // [96][RR_LD]
  double* R = M + RR_MMAX * RR_LD;                      // [96][RR_LD]
  double* Z = R + RR_MMAX * RR_LD;                      // [96][RR_KLD] eigenvectors
  double* H = Z + RR_MMAX * RR_KLD;                     // [32][RR_KLD] k x k problem
  double* Vk = H + RR_KMAX * RR_KLD;                    // [32][RR_KLD]
  double* sc = Vk + RR_KMAX * RR_KLD;                   // [96] unit-diagonal scaling
  double* rdg = sc + RR_MMAX;                           // [96] 1 / diag(R)
  double* dd = rdg + RR_MMAX;                           // [96] diagonal of T
  double* ee = dd + RR_MMAX;                            // [96] off-diagonal of T
  double* e2 = ee + RR_MMAX;                            // [96] squared off-diagonal
  double* bet = e2 + RR_MMAX;                           // [96] reflector scalars
  double* pv = bet + RR_MMAX;                           // [96] work vector
  double* lam = pv + RR_MMAX;                           // [32] shifts
  double* cs = lam + RR_KMAX;                           // [16]
  double* sn = cs + RR_KMAX / 2;                        // [16]
  double* rdk = sn + RR_KMAX / 2;                       // [32] 1 / diag of the k x k factor
  float* d32 = reinterpret_cast<float*>(rdk + RR_KMAX); // [96]
  float* e32 = d32 + RR_MMAX;                           // [96]
  int* perm = reinterpret_cast<int*>(e32 + RR_MMAX);    // [32]
  __shared__ int fail, dropped, nrot;
  __shared__ double sh_alpha, sh_beta, sh_v0, sh_K, sh_lo, sh_hi;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int k = a.k;
  int m = a.m;
  if (tid == 0) dropped = 0;

  // ---------------------------------------------------------------- 1. scale, Cholesky
  for (int attempt = 0; attempt < 2; ++attempt) {
    __syncthreads();
    for (int q = tid; q < m * m; q += RR_T) {
      const int r = q / m, c = q - r * m;
      M[r * RR_LD + c] = 0.5 * (a.G[r * a.m + c] + a.G[c * a.m + r]);
      R[r * RR_LD + c] = 0.5 * (a.G[a.m * a.m + r * a.m + c] + a.G[a.m * a.m + c * a.m + r]);
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int r = tid; r < m; r += RR_T) {
      const double dg = R[r * RR_LD + r];
      if (!(dg > 0.0) || !isfinite(dg)) fail = 1;
      sc[r] = (dg > 0.0) ? frsqrt(dg) : 0.0;
    }
    __syncthreads();
    if (!fail) {
      for (int q = tid; q < m * m; q += RR_T) {
        const int r = q / m, c = q - r * m;
        M[r * RR_LD + c] *= sc[r] * sc[c];
        R[r * RR_LD + c] *= sc[r] * sc[c];
      }
      __syncthreads();
      // right-looking Cholesky: lower factor in R
      for (int j = 0; j < m; ++j) {
        if (tid == 0) {
          const double piv = R[j * RR_LD + j];
          if (!(piv > DEP_TOL)) {
            fail = 1;
          } else {
            const double rj = frsqrt(piv);
            R[j * RR_LD + j] = piv * rj;
            rdg[j] = rj;
          }
        }
        __syncthreads();
        if (fail) break;
        const double rj = rdg[j];
        for (int i = j + 1 + tid; i < m; i += RR_T) R[i * RR_LD + j] *= rj;
        __syncthreads();
        const int t = m - j - 1;
        for (int q = tid; q < t * t; q += RR_T) {
          const int i = j + 1 + q / t, l = j + 1 + q % t;
          if (l <= i) R[i * RR_LD + l] = fma(-R[i * RR_LD + j], R[l * RR_LD + j], R[i * RR_LD + l]);
        }
        __syncthreads();
      }
    }
    __syncthreads();
    if (!fail) break;
    if (attempt == 0 && a.m_nop > 0 && a.m_nop < a.m) {
      m = a.m_nop;
      if (tid == 0) dropped = 1;
      continue;
    }
    if (tid == 0) *a.status = 2;
    return;
  }

  // ---------------------------------------------------------------- 2. M = R^-1 M R^-T
  for (int i = 0; i < m; ++i) {                 // Y = R^-1 M: rows in order
    for (int c = tid; c < m; c += RR_T) M[i * RR_LD + c] *= rdg[i];
    __syncthreads();
    const int t = m - i - 1;
    for (int q = tid; q < t * m; q += RR_T) {
      const int l = i + 1 + q / m, c = q % m;
      M[l * RR_LD + c] = fma(-R[l * RR_LD + i], M[i * RR_LD + c], M[l * RR_LD + c]);
    }
    __syncthreads();
  }
  for (int i = 0; i < m; ++i) {                 // M = Y R^-T: columns in order, rows >= col
    for (int r = i + tid; r < m; r += RR_T) M[r * RR_LD + i] *= rdg[i];
    __syncthreads();
    const int t = m - i - 1;
    for (int q = tid; q < t * t; q += RR_T) {
      const int l = i + 1 + q / t, r = i + 1 + q % t;
      if (r >= l) M[r * RR_LD + l] = fma(-M[r * RR_LD + i], R[l * RR_LD + i], M[r * RR_LD + l]);
    }
    __syncthreads();
  }
  // (the tridiagonal reduction below reads the lower triangle only)

  // ---------------------------------------------------------------- 3. tridiagonal
  for (int j = 0; j + 2 < m; ++j) {
    const int n1 = m - j - 1;
    double* col = M + (j + 1) * RR_LD + j;       // x_i = col[i * RR_LD]
    if (tid < 32) {
      double s = 0.0;
      for (int i = tid; i < n1; i += 32) s = fma(col[i * RR_LD], col[i * RR_LD], s);
      s = warp_sum(s);
      if (tid == 0) {
        const double x0 = col[0];
        const double tail = s - x0 * x0;
        if (!(tail > 0.0)) {
          sh_beta = 0.0;
          sh_alpha = x0;
          sh_v0 = 0.0;
        } else {
          const double nrm = s * frsqrt(s);
          const double al = (x0 >= 0.0) ? -nrm : nrm;
          const double v0 = x0 - al;
          sh_alpha = al;
          sh_v0 = v0;
          sh_beta = 2.0 * frcp(fma(v0, v0, tail));
        }
      }
    }
    __syncthreads();
    const double beta = sh_beta;
    if (tid == 0) {
      dd[j] = M[j * RR_LD + j];
      ee[j] = sh_alpha;
      bet[j] = beta;
      if (beta != 0.0) col[0] = sh_v0;          // reflector vector stored below the diagonal
    }
    __syncthreads();
    if (beta == 0.0) continue;
    double* A1 = M + (j + 1) * RR_LD + (j + 1);  // trailing n1 x n1 block
    // p = beta A1 v  (eight threads per row; A1 is kept in its lower triangle)
    for (int row0 = 0; row0 < n1; row0 += RR_T / 8) {
      const int row = row0 + (tid >> 3), part = tid & 7;
      double s = 0.0;
      if (row < n1)
        for (int c = part; c < n1; c += 8) {
          const double av = (c <= row) ? A1[row * RR_LD + c] : A1[c * RR_LD + row];
          s = fma(av, col[c * RR_LD], s);
        }
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      if (row < n1 && part == 0) pv[row] = beta * s;
    }
    __syncthreads();
    if (tid < 32) {
      double s = 0.0;
      for (int i = tid; i < n1; i += 32) s = fma(col[i * RR_LD], pv[i], s);
      s = warp_sum(s);
      if (tid == 0) sh_K = 0.5 * beta * s;
    }
    __syncthreads();
    for (int i = tid; i < n1; i += RR_T) pv[i] = fma(-sh_K, col[i * RR_LD], pv[i]);   // w
    __syncthreads();
    for (int q = tid; q < n1 * n1; q += RR_T) {
      const int r = q / n1, c = q - r * n1;
      if (c <= r)
        A1[r * RR_LD + c] = fma(-col[r * RR_LD], pv[c], fma(-pv[r], col[c * RR_LD], A1[r * RR_LD + c]));
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2) {
      dd[m - 2] = M[(m - 2) * RR_LD + (m - 2)];
      ee[m - 2] = M[(m - 1) * RR_LD + (m - 2)];
      bet[m - 2] = 0.0;
    }
    dd[m - 1] = M[(m - 1) * RR_LD + (m - 1)];
    ee[m - 1] = 0.0;
    double lo = 1e300, hi = -1e300;               // Gershgorin interval
    for (int i = 0; i < m; ++i) {
      const double rad = fabs(ee[i]) + (i > 0 ? fabs(ee[i - 1]) : 0.0);
      lo = fmin(lo, dd[i] - rad);
      hi = fmax(hi, dd[i] + rad);
    }
    sh_lo = lo;
    sh_hi = hi;
  }
  __syncthreads();
  for (int i = tid; i < m; i += RR_T) {
    e2[i] = ee[i] * ee[i];
    d32[i] = (float)dd[i];
    e32[i] = (float)(ee[i] * ee[i]);
  }
  __syncthreads();
  const double tn = fmax(fabs(sh_lo), fabs(sh_hi));
  const double tiny = 4.0 * 2.2e-16 * tn + 1e-300;

  // ---------------------------------------------------------------- 4. FP32 multisection shifts
  for (int j = wid; j < k; j += RR_T / 32) {
    float lo = (float)sh_lo, hi = (float)sh_hi;
    lo -= 1e-6f * fabsf(lo) + 1e-30f;
    hi += 1e-6f * fabsf(hi) + 1e-30f;
    const float stop = 4.0f * 6e-8f * (float)tn + 1e-30f;
    for (int round = 0; round < 10 && hi - lo > stop; ++round) {
      const float w = (hi - lo) * (1.0f / 33.0f);
      const float x = lo + w * (float)(lane + 1);
      const unsigned above = __ballot_sync(0xffffffffu, sturm_count_f(d32, e32, m, x) > j);
      const int first = above ? __ffs(above) - 1 : 32;     // first point with more than j below
      const float nlo = (first == 0) ? lo : lo + w * (float)first;
      const float nhi = (first == 32) ? hi : lo + w * (float)(first + 1);
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) lam[j] = 0.5 * ((double)lo + (double)hi);
  }
  __syncthreads();

  // ---------------------------------------------------------------- 5. inverse iteration
  if (tid < k) {
    double b[RR_MMAX], f[RR_MMAX], ri[RR_MMAX], u1[RR_MMAX], u2[RR_MMAX];
    unsigned char sw[RR_MMAX];
    tri_factor(dd, ee, m, lam[tid], tiny, f, sw, ri, u1, u2);
    for (int i = 0; i < m; ++i) b[i] = 1.0 + 0.25 * (double)(((i + 1) * (tid + 3) * 7919) % 97) / 97.0;
    for (int rep = 0; rep < 4; ++rep) {
      tri_solve(m, f, sw, ri, u1, u2, b);
      double nrm0 = 0.0, nrm1 = 0.0;
      for (int i = 0; i + 1 < m; i += 2) {
        nrm0 = fmax(nrm0, fabs(b[i]));
        nrm1 = fmax(nrm1, fabs(b[i + 1]));
      }
      if (m & 1) nrm0 = fmax(nrm0, fabs(b[m - 1]));
      const double nrm = fmax(nrm0, nrm1);
      const double inv = (nrm > 0.0 && isfinite(nrm)) ? frcp(nrm) : 1.0;
      for (int i = 0; i < m; ++i) b[i] *= inv;
    }
    for (int i = 0; i < m; ++i) Z[i * RR_KLD + tid] = b[i];
  }
  __syncthreads();

  // ---------------------------------------------------------------- 6. Cholesky QR twice, k x k Rayleigh-Ritz
  for (int pass = 0; pass < 2; ++pass) {
    for (int q = tid; q < k * k; q += RR_T) {        // G = Z^T Z (lower part used)
      const int i = q / k, j = q - i * k;
      if (j <= i) {
        double s0 = 0.0, s1 = 0.0;
        int r = 0;
        for (; r + 1 < m; r += 2) {
          s0 = fma(Z[r * RR_KLD + i], Z[r * RR_KLD + j], s0);
          s1 = fma(Z[(r + 1) * RR_KLD + i], Z[(r + 1) * RR_KLD + j], s1);
        }
        if (r < m) s0 = fma(Z[r * RR_KLD + i], Z[r * RR_KLD + j], s0);
        H[i * RR_KLD + j] = s0 + s1;
      }
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {                   // G = L L^T, right-looking
      if (tid == 0) {
        const double piv = H[j * RR_KLD + j];
        const double rj = (piv > 0.0) ? frsqrt(piv) : 0.0;
        H[j * RR_KLD + j] = piv * rj;
        rdk[j] = rj;
      }
      __syncthreads();
      const double rj = rdk[j];
      for (int i = j + 1 + tid; i < k; i += RR_T) H[i * RR_KLD + j] *= rj;
      __syncthreads();
      const int t = k - j - 1;
      for (int q = tid; q < t * t; q += RR_T) {
        const int i = j + 1 + q / t, l = j + 1 + q % t;
        if (l <= i) H[i * RR_KLD + l] = fma(-H[i * RR_KLD + j], H[l * RR_KLD + j], H[i * RR_KLD + l]);
      }
      __syncthreads();
    }
    for (int j = 0; j < k; ++j) {                   // Z <- Z L^-T, columns in order
      for (int r = tid; r < m; r += RR_T) Z[r * RR_KLD + j] *= rdk[j];
      __syncthreads();
      const int t = k - j - 1;
      for (int q = tid; q < t * m; q += RR_T) {
        const int l = j + 1 + q / m, r = q % m;
        Z[r * RR_KLD + l] = fma(-Z[r * RR_KLD + j], H[l * RR_KLD + j], Z[r * RR_KLD + l]);
      }
      __syncthreads();
    }
  }
  // H = Z^T T Z
  for (int q = tid; q < k * k; q += RR_T) {
    const int i = q / k, j = q - i * k;
    double s = 0.0;
    for (int r = 0; r < m; ++r) {
      double tz = dd[r] * Z[r * RR_KLD + j];
      if (r > 0) tz = fma(ee[r - 1], Z[(r - 1) * RR_KLD + j], tz);
      if (r + 1 < m) tz = fma(ee[r], Z[(r + 1) * RR_KLD + j], tz);
      s = fma(Z[r * RR_KLD + i], tz, s);
    }
    H[i * RR_KLD + j] = s;
  }
  __syncthreads();
  const int kp = k + (k & 1);
  for (int q = tid; q < kp * kp; q += RR_T) {
    const int i = q / kp, j = q - i * kp;
    if (i < k && j < k) {
      if (i < j) {
        const double v = 0.5 * (H[i * RR_KLD + j] + H[j * RR_KLD + i]);
        H[i * RR_KLD + j] = v;
        H[j * RR_KLD + i] = v;
      }
    } else {
      H[i * RR_KLD + j] = (i == j) ? 1e300 : 0.0;
    }
    Vk[i * RR_KLD + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (kp > 1) {
    for (int sweep = 0; sweep < 30; ++sweep) {
      if (tid == 0) nrot = 0;
      __syncthreads();
      for (int step = 0; step < kp - 1; ++step) {
        for (int i = tid; i < kp / 2; i += RR_T) {
          int p, q;
          jacobi_pair_k(step, i, kp, p, q);
          const double apq = H[p * RR_KLD + q], app = H[p * RR_KLD + p], aqq = H[q * RR_KLD + q];
          double c = 1.0, s = 0.0;
          // rotate unless the coupling is below 1e-13 of the diagonal entries: the
          // eigenvalue change it could make is then below rounding
          if (fabs(apq) > 1e-13 * (fabs(app) + fabs(aqq)) + 1e-300) {
            const double tau = (aqq - app) * frcp(2.0 * apq);
            double t;
            if (fabs(tau) > 1e14) {
              t = 0.5 / tau;
            } else {
              const double u = fma(tau, tau, 1.0);
              const double root = u * frsqrt(u);
              t = (tau >= 0.0) ? frcp(tau + root) : -frcp(root - tau);
            }
            c = frsqrt(fma(t, t, 1.0));
            s = t * c;
            atomicAdd(&nrot, 1);
          }
          cs[i] = c;
          sn[i] = s;
        }
        __syncthreads();
        for (int q2 = tid; q2 < (kp / 2) * kp; q2 += RR_T) {
          const int i = q2 / kp, j = q2 - i * kp;
          if (sn[i] == 0.0) continue;
          int p, q;
          jacobi_pair_k(step, i, kp, p, q);
          const double x = H[p * RR_KLD + j], y = H[q * RR_KLD + j];
          H[p * RR_KLD + j] = cs[i] * x - sn[i] * y;
          H[q * RR_KLD + j] = sn[i] * x + cs[i] * y;
        }
        __syncthreads();
        for (int q2 = tid; q2 < (kp / 2) * kp; q2 += RR_T) {
          const int i = q2 / kp, r = q2 - i * kp;
          if (sn[i] == 0.0) continue;
          int p, q;
          jacobi_pair_k(step, i, kp, p, q);
          const double x = H[r * RR_KLD + p], y = H[r * RR_KLD + q];
          H[r * RR_KLD + p] = cs[i] * x - sn[i] * y;
          H[r * RR_KLD + q] = sn[i] * x + cs[i] * y;
          const double vx = Vk[r * RR_KLD + p], vy = Vk[r * RR_KLD + q];
          Vk[r * RR_KLD + p] = cs[i] * vx - sn[i] * vy;
          Vk[r * RR_KLD + q] = sn[i] * vx + cs[i] * vy;
        }
        __syncthreads();
      }
      if (nrot == 0) break;
      __syncthreads();
    }
  }
  for (int i = tid; i < k; i += RR_T) {
    const double li = H[i * RR_KLD + i];
    int rank = 0;
    for (int j = 0; j < k; ++j) {
      const double lj = H[j * RR_KLD + j];
      rank += (lj < li) || (lj == li && j < i);
    }
    perm[rank] = i;
  }
  __syncthreads();
  // Z <- Z Vk[:, perm], row by row
  for (int r = tid; r < m; r += RR_T) {
    double zr[RR_KMAX];
    for (int i = 0; i < k; ++i) zr[i] = Z[r * RR_KLD + i];
    for (int j = 0; j < k; ++j) {
      const int col = perm[j];
      double s = 0.0;
      for (int i = 0; i < k; ++i) s = fma(zr[i], Vk[i * RR_KLD + col], s);
      Z[r * RR_KLD + j] = s;
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- 7. back-transform, C
  // each warp applies all reflectors, last to first, to its own columns
  for (int c = wid; c < k; c += RR_T / 32) {
    for (int j = m - 3; j >= 0; --j) {
      const double beta = bet[j];
      if (beta == 0.0) continue;
      const int n1 = m - j - 1;
      const double* col = M + (j + 1) * RR_LD + j;
      double s = 0.0;
      for (int i = lane; i < n1; i += 32) s = fma(col[i * RR_LD], Z[(j + 1 + i) * RR_KLD + c], s);
      s = beta * warp_sum(s);
      for (int i = lane; i < n1; i += 32)
        Z[(j + 1 + i) * RR_KLD + c] = fma(-col[i * RR_LD], s, Z[(j + 1 + i) * RR_KLD + c]);
      __syncwarp();
    }
  }
  __syncthreads();
  // C = R^-T Z: rows from the bottom, all columns in parallel
  for (int i = m - 1; i >= 0; --i) {
    for (int c = tid; c < k; c += RR_T) Z[i * RR_KLD + c] *= rdg[i];
    __syncthreads();
    for (int q = tid; q < i * k; q += RR_T) {
      const int p = q / k, c = q - p * k;
      Z[p * RR_KLD + c] = fma(-R[i * RR_LD + p], Z[i * RR_KLD + c], Z[p * RR_KLD + c]);
    }
    __syncthreads();
  }
  for (int q = tid; q < a.m * k; q += RR_T) {
    const int r = q / k, c = q - r * k;
    a.C[q] = (r < m) ? Z[r * RR_KLD + c] * sc[r] : 0.0;
  }
  if (tid < k) {
    const double th = H[perm[tid] * RR_KLD + perm[tid]];
    a.theta[tid] = th;
    if (a.theta_hist) a.theta_hist[tid] = th;
    if (!isfinite(th)) *a.status = 3;
  }
  if (tid == 0 && dropped && a.restarts) *a.restarts += 1;
  if (!a.Cp) return;
  // Coefficients of the next P, B-orthogonal to the next X:  Cw = C with the X rows
  // zeroed,  Z2 = C^T G_B Cw  (k x k),  Cp = Cw - C Z2.
  __syncthreads();
  const int mm = a.m;
  double* Cs = M;                    // [mm][k]
  double* T1 = M + mm * k;           // [mm][k]
  double* Z2 = T1 + mm * k;          // [k][k]
  for (int q = tid; q < mm * k; q += RR_T) Cs[q] = a.C[q];
  __syncthreads();
  const double* GBg = a.G + (size_t)mm * mm;
  for (int q = tid; q < mm * k; q += RR_T) {
    const int r = q / k, j = q - r * k;
    double acc0 = 0.0, acc1 = 0.0;
    int b = k;
    for (; b + 1 < mm; b += 2) {
      acc0 = fma(GBg[r * mm + b], Cs[b * k + j], acc0);
      acc1 = fma(GBg[r * mm + b + 1], Cs[(b + 1) * k + j], acc1);
    }
    if (b < mm) acc0 = fma(GBg[r * mm + b], Cs[b * k + j], acc0);
    T1[q] = acc0 + acc1;
  }
  __syncthreads();
  for (int q = tid; q < k * k; q += RR_T) {
    const int i = q / k, j = q - i * k;
    double acc0 = 0.0, acc1 = 0.0;
    int r = 0;
    for (; r + 1 < mm; r += 2) {
      acc0 = fma(Cs[r * k + i], T1[r * k + j], acc0);
      acc1 = fma(Cs[(r + 1) * k + i], T1[(r + 1) * k + j], acc1);
    }
    if (r < mm) acc0 = fma(Cs[r * k + i], T1[r * k + j], acc0);
    Z2[q] = acc0 + acc1;
  }
  __syncthreads();
  for (int q = tid; q < mm * k; q += RR_T) {
    const int r = q / k, j = q - r * k;
    double acc = (r >= k) ? Cs[q] : 0.0;
    for (int i = 0; i < k; ++i) acc = fma(-Cs[r * k + i], Z2[i * k + j], acc);
    a.Cp[q] = acc;
  }
}

size_t rr_smem_bytes() {
  return (size_t)(2 * RR_MMAX * RR_LD + RR_MMAX * RR_KLD + 2 * RR_KMAX * RR_KLD + 7 * RR_MMAX +
                  3 * RR_KMAX) * sizeof(double) + 2 * RR_MMAX * sizeof(float) + RR_KMAX * sizeof(int);
}

}  // namespace

int bf_rr_launch(const RRParams& a, cudaStream_t s) {
  static bool init = false;
  const size_t sm = rr_smem_bytes();
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(k_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return bf_cuda_fail(e, "cudaFuncSetAttribute(k_rr)");
    init = true;
  }
  BF_LAUNCH(k_rr<<<1, RR_T, sm, s>>>(a));
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
  return bf_rr_launch(a, (cudaStream_t)stream);
}
