// The small Rayleigh-Ritz problem of block LOBPCG (Algorithm 3, Section 6), solved in
// FP64 by one CTA: the k smallest eigenpairs of the pencil (G_A, G_B) of size m <= 96.
//
// GB300 runs FP64 at 1/64 of the FP32 rate, so the solver is built to keep FP64 work near
// m^3 instead of the ~36 m^3 of a cyclic Jacobi eigensolver:
//   1. symmetrise, scale to unit diag(G_B), Cholesky G_B = R R^T (a squared pivot
//      <= 1e-10 means a dependent trial basis: retry on the leading m_nop block, i.e.
//      without P, else report a breakdown);
//   2. standard form M = R^-1 G_A R^-T by two in-place triangular solves;
//   3. Householder reduction M = Q T Q^T to a tridiagonal T (reflectors kept in M);
//   4. the k smallest eigenvalues of T by bisection on Sturm counts (sign changes of
//      the characteristic-polynomial recurrence, rescaled by powers of two: no division);
//   5. one eigenvector per eigenvalue by two steps of inverse iteration on T - lambda I
//      (tridiagonal elimination with row interchanges), all k in parallel;
//   6. modified Gram-Schmidt (twice) on those k vectors and a k x k Rayleigh-Ritz on T
//      (cyclic Jacobi; the matrix is diagonal up to rounding except inside clusters);
//   7. back-transformation by the reflectors, C = R^-T Y and the unit-diagonal scaling
//      undone; with Cp requested, the coefficients of the next P made B-orthogonal to
//      the next X (see the driver).
#include <math.h>

#include "bf_internal.cuh"
#include "bf_rr.cuh"

#define RR_T 512
#define RR_LD 97            // padded leading dimension of the m x m work matrices
#define RR_KLD 33           // padded leading dimension of the m x k work matrices
#define DEP_TOL 1e-10

namespace {

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < RR_T / 32; ++w) s += red[w];
  return s;
}

// Number of eigenvalues of the symmetric tridiagonal T (diagonal d, squared off-diagonal
// e2) smaller than x: sign changes along p_0 = 1, p_1 = d_0 - x,
// p_i = (d_{i-1} - x) p_{i-1} - e2_{i-2} p_{i-2}.  A zero p_i is counted as a sign change
// (as if it were a tiny number of the opposite sign).  The pair (p_{i-1}, p_i) is
// rescaled by a power of two whenever p_i leaves [2^-600, 2^600].
__device__ int sturm_count(const double* d, const double* e2, int m, double x) {
  double p0 = 1.0, p1 = d[0] - x;
  int cnt = 0;
  if (p1 == 0.0) p1 = -0x1p-200;
  cnt += (p1 < 0.0);
  for (int i = 1; i < m; ++i) {
    double p2 = (d[i] - x) * p1 - e2[i - 1] * p0;
    if (p2 == 0.0) p2 = -p1 * 0x1p-200;
    cnt += ((p2 < 0.0) != (p1 < 0.0));
    p0 = p1;
    p1 = p2;
    const double a = fabs(p1);
    if (a > 0x1p600 || a < 0x1p-600) {
      const double sc = scalbn(1.0, -ilogb(p1));
      p0 *= sc;
      p1 *= sc;
    }
  }
  return cnt;
}

// Solve (T - lambda I) x = b in place (b -> x) by elimination with row interchanges:
// the working row (pivot candidates in columns i, i+1, i+2) is compared with the next
// original row and the larger entry in column i is the pivot.  u0/u1/u2 hold the rows of
// U, y the transformed right-hand side.  Zero pivots are replaced by `tiny`.
__device__ void tri_solve(const double* d, const double* e, int m, double lambda, double tiny,
                          double* b, double* u0, double* u1, double* u2) {
  double r0 = d[0] - lambda, r1 = (m > 1) ? e[0] : 0.0, r2 = 0.0, rb = b[0];
  for (int i = 0; i < m - 1; ++i) {
    const double n0 = e[i], n1 = d[i + 1] - lambda, n2 = (i + 2 < m) ? e[i + 1] : 0.0;
    const double nb = b[i + 1];
    double p0, p1, p2, pb, o0, o1, o2, ob;
    if (fabs(r0) >= fabs(n0)) {
      p0 = r0; p1 = r1; p2 = r2; pb = rb;
      o0 = n0; o1 = n1; o2 = n2; ob = nb;
    } else {
      p0 = n0; p1 = n1; p2 = n2; pb = nb;
      o0 = r0; o1 = r1; o2 = r2; ob = rb;
    }
    if (p0 == 0.0) p0 = tiny;
    const double f = o0 / p0;
    u0[i] = p0;
    u1[i] = p1;
    u2[i] = p2;
    b[i] = pb;
    r0 = o1 - f * p1;
    r1 = o2 - f * p2;
    r2 = 0.0;
    rb = ob - f * pb;
  }
  if (r0 == 0.0) r0 = tiny;
  u0[m - 1] = r0;
  b[m - 1] = rb;
  // back substitution
  b[m - 1] /= u0[m - 1];
  if (m > 1) b[m - 2] = (b[m - 2] - u1[m - 2] * b[m - 1]) / u0[m - 2];
  for (int i = m - 3; i >= 0; --i) b[i] = (b[i] - u1[i] * b[i + 1] - u2[i] * b[i + 2]) / u0[i];
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
  double* sc = Vk + RR_KMAX * RR_KLD;                   // [96]
  double* tv = sc + RR_MMAX;                            // [96]
  double* dd = tv + RR_MMAX;                            // [96] diagonal of T
  double* ee = dd + RR_MMAX;                            // [96] off-diagonal of T
  double* e2 = ee + RR_MMAX;                            // [96] squared off-diagonal
  double* bet = e2 + RR_MMAX;                           // [96] reflector scalars
  double* pv = bet + RR_MMAX;                           // [96] work vector
  double* lam = pv + RR_MMAX;                           // [32]
  double* cs = lam + RR_KMAX;                           // [16]
  double* sn = cs + RR_KMAX / 2;                        // [16]
  double* red = sn + RR_KMAX / 2;                       // [32]
  int* perm = reinterpret_cast<int*>(red + 32);         // [32]
  __shared__ int fail, dropped, nrot;
  __shared__ double sh_alpha, sh_beta, sh_v0, sh_K, sh_lo, sh_hi;
  const int tid = threadIdx.x;
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
      sc[r] = (dg > 0.0) ? 1.0 / sqrt(dg) : 0.0;
    }
    __syncthreads();
    if (!fail) {
      for (int q = tid; q < m * m; q += RR_T) {
        const int r = q / m, c = q - r * m;
        M[r * RR_LD + c] *= sc[r] * sc[c];
        R[r * RR_LD + c] *= sc[r] * sc[c];
      }
      __syncthreads();
      for (int j = 0; j < m && !fail; ++j) {
        for (int i = j + tid; i < m; i += RR_T) {
          double s = R[i * RR_LD + j];
          for (int p = 0; p < j; ++p) s -= R[i * RR_LD + p] * R[j * RR_LD + p];
          tv[i] = s;
        }
        __syncthreads();
        if (tid == 0) {
          if (!(tv[j] > DEP_TOL)) fail = 1;
          else tv[j] = sqrt(tv[j]);
        }
        __syncthreads();
        if (!fail)
          for (int i = j + tid; i < m; i += RR_T) R[i * RR_LD + j] = (i == j) ? tv[j] : tv[i] / tv[j];
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
  for (int c = tid; c < m; c += RR_T) {          // Y = R^-1 M, column c in place
    for (int i = 0; i < m; ++i) {
      double s = M[i * RR_LD + c];
      for (int p = 0; p < i; ++p) s -= R[i * RR_LD + p] * M[p * RR_LD + c];
      M[i * RR_LD + c] = s / R[i * RR_LD + i];
    }
  }
  __syncthreads();
  for (int r = tid; r < m; r += RR_T) {          // Z = Y R^-T, row r in place
    for (int i = 0; i < m; ++i) {
      double s = M[r * RR_LD + i];
      for (int p = 0; p < i; ++p) s -= R[i * RR_LD + p] * M[r * RR_LD + p];
      M[r * RR_LD + i] = s / R[i * RR_LD + i];
    }
  }
  __syncthreads();
  for (int q = tid; q < m * m; q += RR_T) {
    const int r = q / m, c = q - r * m;
    if (r < c) {
      const double v = 0.5 * (M[r * RR_LD + c] + M[c * RR_LD + r]);
      M[r * RR_LD + c] = v;
      M[c * RR_LD + r] = v;
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- 3. tridiagonal
  for (int j = 0; j + 2 < m; ++j) {
    const int n1 = m - j - 1;
    double* col = M + (j + 1) * RR_LD + j;       // x_i = col[i * RR_LD]
    if (tid < 32) {
      double s = 0.0;
      for (int i = tid; i < n1; i += 32) s += col[i * RR_LD] * col[i * RR_LD];
      s = warp_sum(s);
      if (tid == 0) {
        const double x0 = col[0];
        const double tail = s - x0 * x0;
        if (!(tail > 0.0)) {
          sh_beta = 0.0;
          sh_alpha = x0;
          sh_v0 = 0.0;
        } else {
          const double al = (x0 >= 0.0) ? -sqrt(s) : sqrt(s);
          const double v0 = x0 - al;
          sh_alpha = al;
          sh_v0 = v0;
          sh_beta = 2.0 / (tail + v0 * v0);
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
    // p = beta A1 v  (four threads per row)
    {
      const int row = tid >> 2, part = tid & 3;
      double s = 0.0;
      if (row < n1)
        for (int c = part; c < n1; c += 4) s += A1[row * RR_LD + c] * col[c * RR_LD];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (row < n1 && part == 0) pv[row] = beta * s;
    }
    __syncthreads();
    if (tid < 32) {
      double s = 0.0;
      for (int i = tid; i < n1; i += 32) s += col[i * RR_LD] * pv[i];
      s = warp_sum(s);
      if (tid == 0) sh_K = 0.5 * beta * s;
    }
    __syncthreads();
    for (int i = tid; i < n1; i += RR_T) pv[i] -= sh_K * col[i * RR_LD];   // w
    __syncthreads();
    for (int q = tid; q < n1 * n1; q += RR_T) {
      const int r = q / n1, c = q - r * n1;
      A1[r * RR_LD + c] -= col[r * RR_LD] * pv[c] + pv[r] * col[c * RR_LD];
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
    // Gershgorin interval
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
      const double rad = fabs(ee[i]) + (i > 0 ? fabs(ee[i - 1]) : 0.0);
      lo = fmin(lo, dd[i] - rad);
      hi = fmax(hi, dd[i] + rad);
    }
    sh_lo = lo;
    sh_hi = hi;
  }
  __syncthreads();
  for (int i = tid; i < m; i += RR_T) e2[i] = ee[i] * ee[i];
  __syncthreads();
  const double tn = fmax(fabs(sh_lo), fabs(sh_hi));
  const double tiny = 4.0 * 2.2e-16 * tn + 1e-300;

  // ---------------------------------------------------------------- 4-5. bisection, inverse iteration
  if (tid < k) {
    double lo = sh_lo, hi = sh_hi;
    for (int it = 0; it < 80 && hi - lo > tiny; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (sturm_count(dd, e2, m, mid) > tid) hi = mid;
      else lo = mid;
    }
    const double lmb = 0.5 * (lo + hi);
    lam[tid] = lmb;
    double b[RR_MMAX], u0[RR_MMAX], u1[RR_MMAX], u2[RR_MMAX];
    for (int i = 0; i < m; ++i) b[i] = 1.0 + 0.25 * (double)(((i + 1) * (tid + 3) * 7919) % 97) / 97.0;
    for (int rep = 0; rep < 2; ++rep) {
      tri_solve(dd, ee, m, lmb, tiny, b, u0, u1, u2);
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm = fmax(nrm, fabs(b[i]));
      const double inv = (nrm > 0.0 && isfinite(nrm)) ? 1.0 / nrm : 1.0;
      for (int i = 0; i < m; ++i) b[i] *= inv;
    }
    for (int i = 0; i < m; ++i) Z[i * RR_KLD + tid] = b[i];
  }
  __syncthreads();

  // ---------------------------------------------------------------- 6. MGS twice, k x k Rayleigh-Ritz
  for (int j = 0; j < k; ++j) {
    for (int pass = 0; pass < 2; ++pass) {
      // dots with the finished columns i < j: warp w takes columns w, w + 16, ...
      const int lane = tid & 31, wid = tid >> 5;
      for (int i = wid; i < j; i += RR_T / 32) {
        double s = 0.0;
        for (int r = lane; r < m; r += 32) s += Z[r * RR_KLD + i] * Z[r * RR_KLD + j];
        s = warp_sum(s);
        if (lane == 0) H[i] = s;
      }
      __syncthreads();
      for (int r = tid; r < m; r += RR_T) {
        double v = Z[r * RR_KLD + j];
        for (int i = 0; i < j; ++i) v -= H[i] * Z[r * RR_KLD + i];
        Z[r * RR_KLD + j] = v;
      }
      __syncthreads();
    }
    double s = 0.0;
    for (int r = tid; r < m; r += RR_T) s += Z[r * RR_KLD + j] * Z[r * RR_KLD + j];
    s = block_sum_d(s, red);
    const double inv = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    for (int r = tid; r < m; r += RR_T) Z[r * RR_KLD + j] *= inv;
    __syncthreads();
  }
  // H = Z^T T Z
  for (int q = tid; q < k * k; q += RR_T) {
    const int i = q / k, j = q - i * k;
    double s = 0.0;
    for (int r = 0; r < m; ++r) {
      double tz = dd[r] * Z[r * RR_KLD + j];
      if (r > 0) tz += ee[r - 1] * Z[(r - 1) * RR_KLD + j];
      if (r + 1 < m) tz += ee[r] * Z[(r + 1) * RR_KLD + j];
      s += Z[r * RR_KLD + i] * tz;
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
          if (apq != 0.0 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (fabs(tau) > 1e150) ? 0.5 / tau
                                                   : ((tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                                                   : -1.0 / (-tau + sqrt(1.0 + tau * tau)));
            c = 1.0 / sqrt(1.0 + t * t);
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
      for (int i = 0; i < k; ++i) s += zr[i] * Vk[i * RR_KLD + col];
      Z[r * RR_KLD + j] = s;
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- 7. back-transform, C
  for (int j = m - 3; j >= 0; --j) {
    const double beta = bet[j];
    if (beta == 0.0) continue;
    const int n1 = m - j - 1;
    const double* col = M + (j + 1) * RR_LD + j;
    // dots v^T Z[j+1.., c] for every column c (one warp per column)
    const int lane = tid & 31, wid = tid >> 5;
    for (int c = wid; c < k; c += RR_T / 32) {
      double s = 0.0;
      for (int i = lane; i < n1; i += 32) s += col[i * RR_LD] * Z[(j + 1 + i) * RR_KLD + c];
      s = warp_sum(s);
      if (lane == 0) pv[c] = beta * s;
    }
    __syncthreads();
    for (int q = tid; q < n1 * k; q += RR_T) {
      const int i = q / k, c = q - i * k;
      Z[(j + 1 + i) * RR_KLD + c] -= col[i * RR_LD] * pv[c];
    }
    __syncthreads();
  }
  // C = R^-T Z: columns in parallel, 16 lanes per column
  {
    const int c = tid >> 4, l16 = tid & 15;
    for (int i = m - 1; i >= 0; --i) {
      double s = 0.0;
      if (c < k)
        for (int p = i + 1 + l16; p < m; p += 16) s += R[p * RR_LD + i] * Z[p * RR_KLD + c];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      s += __shfl_xor_sync(0xffffffffu, s, 8);
      if (c < k && l16 == 0) Z[i * RR_KLD + c] = (Z[i * RR_KLD + c] - s) / R[i * RR_LD + i];
      __syncwarp();
    }
  }
  __syncthreads();
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
    double acc = 0.0;
    for (int b = k; b < mm; ++b) acc += 0.5 * (GBg[r * mm + b] + GBg[b * mm + r]) * Cs[b * k + j];
    T1[q] = acc;
  }
  __syncthreads();
  for (int q = tid; q < k * k; q += RR_T) {
    const int i = q / k, j = q - i * k;
    double acc = 0.0;
    for (int r = 0; r < mm; ++r) acc += Cs[r * k + i] * T1[r * k + j];
    Z2[q] = acc;
  }
  __syncthreads();
  for (int q = tid; q < mm * k; q += RR_T) {
    const int r = q / k, j = q - r * k;
    double acc = (r >= k) ? Cs[q] : 0.0;
    for (int i = 0; i < k; ++i) acc -= Cs[r * k + i] * Z2[i * k + j];
    a.Cp[q] = acc;
  }
}

size_t rr_smem_bytes() {
  return (size_t)(2 * RR_MMAX * RR_LD + RR_MMAX * RR_KLD + 2 * RR_KMAX * RR_KLD + 7 * RR_MMAX +
                  RR_KMAX + RR_KMAX + 32) * sizeof(double) + RR_KMAX * sizeof(int);
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
