// The guided filter of Section 3 as a graph operator (Algorithm 1, Eqs. 5-6).
//
// Windows omega_k (square, radius r; 1D: an interval) are truncated at the border: N_k
// in-image pixels, mu_k and sigma_k^2 their mean and variance.  The symmetric matrix
//   Wt_ij = sum_{k : i, j in omega_k} (1 / N_k) (1 + (g_i - mu_k)(g_j - mu_k) / (sigma_k^2 + eps))
// has row sums N_i, so D = diag(N), L = D - Wt, and Algorithm 1 computes y = D^-1 Wt x;
// away from the border Wt / |omega| is Eq. 6.
//
// The apply works in difference form so that smooth vectors (L x << D x) keep their
// relative accuracy: per window k (stage A)
//   d_k = sum_j (x_j - x_k) / N_k,   a_k = sum_j (g_j - mu_k)(x_j - x_k) / N_k / (sigma_k^2 + eps)
// and per pixel i (stage B)
//   (L x)_i = sum_{k : i in omega_k} [(x_i - x_k) - d_k - (g_i - mu_k) a_k],
// which equals N_i x_i - sum_k (mean_k(x) + (g_i - mu_k) a_k) because the deviations
// g_j - mu_k sum to zero over a window.  Every term is a difference of nearby values.
#include <math.h>

#include <algorithm>

#include "bf_internal.cuh"

#define GF_KC 4             // columns per pass of the apply (1 for a single column)

namespace {

struct GfGeom {
  int nx, ny, r, ry;        // ry = r (2D) or 0 (1D)
};

// N_k, mu_k, 1 / (sigma_k^2 + eps) of every window (two passes over it: the mean, then the
// mean squared deviation), and d = N, 1/d, d^-1/2; a non-finite guide value sets *flag.
template <typename T>
__global__ void __launch_bounds__(256) k_guided_prep(const GfGeom gg, const T* __restrict__ guide, T eps,
                                                     int64_t n, T* d, T* dinv, T* dis, T* dls, T* mu,
                                                     T* ivar, int* flag) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int ky = (int)(k / gg.nx), kx = (int)(k - (int64_t)ky * gg.nx);
    const int y0 = max(ky - gg.ry, 0), y1 = min(ky + gg.ry, gg.ny - 1);
    const int x0 = max(kx - gg.r, 0), x1 = min(kx + gg.r, gg.nx - 1);
    T s = T(0);
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) s += guide[(int64_t)y * gg.nx + x];
    const T cnt = (T)((y1 - y0 + 1) * (x1 - x0 + 1));
    const T m = s / cnt;
    T v = T(0);
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) {
        const T dv = guide[(int64_t)y * gg.nx + x] - m;
        v = fma(dv, dv, v);
      }
    const T var = v / cnt;
    if (!isfinite(m) || !isfinite(var)) *flag = 1;
    mu[k] = m;
    ivar[k] = T(1) / (var + eps);
    d[k] = cnt;
    dinv[k] = T(1) / cnt;
    dis[k] = T(1) / sqrt(cnt);
    dls[k] = T(0);
  }
}

template <typename T>
struct GfApply {
  const T* X;
  int64_t ldx;
  T* Y;
  int64_t ldy;
  int k;
  int op;
  const T* guide;           // the guide of the windows' statistics
  const T* mu;
  const T* ivar;
  const T* d;               // N
  const T* dis;             // N^-1/2 (NSYM)
  double* dots;             // [k] or NULL: x^T y per column
};

// Stage A sum of window k (staged at sk): ds = sum_j (x_j - x_k), cs = sum_j (g_j - mu_k)(x_j - x_k)
// over the window's in-image members (CHECK: near the border; else all are in the image).
template <typename T, int KC, int RT, bool ONED, bool CHECK>
__device__ __forceinline__ int gf_stage_a(int r, int hw, int nx, int ny, int kx, int ky, const Vec<T, KC>* sx,
                                          const T* sg, int sk, T muk, Vec<T, KC>& ds, Vec<T, KC>& cs) {
  const int rr = RT > 0 ? RT : r;
  const int ry = ONED ? 0 : rr;
  const Vec<T, KC> xk = sx[sk];
  int cnt = 0;
#pragma unroll
  for (int dy = -ry; dy <= ry; ++dy) {
    if (CHECK && (ky + dy < 0 || ky + dy >= ny)) continue;
#pragma unroll
    for (int dx = -rr; dx <= rr; ++dx) {
      if (CHECK && (kx + dx < 0 || kx + dx >= nx)) continue;
      const int sj = sk + dy * hw + dx;
      const T gd = sg[sj] - muk;
      const Vec<T, KC> xj = sx[sj];
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const T xd = xj.v[c] - xk.v[c];
        ds.v[c] += xd;
        cs.v[c] = fma(gd, xd, cs.v[c]);
      }
      ++cnt;
    }
  }
  return cnt;
}

// Stage B sum of pixel i (staged at si, region-A position qi): the windows containing it.
template <typename T, int KC, int RT, bool ONED, bool CHECK>
__device__ __forceinline__ void gf_stage_b(int r, int hw, int aw, int nx, int ny, int ix, int iy, const Vec<T, KC>* sx,
                                           const Vec<T, KC>* sdk, const Vec<T, KC>* sak, const T* smu,
                                           int si, int qi, T gi, const Vec<T, KC>& xi, T (&lv)[KC]) {
  const int rr = RT > 0 ? RT : r;
  const int ry = ONED ? 0 : rr;
#pragma unroll
  for (int dy = -ry; dy <= ry; ++dy) {
    if (CHECK && (iy + dy < 0 || iy + dy >= ny)) continue;
#pragma unroll
    for (int dx = -rr; dx <= rr; ++dx) {
      if (CHECK && (ix + dx < 0 || ix + dx >= nx)) continue;
      const int qa = qi + dy * aw + dx;
      const int sk = si + dy * hw + dx;
      const T gdi = gi - smu[qa];
      const Vec<T, KC> xk = sx[sk], dk = sdk[qa], ak = sak[qa];
#pragma unroll
      for (int c = 0; c < KC; ++c) lv[c] += ((xi.v[c] - xk.v[c]) - dk.v[c]) - gdi * ak.v[c];
    }
  }
}

// One TW x TH tile of outputs (one per thread); x and g staged on the tile plus a halo of
// 2r, the windows' d_k and a_k on the tile plus r, KC columns per pass interleaved in
// shared memory (one vector load per tap).  RT > 0: the radius at compile time.  Tiles
// whose staged region lies inside the image skip all border tests.
template <typename T, int KC, int TW, int TH, int RT>
__global__ void __launch_bounds__(TW * TH) k_guided_apply(const GfGeom gg, const GfApply<T> a) {
  static_assert(TW * TH == 256, "one output per thread");
  constexpr bool ONED = (TH == 1);
  typedef Vec<T, KC> V;
  extern __shared__ __align__(32) unsigned char smem[];
  const int r = RT > 0 ? RT : gg.r, ry = ONED ? 0 : r, nx = gg.nx, ny = gg.ny;
  const int hw = TW + 4 * r, hh = TH + 4 * ry, hp = hw * hh;
  const int aw = TW + 2 * r, ah = TH + 2 * ry, ap = aw * ah;
  V* sx = reinterpret_cast<V*>(smem);           // [hp] operand, KC columns
  V* sdk = sx + hp;                             // [ap] d_k
  V* sak = sdk + ap;                            // [ap] a_k
  T* sg = reinterpret_cast<T*>(sak + ap);       // [hp] guide
  T* smu = sg + hp;                             // [ap] mu_k
  T* siv = smu + ap;                            // [ap] 1 / (sigma_k^2 + eps)
  const int bx = blockIdx.x * TW, by = blockIdx.y * TH;
  const bool interior = bx - 2 * r >= 0 && bx + TW + 2 * r <= nx && by - 2 * ry >= 0 && by + TH + 2 * ry <= ny;
  for (int q = threadIdx.x; q < hp; q += TW * TH) {
    const int hy = q / hw, hx = q - hy * hw;
    const int gy = by - 2 * ry + hy, gx = bx - 2 * r + hx;
    sg[q] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? a.guide[(int64_t)gy * nx + gx] : T(0);
  }
  for (int q = threadIdx.x; q < ap; q += TW * TH) {
    const int ay = q / aw, ax = q - ay * aw;
    const int gy = by - ry + ay, gx = bx - r + ax;
    const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    smu[q] = in ? a.mu[(int64_t)gy * nx + gx] : T(0);
    siv[q] = in ? a.ivar[(int64_t)gy * nx + gx] : T(0);
  }
  const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
  const int ix = bx + lx, iy = by + ly;
  const bool act = ix < nx && iy < ny;
  const int64_t i = (int64_t)iy * nx + ix;
  const int si = (ly + 2 * ry) * hw + (lx + 2 * r);
  const int qi = (ly + ry) * aw + (lx + r);
  const bool nsym = (a.op == BF_OP_NSYM);
  T* sxs = reinterpret_cast<T*>(sx);
  for (int c0 = 0; c0 < a.k; c0 += KC) {
    __syncthreads();                            // the previous pass's readers are done
    for (int q = threadIdx.x; q < hp * KC; q += TW * TH) {
      const int p = q / KC, c = q - p * KC;
      const int hy = p / hw, hx = p - hy * hw;
      const int gy = by - 2 * ry + hy, gx = bx - 2 * r + hx;
      T v = T(0);
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && c0 + c < a.k) {
        const int64_t gp = (int64_t)gy * nx + gx;
        v = a.X[gp * a.ldx + c0 + c];
        if (nsym) v *= a.dis[gp];
      }
      sxs[q] = v;                               // = sx[p].v[c]
    }
    __syncthreads();
    // stage A: the windows centred on the tile plus r
    for (int q = threadIdx.x; q < ap; q += TW * TH) {
      const int ay = q / aw, ax = q - ay * aw;
      const int ky = by - ry + ay, kx = bx - r + ax;
      V ds, cs;
#pragma unroll
      for (int c = 0; c < KC; ++c) ds.v[c] = cs.v[c] = T(0);
      if (kx >= 0 && kx < nx && ky >= 0 && ky < ny) {
        const int sk = (ay + ry) * hw + (ax + r);
        const int cnt = interior ? gf_stage_a<T, KC, RT, ONED, false>(r, hw, nx, ny, kx, ky, sx, sg, sk, smu[q], ds, cs)
                                 : gf_stage_a<T, KC, RT, ONED, true>(r, hw, nx, ny, kx, ky, sx, sg, sk, smu[q], ds, cs);
        const T inv = T(1) / (T)cnt, ivk = siv[q] * inv;
#pragma unroll
        for (int c = 0; c < KC; ++c) {
          ds.v[c] *= inv;
          cs.v[c] *= ivk;
        }
      }
      sdk[q] = ds;
      sak[q] = cs;
    }
    __syncthreads();
    // stage B: (L x)_i over the windows that contain i, then the operator's epilogue
    const V xi = sx[si];
    T lv[KC], yv[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) lv[c] = yv[c] = T(0);
    if (act) {
      const T gi = sg[si];
      if (interior) gf_stage_b<T, KC, RT, ONED, false>(r, hw, aw, nx, ny, ix, iy, sx, sdk, sak, smu, si, qi, gi, xi, lv);
      else          gf_stage_b<T, KC, RT, ONED, true>(r, hw, aw, nx, ny, ix, iy, sx, sdk, sak, smu, si, qi, gi, xi, lv);
      const T ni = a.d[i];
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        switch (a.op) {
          case BF_OP_W:      yv[c] = fma(ni, xi.v[c], -lv[c]); break;
          case BF_OP_DINV_W: yv[c] = xi.v[c] - lv[c] / ni; break;
          case BF_OP_D:      yv[c] = ni * xi.v[c]; break;
          case BF_OP_NSYM:   yv[c] = a.dis[i] * lv[c]; break;
          default:           yv[c] = lv[c]; break;        // L
        }
        if (c0 + c < a.k) a.Y[i * a.ldy + c0 + c] = yv[c];
      }
    }
    if (a.dots) {
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        if (c0 + c >= a.k) break;                 // the same in every thread
        const T xu = (act && nsym) ? a.X[i * a.ldx + c0 + c] : xi.v[c];
        const T s = warp_sum(act ? xu * yv[c] : T(0));
        if ((threadIdx.x & 31) == 0) atomicAdd(&a.dots[c0 + c], (double)s);
      }
    }
  }
}

template <typename T, int KC, int TW, int TH, int RT>
static int launch_guided(const bf_graph* g, const GfApply<T>& a, cudaStream_t s) {
  const GfGeom gg{g->nx, g->ny, g->rx, g->ry};
  const size_t hp = (size_t)(TW + 4 * gg.r) * (TH + 4 * gg.ry);
  const size_t ap = (size_t)(TW + 2 * gg.r) * (TH + 2 * gg.ry);
  const size_t sm = ((1 + KC) * hp + (2 + 2 * KC) * ap) * sizeof(T);
  if (sm > 227 * 1024) return bf_fail(BF_EINVAL, "guided apply: window too large for shared memory");
  {
    const int rc_ = bf_smem_attr((const void*)k_guided_apply<T, KC, TW, TH, RT>, 227 * 1024,
                                 "cudaFuncSetAttribute(k_guided_apply)");
    if (rc_) return rc_;
  }
  const dim3 grid((unsigned)((g->nx + TW - 1) / TW), (unsigned)((g->ny + TH - 1) / TH), 1);
  BF_LAUNCH(k_guided_apply<T, KC, TW, TH, RT><<<grid, TW * TH, sm, s>>>(gg, a));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

// the radius at compile time for the common windows
template <typename T, int KC>
static int launch_guided_r(const bf_graph* g, const GfApply<T>& a, cudaStream_t s) {
  if (g->ny == 1 && g->ry == 0) {
    if (g->rx == 2) return launch_guided<T, KC, 256, 1, 2>(g, a, s);
    return launch_guided<T, KC, 256, 1, 0>(g, a, s);
  }
  switch (g->rx) {
    case 1: return launch_guided<T, KC, 32, 8, 1>(g, a, s);
    case 2: return launch_guided<T, KC, 32, 8, 2>(g, a, s);
    case 3: return launch_guided<T, KC, 32, 8, 3>(g, a, s);
  }
  return launch_guided<T, KC, 32, 8, 0>(g, a, s);
}

}  // namespace

// Y = op X for a guided graph (ops W, L, D^-1 W, D, D^-1/2 L D^-1/2), k columns.
template <typename T>
int bf_guided_apply(const bf_graph* g, int op, const T* X, int64_t ldx, int k, T* Y, int64_t ldy,
                    double* dots, const T* guide, cudaStream_t s) {
  if (op == BF_OP_NDIAGL) return bf_fail(BF_EINVAL, "bf_apply: (diag L)-normalised form not defined for a guided graph");
  if (op < BF_OP_W || op > BF_OP_NSYM) return bf_fail(BF_EINVAL, "bf_apply: bad op");
  GfApply<T> a;
  a.X = X;
  a.ldx = ldx;
  a.Y = Y;
  a.ldy = ldy;
  a.k = k;
  a.op = op;
  a.guide = guide ? guide : (const T*)g->guide;
  a.mu = (const T*)g->gmu;
  a.ivar = (const T*)g->givar;
  a.d = (const T*)g->d;
  a.dis = (const T*)g->dis;
  a.dots = dots;                                  // zeroed by the caller
  return k == 1 ? launch_guided_r<T, 1>(g, a, s) : launch_guided_r<T, GF_KC>(g, a, s);
}
template int bf_guided_apply<float>(const bf_graph*, int, const float*, int64_t, int, float*, int64_t,
                                    double*, const float*, cudaStream_t);
template int bf_guided_apply<double>(const bf_graph*, int, const double*, int64_t, int, double*, int64_t,
                                     double*, const double*, cudaStream_t);

// Window statistics of g for the guide `guide` (copied into g->guide); a non-finite value
// sets g->flag.
int bf_guided_prep(bf_graph* g, const void* guide, cudaStream_t s) {
  const size_t nb = (size_t)g->n * g->esize;
  BF_CUDA(cudaMemcpyAsync(g->guide, guide, nb, cudaMemcpyDeviceToDevice, s));
  const GfGeom gg{g->nx, g->ny, g->rx, g->ry};
  const unsigned blocks = (unsigned)std::min<int64_t>((g->n + 255) / 256, 65535);
  if (g->esize == 4)
    BF_LAUNCH(k_guided_prep<float><<<blocks, 256, 0, s>>>(gg, (const float*)g->guide, (float)g->eps, g->n,
                                                          (float*)g->d, (float*)g->dinv, (float*)g->dis,
                                                          (float*)g->dls, (float*)g->gmu, (float*)g->givar,
                                                          g->flag));
  else
    BF_LAUNCH(k_guided_prep<double><<<blocks, 256, 0, s>>>(gg, (const double*)g->guide, g->eps, g->n,
                                                           (double*)g->d, (double*)g->dinv, (double*)g->dis,
                                                           (double*)g->dls, (double*)g->gmu, (double*)g->givar,
                                                           g->flag));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}
