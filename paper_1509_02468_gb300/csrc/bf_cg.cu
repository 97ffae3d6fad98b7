// Algorithm 2 (Section 5): preconditioned CG for L x = 0 -- or the shifted system
// (L + sigma I) x = sigma x0 -- as a polynomial filter, with the flexible beta.
//
// Per iteration two kernels, all scalars kept on the device in FP64:
//   k_cg_dir:    p = s + beta p on the tile and its halo, q = (L + sigma I) p (matrix-free,
//                weights from the guide or the stored ones), block sums of p^T q, and in the
//                last block alpha = s^T r / p^T q with the breakdown tests;
//   k_cg_update: x += alpha p, r -= alpha q, s = T r, sums of s^T r, s^T q, s^T s, r^T r,
//                and in the last block beta for the next iteration:
//                s^T (r - r_old) = -alpha s^T q, divided by s_old^T r_old (flexible) or
//                s_old^T s_old (as printed).
// Once a kernel records a stop (converged, breakdown, non-finite) the remaining launches
// return at once, so the host loop needs no read-back.
#include <math.h>

#include <cmath>

#include <algorithm>
#include <mutex>

#include "bf_internal.cuh"
#include "bf_window_fast.cuh"
#include "bf_strip.cuh"

int bf_apply_f32(const bf_graph* g, int op, const float* X, int64_t ldx, int k, float* Y,
                 int64_t ldy, double* dots, cudaStream_t s);
int bf_apply_f64(const bf_graph* g, int op, const double* X, int64_t ldx, int k, double* Y,
                 int64_t ldy, double* dots, cudaStream_t s);
int bf_net_apply_f32(const bf_net* net, const bf_graph* g, const float* R, int64_t ldr, int k, float* Z,
                     int64_t ldz, cudaStream_t s, const int* stop);
int bf_spd_apply_f32(const bf_spd* T, const bf_graph* g, const float* R, int64_t ldr, int k, float* Z,
                     int64_t ldz, cudaStream_t s);

namespace {

int cg_num_sms() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 1;
  }
  return nsm;
}

enum { CG_RUN = 0, CG_CONV = 1, CG_BREAK = 2, CG_NONFINITE = 3 };
#define CG_POLL 64

// s = T r with the learned preconditioner (FP32 graphs; cg_filter checks the dtype)
inline int net_precond(const bf_net* net, const bf_graph* g, const float* r, float* s, cudaStream_t st,
                       const int* stop) {
  return bf_net_apply_f32(net, g, r, 1, 1, s, 1, st, stop);
}
inline int net_precond(const bf_net*, const bf_graph*, const double*, double*, cudaStream_t, const int*) {
  return bf_fail(BF_EINVAL, "cg_filter: the net preconditioner needs an FP32 graph");
}
// s = T r with the learned SPD preconditioner, or the net (the two T that are applied by
// kernels of their own after the update of x and r)
inline int own_precond(const bf_cg_opts& o, const bf_graph* g, const float* r, float* s, cudaStream_t st,
                       const int* stop) {
  if (o.precond == BF_PRECOND_SPD) return bf_spd_apply_f32(o.spd, g, r, 1, 1, s, 1, st);
  return net_precond(o.net, g, r, s, st, stop);
}
inline int own_precond(const bf_cg_opts& o, const bf_graph* g, const double* r, double* s, cudaStream_t st,
                       const int* stop) {
  if (o.precond == BF_PRECOND_SPD) return bf_fail(BF_EINVAL, "cg_filter: the SPD preconditioner needs an FP32 graph");
  return net_precond(o.net, g, r, s, st, stop);
}

struct CgState {
  double sr;        // s^T r of the current residual
  double ss;        // s^T s
  double rr;        // r^T r
  double pq;        // p^T q
  double alpha;
  double beta;      // beta to use in the next direction update
  double ref2;      // ||b||^2 (or ||r_0||^2 when b = 0)
  double tol2;
  int status;
  int iter;         // completed iterations
  int beta_mode;
  int pad;
  unsigned int counter;
  unsigned int pad2;
};

template <typename T>
struct CgArgs {
  const T* x0;
  T* x;
  T* r;
  T* s;
  T* q;
  const T* p_old;
  T* p_new;
  const T* guide;
  const T* dinv;       // Jacobi preconditioner (NULL: identity)
  const T* d;          // degree (the strip path divides by it)
  const void* wf;
  int wmode;
  int64_t n;
  T shift;
  int first;           // first iteration: p = s
  double* partials;
  CgState* st;
  double* hist;        // [2 kmax] or NULL
};

// The scalar state of a run, written on the device (so that a fixed-count run enqueues
// no host-to-device copy and can be captured in a CUDA graph).  The block counter of the
// grid reductions must start at zero.
__global__ void k_cg_state_init(CgState* st, double tol2, int beta_mode) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  CgState z;
  z.sr = z.ss = z.rr = z.pq = z.alpha = z.beta = z.ref2 = 0.0;
  z.tol2 = tol2;
  z.status = CG_RUN;
  z.iter = 0;
  z.beta_mode = beta_mode;
  z.pad = 0;
  z.counter = 0u;
  z.pad2 = 0u;
  *st = z;
}

// Stage one scalar field (with halo) into shared memory; `f(gp)` gives the value at an
// in-image pixel, 0 is stored outside.
template <typename T, class F>
__device__ __forceinline__ void stage1(const Geom<T>& g, const Tile& t, Vec<T, 1>* sx, T* sg,
                                       const T* guide, bool otf, F f) {
  for (int hp = threadIdx.x; hp < t.hp; hp += BF_THREADS) {
    const int hy = hp / t.hw, hx = hp - hy * t.hw;
    const int gy = t.by - g.ry + hy, gx = t.bx - g.rx + hx;
    T v = T(0), gv = T(0);
    if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) {
      const int64_t gp = (int64_t)gy * g.nx + gx;
      v = f(gp);
      if (otf) gv = guide[gp];
    }
    sx[hp].v[0] = v;
    if (otf) sg[hp] = gv;
  }
}

// r = -L x0 (= b - A x0 for either system), x = x0, s = T r; sums s^T r, s^T s, r^T r, x0^T x0.
template <typename T>
__global__ void __launch_bounds__(BF_THREADS) k_cg_init(const Geom<T> g, const CgArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[4 * (BF_THREADS / 32)];
  __shared__ int last;
  const Tile t = make_tile(g);
  Vec<T, 1>* sx = reinterpret_cast<Vec<T, 1>*>(smem);
  T* sg = reinterpret_cast<T*>(sx + t.hp);
  const bool otf = a.wmode == BF_W_ONTHEFLY;
  stage1<T>(g, t, sx, sg, a.guide, otf, [&](int64_t gp) { return a.x0[gp]; });
  __syncthreads();
  T v[4] = {T(0), T(0), T(0), T(0)};
  if (t.active) {
    const int64_t i = (int64_t)t.y * g.nx + t.x;
    T xi[1] = {sx[t.hp0].v[0]}, acc[1] = {T(0)}, ws = T(0);
    window_sum<T, 1, true>(g, t, sg, sx, a.wf, a.wmode, a.n, xi, acc, ws);
    const T r = -acc[0];
    const T s = a.dinv ? r * a.dinv[i] : r;
    a.x[i] = xi[0];
    a.r[i] = r;
    a.s[i] = s;
    v[0] = s * r;
    v[1] = s * s;
    v[2] = r * r;
    v[3] = xi[0] * xi[0];
  }
  double blk[4], tot[4];
  block_sum<4, T>(v, red, blk);
  if (grid_sum_last<4>(blk, a.partials, &a.st->counter, tot, &last)) {
    CgState* st = a.st;
    st->sr = tot[0];
    st->ss = tot[1];
    st->rr = tot[2];
    const double b2 = (double)a.shift * (double)a.shift * tot[3];
    st->ref2 = b2 > 0.0 ? b2 : tot[2];
    st->beta = 0.0;
    st->alpha = 0.0;
    st->iter = 0;
    st->status = (isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2])) ? CG_RUN : CG_NONFINITE;
  }
}

// p = s + beta p_old (first: p = s) on tile + halo, q = (L + shift I) p, p^T q, alpha.
template <typename T>
__global__ void __launch_bounds__(BF_THREADS) k_cg_dir(const Geom<T> g, const CgArgs<T> a) {
  if (a.st->status != CG_RUN) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[1 * (BF_THREADS / 32)];
  __shared__ int last;
  const Tile t = make_tile(g);
  Vec<T, 1>* sx = reinterpret_cast<Vec<T, 1>*>(smem);
  T* sg = reinterpret_cast<T*>(sx + t.hp);
  const bool otf = a.wmode == BF_W_ONTHEFLY;
  const T beta = (T)a.st->beta;
  if (a.first)
    stage1<T>(g, t, sx, sg, a.guide, otf, [&](int64_t gp) { return a.s[gp]; });
  else
    stage1<T>(g, t, sx, sg, a.guide, otf, [&](int64_t gp) { return fma(beta, a.p_old[gp], a.s[gp]); });
  __syncthreads();
  T v[1] = {T(0)};
  if (t.active) {
    const int64_t i = (int64_t)t.y * g.nx + t.x;
    T pi[1] = {sx[t.hp0].v[0]}, acc[1] = {T(0)}, ws = T(0);
    window_sum<T, 1, true>(g, t, sg, sx, a.wf, a.wmode, a.n, pi, acc, ws);
    const T q = fma(a.shift, pi[0], acc[0]);
    a.p_new[i] = pi[0];
    a.q[i] = q;
    v[0] = pi[0] * q;
  }
  double blk[1], tot[1];
  block_sum<1, T>(v, red, blk);
  if (grid_sum_last<1>(blk, a.partials, &a.st->counter, tot, &last)) {
    CgState* st = a.st;
    st->pq = tot[0];
    if (st->sr == 0.0) {
      st->status = CG_CONV;
    } else if (!isfinite(tot[0])) {
      st->status = CG_NONFINITE;
    } else if (!(tot[0] > 0.0)) {
      st->status = CG_BREAK;
    } else {
      st->alpha = st->sr / tot[0];
    }
  }
}

// Last block of an update: record alpha/beta, beta for the next direction from
// s^T (r - r_old) = -alpha s^T q, new sums, convergence and finiteness tests.
template <typename T>
__device__ void cg_step_tail(const CgArgs<T>& a, const double* tot) {
  CgState* st = a.st;
  const int it = st->iter;
  if (a.hist) {
    a.hist[2 * it] = st->alpha;
    a.hist[2 * it + 1] = a.first ? 0.0 : st->beta;
  }
  st->iter = it + 1;
  const double den = (st->beta_mode == BF_BETA_PRINTED) ? st->ss : st->sr;
  const double beta_next = -st->alpha * tot[1] / den;
  st->sr = tot[0];
  st->ss = tot[2];
  st->rr = tot[3];
  st->beta = beta_next;
  if (!(isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2]) && isfinite(tot[3])))
    st->status = CG_NONFINITE;
  else if (st->tol2 > 0.0 && tot[3] <= st->tol2 * st->ref2)
    st->status = CG_CONV;
}

// x += alpha p, r -= alpha q, s = T r; s^T r, s^T q, s^T s, r^T r; beta for the next step.
template <typename T>
__global__ void __launch_bounds__(BF_THREADS) k_cg_update(const CgArgs<T> a) {
  if (a.st->status != CG_RUN) return;
  __shared__ double red[4 * (BF_THREADS / 32)];
  __shared__ int last;
  const T alpha = (T)a.st->alpha;
  T v[4] = {T(0), T(0), T(0), T(0)};
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * BF_THREADS) {
    const T p = a.p_new[i], q = a.q[i];
    a.x[i] = fma(alpha, p, a.x[i]);
    const T r = fma(-alpha, q, a.r[i]);
    const T s = a.dinv ? r * a.dinv[i] : r;
    a.r[i] = r;
    a.s[i] = s;
    v[0] += s * r;
    v[1] += s * q;
    v[2] += s * s;
    v[3] += r * r;
  }
  double blk[4], tot[4];
  block_sum<4, T>(v, red, blk);
  if (grid_sum_last<4>(blk, a.partials, &a.st->counter, tot, &last)) cg_step_tail(a, tot);
}

// x += alpha p, r -= alpha q only: with the net preconditioner s = T r is computed next
// by its own kernels, then k_cg_sdots takes the sums.
template <typename T>
__global__ void __launch_bounds__(BF_THREADS) k_cg_xr(const CgArgs<T> a) {
  if (a.st->status != CG_RUN) return;
  const T alpha = (T)a.st->alpha;
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * BF_THREADS) {
    a.x[i] = fma(alpha, a.p_new[i], a.x[i]);
    a.r[i] = fma(-alpha, a.q[i], a.r[i]);
  }
}

// The sums of k_cg_update for a given s (the net's output); init: after k_cg_init only
// s^T r and s^T s are refreshed.
template <typename T>
__global__ void __launch_bounds__(BF_THREADS) k_cg_sdots(const CgArgs<T> a, int init) {
  if (a.st->status != CG_RUN) return;
  __shared__ double red[4 * (BF_THREADS / 32)];
  __shared__ int last;
  T v[4] = {T(0), T(0), T(0), T(0)};
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * BF_THREADS) {
    const T r = a.r[i], s = a.s[i], q = init ? T(0) : a.q[i];
    v[0] += s * r;
    v[1] += s * q;
    v[2] += s * s;
    v[3] += r * r;
  }
  double blk[4], tot[4];
  block_sum<4, T>(v, red, blk);
  if (grid_sum_last<4>(blk, a.partials, &a.st->counter, tot, &last)) {
    if (init) {
      a.st->sr = tot[0];
      a.st->ss = tot[2];
      if (!(isfinite(tot[0]) && isfinite(tot[2]))) a.st->status = CG_NONFINITE;
    } else {
      cg_step_tail(a, tot);
    }
  }
}

// ---- operator applied by its own kernel (guided graphs): q holds L x0, then L p
// x = x0, r = -L x0, s = T r and the sums of k_cg_init.
template <typename T>
__global__ void __launch_bounds__(BF_THREADS) k_cg_init_lx(const CgArgs<T> a) {
  __shared__ double red[4 * (BF_THREADS / 32)];
  __shared__ int last;
  T v[4] = {T(0), T(0), T(0), T(0)};
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * BF_THREADS) {
    const T x0 = a.x0[i], r = -a.q[i];
    const T s = a.dinv ? r * a.dinv[i] : r;
    a.x[i] = x0;
    a.r[i] = r;
    a.s[i] = s;
    v[0] += s * r;
    v[1] += s * s;
    v[2] += r * r;
    v[3] += x0 * x0;
  }
  double blk[4], tot[4];
  block_sum<4, T>(v, red, blk);
  if (grid_sum_last<4>(blk, a.partials, &a.st->counter, tot, &last)) {
    CgState* st = a.st;
    st->sr = tot[0];
    st->ss = tot[1];
    st->rr = tot[2];
    const double b2 = (double)a.shift * (double)a.shift * tot[3];
    st->ref2 = b2 > 0.0 ? b2 : tot[2];
    st->beta = 0.0;
    st->alpha = 0.0;
    st->iter = 0;
    st->status = (isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2])) ? CG_RUN : CG_NONFINITE;
  }
}

// p = s + beta p_old (first: p = s).
template <typename T>
__global__ void __launch_bounds__(BF_THREADS) k_cg_pdir(const CgArgs<T> a) {
  if (a.st->status != CG_RUN) return;
  const T beta = (T)a.st->beta;
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * BF_THREADS)
    a.p_new[i] = a.first ? a.s[i] : fma(beta, a.p_old[i], a.s[i]);
}

// q = L p (in q) + shift p, p^T q, alpha: the tail of k_cg_dir.
template <typename T>
__global__ void __launch_bounds__(BF_THREADS) k_cg_pq(const CgArgs<T> a) {
  if (a.st->status != CG_RUN) return;
  __shared__ double red[1 * (BF_THREADS / 32)];
  __shared__ int last;
  T v[1] = {T(0)};
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * BF_THREADS) {
    const T p = a.p_new[i];
    const T q = fma(a.shift, p, a.q[i]);
    a.q[i] = q;
    v[0] += p * q;
  }
  double blk[1], tot[1];
  block_sum<1, T>(v, red, blk);
  if (grid_sum_last<1>(blk, a.partials, &a.st->counter, tot, &last)) {
    CgState* st = a.st;
    st->pq = tot[0];
    if (st->sr == 0.0) {
      st->status = CG_CONV;
    } else if (!isfinite(tot[0])) {
      st->status = CG_NONFINITE;
    } else if (!(tot[0] > 0.0)) {
      st->status = CG_BREAK;
    } else {
      st->alpha = st->sr / tot[0];
    }
  }
}

// ---- specialised-window versions of k_cg_init / k_cg_dir (float graphs, common windows)
template <class SH, class F>
__device__ __forceinline__ void stage1_fast(const Geom<float>& g, int bx, int by, float* sx,
                                            float* sg, float* sval, const float* guide,
                                            bool need_guide, F f) {
  for (int hp = threadIdx.x; hp < SH::hp; hp += BF_THREADS) {
    const int hy = hp / SH::hw, hx = hp - hy * SH::hw;
    const int gy = by - SH::ry + hy, gx = bx - SH::rx + hx;
    const bool in = (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny);
    float v = 0.0f, gv = 0.0f;
    if (in) {
      const int64_t gp = (int64_t)gy * g.nx + gx;
      v = f(gp);
      if (need_guide) gv = guide[gp];
    }
    sx[hp] = v;
    if (need_guide) sg[hp] = gv;
    sval[hp] = in ? 1.0f : 0.0f;
  }
}

template <class SH, bool STORED>
__global__ void __launch_bounds__(BF_THREADS) k_cg_init_fast(const Geom<float> g, const CgArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[4 * (BF_THREADS / 32)];
  __shared__ int last;
  float* sx = reinterpret_cast<float*>(smem);
  float* sg = sx + SH::hp;
  float* sval = sg + SH::hp;
  const int ntx = (g.nx + SH::tw - 1) / SH::tw, ntiles = ntx * ((g.ny + SH::th - 1) / SH::th);
  const int lx = threadIdx.x % SH::tw, ly = threadIdx.x / SH::tw;
  const int hp0 = (ly + SH::ry) * SH::hw + (lx + SH::rx);
  float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {      // persistent over the tiles
    const int bx = (t % ntx) * SH::tw, by = (t / ntx) * SH::th;
    const bool mask = !(bx - SH::rx >= 0 && bx + SH::tw + SH::rx <= g.nx && by - SH::ry >= 0 &&
                        by + SH::th + SH::ry <= g.ny);
    __syncthreads();                                          // the previous tile is read
    stage1_fast<SH>(g, bx, by, sx, sg, sval, a.guide, !STORED, [&](int64_t gp) { return a.x0[gp]; });
    __syncthreads();
    const int x = bx + lx, y = by + ly;
    if (x < g.nx && y < g.ny) {
      const int64_t i = (int64_t)y * g.nx + x;
      float xi[1] = {sx[hp0]}, acc[1] = {0.0f}, ws = 0.0f;
      window_fast<SH, 1, STORED>(g, hp0, i, g.nx, sg, sval, mask,
                                 reinterpret_cast<const Vec<float, 1>*>(sx), a.wf, a.wmode, a.n, xi, acc, ws);
      const float r = -acc[0];
      const float sv = a.dinv ? r * a.dinv[i] : r;
      a.x[i] = xi[0];
      a.r[i] = r;
      a.s[i] = sv;
      v[0] += sv * r;
      v[1] += sv * sv;
      v[2] += r * r;
      v[3] += xi[0] * xi[0];
    }
  }
  double blk[4], tot[4];
  block_sum<4, float>(v, red, blk);
  if (grid_sum_last<4>(blk, a.partials, &a.st->counter, tot, &last)) {
    CgState* st = a.st;
    st->sr = tot[0];
    st->ss = tot[1];
    st->rr = tot[2];
    const double b2 = (double)a.shift * (double)a.shift * tot[3];
    st->ref2 = b2 > 0.0 ? b2 : tot[2];
    st->beta = 0.0;
    st->alpha = 0.0;
    st->iter = 0;
    st->status = (isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2])) ? CG_RUN : CG_NONFINITE;
  }
}

template <class SH, bool STORED>
__global__ void __launch_bounds__(BF_THREADS) k_cg_dir_fast(const Geom<float> g, const CgArgs<float> a) {
  if (a.st->status != CG_RUN) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[1 * (BF_THREADS / 32)];
  __shared__ int last;
  float* sx = reinterpret_cast<float*>(smem);
  float* sg = sx + SH::hp;
  float* sval = sg + SH::hp;
  const float beta = (float)a.st->beta;
  const int ntx = (g.nx + SH::tw - 1) / SH::tw, ntiles = ntx * ((g.ny + SH::th - 1) / SH::th);
  const int lx = threadIdx.x % SH::tw, ly = threadIdx.x / SH::tw;
  const int hp0 = (ly + SH::ry) * SH::hw + (lx + SH::rx);
  float v[1] = {0.0f};
  // persistent over the tiles: one block partial for the whole launch, so the grid
  // reduction sums a few hundred partials instead of one per tile
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int bx = (t % ntx) * SH::tw, by = (t / ntx) * SH::th;
    const bool mask = !(bx - SH::rx >= 0 && bx + SH::tw + SH::rx <= g.nx && by - SH::ry >= 0 &&
                        by + SH::th + SH::ry <= g.ny);
    __syncthreads();                                          // the previous tile is read
    if (a.first)
      stage1_fast<SH>(g, bx, by, sx, sg, sval, a.guide, !STORED, [&](int64_t gp) { return a.s[gp]; });
    else
      stage1_fast<SH>(g, bx, by, sx, sg, sval, a.guide, !STORED,
                      [&](int64_t gp) { return fmaf(beta, a.p_old[gp], a.s[gp]); });
    __syncthreads();
    const int x = bx + lx, y = by + ly;
    if (x < g.nx && y < g.ny) {
      const int64_t i = (int64_t)y * g.nx + x;
      float pi[1] = {sx[hp0]}, acc[1] = {0.0f}, ws = 0.0f;
      window_fast<SH, 1, STORED>(g, hp0, i, g.nx, sg, sval, mask,
                                 reinterpret_cast<const Vec<float, 1>*>(sx), a.wf, a.wmode, a.n, pi, acc, ws);
      const float q = fmaf(a.shift, pi[0], acc[0]);
      a.p_new[i] = pi[0];
      a.q[i] = q;
      v[0] += pi[0] * q;
    }
  }
  double blk[1], tot[1];
  block_sum<1, float>(v, red, blk);
  if (grid_sum_last<1>(blk, a.partials, &a.st->counter, tot, &last)) {
    CgState* st = a.st;
    st->pq = tot[0];
    if (st->sr == 0.0) {
      st->status = CG_CONV;
    } else if (!isfinite(tot[0])) {
      st->status = CG_NONFINITE;
    } else if (!(tot[0] > 0.0)) {
      st->status = CG_BREAK;
    } else {
      st->alpha = st->sr / tot[0];
    }
  }
}

// ---- strip path: FP32 graphs with the 7 x 7 window, T = Jacobi or identity -----------
static_assert(STRIP_THREADS == BF_THREADS, "the block reductions assume BF_THREADS threads");
// The vectors are x, s = T r (r itself is not stored: r = d s for Jacobi, r = s for the
// identity), p (two buffers) and q.  Per iteration:
//   k_cgs_dir:    p = s + beta p_old on the tile and its halo (staged by cp.async, the next
//                 tile's copies in flight), q = (L + sigma I) p by strip window sums, p^T q,
//                 and in the last block alpha;
//   k_cgs_update: x += alpha p, s -= alpha T q, the sums s^T r, s^T q, s^T s, r^T r and
//                 beta (four-pixel vectors).
// Reads and writes per pixel and iteration: 20 B (direction) + 28 B (update).

// r = -L x0, x = x0, s = T r; sums s^T r, s^T s, r^T r, x0^T x0.
template <int WM>
__global__ void __launch_bounds__(STRIP_THREADS, 2) k_cgs_init(const Geom<float> g, const CgArgs<float> a) {
  __shared__ double red[4 * (STRIP_THREADS / 32)];
  __shared__ int last;
  const int nx = g.nx, ny = g.ny;
  float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const float* src[2] = {a.x0, WM == BF_W_ONTHEFLY ? a.guide : nullptr};
  const int64_t ld[2] = {1, 1};
  auto epi = [&](int bx, int by, int lx, int ly0, const float (&xi)[STRIP_P], const float (&acc)[STRIP_P]) {
    const int x = bx + lx;
#pragma unroll
    for (int j = 0; j < STRIP_P; ++j) {
      const int y = by + ly0 + j;
      if (x < nx && y < ny) {
        const int64_t i = (int64_t)y * nx + x;
        const float r = -acc[j];
        const float sj = a.dinv ? __fdiv_rn(r, a.d[i]) : r;
        a.x[i] = xi[j];
        a.s[i] = sj;
        v[0] = fmaf(sj, r, v[0]);
        v[1] = fmaf(sj, sj, v[1]);
        v[2] = fmaf(r, r, v[2]);
        v[3] = fmaf(xi[j], xi[j], v[3]);
      }
    }
  };
  strip_run<WM, 2, false>(g, a.wf, a.n, src, ld, 1, [](float*) {}, epi);
  double blk[4], tot[4];
  block_sum<4, float>(v, red, blk);
  if (grid_sum_last<4>(blk, a.partials, &a.st->counter, tot, &last)) {
    CgState* st = a.st;
    st->sr = tot[0];
    st->ss = tot[1];
    st->rr = tot[2];
    const double b2 = (double)a.shift * (double)a.shift * tot[3];
    st->ref2 = b2 > 0.0 ? b2 : tot[2];
    st->beta = 0.0;
    st->alpha = 0.0;
    st->iter = 0;
    st->status = (isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2])) ? CG_RUN : CG_NONFINITE;
  }
}

// p = s + beta p_old (first: p = s), q = (L + shift I) p, p^T q, alpha.
template <int WM>
__global__ void __launch_bounds__(STRIP_THREADS, 2) k_cgs_dir(const Geom<float> g, const CgArgs<float> a) {
  if (a.st->status != CG_RUN) return;
  __shared__ double red[STRIP_THREADS / 32];
  __shared__ int last;
  const float beta = (float)a.st->beta;
  const int nx = g.nx, ny = g.ny;
  float v[1] = {0.0f};
  const bool first = a.first != 0;
  const float* src[3] = {a.s, first ? nullptr : a.p_old, WM == BF_W_ONTHEFLY ? a.guide : nullptr};
  const int64_t ld[3] = {1, 1, 1};
  auto combine = [&](float* st) {
    if (first) return;
    for (int hp = threadIdx.x; hp < STRIP_HP; hp += STRIP_THREADS) st[hp] = fmaf(beta, st[STRIP_HP + hp], st[hp]);
  };
  auto epi = [&](int bx, int by, int lx, int ly0, const float (&pi)[STRIP_P], const float (&acc)[STRIP_P]) {
    const int x = bx + lx;
#pragma unroll
    for (int j = 0; j < STRIP_P; ++j) {
      const int y = by + ly0 + j;
      if (x < nx && y < ny) {
        const int64_t i = (int64_t)y * nx + x;
        const float q = fmaf(a.shift, pi[j], acc[j]);
        a.p_new[i] = pi[j];
        a.q[i] = q;
        v[0] = fmaf(pi[j], q, v[0]);
      }
    }
  };
  strip_run<WM, 3, true>(g, a.wf, a.n, src, ld, 2, combine, epi);
  double blk[1], tot[1];
  block_sum<1, float>(v, red, blk);
  if (grid_sum_last<1>(blk, a.partials, &a.st->counter, tot, &last)) {
    CgState* st = a.st;
    st->pq = tot[0];
    if (st->sr == 0.0) {
      st->status = CG_CONV;
    } else if (!isfinite(tot[0])) {
      st->status = CG_NONFINITE;
    } else if (!(tot[0] > 0.0)) {
      st->status = CG_BREAK;
    } else {
      st->alpha = st->sr / tot[0];
    }
  }
}

// One pixel of the update: x += alpha p, s -= alpha T q, and the four sums.
__device__ __forceinline__ void cgs_upd1(float alpha, bool jac, float q, float d, float p, float& x, float& s,
                                         float (&v)[4]) {
  x = fmaf(alpha, p, x);
  float r;
  if (jac) {
    s = fmaf(-alpha, __fdiv_rn(q, d), s);
    r = d * s;
  } else {
    s = fmaf(-alpha, q, s);
    r = s;
  }
  v[0] = fmaf(s, r, v[0]);
  v[1] = fmaf(s, q, v[1]);
  v[2] = fmaf(s, s, v[2]);
  v[3] = fmaf(r, r, v[3]);
}

// x += alpha p, s -= alpha T q (T = D^-1: s -= alpha q / d; r = d s), sums, beta.  Four
// pixels per vector access (all arrays 16-byte aligned), the n % 4 tail by the last block.
__global__ void __launch_bounds__(BF_THREADS) k_cgs_update(const CgArgs<float> a) {
  if (a.st->status != CG_RUN) return;
  __shared__ double red[4 * (BF_THREADS / 32)];
  __shared__ int last;
  const float alpha = (float)a.st->alpha;
  const bool jac = a.dinv != nullptr;
  float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const int64_t n4 = a.n >> 2;
  const float4* q4 = reinterpret_cast<const float4*>(a.q);
  const float4* d4 = reinterpret_cast<const float4*>(a.d);
  const float4* p4 = reinterpret_cast<const float4*>(a.p_new);
  float4* x4 = reinterpret_cast<float4*>(a.x);
  float4* s4 = reinterpret_cast<float4*>(a.s);
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < n4; i += (int64_t)gridDim.x * BF_THREADS) {
    const float4 q = q4[i], p = p4[i];
    const float4 d = jac ? d4[i] : make_float4(1.0f, 1.0f, 1.0f, 1.0f);
    float4 x = x4[i], sv = s4[i];
    cgs_upd1(alpha, jac, q.x, d.x, p.x, x.x, sv.x, v);
    cgs_upd1(alpha, jac, q.y, d.y, p.y, x.y, sv.y, v);
    cgs_upd1(alpha, jac, q.z, d.z, p.z, x.z, sv.z, v);
    cgs_upd1(alpha, jac, q.w, d.w, p.w, x.w, sv.w, v);
    x4[i] = x;
    s4[i] = sv;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x < (a.n & 3)) {
    const int64_t i = 4 * n4 + threadIdx.x;
    float x = a.x[i], sv = a.s[i];
    cgs_upd1(alpha, jac, a.q[i], jac ? a.d[i] : 1.0f, a.p_new[i], x, sv, v);
    a.x[i] = x;
    a.s[i] = sv;
  }
  double blk[4], tot[4];
  block_sum<4, float>(v, red, blk);
  if (grid_sum_last<4>(blk, a.partials, &a.st->counter, tot, &last)) cg_step_tail(a, tot);
}

// Launch the init / direction kernels: specialised window when the graph has one.
template <class SH, bool STORED>
static void cg_launch_fast(bool init, dim3 tg, cudaStream_t s, const bf_graph* g, const CgArgs<float>& a) {
  const size_t sm = 3 * SH::hp * sizeof(float);
  const unsigned grid = std::min<unsigned>(tg.x * tg.y, 8u * (unsigned)cg_num_sms());   // persistent, 8 per SM
  if (init) BF_LAUNCH(k_cg_init_fast<SH, STORED><<<grid, BF_THREADS, sm, s>>>(g->gf, a));
  else BF_LAUNCH(k_cg_dir_fast<SH, STORED><<<grid, BF_THREADS, sm, s>>>(g->gf, a));
}

template <class SH>
static void cg_launch_fast_w(bool init, dim3 tg, cudaStream_t s, const bf_graph* g, const CgArgs<float>& a) {
  if (g->p.weight_mode == BF_W_ONTHEFLY) cg_launch_fast<SH, false>(init, tg, s, g, a);
  else cg_launch_fast<SH, true>(init, tg, s, g, a);
}

template <typename T>
static void cg_launch_window(bool init, dim3 tg, size_t sm, cudaStream_t s, const bf_graph* g,
                             const CgArgs<T>& a) {
  if (sizeof(T) == 4) {
    const CgArgs<float>& af = reinterpret_cast<const CgArgs<float>&>(a);
    switch (fast_shape(g)) {
      case FAST_R3_2D: cg_launch_fast_w<ShapeR3>(init, tg, s, g, af); return;
      case FAST_R5_1D: cg_launch_fast_w<ShapeR5>(init, tg, s, g, af); return;
      case FAST_CROSS1: cg_launch_fast_w<ShapeX1>(init, tg, s, g, af); return;
    }
  }
  if (init) BF_LAUNCH(k_cg_init<T><<<tg, BF_THREADS, sm, s>>>(geom_of<T>(g), a));
  else BF_LAUNCH(k_cg_dir<T><<<tg, BF_THREADS, sm, s>>>(geom_of<T>(g), a));
}

// The kernels of the generic path (any window, FP32/FP64, guided graphs, the net T).
template <typename T>
int cg_generic_loop(const bf_graph* g, CgArgs<T>& a, int kmax, const bf_cg_opts& o, cudaStream_t s,
                    T* const* pbuf, dim3 tg, size_t sm, unsigned nb_elem) {
  const bool net = (o.precond == BF_PRECOND_NET || o.precond == BF_PRECOND_SPD);
  const bool guided = (g->kind == BF_KIND_GUIDED);
  int rc = BF_OK;
  if (guided) {
    if ((rc = bf_guided_apply<T>(g, BF_OP_L, a.x0, 1, 1, a.q, 1, nullptr, nullptr, s))) return rc;
    BF_LAUNCH(k_cg_init_lx<T><<<nb_elem, BF_THREADS, 0, s>>>(a));
  } else {
    cg_launch_window<T>(true, tg, sm, s, g, a);
  }
  BF_CUDA(cudaGetLastError());
  if (net) {
    if ((rc = own_precond(o, g, a.r, a.s, s, &a.st->status))) return rc;
    BF_LAUNCH(k_cg_sdots<T><<<nb_elem, BF_THREADS, 0, s>>>(a, 1));
  }
  for (int it = 0; it < kmax; ++it) {
    a.first = (it == 0);
    a.p_old = pbuf[it & 1];
    a.p_new = pbuf[(it + 1) & 1];
    if (guided) {
      BF_LAUNCH(k_cg_pdir<T><<<nb_elem, BF_THREADS, 0, s>>>(a));
      if ((rc = bf_guided_apply<T>(g, BF_OP_L, a.p_new, 1, 1, a.q, 1, nullptr, nullptr, s))) return rc;
      BF_LAUNCH(k_cg_pq<T><<<nb_elem, BF_THREADS, 0, s>>>(a));
    } else {
      cg_launch_window<T>(false, tg, sm, s, g, a);
    }
    if (net) {
      BF_LAUNCH(k_cg_xr<T><<<nb_elem, BF_THREADS, 0, s>>>(a));
      if ((rc = own_precond(o, g, a.r, a.s, s, &a.st->status))) return rc;
      BF_LAUNCH(k_cg_sdots<T><<<nb_elem, BF_THREADS, 0, s>>>(a, 0));
    } else {
      BF_LAUNCH(k_cg_update<T><<<nb_elem, BF_THREADS, 0, s>>>(a));
    }
    // with a tolerance, look at the status every CG_POLL iterations so that a converged
    // run stops enqueueing (a fixed-count run never reads back and can be captured)
    if (o.tol > 0.0 && (it + 1) % CG_POLL == 0 && it + 1 < kmax) {
      int stv = 0;
      BF_CUDA(cudaMemcpyAsync(&stv, &a.st->status, sizeof(int), cudaMemcpyDeviceToHost, s));
      BF_CUDA(cudaStreamSynchronize(s));
      if (stv != CG_RUN) break;
    }
  }
  return BF_OK;
}

template <int WM>
int strip_grid(const bf_graph* g, const void* fn) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, STRIP_THREADS, STRIP_SMEM_BYTES) != cudaSuccess || v < 1)
      v = 1;
    per_sm = v;
  }
  const int64_t ntiles = (int64_t)strip_tiles_x(g->nx) * strip_tiles_y(g->ny);
  return (int)std::min<int64_t>(ntiles, (int64_t)per_sm * cg_num_sms());
}

template <int WM>
int cg_strip_loop_w(const bf_graph* g, CgArgs<float>& a, int kmax, double tol, cudaStream_t s,
                    float* const* pbuf) {
  const unsigned nb_vec =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.n / 4 + BF_THREADS - 1) / BF_THREADS, 8 * cg_num_sms()));
  a.d = (const float*)g->d;
  const int gi = strip_grid<WM>(g, (const void*)k_cgs_init<WM>);
  const int gd = strip_grid<WM>(g, (const void*)k_cgs_dir<WM>);
  BF_LAUNCH(k_cgs_init<WM><<<gi, STRIP_THREADS, STRIP_SMEM_BYTES, s>>>(g->gf, a));
  for (int it = 0; it < kmax; ++it) {
    a.first = (it == 0);
    a.p_old = pbuf[it & 1];
    a.p_new = pbuf[(it + 1) & 1];
    BF_LAUNCH(k_cgs_dir<WM><<<gd, STRIP_THREADS, STRIP_SMEM_BYTES, s>>>(g->gf, a));
    BF_LAUNCH(k_cgs_update<<<nb_vec, BF_THREADS, 0, s>>>(a));
    if (tol > 0.0 && (it + 1) % CG_POLL == 0 && it + 1 < kmax) {
      int stv = 0;
      BF_CUDA(cudaMemcpyAsync(&stv, &a.st->status, sizeof(int), cudaMemcpyDeviceToHost, s));
      BF_CUDA(cudaStreamSynchronize(s));
      if (stv != CG_RUN) break;
    }
  }
  return BF_OK;
}

int cg_strip_loop(const bf_graph* g, CgArgs<float>& a, int kmax, double tol, cudaStream_t s,
                  float* const* pbuf) {
  switch (g->p.weight_mode) {
    case BF_W_STORED_F32: return cg_strip_loop_w<BF_W_STORED_F32>(g, a, kmax, tol, s, pbuf);
    case BF_W_STORED_BF16: return cg_strip_loop_w<BF_W_STORED_BF16>(g, a, kmax, tol, s, pbuf);
  }
  return cg_strip_loop_w<BF_W_ONTHEFLY>(g, a, kmax, tol, s, pbuf);
}

// Device buffers of one CG run: residual r, preconditioned residual s, q = A p, the two
// direction buffers, the block partial sums of the grid reductions and the scalar state.
template <typename T>
struct CgBufs {
  T* r;
  T* s;
  T* q;
  T* p[2];
  double* partials;
  CgState* st;
};

// Algorithm 2 on the buffers `b` (cg_filter: the graph's workspace; cg_filter_noalloc: the
// library's static array).  `who` names the entry point in error messages.
template <typename T>
int cg_exec(const bf_graph* g, const T* x0, int kmax, const bf_cg_opts& o, T* x_out,
            bf_info* info, cudaStream_t s, const CgBufs<T>& b, const char* who) {
  const int64_t n = g->n;
  const dim3 tg = tile_grid(g);
  const unsigned nb_elem = (unsigned)std::min<int64_t>((n + BF_THREADS - 1) / BF_THREADS, 8 * cg_num_sms());
  CgArgs<T> a;
  a.r = b.r;
  a.s = b.s;
  a.q = b.q;
  a.partials = b.partials;
  a.st = b.st;
  a.x0 = x0;
  a.x = x_out;
  a.guide = (const T*)g->guide;
  a.dinv = o.precond == BF_PRECOND_JACOBI ? (const T*)g->dinv : nullptr;
  a.d = (const T*)g->d;
  a.wf = g->wf;
  a.wmode = g->p.weight_mode;
  a.n = n;
  a.shift = (T)o.shift;
  a.hist = o.hist;
  a.first = 1;
  a.p_old = b.p[0];
  a.p_new = b.p[1];
  BF_LAUNCH(k_cg_state_init<<<1, 32, 0, s>>>(a.st, o.tol > 0 ? o.tol * o.tol : 0.0, o.beta));
  const bool one_d = (g->ny == 1 && g->ry == 0);
  const size_t hp = (size_t)((one_d ? BF_TW1 : BF_TW2) + 2 * g->rx) * ((one_d ? 1 : BF_TH2) + 2 * g->ry);
  const size_t sm = hp * 2 * sizeof(T);
  const bool net = (o.precond == BF_PRECOND_NET || o.precond == BF_PRECOND_SPD);
  const bool guided = (g->kind == BF_KIND_GUIDED);
  int rc = BF_OK;
  if (!guided && !net && sizeof(T) == 4 && fast_shape(g) == FAST_R3_2D && ((uintptr_t)x_out & 15) == 0) {
    rc = cg_strip_loop(g, reinterpret_cast<CgArgs<float>&>(a), kmax, o.tol, s,
                       reinterpret_cast<float* const*>(b.p));
    if (rc) return rc;
  } else {
    rc = cg_generic_loop<T>(g, a, kmax, o, s, b.p, tg, sm, nb_elem);
    if (rc) return rc;
  }
  BF_CUDA(cudaGetLastError());
  if (info) {
    CgState h;
    BF_CUDA(cudaMemcpyAsync(&h, a.st, sizeof(h), cudaMemcpyDeviceToHost, s));
    BF_CUDA(cudaStreamSynchronize(s));
    info->iters = h.iter;
    info->status = h.status == CG_CONV ? BF_CG_CONVERGED : (h.status == CG_BREAK ? BF_CG_BREAKDOWN : 0);
    info->restarts = 0;
    info->reserved = 0;
    info->rnorm = sqrt(h.rr);
    info->ref = sqrt(h.ref2);
    if (h.status == CG_BREAK) return bf_fail(BF_EBREAKDOWN, std::string(who) + ": p^T q <= 0 (breakdown)");
    if (h.status == CG_NONFINITE) return bf_fail(BF_ENONFINITE, std::string(who) + ": non-finite scalar");
  }
  return BF_OK;
}

// Partial-sum slots a run needs: one per block of the widest launch.
inline unsigned cg_partial_slots(const bf_graph* g) {
  const dim3 tg = tile_grid(g);
  const unsigned nb_tile = tg.x * tg.y;
  const unsigned nb_elem = (unsigned)std::min<int64_t>((g->n + BF_THREADS - 1) / BF_THREADS, 8 * cg_num_sms());
  return std::max(nb_tile, nb_elem);
}

template <typename T>
int cg_run(const bf_graph* g, const T* x0, int kmax, const bf_cg_opts& o, T* x_out,
           bf_info* info, cudaStream_t s) {
  bf_graph* gm = const_cast<bf_graph*>(g);
  const size_t vb = ((size_t)g->n * sizeof(T) + 255) & ~(size_t)255;
  const size_t pb = ((size_t)cg_partial_slots(g) * 4 * sizeof(double) + 255) & ~(size_t)255;
  int rc = bf_ws_reserve(gm, BF_WS_CG, 5 * vb + pb + 256);
  if (rc) return rc;
  char* w = (char*)gm->ws[BF_WS_CG];
  CgBufs<T> b;
  b.r = (T*)(w);
  b.s = (T*)(w + vb);
  b.q = (T*)(w + 2 * vb);
  b.p[0] = (T*)(w + 3 * vb);
  b.p[1] = (T*)(w + 4 * vb);
  b.partials = (double*)(w + 5 * vb);
  b.st = (CgState*)(w + 5 * vb + pb);
  return cg_exec<T>(g, x0, kmax, o, x_out, info, s, b, "cg_filter");
}

}  // namespace

extern "C" int cg_filter(const bf_graph* g, const void* x0, int kmax, const bf_cg_opts* opts,
                         void* x_out, bf_info* info, void* stream) {
  if (!g || !x0 || !x_out) return bf_fail(BF_EINVAL, "cg_filter: NULL argument");
  if (kmax < 0) return bf_fail(BF_EINVAL, "cg_filter: kmax < 0");
  bf_cg_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.precond != BF_PRECOND_JACOBI && o.precond != BF_PRECOND_IDENTITY && o.precond != BF_PRECOND_NET &&
      o.precond != BF_PRECOND_SPD)
    return bf_fail(BF_EINVAL, "cg_filter: bad precond");
  if (o.precond == BF_PRECOND_NET && (!o.net || g->esize != 4 || g->kind != BF_KIND_BILATERAL))
    return bf_fail(BF_EINVAL, "cg_filter: BF_PRECOND_NET needs a net and an FP32 bilateral graph");
  if (o.precond == BF_PRECOND_SPD && (!o.spd || g->esize != 4 || g->kind != BF_KIND_BILATERAL))
    return bf_fail(BF_EINVAL, "cg_filter: BF_PRECOND_SPD needs a bf_spd and an FP32 bilateral graph");
  if (o.beta != BF_BETA_FLEXIBLE && o.beta != BF_BETA_PRINTED)
    return bf_fail(BF_EINVAL, "cg_filter: bad beta");
  if (!(o.shift >= 0.0) || !(o.tol >= 0.0)) return bf_fail(BF_EINVAL, "cg_filter: shift and tol must be >= 0");
  if ((uintptr_t)x0 % g->esize || (uintptr_t)x_out % g->esize)
    return bf_fail(BF_EINVAL, "cg_filter: misaligned vector");
  cudaStream_t s = (cudaStream_t)stream;
  if (g->esize == 4) return cg_run<float>(g, (const float*)x0, kmax, o, (float*)x_out, info, s);
  return cg_run<double>(g, (const double*)x0, kmax, o, (double*)x_out, info, s);
}

// ==================================================================== refinement
// (L + sigma I) x = sigma x0 to a TRUE relative residual: each outer step forms the
// residual r = sigma (x0 - x) - L x in FP64 on the FP64 graph, and solves the correction
// (L + sigma I) e = r by the FP32 CG filter on the FP32 graph to an inner tolerance; the
// FP32 recurrence alone stalls near eps_32 times the condition number.
namespace {

// r = sigma (x0 - x) - q (q = L x), rhs = r / sigma in FP32; sums r^T r and x0^T x0.
__global__ void __launch_bounds__(BF_THREADS) k_ref_resid(const double* x0, const double* x, const double* q,
                                                          double sigma, int64_t n, float* rhs, double* partials,
                                                          unsigned* counter, double* out) {
  __shared__ double red[2 * (BF_THREADS / 32)];
  __shared__ int last;
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * BF_THREADS) {
    const double r = sigma * (x0[i] - x[i]) - q[i];
    rhs[i] = (float)(r / sigma);
    v[0] = fma(r, r, v[0]);
    v[1] = fma(x0[i], x0[i], v[1]);
  }
  double blk[2], tot[2];
  block_sum<2, double>(v, red, blk);
  if (grid_sum_last<2>(blk, partials, counter, tot, &last)) {
    out[0] = tot[0];
    out[1] = tot[1];
  }
}

// x += e (the FP32 correction) and x = x0.
__global__ void __launch_bounds__(BF_THREADS) k_ref_add(double* x, const float* e, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * BF_THREADS)
    x[i] += (double)e[i];
}

}  // namespace

extern "C" int cg_refine(const bf_graph* g64, const bf_graph* g32, const double* x0, double shift, double tol,
                         const bf_cg_opts* inner, int inner_kmax, int outer_max, double* x_out, bf_info* info,
                         void* stream) {
  if (!g64 || !g32 || !x0 || !x_out) return bf_fail(BF_EINVAL, "cg_refine: NULL argument");
  if (g64->esize != 8 || g32->esize != 4 || g64->n != g32->n || g64->nx != g32->nx || g64->ny != g32->ny)
    return bf_fail(BF_EINVAL, "cg_refine: needs an FP64 and an FP32 graph of the same shape");
  if (!(shift > 0.0) || !(tol > 0.0) || inner_kmax < 1 || outer_max < 0)
    return bf_fail(BF_EINVAL, "cg_refine: need shift > 0, tol > 0, inner_kmax >= 1, outer_max >= 0");
  if ((uintptr_t)x0 % 8 || (uintptr_t)x_out % 8) return bf_fail(BF_EINVAL, "cg_refine: misaligned vector");
  bf_cg_opts o;
  memset(&o, 0, sizeof(o));
  if (inner) o = *inner;
  if (!(o.tol > 0.0)) o.tol = 1e-3;
  o.shift = shift;
  o.hist = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g64->n;
  // the refinement's vectors live in the FP64 graph's CG workspace (the inner CG uses the
  // FP32 graph's): q (FP64), rhs and e (FP32), partial sums, counter and the two sums
  bf_graph* gm = const_cast<bf_graph*>(g64);
  const size_t vd = ((size_t)n * 8 + 255) & ~(size_t)255, vf = ((size_t)n * 4 + 255) & ~(size_t)255;
  const unsigned nb = (unsigned)std::min<int64_t>((n + BF_THREADS - 1) / BF_THREADS, 8 * cg_num_sms());
  const size_t pb = (((size_t)nb * 2 * sizeof(double)) + 255) & ~(size_t)255;
  int rc = bf_ws_reserve(gm, BF_WS_CG, vd + 2 * vf + pb + 256);
  if (rc) return rc;
  char* w = (char*)gm->ws[BF_WS_CG];
  double* q = (double*)w;
  float* rhs = (float*)(w + vd);
  float* e = (float*)(w + vd + vf);
  double* partials = (double*)(w + vd + 2 * vf);
  unsigned* counter = (unsigned*)(w + vd + 2 * vf + pb);
  double* sums = (double*)(w + vd + 2 * vf + pb + 16);
  BF_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
  if (x_out != x0) BF_CUDA(cudaMemcpyAsync(x_out, x0, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
  int inner_total = 0, outer = 0;
  double rel = 0.0, rr = 0.0, bb = 0.0;
  for (;; ++outer) {
    if ((rc = bf_apply_f64(g64, BF_OP_L, x_out, 1, 1, q, 1, nullptr, s))) return rc;
    BF_LAUNCH(k_ref_resid<<<nb, BF_THREADS, 0, s>>>(x0, x_out, q, shift, n, rhs, partials, counter, sums));
    BF_CUDA(cudaGetLastError());
    double h[2];
    BF_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s));
    BF_CUDA(cudaStreamSynchronize(s));
    rr = h[0];
    bb = shift * shift * h[1];
    if (!std::isfinite(rr)) return bf_fail(BF_ENONFINITE, "cg_refine: non-finite residual");
    rel = bb > 0.0 ? std::sqrt(rr / bb) : std::sqrt(rr);
    if (rel <= tol || outer == outer_max) break;
    bf_info ii;
    if ((rc = cg_filter(g32, rhs, inner_kmax, &o, e, &ii, stream))) return rc;
    inner_total += ii.iters;
    BF_LAUNCH(k_ref_add<<<nb, BF_THREADS, 0, s>>>(x_out, e, n));
  }
  if (info) {
    info->iters = inner_total;
    info->status = rel <= tol ? BF_CG_CONVERGED : 0;
    info->restarts = outer;
    info->reserved = 0;
    info->rnorm = std::sqrt(rr);
    info->ref = std::sqrt(bb);
  }
  return BF_OK;
}

// r = shift (x0 - x) - L x: the residual of (L + shift I) x = shift x0 (the training pairs
// of the learned preconditioner are built from it).
namespace {
template <typename T>
__global__ void __launch_bounds__(BF_THREADS) k_shifted_resid(const T* x0, const T* x, T shift, int64_t n, T* r) {
  for (int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * BF_THREADS)
    r[i] = fma(shift, x0[i] - x[i], -r[i]);
}
}  // namespace

extern "C" int bf_shifted_residual(const bf_graph* g, const void* x0, const void* x, double shift, void* r_out,
                                   void* stream) {
  if (!g || !x0 || !x || !r_out) return bf_fail(BF_EINVAL, "bf_shifted_residual: NULL argument");
  if (!(shift >= 0.0)) return bf_fail(BF_EINVAL, "bf_shifted_residual: shift must be >= 0");
  if ((uintptr_t)x0 % g->esize || (uintptr_t)x % g->esize || (uintptr_t)r_out % g->esize)
    return bf_fail(BF_EINVAL, "bf_shifted_residual: misaligned vector");
  if (r_out == x || r_out == x0) return bf_fail(BF_EINVAL, "bf_shifted_residual: r_out must not alias x0 or x");
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned nb = (unsigned)std::min<int64_t>((g->n + BF_THREADS - 1) / BF_THREADS, 8 * cg_num_sms());
  int rc;
  if (g->esize == 4) {
    if ((rc = bf_apply_f32(g, BF_OP_L, (const float*)x, 1, 1, (float*)r_out, 1, nullptr, s))) return rc;
    BF_LAUNCH(k_shifted_resid<float><<<nb, BF_THREADS, 0, s>>>((const float*)x0, (const float*)x, (float)shift,
                                                               g->n, (float*)r_out));
  } else {
    if ((rc = bf_apply_f64(g, BF_OP_L, (const double*)x, 1, 1, (double*)r_out, 1, nullptr, s))) return rc;
    BF_LAUNCH(k_shifted_resid<double><<<nb, BF_THREADS, 0, s>>>((const double*)x0, (const double*)x, shift, g->n,
                                                                (double*)r_out));
  }
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

// ==================================================================== allocation-free CG
// cg_filter keeps its vectors in the graph's workspace, which grows with cudaMalloc (and
// cudaFree, which synchronises the whole device) the first time a larger problem comes
// along.  Some callers cannot allow that: code that must not allocate device memory at
// all once it is running (a fixed memory budget owned by another allocator, a loop that
// cannot afford the implicit device synchronisation).  cg_filter_noalloc runs the same
// body (cg_exec: the same kernels, launches and early-stop polling) with its scratch in
// the file-scope array below instead: five n-vectors, the per-block partial sums and the
// scalar state.  The array is a fixed part of the library
// image, so every GPU that loads the library holds it until the process exits.
#define BF_NOALLOC_MAX_N (1 << 18)              // samples (a 512 x 512 image)
#define BF_NOALLOC_MAX_BLOCKS (1 << 16)         // operator tiles (partial-sum slots)
#define BF_NOALLOC_VEC_BYTES ((size_t)BF_NOALLOC_MAX_N * sizeof(double))
#define BF_NOALLOC_BYTES (5 * BF_NOALLOC_VEC_BYTES + (size_t)BF_NOALLOC_MAX_BLOCKS * 4 * sizeof(double) + 256)

static __device__ __align__(256) unsigned char g_cg_noalloc_scratch[BF_NOALLOC_BYTES];

namespace {

// Device address of the scratch array on the current device, looked up once per device.
// (In host code the array's name is only a host-side stand-in for the symbol.)
int noalloc_scratch(unsigned char** out) {
  static std::mutex mu;
  static unsigned char* addr[256] = {nullptr};
  int dev = 0;
  BF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return bf_fail(BF_EINVAL, "cg_filter_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_cg_noalloc_scratch);
    if (e != cudaSuccess) return bf_cuda_fail(e, "cudaGetSymbolAddress(g_cg_noalloc_scratch)");
    addr[dev] = (unsigned char*)p;
  }
  *out = addr[dev];
  return BF_OK;
}

template <typename T>
int cg_run_noalloc(const bf_graph* g, const T* x0, int kmax, const bf_cg_opts& o, T* x_out,
                   bf_info* info, cudaStream_t s) {
  if (g->n > BF_NOALLOC_MAX_N)
    return bf_fail(BF_EINVAL, "cg_filter_noalloc: n exceeds the static scratch limit of 262144 samples");
  if (cg_partial_slots(g) > BF_NOALLOC_MAX_BLOCKS)
    return bf_fail(BF_EINVAL, "cg_filter_noalloc: image shape needs more than 65536 operator tiles");
  unsigned char* w = nullptr;
  int rc = noalloc_scratch(&w);
  if (rc) return rc;
  // The array keeps whatever the previous call left: cg_exec rewrites the scalar state
  // (including the block counter of the grid reductions, which must start at 0) with a
  // kernel before anything reads it, and every vector is written before it is read.
  CgBufs<T> b;
  b.r = (T*)(w);
  b.s = (T*)(w + BF_NOALLOC_VEC_BYTES);
  b.q = (T*)(w + 2 * BF_NOALLOC_VEC_BYTES);
  b.p[0] = (T*)(w + 3 * BF_NOALLOC_VEC_BYTES);
  b.p[1] = (T*)(w + 4 * BF_NOALLOC_VEC_BYTES);
  b.partials = (double*)(w + 5 * BF_NOALLOC_VEC_BYTES);
  b.st = (CgState*)(w + 5 * BF_NOALLOC_VEC_BYTES + (size_t)BF_NOALLOC_MAX_BLOCKS * 4 * sizeof(double));
  return cg_exec<T>(g, x0, kmax, o, x_out, info, s, b, "cg_filter_noalloc");
}

}  // namespace

extern "C" int cg_filter_noalloc(const bf_graph* g, const void* x0, int kmax,
                                 const bf_cg_opts* opts, void* x_out, bf_info* info,
                                 void* stream) {
  if (!g || !x0 || !x_out) return bf_fail(BF_EINVAL, "cg_filter_noalloc: NULL argument");
  if (kmax < 0) return bf_fail(BF_EINVAL, "cg_filter_noalloc: kmax < 0");
  if (g->kind != BF_KIND_BILATERAL) return bf_fail(BF_EINVAL, "cg_filter_noalloc: takes bilateral graphs");
  bf_cg_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.precond != BF_PRECOND_JACOBI && o.precond != BF_PRECOND_IDENTITY)
    return bf_fail(BF_EINVAL, "cg_filter_noalloc: bad precond");
  if (o.beta != BF_BETA_FLEXIBLE && o.beta != BF_BETA_PRINTED)
    return bf_fail(BF_EINVAL, "cg_filter_noalloc: bad beta");
  if (!(o.shift >= 0.0) || !(o.tol >= 0.0))
    return bf_fail(BF_EINVAL, "cg_filter_noalloc: shift and tol must be >= 0");
  if ((uintptr_t)x0 % g->esize || (uintptr_t)x_out % g->esize)
    return bf_fail(BF_EINVAL, "cg_filter_noalloc: misaligned vector");
  cudaStream_t s = (cudaStream_t)stream;
  if (g->esize == 4) return cg_run_noalloc<float>(g, (const float*)x0, kmax, o, (float*)x_out, info, s);
  return cg_run_noalloc<double>(g, (const double*)x0, kmax, o, (double*)x_out, info, s);
}
