// The bilateral-filter graph (Section 2, Eqs. 1-4; Section 4): building it (bf_weights),
// exporting it, and the matrix-free operator Y = op X (bf_apply), plus the simple
// iteration x <- D^-1 W x (bf_simple_filter).
#include <math.h>
#include <stdio.h>

#include <cmath>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <map>
#include <set>
#include <vector>

#include "bf_internal.cuh"
#include "bf_window_fast.cuh"
#include "bf_strip.cuh"
#include "bf_hrun.cuh"

// ================================================================== errors
static thread_local std::string g_last_error;

void bf_set_error(const std::string& msg) { g_last_error = msg; }
int bf_fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int bf_cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? BF_ENOMEM : BF_ECUDA;
}

extern "C" const char* bf_last_error(void) { return g_last_error.c_str(); }

static std::atomic<unsigned long long> g_launches{0};
void bf_count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
extern "C" uint64_t bf_launch_count(void) { return (uint64_t)g_launches.load(); }

int bf_smem_attr(const void* fn, int bytes, const char* what) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> done;   // largest size set so far
  int dev = 0;
  BF_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find({dev, fn});
  if (it != done.end() && it->second >= bytes) return BF_OK;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return bf_cuda_fail(e, what);
  done[{dev, fn}] = bytes;
  return BF_OK;
}

int bf_ws_reserve(bf_graph* g, int slot, size_t bytes) {
  if (bytes <= g->ws_bytes[slot]) return BF_OK;
  if (g->ws[slot]) {
    BF_CUDA(cudaDeviceSynchronize());
    BF_CUDA(cudaFree(g->ws[slot]));
    g->ws[slot] = nullptr;
    g->ws_bytes[slot] = 0;
  }
  bytes = (bytes + 4095) & ~(size_t)4095;
  BF_CUDA(cudaMalloc(&g->ws[slot], bytes));
  g->ws_bytes[slot] = bytes;
  return BF_OK;
}

// ================================================================== weights kernel
// One thread per pixel: sum_{j != i} w_ij over the window (same tap order and the same
// arithmetic as the operator kernels, so d is consistent with every apply), the derived
// per-pixel scalings, and in the stored modes the forward half-window weights rounded to
// the storage type (sums use the rounded values: the stored operator is a graph in its own
// right).
template <typename T>
__global__ void __launch_bounds__(BF_THREADS)
k_weights(const Geom<T> g, const T* __restrict__ guide, int64_t n, T* d, T* dinv, T* dis,
          T* dls, void* wf, int wmode, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x;
  if (i >= n) return;
  const int x = (int)(i % g.nx), y = (int)(i / g.nx);
  const T gi = guide[i];
  if (!isfinite((double)gi)) atomicOr(flag, 1);
  const int bw = 2 * g.rx + 1;
  T wsum = T(0);
  for (int dy = -g.ry; dy <= g.ry; ++dy) {
    const int yy = y + dy;
    for (int dx = -g.rx; dx <= g.rx; ++dx) {
      if (dx == 0 && dy == 0) continue;
      if (g.cross && dx != 0 && dy != 0) continue;
      const int cell = (dy + g.ry) * bw + (dx + g.rx);
      const int f = g.fmap[cell];
      const int xx = x + dx;
      const bool in = (yy >= 0 && yy < g.ny && xx >= 0 && xx < g.nx);
      T w = T(0);
      if (in) {
        const T dl = gi - guide[(int64_t)yy * g.nx + xx];
        w = bf_exp_w(fma(-dl * g.a_r, dl, g.ls[cell]));
        if (wmode == BF_W_STORED_BF16) w = (T)__bfloat162float(__float2bfloat16_rn((float)w));
        else if (wmode == BF_W_STORED_F32) w = (T)(float)w;
        wsum += w;
      }
      if (wmode != BF_W_ONTHEFLY && f >= 0) {
        if (wmode == BF_W_STORED_BF16)
          ((__nv_bfloat16*)wf)[(int64_t)f * n + i] = __float2bfloat16_rn((float)w);
        else
          ((float*)wf)[(int64_t)f * n + i] = (float)w;
      }
    }
  }
  const T dd = T(1) + wsum;
  d[i] = dd;
  dinv[i] = T(1) / dd;
  dis[i] = T(1) / sqrt(dd);
  dls[i] = (wsum > T(1e-30)) ? T(1) / sqrt(wsum) : T(0);
}

// Export every window weight in canonical tap order (centre = 1, 0 off the image).
template <typename T>
__global__ void __launch_bounds__(BF_THREADS)
k_export(const Geom<T> g, const T* __restrict__ guide, int64_t n, const void* wf, int wmode,
         int ntaps, T* out) {
  const int64_t i = (int64_t)blockIdx.x * BF_THREADS + threadIdx.x;
  if (i >= n) return;
  const int x = (int)(i % g.nx), y = (int)(i / g.nx);
  const int bw = 2 * g.rx + 1;
  int t = 0;
  for (int dy = -g.ry; dy <= g.ry; ++dy) {
    for (int dx = -g.rx; dx <= g.rx; ++dx) {
      if (g.cross && dx != 0 && dy != 0) continue;
      const int yy = y + dy, xx = x + dx;
      T w = T(0);
      if (dx == 0 && dy == 0) {
        w = T(1);
      } else if (yy >= 0 && yy < g.ny && xx >= 0 && xx < g.nx) {
        const int cell = (dy + g.ry) * bw + (dx + g.rx);
        const int64_t j = (int64_t)yy * g.nx + xx;
        if (wmode == BF_W_ONTHEFLY) {
          const T dl = guide[i] - guide[j];
          w = bf_exp_w(fma(-dl * g.a_r, dl, g.ls[cell]));
        } else {
          const int f = g.fmap[cell];
          if (f >= 0) w = (T)ld_weight(wf, (int64_t)f * n + i, wmode);
          else w = (T)ld_weight(wf, (int64_t)g.fmap[(g.ry - dy) * bw + (g.rx - dx)] * n + j, wmode);
        }
      }
      out[i * ntaps + t] = w;
      ++t;
    }
  }
}

// ================================================================== operator kernel
template <typename T>
struct ApplyArgs {
  const T* X;
  int64_t ldx;
  T* Y;
  int64_t ldy;
  const T* guide;
  const T* scale;   // per-pixel scaling of the operand (NSYM: d^-1/2, NDIAGL: (diag L)^-1/2)
  const void* wf;
  int wmode;
  int op;
  int64_t n;
  double* dots;     // [K] or NULL
};

template <typename T, int K>
__global__ void __launch_bounds__(BF_THREADS) k_apply(const Geom<T> g, const ApplyArgs<T> a) {
  constexpr int V = VecW<T, K>::value;
  constexpr int NC = K / V;
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile t = make_tile(g);
  Vec<T, V>* sx = reinterpret_cast<Vec<T, V>*>(smem);
  T* sg = reinterpret_cast<T*>(sx + (size_t)NC * t.hp);
  const bool otf = (a.wmode == BF_W_ONTHEFLY);
  // ---- stage the halo tile: operand (optionally scaled) and guide
  for (int idx = threadIdx.x; idx < t.hp * NC; idx += BF_THREADS) {
    const int hp = idx / NC, c = idx - hp * NC;
    const int hy = hp / t.hw, hx = hp - hy * t.hw;
    const int gy = t.by - g.ry + hy, gx = t.bx - g.rx + hx;
    Vec<T, V> v;
    if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) {
      const int64_t gp = (int64_t)gy * g.nx + gx;
      v = *reinterpret_cast<const Vec<T, V>*>(a.X + gp * a.ldx + c * V);
      if (a.scale) {
        const T s = a.scale[gp];
#pragma unroll
        for (int e = 0; e < V; ++e) v.v[e] *= s;
      }
      if (otf && c == 0) sg[hp] = a.guide[gp];
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) v.v[e] = T(0);
      if (otf && c == 0) sg[hp] = T(0);
    }
    sx[c * t.hp + hp] = v;
  }
  __syncthreads();
  // ---- window sum and epilogue
  const bool diff = (a.op == BF_OP_L || a.op == BF_OP_NSYM || a.op == BF_OP_NDIAGL);
  T xi[K], acc[K], y[K];
  T wsum = T(0);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const Vec<T, V> v = sx[c * t.hp + t.hp0];
#pragma unroll
    for (int e = 0; e < V; ++e) xi[c * V + e] = v.v[e];
  }
#pragma unroll
  for (int c = 0; c < K; ++c) { acc[c] = T(0); y[c] = T(0); }
  const int64_t i = (int64_t)t.y * g.nx + t.x;
  if (t.active) {
    if (diff) window_sum<T, K, true>(g, t, sg, sx, a.wf, a.wmode, a.n, xi, acc, wsum);
    else      window_sum<T, K, false>(g, t, sg, sx, a.wf, a.wmode, a.n, xi, acc, wsum);
    T s_i = T(1);
    if (a.scale) s_i = a.scale[i];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      switch (a.op) {
        case BF_OP_W:      y[c] = acc[c] + xi[c]; break;
        case BF_OP_L:      y[c] = acc[c]; break;
        case BF_OP_DINV_W: y[c] = (acc[c] + xi[c]) / (T(1) + wsum); break;
        case BF_OP_D:      y[c] = (T(1) + wsum) * xi[c]; break;
        default:           y[c] = s_i * acc[c]; break;   // NSYM, NDIAGL
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      Vec<T, V> o;
#pragma unroll
      for (int e = 0; e < V; ++e) o.v[e] = y[c * V + e];
      *reinterpret_cast<Vec<T, V>*>(a.Y + i * a.ldy + c * V) = o;
    }
  }
  if (a.dots) {
    // dots use the unscaled operand
    if (a.scale && t.active) {
#pragma unroll
      for (int c = 0; c < K; ++c) xi[c] = a.X[i * a.ldx + c];
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const T pr = t.active ? xi[c] * y[c] : T(0);
      const T s = warp_sum(pr);
      if ((threadIdx.x & 31) == 0) atomicAdd(&a.dots[c], (double)s);
    }
  }
}

// Laplacian-type operators (L, NSYM, NDIAGL) and the BF step D^-1 W of float graphs with a
// specialised window; the step in difference form, y_i = x_i - sum_j w_ij (x_i - x_j) / d_i
// with d_i = 1 + sum_{j != i} w_ij (Eqs. 1, 3).
template <class SH, int K, bool STORED>
__global__ void __launch_bounds__(BF_THREADS) k_apply_fast(const Geom<float> g, const ApplyArgs<float> a) {
  constexpr int V = VecW<float, K>::value;
  constexpr int NC = K / V;
  extern __shared__ __align__(16) unsigned char smem[];
  Vec<float, V>* sx = reinterpret_cast<Vec<float, V>*>(smem);
  float* sg = reinterpret_cast<float*>(sx + (size_t)NC * SH::hp);
  float* sval = sg + SH::hp;
  const int bx = blockIdx.x * SH::tw, by = blockIdx.y * SH::th;
  const bool mask = !(bx - SH::rx >= 0 && bx + SH::tw + SH::rx <= g.nx && by - SH::ry >= 0 &&
                      by + SH::th + SH::ry <= g.ny);
  stage_fast<SH, K>(g, bx, by, a.X, a.ldx, a.scale, a.guide, !STORED, sx, sg, sval);
  __syncthreads();
  const int lx = threadIdx.x % SH::tw, ly = threadIdx.x / SH::tw;
  const int x = bx + lx, y = by + ly;
  const bool active = x < g.nx && y < g.ny;
  const int hp0 = (ly + SH::ry) * SH::hw + (lx + SH::rx);
  float xi[K], acc[K], yv[K];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const Vec<float, V> v = sx[c * SH::hp + hp0];
#pragma unroll
    for (int e = 0; e < V; ++e) xi[c * V + e] = v.v[e];
  }
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = yv[c] = 0.0f;
  float wsum = 0.0f;
  const int64_t i = (int64_t)y * g.nx + x;
  if (active) {
    window_fast<SH, K, STORED>(g, hp0, i, g.nx, sg, sval, mask, sx, a.wf, a.wmode, a.n, xi, acc, wsum);
    const float s_i = a.scale ? a.scale[i] : 1.0f;
    if (a.op == BF_OP_DINV_W) {
      const float di = 1.0f / (1.0f + wsum);
#pragma unroll
      for (int c = 0; c < K; ++c) yv[c] = fmaf(-acc[c], di, xi[c]);
    } else {
#pragma unroll
      for (int c = 0; c < K; ++c) yv[c] = a.scale ? s_i * acc[c] : acc[c];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      Vec<float, V> o;
#pragma unroll
      for (int e = 0; e < V; ++e) o.v[e] = yv[c * V + e];
      *reinterpret_cast<Vec<float, V>*>(a.Y + i * a.ldy + c * V) = o;
    }
  }
  if (a.dots) {
    if (a.scale && active) {
#pragma unroll
      for (int c = 0; c < K; ++c) xi[c] = a.X[i * a.ldx + c];
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const float s = warp_sum(active ? xi[c] * yv[c] : 0.0f);
      if ((threadIdx.x & 31) == 0) atomicAdd(&a.dots[c], (double)s);
    }
  }
}

// One column (k = 1) through the 7 x 7 window, L-type operators (L, D^-1/2 L D^-1/2,
// (diag L)^-1/2 L (diag L)^-1/2): strip-blocked window sums (bf_strip.cuh), persistent over
// 32 x 32 tiles, optional fused dot x^T y.
template <int WM>
__global__ void __launch_bounds__(STRIP_THREADS, 2) k_apply1_strip(const Geom<float> g, const ApplyArgs<float> a) {
  const int nx = g.nx, ny = g.ny;
  float dsum = 0.0f;
  const float* src[3] = {a.X, a.scale, WM == BF_W_ONTHEFLY ? a.guide : nullptr};
  const int64_t ld[3] = {a.ldx, 1, 1};
  const bool scaled = a.scale != nullptr;
  auto combine = [&](float* st) {           // operand of the scaled operators: x * scale
    if (!scaled) return;
    for (int hp = threadIdx.x; hp < STRIP_HP; hp += STRIP_THREADS) st[hp] *= st[STRIP_HP + hp];
  };
  auto epi = [&](int bx, int by, int lx, int ly0, const float (&vi)[STRIP_P], const float (&acc)[STRIP_P]) {
    const int x = bx + lx;
#pragma unroll
    for (int j = 0; j < STRIP_P; ++j) {
      const int y = by + ly0 + j;
      if (x < nx && y < ny) {
        const int64_t i = (int64_t)y * nx + x;
        const float yv = scaled ? a.scale[i] * acc[j] : acc[j];
        a.Y[i * a.ldy] = yv;
        if (a.dots) dsum = fmaf(scaled ? a.X[i * a.ldx] : vi[j], yv, dsum);
      }
    }
  };
  strip_run<WM, 3, true>(g, a.wf, a.n, src, ld, 2, combine, epi);
  if (a.dots) {
    const float w = warp_sum(dsum);
    if ((threadIdx.x & 31) == 0) atomicAdd(a.dots, (double)w);
  }
}

// One column (k = 1) with stored weights through the 7 x 7 window by horizontal runs
// (bf_hrun.cuh): L-type operators, optional fused dot x^T y.  Needs nx % 4 == 0 and a
// contiguous operand.
template <int WM>
__global__ void __launch_bounds__(HRUN_THREADS, 3) k_apply1_hrun(const Geom<float> g, const ApplyArgs<float> a) {
  const int nx = g.nx, ny = g.ny;
  float dsum = 0.0f;
  const bool scaled = a.scale != nullptr;
  const float* src[2] = {a.X, a.scale};
  auto combine = [&](float* st) {           // operand of the scaled operators: x * scale
    if (!scaled) return;
    for (int e = threadIdx.x; e < HRUN_HP; e += HRUN_THREADS) st[e] *= st[HRUN_HP + e];
  };
  auto epi = [&](int bx, int by, int cx, int ry, const float (&vi)[HRUN_P], const float (&acc)[HRUN_P]) {
    const int y = by + ry;
    if (y >= ny) return;
#pragma unroll
    for (int j = 0; j < HRUN_P; ++j) {
      const int x = bx + cx + j;
      if (x < nx) {
        const int64_t i = (int64_t)y * nx + x;
        const float yv = scaled ? a.scale[i] * acc[j] : acc[j];
        a.Y[i * a.ldy] = yv;
        if (a.dots) dsum = fmaf(scaled ? a.X[i] : vi[j], yv, dsum);
      }
    }
  };
  hrun_run<WM, 2>(nx, ny, a.wf, a.n, src, combine, epi);
  if (a.dots) {
    const float w = warp_sum(dsum);
    if ((threadIdx.x & 31) == 0) atomicAdd(a.dots, (double)w);
  }
}

// Register-blocked operator for the 7 x 7 window (see RBTile): L-type operators, K >= 4.
template <int K, bool STORED>
__global__ void __launch_bounds__(BF_THREADS, 2) k_apply_rb(const Geom<float> g, const ApplyArgs<float> a) {
  typedef RBTile<K> TT;
  constexpr int CS = TT::cs, NG = TT::ng, NC4 = K / 4, CS4 = CS / 4;
  extern __shared__ __align__(16) unsigned char smem[];
  float4* sx = reinterpret_cast<float4*>(smem);                 // [NC4][hp]
  float* sg = reinterpret_cast<float*>(sx + NC4 * TT::hp);      // [hp]
  float* sval = sg + TT::hp;                                    // [hp]
  const int bx = blockIdx.x * TT::tw, by = blockIdx.y * TT::th;
  const bool mask = !(bx - 3 >= 0 && bx + TT::tw + 3 <= g.nx && by - 3 >= 0 && by + TT::th + 3 <= g.ny);
  for (int idx = threadIdx.x; idx < TT::hp * NC4; idx += BF_THREADS) {
    const int hp = idx / NC4, c = idx - hp * NC4;
    const int hy = hp / TT::hw, hx = hp - hy * TT::hw;
    const int gy = by - 3 + hy, gx = bx - 3 + hx;
    const bool in = (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny);
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (in) {
      const int64_t gp = (int64_t)gy * g.nx + gx;
      v = *reinterpret_cast<const float4*>(a.X + gp * a.ldx + c * 4);
      if (a.scale) {
        const float sc = a.scale[gp];
        v.x *= sc; v.y *= sc; v.z *= sc; v.w *= sc;
      }
      if (c == 0 && !STORED) sg[hp] = a.guide[gp];
    } else if (c == 0 && !STORED) {
      sg[hp] = 0.0f;
    }
    if (c == 0) sval[hp] = in ? 1.0f : 0.0f;
    sx[c * TT::hp + hp] = v;
  }
  __syncthreads();
  const int lx = threadIdx.x & 31;
  const int rest = threadIdx.x >> 5;
  const int grp = rest % NG, strip = rest / NG;
  const int x = bx + lx;
  const int row0 = strip * RB_P;                 // first strip row within the tile
  float xi[RB_P][CS], gi[RB_P];
  unsigned long long acc2[RB_P][CS / 2], xi2[RB_P][CS / 2];
  int64_t ip[RB_P];
  bool act[RB_P];
#pragma unroll
  for (int p = 0; p < RB_P; ++p) {
    const int hp = (row0 + p + 3) * TT::hw + lx + 3;
#pragma unroll
    for (int c4 = 0; c4 < CS4; ++c4) {
      const float4 v = sx[(grp * CS4 + c4) * TT::hp + hp];
      xi[p][4 * c4] = v.x; xi[p][4 * c4 + 1] = v.y; xi[p][4 * c4 + 2] = v.z; xi[p][4 * c4 + 3] = v.w;
    }
    gi[p] = STORED ? 0.0f : sg[hp];
    const int y = by + row0 + p;
    act[p] = (x < g.nx && y < g.ny);
    ip[p] = (int64_t)y * g.nx + x;
#pragma unroll
    for (int c = 0; c < CS / 2; ++c) {
      acc2[p][c] = f2_pack(0.0f, 0.0f);
      xi2[p][c] = f2_pack(xi[p][2 * c], xi[p][2 * c + 1]);
    }
  }
#pragma unroll
  for (int r = 0; r < RB_P + 6; ++r) {
#pragma unroll
    for (int dx = -3; dx <= 3; ++dx) {
      const int hp = (row0 + r) * TT::hw + lx + 3 + dx;
      unsigned long long xj2[CS / 2];
#pragma unroll
      for (int c4 = 0; c4 < CS4; ++c4) {
        const float4 v = sx[(grp * CS4 + c4) * TT::hp + hp];
        xj2[2 * c4] = f2_pack(v.x, v.y);
        xj2[2 * c4 + 1] = f2_pack(v.z, v.w);
      }
      const float gj = STORED ? 0.0f : sg[hp];
      const float vj = mask ? sval[hp] : 1.0f;
#pragma unroll
      for (int p = 0; p < RB_P; ++p) {
        const int dy = r - 3 - p;
        if (dy < -3 || dy > 3 || (dy == 0 && dx == 0)) continue;
        float w;
        if (STORED) {
          const bool ok = act[p] && vj != 0.0f;
          if (dy > 0 || (dy == 0 && dx > 0)) {
            const int f = ShapeR3::fwd_index(dy, dx);
            w = ok ? ld_weight(a.wf, (int64_t)f * a.n + ip[p], a.wmode) : 0.0f;
          } else {
            const int f = ShapeR3::fwd_index(-dy, -dx);
            w = ok ? ld_weight(a.wf, (int64_t)f * a.n + ip[p] + (int64_t)dy * g.nx + dx, a.wmode) : 0.0f;
          }
        } else {
          w = rb_exp(gi[p], gj, g.a_r, g.ls[(dy + 3) * 7 + (dx + 3)]) * vj;
        }
        const unsigned long long w2 = f2_pack(w, w);
#pragma unroll
        for (int c = 0; c < CS / 2; ++c) acc2[p][c] = f2_diff_fma(w2, xi2[p][c], xj2[c], acc2[p][c]);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < RB_P; ++p) {
    if (!act[p]) continue;
    const float s_i = a.scale ? a.scale[ip[p]] : 1.0f;
#pragma unroll
    for (int c4 = 0; c4 < CS4; ++c4) {
      float4 o;
      f2_unpack(acc2[p][2 * c4], o.x, o.y);
      f2_unpack(acc2[p][2 * c4 + 1], o.z, o.w);
      o.x *= s_i; o.y *= s_i; o.z *= s_i; o.w *= s_i;
      *reinterpret_cast<float4*>(a.Y + ip[p] * a.ldy + (grp * CS4 + c4) * 4) = o;
    }
  }
}

// Persistent, double-buffered form of k_apply_rb for the L operator with weights on the
// fly (unscaled operand): one CTA per SM walks tiles of 32 x th pixels; while it computes
// one tile the halo of its next tile is copied by cp.async (X in 16-byte pieces, zero
// outside the image; the guide in 4-byte pieces, +inf outside the image so that the range
// term gives a zero weight there and no mask is needed).  At K = 16 one thread carries all
// 16 columns of its 4-pixel strip (each weight computed once, 256 threads, ~200 registers);
// the other widths split the columns into groups of 8 (512 threads, <= 128 registers), as
// two halo buffers of a 16-column-per-thread tile would not fit in shared memory at K = 32.
template <int K>
struct PipeTile {
  static constexpr int threads = (K == 16) ? 256 : 512;
  static constexpr int cs = (K == 16) ? 16 : ((K < RB_CS) ? K : RB_CS);
  static constexpr int ng = K / cs;
  static constexpr int strips = threads / (32 * ng);
  static constexpr int tw = 32, th = RB_P * strips;
  static constexpr int hw = tw + 6, hh = th + 6, hp = hw * hh;
  static constexpr int nc4 = K / 4;
  // column-group stride in float4 units, = 2 (mod 8) so the four groups of one pixel fall
  // in different bank quads when the halo is written
  static constexpr int cst = hp + ((10 - hp % 8) % 8);
  static constexpr size_t xbytes = (size_t)cst * nc4 * 16;
  static constexpr size_t stage = xbytes + (((size_t)hp * 4 + 15) / 16) * 16;
  static constexpr size_t smem = 2 * stage;
};

// 2^a by the SFU's approximate exponential, subnormal results flushed to zero (weights
// below 2^-126 contribute nothing at FP32 precision); +inf / -inf arguments give +inf / 0.
__device__ __forceinline__ float rb_exp_ftz(float gi, float gj, float a_r, float ls) {
  const float dl = gi - gj;
  const float a = fmaf(-dl * a_r, dl, ls);
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

template <int K>
__device__ __forceinline__ void pipe_stage(const Geom<float>& g, const ApplyArgs<float>& a, int bx, int by,
                                           unsigned char* buf) {
  typedef PipeTile<K> TT;
  constexpr int NC4 = TT::nc4;
  const unsigned sx = (unsigned)__cvta_generic_to_shared(buf);
  const unsigned sg = sx + (unsigned)TT::xbytes;
  for (int idx = threadIdx.x; idx < TT::hp * NC4; idx += TT::threads) {
    const int hp = idx / NC4, c = idx - hp * NC4;
    const int hy = hp / TT::hw, hx = hp - hy * TT::hw;
    const int gy = by - 3 + hy, gx = bx - 3 + hx;
    const bool in = (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny);
    const float* src = in ? a.X + ((int64_t)gy * g.nx + gx) * a.ldx + c * 4 : a.X;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sx + (unsigned)(c * TT::cst + hp) * 16u),
                 "l"(src), "r"(in ? 16 : 0)
                 : "memory");
  }
  float* sgp = reinterpret_cast<float*>(buf + TT::xbytes);
  for (int hp = threadIdx.x; hp < TT::hp; hp += TT::threads) {
    const int hy = hp / TT::hw, hx = hp - hy * TT::hw;
    const int gy = by - 3 + hy, gx = bx - 3 + hx;
    if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) {
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sg + (unsigned)hp * 4u),
                   "l"(a.guide + (int64_t)gy * g.nx + gx)
                   : "memory");
    } else {
      sgp[hp] = __int_as_float(0x7f800000);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(PipeTile<K>::threads, 1) k_apply_pipe(const Geom<float> g, const ApplyArgs<float> a) {
  bf_pdl_enter();
  typedef PipeTile<K> TT;
  constexpr int CS = TT::cs, NG = TT::ng, CS4 = CS / 4;
  extern __shared__ __align__(16) unsigned char smem[];
  const int ntx = (g.nx + TT::tw - 1) / TT::tw;
  const int ntiles = ntx * ((g.ny + TT::th - 1) / TT::th);
  const int lx = threadIdx.x & 31;
  const int rest = threadIdx.x >> 5;
  const int grp = rest % NG, strip = rest / NG;
  const int row0 = strip * RB_P;
  int t = blockIdx.x;
  if (t < ntiles) pipe_stage<K>(g, a, (t % ntx) * TT::tw, (t / ntx) * TT::th, smem);
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int b = 0; t < ntiles; t += gridDim.x, b ^= 1) {
    const int tn = t + gridDim.x;
    if (tn < ntiles) pipe_stage<K>(g, a, (tn % ntx) * TT::tw, (tn / ntx) * TT::th, smem + (b ^ 1) * TT::stage);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    const float4* sx = reinterpret_cast<const float4*>(smem + b * TT::stage);
    const float* sg = reinterpret_cast<const float*>(smem + b * TT::stage + TT::xbytes);
    const int bx = (t % ntx) * TT::tw, by = (t / ntx) * TT::th;
    const int x = bx + lx;
    float gi[RB_P];
    unsigned long long acc2[RB_P][CS / 2], xi2[RB_P][CS / 2];
#pragma unroll
    for (int p = 0; p < RB_P; ++p) {
      const int hp = (row0 + p + 3) * TT::hw + lx + 3;
#pragma unroll
      for (int c4 = 0; c4 < CS4; ++c4) {
        const float4 v = sx[(grp * CS4 + c4) * TT::cst + hp];
        xi2[p][2 * c4] = f2_pack(v.x, v.y);
        xi2[p][2 * c4 + 1] = f2_pack(v.z, v.w);
      }
      gi[p] = sg[hp];
#pragma unroll
      for (int c = 0; c < CS / 2; ++c) acc2[p][c] = f2_pack(0.0f, 0.0f);
    }
#pragma unroll
    for (int r = 0; r < RB_P + 6; ++r) {
#pragma unroll
      for (int dx = -3; dx <= 3; ++dx) {
        const int hp = (row0 + r) * TT::hw + lx + 3 + dx;
        unsigned long long xj2[CS / 2];
#pragma unroll
        for (int c4 = 0; c4 < CS4; ++c4) {
          const float4 v = sx[(grp * CS4 + c4) * TT::cst + hp];
          xj2[2 * c4] = f2_pack(v.x, v.y);
          xj2[2 * c4 + 1] = f2_pack(v.z, v.w);
        }
        const float gj = sg[hp];
#pragma unroll
        for (int p = 0; p < RB_P; ++p) {
          const int dy = r - 3 - p;
          if (dy < -3 || dy > 3 || (dy == 0 && dx == 0)) continue;
          const float w = rb_exp_ftz(gi[p], gj, g.a_r, g.ls[(dy + 3) * 7 + (dx + 3)]);
          const unsigned long long w2 = f2_pack(w, w);
#pragma unroll
          for (int c = 0; c < CS / 2; ++c) acc2[p][c] = f2_diff_fma(w2, xi2[p][c], xj2[c], acc2[p][c]);
        }
      }
    }
#pragma unroll
    for (int p = 0; p < RB_P; ++p) {
      const int y = by + row0 + p;
      if (x >= g.nx || y >= g.ny) continue;
      float* yp = a.Y + ((int64_t)y * g.nx + x) * a.ldy + grp * CS;
#pragma unroll
      for (int c4 = 0; c4 < CS4; ++c4) {
        float4 o;
        f2_unpack(acc2[p][2 * c4], o.x, o.y);
        f2_unpack(acc2[p][2 * c4 + 1], o.z, o.w);
        *reinterpret_cast<float4*>(yp + 4 * c4) = o;
      }
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

static int num_sms() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 1;
  }
  return nsm;
}

template <int K>
static int launch_apply_pipe(const bf_graph* g, const ApplyArgs<float>& a, cudaStream_t s) {
  typedef PipeTile<K> TT;
  static_assert(TT::smem <= 227 * 1024, "pipelined apply tile does not fit in shared memory");
  {
    const int rc_ = bf_smem_attr((const void*)k_apply_pipe<K>, (int)TT::smem, "cudaFuncSetAttribute(k_apply_pipe)");
    if (rc_) return rc_;
  }
  const int64_t ntiles = ((g->nx + TT::tw - 1) / TT::tw) * (int64_t)((g->ny + TT::th - 1) / TT::th);
  const int grid = (int)std::min<int64_t>(ntiles, num_sms());
  BF_LAUNCH_PDL(k_apply_pipe<K>, grid, TT::threads, TT::smem, s, g->gf, a);
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

template <int K, bool STORED>
static int launch_apply_rb(const bf_graph* g, const ApplyArgs<float>& a, cudaStream_t s) {
  typedef RBTile<K> TT;
  const size_t sm = (size_t)TT::hp * (K / 4) * sizeof(float4) + 2 * TT::hp * sizeof(float);
  {
    const int rc_ = bf_smem_attr((const void*)k_apply_rb<K, STORED>, 227 * 1024, "cudaFuncSetAttribute(k_apply_rb)");
    if (rc_) return rc_;
  }
  const dim3 grid((unsigned)((g->nx + TT::tw - 1) / TT::tw), (unsigned)((g->ny + TT::th - 1) / TT::th), 1);
  BF_LAUNCH(k_apply_rb<K, STORED><<<grid, BF_THREADS, sm, s>>>(g->gf, a));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

template <int K>
static int launch_apply_rb_w(const bf_graph* g, const ApplyArgs<float>& a, cudaStream_t s) {
  if (g->p.weight_mode == BF_W_ONTHEFLY && a.op == BF_OP_L && !a.scale && g->gf.a_r > 0.0f &&
      ((uintptr_t)a.X & 15) == 0 && ((uintptr_t)a.Y & 15) == 0 && a.ldx % 4 == 0 && a.ldy % 4 == 0)
    return launch_apply_pipe<K>(g, a, s);
  if (g->p.weight_mode == BF_W_ONTHEFLY) return launch_apply_rb<K, false>(g, a, s);
  return launch_apply_rb<K, true>(g, a, s);
}

template <class SH, int K, bool STORED>
static int launch_apply_fast(const bf_graph* g, const ApplyArgs<float>& a, cudaStream_t s) {
  constexpr int V = VecW<float, K>::value;
  const size_t sm = (size_t)SH::hp * (K / V) * sizeof(Vec<float, V>) + 2 * SH::hp * sizeof(float);
  {
    const int rc_ = bf_smem_attr((const void*)k_apply_fast<SH, K, STORED>, 227 * 1024, "cudaFuncSetAttribute(k_apply_fast)");
    if (rc_) return rc_;
  }
  BF_LAUNCH(k_apply_fast<SH, K, STORED><<<tile_grid(g), BF_THREADS, sm, s>>>(g->gf, a));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

template <class SH, int K>
static int launch_apply_fast_w(const bf_graph* g, const ApplyArgs<float>& a, cudaStream_t s) {
  if (g->p.weight_mode == BF_W_ONTHEFLY) return launch_apply_fast<SH, K, false>(g, a, s);
  return launch_apply_fast<SH, K, true>(g, a, s);
}

static int strip_occupancy(const void* fn) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, STRIP_THREADS, STRIP_SMEM_BYTES) != cudaSuccess ||
      per < 1)
    per = 1;
  return per;
}

template <int WM>
static int launch_apply1_strip(const bf_graph* g, const ApplyArgs<float>& a, cudaStream_t s) {
  static int per_sm = 0;
  if (per_sm == 0) per_sm = strip_occupancy((const void*)k_apply1_strip<WM>);
  const int64_t ntiles = (int64_t)strip_tiles_x(g->nx) * strip_tiles_y(g->ny);
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)per_sm * num_sms());
  BF_LAUNCH(k_apply1_strip<WM><<<grid, STRIP_THREADS, STRIP_SMEM_BYTES, s>>>(g->gf, a));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

template <int WM>
static int launch_apply1_hrun(const bf_graph* g, const ApplyArgs<float>& a, cudaStream_t s) {
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply1_hrun<WM>, HRUN_THREADS, HRUN_SMEM_BYTES) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  const int64_t ntiles = (int64_t)((g->nx + HRUN_TW - 1) / HRUN_TW) * ((g->ny + HRUN_TH - 1) / HRUN_TH);
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)per_sm * num_sms());
  BF_LAUNCH(k_apply1_hrun<WM><<<grid, HRUN_THREADS, HRUN_SMEM_BYTES, s>>>(g->gf, a));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

static int launch_apply1_strip_w(const bf_graph* g, const ApplyArgs<float>& a, cudaStream_t s) {
  // stored weights by horizontal runs when the rows are whole 16-byte vectors of the planes
  if (g->p.weight_mode != BF_W_ONTHEFLY && g->nx % 4 == 0 && a.ldx == 1 && ((uintptr_t)g->wf & 15) == 0) {
    if (g->p.weight_mode == BF_W_STORED_BF16) return launch_apply1_hrun<BF_W_STORED_BF16>(g, a, s);
    return launch_apply1_hrun<BF_W_STORED_F32>(g, a, s);
  }
  switch (g->p.weight_mode) {
    case BF_W_STORED_F32: return launch_apply1_strip<BF_W_STORED_F32>(g, a, s);
    case BF_W_STORED_BF16: return launch_apply1_strip<BF_W_STORED_BF16>(g, a, s);
  }
  return launch_apply1_strip<BF_W_ONTHEFLY>(g, a, s);
}

// Returns 1 when it launched the specialised kernel for this chunk width.
template <class SH>
static int apply_fast_shape(const bf_graph* g, int K, const ApplyArgs<float>& a, cudaStream_t s, int* rc) {
  switch (K) {
    case 1: *rc = launch_apply_fast_w<SH, 1>(g, a, s); return 1;
    case 4: *rc = launch_apply_fast_w<SH, 4>(g, a, s); return 1;
    case 8: *rc = launch_apply_fast_w<SH, 8>(g, a, s); return 1;
    case 16: *rc = launch_apply_fast_w<SH, 16>(g, a, s); return 1;
    case 32: *rc = launch_apply_fast_w<SH, 32>(g, a, s); return 1;
  }
  return 0;
}

static int try_apply_fast(const bf_graph* g, int K, const ApplyArgs<float>& a, cudaStream_t s, int* rc) {
  if (!(a.op == BF_OP_L || a.op == BF_OP_NSYM || a.op == BF_OP_NDIAGL || a.op == BF_OP_DINV_W)) return 0;
  if (fast_shape(g) == FAST_R3_2D && K == 1 && a.op != BF_OP_DINV_W) {
    *rc = launch_apply1_strip_w(g, a, s);
    return 1;
  }
  if (fast_shape(g) == FAST_R3_2D && !a.dots && a.op != BF_OP_DINV_W) {
    switch (K) {
      case 4: *rc = launch_apply_rb_w<4>(g, a, s); return 1;
      case 8: *rc = launch_apply_rb_w<8>(g, a, s); return 1;
      case 16: *rc = launch_apply_rb_w<16>(g, a, s); return 1;
      case 32: *rc = launch_apply_rb_w<32>(g, a, s); return 1;
    }
  }
  switch (fast_shape(g)) {
    case FAST_R3_2D: return apply_fast_shape<ShapeR3>(g, K, a, s, rc);
    case FAST_R5_1D: return apply_fast_shape<ShapeR5>(g, K, a, s, rc);
    case FAST_CROSS1: return apply_fast_shape<ShapeX1>(g, K, a, s, rc);
  }
  return 0;
}

template <typename T, int K>
static size_t apply_smem(const bf_graph* g) {
  const bool one_d = (g->ny == 1 && g->ry == 0);
  const int hw = (one_d ? BF_TW1 : BF_TW2) + 2 * g->rx;
  const int hh = (one_d ? 1 : BF_TH2) + 2 * g->ry;
  return (size_t)hw * hh * (K + 1) * sizeof(T);
}

template <typename T, int K>
static int launch_apply(const bf_graph* g, const ApplyArgs<T>& a, cudaStream_t s) {
  const size_t sm = apply_smem<T, K>(g);
  {
    const int rc_ = bf_smem_attr((const void*)k_apply<T, K>, 227 * 1024, "cudaFuncSetAttribute(k_apply)");
    if (rc_) return rc_;
  }
  if (sm > 227 * 1024) return bf_fail(BF_EINVAL, "bf_apply: tile does not fit in shared memory");
  BF_LAUNCH(k_apply<T, K><<<tile_grid(g), BF_THREADS, sm, s>>>(geom_of<T>(g), a));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

template <typename T>
static int apply_chunk(const bf_graph* g, int K, const ApplyArgs<T>& a, cudaStream_t s) {
  if (sizeof(T) == 4) {
    int rc = BF_OK;
    if (try_apply_fast(g, K, reinterpret_cast<const ApplyArgs<float>&>(a), s, &rc)) return rc;
  }
  switch (K) {
    case 1: return launch_apply<T, 1>(g, a, s);
    case 2: return launch_apply<T, 2>(g, a, s);
    case 4: return launch_apply<T, 4>(g, a, s);
    case 8: return launch_apply<T, 8>(g, a, s);
    case 16: return launch_apply<T, 16>(g, a, s);
    case 32: return launch_apply<T, 32>(g, a, s);
  }
  return bf_fail(BF_EINVAL, "bf_apply: bad chunk width");
}

// Apply op to k columns, split into power-of-two chunks whose vector loads are aligned.
template <typename T>
static int apply_block(const bf_graph* g, int op, const T* X, int64_t ldx, int k, T* Y,
                       int64_t ldy, double* dots, cudaStream_t s) {
  if (g->kind == BF_KIND_GUIDED) return bf_guided_apply<T>(g, op, X, ldx, k, Y, ldy, dots, nullptr, s);
  ApplyArgs<T> a;
  a.guide = (const T*)g->guide;
  a.scale = op == BF_OP_NSYM ? (const T*)g->dis : (op == BF_OP_NDIAGL ? (const T*)g->dls : nullptr);
  a.wf = g->wf;
  a.wmode = g->p.weight_mode;
  a.op = op;
  a.n = g->n;
  a.ldx = ldx;
  a.ldy = ldy;
  const int kmax_chunk = sizeof(T) == 8 ? 16 : 32;
  int c0 = 0;
  while (c0 < k) {
    int K = kmax_chunk;
    while (K > k - c0) K >>= 1;
    // shrink until the chunk's vector loads/stores are aligned
    for (;;) {
      const int V = (K % (16 / (int)sizeof(T)) == 0) ? 16 / (int)sizeof(T) : ((K % 2 == 0) ? 2 : 1);
      const size_t vb = (size_t)V * sizeof(T);
      const bool ok = ((uintptr_t)(X + c0) % vb == 0) && ((uintptr_t)(Y + c0) % vb == 0) &&
                      (ldx % V == 0) && (ldy % V == 0);
      if (ok || K == 1) break;
      K >>= 1;
    }
    a.X = X + c0;
    a.Y = Y + c0;
    a.dots = dots ? dots + c0 : nullptr;
    int rc = apply_chunk<T>(g, K, a, s);
    if (rc) return rc;
    c0 += K;
  }
  return BF_OK;
}

// Exposed to the solver translation units.
int bf_apply_f32(const bf_graph* g, int op, const float* X, int64_t ldx, int k, float* Y,
                 int64_t ldy, double* dots, cudaStream_t s) {
  return apply_block<float>(g, op, X, ldx, k, Y, ldy, dots, s);
}
int bf_apply_f64(const bf_graph* g, int op, const double* X, int64_t ldx, int k, double* Y,
                 int64_t ldy, double* dots, cudaStream_t s) {
  return apply_block<double>(g, op, X, ldx, k, Y, ldy, dots, s);
}

// One BF step y = D^-1 W x (one column) whose on-the-fly weights take `guide` instead of
// the graph's own guide (the re-guided iteration: guide = x).
template <typename T>
static int apply_bf_step_with_guide(const bf_graph* g, const T* guide, const T* X, T* Y, cudaStream_t s) {
  ApplyArgs<T> a;
  a.guide = guide;
  a.scale = nullptr;
  a.wf = g->wf;
  a.wmode = g->p.weight_mode;
  a.op = BF_OP_DINV_W;
  a.n = g->n;
  a.ldx = 1;
  a.ldy = 1;
  a.X = X;
  a.Y = Y;
  a.dots = nullptr;
  return apply_chunk<T>(g, 1, a, s);
}

// ================================================================== host: graph
template <typename T>
static void fill_geom(Geom<T>& G, const bf_params& p, int nx, int ny, int rx, int ry,
                      int nfwd, const std::vector<short>& fmap) {
  memset(&G, 0, sizeof(G));
  G.nx = nx;
  G.ny = ny;
  G.rx = rx;
  G.ry = ry;
  G.cross = (p.window == BF_WINDOW_CROSS);
  G.nfwd = nfwd;
  const bool is_f = sizeof(T) == 4;
  const double log2e = 1.4426950408889634;
  const double ar = std::isinf(p.sigma_r) ? 0.0 : 1.0 / (2.0 * p.sigma_r * p.sigma_r);
  const double as = std::isinf(p.sigma_s) ? 0.0 : 1.0 / (2.0 * p.sigma_s * p.sigma_s);
  G.a_r = (T)(is_f ? ar * log2e : ar);
  const int bw = 2 * rx + 1;
  for (int dy = -ry; dy <= ry; ++dy)
    for (int dx = -rx; dx <= rx; ++dx) {
      const int cell = (dy + ry) * bw + (dx + rx);
      const double l = -(double)(dx * dx + dy * dy) * as;
      G.ls[cell] = (T)(is_f ? l * log2e : l);
      G.fmap[cell] = fmap[cell];
    }
}

static int compute_weights(bf_graph* g, const void* guide, cudaStream_t s);

extern "C" int bf_weights(const bf_params* p, const void* guide, bf_graph** out, void* stream) {
  if (!p || !guide || !out) return bf_fail(BF_EINVAL, "bf_weights: NULL argument");
  *out = nullptr;
  if (p->ndim != 1 && p->ndim != 2) return bf_fail(BF_EINVAL, "bf_weights: ndim must be 1 or 2");
  if (p->nx < 1 || p->ny < 1) return bf_fail(BF_EINVAL, "bf_weights: empty signal");
  if (p->ndim == 1 && p->ny != 1) return bf_fail(BF_EINVAL, "bf_weights: ndim 1 needs ny = 1");
  if (p->nx > INT32_MAX || p->ny > INT32_MAX || p->nx * p->ny > ((int64_t)1 << 40))
    return bf_fail(BF_EINVAL, "bf_weights: signal too large");
  const int rmax = p->ndim == 2 ? BF_MAX_R2D : BF_MAX_R1D;
  if (p->radius < 1 || p->radius > rmax) return bf_fail(BF_EINVAL, "bf_weights: radius out of range");
  if (p->window != BF_WINDOW_SQUARE && p->window != BF_WINDOW_CROSS)
    return bf_fail(BF_EINVAL, "bf_weights: bad window");
  if (p->weight_mode < BF_W_ONTHEFLY || p->weight_mode > BF_W_STORED_BF16)
    return bf_fail(BF_EINVAL, "bf_weights: bad weight_mode");
  if (p->dtype != BF_F32 && p->dtype != BF_F64) return bf_fail(BF_EINVAL, "bf_weights: bad dtype");
  if (p->reserved != 0) return bf_fail(BF_EINVAL, "bf_weights: reserved must be 0");
  if (!(p->sigma_s > 0) || !(p->sigma_r > 0)) return bf_fail(BF_EINVAL, "bf_weights: sigmas must be > 0");
  const size_t esz = p->dtype == BF_F64 ? 8 : 4;
  if ((uintptr_t)guide % esz) return bf_fail(BF_EINVAL, "bf_weights: misaligned guide");
  cudaStream_t s = (cudaStream_t)stream;

  bf_graph* g = new bf_graph();
  memset(g, 0, sizeof(*g));
  g->p = *p;
  g->nx = (int)p->nx;
  g->ny = (int)p->ny;
  g->n = p->nx * p->ny;
  g->rx = p->radius;
  g->ry = p->ndim == 2 ? p->radius : 0;
  g->esize = esz;
  cudaGetDevice(&g->device);
  // taps and forward map
  const int bw = 2 * g->rx + 1, bh = 2 * g->ry + 1;
  std::vector<short> fmap(bw * bh, -1);
  int ntaps = 0, nfwd = 0;
  for (int dy = -g->ry; dy <= g->ry; ++dy)
    for (int dx = -g->rx; dx <= g->rx; ++dx) {
      if (p->window == BF_WINDOW_CROSS && dx != 0 && dy != 0) continue;
      ++ntaps;
      if (dy > 0 || (dy == 0 && dx > 0)) fmap[(dy + g->ry) * bw + (dx + g->rx)] = (short)nfwd++;
    }
  g->ntaps = ntaps;
  g->nfwd = nfwd;
  fill_geom<float>(g->gf, *p, g->nx, g->ny, g->rx, g->ry, nfwd, fmap);
  fill_geom<double>(g->gd, *p, g->nx, g->ny, g->rx, g->ry, nfwd, fmap);

  const size_t nb = (size_t)g->n * esz;
  auto cleanup = [&](int code) {
    bf_graph_free(g);
    return code;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&g->guide, nb)) != cudaSuccess) return cleanup(bf_cuda_fail(e, "cudaMalloc(guide)"));
  if ((e = cudaMalloc(&g->d, nb)) != cudaSuccess) return cleanup(bf_cuda_fail(e, "cudaMalloc(d)"));
  if ((e = cudaMalloc(&g->dinv, nb)) != cudaSuccess) return cleanup(bf_cuda_fail(e, "cudaMalloc(dinv)"));
  if ((e = cudaMalloc(&g->dis, nb)) != cudaSuccess) return cleanup(bf_cuda_fail(e, "cudaMalloc(dis)"));
  if ((e = cudaMalloc(&g->dls, nb)) != cudaSuccess) return cleanup(bf_cuda_fail(e, "cudaMalloc(dls)"));
  if (p->weight_mode != BF_W_ONTHEFLY) {
    if (p->weight_mode == BF_W_STORED_BF16 && p->dtype != BF_F32)
      return cleanup(bf_fail(BF_EINVAL, "bf_weights: bf16 weights need dtype BF_F32"));
    const size_t wb = (size_t)nfwd * g->n * (p->weight_mode == BF_W_STORED_BF16 ? 2 : 4);
    if ((e = cudaMalloc(&g->wf, wb)) != cudaSuccess) return cleanup(bf_cuda_fail(e, "cudaMalloc(weights)"));
  }
  if ((e = cudaMalloc(&g->flag, sizeof(int))) != cudaSuccess) return cleanup(bf_cuda_fail(e, "cudaMalloc(flag)"));
  const int rc = compute_weights(g, guide, s);
  if (rc) return cleanup(rc);
  *out = g;
  return BF_OK;
}

// Copy the guide into the graph and compute the degree, the scalings and (stored modes)
// the weights; synchronises s to report a non-finite guide.
// Eq. 2 weights, degree and scalings of g for a new guide, enqueued on s; a non-finite
// guide value sets g->flag (which the caller clears and reads).
static int launch_weights(bf_graph* g, const void* guide, cudaStream_t s) {
  if (g->kind == BF_KIND_GUIDED) return bf_guided_prep(g, guide, s);
  const size_t nb = (size_t)g->n * g->esize;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(g->guide, guide, nb, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return bf_cuda_fail(e, "cudaMemcpyAsync(guide)");
  const unsigned blocks = (unsigned)((g->n + BF_THREADS - 1) / BF_THREADS);
  if (g->esize == 4)
    BF_LAUNCH(k_weights<float><<<blocks, BF_THREADS, 0, s>>>(g->gf, (const float*)g->guide, g->n, (float*)g->d,
                                                   (float*)g->dinv, (float*)g->dis, (float*)g->dls,
                                                   g->wf, g->p.weight_mode, g->flag));
  else
    BF_LAUNCH(k_weights<double><<<blocks, BF_THREADS, 0, s>>>(g->gd, (const double*)g->guide, g->n, (double*)g->d,
                                                    (double*)g->dinv, (double*)g->dis, (double*)g->dls,
                                                    g->wf, g->p.weight_mode, g->flag));
  if ((e = cudaGetLastError()) != cudaSuccess) return bf_cuda_fail(e, "k_weights launch");
  return BF_OK;
}

static int read_flag(bf_graph* g, cudaStream_t s, const char* what) {
  cudaError_t e;
  int hflag = 0;
  if ((e = cudaMemcpyAsync(&hflag, g->flag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return bf_cuda_fail(e, "cudaMemcpyAsync(flag)");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bf_cuda_fail(e, "weights sync");
  if (hflag) return bf_fail(BF_ENONFINITE, what);
  return BF_OK;
}

static int compute_weights(bf_graph* g, const void* guide, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(g->flag, 0, sizeof(int), s)) != cudaSuccess) return bf_cuda_fail(e, "memset(flag)");
  const int rc = launch_weights(g, guide, s);
  if (rc) return rc;
  return read_flag(g, s, "bf_weights: guide holds NaN or Inf");
}

extern "C" int bf_graph_update(bf_graph* g, const void* guide, void* stream) {
  if (!g || !guide) return bf_fail(BF_EINVAL, "bf_graph_update: NULL argument");
  if ((uintptr_t)guide % g->esize) return bf_fail(BF_EINVAL, "bf_graph_update: misaligned guide");
  return compute_weights(g, guide, (cudaStream_t)stream);
}

// The guided filter's graph (Section 3, Algorithm 1, Eq. 6): window statistics of the
// guide; the operator itself is applied matrix-free (bf_guided.cu).
extern "C" int bf_guided_graph(const bf_guided_params* p, const void* guide, bf_graph** out, void* stream) {
  if (!p || !guide || !out) return bf_fail(BF_EINVAL, "bf_guided_graph: NULL argument");
  *out = nullptr;
  if (p->ndim != 1 && p->ndim != 2) return bf_fail(BF_EINVAL, "bf_guided_graph: ndim must be 1 or 2");
  if (p->nx < 1 || p->ny < 1) return bf_fail(BF_EINVAL, "bf_guided_graph: empty signal");
  if (p->ndim == 1 && p->ny != 1) return bf_fail(BF_EINVAL, "bf_guided_graph: ndim 1 needs ny = 1");
  if (p->nx > INT32_MAX || p->ny > INT32_MAX || p->nx * p->ny > ((int64_t)1 << 40))
    return bf_fail(BF_EINVAL, "bf_guided_graph: signal too large");
  const int rmax = p->ndim == 2 ? BF_GF_MAX_R2D : BF_GF_MAX_R1D;
  if (p->radius < 1 || p->radius > rmax) return bf_fail(BF_EINVAL, "bf_guided_graph: radius out of range");
  if (p->dtype != BF_F32 && p->dtype != BF_F64) return bf_fail(BF_EINVAL, "bf_guided_graph: bad dtype");
  if (p->reserved != 0) return bf_fail(BF_EINVAL, "bf_guided_graph: reserved must be 0");
  if (!(p->eps > 0) || !std::isfinite(p->eps)) return bf_fail(BF_EINVAL, "bf_guided_graph: eps must be > 0");
  const size_t esz = p->dtype == BF_F64 ? 8 : 4;
  if ((uintptr_t)guide % esz) return bf_fail(BF_EINVAL, "bf_guided_graph: misaligned guide");
  cudaStream_t s = (cudaStream_t)stream;
  bf_graph* g = new bf_graph();
  memset(g, 0, sizeof(*g));
  g->kind = BF_KIND_GUIDED;
  g->eps = p->eps;
  g->p.ndim = p->ndim;
  g->p.radius = p->radius;
  g->p.nx = p->nx;
  g->p.ny = p->ny;
  g->p.window = BF_WINDOW_SQUARE;
  g->p.weight_mode = BF_W_ONTHEFLY;
  g->p.dtype = p->dtype;
  g->p.sigma_s = g->p.sigma_r = INFINITY;
  g->nx = (int)p->nx;
  g->ny = (int)p->ny;
  g->n = p->nx * p->ny;
  g->rx = p->radius;
  g->ry = p->ndim == 2 ? p->radius : 0;
  g->ntaps = (2 * g->rx + 1) * (2 * g->ry + 1);
  g->esize = esz;
  cudaGetDevice(&g->device);
  const size_t nb = (size_t)g->n * esz;
  auto cleanup = [&](int code) {
    bf_graph_free(g);
    return code;
  };
  cudaError_t e;
  void** bufs[] = {&g->guide, &g->d, &g->dinv, &g->dis, &g->dls, &g->gmu, &g->givar};
  for (void** b : bufs)
    if ((e = cudaMalloc(b, nb)) != cudaSuccess) return cleanup(bf_cuda_fail(e, "cudaMalloc(guided graph)"));
  if ((e = cudaMalloc(&g->flag, sizeof(int))) != cudaSuccess) return cleanup(bf_cuda_fail(e, "cudaMalloc(flag)"));
  if ((e = cudaMemsetAsync(g->flag, 0, sizeof(int), s)) != cudaSuccess) return cleanup(bf_cuda_fail(e, "memset(flag)"));
  int rc = bf_guided_prep(g, guide, s);
  if (!rc) rc = read_flag(g, s, "bf_guided_graph: guide holds NaN or Inf");
  if (rc) return cleanup(rc);
  *out = g;
  return BF_OK;
}

// Section 2, the first way of iterating the filter: every step takes the current iterate
// as the guide of Eq. 2, then applies one step x <- D^-1 W x; g ends up holding the graph
// (weights, degree, scalings) of the last guide.  The non-finite check of that guide is
// read once, after the last step (a NaN or Inf in an earlier iterate reaches it through
// the window sums).
extern "C" int bf_reguided_filter(bf_graph* g, const void* x0, int iters, void* x_out, void* stream) {
  if (!g || !x0 || !x_out) return bf_fail(BF_EINVAL, "bf_reguided_filter: NULL argument");
  if (iters < 0) return bf_fail(BF_EINVAL, "bf_reguided_filter: iters < 0");
  if ((uintptr_t)x0 % g->esize || (uintptr_t)x_out % g->esize)
    return bf_fail(BF_EINVAL, "bf_reguided_filter: misaligned vector");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nb = (size_t)g->n * g->esize;
  if (iters == 0) {
    if (x0 != x_out) BF_CUDA(cudaMemcpyAsync(x_out, x0, nb, cudaMemcpyDeviceToDevice, s));
    return BF_OK;
  }
  const size_t nba = (nb + 255) & ~(size_t)255;
  int rc = bf_ws_reserve(g, BF_WS_SIMPLE, 2 * nba);
  if (rc) return rc;
  void* tmp[2] = {g->ws[BF_WS_SIMPLE], (char*)g->ws[BF_WS_SIMPLE] + nba};
  BF_CUDA(cudaMemsetAsync(g->flag, 0, sizeof(int), s));
  // on-the-fly weights: one kernel per step, the iterate staged as its own guide; the graph
  // is rebuilt once, for the last guide.  Stored weights: rebuilt every step.
  const bool otf = g->p.weight_mode == BF_W_ONTHEFLY && g->kind == BF_KIND_BILATERAL;
  const void* src = x0;
  for (int it = 0; it < iters; ++it) {
    const bool last = (it == iters - 1);
    void* dst = (last && x_out != src) ? x_out : tmp[it & 1];
    if (!otf) {
      rc = launch_weights(g, src, s);
      if (rc) return rc;
    }
    if (g->kind == BF_KIND_GUIDED)                   // the window statistics of src are in g
      rc = (g->esize == 4)
               ? bf_guided_apply<float>(g, BF_OP_DINV_W, (const float*)src, 1, 1, (float*)dst, 1, nullptr, nullptr, s)
               : bf_guided_apply<double>(g, BF_OP_DINV_W, (const double*)src, 1, 1, (double*)dst, 1, nullptr, nullptr, s);
    else
      rc = (g->esize == 4)
               ? apply_bf_step_with_guide<float>(g, (const float*)src, (const float*)src, (float*)dst, s)
               : apply_bf_step_with_guide<double>(g, (const double*)src, (const double*)src, (double*)dst, s);
    if (rc) return rc;
    if (last && otf) {
      rc = launch_weights(g, src, s);              // src is intact: dst differs from it
      if (rc) return rc;
    }
    if (last && dst != x_out) BF_CUDA(cudaMemcpyAsync(x_out, dst, nb, cudaMemcpyDeviceToDevice, s));
    src = dst;
  }
  return read_flag(g, s, "bf_reguided_filter: an iterate holds NaN or Inf");
}

extern "C" int bf_graph_free(bf_graph* g) {
  if (!g) return BF_OK;
  void* bufs[] = {g->guide, g->d, g->dinv, g->dis, g->dls, g->wf, g->ws[0], g->ws[1], g->ws[2], g->flag,
                  g->gmu, g->givar};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete g;
  return BF_OK;
}

extern "C" int bf_graph_info(const bf_graph* g, int64_t* n, int32_t* taps, int32_t* dtype) {
  if (!g) return bf_fail(BF_EINVAL, "bf_graph_info: NULL graph");
  if (n) *n = g->n;
  if (taps) *taps = g->ntaps;
  if (dtype) *dtype = g->p.dtype;
  return BF_OK;
}

extern "C" int bf_graph_degree(const bf_graph* g, void* d_out, void* stream) {
  if (!g || !d_out) return bf_fail(BF_EINVAL, "bf_graph_degree: NULL argument");
  BF_CUDA(cudaMemcpyAsync(d_out, g->d, (size_t)g->n * g->esize, cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream));
  return BF_OK;
}

extern "C" int bf_graph_export_weights(const bf_graph* g, void* out, void* stream) {
  if (!g || !out) return bf_fail(BF_EINVAL, "bf_graph_export_weights: NULL argument");
  if (g->kind == BF_KIND_GUIDED)
    return bf_fail(BF_EINVAL, "bf_graph_export_weights: a guided graph has no per-tap weights");
  if ((uintptr_t)out % g->esize) return bf_fail(BF_EINVAL, "bf_graph_export_weights: misaligned output");
  const unsigned blocks = (unsigned)((g->n + BF_THREADS - 1) / BF_THREADS);
  cudaStream_t s = (cudaStream_t)stream;
  if (g->esize == 4)
    BF_LAUNCH(k_export<float><<<blocks, BF_THREADS, 0, s>>>(g->gf, (const float*)g->guide, g->n, g->wf,
                                                  g->p.weight_mode, g->ntaps, (float*)out));
  else
    BF_LAUNCH(k_export<double><<<blocks, BF_THREADS, 0, s>>>(g->gd, (const double*)g->guide, g->n, g->wf,
                                                   g->p.weight_mode, g->ntaps, (double*)out));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

// ================================================================== host: operator
extern "C" int bf_apply(const bf_graph* g, int op, const void* X, int64_t ldx, int k, void* Y,
                        int64_t ldy, double* dots, void* stream) {
  if (!g || !X || !Y) return bf_fail(BF_EINVAL, "bf_apply: NULL argument");
  if (op < BF_OP_W || op > BF_OP_NDIAGL) return bf_fail(BF_EINVAL, "bf_apply: bad op");
  if (k < 1 || ldx < k || ldy < k) return bf_fail(BF_EINVAL, "bf_apply: need k >= 1 and ld >= k");
  if ((uintptr_t)X % g->esize || (uintptr_t)Y % g->esize)
    return bf_fail(BF_EINVAL, "bf_apply: misaligned X or Y");
  const char* xb = (const char*)X;
  const char* yb = (const char*)Y;
  const size_t xspan = ((size_t)(g->n - 1) * ldx + k) * g->esize;
  const size_t yspan = ((size_t)(g->n - 1) * ldy + k) * g->esize;
  if (xb < yb + yspan && yb < xb + xspan) return bf_fail(BF_EINVAL, "bf_apply: X and Y overlap");
  cudaStream_t s = (cudaStream_t)stream;
  if (dots) BF_CUDA(cudaMemsetAsync(dots, 0, sizeof(double) * k, s));
  if (g->esize == 4) return bf_apply_f32(g, op, (const float*)X, ldx, k, (float*)Y, ldy, dots, s);
  return bf_apply_f64(g, op, (const double*)X, ldx, k, (double*)Y, ldy, dots, s);
}

extern "C" int bf_simple_filter(const bf_graph* g, const void* x0, int iters, void* x_out,
                                void* stream) {
  if (!g || !x0 || !x_out) return bf_fail(BF_EINVAL, "bf_simple_filter: NULL argument");
  if (iters < 0) return bf_fail(BF_EINVAL, "bf_simple_filter: iters < 0");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nb = (size_t)g->n * g->esize;
  if (iters == 0) {
    if (x0 != x_out) BF_CUDA(cudaMemcpyAsync(x_out, x0, nb, cudaMemcpyDeviceToDevice, s));
    return BF_OK;
  }
  bf_graph* gm = const_cast<bf_graph*>(g);
  const size_t nba = (nb + 255) & ~(size_t)255;
  int rc = bf_ws_reserve(gm, BF_WS_SIMPLE, 2 * nba);
  if (rc) return rc;
  void* tmp[2] = {gm->ws[BF_WS_SIMPLE], (char*)gm->ws[BF_WS_SIMPLE] + nba};
  // ping-pong through two temporaries; the last step writes x_out unless it aliases x0
  const void* src = x0;
  for (int it = 0; it < iters; ++it) {
    const bool last = (it == iters - 1);
    void* dst = (last && x_out != src) ? x_out : tmp[it & 1];
    rc = (g->esize == 4)
             ? bf_apply_f32(g, BF_OP_DINV_W, (const float*)src, 1, 1, (float*)dst, 1, nullptr, s)
             : bf_apply_f64(g, BF_OP_DINV_W, (const double*)src, 1, 1, (double*)dst, 1, nullptr, s);
    if (rc) return rc;
    if (last && dst != x_out) BF_CUDA(cudaMemcpyAsync(x_out, dst, nb, cudaMemcpyDeviceToDevice, s));
    src = dst;
  }
  return BF_OK;
}
