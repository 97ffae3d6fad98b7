// Specialised window sum of the Laplacian-type operators (L, D^-1/2 L D^-1/2,
// (diag L)^-1/2 L (diag L)^-1/2) for the window shapes the filters use: the 7 x 7 image
// window (radius 3), the 11-tap signal window (radius 5) and the 5-point lattice (cross,
// radius 1).  With the shape known at compile time the tap loop is fully unrolled: tap
// offsets, halo addresses and spatial factors are immediates.  Blocks whose halo lies
// inside the image take the unmasked path; border blocks multiply each weight by the
// staged 0/1 validity of the neighbour (neighbours outside the image do not exist), so
// every lane follows the same code.  Column arithmetic uses packed f32x2 instructions
// (two columns per instruction) in the difference form acc += w (x_i - x_j).
#pragma once

#include "bf_internal.cuh"

// Window of radii RX, RY (CROSS: the 5-point-like cross) on tiles of TW x TH pixels.
template <int RX, int RY, bool CROSS, int TW = (RY == 0 ? BF_TW1 : BF_TW2), int TH = (RY == 0 ? 1 : BF_TH2)>
struct WinShapeT {
  static constexpr int rx = RX, ry = RY;
  static constexpr bool cross = CROSS;
  static constexpr bool one_d = (RY == 0);
  static constexpr int tw = TW;
  static constexpr int th = TH;
  static constexpr int hw = tw + 2 * RX;
  static constexpr int hh = th + 2 * RY;
  static constexpr int hp = hw * hh;
  static constexpr int bw = 2 * RX + 1;
  __host__ __device__ static constexpr bool in_window(int dy, int dx) {
    return !(dy == 0 && dx == 0) && !(CROSS && dx != 0 && dy != 0);
  }
  __host__ __device__ static constexpr bool forward(int dy, int dx) { return dy > 0 || (dy == 0 && dx > 0); }
  // index of a forward cell among the forward cells of the window, row-major
  __host__ __device__ static constexpr int fwd_index(int dy, int dx) {
    int f = 0;
    for (int yy = -RY; yy <= RY; ++yy)
      for (int xx = -RX; xx <= RX; ++xx) {
        if (yy == dy && xx == dx) return f;
        if (in_window(yy, xx) && forward(yy, xx)) ++f;
      }
    return -1;
  }
};

__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
// acc += w * (xi - xj) on two packed columns
__device__ __forceinline__ unsigned long long f2_diff_fma(unsigned long long w2, unsigned long long xi,
                                                          unsigned long long xj, unsigned long long acc) {
  unsigned long long d, r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(xi), "l"(xj));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(w2), "l"(d), "l"(acc));
  return r;
}

// Window sum for this thread's pixel, float operand tile [K / V][hp] in shared memory.
// acc[c] += w_ij (xi[c] - x_j[c]) over the window's existing neighbours; wsum = sum w_ij.
// STORED: weights from the forward half-window array; else from the guide tile (Eq. 2).
// `mask` (block-uniform): multiply by the staged validity sval[hp].
template <class SH, int K, bool STORED>
__device__ __forceinline__ void window_fast(const Geom<float>& g, int hp0, int64_t i, int nx,
                                            const float* sg, const float* sval, bool mask,
                                            const Vec<float, VecW<float, K>::value>* sx,
                                            const void* wf, int wmode, int64_t n,
                                            const float (&xi)[K], float (&acc)[K], float& wsum) {
  constexpr int V = VecW<float, K>::value;
  constexpr int NC = K / V;
  const float gi = STORED ? 0.0f : sg[hp0];
  unsigned long long a2[(K + 1) / 2], xi2[(K + 1) / 2];
  if (K >= 2) {
#pragma unroll
    for (int c = 0; c < K / 2; ++c) {
      a2[c] = f2_pack(acc[2 * c], acc[2 * c + 1]);
      xi2[c] = f2_pack(xi[2 * c], xi[2 * c + 1]);
    }
  }
#pragma unroll
  for (int dy = -SH::ry; dy <= SH::ry; ++dy) {
#pragma unroll
    for (int dx = -SH::rx; dx <= SH::rx; ++dx) {
      if (!SH::in_window(dy, dx)) continue;
      const int hp = hp0 + dy * SH::hw + dx;
      const int cell = (dy + SH::ry) * SH::bw + (dx + SH::rx);
      float w;
      if (STORED) {
        const bool ok = !mask || sval[hp] != 0.0f;
        if (SH::forward(dy, dx)) {
          const int f = SH::fwd_index(dy, dx);
          w = ok ? ld_weight(wf, (int64_t)f * n + i, wmode) : 0.0f;
        } else {
          const int f = SH::fwd_index(-dy, -dx);
          w = ok ? ld_weight(wf, (int64_t)f * n + i + (int64_t)dy * nx + dx, wmode) : 0.0f;
        }
      } else {
        const float dl = gi - sg[hp];
        w = exp2f(fmaf(-dl * g.a_r, dl, g.ls[cell]));
        if (mask) w *= sval[hp];
      }
      wsum += w;
      if (K == 1) {
        acc[0] = fmaf(w, xi[0] - sx[hp].v[0], acc[0]);
      } else {
        const unsigned long long w2 = f2_pack(w, w);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const Vec<float, V> xj = sx[c * SH::hp + hp];
#pragma unroll
          for (int e = 0; e < V; e += 2) {
            const int q = (c * V + e) / 2;
            a2[q] = f2_diff_fma(w2, xi2[q], f2_pack(xj.v[e], xj.v[e + 1]), a2[q]);
          }
        }
      }
    }
  }
  if (K >= 2) {
#pragma unroll
    for (int c = 0; c < K / 2; ++c) f2_unpack(a2[c], acc[2 * c], acc[2 * c + 1]);
  }
}

template <int RX, int RY, bool CROSS>
using WinShape = WinShapeT<RX, RY, CROSS>;

// Which specialised shape (if any) a graph's window has.
enum { FAST_NONE = 0, FAST_R3_2D = 1, FAST_R5_1D = 2, FAST_CROSS1 = 3 };
inline int fast_shape(const bf_graph* g) {
  if (g->esize != 4) return FAST_NONE;
  const bool cross = g->p.window == BF_WINDOW_CROSS;
  const bool one_d = (g->ny == 1 && g->ry == 0);
  if (!one_d && !cross && g->rx == 3 && g->ry == 3) return FAST_R3_2D;
  if (one_d && !cross && g->rx == 5) return FAST_R5_1D;
  if (!one_d && cross && g->rx == 1 && g->ry == 1) return FAST_CROSS1;
  return FAST_NONE;
}
typedef WinShape<3, 3, false> ShapeR3;
typedef WinShape<5, 0, false> ShapeR5;
typedef WinShape<1, 1, true> ShapeX1;

// Stage the operand tile [K / V][hp] (optionally scaled per pixel), the guide and the 0/1
// validity of every halo pixel.
template <class SH, int K>
__device__ __forceinline__ void stage_fast(const Geom<float>& g, int bx, int by, const float* X,
                                           int64_t ldx, const float* scale, const float* guide,
                                           bool need_guide, Vec<float, VecW<float, K>::value>* sx,
                                           float* sg, float* sval) {
  constexpr int V = VecW<float, K>::value;
  constexpr int NC = K / V;
  for (int idx = threadIdx.x; idx < SH::hp * NC; idx += BF_THREADS) {
    const int hp = idx / NC, c = idx - hp * NC;
    const int hy = hp / SH::hw, hx = hp - hy * SH::hw;
    const int gy = by - SH::ry + hy, gx = bx - SH::rx + hx;
    Vec<float, V> v;
    const bool in = (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny);
    if (in) {
      const int64_t gp = (int64_t)gy * g.nx + gx;
      v = *reinterpret_cast<const Vec<float, V>*>(X + gp * ldx + c * V);
      if (scale) {
        const float s = scale[gp];
#pragma unroll
        for (int e = 0; e < V; ++e) v.v[e] *= s;
      }
      if (c == 0 && need_guide) sg[hp] = guide[gp];
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) v.v[e] = 0.0f;
      if (c == 0 && need_guide) sg[hp] = 0.0f;
    }
    if (c == 0) sval[hp] = in ? 1.0f : 0.0f;
    sx[c * SH::hp + hp] = v;
  }
}

// ---------------------------------------------------------------- register-blocked 7 x 7
// Each thread owns a vertical strip of RB_P pixels and RB_CS columns: the operand of a halo
// pixel is read from shared memory once per (row, dx) and used by every strip pixel whose
// window contains it, which divides the shared-memory traffic by about 2.7 against one
// pixel per thread.  Tile: 32 pixels wide, RB_P * (256 / (32 * K / RB_CS)) rows.
#define RB_P 4
#define RB_CS 8

template <int K>
struct RBTile {
  static constexpr int cs = (K < RB_CS) ? K : RB_CS;           // columns per thread
  static constexpr int ng = K / cs;                            // column groups
  static constexpr int strips = BF_THREADS / (32 * ng);        // strips per tile column
  static constexpr int tw = 32, th = RB_P * strips;
  static constexpr int rx = 3, ry = 3;
  static constexpr int hw = tw + 2 * rx, hh = th + 2 * ry, hp = hw * hh;
  static constexpr int v = 4;                                  // float4 staging (K % 4 == 0)
};

__device__ __forceinline__ float rb_exp(float gi, float gj, float a_r, float ls) {
  const float dl = gi - gj;
  return exp2f(fmaf(-dl * a_r, dl, ls));
}
