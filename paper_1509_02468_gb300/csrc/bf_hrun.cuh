// Window sums of the 7 x 7 image window for one column of values (k = 1) with STORED
// weights, by horizontal runs: bf_apply at k = 1 in the stored weight modes.
//
// The stored weights are planes wf[f][i] of the 24 forward taps (Eq. 2's w_ij for the
// half-window dy > 0 or dy = 0, dx > 0); the backward tap (dy, dx) of pixel i is the
// forward tap (-dy, -dx) of its neighbour.  A thread owns a run of HRUN_P = 4 consecutive
// pixels of one row, so a forward plane is one 16-byte (FP32) or 8-byte (BF16) vector
// load per run, and a backward plane two aligned vectors from which the run's four
// weights are selected: 69 vector loads per four pixels instead of 192 scalar ones.  The
// values (tile plus radius-3 halo) are staged in shared memory by cp.async with the next
// tile's copies in flight; each window row of the run is read as three 16-byte vectors.
// Tiles whose window reaches the image border (or one column beyond the halo, where the
// vector windows end) use guarded scalar loads instead: neighbours outside the image do
// not exist.  Needs nx % 4 == 0 (rows start on 16-byte boundaries of the planes).
#pragma once

#include "bf_internal.cuh"
#include "bf_strip.cuh"
#include "bf_window_fast.cuh"

#define HRUN_P 4
#define HRUN_TW 64
#define HRUN_TH 16
#define HRUN_THREADS (HRUN_TW * HRUN_TH / HRUN_P)
#define HRUN_HW (HRUN_TW + 2 * STRIP_R)        // 70 staged columns, bx - 3 .. bx + 66
#define HRUN_XS 72                             // staged row stride (16-byte aligned runs)
#define HRUN_HH (HRUN_TH + 2 * STRIP_R)        // 22 staged rows, by - 3 .. by + 18
#define HRUN_HP (HRUN_HH * HRUN_XS)
#define HRUN_NA 2
#define HRUN_SMEM_BYTES (2 * HRUN_NA * HRUN_HP * 4)

// Four consecutive stored weights starting at element e (e % 4 == 0).
template <int WM>
__device__ __forceinline__ float4 hrun_ld4(const void* wf, int64_t e) {
  if (WM == BF_W_STORED_BF16) {
    const uint2 h = __ldg(reinterpret_cast<const uint2*>((const unsigned short*)wf + e));
    return make_float4(__uint_as_float(h.x << 16), __uint_as_float(h.x & 0xffff0000u),
                       __uint_as_float(h.y << 16), __uint_as_float(h.y & 0xffff0000u));
  }
  return __ldg(reinterpret_cast<const float4*>((const float*)wf + e));
}

__device__ __forceinline__ float hrun_pick(const float4& a, const float4& b, int k) {
  switch (k) {
    case 0: return a.x;
    case 1: return a.y;
    case 2: return a.z;
    case 3: return a.w;
    case 4: return b.x;
    case 5: return b.y;
    case 6: return b.z;
    default: return b.w;
  }
}

// Whether the tile at (bx, by) takes the vector form: its window, and one column beyond it
// on each side, lies in the image.
__device__ __forceinline__ bool hrun_interior(int bx, int by, int nx, int ny) {
  return bx - STRIP_R - 1 >= 0 && bx + HRUN_TW + STRIP_R + 1 <= nx && by - STRIP_R >= 0 &&
         by + HRUN_TH + STRIP_R <= ny;
}

// acc[j] = sum_{(dy,dx) != 0} w_ij (v_i - v_j) for the run (x0 + j, y), j < HRUN_P.  sv:
// staged values, row stride HRUN_XS, origin (bx - 3, by - 3); (cx, ry) the run's position
// in the tile.  MASK: guarded scalar loads (border tiles).
template <int WM, bool MASK>
__device__ __forceinline__ void hrun_lsum(const float* sv, int cx, int ry, int x0, int y, int nx, int ny,
                                          const void* wf, int64_t n, float (&vi)[HRUN_P], float (&acc)[HRUN_P]) {
  typedef WinShape<3, 3, false> SH;
  const int64_t i0 = (int64_t)y * nx + x0;
  {
    const float4 c0 = *reinterpret_cast<const float4*>(sv + (ry + STRIP_R) * HRUN_XS + cx);
    const float4 c1 = *reinterpret_cast<const float4*>(sv + (ry + STRIP_R) * HRUN_XS + cx + 4);
    vi[0] = c0.w;
    vi[1] = c1.x;
    vi[2] = c1.y;
    vi[3] = c1.z;
  }
#pragma unroll
  for (int j = 0; j < HRUN_P; ++j) acc[j] = 0.0f;
#pragma unroll
  for (int dy = -STRIP_R; dy <= STRIP_R; ++dy) {
    float vr[12];
    {
      const float* row = sv + (ry + STRIP_R + dy) * HRUN_XS + cx;
      const float4 a = *reinterpret_cast<const float4*>(row);
      const float4 b = *reinterpret_cast<const float4*>(row + 4);
      const float4 c = *reinterpret_cast<const float4*>(row + 8);
      vr[0] = a.x; vr[1] = a.y; vr[2] = a.z; vr[3] = a.w;
      vr[4] = b.x; vr[5] = b.y; vr[6] = b.z; vr[7] = b.w;
      vr[8] = c.x; vr[9] = c.y; vr[10] = c.z; vr[11] = c.w;
    }
    const bool yin = !MASK || ((unsigned)y < (unsigned)ny && (unsigned)(y + dy) < (unsigned)ny);
#pragma unroll
    for (int dx = -STRIP_R; dx <= STRIP_R; ++dx) {
      if (dx == 0 && dy == 0) continue;
      float w[HRUN_P];
      const bool fwd = SH::forward(dy, dx);
      const int f = fwd ? SH::fwd_index(dy, dx) : SH::fwd_index(-dy, -dx);
      if (MASK) {
#pragma unroll
        for (int j = 0; j < HRUN_P; ++j) {
          const bool in = yin && (unsigned)(x0 + j) < (unsigned)nx && (unsigned)(x0 + j + dx) < (unsigned)nx;
          const int64_t e = (int64_t)f * n + i0 + j + (fwd ? 0 : (int64_t)dy * nx + dx);
          w[j] = in ? strip_ld_w<WM>(wf, e) : 0.0f;
        }
      } else if (fwd) {
        const float4 a = hrun_ld4<WM>(wf, (int64_t)f * n + i0);
        w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
      } else {
        const int64_t e0 = (int64_t)f * n + i0 + (int64_t)dy * nx;     // 4-aligned
        if (dx == 0) {
          const float4 a = hrun_ld4<WM>(wf, e0);
          w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
        } else {
          const int64_t base = dx < 0 ? e0 - 4 : e0;
          const float4 a = hrun_ld4<WM>(wf, base);
          const float4 b = hrun_ld4<WM>(wf, base + 4);
#pragma unroll
          for (int j = 0; j < HRUN_P; ++j) w[j] = hrun_pick(a, b, (dx < 0 ? 4 : 0) + dx + j);
        }
      }
#pragma unroll
      for (int j = 0; j < HRUN_P; ++j) acc[j] = fmaf(w[j], vi[j] - vr[j + STRIP_R + dx], acc[j]);
    }
  }
}

// Issue the cp.async copies of tile (bx, by): array a of the stage receives src[a][gp]
// (0 outside the image), src[a] NULL: not staged.
template <int NA>
__device__ __forceinline__ void hrun_issue(int bx, int by, int nx, int ny, const float* const (&src)[NA], float* stage) {
  const unsigned base = (unsigned)__cvta_generic_to_shared(stage);
  for (int hp = threadIdx.x; hp < HRUN_HH * HRUN_HW; hp += HRUN_THREADS) {
    const int hy = hp / HRUN_HW, hx = hp - hy * HRUN_HW;
    const int gy = by - STRIP_R + hy, gx = bx - STRIP_R + hx;
    const bool in = (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny;
    const int64_t gp = in ? (int64_t)gy * nx + gx : 0;
#pragma unroll
    for (int a = 0; a < NA; ++a)
      if (src[a]) strip_cp4(base + 4u * (unsigned)(a * HRUN_HP + hy * HRUN_XS + hx), src[a] + gp, in);
  }
}

// Walk this CTA's 64 x 16 tiles with the next tile's copies in flight.  combine(stage)
// may rewrite array 0 (the values v) from array 1 (HRUN_HP floats apart);
// epi(bx, by, cx, ry, vi, acc) consumes the run's sums.  Dynamic smem: HRUN_SMEM_BYTES.
template <int WM, int NA, class Combine, class Epi>
__device__ __forceinline__ void hrun_run(int nx, int ny, const void* wf, int64_t n, const float* const (&src)[NA],
                                         Combine combine, Epi epi) {
  extern __shared__ __align__(16) float hrun_smem[];
  const int ntx = (nx + HRUN_TW - 1) / HRUN_TW, ntiles = ntx * ((ny + HRUN_TH - 1) / HRUN_TH);
  const int cx = 4 * (threadIdx.x & 15), ry = threadIdx.x >> 4;
  int t = blockIdx.x;
  if (t < ntiles) hrun_issue<NA>((t % ntx) * HRUN_TW, (t / ntx) * HRUN_TH, nx, ny, src, hrun_smem);
  strip_commit();
  for (int b = 0; t < ntiles; t += gridDim.x, b ^= 1) {
    const int tn = t + gridDim.x;
    float* cur = hrun_smem + b * HRUN_NA * HRUN_HP;
    if (tn < ntiles)
      hrun_issue<NA>((tn % ntx) * HRUN_TW, (tn / ntx) * HRUN_TH, nx, ny, src,
                     hrun_smem + (b ^ 1) * HRUN_NA * HRUN_HP);
    strip_commit();
    strip_wait_prev();
    __syncthreads();
    combine(cur);
    __syncthreads();
    const int bx = (t % ntx) * HRUN_TW, by = (t / ntx) * HRUN_TH;
    float vi[HRUN_P], acc[HRUN_P];
    if (hrun_interior(bx, by, nx, ny))
      hrun_lsum<WM, false>(cur, cx, ry, bx + cx, by + ry, nx, ny, wf, n, vi, acc);
    else
      hrun_lsum<WM, true>(cur, cx, ry, bx + cx, by + ry, nx, ny, wf, n, vi, acc);
    epi(bx, by, cx, ry, vi, acc);
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}
