// Strip-blocked window sums of the 7 x 7 image window for one column of values (k = 1):
// the inner loop of the CG filter (Algorithm 2, q = L p) and of bf_apply at k = 1.
//
// A CTA owns a 32 x 32 tile of pixels; thread (lx, ly) owns the vertical strip of
// STRIP_P pixels in column lx, rows ly * STRIP_P .. ly * STRIP_P + STRIP_P - 1.  The
// tile plus its radius-3 halo (38 x 38) of the values v and of the guide g is staged in
// shared memory.  For each of the 7 window columns dx the thread reads the STRIP_P + 6
// staged values of that column once and applies them to all STRIP_P pixels of its strip:
// 35 shared-memory loads per pixel instead of 96 for one pixel per thread.
//
// L is applied in difference form, acc_i = sum_j w_ij (v_i - v_j) (no D - W cancellation
// on smooth v).  Weights (Eq. 2) are either recomputed from the staged guide,
//   w_ij = 2^(ls(dy, dx) - a_r (g_i - g_j)^2)   (ls, a_r in base 2: Geom<float>),
// or read from the stored forward half-window planes wf[f][i] (FP32 or BF16), the
// backward tap (dy, dx) of pixel i being the forward tap (-dy, -dx) of its neighbour.
// Tiles whose halo crosses the image border (MASK) test every neighbour's coordinates:
// neighbours outside the image do not exist (their weight is 0, and a stored backward
// weight of an outside neighbour is never read).
#pragma once

#include "bf_internal.cuh"
#include "bf_window_fast.cuh"

#define STRIP_P 4
#define STRIP_TW 32
#define STRIP_TH 32
#define STRIP_R 3
#define STRIP_HW (STRIP_TW + 2 * STRIP_R)
#define STRIP_HH (STRIP_TH + 2 * STRIP_R)
#define STRIP_HP (STRIP_HW * STRIP_HH)
#define STRIP_THREADS (STRIP_TW * STRIP_TH / STRIP_P)

__device__ __forceinline__ float strip_ex2(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

// Stored weight idx of mode WM (BF_W_STORED_F32 or BF_W_STORED_BF16).
template <int WM>
__device__ __forceinline__ float strip_ld_w(const void* wf, int64_t idx) {
  if (WM == BF_W_STORED_BF16) return __uint_as_float((unsigned)__ldg((const unsigned short*)wf + idx) << 16);
  return __ldg((const float*)wf + idx);
}

// Number of 32 x 32 tiles of an image.
__host__ __device__ inline int strip_tiles_x(int nx) { return (nx + STRIP_TW - 1) / STRIP_TW; }
__host__ __device__ inline int strip_tiles_y(int ny) { return (ny + STRIP_TH - 1) / STRIP_TH; }

// Whether tile (bx, by) (pixel origin) has neighbours outside the image.
__device__ __forceinline__ bool strip_border(int bx, int by, int nx, int ny) {
  return !(bx - STRIP_R >= 0 && bx + STRIP_TW + STRIP_R <= nx && by - STRIP_R >= 0 &&
           by + STRIP_TH + STRIP_R <= ny);
}

// acc[j] = sum_{(dy,dx) != 0} w (v_i - v_j) for the strip's pixels i = (x, y0 + j).
// sv, sg: staged values and guide ([STRIP_HH][STRIP_HW], halo origin (bx - 3, by - 3)).
// vi[j] returns the strip's own values.  i0 = y0 * nx + x.  In the stored modes sg is
// unused; pixels of the strip outside the image produce garbage that the caller drops.
// WM is the weight mode (BF_W_*).
template <int WM, bool MASK>
__device__ __forceinline__ void strip_lsum(const Geom<float>& g, const float* sv, const float* sg, int lx,
                                           int ly0, int x, int y0, int64_t i0, const void* wf,
                                           int64_t n, float (&vi)[STRIP_P], float (&acc)[STRIP_P]) {
  typedef WinShape<3, 3, false> SH;
  constexpr bool STORED = (WM != BF_W_ONTHEFLY);
  float gi[STRIP_P];
#pragma unroll
  for (int j = 0; j < STRIP_P; ++j) {
    const int hp = (ly0 + j + STRIP_R) * STRIP_HW + lx + STRIP_R;
    vi[j] = sv[hp];
    gi[j] = STORED ? 0.0f : sg[hp];
    acc[j] = 0.0f;
  }
  const int nx = g.nx, ny = g.ny;
#pragma unroll
  for (int dx = -STRIP_R; dx <= STRIP_R; ++dx) {
    float vc[STRIP_P + 2 * STRIP_R], gc[STRIP_P + 2 * STRIP_R];
#pragma unroll
    for (int m = 0; m < STRIP_P + 2 * STRIP_R; ++m) {
      const int hp = (ly0 + m) * STRIP_HW + lx + STRIP_R + dx;
      vc[m] = sv[hp];
      if (!STORED) gc[m] = sg[hp];
    }
    // (MASK) the pixel itself and its neighbour must both lie in the image
    const bool xin = !MASK || ((unsigned)x < (unsigned)nx && (unsigned)(x + dx) < (unsigned)nx);
#pragma unroll
    for (int j = 0; j < STRIP_P; ++j) {
      const bool yself = !MASK || (unsigned)(y0 + j) < (unsigned)ny;
#pragma unroll
      for (int dy = -STRIP_R; dy <= STRIP_R; ++dy) {
        if (dx == 0 && dy == 0) continue;
        const int m = j + STRIP_R + dy;
        const bool in = !MASK || (xin && yself && (unsigned)(y0 + j + dy) < (unsigned)ny);
        float w;
        if (STORED) {
          const int64_t i = i0 + (int64_t)j * nx;
          if (SH::forward(dy, dx)) {
            w = in ? strip_ld_w<WM>(wf, (int64_t)SH::fwd_index(dy, dx) * n + i) : 0.0f;
          } else {
            w = in ? strip_ld_w<WM>(wf, (int64_t)SH::fwd_index(-dy, -dx) * n + i + (int64_t)dy * nx + dx)
                   : 0.0f;
          }
        } else {
          const float dl = gi[j] - gc[m];
          w = strip_ex2(fmaf(-dl * g.a_r, dl, g.ls[(dy + STRIP_R) * 7 + dx + STRIP_R]));
          if (MASK && !in) w = 0.0f;
        }
        acc[j] = fmaf(w, vi[j] - vc[m], acc[j]);
      }
    }
  }
}

// ---- asynchronous double-buffered staging -----------------------------------------------
// A stage holds up to STRIP_NA arrays of the tile plus halo ([STRIP_NA][STRIP_HP] floats),
// copied by cp.async in 4-byte pieces (zero-filled outside the image), so that the next
// tile's copies are in flight while the current tile is computed.
#define STRIP_NA 3
#define STRIP_STAGE_FLOATS (STRIP_NA * STRIP_HP)
#define STRIP_SMEM_BYTES (2 * STRIP_STAGE_FLOATS * 4)

__device__ __forceinline__ void strip_cp4(unsigned dst, const float* src, bool in) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(in ? 4 : 0) : "memory");
}
__device__ __forceinline__ void strip_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void strip_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Issue the copies of the tile at (bx, by): array a of the stage receives src[a][gp * ld[a]]
// for every halo pixel gp (0 outside the image).
template <int NA>
__device__ __forceinline__ void strip_issue(int bx, int by, int nx, int ny, const float* const (&src)[NA],
                                            const int64_t (&ld)[NA], float* stage) {
  const unsigned base = (unsigned)__cvta_generic_to_shared(stage);
#pragma unroll 2
  for (int hp = threadIdx.x; hp < STRIP_HP; hp += STRIP_THREADS) {
    const int hy = hp / STRIP_HW, hx = hp - hy * STRIP_HW;
    const int gy = by - STRIP_R + hy, gx = bx - STRIP_R + hx;
    const bool in = (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny;
    const int64_t gp = in ? (int64_t)gy * nx + gx : 0;
#pragma unroll
    for (int a = 0; a < NA; ++a)
      if (src[a]) strip_cp4(base + 4u * (unsigned)(a * STRIP_HP + hp), src[a] + gp * ld[a], in);
  }
}

// Window sum of the tile at (bx, by), border tiles through the masked form.
template <int WM>
__device__ __forceinline__ void strip_tile_lsum(const Geom<float>& g, const float* sv, const float* sg, int bx,
                                                int by, int lx, int ly0, const void* wf, int64_t n,
                                                float (&vi)[STRIP_P], float (&acc)[STRIP_P]) {
  const int x = bx + lx, y0 = by + ly0;
  const int64_t i0 = (int64_t)y0 * g.nx + x;
  if (strip_border(bx, by, g.nx, g.ny))
    strip_lsum<WM, true>(g, sv, sg, lx, ly0, x, y0, i0, wf, n, vi, acc);
  else
    strip_lsum<WM, false>(g, sv, sg, lx, ly0, x, y0, i0, wf, n, vi, acc);
}

// Walk this CTA's tiles (grid-stride over the 32 x 32 tiles of the image) with the next
// tile's copies in flight: src[a] (NULL: not staged) with element stride ld[a]; array
// `garr` of the stage is the guide (weights on the fly).  combine(stage) runs between the
// arrival of a tile and its window sums (it may rewrite array 0, the values v, from the
// other arrays); epi(bx, by, lx, ly0, vi, acc) consumes the sums of the thread's strip.
// Dynamic shared memory: STRIP_SMEM_BYTES.
template <int WM, int NA, bool COMBINE, class Combine, class Epi>
__device__ __forceinline__ void strip_run(const Geom<float>& g, const void* wf, int64_t n,
                                          const float* const (&src)[NA], const int64_t (&ld)[NA], int garr,
                                          Combine combine, Epi epi) {
  extern __shared__ __align__(16) float strip_smem[];
  const int nx = g.nx, ny = g.ny;
  const int ntx = strip_tiles_x(nx), ntiles = ntx * strip_tiles_y(ny);
  const int lx = threadIdx.x & 31, ly0 = (threadIdx.x >> 5) * STRIP_P;
  int t = blockIdx.x;
  if (t < ntiles) strip_issue<NA>((t % ntx) * STRIP_TW, (t / ntx) * STRIP_TH, nx, ny, src, ld, strip_smem);
  strip_commit();
  for (int b = 0; t < ntiles; t += gridDim.x, b ^= 1) {
    const int tn = t + gridDim.x;
    float* cur = strip_smem + b * STRIP_STAGE_FLOATS;
    if (tn < ntiles)
      strip_issue<NA>((tn % ntx) * STRIP_TW, (tn / ntx) * STRIP_TH, nx, ny, src, ld,
                      strip_smem + (b ^ 1) * STRIP_STAGE_FLOATS);
    strip_commit();
    strip_wait_prev();                      // this tile's copies have landed (own thread)
    __syncthreads();                        // ... and every other thread's
    if (COMBINE) {
      combine(cur);
      __syncthreads();
    }
    const int bx = (t % ntx) * STRIP_TW, by = (t / ntx) * STRIP_TH;
    float vi[STRIP_P], acc[STRIP_P];
    strip_tile_lsum<WM>(g, cur, cur + garr * STRIP_HP, bx, by, lx, ly0, wf, n, vi, acc);
    epi(bx, by, lx, ly0, vi, acc);
    __syncthreads();                        // the stage is refilled in the next iteration
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}
