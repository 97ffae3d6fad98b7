// Internal definitions shared by the libbf translation units: the graph object, launch
// geometry, error plumbing, and the device building blocks of the matrix-free operator.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include <string>

#include "../../include/bf.h"

// ------------------------------------------------------------------ limits
#define BF_MAX_R2D 7          // 2D window radius limit (15 x 15 box)
#define BF_MAX_R1D 32         // 1D window radius limit
#define BF_MAX_BOX 225        // (2 * 7 + 1)^2 >= 2 * 32 + 1
#define BF_THREADS 256        // threads per tile CTA: one output pixel each
#define BF_TW2 32             // 2D tile width  (pixels)
#define BF_TH2 8              // 2D tile height (pixels)
#define BF_TW1 256            // 1D tile length

// ------------------------------------------------------------------ errors
void bf_set_error(const std::string& msg);
int bf_fail(int code, const std::string& msg);
int bf_cuda_fail(cudaError_t e, const char* what);

// Allow kernel `fn` `bytes` of dynamic shared memory on the current device.  The attribute
// belongs to the device's context: it is set per (device, kernel), under a lock, again
// whenever a larger size is asked for.
int bf_smem_attr(const void* fn, int bytes, const char* what);

// Every kernel launch of the library goes through BF_LAUNCH, which counts it (the count
// is exported by bf_launch_count for diagnostics and benchmarks).
void bf_count_launches(int n);
#define BF_LAUNCH(...)          \
  do {                          \
    __VA_ARGS__;                \
    bf_count_launches(1);       \
  } while (0)

// Programmatic dependent launch for the kernels of the block-LOBPCG iteration chain: a
// kernel launched by BF_LAUNCH_PDL may be scheduled while its predecessor in the stream
// still runs, once every CTA of the predecessor has called bf_pdl_enter (or exited); it
// must itself call bf_pdl_enter before touching anything the predecessor writes, since
// the wait in it returns only when the predecessor grid has completed and its memory
// operations are visible.  Without the launch attribute the wait returns at once, so a
// kernel that calls bf_pdl_enter can be launched either way.
__device__ __forceinline__ void bf_pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t bf_launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                 Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}
// a launch error is left for the caller's cudaGetLastError, as with <<< >>>
#define BF_LAUNCH_PDL(kern, grid, block, smem, stream, ...)                   \
  do {                                                                        \
    (void)bf_launch_pdl(kern, grid, block, smem, stream, __VA_ARGS__);        \
    bf_count_launches(1);                                                     \
  } while (0)

#define BF_CUDA(call)                                               \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return bf_cuda_fail(e_, #call);          \
  } while (0)

// ------------------------------------------------------------------ geometry
// Window description handed to every operator kernel by value.  `ls` holds, per cell of
// the (2 ry + 1) x (2 rx + 1) box (row-major by dy, dx), the logarithm of the spatial
// factor of Eq. 2: base 2 in the float path (used with exp2), base e in the double path.
// `fmap` gives, per cell, the index of its forward tap in the stored weights (-1 for the
// centre and for cells outside a cross window); a backward cell is looked up through its
// mirror image.
template <typename T>
struct Geom {
  int nx, ny;        // image extent (ny = 1 for signals)
  int rx, ry;        // window radii (ry = 0 for signals)
  int cross;         // BF_WINDOW_CROSS
  int nfwd;          // number of forward taps
  T a_r;             // range coefficient: log2(e) / (2 sigma_r^2) (float) or 1/(2 sigma_r^2)
  T ls[BF_MAX_BOX];
  short fmap[BF_MAX_BOX];
};

struct bf_graph {
  bf_params p;
  int64_t n;
  int nx, ny, rx, ry;
  int ntaps, nfwd;
  int device;
  size_t esize;          // sizeof(element)
  void* guide;           // [n]
  void* d;               // [n] degree, w_ii = 1 included
  void* dinv;            // [n] 1 / d
  void* dis;             // [n] d^-1/2
  void* dls;             // [n] (diag L)^-1/2, 0 where diag L <= 1e-30
  void* wf;              // [nfwd][n] forward weights (stored modes) or NULL
  Geom<float> gf;
  Geom<double> gd;
  void* ws[3];           // grow-only workspaces, one per filter family (BF_WS_*)
  size_t ws_bytes[3];
  int* flag;             // [1] non-finite guide flag of the weights kernel
  int kind;              // BF_KIND_*
  double eps;            // guided: epsilon of Algorithm 1
  void* gmu;             // guided: [n] mean of the guide over each window
  void* givar;           // guided: [n] 1 / (variance of the guide over each window + eps)
};

#define BF_KIND_BILATERAL 0   // Eq. 2 weights (bf_weights)
#define BF_KIND_GUIDED    1   // the guided filter's matrix, Eq. 6 (bf_guided_graph)
#define BF_GF_MAX_R2D 8
#define BF_GF_MAX_R1D 32

// Guided graphs (bf_guided.cu): Y = op X for ops W, L, D^-1 W, D, NSYM (dots: x^T y per
// column, zeroed by the caller; guide NULL: the graph's own), and the window statistics
// for a new guide (a non-finite value sets g->flag).
template <typename T>
int bf_guided_apply(const bf_graph* g, int op, const T* X, int64_t ldx, int k, T* Y, int64_t ldy,
                    double* dots, const T* guide, cudaStream_t s);
int bf_guided_prep(bf_graph* g, const void* guide, cudaStream_t s);

// Workspace slots: CG and LOBPCG keep their own, so one call of each may run at the same
// time on different streams.
enum { BF_WS_CG = 0, BF_WS_LOB = 1, BF_WS_SIMPLE = 2 };

// Grow workspace `slot` of the graph to at least `bytes` (synchronises the device when it
// grows).
int bf_ws_reserve(bf_graph* g, int slot, size_t bytes);

template <typename T> inline const Geom<T>& geom_of(const bf_graph* g);
template <> inline const Geom<float>& geom_of<float>(const bf_graph* g) { return g->gf; }
template <> inline const Geom<double>& geom_of<double>(const bf_graph* g) { return g->gd; }

inline dim3 tile_grid(const bf_graph* g) {
  if (g->ny == 1 && g->p.ndim == 1) return dim3((unsigned)((g->nx + BF_TW1 - 1) / BF_TW1), 1, 1);
  return dim3((unsigned)((g->nx + BF_TW2 - 1) / BF_TW2), (unsigned)((g->ny + BF_TH2 - 1) / BF_TH2), 1);
}

// Vector width (elements) used for a chunk of K columns of type T.
template <typename T, int K>
struct VecW {
  static constexpr int v16 = 16 / (int)sizeof(T);
  static constexpr int value = (K % v16 == 0) ? v16 : ((K % 2 == 0) ? 2 : 1);
};

template <typename T, int V> struct alignas(sizeof(T) * V) Vec { T v[V]; };

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ float bf_exp_w(float arg) { return exp2f(arg); }
__device__ __forceinline__ double bf_exp_w(double arg) { return exp(arg); }

__device__ __forceinline__ float ld_weight(const void* wf, int64_t idx, int mode) {
  if (mode == BF_W_STORED_BF16) return __bfloat162float(((const __nv_bfloat16*)wf)[idx]);
  return ((const float*)wf)[idx];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Tile bookkeeping shared by the operator kernels: a CTA owns TW x TH output pixels and
// stages TW + 2 rx by TH + 2 ry input pixels (the halo) in shared memory.
struct Tile {
  int tw, th, hw, hh, hp;      // tile and halo extents, halo pixel count
  int bx, by;                  // tile origin
  int lx, ly;                  // this thread's pixel within the tile
  int x, y;                    // this thread's pixel in the image
  bool active;                 // inside the image
  int hp0;                     // this thread's pixel index within the halo tile
};

template <typename T>
__device__ __forceinline__ Tile make_tile(const Geom<T>& g) {
  Tile t;
  const bool one_d = (g.ny == 1 && g.ry == 0);
  t.tw = one_d ? BF_TW1 : BF_TW2;
  t.th = one_d ? 1 : BF_TH2;
  t.hw = t.tw + 2 * g.rx;
  t.hh = t.th + 2 * g.ry;
  t.hp = t.hw * t.hh;
  t.bx = blockIdx.x * t.tw;
  t.by = blockIdx.y * t.th;
  t.lx = threadIdx.x % t.tw;
  t.ly = threadIdx.x / t.tw;
  t.x = t.bx + t.lx;
  t.y = t.by + t.ly;
  t.active = (t.x < g.nx) && (t.y < g.ny);
  t.hp0 = (t.ly + g.ry) * t.hw + (t.lx + g.rx);
  return t;
}

// Weighted window sum for this thread's pixel over a K-column tile held in shared memory
// as [K / V][hp] vectors.  DIFF: acc += w_ij (x_i - x_j)  (L-type operators, no
// cancellation for smooth x);  otherwise acc += w_ij x_j.  wsum = sum_{j != i} w_ij.
// Weights come from the guide tile (mode BF_W_ONTHEFLY, Eq. 2) or the stored forward
// weights.  Neighbours outside the image are skipped (they do not exist).
template <typename T, int K, bool DIFF>
__device__ __forceinline__ void window_sum(const Geom<T>& g, const Tile& t, const T* sg,
                                           const Vec<T, VecW<T, K>::value>* sx,
                                           const void* wf, int wmode, int64_t n,
                                           const T (&xi)[K], T (&acc)[K], T& wsum) {
  constexpr int V = VecW<T, K>::value;
  constexpr int NC = K / V;
  const int bw = 2 * g.rx + 1;
  const T gi = (wmode == BF_W_ONTHEFLY) ? sg[t.hp0] : T(0);
  const int64_t i = (int64_t)t.y * g.nx + t.x;
  for (int dy = -g.ry; dy <= g.ry; ++dy) {
    const int yy = t.y + dy;
    if (yy < 0 || yy >= g.ny) continue;
    for (int dx = -g.rx; dx <= g.rx; ++dx) {
      if (dx == 0 && dy == 0) continue;
      if (g.cross && dx != 0 && dy != 0) continue;
      const int xx = t.x + dx;
      if (xx < 0 || xx >= g.nx) continue;
      const int cell = (dy + g.ry) * bw + (dx + g.rx);
      const int hp = t.hp0 + dy * t.hw + dx;
      T w;
      if (wmode == BF_W_ONTHEFLY) {
        const T dl = gi - sg[hp];
        w = bf_exp_w(fma(-dl * g.a_r, dl, g.ls[cell]));
      } else {
        const int f = g.fmap[cell];
        if (f >= 0) {
          w = (T)ld_weight(wf, (int64_t)f * n + i, wmode);
        } else {
          const int mcell = (g.ry - dy) * bw + (g.rx - dx);
          const int64_t j = i + (int64_t)dy * g.nx + dx;
          w = (T)ld_weight(wf, (int64_t)g.fmap[mcell] * n + j, wmode);
        }
      }
      wsum += w;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const Vec<T, V> xj = sx[c * t.hp + hp];
#pragma unroll
        for (int e = 0; e < V; ++e) {
          if (DIFF) acc[c * V + e] = fma(w, xi[c * V + e] - xj.v[e], acc[c * V + e]);
          else      acc[c * V + e] = fma(w, xj.v[e], acc[c * V + e]);
        }
      }
    }
  }
}

// Block-wide sum of NV values per thread: warp sums in the element type T, the per-warp
// results added in FP64.  The result is valid in thread 0.  `red` must hold
// NV * (BF_THREADS / 32) doubles.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(const T (&v)[NV], double* red, double (&out)[NV]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T w[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) w[j] = warp_sum(v[j]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) red[j * (BF_THREADS / 32) + wid] = (double)w[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = 0.0;
      for (int q = 0; q < BF_THREADS / 32; ++q) s += red[j * (BF_THREADS / 32) + q];
      out[j] = s;
    }
  }
}

// Grid-wide deterministic FP64 reduction ("last block" pattern).  Every block calls it
// with its block sums (valid in thread 0).  Returns true in thread 0 of the last block to
// arrive, whose `tot` then holds the sums over all blocks in block order.
template <int NV>
__device__ __forceinline__ bool grid_sum_last(const double (&blk)[NV], double* partials,
                                              unsigned int* counter, double (&tot)[NV],
                                              int* is_last_sh) {
  const unsigned nb = gridDim.x * gridDim.y;
  const unsigned b = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) partials[(size_t)b * NV + j] = blk[j];
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    *is_last_sh = (prev == nb - 1);
  }
  __syncthreads();
  if (!*is_last_sh) return false;
  __threadfence();
  // the last block sums the partials: thread t takes blocks t, t + 256, ... in order
  double v[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = 0.0;
  for (unsigned q = threadIdx.x; q < nb; q += BF_THREADS) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] += ((volatile double*)partials)[(size_t)q * NV + j];
  }
  __shared__ double red2[NV * (BF_THREADS / 32)];
  block_sum<NV, double>(v, red2, tot);
  if (threadIdx.x == 0) *counter = 0u;
  return threadIdx.x == 0;
}
