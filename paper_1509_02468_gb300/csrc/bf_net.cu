// The learned preconditioner T of the flexible CG and LOBPCG filters (the preconditioner of
// Algorithms 2 and 3, left open by the paper; Section 5's flexible beta admits a variable,
// nonlinear T): a three-layer 3 x 3 conv net on the image-shaped residual r,
//
//   C  = [ (D^-1 r) / rho,  g,  1 / d ],  rho = rms(D^-1 r)
//   A1 = conv(C, W1) (16 ch),  A2 = conv(relu(A1), W2) (16 ch),  O = conv(relu(A2), W3)
//   T(r) = rho O
//
// (cross-correlations without bias, zero outside the image).  Weights are kept in FP32
// (the trained master copy) and used rounded to BF16; every product is accumulated in
// FP32.  Training pairs (r, z) solve (L + sigma I) z = r; the loss of a pair is
// ||T(r) - z||^2 / ||z||^2, its gradient is accumulated by bf_net_accumulate and applied
// by bf_net_adam (Adam, Kingma and Ba).
//
// Kernels work on 32 x 8 pixel tiles with a one-pixel halo staged channel-major in shared
// memory; activations are stored pixel-major [n][16].
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "bf_internal.cuh"

#define NET_CH 16
#define NET_CIN 3
#define NET_TW 32
#define NET_TH 8
#define NET_HW (NET_TW + 2)
#define NET_HH (NET_TH + 2)
#define NET_HP (NET_HW * NET_HH)
#define NET_W1 0
#define NET_W2 (NET_CH * NET_CIN * 9)
#define NET_W3 (NET_W2 + NET_CH * NET_CH * 9)
#define NET_NW (NET_W3 + NET_CH * 9)
#define NET_COLS 4                         // columns per pass of bf_net_apply

struct bf_net {
  int device;
  float* w;       // [NET_NW] FP32 master weights
  float* wq;      // [NET_NW] weights rounded to BF16 (as FP32)
  float* m;       // Adam moments
  float* v;
  float* grad;    // [NET_NW] accumulated gradient
  double* loss;   // [1] accumulated loss
  int t;          // Adam steps taken
  void* ws;       // activations, partial sums
  size_t ws_bytes;
};

namespace {

enum { IN_NET = 0, IN_RELU = 1, IN_PLAIN = 2 };
enum { OUT_ACT = 0, OUT_PRECOND = 1, OUT_MASKED = 2 };

struct NetArgs {
  int nx, ny;
  int64_t n;
  const float* r;        // IN_NET: residual columns, r[i * ldr + col]
  int64_t ldr;
  const float* guide;
  const float* d;
  const float* rho;      // [cols]
  const float* in;       // [cols][n][cin] activations
  float* out;            // [cols][n][cout]
  const float* mask;     // OUT_MASKED: [cols][n][cout] pre-activations
  float* z;              // OUT_PRECOND: z[i * ldz + col]
  int64_t ldz;
  const float* w;        // layer weights as stored: [cout_l][cin_l][9]
  int transpose;         // use the adjoint (flipped, transposed) weights
  const int* stop;       // optional solver status: nonzero = stopped, skip the work
};

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Stage the input tile (with halo) channel-major: s[c * NET_HP + hp].
template <int CIN, int IN>
__device__ __forceinline__ void net_stage(const NetArgs& a, int col, int bx, int by, float* s) {
  for (int hp = threadIdx.x; hp < NET_HP; hp += NET_TW * NET_TH) {
    const int hy = hp / NET_HW, hx = hp - hy * NET_HW;
    const int gy = by - 1 + hy, gx = bx - 1 + hx;
    const bool inside = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;
    const int64_t i = (int64_t)gy * a.nx + gx;
    if (IN == IN_NET) {
      float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
      if (inside) {
        const float rh = a.rho[col];
        const float di = a.d[i];
        c0 = rh > 0.0f ? a.r[i * a.ldr + col] / (di * rh) : 0.0f;
        c1 = a.guide[i];
        c2 = 1.0f / di;
      }
      s[0 * NET_HP + hp] = c0;
      s[1 * NET_HP + hp] = c1;
      s[2 * NET_HP + hp] = c2;
    } else {
      const float* src = a.in + ((int64_t)col * a.n + i) * CIN;
#pragma unroll
      for (int c4 = 0; c4 < CIN; c4 += 4) {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (inside) {
          if (CIN % 4 == 0) {
            v = *reinterpret_cast<const float4*>(src + c4);
          } else {
            v.x = src[c4];
            if (c4 + 1 < CIN) v.y = src[c4 + 1];
            if (c4 + 2 < CIN) v.z = src[c4 + 2];
            if (c4 + 3 < CIN) v.w = src[c4 + 3];
          }
          if (IN == IN_RELU) {
            v.x = fmaxf(v.x, 0.0f);
            v.y = fmaxf(v.y, 0.0f);
            v.z = fmaxf(v.z, 0.0f);
            v.w = fmaxf(v.w, 0.0f);
          }
        }
        s[(c4 + 0) * NET_HP + hp] = v.x;
        if (c4 + 1 < CIN) s[(c4 + 1) * NET_HP + hp] = v.y;
        if (c4 + 2 < CIN) s[(c4 + 2) * NET_HP + hp] = v.z;
        if (c4 + 3 < CIN) s[(c4 + 3) * NET_HP + hp] = v.w;
      }
    }
  }
}

// One 3 x 3 conv layer (CIN -> COUT) on a tile; blockIdx.z is the column.
template <int CIN, int COUT, int IN, int OUT>
__global__ void __launch_bounds__(NET_TW * NET_TH) k_net_conv(const NetArgs a) {
  constexpr int COUTP = (COUT + 3) & ~3;
  if (a.stop && *a.stop != 0) return;
  __shared__ __align__(16) float sx[CIN * NET_HP];
  __shared__ __align__(16) float sw[CIN * 9 * COUTP];       // [c][tap][o]
  const int col = blockIdx.z;
  const int bx = blockIdx.x * NET_TW, by = blockIdx.y * NET_TH;
  for (int e = threadIdx.x; e < CIN * 9 * COUTP; e += NET_TW * NET_TH) {
    const int o = e % COUTP, ct = e / COUTP, c = ct / 9, t = ct - c * 9;
    float wv = 0.0f;
    if (o < COUT) wv = a.transpose ? a.w[(c * COUT + o) * 9 + (8 - t)] : a.w[(o * CIN + c) * 9 + t];
    sw[e] = wv;
  }
  net_stage<CIN, IN>(a, col, bx, by, sx);
  __syncthreads();
  const int lx = threadIdx.x % NET_TW, ly = threadIdx.x / NET_TW;
  const int x = bx + lx, y = by + ly;
  if (x >= a.nx || y >= a.ny) return;
  float acc[COUTP];
#pragma unroll
  for (int o = 0; o < COUTP; ++o) acc[o] = 0.0f;
  for (int c = 0; c < CIN; ++c) {
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int ty = t / 3, tx = t - 3 * (t / 3);
      const float xv = sx[c * NET_HP + (ly + ty) * NET_HW + lx + tx];
      const float4* w4 = reinterpret_cast<const float4*>(sw + (c * 9 + t) * COUTP);
#pragma unroll
      for (int o4 = 0; o4 < COUTP / 4; ++o4) {
        const float4 wv = w4[o4];
        acc[4 * o4 + 0] = fmaf(wv.x, xv, acc[4 * o4 + 0]);
        acc[4 * o4 + 1] = fmaf(wv.y, xv, acc[4 * o4 + 1]);
        acc[4 * o4 + 2] = fmaf(wv.z, xv, acc[4 * o4 + 2]);
        acc[4 * o4 + 3] = fmaf(wv.w, xv, acc[4 * o4 + 3]);
      }
    }
  }
  const int64_t i = (int64_t)y * a.nx + x;
  if (OUT == OUT_PRECOND) {
    a.z[i * a.ldz + col] = a.rho[col] * acc[0];
  } else {
    float* dst = a.out + ((int64_t)col * a.n + i) * COUT;
    const float* mk = (OUT == OUT_MASKED) ? a.mask + ((int64_t)col * a.n + i) * COUT : nullptr;
    if (COUT % 4 == 0) {
#pragma unroll
      for (int o4 = 0; o4 < COUT / 4; ++o4) {
        float4 v = make_float4(acc[4 * o4], acc[4 * o4 + 1], acc[4 * o4 + 2], acc[4 * o4 + 3]);
        if (OUT == OUT_MASKED) {
          const float4 m = reinterpret_cast<const float4*>(mk)[o4];
          v.x = m.x > 0.0f ? v.x : 0.0f;
          v.y = m.y > 0.0f ? v.y : 0.0f;
          v.z = m.z > 0.0f ? v.z : 0.0f;
          v.w = m.w > 0.0f ? v.w : 0.0f;
        }
        reinterpret_cast<float4*>(dst)[o4] = v;
      }
    } else {
#pragma unroll
      for (int o = 0; o < COUT; ++o) dst[o] = (OUT == OUT_MASKED) ? (mk[o] > 0.0f ? acc[o] : 0.0f) : acc[o];
    }
  }
}

// Per-block sums for rho (sum (r/d)^2) and, with z, sum z^2; blockIdx.y is the column.
__global__ void __launch_bounds__(256) k_net_sums(const float* r, int64_t ldr, const float* d, const float* z,
                                                  int64_t n, double* partials, const int* stop) {
  if (stop && *stop != 0) return;
  __shared__ double red[2 * 8];
  const int col = blockIdx.y;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const float c = r[i * ldr + col] / d[i];
    s0 += (double)(c * c);
    if (z) s1 += (double)z[i] * (double)z[i];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = s0;
    red[8 + (threadIdx.x >> 5)] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < 8; ++w) {
      a0 += red[w];
      a1 += red[8 + w];
    }
    partials[((int64_t)col * gridDim.x + blockIdx.x) * 2 + 0] = a0;
    partials[((int64_t)col * gridDim.x + blockIdx.x) * 2 + 1] = a1;
  }
}

// rho[col] = sqrt(mean), zz = sum z^2 (column 0), summed over blocks in order.
__global__ void k_net_rho(const double* partials, int nblocks, int64_t n, float* rho, double* zz,
                          const int* stop) {
  if (stop && *stop != 0) return;
  const int col = blockIdx.x;
  double a0 = 0.0, a1 = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) {
    a0 += partials[((int64_t)col * nblocks + b) * 2];
    a1 += partials[((int64_t)col * nblocks + b) * 2 + 1];
  }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  if (threadIdx.x == 0) {
    rho[col] = (float)sqrt(a0 / (double)n);
    if (zz && col == 0) *zz = a1;
  }
}

// G3 = 2 rho (rho O - z) / zz and per-block sums of (rho O - z)^2.
__global__ void __launch_bounds__(256) k_net_loss(const float* O, const float* z, const float* rho,
                                                  const double* zz, int64_t n, float* G3, double* partials) {
  __shared__ double red[8];
  const float rh = rho[0];
  const float sc = (float)(2.0 * (double)rh / *zz);
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const float e = rh * O[i] - z[i];
    G3[i] = sc * e;
    s += (double)e * (double)e;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void k_net_loss_final(const double* partials, int nblocks, const double* zz, double* loss) {
  double t = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) t += partials[b];
  t = warp_sum(t);
  if (threadIdx.x == 0) *loss += t / *zz;
}

// Per-block weight gradient dW[o][c][t] = sum_px G[px][o] X[px + t][c] over the block's
// tile (X staged like a conv input); partials[block][(o * CIN + c) * 9 + t].
template <int CIN, int COUT, int IN>
__global__ void __launch_bounds__(NET_TW * NET_TH) k_net_wgrad(const NetArgs a, const float* G, float* partials) {
  __shared__ __align__(16) float sx[CIN * NET_HP];
  __shared__ float sg[COUT * NET_TW * NET_TH];               // [o][px]
  const int bx = blockIdx.x * NET_TW, by = blockIdx.y * NET_TH;
  net_stage<CIN, IN>(a, 0, bx, by, sx);
  for (int e = threadIdx.x; e < COUT * NET_TW * NET_TH; e += NET_TW * NET_TH) {
    const int o = e / (NET_TW * NET_TH), p = e - o * (NET_TW * NET_TH);
    const int ly = p / NET_TW, lx = p - ly * NET_TW;
    const int x = bx + lx, y = by + ly;
    sg[e] = (x < a.nx && y < a.ny) ? G[((int64_t)y * a.nx + x) * COUT + o] : 0.0f;
  }
  __syncthreads();
  const int blk = blockIdx.y * gridDim.x + blockIdx.x;
  for (int e = threadIdx.x; e < COUT * CIN * 9; e += NET_TW * NET_TH) {
    const int o = e / (CIN * 9), ct = e - o * (CIN * 9), c = ct / 9, t = ct - c * 9;
    const int ty = t / 3, tx = t - 3 * ty;
    float s0 = 0.0f, s1 = 0.0f;
    for (int ly = 0; ly < NET_TH; ++ly) {
      const float* xs = sx + c * NET_HP + (ly + ty) * NET_HW + tx;
      const float* gs = sg + o * NET_TW * NET_TH + ly * NET_TW;
#pragma unroll 8
      for (int lx = 0; lx < NET_TW; lx += 2) {
        s0 = fmaf(gs[lx], xs[lx], s0);
        s1 = fmaf(gs[lx + 1], xs[lx + 1], s1);
      }
    }
    partials[(int64_t)blk * (COUT * CIN * 9) + e] = s0 + s1;
  }
}

// grad[off + e] += sum_b partials[b][e]
__global__ void k_net_wgrad_reduce(const float* partials, int nblocks, int ne, float* grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += (double)partials[(int64_t)b * ne + e];
  grad[e] += (float)s;
}

__global__ void k_net_adam(float* w, float* wq, float* m, float* v, float* grad, int n, float lr, float b1,
                           float b2, float eps, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float g = grad[e];
  const float mm = b1 * m[e] + (1.0f - b1) * g;
  const float vv = b2 * v[e] + (1.0f - b2) * g * g;
  m[e] = mm;
  v[e] = vv;
  const float wn = w[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  w[e] = wn;
  wq[e] = bf16_round(wn);
  grad[e] = 0.0f;
}

__global__ void k_net_scale(float* g, int n, float scale) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) g[e] *= scale;
}

__global__ void k_net_round(const float* w, float* wq, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) wq[e] = bf16_round(w[e]);
}

// ------------------------------------------------------------------ host side
struct Bufs {
  float* A1;        // [cols][n][16]
  float* A2;        // [cols][n][16]
  float* O;         // [n]
  float* G3;        // [n]
  float* G2;        // [n][16]
  float* G1;        // [n][16]
  float* rho;       // [cols]
  double* zz;       // [1]
  double* dpart;    // [cols][nb][2]
  float* wpart;     // [tiles][2304]
};

int net_ws(bf_net* net, const bf_graph* g, int cols, bool train, Bufs* b) {
  const int64_t n = g->n;
  const int nb_red = (int)std::min<int64_t>((n + 255) / 256, 1024);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t act = al((size_t)cols * n * NET_CH * sizeof(float));
  const size_t vec = al((size_t)n * sizeof(float));
  const size_t act1 = al((size_t)n * NET_CH * sizeof(float));
  const size_t ntile = (size_t)((g->nx + NET_TW - 1) / NET_TW) * (size_t)((g->ny + NET_TH - 1) / NET_TH);
  size_t bytes = 2 * act + al(cols * sizeof(float)) + al(sizeof(double)) +
                 al((size_t)cols * nb_red * 2 * sizeof(double));
  if (train) bytes += 2 * vec + 2 * act1 + al(ntile * NET_CH * NET_CH * 9 * sizeof(float));
  if (bytes > net->ws_bytes) {
    if (net->ws) cudaFree(net->ws);
    net->ws = nullptr;
    net->ws_bytes = 0;
    cudaError_t e = cudaMalloc(&net->ws, bytes);
    if (e != cudaSuccess) return bf_cuda_fail(e, "cudaMalloc(net workspace)");
    net->ws_bytes = bytes;
  }
  char* p = (char*)net->ws;
  b->A1 = (float*)p; p += act;
  b->A2 = (float*)p; p += act;
  b->rho = (float*)p; p += al(cols * sizeof(float));
  b->zz = (double*)p; p += al(sizeof(double));
  b->dpart = (double*)p; p += al((size_t)cols * nb_red * 2 * sizeof(double));
  b->O = b->G3 = nullptr;
  b->G2 = b->G1 = nullptr;
  b->wpart = nullptr;
  if (train) {
    b->O = (float*)p; p += vec;
    b->G3 = (float*)p; p += vec;
    b->G2 = (float*)p; p += act1;
    b->G1 = (float*)p; p += act1;
    b->wpart = (float*)p;
  }
  return BF_OK;
}

NetArgs net_args(const bf_net* net, const bf_graph* g) {
  NetArgs a;
  memset(&a, 0, sizeof(a));
  a.nx = (int)g->nx;
  a.ny = (int)g->ny;
  a.n = g->n;
  a.guide = (const float*)g->guide;
  a.d = (const float*)g->d;
  (void)net;
  return a;
}

template <int CIN, int COUT, int IN, int OUT>
int launch_conv(const NetArgs& a, int cols, cudaStream_t s) {
  const dim3 grid((unsigned)((a.nx + NET_TW - 1) / NET_TW), (unsigned)((a.ny + NET_TH - 1) / NET_TH), (unsigned)cols);
  BF_LAUNCH((k_net_conv<CIN, COUT, IN, OUT><<<grid, NET_TW * NET_TH, 0, s>>>(a)));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

// rho of `cols` columns of r (and zz of z when given)
int net_sums(const bf_graph* g, const float* r, int64_t ldr, const float* z, int cols, const Bufs& b,
             cudaStream_t s, const int* stop = nullptr) {
  const int64_t n = g->n;
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  BF_LAUNCH((k_net_sums<<<dim3(nb, cols), 256, 0, s>>>(r, ldr, (const float*)g->d, z, n, b.dpart, stop)));
  BF_LAUNCH((k_net_rho<<<cols, 32, 0, s>>>(b.dpart, nb, n, b.rho, z ? b.zz : nullptr, stop)));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

int check_pair(const bf_net* net, const bf_graph* g) {
  if (!net || !g) return bf_fail(BF_EINVAL, "bf_net: NULL argument");
  if (g->esize != 4) return bf_fail(BF_EINVAL, "bf_net: the net works on FP32 graphs");
  if (g->nx > 0x7fffffff / 2 || g->ny > 65535 * NET_TH) return bf_fail(BF_EINVAL, "bf_net: image too large");
  return BF_OK;
}

}  // namespace

// ------------------------------------------------------------------ exported
int bf_net_apply_f32(const bf_net* net_c, const bf_graph* g, const float* R, int64_t ldr, int k, float* Z,
                     int64_t ldz, cudaStream_t s, const int* stop) {
  bf_net* net = const_cast<bf_net*>(net_c);
  int rc = check_pair(net, g);
  if (rc) return rc;
  for (int c0 = 0; c0 < k; c0 += NET_COLS) {
    const int cols = std::min(NET_COLS, k - c0);
    Bufs b;
    rc = net_ws(net, g, cols, false, &b);
    if (rc) return rc;
    rc = net_sums(g, R + c0, ldr, nullptr, cols, b, s, stop);
    if (rc) return rc;
    NetArgs a = net_args(net, g);
    a.stop = stop;
    a.r = R + c0;
    a.ldr = ldr;
    a.rho = b.rho;
    a.w = net->wq + NET_W1;
    a.out = b.A1;
    if ((rc = launch_conv<NET_CIN, NET_CH, IN_NET, OUT_ACT>(a, cols, s))) return rc;
    a.in = b.A1;
    a.w = net->wq + NET_W2;
    a.out = b.A2;
    if ((rc = launch_conv<NET_CH, NET_CH, IN_RELU, OUT_ACT>(a, cols, s))) return rc;
    a.in = b.A2;
    a.w = net->wq + NET_W3;
    a.z = Z + c0;
    a.ldz = ldz;
    if ((rc = launch_conv<NET_CH, 1, IN_RELU, OUT_PRECOND>(a, cols, s))) return rc;
  }
  return BF_OK;
}

extern "C" int bf_net_create(const float* w_host, bf_net** out) {
  if (!w_host || !out) return bf_fail(BF_EINVAL, "bf_net_create: NULL argument");
  *out = nullptr;
  bf_net* net = new bf_net();
  memset(net, 0, sizeof(*net));
  BF_CUDA(cudaGetDevice(&net->device));
  const size_t wb = NET_NW * sizeof(float);
  cudaError_t e = cudaMalloc(&net->w, 5 * wb + 256);
  if (e != cudaSuccess) {
    delete net;
    return bf_cuda_fail(e, "cudaMalloc(net)");
  }
  net->wq = net->w + NET_NW;
  net->m = net->wq + NET_NW;
  net->v = net->m + NET_NW;
  net->grad = net->v + NET_NW;
  net->loss = reinterpret_cast<double*>(net->grad + NET_NW + (NET_NW & 1));
  BF_CUDA(cudaMemcpy(net->w, w_host, wb, cudaMemcpyHostToDevice));
  BF_CUDA(cudaMemset(net->m, 0, 3 * wb + 2 * sizeof(double)));
  BF_LAUNCH((k_net_round<<<(NET_NW + 255) / 256, 256>>>(net->w, net->wq, NET_NW)));
  BF_CUDA(cudaDeviceSynchronize());
  *out = net;
  return BF_OK;
}

extern "C" int bf_net_free(bf_net* net) {
  if (!net) return BF_OK;
  if (net->ws) cudaFree(net->ws);
  if (net->w) cudaFree(net->w);
  delete net;
  return BF_OK;
}

extern "C" int bf_net_nweights(void) { return NET_NW; }

extern "C" int bf_net_weights(const bf_net* net, float* w_host, int rounded) {
  if (!net || !w_host) return bf_fail(BF_EINVAL, "bf_net_weights: NULL argument");
  BF_CUDA(cudaMemcpy(w_host, rounded ? net->wq : net->w, NET_NW * sizeof(float), cudaMemcpyDeviceToHost));
  return BF_OK;
}

extern "C" int bf_net_apply(const bf_net* net, const bf_graph* g, const float* R, int64_t ldr, int k, float* Z,
                            int64_t ldz, void* stream) {
  if (!R || !Z) return bf_fail(BF_EINVAL, "bf_net_apply: NULL argument");
  if (k < 1 || ldr < k || ldz < k) return bf_fail(BF_EINVAL, "bf_net_apply: need 1 <= k <= ld");
  return bf_net_apply_f32(net, g, R, ldr, k, Z, ldz, (cudaStream_t)stream, nullptr);
}

extern "C" int bf_net_zero_grad(bf_net* net, void* stream) {
  if (!net) return bf_fail(BF_EINVAL, "bf_net_zero_grad: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  BF_CUDA(cudaMemsetAsync(net->grad, 0, NET_NW * sizeof(float), s));
  BF_CUDA(cudaMemsetAsync(net->loss, 0, sizeof(double), s));
  return BF_OK;
}

extern "C" int bf_net_accumulate(bf_net* net, const bf_graph* g, const float* r, const float* z, void* stream) {
  int rc = check_pair(net, g);
  if (rc) return rc;
  if (!r || !z) return bf_fail(BF_EINVAL, "bf_net_accumulate: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  Bufs b;
  if ((rc = net_ws(net, g, 1, true, &b))) return rc;
  if ((rc = net_sums(g, r, 1, z, 1, b, s))) return rc;
  NetArgs a = net_args(net, g);
  a.r = r;
  a.ldr = 1;
  a.rho = b.rho;
  // forward, keeping the pre-activations
  a.w = net->wq + NET_W1;
  a.out = b.A1;
  if ((rc = launch_conv<NET_CIN, NET_CH, IN_NET, OUT_ACT>(a, 1, s))) return rc;
  a.in = b.A1;
  a.w = net->wq + NET_W2;
  a.out = b.A2;
  if ((rc = launch_conv<NET_CH, NET_CH, IN_RELU, OUT_ACT>(a, 1, s))) return rc;
  a.in = b.A2;
  a.w = net->wq + NET_W3;
  a.out = b.O;
  if ((rc = launch_conv<NET_CH, 1, IN_RELU, OUT_ACT>(a, 1, s))) return rc;
  // loss and dL/dO
  const int64_t n = g->n;
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  BF_LAUNCH((k_net_loss<<<nb, 256, 0, s>>>(b.O, z, b.rho, b.zz, n, b.G3, b.dpart)));
  BF_LAUNCH((k_net_loss_final<<<1, 32, 0, s>>>(b.dpart, nb, b.zz, net->loss)));
  // backward: G2 = conv^T(G3, W3) * (A2 > 0), G1 = conv^T(G2, W2) * (A1 > 0)
  a.transpose = 1;
  a.in = b.G3;
  a.w = net->wq + NET_W3;
  a.out = b.G2;
  a.mask = b.A2;
  if ((rc = launch_conv<1, NET_CH, IN_PLAIN, OUT_MASKED>(a, 1, s))) return rc;
  a.in = b.G2;
  a.w = net->wq + NET_W2;
  a.out = b.G1;
  a.mask = b.A1;
  if ((rc = launch_conv<NET_CH, NET_CH, IN_PLAIN, OUT_MASKED>(a, 1, s))) return rc;
  a.transpose = 0;
  // weight gradients: dW3 = corr(G3, relu(A2)), dW2 = corr(G2, relu(A1)), dW1 = corr(G1, C)
  const dim3 tg((unsigned)((a.nx + NET_TW - 1) / NET_TW), (unsigned)((a.ny + NET_TH - 1) / NET_TH));
  const int ntile = (int)(tg.x * tg.y);
  a.in = b.A2;
  BF_LAUNCH((k_net_wgrad<NET_CH, 1, IN_RELU><<<tg, NET_TW * NET_TH, 0, s>>>(a, b.G3, b.wpart)));
  BF_LAUNCH((k_net_wgrad_reduce<<<(NET_CH * 9 + 127) / 128, 128, 0, s>>>(b.wpart, ntile, NET_CH * 9, net->grad + NET_W3)));
  a.in = b.A1;
  BF_LAUNCH((k_net_wgrad<NET_CH, NET_CH, IN_RELU><<<tg, NET_TW * NET_TH, 0, s>>>(a, b.G2, b.wpart)));
  BF_LAUNCH((k_net_wgrad_reduce<<<(NET_CH * NET_CH * 9 + 127) / 128, 128, 0, s>>>(b.wpart, ntile, NET_CH * NET_CH * 9,
                                                                                   net->grad + NET_W2)));
  BF_LAUNCH((k_net_wgrad<NET_CIN, NET_CH, IN_NET><<<tg, NET_TW * NET_TH, 0, s>>>(a, b.G1, b.wpart)));
  BF_LAUNCH((k_net_wgrad_reduce<<<(NET_CH * NET_CIN * 9 + 127) / 128, 128, 0, s>>>(b.wpart, ntile, NET_CH * NET_CIN * 9,
                                                                                    net->grad + NET_W1)));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

extern "C" int bf_net_grad(const bf_net* net, float* grad_host, double* loss_host, void* stream) {
  if (!net) return bf_fail(BF_EINVAL, "bf_net_grad: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (grad_host) BF_CUDA(cudaMemcpyAsync(grad_host, net->grad, NET_NW * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (loss_host) BF_CUDA(cudaMemcpyAsync(loss_host, net->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  BF_CUDA(cudaStreamSynchronize(s));
  return BF_OK;
}

extern "C" int bf_net_adam(bf_net* net, float lr, float scale, void* stream) {
  if (!net) return bf_fail(BF_EINVAL, "bf_net_adam: NULL argument");
  if (!(lr >= 0.0f) || !(scale > 0.0f)) return bf_fail(BF_EINVAL, "bf_net_adam: bad lr or scale");
  cudaStream_t s = (cudaStream_t)stream;
  net->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)net->t), c2 = 1.0f - powf(b2, (float)net->t);
  if (scale != 1.0f) {
    // the accumulated gradient is a sum over pairs: scale = 1 / pairs makes it a mean
    BF_LAUNCH((k_net_scale<<<(NET_NW + 255) / 256, 256, 0, s>>>(net->grad, NET_NW, scale)));
  }
  BF_LAUNCH((k_net_adam<<<(NET_NW + 255) / 256, 256, 0, s>>>(net->w, net->wq, net->m, net->v, net->grad, NET_NW, lr,
                                                              b1, b2, 1e-8f, c1, c2)));
  BF_CUDA(cudaMemsetAsync(net->loss, 0, sizeof(double), s));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}
