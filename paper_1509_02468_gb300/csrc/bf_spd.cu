// A learned symmetric positive definite preconditioner T for Algorithms 2 and 3:
//
//     T r = D^-1/2 (u + K^T K u),      u = D^-1/2 r,
//
// K a (2h + 1) x (2h + 1) cross-correlation of the image-shaped u with zeros outside the
// image, K^T its adjoint (the correlation with K turned by 180 degrees).  The paper leaves
// T open (Section 5; Section 8 names better preconditioners as future work); this one is
// linear, symmetric and positive definite by construction (I + K^T K >= I), so CG keeps
// the A-norm optimality of Section 5 and LOBPCG's Ritz vectors stay sign-free.  K = 0 is
// Jacobi.  Training minimises, over pairs (r, z) with A z = r and A = L + sigma I, the
// A-norm error of T r relative to z: (z - T r)^T A (z - T r) / z^T A z.
//
// One application is two tiled stencil passes over FP32 data (w = K u, then
// s = D^-1/2 (u + K^T w)), each staging its tile and halo in shared memory.
#include <math.h>

#include <algorithm>

#include "bf_internal.cuh"

int bf_apply_f32(const bf_graph* g, int op, const float* X, int64_t ldx, int k, float* Y,
                 int64_t ldy, double* dots, cudaStream_t s);

#define SPD_HMAX 4            // largest half-width (9 x 9 kernel)
#define SPD_NKMAX ((2 * SPD_HMAX + 1) * (2 * SPD_HMAX + 1))
#define SPD_TW 32
#define SPD_TH 8
#define SPD_T (SPD_TW * SPD_TH)

struct bf_spd {
  int device;
  int half, ks, nk;
  int t;                 // Adam steps taken
  float* K;              // [nk] the kernel, row-major over (dy, dx)
  float* m;              // [nk] Adam moments
  float* v;              // [nk]
  double* grad;          // [nk] accumulated gradient
  double* scal;          // [4]: accumulated loss, -2 / z^T A z of the current pair, spare
  void* ws;              // grow-only workspace
  size_t ws_bytes;
};

namespace {

// out(p) = post(p) * (add(p) * adds(p) + sum_a Kx[a] x(p + a) xs(p + a)), Kx = K or K
// turned by 180 degrees; with zsub: out(p) = zsub(p) - that.  Column c = blockIdx.z of
// pixel-major blocks (x: ldx, add: ldadd, zsub and out: ldo).  NULL scale pointers mean 1,
// a NULL add means 0.
struct SpdCorr {
  int nx, ny, h, ks;
  int flip;
  const float* K;
  const float* x;
  int64_t ldx;
  const float* xs;
  const float* add;
  int64_t ldadd;
  const float* adds;
  const float* post;
  const float* zsub;
  float* out;
  int64_t ldo;
};

__global__ void __launch_bounds__(SPD_T) k_spd_corr(const SpdCorr a) {
  bf_pdl_enter();
  __shared__ float sK[SPD_NKMAX];
  __shared__ float tile[(SPD_TH + 2 * SPD_HMAX) * (SPD_TW + 2 * SPD_HMAX)];
  const int h = a.h, ks = a.ks, nk = ks * ks;
  const int c = blockIdx.z;
  const int bx = blockIdx.x * SPD_TW, by = blockIdx.y * SPD_TH;
  const int hw = SPD_TW + 2 * h, hh = SPD_TH + 2 * h;
  for (int i = threadIdx.x; i < nk; i += SPD_T) sK[i] = a.K[a.flip ? nk - 1 - i : i];
  for (int i = threadIdx.x; i < hw * hh; i += SPD_T) {
    const int ty = i / hw, tx = i - ty * hw;
    const int gy = by + ty - h, gx = bx + tx - h;
    float v = 0.0f;
    if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny) {
      const int64_t p = (int64_t)gy * a.nx + gx;
      v = a.x[p * a.ldx + c];
      if (a.xs) v *= a.xs[p];
    }
    tile[i] = v;
  }
  __syncthreads();
  const int lx = threadIdx.x % SPD_TW, ly = threadIdx.x / SPD_TW;
  const int gx = bx + lx, gy = by + ly;
  if (gx >= a.nx || gy >= a.ny) return;
  float acc = 0.0f;
  for (int dy = 0; dy < ks; ++dy) {
    const float* row = tile + (ly + dy) * hw + lx;
    const float* kr = sK + dy * ks;
    for (int dx = 0; dx < ks; ++dx) acc = fmaf(kr[dx], row[dx], acc);
  }
  const int64_t p = (int64_t)gy * a.nx + gx;
  if (a.add) acc += a.add[p * a.ldadd + c] * (a.adds ? a.adds[p] : 1.0f);
  if (a.post) acc *= a.post[p];
  if (a.zsub) acc = a.zsub[p * a.ldo + c] - acc;
  a.out[p * a.ldo + c] = acc;
}

// Partial sums over pixels of e^T (L e + sigma e) and z^T (L z + sigma z) (FP64).
__global__ void __launch_bounds__(256) k_spd_dots(const float* e, const float* le, const float* z, const float* lz,
                                                  float sigma, int64_t n, double* partials) {
  __shared__ double red[2][256 / 32];
  double se = 0.0, sz = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    se += (double)e[i] * (double)fmaf(sigma, e[i], le[i]);
    sz += (double)z[i] * (double)fmaf(sigma, z[i], lz[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sz += __shfl_xor_sync(0xffffffffu, sz, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = se;
    red[1][w] = sz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < 256 / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// loss += eAe / zAz; scal[1] = -2 / zAz (the factor of dloss/dt = -2 A e / zAz)
__global__ void k_spd_loss(const double* partials, int nb, double* scal) {
  if (threadIdx.x != 0) return;
  double eae = 0.0, zaz = 0.0;
  for (int b = 0; b < nb; ++b) {
    eae += partials[2 * b];
    zaz += partials[2 * b + 1];
  }
  scal[0] += eae / zaz;
  scal[1] = -2.0 / zaz;
}

// h(p) = d^-1/2(p) * scal[1] * (L e + sigma e)(p)
__global__ void __launch_bounds__(256) k_spd_hvec(const float* e, const float* le, const float* dis, float sigma,
                                                  const double* scal, int64_t n, float* hv) {
  const float f = (float)scal[1];
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
    hv[i] = dis[i] * f * fmaf(sigma, e[i], le[i]);
}

// Per tile: part[tile][a] = sum_{p in tile} w(p) h(p + a) + (K h)(p) u(p + a), u = d^-1/2 r,
// h and u zero outside the image; a over the kernel's taps, row-major (dy, dx).
__global__ void __launch_bounds__(SPD_T) k_spd_wgrad(int nx, int ny, int h, const float* w, const float* kh,
                                                     const float* hv, const float* r, const float* dis, float* part) {
  __shared__ float th[(SPD_TH + 2 * SPD_HMAX) * (SPD_TW + 2 * SPD_HMAX)];
  __shared__ float tu[(SPD_TH + 2 * SPD_HMAX) * (SPD_TW + 2 * SPD_HMAX)];
  __shared__ float red[SPD_T / 32][SPD_NKMAX];
  const int ks = 2 * h + 1, nk = ks * ks;
  const int bx = blockIdx.x * SPD_TW, by = blockIdx.y * SPD_TH;
  const int hw = SPD_TW + 2 * h, hh = SPD_TH + 2 * h;
  for (int i = threadIdx.x; i < hw * hh; i += SPD_T) {
    const int ty = i / hw, tx = i - ty * hw;
    const int gy = by + ty - h, gx = bx + tx - h;
    float vh = 0.0f, vu = 0.0f;
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
      const int64_t p = (int64_t)gy * nx + gx;
      vh = hv[p];
      vu = r[p] * dis[p];
    }
    th[i] = vh;
    tu[i] = vu;
  }
  __syncthreads();
  const int lx = threadIdx.x % SPD_TW, ly = threadIdx.x / SPD_TW;
  const int gx = bx + lx, gy = by + ly;
  const bool in = gx < nx && gy < ny;
  float wp = 0.0f, kp = 0.0f;
  if (in) {
    const int64_t p = (int64_t)gy * nx + gx;
    wp = w[p];
    kp = kh[p];
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int dy = 0; dy < ks; ++dy)
    for (int dx = 0; dx < ks; ++dx) {
      const int o = (ly + dy) * hw + lx + dx;
      float v = fmaf(wp, th[o], kp * tu[o]);
      for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
      if (lane == 0) red[wid][dy * ks + dx] = v;
    }
  __syncthreads();
  const int64_t tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
  for (int t = threadIdx.x; t < nk; t += SPD_T) {
    float s = 0.0f;
    for (int i = 0; i < SPD_T / 32; ++i) s += red[i][t];
    part[tile * nk + t] = s;
  }
}

// grad[a] += sum over tiles of part[tile][a]
__global__ void k_spd_grad_reduce(const float* part, int64_t ntiles, int nk, double* grad) {
  const int a = blockIdx.x;
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) s += (double)part[t * nk + a];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) tot += red[i];
    grad[a] += tot;
  }
}

// One Adam step (Kingma and Ba) on the kernel from the accumulated gradient times scale;
// the gradient and the loss accumulator are cleared.
__global__ void k_spd_adam(float* K, float* m, float* v, double* grad, double* scal, int nk, float lr, float scale,
                           float b1, float b2, float eps, float c1, float c2) {
  const int e = threadIdx.x;
  if (e < nk) {
    const float g = (float)(grad[e] * (double)scale);
    const float mm = b1 * m[e] + (1.0f - b1) * g;
    const float vv = b2 * v[e] + (1.0f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    K[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    grad[e] = 0.0;
  }
  if (e == 0) scal[0] = 0.0;
}

int spd_check(const bf_spd* T, const bf_graph* g, const char* who) {
  if (!T || !g) return bf_fail(BF_EINVAL, std::string(who) + ": NULL argument");
  if (g->esize != 4) return bf_fail(BF_EINVAL, std::string(who) + ": needs an FP32 graph");
  if (g->kind != BF_KIND_BILATERAL) return bf_fail(BF_EINVAL, std::string(who) + ": needs a bilateral graph");
  int dev = 0;
  BF_CUDA(cudaGetDevice(&dev));
  if (dev != T->device || dev != g->device)
    return bf_fail(BF_EINVAL, std::string(who) + ": preconditioner, graph and current device differ");
  return BF_OK;
}

// grow-only workspace of the preconditioner (a larger image frees and reallocates it: the
// device is synchronised first)
int spd_ws(bf_spd* T, size_t bytes, char** out) {
  if (bytes > T->ws_bytes) {
    if (T->ws) {
      BF_CUDA(cudaDeviceSynchronize());
      BF_CUDA(cudaFree(T->ws));
      T->ws = nullptr;
      T->ws_bytes = 0;
    }
    bytes = (bytes + 4095) & ~(size_t)4095;
    BF_CUDA(cudaMalloc(&T->ws, bytes));
    T->ws_bytes = bytes;
  }
  *out = (char*)T->ws;
  return BF_OK;
}

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

SpdCorr corr_args(const bf_spd* T, const bf_graph* g) {
  SpdCorr a;
  memset(&a, 0, sizeof(a));
  a.nx = g->nx;
  a.ny = g->ny;
  a.h = T->half;
  a.ks = T->ks;
  a.K = T->K;
  return a;
}

void launch_corr(const SpdCorr& a, int k, cudaStream_t s) {
  const dim3 grid((unsigned)((a.nx + SPD_TW - 1) / SPD_TW), (unsigned)((a.ny + SPD_TH - 1) / SPD_TH), (unsigned)k);
  BF_LAUNCH_PDL(k_spd_corr, grid, SPD_T, 0, s, a);
}

}  // namespace

// Z = T R for k columns (pixel-major, ld >= k); Z may equal R.  Used by cg_filter and
// lobpcg_filter with BF_PRECOND_SPD.
int bf_spd_apply_f32(const bf_spd* Tc, const bf_graph* g, const float* R, int64_t ldr, int k, float* Z,
                     int64_t ldz, cudaStream_t s) {
  int rc = spd_check(Tc, g, "bf_spd_apply");
  if (rc) return rc;
  bf_spd* T = const_cast<bf_spd*>(Tc);
  char* w = nullptr;
  if ((rc = spd_ws(T, al256((size_t)g->n * k * sizeof(float)), &w))) return rc;
  float* W = (float*)w;                                  // w = K u, [n][k]
  SpdCorr a = corr_args(T, g);
  a.flip = 0;
  a.x = R;
  a.ldx = ldr;
  a.xs = (const float*)g->dis;
  a.out = W;
  a.ldo = k;
  launch_corr(a, k, s);
  SpdCorr b = corr_args(T, g);                           // Z = D^-1/2 (D^-1/2 R + K^T w)
  b.flip = 1;
  b.x = W;
  b.ldx = k;
  b.add = R;
  b.ldadd = ldr;
  b.adds = (const float*)g->dis;
  b.post = (const float*)g->dis;
  b.out = Z;
  b.ldo = ldz;
  launch_corr(b, k, s);
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

extern "C" int bf_spd_create(int half, const float* K_host, bf_spd** out) {
  if (!out) return bf_fail(BF_EINVAL, "bf_spd_create: NULL argument");
  *out = nullptr;
  if (half < 1 || half > SPD_HMAX) return bf_fail(BF_EINVAL, "bf_spd_create: half-width must be 1..4");
  bf_spd* T = new bf_spd();
  memset(T, 0, sizeof(*T));
  T->half = half;
  T->ks = 2 * half + 1;
  T->nk = T->ks * T->ks;
  cudaError_t e = cudaGetDevice(&T->device);
  if (e == cudaSuccess) e = cudaMalloc(&T->grad, (size_t)T->nk * sizeof(double) + 4 * sizeof(double) + 3 * T->nk * sizeof(float));
  if (e != cudaSuccess) {
    delete T;
    return bf_cuda_fail(e, "cudaMalloc(bf_spd)");
  }
  T->scal = T->grad + T->nk;
  T->K = reinterpret_cast<float*>(T->scal + 4);
  T->m = T->K + T->nk;
  T->v = T->m + T->nk;
  int rc = BF_OK;
  if (K_host) {
    if (cudaMemcpy(T->K, K_host, T->nk * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = bf_fail(BF_ECUDA, "bf_spd_create: copy of K");
  } else if (cudaMemset(T->K, 0, T->nk * sizeof(float)) != cudaSuccess) {
    rc = bf_fail(BF_ECUDA, "bf_spd_create: clear K");
  }
  if (!rc && (cudaMemset(T->grad, 0, T->nk * sizeof(double) + 4 * sizeof(double)) != cudaSuccess ||
              cudaMemset(T->m, 0, 2 * T->nk * sizeof(float)) != cudaSuccess))
    rc = bf_fail(BF_ECUDA, "bf_spd_create: clear state");
  if (rc) {
    cudaFree(T->grad);
    delete T;
    return rc;
  }
  *out = T;
  return BF_OK;
}

extern "C" int bf_spd_free(bf_spd* T) {
  if (!T) return BF_OK;
  if (T->ws) cudaFree(T->ws);
  if (T->grad) cudaFree(T->grad);
  delete T;
  return BF_OK;
}

extern "C" int bf_spd_size(const bf_spd* T) { return T ? T->nk : 0; }

extern "C" int bf_spd_weights(const bf_spd* T, float* K_host) {
  if (!T || !K_host) return bf_fail(BF_EINVAL, "bf_spd_weights: NULL argument");
  BF_CUDA(cudaMemcpy(K_host, T->K, T->nk * sizeof(float), cudaMemcpyDeviceToHost));
  return BF_OK;
}

extern "C" int bf_spd_apply(const bf_spd* T, const bf_graph* g, const float* R, int64_t ldr, int k, float* Z,
                            int64_t ldz, void* stream) {
  if (!R || !Z) return bf_fail(BF_EINVAL, "bf_spd_apply: NULL argument");
  if (k < 1 || ldr < k || ldz < k) return bf_fail(BF_EINVAL, "bf_spd_apply: need 1 <= k <= ld");
  return bf_spd_apply_f32(T, g, R, ldr, k, Z, ldz, (cudaStream_t)stream);
}

extern "C" int bf_spd_zero_grad(bf_spd* T, void* stream) {
  if (!T) return bf_fail(BF_EINVAL, "bf_spd_zero_grad: NULL argument");
  BF_CUDA(cudaMemsetAsync(T->grad, 0, (size_t)T->nk * sizeof(double) + sizeof(double), (cudaStream_t)stream));
  return BF_OK;
}

extern "C" int bf_spd_accumulate(bf_spd* T, const bf_graph* g, double shift, const float* r, const float* z,
                                 void* stream) {
  int rc = spd_check(T, g, "bf_spd_accumulate");
  if (rc) return rc;
  if (!r || !z) return bf_fail(BF_EINVAL, "bf_spd_accumulate: NULL argument");
  if (!(shift >= 0.0) || !isfinite(shift)) return bf_fail(BF_EINVAL, "bf_spd_accumulate: shift must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n;
  const size_t vb = al256((size_t)n * sizeof(float));
  const dim3 tg((unsigned)((g->nx + SPD_TW - 1) / SPD_TW), (unsigned)((g->ny + SPD_TH - 1) / SPD_TH));
  const int64_t ntiles = (int64_t)tg.x * tg.y;
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  char* w = nullptr;
  if ((rc = spd_ws(T, 6 * vb + al256((size_t)ntiles * T->nk * sizeof(float)) + al256((size_t)nb * 2 * sizeof(double)),
                   &w)))
    return rc;
  float* W = (float*)w;                 // K u
  float* E = (float*)(w + vb);          // e = z - T r
  float* LE = (float*)(w + 2 * vb);     // L e
  float* LZ = (float*)(w + 3 * vb);     // L z
  float* HV = (float*)(w + 4 * vb);     // h = D^-1/2 dloss/dt
  float* KH = (float*)(w + 5 * vb);     // K h
  float* part = (float*)(w + 6 * vb);
  double* dpart = (double*)(w + 6 * vb + al256((size_t)ntiles * T->nk * sizeof(float)));
  const float* dis = (const float*)g->dis;
  // forward: w = K u, e = z - D^-1/2 (u + K^T w)
  SpdCorr a = corr_args(T, g);
  a.x = r;
  a.ldx = 1;
  a.xs = dis;
  a.out = W;
  a.ldo = 1;
  launch_corr(a, 1, s);
  SpdCorr b = corr_args(T, g);
  b.flip = 1;
  b.x = W;
  b.ldx = 1;
  b.add = r;
  b.ldadd = 1;
  b.adds = dis;
  b.post = dis;
  b.zsub = z;
  b.out = E;
  b.ldo = 1;
  launch_corr(b, 1, s);
  // A-norms: L e, L z by the operator, then e^T A e, z^T A z, the loss and h
  if ((rc = bf_apply_f32(g, BF_OP_L, E, 1, 1, LE, 1, nullptr, s))) return rc;
  if ((rc = bf_apply_f32(g, BF_OP_L, z, 1, 1, LZ, 1, nullptr, s))) return rc;
  const float sig = (float)shift;
  BF_LAUNCH((k_spd_dots<<<nb, 256, 0, s>>>(E, LE, z, LZ, sig, n, dpart)));
  BF_LAUNCH((k_spd_loss<<<1, 32, 0, s>>>(dpart, nb, T->scal)));
  BF_LAUNCH((k_spd_hvec<<<nb, 256, 0, s>>>(E, LE, dis, sig, T->scal, n, HV)));
  // K h, then the per-tap correlations
  SpdCorr c = corr_args(T, g);
  c.x = HV;
  c.ldx = 1;
  c.out = KH;
  c.ldo = 1;
  launch_corr(c, 1, s);
  BF_LAUNCH((k_spd_wgrad<<<tg, SPD_T, 0, s>>>(g->nx, g->ny, T->half, W, KH, HV, r, dis, part)));
  BF_LAUNCH((k_spd_grad_reduce<<<T->nk, 256, 0, s>>>(part, ntiles, T->nk, T->grad)));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

extern "C" int bf_spd_grad(const bf_spd* T, double* grad_host, double* loss_host, void* stream) {
  if (!T) return bf_fail(BF_EINVAL, "bf_spd_grad: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (grad_host) BF_CUDA(cudaMemcpyAsync(grad_host, T->grad, T->nk * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (loss_host) BF_CUDA(cudaMemcpyAsync(loss_host, T->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  BF_CUDA(cudaStreamSynchronize(s));
  return BF_OK;
}

extern "C" int bf_spd_adam(bf_spd* T, float lr, float scale, void* stream) {
  if (!T) return bf_fail(BF_EINVAL, "bf_spd_adam: NULL argument");
  if (!(lr >= 0.0f) || !(scale > 0.0f)) return bf_fail(BF_EINVAL, "bf_spd_adam: bad lr or scale");
  T->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)T->t), c2 = 1.0f - powf(b2, (float)T->t);
  BF_LAUNCH((k_spd_adam<<<1, 128, 0, (cudaStream_t)stream>>>(T->K, T->m, T->v, T->grad, T->scal, T->nk, lr, scale, b1,
                                                             b2, 1e-8f, c1, c2)));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}
