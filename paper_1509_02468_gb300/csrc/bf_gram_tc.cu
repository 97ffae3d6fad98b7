// Gram products of the Rayleigh-Ritz step of block LOBPCG (Algorithm 3, Section 6) on the
// fifth-generation tensor cores: [G_A | G_B] = S^T [A S | B S] for the trial basis
// S = [X W P] (n x m, m = 2k or 3k <= 96), as one BF16 GEMM with FP32 accumulation
// (M = 128 rows of S^T, N = 2m rounded up to 16, K = the pixels), split over the CTAs by
// chunks of 64 pixels.
//
// Per chunk the CTA converts S, A S and B S = diag(b) S from FP32 (pixel-major blocks) to
// BF16 and writes them transposed into shared memory in the K-major, unswizzled canonical
// layout (8-row x 16-byte core matrices, 128 B apart along K, 1024 B apart along rows);
// one thread issues the tcgen05.mma instructions, whose accumulator stays in tensor
// memory for the whole split-K range; tcgen05.commit arrives on an mbarrier per buffer,
// so staging of the next chunk overlaps the MMAs of the current one.  With `split` each
// operand is x = hi + lo (both BF16) and the products hi*hi + hi*lo + lo*hi are
// accumulated (about 16 significant bits).  At the end the accumulator is read with
// tcgen05.ld and the FP32 partials of all CTAs are summed in FP64.
//
// Every mbarrier wait is bounded: on a timeout the kernel records an error, waits once
// more (bounded) for its own MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "bf_internal.cuh"

#define TC_THREADS 256
#define TC_KT 64                   // pixels per chunk (K per stage)
#define TC_M 128                   // MMA rows (rows of S^T, m padded)
#define TC_TMEM_COLS 256           // tensor-memory columns allocated (>= N)
#define TC_WAIT_ITERS (1 << 22)    // bound on mbarrier polls

namespace {

struct TcArgs {
  const float* S[3];
  const float* AS[3];
  const float* b;                  // B diagonal (NULL: I)
  int nblk, k, m, N;
  int64_t n;
  float* partials;                 // [gridDim.x][m][2m]
  const int* status;               // LOBPCG status: nonzero = stopped
  int* err;                        // set to 4 on a wait timeout
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int iters = TC_WAIT_ITERS) {
  for (int i = 0; i < iters; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (row-group) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M.
__host__ __device__ constexpr uint32_t idesc_bf16(int N, int M) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive accumulator columns of this thread's lane (32x32b shape).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive accumulator columns of this thread's lane; the caller waits
// (tcgen05.wait::ld) before using them, so several loads can be in flight.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Byte offset of (row, pixel) in a K-major unswizzled operand tile of TC_KT pixels.
__device__ __forceinline__ uint32_t tc_off(int row, int pix) {
  return (uint32_t)((row >> 3) * 1024 + (pix >> 3) * 128 + (row & 7) * 16 + (pix & 7) * 2);
}

template <bool SPLIT>
__device__ __forceinline__ void put_pair(unsigned char* hi, unsigned char* lo, int row, int pix, float x0, float x1) {
  const uint32_t off = tc_off(row, pix);
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  *reinterpret_cast<__nv_bfloat162*>(hi + off) = h;
  if (SPLIT) {
    const float2 hf = __bfloat1622float2(h);
    *reinterpret_cast<__nv_bfloat162*>(lo + off) = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  }
}

// Stage chunk c (pixels c * TC_KT ...) into the operand tiles: A rows = columns of S,
// B rows = columns of A S, then of B S.  A thread owns tasks tid, tid + TC_THREADS, ...
// (a pixel pair and four columns of one block); all its global loads are issued before
// any conversion so that they are in flight together.
#define TC_MAXT 6                  // tasks per thread: 2 * (m / 4) * 32 / 256 <= 6 for m <= 96
template <bool SPLIT>
__device__ void tc_stage(const TcArgs& a, int64_t c, unsigned char* Ahi, unsigned char* Alo, unsigned char* Bhi,
                         unsigned char* Blo) {
  const int kq = a.k >> 2;
  const int per = a.nblk * (TC_KT / 2) * kq;
  const int64_t p0 = c * TC_KT;
  float4 v0[TC_MAXT], v1[TC_MAXT];
#pragma unroll
  for (int u = 0; u < TC_MAXT; ++u) {
    const int t = threadIdx.x + u * TC_THREADS;
    v0[u] = v1[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (t < 2 * per) {
      const bool is_as = t >= per;
      const int tt = is_as ? t - per : t;
      const int cq = tt % kq, rest = tt / kq;
      const int pp = rest % (TC_KT / 2), bk = rest / (TC_KT / 2);
      const int64_t p = p0 + 2 * pp;
      // selects rather than a runtime index into the parameter arrays (which would copy
      // them to local memory)
      const float* const* blocks = is_as ? a.AS : a.S;
      const float* src = bk == 0 ? blocks[0] : (bk == 1 ? blocks[1] : blocks[2]);
      if (p < a.n) v0[u] = __ldg(reinterpret_cast<const float4*>(src + p * a.k + 4 * cq));
      if (p + 1 < a.n) v1[u] = __ldg(reinterpret_cast<const float4*>(src + (p + 1) * a.k + 4 * cq));
    }
  }
#pragma unroll
  for (int u = 0; u < TC_MAXT; ++u) {
    const int t = threadIdx.x + u * TC_THREADS;
    if (t >= 2 * per) break;
    const bool is_as = t >= per;
    const int tt = is_as ? t - per : t;
    const int cq = tt % kq, rest = tt / kq;
    const int pp = rest % (TC_KT / 2), bk = rest / (TC_KT / 2);
    const int64_t p = p0 + 2 * pp;
    const int col = bk * a.k + 4 * cq;
    const float x0[4] = {v0[u].x, v0[u].y, v0[u].z, v0[u].w}, x1[4] = {v1[u].x, v1[u].y, v1[u].z, v1[u].w};
    if (!is_as) {
      const float b0 = (a.b && p < a.n) ? a.b[p] : 1.0f;
      const float b1 = (a.b && p + 1 < a.n) ? a.b[p + 1] : 1.0f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        put_pair<SPLIT>(Ahi, Alo, col + i, 2 * pp, x0[i], x1[i]);
        put_pair<SPLIT>(Bhi, Blo, a.m + col + i, 2 * pp, b0 * x0[i], b1 * x1[i]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) put_pair<SPLIT>(Bhi, Blo, col + i, 2 * pp, x0[i], x1[i]);
    }
  }
}

template <bool SPLIT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_gram_tc(const TcArgs a) {
  if (a.status && *a.status != 0) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const uint32_t a_bytes = TC_M * TC_KT * 2;                 // 16 KB
  const uint32_t b_bytes = (uint32_t)a.N * TC_KT * 2;
  const uint32_t half = a_bytes + b_bytes;                   // hi (or lo) part of one buffer
  const uint32_t buf_bytes = (SPLIT ? 2 : 1) * half;
  for (uint32_t i = tid; i < 2 * buf_bytes / 16; i += TC_THREADS)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);   // padding rows stay zero
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const int64_t nch = (a.n + TC_KT - 1) / TC_KT;
  const int my = (int)((nch - blockIdx.x + gridDim.x - 1) / gridDim.x);   // chunks blockIdx.x + j * grid
  const uint32_t idesc = idesc_bf16(a.N, TC_M);
  bool ok = true;
  uint32_t phase0 = 0u, phase1 = 0u;            // mbarrier phases of the two buffers
  if (my > 0) {
    unsigned char* b0 = smem;
    tc_stage<SPLIT>(a, blockIdx.x, b0, b0 + half, b0 + a_bytes, b0 + half + a_bytes);
    proxy_fence();
  }
  __syncthreads();
  for (int j = 0; j < my; ++j) {
    const int cb = j & 1;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t base = smem_u32(smem + cb * buf_bytes);
      const uint32_t Ah = base, Bh = base + a_bytes, Al = base + half, Bl = base + half + a_bytes;
#pragma unroll
      for (int s = 0; s < TC_KT / 16; ++s) {
        const uint32_t ko = s * 256;
        umma_bf16(tmem, smem_desc(Ah + ko, 128, 1024), smem_desc(Bh + ko, 128, 1024), idesc, (j > 0 || s > 0));
        if (SPLIT) {
          umma_bf16(tmem, smem_desc(Ah + ko, 128, 1024), smem_desc(Bl + ko, 128, 1024), idesc, 1u);
          umma_bf16(tmem, smem_desc(Al + ko, 128, 1024), smem_desc(Bh + ko, 128, 1024), idesc, 1u);
        }
      }
      umma_commit(&bars[cb]);
    }
    if (j + 1 < my) {
      const int nb = (j + 1) & 1;
      if (j >= 1) {                       // buffer nb was read by the MMAs of chunk j - 1
        ok = mbar_wait(&bars[nb], nb ? phase1 : phase0) && ok;
        if (nb) phase1 ^= 1u;
        else phase0 ^= 1u;
      }
      unsigned char* bn = smem + nb * buf_bytes;
      tc_stage<SPLIT>(a, blockIdx.x + (int64_t)(j + 1) * gridDim.x, bn, bn + half, bn + a_bytes,
                      bn + half + a_bytes);
      proxy_fence();
    }
    __syncthreads();
  }
  if (my > 0) {                           // the last commit covers every MMA issued before it
    const int lb = (my - 1) & 1;
    const uint32_t ph = lb ? phase1 : phase0;
    if (!mbar_wait(&bars[lb], ph)) {
      ok = false;
      mbar_wait(&bars[lb], ph);
    }
  }
  tc_fence_after();
  // accumulator rows = columns of S (lanes), columns = columns of [A S | B S]
  const int q = wid & 3, hcol = wid >> 2;
  const int row = 32 * q + lane;
  const int m2 = 2 * a.m;
  float* out = a.partials + (size_t)blockIdx.x * a.m * m2;
  for (int c0 = hcol * (a.N / 2); c0 < (hcol + 1) * (a.N / 2); c0 += 8) {
    float v[8];
    tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
    if (row < a.m) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (c0 + i < m2) out[(size_t)row * m2 + c0 + i] = (my > 0) ? v[i] : 0.0f;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
  if (!ok && tid == 0 && a.err) atomicExch(a.err, 4);
}

// ---- three-way split with per-chunk folding (BF_GRAM_BF16X6, m <= 48) ---------------------
// x = hi + mid + lo, each BF16 (24 significant bits: an FP32 value exactly, barring
// underflow); the products hi*hi, hi*mid, mid*hi, mid*mid, hi*lo, lo*hi are accumulated
// (the dropped ones are below 2^-24 relative).  The tensor-memory accumulators start fresh
// every TC6_FOLD chunks of TC_KT pixels -- hi*hi in one region, the five smaller products
// in another -- so an FP32 accumulator sums at most TC6_FOLD TC_KT / 16 (hi*hi) or
// 5 TC6_FOLD TC_KT / 16 (corrections, 2^-8 smaller) MMA results; then the two are read with
// tcgen05.ld and added into double-float (hi, lo FP32 pair) sums in shared memory, while
// the next chunks are multiplied into the other pair of regions.  The CTA writes its sums
// as FP64 partials at the end.  Long FP32 accumulations in tensor memory, not the operands'
// rounding, are what moved the Ritz values of the one- and two-term modes.
#define TC6_MAXM 48

__device__ __forceinline__ void put_triple(unsigned char* hi, unsigned char* mid, unsigned char* lo, int row,
                                           int pix, float x0, float x1) {
  const uint32_t off = tc_off(row, pix);
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const float r0 = x0 - hf.x, r1 = x1 - hf.y;                 // exact in FP32
  const __nv_bfloat162 md = __floats2bfloat162_rn(r0, r1);
  const float2 mf = __bfloat1622float2(md);
  *reinterpret_cast<__nv_bfloat162*>(hi + off) = h;
  *reinterpret_cast<__nv_bfloat162*>(mid + off) = md;
  *reinterpret_cast<__nv_bfloat162*>(lo + off) = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
}

// Stage chunk c into the three planes of A (columns of S) and of B (columns of A S, then
// B S); the tasks and loads as in tc_stage.
__device__ void tc_stage6(const TcArgs& a, int64_t c, unsigned char* const (&A)[3], unsigned char* const (&B)[3]) {
  const int kq = a.k >> 2;
  const int per = a.nblk * (TC_KT / 2) * kq;
  const int64_t p0 = c * TC_KT;
  float4 v0[TC_MAXT], v1[TC_MAXT];
#pragma unroll
  for (int u = 0; u < TC_MAXT; ++u) {
    const int t = threadIdx.x + u * TC_THREADS;
    v0[u] = v1[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (t < 2 * per) {
      const bool is_as = t >= per;
      const int tt = is_as ? t - per : t;
      const int cq = tt % kq, rest = tt / kq;
      const int pp = rest % (TC_KT / 2), bk = rest / (TC_KT / 2);
      const int64_t p = p0 + 2 * pp;
      const float* const* blocks = is_as ? a.AS : a.S;
      const float* src = bk == 0 ? blocks[0] : (bk == 1 ? blocks[1] : blocks[2]);
      if (p < a.n) v0[u] = __ldg(reinterpret_cast<const float4*>(src + p * a.k + 4 * cq));
      if (p + 1 < a.n) v1[u] = __ldg(reinterpret_cast<const float4*>(src + (p + 1) * a.k + 4 * cq));
    }
  }
#pragma unroll
  for (int u = 0; u < TC_MAXT; ++u) {
    const int t = threadIdx.x + u * TC_THREADS;
    if (t >= 2 * per) break;
    const bool is_as = t >= per;
    const int tt = is_as ? t - per : t;
    const int cq = tt % kq, rest = tt / kq;
    const int pp = rest % (TC_KT / 2), bk = rest / (TC_KT / 2);
    const int64_t p = p0 + 2 * pp;
    const int col = bk * a.k + 4 * cq;
    const float x0[4] = {v0[u].x, v0[u].y, v0[u].z, v0[u].w}, x1[4] = {v1[u].x, v1[u].y, v1[u].z, v1[u].w};
    if (!is_as) {
      const float b0 = (a.b && p < a.n) ? a.b[p] : 1.0f;
      const float b1 = (a.b && p + 1 < a.n) ? a.b[p + 1] : 1.0f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        put_triple(A[0], A[1], A[2], col + i, 2 * pp, x0[i], x1[i]);
        put_triple(B[0], B[1], B[2], a.m + col + i, 2 * pp, b0 * x0[i], b1 * x1[i]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) put_triple(B[0], B[1], B[2], col + i, 2 * pp, x0[i], x1[i]);
    }
  }
}

// acc (hi, lo) += v without loss: Knuth's two-sum of hi and v, the error into lo.
__device__ __forceinline__ void df_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (v - bp);
  hi = s;
  lo += e;
}

#define TC6_TMEM_COLS 512         // two regions of accumulators (hi*hi and corrections): 4 N <= 384
#define TC6_FOLD 2                // chunks per accumulator region between folds

__global__ void __launch_bounds__(TC_THREADS, 1) k_gram_tc6(const TcArgs a, double* part) {
  if (a.status && *a.status != 0) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const uint32_t a_bytes = TC_M * TC_KT * 2;                 // 16 KB per plane of A
  const uint32_t b_bytes = (uint32_t)a.N * TC_KT * 2;
  const uint32_t pl = a_bytes + b_bytes;                     // one plane of A and of B
  const uint32_t buf_bytes = 3 * pl;
  const int m = a.m, m2 = 2 * a.m, ls = m2 + 1;              // row stride of the sums (no bank conflicts)
  const uint32_t N = (uint32_t)a.N;
  float* accH = reinterpret_cast<float*>(smem + 2 * buf_bytes);
  float* accL = accH + m * ls;
  for (uint32_t i = tid; i < 2 * buf_bytes / 16; i += TC_THREADS)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);   // padding rows stay zero
  for (int i = tid; i < 2 * m * ls; i += TC_THREADS) accH[i] = 0.0f;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                 "r"(TC6_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const int64_t nch = (a.n + TC_KT - 1) / TC_KT;
  const int my = (int)((nch - blockIdx.x + gridDim.x - 1) / gridDim.x);
  const uint32_t idesc = idesc_bf16(a.N, TC_M);
  bool ok = true;
  uint32_t phase[2] = {0u, 0u};
  auto planes = [&](int b, unsigned char* (&A)[3], unsigned char* (&B)[3]) {
    unsigned char* base = smem + b * buf_bytes;
    for (int q = 0; q < 3; ++q) {
      A[q] = base + q * pl;
      B[q] = base + q * pl + a_bytes;
    }
  };
  // chunk j uses smem buffer j & 1 and accumulator region (j / TC6_FOLD) & 1: hi*hi in
  // columns [2N r, 2N r + N), the corrections in [2N r + N, 2N r + 2N); a region starts
  // fresh at the first chunk of its period and is folded after the last one
  auto issue = [&](int j) {
    tc_fence_after();
    const int cb = j & 1;
    const uint32_t base = smem_u32(smem + cb * buf_bytes);
    const uint32_t Ah = base, Bh = base + a_bytes, Am = base + pl, Bm = base + pl + a_bytes;
    const uint32_t Al = base + 2 * pl, Bl = base + 2 * pl + a_bytes;
    const uint32_t tm = tmem + 2 * N * (uint32_t)((j / TC6_FOLD) & 1), tc = tm + N;
    const bool fresh = (j % TC6_FOLD) == 0;
#pragma unroll
    for (int s = 0; s < TC_KT / 16; ++s) {
      const uint32_t ko = s * 256;
      umma_bf16(tm, smem_desc(Ah + ko, 128, 1024), smem_desc(Bh + ko, 128, 1024), idesc, !fresh || s > 0);
      umma_bf16(tc, smem_desc(Ah + ko, 128, 1024), smem_desc(Bm + ko, 128, 1024), idesc, !fresh || s > 0);
      umma_bf16(tc, smem_desc(Am + ko, 128, 1024), smem_desc(Bh + ko, 128, 1024), idesc, 1u);
      umma_bf16(tc, smem_desc(Am + ko, 128, 1024), smem_desc(Bm + ko, 128, 1024), idesc, 1u);
      umma_bf16(tc, smem_desc(Ah + ko, 128, 1024), smem_desc(Bl + ko, 128, 1024), idesc, 1u);
      umma_bf16(tc, smem_desc(Al + ko, 128, 1024), smem_desc(Bh + ko, 128, 1024), idesc, 1u);
    }
    umma_commit(&bars[cb]);
  };
  if (my > 0) {
    unsigned char *A[3], *B[3];
    planes(0, A, B);
    tc_stage6(a, blockIdx.x, A, B);
    proxy_fence();
  }
  __syncthreads();
  if (my > 0 && tid == 0) issue(0);
  const int q = wid & 3, hcol = wid >> 2;                    // TMEM lane quadrant, column half
  const int row = 32 * q + lane;
  for (int j = 0; j < my; ++j) {
    const int cb = j & 1;
    if (j + 1 < my) {                  // buffer cb ^ 1 was read by chunk j - 1, already waited for
      unsigned char *A[3], *B[3];
      planes(cb ^ 1, A, B);
      tc_stage6(a, blockIdx.x + (int64_t)(j + 1) * gridDim.x, A, B);
      proxy_fence();
    }
    if (!mbar_wait(&bars[cb], phase[cb])) ok = false;
    phase[cb] ^= 1u;
    tc_fence_before();
    __syncthreads();                   // chunk j + 1 staged by every thread; chunk j's MMAs done
    tc_fence_after();
    if (j + 1 < my && tid == 0) issue(j + 1);   // its region was folded before this barrier
    // at the end of a period, fold its region (rows < m) while the next chunk is multiplied
    const bool fold = ((j + 1) % TC6_FOLD) == 0 || j + 1 == my;
    if (fold && 32 * q < m) {
      // column halves split at a multiple of 16 (the load width); columns >= 2m are ignored
      const int half = ((a.N / 2 + 15) / 16) * 16;
      const int cbeg = hcol ? half : 0, cend = hcol ? a.N : half;
      const uint32_t tm = tmem + ((uint32_t)(32 * q) << 16) + 2 * N * (uint32_t)((j / TC6_FOLD) & 1);
      for (int c0 = cbeg; c0 < cend; c0 += 16) {
        uint32_t vm[16], vc[16];
        tmem_ld16_nowait(tm + (uint32_t)c0, vm);
        tmem_ld16_nowait(tm + N + (uint32_t)c0, vc);
        tmem_wait_ld();
        if (row < m) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            if (c < m2) {
              float h = accH[row * ls + c], l = accL[row * ls + c];
              df_add(h, l, __uint_as_float(vm[i]));
              df_add(h, l, __uint_as_float(vc[i]));
              accH[row * ls + c] = h;
              accL[row * ls + c] = l;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  for (int i = tid; i < m * m2; i += TC_THREADS) {
    const int r = i / m2, c = i - r * m2;
    part[(size_t)blockIdx.x * m * m2 + i] = (double)accH[r * ls + c] + (double)accL[r * ls + c];
  }
  if (wid == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC6_TMEM_COLS) : "memory");
  }
  if (!ok && tid == 0 && a.err) atomicExch(a.err, 4);
}

// G from the CTAs' FP64 partials of k_gram_tc6: one warp per entry.
__global__ void k_gram_tc6_reduce(const double* part, int nblocks, int m, double* G, const int* status) {
  if (status && *status != 0) return;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = gtid >> 5, lanei = gtid & 31;
  const int m2 = 2 * m;
  const bool ok = e < m * m2;
  double s = 0.0;
  if (ok)
    for (int bl = lanei; bl < nblocks; bl += 32) s += part[(size_t)bl * m * m2 + e];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (!ok || lanei != 0) return;
  const int i = e / m2, jj = e - i * m2;
  if (jj < m) G[(size_t)i * m + jj] = s;
  else G[(size_t)m * m + (size_t)i * m + (jj - m)] = s;
}

// G[0] = S^T A S, G[1] = S^T B S (FP64, [2][m][m]) from the CTAs' FP32 partials: one warp
// per entry, each lane a strided share of the CTAs, combined by shuffles.
__global__ void k_gram_tc_reduce(const float* partials, int nblocks, int m, double* G, const int* status) {
  if (status && *status != 0) return;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = gtid >> 5, part = gtid & 31;
  const int m2 = 2 * m;
  const bool ok = e < m * m2;
  double s = 0.0;
  if (ok)
    for (int bl = part; bl < nblocks; bl += 32) s += (double)partials[(size_t)bl * m * m2 + e];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (!ok || part != 0) return;
  const int i = e / m2, j = e - i * m2;
  if (j < m) G[(size_t)i * m + j] = s;
  else G[(size_t)m * m + (size_t)i * m + (j - m)] = s;
}

// The bounded mbarrier wait of k_gram_tc on a barrier of its own (arrival count 1): with
// `arrive` thread 0 completes phase 0 and every thread's wait succeeds; without it nothing
// arrives and every wait gives up after `iters` polls.  out = 0 or 4 (timeout).
__global__ void k_wait_test(int iters, int arrive, int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0)
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(&bar))
                 : "memory");
  const bool ok = mbar_wait(&bar, 0u, iters);
  const bool all = __syncthreads_and(ok);
  if (threadIdx.x == 0) *out = all ? 0 : 4;
}

}  // namespace

extern "C" int bf_wait_test(int iters, int arrive, void* stream) {
  if (iters < 1 || iters > (1 << 20)) return bf_fail(BF_EINVAL, "bf_wait_test: need 1 <= iters <= 2^20");
  int* out = nullptr;
  BF_CUDA(cudaMalloc(&out, sizeof(int)));
  cudaStream_t s = (cudaStream_t)stream;
  int h = -1;
  k_wait_test<<<1, 32, 0, s>>>(iters, arrive, out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, out, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(out);
  if (e != cudaSuccess) return bf_cuda_fail(e, "bf_wait_test");
  bf_count_launches(1);
  if (h == 4) return bf_fail(BF_ETIMEOUT, "bf_wait_test: the bounded wait gave up");
  return h == 0 ? BF_OK : bf_fail(BF_ECUDA, "bf_wait_test: no result");
}

// Launch the tensor-core Gram in mode BF_GRAM_BF16, BF_GRAM_BF16X3 or BF_GRAM_BF16X6:
// returns BF_EINVAL for shapes it does not cover (k not a multiple of 4, m > 96, or m > 48
// for BF16X6), so the caller can use the FP32 kernel instead.  partials: grid * m * 2m
// doubles.
int bf_gram_tc(const float* const* S, const float* const* AS, const float* b, int nblk, int k, int64_t n,
               int mode, double* partials, int grid, double* G, const int* status, int* err, cudaStream_t s) {
  const int m = nblk * k;
  if (k % 4 != 0 || m > 96 || n < 1) return BF_EINVAL;
  if (mode == BF_GRAM_BF16X6 && m > TC6_MAXM) return BF_EINVAL;
  TcArgs a;
  for (int i = 0; i < 3; ++i) {
    a.S[i] = i < nblk ? S[i] : nullptr;
    a.AS[i] = i < nblk ? AS[i] : nullptr;
  }
  a.b = b;
  a.nblk = nblk;
  a.k = k;
  a.m = m;
  a.N = (2 * m + 15) & ~15;
  a.n = n;
  a.partials = reinterpret_cast<float*>(partials);
  a.status = status;
  a.err = err;
  const size_t plane = (size_t)TC_M * TC_KT * 2 + (size_t)a.N * TC_KT * 2;
  const int64_t nch = (n + TC_KT - 1) / TC_KT;
  grid = (int)std::min<int64_t>(grid, nch);
  const int ne = m * 2 * m;
  if (mode == BF_GRAM_BF16X6) {
    const size_t sm = 2 * 3 * plane + 2 * (size_t)m * (2 * m + 1) * sizeof(float);
    int rc = bf_smem_attr((const void*)k_gram_tc6, (int)sm, "cudaFuncSetAttribute(k_gram_tc6)");
    if (rc) return rc;
    BF_LAUNCH((k_gram_tc6<<<grid, TC_THREADS, sm, s>>>(a, partials)));
    BF_LAUNCH((k_gram_tc6_reduce<<<(ne * 32 + 255) / 256, 256, 0, s>>>(partials, grid, m, G, status)));
    BF_CUDA(cudaGetLastError());
    return BF_OK;
  }
  const bool split = (mode == BF_GRAM_BF16X3);
  const size_t sm = 2 * (split ? 2 : 1) * plane;
  {
    const int rc_ = split ? bf_smem_attr((const void*)k_gram_tc<true>, 200 * 1024, "cudaFuncSetAttribute(k_gram_tc)")
                          : bf_smem_attr((const void*)k_gram_tc<false>, 200 * 1024, "cudaFuncSetAttribute(k_gram_tc)");
    if (rc_) return rc_;
  }
  if (split) BF_LAUNCH((k_gram_tc<true><<<grid, TC_THREADS, sm, s>>>(a)));
  else BF_LAUNCH((k_gram_tc<false><<<grid, TC_THREADS, sm, s>>>(a)));
  BF_LAUNCH((k_gram_tc_reduce<<<(ne * 32 + 255) / 256, 256, 0, s>>>(a.partials, grid, m, G, status)));
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

// Test entry point (include/bf_testing.h): the tensor-core Gram of given blocks.
extern "C" int bf_gram_tc_test(const float* S0, const float* S1, const float* S2, const float* AS0, const float* AS1,
                               const float* AS2, const float* b, int nblk, int k, int64_t n, int mode, double* G,
                               void* stream) {
  if (nblk < 1 || nblk > 3 || !S0 || !AS0 || !G) return bf_fail(BF_EINVAL, "bf_gram_tc_test: bad arguments");
  if (k % 4 != 0 || nblk * k > 96) return bf_fail(BF_EINVAL, "bf_gram_tc_test: need k % 4 == 0 and nblk * k <= 96");
  if (mode != BF_GRAM_BF16 && mode != BF_GRAM_BF16X3 && mode != BF_GRAM_BF16X6)
    return bf_fail(BF_EINVAL, "bf_gram_tc_test: bad mode");
  if (mode == BF_GRAM_BF16X6 && nblk * k > TC6_MAXM)
    return bf_fail(BF_EINVAL, "bf_gram_tc_test: BF_GRAM_BF16X6 needs nblk * k <= 48");
  const float* S[3] = {S0, S1, S2};
  const float* AS[3] = {AS0, AS1, AS2};
  int dev = 0, nsm = 0;
  BF_CUDA(cudaGetDevice(&dev));
  BF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int m = nblk * k;
  double* part = nullptr;
  int* flag = nullptr;
  BF_CUDA(cudaMalloc(&part, (size_t)nsm * m * 2 * m * sizeof(double)));
  BF_CUDA(cudaMalloc(&flag, sizeof(int)));
  cudaStream_t s = (cudaStream_t)stream;
  BF_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  int rc = bf_gram_tc(S, AS, b, nblk, k, n, mode, part, nsm, G, flag, flag, s);
  int h = 0;
  if (rc == BF_OK) {
    BF_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    BF_CUDA(cudaStreamSynchronize(s));
  }
  cudaFree(part);
  cudaFree(flag);
  if (rc) return rc;
  if (h) return bf_fail(BF_ETIMEOUT, "bf_gram_tc_test: a bounded wait gave up");
  return BF_OK;
}
