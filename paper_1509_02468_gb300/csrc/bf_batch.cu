// Batched CG filters (Algorithm 2, Section 5) over many instances of uneven size -- images
// and signals -- in one launch sequence, captured once as a CUDA graph and replayed.
//
// All instances' tiles form one work list per window shape (7 x 7 images, 11-tap signals,
// 5-point lattices); one block handles one tile, so a launch covers the whole batch and
// the GPU stays full however small the single instances are.  The tiles of an instance
// are consecutive in its list; the last block of an instance to finish (per-instance
// arrival counter) sums that instance's block partials in a fixed order and updates its
// FP64 scalars (alpha, beta, the stopping tests), exactly as the single-instance kernels
// do for the whole grid.  Per iteration: one direction kernel (p, q = (L + sigma I) p,
// p^T q, alpha) per shape class and one update kernel (x, r, s = T r, the sums, beta) per
// class.  Instances that have stopped return at once.
//
// The autotuner (bf_batch_tune) times the candidate tile shapes of the image class on the
// batch itself and keeps the fastest for later runs.
#include <math.h>

#include <algorithm>
#include <string>
#include <thread>
#include <vector>

#include "bf_internal.cuh"
#include "bf_window_fast.cuh"

namespace {

enum { B_RUN = 0, B_CONV = 1, B_BREAK = 2, B_NONFINITE = 3 };

struct BState {
  double sr, ss, rr, pq, alpha, beta, ref2;
  int status, iter;
};

struct BInst {
  int nx, ny;
  int64_t n;
  const float* guide;
  const float* dinv;      // NULL: identity preconditioner
  const float* x0;
  float* x;
  float* r;
  float* s;
  float* q;
  float* p[2];
  int job0, njobs;        // range in the class work list (per tile shape)
  int upd0, nupd;         // range in the class update list (chunks of BUPD_CHUNK samples)
  unsigned counter;
  BState st;
};

struct BJob {
  int inst;
  int bx, by;             // operator jobs: first tile; update jobs: first sample, count
  int nt;                 // operator jobs: tiles in the group (consecutive along x)
};

struct BArgs {
  BInst* inst;
  const BJob* jobs;
  double* partials;       // [jobs][4] of this class
  float shift;
  double tol2;
  int beta_mode;
};

// Last block of an instance: sums the instance's partials (j0 .. j0 + nj of the launch's
// list) in order.
template <int NV>
__device__ __forceinline__ bool inst_sum_last(const double (&blk)[NV], const BArgs& a, BInst& in, int job,
                                              double (&tot)[NV], int* is_last, int j0, int nj) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) a.partials[(size_t)job * 4 + j] = blk[j];
    __threadfence();
    const unsigned prev = atomicAdd(&in.counter, 1u);
    *is_last = (prev == (unsigned)nj - 1);
  }
  __syncthreads();
  if (!*is_last) return false;
  __threadfence();
  double v[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = 0.0;
  for (int q = threadIdx.x; q < nj; q += BF_THREADS) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] += ((volatile double*)a.partials)[(size_t)(j0 + q) * 4 + j];
  }
  __shared__ double red2[NV * (BF_THREADS / 32)];
  block_sum<NV, double>(v, red2, tot);
  if (threadIdx.x == 0) in.counter = 0u;
  return threadIdx.x == 0;
}

template <class SH, class F>
__device__ __forceinline__ void bstage(const BInst& in, int bx, int by, float* sx, float* sg, float* sval, F f) {
  for (int hp = threadIdx.x; hp < SH::hp; hp += BF_THREADS) {
    const int hy = hp / SH::hw, hx = hp - hy * SH::hw;
    const int gy = by - SH::ry + hy, gx = bx - SH::rx + hx;
    const bool inside = gx >= 0 && gx < in.nx && gy >= 0 && gy < in.ny;
    float v = 0.0f, gv = 0.0f;
    if (inside) {
      const int64_t gp = (int64_t)gy * in.nx + gx;
      v = f(gp);
      gv = in.guide[gp];
    }
    sx[hp] = v;
    sg[hp] = gv;
    sval[hp] = inside ? 1.0f : 0.0f;
  }
}

// r = -L x0, x = x0, s = T r; sums s^T r, s^T s, r^T r, x0^T x0; state of the instance.
template <class SH>
__device__ __forceinline__ void bcg_init_job(const Geom<float>& g, const BArgs& a, int job, unsigned char* smem) {
  __shared__ double red[4 * (BF_THREADS / 32)];
  __shared__ int last;
  float* sx = reinterpret_cast<float*>(smem);
  float* sg = sx + SH::hp;
  float* sval = sg + SH::hp;
  const BJob jb = a.jobs[job];
  BInst& in = a.inst[jb.inst];
  const int lx = threadIdx.x % SH::tw, ly = threadIdx.x / SH::tw;
  const int hp0 = (ly + SH::ry) * SH::hw + (lx + SH::rx);
  float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int t = 0; t < jb.nt; ++t) {                 // the group's tiles, one after another
    const int bx = jb.bx + t * SH::tw;
    const bool mask = !(bx - SH::rx >= 0 && bx + SH::tw + SH::rx <= in.nx && jb.by - SH::ry >= 0 &&
                        jb.by + SH::th + SH::ry <= in.ny);
    if (t) __syncthreads();                         // the previous tile is read
    bstage<SH>(in, bx, jb.by, sx, sg, sval, [&](int64_t gp) { return in.x0[gp]; });
    __syncthreads();
    const int x = bx + lx, y = jb.by + ly;
    if (x < in.nx && y < in.ny) {
      const int64_t i = (int64_t)y * in.nx + x;
      float xi[1] = {sx[hp0]}, acc[1] = {0.0f}, ws = 0.0f;
      window_fast<SH, 1, false>(g, hp0, i, in.nx, sg, sval, mask, reinterpret_cast<const Vec<float, 1>*>(sx),
                                nullptr, BF_W_ONTHEFLY, in.n, xi, acc, ws);
      const float r = -acc[0];
      const float sv = in.dinv ? r * in.dinv[i] : r;
      in.x[i] = xi[0];
      in.r[i] = r;
      in.s[i] = sv;
      v[0] += sv * r;
      v[1] += sv * sv;
      v[2] += r * r;
      v[3] += xi[0] * xi[0];
    }
  }
  double blk[4], tot[4];
  block_sum<4, float>(v, red, blk);
  if (inst_sum_last<4>(blk, a, in, job, tot, &last, in.job0, in.njobs)) {
    BState& st = in.st;
    st.sr = tot[0];
    st.ss = tot[1];
    st.rr = tot[2];
    const double b2 = (double)a.shift * (double)a.shift * tot[3];
    st.ref2 = b2 > 0.0 ? b2 : tot[2];
    st.beta = 0.0;
    st.alpha = 0.0;
    st.iter = 0;
    st.status = (isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2])) ? B_RUN : B_NONFINITE;
  }
}

template <class SH>
__global__ void __launch_bounds__(BF_THREADS) k_bcg_init(const Geom<float> g, const BArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  bcg_init_job<SH>(g, a, blockIdx.x, smem);
}

// p = s + beta p_old on tile + halo (first iteration: p = s), q = (L + shift I) p, p^T q, alpha.
// (An instance's status changes only in the last block of its jobs in a phase, after all
// others have finished theirs, so every block reads the same value.)
template <class SH>
__device__ __forceinline__ void bcg_dir_job(const Geom<float>& g, const BArgs& a, int job, unsigned char* smem) {
  const BJob jb = a.jobs[job];
  BInst& in = a.inst[jb.inst];
  if (in.st.status != B_RUN) return;
  __shared__ double red[BF_THREADS / 32];
  __shared__ int last;
  float* sx = reinterpret_cast<float*>(smem);
  float* sg = sx + SH::hp;
  float* sval = sg + SH::hp;
  const int it = in.st.iter;
  const float* p_old = in.p[it & 1];
  float* p_new = in.p[(it + 1) & 1];
  const float beta = (float)in.st.beta;
  const int lx = threadIdx.x % SH::tw, ly = threadIdx.x / SH::tw;
  const int hp0 = (ly + SH::ry) * SH::hw + (lx + SH::rx);
  float v[1] = {0.0f};
  for (int t = 0; t < jb.nt; ++t) {                 // the group's tiles, one after another
    const int bx = jb.bx + t * SH::tw;
    const bool mask = !(bx - SH::rx >= 0 && bx + SH::tw + SH::rx <= in.nx && jb.by - SH::ry >= 0 &&
                        jb.by + SH::th + SH::ry <= in.ny);
    if (t) __syncthreads();                         // the previous tile is read
    if (it == 0)
      bstage<SH>(in, bx, jb.by, sx, sg, sval, [&](int64_t gp) { return in.s[gp]; });
    else
      bstage<SH>(in, bx, jb.by, sx, sg, sval, [&](int64_t gp) { return fmaf(beta, p_old[gp], in.s[gp]); });
    __syncthreads();
    const int x = bx + lx, y = jb.by + ly;
    if (x < in.nx && y < in.ny) {
      const int64_t i = (int64_t)y * in.nx + x;
      float pi[1] = {sx[hp0]}, acc[1] = {0.0f}, ws = 0.0f;
      window_fast<SH, 1, false>(g, hp0, i, in.nx, sg, sval, mask, reinterpret_cast<const Vec<float, 1>*>(sx),
                                nullptr, BF_W_ONTHEFLY, in.n, pi, acc, ws);
      const float q = fmaf(a.shift, pi[0], acc[0]);
      p_new[i] = pi[0];
      in.q[i] = q;
      v[0] += pi[0] * q;
    }
  }
  double blk[1], tot[1];
  block_sum<1, float>(v, red, blk);
  if (inst_sum_last<1>(blk, a, in, job, tot, &last, in.job0, in.njobs)) {
    BState& st = in.st;
    st.pq = tot[0];
    if (st.sr == 0.0) st.status = B_CONV;
    else if (!isfinite(tot[0])) st.status = B_NONFINITE;
    else if (!(tot[0] > 0.0)) st.status = B_BREAK;
    else st.alpha = st.sr / tot[0];
  }
}

template <class SH>
__global__ void __launch_bounds__(BF_THREADS) k_bcg_dir(const Geom<float> g, const BArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  bcg_dir_job<SH>(g, a, blockIdx.x, smem);
}

// x += alpha p, r -= alpha q, s = T r on a chunk of up to BUPD_CHUNK consecutive samples of
// one instance; sums; beta and the stopping tests.
__device__ __forceinline__ void bcg_update_job(const BArgs& a, int job) {
  const BJob jb = a.jobs[job];
  BInst& in = a.inst[jb.inst];
  if (in.st.status != B_RUN) return;
  __shared__ double red[4 * (BF_THREADS / 32)];
  __shared__ int last;
  const float alpha = (float)in.st.alpha;
  const float* p = in.p[(in.st.iter + 1) & 1];
  const int64_t i0 = jb.bx, i1 = i0 + jb.by;
  float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int64_t i = i0 + threadIdx.x; i < i1; i += BF_THREADS) {
    const float pi = p[i], q = in.q[i];
    in.x[i] = fmaf(alpha, pi, in.x[i]);
    const float r = fmaf(-alpha, q, in.r[i]);
    const float sv = in.dinv ? r * in.dinv[i] : r;
    in.r[i] = r;
    in.s[i] = sv;
    v[0] += sv * r;
    v[1] += sv * q;
    v[2] += sv * sv;
    v[3] += r * r;
  }
  double blk[4], tot[4];
  block_sum<4, float>(v, red, blk);
  if (inst_sum_last<4>(blk, a, in, job, tot, &last, in.upd0, in.nupd)) {
    BState& st = in.st;
    st.iter += 1;
    const double den = (a.beta_mode == BF_BETA_PRINTED) ? st.ss : st.sr;
    st.beta = -st.alpha * tot[1] / den;
    st.sr = tot[0];
    st.ss = tot[2];
    st.rr = tot[3];
    if (!(isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2]) && isfinite(tot[3]))) st.status = B_NONFINITE;
    else if (a.tol2 > 0.0 && tot[3] <= a.tol2 * st.ref2) st.status = B_CONV;
  }
}

template <class SH>
__global__ void __launch_bounds__(BF_THREADS) k_bcg_update(const BArgs a) {
  bcg_update_job(a, blockIdx.x);
}

// candidate tile shapes of the image class (the autotuner's choices)
typedef WinShapeT<3, 3, false, 32, 8> R3_32x8;
typedef WinShapeT<3, 3, false, 64, 4> R3_64x4;
typedef WinShapeT<3, 3, false, 16, 16> R3_16x16;
enum { CLS_R3 = 0, CLS_R5 = 1, CLS_X1 = 2, NCLS = 3 };
#define BUPD_CHUNK 4096           // samples per block of the update kernel (16 per thread)
#define BTILE_GROUP 8             // consecutive tiles of one row per block of the operator kernels
const int R3_TW[3] = {32, 64, 16}, R3_TH[3] = {8, 4, 16};

// ---- persistent form: one cooperative launch for the whole run ----------------------------
// Every CTA walks the work lists of all classes phase by phase (start; then per iteration
// the direction jobs, then the update jobs), the phases separated by a grid barrier.  The
// per-instance reductions are those of the per-phase kernels (same jobs, same order), so
// the results are identical.  The barrier is bounded: a CTA that waits longer than
// BAR_WAIT_NS records a timeout and leaves; so does every other CTA at its next wait.
#define BAR_WAIT_NS 1000000000ull      // 1 s

struct BGeoms {
  Geom<float> g[NCLS];
};

struct BPArgs {
  BArgs op[NCLS];                      // operator work lists
  BArgs up[NCLS];                      // update work lists
  int njobs[NCLS], nupd[NCLS];
  int has[NCLS];
  int kmax;
  unsigned* bar;                       // [0]: arrivals, [1]: generation
  int* err;                            // 1: a barrier wait gave up
  int skip;                            // testing: CTA 0 leaves without arriving at barrier 1
};

__device__ __forceinline__ unsigned long long b_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a bounded wait; returns false (block-uniform) when it gave up or
// an earlier wait of the run did.
__device__ bool b_grid_barrier(const BPArgs& pa, int index) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = *(volatile int*)pa.err == 0;
    if (ok && pa.skip && index == 1 && blockIdx.x == 0) ok = 0;   // testing: never arrives
    if (ok) {
      volatile unsigned* gen = pa.bar + 1;
      const unsigned g0 = *gen;
      __threadfence();
      if (atomicAdd(pa.bar, 1u) == gridDim.x - 1) {
        pa.bar[0] = 0u;
        __threadfence();
        atomicAdd(pa.bar + 1, 1u);
      } else {
        const unsigned long long t0 = b_now_ns();
        while (*gen == g0) {
          if (*(volatile int*)pa.err) {       // another CTA gave up: leave now
            ok = 0;
            break;
          }
          if (b_now_ns() - t0 > BAR_WAIT_NS) {
            atomicExch(pa.err, 1);
            ok = 0;
            break;
          }
        }
      }
      __threadfence();
    }
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

template <class SHR3>
__device__ __forceinline__ void b_phase(const BGeoms& G, const BPArgs& pa, int phase, unsigned char* smem) {
  for (int c = 0; c < NCLS; ++c) {
    if (!pa.has[c]) continue;
    const int nj = phase == 2 ? pa.nupd[c] : pa.njobs[c];
    for (int job = blockIdx.x; job < nj; job += gridDim.x) {
      if (phase == 2) {
        bcg_update_job(pa.up[c], job);
      } else if (c == CLS_R3) {
        if (phase == 0) bcg_init_job<SHR3>(G.g[c], pa.op[c], job, smem);
        else bcg_dir_job<SHR3>(G.g[c], pa.op[c], job, smem);
      } else if (c == CLS_R5) {
        if (phase == 0) bcg_init_job<ShapeR5>(G.g[c], pa.op[c], job, smem);
        else bcg_dir_job<ShapeR5>(G.g[c], pa.op[c], job, smem);
      } else {
        if (phase == 0) bcg_init_job<ShapeX1>(G.g[c], pa.op[c], job, smem);
        else bcg_dir_job<ShapeX1>(G.g[c], pa.op[c], job, smem);
      }
      __syncthreads();                 // the job's shared memory is free
    }
  }
}

template <class SHR3>
__global__ void __launch_bounds__(BF_THREADS) k_bcg_persistent(const __grid_constant__ BGeoms G, const BPArgs pa) {
  extern __shared__ __align__(16) unsigned char smem[];
  int bi = 0;
  b_phase<SHR3>(G, pa, 0, smem);
  if (!b_grid_barrier(pa, ++bi)) return;
  for (int it = 0; it < pa.kmax; ++it) {
    b_phase<SHR3>(G, pa, 1, smem);
    if (!b_grid_barrier(pa, ++bi)) return;
    b_phase<SHR3>(G, pa, 2, smem);
    if (it + 1 < pa.kmax && !b_grid_barrier(pa, ++bi)) return;
  }
}

}  // namespace

struct bf_batch {
  int count;
  int device;
  std::vector<const bf_graph*> graphs;
  std::vector<int> cls;              // class of each instance
  Geom<float> geom[NCLS];
  bool has[NCLS];
  int r3_variant;                    // tile shape of the image class (autotuned)
  int njobs[NCLS];                   // operator jobs (groups of tiles) per class
  int64_t ntiles[NCLS];              // operator tiles per class
  int nupd[NCLS];                    // update chunks per class
  BInst* d_inst;                     // [count]
  BJob* d_jobs[NCLS];
  BJob* d_upd[NCLS];                 // update chunks {instance, first sample, count}
  double* d_part[NCLS];
  void* d_vec;                       // r, s, q, p0, p1 of every instance
  void* d_bar;                       // persistent run: barrier counters and timeout flag
  std::vector<cudaStream_t> lob_streams;   // batched LOBPCG: internal streams
  std::vector<cudaEvent_t> lob_events;     // one per internal stream, and one for the start
  std::vector<BInst> h_inst;
  // captured run
  cudaGraphExec_t exec;
  uint64_t graph_kernels;            // kernels in the captured graph
  int exec_kmax;
  bf_cg_opts exec_opts;
  int exec_variant;
};

namespace {

template <class SH>
size_t bsmem() { return 3 * SH::hp * sizeof(float); }

int build_jobs(bf_batch* b) {
  std::vector<BJob> jobs[NCLS], upd[NCLS];
  for (int c = 0; c < NCLS; ++c) b->ntiles[c] = 0;
  for (int i = 0; i < b->count; ++i) {
    const int c = b->cls[i];
    const int tw = (c == CLS_R3) ? R3_TW[b->r3_variant] : (c == CLS_R5 ? ShapeR5::tw : ShapeX1::tw);
    const int th = (c == CLS_R3) ? R3_TH[b->r3_variant] : (c == CLS_R5 ? ShapeR5::th : ShapeX1::th);
    BInst& in = b->h_inst[i];
    in.job0 = (int)jobs[c].size();
    for (int by = 0; by < in.ny; by += th)
      for (int bx = 0; bx < in.nx; bx += BTILE_GROUP * tw) {
        const int nt = std::min(BTILE_GROUP, (in.nx - bx + tw - 1) / tw);
        jobs[c].push_back(BJob{i, bx, by, nt});
        b->ntiles[c] += nt;
      }
    in.njobs = (int)jobs[c].size() - in.job0;
    in.upd0 = (int)upd[c].size();
    for (int64_t i0 = 0; i0 < in.n; i0 += BUPD_CHUNK)
      upd[c].push_back(BJob{i, (int)i0, (int)std::min<int64_t>(BUPD_CHUNK, in.n - i0), 0});
    in.nupd = (int)upd[c].size() - in.upd0;
  }
  for (int c = 0; c < NCLS; ++c) {
    if (b->d_jobs[c]) cudaFree(b->d_jobs[c]);
    if (b->d_upd[c]) cudaFree(b->d_upd[c]);
    if (b->d_part[c]) cudaFree(b->d_part[c]);
    b->d_jobs[c] = nullptr;
    b->d_upd[c] = nullptr;
    b->d_part[c] = nullptr;
    b->njobs[c] = (int)jobs[c].size();
    b->nupd[c] = (int)upd[c].size();
    if (jobs[c].empty()) continue;
    const size_t np = std::max(jobs[c].size(), upd[c].size());
    BF_CUDA(cudaMalloc(&b->d_jobs[c], jobs[c].size() * sizeof(BJob)));
    BF_CUDA(cudaMalloc(&b->d_upd[c], upd[c].size() * sizeof(BJob)));
    BF_CUDA(cudaMalloc(&b->d_part[c], np * 4 * sizeof(double)));
    BF_CUDA(cudaMemcpy(b->d_jobs[c], jobs[c].data(), jobs[c].size() * sizeof(BJob), cudaMemcpyHostToDevice));
    BF_CUDA(cudaMemcpy(b->d_upd[c], upd[c].data(), upd[c].size() * sizeof(BJob), cudaMemcpyHostToDevice));
  }
  return BF_OK;
}

BArgs make_args(const bf_batch* b, int c, const bf_cg_opts& o) {
  BArgs a;
  a.inst = b->d_inst;
  a.jobs = b->d_jobs[c];
  a.partials = b->d_part[c];
  a.shift = (float)o.shift;
  a.tol2 = o.tol > 0 ? o.tol * o.tol : 0.0;
  a.beta_mode = o.beta;
  return a;
}

template <class SH>
void launch_phase(int phase, const bf_batch* b, int c, const BArgs& a, cudaStream_t s) {
  const unsigned nj = (unsigned)b->njobs[c];
  if (!nj) return;
  if (phase == 0) BF_LAUNCH(k_bcg_init<SH><<<nj, BF_THREADS, bsmem<SH>(), s>>>(b->geom[c], a));
  else if (phase == 1) BF_LAUNCH(k_bcg_dir<SH><<<nj, BF_THREADS, bsmem<SH>(), s>>>(b->geom[c], a));
  else {
    BArgs au = a;
    au.jobs = b->d_upd[c];
    BF_LAUNCH(k_bcg_update<SH><<<(unsigned)b->nupd[c], BF_THREADS, 0, s>>>(au));
  }
}

void launch_all(int phase, const bf_batch* b, const bf_cg_opts& o, int r3v, cudaStream_t s) {
  for (int c = 0; c < NCLS; ++c) {
    if (!b->has[c]) continue;
    const BArgs a = make_args(b, c, o);
    if (c == CLS_R3) {
      if (r3v == 0) launch_phase<R3_32x8>(phase, b, c, a, s);
      else if (r3v == 1) launch_phase<R3_64x4>(phase, b, c, a, s);
      else launch_phase<R3_16x16>(phase, b, c, a, s);
    } else if (c == CLS_R5) {
      launch_phase<ShapeR5>(phase, b, c, a, s);
    } else {
      launch_phase<ShapeX1>(phase, b, c, a, s);
    }
  }
}

int enqueue_run(const bf_batch* b, int kmax, const bf_cg_opts& o, cudaStream_t s) {
  launch_all(0, b, o, b->r3_variant, s);
  for (int it = 0; it < kmax; ++it) {
    launch_all(1, b, o, b->r3_variant, s);
    launch_all(2, b, o, b->r3_variant, s);
  }
  BF_CUDA(cudaGetLastError());
  return BF_OK;
}

bool same_opts(const bf_cg_opts& a, const bf_cg_opts& b) {
  return a.precond == b.precond && a.beta == b.beta && a.shift == b.shift && a.tol == b.tol;
}

}  // namespace

extern "C" int bf_batch_create(const bf_graph* const* graphs, int count, bf_batch** out) {
  if (!graphs || !out || count < 1) return bf_fail(BF_EINVAL, "bf_batch_create: need graphs and count >= 1");
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!graphs[i] || graphs[i]->kind != BF_KIND_BILATERAL)
      return bf_fail(BF_EINVAL, "bf_batch_create: the batched driver takes bilateral graphs");
  bf_batch* b = new bf_batch();
  b->count = count;
  b->graphs.assign(graphs, graphs + count);
  b->cls.resize(count);
  b->h_inst.resize(count);
  b->r3_variant = 0;
  b->d_inst = nullptr;
  b->d_vec = nullptr;
  b->d_bar = nullptr;
  b->exec = nullptr;
  b->graph_kernels = 0;
  b->exec_kmax = -1;
  b->exec_variant = -1;
  for (int c = 0; c < NCLS; ++c) {
    b->has[c] = false;
    b->d_jobs[c] = nullptr;
    b->d_upd[c] = nullptr;
    b->d_part[c] = nullptr;
    b->njobs[c] = 0;
    b->ntiles[c] = 0;
    b->nupd[c] = 0;
  }
  cudaGetDevice(&b->device);
  size_t vtot = 0;
  for (int i = 0; i < count; ++i) {
    const bf_graph* g = graphs[i];
    if (!g || g->esize != 4 || g->p.weight_mode != BF_W_ONTHEFLY) {
      delete b;
      return bf_fail(BF_EINVAL, "bf_batch_create: every graph must be FP32 with on-the-fly weights");
    }
    const int fs = fast_shape(g);
    const int c = fs == FAST_R3_2D ? CLS_R3 : fs == FAST_R5_1D ? CLS_R5 : fs == FAST_CROSS1 ? CLS_X1 : -1;
    if (c < 0) {
      delete b;
      return bf_fail(BF_EINVAL, "bf_batch_create: window must be 7x7 (images), 11 taps (signals) or the 5-point cross");
    }
    if (!b->has[c]) {
      b->has[c] = true;
      b->geom[c] = g->gf;
    } else {
      const Geom<float>& r = b->geom[c];
      bool same = r.a_r == g->gf.a_r;
      for (int t = 0; t < BF_MAX_BOX && same; ++t) same = (r.ls[t] == g->gf.ls[t]);
      if (!same) {
        delete b;
        return bf_fail(BF_EINVAL, "bf_batch_create: instances of one window shape must share sigma_s and sigma_r");
      }
    }
    b->cls[i] = c;
    BInst& in = b->h_inst[i];
    memset(&in, 0, sizeof(in));
    in.nx = g->nx;
    in.ny = g->ny;
    in.n = g->n;
    in.guide = (const float*)g->guide;
    vtot += ((size_t)g->n * sizeof(float) + 255) & ~(size_t)255;
  }
  cudaError_t e = cudaMalloc(&b->d_vec, 5 * vtot);
  if (e != cudaSuccess) {
    delete b;
    return bf_cuda_fail(e, "cudaMalloc(batch vectors)");
  }
  char* p = (char*)b->d_vec;
  for (int i = 0; i < count; ++i) {
    const size_t vb = ((size_t)b->h_inst[i].n * sizeof(float) + 255) & ~(size_t)255;
    BInst& in = b->h_inst[i];
    in.r = (float*)p; p += vb;
    in.s = (float*)p; p += vb;
    in.q = (float*)p; p += vb;
    in.p[0] = (float*)p; p += vb;
    in.p[1] = (float*)p; p += vb;
  }
  e = cudaMalloc(&b->d_inst, count * sizeof(BInst));
  if (e != cudaSuccess) {
    cudaFree(b->d_vec);
    delete b;
    return bf_cuda_fail(e, "cudaMalloc(batch instances)");
  }
  int rc = build_jobs(b);
  if (rc) return rc;
  *out = b;
  return BF_OK;
}

extern "C" int bf_batch_free(bf_batch* b) {
  if (!b) return BF_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (int c = 0; c < NCLS; ++c) {
    if (b->d_jobs[c]) cudaFree(b->d_jobs[c]);
    if (b->d_upd[c]) cudaFree(b->d_upd[c]);
    if (b->d_part[c]) cudaFree(b->d_part[c]);
  }
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->d_vec) cudaFree(b->d_vec);
  if (b->d_bar) cudaFree(b->d_bar);
  for (cudaStream_t st : b->lob_streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->lob_events) cudaEventDestroy(ev);
  delete b;
  return BF_OK;
}

extern "C" int bf_batch_tiles(const bf_batch* b, int64_t* tiles_out, int* variant_out) {
  if (!b) return bf_fail(BF_EINVAL, "bf_batch_tiles: NULL batch");
  if (tiles_out) *tiles_out = b->ntiles[0] + b->ntiles[1] + b->ntiles[2];
  if (variant_out) *variant_out = b->r3_variant;
  return BF_OK;
}

static int batch_upload(bf_batch* b, const float* const* x0, float* const* x_out, const bf_cg_opts& o,
                        cudaStream_t s) {
  for (int i = 0; i < b->count; ++i) {
    BInst& in = b->h_inst[i];
    const bf_graph* g = b->graphs[i];
    in.x0 = x0[i];
    in.x = x_out[i];
    in.dinv = o.precond == BF_PRECOND_JACOBI ? (const float*)g->dinv : nullptr;
    in.counter = 0;
    memset(&in.st, 0, sizeof(in.st));
  }
  BF_CUDA(cudaMemcpyAsync(b->d_inst, b->h_inst.data(), b->count * sizeof(BInst), cudaMemcpyHostToDevice, s));
  return BF_OK;
}

extern "C" int bf_batch_cg(bf_batch* b, const float* const* x0, float* const* x_out, int kmax,
                           const bf_cg_opts* opts, bf_info* infos, void* stream) {
  if (!b || !x0 || !x_out) return bf_fail(BF_EINVAL, "bf_batch_cg: NULL argument");
  if (kmax < 0) return bf_fail(BF_EINVAL, "bf_batch_cg: kmax < 0");
  bf_cg_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.precond != BF_PRECOND_JACOBI && o.precond != BF_PRECOND_IDENTITY)
    return bf_fail(BF_EINVAL, "bf_batch_cg: precond must be Jacobi or identity");
  if (o.beta != BF_BETA_FLEXIBLE && o.beta != BF_BETA_PRINTED) return bf_fail(BF_EINVAL, "bf_batch_cg: bad beta");
  if (!(o.shift >= 0.0) || !(o.tol >= 0.0)) return bf_fail(BF_EINVAL, "bf_batch_cg: shift and tol must be >= 0");
  for (int i = 0; i < b->count; ++i)
    if (!x0[i] || !x_out[i]) return bf_fail(BF_EINVAL, "bf_batch_cg: NULL instance vector");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = batch_upload(b, x0, x_out, o, s);
  if (rc) return rc;
  // the whole run is one CUDA graph, captured once per (kmax, options, tile shape)
  if (!b->exec || b->exec_kmax != kmax || !same_opts(b->exec_opts, o) || b->exec_variant != b->r3_variant) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    cudaStream_t cs;
    BF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    BF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const uint64_t c0 = bf_launch_count();
    rc = enqueue_run(b, kmax, o, cs);
    b->graph_kernels = bf_launch_count() - c0;   // captured, not run: counted per replay
    bf_count_launches(-(int)b->graph_kernels);
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (rc) return rc;
    if (e != cudaSuccess) return bf_cuda_fail(e, "cudaStreamEndCapture(batch)");
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bf_cuda_fail(e, "cudaGraphInstantiate(batch)");
    b->exec_kmax = kmax;
    b->exec_opts = o;
    b->exec_variant = b->r3_variant;
  }
  BF_CUDA(cudaGraphLaunch(b->exec, s));
  bf_count_launches((int)b->graph_kernels);
  if (infos) {
    std::vector<BInst> h(b->count);
    BF_CUDA(cudaMemcpyAsync(h.data(), b->d_inst, b->count * sizeof(BInst), cudaMemcpyDeviceToHost, s));
    BF_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < b->count; ++i) {
      const BState& st = h[i].st;
      infos[i].iters = st.iter;
      infos[i].status = st.status == B_CONV ? BF_CG_CONVERGED : (st.status == B_BREAK ? BF_CG_BREAKDOWN : 0);
      infos[i].restarts = 0;
      infos[i].reserved = st.status == B_NONFINITE ? 1 : 0;
      infos[i].rnorm = sqrt(st.rr);
      infos[i].ref = sqrt(st.ref2);
    }
  }
  return BF_OK;
}

template <class SHR3>
static int launch_persistent(bf_batch* b, const BGeoms& G, const BPArgs& pa, size_t smem, cudaStream_t s) {
  const void* fn = (const void*)k_bcg_persistent<SHR3>;
  int rc = bf_smem_attr(fn, (int)smem, "cudaFuncSetAttribute(k_bcg_persistent)");
  if (rc) return rc;
  int per = 0, nsm = 0;
  BF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bcg_persistent<SHR3>, BF_THREADS, smem));
  BF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
  int most = 1;
  for (int c = 0; c < NCLS; ++c) most = std::max(most, std::max(b->njobs[c], b->nupd[c]));
  const int grid = std::max(1, std::min(per * nsm, most));
  BGeoms g = G;
  BPArgs a = pa;
  void* args[] = {(void*)&g, (void*)&a};
  BF_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(BF_THREADS), args, smem, s));
  bf_count_launches(1);
  return BF_OK;
}

// The persistent run: one cooperative launch; skip (testing) makes CTA 0 leave before its
// first barrier.
static int batch_run_persistent(bf_batch* b, const float* const* x0, float* const* x_out, int kmax,
                                const bf_cg_opts* opts, bf_info* infos, int skip, cudaStream_t s) {
  if (!b || !x0 || !x_out) return bf_fail(BF_EINVAL, "bf_batch_cg_persistent: NULL argument");
  if (kmax < 0) return bf_fail(BF_EINVAL, "bf_batch_cg_persistent: kmax < 0");
  bf_cg_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.precond != BF_PRECOND_JACOBI && o.precond != BF_PRECOND_IDENTITY)
    return bf_fail(BF_EINVAL, "bf_batch_cg_persistent: precond must be Jacobi or identity");
  if (o.beta != BF_BETA_FLEXIBLE && o.beta != BF_BETA_PRINTED)
    return bf_fail(BF_EINVAL, "bf_batch_cg_persistent: bad beta");
  if (!(o.shift >= 0.0) || !(o.tol >= 0.0))
    return bf_fail(BF_EINVAL, "bf_batch_cg_persistent: shift and tol must be >= 0");
  for (int i = 0; i < b->count; ++i)
    if (!x0[i] || !x_out[i]) return bf_fail(BF_EINVAL, "bf_batch_cg_persistent: NULL instance vector");
  if (!b->d_bar) BF_CUDA(cudaMalloc(&b->d_bar, 4 * sizeof(unsigned)));
  int rc = batch_upload(b, x0, x_out, o, s);
  if (rc) return rc;
  BF_CUDA(cudaMemsetAsync(b->d_bar, 0, 4 * sizeof(unsigned), s));
  BGeoms G;
  BPArgs pa;
  memset(&pa, 0, sizeof(pa));
  size_t smem = 0;
  for (int c = 0; c < NCLS; ++c) {
    G.g[c] = b->geom[c];
    pa.has[c] = b->has[c] ? 1 : 0;
    if (!b->has[c]) continue;
    pa.op[c] = make_args(b, c, o);
    pa.up[c] = pa.op[c];
    pa.up[c].jobs = b->d_upd[c];
    pa.njobs[c] = b->njobs[c];
    pa.nupd[c] = b->nupd[c];
  }
  if (b->has[CLS_R3]) {
    const size_t r3[3] = {bsmem<R3_32x8>(), bsmem<R3_64x4>(), bsmem<R3_16x16>()};
    smem = std::max(smem, r3[b->r3_variant]);
  }
  if (b->has[CLS_R5]) smem = std::max(smem, bsmem<ShapeR5>());
  if (b->has[CLS_X1]) smem = std::max(smem, bsmem<ShapeX1>());
  pa.kmax = kmax;
  pa.bar = reinterpret_cast<unsigned*>(b->d_bar);
  pa.err = reinterpret_cast<int*>(b->d_bar) + 2;
  pa.skip = skip;
  if (b->r3_variant == 1) rc = launch_persistent<R3_64x4>(b, G, pa, smem, s);
  else if (b->r3_variant == 2) rc = launch_persistent<R3_16x16>(b, G, pa, smem, s);
  else rc = launch_persistent<R3_32x8>(b, G, pa, smem, s);
  if (rc) return rc;
  std::vector<BInst> h(b->count);
  int err = 0;
  BF_CUDA(cudaMemcpyAsync(&err, pa.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (infos) BF_CUDA(cudaMemcpyAsync(h.data(), b->d_inst, b->count * sizeof(BInst), cudaMemcpyDeviceToHost, s));
  BF_CUDA(cudaStreamSynchronize(s));
  if (err) return bf_fail(BF_ETIMEOUT, "bf_batch_cg_persistent: a grid-barrier wait gave up");
  if (infos) {
    for (int i = 0; i < b->count; ++i) {
      const BState& st = h[i].st;
      infos[i].iters = st.iter;
      infos[i].status = st.status == B_CONV ? BF_CG_CONVERGED : (st.status == B_BREAK ? BF_CG_BREAKDOWN : 0);
      infos[i].restarts = 0;
      infos[i].reserved = st.status == B_NONFINITE ? 1 : 0;
      infos[i].rnorm = sqrt(st.rr);
      infos[i].ref = sqrt(st.ref2);
    }
  }
  return BF_OK;
}

extern "C" int bf_batch_cg_persistent(bf_batch* b, const float* const* x0, float* const* x_out, int kmax,
                                      const bf_cg_opts* opts, bf_info* infos, void* stream) {
  return batch_run_persistent(b, x0, x_out, kmax, opts, infos, 0, (cudaStream_t)stream);
}

extern "C" int bf_batch_barrier_test(bf_batch* b, const float* const* x0, float* const* x_out, int kmax,
                                     void* stream) {
  return batch_run_persistent(b, x0, x_out, kmax, nullptr, nullptr, 1, (cudaStream_t)stream);
}

// ---- batched LOBPCG ---------------------------------------------------------------------------
// Algorithm 3 on every instance: instance i runs lobpcg_filter on internal stream i % S,
// enqueued by S host threads (one per stream), so that the Rayleigh-Ritz solves of the
// instances -- each on one SM -- and their data-parallel kernels run side by side.  Each
// graph keeps its own LOBPCG workspace, so the instances do not share memory.
extern "C" int bf_batch_lobpcg(bf_batch* b, const float* const* X0, int k, int kmax, const bf_lobpcg_opts* opts,
                               double* const* theta_out, float* const* y_out, int nstreams, bf_info* infos,
                               void* stream) {
  if (!b || !X0) return bf_fail(BF_EINVAL, "bf_batch_lobpcg: NULL argument");
  if (k < 1 || kmax < 0) return bf_fail(BF_EINVAL, "bf_batch_lobpcg: need k >= 1 and kmax >= 0");
  for (int i = 0; i < b->count; ++i) {
    if (!X0[i]) return bf_fail(BF_EINVAL, "bf_batch_lobpcg: NULL instance block");
    if (3 * (int64_t)k > b->graphs[i]->n) return bf_fail(BF_EINVAL, "bf_batch_lobpcg: an instance has n < 3k");
  }
  const int S = std::max(1, std::min(nstreams, std::min(64, b->count)));
  int dev = 0;
  BF_CUDA(cudaGetDevice(&dev));
  while ((int)b->lob_streams.size() < S) {
    cudaStream_t st;
    BF_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    b->lob_streams.push_back(st);
  }
  while ((int)b->lob_events.size() < S + 1) {
    cudaEvent_t ev;
    BF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->lob_events.push_back(ev);
  }
  cudaStream_t s = (cudaStream_t)stream;
  BF_CUDA(cudaEventRecord(b->lob_events[S], s));                 // the inputs are ready
  for (int t = 0; t < S; ++t) BF_CUDA(cudaStreamWaitEvent(b->lob_streams[t], b->lob_events[S], 0));
  std::vector<int> rc(S, BF_OK);
  std::vector<std::string> msg(S);
  auto worker = [&](int t) {
    if (cudaSetDevice(dev) != cudaSuccess) {
      rc[t] = BF_ECUDA;
      msg[t] = "bf_batch_lobpcg: cudaSetDevice failed in a worker";
      return;
    }
    for (int i = t; i < b->count; i += S) {
      const int r = lobpcg_filter(b->graphs[i], X0[i], k, k, kmax, opts, nullptr, theta_out ? theta_out[i] : nullptr,
                                  nullptr, y_out ? y_out[i] : nullptr, infos ? &infos[i] : nullptr,
                                  (void*)b->lob_streams[t]);
      if (r != BF_OK) {
        rc[t] = r;
        msg[t] = std::string("bf_batch_lobpcg: instance ") + std::to_string(i) + ": " + bf_last_error();
        return;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < S; ++t) pool.emplace_back(worker, t);
  worker(0);
  for (std::thread& th : pool) th.join();
  for (int t = 0; t < S; ++t) {
    BF_CUDA(cudaEventRecord(b->lob_events[t], b->lob_streams[t]));
    BF_CUDA(cudaStreamWaitEvent(s, b->lob_events[t], 0));      // the caller's stream waits for all
  }
  for (int t = 0; t < S; ++t)
    if (rc[t] != BF_OK) return bf_fail(rc[t], msg[t]);
  return BF_OK;
}

// Autotune the image class's tile shape: time `iters` CG iterations of the batch with each
// candidate (32 x 8, 64 x 4, 16 x 16) on the given vectors and keep the fastest.
extern "C" int bf_batch_tune(bf_batch* b, const float* const* x0, float* const* x_out, int iters,
                             float* ms_out, void* stream) {
  if (!b || !x0 || !x_out) return bf_fail(BF_EINVAL, "bf_batch_tune: NULL argument");
  if (!b->has[CLS_R3]) return BF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  bf_cg_opts o;
  memset(&o, 0, sizeof(o));
  cudaEvent_t e0, e1;
  BF_CUDA(cudaEventCreate(&e0));
  BF_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bestv = 0;
  for (int v = 0; v < 3; ++v) {
    b->r3_variant = v;
    int rc = build_jobs(b);
    if (rc) return rc;
    for (int rep = 0; rep < 2; ++rep) {          // first repetition warms up
      if ((rc = batch_upload(b, x0, x_out, o, s))) return rc;
      BF_CUDA(cudaEventRecord(e0, s));
      if ((rc = enqueue_run(b, iters, o, s))) return rc;
      BF_CUDA(cudaEventRecord(e1, s));
    }
    BF_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    BF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms_out) ms_out[v] = ms;
    if (ms < best) {
      best = ms;
      bestv = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->r3_variant = bestv;
  return build_jobs(b);
}
