// b3sim.cu -- host runtime and C ABI of the population simulator.
//
// The library owns every device buffer.  A population is packed once into a
// structure-of-arrays model (per variant: [field][32 body slots]), sorted by
// robot size, with the robots that are one free body (centred on their frame
// origin) after them, and robots larger than one warp (long chains) last, in
// a layout of their own (64 body slots).  Steps run as persistent launches of
// chain_kernel for the long chains (one block of two warps per robot), of
// step_kernel (one warp per robot, many steps per launch, slowest robots
// first) and of free_body_kernel for the single free bodies (one thread per
// robot); the launch sequence for a given step count is captured once in a
// CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "b3sim.h"
#include "chain_layout.h"
#include "free_body.cuh"
#include "model_pack.h"
#include "step_kernel.cuh"

using b3::Counters;
using b3::StepParams;

constexpr int kDefaultStepsPerLaunch = 5000;

struct sim_ctx {
  sim_config cfg{};
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n = 0;
  int n_free = 0;         // single free bodies, packed after the warp robots (one-body step)
  int n_chain = 0;        // long chains, the last packed robots (chain layout)
  std::vector<int> perm;  // packed index -> caller index
  std::vector<int> inv;   // caller index -> packed index
  float* d_mf = nullptr;
  int* d_mi = nullptr;
  int4* d_meta = nullptr;
  uint16_t* d_pairs = nullptr;
  int* d_perm = nullptr;
  float* d_q = nullptr;
  float* d_v = nullptr;
  float* d_s = nullptr;
  float* d_fit0 = nullptr;
  unsigned* d_status = nullptr;
  Counters* d_counters = nullptr;
  float* d_scratch = nullptr;
  int* d_lastnc = nullptr;
  int* d_order = nullptr;        // launch slot -> packed index (slowest first)
  unsigned* d_order_hist = nullptr;  // cost-bucket counts and cursors (2 x kCostBuckets)
  float* d_stage = nullptr;  // caller-order staging: q | v | s rows
  unsigned* d_stage_st = nullptr;
  // long chains (packed n - n_chain .. n - 1): model, state rows with the
  // host strides, scratch
  float* d_cmf = nullptr;
  int* d_cmi = nullptr;
  unsigned long long* d_cmask = nullptr;
  int4* d_cmeta = nullptr;
  uint16_t* d_cpairs = nullptr;
  float* d_cq = nullptr;
  float* d_cv = nullptr;
  float* d_cs = nullptr;
  float* d_cscratch = nullptr;
  StepParams P{};
  // Steps per persistent launch.  A launch lasts as long as its slowest
  // robot, and which robot is slowest changes as contacts come and go, so a
  // long launch (the maximum over robots of a sum over steps) beats many
  // short ones (a sum over launches of maxima): 5000-step launches measured
  // 16 % faster than 500-step ones on 4096 grammar robots.
  int steps_per_launch = kDefaultStepsPerLaunch;
  // one warp per block: the compiler then knows a block is one warp, and
  // the code of that instance is the smallest (the step is bound by
  // instruction fetch)
  int wpb = 1;
  bool lock = false;  // phase-locked launches (warps of a block in step)
  int wpsm = 16;      // resident warps per SM the kernel's registers are sized for
  std::map<long long, cudaGraphExec_t> graphs;
};

namespace {

// errors of calls without a context (sim_create, sim_step_n_noalloc), one
// slot per host thread: sim_last_error(NULL) reads the calling thread's own
thread_local const char* g_create_error = "";
thread_local std::string g_create_error_buf;

int fail(sim_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(sim_ctx* c, cudaError_t e, const char* what) {
  return fail(c, SIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_population(sim_ctx* ctx) {
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
  dfree(ctx->d_mf);
  dfree(ctx->d_mi);
  dfree(ctx->d_meta);
  dfree(ctx->d_pairs);
  dfree(ctx->d_perm);
  dfree(ctx->d_q);
  dfree(ctx->d_v);
  dfree(ctx->d_s);
  dfree(ctx->d_fit0);
  dfree(ctx->d_status);
  dfree(ctx->d_counters);
  dfree(ctx->d_scratch);
  dfree(ctx->d_lastnc);
  dfree(ctx->d_order);
  dfree(ctx->d_order_hist);
  dfree(ctx->d_stage);
  dfree(ctx->d_stage_st);
  dfree(ctx->d_cmf);
  dfree(ctx->d_cmi);
  dfree(ctx->d_cmask);
  dfree(ctx->d_cmeta);
  dfree(ctx->d_cpairs);
  dfree(ctx->d_cq);
  dfree(ctx->d_cv);
  dfree(ctx->d_cs);
  dfree(ctx->d_cscratch);
  ctx->n = 0;
  ctx->n_chain = 0;
  ctx->perm.clear();
  ctx->inv.clear();
}

// Packed state rows: robots [0, n_short) in the warp layout (q, v rows of 32
// floats, CPG rows of 64), long chains [n_short, n) in rows with the host
// strides (cq, cv, cs).
struct StateRows {
  float* q;
  float* v;
  float* s;
  float* cq;
  float* cv;
  float* cs;
  int n_short;
};

// caller rows -> packed rows (+ fitness origin, status reset); 128 threads
__global__ void scatter_state(const float* __restrict__ sq, const float* __restrict__ sv,
                              const float* __restrict__ ss, const int* __restrict__ inv_first, int first,
                              int count, int with_cpg, StateRows d, float* fit0, unsigned* status) {
  int i = blockIdx.x;
  if (i >= count) return;
  const int p = inv_first[first + i];
  const int t = threadIdx.x;
  if (p < d.n_short) {
    if (t < 32) d.q[(size_t)p * 32 + t] = sq[(size_t)i * SIM_QW + t];
    if (t < 32) d.v[(size_t)p * 32 + t] = sv[(size_t)i * SIM_VW + t];
    if (with_cpg && t < 64) d.s[(size_t)p * 64 + t] = ss[(size_t)i * SIM_SW + t];
  } else {
    const size_t c = (size_t)(p - d.n_short);
    if (t < SIM_QW) d.cq[c * SIM_QW + t] = sq[(size_t)i * SIM_QW + t];
    if (t < SIM_VW) d.cv[c * SIM_VW + t] = sv[(size_t)i * SIM_VW + t];
    if (with_cpg && t < SIM_SW) d.cs[c * SIM_SW + t] = ss[(size_t)i * SIM_SW + t];
  }
  if (t == 0) {
    fit0[2 * p] = sq[(size_t)i * SIM_QW];
    fit0[2 * p + 1] = sq[(size_t)i * SIM_QW + 1];
    status[p] = 0u;
  }
}

// packed rows -> caller rows (tails past the warp layout's rows are zero); 128 threads
__global__ void gather_state(StateRows d, const unsigned* __restrict__ status, const int* __restrict__ inv_first,
                             int first, int count, float* dq, float* dv, float* ds, unsigned* dst) {
  int i = blockIdx.x;
  if (i >= count) return;
  const int p = inv_first[first + i];
  const int t = threadIdx.x;
  if (p < d.n_short) {
    if (t < SIM_QW) dq[(size_t)i * SIM_QW + t] = t < 32 ? d.q[(size_t)p * 32 + t] : 0.f;
    if (t < SIM_VW) dv[(size_t)i * SIM_VW + t] = t < 32 ? d.v[(size_t)p * 32 + t] : 0.f;
    if (t < SIM_SW) ds[(size_t)i * SIM_SW + t] = t < 64 ? d.s[(size_t)p * 64 + t] : 0.f;
  } else {
    const size_t c = (size_t)(p - d.n_short);
    if (t < SIM_QW) dq[(size_t)i * SIM_QW + t] = d.cq[c * SIM_QW + t];
    if (t < SIM_VW) dv[(size_t)i * SIM_VW + t] = d.cv[c * SIM_VW + t];
    if (t < SIM_SW) ds[(size_t)i * SIM_SW + t] = d.cs[c * SIM_SW + t];
  }
  if (t == 0) dst[i] = status[p];
}
static_assert(SIM_SW <= 128 && SIM_QW <= 128 && SIM_VW <= 128, "scatter/gather run 128 threads per row");

__global__ void fitness_kernel(StateRows d, const float* __restrict__ fit0, const int* __restrict__ inv, int n,
                               float* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = inv[i];
  const float* q = p < d.n_short ? d.q + (size_t)p * 32 : d.cq + (size_t)(p - d.n_short) * SIM_QW;
  float dx = q[0] - fit0[2 * p];
  float dy = q[1] - fit0[2 * p + 1];
  out[i] = sqrtf(dx * dx + dy * dy);
}

size_t smem_bytes(int wpb) { return (size_t)wpb * sizeof(b3::WarpSmem); }

struct LaunchArgs {
  const float* mf;
  const int* mi;
  const int4* meta;
  const uint16_t* pairs;
  float* q;
  float* v;
  float* s;
  unsigned* status;
  Counters* counters;
  float* scratch;
  int* lastnc;
  int* order;          // NULL: slot = packed index
  unsigned* order_hist;
  int n;               // robots of the warp-per-robot step: packed [0, n)
  StepParams P;
  cudaStream_t stream;
  int n_free;          // single free bodies after them: packed [n, n + n_free)
  // long chains: packed [n + n_free, n + n_free + n_chain), model and state
  // in the chain layout; status, counters and last_nc indexed by packed index
  int n_chain;
  const float* cmf;
  const int* cmi;
  const unsigned long long* cmask;
  const int4* cmeta;
  const uint16_t* cpairs;
  float* cq;
  float* cv;
  float* cs;
  float* cscratch;
};

}  // namespace

namespace b3 {
// chain.cu
cudaError_t launch_chain(const ChainLaunch& a, int nsteps, const StepParams& P, cudaStream_t stream);
}

namespace {

// Long chains, one block of two warps per robot (chain_kernel.cuh, launched
// from its own translation unit).
cudaError_t launch_chains(const LaunchArgs& a, int nsteps) {
  const int first = a.n + a.n_free;
  const b3::ChainLaunch c{a.cmf,    a.cmi,      a.cmask,        a.cmeta,   a.cpairs,           a.cq, a.cv,
                          a.cs,     a.status + first, a.counters + first, a.cscratch, a.lastnc + first, a.n_chain};
  return b3::launch_chain(c, nsteps, a.P, a.stream);
}

// One thread per single free body (a box or a sphere whose centre is its
// frame origin): the one-body closed form of the step (free_body.cuh) for
// nsteps steps, with the same per-robot state, status, counters and
// inspection block as the warp-per-robot kernel.
__global__ void __launch_bounds__(128) free_body_kernel(const float* __restrict__ mf, float* __restrict__ qg,
                                                        float* __restrict__ vg, unsigned* __restrict__ status,
                                                        b3::Counters* __restrict__ counters,
                                                        float* __restrict__ scratch, int* __restrict__ last_nc,
                                                        int first, int count, int nsteps, b3::StepParams P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int var = first + i;
  const float* F = mf + (size_t)var * b3::NF * 32;
  float* qv = qg + (size_t)var * 32;
  float* vv = vg + (size_t)var * 32;
  float q[7], v[6];
  for (int k = 0; k < 7; ++k) q[k] = qv[k];
  for (int k = 0; k < 6; ++k) v[k] = vv[k];
  unsigned st = status[var];
  unsigned long long n_contacts = 0, n_steps = 0;
  b3::FreeBodyOut fo;
  fo.nc = last_nc[var];
  const long long t0 = clock64();
  for (int t = 0; t < nsteps && !(st & 5u); ++t) {
    if (b3::free_body_step(F, P, q, v, st, fo)) {
      n_contacts += (unsigned)fo.nc;
      ++n_steps;
    }
  }
  const long long cyc = clock64() - t0;
  for (int k = 0; k < 7; ++k) qv[k] = q[k];
  for (int k = 0; k < 6; ++k) vv[k] = v[k];
  status[var] = st;
  b3::Counters c = counters[var];
  c.contacts += n_contacts;
  c.steps += n_steps;
  c.cycles += (unsigned long long)cyc;
  counters[var] = c;
  if (n_steps == 0) return;
  last_nc[var] = fo.nc;
  // the last step's contacts (candidate layout) and inspection block
  float* cand = scratch + (size_t)var * b3::kScratchFloats;
  for (int k = 0; k < fo.nc; ++k) {
    float* row = cand + (size_t)k * b3::kCandW;
    row[0] = fo.p[k][0]; row[1] = fo.p[k][1]; row[2] = fo.p[k][2];
    row[3] = 0.f; row[4] = 0.f; row[5] = 1.f;
    row[6] = fo.depth[k];
    row[7] = __int_as_float(0 | (255 << 8));
  }
  float* dbg = cand + b3::kDbgOffset;
  for (int k = 0; k < 32; ++k) dbg[k] = k < 6 ? fo.vfree[k] : 0.f;
  dbg[31] = (float)cyc / (float)n_steps;
  for (int k = 0; k < fo.nc; ++k)
    for (int t = 0; t < 3; ++t) dbg[32 + 4 * k + t] = fo.lam[k][t];
  for (int k = 0; k < b3::kPhases; ++k) dbg[32 + 4 * b3::kCapMax + k] = 0.f;
}

// Slowest-first scheduling.  A launch lasts as long as its slowest robot, and
// robots differ in cost by an order of magnitude (bodies, contacts, near
// pairs), so before each launch the robots are bucketed by the SM cycles per
// step they took in the previous launch (8 buckets per octave, descending) and
// launched in that order: expensive robots start first and cheap ones fill
// the SMs behind them (longest-processing-time-first list scheduling).  Only
// the launch order changes; every robot's arithmetic is the same in any order.
constexpr int kCostBuckets = 256;

__device__ __forceinline__ int cost_bucket(float cycles_per_step) {
  float c = cycles_per_step;
  if (!(c >= 1.f)) c = 1.f;  // not yet measured, frozen, or not a number
  if (c > 1e30f) c = 1e30f;
  const int b = (int)(log2f(c) * 8.f);
  return kCostBuckets - 1 - min(b, kCostBuckets - 1);
}

__global__ void cost_histogram(const float* __restrict__ scratch, int n, unsigned* __restrict__ hist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  atomicAdd(&hist[cost_bucket(scratch[(size_t)i * b3::kScratchFloats + b3::kDbgOffset + 31])], 1u);
}

// every block scans the (small) histogram itself, then places its robots
__global__ void cost_scatter(const float* __restrict__ scratch, int n, unsigned* __restrict__ hist,
                             int* __restrict__ order) {
  __shared__ unsigned off[kCostBuckets];
  if (threadIdx.x == 0) {
    unsigned acc = 0;
    for (int b = 0; b < kCostBuckets; ++b) {
      off[b] = acc;
      acc += hist[b];
    }
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = cost_bucket(scratch[(size_t)i * b3::kScratchFloats + b3::kDbgOffset + 31]);
  order[off[b] + atomicAdd(&hist[kCostBuckets + b], 1u)] = i;
}

// before the first launch: cost ~ bodies^2 (the launch order is then by size)
__global__ void cost_init(const int4* __restrict__ meta, int n, float* __restrict__ scratch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float nb = (float)meta[i].x;
  scratch[(size_t)i * b3::kScratchFloats + b3::kDbgOffset + 31] = 1000.f * nb * nb;
}

// Up to kSortMax robots the order is deterministic: one block sorts the keys
// (bucket << 24 | robot) with a bitonic network in shared memory, so robots
// of equal cost keep their packed order and every run launches robots in the
// same order.  Larger populations use the atomic bucket scatter above (the
// order inside a bucket then varies from run to run; only timing depends on it).
constexpr int kSortMax = 8192;  // 32 KB of static shared memory

__global__ void __launch_bounds__(1024) cost_sort(const float* __restrict__ scratch, int n, int* __restrict__ order) {
  __shared__ unsigned key[kSortMax];
  int m = 1;
  while (m < n) m <<= 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    key[i] = i < n ? ((unsigned)cost_bucket(scratch[(size_t)i * b3::kScratchFloats + b3::kDbgOffset + 31]) << 24) |
                         (unsigned)i
                   : 0xffffffffu;
  __syncthreads();
  for (int size = 2; size <= m; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const unsigned a = key[i], b = key[j];
          if ((a > b) == up) { key[i] = b; key[j] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) order[i] = (int)(key[i] & 0xffffffu);
}

cudaError_t cost_order(const LaunchArgs& a) {
  if (a.n <= kSortMax) {
    cost_sort<<<1, 1024, 0, a.stream>>>(a.scratch, a.n, a.order);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(a.order_hist, 0, 2 * kCostBuckets * sizeof(unsigned), a.stream);
  if (e != cudaSuccess) return e;
  const int nb = (a.n + 255) / 256;
  cost_histogram<<<nb, 256, 0, a.stream>>>(a.scratch, a.n, a.order_hist);
  cost_scatter<<<nb, 256, 0, a.stream>>>(a.scratch, a.n, a.order_hist, a.order);
  return cudaGetLastError();
}

template <int WPB, bool LOCK, int WPSM>
cudaError_t launch_wpb(const LaunchArgs& a, int nsteps) {
  const size_t sm = smem_bytes(WPB);
  // the shared-memory attribute is per device: set it once on each device used
  constexpr int kMaxDevices = 64;
  static std::atomic<bool> attr_done[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices || !attr_done[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(b3::step_kernel<WPB, LOCK, WPSM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices) attr_done[dev].store(true, std::memory_order_release);
  }
  dim3 grid((a.n + WPB - 1) / WPB), block(32 * WPB);
  b3::step_kernel<WPB, LOCK, WPSM><<<grid, block, sm, a.stream>>>(a.mf, a.mi, a.meta, a.pairs, a.q, a.v, a.s,
                                                                 a.status, a.counters, a.scratch, a.lastnc,
                                                                 a.order, a.n, nsteps, a.P);
  return cudaGetLastError();
}

template <int WPSM>
cudaError_t launch_shape(const LaunchArgs& a, int nsteps, int wpb, bool lock) {
  // phase locking needs a block of several warps; with one warp it is a no-op
  switch (wpb) {
    case 1: return launch_wpb<1, false, WPSM>(a, nsteps);
    case 2: return lock ? launch_wpb<2, true, WPSM>(a, nsteps) : launch_wpb<2, false, WPSM>(a, nsteps);
    case 4: return lock ? launch_wpb<4, true, WPSM>(a, nsteps) : launch_wpb<4, false, WPSM>(a, nsteps);
    default: return cudaErrorInvalidValue;
  }
}

// a launch shape: warps per block, phase lock, resident warps per SM (16 or
// 12; blocks of 8 warps only with 16)
bool shape_ok(int wpb, int wpsm) {
  return (wpsm == 16 && (wpb == 1 || wpb == 2 || wpb == 4 || wpb == 8)) ||
         (wpsm == 12 && (wpb == 1 || wpb == 2 || wpb == 4));
}

cudaError_t launch_chunk(const LaunchArgs& a, int nsteps, int wpb, bool lock, int wpsm) {
  if (!shape_ok(wpb, wpsm)) return cudaErrorInvalidValue;
  if (wpsm == 12) return launch_shape<12>(a, nsteps, wpb, lock);
  if (wpb == 8) return lock ? launch_wpb<8, true, 16>(a, nsteps) : launch_wpb<8, false, 16>(a, nsteps);
  return launch_shape<16>(a, nsteps, wpb, lock);
}

cudaError_t enqueue_launches(const LaunchArgs& a, int n_steps, int wpb, bool lock, int wpsm, int spl) {
  for (int done = 0; done < n_steps; done += spl) {
    const int chunk = std::min(spl, n_steps - done);
    if (a.n_chain > 0) {
      cudaError_t e = launch_chains(a, chunk);
      if (e != cudaSuccess) return e;
    }
    if (a.n > 0) {
      if (a.order) {
        cudaError_t e = cost_order(a);
        if (e != cudaSuccess) return e;
      }
      cudaError_t e = launch_chunk(a, chunk, wpb, lock, wpsm);
      if (e != cudaSuccess) return e;
    }
    if (a.n_free > 0) {
      free_body_kernel<<<(a.n_free + 127) / 128, 128, 0, a.stream>>>(a.mf, a.q, a.v, a.status, a.counters,
                                                                      a.scratch, a.lastnc, a.n, a.n_free, chunk,
                                                                      a.P);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

LaunchArgs ctx_args(sim_ctx* ctx) {
  return LaunchArgs{ctx->d_mf,     ctx->d_mi,     ctx->d_meta,   ctx->d_pairs,
                    ctx->d_q,      ctx->d_v,      ctx->d_s,      ctx->d_status,
                    ctx->d_counters, ctx->d_scratch, ctx->d_lastnc, ctx->d_order,
                    ctx->d_order_hist, ctx->n - ctx->n_free - ctx->n_chain, ctx->P, ctx->stream,
                    ctx->n_free,   ctx->n_chain,  ctx->d_cmf,    ctx->d_cmi,
                    ctx->d_cmask,  ctx->d_cmeta,  ctx->d_cpairs, ctx->d_cq,
                    ctx->d_cv,     ctx->d_cs,     ctx->d_cscratch};
}

StateRows ctx_rows(sim_ctx* ctx) {
  return StateRows{ctx->d_q, ctx->d_v, ctx->d_s, ctx->d_cq, ctx->d_cv, ctx->d_cs, ctx->n - ctx->n_chain};
}

cudaError_t enqueue_steps(sim_ctx* ctx, int n_steps, int wpb, bool lock, int wpsm, int spl, bool chains = true) {
  LaunchArgs a = ctx_args(ctx);
  if (!chains) a.n_chain = 0;
  return enqueue_launches(a, n_steps, wpb, lock, wpsm, spl);
}

bool config_ok(const sim_config* cfg) {
  return cfg->dt > 0.0 && cfg->pgs_iters >= 1 && cfg->contact_cap >= 1 &&
         cfg->contact_cap <= SIM_MAX_CONTACT_CAP && cfg->soft_tau > 0.f && cfg->soft_zeta >= 0.f &&
         cfg->mu >= 0.f && cfg->steps_per_launch >= 0 && cfg->max_correct_vel > 0.f && cfg->min_cfm >= 0.f &&
         (cfg->warps_per_block == 0 || cfg->warps_per_block == 1 || cfg->warps_per_block == 2 ||
          cfg->warps_per_block == 4 || cfg->warps_per_block == 8) &&
         (cfg->phase_lock == 0 || cfg->phase_lock == 1) &&
         (cfg->warps_per_sm == 0 || cfg->warps_per_sm == 12 || cfg->warps_per_sm == 16) &&
         !(cfg->warps_per_sm == 12 && cfg->warps_per_block == 8);
}

// FP32 step constants from a configuration (ERP / CFM of the soft contacts
// computed in double, then rounded)
StepParams make_params(const sim_config* cfg) {
  StepParams P{};
  const double dt = cfg->dt;
  const double omg = 2.0 * 3.14159265358979323846 / (double)cfg->soft_tau;
  const double kden = dt * omg * omg + 2.0 * (double)cfg->soft_zeta * omg;
  P.dt = (float)dt;
  P.gx = cfg->gravity[0];
  P.gy = cfg->gravity[1];
  P.gz = cfg->gravity[2];
  P.iters = cfg->pgs_iters;
  P.mu = cfg->mu;
  P.erp = (float)(dt * omg * omg / kden);
  P.kappa = (float)(1.0 / (dt * kden));
  P.cap = cfg->contact_cap;
  P.kp = cfg->kp;
  P.kd = cfg->kd;
  P.tau_max = cfg->tau_max;
  P.theta_max = cfg->theta_max;
  P.armature = cfg->armature;
  P.ground = cfg->ground ? 1 : 0;
  P.box_box = cfg->box_box ? 1 : 0;
  P.actuate = cfg->actuate ? 1 : 0;
  P.max_correct_vel = cfg->max_correct_vel;
  P.min_cfm = cfg->min_cfm;
  return P;
}


// ---------------------------------------------------------------------------
// Allocation-free stepping.  The step kernel needs per-variant global scratch
// (contact candidates, contact Jacobian rows); here it lives in file-scope
// device arrays sized for SIM_NOALLOC_MAX_VARIANTS variants, which every
// device that loads this library keeps until the process exits.  In host code
// these names are host-side stand-ins, not device addresses, so the device
// addresses are looked up once per device and passed to the kernel.
static __device__ __align__(256) float g_noalloc_scratch[SIM_NOALLOC_MAX_VARIANTS * b3::kScratchFloats];
static __device__ __align__(256) Counters g_noalloc_counters[SIM_NOALLOC_MAX_VARIANTS];
static __device__ __align__(256) int g_noalloc_lastnc[SIM_NOALLOC_MAX_VARIANTS];

constexpr int kMaxDevices = 64;
struct NoallocAddrs {
  bool ready = false;
  float* scratch = nullptr;
  Counters* counters = nullptr;
  int* lastnc = nullptr;
};
NoallocAddrs g_noalloc[kMaxDevices];
std::mutex g_noalloc_mutex;

// once per device, with that device current
cudaError_t noalloc_setup(int dev, NoallocAddrs* out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoallocAddrs& a = g_noalloc[dev];
  if (!a.ready) {
    cudaError_t e = cudaGetSymbolAddress((void**)&a.scratch, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress((void**)&a.counters, g_noalloc_counters);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress((void**)&a.lastnc, g_noalloc_lastnc);
    if (e != cudaSuccess) return e;
    a.ready = true;
  }
  *out = a;
  return cudaSuccess;
}

// FP32 FMA throughput: independent chains x_k <- x_k a + b (a < 1, so the
// values settle at b / (1 - a) and stay finite), 8 per thread, unrolled 16
// times per loop trip; the final sum is stored only if it takes a value it
// cannot take, which keeps every chain live without memory traffic.
constexpr int kFfmaThreads = 256;
constexpr int kFfmaBlocksPerSm = 8;  // 64 resident warps per SM
constexpr int kFfmaChains = 8;
constexpr int kFfmaUnroll = 16;
constexpr int kFfmaPerIter = kFfmaChains * kFfmaUnroll;

__global__ void __launch_bounds__(kFfmaThreads) ffma_loop(float* out, float a, float b, int iters) {
  float x[kFfmaChains];
#pragma unroll
  for (int k = 0; k < kFfmaChains; ++k) x[k] = 1e-3f * (float)threadIdx.x + (float)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kFfmaUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kFfmaChains; ++k) x[k] = fmaf(x[k], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kFfmaChains; ++k) s += x[k];
  if (s == -1.f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" {

int sim_robot_cost(sim_ctx_t* ctx, float* out, int32_t n) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_robot_cost: no population");
  if (!out || n < 0 || n > ctx->n) return fail(ctx, SIM_EINVAL, "sim_robot_cost: bad n or NULL out");
  if (n == 0) return SIM_OK;
  CK(cudaSetDevice(ctx->cfg.device));
  const int n_short = ctx->n - ctx->n_chain;
  std::vector<float> packed(ctx->n);
  // one float per robot, kScratchFloats (chains: kChainScratchFloats) apart
  if (n_short > 0)
    CK(cudaMemcpy2DAsync(packed.data(), sizeof(float), ctx->d_scratch + b3::kDbgOffset + 31,
                         b3::kScratchFloats * sizeof(float), sizeof(float), n_short, cudaMemcpyDeviceToHost,
                         ctx->stream));
  if (ctx->n_chain > 0)
    CK(cudaMemcpy2DAsync(packed.data() + n_short, sizeof(float),
                         ctx->d_cscratch + b3::kCDbgOffset + b3::kCDbgCycles,
                         b3::kChainScratchFloats * sizeof(float), sizeof(float), ctx->n_chain,
                         cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < n; ++i) out[i] = packed[ctx->inv[i]];
  return SIM_OK;
}

int sim_debug_sincos(const double* x, int32_t n, double* s, double* c) {
  if (!x || !s || !c || n < 0) return SIM_EINVAL;
  for (int32_t i = 0; i < n; ++i) b3::sincos_f64(x[i], &s[i], &c[i]);
  return SIM_OK;
}

int sim_step_n_noalloc(const sim_config* cfg, const sim_device_population* pop, int32_t n_steps) {
  if (!cfg || !pop) {
    g_create_error = "sim_step_n_noalloc: cfg or pop is NULL";
    return SIM_EINVAL;
  }
  if (!config_ok(cfg)) {
    g_create_error = "sim_step_n_noalloc: configuration out of range";
    return SIM_EINVAL;
  }
  if (pop->n < 1 || pop->n > SIM_NOALLOC_MAX_VARIANTS) {
    g_create_error = "sim_step_n_noalloc: n must be 1..SIM_NOALLOC_MAX_VARIANTS (64): the static scratch holds 64 variants";
    return SIM_EINVAL;
  }
  if (n_steps < 0) {
    g_create_error = "sim_step_n_noalloc: n_steps < 0";
    return SIM_EINVAL;
  }
  if (!pop->model_f || !pop->model_i || !pop->meta || !pop->pairs || !pop->q || !pop->v || !pop->cpg ||
      !pop->status) {
    g_create_error = "sim_step_n_noalloc: a device pointer is NULL";
    return SIM_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(pop->meta) & 15u) {
    // the step kernel reads each variant's meta row as one 16-byte vector
    g_create_error = "sim_step_n_noalloc: meta must be 16-byte aligned";
    return SIM_EINVAL;
  }
  if (cfg->device < 0 || cfg->device >= kMaxDevices) {
    g_create_error = "sim_step_n_noalloc: device ordinal out of range";
    return SIM_EINVAL;
  }
  if (n_steps == 0) return SIM_OK;
  cudaError_t e = cudaSetDevice(cfg->device);
  NoallocAddrs a;
  if (e == cudaSuccess) e = noalloc_setup(cfg->device, &a);
  if (e != cudaSuccess) {
    g_create_error_buf = std::string("sim_step_n_noalloc: ") + cudaGetErrorString(e);
    g_create_error = g_create_error_buf.c_str();
    return SIM_ECUDA;
  }
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cfg->stream);
  const size_t n = (size_t)pop->n;
  // counters and the last-step contact counts start at zero on every call;
  // the rest of the scratch is written before it is read within each step
  e = cudaMemsetAsync(a.counters, 0, n * sizeof(Counters), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.lastnc, 0, n * sizeof(int), stream);
  if (e == cudaSuccess) {
    LaunchArgs args{pop->model_f, pop->model_i, reinterpret_cast<const int4*>(pop->meta), pop->pairs,
                    pop->q,       pop->v,       pop->cpg, pop->status, a.counters, a.scratch, a.lastnc,
                    nullptr,      nullptr,      pop->n,   make_params(cfg), stream, 0,
                    0,            nullptr,      nullptr,  nullptr,     nullptr,    nullptr,   nullptr,
                    nullptr,      nullptr,      nullptr};
    const int wpb = cfg->warps_per_block > 0 ? cfg->warps_per_block : 1;
    const int wpsm = cfg->warps_per_sm > 0 ? cfg->warps_per_sm : 16;
    const int spl = cfg->steps_per_launch > 0 ? cfg->steps_per_launch : kDefaultStepsPerLaunch;
    e = enqueue_launches(args, n_steps, wpb, cfg->phase_lock == 1, wpsm, spl);
  }
  if (e != cudaSuccess) {
    g_create_error_buf = std::string("sim_step_n_noalloc: ") + cudaGetErrorString(e);
    g_create_error = g_create_error_buf.c_str();
    return SIM_ECUDA;
  }
  return SIM_OK;
}


int sim_create(const sim_config* cfg, sim_ctx_t** out) {
  if (!out) return SIM_EINVAL;
  *out = nullptr;
  if (!cfg) {
    g_create_error = "sim_create: cfg is NULL";
    return SIM_EINVAL;
  }
  if (!config_ok(cfg)) {
    g_create_error = "sim_create: configuration out of range";
    return SIM_EINVAL;
  }
  sim_ctx* ctx = new (std::nothrow) sim_ctx();
  if (!ctx) return SIM_ENOMEM;
  ctx->cfg = *cfg;
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    g_create_error_buf = std::string("sim_create: cudaSetDevice: ") + cudaGetErrorString(e);
    g_create_error = g_create_error_buf.c_str();
    delete ctx;
    return SIM_ECUDA;
  }
  if (cfg->stream) {
    ctx->stream = reinterpret_cast<cudaStream_t>(cfg->stream);
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      g_create_error_buf = std::string("sim_create: cudaStreamCreate: ") + cudaGetErrorString(e);
      g_create_error = g_create_error_buf.c_str();
      delete ctx;
      return SIM_ECUDA;
    }
    ctx->own_stream = true;
  }
  ctx->P = make_params(cfg);
  if (cfg->steps_per_launch > 0) ctx->steps_per_launch = cfg->steps_per_launch;
  if (cfg->warps_per_block > 0) ctx->wpb = cfg->warps_per_block;
  if (cfg->warps_per_sm > 0) ctx->wpsm = cfg->warps_per_sm;
  ctx->lock = cfg->phase_lock == 1;
  *out = ctx;
  return SIM_OK;
}

int sim_destroy(sim_ctx_t* ctx) {
  if (!ctx) return SIM_OK;
  cudaSetDevice(ctx->cfg.device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_population(ctx);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return SIM_OK;
}

int sim_set_population(sim_ctx_t* ctx, const sim_variant_desc* v, int32_t n) {
  if (!ctx) return SIM_EINVAL;
  if (!v || n < 1) return fail(ctx, SIM_EINVAL, "sim_set_population: need n >= 1 variants");
  CK(cudaSetDevice(ctx->cfg.device));
  {
    const std::string why = b3::validate_population(v, n, "sim_set_population");
    if (!why.empty()) return fail(ctx, SIM_EINVAL, why);
  }
  free_population(ctx);
  b3::PackedPopulation pk;
  b3::pack_population(v, n, pk);
  const int n_short = n - pk.n_chain;  // warp robots and single free bodies
  const int n_chain = pk.n_chain;
  std::vector<int4> meta((size_t)std::max(n_short, 1));
  for (int k = 0; k < n_short; ++k)
    meta[k] = make_int4(pk.meta[4 * k], pk.meta[4 * k + 1], pk.meta[4 * k + 2], pk.meta[4 * k + 3]);
  std::vector<int4> cmeta((size_t)std::max(n_chain, 1));
  for (int c = 0; c < n_chain; ++c)
    cmeta[c] = make_int4(pk.cmeta[4 * c], pk.cmeta[4 * c + 1], pk.cmeta[4 * c + 2], pk.cmeta[4 * c + 3]);
  ctx->n = n;
  ctx->n_free = pk.n_free;
  ctx->n_chain = n_chain;
  ctx->perm = pk.perm;
  ctx->inv = pk.inv;
  const size_t N = (size_t)n;
  const size_t NS = (size_t)std::max(n_short, 1), NC = (size_t)std::max(n_chain, 1);
  cudaError_t e;
#define ALLOC(ptr, bytes)                                         \
  e = cudaMalloc(&(ptr), (bytes));                                \
  if (e != cudaSuccess) {                                         \
    free_population(ctx);                                         \
    return fail(ctx, SIM_ENOMEM, std::string("cudaMalloc ") + #ptr); \
  }
  ALLOC(ctx->d_mf, std::max(pk.mf.size(), (size_t)1) * sizeof(float));
  ALLOC(ctx->d_mi, std::max(pk.mi.size(), (size_t)1) * sizeof(int));
  ALLOC(ctx->d_meta, NS * sizeof(int4));
  ALLOC(ctx->d_pairs, pk.pairs.size() * sizeof(uint16_t));
  ALLOC(ctx->d_perm, N * sizeof(int));
  ALLOC(ctx->d_q, NS * 32 * sizeof(float));
  ALLOC(ctx->d_v, NS * 32 * sizeof(float));
  ALLOC(ctx->d_s, NS * 64 * sizeof(float));
  ALLOC(ctx->d_fit0, N * 2 * sizeof(float));
  ALLOC(ctx->d_status, N * sizeof(unsigned));
  ALLOC(ctx->d_counters, N * sizeof(Counters));
  ALLOC(ctx->d_scratch, NS * b3::kScratchFloats * sizeof(float));
  ALLOC(ctx->d_lastnc, N * sizeof(int));
  ALLOC(ctx->d_order, NS * sizeof(int));
  ALLOC(ctx->d_order_hist, 2 * kCostBuckets * sizeof(unsigned));
  ALLOC(ctx->d_stage, N * (SIM_QW + SIM_VW + SIM_SW) * sizeof(float));
  ALLOC(ctx->d_stage_st, N * sizeof(unsigned));
  ALLOC(ctx->d_cmf, std::max(pk.cmf.size(), (size_t)1) * sizeof(float));
  ALLOC(ctx->d_cmi, std::max(pk.cmi.size(), (size_t)1) * sizeof(int));
  ALLOC(ctx->d_cmask, std::max(pk.cmask.size(), (size_t)1) * sizeof(unsigned long long));
  ALLOC(ctx->d_cmeta, NC * sizeof(int4));
  ALLOC(ctx->d_cpairs, pk.cpairs.size() * sizeof(uint16_t));
  ALLOC(ctx->d_cq, NC * SIM_QW * sizeof(float));
  ALLOC(ctx->d_cv, NC * SIM_VW * sizeof(float));
  ALLOC(ctx->d_cs, NC * SIM_SW * sizeof(float));
  ALLOC(ctx->d_cscratch, NC * b3::kChainScratchFloats * sizeof(float));
#undef ALLOC
  CK(cudaMemcpyAsync(ctx->d_mf, pk.mf.data(), pk.mf.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_mi, pk.mi.data(), pk.mi.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_meta, meta.data(), NS * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_pairs, pk.pairs.data(), pk.pairs.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_perm, ctx->inv.data(), N * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_cmf, pk.cmf.data(), pk.cmf.size() * sizeof(float), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_cmi, pk.cmi.data(), pk.cmi.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_cmask, pk.cmask.data(), pk.cmask.size() * sizeof(unsigned long long),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_cmeta, cmeta.data(), NC * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_cpairs, pk.cpairs.data(), pk.cpairs.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemsetAsync(ctx->d_q, 0, NS * 32 * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_v, 0, NS * 32 * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_s, 0, NS * 64 * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_cq, 0, NC * SIM_QW * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_cv, 0, NC * SIM_VW * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_cs, 0, NC * SIM_SW * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_fit0, 0, N * 2 * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status, 0, N * sizeof(unsigned), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_counters, 0, N * sizeof(Counters), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_lastnc, 0, N * sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->d_cscratch, 0, NC * b3::kChainScratchFloats * sizeof(float), ctx->stream));
  // zero scratch, then the size-based cost estimate the first launch is ordered by
  CK(cudaMemsetAsync(ctx->d_scratch, 0, NS * b3::kScratchFloats * sizeof(float), ctx->stream));
  if (n_short > 0) {
    cost_init<<<(n_short + 255) / 256, 256, 0, ctx->stream>>>(ctx->d_meta, n_short, ctx->d_scratch);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return SIM_OK;
}

int sim_set_state(sim_ctx_t* ctx, int32_t first, int32_t count, const float* q, const float* v, const float* cpg) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_set_state: no population");
  if (!q || !v || first < 0 || count < 0 || first + count > ctx->n)
    return fail(ctx, SIM_EINVAL, "sim_set_state: bad range or NULL q/v");
  if (count == 0) return SIM_OK;
  CK(cudaSetDevice(ctx->cfg.device));
  float* sq = ctx->d_stage;
  float* sv = sq + (size_t)count * SIM_QW;
  float* ss = sv + (size_t)count * SIM_VW;
  CK(cudaMemcpyAsync(sq, q, (size_t)count * SIM_QW * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(sv, v, (size_t)count * SIM_VW * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  if (cpg)
    CK(cudaMemcpyAsync(ss, cpg, (size_t)count * SIM_SW * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  scatter_state<<<count, 128, 0, ctx->stream>>>(sq, sv, ss, ctx->d_perm, first, count, cpg ? 1 : 0, ctx_rows(ctx),
                                                ctx->d_fit0, ctx->d_status);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  return SIM_OK;
}

int sim_step_n(sim_ctx_t* ctx, int32_t n_steps) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_step_n: no population");
  if (n_steps < 0) return fail(ctx, SIM_EINVAL, "sim_step_n: n_steps < 0");
  if (n_steps == 0) return SIM_OK;
  CK(cudaSetDevice(ctx->cfg.device));
  const long long key = ((long long)n_steps << 8) | (ctx->wpsm == 12 ? 32 : 0) | (ctx->lock ? 16 : 0) | ctx->wpb;
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = enqueue_steps(ctx, n_steps, ctx->wpb, ctx->lock, ctx->wpsm, ctx->steps_per_launch);
    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
    if (le != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(ctx, le, "sim_step_n: launch");
    }
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "sim_step_n: capture");
    cudaGraphExec_t ge = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_fail(ctx, ie, "sim_step_n: instantiate");
    it = ctx->graphs.emplace(key, ge).first;
  }
  CK(cudaGraphLaunch(it->second, ctx->stream));
  return SIM_OK;
}

int sim_read_state(sim_ctx_t* ctx, int32_t first, int32_t count, float* q, float* v, float* cpg, uint32_t* status) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_read_state: no population");
  if (first < 0 || count < 0 || first + count > ctx->n) return fail(ctx, SIM_EINVAL, "sim_read_state: bad range");
  if (count == 0) return SIM_OK;
  CK(cudaSetDevice(ctx->cfg.device));
  float* dq = ctx->d_stage;
  float* dv = dq + (size_t)count * SIM_QW;
  float* ds = dv + (size_t)count * SIM_VW;
  gather_state<<<count, 128, 0, ctx->stream>>>(ctx_rows(ctx), ctx->d_status, ctx->d_perm, first, count, dq, dv, ds,
                                               ctx->d_stage_st);
  CK(cudaGetLastError());
  if (q) CK(cudaMemcpyAsync(q, dq, (size_t)count * SIM_QW * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  if (v) CK(cudaMemcpyAsync(v, dv, (size_t)count * SIM_VW * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  if (cpg)
    CK(cudaMemcpyAsync(cpg, ds, (size_t)count * SIM_SW * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  if (status)
    CK(cudaMemcpyAsync(status, ctx->d_stage_st, (size_t)count * sizeof(unsigned), cudaMemcpyDeviceToHost,
                       ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SIM_OK;
}

int sim_fitness(sim_ctx_t* ctx, float* out, int32_t n) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_fitness: no population");
  if (!out || n < 0 || n > ctx->n) return fail(ctx, SIM_EINVAL, "sim_fitness: bad n or NULL out");
  if (n == 0) return SIM_OK;
  CK(cudaSetDevice(ctx->cfg.device));
  float* d_out = ctx->d_stage;
  fitness_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(ctx_rows(ctx), ctx->d_fit0, ctx->d_perm, n, d_out);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, d_out, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SIM_OK;
}

// a caller buffer for the _dev entry points: device (or managed) memory
// reachable from the context's device, or NULL where allowed
static bool dev_ptr_ok(const sim_ctx_t* ctx, const void* p) {
  if (!p) return true;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == ctx->cfg.device;
}

int sim_set_state_dev(sim_ctx_t* ctx, int32_t first, int32_t count, const float* q, const float* v,
                      const float* cpg) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_set_state_dev: no population");
  if (!q || !v || first < 0 || count < 0 || first + count > ctx->n)
    return fail(ctx, SIM_EINVAL, "sim_set_state_dev: bad range or NULL q/v");
  if (count == 0) return SIM_OK;
  CK(cudaSetDevice(ctx->cfg.device));
  if (!dev_ptr_ok(ctx, q) || !dev_ptr_ok(ctx, v) || !dev_ptr_ok(ctx, cpg))
    return fail(ctx, SIM_EINVAL, "sim_set_state_dev: a buffer is not device memory of the context's device");
  scatter_state<<<count, 128, 0, ctx->stream>>>(q, v, cpg, ctx->d_perm, first, count, cpg ? 1 : 0, ctx_rows(ctx),
                                                ctx->d_fit0, ctx->d_status);
  CK(cudaGetLastError());
  return SIM_OK;
}

int sim_read_state_dev(sim_ctx_t* ctx, int32_t first, int32_t count, float* q, float* v, float* cpg,
                       uint32_t* status) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_read_state_dev: no population");
  if (first < 0 || count < 0 || first + count > ctx->n)
    return fail(ctx, SIM_EINVAL, "sim_read_state_dev: bad range");
  if (count == 0) return SIM_OK;
  CK(cudaSetDevice(ctx->cfg.device));
  if (!dev_ptr_ok(ctx, q) || !dev_ptr_ok(ctx, v) || !dev_ptr_ok(ctx, cpg) || !dev_ptr_ok(ctx, status))
    return fail(ctx, SIM_EINVAL, "sim_read_state_dev: a buffer is not device memory of the context's device");
  // outputs the caller does not want land in the staging area
  float* dq = ctx->d_stage;
  float* dv = dq + (size_t)count * SIM_QW;
  float* ds = dv + (size_t)count * SIM_VW;
  gather_state<<<count, 128, 0, ctx->stream>>>(ctx_rows(ctx), ctx->d_status, ctx->d_perm, first, count, q ? q : dq,
                                               v ? v : dv, cpg ? cpg : ds, status ? status : ctx->d_stage_st);
  CK(cudaGetLastError());
  return SIM_OK;
}

int sim_fitness_dev(sim_ctx_t* ctx, float* out, int32_t n) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_fitness_dev: no population");
  if (!out || n < 0 || n > ctx->n) return fail(ctx, SIM_EINVAL, "sim_fitness_dev: bad n or NULL out");
  if (n == 0) return SIM_OK;
  CK(cudaSetDevice(ctx->cfg.device));
  if (!dev_ptr_ok(ctx, out))
    return fail(ctx, SIM_EINVAL, "sim_fitness_dev: out is not device memory of the context's device");
  fitness_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(ctx_rows(ctx), ctx->d_fit0, ctx->d_perm, n, out);
  CK(cudaGetLastError());
  return SIM_OK;
}

int sim_stream(const sim_ctx_t* ctx, uint64_t* stream) {
  if (!ctx || !stream) return SIM_EINVAL;
  *stream = reinterpret_cast<uint64_t>(ctx->stream);
  return SIM_OK;
}

int sim_autotune(sim_ctx_t* ctx, int32_t probe_steps) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_autotune: no population");
  if (probe_steps < 1) return fail(ctx, SIM_EINVAL, "sim_autotune: probe_steps < 1");
  CK(cudaSetDevice(ctx->cfg.device));
  // the launch shapes are those of the warp-per-robot kernel: long chains
  // (one block each) sit out the probes and keep their state
  if (ctx->n == ctx->n_chain) return SIM_OK;
  const size_t N = (size_t)ctx->n;
  const size_t NS = (size_t)(ctx->n - ctx->n_chain);
  // save state and counters
  std::vector<float> q(NS * 32), v(NS * 32), s(NS * 64);
  std::vector<unsigned> st(N);
  std::vector<Counters> cn(N);
  CK(cudaMemcpyAsync(q.data(), ctx->d_q, q.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(v.data(), ctx->d_v, v.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(s.data(), ctx->d_s, s.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(st.data(), ctx->d_status, N * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(cn.data(), ctx->d_counters, N * sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  auto restore = [&]() -> cudaError_t {
    cudaMemcpyAsync(ctx->d_q, q.data(), q.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_v, v.data(), v.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_s, s.data(), s.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_status, st.data(), N * 4, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_counters, cn.data(), N * sizeof(Counters), cudaMemcpyHostToDevice, ctx->stream);
    return cudaStreamSynchronize(ctx->stream);
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // warps per block x resident warps per SM (unless configured); the phase
  // lock stays as configured: a short probe from one state does not show
  // its cost in later steps, where the slowest robot of a block sets the
  // pace of every phase boundary
  const int cands[4] = {1, 2, 4, 8};
  const int occs[2] = {16, 12};
  float best_ms = 1e30f;
  int best = ctx->wpb, best_occ = ctx->wpsm;
  for (const int occ : occs) {
    if (ctx->cfg.warps_per_sm > 0 && occ != ctx->cfg.warps_per_sm) continue;
    for (const int c : cands) {
      if (!shape_ok(c, occ)) continue;
      const bool lk = ctx->lock;
      cudaError_t e = restore();
      if (e != cudaSuccess) break;
      e = enqueue_steps(ctx, probe_steps, c, lk, occ, probe_steps, false);  // warm-up (and attribute set-up)
      if (e != cudaSuccess) continue;
      restore();
      cudaEventRecord(e0, ctx->stream);
      e = enqueue_steps(ctx, probe_steps, c, lk, occ, probe_steps, false);
      cudaEventRecord(e1, ctx->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess || e != cudaSuccess) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
        best_occ = occ;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(restore());
  ctx->wpb = best;
  ctx->wpsm = best_occ;
  return SIM_OK;
}

int sim_launch_shape(const sim_ctx_t* ctx, int32_t* warps_per_block, int32_t* phase_lock,
                     int32_t* steps_per_launch, int32_t* warps_per_sm) {
  if (!ctx) return SIM_EINVAL;
  if (warps_per_sm) *warps_per_sm = ctx->wpsm;
  if (warps_per_block) *warps_per_block = ctx->wpb;
  if (phase_lock) *phase_lock = ctx->lock ? 1 : 0;
  if (steps_per_launch) *steps_per_launch = ctx->steps_per_launch;
  return SIM_OK;
}

int sim_counters_read(sim_ctx_t* ctx, sim_counters* out) {
  if (!ctx || !out) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_counters_read: no population");
  CK(cudaSetDevice(ctx->cfg.device));
  std::vector<Counters> cn(ctx->n);
  CK(cudaMemcpyAsync(cn.data(), ctx->d_counters, cn.size() * sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  sim_counters r{};
  for (const Counters& c : cn) {
    r.contacts += (double)c.contacts;
    r.narrow_pairs += (double)c.narrow;
    r.broad_pairs += (double)c.broad;
    r.variant_steps += (double)c.steps;
    r.sm_cycles += (double)c.cycles;
  }
  *out = r;
  return SIM_OK;
}

int sim_debug_contacts(sim_ctx_t* ctx, int32_t i, int32_t max_contacts, float* rows, int32_t* b_out,
                       int32_t* n_out) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_debug_contacts: no population");
  if (i < 0 || i >= ctx->n || max_contacts < 0 || !n_out || (max_contacts > 0 && (!rows || !b_out)))
    return fail(ctx, SIM_EINVAL, "sim_debug_contacts: bad arguments");
  CK(cudaSetDevice(ctx->cfg.device));
  const int d = ctx->inv[i];
  int nc = 0;
  CK(cudaMemcpyAsync(&nc, ctx->d_lastnc + d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int m = std::min(nc, (int)max_contacts);
  std::vector<float> buf((size_t)std::max(m, 1) * b3::kCandW);
  if (m > 0) {
    const int n_short = ctx->n - ctx->n_chain;
    const float* src = d < n_short ? ctx->d_scratch + (size_t)d * b3::kScratchFloats
                                   : ctx->d_cscratch + (size_t)(d - n_short) * b3::kChainScratchFloats;
    CK(cudaMemcpyAsync(buf.data(), src, (size_t)m * b3::kCandW * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  for (int k = 0; k < m; ++k) {
    const float* r = buf.data() + (size_t)k * b3::kCandW;
    int ab;
    std::memcpy(&ab, r + 7, 4);
    for (int t = 0; t < 7; ++t) rows[8 * k + t] = r[t];
    rows[8 * k + 7] = (float)(ab & 0xff);
    const int b = (ab >> 8) & 0xff;
    b_out[k] = b == 255 ? -1 : b;
  }
  *n_out = nc;
  return SIM_OK;
}

int sim_debug_solver(sim_ctx_t* ctx, int32_t i, float* vfree, float* lambda, int32_t* n_out,
                     float* cycles_per_step) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "sim_debug_solver: no population");
  if (i < 0 || i >= ctx->n || !vfree || !lambda || !n_out) return fail(ctx, SIM_EINVAL, "sim_debug_solver: bad arguments");
  CK(cudaSetDevice(ctx->cfg.device));
  const int d = ctx->inv[i];
  const int n_short = ctx->n - ctx->n_chain;
  int nc = 0;
  CK(cudaMemcpyAsync(&nc, ctx->d_lastnc + d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  for (int k = 0; k < SIM_VW; ++k) vfree[k] = 0.f;
  if (d < n_short) {
    // warp layout: v_free (32), cycles per step at [31], impulses at 32 + 4k, phases after them
    std::vector<float> buf(32 + 4 * b3::kCapMax + 16);
    CK(cudaMemcpyAsync(buf.data(), ctx->d_scratch + (size_t)d * b3::kScratchFloats + b3::kDbgOffset,
                       buf.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 31; ++k) vfree[k] = buf[k];
    if (cycles_per_step) {
      cycles_per_step[0] = buf[31];
      for (int k = 0; k < b3::kPhases; ++k) cycles_per_step[1 + k] = buf[32 + 4 * b3::kCapMax + k];
    }
    for (int k = 0; k < nc; ++k)
      for (int t = 0; t < 3; ++t) lambda[3 * k + t] = buf[32 + 4 * k + t];
  } else {
    // chain layout (chain_kernel.cuh)
    std::vector<float> buf(b3::kCDbgPh + 16);
    CK(cudaMemcpyAsync(buf.data(), ctx->d_cscratch + (size_t)(d - n_short) * b3::kChainScratchFloats + b3::kCDbgOffset,
                       buf.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < b3::kCV && k < SIM_VW; ++k) vfree[k] = buf[k];
    if (cycles_per_step) {
      cycles_per_step[0] = buf[b3::kCDbgCycles];
      for (int k = 0; k < b3::kPhases; ++k) cycles_per_step[1 + k] = buf[b3::kCDbgPh + k];
    }
    for (int k = 0; k < nc; ++k)
      for (int t = 0; t < 3; ++t) lambda[3 * k + t] = buf[b3::kCDbgLam + 4 * k + t];
  }
  *n_out = nc;
  return SIM_OK;
}

int sim_fp32_peak(int32_t device, int32_t launches, double* flops, float* ms, int32_t* sm_count) {
  if (launches < 1 || !flops || !ms || !sm_count) {
    g_create_error = "sim_fp32_peak: launches < 1 or a NULL output";
    return SIM_EINVAL;
  }
  cudaError_t e = cudaSetDevice(device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float* out = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * (size_t)sms * kFfmaBlocksPerSm);
  const int grid = sms * kFfmaBlocksPerSm;
  const int iters = 40000;
  if (e == cudaSuccess) {
    ffma_loop<<<grid, kFfmaThreads, 0, st>>>(out, 0.9999f, 1e-4f, 100);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int l = 0; l < launches && e == cudaSuccess; ++l) {
    ffma_loop<<<grid, kFfmaThreads, 0, st>>>(out, 0.9999f, 1e-4f, iters);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) {
    g_create_error_buf = std::string("sim_fp32_peak: ") + cudaGetErrorString(e);
    g_create_error = g_create_error_buf.c_str();
    return SIM_ECUDA;
  }
  *flops = (double)launches * grid * kFfmaThreads * (double)iters * kFfmaPerIter * 2.0;
  *ms = t;
  *sm_count = sms;
  return SIM_OK;
}

const char* sim_last_error(const sim_ctx_t* ctx) {
  if (!ctx) return g_create_error;
  return ctx->err.c_str();
}

}  // extern "C"
