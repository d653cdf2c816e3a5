// b3sur.cu -- learned fitness surrogate: BF16 MLP 128 -> 256 -> 256 -> 1 on
// the tcgen05 tensor cores (TMA-fed, accumulator in tensor memory, FP32
// accumulation), Adam on FP32 master weights, GPU genotype encoding and top-k
// selection.
//
// Every dense layer, forward and backward, runs on one GEMM kernel,
// gemm_umma: C(m, n) = sum over operand pairs of A(m, k) B(n, k) with both
// operands K-major, the forward epilogue fused with the layer's bias + ReLU.
// The weight gradients reduce over the batch, so their operands are first
// copied transposed (K = the batch along a row).  Weights and inputs are
// BF16; activations and backward operands are carried as BF16 pairs (value =
// hi + lo, both BF16) and the GEMMs accumulate over both parts, so only the
// weights and inputs are rounded to 8 mantissa bits.
#include <cuda.h>  // CUtensorMap and its enums (the driver entry point is fetched at run time)
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <initializer_list>
#include <new>
#include <string>
#include <vector>

#include "b3sur.h"

typedef __nv_bfloat16 bf16;

namespace {

constexpr int IN = SUR_IN_DIM;
constexpr int HID = SUR_HIDDEN;
constexpr int NP = SUR_NPARAMS;
constexpr int kEncSlots = 20;               // brick slots of the encoding
constexpr int kEncBodies = kEncSlots + 1;   // core + bricks
static_assert(6 * kEncSlots <= IN, "six features per brick slot");
constexpr int OW1 = 0;
constexpr int OB1 = OW1 + HID * IN;
constexpr int OW2 = OB1 + HID;
constexpr int OB2 = OW2 + HID * HID;
constexpr int OW3 = OB2 + HID;
constexpr int OB3 = OW3 + HID;

// epilogues: store FP32, or bias + ReLU + BF16 (hi, lo) split
enum Epi { EPI_F32 = 0, EPI_BIAS_RELU_BF16 = 1 };

// ---------------------------------------------------------------------------
// Dense layers on the tcgen05 tensor cores, fed by TMA.
//
// C(m, n) = sum over parts p of sum_k A_p(m, k) B_p(n, k) for a tile of 128
// rows and all BN (256 or 128) columns per CTA; every operand is K-major
// (row-major with K contiguous: the forward activations and weights as they
// are, the backward operands through transposed copies).  K runs in chunks of
// 64 through a two-stage shared-memory ring.  One thread produces and issues:
// per chunk it arms the stage's `full` mbarrier with the chunk's byte count
// and starts 16 tensor copies (cp.async.bulk.tensor.2d), each an 8-element K
// slice of 128 A rows or BN B rows (2 KB / BN x 16 B); a box of 8 BF16 x rows
// lands as rows x 16 B, which is the no-swizzle K-major core-matrix layout
// with 8-row groups 128 B apart and K-adjacent core matrices one slice apart.
// Once a stage is full it issues the chunk's four tcgen05.mma (M 128, N BN,
// K 16; BF16 operands, FP32 accumulator in tensor memory) and commits them to
// the stage's `empty` mbarrier, then refills the stage the previous chunk
// used as soon as that chunk's MMAs have drained it, so copies overlap the
// tensor core.  A last commit to the `done` mbarrier releases the epilogue:
// tcgen05.ld (thread = row, 16 columns at a time) with bias + ReLU + the BF16
// (hi, lo) split, or an FP32 store.  Every wait has an iteration limit; a
// give-up sets a device flag that the host checks after its next
// synchronisation.
constexpr int UM_M = 128, UM_KC = 64, UM_STAGES = 2, UM_MAXPARTS = 3;
// the weight gradients reduce over the batch (K up to the batch size): their
// K is split over up to this many CTAs per 128-row tile
constexpr int UM_MAXSPLIT = 16;
constexpr int UM_A_SLICE = UM_M * 16;  // bytes per 8-wide K slice of A
// requested dynamic shared memory: at most two CTAs per SM, so their tensor-
// memory columns (at most 2 x 256) always fit the SM's 512 and an
// allocation never waits
constexpr int UM_SMEM = 100 * 1024;
constexpr unsigned UM_SPIN = 1u << 22;
template <int BN>
struct UmmaShape {
  static constexpr int B_SLICE = BN * 16;
  static constexpr int A_STAGE = UM_A_SLICE * (UM_KC / 8), B_STAGE = B_SLICE * (UM_KC / 8);
  static constexpr int STAGE = A_STAGE + B_STAGE;
  // kind::f16 instruction descriptor: FP32 accumulator (bit 4), BF16 A (bit 7)
  // and B (bit 10), both K-major, N / 8 at bit 17, M / 16 at bit 24
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(UM_M >> 4) << 24);
  static_assert(UM_STAGES * STAGE <= UM_SMEM, "the ring fits the shared memory");
};

struct UmmaArgs {
  int M, K, parts;   // K a multiple of UM_KC; parts 1..UM_MAXPARTS operand pairs
  int kslice;        // K chunks per CTA along gridDim.y (split K); every CTA has at least one
  long part_stride;  // split K: CTA y writes its FP32 partial to Cf + y * part_stride
  const float* bias; // EPI_BIAS_RELU_BF16
  float* Cf;         // EPI_F32 output, row stride BN
  bf16* Cb;          // EPI_BIAS_RELU_BF16 outputs (hi, lo), row stride BN
  bf16* Cb_lo;
  int epi;
  int* err;          // set to 1 when a wait gives up
};

// the operand pairs' tensor maps (a kernel parameter: the maps live in the
// parameter space the copies read them from)
struct UmmaMaps {
  CUtensorMap a[UM_MAXPARTS];
  CUtensorMap b[UM_MAXPARTS];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading byte offset (between
// K-adjacent core matrices: one slice), stride byte offset (between 8-row
// groups: 128 B), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t slice_bytes) {
  return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)(slice_bytes >> 4) << 16) | ((uint64_t)(128u >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (unsigned it = 0; it < UM_SPIN && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  return done != 0;
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

template <int BN>
__global__ void __launch_bounds__(128) gemm_umma(const __grid_constant__ UmmaMaps maps, UmmaArgs g) {
  using Sh = UmmaShape<BN>;
  extern __shared__ __align__(1024) unsigned char um_smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ int failed;
  __shared__ __align__(8) uint64_t full_bar[UM_STAGES], empty_bar[UM_STAGES], done_bar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * UM_M;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < UM_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    failed = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  // this CTA's K chunks: kc0 .. kc0 + nk - 1 of every operand pair
  const int nk_all = g.K / UM_KC, kc0 = blockIdx.y * g.kslice;
  const int nk = min(g.kslice, nk_all - kc0), nchunks = g.parts * nk;
  if (tid == 0) {
    const uint32_t ring = smem_u32(um_smem);
    auto load = [&](int c) {
      const int s = c % UM_STAGES, part = c / nk, k0 = (kc0 + c % nk) * UM_KC;
      const uint32_t a = ring + s * Sh::STAGE, b = a + Sh::A_STAGE, bar = smem_u32(&full_bar[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(Sh::STAGE) : "memory");
      for (int j = 0; j < UM_KC / 8; ++j) {
        tma_2d(a + j * UM_A_SLICE, &maps.a[part], k0 + 8 * j, m0, bar);
        tma_2d(b + j * Sh::B_SLICE, &maps.b[part], k0 + 8 * j, 0, bar);
      }
    };
    bool ok = true;
    load(0);
    if (nchunks > 1) load(1);
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s = c % UM_STAGES;
      ok = mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((c / UM_STAGES) & 1));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a = ring + s * Sh::STAGE, b = a + Sh::A_STAGE;
#pragma unroll
      for (int ks = 0; ks < UM_KC / 16; ++ks) {
        const uint32_t acc = (c | ks) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}\n" ::"r"(tmem),
            "l"(umma_desc(a + 2 * ks * UM_A_SLICE, UM_A_SLICE)),
            "l"(umma_desc(b + 2 * ks * Sh::B_SLICE, Sh::B_SLICE)), "r"(Sh::IDESC), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty_bar[s]))
                   : "memory");
      // refill the stage the previous chunk used once its MMAs have read it
      if (c >= 1 && c + 1 < nchunks) {
        const int sp = (c - 1) % UM_STAGES;
        ok = mbar_wait(smem_u32(&empty_bar[sp]), (uint32_t)(((c - 1) / UM_STAGES) & 1));
        if (ok) load(c + 1);
      }
    }
    if (ok) {
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&done_bar))
                   : "memory");
    } else {
      failed = 1;
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&done_bar)) : "memory");
    }
  }
  const bool done = mbar_wait(smem_u32(&done_bar), 0u);
  const bool ok = __syncthreads_and(done && !failed) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok) {
    if (tid == 0) atomicExch(g.err, 1);
  } else {
    const int row = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row >= g.M) continue;
      if (g.epi == EPI_F32) {
        float4* o = reinterpret_cast<float4*>(g.Cf + blockIdx.y * g.part_stride + (size_t)row * BN + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          o[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]), __uint_as_float(v[4 * q + 2]),
                             __uint_as_float(v[4 * q + 3]));
      } else {
        __align__(16) bf16 hi[16], lo[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float x = fmaxf(__uint_as_float(v[j]) + g.bias[c0 + j], 0.f);
          hi[j] = __float2bfloat16(x);
          lo[j] = __float2bfloat16(x - __bfloat162float(hi[j]));
        }
        uint4* oh = reinterpret_cast<uint4*>(g.Cb + (size_t)row * BN + c0);
        uint4* ol = reinterpret_cast<uint4*>(g.Cb_lo + (size_t)row * BN + c0);
        oh[0] = reinterpret_cast<const uint4*>(hi)[0];
        oh[1] = reinterpret_cast<const uint4*>(hi)[1];
        ol[0] = reinterpret_cast<const uint4*>(lo)[0];
        ol[1] = reinterpret_cast<const uint4*>(lo)[1];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// dst[c][r] = src[r][c] for r < rows (valid rows), 0 for rows <= r < rows_pad;
// dst has row stride ld_dst (the transposed operands' K runs along a row)
__global__ void transpose_pad(const bf16* __restrict__ src, int rows, int cols, int rows_pad, bf16* __restrict__ dst,
                              long ld_dst) {
  __shared__ bf16 t[32][34];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + tx;
    t[k][tx] = (r < rows && c < cols) ? src[(size_t)r * cols + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + tx;
    if (c < cols && r < rows_pad) dst[(size_t)c * ld_dst + r] = t[tx][k];
  }
}

// split-K: out[i] = sum over the S partials, in partial order (deterministic)
__global__ void splitk_sum(const float4* __restrict__ part, int S, long n4, float4* __restrict__ out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  float4 a = part[i];
  for (int y = 1; y < S; ++y) {
    const float4 b = part[(long)y * n4 + i];
    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
  }
  out[i] = a;
}

// h = relu(z + b) as FP32 and as a BF16 pair (hi, lo)
__global__ void bias_relu_split(const float* __restrict__ z, const float* __restrict__ b, int n, float* hf, bf16* hi_out,
                                bf16* lo_out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)n * HID) return;
  const float v = fmaxf(z[i] + b[i % HID], 0.f);
  hf[i] = v;
  const bf16 hi = __float2bfloat16(v);
  hi_out[i] = hi;
  lo_out[i] = __float2bfloat16(v - __bfloat162float(hi));
}

// y[m] = sum_j H2[m, j] W3[j] + b3 (warp per row)
__global__ void out_layer(const float* __restrict__ H2, const bf16* __restrict__ W3, const float* __restrict__ b3,
                          int n, float* y) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float s = 0.f;
  for (int j = lane; j < HID; j += 32) s += H2[(long)row * HID + j] * __bfloat162float(W3[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s + b3[0];
}

// dy = 2 (y - t) / n, per-block partial sums of (y - t)^2
__global__ void loss_grad(const float* __restrict__ y, const float* __restrict__ t, int n, float* dy, float* part) {
  __shared__ float red[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float e = 0.f;
  if (i < n) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)n;
    e = d * d;
  }
  red[threadIdx.x] = e;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// acc += the batch's squared-error partials (one thread, fixed order)
__global__ void loss_accumulate(const float* __restrict__ part, int nblk, double* acc) {
  double s = *acc;
  for (int q = 0; q < nblk; ++q) s += part[q];
  *acc = s;
}

// dZ2 = dy * W3 * (H2 > 0) as a BF16 pair (hi, lo = remainder) for the next GEMMs
__global__ void dz2_kernel(const float* __restrict__ dy, const bf16* __restrict__ W3, const float* __restrict__ H2,
                           int n, bf16* dZ2, bf16* dZ2lo) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)n * HID) return;
  const int m = (int)(i / HID), j = (int)(i % HID);
  const float on = H2[i] > 0.f ? 1.f : 0.f;
  const float v = dy[m] * __bfloat162float(W3[j]) * on;
  const bf16 hi = __float2bfloat16(v);
  dZ2[i] = hi;
  dZ2lo[i] = __float2bfloat16(v - __bfloat162float(hi));
}

// dZ1 = dH1 * (H1 > 0): FP32 in place and as a BF16 pair (hi, lo)
__global__ void relu_mask_split(float* __restrict__ dz, const bf16* __restrict__ H1, const bf16* __restrict__ H1lo,
                                int n, bf16* hi_out, bf16* lo_out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)n * HID) return;
  const float h = __bfloat162float(H1[i]) + __bfloat162float(H1lo[i]);
  const float v = h > 0.f ? dz[i] : 0.f;
  dz[i] = v;
  const bf16 hi = __float2bfloat16(v);
  hi_out[i] = hi;
  lo_out[i] = __float2bfloat16(v - __bfloat162float(hi));
}

// column sums over the batch: gb2, gW3 (from dy, W3, H2 in FP32) and gb1
// (from the FP32 dZ1).  Block (x, y): 32 columns x 8 row lanes over batch
// slab y (rows y, y + S, ...  with S = gridDim.y slabs, 8 lanes apart); the
// x = HID / 32 blocks sum dy for gb3.  Each block writes its partial sums;
// col_sums_finish adds the slabs in a fixed order.
constexpr int kColSlabs = 16;
__global__ void col_sums(const float* __restrict__ dy, const bf16* __restrict__ W3, const float* __restrict__ H2,
                         const float* __restrict__ dZ1, int n, float* __restrict__ part) {
  __shared__ float acc[3][8][33];
  const int tx = threadIdx.x, ty = threadIdx.y, slab = blockIdx.y, S = gridDim.y;
  float b2 = 0.f, w3 = 0.f, b1 = 0.f;
  if (blockIdx.x < HID / 32) {
    const int j = blockIdx.x * 32 + tx;
    const float w3j = __bfloat162float(W3[j]);
    for (int m = slab * 8 + ty; m < n; m += 8 * S) {
      const float h = H2[(long)m * HID + j];
      b2 += h > 0.f ? dy[m] * w3j : 0.f;
      w3 += dy[m] * h;
      b1 += dZ1[(long)m * HID + j];
    }
  } else {
    for (int m = slab * 256 + ty * 32 + tx; m < n; m += 256 * S) b2 += dy[m];
  }
  acc[0][ty][tx] = b2;
  acc[1][ty][tx] = w3;
  acc[2][ty][tx] = b1;
  __syncthreads();
  if (ty != 0) return;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int r = 0; r < 8; ++r) {
    s0 += acc[0][r][tx];
    s1 += acc[1][r][tx];
    s2 += acc[2][r][tx];
  }
  // partial layout: [slab][3][HID + 32] (the last 32 columns: the dy lanes)
  float* o = part + (size_t)slab * 3 * (HID + 32);
  const int c = blockIdx.x * 32 + tx;
  o[c] = s0;
  o[(HID + 32) + c] = s1;
  o[2 * (HID + 32) + c] = s2;
}

__global__ void col_sums_finish(const float* __restrict__ part, int S, float* __restrict__ grads) {
  const int c = threadIdx.x;  // HID + 32 threads
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int y = 0; y < S; ++y) {
    const float* o = part + (size_t)y * 3 * (HID + 32);
    s0 += o[c];
    s1 += o[(HID + 32) + c];
    s2 += o[2 * (HID + 32) + c];
  }
  if (c < HID) {
    grads[OB2 + c] = s0;
    grads[OW3 + c] = s1;
    grads[OB1 + c] = s2;
  } else {
    // the dy lanes' sums, in lane order, for gb3
    __shared__ float lanes[32];
    lanes[c - HID] = s0;
    __syncwarp();
    if (c == HID) {
      float t = 0.f;
      for (int l = 0; l < 32; ++l) t += lanes[l];
      grads[OB3] = t;
    }
  }
}

// Adam's step count lives on the device (so that a captured training epoch
// replays with the right bias corrections): advance it and the running
// powers b1^t, b2^t (FP64 products), and give 1 - b1^t, 1 - b2^t in FP32
__global__ void adam_prep(long long* step, double* pw, double b1, double b2, float* bc) {
  const long long t = *step + 1;
  *step = t;
  const double p1 = (t == 1 ? 1.0 : pw[0]) * b1, p2 = (t == 1 ? 1.0 : pw[1]) * b2;
  pw[0] = p1;
  pw[1] = p2;
  bc[0] = (float)(1.0 - p1);
  bc[1] = (float)(1.0 - p2);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                            const float* __restrict__ bc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float bc1 = bc[0], bc2 = bc[1];
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void to_bf16(const float* __restrict__ src, bf16* __restrict__ dst, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16(src[i]);
}

// batch gather: rows perm[b0 + i] of the full (device) training set
__global__ void gather_rows(const float* __restrict__ X, const float* __restrict__ t, const int* __restrict__ perm,
                            int b0, int nb, bf16* Xb, float* tb) {
  const int i = blockIdx.x;
  if (i >= nb) return;
  const int r = perm[b0 + i];
  for (int j = threadIdx.x; j < IN; j += blockDim.x) Xb[(long)i * IN + j] = __float2bfloat16(X[(long)r * IN + j]);
  if (threadIdx.x == 0) tb[i] = t[r];
}

// genotype encoding: 20 brick slots x (present, parent/20, face/5, rot/3,
// CPG weight), coupling weights of bricks 2..20, zeros
// Encoding of a robot (one thread per robot): zero-pose kinematics on the
// integer millimetre lattice (joint rotations rounded to their integer
// entries, offsets and box centres to whole millimetres; parents precede
// children), the bricks ordered by box centre (z, then x, then y), then per
// slot (x, y, z) / 256 mm, hinge-axis code (1 + index of the core-frame axis
// it lies along) / 3, CPG weight, coupling weight to a parent hinge (0 on
// the core); slots 20 and beyond, and columns 120..127, are zero.
__global__ void __launch_bounds__(128) encode_kernel(const int8_t* __restrict__ parent,
                                                     const int8_t* __restrict__ axis,
                                                     const float* __restrict__ R_fix,
                                                     const float* __restrict__ p_fix,
                                                     const float* __restrict__ com,
                                                     const float* __restrict__ w_int,
                                                     const float* __restrict__ w_cpl,
                                                     const int* __restrict__ nbod, int n, float* X) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  constexpr int B = kEncBodies;
  const int nb = nbod[r];  // 1 .. kEncBodies (checked by the caller)
  const long o = (long)r * 32;
  int R[B][9], org[B][3], cen[B][3];
  unsigned long long key[B];
  int idx[B];
#pragma unroll
  for (int t = 0; t < 9; ++t) R[0][t] = (t % 4 == 0) ? 1 : 0;
  org[0][0] = org[0][1] = org[0][2] = 0;
  int nbr = 0;
#pragma unroll 1
  for (int b = 1; b < nb; ++b) {
    const int p = parent[o + b];
    int Rf[9], pf[3], cb[3];
#pragma unroll
    for (int t = 0; t < 9; ++t) Rf[t] = (int)rintf(R_fix[(o + b) * 9 + t]);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      pf[t] = (int)rintf(p_fix[(o + b) * 3 + t] * 1000.f);
      cb[t] = (int)rintf(com[(o + b) * 3 + t] * 1000.f);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int j = 0; j < 3; ++j)
        R[b][3 * i + j] = R[p][3 * i] * Rf[j] + R[p][3 * i + 1] * Rf[3 + j] + R[p][3 * i + 2] * Rf[6 + j];
      org[b][i] = org[p][i] + R[p][3 * i] * pf[0] + R[p][3 * i + 1] * pf[1] + R[p][3 * i + 2] * pf[2];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
      cen[b][i] = org[b][i] + R[b][3 * i] * cb[0] + R[b][3 * i + 1] * cb[1] + R[b][3 * i + 2] * cb[2];
    // lexicographic (z, x, y), each offset into 13 bits (|coordinate| < 4096 mm)
    const unsigned long long k = ((unsigned long long)(cen[b][2] + 4096) << 26) |
                                 ((unsigned long long)(cen[b][0] + 4096) << 13) |
                                 (unsigned long long)(cen[b][1] + 4096);
    // insertion into the sorted list of the bricks so far
    int pos = nbr;
    while (pos > 0 && key[pos - 1] > k) {
      key[pos] = key[pos - 1];
      idx[pos] = idx[pos - 1];
      --pos;
    }
    key[pos] = k;
    idx[pos] = b;
    ++nbr;
  }
  float* x = X + (long)r * IN;
#pragma unroll 1
  for (int j = 0; j < IN; ++j) x[j] = 0.f;
#pragma unroll 1
  for (int i = 0; i < nbr && i < kEncSlots; ++i) {
    const int b = idx[i];
    const int ax = axis[o + b];
    // column ax of R_b is the hinge axis, a signed unit vector along x, y or z
    const int code = (R[b][ax] != 0) ? 1 : ((R[b][3 + ax] != 0) ? 2 : 3);
    x[6 * i + 0] = (float)cen[b][0] / 256.f;
    x[6 * i + 1] = (float)cen[b][1] / 256.f;
    x[6 * i + 2] = (float)cen[b][2] / 256.f;
    x[6 * i + 3] = (float)code / 3.f;
    x[6 * i + 4] = w_int[o + b];
    x[6 * i + 5] = parent[o + b] >= 1 ? w_cpl[o + b] : 0.f;
  }
}

// monotone float -> uint32 key (larger float, larger key)
__device__ __forceinline__ unsigned fkey(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Top-k in one block: radix select of the k-th largest key (4 passes of 8
// bits), then an index-ordered compaction (ties to the lower index) and a
// bitonic sort of the selection by (key descending, index ascending).
__global__ void __launch_bounds__(1024) topk_kernel(const float* __restrict__ s, int n, int k, int* out,
                                                    unsigned long long* work) {
  __shared__ unsigned hist[256];
  __shared__ unsigned sh_prefix, sh_mask, sh_kk;
  __shared__ int scan[1024];
  const int tid = threadIdx.x;
  if (tid == 0) { sh_prefix = 0u; sh_mask = 0u; sh_kk = (unsigned)k; }
  __syncthreads();
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    if (tid < 256) hist[tid] = 0u;
    __syncthreads();
    const unsigned prefix = sh_prefix, mask = sh_mask;
    for (int i = tid; i < n; i += blockDim.x) {
      const unsigned key = fkey(s[i]);
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      unsigned kk = sh_kk, cum = 0;
      int d = 255;
      for (; d > 0; --d) {
        if (cum + hist[d] >= kk) break;
        cum += hist[d];
      }
      sh_kk = kk - cum;
      sh_prefix = prefix | ((unsigned)d << shift);
      sh_mask = mask | (255u << shift);
    }
    __syncthreads();
  }
  const unsigned T = sh_prefix;
  const int ties_needed = (int)sh_kk;
  // contiguous chunk per thread keeps index order
  const int chunk = (n + blockDim.x - 1) / blockDim.x;
  const int lo = tid * chunk, hi = min(n, lo + chunk);
  int ties = 0;
  for (int i = lo; i < hi; ++i) ties += fkey(s[i]) == T ? 1 : 0;
  scan[tid] = ties;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int v = tid >= o ? scan[tid - o] : 0;
    __syncthreads();
    scan[tid] += v;
    __syncthreads();
  }
  int tie_before = scan[tid] - ties;
  __syncthreads();
  int sel = 0;
  {
    int tb = tie_before;
    for (int i = lo; i < hi; ++i) {
      const unsigned key = fkey(s[i]);
      if (key > T) ++sel;
      else if (key == T) { if (tb < ties_needed) ++sel; ++tb; }
    }
  }
  scan[tid] = sel;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int v = tid >= o ? scan[tid - o] : 0;
    __syncthreads();
    scan[tid] += v;
    __syncthreads();
  }
  int pos = scan[tid] - sel;
  {
    int tb = tie_before;
    for (int i = lo; i < hi; ++i) {
      const unsigned key = fkey(s[i]);
      bool take = false;
      if (key > T) take = true;
      else if (key == T) { take = tb < ties_needed; ++tb; }
      if (take) work[pos++] = ((unsigned long long)(~key) << 32) | (unsigned)i;
    }
  }
  __syncthreads();
  // bitonic sort ascending of (~key, index) = key descending, index ascending
  int P2 = 1;
  while (P2 < k) P2 <<= 1;
  for (int i = k + tid; i < P2; i += blockDim.x) work[i] = ~0ull;
  __syncthreads();
  for (int size = 2; size <= P2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < P2; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const unsigned long long a = work[i], b = work[j];
          if ((a > b) == up) { work[i] = b; work[j] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < k; i += blockDim.x) out[i] = (int)(work[i] & 0xffffffffu);
}

uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double uniform01(uint64_t& x) { return (double)(splitmix(x) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

struct sur_ctx {
  sur_config cfg{};
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float* p = nullptr;      // FP32 master parameters
  float* g = nullptr;      // gradients
  float* m = nullptr;      // Adam moments
  float* v = nullptr;
  bf16* w1b = nullptr;     // BF16 weight copies
  bf16* w2b = nullptr;
  bf16* w3b = nullptr;
  bf16* xb = nullptr;      // batch activations
  bf16* h1 = nullptr;
  bf16* h2 = nullptr;
  bf16* dz2 = nullptr;
  bf16* dz1 = nullptr;
  bf16* dz2lo = nullptr;
  bf16* dz1lo = nullptr;
  bf16* h1lo = nullptr;
  bf16* h2lo = nullptr;
  float* h2f = nullptr;
  float* z2f = nullptr;
  float* dz1f = nullptr;
  float* y = nullptr;
  float* dy = nullptr;
  float* tb = nullptr;
  float* part = nullptr;
  float* xfull = nullptr;  // training set / inputs on the device
  float* tfull = nullptr;
  int* perm = nullptr;
  size_t cap_rows = 0;
  long step = 0;
  double mu = 0.0, sigma = 1.0;
  unsigned long long* topk_work = nullptr;
  float* scores = nullptr;
  int* idx = nullptr;
  size_t cap_scores = 0;
  int* uerr = nullptr;     // set by gemm_umma when a tensor-core wait gives up
  float* kpart = nullptr;  // split-K partials of the weight gradients (UM_MAXSPLIT x HID x HID)
  long long* dstep = nullptr;  // Adam's step count (device)
  double* dpow = nullptr;      // b1^t, b2^t
  float* colpart = nullptr;    // column-sum partials (kColSlabs x 3 x (HID + 32))
  float* bc = nullptr;         // its bias corrections 1 - b1^t, 1 - b2^t
  double* loss_acc = nullptr;  // sum of squared errors of an epoch (device)
  // one captured training epoch (batches of the permuted set), keyed by (n, batch)
  cudaGraphExec_t epoch_graph = nullptr;
  int graph_n = 0, graph_batch = 0;
  // K-major (transposed) copies of the backward operands: [column][batch row],
  // row stride SUR_MAX_BATCH, batch rows padded with zeros to a multiple of 64
  bf16* dz2T = nullptr;
  bf16* dz2loT = nullptr;
  bf16* h1T = nullptr;
  bf16* h1loT = nullptr;
  bf16* dz1T = nullptr;
  bf16* dz1loT = nullptr;
  bf16* xT = nullptr;
  bf16* w2T = nullptr;     // W2 transposed (HID x HID)
  // TMA maps: A operands in boxes of 8 x 128 rows, B operands in boxes of 8 x N rows
  CUtensorMap tm_x{}, tm_h1{}, tm_h1lo{}, tm_dz2{}, tm_dz2lo{}, tm_dz2T{}, tm_dz2loT{}, tm_dz1T{}, tm_dz1loT{};
  CUtensorMap tm_w1{}, tm_w2{}, tm_w2T{}, tm_h1T{}, tm_h1loT{}, tm_xT{};
};

namespace {

const char* g_err = "";

int fail(sur_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(ctx, SUR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, count * sizeof(T));
}

cudaError_t transpose(cudaStream_t st, const bf16* src, int rows, int cols, int rows_pad, bf16* dst, long ld_dst) {
  dim3 grid((rows_pad + 31) / 32, (cols + 31) / 32), block(32, 8);
  transpose_pad<<<grid, block, 0, st>>>(src, rows, cols, rows_pad, dst, ld_dst);
  return cudaGetLastError();
}

cudaError_t refresh_bf16(sur_ctx* c) {
  to_bf16<<<(HID * IN + 255) / 256, 256, 0, c->stream>>>(c->p + OW1, c->w1b, HID * IN);
  to_bf16<<<(HID * HID + 255) / 256, 256, 0, c->stream>>>(c->p + OW2, c->w2b, HID * HID);
  to_bf16<<<1, 256, 0, c->stream>>>(c->p + OW3, c->w3b, HID);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return transpose(c->stream, c->w2b, HID, HID, HID, c->w2T, HID);
}

template <int BN>
cudaError_t launch_umma(sur_ctx* c, int M, int K, std::initializer_list<const CUtensorMap*> a,
                        std::initializer_list<const CUtensorMap*> b, UmmaArgs g, int splits = 1) {
  UmmaMaps maps{};
  int p = 0;
  for (const CUtensorMap* m : a) maps.a[p++] = *m;
  p = 0;
  for (const CUtensorMap* m : b) maps.b[p++] = *m;
  g.M = M;
  g.K = K;
  g.parts = p;
  g.err = c->uerr;
  const int nk = K / UM_KC;
  g.kslice = (nk + splits - 1) / splits;
  const int sy = (nk + g.kslice - 1) / g.kslice;  // every CTA row gets at least one chunk
  g.part_stride = 0;
  float* dst = g.Cf;
  if (sy > 1) {
    // the CTAs of one 128-row tile split K; each writes an FP32 partial,
    // then one pass sums them in a fixed order
    g.Cf = c->kpart;
    g.part_stride = (long)M * BN;
  }
  gemm_umma<BN><<<dim3((M + UM_M - 1) / UM_M, sy), 128, UM_SMEM, c->stream>>>(maps, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || sy == 1) return e;
  const long n4 = (long)M * BN / 4;
  splitk_sum<<<(int)((n4 + 255) / 256), 256, 0, c->stream>>>(reinterpret_cast<const float4*>(c->kpart), sy, n4,
                                                            reinterpret_cast<float4*>(dst));
  return cudaGetLastError();
}

// forward of a batch already in c->xb; y in c->y.  Hidden activations are
// carried as BF16 pairs (hi + lo) and each GEMM consuming them runs on both
// parts, so the forward pass rounds only the weights and inputs to BF16.
cudaError_t forward_batch(sur_ctx* c, int n) {
  // layer 1: H1 = relu(X W1^T + b1) as a BF16 pair; layer 2: Z2 = (H1 + H1lo) W2^T
  // with both parts accumulated in one tensor-memory accumulator
  UmmaArgs g{};
  g.bias = c->p + OB1; g.Cb = c->h1; g.Cb_lo = c->h1lo; g.epi = EPI_BIAS_RELU_BF16;
  cudaError_t e = launch_umma<HID>(c, n, IN, {&c->tm_x}, {&c->tm_w1}, g);
  if (e != cudaSuccess) return e;
  UmmaArgs h{};
  h.Cf = c->z2f; h.epi = EPI_F32;
  e = launch_umma<HID>(c, n, HID, {&c->tm_h1, &c->tm_h1lo}, {&c->tm_w2, &c->tm_w2}, h);
  if (e != cudaSuccess) return e;
  bias_relu_split<<<(int)(((long)n * HID + 255) / 256), 256, 0, c->stream>>>(c->z2f, c->p + OB2, n, c->h2f, c->h2,
                                                                           c->h2lo);
  out_layer<<<(n + 7) / 8, 256, 0, c->stream>>>(c->h2f, c->w3b, c->p + OB3, n, c->y);
  return cudaGetLastError();
}

// gradients of the batch (targets in c->tb) into c->g; loss partials in c->part.
// The backward operands dZ2 and dZ1 are carried as BF16 pairs (hi + lo) and
// every GEMM that consumes them runs on both parts, so their rounding is
// ~2^-16 instead of BF16's 2^-8.
cudaError_t backward_batch(sur_ctx* c, int n) {
  const int nblk = (n + 255) / 256;
  const int kp = (n + UM_KC - 1) / UM_KC * UM_KC;  // batch padded to whole K chunks
  const long ld = SUR_MAX_BATCH;
  loss_grad<<<nblk, 256, 0, c->stream>>>(c->y, c->tb, n, c->dy, c->part);
  dz2_kernel<<<(int)(((long)n * HID + 255) / 256), 256, 0, c->stream>>>(c->dy, c->w3b, c->h2f, n, c->dz2, c->dz2lo);
  cudaError_t e = cudaGetLastError();
  // K-major copies for the weight gradients (K = the batch)
  if (e == cudaSuccess) e = transpose(c->stream, c->dz2, n, HID, kp, c->dz2T, ld);
  if (e == cudaSuccess) e = transpose(c->stream, c->dz2lo, n, HID, kp, c->dz2loT, ld);
  if (e == cudaSuccess) e = transpose(c->stream, c->h1, n, HID, kp, c->h1T, ld);
  if (e == cudaSuccess) e = transpose(c->stream, c->h1lo, n, HID, kp, c->h1loT, ld);
  if (e == cudaSuccess) e = transpose(c->stream, c->xb, n, IN, kp, c->xT, ld);
  if (e != cudaSuccess) return e;
  // dW2(i, j) = sum_m dZ2(m, i) H1(m, j): hi*hi + lo*hi + hi*lo in one accumulator
  UmmaArgs g{};
  g.Cf = c->g + OW2; g.epi = EPI_F32;
  e = launch_umma<HID>(c, HID, kp, {&c->tm_dz2T, &c->tm_dz2loT, &c->tm_dz2T}, {&c->tm_h1T, &c->tm_h1T, &c->tm_h1loT},
                       g, UM_MAXSPLIT);
  if (e != cudaSuccess) return e;
  // dH1(m, j) = sum_i dZ2(m, i) W2(i, j): both parts of dZ2 against W2 transposed
  UmmaArgs h{};
  h.Cf = c->dz1f; h.epi = EPI_F32;
  e = launch_umma<HID>(c, n, HID, {&c->tm_dz2, &c->tm_dz2lo}, {&c->tm_w2T, &c->tm_w2T}, h);
  if (e != cudaSuccess) return e;
  relu_mask_split<<<(int)(((long)n * HID + 255) / 256), 256, 0, c->stream>>>(c->dz1f, c->h1, c->h1lo, n, c->dz1,
                                                                           c->dz1lo);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = transpose(c->stream, c->dz1, n, HID, kp, c->dz1T, ld);
  if (e == cudaSuccess) e = transpose(c->stream, c->dz1lo, n, HID, kp, c->dz1loT, ld);
  if (e != cudaSuccess) return e;
  // dW1(i, j) = sum_m dZ1(m, i) X(m, j): both parts of dZ1
  UmmaArgs w{};
  w.Cf = c->g + OW1; w.epi = EPI_F32;
  e = launch_umma<IN>(c, HID, kp, {&c->tm_dz1T, &c->tm_dz1loT}, {&c->tm_xT, &c->tm_xT}, w, UM_MAXSPLIT);
  if (e != cudaSuccess) return e;
  col_sums<<<dim3(HID / 32 + 1, kColSlabs), dim3(32, 8), 0, c->stream>>>(c->dy, c->w3b, c->h2f, c->dz1f, n,
                                                                       c->colpart);
  col_sums_finish<<<1, HID + 32, 0, c->stream>>>(c->colpart, kColSlabs, c->g);
  return cudaGetLastError();
}

cudaError_t adam_update(sur_ctx* c) {
  c->step += 1;  // host mirror of the device count
  adam_prep<<<1, 1, 0, c->stream>>>(c->dstep, c->dpow, (double)c->cfg.beta1, (double)c->cfg.beta2, c->bc);
  adam_kernel<<<(NP + 255) / 256, 256, 0, c->stream>>>(c->p, c->g, c->m, c->v, NP, c->cfg.lr, c->cfg.beta1,
                                                     c->cfg.beta2, c->cfg.eps, c->bc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return refresh_bf16(c);
}

int ensure_rows(sur_ctx* ctx, size_t n) {
  if (n <= ctx->cap_rows) return SUR_OK;
  // a captured epoch reads the old training-set buffers: drop it
  if (ctx->epoch_graph) cudaGraphExecDestroy(ctx->epoch_graph);
  ctx->epoch_graph = nullptr;
  ctx->graph_n = ctx->graph_batch = 0;
  cudaFree(ctx->xfull);
  cudaFree(ctx->tfull);
  cudaFree(ctx->perm);
  ctx->xfull = nullptr; ctx->tfull = nullptr; ctx->perm = nullptr; ctx->cap_rows = 0;
  if (dalloc(&ctx->xfull, n * IN) != cudaSuccess || dalloc(&ctx->tfull, n) != cudaSuccess ||
      dalloc(&ctx->perm, n) != cudaSuccess)
    return fail(ctx, SUR_ENOMEM, "device allocation for the training set failed");
  ctx->cap_rows = n;
  return SUR_OK;
}

int ensure_scores(sur_ctx* ctx, size_t n) {
  if (n <= ctx->cap_scores) return SUR_OK;
  cudaFree(ctx->scores);
  cudaFree(ctx->idx);
  ctx->scores = nullptr; ctx->idx = nullptr; ctx->cap_scores = 0;
  if (dalloc(&ctx->scores, n) != cudaSuccess || dalloc(&ctx->idx, n) != cudaSuccess)
    return fail(ctx, SUR_ENOMEM, "device allocation for scores failed");
  ctx->cap_scores = n;
  return SUR_OK;
}

void free_all(sur_ctx* c) {
  void* ptrs[] = {c->p, c->g, c->m, c->v, c->w1b, c->w2b, c->w3b, c->xb, c->h1, c->h2, c->dz2, c->dz1,
                  c->dz2lo, c->dz1lo, c->h1lo, c->h2lo, c->h2f, c->z2f, c->dz1f, c->y, c->dy, c->tb, c->part, c->xfull, c->tfull, c->perm, c->topk_work, c->scores,
                  c->idx, c->uerr, c->dz2T, c->dz2loT, c->h1T, c->h1loT, c->dz1T, c->dz1loT, c->xT, c->w2T,
                  c->kpart, c->dstep, c->bc, c->loss_acc, c->dpow, c->colpart};
  if (c->epoch_graph) cudaGraphExecDestroy(c->epoch_graph);
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

// after a stream synchronisation: did a tensor-core wait give up?
int check_umma(sur_ctx* ctx) {
  int h = 0;
  CK(cudaMemcpy(&h, ctx->uerr, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) return fail(ctx, SUR_ECUDA, "gemm_umma: a tensor-core completion wait gave up");
  return SUR_OK;
}

int read_loss(sur_ctx* ctx, int n, float* loss_out) {
  const int nblk = (n + 255) / 256;
  std::vector<float> part(nblk);
  CK(cudaMemcpyAsync(part.data(), ctx->part, nblk * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (int rc = check_umma(ctx)) return rc;
  double s = 0.0;
  for (float x : part) s += x;
  if (loss_out) *loss_out = (float)(s / n);
  return SUR_OK;
}

// upload n rows of X (and t) into xfull / tfull, gather them as one batch
int stage_batch(sur_ctx* ctx, const float* X, const float* t, int n) {
  int rc = ensure_rows(ctx, (size_t)n);
  if (rc != SUR_OK) return rc;
  CK(cudaMemcpyAsync(ctx->xfull, X, (size_t)n * IN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<int> id(n);
  for (int i = 0; i < n; ++i) id[i] = i;
  CK(cudaMemcpyAsync(ctx->perm, id.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  if (t) CK(cudaMemcpyAsync(ctx->tfull, t, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  else CK(cudaMemsetAsync(ctx->tfull, 0, (size_t)n * sizeof(float), ctx->stream));
  gather_rows<<<n, 128, 0, ctx->stream>>>(ctx->xfull, ctx->tfull, ctx->perm, 0, n, ctx->xb, ctx->tb);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  return SUR_OK;
}

}  // namespace

namespace {

// TMA map of a row-major BF16 matrix (rows x cols) read in boxes of 8 columns
// x box_rows rows; cuTensorMapEncodeTiled is taken from the driver at run time
bool make_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * sizeof(bf16)};
  const cuuint32_t box[2] = {8, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" {

int sur_create(const sur_config* cfg, sur_ctx_t** out) {
  if (!out) return SUR_EINVAL;
  *out = nullptr;
  if (!cfg || !(cfg->lr > 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
      !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps > 0.f)) {
    g_err = "sur_create: NULL or out-of-range configuration";
    return SUR_EINVAL;
  }
  sur_ctx* ctx = new (std::nothrow) sur_ctx();
  if (!ctx) return SUR_ENOMEM;
  ctx->cfg = *cfg;
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    g_err = "sur_create: cudaSetDevice failed";
    delete ctx;
    return SUR_ECUDA;
  }
  if (cfg->stream) {
    ctx->stream = reinterpret_cast<cudaStream_t>(cfg->stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      g_err = "sur_create: cudaStreamCreate failed";
      delete ctx;
      return SUR_ECUDA;
    }
    ctx->own_stream = true;
  }
  const size_t B = SUR_MAX_BATCH;
  bool ok = dalloc(&ctx->p, NP) == cudaSuccess && dalloc(&ctx->g, NP) == cudaSuccess &&
            dalloc(&ctx->m, NP) == cudaSuccess && dalloc(&ctx->v, NP) == cudaSuccess &&
            dalloc(&ctx->w1b, (size_t)HID * IN) == cudaSuccess && dalloc(&ctx->w2b, (size_t)HID * HID) == cudaSuccess &&
            dalloc(&ctx->w3b, (size_t)HID) == cudaSuccess && dalloc(&ctx->xb, B * IN) == cudaSuccess &&
            dalloc(&ctx->h1, B * HID) == cudaSuccess && dalloc(&ctx->h2, B * HID) == cudaSuccess &&
            dalloc(&ctx->dz2, B * HID) == cudaSuccess && dalloc(&ctx->dz1, B * HID) == cudaSuccess &&
            dalloc(&ctx->dz2lo, B * HID) == cudaSuccess && dalloc(&ctx->dz1lo, B * HID) == cudaSuccess &&
            dalloc(&ctx->h1lo, B * HID) == cudaSuccess && dalloc(&ctx->h2lo, B * HID) == cudaSuccess &&
            dalloc(&ctx->h2f, B * HID) == cudaSuccess && dalloc(&ctx->z2f, B * HID) == cudaSuccess &&
            dalloc(&ctx->dz1f, B * HID) == cudaSuccess && dalloc(&ctx->y, B) == cudaSuccess &&
            dalloc(&ctx->dy, B) == cudaSuccess && dalloc(&ctx->tb, B) == cudaSuccess &&
            dalloc(&ctx->part, (B + 255) / 256) == cudaSuccess &&
            dalloc(&ctx->topk_work, (size_t)2 * SUR_MAX_TOPK) == cudaSuccess && dalloc(&ctx->uerr, 1) == cudaSuccess &&
            dalloc(&ctx->dz2T, (size_t)HID * B) == cudaSuccess && dalloc(&ctx->dz2loT, (size_t)HID * B) == cudaSuccess &&
            dalloc(&ctx->h1T, (size_t)HID * B) == cudaSuccess && dalloc(&ctx->h1loT, (size_t)HID * B) == cudaSuccess &&
            dalloc(&ctx->dz1T, (size_t)HID * B) == cudaSuccess && dalloc(&ctx->dz1loT, (size_t)HID * B) == cudaSuccess &&
            dalloc(&ctx->xT, (size_t)IN * B) == cudaSuccess && dalloc(&ctx->w2T, (size_t)HID * HID) == cudaSuccess &&
            dalloc(&ctx->kpart, (size_t)UM_MAXSPLIT * HID * HID) == cudaSuccess &&
            dalloc(&ctx->dstep, 1) == cudaSuccess && dalloc(&ctx->bc, 2) == cudaSuccess &&
            dalloc(&ctx->dpow, 2) == cudaSuccess &&
            dalloc(&ctx->colpart, (size_t)kColSlabs * 3 * (HID + 32)) == cudaSuccess &&
            dalloc(&ctx->loss_acc, 1) == cudaSuccess && cudaMemset(ctx->dstep, 0, sizeof(long long)) == cudaSuccess &&
            cudaMemset(ctx->uerr, 0, sizeof(int)) == cudaSuccess &&
            cudaFuncSetAttribute(gemm_umma<HID>, cudaFuncAttributeMaxDynamicSharedMemorySize, UM_SMEM) == cudaSuccess &&
            cudaFuncSetAttribute(gemm_umma<IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, UM_SMEM) == cudaSuccess &&
            // A operands (boxes of 128 rows)
            make_map(&ctx->tm_x, ctx->xb, B, IN, UM_M) && make_map(&ctx->tm_h1, ctx->h1, B, HID, UM_M) &&
            make_map(&ctx->tm_h1lo, ctx->h1lo, B, HID, UM_M) && make_map(&ctx->tm_dz2, ctx->dz2, B, HID, UM_M) &&
            make_map(&ctx->tm_dz2lo, ctx->dz2lo, B, HID, UM_M) && make_map(&ctx->tm_dz2T, ctx->dz2T, HID, B, UM_M) &&
            make_map(&ctx->tm_dz2loT, ctx->dz2loT, HID, B, UM_M) && make_map(&ctx->tm_dz1T, ctx->dz1T, HID, B, UM_M) &&
            make_map(&ctx->tm_dz1loT, ctx->dz1loT, HID, B, UM_M) &&
            // B operands (boxes of N rows)
            make_map(&ctx->tm_w1, ctx->w1b, HID, IN, HID) && make_map(&ctx->tm_w2, ctx->w2b, HID, HID, HID) &&
            make_map(&ctx->tm_w2T, ctx->w2T, HID, HID, HID) && make_map(&ctx->tm_h1T, ctx->h1T, HID, B, HID) &&
            make_map(&ctx->tm_h1loT, ctx->h1loT, HID, B, HID) && make_map(&ctx->tm_xT, ctx->xT, IN, B, IN);
  if (!ok) {
    free_all(ctx);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    g_err = "sur_create: device allocation failed";
    return SUR_ENOMEM;
  }
  // He-uniform weights from the seed, zero biases
  std::vector<float> p(NP, 0.f);
  uint64_t st = cfg->seed ^ 0x5DEECE66DULL;
  auto fill = [&](int off, int rows, int cols) {
    const double lim = std::sqrt(6.0 / cols);
    for (int i = 0; i < rows * cols; ++i) p[off + i] = (float)((2.0 * uniform01(st) - 1.0) * lim);
  };
  fill(OW1, HID, IN);
  fill(OW2, HID, HID);
  fill(OW3, 1, HID);
  *out = ctx;
  return sur_set_params(ctx, p.data());
}

int sur_destroy(sur_ctx_t* ctx) {
  if (!ctx) return SUR_OK;
  cudaSetDevice(ctx->cfg.device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return SUR_OK;
}

int sur_set_params(sur_ctx_t* ctx, const float* params) {
  if (!ctx || !params) return fail(ctx, SUR_EINVAL, "sur_set_params: NULL");
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaMemcpyAsync(ctx->p, params, NP * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->m, 0, NP * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->v, 0, NP * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->dstep, 0, sizeof(long long), ctx->stream));
  ctx->step = 0;
  ctx->mu = 0.0;
  ctx->sigma = 1.0;
  CK(refresh_bf16(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  return SUR_OK;
}

int sur_get_params(sur_ctx_t* ctx, float* params) {
  if (!ctx || !params) return fail(ctx, SUR_EINVAL, "sur_get_params: NULL");
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaMemcpyAsync(params, ctx->p, NP * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SUR_OK;
}

int sur_encode(sur_ctx_t* ctx, const int8_t* parent, const int8_t* axis, const float* R_fix, const float* p_fix,
               const float* box_center, const float* w_int, const float* w_cpl, const int32_t* n_bodies, int32_t n,
               float* X_out) {
  if (!ctx) return SUR_EINVAL;
  if (n < 1 || !parent || !axis || !R_fix || !p_fix || !box_center || !w_int || !w_cpl || !n_bodies || !X_out)
    return fail(ctx, SUR_EINVAL, "sur_encode: bad arguments");
  for (int32_t r = 0; r < n; ++r) {
    const int nb = n_bodies[r];
    if (nb < 1 || nb > kEncBodies) return fail(ctx, SUR_EINVAL, "sur_encode: n_bodies outside 1..21");
    for (int b = 1; b < nb; ++b) {
      const int p = parent[(size_t)r * 32 + b], a = axis[(size_t)r * 32 + b];
      if (p < 0 || p >= b || a < 0 || a > 2) return fail(ctx, SUR_EINVAL, "sur_encode: bad parent or hinge axis");
    }
  }
  CK(cudaSetDevice(ctx->cfg.device));
  int8_t *dp = nullptr, *da = nullptr;
  float *dR = nullptr, *dpf = nullptr, *dc = nullptr, *dwi = nullptr, *dwc = nullptr, *dX = nullptr;
  int* dn = nullptr;
  const size_t N = (size_t)n;
  bool ok = dalloc(&dp, N * 32) == cudaSuccess && dalloc(&da, N * 32) == cudaSuccess &&
            dalloc(&dR, N * 32 * 9) == cudaSuccess && dalloc(&dpf, N * 32 * 3) == cudaSuccess &&
            dalloc(&dc, N * 32 * 3) == cudaSuccess && dalloc(&dwi, N * 32) == cudaSuccess &&
            dalloc(&dwc, N * 32) == cudaSuccess && dalloc(&dn, N) == cudaSuccess && dalloc(&dX, N * IN) == cudaSuccess;
  int rc = SUR_OK;
  if (!ok) {
    rc = fail(ctx, SUR_ENOMEM, "sur_encode: device allocation failed");
  } else {
    cudaMemcpyAsync(dp, parent, N * 32, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(da, axis, N * 32, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dR, R_fix, N * 32 * 9 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dpf, p_fix, N * 32 * 3 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dc, box_center, N * 32 * 3 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dwi, w_int, N * 32 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dwc, w_cpl, N * 32 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dn, n_bodies, N * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    encode_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(dp, da, dR, dpf, dc, dwi, dwc, dn, n, dX);
    cudaMemcpyAsync(X_out, dX, N * IN * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) rc = fail(ctx, SUR_ECUDA, std::string("sur_encode: ") + cudaGetErrorString(e));
  }
  cudaFree(dp); cudaFree(da); cudaFree(dR); cudaFree(dpf); cudaFree(dc); cudaFree(dwi); cudaFree(dwc);
  cudaFree(dn); cudaFree(dX);
  return rc;
}

int sur_predict(sur_ctx_t* ctx, const float* X, int32_t n, float* y_out) {
  if (!ctx) return SUR_EINVAL;
  if (!X || !y_out || n < 1) return fail(ctx, SUR_EINVAL, "sur_predict: bad arguments");
  CK(cudaSetDevice(ctx->cfg.device));
  int rc = ensure_rows(ctx, (size_t)n);
  if (rc != SUR_OK) return rc;
  CK(cudaMemcpyAsync(ctx->xfull, X, (size_t)n * IN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<int> id(n);
  for (int i = 0; i < n; ++i) id[i] = i;
  CK(cudaMemcpyAsync(ctx->perm, id.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->tfull, 0, (size_t)n * sizeof(float), ctx->stream));
  std::vector<float> tmp(SUR_MAX_BATCH);
  for (int b0 = 0; b0 < n; b0 += SUR_MAX_BATCH) {
    const int nb = std::min(SUR_MAX_BATCH, n - b0);
    gather_rows<<<nb, 128, 0, ctx->stream>>>(ctx->xfull, ctx->tfull, ctx->perm, b0, nb, ctx->xb, ctx->tb);
    CK(cudaGetLastError());
    CK(forward_batch(ctx, nb));
    CK(cudaMemcpyAsync(tmp.data(), ctx->y, nb * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (int rc2 = check_umma(ctx)) return rc2;
    for (int i = 0; i < nb; ++i) y_out[b0 + i] = (float)(ctx->mu + ctx->sigma * (double)tmp[i]);
  }
  return SUR_OK;
}

int sur_gradients(sur_ctx_t* ctx, const float* X, const float* y, int32_t n, float* grads, float* loss_out) {
  if (!ctx) return SUR_EINVAL;
  if (!X || !y || !grads || n < 1 || n > SUR_MAX_BATCH) return fail(ctx, SUR_EINVAL, "sur_gradients: bad arguments");
  CK(cudaSetDevice(ctx->cfg.device));
  int rc = stage_batch(ctx, X, y, n);
  if (rc != SUR_OK) return rc;
  CK(forward_batch(ctx, n));
  CK(backward_batch(ctx, n));
  CK(cudaMemcpyAsync(grads, ctx->g, NP * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  return read_loss(ctx, n, loss_out);
}

int sur_train_step(sur_ctx_t* ctx, const float* X, const float* y, int32_t n, float* loss_out) {
  if (!ctx) return SUR_EINVAL;
  if (!X || !y || n < 1 || n > SUR_MAX_BATCH) return fail(ctx, SUR_EINVAL, "sur_train_step: bad arguments");
  CK(cudaSetDevice(ctx->cfg.device));
  int rc = stage_batch(ctx, X, y, n);
  if (rc != SUR_OK) return rc;
  CK(forward_batch(ctx, n));
  CK(backward_batch(ctx, n));
  CK(adam_update(ctx));
  return read_loss(ctx, n, loss_out);
}

int sur_train(sur_ctx_t* ctx, const float* X, const float* y, int32_t n, int32_t epochs, int32_t batch,
              float* loss_out) {
  if (!ctx) return SUR_EINVAL;
  if (!X || !y || n < 2 || epochs < 1 || batch < 1 || batch > SUR_MAX_BATCH)
    return fail(ctx, SUR_EINVAL, "sur_train: bad arguments");
  CK(cudaSetDevice(ctx->cfg.device));
  int rc = ensure_rows(ctx, (size_t)n);
  if (rc != SUR_OK) return rc;
  double mu = 0.0, var = 0.0;
  for (int i = 0; i < n; ++i) mu += y[i];
  mu /= n;
  for (int i = 0; i < n; ++i) var += (y[i] - mu) * (y[i] - mu);
  const double sigma = std::sqrt(var / n) > 1e-12 ? std::sqrt(var / n) : 1.0;
  std::vector<float> t(n);
  for (int i = 0; i < n; ++i) t[i] = (float)((y[i] - mu) / sigma);
  ctx->mu = mu;
  ctx->sigma = sigma;
  CK(cudaMemcpyAsync(ctx->xfull, X, (size_t)n * IN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->tfull, t.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<int> perm(n);
  uint64_t st = ctx->cfg.seed * 0x2545F4914F6CDD1DULL + (uint64_t)ctx->step;
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = n - 1; i > 0; --i) {
      const int j = (int)(splitmix(st) % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    CK(cudaMemcpyAsync(ctx->perm, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    // one epoch = one graph launch: every batch's gather, forward, backward,
    // Adam update and loss partials, captured once per (n, batch)
    if (!ctx->epoch_graph || ctx->graph_n != n || ctx->graph_batch != batch) {
      if (ctx->epoch_graph) cudaGraphExecDestroy(ctx->epoch_graph);
      ctx->epoch_graph = nullptr;
      cudaGraph_t gr = nullptr;
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t ce = cudaSuccess;
      for (int b0 = 0; b0 < n && ce == cudaSuccess; b0 += batch) {
        const int nb = std::min(batch, n - b0);
        gather_rows<<<nb, 128, 0, ctx->stream>>>(ctx->xfull, ctx->tfull, ctx->perm, b0, nb, ctx->xb, ctx->tb);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = forward_batch(ctx, nb);
        if (ce == cudaSuccess) ce = backward_batch(ctx, nb);
        if (ce == cudaSuccess) ce = adam_update(ctx);
        if (ce == cudaSuccess) {
          loss_accumulate<<<1, 1, 0, ctx->stream>>>(ctx->part, (nb + 255) / 256, ctx->loss_acc);
          ce = cudaGetLastError();
        }
      }
      cudaError_t ee = cudaStreamEndCapture(ctx->stream, &gr);
      if (ce != cudaSuccess || ee != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return fail(ctx, SUR_ECUDA, std::string("sur_train: epoch capture: ") +
                                        cudaGetErrorString(ce != cudaSuccess ? ce : ee));
      }
      cudaError_t ie = cudaGraphInstantiate(&ctx->epoch_graph, gr, 0);
      cudaGraphDestroy(gr);
      if (ie != cudaSuccess) {
        ctx->epoch_graph = nullptr;
        return fail(ctx, SUR_ECUDA, std::string("sur_train: instantiate: ") + cudaGetErrorString(ie));
      }
      ctx->graph_n = n;
      ctx->graph_batch = batch;
      // the capture advanced the host mirror of the step count without running
      ctx->step -= (n + batch - 1) / batch;
    }
    CK(cudaMemsetAsync(ctx->loss_acc, 0, sizeof(double), ctx->stream));
    CK(cudaGraphLaunch(ctx->epoch_graph, ctx->stream));
    ctx->step += (n + batch - 1) / batch;
    if (ep == epochs - 1) {
      double acc = 0.0;
      CK(cudaMemcpyAsync(&acc, ctx->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      last = acc / n;
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (loss_out) *loss_out = (float)last;
  return SUR_OK;
}

int sur_topk(sur_ctx_t* ctx, const float* scores, int32_t n, int32_t k, int32_t* idx_out) {
  if (!ctx) return SUR_EINVAL;
  if (!scores || !idx_out || n < 1 || k < 1 || k > n || k > SUR_MAX_TOPK)
    return fail(ctx, SUR_EINVAL, "sur_topk: bad arguments");
  CK(cudaSetDevice(ctx->cfg.device));
  int rc = ensure_scores(ctx, (size_t)n);
  if (rc != SUR_OK) return rc;
  CK(cudaMemcpyAsync(ctx->scores, scores, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  topk_kernel<<<1, 1024, 0, ctx->stream>>>(ctx->scores, n, k, ctx->idx, ctx->topk_work);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(idx_out, ctx->idx, (size_t)k * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SUR_OK;
}

const char* sur_last_error(const sur_ctx_t* ctx) {
  if (!ctx) return g_err;
  return ctx->err.c_str();
}

}  // extern "C"
