// chain.cu -- launcher of the block-per-robot chain step (chain_kernel.cuh).
// A translation unit of its own, so that the chain kernel and the
// narrow-phase helpers it instantiates for 64 body slots leave the code
// generated for the warp-per-robot kernel in b3sim.cu unchanged.
#include <cuda_runtime.h>

#include <atomic>

#include "b3sim.h"
#include "chain_kernel.cuh"

namespace b3 {

static_assert(SIM_QW == kCQS && SIM_VW == kCVS && SIM_SW == kCSS, "chain rows use the host strides");
static_assert(SIM_MAX_BODIES <= kCB && SIM_MAX_BODIES + 5 <= kCV, "chain layout holds the largest robot");
static_assert(SIM_MAX_CONTACT_CAP <= kCapMax, "chain inspection block holds every kept contact");
static_assert(SIM_MAX_CANDIDATES_CHAIN == kCCand, "chain candidate capacity as documented");
static_assert(2 * (chain_smem_bytes(SIM_MAX_CONTACT_CAP) + 1024) <= 228 * 1024, "two chain robots per SM");

cudaError_t launch_chain(const ChainLaunch& a, int nsteps, const StepParams& P, cudaStream_t stream) {
  // the shared-memory attribute is per device: set it once on each device
  // used, for the largest contact cap
  constexpr int kMaxDevices = 64;
  static std::atomic<bool> attr_done[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices || !attr_done[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chain_smem_bytes(SIM_MAX_CONTACT_CAP));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices) attr_done[dev].store(true, std::memory_order_release);
  }
  if (P.cap < 1 || P.cap > SIM_MAX_CONTACT_CAP) return cudaErrorInvalidValue;
  chain_kernel<<<a.n, kCT, chain_smem_bytes(P.cap), stream>>>(
      a.mf, a.mi, a.mk, static_cast<const int4*>(a.meta), a.pairs, a.q, a.v, a.s, a.status,
      static_cast<Counters*>(a.counters), a.scratch, a.last_nc, a.n, nsteps, P);
  return cudaGetLastError();
}

}  // namespace b3
