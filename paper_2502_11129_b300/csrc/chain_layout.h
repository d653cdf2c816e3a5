// chain_layout.h -- sizes and scratch layout of the block-per-robot chain
// step (chain_kernel.cuh), shared with the host runtime that allocates its
// buffers and reads its inspection block.
#pragma once
#include <stddef.h>

#include "step_common.cuh"

namespace b3 {

constexpr int kCB = kChainSlots;                 // body slots (64)
constexpr int kCV = 72;                          // dof slots (nv <= 69)
constexpr int kCT = 64;                          // threads per robot
constexpr int kCTri = kCV * (kCV + 1) / 2;       // packed lower triangle of M / L
constexpr int kYS = 73;                          // Y row stride: odd, so rows read one per thread hit distinct banks
constexpr int kCMaxPairs = kCB * (kCB - 1) / 2;
constexpr int kCCand = 512;                      // contact candidates per step: every vertex of 64 boxes
// device state rows of the chain layout (the host row strides)
constexpr int kCQS = 72, kCVS = 72, kCSS = 128;

// global scratch per chain robot: the last step's contacts (candidate
// layout), the narrow phase's staging rows (8 per thread), then the
// inspection block: v_free [kCV], SM cycles per step, impulses (4 floats per
// contact), per-phase cycles
constexpr size_t kCStageOffset = (size_t)kCand * kCandW;
constexpr size_t kCDbgOffset = kCStageOffset + (size_t)kCT * 8 * kCandW;
constexpr int kCDbgCycles = kCV;
constexpr int kCDbgLam = kCV + 8;
constexpr int kCDbgPh = kCDbgLam + 4 * 64;
constexpr size_t kChainScratchFloats = kCDbgOffset + kCDbgPh + 16;

// one launch of the chain step: model (chain layout), state rows, and the
// per-robot status, counters (b3::Counters) and last contact counts of the
// chain robots
struct ChainLaunch {
  const float* mf;
  const int* mi;
  const unsigned long long* mk;
  const void* meta;  // int4 per robot
  const uint16_t* pairs;
  float* q;
  float* v;
  float* s;
  unsigned* status;
  void* counters;
  float* scratch;
  int* last_nc;
  int n;
};

}  // namespace b3
