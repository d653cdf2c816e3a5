// step_kernel.cuh -- persistent population-step kernel for sm_103a.
//
// One warp advances one robot ("variant", the unit of work of the paper's
// benchmarks, Sec. 4 "Simulation Parameters") for many steps without leaving
// the SM: the static model and the state live in registers and shared memory
// across steps, and only the launch's first load and last store touch HBM.
//
// Lane roles inside a warp (nb <= 26 bodies, nv = nb + 5 <= 31 dofs):
//   * lane = body    for the tree passes (FK, velocities, inertias, CPG);
//   * lane = field   for the leaf-to-root accumulations (one lane per spatial
//                    force / inertia component, serial over bodies);
//   * lane = row     for the Cholesky columns, the contact Jacobian rows and
//                    the Gauss-Seidel sweep of up to 10 contacts;
//   * lane = contact for the sweep of 11 to 32 contacts;
//   * lane = dof     for the triangular solves and the sweep of more;
//   * lane = pair    for the box/box broad and narrow phases.
//
// Gauss-Seidel works with Y_r = L^-1 J_r^T: the row residual J_r v =
// J_r v_free + Y_r . u with u = L^T (v - v_free), and the update
// v += M^-1 J_r^T dl is u += Y_r dl.  Up to 32 contacts the sweep runs in
// contact space on the residuals themselves (w += A_r. dl with the Delassus
// matrix A = Y Y^T), beyond in dof space on u; both are the iteration of
// sweeping in v (identical in exact arithmetic).  After the sweeps
// v+ = v_free + L^-T u.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "step_common.cuh"

namespace b3 {

constexpr unsigned kFull = 0xffffffffu;

// global scratch per variant: candidate rows, the narrow phase's per-lane
// staging rows, Y rows (32 floats each), the Gauss-Seidel constants of each
// contact (kCstG floats: b, 1/(A+R), R of its three rows, the normal-tangent
// couplings A_t1n, A_t2n, a zero, then the 3 x 3 block B_k = Y_(k+1) Y_k^T
// that couples it to the next contact of the sweep, row-major, and three
// zeros), the last step's v_free and impulses (inspection only), then the
// Delassus matrix of the lane-per-contact sweep (up to kLaneContacts^2 blocks
// of 3 x 3 floats, 12 apart)
constexpr int kCstG = 24;
constexpr int kLaneContacts = 32;  // lane-per-contact sweeps up to this many contacts
constexpr size_t kStageOffset = (size_t)kCand * kCandW;            // 32 lanes x 8 points x 8 floats
constexpr size_t kYOffset = kStageOffset + (size_t)32 * 8 * kCandW;
constexpr size_t kCstOffset = kYOffset + (size_t)kYRows * 32;
constexpr size_t kDbgOffset = kCstOffset + (size_t)kCapMax * kCstG;
constexpr int kPhases = 10;  // per-phase cycle counters (inspection only)
constexpr size_t kAOffset = kDbgOffset + 32 + 4 * kCapMax + 16;
constexpr size_t kScratchFloats = kAOffset + (size_t)kLaneContacts * kLaneContacts * 12;
static_assert(kAOffset % 4 == 0 && kScratchFloats % 4 == 0, "float4 rows of the scratch stay aligned");

struct __align__(16) WarpSmem {
  float R[9][32];          // body rotations (lane = body)
  float r[3][32];          // body frame origins relative to the core origin
  float c[3][32];          // box centres relative to the core origin
  float S[6][32];          // dof-indexed motion subspace columns
  // one region, four lifetimes within a step: the dynamics' accumulators,
  // then the contact generation's near pairs and kept-candidate masks, then
  // the contact rows and the Delassus matrix
  union {
    float acc[16][33];     // per-body f (6) + composite inertia (10), padded (steps 1-4)
    struct {
      uint16_t nearp[kMaxPairs];  // near body pairs of the step, (a << 8) | b (step 6)
      unsigned keep[kCand / 32];  // candidates kept under the cap (step 6)
    };
    float Yt[32][32];      // contact rows under construction, [dof][row] (step 7),
                           // then the Delassus matrix [row][row] (step 8)
  };
  float M[kTri];           // mass matrix, then its Cholesky factor (packed lower)
  float invd[32];
  float vfree[32];
  int8_t parent[32];
  unsigned path[32];
  unsigned long long ph[kPhases];  // per-phase SM cycles (inspection only)
};
// 16 warps of this (plus the 1 KB the SM reserves per block) fit a 164 KB
// shared-memory carve-out, which leaves the rest of the SM's 256 KB to L1
static_assert(16 * (sizeof(WarpSmem) + 1024) <= 164 * 1024, "per-warp shared memory");

__device__ __forceinline__ float shf(float x, int src) { return __shfl_sync(kFull, x, src); }

// Double-float arithmetic (Dekker 1971 products, Knuth two-sum): a value is
// h + l in FP32 with |l| <= ulp(h) / 2, about 44 bits.  The round-to-nearest
// intrinsics keep the compiler from fusing the error-free steps into FMAs.
struct f2 {
  float h, l;
};
__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ f2 quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const f2 s = two_sum(a.h, b.h);
  return quick_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ f2 f2_prod(float a, float b) {  // exact
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ f2 f2_mulf(f2 a, float b) {
  const f2 p = f2_prod(a.h, b);
  return quick_two_sum(p.h, __fmaf_rn(a.l, b, p.l));
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  const f2 p = f2_prod(a.h, b.h);
  return quick_two_sum(p.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l)));
}
__device__ __forceinline__ f2 f2_shf(f2 a, int src) { return {shf(a.h, src), shf(a.l, src)}; }
__device__ __forceinline__ int shfi(int x, int src) { return __shfl_sync(kFull, x, src); }

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Sums of three per-lane values over the warp, delivered to every lane.
// Pairs of values travel together in the first two butterfly levels, so
// three sums cost 9 shuffles instead of 15.
__device__ __forceinline__ void warp_sum3(float& a, float& b, float& c, int lane) {
  const bool h16 = (lane & 16) != 0;
  const float r0 = __shfl_xor_sync(kFull, h16 ? a : c, 16);
  const float r1 = __shfl_xor_sync(kFull, h16 ? b : 0.f, 16);
  const float x0 = (h16 ? c : a) + r0;  // lanes < 16: a, lanes >= 16: c
  const float x1 = (h16 ? 0.f : b) + r1;  // lanes < 16: b, lanes >= 16: 0
  const bool h8 = (lane & 8) != 0;
  float y = (h8 ? x1 : x0) + __shfl_xor_sync(kFull, h8 ? x0 : x1, 8);
  y += __shfl_xor_sync(kFull, y, 4);
  y += __shfl_xor_sync(kFull, y, 2);
  y += __shfl_xor_sync(kFull, y, 1);
  a = __shfl_sync(kFull, y, 0);
  b = __shfl_sync(kFull, y, 8);
  c = __shfl_sync(kFull, y, 16);
}

// forward substitution of L y = b with lane = dof; returns y on each lane
__device__ __forceinline__ float lower_solve(const WarpSmem& sm, float b, int nv, int lane) {
  float acc = b, y = 0.f;
#pragma unroll 1
  for (int i = 0; i < nv; ++i) {
    float yi = shf(acc, i) * sm.invd[i];
    if (lane == i) y = yi;
    if (lane > i && lane < nv) acc -= sm.M[tri(lane) + i] * yi;
  }
  return y;
}

// back substitution of L^T x = y with lane = dof
__device__ __forceinline__ float upper_solve(const WarpSmem& sm, float y, int nv, int lane) {
  float acc = y, x = 0.f;
#pragma unroll 1
  for (int i = nv - 1; i >= 0; --i) {
    float xi = shf(acc, i) * sm.invd[i];
    if (lane == i) x = xi;
    if (lane < i) acc -= sm.M[tri(i) + lane] * xi;
  }
  return x;
}

// Keep the cap deepest of ncand candidates (ties by list order), list order
// kept: ranks of every candidate first, then an in-order compaction
// (destination <= source).  Out of line: it runs only on steps whose
// candidates overflow the cap, and its code stays out of the step loop.
static_assert(kCandW == 8, "a candidate row moves as two float4");
static __device__ __noinline__ void keep_deepest(float* cand, int ncand, int cap, unsigned* keep_bits, int lane) {
#pragma unroll 1
  for (int i0 = 0; i0 < ncand; i0 += 32) {
    const int i = i0 + lane;
    bool keep = false;
    if (i < ncand) {
      const float di = cand[(size_t)i * kCandW + 6];
      int rank = 0;
#pragma unroll 1
      for (int j = 0; j < ncand; ++j) {
        const float dj = cand[(size_t)j * kCandW + 6];
        rank += (dj > di || (dj == di && j < i)) ? 1 : 0;
      }
      keep = rank < cap;
    }
    const unsigned bal = __ballot_sync(kFull, keep);
    if (lane == 0) keep_bits[i0 >> 5] = bal;
  }
  __syncwarp();
  int kept = 0;
#pragma unroll 1
  for (int i0 = 0; i0 < ncand; i0 += 32) {
    const int i = i0 + lane;
    const unsigned bal = keep_bits[i0 >> 5];
    const bool keep = (bal >> lane) & 1u;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (keep) {
      const float4* src = reinterpret_cast<const float4*>(cand + (size_t)i * kCandW);
      r0 = src[0];
      r1 = src[1];
    }
    __syncwarp();
    if (keep) {
      float4* dst = reinterpret_cast<float4*>(cand + (size_t)(kept + __popc(bal & ((1u << lane) - 1u))) * kCandW);
      dst[0] = r0;
      dst[1] = r1;
    }
    kept += __popc(bal);
    __syncwarp();
  }
}

// Gauss-Seidel sweeps of 11 to kLaneContacts contacts in contact space,
// lane c = contact c: the lane keeps the residuals w = J v_free - bias +
// A lam of its contact's three rows, their impulses and their constants in
// registers.  Every lane forms the update of its own contact from its own
// residuals; the sweep takes lane k's, broadcast with three shuffles, and
// every lane adds A_(c,k) dlam_k to its residuals, reading its 3 x 3 block of
// the Delassus matrix A = Y Y^T from the global scratch (built here, blocks
// prefetched two updates ahead).  The same iteration as the dof-space sweep;
// the update's dependency chain has one shuffle and no warp reduction.
// Returns u (this lane's dof) and leaves every contact's impulses in lamS.
static __device__ __noinline__ float lane_contact_sweep(float4* lamS, const float* __restrict__ cstg,
                                                        const float* __restrict__ Yg, float* __restrict__ Ag,
                                                        int nc, int nv, int iters, float mu, int lane) {
  // A = Y Y^T, lane = row r: block (k, c) (rows of contact c, columns of
  // contact k) at Ag + (k nc + c) 12, row-major 3 x 3 with 3 floats of
  // padding.  A is symmetric: lane r forms A_rs for s >= r and writes it to
  // both places, so a pass of 32 rows starts at its own first row.
  const int nr = 3 * nc;
#pragma unroll 1
  for (int r0 = 0; r0 < nr; r0 += 32) {
    const int r = r0 + lane;
    const bool act = r < nr;
    float y[32];
    {
      const float4* Yr = reinterpret_cast<const float4*>(Yg + (size_t)(act ? r : 0) * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 t = Yr[q];
        y[4 * q] = t.x; y[4 * q + 1] = t.y; y[4 * q + 2] = t.z; y[4 * q + 3] = t.w;
      }
    }
    const int c = r / 3, dr = r - 3 * c;
    float* dst = Ag + (size_t)c * 12 + 3 * dr;    // A_rs: block (ks, c), entry (dr, ds)
    float* mir = Ag + (size_t)c * nc * 12 + dr;   // A_sr: block (c, ks), entry (ds, dr)
    int ks = r0 / 3, ds = r0 - 3 * ks;  // column s = 3 ks + ds
#pragma unroll 1
    for (int s = r0; s < nr; ++s) {
      const float4* Ys = reinterpret_cast<const float4*>(Yg + (size_t)s * 32);
      float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        if (4 * q < nv) {
          const float4 t = Ys[q];
          acc0 = fmaf(y[4 * q], t.x, fmaf(y[4 * q + 1], t.y, fmaf(y[4 * q + 2], t.z, fmaf(y[4 * q + 3], t.w, acc0))));
        }
        if (4 * q + 4 < nv) {
          const float4 t = Ys[q + 1];
          acc1 = fmaf(y[4 * q + 4], t.x, fmaf(y[4 * q + 5], t.y, fmaf(y[4 * q + 6], t.z, fmaf(y[4 * q + 7], t.w, acc1))));
        }
      }
      if (act && s >= r) {
        const float a = acc0 + acc1;
        dst[(size_t)ks * nc * 12 + ds] = a;
        mir[(size_t)ks * 12 + 3 * ds] = a;
      }
      if (++ds == 3) {
        ds = 0;
        ++ks;
      }
    }
  }
  // this lane's contact: residuals (from J v_free - bias), impulses and, with
  // g = 1/(A+R), a = 1 - R g, b = g A_tn: (g_n, a_n, g_t1, a_t1, b_t1, g_t2, a_t2, b_t2)
  const bool mine = lane < nc;
  float wn = 0.f, w1 = 0.f, w2 = 0.f;
  float gn = 0.f, an = 1.f, g1 = 0.f, a1 = 1.f, b1 = 0.f, g2 = 0.f, a2 = 1.f, b2 = 0.f;
  if (mine) {
    const float4* c4 = reinterpret_cast<const float4*>(cstg) + 6 * lane;
    // (b_n, g_n, R_n, b_t1), (g_t1, R_t1, b_t2, g_t2), (R_t2, A_t1n, A_t2n, 0)
    const float4 x0 = c4[0], x1 = c4[1], x2 = c4[2];
    wn = x0.x; gn = x0.y; an = fmaf(-x0.z, x0.y, 1.f); w1 = x0.w;
    g1 = x1.x; a1 = fmaf(-x1.y, x1.x, 1.f); b1 = x1.x * x2.y;
    w2 = x1.z; g2 = x1.w; a2 = fmaf(-x2.x, x1.w, 1.f); b2 = x1.w * x2.z;
  }
  __syncwarp();  // the blocks written above are read by other lanes
  float ln = 0.f, l1 = 0.f, l2 = 0.f;
  const float4* A4 = reinterpret_cast<const float4*>(Ag) + 3 * lane;
  const int kstride = 3 * nc;  // float4 between block rows k and k + 1
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // Three register sets hold the blocks of the current contact, the next one
  // and the one after (prefetch distance 2); the loop is unrolled by three so
  // that the sets rotate by name instead of by register moves.
  struct Blk {
    float4 x, y, z;
  };
  Blk A = {mine ? A4[0] : z4, mine ? A4[1] : z4, mine ? A4[2] : z4};
  Blk B = {mine ? A4[kstride] : z4, mine ? A4[kstride + 1] : z4, mine ? A4[kstride + 2] : z4};
  Blk C;
  const int nupd = iters * nc;
  int k = 0, k2 = 2;  // contact of this update, and of the block loaded now
  // one update with the block of contact k in `cur`; the block of contact k2
  // is loaded into `load`
  auto update = [&](const Blk& cur, Blk& load) {
    const float4* An = A4 + (size_t)kstride * k2;
    load.x = mine ? An[0] : z4;
    load.y = mine ? An[1] : z4;
    load.z = mine ? An[2] : z4;
    const float lnn = fmaxf(0.f, fmaf(-gn, wn, an * ln));
    const float dn = lnn - ln;
    const float l1t = fmaf(-b1, dn, fmaf(-g1, w1, a1 * l1));
    const float l2t = fmaf(-b2, dn, fmaf(-g2, w2, a2 * l2));
    const float sc = fminf(1.f, (mu * lnn) * rsqrt_ftz(fmaf(l1t, l1t, l2t * l2t)));
    const float d1 = fmaf(l1t, sc, -l1), d2 = fmaf(l2t, sc, -l2);
    const float Dn = shf(dn, k), D1 = shf(d1, k), D2 = shf(d2, k);
    if (lane == k) {
      ln = lnn;
      l1 = l1t * sc;
      l2 = l2t * sc;
    }
    // block (k, lane) row-major: (a00 a01 a02 a10) (a11 a12 a20 a21) (a22 . . .)
    wn = fmaf(cur.x.z, D2, fmaf(cur.x.y, D1, fmaf(cur.x.x, Dn, wn)));
    w1 = fmaf(cur.y.y, D2, fmaf(cur.y.x, D1, fmaf(cur.x.w, Dn, w1)));
    w2 = fmaf(cur.z.x, D2, fmaf(cur.y.w, D1, fmaf(cur.y.z, Dn, w2)));
    k = k + 1 < nc ? k + 1 : 0;
    k2 = k2 + 1 < nc ? k2 + 1 : 0;
  };
#pragma unroll 1
  for (int upd = 0; upd < nupd; upd += 3) {
    update(A, C);
    if (upd + 1 >= nupd) break;
    update(B, A);
    if (upd + 2 >= nupd) break;
    update(C, B);
  }
  if (mine) lamS[lane] = make_float4(ln, l1, l2, 0.f);
  __syncwarp();
  // u = sum_r Y_r lam_r (lane = dof)
  float u = 0.f;
#pragma unroll 1
  for (int kk = 0; kk < nc; ++kk) {
    const float4 l4 = lamS[kk];
    const float* Yk = Yg + (size_t)(3 * kk) * 32 + lane;
    u += l4.x * Yk[0] + l4.y * Yk[32] + l4.z * Yk[64];
  }
  return u;
}

// Gauss-Seidel sweeps of more than kLaneContacts contacts in dof space; returns u (this
// lane's dof) and leaves every contact's impulses in lamS.  Out of line, so
// that its code sits outside the step loop that most robots run.
static __device__ __noinline__ float dof_space_sweep(float4* lamS, const float* __restrict__ cstg,
                                                     const float* __restrict__ Yg, int nc, int iters, float mu,
                                                     int lane) {
  // Dof space (lane = dof, u = L^T (v - v_free)), one contact of
  // lookahead: the next contact's row products are reduced over the warp
  // from u before the current update lands, then brought up to date with
  // B_k (u changes by Y_k^T dlam_k), so that the five-level reduction
  // runs beside the update instead of ahead of it.  Contact impulses sit
  // in shared memory: every lane computes and stores them alike and reads
  // back its own writes.
#pragma unroll 1
  for (int k0 = lane; k0 < nc; k0 += 32) lamS[k0] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncwarp();
  const float4* c4 = reinterpret_cast<const float4*>(cstg);
  // more than kLaneContacts contacts here: the next contact is never the current one
  int k = 0, kn = 1;
  float y0 = Yg[lane], y1 = Yg[32 + lane], y2 = Yg[64 + lane];
  const float* Zn = Yg + (size_t)(3 * kn) * 32;
  float z0 = Zn[lane], z1 = Zn[32 + lane], z2 = Zn[64 + lane];
  float u = 0.f;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;  // Y_k . u before update k (u = 0 at the start)
  float ln = 0.f, l1 = 0.f, l2 = 0.f;  // impulses of contact k
  const int nupd = iters * nc;
#pragma unroll 1
  for (int upd = 0; upd < nupd; ++upd) {
    const int knn = (kn + 1 < nc) ? kn + 1 : 0;
    // this contact's constants and coupling block B_k (loaded first, used
    // after the reduction's shuffles); the next one's impulses and the
    // rows after it
    const float4 ca = c4[6 * k], cb4 = c4[6 * k + 1], cc4 = c4[6 * k + 2];
    const float4 bq0 = c4[6 * k + 3], bq1 = c4[6 * k + 4], bq2 = c4[6 * k + 5];
    const float4 nl = lamS[kn];
    const float* Zz = Yg + (size_t)(3 * knn) * 32;
    const float zz0 = Zz[lane], zz1 = Zz[32 + lane], zz2 = Zz[64 + lane];
    // the next contact's row products against u before this update
    float p0 = z0 * u, p1 = z1 * u, p2 = z2 * u;
    warp_sum3(p0, p1, p2, lane);
    // constants: (b_n, inv_n, R_n, b_t1), (inv_t1, R_t1, b_t2, inv_t2), (R_t2, A_t1n, A_t2n, 0)
    const float gn = s0 + ca.x + ca.z * ln;
    const float lnn = fmaxf(0.f, ln - gn * ca.y);
    const float dn = lnn - ln;
    const float g1 = s1 + cc4.y * dn + ca.w + cb4.y * l1;
    const float g2 = s2 + cc4.z * dn + cb4.z + cc4.x * l2;
    float l1t = l1 - g1 * cb4.x;
    float l2t = l2 - g2 * cb4.w;
    const float lim = mu * lnn;
    const float nt2 = l1t * l1t + l2t * l2t;
    const float sc = fminf(1.f, lim * rsqrt_ftz(nt2));
    l1t *= sc;
    l2t *= sc;
    const float d1 = l1t - l1, d2 = l2t - l2;
    u += y0 * dn + y1 * d1 + y2 * d2;
    lamS[k] = make_float4(lnn, l1t, l2t, 0.f);
    // B_k row-major in bq0..bq2: (b00 b01 b02 b10) (b11 b12 b20 b21) (b22 ...)
    s0 = p0 + bq0.x * dn + bq0.y * d1 + bq0.z * d2;
    s1 = p1 + bq0.w * dn + bq1.x * d1 + bq1.y * d2;
    s2 = p2 + bq1.z * dn + bq1.w * d1 + bq2.x * d2;
    ln = nl.x;
    l1 = nl.y;
    l2 = nl.z;
    y0 = z0; y1 = z1; y2 = z2;
    z0 = zz0; z1 = zz1; z2 = zz2;
    k = kn;
    kn = knn;
  }
  __syncwarp();
  return u;
}

struct Counters {
  unsigned long long contacts, narrow, broad, steps, cycles;
};

// Resident warps per SM that a kernel instance's register budget is sized
// for (WPSM): 16 (128 registers per thread) or 12 (168).  With 12 the compiler
// keeps more values in registers and each warp runs its step faster, but
// fewer robots run at once: the first wins where a launch lasts as long as
// its slowest robot (a few thousand uneven robots), the second where the
// SMs' throughput decides (tens of thousands of robots).  The autotuner
// times both.

// Block barriers per step of a phase-locked launch (LOCK): the warps of a
// block pass every phase boundary together, so that the SM runs few distinct
// phases at a time (instruction-cache locality) at the cost of waiting for the
// block's slowest robot at each boundary.
constexpr int kLockBarriers = 5;

template <int WPB, bool LOCK, int WPSM>
__global__ void __launch_bounds__(WPB * 32, WPSM / WPB)
step_kernel(const float* __restrict__ mf, const int* __restrict__ mi, const int4* __restrict__ meta,
            const uint16_t* __restrict__ pairs, float* __restrict__ qg, float* __restrict__ vg,
            float* __restrict__ sg, unsigned* __restrict__ status, Counters* __restrict__ counters,
            float* __restrict__ scratch, int* __restrict__ last_nc, const int* __restrict__ order, int nvar,
            int nsteps, StepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int slot = blockIdx.x * WPB + wib;
  if (slot >= nvar) {
    if constexpr (LOCK) {
      // a warp without a robot still takes every block barrier of every step
      for (int step = 0; step < nsteps; ++step)
        for (int b = 0; b < kLockBarriers; ++b) __syncthreads();
    }
    return;
  }
  // launch slot -> variant: slowest-first order when given (see cost_order)
  const int var = order ? __ldg(order + slot) : slot;
  WarpSmem& sm = reinterpret_cast<WarpSmem*>(smem_raw)[wib];

  const int4 md = meta[var];
  const int nb = md.x, maxdepth = md.y, npairs = md.z, pairoff = md.w;
  const int nv = nb + 5;
  const bool body = lane < nb;
  const bool hinge = lane >= 1 && lane < nb;

  // static model: [field][body slot] in global memory (L1/L2 resident), read
  // where it is used; only the topology lives in registers
  const float* __restrict__ F = mf + (size_t)var * NF * 32;
  const int* IM = mi + (size_t)var * NI * 32;
  const int parent = body ? IM[I_PARENT * 32 + lane] : -1;
  const int axis = IM[I_AXIS * 32 + lane];
  const unsigned childm = (unsigned)IM[I_CHILD * 32 + lane];
  const int depth = body ? IM[I_DEPTH * 32 + lane] : 0;
  sm.parent[lane] = parent;
  sm.path[lane] = (unsigned)IM[I_PATH * 32 + lane];
  const int par0 = parent > 0 ? parent : 0;
  auto fld = [&](int f) { return __ldg(F + f * 32 + lane); };

  // ---- state
  float* qv = qg + (size_t)var * 32;
  float* vv = vg + (size_t)var * 32;
  float* sv = sg + (size_t)var * 64;
  float p0x = qv[0], p0y = qv[1], p0z = qv[2];
  float qw = qv[3], qx = qv[4], qy = qv[5], qz = qv[6];
  float theta = hinge ? qv[6 + lane] : 0.f;
  float vd = lane < nv ? vv[lane] : 0.f;
  float xo = hinge ? sv[2 * (lane - 1)] : 0.f;
  float yo = hinge ? sv[2 * (lane - 1) + 1] : 0.f;
  unsigned st = status[var];
  unsigned n_contacts = 0, n_narrow = 0, n_broad = 0, n_steps = 0;
  int nc_last = last_nc[var];
  float vfree_last = 0.f;
  float lam_a[3] = {0.f, 0.f, 0.f}, lam_b[3] = {0.f, 0.f, 0.f};  // impulses of contacts lane, lane + 32

  const long long t_start = clock64();
  // per-phase SM cycles (accumulated by lane 0 in shared memory):
  // 0 CPG+FK, 1 inertias+RNEA+CRBA, 2 Cholesky+v_free, 3 ground contacts,
  // 4 box/box, 5 cap, 6 contact rows, 7 Gauss-Seidel, 8 integration
  if (lane < kPhases) sm.ph[lane] = 0ull;
  long long tph = clock64();
#define B3_PHASE(i)                                                  \
  do {                                                               \
    const long long t_ = clock64();                                  \
    if (lane == 0) sm.ph[i] += (unsigned long long)(t_ - tph);       \
    tph = t_;                                                        \
  } while (0)
#define B3_LOCK()                \
  do {                           \
    if constexpr (LOCK) {        \
      __syncwarp();              \
      __syncthreads();           \
    }                            \
  } while (0)
  float* cand = scratch + (size_t)var * kScratchFloats;
  float* Yg = cand + kYOffset;
  float* cstg = cand + kCstOffset;
  __syncwarp();

  for (int step = 0; step < nsteps; ++step) {
    // frozen (non-finite state or failed factorisation): stop, or under LOCK
    // keep computing on the frozen state without committing it, so that every
    // warp takes the same barriers
    if constexpr (!LOCK) {
      if (st & 5u) break;
    }
    const float dt = P.dt;

    // ---------------- 1. CPG and PD torque (lane = body / hinge)
    float xn = xo, yn = yo, tau_b = 0.f;
    const float thd_b = shf(vd, (5 + lane) & 31);
    if (P.actuate) {
      const float wint = fld(F_WINT), wcpl = fld(F_WCPL);
      sm.acc[0][lane] = (hinge && parent >= 1) ? wcpl * xo : 0.f;
      __syncwarp();
      float dx = wint * yo, dy = -wint * xo;
      const float xp = shf(xo, par0);
      if (hinge && parent >= 1) dx -= wcpl * xp;
#pragma unroll 1
      for (unsigned m = hinge ? childm : 0u; m; m &= m - 1) dx += sm.acc[0][__ffs(m) - 1];
      __syncwarp();
      xn = xo + dt * dx;
      yn = yo + dt * dy;
      if (hinge) {
        float x = fminf(fmaxf(xn, -1.f), 1.f);
        float t = P.kp * (P.theta_max * x - theta) - P.kd * thd_b;
        tau_b = fminf(fmaxf(t, -P.tau_max), P.tau_max);
      }
    }
    float tau_d = shf(tau_b, (lane - 5) & 31);
    if (lane < 6 || lane >= nv) tau_d = 0.f;

    // ---------------- 2. forward kinematics (lane = body, level by level)
    float R0[9];
    quat_to_R(qw, qx, qy, qz, R0);
    float R[9], r[3] = {0.f, 0.f, 0.f};
    // hinge angle sine and cosine in FP64 (the height chain below needs them
    // there); the FP32 kinematics use them rounded
    double sd, cd;
    sincos_f64((double)theta, &sd, &cd);
    const float sth = (float)sd, cth = (float)cd;
    {
      float Rl[9];
      const int k = axis, i = (axis + 1) % 3, j = (axis + 2) % 3;
#pragma unroll
      for (int row = 0; row < 3; ++row) {
        const float fi = fld(F_RFIX + 3 * row + i), fj = fld(F_RFIX + 3 * row + j);
        Rl[3 * row + k] = fld(F_RFIX + 3 * row + k);
        Rl[3 * row + i] = cth * fi + sth * fj;
        Rl[3 * row + j] = -sth * fi + cth * fj;
      }
      const float pf0 = fld(F_PFIX), pf1 = fld(F_PFIX + 1), pf2 = fld(F_PFIX + 2);
#pragma unroll
      for (int k2 = 0; k2 < 9; ++k2) R[k2] = R0[k2];
#pragma unroll 1
      for (int lvl = 1; lvl <= maxdepth; ++lvl) {
        float Rp[9], rp[3];
#pragma unroll
        for (int k2 = 0; k2 < 9; ++k2) Rp[k2] = shf(R[k2], par0);
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) rp[k2] = shf(r[k2], par0);
        if (depth == lvl) {
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
              R[3 * a + b] = Rp[3 * a] * Rl[b] + Rp[3 * a + 1] * Rl[3 + b] + Rp[3 * a + 2] * Rl[6 + b];
#pragma unroll
          for (int a = 0; a < 3; ++a) r[a] = rp[a] + (Rp[3 * a] * pf0 + Rp[3 * a + 1] * pf1 + Rp[3 * a + 2] * pf2);
        }
      }
    }
    // Height chain for the ground contacts in double-float: the third row of
    // R_b and the frame-origin height relative to O.  A contact's push-out
    // speed is ERP * depth / dt with depths of ~0.1 mm, so contact activation
    // and depth are taken from heights about as exact as the FP64 reference's
    // (from the FP32 state); everything else stays FP32.
    f2 hz0, hz1, hz2, hzb = {0.f, 0.f};
    {
      hz0 = f2_add(f2_prod(qx, qz), f2_neg(f2_prod(qw, qy)));
      hz1 = f2_add(f2_prod(qy, qz), f2_prod(qw, qx));
      hz0 = {2.f * hz0.h, 2.f * hz0.l};
      hz1 = {2.f * hz1.h, 2.f * hz1.l};
      const f2 xy = f2_add(f2_prod(qx, qx), f2_prod(qy, qy));
      hz2 = f2_add(f2{1.f, 0.f}, f2{-2.f * xy.h, -2.f * xy.l});
      const f2 cdf = {cth, (float)(cd - (double)cth)}, sdf = {sth, (float)(sd - (double)sth)};
      const int k = axis;  // columns i = k + 1, j = k + 2 (mod 3) mix
      // the fixed frame's rows and offset (exact FP32 model values)
      float Fr[9], Fp[3];
#pragma unroll
      for (int t = 0; t < 9; ++t) Fr[t] = fld(F_RFIX + t);
#pragma unroll
      for (int t = 0; t < 3; ++t) Fp[t] = fld(F_PFIX + t);
      // A lattice joint rotation (every column one entry +-1, the others 0)
      // turns the row-times-matrix product into a signed pick of one entry
      // per column, which is what the double-float products give exactly (a
      // normalised pair times +-1 or 0, plus zeros): taken when every body of
      // the robot has one.
      int rc[3];
      float sg[3];
      bool lat = true;
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        const float a0 = Fr[col], a1 = Fr[3 + col], a2 = Fr[6 + col];
        rc[col] = a0 != 0.f ? 0 : (a1 != 0.f ? 1 : 2);
        sg[col] = a0 + a1 + a2;
        const int nz = (a0 != 0.f) + (a1 != 0.f) + (a2 != 0.f);
        lat = lat && nz == 1 && fabsf(sg[col]) == 1.f;
      }
      const bool lattice = __all_sync(kFull, lat);
#pragma unroll 1
      for (int lvl = 1; lvl <= maxdepth; ++lvl) {
        const f2 p0 = f2_shf(hz0, par0), p1 = f2_shf(hz1, par0), p2 = f2_shf(hz2, par0), pb = f2_shf(hzb, par0);
        if (depth == lvl) {
          // (third row of R_parent) x R_fix, then the hinge rotation mixes columns i, j
          f2 t[3];
          if (lattice) {
#pragma unroll
            for (int col = 0; col < 3; ++col) {
              const f2 pc = rc[col] == 0 ? p0 : (rc[col] == 1 ? p1 : p2);
              t[col] = {pc.h * sg[col], pc.l * sg[col]};
            }
          } else {
#pragma unroll
            for (int col = 0; col < 3; ++col)
              t[col] = f2_add(f2_add(f2_mulf(p0, Fr[col]), f2_mulf(p1, Fr[3 + col])), f2_mulf(p2, Fr[6 + col]));
          }
          const f2 ti = k == 0 ? t[1] : (k == 1 ? t[2] : t[0]);
          const f2 tj = k == 0 ? t[2] : (k == 1 ? t[0] : t[1]);
          const f2 tk = k == 0 ? t[0] : (k == 1 ? t[1] : t[2]);
          const f2 oi = f2_add(f2_mul(cdf, ti), f2_mul(sdf, tj));
          const f2 oj = f2_add(f2_mul(cdf, tj), f2_neg(f2_mul(sdf, ti)));
          // out[k] = tk, out[i] = oi, out[j] = oj with i = k + 1, j = k + 2 (mod 3)
          hz0 = k == 0 ? tk : (k == 1 ? oj : oi);
          hz1 = k == 0 ? oi : (k == 1 ? tk : oj);
          hz2 = k == 0 ? oj : (k == 1 ? oi : tk);
          hzb = f2_add(pb, f2_add(f2_add(f2_mulf(p0, Fp[0]), f2_mulf(p1, Fp[1])), f2_mulf(p2, Fp[2])));
        }
      }
    }
    float cb[3];
    {
      const float c0 = fld(F_COM), c1 = fld(F_COM + 1), c2 = fld(F_COM + 2);
#pragma unroll
      for (int a = 0; a < 3; ++a) cb[a] = r[a] + (R[3 * a] * c0 + R[3 * a + 1] * c1 + R[3 * a + 2] * c2);
    }
    float Sb[6];
    Sb[0] = R[axis]; Sb[1] = R[3 + axis]; Sb[2] = R[6 + axis];
    cross3(r, Sb, Sb + 3);
#pragma unroll
    for (int k = 0; k < 9; ++k) sm.R[k][lane] = R[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) { sm.r[k][lane] = r[k]; sm.c[k][lane] = cb[k]; }
    if (hinge) {
#pragma unroll
      for (int k = 0; k < 6; ++k) sm.S[k][5 + lane] = Sb[k];
    }
    if (lane < 6) {
      float col[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (lane < 3) col[3 + lane] = 1.f;
      else { col[0] = R0[lane - 3]; col[1] = R0[3 + lane - 3]; col[2] = R0[6 + lane - 3]; }
#pragma unroll
      for (int k = 0; k < 6; ++k) sm.S[k][lane] = col[k];
    }

    B3_PHASE(0);
    // ---------------- 3. spatial inertias and RNEA bias forces
    {
      float I[10];
      {
        const float mass = fld(F_MASS), i0 = fld(F_ID), i1 = fld(F_ID + 1), i2 = fld(F_ID + 2);
        float Iw[6];  // xx yy zz xy xz yz of R diag(Id) R^T
        Iw[0] = R[0] * R[0] * i0 + R[1] * R[1] * i1 + R[2] * R[2] * i2;
        Iw[1] = R[3] * R[3] * i0 + R[4] * R[4] * i1 + R[5] * R[5] * i2;
        Iw[2] = R[6] * R[6] * i0 + R[7] * R[7] * i1 + R[8] * R[8] * i2;
        Iw[3] = R[0] * R[3] * i0 + R[1] * R[4] * i1 + R[2] * R[5] * i2;
        Iw[4] = R[0] * R[6] * i0 + R[1] * R[7] * i1 + R[2] * R[8] * i2;
        Iw[5] = R[3] * R[6] * i0 + R[4] * R[7] * i1 + R[5] * R[8] * i2;
        const float cc = cb[0] * cb[0] + cb[1] * cb[1] + cb[2] * cb[2];
        I[0] = mass;
        I[1] = mass * cb[0]; I[2] = mass * cb[1]; I[3] = mass * cb[2];
        I[4] = Iw[0] + mass * (cc - cb[0] * cb[0]);
        I[5] = Iw[1] + mass * (cc - cb[1] * cb[1]);
        I[6] = Iw[2] + mass * (cc - cb[2] * cb[2]);
        I[7] = Iw[3] - mass * cb[0] * cb[1];
        I[8] = Iw[4] - mass * cb[0] * cb[2];
        I[9] = Iw[5] - mass * cb[1] * cb[2];
      }
      const float vlx = shf(vd, 0), vly = shf(vd, 1), vlz = shf(vd, 2);
      const float wbx = shf(vd, 3), wby = shf(vd, 4), wbz = shf(vd, 5);
      float vb[6], ab[6];
      {
        float om[3] = {R0[0] * wbx + R0[1] * wby + R0[2] * wbz, R0[3] * wbx + R0[4] * wby + R0[5] * wbz,
                       R0[6] * wbx + R0[7] * wby + R0[8] * wbz};
        float vl[3] = {vlx, vly, vlz};
        float vxw[3];
        cross3(vl, om, vxw);
        vb[0] = om[0]; vb[1] = om[1]; vb[2] = om[2]; vb[3] = vlx; vb[4] = vly; vb[5] = vlz;
        ab[0] = 0.f; ab[1] = 0.f; ab[2] = 0.f;
        ab[3] = vxw[0] - P.gx; ab[4] = vxw[1] - P.gy; ab[5] = vxw[2] - P.gz;
      }
#pragma unroll 1
      for (int lvl = 1; lvl <= maxdepth; ++lvl) {
        float vp[6], ap[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) { vp[k] = shf(vb[k], par0); ap[k] = shf(ab[k], par0); }
        if (depth == lvl) {
          float Sq[6], cr[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) { Sq[k] = Sb[k] * thd_b; vb[k] = vp[k] + Sq[k]; }
          crm(vb, Sq, cr);
#pragma unroll
          for (int k = 0; k < 6; ++k) ab[k] = ap[k] + cr[k];
        }
      }
      float Ia[6], Iv[6], x[6];
      inertia_apply(I, ab, Ia);
      inertia_apply(I, vb, Iv);
      crf(vb, Iv, x);
#pragma unroll
      for (int k = 0; k < 6; ++k) sm.acc[k][lane] = body ? Ia[k] + x[k] : 0.f;
#pragma unroll
      for (int k = 0; k < 10; ++k) sm.acc[6 + k][lane] = body ? I[k] : 0.f;
    }
    __syncwarp();
    // leaf-to-root sums of forces and inertias, lane = component
    if (lane < 16) {
#pragma unroll 1
      for (int b = nb - 1; b >= 1; --b) {
        const int p = sm.parent[b];
        sm.acc[lane][p] += sm.acc[lane][b];
      }
    }
    __syncwarp();
    float c_d;
    {
      float cbh = 0.f;
      if (hinge) {
        cbh = Sb[0] * sm.acc[0][lane] + Sb[1] * sm.acc[1][lane] + Sb[2] * sm.acc[2][lane] +
              Sb[3] * sm.acc[3][lane] + Sb[4] * sm.acc[4][lane] + Sb[5] * sm.acc[5][lane];
      }
      c_d = shf(cbh, (lane - 5) & 31);
      if (lane < 3) c_d = sm.acc[3 + lane][0];
      else if (lane < 6) {
        const int k = lane - 3;
        c_d = R0[k] * sm.acc[0][0] + R0[3 + k] * sm.acc[1][0] + R0[6 + k] * sm.acc[2][0];
      }
    }

    // ---------------- 4. CRBA mass matrix (packed lower triangle)
    if (lane < nv)
#pragma unroll 1
      for (int j = 0; j <= lane; ++j) sm.M[tri(lane) + j] = 0.f;
    __syncwarp();
    if (hinge) {
      float Ic[10], Fv[6];
#pragma unroll
      for (int k = 0; k < 10; ++k) Ic[k] = sm.acc[6 + k][lane];
      inertia_apply(Ic, Sb, Fv);
      const int i = 5 + lane;
      const int ti = tri(i);
      sm.M[ti + i] = Sb[0] * Fv[0] + Sb[1] * Fv[1] + Sb[2] * Fv[2] + Sb[3] * Fv[3] + Sb[4] * Fv[4] + Sb[5] * Fv[5] +
                     P.armature;
#pragma unroll 1
      for (int j = parent; j > 0; j = sm.parent[j]) {
        const int jj = 5 + j;
        sm.M[ti + jj] = sm.S[0][jj] * Fv[0] + sm.S[1][jj] * Fv[1] + sm.S[2][jj] * Fv[2] + sm.S[3][jj] * Fv[3] +
                        sm.S[4][jj] * Fv[4] + sm.S[5][jj] * Fv[5];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) sm.M[ti + k] = Fv[3 + k];
#pragma unroll
      for (int k = 0; k < 3; ++k) sm.M[ti + 3 + k] = R0[k] * Fv[0] + R0[3 + k] * Fv[1] + R0[6 + k] * Fv[2];
    }
    if (lane < 6) {
      float Ic[10], Sk[6], Fv[6];
#pragma unroll
      for (int k = 0; k < 10; ++k) Ic[k] = sm.acc[6 + k][0];
#pragma unroll
      for (int k = 0; k < 6; ++k) Sk[k] = sm.S[k][lane];
      inertia_apply(Ic, Sk, Fv);
#pragma unroll 1
      for (int l = lane; l < 6; ++l)
        sm.M[tri(l) + lane] = sm.S[0][l] * Fv[0] + sm.S[1][l] * Fv[1] + sm.S[2][l] * Fv[2] + sm.S[3][l] * Fv[3] +
                              sm.S[4][l] * Fv[4] + sm.S[5][l] * Fv[5];
    }
    __syncwarp();

    B3_PHASE(1);
    B3_LOCK();
    // ---------------- 5. Cholesky (left-looking, lane = row) and v_free
    // Column j: every row i >= j forms s_i = sum_{k<j} L_ik L_jk from its own
    // finished row and the broadcast row j (independent loads, no
    // read-modify-write chain through shared memory); lane j turns its value
    // into the pivot, the rows below divide by it.
    bool chol_ok = true;
    {
      const float* Li = sm.M + tri(lane);
      const bool row = lane < nv;
#pragma unroll 1
      for (int j = 0; j < nv; ++j) {
        const float* Lj = sm.M + tri(j);
        float s0 = 0.f, s1 = 0.f;
        if (row && lane >= j) {
          // four terms an iteration with their loads first (one load latency
          // per four terms); even terms to s0, odd to s1, in order
          int k = 0;
#pragma unroll 1
          for (; k + 3 < j; k += 4) {
            const float a0 = Li[k], b0 = Lj[k], a1 = Li[k + 1], b1 = Lj[k + 1];
            const float a2 = Li[k + 2], b2 = Lj[k + 2], a3 = Li[k + 3], b3 = Lj[k + 3];
            s0 += a0 * b0;
            s1 += a1 * b1;
            s0 += a2 * b2;
            s1 += a3 * b3;
          }
          if (k + 1 < j) {
            s0 += Li[k] * Lj[k];
            s1 += Li[k + 1] * Lj[k + 1];
            k += 2;
          }
          if (k < j) s0 += Li[k] * Lj[k];
        }
        const float mij = (row && lane >= j) ? Li[j] - (s0 + s1) : 0.f;
        const float piv = shf(mij, j);
        if (!(piv > 0.f)) { chol_ok = false; break; }
        // the pivot's root and its reciprocal from one SFU reciprocal square
        // root (the rounded square root and division sit on the column chain)
        const float inv = rsqrt_ftz(piv);
        const float d = piv * inv;
        if (lane == j) { sm.M[tri(j) + j] = d; sm.invd[j] = inv; }
        if (row && lane > j) sm.M[tri(lane) + j] = mij * inv;
        __syncwarp();
      }
    }
    if (!chol_ok) {
      st |= 4u;
      if constexpr (!LOCK) break;
    }
    float vfree;
    {
      float y = lower_solve(sm, tau_d - c_d, nv, lane);
      float acc = upper_solve(sm, y, nv, lane);
      vfree = vd + dt * acc;
      sm.vfree[lane] = lane < nv ? vfree : 0.f;
      vfree_last = sm.vfree[lane];
    }

    B3_PHASE(2);
    B3_LOCK();
    // ---------------- 6. contact candidates
    int ncand = 0;
    if (P.ground) {
      // a box's 8 vertices (bit i of k: + half size along axis i); a
      // sphere's lowest point: k = 0 with no half-size offsets, r below
      unsigned mask8 = 0;
      const bool sph = fld(F_GEOM) != 0.f;
      const float hr = fld(F_HALF);
      const float h0 = sph ? 0.f : hr, h1 = sph ? 0.f : fld(F_HALF + 1), h2 = sph ? 0.f : fld(F_HALF + 2);
      const float drop = sph ? hr : 0.f;
      const float c0 = fld(F_COM), c1 = fld(F_COM + 1), c2 = fld(F_COM + 2);
      // vertex height p0z + (hzb + hz . l) - drop in double-float
      auto vheight = [&](int k) {
        const float l0 = c0 + ((k & 1) ? h0 : -h0), l1 = c1 + ((k & 2) ? h1 : -h1), l2 = c2 + ((k & 4) ? h2 : -h2);
        const f2 hl = f2_add(f2_add(f2_mulf(hz0, l0), f2_mulf(hz1, l1)), f2_mulf(hz2, l2));
        return f2_add(f2_add(two_sum(p0z, -drop), hzb), hl);
      };
      auto below = [](f2 h) { return h.h < 0.f || (h.h == 0.f && h.l < 0.f); };
      // the depths of the vertices below the plane wait in the (free)
      // accumulator rows until their candidate slots are known
      if (body) {
        const int nvert = sph ? 1 : 8;
#pragma unroll 1
        for (int k = 0; k < nvert; ++k) {
          const f2 vh = vheight(k);
          if (below(vh)) {
            mask8 |= 1u << k;
            sm.acc[k][lane] = -(vh.h + vh.l);
          }
        }
      }
      const int cnt = __popc(mask8);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
      }
      int off = incl - cnt;
      const float up[3] = {0.f, 0.f, 1.f};
#pragma unroll 1
      for (unsigned mm = mask8; mm; mm &= mm - 1) {
        const int k = __ffs(mm) - 1;
        const float l0 = c0 + ((k & 1) ? h0 : -h0), l1 = c1 + ((k & 2) ? h1 : -h1), l2 = c2 + ((k & 4) ? h2 : -h2);
        float pr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) pr[a] = r[a] + (R[3 * a] * l0 + R[3 * a + 1] * l1 + R[3 * a + 2] * l2);
        pr[2] -= drop;
        if (off < kCand) put_candidate(cand, off, pr, up, sm.acc[k][lane], lane, 255);
        ++off;
      }
      ncand = shfi(incl, 31);
      if (ncand > kCand) st |= 8u;
      ncand = min(ncand, kCand);
    }
    __syncwarp();
    B3_PHASE(3);
    if (P.box_box) {
      // broad phase, lane = pair: the near pairs are compacted in pair order
      // into shared memory, so that the narrow phase below runs once per 32
      // near pairs rather than once per 32 candidate pairs
      int nnear = 0;
#pragma unroll 1
      for (int p0 = 0; p0 < npairs; p0 += 32) {
        const int pi = p0 + lane;
        bool near = false;
        unsigned pr = 0u;
        if (pi < npairs) {
          pr = pairs[pairoff + pi];
          const int a = (int)(pr >> 8), b = (int)(pr & 0xffu);
          const float dx = sm.c[0][b] - sm.c[0][a], dy = sm.c[1][b] - sm.c[1][a], dz = sm.c[2][b] - sm.c[2][a];
          const float rr = __ldg(F + F_RAD * 32 + a) + __ldg(F + F_RAD * 32 + b);
          near = dx * dx + dy * dy + dz * dz <= rr * rr;
        }
        const unsigned nm = __ballot_sync(kFull, near);
        if (near) sm.nearp[nnear + __popc(nm & ((1u << lane) - 1u))] = (uint16_t)pr;
        nnear += __popc(nm);
      }
      n_broad += (unsigned)npairs;
      n_narrow += (unsigned)nnear;
      __syncwarp();
      // narrow phase, lane = near pair; contacts placed in pair order by a warp scan
      float* stage = cand + kStageOffset + (size_t)lane * 8 * kCandW;
#pragma unroll 1
      for (int q0 = 0; q0 < nnear; q0 += 32) {
        const int qi = q0 + lane;
        int cnt = 0;
        if (qi < nnear) {
          const unsigned pr = sm.nearp[qi];
          cnt = body_pair_lane(sm.R, sm.c, F, (int)(pr >> 8), (int)(pr & 0xffu), stage);
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += t;
        }
        const int off = ncand + incl - cnt;
#pragma unroll 1
        for (int i = 0; i < cnt; ++i) {
          if (off + i < kCand) {
#pragma unroll
            for (int k = 0; k < kCandW; ++k) cand[(size_t)(off + i) * kCandW + k] = stage[i * kCandW + k];
          }
        }
        ncand += shfi(incl, 31);
        __syncwarp();
      }
      if (ncand > kCand) { st |= 8u; ncand = kCand; }
    }
    __syncwarp();
    B3_PHASE(4);
    // keep the cap deepest (ties by list order), list order kept: ranks of
    // every candidate first, then an in-order compaction (destination <= source)
    int nc = ncand;
    if (ncand > P.cap) {
      st |= 2u;
      keep_deepest(cand, ncand, P.cap, sm.keep, lane);
      nc = P.cap;
    }
    n_contacts += (unsigned)nc;
    nc_last = nc;
    __syncwarp();

    B3_PHASE(5);
    B3_LOCK();
    // ---------------- 7. contact rows: Y_r = L^-1 J_r^T and Gauss-Seidel constants (lane = row)
    float w_row = 0.f;  // with at most 32 rows: this lane's row residual J_r v_free - bias
#pragma unroll 1
    for (int r0 = 0; r0 < 3 * nc; r0 += 32) {
      const int row = r0 + lane;
      const bool act = row < 3 * nc;
      const int k = act ? row / 3 : 0;
      const int dir = row - 3 * k;
      float pr[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 1.f}, depth_k = 0.f;
      unsigned pa = 0u, pb = 0u;
      float sroot = 0.f;
      if (act) {
        const float4* rw = reinterpret_cast<const float4*>(cand + (size_t)k * kCandW);
        const float4 w0 = rw[0], w1 = rw[1];
        pr[0] = w0.x; pr[1] = w0.y; pr[2] = w0.z;
        const float nrm[3] = {w0.w, w1.x, w1.y};
        depth_k = w1.z;
        const int ab = __float_as_int(w1.w);
        const int a = ab & 0xff, b = (ab >> 8) & 0xff;
        pa = sm.path[a];
        pb = b == 255 ? 0u : sm.path[b];
        sroot = (b == 255) ? 1.f : 0.f;
        float t1[3], t2[3];
        if (b == 255) tangent_basis(nrm, t1, t2);
        else pair_tangent_basis(nrm, t1, t2);
#pragma unroll
        for (int q = 0; q < 3; ++q) d[q] = dir == 0 ? nrm[q] : (dir == 1 ? t1[q] : t2[q]);
      }
      float wa[3];
      cross3(pr, d, wa);
      // J_r into this lane's column of Yt ([dof][row]); compact loops keep the code small
      float* yr = &sm.Yt[0][lane];
      float jv = 0.f;
      // two dofs an iteration with their loads first; an odd last dof is
      // formed twice and counted once
      auto jcoef = [&](int j) {
        if (j < 6) return sroot;
        const int bj = j - 5;
        return (float)((int)((pa >> bj) & 1u) - (int)((pb >> bj) & 1u));
      };
#pragma unroll 1
      for (int j = 0; j < nv; j += 2) {
        const int j1 = j + 1 < nv ? j + 1 : j;
        float Sa[6], Sb[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) { Sa[q] = sm.S[q][j]; Sb[q] = sm.S[q][j1]; }
        const float va = sm.vfree[j], vb = sm.vfree[j1];
        const float Ja = jcoef(j) * (Sa[0] * wa[0] + Sa[1] * wa[1] + Sa[2] * wa[2] + Sa[3] * d[0] + Sa[4] * d[1] + Sa[5] * d[2]);
        const float Jb = jcoef(j1) * (Sb[0] * wa[0] + Sb[1] * wa[1] + Sb[2] * wa[2] + Sb[3] * d[0] + Sb[4] * d[1] + Sb[5] * d[2]);
        jv += Ja * va;
        if (j1 != j) jv += Jb * vb;
        yr[32 * j] = Ja;
        yr[32 * j1] = Jb;
      }
#pragma unroll 1
      for (int j = nv; j < 32; ++j) yr[32 * j] = 0.f;
      // forward substitution y <- L^-1 y, L broadcast from shared memory
      float aa = 0.f;
#pragma unroll 1
      for (int i = 0; i < nv; ++i) {
        const float* Li = sm.M + tri(i);
        float t0 = yr[32 * i], t1 = 0.f;
        int kk = 0;  // four terms an iteration, loads first; even terms to t0, odd to t1
#pragma unroll 1
        for (; kk + 3 < i; kk += 4) {
          const float a0 = Li[kk], b0 = yr[32 * kk], a1 = Li[kk + 1], b1 = yr[32 * (kk + 1)];
          const float a2 = Li[kk + 2], b2 = yr[32 * (kk + 2)], a3 = Li[kk + 3], b3 = yr[32 * (kk + 3)];
          t0 -= a0 * b0;
          t1 -= a1 * b1;
          t0 -= a2 * b2;
          t1 -= a3 * b3;
        }
        if (kk + 1 < i) {
          t0 -= Li[kk] * yr[32 * kk];
          t1 -= Li[kk + 1] * yr[32 * (kk + 1)];
          kk += 2;
        }
        if (kk < i) t0 -= Li[kk] * yr[32 * kk];
        const float yi = (t0 + t1) * sm.invd[i];
        yr[32 * i] = yi;
        aa += yi * yi;
      }
      if (act) {
        float4* dst = reinterpret_cast<float4*>(Yg + (size_t)row * 32);
#pragma unroll 2
        for (int i = 0; i < 8; ++i)
          dst[i] = make_float4(yr[32 * (4 * i)], yr[32 * (4 * i + 1)], yr[32 * (4 * i + 2)], yr[32 * (4 * i + 3)]);
        // softness kappa A (mass-normalised CFM), floored at min_cfm: a row the
        // dofs can barely move would otherwise take an impulse ~ 1/A
        const float Rr = fmaxf(P.kappa * aa, P.min_cfm);
        // a row that no dof can move (J = 0) carries no impulse: 1/(A+R) = 0
        const float inv = aa > kAmin ? 1.f / (aa + Rr) : 0.f;
        // penetration recovery speed, capped (ODE's maximum correcting velocity)
        const float bias = dir == 0 ? jv - fminf(P.erp * depth_k / dt, P.max_correct_vel) : jv;
        float* cs = cstg + (size_t)k * kCstG + 3 * dir;
        cs[0] = bias;
        cs[1] = inv;
        cs[2] = Rr;
        w_row = bias;
      }
      __syncwarp();
    }
    // tangent/normal coupling A_tn = Y_t . Y_n of each contact (lane =
    // contact), and for the dof-space sweep (more than 32 contacts) the block
    // B_k = Y_(k+1) Y_k^T to the next contact in sweep order; up to 10
    // contacts the sweep reads the couplings from the Delassus matrix it
    // builds
    const bool dofspace = nc > kLaneContacts;
#pragma unroll 1
    for (int k0 = 0; 3 * nc > 32 && k0 < nc; k0 += 32) {
      const int k = k0 + lane;
      if (k < nc) {
        const float4* yn = reinterpret_cast<const float4*>(Yg + (size_t)(3 * k) * 32);
        const float4* y1 = yn + 8;
        const float4* y2 = yn + 16;
        const int kn = (k + 1 < nc) ? k + 1 : 0;
        const float4* zn = reinterpret_cast<const float4*>(Yg + (size_t)(3 * kn) * 32);
        float a1 = 0.f, a2 = 0.f;
        float b[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) b[t] = 0.f;
#pragma unroll 1
        for (int i = 0; i < 8; ++i) {
          const float4 n4 = yn[i], p4 = y1[i], q4 = y2[i];
          a1 += p4.x * n4.x + p4.y * n4.y + p4.z * n4.z + p4.w * n4.w;
          a2 += q4.x * n4.x + q4.y * n4.y + q4.z * n4.z + q4.w * n4.w;
          if (dofspace) {
            const float4 ys[3] = {n4, p4, q4};
#pragma unroll
            for (int t = 0; t < 3; ++t) {
              const float4 z4 = zn[8 * t + i];
#pragma unroll
              for (int s2 = 0; s2 < 3; ++s2)
                b[3 * t + s2] += z4.x * ys[s2].x + z4.y * ys[s2].y + z4.z * ys[s2].z + z4.w * ys[s2].w;
            }
          }
        }
        float4* cs4 = reinterpret_cast<float4*>(cstg + (size_t)k * kCstG);
        float* cs = cstg + (size_t)k * kCstG;
        cs[9] = a1;
        cs[10] = a2;
        cs[11] = 0.f;
        if (dofspace) {
          cs4[3] = make_float4(b[0], b[1], b[2], b[3]);
          cs4[4] = make_float4(b[4], b[5], b[6], b[7]);
          cs4[5] = make_float4(b[8], 0.f, 0.f, 0.f);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) { lam_a[t] = 0.f; lam_b[t] = 0.f; }
    __syncwarp();

    B3_PHASE(6);
    B3_LOCK();
    // ---------------- 8. soft projected Gauss-Seidel
    float u = 0.f;
    if (nc > 0 && 3 * nc <= 32) {
      // Up to 10 contacts: sweep in contact space.  Lane r keeps row r of the
      // Delassus matrix A = J M^-1 J^T = Y Y^T (shared memory), its impulse
      // lam_r and its residual w_r = J_r v_free - bias_r + sum_s A_rs lam_s;
      // a contact update reads its three residuals with shuffles and adds
      // A_r. dlam to every row.  Same iteration as the dof-space sweep below.
      {
        // columns 0 .. 4 nq4 - 1 cover the 3 nc rows; the sweep reads no other
        const int nq4 = (3 * nc + 3) >> 2;
        float a[32];
#pragma unroll
        for (int c2 = 0; c2 < 32; ++c2) a[c2] = 0.f;
#pragma unroll 1
        for (int j = 0; j < nv; ++j) {
          const float own = sm.Yt[j][lane];
          const float4* Yj = reinterpret_cast<const float4*>(sm.Yt[j]);
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            if (q4 < nq4) {
              const float4 y4 = Yj[q4];
              a[4 * q4] += own * y4.x;
              a[4 * q4 + 1] += own * y4.y;
              a[4 * q4 + 2] += own * y4.z;
              a[4 * q4 + 3] += own * y4.w;
            }
          }
        }
        __syncwarp();
#pragma unroll
        for (int q4 = 0; q4 < 8; ++q4) {
          if (q4 < nq4) {
#pragma unroll
            for (int t = 0; t < 4; ++t) sm.Yt[4 * q4 + t][lane] = a[4 * q4 + t];  // [col][row], symmetric
          }
        }
        __syncwarp();
      }
      // Staging in the rotation rows of shared memory (free during the
      // sweep): the Gauss-Seidel constants of every contact and the
      // impulses of every contact, which all lanes compute alike and store
      // alike, so each lane later reads back its own write.  With
      // g = 1/(A+R), a = 1 - R g (= A g) and b = g A_tn, a row's projected
      // update l - g (w + R l + A_tn dn) is a l - g w - b dn: the terms
      // known before the normal update leave the dependency chain.  Per
      // contact (g_n, a_n, g_t1, a_t1), (b_t1, g_t2, a_t2, b_t2).
      float4* lamS = reinterpret_cast<float4*>(&sm.R[0][0]);
      float4* cS = lamS + 12;
      if (lane < nc) {
        const float4* c4 = reinterpret_cast<const float4*>(cstg) + 6 * lane;
        // (b_n, g_n, R_n, b_t1), (g_t1, R_t1, b_t2, g_t2), (R_t2, ., ., .)
        const float4 x0 = c4[0], x1 = c4[1], x2 = c4[2];
        // A_t1n, A_t2n: column 3k of rows 3k + 1, 3k + 2 of A ([column][row] above)
        const float at1n = sm.Yt[3 * lane][3 * lane + 1], at2n = sm.Yt[3 * lane][3 * lane + 2];
        cS[2 * lane] = make_float4(x0.y, fmaf(-x0.z, x0.y, 1.f), x1.x, fmaf(-x1.y, x1.x, 1.f));
        cS[2 * lane + 1] = make_float4(x1.x * at1n, x1.w, fmaf(-x2.x, x1.w, 1.f), x1.w * at2n);
        lamS[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncwarp();
      float w = w_row;
      // sweeps over contacts 0 .. nc - 1 in order; the impulses of the next
      // contact are read one update ahead (lamS[nc] is spare: at the last
      // contact of a sweep the read is discarded, and the next sweep starts
      // from contact 0's, written back by its update)
#pragma unroll 1
      for (int it = 0; it < P.iters; ++it) {
        const float4 l0 = lamS[0];
        float ln = l0.x, l1 = l0.y, l2 = l0.z;  // impulses of the contact being updated
        float mn, m1, m2;                        // and of the next one
        // update of contact k from its impulses (ln, l1, l2); the next
        // contact's impulses are read into (bn_, b1_, b2_)
        auto update = [&](int k, float ln, float l1, float l2, float& bn_, float& b1_, float& b2_) {
          const int r = 3 * k;
          // this contact's constants and this lane's row of A in its columns
          // (loaded first, used after the shuffles), the next one's impulses
          const float4 c0 = cS[2 * k], c1 = cS[2 * k + 1];
          const float an = sm.Yt[r][lane], a1 = sm.Yt[r + 1][lane], a2 = sm.Yt[r + 2][lane];
          const float4 nl = lamS[k + 1];
          const float wn = shf(w, r), w1 = shf(w, r + 1), w2 = shf(w, r + 2);
          const float lnn = fmaxf(0.f, fmaf(-c0.x, wn, c0.y * ln));
          const float dn = lnn - ln;
          const float wd = fmaf(an, dn, w);
          const float p1 = fmaf(-c0.z, w1, c0.w * l1), p2 = fmaf(-c1.y, w2, c1.z * l2);
          const float l1t = fmaf(-c1.x, dn, p1), l2t = fmaf(-c1.w, dn, p2);
          // disk cone |l_t| <= mu l_n: scale down when outside (rsqrt(0) =
          // inf gives a factor of 1, or 0 when l_n = 0)
          const float sc = fminf(1.f, (P.mu * lnn) * rsqrt_ftz(fmaf(l1t, l1t, l2t * l2t)));
          const float d1 = fmaf(l1t, sc, -l1), d2 = fmaf(l2t, sc, -l2);
          w = fmaf(a2, d2, fmaf(a1, d1, wd));
          lamS[k] = make_float4(lnn, l1t * sc, l2t * sc, 0.f);
          bn_ = nl.x;
          b1_ = nl.y;
          b2_ = nl.z;
        };
        // two contacts per pass, so that the impulse registers alternate by name
#pragma unroll 1
        for (int k = 0; k < nc; k += 2) {
          update(k, ln, l1, l2, mn, m1, m2);
          if (k + 1 >= nc) break;
          update(k + 1, mn, m1, m2, ln, l1, l2);
        }
      }
      __syncwarp();
      // u = sum_r Y_r lam_r (lane = dof)
#pragma unroll 1
      for (int kk = 0; kk < nc; ++kk) {
        const float4 l4 = lamS[kk];
        const float* Yk = Yg + (size_t)(3 * kk) * 32 + lane;
        u += l4.x * Yk[0] + l4.y * Yk[32] + l4.z * Yk[64];
      }
      if (lane < nc) {
        const float4 l4 = lamS[lane];
        lam_a[0] = l4.x; lam_a[1] = l4.y; lam_a[2] = l4.z;
      }
    } else if (nc > 0) {
      float4* lamS = reinterpret_cast<float4*>(&sm.R[0][0]);
      u = nc <= kLaneContacts ? lane_contact_sweep(lamS, cstg, Yg, cand + kAOffset, nc, nv, P.iters, P.mu, lane)
                              : dof_space_sweep(lamS, cstg, Yg, nc, P.iters, P.mu, lane);
      const float4 la = lane < nc ? lamS[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 lb = lane + 32 < nc ? lamS[lane + 32] : make_float4(0.f, 0.f, 0.f, 0.f);
      lam_a[0] = la.x; lam_a[1] = la.y; lam_a[2] = la.z;
      lam_b[0] = lb.x; lam_b[1] = lb.y; lam_b[2] = lb.z;
    }
    float vplus = vfree + upper_solve(sm, u, nv, lane);
    if (lane >= nv) vplus = 0.f;

    B3_PHASE(7);
    B3_LOCK();
    // ---------------- 9. semi-implicit Euler
    const float vx = shf(vplus, 0), vy = shf(vplus, 1), vz = shf(vplus, 2);
    const float ox = shf(vplus, 3), oy = shf(vplus, 4), oz = shf(vplus, 5);
    const float np0x = p0x + dt * vx, np0y = p0y + dt * vy, np0z = p0z + dt * vz;
    float dq0 = 1.f, dq1 = 0.f, dq2 = 0.f, dq3 = 0.f;
    {
      const float w2 = ox * ox + oy * oy + oz * oz;
      if (w2 >= 1e-24f) {  // |w| >= 1e-12, else the identity
        const float inw = rsqrt_ftz(w2);
        float sa, ca;
        sincosf(0.5f * dt * (w2 * inw), &sa, &ca);
        sa *= inw;
        dq0 = ca; dq1 = sa * ox; dq2 = sa * oy; dq3 = sa * oz;
      }
    }
    float r0 = qw * dq0 - qx * dq1 - qy * dq2 - qz * dq3;
    float r1 = qw * dq1 + qx * dq0 + qy * dq3 - qz * dq2;
    float r2 = qw * dq2 - qx * dq3 + qy * dq0 + qz * dq1;
    float r3 = qw * dq3 + qx * dq2 - qy * dq1 + qz * dq0;
    const float inr = rsqrt_ftz(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
    r0 *= inr; r1 *= inr; r2 *= inr; r3 *= inr;
    const float thp = shf(vplus, (5 + lane) & 31);
    const float ntheta = hinge ? theta + dt * thp : 0.f;
    bool bad = !(isfinite(np0x) && isfinite(np0y) && isfinite(np0z) && isfinite(r0) && isfinite(r1) &&
                 isfinite(r2) && isfinite(r3));
    bad = bad || !isfinite(ntheta) || !isfinite(vplus) || !isfinite(xn) || !isfinite(yn);
    if (__any_sync(kFull, bad)) {
      st |= 1u;
      if constexpr (!LOCK) break;
    }
    if (!(st & 5u)) {
      p0x = np0x; p0y = np0y; p0z = np0z;
      qw = r0; qx = r1; qy = r2; qz = r3;
      theta = ntheta;
      vd = vplus;
      xo = xn; yo = yn;
      ++n_steps;
    }
    B3_PHASE(8);
  }
#undef B3_PHASE
#undef B3_LOCK

  // ---- write back
  __syncwarp();
  if (lane == 0) {
    qv[0] = p0x; qv[1] = p0y; qv[2] = p0z;
    qv[3] = qw; qv[4] = qx; qv[5] = qy; qv[6] = qz;
    status[var] = st;
    last_nc[var] = nc_last;
    Counters c = counters[var];
    c.contacts += n_contacts;
    c.narrow += n_narrow;
    c.broad += n_broad;
    c.steps += n_steps;
    c.cycles += (unsigned long long)(clock64() - t_start);
    counters[var] = c;
  }
  if (hinge) {
    qv[6 + lane] = theta;
    sv[2 * (lane - 1)] = xo;
    sv[2 * (lane - 1) + 1] = yo;
  }
  if (lane < nv) vv[lane] = vd;
  // solver detail of the last step (inspection only)
  float* dbg = scratch + (size_t)var * kScratchFloats + kDbgOffset;
  dbg[lane] = vfree_last;
  if (lane == 31) dbg[31] = n_steps > 0 ? (float)(clock64() - t_start) / (float)n_steps : 0.f;
  if (lane < kPhases) dbg[32 + 4 * kCapMax + lane] = n_steps > 0 ? (float)sm.ph[lane] / (float)n_steps : 0.f;
  if (n_steps > 0) {
    if (lane < nc_last) {
      dbg[32 + 4 * lane] = lam_a[0];
      dbg[32 + 4 * lane + 1] = lam_a[1];
      dbg[32 + 4 * lane + 2] = lam_a[2];
    }
    if (lane + 32 < nc_last) {
      dbg[32 + 4 * (lane + 32)] = lam_b[0];
      dbg[32 + 4 * (lane + 32) + 1] = lam_b[1];
      dbg[32 + 4 * (lane + 32) + 2] = lam_b[2];
    }
  }
}

}  // namespace b3
