// chain_kernel.cuh -- block-per-robot step for robots larger than one warp.
//
// Robots of more than kMaxB bodies (up to 64 bodies, nv = nb + 5 <= 69: long
// chains such as a rope behind a core) take one block of kCT = 64 threads
// (two warps) each, persistent over the launch's steps like step_kernel.  The
// step is the one of step_kernel, in the same order, with the work split as
//   * thread = body    for the CPG, the tree passes (level by level, one block
//                      barrier per level), the inertias and the ground vertices;
//   * thread = field   for the leaf-to-root accumulations (serial over bodies);
//   * thread = row     for the Cholesky columns (rows t and t + 64);
//   * thread = pair    for the broad and narrow phases, thread = candidate for
//                      the contact cap, thread = contact row for Y_r = L^-1 J_r^T;
//   * warp 0 alone     for the triangular solves and the Gauss-Seidel sweep,
//                      lane l holding dofs l, l + 32 and l + 64: both are
//                      sequential in their pivots / contact updates, and a
//                      split over two warps would put a block barrier inside
//                      every contact update.
// Everything the step reads more than once lives in shared memory: the
// topology, the kinematics, the mass matrix and its factor, the candidates,
// the contact rows Y (3 x contact_cap rows, sized at launch) and the
// Gauss-Seidel constants.  The global scratch holds the narrow phase's staging
// rows, a copy of the last step's contacts and the inspection block.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "chain_layout.h"
#include "step_common.cuh"
#include "step_kernel.cuh"

namespace b3 {

static_assert(kCDbgPh == kCDbgLam + 4 * kCapMax, "inspection block sized for kCapMax contacts");

struct __align__(16) ChainSmem {
  float R[9][kCB];          // body rotations
  float r[3][kCB];          // frame origins relative to the core origin
  float c[3][kCB];          // box centres relative to the core origin
  float hzh[4][kCB], hzl[4][kCB];  // double-float third row of R (3) and origin height (1)
  float S[6][kCV];          // dof-indexed motion subspace columns
  float vb[6][kCB], ab[6][kCB];
  float acc[16][kCB + 1];   // per-body f (6) + composite inertia (10), padded
  float M[kCTri];           // mass matrix, then its Cholesky factor (packed lower)
  float invd[kCV], vfree[kCV], vel[kCV], tau[kCV], cvec[kCV], vplus[kCV];
  float xs[kCB];            // CPG x of every oscillator at the start of the step
  float cand[kCCand][kCandW];
  float cst[kCapMax][kCstW];  // b, 1/(A+R), R of the three rows; A_t1n, A_t2n
  float4 lam[kCapMax];
  unsigned long long path[kCB];
  uint16_t nearp[kCMaxPairs];
  int8_t parent[kCB];
  unsigned keep[kCCand / 32];
  int wtot[2];
  float piv;
  unsigned long long ph[kPhases];
};

// dynamic shared memory of a launch: the struct, then 3 cap rows of Y
__host__ __device__ constexpr size_t chain_smem_bytes(int cap) {
  return sizeof(ChainSmem) + (size_t)3 * cap * kYS * sizeof(float);
}

// exclusive prefix sum of one int per thread over the block; total to all
__device__ __forceinline__ int block_scan(int v, int& total, int* wtot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) wtot[w] = incl;
  __syncthreads();
  const int w0 = wtot[0];
  total = w0 + wtot[1];
  __syncthreads();  // wtot is reused by the next scan
  return (w == 1 ? w0 : 0) + incl - v;
}

// value of dof i (0 <= i < 96) held by lane i & 31 in slot i >> 5, to every lane
__device__ __forceinline__ float slot_shf(float x0, float x1, float x2, int i) {
  const int s = i >> 5;
  return shf(s == 0 ? x0 : (s == 1 ? x1 : x2), i & 31);
}

// x <- L^-1 x on warp 0, x_j in lane j & 31, slot j >> 5
__device__ __forceinline__ void lower_solve3(const ChainSmem& sm, float& x0, float& x1, float& x2, int nv,
                                             int lane) {
  float y0 = 0.f, y1 = 0.f, y2 = 0.f;
  for (int i = 0; i < nv; ++i) {
    const float yi = slot_shf(x0, x1, x2, i) * sm.invd[i];
    if (lane == (i & 31)) {
      const int s = i >> 5;
      if (s == 0) y0 = yi;
      else if (s == 1) y1 = yi;
      else y2 = yi;
    }
    const int r0 = lane, r1 = lane + 32, r2 = lane + 64;
    if (r0 > i && r0 < nv) x0 -= sm.M[tri(r0) + i] * yi;
    if (r1 > i && r1 < nv) x1 -= sm.M[tri(r1) + i] * yi;
    if (r2 > i && r2 < nv) x2 -= sm.M[tri(r2) + i] * yi;
  }
  x0 = y0; x1 = y1; x2 = y2;
}

// x <- L^-T x on warp 0, same layout
__device__ __forceinline__ void upper_solve3(const ChainSmem& sm, float& x0, float& x1, float& x2, int nv,
                                             int lane) {
  float y0 = 0.f, y1 = 0.f, y2 = 0.f;
  for (int i = nv - 1; i >= 0; --i) {
    const float xi = slot_shf(x0, x1, x2, i) * sm.invd[i];
    if (lane == (i & 31)) {
      const int s = i >> 5;
      if (s == 0) y0 = xi;
      else if (s == 1) y1 = xi;
      else y2 = xi;
    }
    const float* Li = sm.M + tri(i);
    const int r0 = lane, r1 = lane + 32, r2 = lane + 64;
    if (r0 < i) x0 -= Li[r0] * xi;
    if (r1 < i) x1 -= Li[r1] * xi;
    if (r2 < i) x2 -= Li[r2] * xi;
  }
  x0 = y0; x1 = y1; x2 = y2;
}

__global__ void __launch_bounds__(kCT)
chain_kernel(const float* __restrict__ mf, const int* __restrict__ mi, const unsigned long long* __restrict__ mk,
             const int4* __restrict__ meta, const uint16_t* __restrict__ pairs, float* __restrict__ qg,
             float* __restrict__ vg, float* __restrict__ sg, unsigned* __restrict__ status,
             Counters* __restrict__ counters, float* __restrict__ scratch, int* __restrict__ last_nc, int nvar,
             int nsteps, StepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ChainSmem& sm = *reinterpret_cast<ChainSmem*>(smem_raw);
  float* Ys = reinterpret_cast<float*>(smem_raw + sizeof(ChainSmem));  // [3 cap][kYS]
  const int var = blockIdx.x;
  if (var >= nvar) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

  const int4 md = meta[var];
  const int nb = md.x, maxdepth = md.y, npairs = md.z, pairoff = md.w;
  const int nv = nb + 5;
  const bool body = t < nb;
  const bool hinge = t >= 1 && t < nb;
  const float* __restrict__ F = mf + (size_t)var * NF * kCB;
  const int* IM = mi + (size_t)var * CNI * kCB;
  const unsigned long long* MK = mk + (size_t)var * CNM * kCB;
  const int parent = body ? IM[CI_PARENT * kCB + t] : -1;
  const int axis = IM[CI_AXIS * kCB + t];
  const int depth = body ? IM[CI_DEPTH * kCB + t] : 0;
  const unsigned long long childm = body ? MK[CM_CHILD * kCB + t] : 0ull;
  sm.parent[t] = (int8_t)parent;
  sm.path[t] = body ? MK[CM_PATH * kCB + t] : 0ull;
  auto fld = [&](int f) { return __ldg(F + f * kCB + t); };

  // ---- state: the root in every thread, hinge angle and oscillator per body
  // thread, velocities in shared memory (dof-indexed)
  float* qv = qg + (size_t)var * kCQS;
  float* vv = vg + (size_t)var * kCVS;
  float* sv = sg + (size_t)var * kCSS;
  float p0x = qv[0], p0y = qv[1], p0z = qv[2];
  float qw = qv[3], qx = qv[4], qy = qv[5], qz = qv[6];
  float theta = hinge ? qv[6 + t] : 0.f;
  float xo = hinge ? sv[2 * (t - 1)] : 0.f;
  float yo = hinge ? sv[2 * (t - 1) + 1] : 0.f;
  for (int j = t; j < kCV; j += kCT) sm.vel[j] = j < nv ? vv[j] : 0.f;
  unsigned st = status[var];
  unsigned n_contacts = 0, n_narrow = 0, n_broad = 0, n_steps = 0;
  int nc_last = last_nc[var];
  float* gs = scratch + (size_t)var * kChainScratchFloats;
  float* stage = gs + kCStageOffset + (size_t)t * 8 * kCandW;
  float* dbg = gs + kCDbgOffset;

  const long long t_start = clock64();
  // per-phase SM cycles (thread 0, after the barriers): 0 CPG+FK, 1
  // inertias+RNEA+CRBA, 2 Cholesky+v_free, 3 ground, 4 body pairs, 5 cap,
  // 6 contact rows, 7 Gauss-Seidel, 8 integration
  if (t < kPhases) sm.ph[t] = 0ull;
  long long tph = clock64();
#define C3_PHASE(i)                                                  \
  do {                                                               \
    const long long t_ = clock64();                                  \
    if (t == 0) sm.ph[i] += (unsigned long long)(t_ - tph);          \
    tph = t_;                                                        \
  } while (0)
  __syncthreads();

  for (int step = 0; step < nsteps; ++step) {
    if (st & 5u) break;  // frozen (st is the same in every thread)
    const float dt = P.dt;

    // ---------------- 1. CPG and PD torque (thread = body)
    float xn = xo, yn = yo;
    sm.xs[t] = xo;
    for (int j = t; j < kCV; j += kCT) sm.tau[j] = 0.f;
    __syncthreads();
    if (P.actuate && hinge) {
      const float wint = fld(F_WINT), wcpl = fld(F_WCPL);
      float dx = wint * yo, dy = -wint * xo;
      if (parent >= 1) dx -= wcpl * sm.xs[parent];
      for (unsigned long long m = childm; m; m &= m - 1) {
        const int c = __ffsll((long long)m) - 1;
        dx += __ldg(F + F_WCPL * kCB + c) * sm.xs[c];
      }
      xn = xo + dt * dx;
      yn = yo + dt * dy;
      const float x = fminf(fmaxf(xn, -1.f), 1.f);
      const float tq = P.kp * (P.theta_max * x - theta) - P.kd * sm.vel[5 + t];
      sm.tau[5 + t] = fminf(fmaxf(tq, -P.tau_max), P.tau_max);
    }

    // ---------------- 2. forward kinematics (thread = body, level by level)
    float R0[9];
    quat_to_R(qw, qx, qy, qz, R0);
    double sd, cd;
    sincos_f64((double)theta, &sd, &cd);
    const float sth = (float)sd, cth = (float)cd;
    float R[9], r[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k2 = 0; k2 < 9; ++k2) R[k2] = R0[k2];
    // ground-height chain in double-float, as in step_kernel: the root's
    // third row of R from the quaternion, the origin height relative to O
    f2 hz0, hz1, hz2, hzb = {0.f, 0.f};
    {
      hz0 = f2_add(f2_prod(qx, qz), f2_neg(f2_prod(qw, qy)));
      hz1 = f2_add(f2_prod(qy, qz), f2_prod(qw, qx));
      hz0 = {2.f * hz0.h, 2.f * hz0.l};
      hz1 = {2.f * hz1.h, 2.f * hz1.l};
      const f2 xy = f2_add(f2_prod(qx, qx), f2_prod(qy, qy));
      hz2 = f2_add(f2{1.f, 0.f}, f2{-2.f * xy.h, -2.f * xy.l});
    }
    if (t == 0) {
#pragma unroll
      for (int k2 = 0; k2 < 9; ++k2) sm.R[k2][0] = R0[k2];
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) sm.r[k2][0] = 0.f;
      sm.hzh[0][0] = hz0.h; sm.hzl[0][0] = hz0.l;
      sm.hzh[1][0] = hz1.h; sm.hzl[1][0] = hz1.l;
      sm.hzh[2][0] = hz2.h; sm.hzl[2][0] = hz2.l;
      sm.hzh[3][0] = 0.f; sm.hzl[3][0] = 0.f;
    }
    __syncthreads();
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
      float Fr[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) Fr[q] = fld(F_RFIX + q);
      const f2 cdf = {cth, (float)(cd - (double)cth)}, sdf = {sth, (float)(sd - (double)sth)};
      for (int lvl = 1; lvl <= maxdepth; ++lvl) {
        if (body && depth == lvl) {
          float Rp[9], rp[3];
#pragma unroll
          for (int k2 = 0; k2 < 9; ++k2) Rp[k2] = sm.R[k2][parent];
#pragma unroll
          for (int k2 = 0; k2 < 3; ++k2) rp[k2] = sm.r[k2][parent];
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
              R[3 * a + b] = Rp[3 * a] * Rl[b] + Rp[3 * a + 1] * Rl[3 + b] + Rp[3 * a + 2] * Rl[6 + b];
#pragma unroll
          for (int a = 0; a < 3; ++a) r[a] = rp[a] + (Rp[3 * a] * pf0 + Rp[3 * a + 1] * pf1 + Rp[3 * a + 2] * pf2);
          const f2 p0 = {sm.hzh[0][parent], sm.hzl[0][parent]}, p1 = {sm.hzh[1][parent], sm.hzl[1][parent]};
          const f2 p2 = {sm.hzh[2][parent], sm.hzl[2][parent]}, pb = {sm.hzh[3][parent], sm.hzl[3][parent]};
          f2 tt[3];
#pragma unroll
          for (int col = 0; col < 3; ++col)
            tt[col] = f2_add(f2_add(f2_mulf(p0, Fr[col]), f2_mulf(p1, Fr[3 + col])), f2_mulf(p2, Fr[6 + col]));
          const f2 ti = k == 0 ? tt[1] : (k == 1 ? tt[2] : tt[0]);
          const f2 tj = k == 0 ? tt[2] : (k == 1 ? tt[0] : tt[1]);
          const f2 tk = k == 0 ? tt[0] : (k == 1 ? tt[1] : tt[2]);
          const f2 oi = f2_add(f2_mul(cdf, ti), f2_mul(sdf, tj));
          const f2 oj = f2_add(f2_mul(cdf, tj), f2_neg(f2_mul(sdf, ti)));
          hz0 = k == 0 ? tk : (k == 1 ? oj : oi);
          hz1 = k == 0 ? oi : (k == 1 ? tk : oj);
          hz2 = k == 0 ? oj : (k == 1 ? oi : tk);
          hzb = f2_add(pb, f2_add(f2_add(f2_mulf(p0, pf0), f2_mulf(p1, pf1)), f2_mulf(p2, pf2)));
#pragma unroll
          for (int k2 = 0; k2 < 9; ++k2) sm.R[k2][t] = R[k2];
#pragma unroll
          for (int k2 = 0; k2 < 3; ++k2) sm.r[k2][t] = r[k2];
          sm.hzh[0][t] = hz0.h; sm.hzl[0][t] = hz0.l;
          sm.hzh[1][t] = hz1.h; sm.hzl[1][t] = hz1.l;
          sm.hzh[2][t] = hz2.h; sm.hzl[2][t] = hz2.l;
          sm.hzh[3][t] = hzb.h; sm.hzl[3][t] = hzb.l;
        }
        __syncthreads();
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
    for (int k = 0; k < 3; ++k) sm.c[k][t] = cb[k];
    if (hinge) {
#pragma unroll
      for (int k = 0; k < 6; ++k) sm.S[k][5 + t] = Sb[k];
    }
    if (t < 6) {
      float col[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (t < 3) col[3 + t] = 1.f;
      else { col[0] = R0[t - 3]; col[1] = R0[3 + t - 3]; col[2] = R0[6 + t - 3]; }
#pragma unroll
      for (int k = 0; k < 6; ++k) sm.S[k][t] = col[k];
    }
    C3_PHASE(0);

    // ---------------- 3. spatial inertias and RNEA bias forces (thread = body)
    float I[10];
    {
      const float mass = fld(F_MASS), i0 = fld(F_ID), i1 = fld(F_ID + 1), i2 = fld(F_ID + 2);
      float Iw[6];
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
    float vb[6], ab[6];
    {
      const float vlx = sm.vel[0], vly = sm.vel[1], vlz = sm.vel[2];
      const float wbx = sm.vel[3], wby = sm.vel[4], wbz = sm.vel[5];
      float om[3] = {R0[0] * wbx + R0[1] * wby + R0[2] * wbz, R0[3] * wbx + R0[4] * wby + R0[5] * wbz,
                     R0[6] * wbx + R0[7] * wby + R0[8] * wbz};
      float vl[3] = {vlx, vly, vlz};
      float vxw[3];
      cross3(vl, om, vxw);
      vb[0] = om[0]; vb[1] = om[1]; vb[2] = om[2]; vb[3] = vlx; vb[4] = vly; vb[5] = vlz;
      ab[0] = 0.f; ab[1] = 0.f; ab[2] = 0.f;
      ab[3] = vxw[0] - P.gx; ab[4] = vxw[1] - P.gy; ab[5] = vxw[2] - P.gz;
    }
    if (t == 0) {
#pragma unroll
      for (int k = 0; k < 6; ++k) { sm.vb[k][0] = vb[k]; sm.ab[k][0] = ab[k]; }
    }
    __syncthreads();
    {
      const float thd = sm.vel[(5 + t) % kCV];
      for (int lvl = 1; lvl <= maxdepth; ++lvl) {
        if (body && depth == lvl) {
          float Sq[6], cr[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) { Sq[k] = Sb[k] * thd; vb[k] = sm.vb[k][parent] + Sq[k]; }
          crm(vb, Sq, cr);
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            ab[k] = sm.ab[k][parent] + cr[k];
            sm.vb[k][t] = vb[k];
            sm.ab[k][t] = ab[k];
          }
        }
        __syncthreads();
      }
    }
    {
      float Ia[6], Iv[6], x[6];
      inertia_apply(I, ab, Ia);
      inertia_apply(I, vb, Iv);
      crf(vb, Iv, x);
#pragma unroll
      for (int k = 0; k < 6; ++k) sm.acc[k][t] = body ? Ia[k] + x[k] : 0.f;
#pragma unroll
      for (int k = 0; k < 10; ++k) sm.acc[6 + k][t] = body ? I[k] : 0.f;
    }
    __syncthreads();
    // leaf-to-root sums of forces and inertias, thread = component
    if (t < 16) {
      for (int b = nb - 1; b >= 1; --b) sm.acc[t][sm.parent[b]] += sm.acc[t][b];
    }
    __syncthreads();
    if (hinge)
      sm.cvec[5 + t] = Sb[0] * sm.acc[0][t] + Sb[1] * sm.acc[1][t] + Sb[2] * sm.acc[2][t] + Sb[3] * sm.acc[3][t] +
                       Sb[4] * sm.acc[4][t] + Sb[5] * sm.acc[5][t];
    if (t < 3) sm.cvec[t] = sm.acc[3 + t][0];
    else if (t < 6) {
      const int k = t - 3;
      sm.cvec[t] = R0[k] * sm.acc[0][0] + R0[3 + k] * sm.acc[1][0] + R0[6 + k] * sm.acc[2][0];
    }

    // ---------------- 4. CRBA mass matrix (packed lower triangle)
    for (int idx = t; idx < tri(nv); idx += kCT) sm.M[idx] = 0.f;
    __syncthreads();
    if (hinge) {
      float Ic[10], Fv[6];
#pragma unroll
      for (int k = 0; k < 10; ++k) Ic[k] = sm.acc[6 + k][t];
      inertia_apply(Ic, Sb, Fv);
      const int i = 5 + t;
      const int ti = tri(i);
      sm.M[ti + i] = Sb[0] * Fv[0] + Sb[1] * Fv[1] + Sb[2] * Fv[2] + Sb[3] * Fv[3] + Sb[4] * Fv[4] + Sb[5] * Fv[5] +
                     P.armature;
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
    if (t < 6) {
      float Ic[10], Sk[6], Fv[6];
#pragma unroll
      for (int k = 0; k < 10; ++k) Ic[k] = sm.acc[6 + k][0];
#pragma unroll
      for (int k = 0; k < 6; ++k) Sk[k] = sm.S[k][t];
      inertia_apply(Ic, Sk, Fv);
      for (int l = t; l < 6; ++l)
        sm.M[tri(l) + t] = sm.S[0][l] * Fv[0] + sm.S[1][l] * Fv[1] + sm.S[2][l] * Fv[2] + sm.S[3][l] * Fv[3] +
                           sm.S[4][l] * Fv[4] + sm.S[5][l] * Fv[5];
    }
    __syncthreads();
    C3_PHASE(1);

    // ---------------- 5. Cholesky (left-looking, thread = rows t and t + 64) and v_free
    bool chol_ok = true;
    for (int j = 0; j < nv; ++j) {
      const float* Lj = sm.M + tri(j);
      float mij[2] = {0.f, 0.f};
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int i = t + kCT * s;
        if (i >= j && i < nv) {
          const float* Li = sm.M + tri(i);
          float s0 = 0.f, s1 = 0.f;
          int k = 0;
#pragma unroll 1
          for (; k + 1 < j; k += 2) {
            s0 += Li[k] * Lj[k];
            s1 += Li[k + 1] * Lj[k + 1];
          }
          if (k < j) s0 += Li[k] * Lj[k];
          mij[s] = Li[j] - (s0 + s1);
          if (i == j) sm.piv = mij[s];
        }
      }
      __syncthreads();
      const float piv = sm.piv;
      if (!(piv > 0.f)) { chol_ok = false; break; }
      const float d = sqrtf(piv), inv = 1.f / d;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int i = t + kCT * s;
        if (i == j) { sm.M[tri(j) + j] = d; sm.invd[j] = inv; }
        else if (i > j && i < nv) sm.M[tri(i) + j] = mij[s] * inv;
      }
      __syncthreads();
    }
    if (!chol_ok) {
      st |= 4u;
      break;
    }
    if (warp == 0) {
      float x0 = 0.f, x1 = 0.f, x2 = 0.f;
      if (lane < nv) x0 = sm.tau[lane] - sm.cvec[lane];
      if (lane + 32 < nv) x1 = sm.tau[lane + 32] - sm.cvec[lane + 32];
      if (lane + 64 < nv) x2 = sm.tau[lane + 64] - sm.cvec[lane + 64];
      lower_solve3(sm, x0, x1, x2, nv, lane);
      upper_solve3(sm, x0, x1, x2, nv, lane);
      sm.vfree[lane] = lane < nv ? sm.vel[lane] + dt * x0 : 0.f;
      sm.vfree[lane + 32] = lane + 32 < nv ? sm.vel[lane + 32] + dt * x1 : 0.f;
      if (lane + 64 < kCV) sm.vfree[lane + 64] = lane + 64 < nv ? sm.vel[lane + 64] + dt * x2 : 0.f;
    }
    __syncthreads();
    C3_PHASE(2);

    // ---------------- 6. contact candidates (shared memory, list order)
    int ncand = 0;
    if (P.ground) {
      // a box's 8 vertices (bit i of k: + half size along axis i); a
      // sphere's lowest point; heights p0z + (hzb + hz . l) - drop in double-float
      unsigned mask8 = 0;
      const bool sph = fld(F_GEOM) != 0.f;
      const float hr = fld(F_HALF);
      const float h0 = sph ? 0.f : hr, h1 = sph ? 0.f : fld(F_HALF + 1), h2 = sph ? 0.f : fld(F_HALF + 2);
      const float drop = sph ? hr : 0.f;
      const float c0 = fld(F_COM), c1 = fld(F_COM + 1), c2 = fld(F_COM + 2);
      auto vheight = [&](int k) {
        const float l0 = c0 + ((k & 1) ? h0 : -h0), l1 = c1 + ((k & 2) ? h1 : -h1), l2 = c2 + ((k & 4) ? h2 : -h2);
        const f2 hl = f2_add(f2_add(f2_mulf(hz0, l0), f2_mulf(hz1, l1)), f2_mulf(hz2, l2));
        return f2_add(f2_add(two_sum(p0z, -drop), hzb), hl);
      };
      auto below = [](f2 h) { return h.h < 0.f || (h.h == 0.f && h.l < 0.f); };
      if (body) {
        const int nvert = sph ? 1 : 8;
#pragma unroll 1
        for (int k = 0; k < nvert; ++k)
          if (below(vheight(k))) mask8 |= 1u << k;
      }
      int total;
      int off = block_scan(__popc(mask8), total, sm.wtot);
      const float up[3] = {0.f, 0.f, 1.f};
      for (unsigned mm = mask8; mm; mm &= mm - 1) {
        const int k = __ffs(mm) - 1;
        const float l0 = c0 + ((k & 1) ? h0 : -h0), l1 = c1 + ((k & 2) ? h1 : -h1), l2 = c2 + ((k & 4) ? h2 : -h2);
        float pr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) pr[a] = r[a] + (R[3 * a] * l0 + R[3 * a + 1] * l1 + R[3 * a + 2] * l2);
        pr[2] -= drop;
        if (off < kCCand) {
          const f2 vh = vheight(k);
          put_candidate(&sm.cand[0][0], off, pr, up, -(vh.h + vh.l), t, 255);
        }
        ++off;
      }
      ncand = total;
      if (ncand > kCCand) st |= 8u;
      ncand = min(ncand, kCCand);
    }
    __syncthreads();
    C3_PHASE(3);
    if (P.box_box) {
      // broad phase, thread = pair; near pairs compacted in pair order
      int nnear = 0;
      for (int p0 = 0; p0 < npairs; p0 += kCT) {
        const int pi = p0 + t;
        bool near = false;
        unsigned pr = 0u;
        if (pi < npairs) {
          pr = pairs[pairoff + pi];
          const int a = (int)(pr >> 8), b = (int)(pr & 0xffu);
          const float dx = sm.c[0][b] - sm.c[0][a], dy = sm.c[1][b] - sm.c[1][a], dz = sm.c[2][b] - sm.c[2][a];
          const float rr = __ldg(F + F_RAD * kCB + a) + __ldg(F + F_RAD * kCB + b);
          near = dx * dx + dy * dy + dz * dz <= rr * rr;
        }
        int total;
        const int off = block_scan(near ? 1 : 0, total, sm.wtot);
        if (near) sm.nearp[nnear + off] = (uint16_t)pr;
        nnear += total;
      }
      n_broad += (unsigned)npairs;
      n_narrow += (unsigned)nnear;
      __syncthreads();
      // narrow phase, thread = near pair; rows placed in pair order
      for (int q0 = 0; q0 < nnear; q0 += kCT) {
        const int qi = q0 + t;
        int cnt = 0;
        if (qi < nnear) {
          const unsigned pr = sm.nearp[qi];
          cnt = body_pair_lane<kCB>(sm.R, sm.c, F, (int)(pr >> 8), (int)(pr & 0xffu), stage);
        }
        int total;
        const int off = ncand + block_scan(cnt, total, sm.wtot);
        for (int i = 0; i < cnt; ++i) {
          if (off + i < kCCand) {
#pragma unroll
            for (int k = 0; k < kCandW; ++k) sm.cand[off + i][k] = stage[i * kCandW + k];
          }
        }
        ncand += total;
      }
      if (ncand > kCCand) { st |= 8u; ncand = kCCand; }
    }
    __syncthreads();
    C3_PHASE(4);
    // keep the cap deepest (ties by list order), list order kept
    int nc = ncand;
    if (ncand > P.cap) {
      st |= 2u;
      for (int i0 = 0; i0 < ncand; i0 += kCT) {
        const int i = i0 + t;
        bool keep = false;
        if (i < ncand) {
          const float di = sm.cand[i][6];
          int rank = 0;
          for (int j = 0; j < ncand; ++j) {
            const float dj = sm.cand[j][6];
            rank += (dj > di || (dj == di && j < i)) ? 1 : 0;
          }
          keep = rank < P.cap;
        }
        const unsigned bal = __ballot_sync(kFull, keep);
        if (lane == 0) sm.keep[(i0 >> 5) + warp] = bal;
      }
      __syncthreads();
      int kept = 0;
      for (int i0 = 0; i0 < ncand; i0 += kCT) {
        const int i = i0 + t;
        const unsigned w0 = sm.keep[i0 >> 5], w1 = sm.keep[(i0 >> 5) + 1];
        const unsigned bits = warp == 0 ? w0 : w1;
        const bool keep = (bits >> lane) & 1u;
        const int dst = kept + (warp == 1 ? __popc(w0) : 0) + __popc(bits & ((1u << lane) - 1u));
        float row[kCandW];
        if (keep) {
#pragma unroll
          for (int k = 0; k < kCandW; ++k) row[k] = sm.cand[i][k];
        }
        __syncthreads();
        if (keep) {
#pragma unroll
          for (int k = 0; k < kCandW; ++k) sm.cand[dst][k] = row[k];
        }
        kept += __popc(w0) + __popc(w1);
        __syncthreads();
      }
      nc = P.cap;
    }
    n_contacts += (unsigned)nc;
    nc_last = nc;
    C3_PHASE(5);

    // ---------------- 7. contact rows (thread = row): Y_r = L^-1 J_r^T and the Gauss-Seidel constants
    for (int row = t; row < 3 * nc; row += kCT) {
      const int k = row / 3;
      const int dir = row - 3 * k;
      const float* cw = sm.cand[k];
      const float pr[3] = {cw[0], cw[1], cw[2]};
      const float nrm[3] = {cw[3], cw[4], cw[5]};
      const float depth_k = cw[6];
      const int ab2 = __float_as_int(cw[7]);
      const int a = ab2 & 0xff, b = (ab2 >> 8) & 0xff;
      const unsigned long long pa = sm.path[a], pb = b == 255 ? 0ull : sm.path[b];
      const float sroot = (b == 255) ? 1.f : 0.f;
      float t1[3], t2[3], d[3];
      if (b == 255) tangent_basis(nrm, t1, t2);
      else pair_tangent_basis(nrm, t1, t2);
#pragma unroll
      for (int q = 0; q < 3; ++q) d[q] = dir == 0 ? nrm[q] : (dir == 1 ? t1[q] : t2[q]);
      float wa[3];
      cross3(pr, d, wa);
      float* yr = Ys + (size_t)row * kYS;
      float jv = 0.f;
#pragma unroll 1
      for (int j = 0; j < nv; ++j) {
        float coef;
        if (j < 6) coef = sroot;
        else {
          const int bj = j - 5;
          coef = (float)((int)((pa >> bj) & 1ull) - (int)((pb >> bj) & 1ull));
        }
        const float Jj = coef * (sm.S[0][j] * wa[0] + sm.S[1][j] * wa[1] + sm.S[2][j] * wa[2] + sm.S[3][j] * d[0] +
                                 sm.S[4][j] * d[1] + sm.S[5][j] * d[2]);
        jv += Jj * sm.vfree[j];
        yr[j] = Jj;
      }
      float aa = 0.f;
#pragma unroll 1
      for (int i = 0; i < nv; ++i) {
        const float* Li = sm.M + tri(i);
        float t0 = yr[i], t1s = 0.f;
        int kk = 0;
#pragma unroll 1
        for (; kk + 1 < i; kk += 2) {
          t0 -= Li[kk] * yr[kk];
          t1s -= Li[kk + 1] * yr[kk + 1];
        }
        if (kk < i) t0 -= Li[kk] * yr[kk];
        const float yi = (t0 + t1s) * sm.invd[i];
        yr[i] = yi;
        aa += yi * yi;
      }
      // softness kappa A floored at min_cfm, frozen rows, capped recovery speed: as in step_kernel
      const float Rr = fmaxf(P.kappa * aa, P.min_cfm);
      const float inv = aa > kAmin ? 1.f / (aa + Rr) : 0.f;
      const float bias = dir == 0 ? jv - fminf(P.erp * depth_k / dt, P.max_correct_vel) : jv;
      sm.cst[k][3 * dir] = bias;
      sm.cst[k][3 * dir + 1] = inv;
      sm.cst[k][3 * dir + 2] = Rr;
    }
    __syncthreads();
    // tangent/normal couplings A_tn = Y_t . Y_n (thread = contact)
    for (int k = t; k < nc; k += kCT) {
      const float* yn = Ys + (size_t)(3 * k) * kYS;
      const float* y1 = yn + kYS;
      const float* y2 = y1 + kYS;
      float a1 = 0.f, a2 = 0.f;
#pragma unroll 1
      for (int j = 0; j < nv; ++j) {
        a1 += y1[j] * yn[j];
        a2 += y2[j] * yn[j];
      }
      sm.cst[k][9] = a1;
      sm.cst[k][10] = a2;
      sm.cst[k][11] = 0.f;
    }
    __syncthreads();
    C3_PHASE(6);

    // ---------------- 8. soft projected Gauss-Seidel in u = L^T (v - v_free) (warp 0)
    if (warp == 0) {
      float u0 = 0.f, u1 = 0.f, u2 = 0.f;  // dofs lane, lane + 32, lane + 64
      if (nc > 0) {
        for (int k0 = lane; k0 < nc; k0 += 32) sm.lam[k0] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        const bool j0 = lane < nv, j1 = lane + 32 < nv, j2 = lane + 64 < nv;
        const int nupd = P.iters * nc;
        int k = 0;
        for (int upd = 0; upd < nupd; ++upd) {
          const float* Y0 = Ys + (size_t)(3 * k) * kYS;
          const float* Y1 = Y0 + kYS;
          const float* Y2 = Y1 + kYS;
          const float a00 = j0 ? Y0[lane] : 0.f, a01 = j1 ? Y0[lane + 32] : 0.f, a02 = j2 ? Y0[lane + 64] : 0.f;
          const float a10 = j0 ? Y1[lane] : 0.f, a11 = j1 ? Y1[lane + 32] : 0.f, a12 = j2 ? Y1[lane + 64] : 0.f;
          const float a20 = j0 ? Y2[lane] : 0.f, a21 = j1 ? Y2[lane + 32] : 0.f, a22 = j2 ? Y2[lane + 64] : 0.f;
          const float* cs = sm.cst[k];
          const float4 l4 = sm.lam[k];
          float s0 = a00 * u0 + a01 * u1 + a02 * u2;
          float s1 = a10 * u0 + a11 * u1 + a12 * u2;
          float s2 = a20 * u0 + a21 * u1 + a22 * u2;
          warp_sum3(s0, s1, s2, lane);
          const float ln = l4.x, l1 = l4.y, l2 = l4.z;
          // constants: b_n inv_n R_n | b_t1 inv_t1 R_t1 | b_t2 inv_t2 R_t2 | A_t1n A_t2n
          const float gn = s0 + cs[0] + cs[2] * ln;
          const float lnn = fmaxf(0.f, ln - gn * cs[1]);
          const float dn = lnn - ln;
          const float g1 = s1 + cs[9] * dn + cs[3] + cs[5] * l1;
          const float g2 = s2 + cs[10] * dn + cs[6] + cs[8] * l2;
          float l1t = l1 - g1 * cs[4];
          float l2t = l2 - g2 * cs[7];
          const float lim = P.mu * lnn;
          const float nt2 = l1t * l1t + l2t * l2t;
          const float sc = fminf(1.f, lim * rsqrt_ftz(nt2));
          l1t *= sc;
          l2t *= sc;
          const float d1 = l1t - l1, d2 = l2t - l2;
          u0 += a00 * dn + a10 * d1 + a20 * d2;
          u1 += a01 * dn + a11 * d1 + a21 * d2;
          u2 += a02 * dn + a12 * d1 + a22 * d2;
          // every lane stores the same impulses and later reads back its own store
          sm.lam[k] = make_float4(lnn, l1t, l2t, 0.f);
          k = k + 1 < nc ? k + 1 : 0;
        }
        upper_solve3(sm, u0, u1, u2, nv, lane);
      }
      sm.vplus[lane] = lane < nv ? sm.vfree[lane] + u0 : 0.f;
      sm.vplus[lane + 32] = lane + 32 < nv ? sm.vfree[lane + 32] + u1 : 0.f;
      if (lane + 64 < kCV) sm.vplus[lane + 64] = lane + 64 < nv ? sm.vfree[lane + 64] + u2 : 0.f;
    }
    __syncthreads();
    C3_PHASE(7);

    // ---------------- 9. semi-implicit Euler (root in every thread, thread = body for the hinges)
    const float vx = sm.vplus[0], vy = sm.vplus[1], vz = sm.vplus[2];
    const float ox = sm.vplus[3], oy = sm.vplus[4], oz = sm.vplus[5];
    const float np0x = p0x + dt * vx, np0y = p0y + dt * vy, np0z = p0z + dt * vz;
    float dq0 = 1.f, dq1 = 0.f, dq2 = 0.f, dq3 = 0.f;
    {
      const float nw = sqrtf(ox * ox + oy * oy + oz * oz);
      if (nw >= 1e-12f) {
        float sa, ca;
        sincosf(0.5f * dt * nw, &sa, &ca);
        sa = sa / nw;
        dq0 = ca; dq1 = sa * ox; dq2 = sa * oy; dq3 = sa * oz;
      }
    }
    float r0 = qw * dq0 - qx * dq1 - qy * dq2 - qz * dq3;
    float r1 = qw * dq1 + qx * dq0 + qy * dq3 - qz * dq2;
    float r2 = qw * dq2 - qx * dq3 + qy * dq0 + qz * dq1;
    float r3 = qw * dq3 + qx * dq2 - qy * dq1 + qz * dq0;
    const float nr = sqrtf(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
    r0 /= nr; r1 /= nr; r2 /= nr; r3 /= nr;
    const float ntheta = hinge ? theta + dt * sm.vplus[5 + t] : 0.f;
    bool bad = !(isfinite(np0x) && isfinite(np0y) && isfinite(np0z) && isfinite(r0) && isfinite(r1) &&
                 isfinite(r2) && isfinite(r3));
    bad = bad || (hinge && (!isfinite(ntheta) || !isfinite(xn) || !isfinite(yn)));
    for (int j = t; j < nv; j += kCT) bad = bad || !isfinite(sm.vplus[j]);
    if (__syncthreads_or(bad)) {
      st |= 1u;
      break;
    }
    p0x = np0x; p0y = np0y; p0z = np0z;
    qw = r0; qx = r1; qy = r2; qz = r3;
    theta = ntheta;
    xo = xn; yo = yn;
    for (int j = t; j < kCV; j += kCT) sm.vel[j] = sm.vplus[j];
    ++n_steps;
    C3_PHASE(8);
  }
#undef C3_PHASE

  // ---- write back
  __syncthreads();
  if (t == 0) {
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
    dbg[kCDbgCycles] = n_steps > 0 ? (float)(clock64() - t_start) / (float)n_steps : 0.f;
  }
  if (hinge) {
    qv[6 + t] = theta;
    sv[2 * (t - 1)] = xo;
    sv[2 * (t - 1) + 1] = yo;
  }
  for (int j = t; j < nv; j += kCT) vv[j] = sm.vel[j];
  // the last step's solver detail and contacts (inspection only)
  if (n_steps > 0) {
    for (int j = t; j < kCV; j += kCT) dbg[j] = j < nv ? sm.vfree[j] : 0.f;
    if (t < kPhases) dbg[kCDbgPh + t] = (float)sm.ph[t] / (float)n_steps;
    for (int k = t; k < nc_last; k += kCT) {
      const float4 l4 = sm.lam[k];
      dbg[kCDbgLam + 4 * k] = l4.x;
      dbg[kCDbgLam + 4 * k + 1] = l4.y;
      dbg[kCDbgLam + 4 * k + 2] = l4.z;
      for (int q = 0; q < kCandW; ++q) gs[(size_t)k * kCandW + q] = sm.cand[k][q];
    }
  }
}

}  // namespace b3
