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
//   * lane = row     for the Cholesky trailing update;
//   * lane = dof     for the triangular solves and the Gauss-Seidel sweeps;
//   * lane = contact for building contact Jacobian rows;
//   * lane = axis    for the 15 separating-axis tests of a box/box pair.
//
// Gauss-Seidel runs in the Cholesky-transformed velocity u = L^T (v - v_free):
// with Y_r = L^-1 J_r^T, the row residual J_r v = J_r v_free + Y_r . u and the
// update v += M^-1 J_r^T dl is u += Y_r dl.  This is the same iteration as
// sweeping in v (identical in exact arithmetic), with one nv-vector per row
// instead of two.  After the sweeps v+ = v_free + L^-T u.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace b3 {

constexpr int kMaxB = 26;       // bodies per robot
constexpr int kMaxV = 31;       // dofs per robot
constexpr int kLs = 33;         // row stride of M / L in shared memory
constexpr int kCapMax = 64;     // contacts kept per step
constexpr int kCand = 256;      // contact candidates per step
constexpr int kCandW = 8;       // floats per candidate row
constexpr int kYRows = 3 * kCapMax;
constexpr unsigned kFull = 0xffffffffu;
constexpr float kAmin = 1e-10f;  // rows with J M^-1 J^T at or below this are frozen

// per-variant float model fields, [field][32 body slots]
enum : int {
  F_RFIX = 0,    // 9
  F_PFIX = 9,    // 3
  F_HALF = 12,   // 3
  F_COM = 15,    // 3
  F_MASS = 18,
  F_ID = 19,     // 3: principal inertia about the box centre
  F_WINT = 22,
  F_WCPL = 23,
  F_RAD = 24,    // bounding-sphere radius
  NF = 25
};
// per-variant int model fields, [field][32 body slots]
enum : int { I_PARENT = 0, I_AXIS, I_PATH, I_CHILD, I_DEPTH, NI = 5 };

struct StepParams {
  float dt, gx, gy, gz;
  int iters;
  float mu, erp, kappa;
  int cap;
  float kp, kd, tau_max, theta_max, armature;
  int ground, box_box, actuate;
  float max_correct_vel;
};

// global scratch per variant: candidate rows then Y rows (32 floats each)
constexpr size_t kScratchFloats = (size_t)kCand * kCandW + (size_t)kYRows * 32 + 32 + 4 * kCapMax;
constexpr size_t kDbgOffset = (size_t)kCand * kCandW + (size_t)kYRows * 32;  // last v_free, then lambda

struct WarpSmem {
  float R[9][32];
  float r[3][32];
  float c[3][32];
  float half[3][32];
  float rad[32];
  float S[6][32];          // dof-indexed motion subspace columns
  float acc[16][32];       // per-body f (6) + composite inertia (10)
  float M[32 * kLs];       // mass matrix, then its Cholesky factor (lower)
  float invd[32];
  float vfree[32];
  int parent[32];
  unsigned path[32];
  float poly[2][8][3];     // clipping buffers (lane 0)
  float cst[kCapMax][12];  // per-contact Gauss-Seidel constants
  float lam[kCapMax][4];
  unsigned keep[kCand / 32];
};

__device__ __forceinline__ float shf(float x, int src) { return __shfl_sync(kFull, x, src); }
__device__ __forceinline__ int shfi(int x, int src) { return __shfl_sync(kFull, x, src); }

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ float dot3(const float* a, const float* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void cross3(const float* a, const float* b, float* o) {
  float t0 = a[1] * b[2] - a[2] * b[1];
  float t1 = a[2] * b[0] - a[0] * b[2];
  float t2 = a[0] * b[1] - a[1] * b[0];
  o[0] = t0; o[1] = t1; o[2] = t2;
}

// f = I (omega; v) for I stored as (m, h[3], Ixx, Iyy, Izz, Ixy, Ixz, Iyz)
__device__ __forceinline__ void inertia_apply(const float* I, const float* mv, float* f) {
  const float* om = mv;
  const float* vo = mv + 3;
  float hv[3], hw[3];
  cross3(I + 1, vo, hv);
  cross3(I + 1, om, hw);
  f[0] = I[4] * om[0] + I[7] * om[1] + I[8] * om[2] + hv[0];
  f[1] = I[7] * om[0] + I[5] * om[1] + I[9] * om[2] + hv[1];
  f[2] = I[8] * om[0] + I[9] * om[1] + I[6] * om[2] + hv[2];
  f[3] = I[0] * vo[0] - hw[0];
  f[4] = I[0] * vo[1] - hw[1];
  f[5] = I[0] * vo[2] - hw[2];
}

__device__ __forceinline__ void crm(const float* v, const float* m, float* o) {
  float a[3], b[3], c[3];
  cross3(v, m, a);
  cross3(v, m + 3, b);
  cross3(v + 3, m, c);
  o[0] = a[0]; o[1] = a[1]; o[2] = a[2];
  o[3] = b[0] + c[0]; o[4] = b[1] + c[1]; o[5] = b[2] + c[2];
}

__device__ __forceinline__ void crf(const float* v, const float* f, float* o) {
  float a[3], b[3], c[3];
  cross3(v, f, a);
  cross3(v + 3, f + 3, b);
  cross3(v, f + 3, c);
  o[0] = a[0] + b[0]; o[1] = a[1] + b[1]; o[2] = a[2] + b[2];
  o[3] = c[0]; o[4] = c[1]; o[5] = c[2];
}

__device__ __forceinline__ void quat_to_R(float qw, float qx, float qy, float qz, float* R) {
  R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
  R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
  R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
}

// forward substitution of L y = b with lane = dof; returns y on each lane
__device__ __forceinline__ float lower_solve(const WarpSmem& sm, float b, int nv, int lane) {
  float acc = b, y = 0.f;
  for (int i = 0; i < nv; ++i) {
    float yi = shf(acc, i) * sm.invd[i];
    if (lane == i) y = yi;
    if (lane > i && lane < nv) acc -= sm.M[lane * kLs + i] * yi;
  }
  return y;
}

// back substitution of L^T x = y with lane = dof
__device__ __forceinline__ float upper_solve(const WarpSmem& sm, float y, int nv, int lane) {
  float acc = y, x = 0.f;
  for (int i = nv - 1; i >= 0; --i) {
    float xi = shf(acc, i) * sm.invd[i];
    if (lane == i) x = xi;
    if (lane < i) acc -= sm.M[i * kLs + lane] * xi;
  }
  return x;
}

__device__ __forceinline__ void axis_of(const WarpSmem& sm, int b, int k, float* o) {
  o[0] = sm.R[k][b]; o[1] = sm.R[3 + k][b]; o[2] = sm.R[6 + k][b];
}

__device__ __forceinline__ void put_candidate(float* cand, int n, const float* p, const float* nrm,
                                              float depth, int a, int b) {
  float* row = cand + (size_t)n * kCandW;
  row[0] = p[0]; row[1] = p[1]; row[2] = p[2];
  row[3] = nrm[0]; row[4] = nrm[1]; row[5] = nrm[2];
  row[6] = depth;
  row[7] = __int_as_float((a & 0xff) | ((b & 0xff) << 8));
}

// Box/box narrow phase of bodies a < b: separating-axis test over 15 axes
// (lane = axis), then face clipping or the edge-edge point on lane 0.
// Appends to the candidate list; returns the new count (warp-uniform).
__device__ int box_box_pair(WarpSmem& sm, float* cand, int n, int a, int b, int lane, unsigned& st) {
  float Ax[3][3], Bx[3][3], hA[3], hB[3], D[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    axis_of(sm, a, k, Ax[k]);
    axis_of(sm, b, k, Bx[k]);
    hA[k] = sm.half[k][a];
    hB[k] = sm.half[k][b];
    D[k] = sm.c[k][b] - sm.c[k][a];
  }
  float L[3] = {0.f, 0.f, 0.f};
  bool valid = lane < 15;
  if (lane < 3) {
    L[0] = Ax[lane][0]; L[1] = Ax[lane][1]; L[2] = Ax[lane][2];
  } else if (lane < 6) {
    L[0] = Bx[lane - 3][0]; L[1] = Bx[lane - 3][1]; L[2] = Bx[lane - 3][2];
  } else if (lane < 15) {
    int i = (lane - 6) / 3, j = (lane - 6) % 3;
    cross3(Ax[i], Bx[j], L);
    float nl = sqrtf(dot3(L, L));
    if (nl < 1e-6f) valid = false;
    else { L[0] /= nl; L[1] /= nl; L[2] /= nl; }
  }
  float ov = __int_as_float(0x7f800000);  // +inf
  if (valid) {
    float rA = 0.f, rB = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      rA += hA[k] * fabsf(dot3(Ax[k], L));
      rB += hB[k] * fabsf(dot3(Bx[k], L));
    }
    ov = rA + rB - fabsf(dot3(D, L));
  }
  float mn = ov;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(kFull, mn, o));
  if (!(mn > 0.f)) return n;
  // best face (lanes 0..5) and best edge (lanes 6..14), ties to the lowest index
  float fv = lane < 6 ? ov : __int_as_float(0x7f800000);
  int fi = lane;
  float ev = (lane >= 6 && lane < 15 && valid) ? ov : __int_as_float(0x7f800000);
  int ei = lane;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float fv2 = __shfl_xor_sync(kFull, fv, o);
    int fi2 = __shfl_xor_sync(kFull, fi, o);
    if (fv2 < fv || (fv2 == fv && fi2 < fi)) { fv = fv2; fi = fi2; }
    float ev2 = __shfl_xor_sync(kFull, ev, o);
    int ei2 = __shfl_xor_sync(kFull, ei, o);
    if (ev2 < ev || (ev2 == ev && ei2 < ei)) { ev = ev2; ei = ei2; }
  }
  const bool has_edge = ev < __int_as_float(0x7f800000);
  const bool use_edge = has_edge && ev < 0.95f * fv;
  float Le[3];
  {
    int src = use_edge ? ei : 0;
    Le[0] = shf(L[0], src); Le[1] = shf(L[1], src); Le[2] = shf(L[2], src);
  }
  int added = 0;
  if (lane == 0) {
    if (!use_edge) {
      const bool refA = fi < 3;
      const int ri = refA ? fi : fi - 3;
      float Rx[3][3], Ix[3][3], hR[3], hI[3], cR[3], cI[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          Rx[k][t] = refA ? Ax[k][t] : Bx[k][t];
          Ix[k][t] = refA ? Bx[k][t] : Ax[k][t];
        }
        hR[k] = refA ? hA[k] : hB[k];
        hI[k] = refA ? hB[k] : hA[k];
        cR[k] = refA ? sm.c[k][a] : sm.c[k][b];
        cI[k] = refA ? sm.c[k][b] : sm.c[k][a];
      }
      float toI[3] = {cI[0] - cR[0], cI[1] - cR[1], cI[2] - cR[2]};
      float rax[3] = {Rx[ri][0], Rx[ri][1], Rx[ri][2]};
      float sg = dot3(toI, rax) >= 0.f ? 1.f : -1.f;
      float nref[3] = {sg * rax[0], sg * rax[1], sg * rax[2]};
      float dd[3];
      for (int k = 0; k < 3; ++k) dd[k] = dot3(Ix[k], nref);
      int ki = 0;
      for (int k = 1; k < 3; ++k) if (fabsf(dd[k]) > fabsf(dd[ki])) ki = k;
      float si = dd[ki] > 0.f ? -1.f : 1.f;
      int k1 = (ki + 1) % 3, k2 = (ki + 2) % 3;
      if (k1 > k2) { int t = k1; k1 = k2; k2 = t; }
      float fc[3];
      for (int k = 0; k < 3; ++k) fc[k] = cI[k] + si * hI[ki] * Ix[ki][k];
      const float s1[4] = {1.f, -1.f, -1.f, 1.f}, s2[4] = {1.f, 1.f, -1.f, -1.f};
      int np = 4, cur = 0;
      for (int v = 0; v < 4; ++v)
        for (int k = 0; k < 3; ++k)
          sm.poly[0][v][k] = fc[k] + s1[v] * hI[k1] * Ix[k1][k] + s2[v] * hI[k2] * Ix[k2][k];
      int u1 = (ri + 1) % 3, u2 = (ri + 2) % 3;
      if (u1 > u2) { int t = u1; u1 = u2; u2 = t; }
      for (int pl = 0; pl < 4 && np > 0; ++pl) {
        const int ax = pl < 2 ? u1 : u2;
        const float ps = (pl & 1) ? -1.f : 1.f;
        float u[3] = {Rx[ax][0], Rx[ax][1], Rx[ax][2]};
        const float e = hR[ax];
        float dist[8];
        for (int v = 0; v < np; ++v) {
          float rel[3] = {sm.poly[cur][v][0] - cR[0], sm.poly[cur][v][1] - cR[1], sm.poly[cur][v][2] - cR[2]};
          dist[v] = ps * dot3(rel, u) - e;
        }
        int no = 0;
        for (int v = 0; v < np; ++v) {
          int nx = (v + 1) % np;
          bool in_v = dist[v] <= 0.f, in_n = dist[nx] <= 0.f;
          // at most 8 vertices: a convex quad gains at most one per plane;
          // spurious crossings from rounding past 8 are dropped
          if (in_v && no < 8) {
            for (int k = 0; k < 3; ++k) sm.poly[cur ^ 1][no][k] = sm.poly[cur][v][k];
            ++no;
          }
          if (in_v != in_n && no < 8) {
            float t = dist[v] / (dist[v] - dist[nx]);
            for (int k = 0; k < 3; ++k)
              sm.poly[cur ^ 1][no][k] = sm.poly[cur][v][k] + t * (sm.poly[cur][nx][k] - sm.poly[cur][v][k]);
            ++no;
          }
        }
        np = no;
        cur ^= 1;
      }
      float nrm[3];
      for (int k = 0; k < 3; ++k) nrm[k] = refA ? -nref[k] : nref[k];
      for (int v = 0; v < np; ++v) {
        float pt[3] = {sm.poly[cur][v][0], sm.poly[cur][v][1], sm.poly[cur][v][2]};
        float rel[3] = {pt[0] - cR[0], pt[1] - cR[1], pt[2] - cR[2]};
        float depth = hR[ri] - dot3(rel, nref);
        if (depth > 0.f) {
          if (n + added < kCand) put_candidate(cand, n + added, pt, nrm, depth, a, b);
          else st |= 8u;
          ++added;
        }
      }
    } else {
      const int i = (ei - 6) / 3, j = (ei - 6) % 3;
      float Lv[3] = {Le[0], Le[1], Le[2]};
      if (dot3(D, Lv) < 0.f) { Lv[0] = -Lv[0]; Lv[1] = -Lv[1]; Lv[2] = -Lv[2]; }
      float PA[3], PB[3];
      for (int k = 0; k < 3; ++k) { PA[k] = sm.c[k][a]; PB[k] = sm.c[k][b]; }
      for (int k = 0; k < 3; ++k) {
        if (k != i) {
          float s = dot3(Ax[k], Lv) >= 0.f ? hA[k] : -hA[k];
          for (int t = 0; t < 3; ++t) PA[t] += s * Ax[k][t];
        }
        if (k != j) {
          float s = dot3(Bx[k], Lv) >= 0.f ? hB[k] : -hB[k];
          for (int t = 0; t < 3; ++t) PB[t] -= s * Bx[k][t];
        }
      }
      float wv[3] = {PA[0] - PB[0], PA[1] - PB[1], PA[2] - PB[2]};
      float bb = dot3(Ax[i], Bx[j]);
      float dd = dot3(Ax[i], wv);
      float ee = dot3(Bx[j], wv);
      float den = 1.f - bb * bb;
      float s = (bb * ee - dd) / den;
      float t = (ee - bb * dd) / den;
      s = fminf(fmaxf(s, -hA[i]), hA[i]);
      t = fminf(fmaxf(t, -hB[j]), hB[j]);
      float pt[3], nrm[3] = {-Lv[0], -Lv[1], -Lv[2]};
      for (int k = 0; k < 3; ++k) pt[k] = 0.5f * ((PA[k] + s * Ax[i][k]) + (PB[k] + t * Bx[j][k]));
      if (n < kCand) put_candidate(cand, n, pt, nrm, ev, a, b);
      else st |= 8u;
      added = 1;
    }
  }
  st |= __shfl_sync(kFull, st, 0);
  added = __shfl_sync(kFull, added, 0);
  __syncwarp();
  return n + added;
}

// Duff et al. 2017 ("Building an Orthonormal Basis, Revisited"), JCGT 6(1)
__device__ __forceinline__ void tangent_basis(const float* n, float* t1, float* t2) {
  float s = n[2] >= 0.f ? 1.f : -1.f;
  float a = -1.f / (s + n[2]);
  float b = n[0] * n[1] * a;
  t1[0] = 1.f + s * n[0] * n[0] * a; t1[1] = s * b; t1[2] = -s * n[0];
  t2[0] = b; t2[1] = s + n[1] * n[1] * a; t2[2] = -n[1];
}

struct Counters {
  unsigned long long contacts, narrow, broad, steps;
};

template <int WPB>
__global__ void __launch_bounds__(WPB * 32)
step_kernel(const float* __restrict__ mf, const int* __restrict__ mi, const int4* __restrict__ meta,
            const uint16_t* __restrict__ pairs, float* __restrict__ qg, float* __restrict__ vg,
            float* __restrict__ sg, unsigned* __restrict__ status, Counters* __restrict__ counters,
            float* __restrict__ scratch, int* __restrict__ last_nc, int nvar, int nsteps, StepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int var = blockIdx.x * WPB + wib;
  if (var >= nvar) return;
  WarpSmem& sm = reinterpret_cast<WarpSmem*>(smem_raw)[wib];

  const int4 md = meta[var];
  const int nb = md.x, maxdepth = md.y, npairs = md.z, pairoff = md.w;
  const int nv = nb + 5;
  const bool body = lane < nb;
  const bool hinge = lane >= 1 && lane < nb;

  // ---- static model, lane = body
  const float* F = mf + (size_t)var * NF * 32;
  const int* IM = mi + (size_t)var * NI * 32;
  float Rf[9], pf[3], cm[3], mass, Id[3], wint, wcpl;
#pragma unroll
  for (int k = 0; k < 9; ++k) Rf[k] = F[(F_RFIX + k) * 32 + lane];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    pf[k] = F[(F_PFIX + k) * 32 + lane];
    cm[k] = F[(F_COM + k) * 32 + lane];
    Id[k] = F[(F_ID + k) * 32 + lane];
    sm.half[k][lane] = F[(F_HALF + k) * 32 + lane];
  }
  mass = F[F_MASS * 32 + lane];
  wint = F[F_WINT * 32 + lane];
  wcpl = F[F_WCPL * 32 + lane];
  sm.rad[lane] = F[F_RAD * 32 + lane];
  const int parent = body ? IM[I_PARENT * 32 + lane] : -1;
  const int axis = IM[I_AXIS * 32 + lane];
  const unsigned childm = (unsigned)IM[I_CHILD * 32 + lane];
  const int depth = body ? IM[I_DEPTH * 32 + lane] : 0;
  sm.parent[lane] = parent;
  sm.path[lane] = (unsigned)IM[I_PATH * 32 + lane];
  const int par0 = parent > 0 ? parent : 0;

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
  unsigned long long n_contacts = 0, n_narrow = 0, n_broad = 0, n_steps = 0;
  int nc_last = last_nc[var];
  float vfree_last = 0.f;

  float* cand = scratch + (size_t)var * kScratchFloats;
  float* Yg = cand + (size_t)kCand * kCandW;
  __syncwarp();

  for (int step = 0; step < nsteps; ++step) {
    if (st & 5u) break;  // frozen (non-finite state or failed factorisation)
    const float dt = P.dt;

    // ---------------- 1. CPG and PD torque (lane = body / hinge)
    float xn = xo, yn = yo, tau_b = 0.f;
    const float thd_b = shf(vd, (5 + lane) & 31);
    if (P.actuate) {
      sm.acc[0][lane] = (hinge && parent >= 1) ? wcpl * xo : 0.f;
      __syncwarp();
      float dx = wint * yo, dy = -wint * xo;
      const float xp = shf(xo, par0);
      if (hinge && parent >= 1) dx -= wcpl * xp;
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
    float Rl[9];
    {
      float sth, cth;
      sincosf(theta, &sth, &cth);
      const int k = axis, i = (axis + 1) % 3, j = (axis + 2) % 3;
#pragma unroll
      for (int row = 0; row < 3; ++row) {
        float fi = Rf[3 * row + i], fj = Rf[3 * row + j];
        Rl[3 * row + k] = Rf[3 * row + k];
        Rl[3 * row + i] = cth * fi + sth * fj;
        Rl[3 * row + j] = -sth * fi + cth * fj;
      }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = R0[k];
    for (int lvl = 1; lvl <= maxdepth; ++lvl) {
      float Rp[9], rp[3];
#pragma unroll
      for (int k = 0; k < 9; ++k) Rp[k] = shf(R[k], par0);
#pragma unroll
      for (int k = 0; k < 3; ++k) rp[k] = shf(r[k], par0);
      if (depth == lvl) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b)
            R[3 * a + b] = Rp[3 * a] * Rl[b] + Rp[3 * a + 1] * Rl[3 + b] + Rp[3 * a + 2] * Rl[6 + b];
#pragma unroll
        for (int a = 0; a < 3; ++a)
          r[a] = rp[a] + (Rp[3 * a] * pf[0] + Rp[3 * a + 1] * pf[1] + Rp[3 * a + 2] * pf[2]);
      }
    }
    // FP64 height chain for the ground contacts: the third row of R_b and the
    // frame-origin height relative to O.  A contact's push-out speed is
    // ERP * depth / dt with depths of ~0.1 mm, and FP32 kinematics carries
    // ~5 nm of rounding in heights, which would move a resting robot's
    // one-step velocity by ~1e-5; heights are therefore evaluated in FP64
    // (from the FP32 state), everything else stays FP32.
    double hz0, hz1, hz2, hzb = 0.0;
    {
      const double dw = qw, dx = qx, dy = qy, dz = qz;
      hz0 = 2.0 * (dx * dz - dw * dy);
      hz1 = 2.0 * (dy * dz + dw * dx);
      hz2 = 1.0 - 2.0 * (dx * dx + dy * dy);
      double sd, cd;
      sincos((double)theta, &sd, &cd);
      const int k = axis, i = (axis + 1) % 3, j = (axis + 2) % 3;
      double Ld[9];
#pragma unroll
      for (int row = 0; row < 3; ++row) {
        const double fi = Rf[3 * row + i], fj = Rf[3 * row + j];
        Ld[3 * row + k] = Rf[3 * row + k];
        Ld[3 * row + i] = cd * fi + sd * fj;
        Ld[3 * row + j] = -sd * fi + cd * fj;
      }
      for (int lvl = 1; lvl <= maxdepth; ++lvl) {
        const double p0 = __shfl_sync(kFull, hz0, par0), p1 = __shfl_sync(kFull, hz1, par0);
        const double p2 = __shfl_sync(kFull, hz2, par0), pb = __shfl_sync(kFull, hzb, par0);
        if (depth == lvl) {
          hz0 = p0 * Ld[0] + p1 * Ld[3] + p2 * Ld[6];
          hz1 = p0 * Ld[1] + p1 * Ld[4] + p2 * Ld[7];
          hz2 = p0 * Ld[2] + p1 * Ld[5] + p2 * Ld[8];
          hzb = pb + (p0 * (double)pf[0] + p1 * (double)pf[1] + p2 * (double)pf[2]);
        }
      }
    }
    float cb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) cb[a] = r[a] + (R[3 * a] * cm[0] + R[3 * a + 1] * cm[1] + R[3 * a + 2] * cm[2]);
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

    // ---------------- 3. spatial inertias and RNEA bias forces
    float I[10];
    {
      float Iw[6];  // xx yy zz xy xz yz of R diag(Id) R^T
      Iw[0] = R[0] * R[0] * Id[0] + R[1] * R[1] * Id[1] + R[2] * R[2] * Id[2];
      Iw[1] = R[3] * R[3] * Id[0] + R[4] * R[4] * Id[1] + R[5] * R[5] * Id[2];
      Iw[2] = R[6] * R[6] * Id[0] + R[7] * R[7] * Id[1] + R[8] * R[8] * Id[2];
      Iw[3] = R[0] * R[3] * Id[0] + R[1] * R[4] * Id[1] + R[2] * R[5] * Id[2];
      Iw[4] = R[0] * R[6] * Id[0] + R[1] * R[7] * Id[1] + R[2] * R[8] * Id[2];
      Iw[5] = R[3] * R[6] * Id[0] + R[4] * R[7] * Id[1] + R[5] * R[8] * Id[2];
      float cc = cb[0] * cb[0] + cb[1] * cb[1] + cb[2] * cb[2];
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
    {
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

    // ---------------- 4. CRBA mass matrix (lower triangle, row stride kLs)
    for (int j = 0; j <= lane && lane < nv; ++j) sm.M[lane * kLs + j] = 0.f;
    __syncwarp();
    if (hinge) {
      float Ic[10], Fv[6];
#pragma unroll
      for (int k = 0; k < 10; ++k) Ic[k] = sm.acc[6 + k][lane];
      inertia_apply(Ic, Sb, Fv);
      const int i = 5 + lane;
      sm.M[i * kLs + i] = Sb[0] * Fv[0] + Sb[1] * Fv[1] + Sb[2] * Fv[2] + Sb[3] * Fv[3] + Sb[4] * Fv[4] +
                          Sb[5] * Fv[5] + P.armature;
      for (int j = parent; j > 0; j = sm.parent[j]) {
        const int jj = 5 + j;
        sm.M[i * kLs + jj] = sm.S[0][jj] * Fv[0] + sm.S[1][jj] * Fv[1] + sm.S[2][jj] * Fv[2] +
                             sm.S[3][jj] * Fv[3] + sm.S[4][jj] * Fv[4] + sm.S[5][jj] * Fv[5];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) sm.M[i * kLs + k] = Fv[3 + k];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        sm.M[i * kLs + 3 + k] = R0[k] * Fv[0] + R0[3 + k] * Fv[1] + R0[6 + k] * Fv[2];
    }
    if (lane < 6) {
      float Ic[10], Sk[6], Fv[6];
#pragma unroll
      for (int k = 0; k < 10; ++k) Ic[k] = sm.acc[6 + k][0];
#pragma unroll
      for (int k = 0; k < 6; ++k) Sk[k] = sm.S[k][lane];
      inertia_apply(Ic, Sk, Fv);
      for (int l = lane; l < 6; ++l)
        sm.M[l * kLs + lane] = sm.S[0][l] * Fv[0] + sm.S[1][l] * Fv[1] + sm.S[2][l] * Fv[2] +
                               sm.S[3][l] * Fv[3] + sm.S[4][l] * Fv[4] + sm.S[5][l] * Fv[5];
    }
    __syncwarp();

    // ---------------- 5. Cholesky (right-looking, lane = row) and v_free
    bool chol_ok = true;
    for (int k = 0; k < nv; ++k) {
      const float dkk = sm.M[k * kLs + k];
      if (!(dkk > 0.f)) { chol_ok = false; break; }
      const float d = sqrtf(dkk);
      const float inv = 1.f / d;
      float lik = 0.f;
      if (lane > k && lane < nv) lik = sm.M[lane * kLs + k] * inv;
      __syncwarp();
      if (lane == k) { sm.M[k * kLs + k] = d; sm.invd[k] = inv; }
      if (lane > k && lane < nv) sm.M[lane * kLs + k] = lik;
      __syncwarp();
      for (int j = k + 1; j < nv; ++j) {
        const float ljk = sm.M[j * kLs + k];
        if (lane >= j && lane < nv) sm.M[lane * kLs + j] -= lik * ljk;
      }
      __syncwarp();
    }
    if (!chol_ok) { st |= 4u; break; }
    float vfree;
    {
      float y = lower_solve(sm, tau_d - c_d, nv, lane);
      float acc = upper_solve(sm, y, nv, lane);
      vfree = vd + dt * acc;
      sm.vfree[lane] = lane < nv ? vfree : 0.f;
      vfree_last = sm.vfree[lane];
    }

    // ---------------- 6. contact candidates
    const float Oz = p0z;
    int ncand = 0;
    if (P.ground) {
      unsigned mask8 = 0;
      float lv[8][3];
      float zdepth[8];
      if (body) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
          for (int i = 0; i < 3; ++i)
            lv[k][i] = cm[i] + (((k >> i) & 1) ? 1.f : -1.f) * sm.half[i][lane];
          const double z = (double)Oz + (hzb + (hz0 * (double)lv[k][0] + hz1 * (double)lv[k][1] +
                                                 hz2 * (double)lv[k][2]));
          if (z < 0.0) mask8 |= 1u << k;
          zdepth[k] = (float)(-z);
        }
      }
      int cnt = __popc(mask8);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
      }
      int off = incl - cnt;
      const float up[3] = {0.f, 0.f, 1.f};
      for (unsigned m = mask8; m; m &= m - 1) {
        const int k = __ffs(m) - 1;
        float pr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
          pr[a] = r[a] + (R[3 * a] * lv[k][0] + R[3 * a + 1] * lv[k][1] + R[3 * a + 2] * lv[k][2]);
        if (off < kCand) put_candidate(cand, off, pr, up, zdepth[k], lane, 255);
        ++off;
      }
      ncand = shfi(incl, 31);
      if (ncand > kCand) { st |= 8u; }
      ncand = min(ncand, kCand);
    }
    __syncwarp();
    if (P.box_box) {
      for (int p0 = 0; p0 < npairs; p0 += 32) {
        const int pi = p0 + lane;
        int a = 0, b = 0;
        bool near = false;
        if (pi < npairs) {
          const unsigned pr = pairs[pairoff + pi];
          a = (int)(pr >> 8);
          b = (int)(pr & 0xffu);
          const float dx = sm.c[0][b] - sm.c[0][a], dy = sm.c[1][b] - sm.c[1][a], dz = sm.c[2][b] - sm.c[2][a];
          const float rr = sm.rad[a] + sm.rad[b];
          near = dx * dx + dy * dy + dz * dz <= rr * rr;
        }
        n_broad += (unsigned)max(0, min(32, npairs - p0));
        unsigned cm_ = __ballot_sync(kFull, near);
        while (cm_) {
          const int src = __ffs(cm_) - 1;
          cm_ &= cm_ - 1;
          const int aa = shfi(a, src), bb = shfi(b, src);
          ++n_narrow;
          ncand = box_box_pair(sm, cand, ncand, aa, bb, lane, st);
        }
      }
      if (ncand > kCand) { st |= 8u; ncand = kCand; }
    }
    __syncwarp();
    // keep the cap deepest (ties by list order), list order kept: ranks of
    // every candidate first, then an in-order compaction (destination <= source)
    int nc = ncand;
    if (ncand > P.cap) {
      st |= 2u;
      for (int i0 = 0; i0 < ncand; i0 += 32) {
        const int i = i0 + lane;
        bool keep = false;
        if (i < ncand) {
          const float di = cand[(size_t)i * kCandW + 6];
          int rank = 0;
          for (int j = 0; j < ncand; ++j) {
            const float dj = cand[(size_t)j * kCandW + 6];
            rank += (dj > di || (dj == di && j < i)) ? 1 : 0;
          }
          keep = rank < P.cap;
        }
        const unsigned bal = __ballot_sync(kFull, keep);
        if (lane == 0) sm.keep[i0 >> 5] = bal;
      }
      __syncwarp();
      int kept = 0;
      for (int i0 = 0; i0 < ncand; i0 += 32) {
        const int i = i0 + lane;
        const unsigned bal = sm.keep[i0 >> 5];
        const bool keep = (bal >> lane) & 1u;
        float row[kCandW];
        if (keep) {
#pragma unroll
          for (int k = 0; k < kCandW; ++k) row[k] = cand[(size_t)i * kCandW + k];
        }
        __syncwarp();
        if (keep) {
          const int dst = kept + __popc(bal & ((1u << lane) - 1u));
#pragma unroll
          for (int k = 0; k < kCandW; ++k) cand[(size_t)dst * kCandW + k] = row[k];
        }
        kept += __popc(bal);
        __syncwarp();
      }
      nc = P.cap;
    }
    n_contacts += (unsigned)nc;
    nc_last = nc;
    __syncwarp();

    // ---------------- 7. contact rows: Y = L^-1 J^T and Gauss-Seidel constants (lane = contact)
    for (int k0 = 0; k0 < nc; k0 += 32) {
      const int k = k0 + lane;
      const bool act = k < nc;
      float pr[3] = {0.f, 0.f, 0.f}, nrm[3] = {0.f, 0.f, 1.f}, depth_k = 0.f;
      unsigned pa = 0u, pb = 0u;
      float sroot = 0.f;
      if (act) {
        const float* row = cand + (size_t)k * kCandW;
        pr[0] = row[0]; pr[1] = row[1]; pr[2] = row[2];
        nrm[0] = row[3]; nrm[1] = row[4]; nrm[2] = row[5];
        depth_k = row[6];
        const int ab = __float_as_int(row[7]);
        const int a = ab & 0xff, b = (ab >> 8) & 0xff;
        pa = sm.path[a];
        pb = b == 255 ? 0u : sm.path[b];
        sroot = (b == 255) ? 1.f : 0.f;
      }
      float t1[3], t2[3];
      tangent_basis(nrm, t1, t2);
      float yn[32];
      float cst[12];
#pragma unroll 1
      for (int dir = 0; dir < 3; ++dir) {
        float d[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) d[q] = dir == 0 ? nrm[q] : (dir == 1 ? t1[q] : t2[q]);
        float wa[3];
        cross3(pr, d, wa);
        float y[32];
        float jv = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float Jj = 0.f;
          if (j < nv) {
            float coef;
            if (j < 6) coef = sroot;
            else {
              const int bj = j - 5;
              coef = (float)((int)((pa >> bj) & 1u) - (int)((pb >> bj) & 1u));
            }
            Jj = coef * (sm.S[0][j] * wa[0] + sm.S[1][j] * wa[1] + sm.S[2][j] * wa[2] + sm.S[3][j] * d[0] +
                         sm.S[4][j] * d[1] + sm.S[5][j] * d[2]);
            jv += Jj * sm.vfree[j];
          }
          y[j] = Jj;
        }
        // forward substitution y <- L^-1 y, L broadcast from shared memory
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          if (i < nv) {
            float t = y[i];
#pragma unroll
            for (int kk = 0; kk < i; ++kk) t -= sm.M[i * kLs + kk] * y[kk];
            y[i] = t * sm.invd[i];
          }
        }
        float aa = 0.f, an = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          if (i < nv) {
            aa += y[i] * y[i];
            if (dir > 0) an += y[i] * yn[i];
          }
        }
        if (act) {
          float4* dst = reinterpret_cast<float4*>(Yg + (size_t)(3 * k + dir) * 32);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            dst[i] = make_float4(i * 4 + 0 < nv ? y[i * 4 + 0] : 0.f, i * 4 + 1 < nv ? y[i * 4 + 1] : 0.f,
                                 i * 4 + 2 < nv ? y[i * 4 + 2] : 0.f, i * 4 + 3 < nv ? y[i * 4 + 3] : 0.f);
        }
        const float Rr = P.kappa * aa;
        // a row that no dof can move (J = 0) carries no impulse: 1/(A+R) = 0
        const float inv = aa > kAmin ? 1.f / (aa + Rr) : 0.f;
        if (dir == 0) {
#pragma unroll
          for (int i = 0; i < 32; ++i) yn[i] = y[i];
          // penetration recovery speed, capped (ODE's maximum correcting velocity)
          cst[0] = jv - fminf(P.erp * depth_k / dt, P.max_correct_vel);
          cst[1] = inv;
          cst[2] = Rr;
        } else {
          cst[3 * dir + 0] = jv;
          cst[3 * dir + 1] = inv;
          cst[3 * dir + 2] = Rr;
          cst[8 + dir] = an;
        }
      }
      if (act) {
#pragma unroll
        for (int i = 0; i < 11; ++i) sm.cst[k][i] = cst[i];
        sm.lam[k][0] = 0.f; sm.lam[k][1] = 0.f; sm.lam[k][2] = 0.f;
      }
    }
    __syncwarp();

    // ---------------- 8. soft projected Gauss-Seidel (lane = dof, u = L^T (v - v_free))
    float u = 0.f;
    for (int it = 0; it < P.iters; ++it) {
      for (int k = 0; k < nc; ++k) {
        const float* Yk = Yg + (size_t)(3 * k) * 32;
        const float y0 = Yk[lane], y1 = Yk[32 + lane], y2 = Yk[64 + lane];
        float s0 = y0 * u, s1 = y1 * u, s2 = y2 * u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          s0 += __shfl_xor_sync(kFull, s0, o);
          s1 += __shfl_xor_sync(kFull, s1, o);
          s2 += __shfl_xor_sync(kFull, s2, o);
        }
        const float* cs = sm.cst[k];
        const float ln = sm.lam[k][0], l1 = sm.lam[k][1], l2 = sm.lam[k][2];
        const float gn = s0 + cs[0] + cs[2] * ln;
        const float lnn = fmaxf(0.f, ln - gn * cs[1]);
        const float dn = lnn - ln;
        const float g1 = s1 + cs[9] * dn + cs[3] + cs[5] * l1;
        const float g2 = s2 + cs[10] * dn + cs[6] + cs[8] * l2;
        float l1t = l1 - g1 * cs[4];
        float l2t = l2 - g2 * cs[7];
        const float lim = P.mu * lnn;
        const float nt2 = l1t * l1t + l2t * l2t;
        if (nt2 > lim * lim) {
          const float sc = lim / sqrtf(nt2);
          l1t *= sc;
          l2t *= sc;
        }
        u += y0 * dn + y1 * (l1t - l1) + y2 * (l2t - l2);
        __syncwarp();
        if (lane == 0) { sm.lam[k][0] = lnn; sm.lam[k][1] = l1t; sm.lam[k][2] = l2t; }
        __syncwarp();
      }
    }
    float vplus = vfree + upper_solve(sm, u, nv, lane);
    if (lane >= nv) vplus = 0.f;

    // ---------------- 9. semi-implicit Euler
    const float vx = shf(vplus, 0), vy = shf(vplus, 1), vz = shf(vplus, 2);
    const float ox = shf(vplus, 3), oy = shf(vplus, 4), oz = shf(vplus, 5);
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
    const float thp = shf(vplus, (5 + lane) & 31);
    const float ntheta = hinge ? theta + dt * thp : 0.f;
    bool bad = !(isfinite(np0x) && isfinite(np0y) && isfinite(np0z) && isfinite(r0) && isfinite(r1) &&
                 isfinite(r2) && isfinite(r3));
    bad = bad || !isfinite(ntheta) || !isfinite(vplus) || !isfinite(xn) || !isfinite(yn);
    if (__any_sync(kFull, bad)) { st |= 1u; break; }
    p0x = np0x; p0y = np0y; p0z = np0z;
    qw = r0; qx = r1; qy = r2; qz = r3;
    theta = ntheta;
    vd = vplus;
    xo = xn; yo = yn;
    ++n_steps;
  }

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
  for (int k = lane; k < nc_last && n_steps > 0; k += 32) {
    dbg[32 + 4 * k] = sm.lam[k][0];
    dbg[32 + 4 * k + 1] = sm.lam[k][1];
    dbg[32 + 4 * k + 2] = sm.lam[k][2];
  }
}

}  // namespace b3
