// step_common.cuh -- pieces of the population step shared by the GPU step
// kernel and the host (CPU) engine: model layout, step constants, spatial
// algebra, the box/box and sphere narrow phases, the FP64 sine / cosine and
// the contact tangent basis.  Everything here is __host__ __device__: the same source
// gives both engines the same geometry decisions.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

namespace b3 {

constexpr int kMaxB = 26;       // bodies per robot
constexpr int kMaxV = 31;       // dofs per robot
constexpr int kTri = 32 * 33 / 2;  // packed lower triangle of M / L (row i at i(i+1)/2)
constexpr int kCapMax = 64;     // contacts kept per step
constexpr int kCand = 256;      // contact candidates per step
constexpr int kCandW = 8;       // floats per candidate row
constexpr int kYRows = 3 * kCapMax;
constexpr float kAmin = 1e-10f;  // rows with J M^-1 J^T at or below this are frozen
constexpr float kClipOn = 1e-6f;  // a clipped polygon's vertex this close to a side plane is on it [m]
constexpr int kCstW = 12;        // Gauss-Seidel constants per contact (floats)
constexpr int kMaxPairs = kMaxB * (kMaxB - 1) / 2;  // box/box candidate pairs per robot

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
  F_RAD = 24,    // bounding-sphere radius (a sphere's own radius)
  F_GEOM = 25,   // 0 box, 1 sphere (radius F_HALF)
  NF = 26
};
// per-variant int model fields, [field][32 body slots]
enum : int { I_PARENT = 0, I_AXIS, I_PATH, I_CHILD, I_DEPTH, NI = 5 };
// chain layout (robots of more than kMaxB bodies, up to 64): the float fields
// above over 64 body slots, int fields [CNI][64] and 64-bit masks [CNM][64]
constexpr int kChainSlots = 64;
enum : int { CI_PARENT = 0, CI_AXIS, CI_DEPTH, CNI = 3 };
enum : int { CM_PATH = 0, CM_CHILD, CNM = 2 };

struct StepParams {
  float dt, gx, gy, gz;
  int iters;
  float mu, erp, kappa;
  int cap;
  float kp, kd, tau_max, theta_max, armature;
  int ground, box_box, actuate;
  float max_correct_vel;
  float min_cfm;
};

__host__ __device__ __forceinline__ int tri(int i) { return (i * (i + 1)) >> 1; }

// contact rows carry their two body indices packed in a float slot
__host__ __device__ __forceinline__ float int_bits_as_float(int x) {
#ifdef __CUDA_ARCH__
  return __int_as_float(x);
#else
  float f;
  memcpy(&f, &x, sizeof f);
  return f;
#endif
}
__host__ __device__ __forceinline__ int float_bits_as_int(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_int(f);
#else
  int x;
  memcpy(&x, &f, sizeof x);
  return x;
#endif
}

__host__ __device__ __forceinline__ float dot3(const float* a, const float* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__host__ __device__ __forceinline__ void cross3(const float* a, const float* b, float* o) {
  float t0 = a[1] * b[2] - a[2] * b[1];
  float t1 = a[2] * b[0] - a[0] * b[2];
  float t2 = a[0] * b[1] - a[1] * b[0];
  o[0] = t0; o[1] = t1; o[2] = t2;
}

// f = I (omega; v) for I stored as (m, h[3], Ixx, Iyy, Izz, Ixy, Ixz, Iyz)
__host__ __device__ __forceinline__ void inertia_apply(const float* I, const float* mv, float* f) {
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

__host__ __device__ __forceinline__ void crm(const float* v, const float* m, float* o) {
  float a[3], b[3], c[3];
  cross3(v, m, a);
  cross3(v, m + 3, b);
  cross3(v + 3, m, c);
  o[0] = a[0]; o[1] = a[1]; o[2] = a[2];
  o[3] = b[0] + c[0]; o[4] = b[1] + c[1]; o[5] = b[2] + c[2];
}

__host__ __device__ __forceinline__ void crf(const float* v, const float* f, float* o) {
  float a[3], b[3], c[3];
  cross3(v, f, a);
  cross3(v + 3, f + 3, b);
  cross3(v, f + 3, c);
  o[0] = a[0] + b[0]; o[1] = a[1] + b[1]; o[2] = a[2] + b[2];
  o[3] = c[0]; o[4] = c[1]; o[5] = c[2];
}

__host__ __device__ __forceinline__ void quat_to_R(float qw, float qx, float qy, float qz, float* R) {
  R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
  R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
  R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
}

// 1/sqrt(x) from the special-function unit with subnormals flushed to zero
// (PTX rsqrt.approx.ftz.f32, a few ulp): without the flush the compiler adds
// a subnormal fix-up, which lengthens the Gauss-Seidel update's dependency
// chain by ~15 cycles.  Used for the friction-disk scale min(1, mu l_n / |l_t|),
// the Cholesky pivots, the quaternion normalisation and the separating-axis
// directions, where flushing an argument below 1e-38 changes nothing
// measurable (all of them are far from it, or have a threshold above it).
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}


template <int NS = 32>
__host__ __device__ __forceinline__ void axis_of(const float (*R)[NS], int b, int k, float* o) {
  o[0] = R[k][b]; o[1] = R[3 + k][b]; o[2] = R[6 + k][b];
}

__host__ __device__ __forceinline__ void put_candidate(float* cand, int n, const float* p, const float* nrm,
                                              float depth, int a, int b) {
  float* row = cand + (size_t)n * kCandW;
  row[0] = p[0]; row[1] = p[1]; row[2] = p[2];
  row[3] = nrm[0]; row[4] = nrm[1]; row[5] = nrm[2];
  row[6] = depth;
  row[7] = int_bits_as_float((a & 0xff) | ((b & 0xff) << 8));
}

// Box/box narrow phase of one body pair a < b on one lane: separating-axis
// test over 15 axes (faces of a, faces of b, edge crosses), then face
// clipping (Sutherland-Hodgman, a vertex within kClipOn of a side plane
// counting as on it) or the edge-edge point.  Up to 8 contact rows go to `out`
// (8 floats each, candidate layout); returns their count.  Axis choice:
// minimum overlap, ties to the lowest index, a face unless the best edge
// overlap is below 0.95 x the best face overlap.  Normals point from b to a.
// NS: body slots per field of RR, CC and the model F (32, or 64 for chains).
template <int NS = 32>
__host__ __device__ __noinline__ int box_box_lane(const float (*RR)[NS], const float (*CC)[NS],
                                                  const float* __restrict__ F, int a, int b, float* out) {
  float Ax[3][3], Bx[3][3], hA[3], hB[3], D[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    axis_of<NS>(RR, a, k, Ax[k]);
    axis_of<NS>(RR, b, k, Bx[k]);
    hA[k] = F[(F_HALF + k) * NS + a];
    hB[k] = F[(F_HALF + k) * NS + b];
    D[k] = CC[k][b] - CC[k][a];
  }
  float fbest = 0.f, ebest = 0.f, min_ov = 0.f;
  int fi = -1, ei = -1;
  float Le[3] = {0.f, 0.f, 0.f};
  auto pick = [](const float (*X)[3], int k, float* o) {
#pragma unroll
    for (int t = 0; t < 3; ++t) o[t] = k == 0 ? X[0][t] : (k == 1 ? X[1][t] : X[2][t]);
  };
#pragma unroll 1
  for (int e = 0; e < 15; ++e) {
    float L[3];
    bool valid = true;
    if (e < 3) {
      pick(Ax, e, L);
    } else if (e < 6) {
      pick(Bx, e - 3, L);
    } else {
      float ai[3], bj[3];
      pick(Ax, (e - 6) / 3, ai);
      pick(Bx, (e - 6) % 3, bj);
      cross3(ai, bj, L);
#ifdef __CUDA_ARCH__
      // one SFU reciprocal square root instead of a rounded square root and
      // three divisions (nine edge axes per pair, on one lane's chain)
      const float l2 = dot3(L, L);
      if (l2 < 1e-12f) valid = false;
      else {
        const float il = rsqrt_ftz(l2);
        L[0] *= il; L[1] *= il; L[2] *= il;
      }
#else
      const float nl = sqrtf(dot3(L, L));
      if (nl < 1e-6f) valid = false;
      else { L[0] /= nl; L[1] /= nl; L[2] /= nl; }
#endif
    }
    if (valid) {
      float rA = 0.f, rB = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        rA += hA[k] * fabsf(dot3(Ax[k], L));
        rB += hB[k] * fabsf(dot3(Bx[k], L));
      }
      const float ov = rA + rB - fabsf(dot3(D, L));
      // a separating axis ends the test: the pair has no contact (the same
      // verdict as the minimum over all 15 axes being <= 0)
      if (!(ov > 0.f)) return 0;
      if (e == 0 || ov < min_ov) min_ov = ov;
      if (e < 6) {
        if (fi < 0 || ov < fbest) { fbest = ov; fi = e; }
      } else if (ei < 0 || ov < ebest) {
        ebest = ov; ei = e;
        Le[0] = L[0]; Le[1] = L[1]; Le[2] = L[2];
      }
    }
  }
  if (!(min_ov > 0.f)) return 0;
  const bool use_edge = ei >= 0 && ebest < 0.95f * fbest;
  const int ab = (a & 0xff) | ((b & 0xff) << 8);
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
      cR[k] = refA ? CC[k][a] : CC[k][b];
      cI[k] = refA ? CC[k][b] : CC[k][a];
    }
    const float toI[3] = {cI[0] - cR[0], cI[1] - cR[1], cI[2] - cR[2]};
    const float rax[3] = {Rx[ri][0], Rx[ri][1], Rx[ri][2]};
    const float sg = dot3(toI, rax) >= 0.f ? 1.f : -1.f;
    const float nref[3] = {sg * rax[0], sg * rax[1], sg * rax[2]};
    float dd[3];
    for (int k = 0; k < 3; ++k) dd[k] = dot3(Ix[k], nref);
    int ki = 0;
    for (int k = 1; k < 3; ++k) if (fabsf(dd[k]) > fabsf(dd[ki])) ki = k;
    const float si = dd[ki] > 0.f ? -1.f : 1.f;
    int k1 = (ki + 1) % 3, k2 = (ki + 2) % 3;
    if (k1 > k2) { const int t = k1; k1 = k2; k2 = t; }
    float fc[3];
    for (int k = 0; k < 3; ++k) fc[k] = cI[k] + si * hI[ki] * Ix[ki][k];
    const float s1[4] = {1.f, -1.f, -1.f, 1.f}, s2[4] = {1.f, 1.f, -1.f, -1.f};
    float poly[2][8][3];
    int np = 4, cur = 0;
#pragma unroll 1
    for (int v = 0; v < 4; ++v)
      for (int k = 0; k < 3; ++k)
        poly[0][v][k] = fc[k] + s1[v] * hI[k1] * Ix[k1][k] + s2[v] * hI[k2] * Ix[k2][k];
    int u1 = (ri + 1) % 3, u2 = (ri + 2) % 3;
    if (u1 > u2) { const int t = u1; u1 = u2; u2 = t; }
#pragma unroll 1
    for (int pl = 0; pl < 4 && np > 0; ++pl) {
      const int ax = pl < 2 ? u1 : u2;
      const float ps = (pl & 1) ? -1.f : 1.f;
      const float u[3] = {Rx[ax][0], Rx[ax][1], Rx[ax][2]};
      const float eh = hR[ax];
      // side of every vertex: inside (-1), on the plane (0: within
      // kClipOn of it) or outside (+1); inside and on vertices are kept, and
      // a crossing point only joins an inside vertex to an outside one, so
      // an edge lying on the plane is kept whole
      float dist[8];
      int side[8];
#pragma unroll 1
      for (int v = 0; v < np; ++v) {
        const float rel[3] = {poly[cur][v][0] - cR[0], poly[cur][v][1] - cR[1], poly[cur][v][2] - cR[2]};
        dist[v] = ps * dot3(rel, u) - eh;
        side[v] = fabsf(dist[v]) <= kClipOn ? 0 : (dist[v] < 0.f ? -1 : 1);
      }
      int no = 0;
#pragma unroll 1
      for (int v = 0; v < np; ++v) {
        const int nx = (v + 1) % np;
        const bool in_v = side[v] <= 0;
        // at most 8 vertices: a convex quad gains at most one per plane;
        // spurious crossings from rounding past 8 are dropped
        if (in_v && no < 8) {
          for (int k = 0; k < 3; ++k) poly[cur ^ 1][no][k] = poly[cur][v][k];
          ++no;
        }
        if (side[v] * side[nx] == -1 && no < 8) {
          const float t = dist[v] / (dist[v] - dist[nx]);
          for (int k = 0; k < 3; ++k) poly[cur ^ 1][no][k] = poly[cur][v][k] + t * (poly[cur][nx][k] - poly[cur][v][k]);
          ++no;
        }
      }
      np = no;
      cur ^= 1;
    }
    int n = 0;
#pragma unroll 1
    for (int v = 0; v < np; ++v) {
      const float rel[3] = {poly[cur][v][0] - cR[0], poly[cur][v][1] - cR[1], poly[cur][v][2] - cR[2]};
      const float depth = hR[ri] - dot3(rel, nref);
      if (depth > 0.f) {
        float* row = out + (size_t)n * kCandW;
        row[0] = poly[cur][v][0]; row[1] = poly[cur][v][1]; row[2] = poly[cur][v][2];
        row[3] = refA ? -nref[0] : nref[0];
        row[4] = refA ? -nref[1] : nref[1];
        row[5] = refA ? -nref[2] : nref[2];
        row[6] = depth;
        row[7] = int_bits_as_float(ab);
        ++n;
      }
    }
    return n;
  }
  const int i = (ei - 6) / 3, j = (ei - 6) % 3;
  float Lv[3] = {Le[0], Le[1], Le[2]};
  if (dot3(D, Lv) < 0.f) { Lv[0] = -Lv[0]; Lv[1] = -Lv[1]; Lv[2] = -Lv[2]; }
  float PA[3], PB[3];
  for (int k = 0; k < 3; ++k) { PA[k] = CC[k][a]; PB[k] = CC[k][b]; }
  for (int k = 0; k < 3; ++k) {
    if (k != i) {
      const float sA = dot3(Ax[k], Lv) >= 0.f ? hA[k] : -hA[k];
      for (int t = 0; t < 3; ++t) PA[t] += sA * Ax[k][t];
    }
    if (k != j) {
      const float sB = dot3(Bx[k], Lv) >= 0.f ? hB[k] : -hB[k];
      for (int t = 0; t < 3; ++t) PB[t] -= sB * Bx[k][t];
    }
  }
  const float wv[3] = {PA[0] - PB[0], PA[1] - PB[1], PA[2] - PB[2]};
  const float bb = dot3(Ax[i], Bx[j]);
  const float dd2 = dot3(Ax[i], wv);
  const float ee = dot3(Bx[j], wv);
  const float den = 1.f - bb * bb;
  float s = (bb * ee - dd2) / den;
  float t = (ee - bb * dd2) / den;
  s = fminf(fmaxf(s, -hA[i]), hA[i]);
  t = fminf(fmaxf(t, -hB[j]), hB[j]);
  for (int k = 0; k < 3; ++k) out[k] = 0.5f * ((PA[k] + s * Ax[i][k]) + (PB[k] + t * Bx[j][k]));
  out[3] = -Lv[0]; out[4] = -Lv[1]; out[5] = -Lv[2];
  out[6] = ebest;
  out[7] = int_bits_as_float(ab);
  return 1;
}

// Sphere/box or sphere/sphere contact of one body pair a < b (at least one a
// sphere) on one lane: one row at most, written to `out` (candidate layout);
// returns 0 or 1.  The point lies midway between the two surfaces' deepest
// points along the normal; normals point from b to a.  Sphere/sphere: normal
// along the centre difference, depth r_a + r_b - |d|.  Sphere/box: Q = the
// sphere centre C clamped to the box in box axes; C outside the box: normal
// along C - Q, depth r - |C - Q|; C inside: the nearest face's normal
// (smallest h_k - |C_k|, ties to the lowest k), depth r + h_k - |C_k|.
template <int NS = 32>
__host__ __device__ __noinline__ int sphere_pair_lane(const float (*RR)[NS], const float (*CC)[NS],
                                                      const float* __restrict__ F, int a, int b, float* out) {
  const bool sa = F[F_GEOM * NS + a] != 0.f, sb = F[F_GEOM * NS + b] != 0.f;
  float n[3], p[3], depth;
  if (sa && sb) {
    const float ra = F[F_HALF * NS + a], rb = F[F_HALF * NS + b];
    const float d[3] = {CC[0][a] - CC[0][b], CC[1][a] - CC[1][b], CC[2][a] - CC[2][b]};
    const float dist = sqrtf(dot3(d, d));
    depth = ra + rb - dist;
    if (!(depth > 0.f) || !(dist > 0.f)) return 0;
    for (int k = 0; k < 3; ++k) {
      n[k] = d[k] / dist;
      p[k] = 0.5f * ((CC[k][a] - ra * n[k]) + (CC[k][b] + rb * n[k]));
    }
  } else {
    const int is = sa ? a : b, ix = sa ? b : a;  // the sphere and the box
    const float r = F[F_HALF * NS + is];
    float h[3], D[3], l[3], q[3], e[3];
    for (int k = 0; k < 3; ++k) {
      h[k] = F[(F_HALF + k) * NS + ix];
      D[k] = CC[k][is] - CC[k][ix];
    }
    for (int k = 0; k < 3; ++k) {
      float ax[3];
      axis_of<NS>(RR, ix, k, ax);
      l[k] = dot3(ax, D);
      q[k] = fminf(fmaxf(l[k], -h[k]), h[k]);
      e[k] = l[k] - q[k];
    }
    const float e2 = dot3(e, e);
    float nl[3], pl[3];
    if (e2 > 0.f) {
      const float dist = sqrtf(e2);
      depth = r - dist;
      if (!(depth > 0.f)) return 0;
      for (int k = 0; k < 3; ++k) {
        nl[k] = e[k] / dist;
        pl[k] = q[k] - 0.5f * depth * nl[k];
      }
    } else {
      int kk = 0;
      float pen = h[0] - fabsf(l[0]);
      for (int k = 1; k < 3; ++k) {
        const float pk = h[k] - fabsf(l[k]);
        if (pk < pen) { pen = pk; kk = k; }
      }
      depth = r + pen;
      for (int k = 0; k < 3; ++k) nl[k] = k == kk ? (l[kk] >= 0.f ? 1.f : -1.f) : 0.f;
      for (int k = 0; k < 3; ++k) pl[k] = l[k] + 0.5f * (pen - r) * nl[k];
    }
    const float sg = is == a ? 1.f : -1.f;  // box-to-sphere, flipped when the sphere is b
    for (int k = 0; k < 3; ++k) {
      n[k] = sg * (RR[3 * k][ix] * nl[0] + RR[3 * k + 1][ix] * nl[1] + RR[3 * k + 2][ix] * nl[2]);
      p[k] = CC[k][ix] + (RR[3 * k][ix] * pl[0] + RR[3 * k + 1][ix] * pl[1] + RR[3 * k + 2][ix] * pl[2]);
    }
  }
  put_candidate(out, 0, p, n, depth, a, b);
  return 1;
}

// Narrow phase of one body pair a < b on one lane, by geometry: box/box, or
// sphere/box and sphere/sphere.  Rows to `out` (candidate layout); returns
// their count.
template <int NS = 32>
__host__ __device__ __noinline__ int body_pair_lane(const float (*RR)[NS], const float (*CC)[NS],
                                                    const float* __restrict__ F, int a, int b, float* out) {
  if (F[F_GEOM * NS + a] != 0.f || F[F_GEOM * NS + b] != 0.f) return sphere_pair_lane<NS>(RR, CC, F, a, b, out);
  return box_box_lane<NS>(RR, CC, F, a, b, out);
}

// Double-precision sine and cosine of one argument, compact enough to live in
// the step loop: Cody & Waite (1980) reduction x = k pi/2 + r with pi/2 split
// into a 33-bit head (k * head is exact for |k| < 2^20) and a double tail,
// then the Taylor series of sin and cos on |r| <= pi/4 through r^17 and r^18
// (truncation below 1e-19), and the quadrant swap.  Good to a few ulp for
// |x| < 1e6, far beyond any hinge angle.
__host__ __device__ __forceinline__ void sincos_f64(double x, double* s_out, double* c_out) {
  constexpr double kTwoOverPi = 0.63661977236758138;
  constexpr double kPio2Hi = 1.5707963267341256;     // pi/2 to 33 bits
  constexpr double kPio2Lo = 6.077100506506192e-11;  // pi/2 - kPio2Hi
  const double k = rint(x * kTwoOverPi);
  const double r = (x - k * kPio2Hi) - k * kPio2Lo;
  const double z = r * r;
  // 1/n! for the odd (sin) and even (cos) Taylor terms
  double ps = 1.0 / 355687428096000.0;                 // 1/17!
  ps = ps * z - 1.0 / 1307674368000.0;                 // 1/15!
  ps = ps * z + 1.0 / 6227020800.0;                    // 1/13!
  ps = ps * z - 1.0 / 39916800.0;                      // 1/11!
  ps = ps * z + 1.0 / 362880.0;                        // 1/9!
  ps = ps * z - 1.0 / 5040.0;                          // 1/7!
  ps = ps * z + 1.0 / 120.0;                           // 1/5!
  ps = ps * z - 1.0 / 6.0;                             // 1/3!
  const double sr = r + r * z * ps;
  double pc = -1.0 / 6402373705728000.0;               // 1/18!
  pc = pc * z + 1.0 / 20922789888000.0;                // 1/16!
  pc = pc * z - 1.0 / 87178291200.0;                   // 1/14!
  pc = pc * z + 1.0 / 479001600.0;                     // 1/12!
  pc = pc * z - 1.0 / 3628800.0;                       // 1/10!
  pc = pc * z + 1.0 / 40320.0;                         // 1/8!
  pc = pc * z - 1.0 / 720.0;                           // 1/6!
  pc = pc * z + 1.0 / 24.0;                            // 1/4!
  pc = pc * z - 0.5;                                   // 1/2!
  const double cr = 1.0 + z * pc;
  const int q = (int)((long long)k & 3);
  const double sa = (q & 1) ? cr : sr, ca = (q & 1) ? sr : cr;
  *s_out = (q & 2) ? -sa : sa;
  *c_out = ((q + 1) & 2) ? -ca : ca;
}

// Duff et al. 2017 ("Building an Orthonormal Basis, Revisited"), JCGT 6(1);
// ground contacts (n = +z) get x and y from it
__host__ __device__ __forceinline__ void tangent_basis(const float* n, float* t1, float* t2) {
  float s = n[2] >= 0.f ? 1.f : -1.f;
  float a = -1.f / (s + n[2]);
  float b = n[0] * n[1] * a;
  t1[0] = 1.f + s * n[0] * n[0] * a; t1[1] = s * b; t1[2] = -s * n[0];
  t2[0] = b; t2[1] = s + n[1] * n[1] * a; t2[2] = -n[1];
}

// Tangent directions of a body-pair contact: the same basis built in a fixed
// frame G (rows g1, g2, g3, g3 = (1, sqrt 2, sqrt 3) / sqrt 6) and turned back.
// No basis field on the sphere of normals is continuous everywhere; Duff's
// jumps where n_z changes sign, i.e. on horizontal normals, which bricks
// built on a lattice and lying side by side produce exactly, and the
// Gauss-Seidel result depends on the basis (each tangent row has its own
// step).  In G the jump lies on the normals orthogonal to g3, which no
// lattice direction is.
__host__ __device__ __forceinline__ void pair_tangent_basis(const float* n, float* t1, float* t2) {
  constexpr float kG[3][3] = {{-0.816496580927726f, 0.577350269189626f, 0.f},
                              {-0.408248290463863f, -0.577350269189626f, 0.707106781186548f},
                              {0.408248290463863f, 0.577350269189626f, 0.707106781186548f}};
  float m[3], u1[3], u2[3];
  for (int i = 0; i < 3; ++i) m[i] = kG[i][0] * n[0] + kG[i][1] * n[1] + kG[i][2] * n[2];
  tangent_basis(m, u1, u2);
  for (int k = 0; k < 3; ++k) {
    t1[k] = kG[0][k] * u1[0] + kG[1][k] * u1[1] + kG[2][k] * u1[2];
    t2[k] = kG[0][k] * u2[0] + kG[1][k] * u2[1] + kG[2][k] * u2[2];
  }
}

}  // namespace b3
