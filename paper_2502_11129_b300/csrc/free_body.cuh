// free_body.cuh -- one step of a robot that is a single free body (a box or a
// sphere whose centre is its frame origin), written for one thread (GPU) or
// one host loop iteration (CPU engine).  It is the general step of
// step_kernel.cuh with every tree pass reduced to its one-body closed form:
//   * the mass matrix in (linear velocity of the centre in world axes,
//     angular velocity in body axes) is diag(m, m, m, I_1, I_2, I_3) with the
//     principal moments I_k, so the Cholesky factor is its square root and
//     L^-1 J^T is J scaled per dof;
//   * the bias force is gravity on the linear part and the gyroscopic torque
//     w x (I w) on the angular part (Euler's equations);
//   * contacts are the body's ground points only (8 box vertices or the
//     sphere's lowest point), heights in FP64 as in the general step;
//   * rows, soft constants, the capped penetration recovery, the softness
//     floor and the Gauss-Seidel sweep (dof space, 6 dofs) follow the general
//     step's formulas and order;
//   * semi-implicit Euler as in the general step.
#pragma once
#include "step_common.cuh"

namespace b3 {

constexpr int kFreeMaxContacts = 8;

// what a free-body step reports besides the new state
struct FreeBodyOut {
  int nc;                          // contacts kept this step
  float vfree[6];                  // unconstrained velocity of this step
  float p[kFreeMaxContacts][3];    // kept contacts: points relative to the centre
  float depth[kFreeMaxContacts];   // and depths (normal +z)
  float lam[kFreeMaxContacts][3];  // impulses of the kept contacts
};

// F: the robot's packed model fields [field][32 body slots] (body 0 used);
// q (7), v (6) in place; st gets SIM_ST_* bits (1 non-finite, 2 overflow);
// returns false if the robot froze this step (state left unchanged).
__host__ __device__ inline bool free_body_step(const float* __restrict__ F, const StepParams& P, float* q, float* v,
                                               unsigned& st, FreeBodyOut& out) {
  const float dt = P.dt;
  auto fld = [&](int f) { return F[f * 32]; };
  // ---- pose
  float R[9];
  quat_to_R(q[3], q[4], q[5], q[6], R);
  const double dw = q[3], dx = q[4], dy = q[5], dz = q[6];
  const double hz0 = 2.0 * (dx * dz - dw * dy), hz1 = 2.0 * (dy * dz + dw * dx), hz2 = 1.0 - 2.0 * (dx * dx + dy * dy);
  // ---- dynamics: M = diag(m, m, m, I), c = (-m g, w x I w), v_free = v - dt M^-1 c
  const float m = fld(F_MASS);
  const float Id[3] = {fld(F_ID), fld(F_ID + 1), fld(F_ID + 2)};
  const float invd[6] = {1.f / sqrtf(m), 1.f / sqrtf(m), 1.f / sqrtf(m),
                         1.f / sqrtf(Id[0]), 1.f / sqrtf(Id[1]), 1.f / sqrtf(Id[2])};
  const float w[3] = {v[3], v[4], v[5]};
  const float Iw[3] = {Id[0] * w[0], Id[1] * w[1], Id[2] * w[2]};
  float gyro[3];
  cross3(w, Iw, gyro);
  float vf[6];
  vf[0] = v[0] + dt * P.gx;
  vf[1] = v[1] + dt * P.gy;
  vf[2] = v[2] + dt * P.gz;
  for (int k = 0; k < 3; ++k) vf[3 + k] = w[k] - dt * (gyro[k] / Id[k]);
  for (int k = 0; k < 6; ++k) out.vfree[k] = vf[k];
  // ---- ground contacts: a box's 8 vertices (bit i of k: + half size along
  // axis i) or a sphere's lowest point, in vertex order
  float cp[kFreeMaxContacts][3], cdep[kFreeMaxContacts];
  int ncand = 0;
  if (P.ground) {
    const bool sph = fld(F_GEOM) != 0.f;
    const float hr = fld(F_HALF);
    const float h0 = sph ? 0.f : hr, h1 = sph ? 0.f : fld(F_HALF + 1), h2 = sph ? 0.f : fld(F_HALF + 2);
    const float drop = sph ? hr : 0.f;
    const float c0 = fld(F_COM), c1 = fld(F_COM + 1), c2 = fld(F_COM + 2);
    const int nvert = sph ? 1 : 8;
    for (int k = 0; k < nvert; ++k) {
      const float l0 = c0 + ((k & 1) ? h0 : -h0), l1 = c1 + ((k & 2) ? h1 : -h1), l2 = c2 + ((k & 4) ? h2 : -h2);
      const double h = (double)q[2] + (0.0 + (hz0 * l0 + hz1 * l1 + hz2 * l2)) - (double)drop;
      if (!(h < 0.0)) continue;
      for (int a = 0; a < 3; ++a) cp[ncand][a] = R[3 * a] * l0 + R[3 * a + 1] * l1 + R[3 * a + 2] * l2;
      cp[ncand][2] -= drop;
      cdep[ncand] = (float)(-h);
      ++ncand;
    }
  }
  // keep the cap deepest (ties by list order), list order kept
  int nc = ncand;
  if (ncand > P.cap) {
    st |= 2u;
    bool keep[kFreeMaxContacts];
    for (int i = 0; i < ncand; ++i) {
      int rank = 0;
      for (int j = 0; j < ncand; ++j) rank += (cdep[j] > cdep[i] || (cdep[j] == cdep[i] && j < i)) ? 1 : 0;
      keep[i] = rank < P.cap;
    }
    int kept = 0;
    for (int i = 0; i < ncand; ++i)
      if (keep[i]) {
        for (int a = 0; a < 3; ++a) cp[kept][a] = cp[i][a];
        cdep[kept] = cdep[i];
        ++kept;
      }
    nc = P.cap;
  }
  out.nc = nc;
  for (int k = 0; k < nc; ++k) {
    for (int a = 0; a < 3; ++a) out.p[k][a] = cp[k][a];
    out.depth[k] = cdep[k];
  }
  // ---- contact rows: Y_r = L^-1 J_r^T (J scaled per dof) and the constants
  // b_n inv_n R_n | b_t1 inv_t1 R_t1 | b_t2 inv_t2 R_t2 | A_t1n A_t2n
  float Y[kFreeMaxContacts][3][6], cs[kFreeMaxContacts][11];
  const float up[3] = {0.f, 0.f, 1.f};
  float t1[3], t2[3];
  tangent_basis(up, t1, t2);
  for (int k = 0; k < nc; ++k) {
    for (int dir = 0; dir < 3; ++dir) {
      const float* d = dir == 0 ? up : (dir == 1 ? t1 : t2);
      float wa[3];
      cross3(cp[k], d, wa);
      float J[6];
      J[0] = d[0]; J[1] = d[1]; J[2] = d[2];
      for (int j = 0; j < 3; ++j) J[3 + j] = R[j] * wa[0] + R[3 + j] * wa[1] + R[6 + j] * wa[2];
      float jv = 0.f, aa = 0.f;
      for (int j = 0; j < 6; ++j) {
        jv += J[j] * vf[j];
        const float y = J[j] * invd[j];
        Y[k][dir][j] = y;
        aa += y * y;
      }
      const float Rr = fmaxf(P.kappa * aa, P.min_cfm);
      const float inv = aa > kAmin ? 1.f / (aa + Rr) : 0.f;
      const float bias = dir == 0 ? jv - fminf(P.erp * cdep[k] / dt, P.max_correct_vel) : jv;
      cs[k][3 * dir] = bias;
      cs[k][3 * dir + 1] = inv;
      cs[k][3 * dir + 2] = Rr;
    }
    float a1 = 0.f, a2 = 0.f;
    for (int j = 0; j < 6; ++j) {
      a1 += Y[k][1][j] * Y[k][0][j];
      a2 += Y[k][2][j] * Y[k][0][j];
    }
    cs[k][9] = a1;
    cs[k][10] = a2;
  }
  // ---- soft projected Gauss-Seidel in u = L^T (v - v_free)
  float u[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float lam[kFreeMaxContacts][3];
  for (int k = 0; k < nc; ++k) lam[k][0] = lam[k][1] = lam[k][2] = 0.f;
  for (int it = 0; it < P.iters && nc > 0; ++it) {
    for (int k = 0; k < nc; ++k) {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      for (int j = 0; j < 6; ++j) {
        s0 += Y[k][0][j] * u[j];
        s1 += Y[k][1][j] * u[j];
        s2 += Y[k][2][j] * u[j];
      }
      const float ln = lam[k][0], l1 = lam[k][1], l2 = lam[k][2];
      const float gn = s0 + cs[k][0] + cs[k][2] * ln;
      const float lnn = fmaxf(0.f, ln - gn * cs[k][1]);
      const float dn = lnn - ln;
      const float g1 = s1 + cs[k][9] * dn + cs[k][3] + cs[k][5] * l1;
      const float g2 = s2 + cs[k][10] * dn + cs[k][6] + cs[k][8] * l2;
      float l1t = l1 - g1 * cs[k][4];
      float l2t = l2 - g2 * cs[k][7];
      const float lim = P.mu * lnn;
      const float nt2 = l1t * l1t + l2t * l2t;
      if (nt2 > lim * lim) {
#ifdef __CUDA_ARCH__
        const float sc = lim * rsqrtf(nt2);
#else
        const float sc = lim / sqrtf(nt2);
#endif
        l1t *= sc;
        l2t *= sc;
      }
      const float d1 = l1t - l1, d2 = l2t - l2;
      for (int j = 0; j < 6; ++j) u[j] += Y[k][0][j] * dn + Y[k][1][j] * d1 + Y[k][2][j] * d2;
      lam[k][0] = lnn;
      lam[k][1] = l1t;
      lam[k][2] = l2t;
    }
  }
  for (int k = 0; k < nc; ++k)
    for (int t = 0; t < 3; ++t) out.lam[k][t] = lam[k][t];
  float vp[6];
  for (int j = 0; j < 6; ++j) vp[j] = vf[j] + u[j] * invd[j];
  // ---- semi-implicit Euler: position, quaternion exponential map
  const float np0[3] = {q[0] + dt * vp[0], q[1] + dt * vp[1], q[2] + dt * vp[2]};
  const float ox = vp[3], oy = vp[4], oz = vp[5];
  float dq0 = 1.f, dq1 = 0.f, dq2 = 0.f, dq3 = 0.f;
  {
    const float nw = sqrtf(ox * ox + oy * oy + oz * oz);
    if (nw >= 1e-12f) {
      float sa, ca;
#ifdef __CUDA_ARCH__
      sincosf(0.5f * dt * nw, &sa, &ca);
#else
      sa = sinf(0.5f * dt * nw);
      ca = cosf(0.5f * dt * nw);
#endif
      sa = sa / nw;
      dq0 = ca; dq1 = sa * ox; dq2 = sa * oy; dq3 = sa * oz;
    }
  }
  const float qw = q[3], qx = q[4], qy = q[5], qz = q[6];
  float r0 = qw * dq0 - qx * dq1 - qy * dq2 - qz * dq3;
  float r1 = qw * dq1 + qx * dq0 + qy * dq3 - qz * dq2;
  float r2 = qw * dq2 - qx * dq3 + qy * dq0 + qz * dq1;
  float r3 = qw * dq3 + qx * dq2 - qy * dq1 + qz * dq0;
  const float nr = sqrtf(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
  r0 /= nr; r1 /= nr; r2 /= nr; r3 /= nr;
  bool bad = !(isfinite(np0[0]) && isfinite(np0[1]) && isfinite(np0[2]) && isfinite(r0) && isfinite(r1) &&
               isfinite(r2) && isfinite(r3));
  for (int j = 0; j < 6; ++j) bad = bad || !isfinite(vp[j]);
  if (bad) {
    st |= 1u;
    return false;
  }
  q[0] = np0[0]; q[1] = np0[1]; q[2] = np0[2];
  q[3] = r0; q[4] = r1; q[5] = r2; q[6] = r3;
  for (int j = 0; j < 6; ++j) v[j] = vp[j];
  return true;
}

// a robot the free-body step serves: one body whose centre is its frame origin
inline bool free_body_eligible(int nb, const float* com3) {
  return nb == 1 && com3[0] == 0.f && com3[1] == 0.f && com3[2] == 0.f;
}

}  // namespace b3
