// b3cpu.cu -- host (CPU) engine of the population simulator: the step of
// step_kernel.cuh written as scalar loops over bodies, dofs and contacts for
// one robot at a time, FP32 with FP64 contact heights, on a pool of worker
// threads.  Host code only (nvcc compiles it so that it can include the
// __host__ __device__ helpers it shares with the GPU kernel).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "b3cpu.h"
#include "model_pack.h"
#include "step_common.cuh"
#include "free_body.cuh"

using namespace b3;

namespace {

struct Robot {
  const float* F;       // [NF][32]
  const int* I;         // [NI][32]
  int nb, maxdepth, npairs, pairoff;
};

// per-thread work space of one robot step
struct Work {
  float R[9][32], r[3][32], c[3][32], S[6][32];
  double hz[3][32], hzb[32];
  float acc[16][32];
  float M[kTri], invd[32], vfree[32];
  float cand[kCand][kCandW];
  float Y[kYRows][32];
  float cst[kCapMax][kCstW];
};

// one step of one robot; returns false if the robot froze (status set)
bool step_robot(const Robot& m, const uint16_t* pairs, const StepParams& P, float* q, float* v, float* s,
                unsigned& st, unsigned long long& contacts, Work& w) {
  const int nb = m.nb, nv = nb + 5;
  const float* F = m.F;
  auto fld = [&](int f, int b) { return F[f * 32 + b]; };
  const int* parent = m.I + I_PARENT * 32;
  const int* axis = m.I + I_AXIS * 32;
  const unsigned* path = reinterpret_cast<const unsigned*>(m.I + I_PATH * 32);
  const unsigned* child = reinterpret_cast<const unsigned*>(m.I + I_CHILD * 32);
  const float dt = P.dt;

  // ---- 1. CPG and PD torques (explicit Euler from the old oscillator state)
  float xn[32], yn[32], tau[32];
  for (int j = 0; j < 32; ++j) tau[j] = 0.f;
  for (int b = 1; b < nb; ++b) {
    xn[b] = s[2 * (b - 1)];
    yn[b] = s[2 * (b - 1) + 1];
  }
  if (P.actuate) {
    for (int b = 1; b < nb; ++b) {
      const float xo = s[2 * (b - 1)], yo = s[2 * (b - 1) + 1];
      const float wint = fld(F_WINT, b), wcpl = fld(F_WCPL, b);
      float dx = wint * yo, dy = -wint * xo;
      if (parent[b] >= 1) dx -= wcpl * s[2 * (parent[b] - 1)];
      for (unsigned mm = child[b]; mm; mm &= mm - 1) {
        const int c = __builtin_ctz(mm);
        dx += fld(F_WCPL, c) * s[2 * (c - 1)];
      }
      xn[b] = xo + dt * dx;
      yn[b] = yo + dt * dy;
      const float x = std::fmin(std::fmax(xn[b], -1.f), 1.f);
      const float t = P.kp * (P.theta_max * x - q[6 + b]) - P.kd * v[5 + b];
      tau[5 + b] = std::fmin(std::fmax(t, -P.tau_max), P.tau_max);
    }
  }

  // ---- 2. forward kinematics (parents precede children), FP64 heights
  float R0[9];
  quat_to_R(q[3], q[4], q[5], q[6], R0);
  for (int k = 0; k < 9; ++k) w.R[k][0] = R0[k];
  for (int k = 0; k < 3; ++k) w.r[k][0] = 0.f;
  {
    const double dw = q[3], dx = q[4], dy = q[5], dz = q[6];
    w.hz[0][0] = 2.0 * (dx * dz - dw * dy);
    w.hz[1][0] = 2.0 * (dy * dz + dw * dx);
    w.hz[2][0] = 1.0 - 2.0 * (dx * dx + dy * dy);
    w.hzb[0] = 0.0;
  }
  for (int b = 1; b < nb; ++b) {
    const int p = parent[b];
    double sd, cd;
    sincos_f64((double)q[6 + b], &sd, &cd);
    const float sth = (float)sd, cth = (float)cd;
    const int k = axis[b], i = (k + 1) % 3, j = (k + 2) % 3;
    float Rl[9];
    for (int row = 0; row < 3; ++row) {
      const float fi = fld(F_RFIX + 3 * row + i, b), fj = fld(F_RFIX + 3 * row + j, b);
      Rl[3 * row + k] = fld(F_RFIX + 3 * row + k, b);
      Rl[3 * row + i] = cth * fi + sth * fj;
      Rl[3 * row + j] = -sth * fi + cth * fj;
    }
    float Rp[9], rp[3];
    for (int t = 0; t < 9; ++t) Rp[t] = w.R[t][p];
    for (int t = 0; t < 3; ++t) rp[t] = w.r[t][p];
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c)
        w.R[3 * a + c][b] = Rp[3 * a] * Rl[c] + Rp[3 * a + 1] * Rl[3 + c] + Rp[3 * a + 2] * Rl[6 + c];
    const float pf0 = fld(F_PFIX, b), pf1 = fld(F_PFIX + 1, b), pf2 = fld(F_PFIX + 2, b);
    for (int a = 0; a < 3; ++a) w.r[a][b] = rp[a] + (Rp[3 * a] * pf0 + Rp[3 * a + 1] * pf1 + Rp[3 * a + 2] * pf2);
    // third row of R_b and the frame-origin height, FP64
    const double p0 = w.hz[0][p], p1 = w.hz[1][p], p2 = w.hz[2][p];
    double t3[3];
    for (int col = 0; col < 3; ++col)
      t3[col] = p0 * (double)fld(F_RFIX + col, b) + p1 * (double)fld(F_RFIX + 3 + col, b) +
                p2 * (double)fld(F_RFIX + 6 + col, b);
    double o3[3];
    o3[k] = t3[k];
    o3[i] = cd * t3[i] + sd * t3[j];
    o3[j] = -sd * t3[i] + cd * t3[j];
    for (int t = 0; t < 3; ++t) w.hz[t][b] = o3[t];
    w.hzb[b] = w.hzb[p] + (p0 * (double)pf0 + p1 * (double)pf1 + p2 * (double)pf2);
  }
  for (int b = 0; b < nb; ++b) {
    const float c0 = fld(F_COM, b), c1 = fld(F_COM + 1, b), c2 = fld(F_COM + 2, b);
    for (int a = 0; a < 3; ++a)
      w.c[a][b] = w.r[a][b] + (w.R[3 * a][b] * c0 + w.R[3 * a + 1][b] * c1 + w.R[3 * a + 2][b] * c2);
  }
  // motion subspaces: root (linear world axes, angular body axes), hinges
  for (int d = 0; d < 6; ++d) {
    float col[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (d < 3) col[3 + d] = 1.f;
    else { col[0] = R0[d - 3]; col[1] = R0[3 + d - 3]; col[2] = R0[6 + d - 3]; }
    for (int t = 0; t < 6; ++t) w.S[t][d] = col[t];
  }
  for (int b = 1; b < nb; ++b) {
    float Sb[6];
    Sb[0] = w.R[axis[b]][b]; Sb[1] = w.R[3 + axis[b]][b]; Sb[2] = w.R[6 + axis[b]][b];
    const float rb[3] = {w.r[0][b], w.r[1][b], w.r[2][b]};
    cross3(rb, Sb, Sb + 3);
    for (int t = 0; t < 6; ++t) w.S[t][5 + b] = Sb[t];
  }

  // ---- 3. spatial inertias about O, RNEA (gravity as base acceleration)
  float vb[32][6], ab[32][6];
  {
    const float wb[3] = {v[3], v[4], v[5]};
    const float om[3] = {R0[0] * wb[0] + R0[1] * wb[1] + R0[2] * wb[2], R0[3] * wb[0] + R0[4] * wb[1] + R0[5] * wb[2],
                         R0[6] * wb[0] + R0[7] * wb[1] + R0[8] * wb[2]};
    const float vl[3] = {v[0], v[1], v[2]};
    float vxw[3];
    cross3(vl, om, vxw);
    for (int t = 0; t < 3; ++t) { vb[0][t] = om[t]; vb[0][3 + t] = vl[t]; ab[0][t] = 0.f; }
    ab[0][3] = vxw[0] - P.gx; ab[0][4] = vxw[1] - P.gy; ab[0][5] = vxw[2] - P.gz;
  }
  for (int b = 1; b < nb; ++b) {
    const int p = parent[b];
    float Sq[6], cr[6];
    for (int t = 0; t < 6; ++t) { Sq[t] = w.S[t][5 + b] * v[5 + b]; vb[b][t] = vb[p][t] + Sq[t]; }
    crm(vb[b], Sq, cr);
    for (int t = 0; t < 6; ++t) ab[b][t] = ab[p][t] + cr[t];
  }
  for (int b = 0; b < nb; ++b) {
    float I[10];
    const float mass = fld(F_MASS, b), i0 = fld(F_ID, b), i1 = fld(F_ID + 1, b), i2 = fld(F_ID + 2, b);
    float Rb[9];
    for (int t = 0; t < 9; ++t) Rb[t] = w.R[t][b];
    const float cb[3] = {w.c[0][b], w.c[1][b], w.c[2][b]};
    float Iw[6];
    Iw[0] = Rb[0] * Rb[0] * i0 + Rb[1] * Rb[1] * i1 + Rb[2] * Rb[2] * i2;
    Iw[1] = Rb[3] * Rb[3] * i0 + Rb[4] * Rb[4] * i1 + Rb[5] * Rb[5] * i2;
    Iw[2] = Rb[6] * Rb[6] * i0 + Rb[7] * Rb[7] * i1 + Rb[8] * Rb[8] * i2;
    Iw[3] = Rb[0] * Rb[3] * i0 + Rb[1] * Rb[4] * i1 + Rb[2] * Rb[5] * i2;
    Iw[4] = Rb[0] * Rb[6] * i0 + Rb[1] * Rb[7] * i1 + Rb[2] * Rb[8] * i2;
    Iw[5] = Rb[3] * Rb[6] * i0 + Rb[4] * Rb[7] * i1 + Rb[5] * Rb[8] * i2;
    const float cc = cb[0] * cb[0] + cb[1] * cb[1] + cb[2] * cb[2];
    I[0] = mass;
    I[1] = mass * cb[0]; I[2] = mass * cb[1]; I[3] = mass * cb[2];
    I[4] = Iw[0] + mass * (cc - cb[0] * cb[0]);
    I[5] = Iw[1] + mass * (cc - cb[1] * cb[1]);
    I[6] = Iw[2] + mass * (cc - cb[2] * cb[2]);
    I[7] = Iw[3] - mass * cb[0] * cb[1];
    I[8] = Iw[4] - mass * cb[0] * cb[2];
    I[9] = Iw[5] - mass * cb[1] * cb[2];
    float Ia[6], Iv[6], x[6];
    inertia_apply(I, ab[b], Ia);
    inertia_apply(I, vb[b], Iv);
    crf(vb[b], Iv, x);
    for (int t = 0; t < 6; ++t) w.acc[t][b] = Ia[t] + x[t];
    for (int t = 0; t < 10; ++t) w.acc[6 + t][b] = I[t];
  }
  for (int b = nb - 1; b >= 1; --b)
    for (int t = 0; t < 16; ++t) w.acc[t][parent[b]] += w.acc[t][b];
  float cvec[32];
  for (int b = 1; b < nb; ++b)
    cvec[5 + b] = w.S[0][5 + b] * w.acc[0][b] + w.S[1][5 + b] * w.acc[1][b] + w.S[2][5 + b] * w.acc[2][b] +
                  w.S[3][5 + b] * w.acc[3][b] + w.S[4][5 + b] * w.acc[4][b] + w.S[5][5 + b] * w.acc[5][b];
  for (int k = 0; k < 3; ++k) {
    cvec[k] = w.acc[3 + k][0];
    cvec[3 + k] = R0[k] * w.acc[0][0] + R0[3 + k] * w.acc[1][0] + R0[6 + k] * w.acc[2][0];
  }

  // ---- 4. CRBA (packed lower triangle)
  for (int t = 0; t < tri(nv); ++t) w.M[t] = 0.f;
  for (int b = 1; b < nb; ++b) {
    float Ic[10], Sb[6], Fv[6];
    for (int t = 0; t < 10; ++t) Ic[t] = w.acc[6 + t][b];
    for (int t = 0; t < 6; ++t) Sb[t] = w.S[t][5 + b];
    inertia_apply(Ic, Sb, Fv);
    const int i = 5 + b, ti = tri(i);
    w.M[ti + i] = Sb[0] * Fv[0] + Sb[1] * Fv[1] + Sb[2] * Fv[2] + Sb[3] * Fv[3] + Sb[4] * Fv[4] + Sb[5] * Fv[5] +
                  P.armature;
    for (int j = parent[b]; j > 0; j = parent[j]) {
      const int jj = 5 + j;
      w.M[ti + jj] = w.S[0][jj] * Fv[0] + w.S[1][jj] * Fv[1] + w.S[2][jj] * Fv[2] + w.S[3][jj] * Fv[3] +
                     w.S[4][jj] * Fv[4] + w.S[5][jj] * Fv[5];
    }
    for (int k = 0; k < 3; ++k) w.M[ti + k] = Fv[3 + k];
    for (int k = 0; k < 3; ++k) w.M[ti + 3 + k] = R0[k] * Fv[0] + R0[3 + k] * Fv[1] + R0[6 + k] * Fv[2];
  }
  {
    float Ic[10];
    for (int t = 0; t < 10; ++t) Ic[t] = w.acc[6 + t][0];
    for (int d = 0; d < 6; ++d) {
      float Sk[6], Fv[6];
      for (int t = 0; t < 6; ++t) Sk[t] = w.S[t][d];
      inertia_apply(Ic, Sk, Fv);
      for (int l = d; l < 6; ++l)
        w.M[tri(l) + d] = w.S[0][l] * Fv[0] + w.S[1][l] * Fv[1] + w.S[2][l] * Fv[2] + w.S[3][l] * Fv[3] +
                          w.S[4][l] * Fv[4] + w.S[5][l] * Fv[5];
    }
  }

  // ---- 5. Cholesky (left-looking) and v_free = v + dt M^-1 (tau - c)
  for (int j = 0; j < nv; ++j) {
    const float* Lj = w.M + tri(j);
    float mij[32];
    for (int i = j; i < nv; ++i) {
      const float* Li = w.M + tri(i);
      float s0 = 0.f, s1 = 0.f;
      int k = 0;
      for (; k + 1 < j; k += 2) {
        s0 += Li[k] * Lj[k];
        s1 += Li[k + 1] * Lj[k + 1];
      }
      if (k < j) s0 += Li[k] * Lj[k];
      mij[i] = Li[j] - (s0 + s1);
    }
    const float piv = mij[j];
    if (!(piv > 0.f)) {
      st |= SIM_ST_CHOL;
      return false;
    }
    const float d = std::sqrt(piv), inv = 1.f / d;
    w.M[tri(j) + j] = d;
    w.invd[j] = inv;
    for (int i = j + 1; i < nv; ++i) w.M[tri(i) + j] = mij[i] * inv;
  }
  auto lower_solve = [&](float* x) {  // x <- L^-1 x
    for (int i = 0; i < nv; ++i) {
      float a = x[i];
      for (int k = 0; k < i; ++k) a -= w.M[tri(i) + k] * x[k];
      x[i] = a * w.invd[i];
    }
  };
  auto upper_solve = [&](float* x) {  // x <- L^-T x
    for (int i = nv - 1; i >= 0; --i) {
      const float xi = x[i] * w.invd[i];
      x[i] = xi;
      for (int k = 0; k < i; ++k) x[k] -= w.M[tri(i) + k] * xi;
    }
  };
  {
    float t[32];
    for (int j = 0; j < nv; ++j) t[j] = (j >= 6 ? tau[j] : 0.f) - cvec[j];
    lower_solve(t);
    upper_solve(t);
    for (int j = 0; j < nv; ++j) w.vfree[j] = v[j] + dt * t[j];
  }

  // ---- 6. contact candidates: body/plane points, then body/body pairs
  int ncand = 0;
  if (P.ground) {
    const float up[3] = {0.f, 0.f, 1.f};
    for (int b = 0; b < nb; ++b) {
      // a box's 8 vertices; a sphere's lowest point (no half-size offsets, r below)
      const bool sph = fld(F_GEOM, b) != 0.f;
      const float hr = fld(F_HALF, b);
      const float h0 = sph ? 0.f : hr, h1 = sph ? 0.f : fld(F_HALF + 1, b), h2 = sph ? 0.f : fld(F_HALF + 2, b);
      const float drop = sph ? hr : 0.f;
      const float c0 = fld(F_COM, b), c1 = fld(F_COM + 1, b), c2 = fld(F_COM + 2, b);
      for (int k = 0; k < (sph ? 1 : 8); ++k) {
        const float l0 = c0 + ((k & 1) ? h0 : -h0), l1 = c1 + ((k & 2) ? h1 : -h1), l2 = c2 + ((k & 4) ? h2 : -h2);
        const double h = (double)q[2] + (w.hzb[b] + (w.hz[0][b] * (double)l0 + w.hz[1][b] * (double)l1 +
                                                     w.hz[2][b] * (double)l2)) - (double)drop;
        if (!(h < 0.0)) continue;
        if (ncand < kCand) {
          float pr[3];
          for (int a = 0; a < 3; ++a)
            pr[a] = w.r[a][b] + (w.R[3 * a][b] * l0 + w.R[3 * a + 1][b] * l1 + w.R[3 * a + 2][b] * l2);
          pr[2] -= drop;
          put_candidate(&w.cand[0][0], ncand, pr, up, (float)(-h), b, 255);
        }
        ++ncand;
      }
    }
    if (ncand > kCand) { st |= SIM_ST_CANDIDATES; ncand = kCand; }
  }
  if (P.box_box) {
    float stage[8 * kCandW];
    for (int pi = 0; pi < m.npairs; ++pi) {
      const unsigned pr = pairs[m.pairoff + pi];
      const int a = (int)(pr >> 8), b = (int)(pr & 0xffu);
      const float dx = w.c[0][b] - w.c[0][a], dy = w.c[1][b] - w.c[1][a], dz = w.c[2][b] - w.c[2][a];
      const float rr = fld(F_RAD, a) + fld(F_RAD, b);
      if (!(dx * dx + dy * dy + dz * dz <= rr * rr)) continue;
      const int cnt = body_pair_lane(w.R, w.c, F, a, b, stage);
      for (int t = 0; t < cnt; ++t) {
        if (ncand + t < kCand) std::memcpy(w.cand[ncand + t], stage + t * kCandW, kCandW * sizeof(float));
      }
      ncand += cnt;
    }
    if (ncand > kCand) { st |= SIM_ST_CANDIDATES; ncand = kCand; }
  }
  // keep the cap deepest (ties by list order), list order kept
  int nc = ncand;
  if (ncand > P.cap) {
    st |= SIM_ST_OVERFLOW;
    static thread_local bool keep[kCand];
    for (int i = 0; i < ncand; ++i) {
      const float di = w.cand[i][6];
      int rank = 0;
      for (int j = 0; j < ncand; ++j) {
        const float dj = w.cand[j][6];
        rank += (dj > di || (dj == di && j < i)) ? 1 : 0;
      }
      keep[i] = rank < P.cap;
    }
    int kept = 0;
    for (int i = 0; i < ncand; ++i)
      if (keep[i]) {
        if (kept != i) std::memcpy(w.cand[kept], w.cand[i], kCandW * sizeof(float));
        ++kept;
      }
    nc = P.cap;
  }
  contacts += (unsigned long long)nc;

  // ---- 7. contact rows: Y_r = L^-1 J_r^T and the Gauss-Seidel constants
  for (int row = 0; row < 3 * nc; ++row) {
    const int k = row / 3, dir = row - 3 * k;
    const float* cw = w.cand[k];
    const float pr[3] = {cw[0], cw[1], cw[2]};
    const float nrm[3] = {cw[3], cw[4], cw[5]};
    const float depth_k = cw[6];
    const int ab = float_bits_as_int(cw[7]);
    const int a = ab & 0xff, b = (ab >> 8) & 0xff;
    const unsigned pa = path[a], pb = b == 255 ? 0u : path[b];
    const float sroot = (b == 255) ? 1.f : 0.f;
    float t1[3], t2[3], d[3];
    if (b == 255) tangent_basis(nrm, t1, t2);
    else pair_tangent_basis(nrm, t1, t2);
    for (int t = 0; t < 3; ++t) d[t] = dir == 0 ? nrm[t] : (dir == 1 ? t1[t] : t2[t]);
    float wa[3];
    cross3(pr, d, wa);
    float* yr = w.Y[row];
    float jv = 0.f;
    for (int j = 0; j < nv; ++j) {
      float coef;
      if (j < 6) coef = sroot;
      else {
        const int bj = j - 5;
        coef = (float)((int)((pa >> bj) & 1u) - (int)((pb >> bj) & 1u));
      }
      const float Jj = coef * (w.S[0][j] * wa[0] + w.S[1][j] * wa[1] + w.S[2][j] * wa[2] + w.S[3][j] * d[0] +
                               w.S[4][j] * d[1] + w.S[5][j] * d[2]);
      jv += Jj * w.vfree[j];
      yr[j] = Jj;
    }
    for (int j = nv; j < 32; ++j) yr[j] = 0.f;
    float aa = 0.f;
    for (int i = 0; i < nv; ++i) {
      const float* Li = w.M + tri(i);
      float t0 = yr[i], tt = 0.f;
      int kk = 0;
      for (; kk + 1 < i; kk += 2) {
        t0 -= Li[kk] * yr[kk];
        tt -= Li[kk + 1] * yr[kk + 1];
      }
      if (kk < i) t0 -= Li[kk] * yr[kk];
      const float yi = (t0 + tt) * w.invd[i];
      yr[i] = yi;
      aa += yi * yi;
    }
    const float Rr = std::fmax(P.kappa * aa, P.min_cfm);  // floored softness (see the GPU kernel)
    const float inv = aa > kAmin ? 1.f / (aa + Rr) : 0.f;
    const float bias = dir == 0 ? jv - std::fmin(P.erp * depth_k / dt, P.max_correct_vel) : jv;
    w.cst[k][3 * dir] = bias;
    w.cst[k][3 * dir + 1] = inv;
    w.cst[k][3 * dir + 2] = Rr;
  }
  for (int k = 0; k < nc; ++k) {
    const float *yn = w.Y[3 * k], *y1 = w.Y[3 * k + 1], *y2 = w.Y[3 * k + 2];
    float a1 = 0.f, a2 = 0.f;
    for (int i = 0; i < 32; i += 4) {
      a1 += y1[i] * yn[i] + y1[i + 1] * yn[i + 1] + y1[i + 2] * yn[i + 2] + y1[i + 3] * yn[i + 3];
      a2 += y2[i] * yn[i] + y2[i + 1] * yn[i + 1] + y2[i + 2] * yn[i + 2] + y2[i + 3] * yn[i + 3];
    }
    w.cst[k][9] = a1;
    w.cst[k][10] = a2;
  }

  // ---- 8. soft projected Gauss-Seidel in u = L^T (v - v_free)
  float u[32];
  for (int j = 0; j < 32; ++j) u[j] = 0.f;
  float lam[kCapMax][3];
  for (int k = 0; k < nc; ++k) lam[k][0] = lam[k][1] = lam[k][2] = 0.f;
  for (int it = 0; it < P.iters && nc > 0; ++it) {
    for (int k = 0; k < nc; ++k) {
      const float *y0 = w.Y[3 * k], *y1 = w.Y[3 * k + 1], *y2 = w.Y[3 * k + 2];
      const float* cs = w.cst[k];
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      for (int j = 0; j < nv; ++j) {
        s0 += y0[j] * u[j];
        s1 += y1[j] * u[j];
        s2 += y2[j] * u[j];
      }
      const float ln = lam[k][0], l1 = lam[k][1], l2 = lam[k][2];
      // constants: b_n inv_n R_n | b_t1 inv_t1 R_t1 | b_t2 inv_t2 R_t2 | A_t1n A_t2n
      const float gn = s0 + cs[0] + cs[2] * ln;
      const float lnn = std::fmax(0.f, ln - gn * cs[1]);
      const float dn = lnn - ln;
      const float g1 = s1 + cs[9] * dn + cs[3] + cs[5] * l1;
      const float g2 = s2 + cs[10] * dn + cs[6] + cs[8] * l2;
      float l1t = l1 - g1 * cs[4];
      float l2t = l2 - g2 * cs[7];
      const float lim = P.mu * lnn;
      const float nt2 = l1t * l1t + l2t * l2t;
      if (nt2 > lim * lim) {
        const float sc = lim / std::sqrt(nt2);
        l1t *= sc;
        l2t *= sc;
      }
      const float d1 = l1t - l1, d2 = l2t - l2;
      for (int j = 0; j < nv; ++j) u[j] += y0[j] * dn + y1[j] * d1 + y2[j] * d2;
      lam[k][0] = lnn;
      lam[k][1] = l1t;
      lam[k][2] = l2t;
    }
  }
  upper_solve(u);
  float vplus[32];
  for (int j = 0; j < nv; ++j) vplus[j] = w.vfree[j] + u[j];

  // ---- 9. semi-implicit Euler: root position, quaternion exponential map, hinges
  const float np0[3] = {q[0] + dt * vplus[0], q[1] + dt * vplus[1], q[2] + dt * vplus[2]};
  const float ox = vplus[3], oy = vplus[4], oz = vplus[5];
  float dq0 = 1.f, dq1 = 0.f, dq2 = 0.f, dq3 = 0.f;
  {
    const float nw = std::sqrt(ox * ox + oy * oy + oz * oz);
    if (nw >= 1e-12f) {
      float sa = std::sin(0.5f * dt * nw), ca = std::cos(0.5f * dt * nw);
      sa = sa / nw;
      dq0 = ca; dq1 = sa * ox; dq2 = sa * oy; dq3 = sa * oz;
    }
  }
  const float qw = q[3], qx = q[4], qy = q[5], qz = q[6];
  float r0 = qw * dq0 - qx * dq1 - qy * dq2 - qz * dq3;
  float r1 = qw * dq1 + qx * dq0 + qy * dq3 - qz * dq2;
  float r2 = qw * dq2 - qx * dq3 + qy * dq0 + qz * dq1;
  float r3 = qw * dq3 + qx * dq2 - qy * dq1 + qz * dq0;
  const float nr = std::sqrt(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
  r0 /= nr; r1 /= nr; r2 /= nr; r3 /= nr;
  bool bad = !(std::isfinite(np0[0]) && std::isfinite(np0[1]) && std::isfinite(np0[2]) && std::isfinite(r0) &&
               std::isfinite(r1) && std::isfinite(r2) && std::isfinite(r3));
  float ntheta[32];
  for (int b = 1; b < nb; ++b) {
    ntheta[b] = q[6 + b] + dt * vplus[5 + b];
    bad = bad || !std::isfinite(ntheta[b]) || !std::isfinite(xn[b]) || !std::isfinite(yn[b]);
  }
  for (int j = 0; j < nv; ++j) bad = bad || !std::isfinite(vplus[j]);
  if (bad) {
    st |= SIM_ST_NONFINITE;
    return false;
  }
  q[0] = np0[0]; q[1] = np0[1]; q[2] = np0[2];
  q[3] = r0; q[4] = r1; q[5] = r2; q[6] = r3;
  for (int b = 1; b < nb; ++b) {
    q[6 + b] = ntheta[b];
    s[2 * (b - 1)] = xn[b];
    s[2 * (b - 1) + 1] = yn[b];
  }
  for (int j = 0; j < nv; ++j) v[j] = vplus[j];
  return true;
}

StepParams params_of(const sim_config* cfg) {
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

}  // namespace

struct cpu_ctx {
  sim_config cfg{};
  StepParams P{};
  int threads = 1;
  std::string err;
  PackedPopulation pk;
  int n = 0;
  std::vector<float> q, v, s, fit0;
  std::vector<unsigned> status;
  std::vector<unsigned long long> contacts;  // per robot
  std::vector<double> seconds;               // per robot, last cpu_step_n
};

namespace {
int fail(cpu_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}
}  // namespace

extern "C" {

int cpu_create(const sim_config* cfg, int32_t threads, cpu_ctx_t** out) {
  if (!out) return SIM_EINVAL;
  *out = nullptr;
  if (!cfg || threads < 0 || !(cfg->dt > 0.0) || cfg->pgs_iters < 1 || cfg->contact_cap < 1 ||
      cfg->contact_cap > SIM_MAX_CONTACT_CAP || !(cfg->soft_tau > 0.f) || !(cfg->soft_zeta >= 0.f) ||
      !(cfg->mu >= 0.f) || !(cfg->max_correct_vel > 0.f) || !(cfg->min_cfm >= 0.f))
    return SIM_EINVAL;
  cpu_ctx* ctx = new (std::nothrow) cpu_ctx;
  if (!ctx) return SIM_ENOMEM;
  ctx->cfg = *cfg;
  ctx->P = params_of(cfg);
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  ctx->threads = threads > 0 ? threads : (int)hw;
  *out = ctx;
  return SIM_OK;
}

int cpu_destroy(cpu_ctx_t* ctx) {
  delete ctx;
  return SIM_OK;
}

int cpu_set_population(cpu_ctx_t* ctx, const sim_variant_desc* v, int32_t n) {
  if (!ctx) return SIM_EINVAL;
  // robots of up to SIM_WARP_MAX_BODIES bodies (the warp layout); longer
  // chains are stepped by the GPU simulator only
  const std::string why = validate_population(v, n, "cpu_set_population", SIM_WARP_MAX_BODIES);
  if (!why.empty()) return fail(ctx, SIM_EINVAL, why);
  try {
    pack_population(v, n, ctx->pk);
    ctx->n = n;
    ctx->q.assign((size_t)n * 32, 0.f);
    ctx->v.assign((size_t)n * 32, 0.f);
    ctx->s.assign((size_t)n * 64, 0.f);
    ctx->fit0.assign((size_t)n * 2, 0.f);
    ctx->status.assign(n, 0u);
    ctx->contacts.assign(n, 0ull);
    ctx->seconds.assign(n, 0.0);
  } catch (const std::bad_alloc&) {
    ctx->n = 0;
    return fail(ctx, SIM_ENOMEM, "cpu_set_population: out of host memory");
  }
  return SIM_OK;
}

int cpu_set_state(cpu_ctx_t* ctx, int32_t first, int32_t count, const float* q, const float* v, const float* cpg) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "cpu_set_state: no population");
  if (!q || !v || first < 0 || count < 0 || first + count > ctx->n)
    return fail(ctx, SIM_EINVAL, "cpu_set_state: bad range or NULL q/v");
  for (int i = 0; i < count; ++i) {
    const int d = ctx->pk.inv[first + i];
    // rows of the warp layout: nq, nv <= 32, 2 nh <= 64 (the rest of a host row is ignored)
    std::memcpy(&ctx->q[(size_t)d * 32], q + (size_t)i * SIM_QW, 32 * sizeof(float));
    std::memcpy(&ctx->v[(size_t)d * 32], v + (size_t)i * SIM_VW, 32 * sizeof(float));
    if (cpg) std::memcpy(&ctx->s[(size_t)d * 64], cpg + (size_t)i * SIM_SW, 64 * sizeof(float));
    ctx->fit0[2 * d] = q[(size_t)i * SIM_QW];
    ctx->fit0[2 * d + 1] = q[(size_t)i * SIM_QW + 1];
    ctx->status[d] = 0u;
  }
  return SIM_OK;
}

int cpu_step_n(cpu_ctx_t* ctx, int32_t n_steps) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "cpu_step_n: no population");
  if (n_steps < 0) return fail(ctx, SIM_EINVAL, "cpu_step_n: n_steps < 0");
  if (n_steps == 0) return SIM_OK;
  std::atomic<int> next{0};
  auto worker = [&]() {
    Work* w = new (std::nothrow) Work;
    if (!w) return;
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= ctx->n) break;
      const int* meta = &ctx->pk.meta[4 * (size_t)k];
      const Robot m{ctx->pk.mf.data() + (size_t)k * NF * 32, ctx->pk.mi.data() + (size_t)k * NI * 32, meta[0],
                    meta[1], meta[2], meta[3]};
      unsigned st = ctx->status[k];
      unsigned long long nc = 0;
      const auto t0 = std::chrono::steady_clock::now();
      if (free_body_eligible(m.nb, m.F + F_COM * 32)) {
        // a single free body: the one-body closed form of the step
        FreeBodyOut fo;
        for (int t = 0; t < n_steps && !(st & 5u); ++t)
          if (free_body_step(m.F, ctx->P, &ctx->q[(size_t)k * 32], &ctx->v[(size_t)k * 32], st, fo)) nc += fo.nc;
      } else {
        for (int t = 0; t < n_steps && !(st & 5u); ++t)
          step_robot(m, ctx->pk.pairs.data(), ctx->P, &ctx->q[(size_t)k * 32], &ctx->v[(size_t)k * 32],
                     &ctx->s[(size_t)k * 64], st, nc, *w);
      }
      ctx->seconds[k] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      ctx->status[k] = st;
      ctx->contacts[k] += nc;
    }
    delete w;
  };
  const int nt = std::max(1, std::min(ctx->threads, ctx->n));
  std::vector<std::thread> pool;
  pool.reserve(nt - 1);
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  if (next.load() < ctx->n) return fail(ctx, SIM_ENOMEM, "cpu_step_n: could not allocate a work space");
  return SIM_OK;
}

int cpu_read_state(cpu_ctx_t* ctx, int32_t first, int32_t count, float* q, float* v, float* cpg, uint32_t* status) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "cpu_read_state: no population");
  if (first < 0 || count < 0 || first + count > ctx->n) return fail(ctx, SIM_EINVAL, "cpu_read_state: bad range");
  for (int i = 0; i < count; ++i) {
    const int d = ctx->pk.inv[first + i];
    if (q) {
      std::memcpy(q + (size_t)i * SIM_QW, &ctx->q[(size_t)d * 32], 32 * sizeof(float));
      std::memset(q + (size_t)i * SIM_QW + 32, 0, (SIM_QW - 32) * sizeof(float));
    }
    if (v) {
      std::memcpy(v + (size_t)i * SIM_VW, &ctx->v[(size_t)d * 32], 32 * sizeof(float));
      std::memset(v + (size_t)i * SIM_VW + 32, 0, (SIM_VW - 32) * sizeof(float));
    }
    if (cpg) {
      std::memcpy(cpg + (size_t)i * SIM_SW, &ctx->s[(size_t)d * 64], 64 * sizeof(float));
      std::memset(cpg + (size_t)i * SIM_SW + 64, 0, (SIM_SW - 64) * sizeof(float));
    }
    if (status) status[i] = ctx->status[d];
  }
  return SIM_OK;
}

int cpu_fitness(cpu_ctx_t* ctx, float* out, int32_t n) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "cpu_fitness: no population");
  if (!out || n < 0 || n > ctx->n) return fail(ctx, SIM_EINVAL, "cpu_fitness: bad n or NULL out");
  for (int i = 0; i < n; ++i) {
    const int d = ctx->pk.inv[i];
    const float dx = ctx->q[(size_t)d * 32] - ctx->fit0[2 * d];
    const float dy = ctx->q[(size_t)d * 32 + 1] - ctx->fit0[2 * d + 1];
    out[i] = std::sqrt(dx * dx + dy * dy);
  }
  return SIM_OK;
}

int cpu_robot_seconds(cpu_ctx_t* ctx, double* out, int32_t n) {
  if (!ctx) return SIM_EINVAL;
  if (ctx->n == 0) return fail(ctx, SIM_ESTATE, "cpu_robot_seconds: no population");
  if (!out || n < 0 || n > ctx->n) return fail(ctx, SIM_EINVAL, "cpu_robot_seconds: bad n or NULL out");
  for (int i = 0; i < n; ++i) out[i] = ctx->seconds[ctx->pk.inv[i]];
  return SIM_OK;
}

int cpu_threads(const cpu_ctx_t* ctx) { return ctx ? ctx->threads : 0; }

int cpu_contacts(cpu_ctx_t* ctx, double* out) {
  if (!ctx || !out) return SIM_EINVAL;
  double t = 0.0;
  for (unsigned long long c : ctx->contacts) t += (double)c;
  *out = t;
  return SIM_OK;
}

const char* cpu_last_error(const cpu_ctx_t* ctx) { return ctx ? ctx->err.c_str() : ""; }

}  // extern "C"
