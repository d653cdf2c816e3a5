// model_pack.h -- validation and structure-of-arrays packing of a robot
// population (host code shared by the GPU simulator and the CPU engine).
//
// Layout per packed robot k (robots sorted by body count, largest first,
// stable; single free bodies with their centre at the frame origin last): float fields [NF][32 body slots], int fields [NI][32], meta
// (bodies, tree depth, pair count, pair offset) and the list of body/body
// candidate pairs (a < b, a not the parent of b, not excluded), each packed
// as (a << 8) | b.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "b3sim.h"
#include "step_common.cuh"

namespace b3 {

struct PackedPopulation {
  int n_free = 0;         // single free bodies (free_body.cuh), packed last
  std::vector<int> perm;  // packed index -> caller index
  std::vector<int> inv;   // caller index -> packed index
  std::vector<float> mf;
  std::vector<int> mi;
  std::vector<int> meta;  // 4 ints per robot: bodies, max depth, pair count, pair offset
  std::vector<uint16_t> pairs;
};

inline bool finite_all(const float* p, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Returns an empty string on success, else the reason the population is invalid.
inline std::string validate_population(const sim_variant_desc* v, int n, const char* who) {
  if (!v || n < 1) return std::string(who) + ": need n >= 1 variants";
  for (int i = 0; i < n; ++i) {
    const sim_variant_desc& d = v[i];
    const int nb = d.n_bodies;
    char buf[160];
    if (nb < 1 || nb > SIM_MAX_BODIES) {
      snprintf(buf, sizeof buf, ": variant %d has %d bodies (1..%d)", i, nb, SIM_MAX_BODIES);
      return std::string(who) + buf;
    }
    if (!d.parent || !d.hinge_axis || !d.joint_frame || !d.half_size || !d.box_center || !d.mass) {
      snprintf(buf, sizeof buf, ": variant %d has a NULL model array", i);
      return std::string(who) + buf;
    }
    if (d.parent[0] != -1) {
      snprintf(buf, sizeof buf, ": variant %d: parent[0] must be -1", i);
      return std::string(who) + buf;
    }
    for (int b = 0; b < nb; ++b) {
      if ((b > 0 && (d.parent[b] < 0 || d.parent[b] >= b)) || d.hinge_axis[b] < 0 || d.hinge_axis[b] > 2 ||
          !(d.mass[b] > 0.f) || !finite_all(d.joint_frame + 12 * b, 12) || !finite_all(d.half_size + 3 * b, 3) ||
          !finite_all(d.box_center + 3 * b, 3) || !(d.half_size[3 * b] > 0.f) || !(d.half_size[3 * b + 1] > 0.f) ||
          !(d.half_size[3 * b + 2] > 0.f) ||
          (d.cpg_w_internal && !std::isfinite(d.cpg_w_internal[b])) ||
          (d.cpg_w_couple && !std::isfinite(d.cpg_w_couple[b])) ||
          (d.geom && d.geom[b] != SIM_GEOM_BOX && d.geom[b] != SIM_GEOM_SPHERE) ||
          (d.geom && d.geom[b] == SIM_GEOM_SPHERE &&
           (d.half_size[3 * b + 1] != d.half_size[3 * b] || d.half_size[3 * b + 2] != d.half_size[3 * b]))) {
        snprintf(buf, sizeof buf, ": variant %d body %d is invalid", i, b);
        return std::string(who) + buf;
      }
    }
  }
  return std::string();
}

inline void pack_population(const sim_variant_desc* v, int n, PackedPopulation& out) {
  // pack in size order (largest first, stable), the single free bodies that
  // the one-body step serves last of all
  auto is_free = [&](int i) {
    return v[i].n_bodies == 1 && v[i].box_center[0] == 0.f && v[i].box_center[1] == 0.f &&
           v[i].box_center[2] == 0.f;
  };
  std::vector<int>& perm = out.perm;
  perm.resize(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
    if (v[a].n_bodies != v[b].n_bodies) return v[a].n_bodies > v[b].n_bodies;
    return !is_free(a) && is_free(b);
  });
  out.n_free = 0;
  for (int i = 0; i < n; ++i) out.n_free += is_free(i) ? 1 : 0;
  std::vector<int>& inv = out.inv;
  inv.assign(n, 0);
  for (int k = 0; k < n; ++k) inv[perm[k]] = k;
  std::vector<float>& mf = out.mf;
  mf.assign((size_t)n * b3::NF * 32, 0.f);
  std::vector<int>& mi = out.mi;
  mi.assign((size_t)n * b3::NI * 32, 0);
  std::vector<int>& meta = out.meta;
  meta.assign((size_t)4 * n, 0);
  std::vector<uint16_t>& pairs = out.pairs;
  pairs.clear();
  for (int k = 0; k < n; ++k) {
    const sim_variant_desc& d = v[perm[k]];
    const int nb = d.n_bodies;
    float* F = mf.data() + (size_t)k * b3::NF * 32;
    int* I = mi.data() + (size_t)k * b3::NI * 32;
    int depth[32] = {0};
    unsigned path[32] = {0}, child[32] = {0};
    int maxdepth = 0;
    for (int b = 0; b < nb; ++b) {
      const int p = b == 0 ? -1 : d.parent[b];
      depth[b] = p < 0 ? 0 : depth[p] + 1;
      path[b] = (p < 0 ? 0u : path[p]) | (1u << b);
      if (p >= 0) child[p] |= 1u << b;
      maxdepth = std::max(maxdepth, depth[b]);
    }
    for (int b = 0; b < 32; ++b) {
      I[b3::I_PARENT * 32 + b] = b < nb ? (b == 0 ? -1 : d.parent[b]) : -1;
      I[b3::I_AXIS * 32 + b] = b < nb ? d.hinge_axis[b] : 0;
      I[b3::I_PATH * 32 + b] = (int)(b < nb ? path[b] : 0u);
      I[b3::I_CHILD * 32 + b] = (int)(b < nb ? child[b] : 0u);
      I[b3::I_DEPTH * 32 + b] = b < nb ? depth[b] : 0;
      if (b >= nb) {
        F[(b3::F_RFIX + 0) * 32 + b] = 1.f;
        F[(b3::F_RFIX + 4) * 32 + b] = 1.f;
        F[(b3::F_RFIX + 8) * 32 + b] = 1.f;
        continue;
      }
      for (int t = 0; t < 9; ++t) F[(b3::F_RFIX + t) * 32 + b] = d.joint_frame[12 * b + t];
      for (int t = 0; t < 3; ++t) {
        F[(b3::F_PFIX + t) * 32 + b] = d.joint_frame[12 * b + 9 + t];
        F[(b3::F_HALF + t) * 32 + b] = d.half_size[3 * b + t];
        F[(b3::F_COM + t) * 32 + b] = d.box_center[3 * b + t];
      }
      const double m = d.mass[b];
      const double hx = d.half_size[3 * b], hy = d.half_size[3 * b + 1], hz = d.half_size[3 * b + 2];
      const bool sphere = d.geom && d.geom[b] == SIM_GEOM_SPHERE;
      F[b3::F_MASS * 32 + b] = d.mass[b];
      if (sphere) {  // solid sphere: 2 m r^2 / 5 about every axis
        for (int t = 0; t < 3; ++t) F[(b3::F_ID + t) * 32 + b] = (float)(0.4 * m * hx * hx);
      } else {       // solid box: m (h_j^2 + h_k^2) / 3
        F[(b3::F_ID + 0) * 32 + b] = (float)(m * (hy * hy + hz * hz) / 3.0);
        F[(b3::F_ID + 1) * 32 + b] = (float)(m * (hx * hx + hz * hz) / 3.0);
        F[(b3::F_ID + 2) * 32 + b] = (float)(m * (hx * hx + hy * hy) / 3.0);
      }
      F[b3::F_WINT * 32 + b] = d.cpg_w_internal ? d.cpg_w_internal[b] : 0.f;
      F[b3::F_WCPL * 32 + b] = d.cpg_w_couple ? d.cpg_w_couple[b] : 0.f;
      F[b3::F_RAD * 32 + b] = sphere ? (float)hx : (float)std::sqrt(hx * hx + hy * hy + hz * hz);
      F[b3::F_GEOM * 32 + b] = sphere ? 1.f : 0.f;
    }
    const int off = (int)pairs.size();
    for (int a = 0; a < nb; ++a)
      for (int b = a + 1; b < nb; ++b) {
        if (d.parent[b] == a) continue;
        if (d.exclude && (((d.exclude[a] >> b) & 1u) || ((d.exclude[b] >> a) & 1u))) continue;
        pairs.push_back((uint16_t)((a << 8) | b));
      }
    meta[4 * k] = nb;
    meta[4 * k + 1] = maxdepth;
    meta[4 * k + 2] = (int)pairs.size() - off;
    meta[4 * k + 3] = off;
  }
  if (pairs.empty()) pairs.push_back(0);
}

}  // namespace b3
