// model_pack.h -- validation and structure-of-arrays packing of a robot
// population (host code shared by the GPU simulator and the CPU engine).
//
// Packed order: robots of up to SIM_WARP_MAX_BODIES bodies sorted by body
// count, largest first (stable), then the single free bodies with their
// centre at the frame origin, then the long chains (more than
// SIM_WARP_MAX_BODIES bodies), largest first.  The first two groups use the
// warp layout, per robot: float fields [NF][32 body slots], int fields
// [NI][32], meta (bodies, tree depth, pair count, pair offset) and the list of
// body/body candidate pairs (a < b, a not the parent of b, not excluded),
// each packed as (a << 8) | b.  Long chains use the chain layout: float
// fields [NF][64], int fields [CNI][64] (parent, axis, depth), 64-bit masks
// [2][64] (path to the root, children), meta and pairs as above.
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
  int n_free = 0;         // single free bodies (free_body.cuh), after the warp robots
  int n_chain = 0;        // long chains (chain layout), packed last
  std::vector<int> perm;  // packed index -> caller index
  std::vector<int> inv;   // caller index -> packed index
  // warp layout, packed robots [0, n - n_chain)
  std::vector<float> mf;
  std::vector<int> mi;
  std::vector<int> meta;  // 4 ints per robot: bodies, max depth, pair count, pair offset
  std::vector<uint16_t> pairs;
  // chain layout, packed robots [n - n_chain, n)
  std::vector<float> cmf;
  std::vector<int> cmi;
  std::vector<unsigned long long> cmask;
  std::vector<int> cmeta;
  std::vector<uint16_t> cpairs;
};

inline bool finite_all(const float* p, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Returns an empty string on success, else the reason the population is
// invalid.  max_bodies: the caller's body bound (at most SIM_MAX_BODIES).
inline std::string validate_population(const sim_variant_desc* v, int n, const char* who,
                                       int max_bodies = SIM_MAX_BODIES) {
  if (!v || n < 1) return std::string(who) + ": need n >= 1 variants";
  for (int i = 0; i < n; ++i) {
    const sim_variant_desc& d = v[i];
    const int nb = d.n_bodies;
    char buf[160];
    if (nb < 1 || nb > max_bodies) {
      snprintf(buf, sizeof buf, ": variant %d has %d bodies (1..%d)", i, nb, max_bodies);
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

// float fields of one robot into F ([NF][NS] body slots); slots >= n_bodies
// hold R = identity and zeros
inline void pack_body_fields(const sim_variant_desc& d, float* F, int NS) {
  const int nb = d.n_bodies;
  for (int b = 0; b < NS; ++b) {
    if (b >= nb) {
      F[(F_RFIX + 0) * NS + b] = 1.f;
      F[(F_RFIX + 4) * NS + b] = 1.f;
      F[(F_RFIX + 8) * NS + b] = 1.f;
      continue;
    }
    for (int t = 0; t < 9; ++t) F[(F_RFIX + t) * NS + b] = d.joint_frame[12 * b + t];
    for (int t = 0; t < 3; ++t) {
      F[(F_PFIX + t) * NS + b] = d.joint_frame[12 * b + 9 + t];
      F[(F_HALF + t) * NS + b] = d.half_size[3 * b + t];
      F[(F_COM + t) * NS + b] = d.box_center[3 * b + t];
    }
    const double m = d.mass[b];
    const double hx = d.half_size[3 * b], hy = d.half_size[3 * b + 1], hz = d.half_size[3 * b + 2];
    const bool sphere = d.geom && d.geom[b] == SIM_GEOM_SPHERE;
    F[F_MASS * NS + b] = d.mass[b];
    if (sphere) {  // solid sphere: 2 m r^2 / 5 about every axis
      for (int t = 0; t < 3; ++t) F[(F_ID + t) * NS + b] = (float)(0.4 * m * hx * hx);
    } else {       // solid box: m (h_j^2 + h_k^2) / 3
      F[(F_ID + 0) * NS + b] = (float)(m * (hy * hy + hz * hz) / 3.0);
      F[(F_ID + 1) * NS + b] = (float)(m * (hx * hx + hz * hz) / 3.0);
      F[(F_ID + 2) * NS + b] = (float)(m * (hx * hx + hy * hy) / 3.0);
    }
    F[F_WINT * NS + b] = d.cpg_w_internal ? d.cpg_w_internal[b] : 0.f;
    F[F_WCPL * NS + b] = d.cpg_w_couple ? d.cpg_w_couple[b] : 0.f;
    F[F_RAD * NS + b] = sphere ? (float)hx : (float)std::sqrt(hx * hx + hy * hy + hz * hz);
    F[F_GEOM * NS + b] = sphere ? 1.f : 0.f;
  }
}

// depth, path mask (bodies from the root to b, both included) and child mask
// of every body; returns the tree depth
inline int tree_masks(const sim_variant_desc& d, int* depth, unsigned long long* path, unsigned long long* child) {
  const int nb = d.n_bodies;
  int maxdepth = 0;
  for (int b = 0; b < nb; ++b) {
    depth[b] = 0;
    path[b] = 0ull;
    child[b] = 0ull;
  }
  for (int b = 0; b < nb; ++b) {
    const int p = b == 0 ? -1 : d.parent[b];
    depth[b] = p < 0 ? 0 : depth[p] + 1;
    path[b] = (p < 0 ? 0ull : path[p]) | (1ull << b);
    if (p >= 0) child[p] |= 1ull << b;
    maxdepth = std::max(maxdepth, depth[b]);
  }
  return maxdepth;
}

// body/body candidate pairs of one robot appended to `pairs`; returns their count
inline int append_pairs(const sim_variant_desc& d, std::vector<uint16_t>& pairs) {
  const int nb = d.n_bodies;
  const int off = (int)pairs.size();
  for (int a = 0; a < nb; ++a)
    for (int b = a + 1; b < nb; ++b) {
      if (d.parent[b] == a) continue;
      if (d.exclude && (((d.exclude[a] >> b) & 1ull) || ((d.exclude[b] >> a) & 1ull))) continue;
      pairs.push_back((uint16_t)((a << 8) | b));
    }
  return (int)pairs.size() - off;
}

inline void pack_population(const sim_variant_desc* v, int n, PackedPopulation& out) {
  // group 0: warp robots, 1: single free bodies (one-body step), 2: long chains
  auto is_free = [&](int i) {
    return v[i].n_bodies == 1 && v[i].box_center[0] == 0.f && v[i].box_center[1] == 0.f &&
           v[i].box_center[2] == 0.f;
  };
  auto group = [&](int i) { return v[i].n_bodies > SIM_WARP_MAX_BODIES ? 2 : (is_free(i) ? 1 : 0); };
  std::vector<int>& perm = out.perm;
  perm.resize(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
    if (group(a) != group(b)) return group(a) < group(b);
    return v[a].n_bodies > v[b].n_bodies;
  });
  out.n_free = 0;
  out.n_chain = 0;
  for (int i = 0; i < n; ++i) {
    out.n_free += group(i) == 1 ? 1 : 0;
    out.n_chain += group(i) == 2 ? 1 : 0;
  }
  const int n_short = n - out.n_chain;
  std::vector<int>& inv = out.inv;
  inv.assign(n, 0);
  for (int k = 0; k < n; ++k) inv[perm[k]] = k;

  // warp layout
  out.mf.assign((size_t)n_short * NF * 32, 0.f);
  out.mi.assign((size_t)n_short * NI * 32, 0);
  out.meta.assign((size_t)4 * n_short, 0);
  out.pairs.clear();
  for (int k = 0; k < n_short; ++k) {
    const sim_variant_desc& d = v[perm[k]];
    const int nb = d.n_bodies;
    float* F = out.mf.data() + (size_t)k * NF * 32;
    int* I = out.mi.data() + (size_t)k * NI * 32;
    int depth[SIM_MAX_BODIES];
    unsigned long long path[SIM_MAX_BODIES], child[SIM_MAX_BODIES];
    const int maxdepth = tree_masks(d, depth, path, child);
    for (int b = 0; b < 32; ++b) {
      I[I_PARENT * 32 + b] = b < nb ? (b == 0 ? -1 : d.parent[b]) : -1;
      I[I_AXIS * 32 + b] = b < nb ? d.hinge_axis[b] : 0;
      I[I_PATH * 32 + b] = (int)(unsigned)(b < nb ? path[b] : 0ull);
      I[I_CHILD * 32 + b] = (int)(unsigned)(b < nb ? child[b] : 0ull);
      I[I_DEPTH * 32 + b] = b < nb ? depth[b] : 0;
    }
    pack_body_fields(d, F, 32);
    const int off = (int)out.pairs.size();
    out.meta[4 * k] = nb;
    out.meta[4 * k + 1] = maxdepth;
    out.meta[4 * k + 2] = append_pairs(d, out.pairs);
    out.meta[4 * k + 3] = off;
  }
  if (out.pairs.empty()) out.pairs.push_back(0);

  // chain layout
  const int nch = out.n_chain;
  constexpr int NS = kChainSlots;
  out.cmf.assign((size_t)nch * NF * NS, 0.f);
  out.cmi.assign((size_t)nch * CNI * NS, 0);
  out.cmask.assign((size_t)nch * CNM * NS, 0ull);
  out.cmeta.assign((size_t)4 * nch, 0);
  out.cpairs.clear();
  for (int c = 0; c < nch; ++c) {
    const sim_variant_desc& d = v[perm[n_short + c]];
    const int nb = d.n_bodies;
    float* F = out.cmf.data() + (size_t)c * NF * NS;
    int* I = out.cmi.data() + (size_t)c * CNI * NS;
    unsigned long long* Mk = out.cmask.data() + (size_t)c * CNM * NS;
    int depth[SIM_MAX_BODIES];
    unsigned long long path[SIM_MAX_BODIES], child[SIM_MAX_BODIES];
    const int maxdepth = tree_masks(d, depth, path, child);
    for (int b = 0; b < NS; ++b) {
      I[CI_PARENT * NS + b] = b < nb ? (b == 0 ? -1 : d.parent[b]) : -1;
      I[CI_AXIS * NS + b] = b < nb ? d.hinge_axis[b] : 0;
      I[CI_DEPTH * NS + b] = b < nb ? depth[b] : 0;
      Mk[CM_PATH * NS + b] = b < nb ? path[b] : 0ull;
      Mk[CM_CHILD * NS + b] = b < nb ? child[b] : 0ull;
    }
    pack_body_fields(d, F, NS);
    const int off = (int)out.cpairs.size();
    out.cmeta[4 * c] = nb;
    out.cmeta[4 * c + 1] = maxdepth;
    out.cmeta[4 * c + 2] = append_pairs(d, out.cpairs);
    out.cmeta[4 * c + 3] = off;
  }
  if (out.cpairs.empty()) out.cpairs.push_back(0);
}

}  // namespace b3
