// Pauli strings grouped by their X/Y mask.
//
// P|x> = i^{nY} (-1)^{popcount(x & z)} |x ^ m>  (m = X/Y positions, z = Z/Y
// positions, nY = popcount(m & z)), so terms sharing m act together:
//   (sum_t c_t P_t psi)_x = f(x ^ m) psi_{x ^ m},
//   f(y) = sum_t c_t i^{nY_t} (-1)^{popcount(y & z_t)}.
#pragma once

#include <map>
#include <vector>

#include "kcommon.cuh"

namespace qs {

constexpr int kMaxGroupTerms = 64;
struct PauliGroup {
  u64 m;           // X/Y mask shared by the group
  int h;           // highest bit of m (-1 if m == 0)
  int nt;          // terms in this launch
  u64 z[kMaxGroupTerms];
  double wr[kMaxGroupTerms], wi[kMaxGroupTerms];  // c_t * i^{nY_t}
};

__device__ __forceinline__ void fval(const PauliGroup& g, u64 x, double& fr, double& fi) {
  fr = 0.0; fi = 0.0;
  for (int t = 0; t < g.nt; ++t) {
    const double sgn = (__popcll(x & g.z[t]) & 1) ? -1.0 : 1.0;
    fr += sgn * g.wr[t];
    fi += sgn * g.wi[t];
  }
}


// Group terms by X/Y mask in order of first appearance (deterministic), at
// most kMaxGroupTerms per group.
inline std::vector<PauliGroup> build_pauli_groups(int nterms, const u64* xmask, const u64* zmask,
                                                  const double* coeff) {
  std::vector<PauliGroup> groups;
  std::map<u64, int> idx;
  for (int t = 0; t < nterms; ++t) {
    const u64 m = xmask[t], z = zmask[t];
    auto it = idx.find(m);
    int gi;
    if (it == idx.end() || groups[it->second].nt == kMaxGroupTerms) {
      PauliGroup g{};
      g.m = m;
      g.h = m ? 63 - __builtin_clzll(m) : -1;
      g.nt = 0;
      groups.push_back(g);
      gi = (int)groups.size() - 1;
      idx[m] = gi;
    } else {
      gi = it->second;
    }
    PauliGroup& g = groups[gi];
    const int ny = __builtin_popcountll(m & z) & 3;  // i^{nY}
    const double pr[4] = {1, 0, -1, 0}, pim[4] = {0, 1, 0, -1};
    g.z[g.nt] = z;
    g.wr[g.nt] = coeff[t] * pr[ny];
    g.wi[g.nt] = coeff[t] * pim[ny];
    ++g.nt;
  }
  return groups;
}

}  // namespace qs
