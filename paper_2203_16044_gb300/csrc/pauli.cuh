// Pauli strings grouped by their X/Y mask.
//
// P|x> = i^{nY} (-1)^{popcount(x & z)} |x ^ m>  (m = X/Y positions, z = Z/Y
// positions, nY = popcount(m & z)), so terms sharing m act together:
//   (sum_t c_t P_t psi)_x = f(x ^ m) psi_{x ^ m},
//   f(y) = sum_t c_t i^{nY_t} (-1)^{popcount(y & z_t)}.
#pragma once

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "dfloat.cuh"
#include "kcommon.cuh"

namespace qs {

constexpr int kMaxGroupTerms = 64;
constexpr int kMaxClasses = 8;
struct PauliGroup {
  u64 m;           // X/Y mask shared by the group
  int h;           // highest bit of m (-1 if m == 0)
  int nt;          // terms in this launch
  u64 z[kMaxGroupTerms];
  // w_t = c_t * i^{nY_t} in double-float: real (h, l) and imaginary (h, l)
  float wrh[kMaxGroupTerms], wrl[kMaxGroupTerms], wih[kMaxGroupTerms], wil[kMaxGroupTerms];
  // Z-only groups whose terms each have two Z bits, i apart from j = i + d:
  // terms of equal d and weight form a class, and popcount(x & z_t) is odd
  // exactly when bit i of x ^ (x >> d) is set, so a class of len terms gives
  // w (len - 2 popcount((x ^ (x >> d)) & mask)), mask = the terms' lower
  // bits.  ncls = 0: the term list is used.
  int ncls;
  int cls_d[kMaxClasses], cls_len[kMaxClasses];
  u64 cls_mask[kMaxClasses];
  float cwrh[kMaxClasses], cwrl[kMaxClasses], cwih[kMaxClasses], cwil[kMaxClasses];
};

// f(x) in double-float.  The host sorts a group's terms by weight, so equal
// weights form runs: a run of len terms with weight w contributes
// w (len - 2 odd), odd = the number of its terms with popcount(x & z_t) odd,
// counted with integer operations; one double-float product per run.
__device__ __forceinline__ void fval_df(const PauliGroup& g, u64 x, dfl& fr, dfl& fi) {
  fr = dfl{0.f, 0.f};
  fi = dfl{0.f, 0.f};
  if (g.ncls > 0) {
    for (int c = 0; c < g.ncls; ++c) {
      const dfl k{(float)(g.cls_len[c] - 2 * __popcll((x ^ (x >> g.cls_d[c])) & g.cls_mask[c])), 0.f};
      df_acc(fr, df_mul(dfl{g.cwrh[c], g.cwrl[c]}, k));
      df_acc(fi, df_mul(dfl{g.cwih[c], g.cwil[c]}, k));
    }
    return;
  }
  int len = 0, odd = 0;
  for (int t = 0; t < g.nt; ++t) {
    odd += __popcll(x & g.z[t]) & 1;
    ++len;
    const bool last = t + 1 == g.nt || g.wrh[t + 1] != g.wrh[t] || g.wrl[t + 1] != g.wrl[t] ||
                      g.wih[t + 1] != g.wih[t] || g.wil[t + 1] != g.wil[t];
    if (last) {
      const dfl k{(float)(len - 2 * odd), 0.f};  // exact: |k| <= 64
      df_acc(fr, df_mul(dfl{g.wrh[t], g.wrl[t]}, k));
      df_acc(fi, df_mul(dfl{g.wih[t], g.wil[t]}, k));
      len = 0;
      odd = 0;
    }
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
    const double wr = coeff[t] * pr[ny], wi = coeff[t] * pim[ny];
    g.z[g.nt] = z;
    g.wrh[g.nt] = (float)wr;
    g.wrl[g.nt] = (float)(wr - (double)g.wrh[g.nt]);
    g.wih[g.nt] = (float)wi;
    g.wil[g.nt] = (float)(wi - (double)g.wih[g.nt]);
    ++g.nt;
  }
  // terms of equal weight next to each other (fval_df counts them as a run)
  for (PauliGroup& g : groups) {
    std::vector<int> ord(g.nt);
    for (int i = 0; i < g.nt; ++i) ord[i] = i;
    auto key = [&](int i) { return std::make_tuple(g.wrh[i], g.wrl[i], g.wih[i], g.wil[i]); };
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return key(a) < key(b); });
    PauliGroup s = g;
    for (int i = 0; i < g.nt; ++i) {
      s.z[i] = g.z[ord[i]];
      s.wrh[i] = g.wrh[ord[i]];
      s.wrl[i] = g.wrl[ord[i]];
      s.wih[i] = g.wih[ord[i]];
      s.wil[i] = g.wil[ord[i]];
    }
    g = s;
  }
  // Z-only groups of two-bit terms: classes by (bit distance, weight)
  for (PauliGroup& g : groups) {
    g.ncls = 0;
    if (g.m != 0) continue;
    bool ok = true;
    for (int t = 0; t < g.nt && ok; ++t) {
      if (__builtin_popcountll(g.z[t]) != 2) { ok = false; break; }
      const int i = __builtin_ctzll(g.z[t]), j = 63 - __builtin_clzll(g.z[t]), d = j - i;
      int c = 0;
      for (; c < g.ncls; ++c)
        if (g.cls_d[c] == d && g.cwrh[c] == g.wrh[t] && g.cwrl[c] == g.wrl[t] && g.cwih[c] == g.wih[t] &&
            g.cwil[c] == g.wil[t])
          break;
      if (c == g.ncls) {
        if (g.ncls == kMaxClasses) { ok = false; break; }
        g.cls_d[c] = d;
        g.cls_len[c] = 0;
        g.cls_mask[c] = 0;
        g.cwrh[c] = g.wrh[t];
        g.cwrl[c] = g.wrl[t];
        g.cwih[c] = g.wih[t];
        g.cwil[c] = g.wil[t];
        ++g.ncls;
      }
      if ((g.cls_mask[c] >> i) & 1) { ok = false; break; }  // a repeated term: keep the list
      g.cls_mask[c] |= u64(1) << i;
      ++g.cls_len[c];
    }
    if (!ok) g.ncls = 0;
  }
  return groups;
}

}  // namespace qs
