// Plan policies that move qubits rather than gather them (§III-D).
//
// The paper's distributed simulator can apply a gate only to "local"
// qubits, those inside a process's slice (§III-B).  Two ways to make a
// global qubit local are compared there: swap gates inserted in front of
// the gates that need them (as Qiskit Aer does), each one exchange of half
// the vector, and the fused swap of Listing 1, which exchanges s disjoint
// qubit pairs at once and moves a fraction 1 - 2^-s of the vector.  On one
// GPU the "local" qubits are those a tile pass holds in shared memory; here
// they are the m lowest physical qubits, every tile pass holds exactly
// those (contiguous runs of 2^m amplitudes), and a bit-pair exchange pass in
// HBM (run_bitswap) brings a gate's target in:
//   QS_PLAN_SWAP     one pass per target that is not local, exchanging it
//                    with the local qubit needed furthest in the future
//                    (Belady's rule);
//   QS_PLAN_PERMUTE  one pass per routing point, exchanging every target
//                    that the coming gates need -- as many gates ahead as
//                    fit m distinct targets -- with local qubits not needed
//                    by them (the fused swap: up to m pairs in one pass).
// Gates between routing points are tiled over the m local qubits (their
// controls and phase bits may lie anywhere).  A SWAP gate of the circuit
// costs nothing: it only relabels which physical qubit holds which logical
// one.  The logical -> physical map is undone at the end by at most two
// exchange passes, so the result is in logical order, as the paper requires
// of its fused-swap insertion (§IV-D, §IV-F).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "planner.h"

namespace qs {

std::vector<std::vector<std::pair<int, int>>> permutation_passes(const std::vector<int>& perm, int cap) {
  // Every cycle c_0 -> c_1 -> ... -> c_{m-1} (perm[c_i] = c_{i+1}) is the
  // product of two reflections, r1(i) = -i and then r2(i) = 1 - i (mod m);
  // each reflection exchanges disjoint pairs.
  const int n = (int)perm.size();
  std::vector<std::pair<int, int>> r1, r2;
  std::vector<char> done(n, 0);
  for (int j = 0; j < n; ++j) {
    if (done[j]) continue;
    std::vector<int> cyc;
    for (int c = j; !done[c]; c = perm[c]) {
      done[c] = 1;
      cyc.push_back(c);
    }
    const int m = (int)cyc.size();
    for (int i = 0; i < m; ++i) {
      const int i1 = (m - i) % m;
      if (i < i1) r1.push_back({cyc[i], cyc[i1]});
      const int i2 = ((1 - i) % m + m) % m;
      if (i < i2) r2.push_back({cyc[i], cyc[i2]});
    }
  }
  std::vector<std::vector<std::pair<int, int>>> out;
  for (const auto* r : {&r1, &r2})
    for (size_t o = 0; o < r->size(); o += (size_t)cap)
      out.emplace_back(r->begin() + o, r->begin() + std::min(r->size(), o + (size_t)cap));
  return out;
}

qs_status plan_routed(qs_plan* p, bool fused) {
  const int n = p->n;
  if (n < 4) {  // too small for a tile: per-gate passes
    for (const qs_gate_rec& g : p->gates) p->steps.push_back(unfused_step(g));
    return QS_OK;
  }
  int m = 0, L = 0, G = 0;
  qs_status st = tile_options(p, &m, &L, &G);
  if (st != QS_OK) return st;
  const size_t NG = p->gates.size();
  // per logical qubit, the gates that need it as a tile target, ascending
  std::vector<std::vector<size_t>> uses(n);
  for (size_t i = 0; i < NG; ++i) {
    int tq[2];
    const int nt = tile_targets(p->gates[i], tq);
    for (int j = 0; j < nt; ++j) uses[tq[j]].push_back(i);
  }
  auto next_use = [&](int q, size_t i) {
    const auto it = std::lower_bound(uses[q].begin(), uses[q].end(), i);
    return it == uses[q].end() ? SIZE_MAX : *it;
  };
  std::vector<int> phys(n), logi(n);  // logical -> physical and back
  for (int q = 0; q < n; ++q) phys[q] = logi[q] = q;
  std::vector<qs_gate_rec> seg;  // gates since the last routing point, on physical qubits
  auto flush = [&]() -> qs_status {
    if (seg.empty()) return QS_OK;
    std::vector<const qs_gate_rec*> ptrs;
    for (const qs_gate_rec& g : seg) ptrs.push_back(&g);
    const qs_status r = tile_gates(p, ptrs, m, m, G);
    seg.clear();
    return r;
  };
  auto exchange = [&](const std::vector<std::pair<int, int>>& pairs) {
    if (pairs.empty()) return;
    p->exchanges.push_back(pairs);
    qs_step s{};
    s.type = qs_step::EXCHANGE;
    s.nq = (int)pairs.size();
    s.tile_index = (int)p->exchanges.size() - 1;
    p->steps.push_back(s);
    for (const auto& pr : pairs) {
      std::swap(logi[pr.first], logi[pr.second]);
      phys[logi[pr.first]] = pr.first;
      phys[logi[pr.second]] = pr.second;
    }
  };
  for (size_t i = 0; i < NG; ++i) {
    const qs_gate_rec& g = p->gates[i];
    if (g.kind == QS_GATE_SWAP) {  // a relabelling, no data moves
      std::swap(phys[g.q[0]], phys[g.q[1]]);
      logi[phys[g.q[0]]] = g.q[0];
      logi[phys[g.q[1]]] = g.q[1];
      continue;
    }
    int tq[2];
    const int nt = tile_targets(g, tq);
    bool remote = false;
    for (int j = 0; j < nt; ++j) remote |= phys[tq[j]] >= m;
    if (remote) {
      if ((st = flush()) != QS_OK) return st;
      if (!fused) {
        for (int j = 0; j < nt; ++j) {
          if (phys[tq[j]] < m) continue;
          int best = -1;
          size_t bu = 0;
          for (int s = 0; s < m; ++s) {
            const int lq = logi[s];
            if (lq == tq[0] || (nt > 1 && lq == tq[1])) continue;
            const size_t u = next_use(lq, i);
            if (best < 0 || u > bu) {
              best = s;
              bu = u;
            }
          }
          exchange({{phys[tq[j]], best}});
        }
      } else {
        // the targets of gates i, i+1, ... while at most m distinct ones
        std::vector<char> need(n, 0);
        int cnt = 0;
        for (size_t j = i; j < NG; ++j) {
          if (p->gates[j].kind == QS_GATE_SWAP) break;  // relabels: look no further
          int q2[2];
          const int k2 = tile_targets(p->gates[j], q2);
          int add = 0;
          for (int t = 0; t < k2; ++t) add += !need[q2[t]] && (t == 0 || q2[1] != q2[0]);
          if (cnt + add > m) break;
          for (int t = 0; t < k2; ++t) need[q2[t]] = 1;
          cnt += add;
        }
        std::vector<int> in, slots;
        for (int q = 0; q < n; ++q)
          if (need[q] && phys[q] >= m) in.push_back(phys[q]);
        for (int s = 0; s < m; ++s)
          if (!need[logi[s]]) slots.push_back(s);
        std::stable_sort(slots.begin(), slots.end(),
                         [&](int x, int y) { return next_use(logi[x], i) > next_use(logi[y], i); });
        std::vector<std::pair<int, int>> pairs;
        for (size_t k = 0; k < in.size(); ++k) pairs.push_back({in[k], slots[k]});
        for (size_t o = 0; o < pairs.size(); o += 17)
          exchange(std::vector<std::pair<int, int>>(pairs.begin() + o,
                                                    pairs.begin() + std::min(pairs.size(), o + 17)));
      }
    }
    qs_gate_rec r = g;
    r.q[0] = phys[g.q[0]];
    if (gate_arity(g.kind) == 2) r.q[1] = phys[g.q[1]];
    seg.push_back(r);
  }
  if ((st = flush()) != QS_OK) return st;
  // back to logical order: the bit at physical position x belongs at logi[x]
  for (const auto& pass : permutation_passes(logi, 17)) exchange(pass);
  return QS_OK;
}

}  // namespace qs
