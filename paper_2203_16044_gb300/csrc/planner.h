// Planner internals shared by planner.cpp and tile.cu.
#pragma once
#include "qs_internal.h"

namespace qs {
double step_bytes(const qs_step& st, int n, int S);
qs_step unfused_step(const qs_gate_rec& g);
qs_status run_step(qs_state* s, qs_plan* p, const qs_step& st);
qs_status run_step_dfl(qs_state* s, qs_plan* p, const qs_step& st);
qs_status run_all_steps(qs_state* s, qs_plan* p, cudaEvent_t* ev);
// Fills p->steps (and p->tiles) for QS_PLAN_TILED.
qs_status plan_tiled(qs_plan* p);
// Fills p->steps (and p->blocks) for QS_PLAN_FUSED.
qs_status plan_fused(qs_plan* p);
// Register stages summed over the plan's tile passes.
int tile_stage_count(const qs_plan* p, int* dense);
// Tile options of a plan (tile qubits m, low qubits L, slot qubits G),
// validated with defaults filled in; needs n >= 4.
qs_status tile_options(qs_plan* p, int* m, int* L, int* G);
// Tile passes (L low + up to m - L chosen qubits each) for a gate list,
// appended to p->steps.
qs_status tile_gates(qs_plan* p, std::vector<const qs_gate_rec*> gates, int m, int L, int G);
// The qubits a gate needs inside a tile (its targets); returns their count.
int tile_targets(const qs_gate_rec& g, int* q);
// Fills p->steps for QS_PLAN_SWAP (fused = false) and QS_PLAN_PERMUTE
// (fused = true): tile passes over the lowest qubits, with bit-exchange
// passes bringing gate targets into them (route.cpp).
qs_status plan_routed(qs_plan* p, bool fused);
// A qubit permutation (bit j of an index moves to bit perm[j]) as at most
// two passes of disjoint bit-pair exchanges, each split into passes of at
// most `cap` pairs.
std::vector<std::vector<std::pair<int, int>>> permutation_passes(const std::vector<int>& perm, int cap);
}  // namespace qs
