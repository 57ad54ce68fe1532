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
}  // namespace qs
