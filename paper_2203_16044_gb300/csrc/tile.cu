// Shared-memory tile passes (multi-gate per HBM pass).
#include "planner.h"

struct qs_tile_pass {
  int dummy;
};

namespace qs {

qs_status plan_tiled(qs_plan* p) {
  (void)p;
  return fail(QS_EUNSUPPORTED, "tiled plans are not built yet");
}

qs_status plan_tiles_upload(qs_plan* p, cudaStream_t stream) {
  (void)p;
  (void)stream;
  return QS_OK;
}

qs_status run_tile(qs_state* s, qs_plan* p, int tile_index) {
  (void)s;
  (void)p;
  (void)tile_index;
  return fail(QS_EUNSUPPORTED, "tiled plans are not built yet");
}

void tile_free(qs_tile_pass* t) { delete t; }

}  // namespace qs
