// Autotuning of plan shapes, with a cache that can persist across processes.
//
// A plan's speed depends on the circuit, the qubit count, the dtype and the
// GPU: dense-block width k (4, 5, 6 for complex64; 4, 5 for complex128)
// trades the number of HBM passes against arithmetic per pass, and tile
// passes trade their width and register-slot shape against occupancy.  The
// tuners time candidates on the caller's own state (or batch) and keep the
// fastest (a candidate whose first run is already 1.5x slower than the best
// so far is not run again).  Results are keyed by a 64-bit FNV-1a hash of everything that
// determines the plan -- every gate (kind, qubits, angle bits, parameter
// index), the qubit count(s), the dtype -- and of the GPU (name, SM count,
// compute capability), kept in memory for the process and, when a cache
// file is set, appended to it as one text line per result:
//   qs-tune-v3 <key hex> <what> <mode> <tile> <low> <slots> <gpt> <dense> <fuse> <search> <fuse_min> <ms>
// where <what> is "plan" or "batch".  A file written on another GPU never
// matches (the key covers the device).  Timing runs overwrite the state.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qs_internal.h"

namespace qs {
namespace {

struct TuneRec {
  qs_plan_opts opts;
  double ms;
};

std::mutex g_tune_mu;
std::map<unsigned long long, TuneRec> g_tune;  // key -> best
std::string g_tune_file;

struct Fnv {
  unsigned long long h = 1469598103934665603ull;
  void bytes(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  }
  template <typename T>
  void val(const T& v) {
    bytes(&v, sizeof(v));
  }
};

void hash_circuit(Fnv& f, const qs_circuit* c) {
  const unsigned long long ng = c ? c->gates.size() : 0;
  f.val(ng);
  if (!c) return;
  for (const qs_gate_rec& g : c->gates) {
    f.val(g.kind);
    f.val(g.q[0]);
    f.val(g.q[1]);
    f.bytes(g.p, sizeof(g.p));  // the angles' bit patterns
    f.val(g.param_index);
  }
}

qs_status hash_device(Fnv& f) {
  int dev = 0;
  cudaDeviceProp pr;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&pr, dev);
  if (e != cudaSuccess) return cuda_fail(e, "autotune: device properties");
  f.bytes(pr.name, strnlen(pr.name, sizeof(pr.name)));
  f.val(pr.multiProcessorCount);
  f.val(pr.major);
  f.val(pr.minor);
  return QS_OK;
}

bool lookup(unsigned long long key, qs_plan_opts* best, double* best_ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *best = it->second.opts;
  if (best_ms) *best_ms = it->second.ms;
  return true;
}

void remember(unsigned long long key, const char* what, const qs_plan_opts& o, double ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = TuneRec{o, ms};
  if (g_tune_file.empty()) return;
  FILE* fp = std::fopen(g_tune_file.c_str(), "a");
  if (!fp) return;  // the cache is an optimisation: an unwritable file only loses persistence
  std::fprintf(fp, "qs-tune-v3 %016llx %s %d %d %d %d %d %d %d %d %d %.6f\n", key, what, o.mode, o.tile_qubits,
               o.low_qubits, o.slot_qubits, o.groups_per_thread, o.dense, o.fuse_qubits, o.search, o.fuse_min_qubits, ms);
  std::fclose(fp);
}

// Times `plan` on `st` (CUDA events on the state's stream; the state is
// overwritten): a first run, and when that one is not already slower than
// `prune_ms`, a second run whose time is returned (the first also pays for
// one-time set-up); otherwise the first run's time.
qs_status time_plan(qs_state* st, qs_plan* plan, double prune_ms, float* ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return cuda_fail(e, "autotune: event");
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(e, "autotune: event");
  }
  qs_status r = QS_OK;
  for (int rep = 0; rep < 2 && r == QS_OK; ++rep) {
    cudaEventRecord(e0, st->stream);
    r = qs_run_plan(st, plan);
    cudaEventRecord(e1, st->stream);
    if (r == QS_OK) r = qs_sync(st);
    if (r == QS_OK) {
      e = cudaEventElapsedTime(ms, e0, e1);
      if (e != cudaSuccess) r = cuda_fail(e, "autotune: elapsed time");
    }
    if (rep == 0 && r == QS_OK && *ms > prune_ms) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}

}  // namespace

unsigned long long batch_tune_key(int count, const int* nq, qs_dtype dtype, const qs_circuit* const* circuits,
                                  qs_status* st) {
  Fnv f;
  const char tag[] = "batch";
  f.bytes(tag, sizeof(tag));
  f.val((int)dtype);
  f.val(count);
  for (int i = 0; i < count; ++i) {
    f.val(nq[i]);
    hash_circuit(f, circuits[i]);
  }
  *st = hash_device(f);
  return f.h;
}

bool batch_tune_lookup(unsigned long long key, qs_plan_opts* best, double* best_ms) {
  return lookup(key, best, best_ms);
}

void batch_tune_remember(unsigned long long key, const qs_plan_opts& o, double ms) { remember(key, "batch", o, ms); }

}  // namespace qs

using namespace qs;

extern "C" {

qs_status qs_circuit_hash(const qs_circuit* c, int n, qs_dtype dtype, uint64_t* out) {
  if (!c || !out) return fail(QS_EINVAL, "qs_circuit_hash: NULL argument");
  Fnv f;
  const char tag[] = "plan";
  f.bytes(tag, sizeof(tag));
  f.val(n);
  f.val((int)dtype);
  hash_circuit(f, c);
  *out = f.h;
  return QS_OK;
}

qs_status qs_tune_cache_file(const char* path) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  g_tune_file = path ? path : "";
  if (!path) return QS_OK;
  FILE* fp = std::fopen(path, "r");
  if (!fp) return QS_OK;  // created on the first result
  char line[512];
  while (std::fgets(line, sizeof(line), fp)) {
    unsigned long long key = 0;
    char what[16];
    qs_plan_opts o{};
    double ms = 0.0;
    if (std::sscanf(line, "qs-tune-v3 %llx %15s %d %d %d %d %d %d %d %d %d %lf", &key, what, &o.mode, &o.tile_qubits,
                    &o.low_qubits, &o.slot_qubits, &o.groups_per_thread, &o.dense, &o.fuse_qubits, &o.search,
                    &o.fuse_min_qubits, &ms) == 12)
      g_tune[key] = TuneRec{o, ms};  // a later line for the same key wins
  }
  std::fclose(fp);
  return QS_OK;
}

qs_status qs_plan_autotune(const qs_circuit* c, qs_state* st, qs_plan_opts* best, double* best_ms) {
  if (!c || !st || !best) return fail(QS_EINVAL, "qs_plan_autotune: NULL argument");
  uint64_t ch = 0;
  qs_status r = qs_circuit_hash(c, st->n, st->dtype, &ch);
  if (r != QS_OK) return r;
  Fnv f;
  f.val(ch);
  if ((r = hash_device(f)) != QS_OK) return r;
  const unsigned long long key = f.h;
  if (lookup(key, best, best_ms)) return QS_OK;
  std::vector<qs_plan_opts> cands;
  const int kmax = st->dtype == QS_C64 ? 6 : 5;
  for (int k = 4; k <= kmax && k <= st->n; ++k) {
    qs_plan_opts o{};
    o.mode = QS_PLAN_FUSED;
    o.fuse_qubits = k;
    cands.push_back(o);
  }
  const int tiles[][3] = {{12, 3, 1}, {13, 3, 1}, {13, 4, 1}, {14, 3, 1}, {13, 3, 2}};
  for (const auto& t : tiles) {
    if (st->dtype == QS_C128 && (t[0] > 13 || t[2] == 2)) continue;
    qs_plan_opts o{};
    o.mode = QS_PLAN_TILED;
    o.tile_qubits = t[0];
    o.slot_qubits = t[1];
    o.groups_per_thread = t[2];
    cands.push_back(o);
  }
  double bestt = 1e300;
  qs_plan_opts bo{};
  bool any = false;
  for (const qs_plan_opts& o : cands) {
    qs_plan* p = nullptr;
    if (qs_plan_build(c, st->n, st->dtype, &o, &p) != QS_OK) continue;  // a shape this circuit cannot take
    float ms = 0.f;
    r = time_plan(st, p, 1.5 * bestt, &ms);
    qs_plan_destroy(p);
    if (r != QS_OK) return r;
    if (ms < bestt) {
      bestt = ms;
      bo = o;
      any = true;
    }
  }
  if (!any) return fail(QS_EUNSUPPORTED, "qs_plan_autotune: no candidate plan could be built");
  remember(key, "plan", bo, bestt);
  *best = bo;
  if (best_ms) *best_ms = bestt;
  return QS_OK;
}

}  // extern "C"
