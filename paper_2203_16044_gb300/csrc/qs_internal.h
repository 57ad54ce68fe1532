// Internal declarations of libqs (not installed; the public ABI is qs.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qs.h"

typedef uint64_t u64;

struct qs_state {
  int n = 0;
  qs_dtype dtype = QS_C128;
  void* amp = nullptr;          // 2^n amplitudes, interleaved (re, im)
  bool owns = false;            // allocated by qs_alloc
  cudaStream_t stream = nullptr;
  int device = 0;
  void* scratch = nullptr;      // reduction partials, plan tables
  size_t scratch_bytes = 0;
  double* pinned = nullptr;     // small pinned host buffer for results
  int tiles_per_cta = 1;        // block kernels: at least this many tiles per CTA (batched small states)
};

namespace qs {

// ---- errors ---------------------------------------------------------------
qs_status fail(qs_status code, const char* fmt, ...);
qs_status cuda_fail(cudaError_t e, const char* what);
// Check for a launch error after enqueueing kernels.
qs_status launch_ok(const char* what);

inline int amp_bytes(qs_dtype d) { return d == QS_C64 ? 8 : 16; }
inline u64 state_bytes(const qs_state* s) { return (u64(1) << s->n) * amp_bytes(s->dtype); }

// Grows the state's device scratch buffer to at least `bytes` (stream-ordered).
qs_status ensure_scratch(qs_state* s, size_t bytes);

// SM count of the current device (cached).
int sm_count();

// ---- host-side gate matrices (gatemat.cpp) ---------------------------------
// Writes the 2x2 (nq = 1) or 4x4 (nq = 2) matrix of a named gate; returns nq
// or -1 for an unknown kind.  Bit 0 of a 4x4 index = qubits[0].
int gate_matrix(int kind, const double* params, double* out);
int gate_arity(int kind);
int gate_nparams(int kind);
bool gate_is_diagonal(int kind);

// ---- kernels (gates.cu) ----------------------------------------------------
qs_status run_1q(qs_state* s, int q, const double U[8]);
qs_status run_controlled(qs_state* s, const int* ctrl, int nc, int t, const double U[8]);
qs_status run_diag(qs_state* s, const int* qubits, int k, const double* d);
// unitary: 1 known unitary, 0 not, -1 check (tensor-core path restores group norms)
qs_status run_dense(qs_state* s, const int* qubits, int k, const double* M, int unitary = -1);
// complex64 dense block, 4 <= k <= 6, on the tensor cores (fused_tc.cu)
qs_status run_dense_tc(qs_state* s, const int* qubits, int k, const double* M, int unitary);
qs_status tc_prepare(const int* qubits, int k, const double* M, int* q_sorted, std::vector<float>& B);
qs_status run_dense_tc_prepared(qs_state* s, const int* q_sorted, int k, const float* Bdev, int unitary);
qs_status fused_tc_status();  // QS_ETIMEOUT if a tensor-core wait gave up since the last call
// complex128 dense block, k = 4, 5, on the tensor cores (fused_c128.cu): FP64
// operands split into five 9-bit integer digits, exact FP16 digit products
qs_status run_dense_tc128(qs_state* s, const int* qubits, int k, const double* M);
qs_status tc128_prepare(const int* qubits, int k, const double* M, int* q_sorted, std::vector<uint16_t>& dig,
                        int* F);
qs_status run_dense_tc128_prepared(qs_state* s, const int* q_sorted, int k, const void* Bdig, int F, bool dfl);
qs_status fused_c128_status();
// In-place exchange of disjoint bit pairs (a[i], b[i]), i < npairs.
qs_status run_bitswap(qs_state* s, const int* a, const int* b, int npairs);
qs_status run_set_basis(qs_state* s, u64 x);
// complex128 double-float storage: in-place layout change and the gates on it
qs_status run_layout_dfl(qs_state* s, bool to_dfl);
qs_status run_controlled_dfl(qs_state* s, const int* ctrl, int nc, int t, const double U[8]);
qs_status run_diag_dfl(qs_state* s, const int* qubits, int k, const double* d);

// ---- autotuning cache (tune.cpp) -------------------------------------------
unsigned long long batch_tune_key(int count, const int* nq, qs_dtype dtype, const qs_circuit* const* circuits,
                                  qs_status* st);
bool batch_tune_lookup(unsigned long long key, qs_plan_opts* best, double* best_ms);
void batch_tune_remember(unsigned long long key, const qs_plan_opts& o, double ms);

// ---- reductions (reduce.cu) ------------------------------------------------
qs_status run_norm2(qs_state* s, double* out);
qs_status run_inner(qs_state* a, qs_state* b, double out[2]);
qs_status run_expect(qs_state* s, int nterms, const u64* xmask, const u64* zmask,
                     const double* coeff, double* out);
qs_status expect_pauli_passes(int n, int dtype, int nterms, const u64* xmask, const u64* zmask, int* passes);

}  // namespace qs

// ---- circuits and plans (planner.cpp / tile.cu) -----------------------------
struct qs_gate_rec {
  int kind;
  int q[2];
  double p[3];
  int param_index;
};

struct qs_circuit {
  std::vector<qs_gate_rec> gates;
};

// One step of a compiled plan.
struct qs_step {
  enum Type { GATE_1Q, GATE_CTRL, GATE_DIAG, GATE_SWAP, TILE, BLOCK, EXCHANGE } type;
  int q[4];
  int nq;
  double m[32];         // matrix / diagonal (FP64)
  int tile_index;       // TILE: index into plan->tiles; BLOCK: into plan->blocks;
                        // EXCHANGE: into plan->exchanges
};

// A dense block of a QS_PLAN_FUSED plan: 2^k x 2^k complex matrix over qubits.
struct qs_block {
  int k;
  int q[6];
  std::vector<double> M;  // row-major (re, im)
  // tensor-core blocks (k >= 4): qubits ascending and the offset of the
  // block's B in the plan's tc_B (prepared once, uploaded once per run):
  // complex64 FP32 values, complex128 FP16 digit matrices (two per float
  // slot) on the grid 2^(f128 - 43)
  bool tc = false;
  int q_sorted[6];
  size_t b_off = 0;
  int f128 = 0;
};

struct qs_tile_pass;    // defined in tile.cu

struct qs_plan {
  int n = 0;
  qs_dtype dtype = QS_C128;
  qs_plan_opts opts{};
  std::vector<qs_gate_rec> gates;
  std::vector<qs_step> steps;
  qs_plan_stats stats{};
  // tile passes (host description; owned by the plan, freed by tile_free)
  std::vector<qs_tile_pass*> tiles;
  std::vector<qs_block> blocks;
  std::vector<float> tc_B;  // all tensor-core blocks' B, concatenated
  // EXCHANGE steps: disjoint bit pairs (a_i, b_i) exchanged in one pass
  std::vector<std::vector<std::pair<int, int>>> exchanges;
};

namespace qs {
qs_status run_tile(qs_state* s, qs_plan* p, int tile_index, bool dfl);
void tile_free(qs_tile_pass* t);
}  // namespace qs
