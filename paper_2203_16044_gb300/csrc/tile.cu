// Tile passes: many gates per HBM pass.
//
// The single-GPU form of the paper's local-qubit idea (§III-B): gates on
// "local" qubits need no exchange, so a pass that keeps a set T of m qubits
// resident in shared memory can apply every gate acting on T before the
// amplitudes go back to HBM.  T is the L lowest qubits (contiguous runs of
// 2^L amplitudes keep every HBM access coalesced) plus r = m - L high qubits
// chosen per pass by the planner.  A tile is one assignment of the n - m
// other ("global") bits: 2^r runs of 2^L amplitudes.  Gates whose controls
// or phase bits lie outside T are still absorbed, because those bits are
// constant over a tile (they become per-tile predicates).  This replaces the
// explicit swap / fused-swap insertion of §III-D: no permutation pass is
// needed, since each pass gathers whichever qubits it works on.
//
// Inside a pass the gate list is split into stages.  A stage names G "slot"
// qubits (G = 3 or 4); each thread loads the 2^G amplitudes spanning them
// (for GPT assignments of the other tile bits at once) from shared memory
// into registers, applies every gate of the stage whose target is a slot
// qubit (controls and phases may be on any qubit), and writes them back.
// Each operation is decoded once per stage and thread and applied to all of
// the thread's register groups.  Shared memory is XOR-swizzled so that the
// strided accesses of a stage whose slots include low qubits stay free of
// bank conflicts.
//
// Arithmetic: complex64 in FP32; complex128 in double-float (dfloat.cuh),
// converted from / to the FP64 layout once per pass at load / store.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "planner.h"
#include "tilecore.cuh"

namespace qs {
namespace {

struct TileArgs {
  int L, m, r, nstages;
  u64 ntiles;
  Ins tins;            // zero insertion at the high tile qubits
  int H[kMaxR];
  TStage stages[kMaxStages];
  TOp ops[kMaxOps];
  float mats[kMaxMats * kMatFloats];
};
static_assert(sizeof(TileArgs) < 32000, "kernel parameter block limit");

// ops, stages and dense matrices read straight from the kernel parameter block
struct ParamSrc {
  const TileArgs& A;
  __device__ __forceinline__ const TStage& stage(int s) const { return A.stages[s]; }
  __device__ __forceinline__ const TOp& op(int o) const { return A.ops[o]; }
  __device__ __forceinline__ const float* mat(int i) const { return A.mats + i * kMatFloats; }
};

template <int MODE, int G, int GPT, bool DENSE>
__global__ void __launch_bounds__(kTT) k_tile(void* amp, const __grid_constant__ TileArgs A) {
  typedef typename Elem<MODE>::T E;
  typedef typename std::conditional<MODE == 1, double, float>::type R;  // MODE 2: double-float storage
  constexpr int APP = MODE == 0 ? 2 : 1;  // amplitudes per 16-byte packet
  extern __shared__ __align__(16) unsigned char smem[];
  u64* tab = reinterpret_cast<u64*>(smem);  // [2][64] spread tables
  E* t = reinterpret_cast<E*>(smem + 2 * 64 * sizeof(u64));
  R* a = static_cast<R*>(amp);
  const int L = A.L, m = A.m;
  const int tile = 1 << m;
  build_spread(tab, A.H, A.r);
  __syncthreads();
  const ParamSrc src{A};
  for (u64 ti = blockIdx.x; ti < A.ntiles; ti += gridDim.x) {
    const u64 F = expand(ti << L, A.tins);
    for (int e = threadIdx.x; e < tile / APP; e += kTT) {
      const int la = e * APP;
      load_pk<MODE>(a, tile_global(F, tab, la, L) / APP, t, la);
    }
    __syncthreads();
    run_stages<MODE, G, GPT, DENSE>(t, m, F, src, A.nstages);
    for (int e = threadIdx.x; e < tile / APP; e += kTT) {
      const int la = e * APP;
      store_pk<MODE>(a, tile_global(F, tab, la, L) / APP, t, la);
    }
    __syncthreads();
  }
}

// ---- planner --------------------------------------------------------------

enum GClass { G_DENSE1, G_CNOT, G_XGATE, G_DIAG1, G_PHASE1, G_PHASE2, G_SWAP };

GClass classify(int kind) {
  switch (kind) {
    case QS_GATE_X: return G_XGATE;
    case QS_GATE_CNOT: return G_CNOT;
    case QS_GATE_RZ: return G_DIAG1;
    case QS_GATE_Z: case QS_GATE_S: case QS_GATE_T: case QS_GATE_P: return G_PHASE1;
    case QS_GATE_CZ: case QS_GATE_CP: return G_PHASE2;
    case QS_GATE_SWAP: return G_SWAP;
    default: return G_DENSE1;
  }
}

// Qubits a gate needs inside the tile (its targets).
int tile_needs(const qs_gate_rec& g, int* q) {
  switch (classify(g.kind)) {
    case G_DENSE1: case G_XGATE: q[0] = g.q[0]; return 1;
    case G_CNOT: q[0] = g.q[1]; return 1;
    case G_SWAP: q[0] = g.q[0]; q[1] = g.q[1]; return 2;
    default: return 0;
  }
}

int gate_qubits(const qs_gate_rec& g, int* q) {
  q[0] = g.q[0];
  if (gate_arity(g.kind) == 2) { q[1] = g.q[1]; return 2; }
  return 1;
}

void set_matrix(TOp& op, const double* m, int count, qs_dtype dt) {
  for (int i = 0; i < 16; ++i) op.f[i] = 0.0f;
  for (int i = 0; i < count; ++i) {
    const float h = (float)m[i];
    op.f[i] = h;
    if (dt == QS_C128) op.f[8 + i] = (float)(m[i] - (double)h);
  }
}

// Local tile qubits a gate touches (targets, controls, phase bits) and
// whether it also reads bits outside the tile.
void gate_locality(const qs_gate_rec& g, const std::vector<int>& loc, uint64_t& lq, bool& global) {
  int gq[2];
  const int ng = gate_qubits(g, gq);
  lq = 0;
  global = false;
  for (int i = 0; i < ng; ++i) {
    if (loc[gq[i]] >= 0) lq |= uint64_t(1) << loc[gq[i]];
    else global = true;
  }
}

// Rough per-amplitude instruction costs, used to pick dense or op stages
// (measured shape on GB300: a stage's shared-memory round trip ~12, a dense
// 8x8 stage ~44, a dense one-qubit op ~10, an exchange ~4).
double op_cost(const qs_gate_rec& g) {
  switch (classify(g.kind)) {
    case G_DENSE1: return 10.0;
    case G_DIAG1: return 8.0;
    case G_PHASE1: case G_PHASE2: return 6.0;
    default: return 4.0;
  }
}
constexpr double kStageCost = 12.0, kDenseStageCost = 44.0;

typedef std::complex<double> cd;

// 8x8 matrix of one gate on the slot qubits S (bit i of the index = S[i]).
void gate_on_slots(const qs_gate_rec& g, const std::vector<int>& loc, const std::vector<int>& S, cd (*G8)[8]) {
  auto slot = [&](int q) { return (int)(std::find(S.begin(), S.end(), loc[q]) - S.begin()); };
  for (int r = 0; r < 8; ++r)
    for (int c = 0; c < 8; ++c) G8[r][c] = 0.0;
  double m[32];
  gate_matrix(g.kind, g.p, m);
  switch (classify(g.kind)) {
    case G_DENSE1: case G_XGATE: case G_DIAG1: case G_PHASE1: {
      const int a = slot(g.q[0]);
      for (int k = 0; k < 8; ++k)
        for (int k2 = 0; k2 < 8; ++k2)
          if (((k ^ k2) & ~(1 << a)) == 0) {
            const int ro = (k2 >> a) & 1, co = (k >> a) & 1;
            G8[k2][k] = cd(m[2 * (ro * 2 + co)], m[2 * (ro * 2 + co) + 1]);
          }
    } break;
    case G_CNOT: {
      const int c = slot(g.q[0]), t = slot(g.q[1]);
      for (int k = 0; k < 8; ++k) G8[((k >> c) & 1) ? (k ^ (1 << t)) : k][k] = 1.0;
    } break;
    case G_PHASE2: {
      const int a = slot(g.q[0]), b = slot(g.q[1]);
      for (int k = 0; k < 8; ++k) {
        const int r4 = ((k >> a) & 1) | (((k >> b) & 1) << 1);
        G8[k][k] = cd(m[2 * (r4 * 4 + r4)], m[2 * (r4 * 4 + r4) + 1]);
      }
    } break;
    case G_SWAP: {
      const int a = slot(g.q[0]), b = slot(g.q[1]);
      for (int k = 0; k < 8; ++k) {
        const int ba = (k >> a) & 1, bb = (k >> b) & 1;
        const int k2 = (k & ~((1 << a) | (1 << b))) | (ba << b) | (bb << a);
        G8[k2][k] = 1.0;
      }
    } break;
  }
}

// Build the stages and device ops of one pass from its gate list: greedy
// list scheduling; a gate joins the current stage when no earlier gate left
// for a later stage touches its tile qubits and it fits the stage.  For
// complex64 with three slots a stage may instead be dense: every gate whose
// tile qubits all lie in the three slots (and that reads nothing outside the
// tile) is multiplied into one 8x8 matrix, used when cheaper than the ops.
void build_pass_ops(qs_tile_pass& tp, const std::vector<const qs_gate_rec*>& gates, qs_dtype dt, int n,
                    bool allow_dense) {
  const int G = tp.G;
  const bool dense_ok = allow_dense && dt == QS_C64 && G == 3;
  std::vector<int> loc(n, -1);
  for (int q = 0; q < tp.L; ++q) loc[q] = q;
  for (int i = 0; i < tp.r; ++i) loc[tp.H[i]] = tp.L + i;
  std::vector<const qs_gate_rec*> rest = gates;
  auto finish_slots = [&](std::vector<int>& S, TStage& st) {
    // complete the slot set with unused local qubits, highest first
    for (int l = tp.m - 1; l >= 0 && (int)S.size() < G; --l)
      if (std::find(S.begin(), S.end(), l) == S.end()) S.push_back(l);
    for (int i = 0; i < G; ++i) st.sq[i] = (uint8_t)S[i];
    std::vector<int> srt = S;
    std::sort(srt.begin(), srt.end());
    for (int i = 0; i < G; ++i) st.srt[i] = (uint8_t)srt[i];
  };
  while (!rest.empty()) {
    if (dense_ok && (int)(tp.mats.size() / kMatFloats) < kMaxMats) {
      std::vector<int> S;
      uint64_t blocked = 0;
      std::vector<const qs_gate_rec*> later, taken;
      double cost_ops = kStageCost;
      for (const qs_gate_rec* g : rest) {
        uint64_t lq;
        bool glob;
        gate_locality(*g, loc, lq, glob);
        if ((lq & blocked) || glob) {
          blocked |= lq;
          later.push_back(g);
          continue;
        }
        std::vector<int> need;
        for (int l = 0; l < tp.m; ++l)
          if (((lq >> l) & 1) && std::find(S.begin(), S.end(), l) == S.end()) need.push_back(l);
        if (S.size() + need.size() <= 3) {
          for (int l : need) S.push_back(l);
          taken.push_back(g);
          cost_ops += op_cost(*g);
        } else {
          blocked |= lq;
          later.push_back(g);
        }
      }
      if (!taken.empty() && cost_ops > kDenseStageCost) {
        TStage st{};
        finish_slots(S, st);
        cd M[8][8], G8[8][8], T[8][8];
        for (int r = 0; r < 8; ++r)
          for (int c = 0; c < 8; ++c) M[r][c] = (r == c) ? 1.0 : 0.0;
        for (const qs_gate_rec* g : taken) {
          gate_on_slots(*g, loc, S, G8);
          for (int r = 0; r < 8; ++r)
            for (int c = 0; c < 8; ++c) {
              cd acc = 0.0;
              for (int k = 0; k < 8; ++k) acc += G8[r][k] * M[k][c];
              T[r][c] = acc;
            }
          for (int r = 0; r < 8; ++r)
            for (int c = 0; c < 8; ++c) M[r][c] = T[r][c];
        }
        st.dense = 1;
        st.op_begin = (uint16_t)(tp.mats.size() / kMatFloats);
        st.op_end = st.op_begin;
        for (int r = 0; r < 8; ++r)
          for (int c = 0; c < 8; ++c) {
            tp.mats.push_back((float)M[r][c].real());
            tp.mats.push_back((float)M[r][c].imag());
          }
        tp.stages.push_back(st);
        rest.swap(later);
        continue;
      }
    }
    // op stage: targets in the G slots, controls and phases anywhere
    std::vector<int> S;  // slot -> local qubit
    uint64_t blocked = 0;
    std::vector<const qs_gate_rec*> later, taken;
    for (const qs_gate_rec* g : rest) {
      uint64_t lq;
      bool glob;
      gate_locality(*g, loc, lq, glob);
      if (lq & blocked) {
        blocked |= lq;
        later.push_back(g);
        continue;
      }
      int nq[2];
      const int nn = tile_needs(*g, nq);
      std::vector<int> need;
      for (int i = 0; i < nn; ++i) {
        const int l = loc[nq[i]];
        if (std::find(S.begin(), S.end(), l) == S.end()) need.push_back(l);
      }
      if ((int)(S.size() + need.size()) <= G) {
        for (int l : need) S.push_back(l);
        taken.push_back(g);
      } else {
        blocked |= lq;
        later.push_back(g);
      }
    }
    TStage st{};
    finish_slots(S, st);
    st.op_begin = (uint16_t)tp.ops.size();
    auto slot_of = [&](int q) { return (int)(std::find(S.begin(), S.end(), loc[q]) - S.begin()); };
    auto bit_masks = [&](int q, TOp& op) {
      if (loc[q] >= 0) op.lmask |= 1u << loc[q];
      else op.gmask |= uint64_t(1) << q;
    };
    for (const qs_gate_rec* gp : taken) {
      const qs_gate_rec& g = *gp;
      TOp op{};
      double m[32];
      gate_matrix(g.kind, g.p, m);
      switch (classify(g.kind)) {
        case G_DENSE1:
          op.type = T_U;
          op.a = (uint8_t)slot_of(g.q[0]);
          set_matrix(op, m, 8, dt);
          break;
        case G_XGATE:
          op.type = T_XPERM;
          op.a = (uint8_t)slot_of(g.q[0]);
          break;
        case G_CNOT:
          op.type = T_XPERM;
          op.a = (uint8_t)slot_of(g.q[1]);
          bit_masks(g.q[0], op);
          break;
        case G_PHASE1: {
          op.type = T_PHASE;
          bit_masks(g.q[0], op);
          const double z[2] = {m[6], m[7]};
          set_matrix(op, z, 2, dt);
        } break;
        case G_PHASE2: {
          op.type = T_PHASE;
          bit_masks(g.q[0], op);
          bit_masks(g.q[1], op);
          const double z[2] = {m[30], m[31]};
          set_matrix(op, z, 2, dt);
        } break;
        case G_DIAG1: {
          op.type = T_DIAG1;
          if (loc[g.q[0]] >= 0) { op.a = (uint8_t)loc[g.q[0]]; op.dglobal = 0; }
          else { op.a = (uint8_t)g.q[0]; op.dglobal = 1; }
          const double d[4] = {m[0], m[1], m[6], m[7]};
          set_matrix(op, d, 4, dt);
        } break;
        case G_SWAP: {
          op.type = T_SWAP;
          const int s0 = slot_of(g.q[0]), s1 = slot_of(g.q[1]);
          op.a = (uint8_t)std::min(s0, s1);
          op.b = (uint8_t)std::max(s0, s1);
        } break;
      }
      tp.ops.push_back(op);
    }
    st.op_end = (uint16_t)tp.ops.size();
    tp.stages.push_back(st);
    rest.swap(later);
  }
}

// Defaults from a sweep on GB300 (30- and 26-qubit brick circuits).
int default_tile_qubits(qs_dtype dt) { return dt == QS_C64 ? 13 : 12; }
int default_low_qubits(qs_dtype dt) { return dt == QS_C64 ? 4 : 4; }
int default_slots(qs_dtype dt) { return dt == QS_C64 ? 3 : 3; }
int default_gpt(qs_dtype dt) { return dt == QS_C64 ? 1 : 1; }

template <int MODE, int G, int GPT, bool DENSE>
qs_status launch_tile(qs_state* s, const TileArgs& A, size_t smem, unsigned grid) {
  auto kern = k_tile<MODE, G, GPT, DENSE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "tile: smem attribute");
  kern<<<grid, kTT, smem, s->stream>>>(s->amp, A);
  return launch_ok("k_tile");
}

}  // namespace

int tile_targets(const qs_gate_rec& g, int* q) { return tile_needs(g, q); }

int tile_stage_count(const qs_plan* p, int* dense) {
  int n = 0, d = 0;
  for (const qs_tile_pass* t : p->tiles) {
    n += (int)t->stages.size();
    for (const TStage& s : t->stages) d += s.dense;
  }
  if (dense) *dense = d;
  return n;
}

// Tile options of a plan (validated; defaults filled in); n >= 4.
qs_status tile_options(qs_plan* p, int* m_out, int* L_out, int* G_out) {
  const int n = p->n;
  const qs_plan_opts& o = p->opts;
  int m = o.tile_qubits > 0 ? o.tile_qubits : default_tile_qubits(p->dtype);
  int L = o.low_qubits > 0 ? o.low_qubits : default_low_qubits(p->dtype);
  const int G = o.slot_qubits > 0 ? o.slot_qubits : default_slots(p->dtype);
  const int gpt = o.groups_per_thread > 0 ? o.groups_per_thread : default_gpt(p->dtype);
  const int maxm = p->dtype == QS_C64 ? 14 : 13;
  if (m < 4 || m > maxm) return fail(QS_EINVAL, "qs_plan_build: tile_qubits=%d outside [4, %d]", m, maxm);
  if (L < 1 || L > m) return fail(QS_EINVAL, "qs_plan_build: low_qubits=%d outside [1, tile_qubits]", L);
  if (G != 3 && G != 4) return fail(QS_EINVAL, "qs_plan_build: slot_qubits must be 3 or 4");
  if (gpt != 1 && gpt != 2) return fail(QS_EINVAL, "qs_plan_build: groups_per_thread must be 1 or 2");
  if (o.dense != 0 && o.dense != -1) return fail(QS_EINVAL, "qs_plan_build: dense must be 0 or -1");
  if (m > n) m = n;
  if (L > m) L = m;
  if (m - L > kMaxR) return fail(QS_EINVAL, "qs_plan_build: at most %d high tile qubits", kMaxR);
  p->opts.slot_qubits = G;
  // complex128 with four slots holds 64 floats per group: one group per
  // thread (two would spill registers)
  p->opts.groups_per_thread = (p->dtype == QS_C128 && G == 4) ? 1 : gpt;
  *m_out = m;
  *L_out = L;
  *G_out = G;
  return QS_OK;
}

// Tile passes for a gate list, appended to p->steps: each pass keeps the L
// lowest qubits and up to m - L chosen higher ones resident and absorbs, in
// order, every gate whose targets it holds (a gate left out blocks its
// qubits for the rest of the scan).
qs_status tile_gates(qs_plan* p, std::vector<const qs_gate_rec*> remaining, int m, int L, int G) {
  const int n = p->n;
  const int r = m - L;
  const bool dense = p->opts.dense >= 0;
  while (!remaining.empty()) {
    std::vector<char> inT(n, 0), blocked(n, 0);
    for (int q = 0; q < L; ++q) inT[q] = 1;
    std::vector<int> H;
    std::vector<const qs_gate_rec*> absorbed, rest;
    for (const qs_gate_rec* g : remaining) {
      int gq[2];
      const int ng = gate_qubits(*g, gq);
      bool blk = false;
      for (int i = 0; i < ng; ++i) blk |= blocked[gq[i]] != 0;
      if (!blk) {
        int nq[2];
        const int nn = tile_needs(*g, nq);
        std::vector<int> add;
        for (int i = 0; i < nn; ++i)
          if (!inT[nq[i]]) add.push_back(nq[i]);
        if ((int)(H.size() + add.size()) <= r && (int)absorbed.size() < kMaxOps) {
          for (int q : add) { inT[q] = 1; H.push_back(q); }
          absorbed.push_back(g);
          continue;
        }
      }
      for (int i = 0; i < ng; ++i) blocked[gq[i]] = 1;
      rest.push_back(g);
    }
    if (absorbed.empty())
      return fail(QS_EINVAL, "qs_plan_build: a tile of %d low + %d chosen qubits cannot hold the next gate", L, r);
    // fill the remaining high slots (the kernel's tile shape is fixed)
    for (int q = n - 1; q >= L && (int)H.size() < r; --q)
      if (!inT[q]) { inT[q] = 1; H.push_back(q); }
    std::sort(H.begin(), H.end());
    qs_tile_pass* tp = new qs_tile_pass();
    tp->L = L;
    tp->r = r;
    tp->m = m;
    tp->G = G;
    for (int i = 0; i < r; ++i) tp->H[i] = H[i];
    build_pass_ops(*tp, absorbed, p->dtype, n, dense);
    if ((int)tp->ops.size() > kMaxOps || (int)tp->stages.size() > kMaxStages) {
      // too many stages for one parameter block: split the pass's gates
      delete tp;
      const size_t half = absorbed.size() / 2;
      std::vector<const qs_gate_rec*> again(absorbed.begin() + half, absorbed.end());
      again.insert(again.end(), rest.begin(), rest.end());
      // the first half stays absorbed by a smaller pass over the same tile set
      std::vector<const qs_gate_rec*> first(absorbed.begin(), absorbed.begin() + half);
      tp = new qs_tile_pass();
      tp->L = L; tp->r = r; tp->m = m; tp->G = G;
      for (int i = 0; i < r; ++i) tp->H[i] = H[i];
      build_pass_ops(*tp, first, p->dtype, n, dense);
      if (half == 0 || (int)tp->ops.size() > kMaxOps || (int)tp->stages.size() > kMaxStages) {
        delete tp;
        return fail(QS_EUNSUPPORTED, "qs_plan_build: tile pass too large");
      }
      rest.swap(again);
    }
    p->tiles.push_back(tp);
    qs_step st{};
    st.type = qs_step::TILE;
    st.tile_index = (int)p->tiles.size() - 1;
    p->steps.push_back(st);
    remaining.swap(rest);
  }
  return QS_OK;
}

qs_status plan_tiled(qs_plan* p) {
  if (p->n < 4) {  // a tile needs its slot qubits: per-gate passes instead
    for (const qs_gate_rec& g : p->gates) p->steps.push_back(unfused_step(g));
    return QS_OK;
  }
  int m = 0, L = 0, G = 0;
  qs_status st = tile_options(p, &m, &L, &G);
  if (st != QS_OK) return st;
  std::vector<const qs_gate_rec*> all;
  for (const qs_gate_rec& g : p->gates) all.push_back(&g);
  return tile_gates(p, all, m, L, G);
}

qs_status run_tile(qs_state* s, qs_plan* p, int tile_index, bool dfl) {
  const qs_tile_pass& tp = *p->tiles[tile_index];
  static thread_local TileArgs A;
  A.L = tp.L;
  A.m = tp.m;
  A.r = tp.r;
  A.nstages = (int)tp.stages.size();
  A.ntiles = u64(1) << (s->n - tp.m);
  Ins ins{};
  ins.k = tp.r;
  ins.set = 0;
  for (int i = 0; i < tp.r; ++i) {
    ins.pos[i] = tp.H[i];
    A.H[i] = tp.H[i];
  }
  A.tins = ins;
  std::memcpy(A.stages, tp.stages.data(), tp.stages.size() * sizeof(TStage));
  std::memcpy(A.ops, tp.ops.data(), tp.ops.size() * sizeof(TOp));
  if (!tp.mats.empty()) std::memcpy(A.mats, tp.mats.data(), tp.mats.size() * sizeof(float));
  const size_t esize = s->dtype == QS_C64 ? sizeof(float2) : sizeof(cdf);
  const size_t smem = 2 * 64 * sizeof(u64) + (size_t(1) << tp.m) * esize;
  const int per_sm = (int)std::max<size_t>(1, (227 * 1024) / (smem + 1024));
  const unsigned grid = grid_for(A.ntiles, 1, std::min(per_sm, 8));
  const int gpt = p->opts.groups_per_thread;
  if (s->dtype == QS_C64) {
    if (tp.G == 4) return gpt == 2 ? launch_tile<0, 4, 2, false>(s, A, smem, grid) : launch_tile<0, 4, 1, false>(s, A, smem, grid);
    if (!tp.mats.empty())
      return gpt == 2 ? launch_tile<0, 3, 2, true>(s, A, smem, grid) : launch_tile<0, 3, 1, true>(s, A, smem, grid);
    return gpt == 2 ? launch_tile<0, 3, 2, false>(s, A, smem, grid) : launch_tile<0, 3, 1, false>(s, A, smem, grid);
  }
  if (dfl) {
    if (tp.G == 4) return launch_tile<2, 4, 1, false>(s, A, smem, grid);
    return gpt == 2 ? launch_tile<2, 3, 2, false>(s, A, smem, grid) : launch_tile<2, 3, 1, false>(s, A, smem, grid);
  }
  if (tp.G == 4) return launch_tile<1, 4, 1, false>(s, A, smem, grid);
  return gpt == 2 ? launch_tile<1, 3, 2, false>(s, A, smem, grid) : launch_tile<1, 3, 1, false>(s, A, smem, grid);
}

void tile_free(qs_tile_pass* t) { delete t; }

}  // namespace qs
