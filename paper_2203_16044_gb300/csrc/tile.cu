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
// Inside a pass the gate list is split into stages.  A stage names three
// "slot" qubits; each thread loads the 8 amplitudes spanning them (for one
// assignment of the other tile bits) from shared memory into registers,
// applies every gate of the stage whose target is a slot qubit (controls and
// phases may be on any qubit), and writes them back.
//
// Arithmetic: complex64 in FP32; complex128 in double-float (dfloat.cuh),
// converted from / to the FP64 layout once per pass at load / store.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "dfloat.cuh"
#include "kcommon.cuh"
#include "planner.h"

namespace qs {

enum : uint8_t { T_U = 0, T_XPERM = 1, T_PHASE = 2, T_DIAG1 = 3, T_SWAP = 4 };

// One operation of a tile pass (device format, 80 bytes).
struct alignas(16) TOp {
  uint8_t type;
  uint8_t a;        // slot of the target (T_U, T_XPERM), first slot (T_SWAP), qubit (T_DIAG1)
  uint8_t b;        // second slot (T_SWAP)
  uint8_t dglobal;  // T_DIAG1: a is a global qubit (constant over the tile)
  uint32_t lmask;   // local bits that must all be 1 (controls, phase bits)
  uint64_t gmask;   // global bits that must all be 1
  float f[16];      // complex64: f[0..7] matrix / phase; complex128: hi f[0..7], lo f[8..15]
};
static_assert(sizeof(TOp) == 80, "TOp layout");

struct TStage {
  uint8_t sq[3];    // local qubit of slot 0, 1, 2
  uint8_t srt[3];   // the same, ascending (for index insertion)
  uint16_t op_begin, op_end;
};
static_assert(sizeof(TStage) == 10, "TStage layout");

}  // namespace qs

struct qs_tile_pass {
  int L = 0, r = 0, m = 0;
  int H[24] = {0};
  std::vector<qs::TOp> ops;
  std::vector<qs::TStage> stages;
  size_t ops_off = 0, stages_off = 0;  // byte offsets into the plan's device table
};

namespace qs {
namespace {

constexpr int kTT = 256;         // threads per CTA
constexpr int kTabBits = 6;      // spread tables: 2 x 64 entries
constexpr int kMaxR = 2 * kTabBits;

struct TileArgs {
  int L, m, r, nstages;
  u64 ntiles;
  Ins tins;            // zero insertion at the high tile qubits
  int H[kMaxR];
  const TOp* ops;
  const TStage* stages;
};

template <int MODE> struct Elem;
template <> struct Elem<0> { typedef float2 T; };
template <> struct Elem<1> { typedef cdf T; };

__device__ __forceinline__ int ins1(int x, int p) {
  const int lo = x & ((1 << p) - 1);
  return ((x ^ lo) << 1) | lo;
}

// ---- per-op application on the 8 register amplitudes ----------------------

template <int A>
__device__ __forceinline__ void op_u(float2 (&v)[8], const int (&li)[8], uint32_t lmask, const M2<float>& U) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & (1 << A)) continue;
    if ((li[k] & lmask) == lmask) mv2(U, v[k].x, v[k].y, v[k | (1 << A)].x, v[k | (1 << A)].y);
  }
}
template <int A>
__device__ __forceinline__ void op_u(cdf (&v)[8], const int (&li)[8], uint32_t lmask, const M2df& U) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & (1 << A)) continue;
    if ((li[k] & lmask) == lmask) mv2df(U, v[k], v[k | (1 << A)]);
  }
}
template <int A, typename T>
__device__ __forceinline__ void op_x(T (&v)[8], const int (&li)[8], uint32_t lmask) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k & (1 << A)) continue;
    if ((li[k] & lmask) == lmask) {
      const T t = v[k];
      v[k] = v[k | (1 << A)];
      v[k | (1 << A)] = t;
    }
  }
}
template <int A, int B, typename T>
__device__ __forceinline__ void op_swap(T (&v)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if ((k & (1 << A)) && !(k & (1 << B))) {
      const int k2 = (k ^ (1 << A)) | (1 << B);
      const T t = v[k];
      v[k] = v[k2];
      v[k2] = t;
    }
  }
}

__device__ __forceinline__ void cmul(float2& x, float zr, float zi) {
  const float r = zr * x.x - zi * x.y;
  x.y = zr * x.y + zi * x.x;
  x.x = r;
}

__device__ __forceinline__ void apply_op(const TOp& op, float2 (&v)[8], const int (&li)[8], u64 F) {
  if ((F & op.gmask) != op.gmask) return;
  switch (op.type) {
    case T_U: {
      M2<float> U;
#pragma unroll
      for (int i = 0; i < 8; ++i) U.m[i] = op.f[i];
      if (op.a == 0) op_u<0>(v, li, op.lmask, U);
      else if (op.a == 1) op_u<1>(v, li, op.lmask, U);
      else op_u<2>(v, li, op.lmask, U);
    } break;
    case T_XPERM:
      if (op.a == 0) op_x<0>(v, li, op.lmask);
      else if (op.a == 1) op_x<1>(v, li, op.lmask);
      else op_x<2>(v, li, op.lmask);
      break;
    case T_PHASE:
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if ((li[k] & op.lmask) == op.lmask) cmul(v[k], op.f[0], op.f[1]);
      break;
    case T_DIAG1:
      if (op.dglobal) {
        const int hi = (int)((F >> op.a) & 1u);
        const float zr = op.f[2 * hi], zi = op.f[2 * hi + 1];
#pragma unroll
        for (int k = 0; k < 8; ++k) cmul(v[k], zr, zi);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int hi = (li[k] >> op.a) & 1;
          cmul(v[k], hi ? op.f[2] : op.f[0], hi ? op.f[3] : op.f[1]);
        }
      }
      break;
    case T_SWAP:
      if (op.a == 0 && op.b == 1) op_swap<0, 1>(v);
      else if (op.a == 1 && op.b == 0) op_swap<1, 0>(v);
      else if (op.a == 0 && op.b == 2) op_swap<0, 2>(v);
      else if (op.a == 2 && op.b == 0) op_swap<2, 0>(v);
      else if (op.a == 1 && op.b == 2) op_swap<1, 2>(v);
      else op_swap<2, 1>(v);
      break;
  }
}

__device__ __forceinline__ void apply_op(const TOp& op, cdf (&v)[8], const int (&li)[8], u64 F) {
  if ((F & op.gmask) != op.gmask) return;
  switch (op.type) {
    case T_U: {
      M2df U;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        U.h[i] = op.f[i];
        U.l[i] = op.f[8 + i];
      }
      if (op.a == 0) op_u<0>(v, li, op.lmask, U);
      else if (op.a == 1) op_u<1>(v, li, op.lmask, U);
      else op_u<2>(v, li, op.lmask, U);
    } break;
    case T_XPERM:
      if (op.a == 0) op_x<0>(v, li, op.lmask);
      else if (op.a == 1) op_x<1>(v, li, op.lmask);
      else op_x<2>(v, li, op.lmask);
      break;
    case T_PHASE: {
      const float zh[2] = {op.f[0], op.f[1]}, zl[2] = {op.f[8], op.f[9]};
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if ((li[k] & op.lmask) == op.lmask) cmul_df(zh, zl, v[k]);
    } break;
    case T_DIAG1:
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int hi = op.dglobal ? (int)((F >> op.a) & 1u) : (li[k] >> op.a) & 1;
        const float zh[2] = {op.f[2 * hi], op.f[2 * hi + 1]}, zl[2] = {op.f[8 + 2 * hi], op.f[9 + 2 * hi]};
        cmul_df(zh, zl, v[k]);
      }
      break;
    case T_SWAP:
      if (op.a == 0 && op.b == 1) op_swap<0, 1>(v);
      else if (op.a == 1 && op.b == 0) op_swap<1, 0>(v);
      else if (op.a == 0 && op.b == 2) op_swap<0, 2>(v);
      else if (op.a == 2 && op.b == 0) op_swap<2, 0>(v);
      else if (op.a == 1 && op.b == 2) op_swap<1, 2>(v);
      else op_swap<2, 1>(v);
      break;
  }
}

// ---- HBM <-> shared memory ------------------------------------------------

__device__ __forceinline__ void load_pk(const float* a, u64 p, float2* t, int la) {
  float v[4];
  ld16(a + p * 4, v);
  t[la] = make_float2(v[0], v[1]);
  t[la + 1] = make_float2(v[2], v[3]);
}
__device__ __forceinline__ void store_pk(float* a, u64 p, const float2* t, int la) {
  const float2 x = t[la], y = t[la + 1];
  const float v[4] = {x.x, x.y, y.x, y.y};
  st16(a + p * 4, v);
}
__device__ __forceinline__ void load_pk(const double* a, u64 p, cdf* t, int la) {
  double v[2];
  ld16(a + p * 2, v);
  const dfl r = d2df(v[0]), i = d2df(v[1]);
  t[la] = cdf{r.h, r.l, i.h, i.l};
}
__device__ __forceinline__ void store_pk(double* a, u64 p, const cdf* t, int la) {
  const cdf x = t[la];
  const double v[2] = {df2d(dfl{x.rh, x.rl}), df2d(dfl{x.ih, x.il})};
  st16(a + p * 2, v);
}

template <int MODE>
__global__ void __launch_bounds__(kTT) k_tile(void* amp, const __grid_constant__ TileArgs A) {
  typedef typename Elem<MODE>::T E;
  typedef typename std::conditional<MODE == 0, float, double>::type R;
  constexpr int APP = MODE == 0 ? 2 : 1;  // amplitudes per 16-byte packet
  extern __shared__ __align__(16) unsigned char smem[];
  u64* tab = reinterpret_cast<u64*>(smem);            // [2][64] spread tables
  E* t = reinterpret_cast<E*>(smem + 2 * 64 * sizeof(u64));
  R* a = static_cast<R*>(amp);
  const int L = A.L, m = A.m;
  const int tile = 1 << m;
  const int lmask = (1 << L) - 1;
  // spread tables: j -> OR of 2^H[b] over the set bits b of j
  for (int i = threadIdx.x; i < 128; i += kTT) {
    const int part = i >> 6, j = i & 63;
    u64 s = 0;
    for (int b = 0; b < kTabBits; ++b) {
      const int hb = part * kTabBits + b;
      if (hb < A.r && ((j >> b) & 1)) s |= u64(1) << A.H[hb];
    }
    tab[i] = s;
  }
  __syncthreads();
  for (u64 ti = blockIdx.x; ti < A.ntiles; ti += gridDim.x) {
    const u64 F = expand(ti << L, A.tins);
    // load the tile: run j = la >> L, offset la & lmask
    for (int e = threadIdx.x; e < tile / APP; e += kTT) {
      const int la = e * APP;
      const int j = la >> L;
      const u64 g = F | tab[j & 63] | tab[64 + (j >> kTabBits)] | (u64)(la & lmask);
      load_pk(a, g / APP, t, la);
    }
    __syncthreads();
    for (int s = 0; s < A.nstages; ++s) {
      const TStage st = A.stages[s];
      const int q0 = st.sq[0], q1 = st.sq[1], q2 = st.sq[2];
      for (int gi = threadIdx.x; gi < (tile >> 3); gi += kTT) {
        const int base = ins1(ins1(ins1(gi, st.srt[0]), st.srt[1]), st.srt[2]);
        int li[8];
        E v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          li[k] = base | ((k & 1) << q0) | (((k >> 1) & 1) << q1) | (((k >> 2) & 1) << q2);
          v[k] = t[li[k]];
        }
        for (int o = st.op_begin; o < st.op_end; ++o) apply_op(A.ops[o], v, li, F);
#pragma unroll
        for (int k = 0; k < 8; ++k) t[li[k]] = v[k];
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < tile / APP; e += kTT) {
      const int la = e * APP;
      const int j = la >> L;
      const u64 g = F | tab[j & 63] | tab[64 + (j >> kTabBits)] | (u64)(la & lmask);
      store_pk(a, g / APP, t, la);
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

// Build the stages and device ops of one pass from its gate list.
void build_pass_ops(qs_tile_pass& tp, const std::vector<const qs_gate_rec*>& gates, qs_dtype dt, int n) {
  std::vector<int> loc(n, -1);
  for (int q = 0; q < tp.L; ++q) loc[q] = q;
  for (int i = 0; i < tp.r; ++i) loc[tp.H[i]] = tp.L + i;
  std::vector<const qs_gate_rec*> rest = gates;
  while (!rest.empty()) {
    std::vector<int> S;  // slot -> local qubit
    uint64_t blocked = 0;
    std::vector<const qs_gate_rec*> later;
    std::vector<std::pair<const qs_gate_rec*, std::vector<int>>> taken;
    for (const qs_gate_rec* g : rest) {
      int gq[2];
      const int ng = gate_qubits(*g, gq);
      uint64_t lq = 0;
      for (int i = 0; i < ng; ++i)
        if (loc[gq[i]] >= 0) lq |= uint64_t(1) << loc[gq[i]];
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
      if (S.size() + need.size() <= 3) {
        for (int l : need) S.push_back(l);
        taken.push_back({g, {}});
      } else {
        blocked |= lq;
        later.push_back(g);
      }
    }
    // complete the slot set with unused local qubits, highest first (keeps
    // the low qubits out of the slots: consecutive threads then touch
    // consecutive shared-memory words)
    for (int l = tp.m - 1; l >= 0 && S.size() < 3; --l)
      if (std::find(S.begin(), S.end(), l) == S.end()) S.push_back(l);
    TStage st{};
    for (int i = 0; i < 3; ++i) st.sq[i] = (uint8_t)S[i];
    std::vector<int> srt = S;
    std::sort(srt.begin(), srt.end());
    for (int i = 0; i < 3; ++i) st.srt[i] = (uint8_t)srt[i];
    st.op_begin = (uint16_t)tp.ops.size();
    auto slot_of = [&](int q) { return (int)(std::find(S.begin(), S.end(), loc[q]) - S.begin()); };
    auto bit_masks = [&](int q, TOp& op) {
      if (loc[q] >= 0) op.lmask |= 1u << loc[q];
      else op.gmask |= uint64_t(1) << q;
    };
    for (auto& tk : taken) {
      const qs_gate_rec& g = *tk.first;
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
        case G_SWAP:
          op.type = T_SWAP;
          op.a = (uint8_t)slot_of(g.q[0]);
          op.b = (uint8_t)slot_of(g.q[1]);
          break;
      }
      tp.ops.push_back(op);
    }
    st.op_end = (uint16_t)tp.ops.size();
    tp.stages.push_back(st);
    rest.swap(later);
  }
}

int default_tile_qubits(qs_dtype dt) { return dt == QS_C64 ? 13 : 12; }
int default_low_qubits(qs_dtype dt) { return dt == QS_C64 ? 5 : 4; }

}  // namespace

qs_status plan_tiled(qs_plan* p) {
  const int n = p->n;
  if (n < 3) {  // a tile needs three slot qubits: per-gate passes instead
    for (const qs_gate_rec& g : p->gates) p->steps.push_back(unfused_step(g));
    return QS_OK;
  }
  int m = p->opts.tile_qubits > 0 ? p->opts.tile_qubits : default_tile_qubits(p->dtype);
  int L = p->opts.low_qubits > 0 ? p->opts.low_qubits : default_low_qubits(p->dtype);
  const int maxm = p->dtype == QS_C64 ? 14 : 13;
  if (m < 3 || m > maxm) return fail(QS_EINVAL, "qs_plan_build: tile_qubits=%d outside [3, %d]", m, maxm);
  if (L < 1 || L > m) return fail(QS_EINVAL, "qs_plan_build: low_qubits=%d outside [1, tile_qubits]", L);
  if (m > n) m = n;
  if (L > m) L = m;
  int r = m - L;
  if (r > kMaxR) return fail(QS_EINVAL, "qs_plan_build: at most %d high tile qubits", kMaxR);
  if (p->dtype == QS_C64 && L < 1) L = 1;

  std::vector<const qs_gate_rec*> remaining;
  for (const qs_gate_rec& g : p->gates) remaining.push_back(&g);
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
        if ((int)(H.size() + add.size()) <= r) {
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
    for (int i = 0; i < r; ++i) tp->H[i] = H[i];
    build_pass_ops(*tp, absorbed, p->dtype, n);
    if (tp->ops.size() > 65535 || tp->stages.size() > 65535) {
      delete tp;
      return fail(QS_EUNSUPPORTED, "qs_plan_build: tile pass too large");
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

qs_status plan_tiles_upload(qs_plan* p, cudaStream_t stream) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (p->dev_tables && p->dev_tables_device == dev) return QS_OK;
  if (p->dev_tables) {
    cudaFree(p->dev_tables);
    p->dev_tables = nullptr;
  }
  size_t bytes = 0;
  for (qs_tile_pass* t : p->tiles) {
    t->ops_off = bytes;
    bytes += t->ops.size() * sizeof(TOp);
    bytes = (bytes + 15) & ~size_t(15);
    t->stages_off = bytes;
    bytes += t->stages.size() * sizeof(TStage);
    bytes = (bytes + 15) & ~size_t(15);
  }
  std::vector<unsigned char> host(bytes ? bytes : 16);
  for (qs_tile_pass* t : p->tiles) {
    if (!t->ops.empty()) std::memcpy(host.data() + t->ops_off, t->ops.data(), t->ops.size() * sizeof(TOp));
    if (!t->stages.empty())
      std::memcpy(host.data() + t->stages_off, t->stages.data(), t->stages.size() * sizeof(TStage));
  }
  cudaError_t e = cudaMalloc(&p->dev_tables, host.size());
  if (e != cudaSuccess) {
    p->dev_tables = nullptr;
    return fail(QS_ENOMEM, "plan tables: %s", cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(p->dev_tables, host.data(), host.size(), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "plan tables upload");
  p->dev_tables_bytes = host.size();
  p->dev_tables_device = dev;
  return QS_OK;
}

qs_status run_tile(qs_state* s, qs_plan* p, int tile_index) {
  const qs_tile_pass& tp = *p->tiles[tile_index];
  TileArgs A{};
  A.L = tp.L;
  A.m = tp.m;
  A.r = tp.r;
  A.nstages = (int)tp.stages.size();
  A.ntiles = u64(1) << (s->n - tp.m);
  std::vector<std::pair<int, int>> bits;
  Ins ins{};
  ins.k = tp.r;
  ins.set = 0;
  for (int i = 0; i < tp.r; ++i) {
    ins.pos[i] = tp.H[i];
    A.H[i] = tp.H[i];
  }
  A.tins = ins;
  const unsigned char* base = static_cast<const unsigned char*>(p->dev_tables);
  A.ops = reinterpret_cast<const TOp*>(base + tp.ops_off);
  A.stages = reinterpret_cast<const TStage*>(base + tp.stages_off);
  const size_t esize = s->dtype == QS_C64 ? sizeof(float2) : sizeof(cdf);
  const size_t smem = 2 * 64 * sizeof(u64) + (size_t(1) << tp.m) * esize;
  const int per_sm = (int)std::max<size_t>(1, (227 * 1024) / (smem + 1024));
  const unsigned grid = grid_for(A.ntiles, 1, std::min(per_sm, 8));
  cudaError_t e;
  if (s->dtype == QS_C64) {
    e = cudaFuncSetAttribute(k_tile<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "tile: smem attribute");
    k_tile<0><<<grid, kTT, smem, s->stream>>>(s->amp, A);
  } else {
    e = cudaFuncSetAttribute(k_tile<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "tile: smem attribute");
    k_tile<1><<<grid, kTT, smem, s->stream>>>(s->amp, A);
  }
  return launch_ok("k_tile");
}

void tile_free(qs_tile_pass* t) { delete t; }

}  // namespace qs
