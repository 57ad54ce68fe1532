// Device-side tile-pass machinery shared by the per-pass kernel (tile.cu)
// and the persistent batch kernel (batch.cu).  See tile.cu for the design.
#pragma once

#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "dfloat.cuh"
#include "kcommon.cuh"

namespace qs {

enum : uint8_t { T_U = 0, T_XPERM = 1, T_PHASE = 2, T_DIAG1 = 3, T_SWAP = 4 };

// One operation of a tile pass (device format, 80 bytes = 5 x 16).
struct alignas(16) TOp {
  uint8_t type;
  uint8_t a;        // slot of the target (T_U, T_XPERM), lower slot (T_SWAP), qubit (T_DIAG1)
  uint8_t b;        // upper slot (T_SWAP)
  uint8_t dglobal;  // T_DIAG1: a is a global qubit (constant over the tile)
  uint32_t lmask;   // local bits that must all be 1 (controls, phase bits)
  uint64_t gmask;   // global bits that must all be 1
  float f[16];      // complex64: f[0..7] matrix / phase; complex128: hi f[0..7], lo f[8..15]
};
static_assert(sizeof(TOp) == 80, "TOp layout");

struct TStage {
  uint8_t sq[4];    // local qubit of slot 0..3 (unused slots: 0)
  uint8_t srt[4];   // the slot qubits ascending (for index insertion)
  uint16_t op_begin, op_end;  // ops [op_begin, op_end); dense: op_begin = matrix index
  uint8_t dense;    // 1: the stage is one 8x8 complex64 matrix on its 3 slots
  uint8_t pad[3];
};
static_assert(sizeof(TStage) == 16, "TStage layout");

}  // namespace qs

struct qs_tile_pass {
  int L = 0, r = 0, m = 0, G = 3;
  int H[24] = {0};
  std::vector<qs::TOp> ops;
  std::vector<qs::TStage> stages;
  std::vector<float> mats;  // dense stages: 128 floats each, (re, im) row-major 8x8
};

namespace qs {
namespace {

constexpr int kTT = 256;         // threads per CTA
constexpr int kTabBits = 6;      // spread tables: 2 x 64 entries
constexpr int kMaxR = 2 * kTabBits;
// A pass's ops and stages travel in the kernel parameter block (constant
// bank: uniform, short-latency reads); the planner keeps passes within it.
constexpr int kMaxOps = 200;
constexpr int kMaxStages = 64;
constexpr int kMaxMats = 24;     // dense stage matrices per pass
constexpr int kMatFloats = 128;  // 8 x 8 complex64

template <int MODE> struct Elem;
template <> struct Elem<0> { typedef float2 T; };
template <> struct Elem<1> { typedef cdf T; };
template <> struct Elem<2> { typedef cdf T; };  // complex128 held in double-float storage

__device__ __forceinline__ int ins1(int x, int p) {
  const int lo = x & ((1 << p) - 1);
  return ((x ^ lo) << 1) | lo;
}

// amplitudes per 128-byte shared-memory row: 16 (complex64) or 8 (complex128)
template <int MODE>
__device__ __forceinline__ int swz(int x) {
  constexpr int SW = MODE == 0 ? 4 : 3;
  return x ^ ((x >> SW) & ((1 << SW) - 1));
}

// ---- arithmetic on one pair / one amplitude --------------------------------

struct OpData {
  uint32_t lmask;
  float f[16];
};

__device__ __forceinline__ void pair_u(const OpData& d, float2& x, float2& y) {
  M2<float> U;
#pragma unroll
  for (int i = 0; i < 8; ++i) U.m[i] = d.f[i];
  mv2(U, x.x, x.y, y.x, y.y);
}
__device__ __forceinline__ void pair_u(const OpData& d, cdf& x, cdf& y) {
  M2df U;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    U.h[i] = d.f[i];
    U.l[i] = d.f[8 + i];
  }
  mv2df(U, x, y);
}
__device__ __forceinline__ void amp_mul(float2& x, float zr, float zi, float, float) {
  const float r = zr * x.x - zi * x.y;
  x.y = zr * x.y + zi * x.x;
  x.x = r;
}
__device__ __forceinline__ void amp_mul(cdf& x, float zr, float zi, float zrl, float zil) {
  const float zh[2] = {zr, zi}, zl[2] = {zrl, zil};
  cmul_df(zh, zl, x);
}

// ---- per-op application on the register groups ------------------------------

template <int G, int GPT, int A, bool CTRL, typename E>
__device__ __forceinline__ void apply_u(E (&v)[GPT][1 << G], const int (&base)[GPT], const int (&sk)[1 << G],
                                       const OpData& d) {
#pragma unroll
  for (int j = 0; j < GPT; ++j) {
#pragma unroll
    for (int k = 0; k < (1 << G); ++k) {
      if (k & (1 << A)) continue;
      if (!CTRL || (((base[j] | sk[k]) & d.lmask) == d.lmask)) pair_u(d, v[j][k], v[j][k | (1 << A)]);
    }
  }
}

template <int G, int GPT, int A, bool CTRL, typename E>
__device__ __forceinline__ void apply_x(E (&v)[GPT][1 << G], const int (&base)[GPT], const int (&sk)[1 << G],
                                       uint32_t lmask) {
#pragma unroll
  for (int j = 0; j < GPT; ++j) {
#pragma unroll
    for (int k = 0; k < (1 << G); ++k) {
      if (k & (1 << A)) continue;
      if (!CTRL || (((base[j] | sk[k]) & lmask) == lmask)) {
        const E t = v[j][k];
        v[j][k] = v[j][k | (1 << A)];
        v[j][k | (1 << A)] = t;
      }
    }
  }
}

template <int G, int GPT, int A, int B, typename E>
__device__ __forceinline__ void apply_swap(E (&v)[GPT][1 << G]) {
#pragma unroll
  for (int j = 0; j < GPT; ++j) {
#pragma unroll
    for (int k = 0; k < (1 << G); ++k) {
      if ((k & (1 << A)) && !(k & (1 << B))) {
        const int k2 = (k ^ (1 << A)) | (1 << B);
        const E t = v[j][k];
        v[j][k] = v[j][k2];
        v[j][k2] = t;
      }
    }
  }
}

template <int G, int GPT, typename E>
__device__ __forceinline__ void dispatch_u(int a, bool ctrl, E (&v)[GPT][1 << G], const int (&base)[GPT],
                                           const int (&sk)[1 << G], const OpData& d) {
#define QS_U(A)                                                   \
  if (a == A) {                                                   \
    if (ctrl) apply_u<G, GPT, A, true>(v, base, sk, d);           \
    else apply_u<G, GPT, A, false>(v, base, sk, d);               \
    return;                                                       \
  }
  QS_U(0) QS_U(1) QS_U(2)
  if (G > 3) { QS_U((G > 3 ? 3 : 0)) }
#undef QS_U
}

template <int G, int GPT, typename E>
__device__ __forceinline__ void dispatch_x(int a, bool ctrl, E (&v)[GPT][1 << G], const int (&base)[GPT],
                                           const int (&sk)[1 << G], uint32_t lmask) {
#define QS_X(A)                                                   \
  if (a == A) {                                                   \
    if (ctrl) apply_x<G, GPT, A, true>(v, base, sk, lmask);       \
    else apply_x<G, GPT, A, false>(v, base, sk, lmask);           \
    return;                                                       \
  }
  QS_X(0) QS_X(1) QS_X(2)
  if (G > 3) { QS_X((G > 3 ? 3 : 0)) }
#undef QS_X
}

template <int G, int GPT, typename E>
__device__ __forceinline__ void dispatch_swap(int a, int b, E (&v)[GPT][1 << G]) {
  // a < b (the planner orders them)
  if (a == 0 && b == 1) apply_swap<G, GPT, 0, 1>(v);
  else if (a == 0 && b == 2) apply_swap<G, GPT, 0, 2>(v);
  else if (a == 1 && b == 2) apply_swap<G, GPT, 1, 2>(v);
  else if (G > 3) {
    constexpr int S3 = G > 3 ? 3 : 2;
    if (a == 0) apply_swap<G, GPT, 0, S3>(v);
    else if (a == 1) apply_swap<G, GPT, 1, S3>(v);
    else apply_swap<G, GPT, 2, S3>(v);
  }
}

// ---- HBM <-> shared memory ------------------------------------------------

template <int MODE>
__device__ __forceinline__ void load_pk(const float* a, u64 p, float2* t, int la) {
  float v[4];
  ld16(a + p * 4, v);
  t[swz<MODE>(la)] = make_float2(v[0], v[1]);
  t[swz<MODE>(la + 1)] = make_float2(v[2], v[3]);
}
template <int MODE>
__device__ __forceinline__ void store_pk(float* a, u64 p, const float2* t, int la) {
  const float2 x = t[swz<MODE>(la)], y = t[swz<MODE>(la + 1)];
  const float v[4] = {x.x, x.y, y.x, y.y};
  st16(a + p * 4, v);
}
template <int MODE>
__device__ __forceinline__ void load_pk(const double* a, u64 p, cdf* t, int la) {
  double v[2];
  ld16(a + p * 2, v);
  const dfl r = d2df(v[0]), i = d2df(v[1]);
  t[swz<MODE>(la)] = cdf{r.h, r.l, i.h, i.l};
}
// complex128 in double-float storage: an amplitude is one float4 (re_h, re_l, im_h, im_l)
template <int MODE>
__device__ __forceinline__ void load_pk(const float* a, u64 p, cdf* t, int la) {
  const float4 v = *reinterpret_cast<const float4*>(a + p * 4);
  t[swz<MODE>(la)] = cdf{v.x, v.y, v.z, v.w};
}
template <int MODE>
__device__ __forceinline__ void store_pk(float* a, u64 p, const cdf* t, int la) {
  const cdf x = t[swz<MODE>(la)];
  *reinterpret_cast<float4*>(a + p * 4) = make_float4(x.rh, x.rl, x.ih, x.il);
}
template <int MODE>
__device__ __forceinline__ void store_pk(double* a, u64 p, const cdf* t, int la) {
  const cdf x = t[swz<MODE>(la)];
  const double v[2] = {df2d(dfl{x.rh, x.rl}), df2d(dfl{x.ih, x.il})};
  st16(a + p * 2, v);
}


// Dense stage (complex64, three slots): out[r] = sum_c M[r][c] v[c] for the
// 8 amplitudes spanning the slot qubits, GPT groups per thread sharing each
// matrix element.  M: 8 x 8 complex, (re, im) row-major, uniform over the CTA.
// Rows are produced one at a time and written straight back to the tile:
// the group's 8 inputs are already in registers and no other thread reads
// them during the stage.
template <int GPT>
__device__ __forceinline__ void dense_stage(float2* t, const TStage& st, const float* M, int ngroups) {
  const int q0 = st.sq[0], q1 = st.sq[1], q2 = st.sq[2];
  for (int g0 = threadIdx.x; g0 < ngroups; g0 += kTT * GPT) {
    int base[GPT];
    float2 v[GPT][8];
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      const int gi = g0 + j * kTT;
      int b = gi < ngroups ? gi : 0;
      b = ins1(ins1(ins1(b, st.srt[0]), st.srt[1]), st.srt[2]);
      base[j] = b;
#pragma unroll
      for (int k = 0; k < 8; ++k) v[j][k] = t[swz<0>(b | ((k & 1) << q0) | (((k >> 1) & 1) << q1) | ((k >> 2) << q2))];
    }
#pragma unroll 1
    for (int r = 0; r < 8; ++r) {
      float ar[GPT], ai[GPT];
#pragma unroll
      for (int j = 0; j < GPT; ++j) { ar[j] = 0.f; ai[j] = 0.f; }
      const float* Mr = M + 16 * r;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float mr = Mr[2 * c], mi = Mr[2 * c + 1];
#pragma unroll
        for (int j = 0; j < GPT; ++j) {
          ar[j] = fmaf(mr, v[j][c].x, ar[j]);
          ar[j] = fmaf(-mi, v[j][c].y, ar[j]);
          ai[j] = fmaf(mr, v[j][c].y, ai[j]);
          ai[j] = fmaf(mi, v[j][c].x, ai[j]);
        }
      }
      const int off = ((r & 1) << q0) | (((r >> 1) & 1) << q1) | ((r >> 2) << q2);
#pragma unroll
      for (int j = 0; j < GPT; ++j)
        if (g0 + j * kTT < ngroups) t[swz<0>(base[j] | off)] = make_float2(ar[j], ai[j]);
    }
  }
}

// Runs the stages of one tile pass on the shared-memory tile t (2^m
// amplitudes, swizzled).  SRC supplies the pass's stages and ops:
// stage(s) and op(o).  F: the tile's global bits.
template <int MODE, int G, int GPT, bool DENSE, class SRC>
__device__ __forceinline__ void run_stages(typename Elem<MODE>::T* t, int m, u64 F, const SRC& src, int nstages) {
  typedef typename Elem<MODE>::T E;
  constexpr int NK = 1 << G;
  constexpr int NF = MODE == 0 ? 8 : 16;  // matrix floats an op carries
  const int ngroups = (1 << m) >> G;
  for (int s = 0; s < nstages; ++s) {
    const TStage& st = src.stage(s);
    if constexpr (DENSE && MODE == 0 && G == 3) {
      if (st.dense) {
        dense_stage<GPT>(t, st, src.mat(st.op_begin), ngroups);
        __syncthreads();
        continue;
      }
    }
    int sk[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      int x = 0;
#pragma unroll
      for (int i = 0; i < G; ++i) x |= ((k >> i) & 1) << st.sq[i];
      sk[k] = x;
    }
    for (int g0 = threadIdx.x; g0 < ngroups; g0 += kTT * GPT) {
      int base[GPT];
      E v[GPT][NK];
#pragma unroll
      for (int j = 0; j < GPT; ++j) {
        const int gi = g0 + j * kTT;
        int b = gi < ngroups ? gi : 0;
#pragma unroll
        for (int i = 0; i < G; ++i) b = ins1(b, st.srt[i]);
        base[j] = b;
#pragma unroll
        for (int k = 0; k < NK; ++k) v[j][k] = t[swz<MODE>(b | sk[k])];
      }
      for (int o = st.op_begin; o < st.op_end; ++o) {
        const TOp& op = src.op(o);
        const int type = op.type, oa = op.a;
        const u64 gmask = op.gmask;
        if ((F & gmask) != gmask) continue;
        OpData d;
        d.lmask = op.lmask;
        if (type == T_U || type == T_PHASE || type == T_DIAG1) {
#pragma unroll
          for (int q = 0; q < NF; ++q) d.f[q] = op.f[q];
        }
        if (type == T_U) {
          dispatch_u<G, GPT>(oa, d.lmask != 0, v, base, sk, d);
        } else if (type == T_XPERM) {
          dispatch_x<G, GPT>(oa, d.lmask != 0, v, base, sk, d.lmask);
        } else if (type == T_PHASE) {
#pragma unroll
          for (int j = 0; j < GPT; ++j)
#pragma unroll
            for (int k = 0; k < NK; ++k)
              if (((base[j] | sk[k]) & d.lmask) == d.lmask) amp_mul(v[j][k], d.f[0], d.f[1], d.f[8 % NF], d.f[9 % NF]);
        } else if (type == T_DIAG1) {
          const bool dglobal = op.dglobal != 0;
#pragma unroll
          for (int j = 0; j < GPT; ++j)
#pragma unroll
            for (int k = 0; k < NK; ++k) {
              const int hi = dglobal ? (int)((F >> oa) & 1u) : (((base[j] | sk[k]) >> oa) & 1);
              if (hi) amp_mul(v[j][k], d.f[2], d.f[3], d.f[10 % NF], d.f[11 % NF]);
              else amp_mul(v[j][k], d.f[0], d.f[1], d.f[8 % NF], d.f[9 % NF]);
            }
        } else {  // T_SWAP
          dispatch_swap<G, GPT>(oa, (int)op.b, v);
        }
      }
#pragma unroll
      for (int j = 0; j < GPT; ++j) {
        if (g0 + j * kTT < ngroups) {
#pragma unroll
          for (int k = 0; k < NK; ++k) t[swz<MODE>(base[j] | sk[k])] = v[j][k];
        }
      }
    }
    __syncthreads();
  }
}

// Spread tables: tab[part * 64 + j] = OR of 2^H[part * 6 + b] over the set
// bits b of j (r <= 12 high tile qubits).
__device__ __forceinline__ void build_spread(u64* tab, const int* H, int r) {
  for (int i = threadIdx.x; i < 128; i += kTT) {
    const int part = i >> 6, j = i & 63;
    u64 s = 0;
    for (int b = 0; b < kTabBits; ++b) {
      const int hb = part * kTabBits + b;
      if (hb < r && ((j >> b) & 1)) s |= u64(1) << H[hb];
    }
    tab[i] = s;
  }
}

// Global amplitude index of local tile index la (run j = la >> L).
__device__ __forceinline__ u64 tile_global(u64 F, const u64* tab, int la, int L) {
  const int j = la >> L;
  return F | tab[j & 63] | tab[64 + (j >> kTabBits)] | (u64)(la & ((1 << L) - 1));
}

}  // namespace
}  // namespace qs
