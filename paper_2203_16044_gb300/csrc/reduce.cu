// Reductions over the state vector: norm, inner product, Pauli expectation.
//
// Each thread accumulates over a grid-stride range of elements in
// double-float, flushed into FP64 (see kU); warps combine in FP64 with shuffles, CTAs through shared memory, and the
// per-CTA partials are summed by one CTA in index order.  The grid size
// depends only on the problem size (and, for tile passes, the device), so
// results are bitwise reproducible.
//
// Expectation of Pauli strings: P|x> = i^{nY} (-1)^{popcount(x & z)} |x ^ m>
// (m = X/Y positions, z = Z/Y positions), so
//   <psi|P|psi> = sum_x conj(a_{x^m}) a_x i^{nY} (-1)^{popcount(x & z)}.
// Terms sharing m are evaluated together in one read of the state:
//   f(x) = sum_t c_t i^{nY_t} (-1)^{popcount(x & z_t)}.
// For m != 0 the pairs {x, x^m} are visited once (x with bit h of m clear,
// h = highest set bit of m), each amplitude read once.
//
// Groups whose X/Y bits all lie in one tile's qubit set -- the kTL lowest
// qubits and up to kTH chosen higher ones -- share one read of the state: a
// tile pass loads each tile (one assignment of the other qubits) into
// shared memory once and evaluates every group of the pass on it, since x
// and x ^ m then lie in the same tile.  The transverse-field Ising energy at
// 30 qubits (one Z-only group and 30 single-X groups) takes three such
// passes instead of 31.  Groups that fit no tile get a pass of their own.
//
// Inside a tile pass, single-term groups on one qubit (X or Y) go to
// register stages: a thread holds the amplitudes spanning a few tile qubits
// and forms every qubit's pair products from them (complex64: FP32 products
// and FP32 sums per thread and tile, then exact double-float slots;
// complex128: double-float products, slots flushed to FP64 every 16 tiles);
// the lanes of a warp take tile qubits that the XOR swizzle of the tile
// spreads over distinct banks.  Z-only two-qubit terms go by rows of 16
// amplitudes (complex64), their parity function being linear over GF(2).
// Complex64 tiles arrive by TMA (128-byte swizzle) into two buffers, the
// next tile's copy in flight while the current one is evaluated.  The
// partial sums follow a fixed order for a given grid, which depends on the
// problem size and the device, so results repeat on a given GPU.
#include <algorithm>
#include <cstring>
#include <vector>

#include <type_traits>

#include "dfloat.cuh"
#include "kcommon.cuh"
#include "pauli.cuh"
#include "umma.cuh"

namespace qs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of up to two values over NT threads; result valid in thread 0.
template <int NT = kThreads>
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[NT / 32], sb[NT / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (w == 0) {
    a = l < NT / 32 ? sa[l] : 0.0;
    b = l < NT / 32 ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

unsigned red_grid(u64 npk) {
  const u64 per = (u64)kThreads * 8;
  u64 g = (npk + per - 1) / per;
  const u64 cap = (u64)sm_count() * 4;
  if (g > cap) g = cap;
  return (unsigned)(g ? g : 1);
}

// Per-element arithmetic stays off the FP64 pipe (about 1/64 of FP32 on
// GB300): values enter as double-float (complex64: (x, 0); complex128: its
// (hi, lo) split, integer operations only), products are formed with their
// exact rounding errors (df_mul), and each thread sums them in double-float,
// flushing into its FP64 accumulator every kU elements.  Within a flush
// interval the high part's rounding errors are captured exactly (TwoSum) and
// only the low part rounds (~2^-24 of a few error terms): FP64-level
// accuracy, with 2 FP64 additions per kU elements.  Loads are unrolled kU
// deep so that each thread keeps kU independent 16-byte loads in flight.
constexpr int kU = 4;


template <typename R>
__global__ void __launch_bounds__(kThreads) k_norm2(const R* __restrict__ a, u64 npk, double2* part) {
  constexpr int V = PK<R>::V;
  const u64 stride = (u64)gridDim.x * kThreads;
  double s = 0.0, dummy = 0.0;
  dfl acc{0.f, 0.f};
  u64 p = (u64)blockIdx.x * kThreads + threadIdx.x;
  for (; p + (kU - 1) * stride < npk; p += kU * stride) {
    R v[kU][V];
#pragma unroll
    for (int u = 0; u < kU; ++u) ld16(a + (p + u * stride) * V, v[u]);
#pragma unroll
    for (int u = 0; u < kU; ++u)
#pragma unroll
      for (int c = 0; c < V; ++c) {
        const dfl x = to_df(v[u][c]);
        df_acc(acc, df_mul(x, x));
      }
    df_flush(s, acc);
  }
  for (; p < npk; p += stride) {
    R v[V];
    ld16(a + p * V, v);
#pragma unroll
    for (int c = 0; c < V; ++c) {
      const dfl x = to_df(v[c]);
      df_acc(acc, df_mul(x, x));
    }
  }
  df_flush(s, acc);
  block_sum2(s, dummy);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(s, 0.0);
}

// conj(a) b = (ar br + ai bi) + i (ar bi - ai br), reals c, c + 1 of a packet
template <typename R>
__device__ __forceinline__ void inner_acc(const R* va, const R* vb, int c, dfl& re, dfl& im) {
  const dfl ar = to_df(va[c]), ai = to_df(va[c + 1]), br = to_df(vb[c]), bi = to_df(vb[c + 1]);
  df_acc(re, df_mul(ar, br));
  df_acc(re, df_mul(ai, bi));
  df_acc(im, df_mul(ar, bi));
  df_acc(im, df_mul(dfl{-ai.h, -ai.l}, br));
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_inner(const R* __restrict__ a, const R* __restrict__ b, u64 npk,
                                                    double2* part) {
  constexpr int V = PK<R>::V;
  const u64 stride = (u64)gridDim.x * kThreads;
  double sr = 0.0, si = 0.0;
  dfl re{0.f, 0.f}, im{0.f, 0.f};
  u64 p = (u64)blockIdx.x * kThreads + threadIdx.x;
  for (; p + (kU - 1) * stride < npk; p += kU * stride) {
    R va[kU][V], vb[kU][V];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      ld16(a + (p + u * stride) * V, va[u]);
      ld16(b + (p + u * stride) * V, vb[u]);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u)
#pragma unroll
      for (int c = 0; c < V; c += 2) inner_acc(va[u], vb[u], c, re, im);
    df_flush(sr, re);
    df_flush(si, im);
  }
  for (; p < npk; p += stride) {
    R va[V], vb[V];
    ld16(a + p * V, va);
    ld16(b + p * V, vb);
#pragma unroll
    for (int c = 0; c < V; c += 2) inner_acc(va, vb, c, re, im);
  }
  df_flush(sr, re);
  df_flush(si, im);
  block_sum2(sr, si);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sr, si);
}

// Sum partials [0, n) in index order (one CTA), add into *out if accumulate.
__global__ void __launch_bounds__(kThreads) k_final(const double2* part, int n, double2* out, int accumulate) {
  double sr = 0.0, si = 0.0;
  // fixed assignment: thread t sums t, t+256, ... in order
  for (int i = threadIdx.x; i < n; i += kThreads) {
    sr += part[i].x;
    si += part[i].y;
  }
  block_sum2(sr, si);
  if (threadIdx.x == 0) {
    if (accumulate) { out->x += sr; out->y += si; }
    else *out = make_double2(sr, si);
  }
}

// acc += w f, w and f complex double-float
__device__ __forceinline__ void cacc(dfl& sr, dfl& si, dfl wr, dfl wi, dfl fr, dfl fi) {
  df_acc(sr, df_mul(wr, fr));
  df_acc(sr, df_mul(dfl{-wi.h, -wi.l}, fi));
  df_acc(si, df_mul(wr, fi));
  df_acc(si, df_mul(wi, fr));
}

template <typename R> struct AmpV;
template <> struct AmpV<float> { typedef float2 T; };
template <> struct AmpV<double> { typedef double2 T; };

template <typename R>
__global__ void __launch_bounds__(kThreads) k_pauli(const R* __restrict__ a, int n, const __grid_constant__ PauliGroup g,
                                                    double2* part) {
  typedef typename AmpV<R>::T A;
  const A* av = reinterpret_cast<const A*>(a);
  double sr = 0.0, si = 0.0;
  dfl ar{0.f, 0.f}, ai{0.f, 0.f};
  const u64 N = u64(1) << n;
  const u64 stride = (u64)gridDim.x * kThreads;
  u64 i = (u64)blockIdx.x * kThreads + threadIdx.x;
  if (g.m == 0) {
    // sum_x |a_x|^2 f(x); kU elements per iteration, loads first
    auto term = [&](u64 x, A v) {
      const dfl xr = to_df(v.x), xi = to_df(v.y);
      dfl fr, fi;
      fval_df(g, x, fr, fi);
      dfl w = df_mul(xr, xr);
      df_acc(w, df_mul(xi, xi));
      df_acc(ar, df_mul(w, fr));
      df_acc(ai, df_mul(w, fi));
    };
    for (; i + (kU - 1) * stride < N; i += kU * stride) {
      A v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) v[u] = av[i + u * stride];
#pragma unroll
      for (int u = 0; u < kU; ++u) term(i + u * stride, v[u]);
      df_flush(sr, ar);
      df_flush(si, ai);
    }
    for (; i < N; i += stride) term(i, av[i]);
  } else {
    // pairs {x, y = x ^ m}, x with bit h clear:
    //   conj(a_y) a_x f(x) + conj(a_x) a_y f(y)
    const u64 half = N >> 1;
    const u64 lo_mask = (u64(1) << g.h) - 1;
    auto xof = [&](u64 k) { return ((k & ~lo_mask) << 1) | (k & lo_mask); };
    auto term = [&](u64 x, A vx, A vy) {
      const dfl xr = to_df(vx.x), xi = to_df(vx.y), yr = to_df(vy.x), yi = to_df(vy.y);
      // conj(a_y) a_x = (yr xr + yi xi) + i (yr xi - yi xr); conj(a_x) a_y is its conjugate
      dfl pr = df_mul(yr, xr), pi = df_mul(yr, xi);
      df_acc(pr, df_mul(yi, xi));
      df_acc(pi, df_mul(dfl{-yi.h, -yi.l}, xr));
      dfl fr, fi;
      fval_df(g, x, fr, fi);
      cacc(ar, ai, pr, pi, fr, fi);
      fval_df(g, x ^ g.m, fr, fi);
      cacc(ar, ai, pr, dfl{-pi.h, -pi.l}, fr, fi);
    };
    // one term: f(y) = s_m f(x), s_m = (-1)^popcount(m & z), so the pair gives
    // w s(x) (p + s_m conj(p)) = 2 w s(x) Re p (s_m = 1) or 2 i w s(x) Im p
    const bool one = g.nt == 1;
    const bool sm_odd = one && (__popcll(g.m & g.z[0]) & 1);
    const dfl w_r{2.f * g.wrh[0], 2.f * g.wrl[0]}, w_i{2.f * g.wih[0], 2.f * g.wil[0]};
    auto term1 = [&](u64 x, A vx, A vy) {
      const dfl xr = to_df(vx.x), xi = to_df(vx.y), yr = to_df(vy.x), yi = to_df(vy.y);
      dfl c;
      if (!sm_odd) {  // Re p = yr xr + yi xi
        c = df_mul(yr, xr);
        df_acc(c, df_mul(yi, xi));
      } else {        // Im p = yr xi - yi xr
        c = df_mul(yr, xi);
        df_acc(c, df_mul(dfl{-yi.h, -yi.l}, xr));
      }
      if (__popcll(x & g.z[0]) & 1) c = dfl{-c.h, -c.l};
      if (!sm_odd) {  // (w_r + i w_i) c
        df_acc(ar, df_mul(w_r, c));
        df_acc(ai, df_mul(w_i, c));
      } else {        // (w_r + i w_i) i c
        df_acc(ar, df_mul(dfl{-w_i.h, -w_i.l}, c));
        df_acc(ai, df_mul(w_r, c));
      }
    };
    for (; i + (kU - 1) * stride < half; i += kU * stride) {
      A vx[kU], vy[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const u64 x = xof(i + u * stride);
        vx[u] = av[x];
        vy[u] = av[x ^ g.m];
      }
      if (one) {
#pragma unroll
        for (int u = 0; u < kU; ++u) term1(xof(i + u * stride), vx[u], vy[u]);
      } else {
#pragma unroll
        for (int u = 0; u < kU; ++u) term(xof(i + u * stride), vx[u], vy[u]);
      }
      df_flush(sr, ar);
      df_flush(si, ai);
    }
    for (; i < half; i += stride) {
      const u64 x = xof(i);
      if (one) term1(x, av[x], av[x ^ g.m]);
      else term(x, av[x], av[x ^ g.m]);
    }
  }
  df_flush(sr, ar);
  df_flush(si, ai);
  block_sum2(sr, si);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sr, si);
}

// ---- tile passes shared by several groups ----------------------------------
constexpr int kTL = 4;          // low qubits of every expectation tile (runs of 16 amplitudes)
constexpr int kTH = 9;          // at most this many chosen higher qubits per tile (8 for complex128)
constexpr int kPassGroups = 16; // groups per tile pass

constexpr int kTileThreads64 = 512;  // complex64 tile passes: CTA size
constexpr int kStageThreads = 256;   // ... in two warp groups, each running its own register stages
constexpr int kStageBits = 5;        // at most this many bits per register stage
constexpr int kStageBits128 = 4;     // ... for complex128 (16-byte amplitudes)

// A register stage of a complex64 tile pass: single-term groups on up to
// kStageBits tile-local bits (X or Y on one qubit, Z only on that qubit).
// Thread t holds the 2^nb amplitudes e | c, c over the stage bits, for e =
// t's index bits placed at the tile bits tb[] plus each subset of the tile
// bits dhi.  The lane bits tb[0..3] give the 16 lanes of a half warp
// (8-byte reads) or the 8 lanes of a quarter warp (16-byte pair reads, in
// stages holding bit 0) distinct banks of the swizzled tile.
struct XStage {
  int8_t nb, pair, gen, ntb;  // bits; bit 0 among them; some Y term; thread-index bits used
  int8_t grp;                 // the warp group that runs the stage
  int8_t odd;                 // bit j: bit j's term is Y (Im of the pair products)
  int8_t slot0;               // first accumulator slot of the stage's bits
  int8_t bit[kStageBits];     // ascending tile-local bits
  int8_t gg[kStageBits];      // the group slot of each bit
  int8_t tb[10];              // tile bit of thread-index bit i
  unsigned dhi;               // the tile bits each thread enumerates
};

struct PTilePass {
  int L, r;                    // tile = L low qubits + r high qubits H[0..r)
  int H[kTH];
  Ins tins;                    // zero insertion at the high qubits (the tile base)
  int ng;
  int gi[kPassGroups];         // groups of this pass (indices into the group array)
  int hloc[kPassGroups];       // highest tile-local bit of the group's mask (-1: diagonal group)
  unsigned mloc[kPassGroups];  // the group's X/Y mask in tile-local bits
  // complex64 register stages: single-term groups on one tile-local bit
  // with no Z bit outside it, evaluated from 2^nb amplitudes held in
  // registers (the other groups loop over the tile)
  int nst, nsg;     // stages; staged groups (accumulator slots)
  XStage st[kPassGroups];
  unsigned staged;  // bit gg: group slot gg is evaluated in a stage
  int ngen;         // the other group slots, in order
  int8_t genl[kPassGroups];
  int allst;        // every group staged: no per-amplitude group loop
  int clsg;         // complex64: slot of the Z-class group (-1: none), summed across tiles
  int ggrp;         // complex64: the warp group running the non-staged groups (-1: all threads)
  u64 fmask;        // the qubits outside the tile (the tile base's bits)
  int noflush;      // complex64: only staged and Z-class groups (no per-tile FP64 flush)
  // complex64 tiles by TMA (tma != 0): dimension d of the tensor map is a
  // run of qubits; tgb[d] >= 0: a run outside the tile, coordinate = bits
  // tgb[d] .. tgb[d] + tlen[d] - 1 of the tile number
  int tma, trank;
  int8_t tgb[5], tlen[5];
};

// A TMA tile wait that gave up (about 1 s): reported by qs_expect_pauli.
__device__ int g_expect_timeout;

// h + l renormalised (the accumulators' low parts gather unnormalised error terms)
__device__ __forceinline__ dfl df_norm2(dfl a) {
  dfl r;
  r.h = fast_two_sum(a.h, a.l, r.l);
  return r;
}

// Tile-local index l (bits [0, L) = qubits [0, L), bit L + j = qubit H[j]) to
// the global index, given the tile base F.
__device__ __forceinline__ u64 ptile_global(u64 F, const u64* spreadH, int L, unsigned l) {
  return F | (u64)(l & ((1u << L) - 1)) | spreadH[l >> L];
}

// A tile amplitude in shared memory: complex64 as it is, complex128 as its
// double-float split (converted once per tile, not once per group).
template <typename R> struct TileAmp;
template <> struct TileAmp<float> {
  typedef float2 T;
  // XOR swizzle of the 16-byte pieces (amplitude pairs) of the tile's
  // 16-amplitude (128-byte) rows: strided reads of the register stages stay
  // free of bank conflicts, and a pair stays whole for 16-byte copies
  __host__ __device__ static unsigned sw(unsigned e) { return e ^ (((e >> 4) & 7u) << 1); }
  __device__ static T from(float2 v) { return v; }
  __device__ static void get(const T& v, dfl& re, dfl& im) {
    re = dfl{v.x, 0.f};
    im = dfl{v.y, 0.f};
  }
};
template <> struct TileAmp<double> {
  typedef float4 T;
  // XOR swizzle of the 16-byte amplitudes of the tile's 8-amplitude
  // (128-byte) rows: strided reads of the register stages stay free of bank
  // conflicts
  __host__ __device__ static unsigned sw(unsigned e) { return e ^ ((e >> 3) & 7u); }
  __device__ static T from(double2 v) {
    const dfl r = d2df(v.x), i = d2df(v.y);
    return make_float4(r.h, r.l, i.h, i.l);
  }
  __device__ static void get(const T& v, dfl& re, dfl& im) {
    re = dfl{v.x, v.y};
    im = dfl{v.z, v.w};
  }
};

__device__ __forceinline__ float2 t_as_f2(float2 v) { return v; }

// Stage S of a complex64 tile pass over the (swizzled) tile t: for each
// stage bit j's group, over the pairs x, x ^ 2^b_j of the tile, Re (and,
// for stages with a Y term, Im) of conj(a_y) a_x in FP32, summed per thread
// into re[j] (im[j]).  swt is the swizzled position of this thread's base
// amplitude.  Positions: the swizzle is linear over XOR, and the enumerated
// bits dhi lie above bit 6, where it is the identity, so the amplitude at
// base | c | cur sits at (swt ^ sw(c)) + cur.
template <int NB, bool PAIR, bool GEN>
__device__ __forceinline__ void x_stage(const float2* __restrict__ t, unsigned swt, const XStage& S,
                                        float (&re)[kStageBits], float (&im)[kStageBits]) {
  const char* tb = reinterpret_cast<const char*>(t);
  unsigned off[1 << NB];  // byte offsets
  off[0] = swt * 8u;
#pragma unroll
  for (int c = 1; c < (1 << NB); ++c) {
    int j = 0;
    while (!((c >> j) & 1)) ++j;
    off[c] = off[c & (c - 1)] ^ (TileAmp<float>::sw(1u << S.bit[j]) * 8u);
  }
  float r0[NB], r1[NB], i0[NB], i1[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) r0[j] = r1[j] = i0[j] = i1[j] = 0.f;
  const unsigned dhi = S.dhi;
  unsigned cur = 0;
  do {
    float2 v[1 << NB];
    if constexpr (PAIR) {
#pragma unroll
      for (int c = 0; c < (1 << NB); c += 2) {
        const float4 w = *reinterpret_cast<const float4*>(tb + off[c] + cur * 8u);
        v[c] = make_float2(w.x, w.y);
        v[c + 1] = make_float2(w.z, w.w);
      }
    } else {
#pragma unroll
      for (int c = 0; c < (1 << NB); ++c) v[c] = *reinterpret_cast<const float2*>(tb + off[c] + cur * 8u);
    }
    // products in pair-major order: consecutive FMAs feed different bits'
    // accumulators (Re: x parts into r0, y parts into r1)
#pragma unroll
    for (int c = 0; c < (1 << NB); ++c) {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if ((c >> j) & 1) continue;
        const float2 X = v[c], Y = v[c | (1 << j)];
        r0[j] = fmaf(Y.x, X.x, r0[j]);
        if constexpr (GEN) i0[j] = fmaf(Y.x, X.y, i0[j]);
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if ((c >> j) & 1) continue;
        const float2 X = v[c], Y = v[c | (1 << j)];
        r1[j] = fmaf(Y.y, X.y, r1[j]);
        if constexpr (GEN) i1[j] = fmaf(-Y.y, X.x, i1[j]);
      }
    }
    cur = ((cur | ~dhi) + 1u) & dhi;  // the next subset of dhi
  } while (cur != 0);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    re[j] = r0[j] + r1[j];
    im[j] = i0[j] + i1[j];
  }
}

template <int NB>
__device__ __forceinline__ void x_stage_any(const float2* t, unsigned swt, const XStage& S, float (&re)[kStageBits],
                                            float (&im)[kStageBits]) {
  if (S.pair) {
    if (S.gen) x_stage<NB, true, true>(t, swt, S, re, im);
    else x_stage<NB, true, false>(t, swt, S, re, im);
  } else {
    if (S.gen) x_stage<NB, false, true>(t, swt, S, re, im);
    else x_stage<NB, false, false>(t, swt, S, re, im);
  }
}

// acc += a b + c d for double-float a, b, c, d (given as high and low
// floats): the high products exact (two-product), the four cross products
// and the two product errors in FP32 into the low part, the high products
// added exactly (TwoSum)
__device__ __forceinline__ void df_dot2_acc(dfl& acc, float ah, float al, float bh, float bl, float ch, float cl,
                                            float dh, float dl) {
  const float p1 = ah * bh, e1 = fmaf(ah, bh, -p1);
  const float p2 = ch * dh, e2 = fmaf(ch, dh, -p2);
  const float lo = fmaf(ah, bl, fmaf(al, bh, fmaf(ch, dl, fmaf(cl, dh, e1 + e2))));
  float t1, t2;
  float h = two_sum(acc.h, p1, t1);
  h = two_sum(h, p2, t2);
  acc.h = h;
  acc.l += lo + (t1 + t2);
}

// Stage S of a complex128 tile pass (amplitudes as double-float (re h, re l,
// im h, im l), swizzled by TileAmp<double>::sw): for each stage qubit j,
// Re (and, with a Y term, Im) of conj(a_y) a_x over this thread's pairs
// x, x ^ 2^b_j, in double-float, two accumulators per qubit.  Positions as
// in x_stage: the swizzle is linear over XOR and the identity above bit 5,
// where the enumerated bits lie.
template <int NB, bool GEN>
__device__ __forceinline__ void x_stage128(const float4* __restrict__ t, unsigned swt, const XStage& S,
                                           dfl (&re)[kStageBits], dfl (&im)[kStageBits]) {
  unsigned off[1 << NB];
  off[0] = swt;
#pragma unroll
  for (int c = 1; c < (1 << NB); ++c) {
    int j = 0;
    while (!((c >> j) & 1)) ++j;
    off[c] = off[c & (c - 1)] ^ TileAmp<double>::sw(1u << S.bit[j]);
  }
  dfl r0[NB], r1[NB], i0[NB], i1[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) r0[j] = r1[j] = i0[j] = i1[j] = dfl{0.f, 0.f};
  const unsigned dhi = S.dhi;
  unsigned cur = 0;
  do {
    float4 v[1 << NB];
#pragma unroll
    for (int c = 0; c < (1 << NB); ++c) v[c] = t[off[c] + cur];
#pragma unroll
    for (int c = 0; c < (1 << NB); ++c) {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if ((c >> j) & 1) continue;
        const float4 X = v[c], Y = v[c | (1 << j)];
        // the pairs of bit j alternate between two accumulators
        const bool second = ((c >> (j == 0 ? 1 : 0)) & 1) != 0;
        dfl& r = second ? r1[j] : r0[j];
        df_dot2_acc(r, Y.x, Y.y, X.x, X.y, Y.z, Y.w, X.z, X.w);  // Re: yr xr + yi xi
        if constexpr (GEN) {
          dfl& q = second ? i1[j] : i0[j];
          df_dot2_acc(q, Y.x, Y.y, X.z, X.w, -Y.z, -Y.w, X.x, X.y);  // Im: yr xi - yi xr
        }
      }
    }
    cur = ((cur | ~dhi) + 1u) & dhi;
  } while (cur != 0);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    re[j] = df_add(r0[j], r1[j]);
    im[j] = df_add(i0[j], i1[j]);
  }
}

template <int NB>
__device__ __forceinline__ void x_stage128_any(const float4* t, unsigned swt, const XStage& S, dfl (&re)[kStageBits],
                                               dfl (&im)[kStageBits]) {
  if (S.gen) x_stage128<NB, true>(t, swt, S, re, im);
  else x_stage128<NB, false>(t, swt, S, re, im);
}

// Shared memory of a tile pass: spreadH, then (complex64) the threads'
// stage positions and their double-float stage sums, then the tile
// buffer(s).
__host__ __device__ constexpr size_t ptile_stage_off() { return sizeof(u64) * (size_t(1) << kTH); }
__host__ __device__ constexpr size_t ptile_acc_off(int nst, int nt) {
  return ptile_stage_off() + ((sizeof(uint16_t) * (size_t)nst * (size_t)nt + 15) / 16) * 16;
}
__host__ __device__ constexpr size_t ptile_buf_off(int nst, int nsg, int nt) {
  return ptile_acc_off(nst, nt) + sizeof(float2) * (size_t)nsg * (size_t)nt;
}
constexpr size_t kPtileAlign = 1024;  // the tile buffers' alignment (128-byte swizzle period)
// complex128 stage slots go to FP64 every kSlotTiles tiles: the low float of
// a slot then rounds at most kSlotTiles times its own size, ~2^-44 of the
// summed term magnitudes
constexpr int kSlotTiles = 16;

// ALLST: a complex64 pass whose groups are all in register stages (no
// per-amplitude group code in that instance).
template <typename R, int NT, bool ALLST = false>
__global__ void __launch_bounds__(NT, (std::is_same<R, float>::value ? 1 : 2)) k_pauli_tiles(const R* __restrict__ a, int n,
                                                    const __grid_constant__ PTilePass P,
                                                    const __grid_constant__ CUtensorMap tmap,
                                                    const PauliGroup* __restrict__ groups, double2* part) {
  typedef typename AmpV<R>::T A;
  typedef TileAmp<R> TA;
  typedef typename TA::T E;
  // complex64 single-term and Z-class groups: FP32 products and per-tile
  // FP32 sums (see qs_expect_pauli); complex128 and the other group kinds:
  // exact products in double-float
  constexpr bool kF32 = std::is_same<R, float>::value;
  extern __shared__ __align__(16) unsigned char psm[];
  u64* spreadH = reinterpret_cast<u64*>(psm);             // [2^r]
  constexpr int ST = kStageThreads;
  const unsigned lt = threadIdx.x % ST, grp = threadIdx.x / ST;  // complex64 stages: thread within its warp group
  uint16_t* swt = reinterpret_cast<uint16_t*>(psm + ptile_stage_off());  // [nst][ST]
  float2* sacc = reinterpret_cast<float2*>(psm + ptile_acc_off(P.nst, ST));  // [nsg][ST] (hi, lo)
  __shared__ __align__(8) uint64_t pmbar[2];  // TMA tiles: buffer b filled
  // the Z-class parameters of the pass's class group, read once
  __shared__ struct {
    u64 mask[kMaxClasses];
    int d[kMaxClasses], len[kMaxClasses];
  } ctab;
  const size_t boff = ptile_buf_off(P.nst, P.nsg, ST);
  const uint32_t sbase = smem_u32(psm);
  // (complex64 only: its launch adds kPtileAlign bytes for this pad)
  const size_t bpad = kF32 ? (kPtileAlign - ((sbase + boff) & (kPtileAlign - 1))) & (kPtileAlign - 1) : 0;
  E* const t0 = reinterpret_cast<E*>(psm + boff + bpad);  // [2^(L + r)] (complex64: two)
  E* t = t0;
  const bool use_tma = kF32 && P.tma;
  if (use_tma && threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&pmbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&pmbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const A* av = reinterpret_cast<const A*>(a);
  const int L = P.L, r = P.r, m = L + r;
  const unsigned tile = 1u << m;
  for (unsigned i = threadIdx.x; i < (1u << r); i += NT) {
    u64 sp = 0;
    for (int j = 0; j < r; ++j)
      if ((i >> j) & 1u) sp |= u64(1) << P.H[j];
    spreadH[i] = sp;
  }
  for (int si = 0; si < P.nst; ++si) {  // this thread's swizzled base position in its group's stages
    if (P.st[si].grp != (int)grp) continue;
    unsigned d = 0;
    for (int i = 0; i < P.st[si].ntb; ++i)
      if ((lt >> i) & 1u) d |= 1u << P.st[si].tb[i];
    swt[si * ST + lt] = (uint16_t)TA::sw(d);
    for (int j = 0; j < P.st[si].nb; ++j) sacc[(P.st[si].slot0 + j) * ST + lt] = make_float2(0.f, 0.f);
  }
  if (kF32 && P.clsg >= 0 && threadIdx.x < kMaxClasses) {
    const PauliGroup& cg = groups[P.gi[P.clsg]];
    ctab.mask[threadIdx.x] = cg.cls_mask[threadIdx.x];
    ctab.d[threadIdx.x] = cg.cls_d[threadIdx.x];
    ctab.len[threadIdx.x] = cg.cls_len[threadIdx.x];
  }
  const u64 ntiles = u64(1) << (n - m);
  double sr = 0.0, si = 0.0;
  dfl ar{0.f, 0.f}, ai{0.f, 0.f};
  // complex64: two tile buffers, the next tile's 16-byte pieces copied
  // asynchronously (cp.async) while the current one is evaluated
  auto copy_tile = [&](u64 ti, int buf) {
    const u64 F = expand(ti << L, P.tins);
    const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(t0) + (uint32_t)buf * tile * (uint32_t)sizeof(E);
    for (unsigned c2 = threadIdx.x; c2 < tile / 2; c2 += NT) {
      const unsigned e = 2 * c2;
      const A* src = av + ptile_global(F, spreadH, L, e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + TA::sw(e) * (uint32_t)sizeof(E)), "l"(src)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // ... or (thread 0) one TMA box: the tile's rows of 16 amplitudes with the
  // 128-byte swizzle, which is TileAmp<float>::sw
  auto tma_tile = [&](u64 ti, int buf) {
    int c[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int d = 0; d < 5; ++d)
      if (d < P.trank && P.tgb[d] >= 0) c[d] = (int)((ti >> P.tgb[d]) & ((u64(1) << P.tlen[d]) - 1));
    const uint32_t mb = smem_u32(&pmbar[buf]);
    const uint32_t dst = smem_u32(t0) + (uint32_t)buf * tile * (uint32_t)sizeof(E);
    mbar_expect_tx(mb, tile * (uint32_t)sizeof(E));
    if (P.trank == 3) tma_load_3d(dst, &tmap, c[0], c[1], c[2], mb);
    else if (P.trank == 4) tma_load_4d(dst, &tmap, c, mb);
    else if (P.trank == 5) tma_load_5d(dst, &tmap, c, mb);
    else tma_load_2d(dst, &tmap, c[0], c[1], mb);
  };
  __syncthreads();
  if constexpr (kF32) {
    if ((u64)blockIdx.x < ntiles) {
      if (!use_tma) copy_tile(blockIdx.x, 0);
      else if (threadIdx.x == 0) tma_tile(blockIdx.x, 0);
    }
  }
  // the stage sums, weighted, into the FP64 accumulators: 2 w Re p for
  // X-type terms, 2 i w Im p for Y-type; the slots restart from zero
  auto flush_slots = [&]() {
    for (int sx = 0; sx < P.nst; ++sx) {
      const XStage& S = P.st[sx];
      if (S.grp != (int)grp) continue;
      for (int j = 0; j < S.nb; ++j) {
        float2& a = sacc[(S.slot0 + j) * ST + lt];
        const PauliGroup& g = groups[P.gi[S.gg[j]]];
        const dfl c = df_norm2(dfl{a.x, a.y});
        a = make_float2(0.f, 0.f);
        const dfl w_r{2.f * g.wrh[0], 2.f * g.wrl[0]}, w_i{2.f * g.wih[0], 2.f * g.wil[0]};
        if (!((S.odd >> j) & 1)) {
          df_acc(ar, df_mul(w_r, c));
          df_acc(ai, df_mul(w_i, c));
        } else {
          df_acc(ar, df_mul(dfl{-w_i.h, -w_i.l}, c));
          df_acc(ai, df_mul(w_r, c));
        }
      }
    }
    df_flush(sr, ar);
    df_flush(si, ai);
  };
  // complex64 Z-class sums over the thread's tiles (there is one diagonal
  // group, so at most one class group per pass)
  dfl csum[kMaxClasses];
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) csum[c] = dfl{0.f, 0.f};
  // the non-staged groups: all threads, or (complex64 passes with stages)
  // one warp group while the other runs its stages
  const bool gsplit = kF32 && P.ggrp >= 0;
  const unsigned gt = gsplit ? lt : threadIdx.x, gN = gsplit ? (unsigned)ST : (unsigned)NT;
  const bool gmine = !gsplit || (int)grp == P.ggrp;
  const bool need_F = !(kF32 && (ALLST || P.allst));
  // tile base: the tile number's bits at the qubits outside the tile,
  // advanced by gridDim.x tiles with a masked add (carries skip the tile's
  // qubits)
  u64 F = need_F ? expand((u64)blockIdx.x << L, P.tins) : 0;
  const u64 Fstep = need_F ? expand((u64)gridDim.x << L, P.tins) : 0;
  int it = 0;
  for (u64 ti = blockIdx.x; ti < ntiles; ti += gridDim.x, ++it, F = ((F | ~P.fmask) + Fstep) & P.fmask) {
    if (use_tma) {
      if (threadIdx.x == 0 && ti + gridDim.x < ntiles) tma_tile(ti + gridDim.x, (it + 1) & 1);
      const bool bad = !mbar_wait(smem_u32(&pmbar[it & 1]), (it >> 1) & 1);
      if (__syncthreads_or(bad)) {
        // a copy that never arrived: flag it, give the next tile's copy a
        // bounded wait, and leave without a partial sum
        if (threadIdx.x == 0) {
          atomicExch(&g_expect_timeout, 1);
          if (ti + gridDim.x < ntiles) mbar_wait(smem_u32(&pmbar[(it + 1) & 1]), ((it + 1) >> 1) & 1);
        }
        return;
      }
      t = t0 + (size_t)(it & 1) * tile;
    } else if constexpr (kF32) {
      if (ti + gridDim.x < ntiles) {
        copy_tile(ti + gridDim.x, (it + 1) & 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      t = t0 + (size_t)(it & 1) * tile;
    } else {
      // the tile into shared memory, 4 loads in flight per thread
      for (unsigned e0 = threadIdx.x; e0 < tile; e0 += 4 * NT) {
        A v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned e = e0 + u * NT;
          if (e < tile) v[u] = av[ptile_global(F, spreadH, L, e)];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned e = e0 + u * NT;
          if (e < tile) t[TA::sw(e)] = TA::from(v[u]);
        }
      }
    }
    if (!use_tma) __syncthreads();
    for (int sx = 0; sx < P.nst; ++sx) {
      const XStage& S = P.st[sx];
      if (S.grp != (int)grp || (lt >> S.ntb)) continue;  // another group's; or small tiles: fewer sets than threads
      const int nb = S.nb;
      const unsigned sb = swt[sx * ST + lt];
      if constexpr (kF32) {
        float re[kStageBits], im[kStageBits];
        const float2* tf = reinterpret_cast<const float2*>(t);
        if (nb == 5) x_stage_any<5>(tf, sb, S, re, im);
        else if (nb == 4) x_stage_any<4>(tf, sb, S, re, im);
        else if (nb == 3) x_stage_any<3>(tf, sb, S, re, im);
        else if (nb == 2) x_stage_any<2>(tf, sb, S, re, im);
        else x_stage_any<1>(tf, sb, S, re, im);
        // this tile's FP32 sums into the thread's double-float slots
        // (exact: TwoSum), weighted once at the end
#pragma unroll
        for (int j = 0; j < kStageBits; ++j) {
          if (j >= nb) break;
          float2& a = sacc[(S.slot0 + j) * ST + lt];
          float2 v = a, e;
          v.x = two_sum(v.x, ((S.odd >> j) & 1) ? im[j] : re[j], e.x);
          v.y += e.x;
          a = v;
        }
      } else {
        dfl re[kStageBits], im[kStageBits];
        const float4* tf = reinterpret_cast<const float4*>(t);
        if (nb == 4) x_stage128_any<4>(tf, sb, S, re, im);
        else if (nb == 3) x_stage128_any<3>(tf, sb, S, re, im);
        else if (nb == 2) x_stage128_any<2>(tf, sb, S, re, im);
        else x_stage128_any<1>(tf, sb, S, re, im);
        // this tile's double-float sums into the thread's slots (high parts
        // exactly, TwoSum), weighted and flushed to FP64 every kSlotTiles
        // tiles
#pragma unroll
        for (int j = 0; j < kStageBits128; ++j) {
          if (j >= nb) break;
          float2& a = sacc[(S.slot0 + j) * ST + lt];
          const dfl c = ((S.odd >> j) & 1) ? im[j] : re[j];
          float2 v = a;
          float e;
          v.x = two_sum(v.x, c.h, e);
          v.y += c.l + e;
          a = v;
        }
      }
    }
    for (int gq = 0; !ALLST && need_F && gmine && gq < P.ngen; ++gq) {
      const int gg = P.genl[gq];
      const PauliGroup& g = groups[P.gi[gg]];
      const int h = P.hloc[gg];
      if (h < 0 && g.ncls > 0) {
        // Z-only two-bit terms in classes: f(x) = sum_c w_c k_c(x) with
        // integer k_c, so sum_x p_x f(x) = sum_c w_c sum_x p_x k_c(x): the
        // inner sums are formed first, one double-float chain per class
        const int nc = g.ncls;
        dfl sc[kMaxClasses];
#pragma unroll
        for (int c = 0; c < kMaxClasses; ++c) sc[c] = dfl{0.f, 0.f};
        if constexpr (kF32) {
          // complex64, by rows of 16 amplitudes, in FP32 per thread and
          // tile, then one double-float step per class.  V(x) = (x ^ x >> d)
          // & mask is linear over GF(2), so for a row base xr (bits 0..3
          // clear) and j < 16, V(xr | j) = V(xr) ^ V(j) with V(j) inside
          // bits 0..3: k = base - 2 popc(u_j), base = len - 2 popc(V(xr)
          // above bit 3), u_j = (V(xr) ^ V(j)) & 15, and the row adds
          // base * sum_j p_j - 2 sum_j p_j popc(u_j)
          float s2[kMaxClasses];
#pragma unroll
          for (int c = 0; c < kMaxClasses; ++c) s2[c] = 0.f;
          const float4* t4 = reinterpret_cast<const float4*>(t);
          for (unsigned rho = gt; rho < (tile >> kTL); rho += gN) {
            const u64 xr = F | spreadH[rho];
            float pj[16];
#pragma unroll
            for (int q = 0; q < 8; ++q) {  // the row's 16-byte pieces, unswizzled
              const float4 w = t4[rho * 8 + (q ^ (rho & 7))];
              pj[2 * q] = fmaf(w.x, w.x, w.y * w.y);
              pj[2 * q + 1] = fmaf(w.z, w.z, w.w * w.w);
            }
            float pr[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) pr[q] = pj[2 * q] + pj[2 * q + 1];
            const float prow = ((pr[0] + pr[1]) + (pr[2] + pr[3])) + ((pr[4] + pr[5]) + (pr[6] + pr[7]));
#pragma unroll
            for (int c = 0; c < kMaxClasses; ++c) {
              if (c >= nc) break;
              // (the pass's class group from the shared table; another one,
              // a diagonal group split for its size, from its own record)
              const bool tab = gg == P.clsg;
              const int d = tab ? ctab.d[c] : g.cls_d[c];
              const u64 mk = tab ? ctab.mask[c] : g.cls_mask[c];
              const u64 V = (xr ^ (xr >> d)) & mk;
              const float base = (float)((tab ? ctab.len[c] : g.cls_len[c]) - 2 * __popcll(V & ~u64(15)));
              unsigned bv[4];  // V(2^b), b < 4
#pragma unroll
              for (int b = 0; b < 4; ++b) bv[b] = ((1u << b) ^ (d < 4 ? (1u << b) >> d : 0u)) & (unsigned)mk & 15u;
              unsigned u[16];
              u[0] = (unsigned)V & 15u;
              float a0 = 0.f, a1 = 0.f;
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                if (j) {
                  int b = 0;
                  while (!((j >> b) & 1)) ++b;
                  u[j] = u[j & (j - 1)] ^ bv[b];
                }
                if (j & 1) a1 = fmaf(pj[j], (float)__popc(u[j]), a1);
                else a0 = fmaf(pj[j], (float)__popc(u[j]), a0);
              }
              s2[c] = fmaf(base, prow, fmaf(-2.f, a0 + a1, s2[c]));
            }
          }
#pragma unroll
          for (int c = 0; c < kMaxClasses; ++c) {
            // the pass's first class group: into the thread's double-float
            // class sums (exact: TwoSum), weighted once at the end; any
            // other (a diagonal group split for its size): weighted per tile
            if (c >= nc) break;
            if (gg == P.clsg) {
              float e;
              csum[c].h = two_sum(csum[c].h, s2[c], e);
              csum[c].l += e;
            } else {
              sc[c] = dfl{s2[c], 0.f};
            }
          }
        } else {
          for (unsigned l = gt; l < tile; l += gN) {
            dfl xr, xi;
            TA::get(t[TA::sw(l)], xr, xi);
            dfl pw = df_mul(xr, xr);
            df_acc(pw, df_mul(xi, xi));
            const u64 x = ptile_global(F, spreadH, L, l);
#pragma unroll
            for (int c = 0; c < kMaxClasses; ++c) {
              if (c >= nc) break;
              const float k = (float)(g.cls_len[c] - 2 * __popcll((x ^ (x >> g.cls_d[c])) & g.cls_mask[c]));
              df_acc(sc[c], df_mul(pw, dfl{k, 0.f}));
            }
          }
        }
#pragma unroll
        for (int c = 0; c < kMaxClasses; ++c) {
          if ((kF32 && gg == P.clsg) || c >= nc) break;
          const dfl v = df_norm2(sc[c]);
          df_acc(ar, df_mul(dfl{g.cwrh[c], g.cwrl[c]}, v));
          df_acc(ai, df_mul(dfl{g.cwih[c], g.cwil[c]}, v));
        }
      } else if (h < 0) {  // diagonal group: sum_x |a_x|^2 f(x)
        int since = 0;  // flush the double-float sums into FP64 every kU terms
        for (unsigned l = gt; l < tile; l += gN) {
          dfl xr, xi;
          TA::get(t[TA::sw(l)], xr, xi);
          dfl fr, fi;
          fval_df(g, ptile_global(F, spreadH, L, l), fr, fi);
          dfl w = df_mul(xr, xr);
          df_acc(w, df_mul(xi, xi));
          df_acc(ar, df_mul(w, fr));
          df_acc(ai, df_mul(w, fi));
          if (++since == kU) {
            df_flush(sr, ar);
            df_flush(si, ai);
            since = 0;
          }
        }
      } else if (g.nt == 1) {
        // one term: the pair {x, y = x ^ m} gives 2 w s(x) Re p (m and z of
        // even overlap) or 2 i w s(x) Im p, p = conj(a_y) a_x; the sum of
        // s(x) Re p (or Im p) over this thread's pairs is formed first, in
        // four independent double-float chains, and weighted once
        const unsigned mloc = P.mloc[gg], lo_mask = (1u << h) - 1u;
        const u64 z0 = g.z[0];
        const bool sm_odd = __popcll(g.m & z0) & 1;
        dfl c;
        if constexpr (kF32) {
          // complex64: each pair's Re / Im p in FP32 (one FMA), summed in
          // FP32 over this thread's pairs of the tile in four chains
          float c4[4] = {0.f, 0.f, 0.f, 0.f};
          for (unsigned k0 = gt; k0 < tile / 2; k0 += 4 * gN) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const unsigned k = k0 + u * gN;
              if (k >= tile / 2) break;
              const unsigned l = ((k & ~lo_mask) << 1) | (k & lo_mask);  // bit h clear
              const float2 X = t_as_f2(t[TA::sw(l)]), Y = t_as_f2(t[TA::sw(l ^ mloc)]);
              float cv = !sm_odd ? fmaf(Y.x, X.x, Y.y * X.y) : fmaf(Y.x, X.y, -(Y.y * X.x));
              if (z0 && (__popcll(ptile_global(F, spreadH, L, l) & z0) & 1)) cv = -cv;
              c4[u] += cv;
            }
          }
          c = dfl{(c4[0] + c4[1]) + (c4[2] + c4[3]), 0.f};
        } else {
          dfl c4[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
          for (unsigned k0 = gt; k0 < tile / 2; k0 += 4 * gN) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const unsigned k = k0 + u * gN;
              if (k >= tile / 2) break;
              const unsigned l = ((k & ~lo_mask) << 1) | (k & lo_mask);  // bit h clear
              dfl xr, xi, yr, yi;
              TA::get(t[TA::sw(l)], xr, xi);
              TA::get(t[TA::sw(l ^ mloc)], yr, yi);
              dfl cc;
              if (!sm_odd) {
                cc = df_mul(yr, xr);
                df_acc(cc, df_mul(yi, xi));
              } else {
                cc = df_mul(yr, xi);
                df_acc(cc, df_mul(dfl{-yi.h, -yi.l}, xr));
              }
              if (z0 && (__popcll(ptile_global(F, spreadH, L, l) & z0) & 1)) cc = dfl{-cc.h, -cc.l};
              df_acc(c4[u], cc);
            }
          }
          c = df_add(df_add(df_norm2(c4[0]), df_norm2(c4[1])), df_add(df_norm2(c4[2]), df_norm2(c4[3])));
        }
        const dfl w_r{2.f * g.wrh[0], 2.f * g.wrl[0]}, w_i{2.f * g.wih[0], 2.f * g.wil[0]};
        if (!sm_odd) {
          df_acc(ar, df_mul(w_r, c));
          df_acc(ai, df_mul(w_i, c));
        } else {
          df_acc(ar, df_mul(dfl{-w_i.h, -w_i.l}, c));
          df_acc(ai, df_mul(w_r, c));
        }
      } else {
        const unsigned mloc = P.mloc[gg], lo_mask = (1u << h) - 1u;
        int since = 0;
        for (unsigned k = gt; k < tile / 2; k += gN) {
          const unsigned l = ((k & ~lo_mask) << 1) | (k & lo_mask);  // bit h clear
          dfl xr, xi, yr, yi;
          TA::get(t[TA::sw(l)], xr, xi);
          TA::get(t[TA::sw(l ^ mloc)], yr, yi);
          const u64 x = ptile_global(F, spreadH, L, l);
          dfl pr = df_mul(yr, xr), pi = df_mul(yr, xi);
          df_acc(pr, df_mul(yi, xi));
          df_acc(pi, df_mul(dfl{-yi.h, -yi.l}, xr));
          dfl fr, fi;
          fval_df(g, x, fr, fi);
          cacc(ar, ai, pr, pi, fr, fi);
          fval_df(g, x ^ g.m, fr, fi);
          cacc(ar, ai, pr, dfl{-pi.h, -pi.l}, fr, fi);
          if (++since == kU) {
            df_flush(sr, ar);
            df_flush(si, ai);
            since = 0;
          }
        }
      }
    }
    if (!kF32 && P.nst > 0 && (it % kSlotTiles) == kSlotTiles - 1) flush_slots();
    // into FP64 once per tile (the FP64 pipe is about 1/64 of FP32 on GB300)
    if (!ALLST && !(kF32 && P.noflush)) {
      df_flush(sr, ar);
      df_flush(si, ai);
    }
    __syncthreads();
  }
  flush_slots();
  if constexpr (kF32) {
    if (!ALLST && P.clsg >= 0) {  // the class sums, weighted
      const PauliGroup& g = groups[P.gi[P.clsg]];
#pragma unroll
      for (int c = 0; c < kMaxClasses; ++c) {
        if (c >= g.ncls) break;
        const dfl v = df_norm2(csum[c]);
        df_acc(ar, df_mul(dfl{g.cwrh[c], g.cwrl[c]}, v));
        df_acc(ai, df_mul(dfl{g.cwih[c], g.cwil[c]}, v));
      }
    }
    df_flush(sr, ar);
    df_flush(si, ai);
  }
  block_sum2<NT>(sr, si);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sr, si);
}

qs_status read_result(qs_state* s, const double2* dev, double2* host) {
  cudaError_t e = cudaMemcpyAsync(s->pinned, dev, sizeof(double2), cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reduction readback");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reduction sync");
  host->x = s->pinned[0];
  host->y = s->pinned[1];
  return QS_OK;
}

}  // namespace

qs_status run_norm2(qs_state* s, double* out) {
  const int LA = s->dtype == QS_C64 ? 1 : 0;
  const u64 npk = u64(1) << (s->n - LA);
  const unsigned g = red_grid(npk);
  qs_status st = ensure_scratch(s, sizeof(double2) * (g + 1));
  if (st != QS_OK) return st;
  double2* part = static_cast<double2*>(s->scratch);
  double2* res = part + g;
  if (s->dtype == QS_C64) k_norm2<float><<<g, kThreads, 0, s->stream>>>(static_cast<const float*>(s->amp), npk, part);
  else k_norm2<double><<<g, kThreads, 0, s->stream>>>(static_cast<const double*>(s->amp), npk, part);
  if ((st = launch_ok("k_norm2")) != QS_OK) return st;
  k_final<<<1, kThreads, 0, s->stream>>>(part, g, res, 0);
  if ((st = launch_ok("k_final")) != QS_OK) return st;
  double2 h{0.0, 0.0};
  if ((st = read_result(s, res, &h)) != QS_OK) return st;
  *out = h.x;
  return QS_OK;
}

qs_status run_inner(qs_state* a, qs_state* b, double out[2]) {
  if (a->amp == b->amp) {  // the same vector: <a|a> = the norm, one read of the state
    double v = 0.0;
    const qs_status st = run_norm2(a, &v);
    out[0] = v;
    out[1] = 0.0;
    return st;
  }
  const int LA = a->dtype == QS_C64 ? 1 : 0;
  const u64 npk = u64(1) << (a->n - LA);
  const unsigned g = red_grid(npk);
  qs_status st = ensure_scratch(a, sizeof(double2) * (g + 1));
  if (st != QS_OK) return st;
  // b's pending work must be complete before a's stream reads it
  if (b->stream != a->stream) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qs_inner: sync b");
  }
  double2* part = static_cast<double2*>(a->scratch);
  double2* res = part + g;
  if (a->dtype == QS_C64)
    k_inner<float><<<g, kThreads, 0, a->stream>>>(static_cast<const float*>(a->amp), static_cast<const float*>(b->amp), npk, part);
  else
    k_inner<double><<<g, kThreads, 0, a->stream>>>(static_cast<const double*>(a->amp), static_cast<const double*>(b->amp), npk, part);
  if ((st = launch_ok("k_inner")) != QS_OK) return st;
  k_final<<<1, kThreads, 0, a->stream>>>(part, g, res, 0);
  if ((st = launch_ok("k_final")) != QS_OK) return st;
  double2 h{0.0, 0.0};
  if ((st = read_result(a, res, &h)) != QS_OK) return st;
  out[0] = h.x;
  out[1] = h.y;
  return QS_OK;
}

// Register stages of a complex64 tile pass.  The single-term groups on one
// tile-local bit (X or Y, Z on that bit only) are placed first fit, in
// ascending bit order, into stages of at most kStageBits bits; a stage never
// holds both bits j and j + 3 (j = 1..3), which the swizzle folds onto the
// same bank position.  Lane bits: bit 0 (unless a stage bit: then pairs are
// read as 16 bytes) and, for j = 1..3, bit j or else bit j + 3; then the
// other tile bits ascending.
// Complex128 (c128): 16-byte amplitudes, swizzle e ^ ((e >> 3) & 7): the
// clash pairs are j, j + 3 for j = 0..2, the lanes of a quarter warp take
// qubit j or j + 3, stages hold at most kStageBits128 qubits, one warp group.
void build_stages(PTilePass& q, const std::vector<PauliGroup>& groups, int nt, bool c128) {
  const int m = q.L + q.r;
  const int jlo = c128 ? 0 : 1, jhi = c128 ? 2 : 3, maxnb = c128 ? kStageBits128 : kStageBits;
  int lg_nt = 0;
  while ((1 << lg_nt) < nt) ++lg_nt;
  std::vector<std::pair<int, int>> one;  // (local bit, group slot)
  for (int gg = 0; gg < q.ng; ++gg) {
    const PauliGroup& G = groups[q.gi[gg]];
    if (G.nt == 1 && __builtin_popcount(q.mloc[gg]) == 1 && (G.z[0] & ~G.m) == 0) one.push_back({q.hloc[gg], gg});
  }
  std::sort(one.begin(), one.end());
  std::vector<unsigned> smask;
  for (const auto& bg : one) {
    const int b = bg.first;
    size_t si = 0;
    for (; si < smask.size(); ++si) {
      if (q.st[si].nb >= maxnb) continue;
      bool clash = false;
      for (int j = jlo; j <= jhi; ++j)
        if ((b == j && ((smask[si] >> (j + 3)) & 1)) || (b == j + 3 && ((smask[si] >> j) & 1))) clash = true;
      if (!clash) break;
    }
    if (si == smask.size()) {
      smask.push_back(0);
      q.st[si] = XStage{};
    }
    XStage& S = q.st[si];
    const PauliGroup& G = groups[q.gi[bg.second]];
    if (__builtin_popcountll(G.m & G.z[0]) & 1) {
      S.gen = 1;
      S.odd |= (int8_t)(1 << S.nb);
    }
    S.bit[S.nb] = (int8_t)b;
    S.gg[S.nb] = (int8_t)bg.second;
    ++S.nb;
    smask[si] |= 1u << b;
    q.staged |= 1u << bg.second;
  }
  q.nst = (int)smask.size();
  // the warp groups: longest stage first to the less loaded group (cost per
  // amplitude about nb FMAs plus a load and its address)
  {
    std::vector<int> ord(q.nst);
    for (int i = 0; i < q.nst; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return q.st[a].nb > q.st[b].nb; });
    int load[2] = {0, 0};
    for (int i : ord) {
      const int g = !c128 && load[1] < load[0] ? 1 : 0;
      q.st[i].grp = (int8_t)g;
      load[g] += q.st[i].nb + 3;
    }
  }
  q.nsg = 0;
  for (int si = 0; si < q.nst; ++si) {
    XStage& S = q.st[si];
    S.slot0 = (int8_t)q.nsg;
    q.nsg += S.nb;
    const unsigned sm = smask[si];
    S.pair = (int8_t)(!c128 && (sm & 1u));
    std::vector<int> order;
    if (!c128 && !S.pair) order.push_back(0);
    for (int j = jlo; j <= jhi; ++j) {
      if (j < m && !((sm >> j) & 1)) order.push_back(j);
      else if (j + 3 < m && !((sm >> (j + 3)) & 1)) order.push_back(j + 3);
    }
    for (int b = 0; b < m; ++b)
      if (!((sm >> b) & 1) && std::find(order.begin(), order.end(), b) == order.end()) order.push_back(b);
    const int ntb = std::min<int>(std::min<int>(lg_nt, (int)sizeof(S.tb)), (int)order.size());
    S.ntb = (int8_t)ntb;
    for (int i = 0; i < ntb && i < (int)sizeof(S.tb); ++i) S.tb[i] = (int8_t)order[i];
    S.dhi = 0;
    for (size_t i = S.ntb; i < order.size(); ++i) S.dhi |= 1u << order[i];
  }
}

// Tensor map of a complex64 tile pass: the state as UINT64 amplitudes in
// dimensions that are runs of qubits -- qubits 0..3 (the tile's 128-byte
// rows), then ascending runs of tile qubits (split into pieces of at most 8,
// the box limit) and of the qubits outside the tile (box 1, coordinate from
// the tile number), at most 5 in all, 128-byte swizzled.  The box's row
// order is the tile-local order (high tile qubits ascending).  False: more
// than 5 runs (the pass copies with cp.async).
bool make_ptile_tmap(void* amp, int n, PTilePass& q, CUtensorMap* map, qs_status* st) {
  *st = QS_OK;
  q.tma = 0;
  if (kTL + q.r < 7) return false;  // both buffers 1024-byte aligned: tiles of 128 amplitudes or more
  u64 tmask = (u64(1) << kTL) - 1;
  for (int j = 0; j < q.r; ++j) tmask |= u64(1) << q.H[j];
  struct Dim { int lo, len, tile; };
  std::vector<Dim> dims;
  dims.push_back(Dim{0, kTL, 1});
  for (int b = kTL; b < n;) {
    const int t = (int)((tmask >> b) & 1);
    int e = b;
    while (e < n && (int)((tmask >> e) & 1) == t) ++e;
    if (t)
      for (int x = b; x < e; x += 8) dims.push_back(Dim{x, std::min(8, e - x), 1});
    else
      dims.push_back(Dim{b, e - b, 0});
    b = e;
  }
  if (dims.size() > 5) return false;
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  *st = tmap_encoder(&encode);
  if (*st != QS_OK) return false;
  const int rank = (int)dims.size();
  cuuint64_t gdim[5], gstr[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  for (int d = 0; d < 5; ++d) {
    q.tgb[d] = -1;
    q.tlen[d] = 0;
    if (d >= rank) continue;
    const Dim& D = dims[d];
    gdim[d] = cuuint64_t(1) << D.len;
    box[d] = D.tile ? (1u << D.len) : 1u;
    if (d > 0) gstr[d - 1] = (cuuint64_t(1) << D.lo) * 8;
    if (!D.tile) {
      int below = 0;  // qubits outside the tile under the run: its first tile-number bit
      for (int x = kTL; x < D.lo; ++x) below += !((tmask >> x) & 1);
      q.tgb[d] = (int8_t)below;
      q.tlen[d] = (int8_t)D.len;
    }
  }
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)rank, amp, gdim, gstr, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *st = fail(QS_ECUDA, "cuTensorMapEncodeTiled (expectation tile) failed (%d)", (int)r);
    return false;
  }
  q.trank = rank;
  q.tma = 1;
  return true;
}

// The passes of an expectation over an n-qubit state: tile passes (first
// fit of every group whose mask bits above the kTL low qubits number at most
// kTH, or kTH - 1 for complex128) and the groups that get a pass of their
// own (more high bits, or a state too small for a tile).
static void plan_pauli_passes(int n, qs_dtype dt, const std::vector<PauliGroup>& groups, std::vector<PTilePass>& tp,
                       std::vector<int>& alone) {
  const size_t ng = groups.size();
  // (complex64: one group too -- the tile pass's row and stage paths beat
  // the per-amplitude kernel)
  const bool tiles = n >= kTL + 1 && (ng > 1 || (dt == QS_C64 && n >= kTL + 3));
  const int rmax = dt == QS_C64 ? kTH : kTH - 1;  // tiles of 64 KB
  for (size_t i = 0; i < ng; ++i) {
    const u64 hi = groups[i].m >> kTL;
    if (!tiles || __builtin_popcountll(hi) > rmax) {
      alone.push_back((int)i);
      continue;
    }
    size_t p = 0;
    for (; p < tp.size(); ++p) {
      u64 cur = 0;
      for (int j = 0; j < tp[p].r; ++j) cur |= u64(1) << tp[p].H[j];
      const u64 need = (groups[i].m & ~((u64(1) << kTL) - 1)) | cur;
      if (tp[p].ng < kPassGroups && __builtin_popcountll(need) <= rmax && kTL + __builtin_popcountll(need) <= n)
        break;
    }
    if (p == tp.size()) {
      PTilePass q{};
      q.L = kTL;
      tp.push_back(q);
    }
    PTilePass& q = tp[p];
    u64 need = groups[i].m & ~((u64(1) << kTL) - 1);
    for (int j = 0; j < q.r; ++j) need |= u64(1) << q.H[j];
    q.r = 0;
    for (int b = kTL; b < n; ++b)
      if ((need >> b) & 1) q.H[q.r++] = b;
    q.gi[q.ng++] = (int)i;
  }
  // each pass's tile-local masks, and its tiles at least 2^(kTL + 1) amplitudes
  for (PTilePass& q : tp) {
    // tiles of up to 2^(kTL + rmax) amplitudes: fewer, larger tiles for
    // passes that need few high qubits (the extra qubits are the lowest free)
    {
      u64 used = 0;
      for (int j = 0; j < q.r; ++j) used |= u64(1) << q.H[j];
      for (int b = kTL; b < n && q.r < rmax; ++b)
        if (!((used >> b) & 1)) used |= u64(1) << b, ++q.r;
      q.r = 0;
      for (int b = kTL; b < n; ++b)
        if ((used >> b) & 1) q.H[q.r++] = b;
    }
    q.fmask = (n >= 64 ? ~u64(0) : (u64(1) << n) - 1) & ~((u64(1) << kTL) - 1);
    for (int j = 0; j < q.r; ++j) q.fmask &= ~(u64(1) << q.H[j]);
    q.tins.k = q.r;
    q.tins.set = 0;
    for (int j = 0; j < q.r; ++j) q.tins.pos[j] = q.H[j];
    for (int gg = 0; gg < q.ng; ++gg) {
      const u64 mg = groups[q.gi[gg]].m;
      unsigned ml = (unsigned)(mg & ((u64(1) << kTL) - 1));
      for (int j = 0; j < q.r; ++j)
        if ((mg >> q.H[j]) & 1) ml |= 1u << (kTL + j);
      q.mloc[gg] = ml;
      q.hloc[gg] = ml ? 31 - __builtin_clz(ml) : -1;
    }
    // complex64: single-term groups on one local bit with no Z bit outside
    // it go to register stages
    q.nst = q.nsg = 0;
    q.staged = 0;
    build_stages(q, groups, kStageThreads, dt == QS_C128);
    q.allst = q.ng > 0 && q.staged == (q.ng >= 32 ? ~0u : (1u << q.ng) - 1u);
    q.ngen = 0;
    for (int gg = 0; gg < q.ng; ++gg)
      if (!((q.staged >> gg) & 1u)) q.genl[q.ngen++] = (int8_t)gg;
    q.clsg = -1;
    q.noflush = 1;
    for (int gg = 0; gg < q.ng; ++gg) {
      if ((q.staged >> gg) & 1u) continue;
      if (q.hloc[gg] < 0 && groups[q.gi[gg]].ncls > 0 && q.clsg < 0) q.clsg = gg;
      else q.noflush = 0;
    }
    if (dt != QS_C64) q.clsg = -1, q.noflush = 0;
    // complex64 with stages: the non-staged groups to the warp group with
    // the smaller stage load (cost per amplitude: a stage about nb + 3, a
    // Z-class group about 6, another group about 20)
    q.ggrp = -1;
    if (dt == QS_C64 && q.nst > 0 && !q.allst) {
      int load[2] = {0, 0};
      for (int si = 0; si < q.nst; ++si) load[(int)q.st[si].grp] += q.st[si].nb + 3;
      q.ggrp = load[1] < load[0] ? 1 : 0;
    }
  }
}

qs_status run_expect(qs_state* s, int nterms, const u64* xmask, const u64* zmask, const double* coeff,
                     double* out) {
  const std::vector<PauliGroup> groups = build_pauli_groups(nterms, xmask, zmask, coeff);
  const u64 N = u64(1) << s->n;
  const size_t ng = groups.size();
  std::vector<PTilePass> tp;
  std::vector<int> alone;
  plan_pauli_passes(s->n, (qs_dtype)s->dtype, groups, tp, alone);
  const unsigned gsz = red_grid(N / 2);
  const size_t npart = gsz * (tp.size() + alone.size());
  const size_t gbytes = sizeof(PauliGroup) * ng;
  const size_t goff = ((sizeof(double2) * (npart + 1) + 255) / 256) * 256;
  qs_status st = ensure_scratch(s, goff + gbytes);
  if (st != QS_OK) return st;
  double2* part = static_cast<double2*>(s->scratch);
  double2* res = part + npart;
  PauliGroup* dgroups = reinterpret_cast<PauliGroup*>(static_cast<char*>(s->scratch) + goff);
  size_t pi = 0;
  if (!tp.empty()) {
    cudaError_t e = cudaMemcpyAsync(dgroups, groups.data(), gbytes, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "expectation: group upload");
  }
  bool any_tma = false;
  for (PTilePass& q : tp) {
    const size_t asz = s->dtype == QS_C64 ? sizeof(float2) : sizeof(double2);
    const bool c64 = s->dtype == QS_C64;
    const size_t smem = ptile_buf_off(q.nst, q.nsg, c64 ? kStageThreads : kThreads) +
                        (c64 ? kPtileAlign : 0) + asz * (size_t(1) << (q.L + q.r)) * (c64 ? 2 : 1);
    CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof(tmap));
    q.tma = 0;
    if (c64) {
      make_ptile_tmap(s->amp, s->n, q, &tmap, &st);
      if (st != QS_OK) return st;
      any_tma |= q.tma != 0;
    }
    const u64 ntiles = u64(1) << (s->n - q.L - q.r);
    unsigned g = (unsigned)std::min<u64>(ntiles, (u64)gsz);
    cudaError_t e;
    if (s->dtype == QS_C64) {
      auto kern = q.allst ? k_pauli_tiles<float, kTileThreads64, true> : k_pauli_tiles<float, kTileThreads64, false>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_fail(e, "expectation: smem attribute");
      // one wave of resident CTAs: each runs its tiles' copy/evaluate pipeline
      int occ = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTileThreads64, smem);
      if (e != cudaSuccess) return cuda_fail(e, "expectation: occupancy");
      g = std::min<unsigned>(g, (unsigned)std::max(1, occ) * (unsigned)sm_count());
      kern<<<g, kTileThreads64, smem, s->stream>>>(static_cast<const float*>(s->amp), s->n, q, tmap, dgroups,
                                                   part + gsz * pi);
    } else {
      auto kern = q.allst ? k_pauli_tiles<double, kThreads, true> : k_pauli_tiles<double, kThreads, false>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_fail(e, "expectation: smem attribute");
      int occ = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
      if (e != cudaSuccess) return cuda_fail(e, "expectation: occupancy");
      g = std::min<unsigned>(g, (unsigned)std::max(1, occ) * (unsigned)sm_count());
      kern<<<g, kThreads, smem, s->stream>>>(static_cast<const double*>(s->amp), s->n, q, tmap, dgroups,
                                             part + gsz * pi);
    }
    if ((st = launch_ok("k_pauli_tiles")) != QS_OK) return st;
    // CTAs beyond the tiles write no partial: zero their slots
    if (g < gsz) {
      e = cudaMemsetAsync(part + gsz * pi + g, 0, sizeof(double2) * (gsz - g), s->stream);
      if (e != cudaSuccess) return cuda_fail(e, "expectation: memset");
    }
    ++pi;
  }
  for (int i : alone) {
    if (s->dtype == QS_C64)
      k_pauli<float><<<gsz, kThreads, 0, s->stream>>>(static_cast<const float*>(s->amp), s->n, groups[i], part + gsz * pi);
    else
      k_pauli<double><<<gsz, kThreads, 0, s->stream>>>(static_cast<const double*>(s->amp), s->n, groups[i], part + gsz * pi);
    if ((st = launch_ok("k_pauli")) != QS_OK) return st;
    ++pi;
  }
  k_final<<<1, kThreads, 0, s->stream>>>(part, (int)npart, res, 0);
  if ((st = launch_ok("k_final")) != QS_OK) return st;
  double2 h{0.0, 0.0};
  if ((st = read_result(s, res, &h)) != QS_OK) return st;
  if (any_tma) {
    int flag = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&flag, g_expect_timeout, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "expectation: status read");
    if (flag) {
      const int zero = 0;
      cudaMemcpyToSymbol(g_expect_timeout, &zero, sizeof(int));
      return fail(QS_ETIMEOUT, "expectation: a tile copy wait gave up");
    }
  }
  *out = h.x;
  return QS_OK;
}

qs_status expect_pauli_passes(int n, int dtype, int nterms, const u64* xmask, const u64* zmask, int* passes) {
  std::vector<double> coeff((size_t)nterms, 1.0);
  const std::vector<PauliGroup> groups = build_pauli_groups(nterms, xmask, zmask, coeff.data());
  std::vector<PTilePass> tp;
  std::vector<int> alone;
  plan_pauli_passes(n, (qs_dtype)dtype, groups, tp, alone);
  *passes = (int)(tp.size() + alone.size());
  return QS_OK;
}

}  // namespace qs
