// Reductions over the state vector: norm, inner product, Pauli expectation.
//
// Each thread accumulates over a grid-stride range of elements in
// double-float, flushed into FP64 (see kU); warps combine in FP64 with shuffles, CTAs through shared memory, and the
// per-CTA partials are summed by one CTA in index order.  The grid size
// depends only on the problem size, so results are bitwise reproducible.
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
#include <algorithm>
#include <vector>

#include <type_traits>

#include "dfloat.cuh"
#include "kcommon.cuh"
#include "pauli.cuh"

namespace qs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of up to two values; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kThreads / 32], sb[kThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (w == 0) {
    a = l < kThreads / 32 ? sa[l] : 0.0;
    b = l < kThreads / 32 ? sb[l] : 0.0;
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

struct PTilePass {
  int L, r;                    // tile = L low qubits + r high qubits H[0..r)
  int H[kTH];
  Ins tins;                    // zero insertion at the high qubits (the tile base)
  int ng;
  int gi[kPassGroups];         // groups of this pass (indices into the group array)
  int hloc[kPassGroups];       // highest tile-local bit of the group's mask (-1: diagonal group)
  unsigned mloc[kPassGroups];  // the group's X/Y mask in tile-local bits
  // complex64 register stages: single-term groups on one tile-local bit
  // with no Z bit outside it, up to 3 bits per stage, evaluated from 2^nb
  // amplitudes held in registers (the other groups loop over the tile)
  int nst;
  int8_t snb[kPassGroups];
  int8_t sbit[kPassGroups][3];  // ascending local bits
  int8_t sgg[kPassGroups][3];   // the group slot of each bit
  unsigned staged;              // bit gg: group slot gg is evaluated in a stage
};

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
  // XOR swizzle of the tile's 16-amplitude (128-byte) rows: strided reads
  // of the register stages stay free of bank conflicts
  __device__ static unsigned sw(unsigned e) { return e ^ ((e >> 4) & 15u); }
  __device__ static T from(float2 v) { return v; }
  __device__ static void get(const T& v, dfl& re, dfl& im) {
    re = dfl{v.x, 0.f};
    im = dfl{v.y, 0.f};
  }
};
template <> struct TileAmp<double> {
  typedef float4 T;
  __device__ static unsigned sw(unsigned e) { return e; }
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

// Stage si of a complex64 tile pass: every 2^NB amplitudes spanning the
// stage's bits from the (swizzled) tile into registers, then for each
// bit's group, over the pairs x, x ^ 2^b of the block, Re (or Im) of
// conj(a_y) a_x in FP32, summed per thread; acc[j] receives bit j's sum.
template <int NB>
__device__ __forceinline__ void x_stage(const float2* t, unsigned tile, const PTilePass& P, int si, const bool (&odd)[3],
                                        float (&acc)[3]) {
  // the swizzle is linear over the index bits, so the swizzled offset of
  // base | c's bits is sw(base) ^ sw(c's bits)
  unsigned sp[1 << NB];
  unsigned b[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) b[j] = j < NB ? (unsigned)P.sbit[si][j] : 0u;
#pragma unroll
  for (int c = 0; c < (1 << NB); ++c) {
    unsigned o = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if ((c >> j) & 1) o |= 1u << b[j];
    sp[c] = TileAmp<float>::sw(o);
  }
  for (unsigned i = threadIdx.x; i < (tile >> NB); i += kThreads) {
    unsigned base = i;
#pragma unroll
    for (int j = 0; j < NB; ++j)  // a zero at each stage bit (ascending)
      base = ((base >> b[j]) << (b[j] + 1)) | (base & ((1u << b[j]) - 1u));
    const unsigned sb = TileAmp<float>::sw(base);
    float2 v[1 << NB];
#pragma unroll
    for (int c = 0; c < (1 << NB); ++c) v[c] = t[sb ^ sp[c]];
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int c = 0; c < (1 << NB); ++c) {
        if ((c >> j) & 1) continue;
        const float2 X = v[c], Y = v[c | (1 << j)];
        acc[j] += !odd[j] ? fmaf(Y.x, X.x, Y.y * X.y) : fmaf(Y.x, X.y, -(Y.y * X.x));
      }
  }
}
__device__ __forceinline__ float2 t_as_f2(float4 v) { return make_float2(v.x, v.z); }  // unused (complex128)

template <typename R>
__global__ void __launch_bounds__(kThreads, 1) k_pauli_tiles(const R* __restrict__ a, int n,
                                                          const __grid_constant__ PTilePass P,
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
  E* t = reinterpret_cast<E*>(psm + sizeof(u64) * (1u << kTH));  // [2^(L + r)]
  const A* av = reinterpret_cast<const A*>(a);
  const int L = P.L, r = P.r, m = L + r;
  const unsigned tile = 1u << m;
  for (unsigned i = threadIdx.x; i < (1u << r); i += kThreads) {
    u64 sp = 0;
    for (int j = 0; j < r; ++j)
      if ((i >> j) & 1u) sp |= u64(1) << P.H[j];
    spreadH[i] = sp;
  }
  const u64 ntiles = u64(1) << (n - m);
  double sr = 0.0, si = 0.0;
  dfl ar{0.f, 0.f}, ai{0.f, 0.f};
  __syncthreads();
  for (u64 ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const u64 F = expand(ti << L, P.tins);
    // the tile into shared memory, 4 loads in flight per thread
    for (unsigned e0 = threadIdx.x; e0 < tile; e0 += 4 * kThreads) {
      A v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned e = e0 + u * kThreads;
        if (e < tile) v[u] = av[ptile_global(F, spreadH, L, e)];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned e = e0 + u * kThreads;
        if (e < tile) t[TA::sw(e)] = TA::from(v[u]);
      }
    }
    __syncthreads();
    if constexpr (kF32) {
      for (int si = 0; si < P.nst; ++si) {
        const int nb = P.snb[si];
        bool odd[3] = {false, false, false};
        float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (j >= nb) break;
          const PauliGroup& g = groups[P.gi[P.sgg[si][j]]];
          odd[j] = __popcll(g.m & g.z[0]) & 1;
        }
        const float2* tf = reinterpret_cast<const float2*>(t);
        if (nb == 3) x_stage<3>(tf, tile, P, si, odd, acc);
        else if (nb == 2) x_stage<2>(tf, tile, P, si, odd, acc);
        else x_stage<1>(tf, tile, P, si, odd, acc);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (j >= nb) break;
          const PauliGroup& g = groups[P.gi[P.sgg[si][j]]];
          const dfl c{acc[j], 0.f};
          const dfl w_r{2.f * g.wrh[0], 2.f * g.wrl[0]}, w_i{2.f * g.wih[0], 2.f * g.wil[0]};
          if (!odd[j]) {
            df_acc(ar, df_mul(w_r, c));
            df_acc(ai, df_mul(w_i, c));
          } else {
            df_acc(ar, df_mul(dfl{-w_i.h, -w_i.l}, c));
            df_acc(ai, df_mul(w_r, c));
          }
        }
      }
    }
    for (int gg = 0; gg < P.ng; ++gg) {
      if (kF32 && ((P.staged >> gg) & 1u)) continue;
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
          // complex64: p_x and the class sums in FP32 over this thread's
          // amplitudes of the tile (two chains per class), then one
          // double-float step per class
          float s2[kMaxClasses][2];
#pragma unroll
          for (int c = 0; c < kMaxClasses; ++c) s2[c][0] = s2[c][1] = 0.f;
          int par = 0;
          for (unsigned l = threadIdx.x; l < tile; l += kThreads, par ^= 1) {
            const float2 v = t_as_f2(t[TA::sw(l)]);
            const float pw = fmaf(v.x, v.x, v.y * v.y);
            const u64 x = ptile_global(F, spreadH, L, l);
#pragma unroll
            for (int c = 0; c < kMaxClasses; ++c) {
              if (c >= nc) break;
              const float k = (float)(g.cls_len[c] - 2 * __popcll((x ^ (x >> g.cls_d[c])) & g.cls_mask[c]));
              if (par) s2[c][1] = fmaf(k, pw, s2[c][1]);
              else s2[c][0] = fmaf(k, pw, s2[c][0]);
            }
          }
#pragma unroll
          for (int c = 0; c < kMaxClasses; ++c) sc[c] = dfl{s2[c][0] + s2[c][1], 0.f};
        } else {
          for (unsigned l = threadIdx.x; l < tile; l += kThreads) {
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
          if (c >= nc) break;
          const dfl v = df_norm2(sc[c]);
          df_acc(ar, df_mul(dfl{g.cwrh[c], g.cwrl[c]}, v));
          df_acc(ai, df_mul(dfl{g.cwih[c], g.cwil[c]}, v));
        }
      } else if (h < 0) {  // diagonal group: sum_x |a_x|^2 f(x)
        int since = 0;  // flush the double-float sums into FP64 every kU terms
        for (unsigned l = threadIdx.x; l < tile; l += kThreads) {
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
          for (unsigned k0 = threadIdx.x; k0 < tile / 2; k0 += 4 * kThreads) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const unsigned k = k0 + u * kThreads;
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
          for (unsigned k0 = threadIdx.x; k0 < tile / 2; k0 += 4 * kThreads) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const unsigned k = k0 + u * kThreads;
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
        for (unsigned k = threadIdx.x; k < tile / 2; k += kThreads) {
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
    // into FP64 once per tile (the FP64 pipe is about 1/64 of FP32 on GB300)
    df_flush(sr, ar);
    df_flush(si, ai);
    __syncthreads();
  }
  block_sum2(sr, si);
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
  double2 h;
  if ((st = read_result(s, res, &h)) != QS_OK) return st;
  *out = h.x;
  return QS_OK;
}

qs_status run_inner(qs_state* a, qs_state* b, double out[2]) {
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
  double2 h;
  if ((st = read_result(a, res, &h)) != QS_OK) return st;
  out[0] = h.x;
  out[1] = h.y;
  return QS_OK;
}

qs_status run_expect(qs_state* s, int nterms, const u64* xmask, const u64* zmask, const double* coeff,
                     double* out) {
  const std::vector<PauliGroup> groups = build_pauli_groups(nterms, xmask, zmask, coeff);
  const u64 N = u64(1) << s->n;
  const size_t ng = groups.size();
  // tile passes: first fit of every group whose mask bits above the kTL low
  // qubits number at most kTH; the others (and every group of a state too
  // small for a tile) get a pass of their own
  std::vector<PTilePass> tp;
  std::vector<int> alone;
  const bool tiles = s->n >= kTL + 1 && ng > 1;
  const int rmax = s->dtype == QS_C64 ? kTH : kTH - 1;  // tiles of 64 KB
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
      if (tp[p].ng < kPassGroups && __builtin_popcountll(need) <= rmax && kTL + __builtin_popcountll(need) <= s->n)
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
    for (int b = kTL; b < s->n; ++b)
      if ((need >> b) & 1) q.H[q.r++] = b;
    q.gi[q.ng++] = (int)i;
  }
  // each pass's tile-local masks, and its tiles at least 2^(kTL + 1) amplitudes
  for (PTilePass& q : tp) {
    for (int b = kTL; b < s->n && q.r == 0; ++b) q.H[q.r++] = b;
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
    // it go to register stages of up to 3 bits
    q.nst = 0;
    q.staged = 0;
    if (s->dtype == QS_C64) {
      std::vector<std::pair<int, int>> one;  // (local bit, group slot)
      for (int gg = 0; gg < q.ng; ++gg) {
        const PauliGroup& G = groups[q.gi[gg]];
        if (G.nt == 1 && __builtin_popcount(q.mloc[gg]) == 1 && (G.z[0] & ~G.m) == 0)
          one.push_back({q.hloc[gg], gg});
      }
      std::sort(one.begin(), one.end());
      for (size_t i = 0; i < one.size(); i += 3) {
        const int nb = (int)std::min<size_t>(3, one.size() - i);
        q.snb[q.nst] = (int8_t)nb;
        for (int j = 0; j < nb; ++j) {
          q.sbit[q.nst][j] = (int8_t)one[i + j].first;
          q.sgg[q.nst][j] = (int8_t)one[i + j].second;
          q.staged |= 1u << one[i + j].second;
        }
        ++q.nst;
      }
    }
  }
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
  for (const PTilePass& q : tp) {
    const size_t asz = s->dtype == QS_C64 ? sizeof(float2) : sizeof(double2);
    const size_t smem = sizeof(u64) * (1u << kTH) + asz * (size_t(1) << (q.L + q.r));
    const u64 ntiles = u64(1) << (s->n - q.L - q.r);
    const unsigned g = (unsigned)std::min<u64>(ntiles, (u64)gsz);
    cudaError_t e;
    if (s->dtype == QS_C64) {
      e = cudaFuncSetAttribute(k_pauli_tiles<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_fail(e, "expectation: smem attribute");
      k_pauli_tiles<float><<<g, kThreads, smem, s->stream>>>(static_cast<const float*>(s->amp), s->n, q, dgroups,
                                                             part + gsz * pi);
    } else {
      e = cudaFuncSetAttribute(k_pauli_tiles<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_fail(e, "expectation: smem attribute");
      k_pauli_tiles<double><<<g, kThreads, smem, s->stream>>>(static_cast<const double*>(s->amp), s->n, q, dgroups,
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
  double2 h;
  if ((st = read_result(s, res, &h)) != QS_OK) return st;
  *out = h.x;
  return QS_OK;
}

}  // namespace qs
