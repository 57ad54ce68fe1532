// Adjoint-method gradient of an expectation value.
//
// The paper has no differentiation; this is the standard reverse sweep for
// E(theta) = <psi(theta)|H|psi(theta)>, psi(theta) = U_L ... U_1 |0...0>,
// whose trainable gates are R_P(t) = exp(-i t P / 2), P in {X, Y, Z}:
//   forward:  psi = U_L ... U_1 |0>        (a compiled tile plan per parameter set)
//             lambda = H psi, E = Re <psi|lambda>   (one fused pass, k_hamiltonian)
//   reverse:  for l = L .. 1
//               if gate l is R_P(theta_j):  g_j += Im <lambda|P_q|psi>
//               psi <- U_l^dagger psi ;  lambda <- U_l^dagger lambda
// (dE/dt = 2 Re <lambda_l| (-i P/2) |psi_l> = Im <lambda_l|P|psi_l> with
// psi_l, lambda_l the states right after gate l.)
//
// The reverse sweep runs in steps (build_sweep):
//  * a run of consecutive diagonal gates in one pass (k_adj_diag): their
//    trainable RZ gradients all come from the state at the run's end, since
//    the run's diagonal gates commute with each Z_q;
//  * a layer of one-qubit gates on distinct qubits in one pass (k_adj_layer):
//    each generator commutes with the layer's other gates, so all gradient
//    terms come from the group's values before any of the layer is undone;
//  * any other trainable gate (k_adj_1q), any other fixed gate (per-gate
//    kernels).
//
// Parameter sets are processed Bc at a time.  psi and lambda of the chunk live
// in one buffer [psi_0 .. psi_{Bc-1}, lambda_0 .. lambda_{Bc-1}], which is
// itself a state of n + log2(Bc) + 1 qubits: a fixed gate on qubits < n is
// un-applied to all 2 Bc vectors by one launch of the per-gate kernel, and the
// sweep kernels run over (elements, set).  Bc is the largest power of two
// <= batch whose 2 Bc vectors fit a budget (adj_chunk).  With Bc = 1 psi is
// the caller's state and lambda a second vector.
//
// Arithmetic: complex64 in FP32; complex128 in double-float, with psi and
// lambda held in double-float storage for the whole reverse sweep (each FP64
// value as its (hi, lo) float pair in the same 8 bytes, so an amplitude is one
// float4 and no kernel converts).  Per-element gradient products are FP32
// (complex64) or double-float (complex128), summed per thread in
// double-float; CTA partials are summed in FP64 in a fixed order.
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <map>
#include <vector>

#include "arith.cuh"
#include "planner.h"

namespace qs {
namespace {

constexpr int kAT = 256;

__device__ __forceinline__ double a_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double a_block_sum(double a) {
  __shared__ double sa[kAT / 32];
  a = a_warp_sum(a);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sa[w] = a;
  __syncthreads();
  if (w == 0) {
    a = l < kAT / 32 ? sa[l] : 0.0;
    a = a_warp_sum(a);
  }
  return a;
}

// Amplitude storage of the sweep: complex64 as float2 (re, im); complex128
// in double-float storage as float4 (re_h, re_l, im_h, im_l).
template <typename R> struct Amp;
template <> struct Amp<float> { typedef float2 V; };
template <> struct Amp<double> { typedef float4 V; };

__device__ __forceinline__ void upd(const M2<float>& U, float2& a, float2& b) { mv2(U, a.x, a.y, b.x, b.y); }
__device__ __forceinline__ void upd(const M2df& U, float4& a, float4& b) {
  cdf A{a.x, a.y, a.z, a.w}, B{b.x, b.y, b.z, b.w};
  mv2df(U, A, B);
  a = make_float4(A.rh, A.rl, A.ih, A.il);
  b = make_float4(B.rh, B.rl, B.ih, B.il);
}

// Gradient term of one amplitude pair, Im <lambda|P_q|psi> restricted to the
// pair (a = lambda, b = psi; conj(a) b = (ar br + ai bi) + i (ar bi - ai br)):
//   P = X: Im(conj(a0) b1 + conj(a1) b0)
//   P = Y: Im(-i conj(a0) b1 + i conj(a1) b0) = -Re(conj(a0) b1) + Re(conj(a1) b0)
//   P = Z: Im(conj(a0) b0 - conj(a1) b1)
__device__ __forceinline__ dfl grad_term(int gen, float2 a0, float2 a1, float2 b0, float2 b1) {
  float t;
  if (gen == 1) t = __fmaf_rn(a0.x, b1.y, -a0.y * b1.x) + __fmaf_rn(a1.x, b0.y, -a1.y * b0.x);
  else if (gen == 2) t = __fmaf_rn(a1.x, b0.x, a1.y * b0.y) - __fmaf_rn(a0.x, b1.x, a0.y * b1.y);
  else t = __fmaf_rn(a0.x, b0.y, -a0.y * b0.x) - __fmaf_rn(a1.x, b1.y, -a1.y * b1.x);
  return dfl{t, 0.0f};
}
__device__ __forceinline__ dfl grad_term(int gen, float4 a0, float4 a1, float4 b0, float4 b1) {
  // components: .x re_h, .y re_l, .z im_h, .w im_l
  if (gen == 1)
    return dot4(a0.x, a0.y, b1.z, b1.w, -a0.z, -a0.w, b1.x, b1.y, a1.x, a1.y, b0.z, b0.w, -a1.z, -a1.w, b0.x, b0.y);
  if (gen == 2)
    return dot4(-a0.x, -a0.y, b1.x, b1.y, -a0.z, -a0.w, b1.z, b1.w, a1.x, a1.y, b0.x, b0.y, a1.z, a1.w, b0.z, b0.w);
  return dot4(a0.x, a0.y, b0.z, b0.w, -a0.z, -a0.w, b0.x, b0.y, -a1.x, -a1.y, b1.z, b1.w, a1.z, a1.w, b1.x, b1.y);
}

// Trainable step (gen 1, 2, 3: generator X, Y, Z) for every set b =
// blockIdx.y: psi_b = psi + b N, lambda_b = lam + b N, U^dagger of set b at
// mats[b]; gradient partials part[b * gridDim.x + blockIdx.x].
template <typename V, typename Mat>
__global__ void __launch_bounds__(kAT) k_adj_1q(V* __restrict__ psi, V* __restrict__ lam, u64 N, u64 npairs, int q,
                                                const Mat* __restrict__ mats, int gen, double* __restrict__ part) {
  const int b = blockIdx.y;
  V* ps = psi + N * b;
  V* lm = lam + N * b;
  const Mat U = mats[b];
  const u64 lo_mask = (u64(1) << q) - 1;
  dfl acc{0.0f, 0.0f};
  for (u64 i = (u64)blockIdx.x * kAT + threadIdx.x; i < npairs; i += (u64)gridDim.x * kAT) {
    const u64 x0 = ((i & ~lo_mask) << 1) | (i & lo_mask);
    const u64 x1 = x0 | (lo_mask + 1);
    V p0 = ps[x0], p1 = ps[x1], l0 = lm[x0], l1 = lm[x1];
    df_acc(acc, grad_term(gen, l0, l1, p0, p1));
    upd(U, p0, p1);
    upd(U, l0, l1);
    ps[x0] = p0;
    ps[x1] = p1;
    lm[x0] = l0;
    lm[x1] = l1;
  }
  const double g = a_block_sum((double)acc.h + (double)acc.l);
  if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = g;
}

// A run of consecutive diagonal gates (Z, S, T, P, RZ, CZ, CP) of the reverse
// sweep in one pass.  Every trainable RZ_q in the run has the gradient
// Im <lambda|Z_q|psi> on the state at the run's end: the run's other gates
// are diagonal, commute with Z_q and cancel in <lambda|D Z_q D^dagger|psi>.  So
// the pass takes all of them from one product conj(lambda_x) psi_x, then
// multiplies psi_x and lambda_x by the run's U^dagger diagonal, a product of
// one factor per gate (its entry for the gate's bits of x).
constexpr int kRunF = 64;  // factors per run
constexpr int kRunG = 24;  // trainable gates per run
struct DRun {
  int nf, ng;
  int nlo;                   // factors [0, nlo) act on qubits below the launch's stride bits only
  int q0[kRunF], q1[kRunF];  // q1 < 0: one-qubit factor
  int sign[kRunF];           // 1: -1 when all its bits are set (CZ, Z), else 1 (no table entry used)
  int gq[kRunG];             // qubit of each trainable RZ, in slot order
};
// one factor's U^dagger diagonal entries d[r] (r = bit q0 | bit q1 << 1), double-float
struct DFac {
  float rh[4], rl[4], ih[4], il[4];
};

__device__ __forceinline__ dfl im_conj_mul(float2 l, float2 p) {  // Im(conj(l) p)
  return dfl{__fmaf_rn(l.x, p.y, -l.y * p.x), 0.0f};
}
__device__ __forceinline__ dfl im_conj_mul(float4 l, float4 p) {
  return dot2(l.x, l.y, p.z, p.w, -l.z, -l.w, p.x, p.y);
}
__device__ __forceinline__ void vneg(float2& v) { v = make_float2(-v.x, -v.y); }
__device__ __forceinline__ void vneg(float4& v) { v = make_float4(-v.x, -v.y, -v.z, -v.w); }
__device__ __forceinline__ void fac_mul(const DFac& F, int r, float2& v) {
  const float zr = F.rh[r], zi = F.ih[r];
  v = make_float2(__fmaf_rn(zr, v.x, -zi * v.y), __fmaf_rn(zr, v.y, zi * v.x));
}
__device__ __forceinline__ void fac_mul(const DFac& F, int r, float4& v) {
  const float zh[2] = {F.rh[r], F.ih[r]}, zl[2] = {F.rl[r], F.il[r]};
  cdf a{v.x, v.y, v.z, v.w};
  cmul_df(zh, zl, a);
  v = make_float4(a.rh, a.rl, a.ih, a.il);
}

// complex scalar in double-float (complex64 uses the high parts only)
struct CZf {
  float rh, rl, ih, il;
};
__device__ __forceinline__ void cz_mul(CZf& z, const DFac& F, int r, float2*) {  // z *= d[r], FP32
  const float fr = F.rh[r], fi = F.ih[r];
  const float zr = __fmaf_rn(z.rh, fr, -z.ih * fi);
  z.ih = __fmaf_rn(z.rh, fi, z.ih * fr);
  z.rh = zr;
}
__device__ __forceinline__ void cz_mul(CZf& z, const DFac& F, int r, float4*) {  // double-float
  const float zh[2] = {F.rh[r], F.ih[r]}, zl[2] = {F.rl[r], F.il[r]};
  cdf a{z.rh, z.rl, z.ih, z.il};
  cmul_df(zh, zl, a);
  z = CZf{a.rh, a.rl, a.ih, a.il};
}
__device__ __forceinline__ void cz_apply(const CZf& z, float2& v) {
  v = make_float2(__fmaf_rn(z.rh, v.x, -z.ih * v.y), __fmaf_rn(z.rh, v.y, z.ih * v.x));
}
__device__ __forceinline__ void cz_apply(const CZf& z, float4& v) {
  const float zh[2] = {z.rh, z.ih}, zl[2] = {z.rl, z.il};
  cdf a{v.x, v.y, v.z, v.w};
  cmul_df(zh, zl, a);
  v = make_float4(a.rh, a.rl, a.ih, a.il);
}

// The grid's stride is 2^lgs (a power of two), so the bits of x below lgs
// are this thread's constants: the factors on those bits (the first nlo)
// are multiplied once into a per-thread scalar, and a gradient whose qubit is
// below lgs is +-(the thread's plain sum).  Only factors and gradients on
// higher qubits are evaluated per element.
template <typename V>
__global__ void __launch_bounds__(kAT) k_adj_diag(V* __restrict__ psi, V* __restrict__ lam, u64 N,
                                                  const __grid_constant__ DRun R, const DFac* __restrict__ tab,
                                                  double* __restrict__ part, int Bc, int lgs) {
  const int b = blockIdx.y;
  V* ps = psi + N * b;
  V* lm = lam + N * b;
  const DFac* T = tab + (size_t)b * R.nf;
  const u64 x0 = (u64)blockIdx.x * kAT + threadIdx.x;
  const u64 stride = (u64)gridDim.x * kAT;
  // per-thread constant part of the phase
  CZf zc{1.0f, 0.0f, 0.0f, 0.0f};
  bool neg0 = false, zc_one = true;
  for (int f = 0; f < R.nlo; ++f) {
    const int r = (int)((x0 >> R.q0[f]) & 1) | (R.q1[f] >= 0 ? (int)((x0 >> R.q1[f]) & 1) << 1 : 0);
    if (R.sign[f]) {
      neg0 ^= r == (R.q1[f] >= 0 ? 3 : 1);
    } else {
      cz_mul(zc, T[f], r, (V*)nullptr);
      zc_one = false;
    }
  }
  dfl tot{0.0f, 0.0f};
  dfl acc[kRunG];
#pragma unroll
  for (int s = 0; s < kRunG; ++s) acc[s] = dfl{0.0f, 0.0f};
  for (u64 x = x0; x < N; x += stride) {
    V p = ps[x], l = lm[x];
    const dfl c = im_conj_mul(l, p);
    df_acc(tot, c);
#pragma unroll
    for (int s = 0; s < kRunG; ++s)
      if (s < R.ng && R.gq[s] >= lgs) df_acc(acc[s], ((x >> R.gq[s]) & 1) ? dfl{-c.h, -c.l} : c);
    bool neg = neg0;
    if (!zc_one) {
      cz_apply(zc, p);
      cz_apply(zc, l);
    }
    for (int f = R.nlo; f < R.nf; ++f) {
      const int r = (int)((x >> R.q0[f]) & 1) | (R.q1[f] >= 0 ? (int)((x >> R.q1[f]) & 1) << 1 : 0);
      if (R.sign[f]) {
        neg ^= r == (R.q1[f] >= 0 ? 3 : 1);
      } else {
        fac_mul(T[f], r, p);
        fac_mul(T[f], r, l);
      }
    }
    if (neg) {
      vneg(p);
      vneg(l);
    }
    ps[x] = p;
    lm[x] = l;
  }
#pragma unroll
  for (int s = 0; s < kRunG; ++s) {
    if (s < R.ng) {  // uniform: every thread takes part in each block sum
      dfl v = acc[s];
      if (R.gq[s] < lgs) v = ((x0 >> R.gq[s]) & 1) ? dfl{-tot.h, -tot.l} : tot;
      const double g = a_block_sum((double)v.h + (double)v.l);
      if (threadIdx.x == 0) part[((size_t)s * Bc + b) * gridDim.x + blockIdx.x] = g;
    }
  }
}

// A layer of one-qubit gates on M distinct qubits (trainable RX/RY or fixed
// non-diagonal gates) in one pass.  Gates on distinct qubits commute, and a
// gate's generator commutes with the layer's other gates, so every gradient
// term is taken from the group's values before any of the layer is
// un-applied; then each U^dagger is applied along its bit of the group.
// A thread holds the 2^M amplitudes of psi and lambda over the layer's
// qubits (x with those bits clear, plus every combination).
constexpr int kLayerMax = 4;
template <typename Mat>
struct LayerArgs {
  Ins ins;               // zero insertion at the layer's qubits (sorted)
  int q[kLayerMax];      // qubit of gate j
  int gen[kLayerMax];    // 0: fixed (matrix in fixed[j]); 1, 2, 3: trainable X, Y, Z generator
  int slot[kLayerMax];   // gradient slot (trainable)
  Mat fixed[kLayerMax];  // U^dagger of fixed gates
};

template <typename V, typename Mat, int M>
__global__ void __launch_bounds__(kAT) k_adj_layer(V* __restrict__ psi, V* __restrict__ lam, u64 N,
                                                   const __grid_constant__ LayerArgs<Mat> A,
                                                   const Mat* __restrict__ mats, double* __restrict__ part, int Bc) {
  constexpr int NR = 1 << M;
  const int b = blockIdx.y;
  V* ps = psi + N * b;
  V* lm = lam + N * b;
  Mat U[M];
#pragma unroll
  for (int j = 0; j < M; ++j) U[j] = A.gen[j] ? mats[(size_t)A.slot[j] * Bc + b] : A.fixed[j];
  dfl acc[M];
#pragma unroll
  for (int j = 0; j < M; ++j) acc[j] = dfl{0.0f, 0.0f};
  u64 off[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    u64 o = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) o |= (u64)((r >> j) & 1) << A.q[j];
    off[r] = o;
  }
  const u64 ngroups = N >> M;
  for (u64 gi = (u64)blockIdx.x * kAT + threadIdx.x; gi < ngroups; gi += (u64)gridDim.x * kAT) {
    const u64 base = expand(gi, A.ins);
    V p[NR], l[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      p[r] = ps[base | off[r]];
      l[r] = lm[base | off[r]];
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if (!A.gen[j]) continue;
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (!((r >> j) & 1)) df_acc(acc[j], grad_term(A.gen[j], l[r], l[r | (1 << j)], p[r], p[r | (1 << j)]));
    }
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (!((r >> j) & 1)) {
          upd(U[j], p[r], p[r | (1 << j)]);
          upd(U[j], l[r], l[r | (1 << j)]);
        }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      ps[base | off[r]] = p[r];
      lm[base | off[r]] = l[r];
    }
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    if (A.gen[j]) {  // uniform
      const double g = a_block_sum((double)acc[j].h + (double)acc[j].l);
      if (threadIdx.x == 0) part[((size_t)A.slot[j] * Bc + b) * gridDim.x + blockIdx.x] = g;
    }
  }
}

// H = sum_t c_t P_t with Pauli strings grouped by their X/Y mask m:
// P|x> = i^{nY} (-1)^{popcount(x & z)} |x ^ m>, so
//   (H psi)_x = sum_groups f_g(x ^ m_g) psi_{x ^ m_g},
//   f_g(y) = sum_{t in g} w_t (-1)^{popcount(y & z_t)},  w_t = c_t i^{nY_t}.
struct HGroup {
  u64 m;
  int first, nt;
};
struct HTerm {
  u64 z;
  float wrh, wrl, wih, wil;  // w_t in double-float
};

__device__ __forceinline__ void hmul_acc(const HTerm* __restrict__ T, const HGroup& G, u64 y, float2 py, float2& acc) {
  float fr = 0.0f, fi = 0.0f;
  for (int t = 0; t < G.nt; ++t) {
    const HTerm w = T[G.first + t];
    const bool neg = __popcll(y & w.z) & 1;
    fr += neg ? -w.wrh : w.wrh;
    fi += neg ? -w.wih : w.wih;
  }
  acc.x = __fmaf_rn(fr, py.x, __fmaf_rn(-fi, py.y, acc.x));
  acc.y = __fmaf_rn(fr, py.y, __fmaf_rn(fi, py.x, acc.y));
}
__device__ __forceinline__ void hmul_acc(const HTerm* __restrict__ T, const HGroup& G, u64 y, float4 py,
                                         float4& acc) {
  dfl fr{0.0f, 0.0f}, fi{0.0f, 0.0f};
  for (int t = 0; t < G.nt; ++t) {
    const HTerm w = T[G.first + t];
    const float s = (__popcll(y & w.z) & 1) ? -1.0f : 1.0f;
    df_acc(fr, dfl{s * w.wrh, s * w.wrl});
    df_acc(fi, dfl{s * w.wih, s * w.wil});
  }
  fr.h = fast_two_sum(fr.h, fr.l, fr.l);
  fi.h = fast_two_sum(fi.h, fi.l, fi.l);
  const dfl re = dot2(fr.h, fr.l, py.x, py.y, -fi.h, -fi.l, py.z, py.w);
  const dfl im = dot2(fr.h, fr.l, py.z, py.w, fi.h, fi.l, py.x, py.y);
  const dfl ar = df_add(dfl{acc.x, acc.y}, re), ai = df_add(dfl{acc.z, acc.w}, im);
  acc = make_float4(ar.h, ar.l, ai.h, ai.l);
}
__device__ __forceinline__ void vzero(float2& v) { v = make_float2(0.0f, 0.0f); }
__device__ __forceinline__ void vzero(float4& v) { v = make_float4(0.0f, 0.0f, 0.0f, 0.0f); }
__device__ __forceinline__ dfl re_dot(float2 a, float2 b) { return dfl{__fmaf_rn(a.x, b.x, a.y * b.y), 0.0f}; }
__device__ __forceinline__ dfl re_dot(float4 a, float4 b) { return dot2(a.x, a.y, b.x, b.y, a.z, a.w, b.z, b.w); }

// lambda_b = H psi_b (every set b = blockIdx.y) and the partials of
// E_b = Re <psi_b|lambda_b>, part[b * gridDim.x + blockIdx.x], in one pass.
template <typename V>
__global__ void __launch_bounds__(kAT) k_hamiltonian(const V* __restrict__ psi, V* __restrict__ lam, u64 N,
                                                     const HGroup* __restrict__ groups, int ngroups,
                                                     const HTerm* __restrict__ terms, double* __restrict__ part) {
  const V* ps = psi + N * blockIdx.y;
  V* lm = lam + N * blockIdx.y;
  dfl e{0.0f, 0.0f};
  for (u64 x = (u64)blockIdx.x * kAT + threadIdx.x; x < N; x += (u64)gridDim.x * kAT) {
    V acc;
    vzero(acc);
    for (int g = 0; g < ngroups; ++g) {
      const HGroup G = groups[g];
      const u64 y = x ^ G.m;
      hmul_acc(terms, G, y, ps[y], acc);
    }
    lm[x] = acc;
    df_acc(e, re_dot(ps[x], acc));
  }
  const double s = a_block_sum((double)e.h + (double)e.l);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// out[s] = sum_{b < G} part[s * G + b], in order (one CTA per slot).
__global__ void __launch_bounds__(kAT) k_slot_sums(const double* part, int G, double* out) {
  double s = 0.0;
  const double* p = part + (size_t)blockIdx.x * G;
  for (int i = threadIdx.x; i < G; i += kAT) s += p[i];
  s = a_block_sum(s);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// CTAs per parameter set for every kernel of the sweep (one partial-sum
// layout): enough for the work, about the resident CTAs over the chunk's
// sets (few CTAs, each looping, keep the per-CTA set-up and reduction tail
// small), and a power of two so a thread's low index bits stay fixed.
unsigned adj_grid(u64 work, int Bc) {
  const u64 per = (u64)kAT * 4;
  u64 g = (work + per - 1) / per;
  u64 cap = (u64)sm_count() * 4 / (u64)Bc;
  if (cap < 1) cap = 1;
  if (g > cap) g = cap;
  unsigned p = 1;
  while ((u64)p * 2 <= g) p *= 2;
  return p;
}

// conjugate transpose of a 2x2 matrix
void dagger2(const double* m, double* d) {
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      d[2 * (r * 2 + c)] = m[2 * (c * 2 + r)];
      d[2 * (r * 2 + c) + 1] = -m[2 * (c * 2 + r) + 1];
    }
}

// Chunk budget for psi and lambda of Bc sets.  complex64: about half of L2,
// so the per-gate sweep re-reads the vectors from L2.  complex128: the
// double-float sweep is ALU-bound, and a larger chunk gives each launch more
// CTAs (measured at 20 qubits, 64 sets: 7.4 ms per set at 64 MB, 6.6 ms at
// 1 GB; complex64 2.85 ms at 64 MB, 2.95 ms at 1 GB).
int adj_chunk(int batch, u64 sbytes, bool df) {
  const u64 budget = df ? (1ull << 30) : (64ull << 20);
  int bc = 1;
  while (2 * bc <= batch && 2 * (u64)(2 * bc) * sbytes <= budget) bc *= 2;
  return bc;
}

// Run f on a view of `st` at another address / qubit count; the view borrows
// st's scratch buffer and hands any reallocation back.
template <typename F>
qs_status on_view(qs_state* st, void* amp, int n, F&& f) {
  qs_state v = *st;
  v.amp = amp;
  v.n = n;
  v.owns = false;
  const qs_status rc = f(&v);
  st->scratch = v.scratch;
  st->scratch_bytes = v.scratch_bytes;
  return rc;
}

// U^dagger of a fixed gate on a vector (or the chunk's combined vector);
// complex128 vectors are in double-float storage.
qs_status unapply_fixed(qs_state* v, const qs_gate_rec& g, bool dfl_layout) {
  double m[32];
  const int nq = gate_matrix(g.kind, g.p, m);
  if (nq == 1) {
    double md[8];
    dagger2(m, md);
    return dfl_layout ? run_controlled_dfl(v, nullptr, 0, g.q[0], md) : run_1q(v, g.q[0], md);
  }
  if (g.kind == QS_GATE_CNOT) {  // an exchange: the same in either storage
    double x[8];
    gate_matrix(QS_GATE_X, nullptr, x);
    return run_controlled(v, &g.q[0], 1, g.q[1], x);
  }
  if (g.kind == QS_GATE_SWAP) return run_bitswap(v, &g.q[0], &g.q[1], 1);
  double d[8];  // CZ, CP: conjugate of the diagonal
  for (int r = 0; r < 4; ++r) {
    d[2 * r] = m[2 * (r * 4 + r)];
    d[2 * r + 1] = -m[2 * (r * 4 + r) + 1];
  }
  return dfl_layout ? run_diag_dfl(v, g.q, 2, d) : run_diag(v, g.q, 2, d);
}

bool is_diag_kind(int k) {
  return k == QS_GATE_Z || k == QS_GATE_S || k == QS_GATE_T || k == QS_GATE_RZ || k == QS_GATE_P ||
         k == QS_GATE_CZ || k == QS_GATE_CP;
}

// The reverse sweep as steps: a trainable RX/RY (k_adj_1q), a fixed
// non-diagonal gate (per-gate kernels), or a run of diagonal gates
// (k_adj_diag).  Trainable gates get gradient slots in reverse order.
struct RunInfo {
  DRun R;
  std::vector<int> gates;  // circuit indices, in reverse order (factor order)
  size_t tab_off;          // first DFac of this run in the chunk's table (x Bc sets)
  int slot_base;
};
struct LayerInfo {
  int M;
  int gi[kLayerMax], slot[kLayerMax];
};
struct SweepStep {
  int kind;  // 0 trainable one-qubit, 1 fixed, 2 diagonal run, 3 layer of one-qubit gates
  int gi, slot, run;
};

bool layer_kind(const qs_gate_rec& g) { return gate_arity(g.kind) == 1 && !is_diag_kind(g.kind); }

void build_sweep(const qs_circuit* c, int Bc, int max_layer, int lgs, std::vector<SweepStep>& steps,
                 std::vector<RunInfo>& runs, std::vector<LayerInfo>& layers, size_t& nfac) {
  int slot = 0;
  nfac = 0;
  for (int gi = (int)c->gates.size() - 1; gi >= 0;) {
    const qs_gate_rec& g = c->gates[gi];
    if (layer_kind(g) && max_layer >= 2) {
      // consecutive one-qubit non-diagonal gates on distinct qubits
      LayerInfo li{};
      unsigned long long used = 0;
      int j = gi;
      while (j >= 0 && li.M < max_layer && layer_kind(c->gates[j]) && !((used >> c->gates[j].q[0]) & 1)) {
        used |= 1ull << c->gates[j].q[0];
        li.gi[li.M++] = j;
        --j;
      }
      if (li.M >= 2) {
        for (int k = 0; k < li.M; ++k) li.slot[k] = c->gates[li.gi[k]].param_index >= 0 ? slot++ : -1;
        steps.push_back(SweepStep{3, -1, -1, (int)layers.size()});
        layers.push_back(li);
        gi = j;
        continue;
      }
    }
    if (is_diag_kind(g.kind)) {
      RunInfo ri{};
      ri.slot_base = slot;
      ri.tab_off = nfac;
      while (gi >= 0 && is_diag_kind(c->gates[gi].kind) && ri.R.nf < kRunF) {
        const qs_gate_rec& d = c->gates[gi];
        if (d.param_index >= 0 && ri.R.ng == kRunG) break;
        const int f = ri.R.nf++;
        ri.R.q0[f] = d.q[0];
        ri.R.q1[f] = gate_arity(d.kind) == 2 ? d.q[1] : -1;
        ri.R.sign[f] = (d.kind == QS_GATE_CZ || d.kind == QS_GATE_Z) ? 1 : 0;
        if (d.param_index >= 0) ri.R.gq[ri.R.ng++] = d.q[0];
        ri.gates.push_back(gi);
        --gi;
      }
      // factors on qubits below the stride bits first (they commute)
      {
        std::vector<int> order(ri.R.nf);
        for (int f = 0; f < ri.R.nf; ++f) order[f] = f;
        auto low = [&](int f) { return ri.R.q0[f] < lgs && ri.R.q1[f] < lgs; };
        std::stable_partition(order.begin(), order.end(), low);
        DRun R2 = ri.R;
        std::vector<int> g2(ri.R.nf);
        for (int f = 0; f < ri.R.nf; ++f) {
          R2.q0[f] = ri.R.q0[order[f]];
          R2.q1[f] = ri.R.q1[order[f]];
          R2.sign[f] = ri.R.sign[order[f]];
          g2[f] = ri.gates[order[f]];
        }
        R2.nlo = 0;
        while (R2.nlo < R2.nf && low(order[R2.nlo])) ++R2.nlo;
        ri.R = R2;
        ri.gates = g2;
      }
      slot += ri.R.ng;
      nfac += (size_t)ri.R.nf * Bc;
      steps.push_back(SweepStep{2, -1, ri.slot_base, (int)runs.size()});
      runs.push_back(std::move(ri));
      continue;
    }
    if (g.param_index >= 0) steps.push_back(SweepStep{0, gi, slot++, -1});
    else steps.push_back(SweepStep{1, gi, -1, -1});
    --gi;
  }
}

// U^dagger diagonal of a diagonal gate with angle p (p[0] replaced for a
// trainable gate), as a double-float factor
DFac diag_factor(const qs_gate_rec& g, const double* p) {
  double m[32];
  const int nq = gate_matrix(g.kind, p, m);
  const int D = 1 << nq;
  DFac F{};
  for (int r = 0; r < 4; ++r) {
    const int rr = r < D ? r : 0;
    const double re = m[2 * (rr * D + rr)], im = -m[2 * (rr * D + rr) + 1];  // conjugate
    F.rh[r] = (float)re;
    F.rl[r] = (float)(re - (double)F.rh[r]);
    F.ih[r] = (float)im;
    F.il[r] = (float)(im - (double)F.ih[r]);
  }
  return F;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename V, typename Mat>
qs_status launch_layer(const LayerInfo& li, const qs_circuit* c, V* psi, V* lam, u64 N, unsigned G, int cnt,
                       const Mat* mats, double* part, int Bc, cudaStream_t stream) {
  LayerArgs<Mat> A{};
  int qs_sorted[kLayerMax];
  for (int j = 0; j < li.M; ++j) {
    const qs_gate_rec& g = c->gates[li.gi[j]];
    A.q[j] = g.q[0];
    qs_sorted[j] = g.q[0];
    if (g.param_index >= 0) {
      A.gen[j] = g.kind == QS_GATE_RX ? 1 : g.kind == QS_GATE_RY ? 2 : 3;
      A.slot[j] = li.slot[j];
    } else {
      double m[32], md[8];
      gate_matrix(g.kind, g.p, m);
      dagger2(m, md);
      A.fixed[j] = to_mat(md, typename std::conditional<sizeof(V) == 8, float, double>::type(0));
    }
  }
  small_sort(qs_sorted, li.M, [](int x, int y) { return x < y; });
  A.ins.k = li.M;
  A.ins.set = 0;
  for (int j = 0; j < li.M; ++j) A.ins.pos[j] = qs_sorted[j];
  const dim3 grid(G, cnt);
  if (li.M == 2) {
    k_adj_layer<V, Mat, 2><<<grid, kAT, 0, stream>>>(psi, lam, N, A, mats, part, Bc);
  } else if constexpr (sizeof(V) == 8) {  // complex64 layers of up to 4 (registers)
    if (li.M == 3) k_adj_layer<V, Mat, 3><<<grid, kAT, 0, stream>>>(psi, lam, N, A, mats, part, Bc);
    else if (li.M == 4) k_adj_layer<V, Mat, 4><<<grid, kAT, 0, stream>>>(psi, lam, N, A, mats, part, Bc);
    else return fail(QS_EINVAL, "adjoint layer of %d gates", li.M);
  } else {
    return fail(QS_EINVAL, "adjoint layer of %d gates", li.M);
  }
  return launch_ok("k_adj_layer");
}

template <typename R>
qs_status adjoint_run(qs_state* st, const qs_circuit* c, const double* theta, int nparam, int batch, int nterms,
                      const u64* xmask, const u64* zmask, const double* coeff, double* energy, double* grad) {
  typedef typename Ar<R>::Mat Mat;
  typedef typename Amp<R>::V V;
  const bool df = sizeof(R) == 8;
  const int n = st->n;
  const u64 N = u64(1) << n;
  const size_t sbytes = state_bytes(st);
  const int Bc = adj_chunk(batch, sbytes, df);
  int lb = 0;
  while ((1 << lb) < Bc) ++lb;
  const unsigned G = adj_grid(N >> 1, Bc);

  // trainable gates in reverse order: slot s <-> gate index
  std::vector<int> slot_gate;
  for (int gi = (int)c->gates.size() - 1; gi >= 0; --gi)
    if (c->gates[gi].param_index >= 0) slot_gate.push_back(gi);
  const int nslots = (int)slot_gate.size() + 1;  // trainable gates, then the energy
  const int eslot = nslots - 1;
  std::vector<SweepStep> steps;
  std::vector<RunInfo> runs;
  std::vector<LayerInfo> layers;
  size_t nfac = 0;
  int lgs = 0;  // log2 of a sweep kernel's grid stride
  while ((1ull << lgs) < (u64)G * kAT) ++lgs;
  build_sweep(c, Bc, df ? 2 : 3, lgs, steps, runs, layers, nfac);  // widths measured best

  // Hamiltonian grouped by X/Y mask, in order of first appearance
  std::vector<HGroup> hg;
  std::vector<HTerm> ht;
  {
    std::map<u64, std::vector<int>> by_m;
    std::vector<u64> order;
    for (int t = 0; t < nterms; ++t) {
      if (!by_m.count(xmask[t])) order.push_back(xmask[t]);
      by_m[xmask[t]].push_back(t);
    }
    for (u64 m : order) {
      HGroup g{m, (int)ht.size(), (int)by_m[m].size()};
      hg.push_back(g);
      for (int t : by_m[m]) {
        const int ny = __builtin_popcountll(xmask[t] & zmask[t]) & 3;  // i^{nY}
        const double pr[4] = {1, 0, -1, 0}, pim[4] = {0, 1, 0, -1};
        const double wr = coeff[t] * pr[ny], wi = coeff[t] * pim[ny];
        HTerm w;
        w.z = zmask[t];
        w.wrh = (float)wr;
        w.wrl = (float)(wr - (double)w.wrh);
        w.wih = (float)wi;
        w.wil = (float)(wi - (double)w.wih);
        ht.push_back(w);
      }
    }
  }

  // device: [psi/lambda chunk (Bc > 1) or lambda][partials][sums][mats][groups][terms]
  const size_t vec_b = up256((Bc > 1 ? 2 * (size_t)Bc : 1) * sbytes);
  const size_t part_b = up256(sizeof(double) * (size_t)nslots * Bc * G);
  const size_t sums_b = up256(sizeof(double) * (size_t)nslots * Bc);
  const size_t mats_b = up256(sizeof(Mat) * (size_t)nslots * Bc);
  const size_t grp_b = up256(sizeof(HGroup) * hg.size()), trm_b = up256(sizeof(HTerm) * ht.size());
  const size_t fac_b = up256(sizeof(DFac) * (nfac > 0 ? nfac : 1));
  const size_t bytes = vec_b + part_b + sums_b + mats_b + grp_b + trm_b + fac_b;
  char* dev = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dev), bytes, st->stream);
  if (e != cudaSuccess) return fail(QS_ENOMEM, "qs_adjoint_grad: %zu bytes: %s", bytes, cudaGetErrorString(e));
  char* psi = Bc > 1 ? dev : static_cast<char*>(st->amp);
  char* lam = Bc > 1 ? dev + (size_t)Bc * sbytes : dev;
  double* part = reinterpret_cast<double*>(dev + vec_b);
  double* sums = reinterpret_cast<double*>(dev + vec_b + part_b);
  Mat* mats = reinterpret_cast<Mat*>(dev + vec_b + part_b + sums_b);
  HGroup* dgrp = reinterpret_cast<HGroup*>(dev + vec_b + part_b + sums_b + mats_b);
  HTerm* dtrm = reinterpret_cast<HTerm*>(dev + vec_b + part_b + sums_b + mats_b + grp_b);
  DFac* dfac = reinterpret_cast<DFac*>(dev + vec_b + part_b + sums_b + mats_b + grp_b + trm_b);
  std::vector<DFac> hfac(nfac);
  qs_status rc = QS_OK;
  e = cudaMemcpyAsync(dgrp, hg.data(), sizeof(HGroup) * hg.size(), cudaMemcpyHostToDevice, st->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dtrm, ht.data(), sizeof(HTerm) * ht.size(), cudaMemcpyHostToDevice, st->stream);
  // padded sets of a short last chunk stay finite: they pass through the
  // fixed-gate launches but are never read
  if (e == cudaSuccess && Bc > 1) e = cudaMemsetAsync(dev, 0, 2 * (size_t)Bc * sbytes, st->stream);
  if (e != cudaSuccess) rc = cuda_fail(e, "qs_adjoint_grad: setup");

  // targets of the fixed-gate launches
  std::vector<std::pair<char*, int>> targets;
  if (Bc > 1) targets.push_back({psi, n + lb + 1});
  else targets = {{psi, n}, {lam, n}};

  std::vector<Mat> hmats((size_t)nslots * Bc);
  std::vector<double> hsums((size_t)nslots * Bc);
  qs_circuit cb;
  cb.gates = c->gates;
  for (int c0 = 0; c0 < batch && rc == QS_OK; c0 += Bc) {
    const int cnt = batch - c0 < Bc ? batch - c0 : Bc;
    // forward: one compiled plan per parameter set, run on psi_b
    for (int b = 0; b < cnt && rc == QS_OK; ++b) {
      const double* th = theta + (size_t)(c0 + b) * nparam;
      for (qs_gate_rec& g : cb.gates)
        if (g.param_index >= 0) g.p[0] = th[g.param_index];
      qs_plan* plan = nullptr;
      if ((rc = qs_plan_build(&cb, n, st->dtype, nullptr, &plan)) != QS_OK) break;
      rc = on_view(st, psi + (size_t)b * sbytes, n, [&](qs_state* v) {
        qs_status r = run_set_basis(v, 0);
        return r == QS_OK ? qs_run_plan(v, plan) : r;
      });
      qs_plan_destroy(plan);
      for (size_t s = 0; s < slot_gate.size(); ++s) {  // U^dagger of each trainable gate
        const qs_gate_rec& g = cb.gates[slot_gate[s]];
        if (is_diag_kind(g.kind)) continue;  // in a diagonal run's table
        double m[32], md[8];
        gate_matrix(g.kind, g.p, m);
        dagger2(m, md);
        hmats[s * Bc + b] = to_mat(md, R(0));
      }
      for (const RunInfo& ri : runs)  // diagonal-run factors of this set
        for (int f = 0; f < ri.R.nf; ++f) {
          const qs_gate_rec& g = cb.gates[ri.gates[f]];
          hfac[ri.tab_off + (size_t)b * ri.R.nf + f] = diag_factor(g, g.p);
        }
    }
    if (rc != QS_OK) break;
    if (!slot_gate.empty()) {
      e = cudaMemcpyAsync(mats, hmats.data(), sizeof(Mat) * hmats.size(), cudaMemcpyHostToDevice, st->stream);
      if (e != cudaSuccess) { rc = cuda_fail(e, "qs_adjoint_grad: matrix upload"); break; }
    }
    if (nfac > 0) {
      e = cudaMemcpyAsync(dfac, hfac.data(), sizeof(DFac) * nfac, cudaMemcpyHostToDevice, st->stream);
      if (e != cudaSuccess) { rc = cuda_fail(e, "qs_adjoint_grad: diagonal factor upload"); break; }
    }
    if (df) {  // psi of the chunk to double-float storage; lambda is written in it
      rc = on_view(st, psi, n + lb, [&](qs_state* v) { return run_layout_dfl(v, true); });
      if (rc != QS_OK) break;
    }
    // lambda_b = H psi_b and E_b
    k_hamiltonian<V><<<dim3(G, cnt), kAT, 0, st->stream>>>(reinterpret_cast<const V*>(psi), reinterpret_cast<V*>(lam),
                                                          N, dgrp, (int)hg.size(), dtrm,
                                                          part + (size_t)eslot * Bc * G);
    if ((rc = launch_ok("k_hamiltonian")) != QS_OK) break;
    // reverse sweep
    for (size_t si = 0; si < steps.size() && rc == QS_OK; ++si) {
      const SweepStep& sp = steps[si];
      if (sp.kind == 2) {
        const RunInfo& ri = runs[sp.run];
        k_adj_diag<V><<<dim3(G, cnt), kAT, 0, st->stream>>>(reinterpret_cast<V*>(psi), reinterpret_cast<V*>(lam), N,
                                                           ri.R, dfac + ri.tab_off, part + (size_t)ri.slot_base * Bc * G,
                                                           Bc, lgs);
        rc = launch_ok("k_adj_diag");
        continue;
      }
      if (sp.kind == 3) {
        rc = launch_layer<V, Mat>(layers[sp.run], c, reinterpret_cast<V*>(psi), reinterpret_cast<V*>(lam), N, G, cnt,
                                  mats, part, Bc, st->stream);
        continue;
      }
      const qs_gate_rec& g = c->gates[sp.gi];
      if (sp.kind == 0) {
        const int gen = g.kind == QS_GATE_RX ? 1 : g.kind == QS_GATE_RY ? 2 : 3;
        k_adj_1q<V, Mat><<<dim3(G, cnt), kAT, 0, st->stream>>>(reinterpret_cast<V*>(psi), reinterpret_cast<V*>(lam), N,
                                                               N >> 1, g.q[0], mats + (size_t)sp.slot * Bc, gen,
                                                               part + (size_t)sp.slot * Bc * G);
        rc = launch_ok("k_adj_1q");
        continue;
      }
      for (size_t t = 0; t < targets.size() && rc == QS_OK; ++t)
        rc = on_view(st, targets[t].first, targets[t].second, [&](qs_state* v) { return unapply_fixed(v, g, df); });
    }
    if (rc != QS_OK) break;
    k_slot_sums<<<nslots * Bc, kAT, 0, st->stream>>>(part, (int)G, sums);
    if ((rc = launch_ok("k_slot_sums")) != QS_OK) break;
    e = cudaMemcpyAsync(hsums.data(), sums, sizeof(double) * hsums.size(), cudaMemcpyDeviceToHost, st->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
    if (e != cudaSuccess) { rc = cuda_fail(e, "qs_adjoint_grad: gradient readback"); break; }
    for (int b = 0; b < cnt; ++b) {
      energy[c0 + b] = hsums[(size_t)eslot * Bc + b];
      if (nparam == 0) continue;
      double* gb = grad + (size_t)(c0 + b) * nparam;
      for (int j = 0; j < nparam; ++j) gb[j] = 0.0;
      for (size_t s = 0; s < slot_gate.size(); ++s) gb[c->gates[slot_gate[s]].param_index] += hsums[s * Bc + b];
    }
  }
  // the caller's state back in plain storage
  if (rc == QS_OK && df && Bc == 1) rc = run_layout_dfl(st, false);
  cudaFreeAsync(dev, st->stream);
  if (rc == QS_OK) {
    e = cudaStreamSynchronize(st->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "qs_adjoint_grad: sync");
  }
  return rc;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_adjoint_grad(qs_state* st, const qs_circuit* c, const double* theta, int nparam, int batch,
                                     int nterms, const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                                     double* energy, double* grad) {
  if (!st || !c || !energy || (nparam > 0 && (!theta || !grad)))
    return fail(QS_EINVAL, "qs_adjoint_grad: NULL argument");
  if (nparam < 0 || batch < 1) return fail(QS_EINVAL, "qs_adjoint_grad: nparam >= 0 and batch >= 1 required");
  if (nterms < 1 || nterms > 65536 || !xmask || !zmask || !coeff)
    return fail(QS_EINVAL, "qs_adjoint_grad: need 1 <= nterms <= 65536 and non-NULL term arrays");
  const int n = st->n;
  const uint64_t lim = (1ull << n) - 1;
  for (int t = 0; t < nterms; ++t)
    if ((xmask[t] & ~lim) || (zmask[t] & ~lim)) return fail(QS_EINVAL, "qs_adjoint_grad: term %d acts on a qubit >= n", t);
  for (size_t i = 0; i < c->gates.size(); ++i) {
    const qs_gate_rec& g = c->gates[i];
    if (g.q[0] >= n || g.q[1] >= n) return fail(QS_EINVAL, "qs_adjoint_grad: gate %zu acts on a qubit >= n", i);
    if (g.param_index >= nparam) return fail(QS_EINVAL, "qs_adjoint_grad: gate %zu uses parameter %d >= nparam", i, g.param_index);
  }
  return st->dtype == QS_C64
             ? adjoint_run<float>(st, c, theta, nparam, batch, nterms, xmask, zmask, coeff, energy, grad)
             : adjoint_run<double>(st, c, theta, nparam, batch, nterms, xmask, zmask, coeff, energy, grad);
}
