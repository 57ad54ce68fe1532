// Computational-basis measurement (§II-A: a circuit is a sequence of gates,
// measurements and resets): marginal probabilities, the collapse after a
// single-qubit measurement, and sampling of basis states.
//
// Probabilities follow the Born rule, p_x = |a_x|^2.  The squares are formed
// exactly in double-float (FP32 pairs with their rounding errors) and summed
// in double-float, flushed into FP64 where a sum leaves a thread: FP64-level
// accuracy without the FP64 pipe (about 1/64 of the FP32 rate on GB300).
//
// Sampling inverts the cumulative distribution in index order,
// F(x) = p_0 + ... + p_x: a uniform u gives t = u T (T = F(2^n - 1)) and the
// sample is the x with F(x - 1) <= t < F(x).  The search runs on the GPU in
// three levels of partial sums -- superchunks of 32 chunks, chunks of 32 lane
// ranges, lane ranges of 32 amplitudes -- one warp per shot, each level a
// 32-wide ballot over prefix sums.  Its sums are taken in another order than
// a sequential one, so near a boundary of F (within the rounding of the
// sums, a few 2^-53 T per term) either neighbour can be returned; elsewhere
// the result is the exact inverse.  An index with p_x = 0 is never returned.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "kcommon.cuh"

namespace qs {
namespace {

constexpr int kMT = 256;        // threads per CTA
constexpr int kBins = 8;        // outcomes per marginal pass
// Sampling levels: a lane range is 32 consecutive amplitudes, a chunk 32 lane
// ranges (1024 amplitudes), a superchunk 32 chunks.
constexpr u64 kChunk = 1024;
constexpr int kSuper = 32;
constexpr u64 kShotBatch = u64(1) << 20;
constexpr int kPrefixThreads = 1024;

struct MargArgs {
  Ins ins;          // zero insertion at the measured qubits
  u64 spread[64];   // spread[r]: OR of 2^qubits[i] over the set bits i of r
  u64 free;         // the other qubits' bits (a group base's bits)
  u64 step1, stepU; // masked-add steps: the bases of the groups stride and kMargU strides on
};

// p = x^2 into a double-float sum: the FP32 square exactly as p + e
// (FMA), p added exactly (TwoSum), e and the TwoSum error into the low part
__device__ __forceinline__ void sq_acc(dfl& acc, float x) {
  const float p = __fmul_rn(x, x), e = __fmaf_rn(x, x, -p);
  float t;
  acc.h = two_sum(acc.h, p, t);
  acc.l = __fadd_rn(acc.l, __fadd_rn(e, t));
}
__device__ __forceinline__ void sq_acc(dfl& acc, double x) {
  const dfl d = d2df(x);
  df_acc(acc, df_mul(d, d));
}

// Outcomes [b0, b0 + NB): each thread sums its groups (the other qubits) in
// grid-stride order, kMargU groups at a time (their 8 loads issued first),
// the squares exact in double-float, flushed into FP64 every kMargFlush
// groups (the low float then holds at most 2 kMargFlush rounding errors of
// the TwoSums, ~2^-43 of the sum); the CTA reduces every bin into
// part[blockIdx.x * kBins + j].
constexpr int kMargFlush = 16;
template <int NB> struct MargU { static constexpr int value = NB >= 8 ? 1 : 8 / NB; };
template <typename A, int NB>
__global__ void __launch_bounds__(kMT, (NB >= 8 && sizeof(A) > 8) ? 2 : 3) k_marginal(const A* __restrict__ a, u64 ngroups,
                                                  const __grid_constant__ MargArgs args, int b0,
                                                  double* __restrict__ part) {
  constexpr int kMargU = MargU<NB>::value;
  double acc[NB];
  dfl da[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    acc[j] = 0.0;
    da[j] = dfl{0.f, 0.f};
  }
  // bases of groups g, g + stride, ...: the group index's bits at the
  // other qubits, advanced by masked adds (carries skip the measured qubits)
  const u64 stride = (u64)gridDim.x * kMT;
  u64 g = (u64)blockIdx.x * kMT + threadIdx.x;
  u64 base[kMargU];
  base[0] = expand(g, args.ins);
#pragma unroll
  for (int u = 1; u < kMargU; ++u) base[u] = ((base[u - 1] | ~args.free) + args.step1) & args.free;
  int since = 0;
  for (; g + (kMargU - 1) * stride < ngroups; g += kMargU * stride) {
    A v[kMargU][NB];
#pragma unroll
    for (int u = 0; u < kMargU; ++u)
#pragma unroll
      for (int j = 0; j < NB; ++j) v[u][j] = a[base[u] | args.spread[b0 + j]];
#pragma unroll
    for (int u = 0; u < kMargU; ++u) {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        sq_acc(da[j], v[u][j].x);
        sq_acc(da[j], v[u][j].y);
      }
      base[u] = ((base[u] | ~args.free) + args.stepU) & args.free;
    }
    since += kMargU;
    if (since >= kMargFlush) {
#pragma unroll
      for (int j = 0; j < NB; ++j) df_flush(acc[j], da[j]);
      since = 0;
    }
  }
  for (u64 b = base[0]; g < ngroups; g += stride, b = ((b | ~args.free) + args.step1) & args.free) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const A v = a[b | args.spread[b0 + j]];
      sq_acc(da[j], v.x);
      sq_acc(da[j], v.y);
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) df_flush(acc[j], da[j]);
  __shared__ double red[kMT / 32][kBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    double v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < NB) {
    double s = 0.0;
    for (int w = 0; w < kMT / 32; ++w) s += red[w][threadIdx.x];
    part[(u64)blockIdx.x * kBins + threadIdx.x] = s;
  }
}

// Collapse onto `outcome` of qubit q: the kept amplitude of every pair
// (x, x | 2^q) is scaled by sc, the other set to 0.
template <typename A, typename R>
__global__ void __launch_bounds__(kMT) k_collapse(A* __restrict__ a, u64 npairs, Ins ins, u64 qbit, int outcome,
                                                  R sc) {
  const u64 stride = (u64)gridDim.x * kMT;
  for (u64 i = (u64)blockIdx.x * kMT + threadIdx.x; i < npairs; i += stride) {
    const u64 x0 = expand(i, ins), x1 = x0 | qbit;
    const u64 keep = outcome ? x1 : x0, drop = outcome ? x0 : x1;
    A v = a[keep];
    v.x *= sc;
    v.y *= sc;
    a[keep] = v;
    A z;
    z.x = 0;
    z.y = 0;
    a[drop] = z;
  }
}

// p_x as a double-float: each square exact (TwoProd), their sum rounded once
// in double-float.
__device__ __forceinline__ dfl prob_df(float2 v) {
  const dfl x = to_df(v.x), y = to_df(v.y);
  dfl r = df_mul(x, x);
  df_acc(r, df_mul(y, y));
  return r;
}
__device__ __forceinline__ dfl prob_df(double2 v) {
  const dfl x = to_df(v.x), y = to_df(v.y);
  dfl r = df_mul(x, x);
  df_acc(r, df_mul(y, y));
  return r;
}
__device__ __forceinline__ dfl df_norm(dfl a) {
  dfl r;
  r.h = fast_two_sum(a.h, a.l, r.l);
  return r;
}
__device__ __forceinline__ dfl df_shfl_up(dfl v, int d) {
  return dfl{__shfl_up_sync(0xffffffffu, v.h, d), __shfl_up_sync(0xffffffffu, v.l, d)};
}
__device__ __forceinline__ dfl df_shfl(dfl v, int src) {
  return dfl{__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src)};
}
// a > b for normalised double-floats
__device__ __forceinline__ bool df_gt(dfl a, dfl b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }
// Inclusive prefix over the warp's lanes, in double-float.
__device__ __forceinline__ dfl df_warp_incl(dfl v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const dfl o = df_shfl_up(v, d);
    if (lane >= d) v = df_add(v, o);
  }
  return v;
}
__device__ __forceinline__ double dbl_warp_incl(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}
__device__ __forceinline__ dfl to_dfl_of(double x) {
  dfl r;
  r.h = (float)x;
  r.l = (float)(x - (double)r.h);
  return r;
}

// Level sums: S1[c] for every chunk (1024 amplitudes) and S2[s] for every
// superchunk (32 chunks), one warp per superchunk; lanes read the chunk
// coalesced (amplitude cC + lane + 32 i).
template <typename A>
__global__ void __launch_bounds__(kMT) k_sample_sums(const A* __restrict__ a, u64 N, u64 nch, u64 nsc,
                                                     double* __restrict__ S1, double* __restrict__ S2) {
  const int lane = threadIdx.x & 31;
  const u64 wstride = (u64)gridDim.x * (kMT / 32);
  for (u64 sc = (u64)blockIdx.x * (kMT / 32) + (threadIdx.x >> 5); sc < nsc; sc += wstride) {
    dfl s2{0.f, 0.f};
    for (int j = 0; j < kSuper; ++j) {
      const u64 c = sc * kSuper + j;
      if (c >= nch) break;
      const u64 x0 = c * kChunk;
      dfl acc{0.f, 0.f};
      if (x0 + kChunk <= N) {
#pragma unroll 8
        for (int i = 0; i < 32; ++i) {
          const dfl p = prob_df(a[x0 + lane + 32 * i]);
          df_acc(acc, p);
        }
      } else {
        for (u64 x = x0 + lane; x < N; x += 32) df_acc(acc, prob_df(a[x]));
      }
      acc = df_norm(acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const dfl t{__shfl_xor_sync(0xffffffffu, acc.h, o), __shfl_xor_sync(0xffffffffu, acc.l, o)};
        acc = df_add(acc, t);
      }
      if (lane == 0) S1[c] = (double)acc.h + (double)acc.l;
      s2 = df_add(s2, acc);
    }
    if (lane == 0) S2[sc] = (double)s2.h + (double)s2.l;
  }
}

// Exclusive prefix of the superchunk sums, P2[s] = S2[0] + ... + S2[s - 1],
// and P2[nsc] = T: one CTA, each thread a contiguous run summed in order.
__global__ void __launch_bounds__(kPrefixThreads) k_sample_prefix(const double* __restrict__ S2, u64 nsc,
                                                                  double* __restrict__ P2) {
  __shared__ double wsum[kPrefixThreads / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const u64 run = (nsc + kPrefixThreads - 1) / kPrefixThreads;
  const u64 b = (u64)t * run, e = b + run < nsc ? b + run : nsc;
  double tot = 0.0;
  for (u64 i = b; i < e; ++i) tot += S2[i];
  const double incl = dbl_warp_incl(tot);
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    const double v = wsum[lane];
    const double wi = dbl_warp_incl(v);
    wsum[lane] = wi - v;  // exclusive (rounding only shifts this warp's offset)
    if (lane == 31) P2[nsc] = wi;
  }
  __syncthreads();
  double r = wsum[w] + (incl - tot);
  for (u64 i = b; i < e; ++i) {
    P2[i] = r;
    r += S2[i];
  }
}

// One warp per shot: t = u T, then at each level the 32 candidate partial
// sums are prefixed across the lanes and a ballot picks the first one that
// passes t and is not zero.  Where t sits at T itself after rounding (or on
// a rounding difference between two levels' sums) and no candidate passes,
// the last nonzero candidate is taken, so a returned index always has
// p_x > 0 (in double-float) whenever T > 0.
template <typename A>
__global__ void __launch_bounds__(kMT) k_sample_shots(const A* __restrict__ a, u64 N, u64 nch, u64 nsc,
                                                      const double* __restrict__ S1, const double* __restrict__ S2,
                                                      const double* __restrict__ P2, const double* __restrict__ u,
                                                      u64 nshots, u64* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const double T = P2[nsc];
  const u64 wstride = (u64)gridDim.x * (kMT / 32);
  for (u64 i = (u64)blockIdx.x * (kMT / 32) + (threadIdx.x >> 5); i < nshots; i += wstride) {
    const double t = u[i] * T;
    // superchunk: the largest s with P2[s] <= t (P2[0] = 0 <= t always),
    // 32-ary: each round the lanes probe 32 evenly spaced candidates
    u64 lo = 0, len = nsc;
    while (len > 1) {
      const u64 step = (len + 31) / 32, off = (u64)lane * step;
      const unsigned m = __ballot_sync(0xffffffffu, off < len && P2[lo + off] <= t);
      const u64 j = (u64)(31 - __clz(m));
      lo += j * step;
      len = len - j * step < step ? len - j * step : step;
    }
    u64 sc = lo;
    if (!(S2[sc] > 0.0)) {
      // the nearest superchunk at or below with a nonzero sum (T > 0: one exists)
      for (long long s0 = (long long)sc; s0 >= 0; s0 -= 32) {
        const long long idx = s0 - lane;
        const unsigned mz = __ballot_sync(0xffffffffu, idx >= 0 && S2[idx] > 0.0);
        if (mz) {
          sc = (u64)(s0 - (__ffs(mz) - 1));
          break;
        }
      }
    }
    // chunk within the superchunk
    const double base = P2[sc];
    const u64 c0 = sc * kSuper;
    const double v = c0 + lane < nch ? S1[c0 + lane] : 0.0;
    const double incl = dbl_warp_incl(v);
    unsigned m = __ballot_sync(0xffffffffu, v > 0.0 && base + incl > t);
    int j = m ? __ffs(m) - 1 : 31 - __clz(__ballot_sync(0xffffffffu, v > 0.0));
    j = j < 0 ? 0 : j;  // (S2[sc] > 0, so some v > 0: kept in range regardless)
    const double ex1 = __shfl_sync(0xffffffffu, incl, j > 0 ? j - 1 : 0);
    const double base1 = base + (j > 0 ? ex1 : 0.0);
    const u64 c = c0 + (u64)j;
    const dfl tq = to_dfl_of(t - base1);
    // lane range within the chunk: lane l sums amplitudes cC + 32 l .. + 31
    const u64 xl = c * kChunk + (u64)lane * 32;
    dfl L{0.f, 0.f};
    if (xl + 32 <= N) {
#pragma unroll 8
      for (int k = 0; k < 32; ++k) df_acc(L, prob_df(a[xl + k]));
    } else {
      for (u64 x = xl; x < N; ++x) df_acc(L, prob_df(a[x]));
    }
    L = df_norm(L);
    const dfl inclL = df_warp_incl(L);
    m = __ballot_sync(0xffffffffu, L.h > 0.f && df_gt(inclL, tq));
    int j0 = m ? __ffs(m) - 1 : 31 - __clz(__ballot_sync(0xffffffffu, L.h > 0.f));
    j0 = j0 < 0 ? 0 : j0;
    dfl ex0 = df_shfl(inclL, j0 > 0 ? j0 - 1 : 0);
    if (j0 == 0) ex0 = dfl{0.f, 0.f};
    // amplitude within the lane range
    const u64 x = c * kChunk + (u64)j0 * 32 + lane;
    const dfl p = x < N ? df_norm(prob_df(a[x])) : dfl{0.f, 0.f};
    const dfl inclp = df_add(ex0, df_warp_incl(p));
    m = __ballot_sync(0xffffffffu, p.h > 0.f && df_gt(inclp, tq));
    int j1 = m ? __ffs(m) - 1 : 31 - __clz(__ballot_sync(0xffffffffu, p.h > 0.f));
    j1 = j1 < 0 ? 0 : j1;
    if (lane == 0) out[i] = c * kChunk + (u64)j0 * 32 + (u64)j1;
  }
}

Ins ins_for(const int* qubits, int k) {
  Ins ins{};
  ins.k = k;
  ins.set = 0;
  for (int i = 0; i < k && i < 6; ++i) {  // insertion sort of at most 6 qubits
    int j = i;
    for (; j > 0 && ins.pos[j - 1] > qubits[i]; --j) ins.pos[j] = ins.pos[j - 1];
    ins.pos[j] = qubits[i];
  }
  return ins;
}

qs_status sync_copy(qs_state* s, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? QS_OK : cuda_fail(e, "measure: copy");
}

template <typename A>
qs_status marginal(qs_state* s, const int* qubits, int k, double* out) {
  MargArgs args{};
  args.ins = ins_for(qubits, k);
  for (int r = 0; r < (1 << k); ++r) {
    u64 sp = 0;
    for (int i = 0; i < k; ++i)
      if ((r >> i) & 1) sp |= u64(1) << qubits[i];
    args.spread[r] = sp;
  }
  const u64 ngroups = u64(1) << (s->n - k);
  // one wave of resident CTAs (3 per SM; 2 for complex128 passes of 8 bins)
  const unsigned g = grid_for(ngroups, kMT, ((1 << k) >= kBins && s->dtype == QS_C128) ? 2 : 3);
  args.free = (u64(1) << s->n) - 1;
  for (int i = 0; i < k; ++i) args.free &= ~(u64(1) << qubits[i]);
  const u64 stride = (u64)g * kMT;
  args.step1 = expand(stride, args.ins);
  // every pass writes its own partials; one read-back after the last
  const int npass = ((1 << k) + kBins - 1) / kBins;
  const size_t per = (size_t)kBins * g;
  qs_status st = ensure_scratch(s, sizeof(double) * per * npass);
  if (st != QS_OK) return st;
  double* part = static_cast<double*>(s->scratch);
  std::vector<double> h(per * npass);
  for (int b0 = 0; b0 < (1 << k); b0 += kBins) {
    const int nb = std::min(kBins, (1 << k) - b0);  // 2, 4 or 8
    const A* amp = static_cast<const A*>(s->amp);
    const int U = nb == 2 ? MargU<2>::value : nb == 4 ? MargU<4>::value : MargU<8>::value;
    args.stepU = expand((u64)U * stride, args.ins);
    double* pp = part + per * (size_t)(b0 / kBins);
    if (nb == 2) k_marginal<A, 2><<<g, kMT, 0, s->stream>>>(amp, ngroups, args, b0, pp);
    else if (nb == 4) k_marginal<A, 4><<<g, kMT, 0, s->stream>>>(amp, ngroups, args, b0, pp);
    else k_marginal<A, 8><<<g, kMT, 0, s->stream>>>(amp, ngroups, args, b0, pp);
    if ((st = launch_ok("k_marginal")) != QS_OK) return st;
  }
  if ((st = sync_copy(s, h.data(), part, sizeof(double) * per * npass, cudaMemcpyDeviceToHost)) != QS_OK) return st;
  for (int b0 = 0; b0 < (1 << k); b0 += kBins) {
    const int nb = std::min(kBins, (1 << k) - b0);
    const double* hp = h.data() + per * (size_t)(b0 / kBins);
    for (int j = 0; j < nb; ++j) {
      double sum = 0.0;
      for (unsigned c = 0; c < g; ++c) sum += hp[(size_t)c * kBins + j];
      out[b0 + j] = sum;
    }
  }
  return QS_OK;
}

template <typename A, typename R>
qs_status collapse(qs_state* s, int q, int outcome, double p) {
  const u64 npairs = u64(1) << (s->n - 1);
  const unsigned g = grid_for(npairs, kMT, 8);
  k_collapse<A, R><<<g, kMT, 0, s->stream>>>(static_cast<A*>(s->amp), npairs, ins_for(&q, 1), u64(1) << q, outcome,
                                             (R)(1.0 / std::sqrt(p)));
  return launch_ok("k_collapse");
}

template <typename A>
qs_status sample(qs_state* s, u64 nshots, const double* u, uint64_t* out) {
  const u64 N = u64(1) << s->n;
  const u64 nch = (N + kChunk - 1) / kChunk, nsc = (nch + kSuper - 1) / kSuper;
  const u64 batch = std::min(nshots, kShotBatch);
  // scratch: S1 (nch), S2 (nsc), P2 (nsc + 1), uniforms and results of one
  // batch of shots
  const size_t need = sizeof(double) * (nch + 2 * nsc + 1) + batch * (sizeof(double) + sizeof(u64));
  qs_status st = ensure_scratch(s, need);
  if (st != QS_OK) return st;
  const A* a = static_cast<const A*>(s->amp);
  double* S1 = static_cast<double*>(s->scratch);
  double* S2 = S1 + nch;
  double* P2 = S2 + nsc;
  double* d_u = P2 + nsc + 1;
  u64* d_out = reinterpret_cast<u64*>(d_u + batch);
  k_sample_sums<A><<<grid_for(nsc, kMT / 32, 8), kMT, 0, s->stream>>>(a, N, nch, nsc, S1, S2);
  if ((st = launch_ok("k_sample_sums")) != QS_OK) return st;
  k_sample_prefix<<<1, kPrefixThreads, 0, s->stream>>>(S2, nsc, P2);
  if ((st = launch_ok("k_sample_prefix")) != QS_OK) return st;
  double T = 0.0;
  if ((st = sync_copy(s, &T, P2 + nsc, sizeof(double), cudaMemcpyDeviceToHost)) != QS_OK) return st;
  if (!(T > 0.0) || !std::isfinite(T)) return fail(QS_EINVAL, "qs_sample: the state has zero norm");
  for (u64 b = 0; b < nshots; b += batch) {
    const u64 m = std::min(batch, nshots - b);
    cudaError_t e = cudaMemcpyAsync(d_u, u + b, sizeof(double) * m, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qs_sample: upload");
    k_sample_shots<A><<<grid_for(m, kMT / 32, 16), kMT, 0, s->stream>>>(a, N, nch, nsc, S1, S2, P2, d_u, m, d_out);
    if ((st = launch_ok("k_sample_shots")) != QS_OK) return st;
    if ((st = sync_copy(s, out + b, d_out, sizeof(u64) * m, cudaMemcpyDeviceToHost)) != QS_OK) return st;
  }
  return QS_OK;
}

qs_status check_qubits(const qs_state* s, const int* qubits, int k, const char* fn) {
  for (int i = 0; i < k; ++i) {
    if (qubits[i] < 0 || qubits[i] >= s->n) return fail(QS_EINVAL, "%s: qubit %d out of range", fn, qubits[i]);
    for (int j = 0; j < i; ++j)
      if (qubits[j] == qubits[i]) return fail(QS_EINVAL, "%s: qubit %d repeated", fn, qubits[i]);
  }
  return QS_OK;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" {

qs_status qs_probabilities(qs_state* s, const int* qubits, int k, double* out) {
  if (!s || !qubits || !out) return fail(QS_EINVAL, "qs_probabilities: NULL argument");
  if (k < 1 || k > 6 || k > s->n) return fail(QS_EINVAL, "qs_probabilities: need 1 <= k <= min(6, n), got %d", k);
  qs_status st = check_qubits(s, qubits, k, "qs_probabilities");
  if (st != QS_OK) return st;
  return s->dtype == QS_C64 ? marginal<float2>(s, qubits, k, out) : marginal<double2>(s, qubits, k, out);
}

qs_status qs_measure(qs_state* s, int q, double u, int* outcome, double* prob) {
  if (!s || !outcome) return fail(QS_EINVAL, "qs_measure: NULL argument");
  if (!(u >= 0.0 && u < 1.0)) return fail(QS_EINVAL, "qs_measure: u must lie in [0, 1)");
  qs_status st = check_qubits(s, &q, 1, "qs_measure");
  if (st != QS_OK) return st;
  double p[2];
  if ((st = qs_probabilities(s, &q, 1, p)) != QS_OK) return st;
  const double tot = p[0] + p[1];
  if (!(tot > 0.0) || !std::isfinite(tot)) return fail(QS_EINVAL, "qs_measure: the state has zero norm");
  int o = u * tot < p[0] ? 0 : 1;
  if (!(p[o] > 0.0)) o ^= 1;
  st = s->dtype == QS_C64 ? collapse<float2, float>(s, q, o, p[o]) : collapse<double2, double>(s, q, o, p[o]);
  if (st != QS_OK) return st;
  *outcome = o;
  if (prob) *prob = p[o] / tot;
  return QS_OK;
}

qs_status qs_sample(qs_state* s, uint64_t nshots, const double* u, uint64_t* out) {
  if (!s || (nshots && (!u || !out))) return fail(QS_EINVAL, "qs_sample: NULL argument");
  for (uint64_t i = 0; i < nshots; ++i)
    if (!(u[i] >= 0.0 && u[i] < 1.0)) return fail(QS_EINVAL, "qs_sample: u[%llu] outside [0, 1)", (unsigned long long)i);
  if (!nshots) return QS_OK;
  return s->dtype == QS_C64 ? sample<float2>(s, nshots, u, out) : sample<double2>(s, nshots, u, out);
}

}  // extern "C"
