// Computational-basis measurement (§II-A: a circuit is a sequence of gates,
// measurements and resets): marginal probabilities, the collapse after a
// single-qubit measurement, and sampling of basis states.
//
// Probabilities follow the Born rule, p_x = |a_x|^2.  For the marginals the
// squares are formed exactly in double-float (FP32 pairs with their
// rounding errors) and summed per thread in double-float with an FP64 flush
// every few groups: FP64-level accuracy without the FP64 pipe (about 1/64 of
// the FP32 rate on GB300).  Sampling follows a step-by-step definition whose
// floating-point operations are taken in a fixed order, so the index it
// returns for a given uniform does not depend on the launch shape:
//   p_x = re * re + im * im, each product and the sum rounded on its own;
//   C = min(N, 1024) amplitudes per chunk; chunk sum S_c = 32 lane partials
//   (lane l sums p_{cC + l + 32 i}, i ascending) combined by the butterfly
//   s_l <- s_l + s_{l xor off} for off = 16, 8, 4, 2, 1;
//   P_0 = 0, P_{c+1} = P_c + S_c in order, T = P_{N/C};
//   a uniform u gives t = u T, c = the largest chunk with P_c <= t, and the
//   sample is the first x >= cC at which the running sum r = P_c + p_{cC} +
//   ... + p_x exceeds t (the largest x with p_x > 0 if none does).
#include <algorithm>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "kcommon.cuh"

namespace qs {
namespace {

constexpr int kMT = 256;        // threads per CTA
constexpr u64 kChunk = 1024;    // amplitudes per chunk of the sampling definition
constexpr int kBins = 8;        // outcomes per marginal pass
constexpr u64 kShotBatch = u64(1) << 20;

__device__ __forceinline__ double prob(float2 v) {
  return __dadd_rn(__dmul_rn((double)v.x, (double)v.x), __dmul_rn((double)v.y, (double)v.y));
}
__device__ __forceinline__ double prob(double2 v) { return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)); }

struct MargArgs {
  Ins ins;          // zero insertion at the measured qubits
  u64 spread[64];   // spread[r]: OR of 2^qubits[i] over the set bits i of r
};

// Outcomes [b0, b0 + NB): each thread sums its groups (the other qubits) in
// grid-stride order, the squares exact in double-float, flushed into FP64
// every 4 groups; the CTA reduces every bin into part[blockIdx.x * kBins + j].
template <typename A, int NB>
__global__ void __launch_bounds__(kMT) k_marginal(const A* __restrict__ a, u64 ngroups,
                                                  const __grid_constant__ MargArgs args, int b0,
                                                  double* __restrict__ part) {
  double acc[NB];
  dfl da[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    acc[j] = 0.0;
    da[j] = dfl{0.f, 0.f};
  }
  const u64 stride = (u64)gridDim.x * kMT;
  int since = 0;
  for (u64 g = (u64)blockIdx.x * kMT + threadIdx.x; g < ngroups; g += stride) {
    const u64 base = expand(g, args.ins);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const A v = a[base | args.spread[b0 + j]];
      const dfl x = to_df(v.x), y = to_df(v.y);
      df_acc(da[j], df_mul(x, x));
      df_acc(da[j], df_mul(y, y));
    }
    if (++since == 4) {
#pragma unroll
      for (int j = 0; j < NB; ++j) df_flush(acc[j], da[j]);
      since = 0;
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

// Chunk sums of the sampling definition: one warp per chunk of C amplitudes.
template <typename A>
__global__ void __launch_bounds__(kMT) k_chunk_sums(const A* __restrict__ a, u64 C, u64 nch, double* __restrict__ S) {
  const int lane = threadIdx.x & 31;
  const u64 wstride = (u64)gridDim.x * (kMT / 32);
  for (u64 c = (u64)blockIdx.x * (kMT / 32) + (threadIdx.x >> 5); c < nch; c += wstride) {
    double s = 0.0;
    for (u64 j = (u64)lane; j < C; j += 32) s = __dadd_rn(s, prob(a[c * C + j]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, off));
    if (lane == 0) S[c] = s;
  }
}

// One thread per shot: the running sum from chunk c[i] until it exceeds
// t[i]; ~0 when the end of the state is reached first.
template <typename A>
__global__ void __launch_bounds__(kMT) k_sample_scan(const A* __restrict__ a, u64 N, u64 C, u64 nshots,
                                                     const u64* __restrict__ chunk, const double* __restrict__ p0,
                                                     const double* __restrict__ tt, u64* __restrict__ out) {
  const u64 i = (u64)blockIdx.x * kMT + threadIdx.x;
  if (i >= nshots) return;
  double r = p0[i];
  const double t = tt[i];
  u64 x = chunk[i] * C;
  for (; x < N; ++x) {
    r = __dadd_rn(r, prob(a[x]));
    if (r > t) break;
  }
  out[i] = x < N ? x : ~u64(0);
}

// The largest x with p_x > 0 (the sampling fallback); *out must start at 0.
template <typename A>
__global__ void __launch_bounds__(kMT) k_last_nonzero(const A* __restrict__ a, u64 N, unsigned long long* out) {
  const u64 stride = (u64)gridDim.x * kMT;
  unsigned long long best = 0;
  for (u64 x = (u64)blockIdx.x * kMT + threadIdx.x; x < N; x += stride)
    if (prob(a[x]) > 0.0) best = x;
  if (best) atomicMax(out, best);
}

Ins ins_for(const int* qubits, int k) {
  Ins ins{};
  ins.k = k;
  ins.set = 0;
  int s[6];
  for (int i = 0; i < k; ++i) s[i] = qubits[i];
  std::sort(s, s + k);
  for (int i = 0; i < k; ++i) ins.pos[i] = s[i];
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
  const unsigned g = grid_for(ngroups, kMT, 4);
  qs_status st = ensure_scratch(s, sizeof(double) * kBins * g);
  if (st != QS_OK) return st;
  double* part = static_cast<double*>(s->scratch);
  std::vector<double> h((size_t)kBins * g);
  for (int b0 = 0; b0 < (1 << k); b0 += kBins) {
    const int nb = std::min(kBins, (1 << k) - b0);  // 2, 4 or 8
    const A* amp = static_cast<const A*>(s->amp);
    if (nb == 2) k_marginal<A, 2><<<g, kMT, 0, s->stream>>>(amp, ngroups, args, b0, part);
    else if (nb == 4) k_marginal<A, 4><<<g, kMT, 0, s->stream>>>(amp, ngroups, args, b0, part);
    else k_marginal<A, 8><<<g, kMT, 0, s->stream>>>(amp, ngroups, args, b0, part);
    if ((st = launch_ok("k_marginal")) != QS_OK) return st;
    if ((st = sync_copy(s, h.data(), part, sizeof(double) * kBins * g, cudaMemcpyDeviceToHost)) != QS_OK) return st;
    for (int j = 0; j < nb; ++j) {
      double sum = 0.0;
      for (unsigned c = 0; c < g; ++c) sum += h[(size_t)c * kBins + j];
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
  const u64 N = u64(1) << s->n, C = std::min(N, kChunk), nch = N / C;
  const u64 batch = std::min(nshots, kShotBatch);
  // scratch: chunk sums, then per shot chunk, P_c, t, result
  const size_t need = sizeof(double) * nch + batch * (2 * sizeof(u64) + 2 * sizeof(double)) + sizeof(u64);
  qs_status st = ensure_scratch(s, need);
  if (st != QS_OK) return st;
  const A* a = static_cast<const A*>(s->amp);
  double* S = static_cast<double*>(s->scratch);
  u64* d_chunk = reinterpret_cast<u64*>(S + nch);
  double* d_p0 = reinterpret_cast<double*>(d_chunk + batch);
  double* d_t = d_p0 + batch;
  u64* d_out = reinterpret_cast<u64*>(d_t + batch);
  u64* d_last = d_out + batch;
  k_chunk_sums<A><<<grid_for(nch, kMT / 32, 8), kMT, 0, s->stream>>>(a, C, nch, S);
  if ((st = launch_ok("k_chunk_sums")) != QS_OK) return st;
  std::vector<double> P(nch + 1, 0.0), hS(nch);
  if ((st = sync_copy(s, hS.data(), S, sizeof(double) * nch, cudaMemcpyDeviceToHost)) != QS_OK) return st;
  for (u64 c = 0; c < nch; ++c) P[c + 1] = P[c] + hS[c];
  const double T = P[nch];
  if (!(T > 0.0) || !std::isfinite(T)) return fail(QS_EINVAL, "qs_sample: the state has zero norm");
  u64 last = 0;
  bool have_last = false;
  std::vector<u64> hc(batch);
  std::vector<double> hp(batch), ht(batch);
  for (u64 b = 0; b < nshots; b += batch) {
    const u64 m = std::min(batch, nshots - b);
    for (u64 i = 0; i < m; ++i) {
      const double t = u[b + i] * T;
      const u64 c = (u64)(std::upper_bound(P.begin(), P.begin() + nch, t) - P.begin()) - 1;
      hc[i] = c;
      hp[i] = P[c];
      ht[i] = t;
    }
    cudaError_t e = cudaMemcpyAsync(d_chunk, hc.data(), sizeof(u64) * m, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_p0, hp.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_t, ht.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qs_sample: upload");
    k_sample_scan<A><<<(unsigned)((m + kMT - 1) / kMT), kMT, 0, s->stream>>>(a, N, C, m, d_chunk, d_p0, d_t, d_out);
    if ((st = launch_ok("k_sample_scan")) != QS_OK) return st;
    if ((st = sync_copy(s, out + b, d_out, sizeof(u64) * m, cudaMemcpyDeviceToHost)) != QS_OK) return st;
    for (u64 i = 0; i < m; ++i) {
      if (out[b + i] != ~u64(0)) continue;
      if (!have_last) {
        e = cudaMemsetAsync(d_last, 0, sizeof(u64), s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "qs_sample: memset");
        k_last_nonzero<A><<<grid_for(N, kMT, 4), kMT, 0, s->stream>>>(a, N,
                                                                        reinterpret_cast<unsigned long long*>(d_last));
        if ((st = launch_ok("k_last_nonzero")) != QS_OK) return st;
        if ((st = sync_copy(s, &last, d_last, sizeof(u64), cudaMemcpyDeviceToHost)) != QS_OK) return st;
        have_last = true;
      }
      out[b + i] = last;
    }
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
