// Reductions over the state vector: norm, inner product, Pauli expectation.
//
// Each thread accumulates in FP64 over a grid-stride range of 16-byte
// packets; warps combine with shuffles, CTAs through shared memory, and the
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
#include <algorithm>

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

template <typename R>
__global__ void __launch_bounds__(kThreads) k_norm2(const R* __restrict__ a, u64 npk, double2* part) {
  constexpr int V = PK<R>::V;
  double s = 0.0, dummy = 0.0;
  for (u64 p = (u64)blockIdx.x * kThreads + threadIdx.x; p < npk; p += (u64)gridDim.x * kThreads) {
    R v[V];
    ld16(a + p * V, v);
#pragma unroll
    for (int c = 0; c < V; ++c) s += (double)v[c] * (double)v[c];
  }
  block_sum2(s, dummy);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(s, 0.0);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_inner(const R* __restrict__ a, const R* __restrict__ b, u64 npk,
                                                    double2* part) {
  constexpr int V = PK<R>::V;
  double sr = 0.0, si = 0.0;
  for (u64 p = (u64)blockIdx.x * kThreads + threadIdx.x; p < npk; p += (u64)gridDim.x * kThreads) {
    R va[V], vb[V];
    ld16(a + p * V, va);
    ld16(b + p * V, vb);
#pragma unroll
    for (int c = 0; c < V; c += 2) {
      const double ar = va[c], ai = va[c + 1], br = vb[c], bi = vb[c + 1];
      sr += ar * br + ai * bi;   // conj(a) b
      si += ar * bi - ai * br;
    }
  }
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

template <typename R>
__global__ void __launch_bounds__(kThreads) k_pauli(const R* __restrict__ a, int n, const __grid_constant__ PauliGroup g,
                                                    double2* part) {
  double sr = 0.0, si = 0.0;
  const u64 N = u64(1) << n;
  if (g.m == 0) {
    for (u64 x = (u64)blockIdx.x * kThreads + threadIdx.x; x < N; x += (u64)gridDim.x * kThreads) {
      const double ar = a[2 * x], ai = a[2 * x + 1];
      double fr, fi;
      fval(g, x, fr, fi);
      const double p = ar * ar + ai * ai;
      sr += p * fr;
      si += p * fi;
    }
  } else {
    const u64 half = N >> 1;
    const u64 lo_mask = (u64(1) << g.h) - 1;
    for (u64 i = (u64)blockIdx.x * kThreads + threadIdx.x; i < half; i += (u64)gridDim.x * kThreads) {
      const u64 x = ((i & ~lo_mask) << 1) | (i & lo_mask);  // bit h clear
      const u64 y = x ^ g.m;
      const double xr = a[2 * x], xi = a[2 * x + 1], yr = a[2 * y], yi = a[2 * y + 1];
      double fr, fi;
      // term x: conj(a_y) a_x f(x)
      fval(g, x, fr, fi);
      double pr = yr * xr + yi * xi, pi = yr * xi - yi * xr;
      sr += pr * fr - pi * fi;
      si += pr * fi + pi * fr;
      // term y: conj(a_x) a_y f(y)
      fval(g, y, fr, fi);
      pr = xr * yr + xi * yi;
      pi = xr * yi - xi * yr;
      sr += pr * fr - pi * fi;
      si += pr * fi + pi * fr;
    }
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
  const unsigned gsz = red_grid(N / 2);
  const size_t ng = groups.size();
  qs_status st = ensure_scratch(s, sizeof(double2) * (gsz * ng + 1));
  if (st != QS_OK) return st;
  double2* part = static_cast<double2*>(s->scratch);
  double2* res = part + gsz * ng;
  for (size_t i = 0; i < ng; ++i) {
    if (s->dtype == QS_C64)
      k_pauli<float><<<gsz, kThreads, 0, s->stream>>>(static_cast<const float*>(s->amp), s->n, groups[i], part + gsz * i);
    else
      k_pauli<double><<<gsz, kThreads, 0, s->stream>>>(static_cast<const double*>(s->amp), s->n, groups[i], part + gsz * i);
    if ((st = launch_ok("k_pauli")) != QS_OK) return st;
  }
  k_final<<<1, kThreads, 0, s->stream>>>(part, (int)(gsz * ng), res, 0);
  if ((st = launch_ok("k_final")) != QS_OK) return st;
  double2 h;
  if ((st = read_result(s, res, &h)) != QS_OK) return st;
  *out = h.x;
  return QS_OK;
}

}  // namespace qs
