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
#include <algorithm>

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
