// Per-gate kernels: one HBM pass per gate.
//
//  * pair update (Eq. 4 of §II-A): one-qubit and controlled gates.  A thread
//    takes a compact pair counter i, inserts the target bit (0) and any
//    control bits (1) to get the lower packet index p0, and updates the
//    packets p0 and p0 + 2^t' together.  Consecutive threads touch
//    consecutive packets on both sides of the pair, so every warp access is
//    a coalesced 512-byte transaction whatever the target qubit.
//  * in-packet update: complex64 gates whose target is qubit 0 (both halves
//    of each pair sit in one 16-byte packet).
//  * diagonal: general k-qubit diagonal (every amplitude), and the sparse
//    "phase on all-ones" form (CZ, CP, Z, S, T, P) that touches only the
//    2^(n-k) amplitudes whose k bits are all 1.
//  * dense k-qubit block (k <= 6): a CTA stages 32 groups of 2^k amplitudes
//    in shared memory and multiplies them by the 2^k x 2^k matrix.
//  * bit-field exchange (swap / fused swap of §III-D, Listing 1): an
//    in-place, shared-memory-tiled involution over pairs of 512-byte runs.
//
// Arithmetic: complex64 in FP32.  complex128 pair, diagonal and phase
// updates run in double-float (dfloat.cuh): GB300's FP64 pipe is ~1/64 of
// FP32, so native FP64 would cap these passes near a third of HBM bandwidth.
// X-type gates (X, CNOT, Toffoli-like) are pure exchanges with no arithmetic.
#include <algorithm>
#include <cstring>

#include "arith.cuh"

namespace qs {
namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 2;  // pair kernels: 2 x kUnroll 16-byte loads in flight per thread
constexpr int kU1 = 4;      // one-vector kernels (diagonals, phases): kU1 loads in flight
constexpr int kWaves = 8;

// ---------------------------------------------------------------------------
// Pair update over packets: p0 = expand(i), p1 = p0 + 2^tp.
// jmask selects which amplitudes of a packet take part (complex64 packets
// hold two; a control on qubit 0 restricts the update to the odd one).
// XG: the matrix is X -- exchange, no arithmetic.
// ---------------------------------------------------------------------------
template <typename R, bool XG>
__global__ void __launch_bounds__(kThreads) k_pairs(R* __restrict__ a, u64 nwork, Ins ins, int tp,
                                                    int jmask, typename Ar<R>::Mat U) {
  constexpr int V = PK<R>::V, A = PK<R>::A;
  const u64 step = (u64)gridDim.x * kThreads * kUnroll;
  const u64 dp = u64(1) << tp;
  for (u64 base = (u64)blockIdx.x * kThreads * kUnroll + threadIdx.x; base < nwork; base += step) {
    R x0[kUnroll][V], x1[kUnroll][V];
    u64 p0[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const u64 i = base + (u64)u * kThreads;
      p0[u] = expand(i < nwork ? i : 0, ins);
      ld16(a + p0[u] * V, x0[u]);
      ld16(a + (p0[u] + dp) * V, x1[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < A; ++j) {
        if (!((jmask >> j) & 1)) continue;
        if (XG) {
          const R tr = x0[u][2 * j], ti = x0[u][2 * j + 1];
          x0[u][2 * j] = x1[u][2 * j];
          x0[u][2 * j + 1] = x1[u][2 * j + 1];
          x1[u][2 * j] = tr;
          x1[u][2 * j + 1] = ti;
        } else {
          pair_apply(U, x0[u][2 * j], x0[u][2 * j + 1], x1[u][2 * j], x1[u][2 * j + 1]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (base + (u64)u * kThreads < nwork) {
        st16(a + p0[u] * V, x0[u]);
        st16(a + (p0[u] + dp) * V, x1[u]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// complex64, target qubit 0: the pair (a_2p, a_2p+1) is one packet.
// ---------------------------------------------------------------------------
template <bool XG>
__global__ void __launch_bounds__(kThreads) k_inpkt(float* __restrict__ a, u64 nwork, Ins ins, M2<float> U) {
  const u64 step = (u64)gridDim.x * kThreads * kUnroll;
  for (u64 base = (u64)blockIdx.x * kThreads * kUnroll + threadIdx.x; base < nwork; base += step) {
    float v[kUnroll][4];
    u64 p[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const u64 i = base + (u64)u * kThreads;
      p[u] = expand(i < nwork ? i : 0, ins);
      ld16(a + p[u] * 4, v[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (XG) {
        const float r = v[u][0], i = v[u][1];
        v[u][0] = v[u][2];
        v[u][1] = v[u][3];
        v[u][2] = r;
        v[u][3] = i;
      } else {
        mv2(U, v[u][0], v[u][1], v[u][2], v[u][3]);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
      if (base + (u64)u * kThreads < nwork) st16(a + p[u] * 4, v[u]);
  }
}

// ---------------------------------------------------------------------------
// Diagonal over every amplitude: a_x *= d[r(x)].
// ---------------------------------------------------------------------------
constexpr int kMaxDiagK = 8;
template <typename R>
struct DiagTab {
  int k;
  int q[kMaxDiagK];
  typename Ar<R>::Z d[1 << kMaxDiagK];
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_diag(R* __restrict__ a, u64 npk, const __grid_constant__ DiagTab<R> T) {
  typedef typename Ar<R>::Z Z;
  constexpr int V = PK<R>::V, A = PK<R>::A, LA = PK<R>::LA;
  __shared__ Z sd[1 << kMaxDiagK];
  const int D = 1 << T.k;
  for (int i = threadIdx.x; i < D; i += kThreads) sd[i] = T.d[i];
  __syncthreads();
  const u64 step = (u64)gridDim.x * kThreads * kU1;
  for (u64 base = (u64)blockIdx.x * kThreads * kU1 + threadIdx.x; base < npk; base += step) {
    R v[kU1][V];
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
      const u64 p = base + (u64)u * kThreads;
      if (p < npk) ld16(a + p * V, v[u]);
    }
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
      const u64 p = base + (u64)u * kThreads;
#pragma unroll
      for (int j = 0; j < A; ++j) {
        const u64 x = (p << LA) | (u64)j;
        int r = 0;
        for (int i = 0; i < T.k; ++i) r |= (int)((x >> T.q[i]) & 1u) << i;
        scal_apply(sd[r], v[u][2 * j], v[u][2 * j + 1]);
      }
    }
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
      const u64 p = base + (u64)u * kThreads;
      if (p < npk) st16(a + p * V, v[u]);
    }
  }
}

// ---------------------------------------------------------------------------
// Phase on all-ones: a_x *= z for the x whose selected bits are all 1.
// Packets enumerated by bit insertion; jmask as in k_pairs.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads) k_phase(R* __restrict__ a, u64 nwork, Ins ins, int jmask,
                                                    typename Ar<R>::Z z) {
  constexpr int V = PK<R>::V, A = PK<R>::A;
  const u64 step = (u64)gridDim.x * kThreads * kU1;
  for (u64 base = (u64)blockIdx.x * kThreads * kU1 + threadIdx.x; base < nwork; base += step) {
    R v[kU1][V];
    u64 p[kU1];
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
      const u64 i = base + (u64)u * kThreads;
      p[u] = expand(i < nwork ? i : 0, ins);
      ld16(a + p[u] * V, v[u]);
    }
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
#pragma unroll
      for (int j = 0; j < A; ++j)
        if ((jmask >> j) & 1) scal_apply(z, v[u][2 * j], v[u][2 * j + 1]);
    }
#pragma unroll
    for (int u = 0; u < kU1; ++u)
      if (base + (u64)u * kThreads < nwork) st16(a + p[u] * V, v[u]);
  }
}

// ---------------------------------------------------------------------------
// Dense k-qubit block.  A CTA owns kGroups consecutive groups (compact group
// counter g, amplitudes a[expand(g) | spread(r)], r < 2^k), stages them in
// shared memory, and writes M * v back.  M (2^k x 2^k, real type R) sits in
// shared memory too.
// ---------------------------------------------------------------------------
constexpr int kGroups = 32;
struct DenseArgs {
  Ins ins;        // zero-insertion at the k qubits (amplitude space)
  int k;
  u64 spread[64]; // spread[r] = OR of 2^qubits[i] for bits i of r
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_dense(R* __restrict__ a, u64 ngroups, const R* __restrict__ Mg,
                                                    const __grid_constant__ DenseArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sM = reinterpret_cast<R*>(smem_raw);
  const int D = 1 << args.k;
  R* sv = sM + 2 * D * D;  // [D][kGroups] complex
  for (int i = threadIdx.x; i < 2 * D * D; i += kThreads) sM[i] = Mg[i];
  for (u64 g0 = (u64)blockIdx.x * kGroups; g0 < ngroups; g0 += (u64)gridDim.x * kGroups) {
    __syncthreads();
    for (int e = threadIdx.x; e < D * kGroups; e += kThreads) {
      const int r = e / kGroups, b = e % kGroups;
      const u64 g = g0 + b;
      if (g < ngroups) {
        const u64 x = expand(g, args.ins) | args.spread[r];
        sv[2 * e] = a[2 * x];
        sv[2 * e + 1] = a[2 * x + 1];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < D * kGroups; e += kThreads) {
      const int r = e / kGroups, b = e % kGroups;
      const u64 g = g0 + b;
      R sr = 0, si = 0;
      for (int c = 0; c < D; ++c) {
        const R mr = sM[2 * (r * D + c)], mi = sM[2 * (r * D + c) + 1];
        const R vr = sv[2 * (c * kGroups + b)], vi = sv[2 * (c * kGroups + b) + 1];
        sr += mr * vr - mi * vi;
        si += mr * vi + mi * vr;
      }
      if (g < ngroups) {
        const u64 x = expand(g, args.ins) | args.spread[r];
        a[2 * x] = sr;
        a[2 * x + 1] = si;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Bit-field exchange (involution sigma swapping bit pairs (pa[i], pb[i])).
// A tile is a set of 2^nb runs of 2^R contiguous amplitudes: the low R bits
// plus the bits in B (high partners of low swapped bits).  A CTA loads tile F
// and, when sigma(F) != F, tile sigma(F); then writes new[X] = old[sigma(X)].
// Tiles with sigma(F) < F are left to their partner's CTA.
// ---------------------------------------------------------------------------
struct SwapArgs {
  int npairs;
  int pa[17], pb[17];  // amplitude-space bit pairs, pa < pb
  int R;               // log2 of run length in amplitudes
  int nb;              // |B|
  int B[8];            // ascending
  Ins tins;            // zero-insertion at B (applied to t << R)
  bool skip_fixed;     // no low pairs: tiles with sigma(F) == F are untouched
};

__device__ __forceinline__ u64 sigma(u64 x, const SwapArgs& s) {
  for (int i = 0; i < s.npairs; ++i) {
    const u64 ba = (x >> s.pa[i]) & 1u, bb = (x >> s.pb[i]) & 1u;
    x ^= ((ba ^ bb) << s.pa[i]) | ((ba ^ bb) << s.pb[i]);
  }
  return x;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_bitswap(R* __restrict__ a, u64 ntiles, const __grid_constant__ SwapArgs s) {
  constexpr int V = PK<R>::V, A = PK<R>::A;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int run = 1 << s.R;                 // amplitudes per run
  const int tile = run << s.nb;             // amplitudes per tile
  R* t0 = reinterpret_cast<R*>(smem_raw);   // tile F
  R* t1 = t0 + 2 * tile;                    // tile sigma(F)
  const int pk_per_tile = tile / A;
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const u64 F = expand(t << s.R, s.tins);
    const u64 G = sigma(F, s);
    if (G < F) continue;
    if (G == F && s.skip_fixed) continue;
    const bool two = (G != F);
    __syncthreads();
    // load (packet-wise; a packet never straddles a run since run >= A)
    for (int e = threadIdx.x; e < pk_per_tile; e += kThreads) {
      const int la = e * A;                       // local amplitude index
      const int j = la >> s.R, l = la & (run - 1);
      u64 off = 0;
      for (int i = 0; i < s.nb; ++i) off |= (u64)((j >> i) & 1) << s.B[i];
      R v[V];
      ld16(a + 2 * (F | off | (u64)l), v);
#pragma unroll
      for (int c = 0; c < V; ++c) t0[2 * la + c] = v[c];
      if (two) {
        ld16(a + 2 * (G | off | (u64)l), v);
#pragma unroll
        for (int c = 0; c < V; ++c) t1[2 * la + c] = v[c];
      }
    }
    __syncthreads();
    for (int side = 0; side < (two ? 2 : 1); ++side) {
      const u64 base = side ? G : F;
      const R* src = two ? (side ? t0 : t1) : t0;
      for (int e = threadIdx.x; e < pk_per_tile; e += kThreads) {
        const int la = e * A;
        const int j = la >> s.R, l = la & (run - 1);
        u64 off = 0;
        for (int i = 0; i < s.nb; ++i) off |= (u64)((j >> i) & 1) << s.B[i];
        R v[V];
#pragma unroll
        for (int h = 0; h < A; ++h) {
          const u64 X = base | off | (u64)(l + h);
          const u64 Y = sigma(X, s);
          // local index of Y within its tile
          int jy = 0;
          for (int i = 0; i < s.nb; ++i) jy |= (int)((Y >> s.B[i]) & 1u) << i;
          const int ly = (jy << s.R) | (int)(Y & (u64)(run - 1));
          v[2 * h] = src[2 * ly];
          v[2 * h + 1] = src[2 * ly + 1];
        }
        st16(a + 2 * (base | off | (u64)l), v);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// complex128 in double-float storage: each FP64 value of the vector is held
// as its (hi, lo) float pair in the same 8 bytes, so an amplitude is one
// float4 (re_h, re_l, im_h, im_l).  Plans convert a complex128 state to this
// layout once at the start and back at the end (k_to_dfl / k_from_dfl), so
// the per-gate kernels below do no conversion work.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_to_dfl(double* a, u64 npk) {
  for (u64 p = (u64)blockIdx.x * kThreads + threadIdx.x; p < npk; p += (u64)gridDim.x * kThreads) {
    const double2 v = reinterpret_cast<const double2*>(a)[p];
    const dfl r = d2df(v.x), i = d2df(v.y);
    reinterpret_cast<float4*>(a)[p] = make_float4(r.h, r.l, i.h, i.l);
  }
}
__global__ void __launch_bounds__(kThreads) k_from_dfl(double* a, u64 npk) {
  for (u64 p = (u64)blockIdx.x * kThreads + threadIdx.x; p < npk; p += (u64)gridDim.x * kThreads) {
    const float4 v = reinterpret_cast<const float4*>(a)[p];
    reinterpret_cast<double2*>(a)[p] = make_double2(df2d(dfl{v.x, v.y}), df2d(dfl{v.z, v.w}));
  }
}

__global__ void __launch_bounds__(kThreads) k_pairs_dfl(float4* __restrict__ a, u64 nwork, Ins ins, int tp, M2df U) {
  const u64 step = (u64)gridDim.x * kThreads * kUnroll;
  const u64 dp = u64(1) << tp;
  for (u64 base = (u64)blockIdx.x * kThreads * kUnroll + threadIdx.x; base < nwork; base += step) {
    float4 x0[kUnroll], x1[kUnroll];
    u64 p0[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const u64 i = base + (u64)u * kThreads;
      p0[u] = expand(i < nwork ? i : 0, ins);
      x0[u] = a[p0[u]];
      x1[u] = a[p0[u] + dp];
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      cdf A{x0[u].x, x0[u].y, x0[u].z, x0[u].w}, B{x1[u].x, x1[u].y, x1[u].z, x1[u].w};
      mv2df(U, A, B);
      x0[u] = make_float4(A.rh, A.rl, A.ih, A.il);
      x1[u] = make_float4(B.rh, B.rl, B.ih, B.il);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (base + (u64)u * kThreads < nwork) {
        a[p0[u]] = x0[u];
        a[p0[u] + dp] = x1[u];
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_phase_dfl(float4* __restrict__ a, u64 nwork, Ins ins, Zdf z) {
  const float zh[2] = {z.rh, z.ih}, zl[2] = {z.rl, z.il};
  const u64 step = (u64)gridDim.x * kThreads * kU1;
  for (u64 base = (u64)blockIdx.x * kThreads * kU1 + threadIdx.x; base < nwork; base += step) {
    float4 v[kU1];
    u64 p[kU1];
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
      const u64 i = base + (u64)u * kThreads;
      p[u] = expand(i < nwork ? i : 0, ins);
      v[u] = a[p[u]];
    }
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
      cdf x{v[u].x, v[u].y, v[u].z, v[u].w};
      cmul_df(zh, zl, x);
      v[u] = make_float4(x.rh, x.rl, x.ih, x.il);
    }
#pragma unroll
    for (int u = 0; u < kU1; ++u)
      if (base + (u64)u * kThreads < nwork) a[p[u]] = v[u];
  }
}

__global__ void __launch_bounds__(kThreads) k_diag_dfl(float4* __restrict__ a, u64 npk,
                                                       const __grid_constant__ DiagTab<double> T) {
  __shared__ Zdf sd[1 << kMaxDiagK];
  const int D = 1 << T.k;
  for (int i = threadIdx.x; i < D; i += kThreads) sd[i] = T.d[i];
  __syncthreads();
  const u64 step = (u64)gridDim.x * kThreads * kU1;
  for (u64 base = (u64)blockIdx.x * kThreads * kU1 + threadIdx.x; base < npk; base += step) {
    float4 v[kU1];
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
      const u64 p = base + (u64)u * kThreads;
      if (p < npk) v[u] = a[p];
    }
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
      const u64 p = base + (u64)u * kThreads;
      int r = 0;
      for (int i = 0; i < T.k; ++i) r |= (int)((p >> T.q[i]) & 1u) << i;
      cdf x{v[u].x, v[u].y, v[u].z, v[u].w};
      const Zdf z = sd[r];
      const float zh[2] = {z.rh, z.ih}, zl[2] = {z.rl, z.il};
      cmul_df(zh, zl, x);
      v[u] = make_float4(x.rh, x.rl, x.ih, x.il);
    }
#pragma unroll
    for (int u = 0; u < kU1; ++u) {
      const u64 p = base + (u64)u * kThreads;
      if (p < npk) a[p] = v[u];
    }
  }
}

bool is_x(const double U[8]) {
  return U[0] == 0 && U[1] == 0 && U[2] == 1 && U[3] == 0 && U[4] == 1 && U[5] == 0 && U[6] == 0 && U[7] == 0;
}

Ins make_ins(std::vector<std::pair<int, int>> bits) {  // (position, value)
  std::sort(bits.begin(), bits.end());
  Ins ins{};
  ins.k = (int)bits.size();
  ins.set = 0;
  for (int i = 0; i < ins.k; ++i) {
    ins.pos[i] = bits[i].first;
    if (bits[i].second) ins.set |= u64(1) << bits[i].first;
  }
  return ins;
}

template <typename R>
qs_status pairs_or_inpkt(qs_state* s, const int* ctrl, int nc, int t, const double U[8]) {
  const int LA = PK<R>::LA;
  const int nb = s->n - LA;  // packet-space bits
  R* a = static_cast<R*>(s->amp);
  if (LA == 1 && t == 0) {
    // complex64, target qubit 0: pair inside the packet; controls >= 1.
    std::vector<std::pair<int, int>> bits;
    for (int i = 0; i < nc; ++i) bits.push_back({ctrl[i] - 1, 1});
    const u64 nwork = u64(1) << (nb - nc);
    const unsigned g = grid_for(nwork, (u64)kThreads * kUnroll, kWaves);
    const M2<float> m = to_mat(U, 0.0f);
    if (is_x(U)) k_inpkt<true><<<g, kThreads, 0, s->stream>>>(reinterpret_cast<float*>(a), nwork, make_ins(bits), m);
    else k_inpkt<false><<<g, kThreads, 0, s->stream>>>(reinterpret_cast<float*>(a), nwork, make_ins(bits), m);
    return launch_ok("k_inpkt");
  }
  std::vector<std::pair<int, int>> bits;
  int jmask = (1 << PK<R>::A) - 1;
  int n_in = 0;
  for (int i = 0; i < nc; ++i) {
    if (ctrl[i] < LA) {  // complex64 control on qubit 0: odd amplitude only
      jmask &= 2;
      ++n_in;
    } else {
      bits.push_back({ctrl[i] - LA, 1});
    }
  }
  bits.push_back({t - LA, 0});
  const int nins = (int)bits.size();
  const u64 nwork = u64(1) << (nb - nins);
  const unsigned g = grid_for(nwork, (u64)kThreads * kUnroll, kWaves);
  (void)n_in;
  const typename Ar<R>::Mat m = to_mat(U, R(0));
  if (is_x(U)) k_pairs<R, true><<<g, kThreads, 0, s->stream>>>(a, nwork, make_ins(bits), t - LA, jmask, m);
  else k_pairs<R, false><<<g, kThreads, 0, s->stream>>>(a, nwork, make_ins(bits), t - LA, jmask, m);
  return launch_ok("k_pairs");
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

qs_status run_1q(qs_state* s, int q, const double U[8]) {
  return s->dtype == QS_C64 ? pairs_or_inpkt<float>(s, nullptr, 0, q, U)
                            : pairs_or_inpkt<double>(s, nullptr, 0, q, U);
}

qs_status run_controlled(qs_state* s, const int* ctrl, int nc, int t, const double U[8]) {
  return s->dtype == QS_C64 ? pairs_or_inpkt<float>(s, ctrl, nc, t, U)
                            : pairs_or_inpkt<double>(s, ctrl, nc, t, U);
}

template <typename R>
static qs_status diag_impl(qs_state* s, const int* qubits, int k, const double* d) {
  constexpr int LA = PK<R>::LA;
  const int D = 1 << k;
  R* a = static_cast<R*>(s->amp);
  // Sparse form: every entry but the all-ones one is exactly 1.
  bool sparse = true;
  for (int r = 0; r < D - 1 && sparse; ++r) sparse = (d[2 * r] == 1.0 && d[2 * r + 1] == 0.0);
  if (sparse) {
    if (d[2 * (D - 1)] == 1.0 && d[2 * (D - 1) + 1] == 0.0) return QS_OK;  // identity
    std::vector<std::pair<int, int>> bits;
    int jmask = (1 << PK<R>::A) - 1;
    for (int i = 0; i < k; ++i) {
      if (qubits[i] < LA) jmask &= 2;
      else bits.push_back({qubits[i] - LA, 1});
    }
    const u64 nwork = u64(1) << (s->n - LA - (int)bits.size());
    const unsigned g = grid_for(nwork, (u64)kThreads * kU1, kWaves);
    k_phase<R><<<g, kThreads, 0, s->stream>>>(a, nwork, make_ins(bits), jmask, to_z(d[2 * (D - 1)], d[2 * (D - 1) + 1], R(0)));
    return launch_ok("k_phase");
  }
  DiagTab<R> T{};
  T.k = k;
  for (int i = 0; i < k; ++i) T.q[i] = qubits[i];
  for (int i = 0; i < D; ++i) T.d[i] = to_z(d[2 * i], d[2 * i + 1], R(0));
  const u64 npk = u64(1) << (s->n - LA);
  const unsigned g = grid_for(npk, (u64)kThreads * kU1, kWaves);
  k_diag<R><<<g, kThreads, 0, s->stream>>>(a, npk, T);
  return launch_ok("k_diag");
}

qs_status run_diag(qs_state* s, const int* qubits, int k, const double* d) {
  if (k > kMaxDiagK) return fail(QS_EINVAL, "qs_apply_diag: k=%d exceeds %d", k, kMaxDiagK);
  return s->dtype == QS_C64 ? diag_impl<float>(s, qubits, k, d) : diag_impl<double>(s, qubits, k, d);
}

template <typename R>
static qs_status dense_impl(qs_state* s, const int* qubits, int k, const double* M) {
  const int D = 1 << k;
  DenseArgs args{};
  args.k = k;
  std::vector<std::pair<int, int>> bits;
  for (int i = 0; i < k; ++i) bits.push_back({qubits[i], 0});
  args.ins = make_ins(bits);
  for (int r = 0; r < D; ++r) {
    u64 sp = 0;
    for (int i = 0; i < k; ++i)
      if ((r >> i) & 1) sp |= u64(1) << qubits[i];
    args.spread[r] = sp;
  }
  const size_t mbytes = sizeof(R) * 2 * D * D;
  qs_status st = ensure_scratch(s, mbytes);
  if (st != QS_OK) return st;
  std::vector<R> hm(2 * D * D);
  for (int i = 0; i < 2 * D * D; ++i) hm[i] = (R)M[i];
  cudaError_t e = cudaMemcpyAsync(s->scratch, hm.data(), mbytes, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qs_apply_fused: matrix upload");
  const size_t smem = mbytes + sizeof(R) * 2 * D * kGroups;
  auto kern = k_dense<R>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "qs_apply_fused: smem attribute");
  const u64 ngroups = u64(1) << (s->n - k);
  const unsigned g = grid_for(ngroups, kGroups, 4);
  kern<<<g, kThreads, smem, s->stream>>>(static_cast<R*>(s->amp), ngroups, static_cast<const R*>(s->scratch), args);
  st = launch_ok("k_dense");
  if (st != QS_OK) return st;
  // The host copy of M must outlive the asynchronous upload: pageable
  // cudaMemcpyAsync stages the data before returning, so hm may go.
  return QS_OK;
}

qs_status run_dense(qs_state* s, const int* qubits, int k, const double* M, int unitary) {
  if (s->dtype == QS_C64 && k >= 4) return run_dense_tc(s, qubits, k, M, unitary);
  if (s->dtype == QS_C128 && (k == 4 || k == 5)) return run_dense_tc128(s, qubits, k, M);
  return s->dtype == QS_C64 ? dense_impl<float>(s, qubits, k, M) : dense_impl<double>(s, qubits, k, M);
}

template <typename R>
static qs_status bitswap_impl(qs_state* s, const int* pa, const int* pb, int npairs) {
  constexpr int A = PK<R>::A;
  SwapArgs args{};
  args.npairs = 0;
  const int n = s->n;
  // run of 512 bytes (or the whole state if smaller)
  const int Rfull = (A == 2) ? 6 : 5;
  args.R = std::min(Rfull, n);
  std::vector<int> B;
  bool low_pairs = false;
  for (int i = 0; i < npairs; ++i) {
    int x = std::min(pa[i], pb[i]), y = std::max(pa[i], pb[i]);
    if (x == y) continue;
    args.pa[args.npairs] = x;
    args.pb[args.npairs] = y;
    ++args.npairs;
    if (x < args.R) {
      low_pairs = true;
      if (y >= args.R) B.push_back(y);
    }
  }
  if (args.npairs == 0) return QS_OK;
  std::sort(B.begin(), B.end());
  args.nb = (int)B.size();
  std::vector<std::pair<int, int>> bits;
  for (int i = 0; i < args.nb; ++i) {
    args.B[i] = B[i];
    bits.push_back({B[i], 0});
  }
  args.tins = make_ins(bits);
  args.skip_fixed = !low_pairs;
  const int tile = (1 << args.R) << args.nb;
  const size_t smem = sizeof(R) * 2 * tile * 2;
  auto kern = k_bitswap<R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "bitswap: smem attribute");
  const u64 ntiles = u64(1) << (n - args.R - args.nb);
  const unsigned g = grid_for(ntiles, 1, 8);
  kern<<<g, kThreads, smem, s->stream>>>(static_cast<R*>(s->amp), ntiles, args);
  return launch_ok("k_bitswap");
}

qs_status run_bitswap(qs_state* s, const int* a, const int* b, int npairs) {
  if (npairs > 17) return fail(QS_EINVAL, "bit-field exchange: at most 17 pairs");
  return s->dtype == QS_C64 ? bitswap_impl<float>(s, a, b, npairs) : bitswap_impl<double>(s, a, b, npairs);
}

// ---------------------------------------------------------------------------
// |x>: zero the vector, then write 1 at index x.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_set_one(R* a, u64 x) {
  a[2 * x] = (R)1;
  a[2 * x + 1] = (R)0;
}

qs_status run_layout_dfl(qs_state* s, bool to_dfl) {
  if (s->dtype != QS_C128) return QS_OK;
  const u64 npk = u64(1) << s->n;
  const unsigned g = grid_for(npk, kThreads, kWaves);
  if (to_dfl) k_to_dfl<<<g, kThreads, 0, s->stream>>>(static_cast<double*>(s->amp), npk);
  else k_from_dfl<<<g, kThreads, 0, s->stream>>>(static_cast<double*>(s->amp), npk);
  return launch_ok(to_dfl ? "k_to_dfl" : "k_from_dfl");
}

// complex128 gates on a state in double-float storage (see k_to_dfl).
qs_status run_controlled_dfl(qs_state* s, const int* ctrl, int nc, int t, const double U[8]) {
  if (is_x(U)) return run_controlled(s, ctrl, nc, t, U);  // exchange: layout-agnostic
  std::vector<std::pair<int, int>> bits;
  for (int i = 0; i < nc; ++i) bits.push_back({ctrl[i], 1});
  bits.push_back({t, 0});
  const u64 nwork = u64(1) << (s->n - (int)bits.size());
  const unsigned g = grid_for(nwork, (u64)kThreads * kUnroll, kWaves);
  k_pairs_dfl<<<g, kThreads, 0, s->stream>>>(static_cast<float4*>(s->amp), nwork, make_ins(bits), t,
                                             to_mat(U, 0.0));
  return launch_ok("k_pairs_dfl");
}

qs_status run_diag_dfl(qs_state* s, const int* qubits, int k, const double* d) {
  if (k > kMaxDiagK) return fail(QS_EINVAL, "diag: k=%d exceeds %d", k, kMaxDiagK);
  const int D = 1 << k;
  bool sparse = true;
  for (int r = 0; r < D - 1 && sparse; ++r) sparse = (d[2 * r] == 1.0 && d[2 * r + 1] == 0.0);
  float4* a = static_cast<float4*>(s->amp);
  if (sparse) {
    if (d[2 * (D - 1)] == 1.0 && d[2 * (D - 1) + 1] == 0.0) return QS_OK;
    std::vector<std::pair<int, int>> bits;
    for (int i = 0; i < k; ++i) bits.push_back({qubits[i], 1});
    const u64 nwork = u64(1) << (s->n - k);
    const unsigned g = grid_for(nwork, (u64)kThreads * kU1, kWaves);
    k_phase_dfl<<<g, kThreads, 0, s->stream>>>(a, nwork, make_ins(bits), to_z(d[2 * (D - 1)], d[2 * (D - 1) + 1], 0.0));
    return launch_ok("k_phase_dfl");
  }
  DiagTab<double> T{};
  T.k = k;
  for (int i = 0; i < k; ++i) T.q[i] = qubits[i];
  for (int i = 0; i < D; ++i) T.d[i] = to_z(d[2 * i], d[2 * i + 1], 0.0);
  const u64 npk = u64(1) << s->n;
  const unsigned g = grid_for(npk, (u64)kThreads * kU1, kWaves);
  k_diag_dfl<<<g, kThreads, 0, s->stream>>>(a, npk, T);
  return launch_ok("k_diag_dfl");
}

qs_status run_set_basis(qs_state* s, u64 x) {
  cudaError_t e = cudaMemsetAsync(s->amp, 0, state_bytes(s), s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qs_set_basis: memset");
  if (s->dtype == QS_C64) k_set_one<float><<<1, 1, 0, s->stream>>>(static_cast<float*>(s->amp), x);
  else k_set_one<double><<<1, 1, 0, s->stream>>>(static_cast<double*>(s->amp), x);
  return launch_ok("k_set_one");
}

}  // namespace qs
