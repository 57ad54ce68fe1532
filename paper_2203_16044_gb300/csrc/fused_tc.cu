// Dense k-qubit blocks (k = 4, 5, 6) on the tensor cores, complex64.
//
// For a block over qubits Q (|Q| = k, D = 2^k) every group of D amplitudes
// a[x | spread(r)] (x with the k bits clear) is multiplied by the D x D
// complex matrix M.  With the amplitudes as interleaved reals, a group is a
// row of 2D reals and the block is one real GEMM over all groups:
//   Out[G x 2D] = In[G x 2D] * B[2D x 2D],
//   B[2c][2r] = Re M[r][c], B[2c+1][2r] = -Im M[r][c],
//   B[2c][2r+1] = Im M[r][c], B[2c+1][2r+1] = Re M[r][c].
// Its arithmetic intensity, 2D flops per byte moved at complex64, passes the
// GB300 FP32-SIMT ridge for k >= 4, so it runs on the 5th-generation tensor
// cores (tcgen05.mma, FP32 accumulation in tensor memory).  Each FP32 operand
// is split as x ~ hi + lo and a product is formed from three MMAs, lo*hi +
// hi*lo + hi*hi: with TF32 parts (kind::tf32, "3xTF32") or with FP16 parts
// under exact power-of-two scaling (kind::f16, twice the rate); either way
// about 22 significant bits per product with unbiased rounding, FP32-level
// for the complex64 path.
//
// Two kernels, by the block's qubits (sorted ascending):
//   k_fused_umma_tma   a set forming at most 5 runs with the other qubits
//                      (qubit 0 outside it or in the run 0, 1), or
//                      qubits 0 .. k-1: each tile moves by
//                      TMA (one box of up to 5 dimensions, or 2^k / 16
//                      swizzled 2-D boxes in and out); FP16 parts.
//   k_fused_umma       any other set: per-thread gathers; TF32 parts.
//
// Tensor-core FP32 accumulation truncates its internal sums (rounds toward
// zero), which shrinks every output by about an ulp per block -- a bias, not
// noise, and it compounds over a circuit.  When M is unitary (every block a
// plan builds from circuit gates; qs_apply_fused checks on the host) each
// group's norm is exactly preserved by the true result, so the kernel
// rescales every output group to its input group's norm (both summed in
// FP32, reduced across the row's threads in a fixed order; the correction is
// applied without bias, see norm_correction).
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "kcommon.cuh"
#include "umma.cuh"

namespace qs {
namespace {

// x ~ hi + lo with hi, lo TF32 values (10 explicit significand bits), each
// rounded to nearest (ties away from zero) by adding half a TF32 ulp to the
// bit pattern before clearing the low 13 bits.  Rounding, not truncation:
// truncation shrinks every operand by ~2^-22 on average, a bias that
// compounds over a circuit's blocks.  x - hi is exact in FP32.
__device__ __forceinline__ unsigned round_tf32(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
}
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  const unsigned h = round_tf32(x);
  hi = h;
  lo = round_tf32(x - __uint_as_float(h));
}

struct FusedArgs {
  Ins ins;         // zero insertion at the k qubits (amplitude index space)
  u64 spread[64];  // spread[r]: OR of 2^qubits[i] over the set bits i of r
  RunBox rb;       // k_fused_umma_tma, ROWS = false: the tile's box (make_runs_tmap)
  LowBox lb;       // k_fused_umma_tma, ROWS = true: the tile's pieces (make_lowrun_tmap)
};

// ---------------------------------------------------------------------------
// tcgen05 helpers
// ---------------------------------------------------------------------------

__device__ int g_umma_timeout;

// Instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at 24.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Norm restore for a group whose input norm^2 is nin and output norm^2 nout:
// the output is scaled by sqrt(nin / nout) = 1 + g.  g is formed as a small
// number, g = d / (1 + sqrt(1 + d)) with d = (nin - nout) / nout, and applied
// as o + o g: a scale factor rounded to FP32 next to 1.0 would be biased
// (the FP32 grid is twice as fine just below 1 as just above, so small
// upward corrections round away while downward ones survive), which shrank
// every block's output norm by about one unit roundoff.
__device__ __forceinline__ float norm_correction(float nin, float nout) {
  if (!(nout > 0.f)) return 0.f;
  const float d = (nin - nout) / nout;
  return d / (1.f + sqrtf(1.f + d));
}

// A thread's share of a group's 2^k amplitudes to / from registers, as CH
// 16-byte words w[j] = amplitudes (2 (j0 + j), 2 (j0 + j) + 1) once taken.
// The block's qubits are sorted ascending (the host permutes M to match), so
// when qubit 0 is in the block it is block bit 0.
//   lmode 0: 8-byte accesses.
//   lmode 1 (qubit 0 in the block): amplitudes 2j and 2j + 1 are adjacent,
//            one 16-byte access.
//   lmode 2 (qubit 0 not in the block, full tiles): groups t and t ^ 1 are
//            adjacent; the even lane loads both groups' amplitude 2j, the odd
//            lane both groups' amplitude 2j + 1, and group_take exchanges the
//            halves.  The loads have no dependent instruction until the
//            tile is consumed, so a prefetch stays in flight.
// (Blocks whose tiles are TMA boxes, or on qubits 0 .. k-1, run in
// k_fused_umma_tma instead.)
template <int D, int CH>
__device__ __forceinline__ void group_load(const float2* __restrict__ a, u64 base, bool valid, const u64* spread,
                                           int lmode, int j0, float4 (&w)[CH]) {
  if (lmode == 1) {
#pragma unroll
    for (int j = 0; j < CH; ++j)
      w[j] = valid ? *reinterpret_cast<const float4*>(a + (base | spread[2 * (j0 + j)]))
                   : make_float4(0.f, 0.f, 0.f, 0.f);
  } else if (lmode == 2) {
    const bool odd = threadIdx.x & 1;
    const u64 pb = base & ~u64(1);
#pragma unroll
    for (int j = 0; j < CH; ++j)
      w[j] = *reinterpret_cast<const float4*>(a + (pb | spread[2 * (j0 + j) + (odd ? 1 : 0)]));
  } else {
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const float2 x = valid ? a[base | spread[2 * (j0 + j)]] : make_float2(0.f, 0.f);
      const float2 y = valid ? a[base | spread[2 * (j0 + j) + 1]] : make_float2(0.f, 0.f);
      w[j] = make_float4(x.x, x.y, y.x, y.y);
    }
  }
}
// word j of a group_load as this thread's amplitudes (2j, 2j + 1)
__device__ __forceinline__ float4 group_take(float4 x, int lmode) {
  if (lmode != 2) return x;
  // even lane: x = (own 2j, partner 2j); odd lane: x = (partner 2j + 1, own 2j + 1)
  const bool odd = threadIdx.x & 1;
  const float sx = odd ? x.x : x.z, sy = odd ? x.y : x.w;
  const float rx = __shfl_xor_sync(0xffffffffu, sx, 1), ry = __shfl_xor_sync(0xffffffffu, sy, 1);
  return odd ? make_float4(rx, ry, x.z, x.w) : make_float4(x.x, x.y, rx, ry);
}
// The addresses group_load would read, fetched into L2 only (no registers
// held): issued a few tiles ahead, they keep more bytes in flight than the
// register buffers can, and the later loads hit L2.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
template <int D, int CH>
__device__ __forceinline__ void group_prefetch(const float2* __restrict__ a, u64 base, bool valid, const u64* spread,
                                               int lmode, int j0) {
  if (!valid) return;
  if (lmode == 2) base &= ~u64(1);
  const int odd = lmode == 2 ? (threadIdx.x & 1) : 0;
#pragma unroll
  for (int j = 0; j < CH; ++j) prefetch_l2(a + (base | spread[2 * (j0 + j) + odd]));
}
// o[4j .. 4j + 3] = amplitudes 2 (j0 + j), 2 (j0 + j) + 1 of this thread's
// group; each value is stored as o (1 + g), one rounding (FMA).
template <int D, int CH>
__device__ __forceinline__ void group_store(float2* __restrict__ a, u64 base, bool valid, const u64* spread, int lmode,
                                            int j0, const float* o, float g) {
  auto sc = [g](float v) { return fmaf(v, g, v); };
  if (lmode == 1) {
    if (!valid) return;
#pragma unroll
    for (int j = 0; j < CH; ++j)
      *reinterpret_cast<float4*>(a + (base | spread[2 * (j0 + j)])) =
          make_float4(sc(o[4 * j]), sc(o[4 * j + 1]), sc(o[4 * j + 2]), sc(o[4 * j + 3]));
  } else if (lmode == 2) {
    const bool odd = threadIdx.x & 1;
    const u64 pb = base & ~u64(1);
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      // even lane stores (own 2j, partner 2j); odd lane (partner 2j + 1, own 2j + 1)
      const float m0x = sc(o[4 * j]), m0y = sc(o[4 * j + 1]), m1x = sc(o[4 * j + 2]), m1y = sc(o[4 * j + 3]);
      const float sx = odd ? m0x : m1x, sy = odd ? m0y : m1y;
      const float rx = __shfl_xor_sync(0xffffffffu, sx, 1), ry = __shfl_xor_sync(0xffffffffu, sy, 1);
      *reinterpret_cast<float4*>(a + (pb | spread[2 * (j0 + j) + (odd ? 1 : 0)])) =
          odd ? make_float4(rx, ry, m1x, m1y) : make_float4(m0x, m0y, rx, ry);
    }
  } else if (valid) {
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      a[base | spread[2 * (j0 + j)]] = make_float2(sc(o[4 * j]), sc(o[4 * j + 1]));
      a[base | spread[2 * (j0 + j) + 1]] = make_float2(sc(o[4 * j + 2]), sc(o[4 * j + 3]));
    }
  }
}

// ---------------------------------------------------------------------------
// The block kernel (k = 4, 5, 6).  The MMA's A operand may
// live in tensor memory (lane = row, one 32-bit column per K element), so the
// tile never passes through shared memory: each thread writes its share of
// its row, split into TF32 hi and lo, straight into its own TMEM lane with
// tcgen05.st.  Shared memory holds only B (hi and lo: 8 KB at k = 4, 32 KB at
// k = 5, 128 KB at k = 6), which is what lets k = 6 fit.  TMEM columns: A hi
// [0, 2D), A lo [2D, 4D), accumulator [4D, 6D) (128, 256 or all 512 columns,
// so 4, 2 or 1 CTAs share an SM).  H = 2^(k+1) / 32 threads per row, each
// owning 32 reals (16 amplitudes) of it: 128, 256 or 512 threads.  Per
// tile: take + split + tcgen05.st, one CTA barrier, 3 (2D / 8)
// MMAs issued by one thread, the next tiles' loads issued, the bounded
// mbarrier wait, tcgen05.ld of the thread's 32 accumulator columns, the group
// norm restored across the row's H threads (shared memory), and the scatter.
// Two register buffers keep the next two tiles' loads in flight meanwhile.
// A wait that gives up (about 1 s) sets g_umma_timeout, reported by qs_sync;
// the CTA then stops, frees its TMEM and returns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void umma_tf32_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, uint32_t idesc,
                                             uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bd), "r"(idesc), "r"(acc));
}

template <int K>
struct TaShape {
  static constexpr int D = 1 << K, KR = 2 * D, H = KR / 32, NT = kUT * H;
  static constexpr uint32_t B_BYTES = KR * KR * 4, LBO_B = (KR / 8) * 128, SBO = 128;
  static constexpr uint32_t TCOLS = 3 * KR <= 128 ? 128 : (3 * KR <= 256 ? 256 : 512);  // power of two >= 3 KR
  static constexpr size_t SMEM = 2 * (size_t)B_BYTES + 16 + 2 * H * kUT * sizeof(float);
};

template <int K>
__global__ void __launch_bounds__(TaShape<K>::NT, 512 / TaShape<K>::TCOLS)
    k_fused_umma(float2* __restrict__ a, u64 ngroups, const float* __restrict__ Bg,
                    const __grid_constant__ FusedArgs args, int renorm, int lmode, int pf) {
  typedef TaShape<K> S;
  constexpr int D = S::D, KR = S::KR, H = S::H, NT = S::NT;
  constexpr int CH = 8;  // 16-byte words (amplitude pairs) per thread: 32 reals
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* Bhi = sm;
  unsigned char* Blo = sm + S::B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + S::B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  float* nin_s = reinterpret_cast<float*>(mbar + 2);  // [H][kUT] partial input norms
  float* nout_s = nin_s + H * kUT;                     // [H][kUT] partial output norms
  const int t = threadIdx.x, warp = t >> 5;
  const int row = t & (kUT - 1), h = t / kUT, j0 = h * CH;
  for (int i = t; i < KR * KR; i += NT) {
    const int k = i / KR, n = i % KR;
    unsigned hh, l;
    split_tf32(Bg[i], hh, l);
    const uint32_t off = ((k >> 2) * (KR / 8) + (n >> 3)) * 128 + (n & 7) * 16 + (k & 3) * 4;
    *reinterpret_cast<unsigned*>(Bhi + off) = hh;
    *reinterpret_cast<unsigned*>(Blo + off) = l;
  }
  const uint32_t mb = smem_u32(mbar);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(S::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  // this warp's 32 lanes (= its rows), and this thread's 32 columns in each region
  const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * 32);
  const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
  constexpr uint32_t idesc = umma_idesc(kUT, KR);
  uint32_t phase = 0;
  const u64 gstep = (u64)gridDim.x * kUT;
  u64 gA = (u64)blockIdx.x * kUT, gB = gA + gstep;
  bool vA = gA + row < ngroups, vB = gB + row < ngroups;
  u64 bA = expand(vA ? gA + row : 0, args.ins), bB = expand(vB ? gB + row : 0, args.ins);
  float4 wA[CH], wB[CH];
  auto load = [&](u64 base, bool valid, float4 (&w)[CH]) {
    group_load<D, CH>(a, base, valid, args.spread, lmode, j0, w);
  };
  // L2 prefetch (pf != 0) of the tile two tile-steps ahead of the one
  // being loaded into registers
  auto prefetch = [&](u64 g) {
    if (!pf || g >= ngroups) return;
    const bool v = g + row < ngroups;
    group_prefetch<D, CH>(a, expand(v ? g + row : 0, args.ins), v, args.spread, lmode, j0);
  };
  if (gA < ngroups) load(bA, vA, wA);
  if (gB < ngroups) load(bB, vB, wB);
  prefetch(gA + 2 * gstep);
  prefetch(gA + 3 * gstep);
  auto step = [&](u64& g, bool& valid, u64& base, float4 (&w)[CH]) -> bool {
    if (g >= ngroups) return false;
    float nin = 0.f;
#pragma unroll
    for (int half = 0; half < 2; ++half) {  // 16 columns (4 words) at a time
      unsigned hv[16], lv[16];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 wc = group_take(w[4 * half + j], lmode);
        const float x[4] = {wc.x, wc.y, wc.z, wc.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          nin = fmaf(x[i], x[i], nin);
          split_tf32(x[i], hv[4 * j + i], lv[4 * j + i]);
        }
      }
      tmem_st16(tl + (uint32_t)(16 * half), hv);
      tmem_st16(tl + (uint32_t)(KR + 16 * half), lv);
    }
    nin_s[h * kUT + row] = nin;
    asm volatile("tcgen05.wait::st.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    nin = 0.f;
#pragma unroll
    for (int i = 0; i < H; ++i) nin += nin_s[i * kUT + row];
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < KR / 8; ++ks) {
        const uint32_t bo = ks * 2 * S::LBO_B;
        const uint64_t dbh = umma_desc(bhi + bo, S::LBO_B, S::SBO), dbl = umma_desc(blo + bo, S::LBO_B, S::SBO);
        const uint32_t ahi_t = tmem + (uint32_t)(ks * 8), alo_t = tmem + (uint32_t)(KR + ks * 8);
        umma_tf32_ta(tmem + 2 * KR, alo_t, dbh, idesc, ks > 0 ? 1u : 0u);
        umma_tf32_ta(tmem + 2 * KR, ahi_t, dbl, idesc, 1u);
        umma_tf32_ta(tmem + 2 * KR, ahi_t, dbh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
    }
    const u64 gn = g + 2 * gstep;
    const bool vn = gn + row < ngroups;
    const u64 bn = expand(vn ? gn + row : 0, args.ins);
    if (gn < ngroups) load(bn, vn, w);
    prefetch(gn + 2 * gstep);
    if (!__syncthreads_and(mbar_wait(mb, phase) ? 1 : 0)) {
      if (t == 0) atomicExch(&g_umma_timeout, 1);
      return false;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float o[32];
    tmem_ld16(tl + (uint32_t)(2 * KR), o);
    tmem_ld16(tl + (uint32_t)(2 * KR + 16), o + 16);
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    float gsc = 0.f;  // output = o (1 + gsc)
    if (renorm) {
      float nout = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) nout = fmaf(o[j], o[j], nout);
      nout_s[h * kUT + row] = nout;
      __syncthreads();
      nout = 0.f;
#pragma unroll
      for (int i = 0; i < H; ++i) nout += nout_s[i * kUT + row];
      gsc = norm_correction(nin, nout);
    }
    group_store<D, CH>(a, base, valid, args.spread, lmode, j0, o, gsc);
    asm volatile("tcgen05.fence::before_thread_sync;");
    g = gn;
    valid = vn;
    base = bn;
    return true;
  };
  while (step(gA, vA, bA, wA) && step(gB, vB, bB, wB)) {
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TCOLS));
}

// ---------------------------------------------------------------------------
// FP16 split for the TMA-fed kernel below (kind::f16, twice the TF32 rate).
// Each operand is split x ~ hi + lo with hi = fp16(x), lo = fp16(x - hi),
// both round-to-nearest: 11 significant bits each, the same 22-bit products
// as 3xTF32 from the same three MMAs per K step.  FP16's narrow exponent
// range is handled with exact powers of two: the block matrix is scaled by
// 2^f so that max |b| < 2^14, and each group (row) by 2^e so that its norm,
// hence every |x|, is below 2^14 (e from the row's sum of squares, which the
// norm restore needs anyway); the accumulator is scaled back by 2^-(e + f)
// before the epilogue.  Values far below their row's or the matrix's maximum
// keep an absolute error of about 2^-24 of that maximum.  TMEM: A hi
// [0, D), A lo [D, 2D) (two FP16 values per 32-bit column, even K index in
// the low half), accumulator [2D, 4D).  (With the tile gathered by
// per-thread loads, as in k_fused_umma, this halved the MMA time without
// making the kernel faster: the load issue then took its place.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }  // -126 <= e <= 127
// E with v in [2^E, 2^(E+1)) for a positive normal float (-127 for subnormals)
__device__ __forceinline__ int fexp(float v) { return ((__float_as_int(v) >> 23) & 255) - 127; }
// scale exponent of a value set whose maximum magnitude is below 2^(E+1):
// the scaled maximum stays below 2^14, and e + f stays within [-126, 126]
__device__ __forceinline__ int scale_exp(int E, int lo, int hi) { return max(lo, min(hi, 13 - E)); }
__device__ __forceinline__ uint32_t h2bits(__half2 v) { return *reinterpret_cast<uint32_t*>(&v); }
// (a, b) -> FP16 pairs hi = (fp16(a), fp16(b)), lo = residuals, a in the low half
__device__ __forceinline__ void split_f16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  hi = h2bits(h);
  lo = h2bits(__floats2half2_rn(a - hf.x, b - hf.y));
}
// ---------------------------------------------------------------------------
// Blocks on any qubit set whose qubits, with the others, form at most 5
// runs, qubit 0 outside the set or in the run 0, 1 (windows, two-run sets;
// full tiles):
// k_fused_umma_tma.  A tile of 128 consecutive groups is then one box of a
// view of the state with up to 5 dimensions (make_runs_tmap): a single TMA
// copy (cp.async.bulk.tensor, completion counted on an mbarrier) moves it
// into shared memory, with no per-thread load instructions and no registers
// held; element e of tile row r lands at a position the view's dimension
// order fixes (per-bit multipliers in the kernel arguments).  The stage is
// refilled
// with the next tile as soon as every thread has read the current one, so
// the copy runs under the split, the MMAs and the epilogue.  Two tiles are
// in flight on two TMEM sets (A hi, A lo and the accumulator each): tile j
// is split and its MMAs issued, then tile j-1's epilogue runs while those
// MMAs do (2 x 256 TMEM columns at k = 6, one CTA per SM).  Arithmetic: the
// FP16 split above (kind::f16).  Shared memory at k = 6: stage 64 KB,
// output stage 64 KB, B 64 KB.  Blocks on qubits 0 .. k-1 take the same
// kernel with ROWS set (below).
// ---------------------------------------------------------------------------
// ROWS = false: the run box above; the outputs go out by one TMA store from
// a second stage at k = 6, by 8-byte stores at k = 4, 5.  ROWS = true: the
// block's qubits start with a run 0 .. a-1 of at least 16 amplitudes
// (qubits 0 .. k-1, or such a run plus others, as QFT blocks are): the tile
// moves as 2^a / 16 boxes (make_lowrun_tmap), box b holding amplitudes
// 16 b .. 16 b + 15 of the low run for every row and every value of the
// other block qubits, in 128-byte-swizzled layout (16-byte unit c of smem
// line L stored at unit c ^ (L mod 8)); a thread's 16 amplitudes are one
// line of one box, so the reads and the output writes are conflict-free
// 16-byte accesses, and the outputs leave through a second stage with TMA
// stores (a row per lane would touch 32 cache lines per warp store).
template <int K, bool ROWS>
struct TShape {
  static constexpr int D = 1 << K, KR = 2 * D, H = KR / 32, NT = kUT * H;
  static constexpr uint32_t STAGE = kUT * D * 8;  // one tile: 128 groups x 2^K amplitudes
  // outputs leave through a second stage by TMA stores for qubits 0 .. k-1,
  // and for windows at k = 6 (one CTA per SM there, where the per-thread
  // scatter's store issue was the longest phase)
  static constexpr bool TSTORE = ROWS || K == 6;
  static constexpr uint32_t OUT = TSTORE ? STAGE : 0;
  static constexpr uint32_t B_BYTES = KR * KR * 2, LBO_B = (KR / 8) * 128, SBO = 128;
  static constexpr uint32_t SETCOLS = 2 * KR;  // one tile's TMEM: A hi, A lo (KR / 2 each), accumulator
  static constexpr uint32_t TCOLS = 2 * SETCOLS;  // two tiles in flight
  static constexpr size_t SMEM = STAGE + OUT + 2 * (size_t)B_BYTES + 32 + 2 * H * kUT * sizeof(float);
  static constexpr int MINB = K == 6 ? 1 : (K == 5 ? 2 : 4);  // register-limited
};

template <int K, bool ROWS>
__global__ void __launch_bounds__(TShape<K, ROWS>::NT, TShape<K, ROWS>::MINB)
    k_fused_umma_tma(float2* __restrict__ a, u64 ngroups, const float* __restrict__ Bg,
                     const __grid_constant__ FusedArgs args, const __grid_constant__ CUtensorMap tmap, int renorm) {
  typedef TShape<K, ROWS> S;
  constexpr int D = S::D, KR = S::KR, H = S::H, NT = S::NT;
  constexpr int CH = 8;
  extern __shared__ __align__(1024) unsigned char sm[];
  const float2* stage = reinterpret_cast<const float2*>(sm);
  unsigned char* outst = sm + S::STAGE;  // ROWS: the output stage
  unsigned char* Bhi = sm + S::STAGE + S::OUT;
  unsigned char* Blo = Bhi + S::B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + S::B_BYTES);  // [0] tile loaded, [1 + b] MMAs of set b done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 3);
  uint32_t* bmax_s = tslot + 1;
  float* nin_s = reinterpret_cast<float*>(mbar + 4);  // [H][kUT] partial input norms
  float* nout_s = nin_s + H * kUT;                     // [H][kUT] partial output norms
  const int t = threadIdx.x, warp = t >> 5;
  const int row = t & (kUT - 1), h = t / kUT, j0 = h * CH;
  const uint32_t mb_full = smem_u32(mbar), mb_mma0 = smem_u32(mbar + 1);
  const u64 gstep = (u64)gridDim.x * kUT;
  u64 g = (u64)blockIdx.x * kUT;
  // ROWS: piece b of the low run, for every line, at box b (STAGE / nslice bytes)
  const uint32_t boxb = ROWS ? S::STAGE / (uint32_t)args.lb.nslice : 0;
  auto tile_load = [&](u64 gt) {  // one thread
    mbar_expect_tx(mb_full, S::STAGE);
    if (ROWS) {
      lowrun_load(smem_u32(stage), boxb, &tmap, gt, args.lb, mb_full);
    } else {
      run_load(smem_u32(stage), &tmap, gt, args.rb, 1, mb_full);
    }
  };
  if (t == 0) {
    *bmax_s = 0u;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_full));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_mma0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb_mma0 + 8));
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (g < ngroups) tile_load(g);  // under the B set-up
  }
  __syncthreads();
  {
    float m = 0.f;
    for (int i = t; i < KR * KR; i += NT) m = fmaxf(m, fabsf(Bg[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0) atomicMax(bmax_s, __float_as_uint(m));
  }
  __syncthreads();
  const float bmax = __uint_as_float(*bmax_s);
  const int f = bmax > 0.f ? scale_exp(fexp(bmax), -100, 100) : 0;
  {
    const float sb = pow2f(f);
    for (int i = t; i < KR * KR; i += NT) {
      const int k = i / KR, n = i % KR;
      const float b = Bg[i] * sb;
      const __half hh = __float2half_rn(b);
      const __half ll = __float2half_rn(b - __half2float(hh));
      const uint32_t off = ((k >> 3) * (KR / 8) + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
      *reinterpret_cast<__half*>(Bhi + off) = hh;
      *reinterpret_cast<__half*>(Blo + off) = ll;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(S::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
  constexpr uint32_t idesc = umma_idesc_f16(kUT, KR);
  // ROWS: this thread's 16 amplitudes are piece h mod nslice of the low run
  // in line row + 128 (h / nslice) of its box
  const uint32_t rowoff = ROWS ? (uint32_t)(h % args.lb.nslice) * boxb +
                                     (uint32_t)(row + kUT * (h / args.lb.nslice)) * 128u
                               : 0u;
  // ROWS = false: element 16 h + i of this row at pbase + (multipliers of i's bits)
  const int pbase = ROWS ? 0
                         : run_row_pos(args.rb, row) + ((h & 1) ? args.rb.multe[4] : 0) + ((h & 2) ? args.rb.multe[5] : 0);
  const int pm[4] = {args.rb.multe[0], args.rb.multe[1], args.rb.multe[2], args.rb.multe[3]};
  uint32_t ph_full = 0, ph_mma = 0;  // ph_mma bit b: TMEM set b
  uint32_t outstanding = 0;           // bit b: MMAs of set b issued and not yet waited for

  // Tile gt from the stage into TMEM set b (A hi, A lo), then its MMAs
  // issued; e (the row scale) and nin (the row's input norm^2) for its
  // epilogue.  The next tile's copy starts as soon as every thread has read
  // the stage.  False (in every thread) if a bounded wait gave up.
  auto split_issue = [&](u64 gt, int b, int& e, float& nin) -> bool {
    const bool loaded = mbar_wait(mb_full, ph_full);
    ph_full ^= 1u;
    float2 v[16];
    if (ROWS) {
      // 16-byte unit c of this thread's line sits at c ^ (row mod 8)
      const float4* rowp = reinterpret_cast<const float4*>(sm + rowoff);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 q = rowp[c ^ (row & 7)];
        v[2 * c] = make_float2(q.x, q.y);
        v[2 * c + 1] = make_float2(q.z, q.w);
      }
    } else if (pm[0] == 1) {  // qubits 0, 1 in the block: elements 2j, 2j + 1 adjacent
#pragma unroll
      for (int i = 0; i < 16; i += 2) {
        const float4 q = *reinterpret_cast<const float4*>(stage + run_elem_pos<4>(pbase, pm, i));
        v[i] = make_float2(q.x, q.y);
        v[i + 1] = make_float2(q.z, q.w);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = stage[run_elem_pos<4>(pbase, pm, i)];
    }
    nin = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) nin = fmaf(v[i].x, v[i].x, fmaf(v[i].y, v[i].y, nin));
    nin_s[h * kUT + row] = nin;
    if (!__syncthreads_and(loaded ? 1 : 0)) return false;
    if (t == 0 && gt + gstep < ngroups) tile_load(gt + gstep);  // the stage has been read
    nin = 0.f;
#pragma unroll
    for (int i = 0; i < H; ++i) nin += nin_s[i * kUT + row];
    e = (nin > 0.f && nin < INFINITY) ? scale_exp((fexp(nin) + 2) >> 1, -126 - f, 126 - f) : 0;
    const uint32_t ta = tmem + lanes + (uint32_t)(b * S::SETCOLS + h * 16);
    {
      const float sx = pow2f(e);
      uint32_t hv[16], lv[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) split_f16x2(v[i].x * sx, v[i].y * sx, hv[i], lv[i]);
      tmem_st16(ta, hv);
      tmem_st16(ta + (uint32_t)(KR / 2), lv);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // A of set b written by every thread
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (t == 0) {
      const uint32_t set = tmem + (uint32_t)(b * S::SETCOLS);
#pragma unroll
      for (int ks = 0; ks < KR / 16; ++ks) {
        const uint32_t bo = ks * 2 * S::LBO_B;
        const uint64_t dbh = umma_desc(bhi + bo, S::LBO_B, S::SBO), dbl = umma_desc(blo + bo, S::LBO_B, S::SBO);
        const uint32_t ahi_t = set + (uint32_t)(ks * 8), alo_t = set + (uint32_t)(KR / 2 + ks * 8);
        umma_f16_ta(set + KR, alo_t, dbh, idesc, ks > 0 ? 1u : 0u);
        umma_f16_ta(set + KR, ahi_t, dbl, idesc, 1u);
        umma_f16_ta(set + KR, ahi_t, dbh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb_mma0 + 8 * b));
    }
    outstanding |= 1u << b;
    return true;
  };
  // The outputs of tile gt from TMEM set b: scaled back, the group norm
  // restored, and stored (through the output stage and a TMA store, or
  // directly).
  auto epilogue = [&](u64 gt, int b, int e, float nin) -> bool {
    // the previous tile's TMA stores must have read the output stage
    if (S::TSTORE && t == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    const bool done = mbar_wait(mb_mma0 + 8 * b, (ph_mma >> b) & 1u);
    if (!__syncthreads_and(done ? 1 : 0)) return false;
    ph_mma ^= 1u << b;
    outstanding &= ~(1u << b);
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t td = tmem + lanes + (uint32_t)(b * S::SETCOLS + KR + h * 32);
    float o[32];
    tmem_ld16(td, o);
    tmem_ld16(td + 16, o + 16);
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    const float so = pow2f(-(e + f));
#pragma unroll
    for (int j = 0; j < 32; ++j) o[j] *= so;
    float gsc = 0.f;
    if (renorm) {
      float nout = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) nout = fmaf(o[j], o[j], nout);
      nout_s[h * kUT + row] = nout;
      __syncthreads();
      nout = 0.f;
#pragma unroll
      for (int i = 0; i < H; ++i) nout += nout_s[i * kUT + row];
      gsc = norm_correction(nin, nout);
    }
    if (ROWS) {
      float4* rowo = reinterpret_cast<float4*>(outst + rowoff);
#pragma unroll
      for (int c = 0; c < 8; ++c)
        rowo[c ^ (row & 7)] = make_float4(fmaf(o[4 * c], gsc, o[4 * c]), fmaf(o[4 * c + 1], gsc, o[4 * c + 1]),
                                          fmaf(o[4 * c + 2], gsc, o[4 * c + 2]), fmaf(o[4 * c + 3], gsc, o[4 * c + 3]));
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (t == 0) {
        lowrun_store(&tmap, gt, args.lb, smem_u32(outst), boxb);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    } else if (S::TSTORE) {
      // the output tile in the input stage's layout, then one TMA store
      float2* outw = reinterpret_cast<float2*>(outst);
      if (pm[0] == 1) {
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const int j = 2 * i;
          *reinterpret_cast<float4*>(outw + run_elem_pos<4>(pbase, pm, i)) =
              make_float4(fmaf(o[j], gsc, o[j]), fmaf(o[j + 1], gsc, o[j + 1]), fmaf(o[j + 2], gsc, o[j + 2]),
                          fmaf(o[j + 3], gsc, o[j + 3]));
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = 2 * i;
          outw[run_elem_pos<4>(pbase, pm, i)] = make_float2(fmaf(o[j], gsc, o[j]), fmaf(o[j + 1], gsc, o[j + 1]));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (t == 0) {
        run_store(&tmap, gt, args.rb, 1, smem_u32(outst));
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    } else {
      group_store<D, CH>(a, expand(gt + row, args.ins), true, args.spread, 0, j0, o, gsc);
    }
    return true;
  };

  // Two tiles in flight on the two TMEM sets: tile g is split and its MMAs
  // issued, then the previous tile's epilogue runs while those MMAs do.
  bool fine = true, prev = false;
  u64 gp = 0;
  int ep = 0, it = 0;
  float ninp = 0.f;
  while (g < ngroups) {
    int e = 0;
    float nin = 0.f;
    if (!(fine = split_issue(g, it & 1, e, nin))) break;
    if (prev && !(fine = epilogue(gp, (it - 1) & 1, ep, ninp))) break;
    prev = true;
    gp = g;
    ep = e;
    ninp = nin;
    g += gstep;
    ++it;
  }
  if (fine && prev) fine = epilogue(gp, (it - 1) & 1, ep, ninp);
  if (!fine) {
    if (t == 0) atomicExch(&g_umma_timeout, 1);
    // let MMAs already issued finish before the tensor memory is freed (bounded)
    for (int b2 = 0; b2 < 2; ++b2)
      if ((outstanding >> b2) & 1u) mbar_wait(mb_mma0 + 8 * b2, (ph_mma >> b2) & 1u);
  }
  if (S::TSTORE && t == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TCOLS));
}

// Grid for a block kernel: CTAs per SM from shared memory, registers and TMEM
// columns (the occupancy query does not know about TMEM), times the SMs.
template <int K, typename Kern>
qs_status block_grid(qs_state* s, Kern kern, int nthreads, size_t smem, int tcols, unsigned& grid) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return cuda_fail(e, "fused_tc: smem attribute");
  int dev = 0, smem_sm = 0, smem_rsv = 0;
  cudaFuncAttributes fa{};
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return cuda_fail(e, "fused_tc: occupancy attributes");
  int per_sm = smem_sm / (int)(smem + smem_rsv);
  const int regs = fa.numRegs > 0 ? ((fa.numRegs + 7) & ~7) : 255;
  per_sm = std::min(per_sm, 65536 / (regs * nthreads));
  per_sm = std::min(per_sm, 512 / tcols);
  if (per_sm < 1) per_sm = 1;
  // (a state in a batch asks for several tiles per CTA: each CTA's set-up --
  // tensor memory, barriers, the block matrix -- then serves more tiles, and
  // the batch's concurrent circuits share the SMs)
  grid = grid_for(u64(1) << (s->n - K), (u64)kUT * (u64)std::max(1, s->tiles_per_cta), per_sm);
  return QS_OK;
}

template <int K>
qs_status launch_umma(qs_state* s, const FusedArgs& A, const float* B, int renorm, const int* qubits) {
  const u64 ngroups = u64(1) << (s->n - K);
  const bool full = ngroups >= (u64)kUT;
  unsigned grid = 0;
  // a low run 0 .. a-1 of at least 16 amplitudes (qubits 0 .. K-1 among
  // them): 128-byte swizzled pieces
  {
    FusedArgs AL = A;
    CUtensorMap map;
    qs_status est = QS_OK;
    if (full && make_lowrun_tmap(s->amp, s->n, K, qubits, 1, 16, &map, &AL.lb, &est)) {
      typedef TShape<K, true> ST;
      qs_status st = block_grid<K>(s, k_fused_umma_tma<K, true>, ST::NT, ST::SMEM, ST::TCOLS, grid);
      if (st != QS_OK) return st;
      k_fused_umma_tma<K, true><<<grid, ST::NT, ST::SMEM, s->stream>>>(static_cast<float2*>(s->amp), ngroups, B,
                                                                         AL, map, renorm);
      return launch_ok("k_fused_umma_tma");
    }
    if (est != QS_OK) return est;
  }
  // any other set whose qubits form at most 5 runs (qubit 0 outside it or
  // in the run 0, 1): one TMA box per tile
  {
    FusedArgs AR = A;
    CUtensorMap map;
    qs_status est = QS_OK;
    if (full && make_runs_tmap(s->amp, s->n, K, qubits, 1, &map, &AR.rb, &est)) {
      typedef TShape<K, false> ST;
      qs_status st = block_grid<K>(s, k_fused_umma_tma<K, false>, ST::NT, ST::SMEM, ST::TCOLS, grid);
      if (st != QS_OK) return st;
      k_fused_umma_tma<K, false><<<grid, ST::NT, ST::SMEM, s->stream>>>(static_cast<float2*>(s->amp), ngroups, B,
                                                                          AR, map, renorm);
      return launch_ok("k_fused_umma_tma");
    }
    if (est != QS_OK) return est;
  }
  typedef TaShape<K> S;
  // access mode (see group_load); 8-byte accesses measured faster than the
  // lane-pair exchange at k = 6 once a warp's 32 groups are contiguous
  // (lowest block qubit >= 5); L2 prefetch helped k = 4, 5 and slowed k = 6
  const int lmode = qubits[0] == 0 ? 1 : (full && !(K == 6 && qubits[0] >= 5) ? 2 : 0);
  const int pf = K < 6 && full;
  qs_status st = block_grid<K>(s, k_fused_umma<K>, S::NT, S::SMEM, S::TCOLS, grid);
  if (st != QS_OK) return st;
  k_fused_umma<K><<<grid, S::NT, S::SMEM, s->stream>>>(static_cast<float2*>(s->amp), ngroups, B, A, renorm, lmode, pf);
  return launch_ok("k_fused_umma");
}

}  // namespace

// Host-side preparation of a tensor-core block: the qubits in ascending
// order (q_sorted) and B, the real form of M with its row / column indices
// reordered to match (bit p of a reordered index is bit ord[p] of the
// caller's), B[2c + u][2r + w] as in the header comment.
qs_status tc_prepare(const int* qubits, int k, const double* M, int* q_sorted, std::vector<float>& B) {
  if (k < 4 || k > 6) return fail(QS_EINVAL, "fused_tc: k=%d outside [4, 6]", k);
  const int D = 1 << k, KR = 2 * D;
  int ord[6];
  for (int i = 0; i < k; ++i) ord[i] = i;
  small_sort(ord, k, [&](int x, int y) { return qubits[x] < qubits[y]; });
  for (int p = 0; p < k; ++p) q_sorted[p] = qubits[ord[p]];
  int perm[64];
  for (int rp = 0; rp < D; ++rp) {
    int r = 0;
    for (int p = 0; p < k; ++p) r |= ((rp >> p) & 1) << ord[p];
    perm[rp] = r;
  }
  B.assign((size_t)KR * KR, 0.0f);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      const int pr = perm[r], pc = perm[c];
      const double mr = M[2 * (pr * D + pc)], mi = M[2 * (pr * D + pc) + 1];
      B[(size_t)(2 * c) * KR + 2 * r] = (float)mr;
      B[(size_t)(2 * c + 1) * KR + 2 * r] = (float)-mi;
      B[(size_t)(2 * c) * KR + 2 * r + 1] = (float)mi;
      B[(size_t)(2 * c + 1) * KR + 2 * r + 1] = (float)mr;
    }
  return QS_OK;
}

// Launch a prepared block; Bdev holds its B on the device.
qs_status run_dense_tc_prepared(qs_state* s, const int* q_sorted, int k, const float* Bdev, int unitary) {
  const int D = 1 << k;
  FusedArgs A{};
  A.ins.k = k;
  A.ins.set = 0;
  for (int i = 0; i < k; ++i) A.ins.pos[i] = q_sorted[i];
  for (int r = 0; r < D; ++r) {
    u64 sp = 0;
    for (int i = 0; i < k; ++i)
      if ((r >> i) & 1) sp |= u64(1) << q_sorted[i];
    A.spread[r] = sp;
  }
  switch (k) {
    case 4: return launch_umma<4>(s, A, Bdev, unitary, q_sorted);
    case 5: return launch_umma<5>(s, A, Bdev, unitary, q_sorted);
    case 6: return launch_umma<6>(s, A, Bdev, unitary, q_sorted);
  }
  return fail(QS_EINVAL, "fused_tc: k=%d outside [4, 6]", k);
}

// Dense k-qubit block (complex64, 4 <= k <= 6) on the tensor cores.
// unitary: 1 = M is known unitary (group norms are restored), 0 = not,
// -1 = check on the host (|M M^dagger - I| <= 1e-9 entrywise).
qs_status run_dense_tc(qs_state* s, const int* qubits, int k, const double* M, int unitary) {
  const int D = 1 << k;
  if (unitary < 0) {
    unitary = 1;
    for (int r = 0; r < D && unitary; ++r)
      for (int c = 0; c < D && unitary; ++c) {
        double re = 0.0, im = 0.0;  // (M M^dagger)[r][c]
        for (int j = 0; j < D; ++j) {
          const double ar = M[2 * (r * D + j)], ai = M[2 * (r * D + j) + 1];
          const double br = M[2 * (c * D + j)], bi = -M[2 * (c * D + j) + 1];
          re += ar * br - ai * bi;
          im += ar * bi + ai * br;
        }
        if (std::fabs(re - (r == c ? 1.0 : 0.0)) > 1e-9 || std::fabs(im) > 1e-9) unitary = 0;
      }
  }
  int q[6];
  std::vector<float> B;
  qs_status st = tc_prepare(qubits, k, M, q, B);
  if (st != QS_OK) return st;
  const size_t bbytes = B.size() * sizeof(float);
  if ((st = ensure_scratch(s, bbytes)) != QS_OK) return st;
  cudaError_t e = cudaMemcpyAsync(s->scratch, B.data(), bbytes, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "fused_tc: matrix upload");
  return run_dense_tc_prepared(s, q, k, static_cast<const float*>(s->scratch), unitary);
}

// A tcgen05 wait that gave up since the last call: QS_ETIMEOUT (and clear).
qs_status fused_tc_status() {
  int flag = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&flag, g_umma_timeout, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "fused_tc: status read");
  if (!flag) return QS_OK;
  const int zero = 0;
  cudaMemcpyToSymbol(g_umma_timeout, &zero, sizeof(int));
  return fail(QS_ETIMEOUT, "fused_tc: a tensor-core wait gave up; the state is invalid");
}

}  // namespace qs
