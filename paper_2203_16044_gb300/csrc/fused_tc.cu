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
// GB300 FP32-SIMT ridge for k >= 4, so it runs on the tensor cores:
// mma.sync m16n8k8 with TF32 inputs and FP32 accumulation, each FP32 operand
// split as x ~ hi + lo (hi = x rounded to TF32, lo = x - hi rounded to
// TF32) and the product formed from three MMAs, hi*hi + lo*hi + hi*lo
// ("3xTF32"): about 22 significant bits per product with unbiased rounding,
// FP32-level for the complex64 path.
//
// Tensor-core FP32 accumulation truncates its internal sums (rounds toward
// zero), which shrinks every output by about an ulp per block -- a bias, not
// noise, and it compounds over a circuit.  When M is unitary (every block a
// plan builds from circuit gates; qs_apply_fused checks on the host) each
// group's norm is exactly preserved by the true result, so the kernel
// rescales every output group to its input group's norm (both summed in
// FP32 from the MMA fragments, reduced across each quad in a fixed order).
//
// A CTA (4 warps) takes chunks of 64 groups: gathers them from HBM into
// shared memory (row stride 2D + 4 floats: conflict-free MMA fragment
// loads; each thread owns one group slot, its addresses in registers), each
// warp multiplies 16 groups by all of B (pre-split into TF32 hi/lo fragment
// records in shared memory, one 16-byte load per three MMAs), stages the
// results in shared memory and scatters them back.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kcommon.cuh"

namespace qs {
namespace {

constexpr int kFT = 128;  // threads per CTA (4 warps)
constexpr int kTG = 64;   // groups per chunk (16 per warp)

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

__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct FusedArgs {
  Ins ins;         // zero insertion at the k qubits (amplitude index space)
  u64 spread[64];  // spread[r]: OR of 2^qubits[i] over the set bits i of r
};

template <int K>
__global__ void __launch_bounds__(kFT) k_fused_tc(float2* __restrict__ a, u64 ngroups, const float* __restrict__ Bg,
                                                  const __grid_constant__ FusedArgs args, int renorm) {
  constexpr int D = 1 << K, KR = 2 * D, NT = KR / 8, KS = KR / 8;
  constexpr int BQS = KS * 4 + 4;  // uint4 row stride of Bq: = 4 (mod 8), conflict-free LDS.128
  constexpr int PAD = KR + 4;      // float row stride of As: conflict-free fragment loads
  constexpr int RPT = D / 2;       // amplitudes per thread per chunk (kTG * D / kFT)
  extern __shared__ __align__(16) uint4 smq[];
  uint4* Bq = smq;                                     // [n][ks * 4 + tq] = (hi b0, hi b1, lo b0, lo b1)
  float* As = reinterpret_cast<float*>(smq + KR * BQS);  // [kTG][PAD]
  for (int i = threadIdx.x; i < KR * KS * 4; i += kFT) {
    const int n = i / (KS * 4), rem = i % (KS * 4), ks = rem >> 2, tq = rem & 3;
    unsigned h0, l0, h1, l1;
    split_tf32(Bg[(8 * ks + tq) * KR + n], h0, l0);
    split_tf32(Bg[(8 * ks + tq + 4) * KR + n], h1, l1);
    Bq[n * BQS + ks * 4 + tq] = make_uint4(h0, h1, l0, l1);
  }
  // this thread's group slot within a chunk, and its amplitudes r = rb + 2 j
  const int bslot = threadIdx.x & (kTG - 1), rb = threadIdx.x >> 6;
  u64 spr[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) spr[j] = args.spread[rb + 2 * j];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  const int row0 = warp * 16;
  for (u64 g0 = (u64)blockIdx.x * kTG; g0 < ngroups; g0 += (u64)gridDim.x * kTG) {
    const u64 g = g0 + bslot;
    const bool valid = g < ngroups;
    const u64 base = expand(valid ? g : 0, args.ins);
    __syncthreads();  // previous chunk's scatter (and the set-up) complete
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      const float2 v = valid ? a[base | spr[j]] : make_float2(0.f, 0.f);
      *reinterpret_cast<float2*>(As + bslot * PAD + 2 * (rb + 2 * j)) = v;
    }
    __syncthreads();
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    float n0 = 0.f, n1 = 0.f;  // input sums of squares, rows gq and gq + 8 (this lane's columns)
#pragma unroll 2
    for (int ks = 0; ks < KS; ++ks) {
      const int kk = 8 * ks;
      const float x0 = As[(row0 + gq) * PAD + kk + tq], x1 = As[(row0 + gq + 8) * PAD + kk + tq];
      const float x2 = As[(row0 + gq) * PAD + kk + tq + 4], x3 = As[(row0 + gq + 8) * PAD + kk + tq + 4];
      n0 = fmaf(x0, x0, fmaf(x2, x2, n0));
      n1 = fmaf(x1, x1, fmaf(x3, x3, n1));
      unsigned ah[4], al[4];
      split_tf32(x0, ah[0], al[0]);
      split_tf32(x1, ah[1], al[1]);
      split_tf32(x2, ah[2], al[2]);
      split_tf32(x3, ah[3], al[3]);
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const uint4 bq = Bq[(nt * 8 + gq) * BQS + ks * 4 + tq];
        mma_tf32(acc[nt], al, bq.x, bq.y);
        mma_tf32(acc[nt], ah, bq.z, bq.w);
        mma_tf32(acc[nt], ah, bq.x, bq.y);
      }
    }
    float f0 = 1.f, f1 = 1.f;
    if (renorm) {
      float m0 = 0.f, m1 = 0.f;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        m0 = fmaf(acc[nt][0], acc[nt][0], fmaf(acc[nt][1], acc[nt][1], m0));
        m1 = fmaf(acc[nt][2], acc[nt][2], fmaf(acc[nt][3], acc[nt][3], m1));
      }
      // the four lanes of a quad hold a row's columns between them
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        n0 += __shfl_xor_sync(0xffffffffu, n0, o);
        n1 += __shfl_xor_sync(0xffffffffu, n1, o);
        m0 += __shfl_xor_sync(0xffffffffu, m0, o);
        m1 += __shfl_xor_sync(0xffffffffu, m1, o);
      }
      f0 = m0 > 0.f ? sqrtf(n0 / m0) : 1.f;
      f1 = m1 > 0.f ? sqrtf(n1 / m1) : 1.f;
    }
    __syncthreads();  // every warp is done reading As
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      *reinterpret_cast<float2*>(As + (row0 + gq) * PAD + nt * 8 + 2 * tq) = make_float2(acc[nt][0] * f0, acc[nt][1] * f0);
      *reinterpret_cast<float2*>(As + (row0 + gq + 8) * PAD + nt * 8 + 2 * tq) = make_float2(acc[nt][2] * f1, acc[nt][3] * f1);
    }
    __syncthreads();
    if (valid) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) a[base | spr[j]] = *reinterpret_cast<const float2*>(As + bslot * PAD + 2 * (rb + 2 * j));
    }
  }
}

// ---------------------------------------------------------------------------
// tcgen05 path (k = 4, 5): the same GEMM with the 5th-generation tensor-core
// instructions.  One CTA of 128 threads per tile of 128 groups = the MMA's M;
// thread t owns group (row) t from gather to scatter:
//   1. gathers its 2^k amplitudes from HBM (constant-bank spread offsets),
//      sums their squares, splits each real into TF32 hi + lo (rounded) and
//      writes both rows to shared memory in the tensor core's K-major
//      "core matrix" layout (8 rows x 16 bytes per 128-byte core matrix);
//   2. thread 0 issues 3 x (2D / 8) tcgen05.mma (M = 128, N = 2D, K = 8;
//      lo*hi, hi*lo, hi*hi per K step) into a TMEM accumulator of 2D FP32
//      columns and commits them to an mbarrier;
//   3. every thread waits on the mbarrier (bounded), reads its row of the
//      accumulator with tcgen05.ld (TMEM lane t = row t), restores the
//      group norm and scatters the result to the same addresses.
// B (hi and lo) is staged once per CTA.  Each CTA keeps the next two tiles'
// loads in flight in registers while a tile's MMAs and epilogue run, and
// several CTAs share an SM (shared memory 40 KB at k = 4, 96 KB at k = 5).  A wait that gives up (about 1 s) sets g_umma_timeout,
// reported by qs_sync; the CTA then stops, frees its TMEM and returns.
// ---------------------------------------------------------------------------
constexpr int kUT = 128;  // threads per CTA = groups per tile = MMA M

__device__ int g_umma_timeout;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzle:
// start address, lbo = byte distance between core matrices adjacent along
// K, sbo = between core matrices adjacent along M (or N); bits 46-48 hold
// the fixed value 0b001; base offset 0, swizzle mode 0.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at 24.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* o) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) o[j] = __uint_as_float(r[j]);
}
// mbarrier phase wait with a limit of about 2^31 SM cycles; false on timeout.
// The "memory" clobber keeps the compiler from sinking earlier loads (the
// next tiles' prefetch) below the wait.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

template <int K>
struct UmmaShape {
  static constexpr int D = 1 << K, KR = 2 * D;
  static constexpr uint32_t A_BYTES = kUT * KR * 4, B_BYTES = KR * KR * 4;
  static constexpr uint32_t LBO_A = (kUT / 8) * 128, LBO_B = (KR / 8) * 128, SBO = 128;
  static constexpr size_t SMEM = 2 * (size_t)A_BYTES + 2 * (size_t)B_BYTES + 16 + 2 * 2 * kUT * sizeof(float);
};

// A thread's share of a group's 2^k amplitudes to / from registers, as CH
// 16-byte words w[j] = amplitudes (2 (j0 + j), 2 (j0 + j) + 1) once taken.  The block's qubits are
// sorted ascending (the host permutes M to match), so when qubit 0 is in the
// block it is block bit 0.
//   lmode 0: 8-byte accesses.
//   lmode 1 (qubit 0 in the block): amplitudes 2j and 2j + 1 are adjacent,
//            one 16-byte access.
//   lmode 2 (qubit 0 not in the block, full tiles): groups t and t ^ 1 are
//            adjacent; the even lane loads both groups' amplitude 2j, the odd
//            lane both groups' amplitude 2j + 1, and group_take exchanges the
//            halves.  The loads have no dependent instruction until the
//            tile is consumed, so a prefetch stays in flight.
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
// o[4j .. 4j + 3] = amplitudes 2 (j0 + j), 2 (j0 + j) + 1 of this thread's group
template <int D, int CH>
__device__ __forceinline__ void group_store(float2* __restrict__ a, u64 base, bool valid, const u64* spread, int lmode,
                                            int j0, const float* o, float f) {
  if (lmode == 1) {
    if (!valid) return;
#pragma unroll
    for (int j = 0; j < CH; ++j)
      *reinterpret_cast<float4*>(a + (base | spread[2 * (j0 + j)])) =
          make_float4(o[4 * j] * f, o[4 * j + 1] * f, o[4 * j + 2] * f, o[4 * j + 3] * f);
  } else if (lmode == 2) {
    const bool odd = threadIdx.x & 1;
    const u64 pb = base & ~u64(1);
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      // even lane stores (own 2j, partner 2j); odd lane (partner 2j + 1, own 2j + 1)
      const float m0x = o[4 * j] * f, m0y = o[4 * j + 1] * f, m1x = o[4 * j + 2] * f, m1y = o[4 * j + 3] * f;
      const float sx = odd ? m0x : m1x, sy = odd ? m0y : m1y;
      const float rx = __shfl_xor_sync(0xffffffffu, sx, 1), ry = __shfl_xor_sync(0xffffffffu, sy, 1);
      *reinterpret_cast<float4*>(a + (pb | spread[2 * (j0 + j) + (odd ? 1 : 0)])) =
          odd ? make_float4(rx, ry, m1x, m1y) : make_float4(m0x, m0y, rx, ry);
    }
  } else if (valid) {
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      a[base | spread[2 * (j0 + j)]] = make_float2(o[4 * j] * f, o[4 * j + 1] * f);
      a[base | spread[2 * (j0 + j) + 1]] = make_float2(o[4 * j + 2] * f, o[4 * j + 3] * f);
    }
  }
}

// H threads per group row (H = 1 or 2): thread t owns row t % 128 and the
// half h = t / 128 of its amplitudes (H = 2), so a CTA has 4 H warps.
template <int K, int H>
__global__ void __launch_bounds__(kUT * H, H == 2 ? 2 : 1)
    k_fused_umma(float2* __restrict__ a, u64 ngroups, const float* __restrict__ Bg,
                 const __grid_constant__ FusedArgs args, int renorm, int lmode) {
  typedef UmmaShape<K> S;
  constexpr int D = S::D, KR = S::KR, NT = kUT * H;
  constexpr int CH = D / 2 / H;  // 16-byte words (amplitude pairs) per thread
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* Ahi = sm;
  unsigned char* Alo = sm + S::A_BYTES;
  unsigned char* Bhi = sm + 2 * S::A_BYTES;
  unsigned char* Blo = Bhi + S::B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + S::B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  float* nin_s = reinterpret_cast<float*>(mbar + 2);  // [H][kUT] partial input norms
  float* nout_s = nin_s + 2 * kUT;                     // [H][kUT] partial output norms
  const int t = threadIdx.x, warp = t >> 5;
  const int row = t & (kUT - 1), h = t / kUT, j0 = h * CH;
  // B operand (N x K, K-major): element (n, k) = B[k][n], split hi + lo
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
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(KR));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  // a warp reads TMEM lanes 32 (warp % 4) .. + 31 = its rows; columns of its half
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * (KR / H));
  const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo), bhi = smem_u32(Bhi), blo = smem_u32(Blo);
  const uint32_t row_off = (uint32_t)(row >> 3) * 128 + (uint32_t)(row & 7) * 16;
  constexpr uint32_t idesc = umma_idesc(kUT, KR);
  uint32_t phase = 0;
  // Software pipeline, two tiles deep: register buffers wA and wB hold the
  // next two tiles' amplitudes; a buffer is refilled with the tile two steps
  // ahead as soon as its contents are in shared memory, so its loads stay in
  // flight during this tile's MMAs and epilogue and the next tile's step.
  const u64 gstep = (u64)gridDim.x * kUT;
  u64 gA = (u64)blockIdx.x * kUT, gB = gA + gstep;
  bool vA = gA + row < ngroups, vB = gB + row < ngroups;
  u64 bA = expand(vA ? gA + row : 0, args.ins), bB = expand(vB ? gB + row : 0, args.ins);
  float4 wA[CH], wB[CH];
  if (gA < ngroups) group_load<D, CH>(a, bA, vA, args.spread, lmode, j0, wA);
  if (gB < ngroups) group_load<D, CH>(a, bB, vB, args.spread, lmode, j0, wB);
  auto step = [&](u64& g, bool& valid, u64& base, float4 (&w)[CH]) -> bool {
    if (g >= ngroups) return false;
    float nin = 0.f;
#pragma unroll
    for (int j = 0; j < CH; ++j) {  // 16-byte chunk c = j0 + j = reals 4c .. 4c + 3 = amplitudes 2c, 2c + 1
      const float4 wc = group_take(w[j], lmode);
      const float x[4] = {wc.x, wc.y, wc.z, wc.w};
      unsigned hh[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        nin = fmaf(x[i], x[i], nin);
        split_tf32(x[i], hh[i], l[i]);
      }
      *reinterpret_cast<uint4*>(Ahi + (j0 + j) * S::LBO_A + row_off) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
      *reinterpret_cast<uint4*>(Alo + (j0 + j) * S::LBO_A + row_off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    if (H > 1) nin_s[h * kUT + row] = nin;
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (H > 1) nin += nin_s[(h ^ 1) * kUT + row];
    if (t == 0) {
#pragma unroll
      for (int ks = 0; ks < KR / 8; ++ks) {
        const uint32_t ao = ks * 2 * S::LBO_A, bo = ks * 2 * S::LBO_B;
        const uint64_t dah = umma_desc(ahi + ao, S::LBO_A, S::SBO), dal = umma_desc(alo + ao, S::LBO_A, S::SBO);
        const uint64_t dbh = umma_desc(bhi + bo, S::LBO_B, S::SBO), dbl = umma_desc(blo + bo, S::LBO_B, S::SBO);
        umma_tf32(tmem, dal, dbh, idesc, ks > 0 ? 1u : 0u);
        umma_tf32(tmem, dah, dbl, idesc, 1u);
        umma_tf32(tmem, dah, dbh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
    }
    // refill this buffer with the tile two steps ahead
    const u64 gn = g + 2 * gstep;
    const bool vn = gn + row < ngroups;
    const u64 bn = expand(vn ? gn + row : 0, args.ins);
    if (gn < ngroups) group_load<D, CH>(a, bn, vn, args.spread, lmode, j0, w);
    if (!__syncthreads_and(mbar_wait(mb, phase) ? 1 : 0)) {
      if (t == 0) atomicExch(&g_umma_timeout, 1);
      return false;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float o[KR / H];
#pragma unroll
    for (int c0 = 0; c0 < KR / H; c0 += 16) tmem_ld16(trow + (uint32_t)c0, o + c0);
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    float f = 1.f;
    if (renorm) {
      float nout = 0.f;
#pragma unroll
      for (int j = 0; j < KR / H; ++j) nout = fmaf(o[j], o[j], nout);
      if (H > 1) {
        nout_s[h * kUT + row] = nout;
        __syncthreads();
        nout += nout_s[(h ^ 1) * kUT + row];
      }
      f = nout > 0.f ? sqrtf(nin / nout) : 1.f;
    }
    group_store<D, CH>(a, base, valid, args.spread, lmode, j0, o, f);
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
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(KR));
}

template <int K, int H>
qs_status launch_umma(qs_state* s, const FusedArgs& A, const float* B, int renorm, const int* qubits) {
  const size_t smem = UmmaShape<K>::SMEM;
  auto kern = k_fused_umma<K, H>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return cuda_fail(e, "fused_umma: smem attribute");
  // CTAs per SM from registers, shared memory and TMEM columns (512 per SM)
  int dev = 0, smem_sm = 0, smem_rsv = 0;
  cudaFuncAttributes fa{};
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return cuda_fail(e, "fused_umma: occupancy attributes");
  int per_sm = smem_sm / (int)(smem + smem_rsv);
  const int regs = fa.numRegs > 0 ? ((fa.numRegs + 7) & ~7) : 255;
  per_sm = std::min(per_sm, 65536 / (regs * kUT * H));
  per_sm = std::min(per_sm, 512 / UmmaShape<K>::KR);
  if (per_sm < 1) per_sm = 1;
  const u64 ngroups = u64(1) << (s->n - K);
  const unsigned grid = grid_for(ngroups, kUT, per_sm);
  // qubits ascending (see run_dense_tc)
  const int lmode = qubits[0] == 0 ? 1 : (ngroups >= (u64)kUT ? 2 : 0);
  kern<<<grid, kUT * H, smem, s->stream>>>(static_cast<float2*>(s->amp), ngroups, B, A, renorm, lmode);
  return launch_ok("k_fused_umma");
}

template <int K>
qs_status launch(qs_state* s, const FusedArgs& A, const float* B, int renorm) {
  constexpr int D = 1 << K, KR = 2 * D, KS = KR / 8, BQS = KS * 4 + 4, PAD = KR + 4;
  const size_t smem = sizeof(uint4) * (size_t)KR * BQS + sizeof(float) * (size_t)kTG * PAD;
  auto kern = k_fused_tc<K>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "fused_tc: smem attribute");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFT, smem);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  const u64 ngroups = u64(1) << (s->n - K);
  const unsigned grid = grid_for(ngroups, kTG, per_sm);
  kern<<<grid, kFT, smem, s->stream>>>(static_cast<float2*>(s->amp), ngroups, B, A, renorm);
  return launch_ok("k_fused_tc");
}

}  // namespace

// Dense k-qubit block (complex64, 4 <= k <= 6) on the tensor cores.
// unitary: 1 = M is known unitary (group norms are restored), 0 = not,
// -1 = check on the host (|M M^dagger - I| <= 1e-9 entrywise).
qs_status run_dense_tc(qs_state* s, const int* qubits, int k, const double* M, int unitary) {
  const int D = 1 << k, KR = 2 * D;
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
  // Block qubits in ascending order: bit p of a row / column index r' of the
  // reordered matrix is bit ord[p] of the caller's index (perm(r')).
  int ord[6], q[6];
  for (int i = 0; i < k; ++i) ord[i] = i;
  std::sort(ord, ord + k, [&](int x, int y) { return qubits[x] < qubits[y]; });
  for (int p = 0; p < k; ++p) q[p] = qubits[ord[p]];
  auto perm = [&](int rp) {
    int r = 0;
    for (int p = 0; p < k; ++p) r |= ((rp >> p) & 1) << ord[p];
    return r;
  };
  FusedArgs A{};
  A.ins.k = k;
  A.ins.set = 0;
  for (int i = 0; i < k; ++i) A.ins.pos[i] = q[i];
  for (int r = 0; r < D; ++r) {
    u64 sp = 0;
    for (int i = 0; i < k; ++i)
      if ((r >> i) & 1) sp |= u64(1) << q[i];
    A.spread[r] = sp;
  }
  // real form of the reordered M: B[2c + u][2r + w]
  std::vector<float> B((size_t)KR * KR);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      const int pr = perm(r), pc = perm(c);
      const double mr = M[2 * (pr * D + pc)], mi = M[2 * (pr * D + pc) + 1];
      B[(size_t)(2 * c) * KR + 2 * r] = (float)mr;
      B[(size_t)(2 * c + 1) * KR + 2 * r] = (float)-mi;
      B[(size_t)(2 * c) * KR + 2 * r + 1] = (float)mi;
      B[(size_t)(2 * c + 1) * KR + 2 * r + 1] = (float)mr;
    }
  const size_t bbytes = B.size() * sizeof(float);
  qs_status st = ensure_scratch(s, bbytes);
  if (st != QS_OK) return st;
  cudaError_t e = cudaMemcpyAsync(s->scratch, B.data(), bbytes, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "fused_tc: matrix upload");
  const float* Bd = static_cast<const float*>(s->scratch);
  switch (k) {
    case 4: return launch_umma<4, 1>(s, A, Bd, unitary, q);
    case 5: return launch_umma<5, 2>(s, A, Bd, unitary, q);
    case 6: return launch<6>(s, A, Bd, unitary);
  }
  return fail(QS_EINVAL, "fused_tc: k=%d outside [4, 6]", k);
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
