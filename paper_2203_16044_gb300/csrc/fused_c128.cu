// Dense k-qubit blocks (k = 4, 5) on the tensor cores, complex128.
//
// The block is the real GEMM of the complex64 kernels (fused_tc.cu): every
// group of D = 2^k amplitudes is a row of 2D reals, Out[G x 2D] =
// In[G x 2D] * B[2D x 2D] with B the real form of M^T.  Here the operands are
// FP64 and the state stays in the standard complex128 layout.
//
// FP64 products come from an error-free splitting of both operands into
// small integer digits, after Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numerical Algorithms 59, 2012):
//  * every row of A (one group) is put on a fixed-point grid of its own,
//    a = 2^(E - 43) X with E the row's largest binary exponent (|a| < 2^E)
//    and X an integer with |X| <= 2^43; B likewise with one exponent F for
//    the whole matrix (prepared on the host);
//  * X = sum_{i<5} d_i 2^(9 (4 - i)) with digits d_i in [-256, 256): with the
//    offset kOff (256 at every digit position) added, each digit is a plain
//    9-bit field of X + kOff, so the split is shifts and masks;
//  * digits are exact FP16 values and a digit product is exact in the MMA;
//    level s collects sum_{i + j = s} d_i e_j over the K = 2D reals in an
//    FP32 accumulator of its own in tensor memory.  B's digit matrices sit
//    side by side, [e_0 | e_1 | e_2 | e_3 | e_4] (N = 5 x 2D), and the level
//    accumulators side by side as well, so one MMA per digit i of A and K
//    step, over the first 5 - i blocks of B, adds d_i e_j into level i + j
//    for every j at once;
//  * bounds: |d_0|, |e_0| <= 128 (|X| <= 2^43), the other digits <= 256, so
//    level s <= max(1, s) 2^16 K -- below 2^24, the FP32 range of exact
//    integers, for s <= 4 at k = 4 and s <= 3 at k = 5;
//  * level 5 (pairs (1,4), (2,3), (3,2), (4,1)) is folded into the level-4
//    accumulator through copies of e_1 .. e_4 scaled by 2^-9 (still exact
//    FP16 values), four narrow MMAs per K step: the one FP32 rounding of
//    that accumulator is below 2^-50 of the level-0 scale.  Levels >= 6 are
//    dropped (below 2^-50 as well);
//  * the epilogue sums S = sum_s acc_s 2^(-9 s) in double-float (Knuth's
//    TwoSum on the level values) and assembles S 2^(E + F - 14) as FP64
//    bits with integer operations.
// No FP64 instruction is issued.  Accuracy: the 43-bit grids dominate, an
// error of about 2^-44 of the group's largest value (and of B's largest
// entry) per block.

// Tiles of 128 groups are the MMA's M (= TMEM lanes).  Each thread owns 4
// amplitudes of one row (H = D / 4 threads per row: 512 threads at k = 4,
// 1024 at k = 5, for latency hiding of the integer work).  TMEM: the five digit
// slices of A, D columns each (two FP16 values per 32-bit column: re, im of
// one amplitude), then five level accumulators of 2D FP32 columns: 240
// columns at k = 4 (two CTAs per SM), 480 at k = 5 (one).  Three ways in:
//   MODE 2: the block's qubits start with a run 0 .. a-1 of at least 8
//           amplitudes (qubits 0 .. k-1, or such a run plus others):
//           2^a / 8 TMA boxes (8 amplitudes of the low run x 128 rows x
//           the other block qubits, 128-byte swizzle; make_lowrun_tmap) in,
//           the same boxes out by TMA stores from a second stage;
//   MODE 1: any set without qubit 0 forming at most 5 runs with the other
//           qubits (windows, two-run sets): one TMA box of a view with up
//           to 5 dimensions per tile in (make_runs_tmap), the same box out
//           by a TMA store from a second stage;
//   MODE 0: any other set: per-thread 16-byte gathers and scatters.
// The next tile's TMA copy is issued as soon as the current one has been
// split, so it runs under the MMAs and the epilogue.  Where the time goes
// (clock64 phase timing at k = 5, cycles per tile): split 4,300-5,300, MMAs
// 2,400 (near the FP16 tensor peak for the 15 digit-pair products), epilogue
// 6,400-8,000, against ~6,100 cycles of HBM time: integer and FP32 issue,
// not the tensor cores, bound the kernel.  Every mbarrier wait is
// bounded (about 1 s): a wait that gives up sets g_c128_timeout, reported
// by qs_sync as QS_ETIMEOUT; the CTA then frees its tensor memory and stops.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "dfloat.cuh"
#include "kcommon.cuh"
#include "umma.cuh"

namespace qs {
namespace {

constexpr int kDig = 5;  // digits per value, 9 bits each
// 256 at every digit position: digit i of X + kOff is bits 9 (4 - i) .. +8
constexpr long long kOff = 256LL * (1LL + (1LL << 9) + (1LL << 18) + (1LL << 27) + (1LL << 36));

__device__ int g_c128_timeout;

struct C128Args {
  Ins ins;         // zero insertion at the k qubits
  u64 spread[32];  // spread[r]: OR of 2^qubits[i] over the set bits i of r
  RunBox rb;       // MODE 1: the tile's box (make_runs_tmap)
  LowBox lb;       // MODE 2: the tile's pieces (make_lowrun_tmap)
};

template <int K, int MODE>
struct CShape {
  static constexpr int APT = 4;  // amplitudes per thread
  static constexpr int D = 1 << K, KR = 2 * D, H = D / APT, NT = kUT * H;
  static constexpr uint32_t TILE = kUT * D * 16;            // one tile: 128 groups
  static constexpr uint32_t SET = kDig * D + kDig * KR;     // TMEM columns of one tile: digits, levels
  static constexpr uint32_t TCOLS = SET <= 256 ? 256 : 512;
  static constexpr int NSTAGE = MODE ? 1 : 0;               // TMA input stage
  static constexpr uint32_t OUT = MODE ? TILE : 0;     // output stage (TMA stores)
  static constexpr uint32_t DIG_BYTES = KR * KR * 2;        // one FP16 digit matrix of B
  static constexpr int NBLK = 2 * kDig - 1;                 // e_0 .. e_4, then e_4 .. e_1 scaled by 2^-9
  static constexpr uint32_t NB = NBLK * KR;                 // columns of the digit matrices side by side
  static constexpr uint32_t LBO_B = (NB / 8) * 128, SBO = 128;
  static constexpr size_t SMEM = NSTAGE * (size_t)TILE + OUT + NBLK * (size_t)DIG_BYTES + 64 + H * kUT * sizeof(int);
  static constexpr int MINB = 512 / TCOLS;
  static constexpr int BPR = 8 / APT;  // threads per 8-amplitude box (MODE 2)
};

__device__ __forceinline__ int fp64_exp(unsigned long long b) { return (int)((b >> 52) & 0x7ffu); }

// X + kOff for X = round(a 2^(43 - E)), E = em - 1022 (em: the row's largest
// biased exponent, so |a| < 2^E and |X| <= 2^43).  Subnormal inputs count
// as zero.
__device__ __forceinline__ unsigned long long fixed_point(unsigned long long b, int em) {
  const int e = fp64_exp(b);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int r = em - e + 10;  // >= 10
  const unsigned long long X = (e == 0 || r >= 64) ? 0ull : (m + (1ull << (r - 1))) >> r;
  return (b >> 63) ? (unsigned long long)kOff - X : (unsigned long long)kOff + X;
}

// S = a0 + a1 2^-9 + a2 2^-18 + a3 2^-27 + a4 2^-36 as a normalised
// double-float h + l, from the level sums (exact integers in FP32): the two
// lowest levels in one FMA (error below 2^-27 against a0 up to 2^22), the
// others by TwoSum.
__device__ __forceinline__ dfl levels_to_df(float a0, float a1, float a2, float a3, float a4) {
  const float lo = fmaf(a3, 0x1p-27f, a4 * 0x1p-36f);
  float e1, e2, e3;
  float s = two_sum(a2 * 0x1p-18f, lo, e1);
  s = two_sum(a1 * 0x1p-9f, s, e2);
  s = two_sum(a0, s, e3);
  dfl r;
  r.h = fast_two_sum(s, __fadd_rn(__fadd_rn(e1, e2), e3), r.l);
  return r;
}

// (h + l) 2^delta as FP64 bits, integer operations only (the conversion of
// df2d with the exponent moved by delta); below the normal range: zero.
__device__ __forceinline__ double df2d_scaled(dfl v, int delta) {
  const unsigned hb = __float_as_uint(v.h), lb = __float_as_uint(v.l);
  const int eh = (int)((hb >> 23) & 0xffu);
  const unsigned fh = hb & 0x7fffffu;
  const unsigned long long sg = (unsigned long long)(hb & 0x80000000u) << 32;
  const int ed = eh + 896 + delta;
  if (eh == 0 || ed <= 0) return __longlong_as_double((long long)sg);
  unsigned long long D = sg | ((unsigned long long)ed << 52) | ((unsigned long long)fh << 29);
  const int el = (int)((lb >> 23) & 0xffu);
  if (eh < 52 || el == 0) return __longlong_as_double((long long)D);
  const unsigned ml = 0x800000u | (lb & 0x7fffffu);
  const int sh = el - eh + 29;
  unsigned long long k;
  if (sh >= 0) k = (unsigned long long)ml << sh;
  else if (sh > -24) k = (unsigned long long)(ml >> (-sh));
  else k = 0ull;
  if ((hb ^ lb) & 0x80000000u) D -= (fh == 0u) ? (k << 1) : k;
  else D += k;
  return __longlong_as_double((long long)D);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }  // -126 <= e <= 127
// the two floats of a 64-bit word of double-float storage (low half first)
__device__ __forceinline__ float lo_f(unsigned long long w) { return __uint_as_float((unsigned)w); }
__device__ __forceinline__ float hi_f(unsigned long long w) { return __uint_as_float((unsigned)(w >> 32)); }

// Digits of X ~ x + y (x, y already on the grid: |x + y| < 2^43, y below
// half an ulp of x) as FP32 integers: d_0 .. d_2 rounded to nearest
// multiples of 2^36, 2^27, 2^18 of x (each remainder exact), then y added
// (rounding below 2^-7) and d_3, d_4 to multiples of 2^9 and 1.  Rounding to
// an integer: x 2^-s + 1.5 2^23 rounds once in FP32 (the FMA), and
// subtracting 1.5 2^23 again is exact.  |d_0| <= 128, the others <= 256,
// sum d_i 2^(36 - 9i) within 0.51 of x + y: the FP64 path's digits, by
// floating-point operations instead of integer ones.
__device__ __forceinline__ void digits_df(float x, float y, float (&d)[kDig][4], int i) {
  constexpr float kR = 0x1.8p23f;
  d[0][i] = fmaf(x, 0x1p-36f, kR) - kR;
  x = fmaf(-d[0][i], 0x1p36f, x);
  d[1][i] = fmaf(x, 0x1p-27f, kR) - kR;
  x = fmaf(-d[1][i], 0x1p27f, x);
  d[2][i] = fmaf(x, 0x1p-18f, kR) - kR;
  x = fmaf(-d[2][i], 0x1p18f, x) + y;
  d[3][i] = fmaf(x, 0x1p-9f, kR) - kR;
  x = fmaf(-d[3][i], 0x1p9f, x);
  d[4][i] = (x + kR) - kR;
}

// (h + l) 2^delta of the real and imaginary parts as one 16-byte word of
// double-float storage (re h, re l, im h, im l); delta outside the FP32
// scale range takes scalbnf (rows far from unit scale).
__device__ __forceinline__ double2 scaled_pairs(dfl r, dfl i, int delta) {
  float4 o;
  if (delta >= -126 && delta <= 127) {
    const float p = pow2f(delta);
    o = make_float4(r.h * p, r.l * p, i.h * p, i.l * p);
  } else {
    o = make_float4(scalbnf(r.h, delta), scalbnf(r.l, delta), scalbnf(i.h, delta), scalbnf(i.l, delta));
  }
  return *reinterpret_cast<const double2*>(&o);
}

template <int K, int MODE, int IO>
__global__ void __launch_bounds__(CShape<K, MODE>::NT, CShape<K, MODE>::MINB)
    k_fused_c128(double2* __restrict__ a, u64 ngroups, const uint4* __restrict__ Bdig, int Fexp,
                 const __grid_constant__ C128Args args, const __grid_constant__ CUtensorMap tmap) {
  typedef CShape<K, MODE> S;
  constexpr int D = S::D, KR = S::KR, H = S::H, NT = S::NT, APT = S::APT;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* stage = sm;                             // MODE 1, 2: the input tile
  unsigned char* outst = sm + S::NSTAGE * S::TILE;       // MODE 1, 2: output stage
  unsigned char* Bs = outst + S::OUT;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Bs + S::NBLK * S::DIG_BYTES);  // [0] stage full, [2] MMAs done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 4);
  int* emax_s = reinterpret_cast<int*>(mbar + 6);  // [H][kUT] partial row exponents
  const int t = threadIdx.x, warp = t >> 5;
  const int row = t & (kUT - 1), h = t / kUT;
  const uint32_t mb0 = smem_u32(mbar);
  const u64 gstep = (u64)gridDim.x * kUT;
  // MODE 2: piece b of the low run (8 amplitudes), for every line, at box b
  const uint32_t boxb = MODE == 2 ? S::TILE / (uint32_t)args.lb.nslice : 0;
  auto tile_load = [&](u64 gt, int st) {  // one thread
    const uint32_t mb = mb0 + 8 * st, dst = smem_u32(stage) + st * S::TILE;
    mbar_expect_tx(mb, S::TILE);
    if (MODE == 2) {
      lowrun_load(dst, boxb, &tmap, gt, args.lb, mb);
    } else {
      run_load(dst, &tmap, gt, args.rb, 2, mb);
    }
  };
  u64 g = (u64)blockIdx.x * kUT;
  if (t == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0 + 8 * i));
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (MODE) {  // the first tiles, under the B copy
      for (int st = 0; st < S::NSTAGE; ++st)
        if (g + st * gstep < ngroups) tile_load(g + st * gstep, st);
    }
  }
  // B's digit matrices [e_0 | ... | e_4 | e_4' | e_3' | e_2' | e_1'] (e' = e 2^-9),
  // prepared on the host in the K-major core-matrix layout (8 x 8 FP16 core
  // matrices of 128 bytes), copied as they are
  for (int i = t; i < (int)(S::NBLK * S::DIG_BYTES / 16); i += NT) reinterpret_cast<uint4*>(Bs)[i] = Bdig[i];
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
  const uint32_t bsa = smem_u32(Bs);
  // MODE 1: element APT h + i of this row at pbase + (multipliers of i's bits) (amplitudes)
  int pbase = 0;
  if (MODE == 1) {
    pbase = run_row_pos(args.rb, row);
#pragma unroll
    for (int j = 2; j < 6; ++j)
      if (((APT * h) >> j) & 1) pbase += args.rb.multe[j];
  }
  const int pm[2] = {args.rb.multe[0], args.rb.multe[1]};
  // MODE 2: this thread's amplitudes are units u0 .. u0 + APT - 1 of the
  // 8-amplitude piece h / BPR: piece (h / BPR) mod nslice of the low run, in
  // line row + 128 ((h / BPR) / nslice) of its box
  const int u0 = (h % S::BPR) * APT;
  const uint32_t rowoff = MODE == 2 ? (uint32_t)((h / S::BPR) % args.lb.nslice) * boxb +
                                          (uint32_t)(row + kUT * ((h / S::BPR) / args.lb.nslice)) * 128u
                                    : 0u;
  const __half2 k1280 = __floats2half2_rn(1280.f, 1280.f);
  uint32_t ph_full = 0, ph_mma = 0;  // phase bits (bit b: stage / TMEM set b)

  // Split tile gt into digit slices of TMEM set `buf` (input stage `buf`);
  // returns false if a bounded wait gave up (every thread agrees).
  auto split = [&](u64 gt, int buf, int& em, bool& valid) -> bool {
    bool ok = true;
    valid = true;
    ulonglong2 v[APT];  // amplitudes APT h .. APT h + APT - 1 of this row, raw FP64 bits
    if (MODE == 0) {
      valid = gt + row < ngroups;
      const u64 base = expand(valid ? gt + row : 0, args.ins);
#pragma unroll
      for (int i = 0; i < APT; ++i)
        v[i] = valid ? *reinterpret_cast<const ulonglong2*>(a + (base | args.spread[APT * h + i]))
                     : make_ulonglong2(0ull, 0ull);
    } else {
      ok = mbar_wait(mb0 + 8 * buf, (ph_full >> buf) & 1u);
      ph_full ^= 1u << buf;
      const unsigned char* stg = stage + buf * S::TILE;
      if (MODE == 2) {
        // amplitude APT h + i is unit u0 + i of this thread's line, stored at unit (u0 + i) ^ (row mod 8)
        const unsigned char* rb = stg + rowoff;
#pragma unroll
        for (int i = 0; i < APT; ++i)
          v[i] = *reinterpret_cast<const ulonglong2*>(rb + (((u0 + i) ^ (row & 7)) << 4));
      } else {
        const ulonglong2* st2 = reinterpret_cast<const ulonglong2*>(stg);
#pragma unroll
        for (int i = 0; i < APT; ++i) v[i] = st2[run_elem_pos<2>(pbase, pm, i)];
      }
    }
    em = 0;
    if constexpr (IO == 0) {
#pragma unroll
      for (int i = 0; i < APT; ++i) em = max(em, max(fp64_exp(v[i].x), fp64_exp(v[i].y)));
    } else {  // the high floats bound the values: em = biased FP32 exponent of the largest
      float mx = 0.f;
#pragma unroll
      for (int i = 0; i < APT; ++i) mx = fmaxf(mx, fmaxf(fabsf(lo_f(v[i].x)), fabsf(lo_f(v[i].y))));
      em = (int)(__float_as_uint(mx) >> 23);
    }
    emax_s[h * kUT + row] = em;
    if (!__syncthreads_and(ok ? 1 : 0)) return false;
    em = 0;
#pragma unroll
    for (int j = 0; j < H; ++j) em = max(em, emax_s[j * kUT + row]);
    const uint32_t ta = tmem + lanes + (uint32_t)(buf * S::SET + h * APT);
    if constexpr (IO == 0) {
      unsigned long long xp[2 * APT];
#pragma unroll
      for (int i = 0; i < APT; ++i) {
        xp[2 * i] = fixed_point(v[i].x, em);
        xp[2 * i + 1] = fixed_point(v[i].y, em);
      }
      // digit slice j, column APT h + i: (d_j(re), d_j(im)) of amplitude
      // APT h + i; FP16 bits 0x6400 | u are the value 1024 + u, so subtracting
      // 1280 leaves the digit u - 256 exactly
#pragma unroll
      for (int j = 0; j < kDig; ++j) {
        const int sh = 9 * (4 - j);
        unsigned w[APT];
#pragma unroll
        for (int i = 0; i < APT; ++i) {
          const unsigned ur = (unsigned)(xp[2 * i] >> sh) & 511u, ui = (unsigned)(xp[2 * i + 1] >> sh) & 511u;
          const unsigned raw = 0x64006400u | ur | (ui << 16);
          const __half2 d = __hsub2(*reinterpret_cast<const __half2*>(&raw), k1280);
          w[i] = *reinterpret_cast<const unsigned*>(&d);
        }
        tmem_st4(ta + (uint32_t)(j * D), w);
      }
    } else {
      // scale 2^(43 - E), E = em - 126: two factors where it exceeds 2^127
      // (rows below 2^-85); an all-zero row (em = 0) scales to zero
      const int sc = 169 - em;
      const float s1 = em == 0 ? 0.f : pow2f(min(sc, 127)), s2 = pow2f(max(sc - 127, 0));
      float dr[kDig][APT], di[kDig][APT];
#pragma unroll
      for (int i = 0; i < APT; ++i) {
        float xr = lo_f(v[i].x) * s1, yr = hi_f(v[i].x) * s1, xi = lo_f(v[i].y) * s1, yi = hi_f(v[i].y) * s1;
        if (sc > 127) {
          xr *= s2;
          yr *= s2;
          xi *= s2;
          yi *= s2;
        }
        digits_df(xr, yr, dr, i);
        digits_df(xi, yi, di, i);
      }
#pragma unroll
      for (int j = 0; j < kDig; ++j) {
        unsigned w[APT];
#pragma unroll
        for (int i = 0; i < APT; ++i) {
          const __half2 d = __floats2half2_rn(dr[j][i], di[j][i]);  // exact: integers below 2^9
          w[i] = *reinterpret_cast<const unsigned*>(&d);
        }
        tmem_st4(ta + (uint32_t)(j * D), w);
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // digits written, and every thread is done with the stage
    asm volatile("tcgen05.fence::after_thread_sync;");
    return true;
  };
  // One thread: the MMAs of TMEM set `buf`: d_i times blocks e_0 .. e_(4-i)
  // into levels i .. 4 (at most 256 columns per MMA), and for i >= 1 d_i
  // times e'_(5-i) (level 5) into level 4; then the commit.
  auto issue = [&](int buf) {
    const uint32_t set = tmem + (uint32_t)(buf * S::SET);
    const uint32_t lev = set + (uint32_t)(kDig * D);
#pragma unroll
    for (int ks = 0; ks < KR / 16; ++ks) {
      const uint32_t bk = bsa + (uint32_t)(ks * 2 * S::LBO_B);
#pragma unroll
      for (int i = 0; i < kDig; ++i) {
        const uint32_t ncols = (uint32_t)((kDig - i) * KR), a_t = set + (uint32_t)(i * D + ks * 8);
#pragma unroll
        for (uint32_t c0 = 0; c0 < (uint32_t)(kDig * KR); c0 += 256) {
          if (c0 >= ncols) break;
          const uint32_t nc = ncols - c0 < 256u ? ncols - c0 : 256u;
          umma_f16_ta(lev + (uint32_t)(i * KR) + c0, a_t, umma_desc(bk + (c0 / 8) * 128, S::LBO_B, S::SBO),
                      umma_idesc_f16(kUT, (int)nc), (i > 0 || ks > 0) ? 1u : 0u);
        }
        if (i >= 1)  // e'_(5 - i) is block kDig + i - 1
          umma_f16_ta(lev + (uint32_t)((kDig - 1) * KR), a_t,
                      umma_desc(bk + (uint32_t)(((kDig + i - 1) * KR / 8) * 128), S::LBO_B, S::SBO),
                      umma_idesc_f16(kUT, KR), 1u);
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb0 + 8 * (2 + buf)));
  };
  // Wait for the MMAs of set `buf`, then the outputs of tile gt.
  auto epilogue = [&](u64 gt, int buf, int em, bool valid) -> bool {
    if (MODE && t == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // out stage free
    const bool done = mbar_wait(mb0 + 8 * (2 + buf), (ph_mma >> buf) & 1u);
    ph_mma ^= 1u << buf;
    if (!__syncthreads_and(done ? 1 : 0)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // outputs 2 APT h .. 2 APT h + 2 APT - 1 (amplitude APT h + p: reals 2 p,
    // 2 p + 1) of each level, then S 2^(E + F - 14) with E = em - 1022
    const uint32_t td = tmem + lanes + (uint32_t)(buf * S::SET + kDig * D + h * 2 * APT);
    float acc[kDig][2 * APT];
#pragma unroll
    for (int l = 0; l < kDig; ++l) {
      if (APT == 8) tmem_ld16(td + (uint32_t)(l * KR), acc[l]);
      else tmem_ld8(td + (uint32_t)(l * KR), acc[l]);
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    const int delta = (IO == 0 ? em - 1022 : em - 126) + Fexp - 14;
    const u64 base = MODE ? 0 : expand(valid ? gt + row : 0, args.ins);
#pragma unroll
    for (int p = 0; p < APT; ++p) {
      const dfl vr = levels_to_df(acc[0][2 * p], acc[1][2 * p], acc[2][2 * p], acc[3][2 * p], acc[4][2 * p]);
      const dfl vi =
          levels_to_df(acc[0][2 * p + 1], acc[1][2 * p + 1], acc[2][2 * p + 1], acc[3][2 * p + 1], acc[4][2 * p + 1]);
      double2 o;
      if constexpr (IO == 0) {
        o.x = df2d_scaled(vr, delta);
        o.y = df2d_scaled(vi, delta);
      } else {  // the double-float pairs times 2^delta: (re h, re l, im h, im l)
        o = scaled_pairs(vr, vi, delta);
      }
      if (MODE == 2) {
        *reinterpret_cast<double2*>(outst + rowoff + (((u0 + p) ^ (row & 7)) << 4)) = o;
      } else if (MODE == 1) {
        reinterpret_cast<double2*>(outst)[run_elem_pos<2>(pbase, pm, p)] = o;  // the input stage's layout
      } else if (valid) {
        a[base | args.spread[APT * h + p]] = o;
      }
    }
    if (MODE) {
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (t == 0) {
        if (MODE == 2) {
          lowrun_store(&tmap, gt, args.lb, smem_u32(outst), boxb);
        } else {
          run_store(&tmap, gt, args.rb, 2, smem_u32(outst));
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    return true;
  };

  // one tile at a time: split, MMAs, epilogue.  (Two tiles in flight, with
  // two TMEM sets and one CTA per SM at k = 4, measured slower than two CTAs
  // per SM with one set each.)
  bool fine = true;
  int em = 0;
  bool val = true;
  while (g < ngroups) {
    if (!(fine = split(g, 0, em, val))) break;
    if (t == 0) {
      if (MODE && g + gstep < ngroups) tile_load(g + gstep, 0);
      issue(0);
    }
    if (!(fine = epilogue(g, 0, em, val))) break;
    g += gstep;
  }
  if (!fine && t == 0) atomicExch(&g_c128_timeout, 1);
  if (MODE && t == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TCOLS));
}

// CTAs per SM from shared memory, registers and TMEM columns, times the SMs.
template <typename Kern>
qs_status c128_grid(qs_state* s, int K, Kern kern, int nthreads, size_t smem, int tcols, unsigned& grid) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return cuda_fail(e, "fused_c128: smem attribute");
  int dev = 0, smem_sm = 0, smem_rsv = 0;
  cudaFuncAttributes fa{};
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return cuda_fail(e, "fused_c128: occupancy attributes");
  int per_sm = smem_sm / (int)(smem + smem_rsv);
  const int regs = fa.numRegs > 0 ? ((fa.numRegs + 7) & ~7) : 255;
  per_sm = std::min(per_sm, 65536 / (regs * nthreads));
  per_sm = std::min(per_sm, 512 / tcols);
  if (per_sm < 1) per_sm = 1;
  grid = grid_for(u64(1) << (s->n - K), kUT, per_sm);
  return QS_OK;
}

template <int K, int MODE, int IO>
qs_status launch_io(qs_state* s, const C128Args& A, const uint4* Bdig, int F, const CUtensorMap& map) {
  typedef CShape<K, MODE> S;
  unsigned grid = 0;
  qs_status st = c128_grid(s, K, k_fused_c128<K, MODE, IO>, S::NT, S::SMEM, S::TCOLS, grid);
  if (st != QS_OK) return st;
  k_fused_c128<K, MODE, IO><<<grid, S::NT, S::SMEM, s->stream>>>(static_cast<double2*>(s->amp),
                                                                 u64(1) << (s->n - K), Bdig, F, A, map);
  return launch_ok("k_fused_c128");
}
template <int K, int MODE>
qs_status launch_mode(qs_state* s, const C128Args& A, const uint4* Bdig, int F, const CUtensorMap& map, bool dfl) {
  return dfl ? launch_io<K, MODE, 1>(s, A, Bdig, F, map) : launch_io<K, MODE, 0>(s, A, Bdig, F, map);
}

template <int K>
qs_status launch_c128(qs_state* s, const int* q, const uint4* Bdig, int F, bool dfl) {
  C128Args A{};
  A.ins.k = K;
  A.ins.set = 0;
  for (int i = 0; i < K; ++i) A.ins.pos[i] = q[i];
  for (int r = 0; r < (1 << K); ++r) {
    u64 sp = 0;
    for (int i = 0; i < K; ++i)
      if ((r >> i) & 1) sp |= u64(1) << q[i];
    A.spread[r] = sp;
  }
  const bool full = s->n - K >= 7;  // whole tiles of 128 groups
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  qs_status est = QS_OK;
  if (full && make_lowrun_tmap(s->amp, s->n, K, q, 2, 8, &map, &A.lb, &est)) return launch_mode<K, 2>(s, A, Bdig, F, map, dfl);
  if (est != QS_OK) return est;
  if (full && make_runs_tmap(s->amp, s->n, K, q, 2, &map, &A.rb, &est)) return launch_mode<K, 1>(s, A, Bdig, F, map, dfl);
  if (est != QS_OK) return est;
  return launch_mode<K, 0>(s, A, Bdig, F, map, dfl);
}

// FP16 bit pattern of d 2^-p for an integer |d| < 2^11 whose value stays in
// FP16's normal range (exact).
uint16_t f16_of_scaled(int d, int p) {
  if (d == 0) return 0;
  const unsigned sg = d < 0 ? 0x8000u : 0u;
  const unsigned m = (unsigned)(d < 0 ? -d : d);
  int e = 0;
  while ((m >> (e + 1)) != 0) ++e;  // floor(log2 m)
  return (uint16_t)(sg | ((unsigned)(e - p + 15) << 10) | ((m << (10 - e)) & 0x3ffu));
}
uint16_t f16_of_int(int d) { return f16_of_scaled(d, 0); }

}  // namespace

// Host-side preparation of a complex128 tensor-core block: the qubits in
// ascending order, B (the real form of M^T with rows and columns reordered
// to match, as for the complex64 blocks) on the fixed-point grid
// b = 2^(F - 43) Z, |Z| <= 2^43, and Z's digit matrices e_0 .. e_4 and
// e_4, e_3, e_2, e_1 scaled by 2^-9 as FP16 matrices side by side
// (2D x 18D), in the layout the kernel copies into shared memory.
qs_status tc128_prepare(const int* qubits, int k, const double* M, int* q_sorted, std::vector<uint16_t>& dig,
                        int* F) {
  if (k < 4 || k > 5) return fail(QS_EINVAL, "fused_c128: k=%d outside [4, 5]", k);
  const int D = 1 << k, KR = 2 * D;
  int ord[6];
  for (int i = 0; i < k; ++i) ord[i] = i;
  small_sort(ord, k, [&](int x, int y) { return qubits[x] < qubits[y]; });
  for (int p = 0; p < k; ++p) q_sorted[p] = qubits[ord[p]];
  int perm[32];
  for (int rp = 0; rp < D; ++rp) {
    int r = 0;
    for (int p = 0; p < k; ++p) r |= ((rp >> p) & 1) << ord[p];
    perm[rp] = r;
  }
  std::vector<double> B((size_t)KR * KR, 0.0);  // B[kk][n], kk = input real, n = output real
  double bmax = 0.0;
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      const int pr = perm[r], pc = perm[c];
      const double mr = M[2 * (pr * D + pc)], mi = M[2 * (pr * D + pc) + 1];
      B[(size_t)(2 * c) * KR + 2 * r] = mr;
      B[(size_t)(2 * c + 1) * KR + 2 * r] = -mi;
      B[(size_t)(2 * c) * KR + 2 * r + 1] = mi;
      B[(size_t)(2 * c + 1) * KR + 2 * r + 1] = mr;
      bmax = std::max(bmax, std::max(std::fabs(mr), std::fabs(mi)));
    }
  if (!std::isfinite(bmax)) return fail(QS_EINVAL, "fused_c128: matrix entries must be finite");
  int e = 0;
  if (bmax > 0.0) std::frexp(bmax, &e);  // bmax < 2^e
  *F = e;
  constexpr int kBlk = 2 * kDig - 1;  // e_0 .. e_4, then e_4 .. e_1 scaled by 2^-9
  dig.assign((size_t)kBlk * KR * KR, 0);
  for (int kk = 0; kk < KR; ++kk)
    for (int n = 0; n < KR; ++n) {
      const long long Z = std::llround(std::ldexp(B[(size_t)kk * KR + n], 43 - e));
      const unsigned long long Zp = (unsigned long long)(Z + kOff);
      for (int j = 0; j < kDig; ++j) {
        const int d = (int)((Zp >> (9 * (4 - j))) & 511u) - 256;
        // block j: e_j; block kDig + (4 - j): e_j 2^-9 (j >= 1), exact in FP16
        const int blocks[2] = {j, j >= 1 ? kDig + (4 - j) : -1};
        for (int bi = 0; bi < 2; ++bi) {
          if (blocks[bi] < 0) continue;
          const int nn = blocks[bi] * KR + n;  // column of the side-by-side matrices, K-major core matrices
          const size_t off = (size_t)((kk >> 3) * (kBlk * KR / 8) + (nn >> 3)) * 64 + (nn & 7) * 8 + (kk & 7);
          dig[off] = bi == 0 ? f16_of_int(d) : f16_of_scaled(d, 9);
        }
      }
    }
  return QS_OK;
}

// Launch a prepared block; Bdig (device, 16-byte aligned) holds its digits.
// dfl: the state is in double-float storage (re h, re l, im h, im l per
// amplitude, as complex128 plans hold it) rather than FP64.
qs_status run_dense_tc128_prepared(qs_state* s, const int* q_sorted, int k, const void* Bdig, int F, bool dfl) {
  const uint4* b = static_cast<const uint4*>(Bdig);
  switch (k) {
    case 4: return launch_c128<4>(s, q_sorted, b, F, dfl);
    case 5: return launch_c128<5>(s, q_sorted, b, F, dfl);
  }
  return fail(QS_EINVAL, "fused_c128: k=%d outside [4, 5]", k);
}

// Dense k-qubit block (complex128, k = 4, 5) on the tensor cores.
qs_status run_dense_tc128(qs_state* s, const int* qubits, int k, const double* M) {
  int q[6], F = 0;
  std::vector<uint16_t> dig;
  qs_status st = tc128_prepare(qubits, k, M, q, dig, &F);
  if (st != QS_OK) return st;
  const size_t bytes = dig.size() * sizeof(uint16_t);
  if ((st = ensure_scratch(s, bytes)) != QS_OK) return st;
  cudaError_t e = cudaMemcpyAsync(s->scratch, dig.data(), bytes, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "fused_c128: digit upload");
  return run_dense_tc128_prepared(s, q, k, s->scratch, F, false);
}

// A complex128 tensor-core wait that gave up since the last call: QS_ETIMEOUT (and clear).
qs_status fused_c128_status() {
  int flag = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&flag, g_c128_timeout, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "fused_c128: status read");
  if (!flag) return QS_OK;
  const int zero = 0;
  cudaMemcpyToSymbol(g_c128_timeout, &zero, sizeof(int));
  return fail(QS_ETIMEOUT, "fused_c128: a tensor-core wait gave up; the state is invalid");
}

}  // namespace qs
