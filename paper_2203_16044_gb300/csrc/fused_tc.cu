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
  FusedArgs A{};
  std::vector<std::pair<int, int>> bits;
  for (int i = 0; i < k; ++i) bits.push_back({qubits[i], 0});
  std::sort(bits.begin(), bits.end());
  A.ins.k = k;
  A.ins.set = 0;
  for (int i = 0; i < k; ++i) A.ins.pos[i] = bits[i].first;
  for (int r = 0; r < D; ++r) {
    u64 sp = 0;
    for (int i = 0; i < k; ++i)
      if ((r >> i) & 1) sp |= u64(1) << qubits[i];
    A.spread[r] = sp;
  }
  // real form of M: B[2c + u][2r + w]
  std::vector<float> B((size_t)KR * KR);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      const double mr = M[2 * (r * D + c)], mi = M[2 * (r * D + c) + 1];
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
    case 4: return launch<4>(s, A, Bd, unitary);
    case 5: return launch<5>(s, A, Bd, unitary);
    case 6: return launch<6>(s, A, Bd, unitary);
  }
  return fail(QS_EINVAL, "fused_tc: k=%d outside [4, 6]", k);
}

}  // namespace qs
