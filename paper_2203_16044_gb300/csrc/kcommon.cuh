// Device-side helpers shared by the libqs kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "qs_internal.h"

namespace qs {

// A "packet" is one 16-byte (128-bit) access: one complex128 amplitude or two
// consecutive complex64 amplitudes.  Every kernel moves state data in packets
// so that each warp access is a fully used, coalesced 512-byte transaction.
template <typename R>
struct PK {
  static constexpr int V = 16 / sizeof(R);  // reals per packet
  static constexpr int A = V / 2;           // amplitudes per packet
  static constexpr int LA = (A == 2) ? 1 : 0;  // log2(A)
};

__device__ __forceinline__ void ld16(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld16(const double* p, double (&v)[2]) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void st16(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st16(double* p, const double (&v)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

// Ascending insertion sort of a few ints under `less` (host; qubit lists).
template <typename Less>
inline void small_sort(int* a, int k, Less less) {
  for (int i = 1; i < k; ++i) {
    const int v = a[i];
    int j = i;
    for (; j > 0 && less(v, a[j - 1]); --j) a[j] = a[j - 1];
    a[j] = v;
  }
}

// Bit insertion: positions sorted ascending, each inserted as a 0 into the
// compact counter i; `set` then ORs the bits that must be 1.
struct Ins {
  int k;
  int pos[12];
  u64 set;
};

__host__ __device__ __forceinline__ u64 expand(u64 i, const Ins& ins) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int j = 0; j < 12; ++j) {
    if (j < ins.k) {
      const u64 lo = i & ((u64(1) << ins.pos[j]) - 1);
      i = ((i ^ lo) << 1) | lo;
    }
  }
  return i | ins.set;
}

// 2x2 complex matrix in the kernel's real type: m00 m01 m10 m11, (re, im).
template <typename R>
struct M2 {
  R m[8];
};

template <typename R>
__device__ __forceinline__ void mv2(const M2<R>& U, R& ar, R& ai, R& br, R& bi) {
  const R xr = U.m[0] * ar - U.m[1] * ai + U.m[2] * br - U.m[3] * bi;
  const R xi = U.m[0] * ai + U.m[1] * ar + U.m[2] * bi + U.m[3] * br;
  const R yr = U.m[4] * ar - U.m[5] * ai + U.m[6] * br - U.m[7] * bi;
  const R yi = U.m[4] * ai + U.m[5] * ar + U.m[6] * bi + U.m[7] * br;
  ar = xr; ai = xi; br = yr; bi = yi;
}

// Grid for a grid-stride kernel: enough CTAs to cover `work` items at
// `per_cta` items each, capped at `waves` CTAs per SM.
inline unsigned grid_for(u64 work, u64 per_cta, int waves) {
  const u64 need = (work + per_cta - 1) / per_cta;
  const u64 cap = (u64)sm_count() * waves;
  return (unsigned)(need < cap ? (need ? need : 1) : cap);
}

}  // namespace qs
