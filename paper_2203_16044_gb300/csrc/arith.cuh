// Per-amplitude arithmetic shared by the per-gate and adjoint kernels:
// FP32 for complex64, double-float for complex128 (see dfloat.cuh).
#pragma once

#include "dfloat.cuh"
#include "kcommon.cuh"

namespace qs {

// ---------------------------------------------------------------------------
// Per-amplitude-pair arithmetic: FP32 for complex64, double-float for
// complex128 (values converted from / to FP64 with integer operations).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pair_apply(const M2<float>& U, float& ar, float& ai, float& br, float& bi) {
  mv2(U, ar, ai, br, bi);
}
__device__ __forceinline__ void pair_apply(const M2df& U, double& ar, double& ai, double& br, double& bi) {
  const dfl xr = d2df(ar), xi = d2df(ai), yr = d2df(br), yi = d2df(bi);
  cdf x{xr.h, xr.l, xi.h, xi.l}, y{yr.h, yr.l, yi.h, yi.l};
  mv2df(U, x, y);
  ar = df2d(dfl{x.rh, x.rl});
  ai = df2d(dfl{x.ih, x.il});
  br = df2d(dfl{y.rh, y.rl});
  bi = df2d(dfl{y.ih, y.il});
}

// Complex scalar in the kernel's arithmetic: FP32, or double-float (h, l).
struct Zf { float r, i; };
struct Zdf { float rh, rl, ih, il; };

__device__ __forceinline__ void scal_apply(const Zf& z, float& xr, float& xi) {
  const float r = z.r * xr - z.i * xi;
  xi = z.r * xi + z.i * xr;
  xr = r;
}
__device__ __forceinline__ void scal_apply(const Zdf& z, double& xr, double& xi) {
  const dfl a = d2df(xr), b = d2df(xi);
  cdf x{a.h, a.l, b.h, b.l};
  const float zh[2] = {z.rh, z.ih}, zl[2] = {z.rl, z.il};
  cmul_df(zh, zl, x);
  xr = df2d(dfl{x.rh, x.rl});
  xi = df2d(dfl{x.ih, x.il});
}

template <typename R> struct Ar;
template <> struct Ar<float> { typedef M2<float> Mat; typedef Zf Z; };
template <> struct Ar<double> { typedef M2df Mat; typedef Zdf Z; };

inline Ar<float>::Mat to_mat(const double U[8], float) {
  M2<float> m;
  for (int i = 0; i < 8; ++i) m.m[i] = (float)U[i];
  return m;
}
inline Ar<double>::Mat to_mat(const double U[8], double) {
  M2df m;
  for (int i = 0; i < 8; ++i) {
    m.h[i] = (float)U[i];
    m.l[i] = (float)(U[i] - (double)m.h[i]);
  }
  return m;
}
inline Zf to_z(double re, double im, float) { return Zf{(float)re, (float)im}; }
inline Zdf to_z(double re, double im, double) {
  const float rh = (float)re, ih = (float)im;
  return Zdf{rh, (float)(re - (double)rh), ih, (float)(im - (double)ih)};
}

}  // namespace qs
