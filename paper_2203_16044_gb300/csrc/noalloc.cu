// qs_inner_noalloc: the inner product <a|b> with no allocation at all.
//
// Some callers cannot let a library allocate device memory: a framework
// whose caching allocator has already reserved the GPU's memory (a library
// cudaMalloc then fails or fragments the pool), code on a latency-critical
// loop where cudaMalloc / cudaFree would synchronise the device, or hosts
// whose memory policy forbids allocations outside their own allocator.
// qs_inner (reduce.cu) grows a per-state scratch buffer for its per-CTA
// partial sums and needs a qs_state handle (which holds a pinned host word);
// this variant takes plain device pointers and keeps its partial sums in the
// fixed array below instead.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds it (16 KiB + 16 B) until the process exits.  Host code must
// not pass the array's name to a kernel -- on the host that name is only a
// stand-in, not a device address -- so the first call on each device looks
// up the device address with cudaGetSymbolAddress (with that device current)
// and caches it once the lookup has succeeded (a failed lookup is retried by
// the next call).  That first call therefore does a little set-up work; make
// it before any stream capture begins.
//
// Every call shares the one array and the last call's partial sums stay in
// it.  Nothing has to start at zero: each CTA overwrites its own partial
// before the final pass reads exactly those partials.  Calls whose work
// overlaps on the GPU (different streams, or different host threads, on the
// same device) race on the array: serialise them.
#include <atomic>
#include <mutex>

#include "kcommon.cuh"

namespace {

constexpr int kNaThreads = 256;
// Largest number of per-CTA partial sums the static scratch holds.
constexpr int kNaMaxPartials = 1024;
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double2 g_inner_scratch[kNaMaxPartials + 1];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void na_block_sum2(double& a, double& b) {
  __shared__ double sa[kNaThreads / 32], sb[kNaThreads / 32];
  a = na_warp_sum(a);
  b = na_warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (w == 0) {
    a = l < kNaThreads / 32 ? sa[l] : 0.0;
    b = l < kNaThreads / 32 ? sb[l] : 0.0;
    a = na_warp_sum(a);
    b = na_warp_sum(b);
  }
}

// Per-CTA partial of sum_x conj(a_x) b_x over a grid-stride range of packets.
template <typename R>
__global__ void __launch_bounds__(kNaThreads) k_inner_static(const R* __restrict__ a, const R* __restrict__ b,
                                                             u64 npk, double2* part) {
  constexpr int V = qs::PK<R>::V;
  double sr = 0.0, si = 0.0;
  for (u64 p = (u64)blockIdx.x * kNaThreads + threadIdx.x; p < npk; p += (u64)gridDim.x * kNaThreads) {
    R va[V], vb[V];
    qs::ld16(a + p * V, va);
    qs::ld16(b + p * V, vb);
#pragma unroll
    for (int c = 0; c < V; c += 2) {
      const double ar = va[c], ai = va[c + 1], br = vb[c], bi = vb[c + 1];
      sr += ar * br + ai * bi;
      si += ar * bi - ai * br;
    }
  }
  na_block_sum2(sr, si);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sr, si);
}

// Sums part[0..n) in a fixed order into *out.
__global__ void __launch_bounds__(kNaThreads) k_inner_static_final(const double2* part, int n, double2* out) {
  double sr = 0.0, si = 0.0;
  for (int i = threadIdx.x; i < n; i += kNaThreads) {
    sr += part[i].x;
    si += part[i].y;
  }
  na_block_sum2(sr, si);
  if (threadIdx.x == 0) *out = make_double2(sr, si);
}

// Device address of g_inner_scratch per device, set once a lookup succeeds.
std::atomic<double2*> g_scratch_ptr[kNaMaxDevices];
std::mutex g_scratch_mu;

// The scratch array's device address on `dev` (the current device).
cudaError_t scratch_address(int dev, double2** out) {
  double2* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (p) {
    *out = p;
    return cudaSuccess;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  p = g_scratch_ptr[dev].load(std::memory_order_relaxed);
  if (!p) {
    const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_inner_scratch);
    if (e != cudaSuccess || !p) return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    g_scratch_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" qs_status qs_inner_noalloc(const void* a, const void* b, int n, qs_dtype dtype, void* stream,
                                      double out[2]) {
  using namespace qs;
  if (!a || !b || !out) return fail(QS_EINVAL, "qs_inner_noalloc: NULL argument");
  if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15)
    return fail(QS_EINVAL, "qs_inner_noalloc: device pointers must be 16-byte aligned");
  if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "qs_inner_noalloc: n=%d outside [1, %d]", n, QS_MAX_QUBITS);
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "qs_inner_noalloc: bad dtype %d", (int)dtype);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "qs_inner_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kNaMaxDevices) return fail(QS_EUNSUPPORTED, "qs_inner_noalloc: device %d >= %d", dev, kNaMaxDevices);
  double2* scratch = nullptr;
  e = scratch_address(dev, &scratch);
  if (e != cudaSuccess) return cuda_fail(e, "qs_inner_noalloc: cudaGetSymbolAddress");
  const int LA = dtype == QS_C64 ? 1 : 0;
  const u64 npk = u64(1) << (n - LA);
  // Same grid rule as qs_inner: at most 4 CTAs per SM, 2048 packets per CTA.
  const u64 per = (u64)kNaThreads * 8;
  u64 grid = (npk + per - 1) / per;
  const u64 cap = (u64)sm_count() * 4;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  if (grid > (u64)kNaMaxPartials)
    return fail(QS_EUNSUPPORTED, "qs_inner_noalloc: needs %llu partial sums, the static scratch holds %d",
                (unsigned long long)grid, kNaMaxPartials);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double2* part = scratch;
  double2* res = scratch + kNaMaxPartials;
  if (dtype == QS_C64)
    k_inner_static<float><<<(unsigned)grid, kNaThreads, 0, s>>>(static_cast<const float*>(a), static_cast<const float*>(b), npk, part);
  else
    k_inner_static<double><<<(unsigned)grid, kNaThreads, 0, s>>>(static_cast<const double*>(a), static_cast<const double*>(b), npk, part);
  qs_status st = launch_ok("qs_inner_noalloc: k_inner_static");
  if (st != QS_OK) return st;
  k_inner_static_final<<<1, kNaThreads, 0, s>>>(part, (int)grid, res);
  if ((st = launch_ok("qs_inner_noalloc: k_inner_static_final")) != QS_OK) return st;
  e = cudaMemcpyAsync(out, res, sizeof(double2), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "qs_inner_noalloc: result copy");
  e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_inner_noalloc: sync");
}
