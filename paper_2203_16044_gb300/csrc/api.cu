// C ABI of libqs: argument validation, state lifetime, dispatch to kernels.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "qs_internal.h"
#include "planner.h"

namespace qs {

static thread_local char g_err[512] = "";

qs_status fail(qs_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

qs_status cuda_fail(cudaError_t e, const char* what) {
  return fail(QS_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

qs_status launch_ok(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QS_OK : cuda_fail(e, what);
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cached[dev] = v;
  }
  return cached[dev];
}

qs_status ensure_scratch(qs_state* s, size_t bytes) {
  if (s->scratch_bytes >= bytes) return QS_OK;
  size_t want = bytes < 4096 ? 4096 : bytes;
  if (s->scratch) {
    cudaError_t e = cudaFreeAsync(s->scratch, s->stream);
    s->scratch = nullptr;
    s->scratch_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e, "scratch free");
  }
  cudaError_t e = cudaMallocAsync(&s->scratch, want, s->stream);
  if (e != cudaSuccess) {
    s->scratch = nullptr;
    return fail(QS_ENOMEM, "scratch allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  s->scratch_bytes = want;
  return QS_OK;
}

}  // namespace qs

using namespace qs;

#define CHECK_STATE(s)                                                        \
  do {                                                                        \
    if (!(s)) return fail(QS_EINVAL, "%s: state is NULL", __func__);          \
  } while (0)

static bool distinct(const int* q, int k, int n) {
  for (int i = 0; i < k; ++i) {
    if (q[i] < 0 || q[i] >= n) return false;
    for (int j = 0; j < i; ++j)
      if (q[i] == q[j]) return false;
  }
  return true;
}

static qs_status make_state(int n, qs_dtype dt, void* ptr, bool owns, qs_state** out) {
  qs_state* s = new (std::nothrow) qs_state();
  if (!s) return fail(QS_ENOMEM, "host allocation failed");
  s->n = n;
  s->dtype = dt;
  s->amp = ptr;
  s->owns = owns;
  s->stream = nullptr;
  cudaGetDevice(&s->device);
  cudaError_t e = cudaMallocHost(&s->pinned, 64);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "pinned result buffer");
  }
  *out = s;
  return QS_OK;
}

extern "C" {

const char* qs_last_error(void) { return g_err; }
const char* qs_version(void) { return "qs-gb300 0.1 (sm_103a)"; }

qs_status qs_alloc(int n, qs_dtype dtype, qs_state** out) {
  if (!out) return fail(QS_EINVAL, "qs_alloc: out is NULL");
  *out = nullptr;
  if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "qs_alloc: n=%d outside [1, %d]", n, QS_MAX_QUBITS);
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "qs_alloc: bad dtype %d", (int)dtype);
  const size_t bytes = (size_t(1) << n) * amp_bytes(dtype);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(QS_ENOMEM, "qs_alloc: %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  qs_state* s = nullptr;
  qs_status st = make_state(n, dtype, p, true, &s);
  if (st != QS_OK) {
    cudaFree(p);
    return st;
  }
  st = run_set_basis(s, 0);
  if (st != QS_OK) {
    qs_free(s);
    return st;
  }
  *out = s;
  return QS_OK;
}

qs_status qs_wrap(int n, qs_dtype dtype, void* dev_ptr, qs_state** out) {
  if (!out) return fail(QS_EINVAL, "qs_wrap: out is NULL");
  *out = nullptr;
  if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "qs_wrap: n=%d outside [1, %d]", n, QS_MAX_QUBITS);
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "qs_wrap: bad dtype %d", (int)dtype);
  if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 15))
    return fail(QS_EINVAL, "qs_wrap: device pointer must be non-NULL and 16-byte aligned");
  return make_state(n, dtype, dev_ptr, false, out);
}

qs_status qs_free(qs_state* s) {
  if (!s) return QS_OK;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (s->scratch) cudaFree(s->scratch);
  if (s->owns && s->amp) cudaFree(s->amp);
  if (s->pinned) cudaFreeHost(s->pinned);
  delete s;
  return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_free: pending device error");
}

qs_status qs_set_stream(qs_state* s, void* stream) {
  CHECK_STATE(s);
  if (s->stream != static_cast<cudaStream_t>(stream)) {
    // keep scratch reuse ordered: finish the old stream's work first
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "qs_set_stream: sync old stream");
  }
  s->stream = static_cast<cudaStream_t>(stream);
  return QS_OK;
}

qs_status qs_sync(qs_state* s) {
  CHECK_STATE(s);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qs_sync");
  const qs_status r64 = fused_tc_status();
  const qs_status r128 = fused_c128_status();
  return r64 != QS_OK ? r64 : r128;
}

qs_status qs_data(qs_state* s, void** dev_ptr, size_t* bytes) {
  CHECK_STATE(s);
  if (dev_ptr) *dev_ptr = s->amp;
  if (bytes) *bytes = state_bytes(s);
  return QS_OK;
}

qs_status qs_set_basis(qs_state* s, uint64_t x) {
  CHECK_STATE(s);
  if (x >> s->n) return fail(QS_EINVAL, "qs_set_basis: x=%llu >= 2^%d", (unsigned long long)x, s->n);
  return run_set_basis(s, x);
}

qs_status qs_copy_to_host(qs_state* s, void* dst) {
  CHECK_STATE(s);
  if (!dst) return fail(QS_EINVAL, "qs_copy_to_host: dst is NULL");
  cudaError_t e = cudaMemcpyAsync(dst, s->amp, state_bytes(s), cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qs_copy_to_host");
  e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_copy_to_host: sync");
}

qs_status qs_copy_from_host(qs_state* s, const void* src) {
  CHECK_STATE(s);
  if (!src) return fail(QS_EINVAL, "qs_copy_from_host: src is NULL");
  cudaError_t e = cudaMemcpyAsync(s->amp, src, state_bytes(s), cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qs_copy_from_host");
  e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_copy_from_host: sync");
}

qs_status qs_copy_from_host_async(qs_state* s, const void* src) {
  CHECK_STATE(s);
  if (!src) return fail(QS_EINVAL, "qs_copy_from_host_async: src is NULL");
  const cudaError_t e = cudaMemcpyAsync(s->amp, src, state_bytes(s), cudaMemcpyHostToDevice, s->stream);
  return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_copy_from_host_async");
}

qs_status qs_apply_1q(qs_state* s, int q, const double U[8]) {
  CHECK_STATE(s);
  if (!U) return fail(QS_EINVAL, "qs_apply_1q: U is NULL");
  if (q < 0 || q >= s->n) return fail(QS_EINVAL, "qs_apply_1q: qubit %d outside [0, %d)", q, s->n);
  return run_1q(s, q, U);
}

qs_status qs_apply_controlled(qs_state* s, const int* controls, int nc, int target, const double U[8]) {
  CHECK_STATE(s);
  if (!U) return fail(QS_EINVAL, "qs_apply_controlled: U is NULL");
  if (nc < 0 || nc > 8 || (nc > 0 && !controls))
    return fail(QS_EINVAL, "qs_apply_controlled: nc=%d (0..8, controls non-NULL)", nc);
  int q[9];
  for (int i = 0; i < nc; ++i) q[i] = controls[i];
  q[nc] = target;
  if (nc + 1 > s->n || !distinct(q, nc + 1, s->n))
    return fail(QS_EINVAL, "qs_apply_controlled: qubits must be distinct and in [0, %d)", s->n);
  return run_controlled(s, controls, nc, target, U);
}

qs_status qs_apply_diag(qs_state* s, const int* qubits, int k, const double* d) {
  CHECK_STATE(s);
  if (!qubits || !d || k < 1 || k > 8 || k > s->n)
    return fail(QS_EINVAL, "qs_apply_diag: need 1 <= k <= min(8, n) and non-NULL arrays (k=%d)", k);
  if (!distinct(qubits, k, s->n)) return fail(QS_EINVAL, "qs_apply_diag: qubits must be distinct and in range");
  return run_diag(s, qubits, k, d);
}

qs_status qs_apply_fused(qs_state* s, const int* qubits, int k, const double* M) {
  CHECK_STATE(s);
  if (!qubits || !M || k < 1 || k > 6 || k > s->n)
    return fail(QS_EINVAL, "qs_apply_fused: need 1 <= k <= min(6, n) and non-NULL arrays (k=%d)", k);
  if (!distinct(qubits, k, s->n)) return fail(QS_EINVAL, "qs_apply_fused: qubits must be distinct and in range");
  return run_dense(s, qubits, k, M);
}

qs_status qs_fused_swap(qs_state* s, int p, int q, int sw) {
  CHECK_STATE(s);
  if (sw < 0 || p < 0 || q < 0 || p + sw > s->n || q + sw > s->n)
    return fail(QS_EINVAL, "qs_fused_swap: ranges [%d,%d) and [%d,%d) outside [0, %d)", p, p + sw, q, q + sw, s->n);
  if (sw > 0 && !(p + sw <= q || q + sw <= p))
    return fail(QS_EINVAL, "qs_fused_swap: ranges [%d,%d) and [%d,%d) overlap", p, p + sw, q, q + sw);
  if (sw == 0 || p == q) return QS_OK;
  std::vector<int> a(sw), b(sw);
  for (int i = 0; i < sw; ++i) {
    a[i] = p + i;
    b[i] = q + i;
  }
  return run_bitswap(s, a.data(), b.data(), sw);
}

qs_status qs_permute_qubits(qs_state* s, const int* perm) {
  CHECK_STATE(s);
  if (!perm) return fail(QS_EINVAL, "qs_permute_qubits: perm is NULL");
  const int n = s->n;
  std::vector<int> seen(n, 0);
  for (int j = 0; j < n; ++j) {
    if (perm[j] < 0 || perm[j] >= n || seen[perm[j]])
      return fail(QS_EINVAL, "qs_permute_qubits: not a permutation of 0..%d", n - 1);
    seen[perm[j]] = 1;
  }
  // at most two passes of disjoint bit-pair exchanges (17 pairs per pass)
  for (const auto& pass : permutation_passes(std::vector<int>(perm, perm + n), 17)) {
    int a[17], b[17];
    for (size_t i = 0; i < pass.size(); ++i) {
      a[i] = pass[i].first;
      b[i] = pass[i].second;
    }
    qs_status st = run_bitswap(s, a, b, (int)pass.size());
    if (st != QS_OK) return st;
  }
  return QS_OK;
}

qs_status qs_norm2(qs_state* s, double* out) {
  CHECK_STATE(s);
  if (!out) return fail(QS_EINVAL, "qs_norm2: out is NULL");
  return run_norm2(s, out);
}

qs_status qs_inner(qs_state* a, qs_state* b, double out[2]) {
  if (!a || !b || !out) return fail(QS_EINVAL, "qs_inner: NULL argument");
  if (a->n != b->n || a->dtype != b->dtype) return fail(QS_EINVAL, "qs_inner: states differ in n or dtype");
  return run_inner(a, b, out);
}

qs_status qs_expect_pauli(qs_state* s, int nterms, const uint64_t* xmask, const uint64_t* zmask,
                          const double* coeff, double* out) {
  CHECK_STATE(s);
  if (nterms < 1 || nterms > 65536 || !xmask || !zmask || !coeff || !out)
    return fail(QS_EINVAL, "qs_expect_pauli: need 1 <= nterms <= 65536 and non-NULL arrays");
  const uint64_t lim = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
  for (int t = 0; t < nterms; ++t)
    if ((xmask[t] & ~lim) || (zmask[t] & ~lim))
      return fail(QS_EINVAL, "qs_expect_pauli: term %d acts on a qubit >= n", t);
  return run_expect(s, nterms, xmask, zmask, coeff, out);
}

qs_status qs_expect_pauli_passes(int n, qs_dtype dtype, int nterms, const uint64_t* xmask, const uint64_t* zmask,
                                 int* passes) {
  if (n < 1 || n > 34 || (dtype != QS_C64 && dtype != QS_C128))
    return fail(QS_EINVAL, "qs_expect_pauli_passes: need 1 <= n <= 34 and a known dtype");
  if (nterms < 1 || nterms > 65536 || !xmask || !zmask || !passes)
    return fail(QS_EINVAL, "qs_expect_pauli_passes: need 1 <= nterms <= 65536 and non-NULL arrays");
  const uint64_t lim = (1ull << n) - 1;
  for (int t = 0; t < nterms; ++t)
    if ((xmask[t] & ~lim) || (zmask[t] & ~lim))
      return fail(QS_EINVAL, "qs_expect_pauli_passes: term %d acts on a qubit >= n", t);
  return expect_pauli_passes(n, (int)dtype, nterms, xmask, zmask, passes);
}

}  // extern "C"
