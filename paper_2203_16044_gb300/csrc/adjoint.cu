// Adjoint-method gradient of an expectation value.
//
// The paper has no differentiation; this is the standard reverse sweep for
// E(theta) = <psi(theta)|H|psi(theta)>, psi(theta) = U_L ... U_1 |0...0>,
// whose trainable gates are R_P(t) = exp(-i t P / 2), P in {X, Y, Z}:
//   forward:  psi = U_L ... U_1 |0>        (a compiled tile plan)
//             lambda = H psi               (k_pauli_apply, one pass per X/Y mask)
//             E = Re <psi|lambda>
//   reverse:  for l = L .. 1
//               if gate l is R_P(theta_j):  g_j += Im <lambda|P_q|psi>
//               psi <- U_l^dagger psi ;  lambda <- U_l^dagger lambda
// (dE/dt = 2 Re <lambda_l| (-i P/2) |psi_l> = Im <lambda_l|P|psi_l> with
// psi_l, lambda_l the states right after gate l.)
//
// One-qubit steps run as one fused kernel (k_adj_1q): it reads the pair
// (psi_x0, psi_x1) and (lambda_x0, lambda_x1) once, accumulates the
// gradient term in FP64 (per-CTA partials, summed in a fixed order), and
// writes back U^dagger applied to both -- one pass over two vectors instead of
// three.  Two-qubit gates (CNOT, CZ, CP, SWAP) are un-applied with the
// per-gate kernels.  complex128 uses double-float arithmetic, complex64 FP32;
// gradients accumulate in FP64 for both.
#include <cmath>
#include <cstring>
#include <vector>

#include "arith.cuh"
#include "pauli.cuh"
#include "planner.h"

namespace qs {
namespace {

constexpr int kAT = 256;

__device__ __forceinline__ double a_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double a_block_sum(double a) {
  __shared__ double sa[kAT / 32];
  a = a_warp_sum(a);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sa[w] = a;
  __syncthreads();
  if (w == 0) {
    a = l < kAT / 32 ? sa[l] : 0.0;
    a = a_warp_sum(a);
  }
  return a;
}

// gen: 0 none, 1 X, 2 Y, 3 Z (the generator of the trainable gate).
template <typename R>
__global__ void __launch_bounds__(kAT) k_adj_1q(R* __restrict__ psi, R* __restrict__ lam, u64 npairs, int q,
                                                typename Ar<R>::Mat Udag, int gen, double* part) {
  const u64 lo_mask = (u64(1) << q) - 1;
  double g = 0.0;
  for (u64 i = (u64)blockIdx.x * kAT + threadIdx.x; i < npairs; i += (u64)gridDim.x * kAT) {
    const u64 x0 = ((i & ~lo_mask) << 1) | (i & lo_mask);
    const u64 x1 = x0 | (lo_mask + 1);
    R p0r = psi[2 * x0], p0i = psi[2 * x0 + 1], p1r = psi[2 * x1], p1i = psi[2 * x1 + 1];
    R l0r = lam[2 * x0], l0i = lam[2 * x0 + 1], l1r = lam[2 * x1], l1i = lam[2 * x1 + 1];
    if (gen) {
      // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
      const double a0r = l0r, a0i = l0i, a1r = l1r, a1i = l1i;
      const double b0r = p0r, b0i = p0i, b1r = p1r, b1i = p1i;
      if (gen == 1) {         // Im(conj(l0) p1 + conj(l1) p0)
        g += (a0r * b1i - a0i * b1r) + (a1r * b0i - a1i * b0r);
      } else if (gen == 2) {  // Im(-i conj(l0) p1 + i conj(l1) p0) = -Re(conj(l0) p1) + Re(conj(l1) p0)
        g += -(a0r * b1r + a0i * b1i) + (a1r * b0r + a1i * b0i);
      } else {                // Im(conj(l0) p0 - conj(l1) p1)
        g += (a0r * b0i - a0i * b0r) - (a1r * b1i - a1i * b1r);
      }
    }
    pair_apply(Udag, p0r, p0i, p1r, p1i);
    pair_apply(Udag, l0r, l0i, l1r, l1i);
    psi[2 * x0] = p0r; psi[2 * x0 + 1] = p0i; psi[2 * x1] = p1r; psi[2 * x1 + 1] = p1i;
    lam[2 * x0] = l0r; lam[2 * x0 + 1] = l0i; lam[2 * x1] = l1r; lam[2 * x1 + 1] = l1i;
  }
  if (gen) {
    g = a_block_sum(g);
    if (threadIdx.x == 0) part[blockIdx.x] = g;
  }
}

// out (=, or += if accumulate) f(x ^ m) psi_{x ^ m} for one Pauli group.
template <typename R>
__global__ void __launch_bounds__(kAT) k_pauli_apply(const R* __restrict__ psi, R* __restrict__ out, u64 N,
                                                     const __grid_constant__ PauliGroup g, int accumulate) {
  for (u64 x = (u64)blockIdx.x * kAT + threadIdx.x; x < N; x += (u64)gridDim.x * kAT) {
    const u64 y = x ^ g.m;
    double fr, fi;
    fval(g, y, fr, fi);
    const double yr = psi[2 * y], yi = psi[2 * y + 1];
    double r = fr * yr - fi * yi, im = fr * yi + fi * yr;
    if (accumulate) {
      r += (double)out[2 * x];
      im += (double)out[2 * x + 1];
    }
    out[2 * x] = (R)r;
    out[2 * x + 1] = (R)im;
  }
}

// out[s] = sum_{b < G} part[s * G + b], in order (one CTA per slot).
__global__ void __launch_bounds__(kAT) k_slot_sums(const double* part, int G, double* out) {
  double s = 0.0;
  const double* p = part + (size_t)blockIdx.x * G;
  for (int i = threadIdx.x; i < G; i += kAT) s += p[i];
  s = a_block_sum(s);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

unsigned adj_grid(u64 work) {
  const u64 per = (u64)kAT * 4;
  u64 g = (work + per - 1) / per;
  const u64 cap = (u64)sm_count() * 8;
  if (g > cap) g = cap;
  return (unsigned)(g ? g : 1);
}

// conjugate transpose of a 2x2 matrix
void dagger2(const double* m, double* d) {
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      d[2 * (r * 2 + c)] = m[2 * (c * 2 + r)];
      d[2 * (r * 2 + c) + 1] = -m[2 * (c * 2 + r) + 1];
    }
}

template <typename R>
qs_status adj_step_1q(qs_state* psi, qs_state* lam, int q, const double* Udag, int gen, double* part) {
  const u64 npairs = u64(1) << (psi->n - 1);
  const unsigned g = adj_grid(npairs);
  k_adj_1q<R><<<g, kAT, 0, psi->stream>>>(static_cast<R*>(psi->amp), static_cast<R*>(lam->amp), npairs, q,
                                          to_mat(Udag, R(0)), gen, part);
  return launch_ok("k_adj_1q");
}

template <typename R>
qs_status pauli_apply(qs_state* psi, qs_state* out, const std::vector<PauliGroup>& groups) {
  const u64 N = u64(1) << psi->n;
  const unsigned g = adj_grid(N);
  for (size_t i = 0; i < groups.size(); ++i) {
    k_pauli_apply<R><<<g, kAT, 0, psi->stream>>>(static_cast<const R*>(psi->amp), static_cast<R*>(out->amp), N,
                                                 groups[i], i > 0 ? 1 : 0);
    qs_status st = launch_ok("k_pauli_apply");
    if (st != QS_OK) return st;
  }
  return QS_OK;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" qs_status qs_adjoint_grad(qs_state* st, const qs_circuit* c, const double* theta, int nparam, int batch,
                                     int nterms, const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                                     double* energy, double* grad) {
  if (!st || !c || !energy || (nparam > 0 && (!theta || !grad)))
    return fail(QS_EINVAL, "qs_adjoint_grad: NULL argument");
  if (nparam < 0 || batch < 1) return fail(QS_EINVAL, "qs_adjoint_grad: nparam >= 0 and batch >= 1 required");
  if (nterms < 1 || nterms > 65536 || !xmask || !zmask || !coeff)
    return fail(QS_EINVAL, "qs_adjoint_grad: need 1 <= nterms <= 65536 and non-NULL term arrays");
  const int n = st->n;
  const uint64_t lim = (1ull << n) - 1;
  for (int t = 0; t < nterms; ++t)
    if ((xmask[t] & ~lim) || (zmask[t] & ~lim)) return fail(QS_EINVAL, "qs_adjoint_grad: term %d acts on a qubit >= n", t);
  int nparam_gates = 0;
  for (size_t i = 0; i < c->gates.size(); ++i) {
    const qs_gate_rec& g = c->gates[i];
    if (g.q[0] >= n || g.q[1] >= n) return fail(QS_EINVAL, "qs_adjoint_grad: gate %zu acts on a qubit >= n", i);
    if (g.param_index >= nparam) return fail(QS_EINVAL, "qs_adjoint_grad: gate %zu uses parameter %d >= nparam", i, g.param_index);
    if (g.param_index >= 0) ++nparam_gates;
  }
  const std::vector<PauliGroup> groups = build_pauli_groups(nterms, xmask, zmask, coeff);
  const bool c64 = st->dtype == QS_C64;
  const size_t sbytes = state_bytes(st);
  const unsigned G = adj_grid(u64(1) << (n - 1));
  // lambda vector and per-gate gradient partials (stream-ordered allocation)
  void* lam_buf = nullptr;
  double* part = nullptr;
  cudaError_t e = cudaMallocAsync(&lam_buf, sbytes, st->stream);
  if (e != cudaSuccess) return fail(QS_ENOMEM, "qs_adjoint_grad: lambda (%zu bytes): %s", sbytes, cudaGetErrorString(e));
  const size_t pbytes = sizeof(double) * ((size_t)G * (nparam_gates + 1) + nparam_gates + 1);
  e = cudaMallocAsync(reinterpret_cast<void**>(&part), pbytes, st->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(lam_buf, st->stream);
    return fail(QS_ENOMEM, "qs_adjoint_grad: partials: %s", cudaGetErrorString(e));
  }
  double* sums = part + (size_t)G * (nparam_gates + 1);
  qs_state lam;
  lam.n = n;
  lam.dtype = st->dtype;
  lam.amp = lam_buf;
  lam.owns = false;
  lam.stream = st->stream;
  lam.device = st->device;
  lam.pinned = st->pinned;
  std::vector<double> hsums(nparam_gates + 1);
  qs_status rc = QS_OK;
  for (int b = 0; b < batch && rc == QS_OK; ++b) {
    const double* th = theta ? theta + (size_t)b * nparam : nullptr;
    // forward with this parameter set
    qs_circuit cb;
    cb.gates = c->gates;
    for (qs_gate_rec& g : cb.gates)
      if (g.param_index >= 0) g.p[0] = th[g.param_index];
    qs_plan* plan = nullptr;
    if ((rc = qs_plan_build(&cb, n, st->dtype, nullptr, &plan)) != QS_OK) break;
    rc = run_set_basis(st, 0);
    if (rc == QS_OK) rc = qs_run_plan(st, plan);
    qs_plan_destroy(plan);
    if (rc != QS_OK) break;
    // lambda = H psi, E = Re <psi|lambda>
    rc = c64 ? pauli_apply<float>(st, &lam, groups) : pauli_apply<double>(st, &lam, groups);
    if (rc != QS_OK) break;
    double ip[2];
    if ((rc = run_inner(st, &lam, ip)) != QS_OK) break;
    energy[b] = ip[0];
    // reverse sweep
    int slot = 0;
    for (int gi = (int)cb.gates.size() - 1; gi >= 0 && rc == QS_OK; --gi) {
      const qs_gate_rec& g = cb.gates[gi];
      double m[32];
      const int nq = gate_matrix(g.kind, g.p, m);
      if (nq == 1) {
        double md[8];
        dagger2(m, md);
        int gen = 0;
        double* pp = part + (size_t)G * nparam_gates;  // unused slot for fixed gates
        if (g.param_index >= 0) {
          gen = g.kind == QS_GATE_RX ? 1 : g.kind == QS_GATE_RY ? 2 : 3;
          pp = part + (size_t)G * slot;
          ++slot;
        }
        rc = c64 ? adj_step_1q<float>(st, &lam, g.q[0], md, gen, pp)
                 : adj_step_1q<double>(st, &lam, g.q[0], md, gen, pp);
      } else if (g.kind == QS_GATE_CNOT) {
        double x[8];
        gate_matrix(QS_GATE_X, nullptr, x);
        rc = run_controlled(st, &g.q[0], 1, g.q[1], x);
        if (rc == QS_OK) rc = run_controlled(&lam, &g.q[0], 1, g.q[1], x);
      } else if (g.kind == QS_GATE_SWAP) {
        rc = run_bitswap(st, &g.q[0], &g.q[1], 1);
        if (rc == QS_OK) rc = run_bitswap(&lam, &g.q[0], &g.q[1], 1);
      } else {  // CZ, CP: conjugate of the diagonal
        double d[8];
        for (int r = 0; r < 4; ++r) {
          d[2 * r] = m[2 * (r * 4 + r)];
          d[2 * r + 1] = -m[2 * (r * 4 + r) + 1];
        }
        rc = run_diag(st, g.q, 2, d);
        if (rc == QS_OK) rc = run_diag(&lam, g.q, 2, d);
      }
    }
    if (rc != QS_OK) break;
    if (nparam_gates > 0) {
      k_slot_sums<<<nparam_gates, kAT, 0, st->stream>>>(part, (int)G, sums);
      if ((rc = launch_ok("k_slot_sums")) != QS_OK) break;
      e = cudaMemcpyAsync(hsums.data(), sums, sizeof(double) * nparam_gates, cudaMemcpyDeviceToHost, st->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st->stream);
      if (e != cudaSuccess) { rc = cuda_fail(e, "qs_adjoint_grad: gradient readback"); break; }
    }
    double* gb = grad + (size_t)b * nparam;
    for (int j = 0; j < nparam; ++j) gb[j] = 0.0;
    slot = 0;
    for (int gi = (int)cb.gates.size() - 1; gi >= 0; --gi)
      if (cb.gates[gi].param_index >= 0) gb[cb.gates[gi].param_index] += hsums[slot++];
  }
  cudaFreeAsync(part, st->stream);
  cudaFreeAsync(lam_buf, st->stream);
  if (rc == QS_OK) {
    e = cudaStreamSynchronize(st->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "qs_adjoint_grad: sync");
  }
  return rc;
}
