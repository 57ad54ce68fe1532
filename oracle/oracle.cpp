// Plain FP64 CPU oracle for state-vector gate application.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
// call this file: only tests/, the package smoke check and the CPU-baseline
// leg of the benchmark use it.  It shares no code with the CUDA library.
//
// Everything here is the plain definition, written out with
// std::complex<double> and one sequential loop per operation; the only
// parallelism is an OpenMP "parallel for" over loop iterations that write
// disjoint amplitudes, so results do not depend on the thread count.
// Reductions use a fixed chunking (partials of 4096 amplitudes, summed in
// index order), also independent of the thread count.
//
// State layout (§II-A, Eq. 2): amplitude a_x of basis state |x> at index x,
// bit q of x is qubit q (qubit 0 least significant); 2^n complex doubles,
// 2^(n+4) bytes, interleaved (re, im) -- the numpy complex128 layout.
//
// Matrix conventions: a 2x2 matrix is 8 doubles, row-major, (re, im) per
// entry.  A k-qubit matrix over qubits[0..k-1] is 2^k x 2^k row-major; bit i
// of its row/column index r corresponds to qubits[i].
//
// Parity status of each function is recorded in the test suite: every
// function below is pinned by tests that do not reuse it (Kronecker-product
// brute force, closed forms, identities); none is "parity unpinned".

#include <algorithm>
#include <complex>
#include <cstdint>
#include <cstring>
#include <cmath>
#include <vector>

typedef std::complex<double> cplx;
typedef uint64_t u64;
typedef long long i64;

static inline cplx* as_c(double* p) { return reinterpret_cast<cplx*>(p); }
static inline const cplx* as_c(const double* p) { return reinterpret_cast<const cplx*>(p); }

// Gate kinds understood by or_gate_matrix / or_run_circuit (the oracle's own
// numbering; the Python wrapper maps gate names onto it).
enum {
  OR_H = 0, OR_X, OR_Y, OR_Z, OR_S, OR_T, OR_RX, OR_RY, OR_RZ, OR_P, OR_U3,
  OR_CNOT = 16, OR_CZ, OR_CP, OR_SWAP
};

extern "C" {

// ---------------------------------------------------------------------------
// One-qubit gate, Eq. (4) of §II-A: for every x with bit q clear and
// y = x | 2^q, (a_x, a_y) <- U (a_x, a_y).
// ---------------------------------------------------------------------------
void or_apply_1q(double* state, int n, int q, const double* U) {
  cplx* a = as_c(state);
  const u64 N = 1ull << n, bit = 1ull << q;
  const cplx u00(U[0], U[1]), u01(U[2], U[3]), u10(U[4], U[5]), u11(U[6], U[7]);
#pragma omp parallel for schedule(static)
  for (i64 xi = 0; xi < (i64)N; ++xi) {
    const u64 x = (u64)xi;
    if (x & bit) continue;
    const u64 y = x | bit;
    const cplx ax = a[x], ay = a[y];
    a[x] = u00 * ax + u01 * ay;
    a[y] = u10 * ax + u11 * ay;
  }
}

// ---------------------------------------------------------------------------
// Controlled one-qubit gate: Eq. (4) restricted to the indices whose control
// bits are all 1 (the CNOT layers of §IV-F are the case U = X, one control).
// ---------------------------------------------------------------------------
void or_apply_controlled(double* state, int n, const int* ctrl, int nc, int t,
                         const double* U) {
  cplx* a = as_c(state);
  const u64 N = 1ull << n, bit = 1ull << t;
  u64 cmask = 0;
  for (int i = 0; i < nc; ++i) cmask |= 1ull << ctrl[i];
  const cplx u00(U[0], U[1]), u01(U[2], U[3]), u10(U[4], U[5]), u11(U[6], U[7]);
#pragma omp parallel for schedule(static)
  for (i64 xi = 0; xi < (i64)N; ++xi) {
    const u64 x = (u64)xi;
    if (x & bit) continue;
    if ((x & cmask) != cmask) continue;
    const u64 y = x | bit;
    const cplx ax = a[x], ay = a[y];
    a[x] = u00 * ax + u01 * ay;
    a[y] = u10 * ax + u11 * ay;
  }
}

// ---------------------------------------------------------------------------
// Diagonal gate on k qubits: a_x <- d[r(x)] a_x, where bit i of r(x) is bit
// qubits[i] of x.  d holds 2^k complex entries.
// ---------------------------------------------------------------------------
void or_apply_diag(double* state, int n, const int* qubits, int k, const double* d) {
  cplx* a = as_c(state);
  const cplx* dd = as_c(d);
  const u64 N = 1ull << n;
#pragma omp parallel for schedule(static)
  for (i64 xi = 0; xi < (i64)N; ++xi) {
    const u64 x = (u64)xi;
    u64 r = 0;
    for (int i = 0; i < k; ++i) r |= ((x >> qubits[i]) & 1ull) << i;
    a[x] = dd[r] * a[x];
  }
}

// ---------------------------------------------------------------------------
// Dense k-qubit gate: for every base index x with all k bits clear, gather
// v[r] = a[x | spread(r)], set v <- M v, scatter back.
// ---------------------------------------------------------------------------
void or_apply_dense(double* state, int n, const int* qubits, int k, const double* M) {
  cplx* a = as_c(state);
  const cplx* m = as_c(M);
  const u64 N = 1ull << n, D = 1ull << k;
  u64 kmask = 0;
  for (int i = 0; i < k; ++i) kmask |= 1ull << qubits[i];
  std::vector<u64> spread(D);
  for (u64 r = 0; r < D; ++r) {
    u64 s = 0;
    for (int i = 0; i < k; ++i)
      if ((r >> i) & 1ull) s |= 1ull << qubits[i];
    spread[r] = s;
  }
#pragma omp parallel
  {
    std::vector<cplx> v(D), w(D);
#pragma omp for schedule(static)
    for (i64 xi = 0; xi < (i64)N; ++xi) {
      const u64 x = (u64)xi;
      if (x & kmask) continue;
      for (u64 r = 0; r < D; ++r) v[r] = a[x | spread[r]];
      for (u64 r = 0; r < D; ++r) {
        cplx s = 0.0;
        for (u64 c = 0; c < D; ++c) s += m[r * D + c] * v[c];
        w[r] = s;
      }
      for (u64 r = 0; r < D; ++r) a[x | spread[r]] = w[r];
    }
  }
}

// ---------------------------------------------------------------------------
// swap(i, j) of §III-D: exchange a_x and a_x' where x' is x with bits i and j
// exchanged; only indices whose two bits differ move.
// ---------------------------------------------------------------------------
void or_swap(double* state, int n, int i, int j) {
  cplx* a = as_c(state);
  const u64 N = 1ull << n, bi = 1ull << i, bj = 1ull << j;
#pragma omp parallel for schedule(static)
  for (i64 xi = 0; xi < (i64)N; ++xi) {
    const u64 x = (u64)xi;
    if ((x & bi) && !(x & bj)) {
      const u64 y = (x ^ bi) | bj;
      const cplx t = a[x];
      a[x] = a[y];
      a[y] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// fused_swap(p, q, s) of §III-D (Listing 1): the s swaps swap(p+i, q+i),
// i = 0..s-1, applied one after another; the ranges [p, p+s) and [q, q+s)
// must not overlap.  Returns the number of amplitudes whose index the fused
// operation changes (those whose two s-bit fields differ), or -1 on bad
// arguments.
// ---------------------------------------------------------------------------
i64 or_fused_swap(double* state, int n, int p, int q, int s) {
  if (s < 0 || p < 0 || q < 0 || p + s > n || q + s > n) return -1;
  if (!(p + s <= q || q + s <= p)) return -1;
  for (int i = 0; i < s; ++i) or_swap(state, n, p + i, q + i);
  const u64 N = 1ull << n;
  i64 moved = 0;
  for (u64 x = 0; x < N; ++x) {
    const u64 fp = (x >> p) & ((1ull << s) - 1), fq = (x >> q) & ((1ull << s) - 1);
    if (fp != fq) ++moved;
  }
  return moved;
}

// ---------------------------------------------------------------------------
// General qubit permutation: out[pi(x)] = in[x], where pi moves bit j of x to
// bit perm[j].  (A fused swap is the permutation exchanging two disjoint bit
// fields.)  Out of place; perm must be a permutation of 0..n-1.
// ---------------------------------------------------------------------------
int or_permute(const double* in, double* out, int n, const int* perm) {
  std::vector<int> seen(n, 0);
  for (int j = 0; j < n; ++j) {
    if (perm[j] < 0 || perm[j] >= n || seen[perm[j]]) return -1;
    seen[perm[j]] = 1;
  }
  const cplx* a = as_c(in);
  cplx* b = as_c(out);
  const u64 N = 1ull << n;
#pragma omp parallel for schedule(static)
  for (i64 xi = 0; xi < (i64)N; ++xi) {
    const u64 x = (u64)xi;
    u64 y = 0;
    for (int j = 0; j < n; ++j) y |= ((x >> j) & 1ull) << perm[j];
    b[y] = a[x];
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Gate matrices (textbook definitions; the paper does not fix them).
//   H = [[1,1],[1,-1]]/sqrt2, X, Y, Z, S = diag(1,i), T = diag(1,e^{i pi/4}),
//   RX(t) = cos(t/2) I - i sin(t/2) X, RY(t) = cos(t/2) I - i sin(t/2) Y,
//   RZ(t) = diag(e^{-it/2}, e^{it/2}), P(l) = diag(1, e^{il}),
//   U3(t,p,l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]].
// Two-qubit (4x4, bit 0 of the index = qubits[0]):
//   CNOT(control = qubits[0], target = qubits[1]), CZ = diag(1,1,1,-1),
//   CP(l) = diag(1,1,1,e^{il}), SWAP.
// Writes 8 (one-qubit) or 32 (two-qubit) doubles; returns the number of
// qubits, or -1 for an unknown kind.
// ---------------------------------------------------------------------------
int or_gate_matrix(int kind, const double* prm, double* out) {
  const cplx I(0.0, 1.0);
  cplx m[16];
  for (int i = 0; i < 16; ++i) m[i] = 0.0;
  int nq = 1;
  switch (kind) {
    case OR_H: {
      const double r = 1.0 / std::sqrt(2.0);
      m[0] = r; m[1] = r; m[2] = r; m[3] = -r;
    } break;
    case OR_X: m[1] = 1.0; m[2] = 1.0; break;
    case OR_Y: m[1] = -I; m[2] = I; break;
    case OR_Z: m[0] = 1.0; m[3] = -1.0; break;
    case OR_S: m[0] = 1.0; m[3] = I; break;
    case OR_T: m[0] = 1.0; m[3] = std::exp(I * (M_PI / 4.0)); break;
    case OR_RX: {
      const double c = std::cos(prm[0] / 2), s = std::sin(prm[0] / 2);
      m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c;
    } break;
    case OR_RY: {
      const double c = std::cos(prm[0] / 2), s = std::sin(prm[0] / 2);
      m[0] = c; m[1] = -s; m[2] = s; m[3] = c;
    } break;
    case OR_RZ:
      m[0] = std::exp(-I * (prm[0] / 2)); m[3] = std::exp(I * (prm[0] / 2));
      break;
    case OR_P: m[0] = 1.0; m[3] = std::exp(I * prm[0]); break;
    case OR_U3: {
      const double c = std::cos(prm[0] / 2), s = std::sin(prm[0] / 2);
      m[0] = c;
      m[1] = -std::exp(I * prm[2]) * s;
      m[2] = std::exp(I * prm[1]) * s;
      m[3] = std::exp(I * (prm[1] + prm[2])) * c;
    } break;
    case OR_CNOT:
      nq = 2;
      // index r = b0 + 2 b1, b0 = control, b1 = target: flip b1 when b0 = 1.
      m[0 * 4 + 0] = 1.0; m[2 * 4 + 2] = 1.0; m[1 * 4 + 3] = 1.0; m[3 * 4 + 1] = 1.0;
      break;
    case OR_CZ:
      nq = 2; m[0] = 1.0; m[5] = 1.0; m[10] = 1.0; m[15] = -1.0;
      break;
    case OR_CP:
      nq = 2; m[0] = 1.0; m[5] = 1.0; m[10] = 1.0; m[15] = std::exp(I * prm[0]);
      break;
    case OR_SWAP:
      nq = 2; m[0] = 1.0; m[1 * 4 + 2] = 1.0; m[2 * 4 + 1] = 1.0; m[15] = 1.0;
      break;
    default: return -1;
  }
  const int D = 1 << nq;
  for (int i = 0; i < D * D; ++i) {
    out[2 * i] = m[i].real();
    out[2 * i + 1] = m[i].imag();
  }
  return nq;
}

// ---------------------------------------------------------------------------
// Run a circuit, an ordered gate sequence (§II-A), one gate at a time:
// one-qubit gates by Eq. (4), CNOT as controlled X, CZ and CP as diagonal
// gates, SWAP by swap(i, j).  kinds[g], qubits[2g..2g+1], params[3g..3g+2].
// Returns 0, or -1 at the first unknown kind.
// ---------------------------------------------------------------------------
int or_run_circuit(double* state, int n, int ngates, const int* kinds,
                   const int* qubits, const double* params) {
  for (int g = 0; g < ngates; ++g) {
    const int kind = kinds[g];
    const int* q = qubits + 2 * g;
    const double* p = params + 3 * g;
    double m[32];
    const int nq = or_gate_matrix(kind, p, m);
    if (nq < 0) return -1;
    if (nq == 1) {
      or_apply_1q(state, n, q[0], m);
    } else if (kind == OR_CNOT) {
      double x[8];
      or_gate_matrix(OR_X, p, x);
      or_apply_controlled(state, n, &q[0], 1, q[1], x);
    } else if (kind == OR_SWAP) {
      or_swap(state, n, q[0], q[1]);
    } else {  // CZ, CP: the diagonal of the 4x4 matrix
      double d[8];
      for (int r = 0; r < 4; ++r) {
        d[2 * r] = m[2 * (r * 4 + r)];
        d[2 * r + 1] = m[2 * (r * 4 + r) + 1];
      }
      or_apply_diag(state, n, q, 2, d);
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// <a|b> = sum_x conj(a_x) b_x, in fixed-order chunked summation.
// ---------------------------------------------------------------------------
void or_inner(const double* av, const double* bv, int n, double* out) {
  const cplx* a = as_c(av);
  const cplx* b = as_c(bv);
  const u64 N = 1ull << n, CH = 4096;
  const u64 nch = (N + CH - 1) / CH;
  std::vector<cplx> part(nch);
#pragma omp parallel for schedule(static)
  for (i64 c = 0; c < (i64)nch; ++c) {
    cplx s = 0.0;
    const u64 lo = (u64)c * CH, hi = lo + CH < N ? lo + CH : N;
    for (u64 x = lo; x < hi; ++x) s += std::conj(a[x]) * b[x];
    part[c] = s;
  }
  cplx s = 0.0;
  for (u64 c = 0; c < nch; ++c) s += part[c];
  out[0] = s.real();
  out[1] = s.imag();
}

// ---------------------------------------------------------------------------
// Expectation of a weighted sum of Pauli strings, sum_t coeff[t] <psi|P_t|psi>.
// P_t has X on the qubits set only in xmask[t], Z on those only in zmask[t],
// Y on those set in both.  Each term: copy psi, apply its factors as
// one-qubit gates, take the real part of <psi|P psi>.
// ---------------------------------------------------------------------------
double or_expect_pauli(const double* state, int n, int nterms, const u64* xmask,
                       const u64* zmask, const double* coeff) {
  const u64 N = 1ull << n;
  std::vector<double> phi(2 * N);
  double X[8], Y[8], Z[8];
  or_gate_matrix(OR_X, nullptr, X);
  or_gate_matrix(OR_Y, nullptr, Y);
  or_gate_matrix(OR_Z, nullptr, Z);
  double total = 0.0;
  for (int t = 0; t < nterms; ++t) {
    std::memcpy(phi.data(), state, sizeof(double) * 2 * N);
    for (int q = 0; q < n; ++q) {
      const bool x = (xmask[t] >> q) & 1ull, z = (zmask[t] >> q) & 1ull;
      if (x && z) or_apply_1q(phi.data(), n, q, Y);
      else if (x) or_apply_1q(phi.data(), n, q, X);
      else if (z) or_apply_1q(phi.data(), n, q, Z);
    }
    double ip[2];
    or_inner(state, phi.data(), n, ip);
    total += coeff[t] * ip[0];
  }
  return total;
}

// ---------------------------------------------------------------------------
// Apply a weighted sum of Pauli strings to psi: out = sum_t coeff[t] P_t psi.
// Same Pauli convention as or_expect_pauli.
// ---------------------------------------------------------------------------
void or_apply_pauli_sum(const double* state, double* out, int n, int nterms,
                        const u64* xmask, const u64* zmask, const double* coeff) {
  const u64 N = 1ull << n;
  std::vector<double> phi(2 * N);
  double X[8], Y[8], Z[8];
  or_gate_matrix(OR_X, nullptr, X);
  or_gate_matrix(OR_Y, nullptr, Y);
  or_gate_matrix(OR_Z, nullptr, Z);
  std::memset(out, 0, sizeof(double) * 2 * N);
  for (int t = 0; t < nterms; ++t) {
    std::memcpy(phi.data(), state, sizeof(double) * 2 * N);
    for (int q = 0; q < n; ++q) {
      const bool x = (xmask[t] >> q) & 1ull, z = (zmask[t] >> q) & 1ull;
      if (x && z) or_apply_1q(phi.data(), n, q, Y);
      else if (x) or_apply_1q(phi.data(), n, q, X);
      else if (z) or_apply_1q(phi.data(), n, q, Z);
    }
    for (u64 i = 0; i < 2 * N; ++i) out[i] += coeff[t] * phi[i];
  }
}

// ---------------------------------------------------------------------------
// Adjoint-method gradient of E(theta) = <psi(theta)|H|psi(theta)>,
// psi(theta) = U_L ... U_1 |psi0>, for circuits whose parameterised gates are
// RX/RY/RZ(theta_j) = exp(-i theta_j G / 2), G in {X, Y, Z}.  The paper has no
// differentiation; this is the textbook reverse sweep:
//   psi = psi_L, lambda = H psi_L;
//   for l = L .. 1:
//     if gate l is exp(-i t G / 2) with parameter j:
//        grad[j] += 2 Re( <lambda| (-i G / 2) |psi> ) = Im <lambda|G|psi>
//     psi <- U_l^dagger psi;  lambda <- U_l^dagger lambda.
// (dE/dt = 2 Re <psi_L|H dpsi_L/dt>, and dpsi_L/dt = U_L..U_{l+1} (-iG/2) psi_l
// with psi_l the state right after gate l.)
// param_index[g] >= 0 marks a parameterised gate; grad has nparam entries and
// is overwritten.  Returns E, or NaN on an unsupported gate.
// ---------------------------------------------------------------------------
double or_adjoint_grad(const double* psi0, int n, int ngates, const int* kinds,
                       const int* qubits, const double* params, const int* param_index,
                       int nparam, int nterms, const u64* xmask, const u64* zmask,
                       const double* coeff, double* grad) {
  const u64 N = 1ull << n;
  std::vector<double> psi(psi0, psi0 + 2 * N), lam(2 * N), tmp(2 * N);
  if (or_run_circuit(psi.data(), n, ngates, kinds, qubits, params) != 0) return NAN;
  or_apply_pauli_sum(psi.data(), lam.data(), n, nterms, xmask, zmask, coeff);
  double e[2];
  or_inner(psi.data(), lam.data(), n, e);
  for (int j = 0; j < nparam; ++j) grad[j] = 0.0;
  for (int g = ngates - 1; g >= 0; --g) {
    const int kind = kinds[g];
    const int* q = qubits + 2 * g;
    const double* p = params + 3 * g;
    if (param_index[g] >= 0) {
      int gen;
      if (kind == OR_RX) gen = OR_X;
      else if (kind == OR_RY) gen = OR_Y;
      else if (kind == OR_RZ) gen = OR_Z;
      else return NAN;
      double G[8];
      or_gate_matrix(gen, nullptr, G);
      std::memcpy(tmp.data(), psi.data(), sizeof(double) * 2 * N);
      or_apply_1q(tmp.data(), n, q[0], G);
      double ip[2];
      or_inner(lam.data(), tmp.data(), n, ip);
      grad[param_index[g]] += ip[1];
    }
    // Un-apply gate g: U^dagger, from the conjugate transpose of its matrix.
    double m[32];
    const int nq = or_gate_matrix(kind, p, m);
    if (nq < 0) return NAN;
    if (nq == 1) {
      double md[8];
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
          md[2 * (r * 2 + c)] = m[2 * (c * 2 + r)];
          md[2 * (r * 2 + c) + 1] = -m[2 * (c * 2 + r) + 1];
        }
      or_apply_1q(psi.data(), n, q[0], md);
      or_apply_1q(lam.data(), n, q[0], md);
    } else {
      double md[32];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          md[2 * (r * 4 + c)] = m[2 * (c * 4 + r)];
          md[2 * (r * 4 + c) + 1] = -m[2 * (c * 4 + r) + 1];
        }
      or_apply_dense(psi.data(), n, q, 2, md);
      or_apply_dense(lam.data(), n, q, 2, md);
    }
  }
  return e[0];
}

// ---------------------------------------------------------------------------
// Measurement in the computational basis (§II-A: a circuit is a sequence of
// gates, measurements and resets).  Outcome probabilities follow the Born
// rule, p_x = |a_x|^2.  The paper gives no procedure for them; the functions
// below are the plain definitions.
// ---------------------------------------------------------------------------

// Born-rule probability of one amplitude.
static double prob_of(const cplx& a) { return a.real() * a.real() + a.imag() * a.imag(); }

// Marginal probabilities of k qubits: out[r] = sum of p_x over x whose bits
// at qubits[0..k-1] form r (bit i of r = qubits[i]), summed in index order.
void or_probabilities(const double* state, int n, const int* qubits, int k, double* out) {
  const u64 N = u64(1) << n;
  const cplx* a = as_c(state);
  for (int r = 0; r < (1 << k); ++r) out[r] = 0.0;
  for (u64 x = 0; x < N; ++x) {
    int r = 0;
    for (int i = 0; i < k; ++i) r |= (int)((x >> qubits[i]) & 1) << i;
    out[r] += prob_of(a[x]);
  }
}

// The state after measuring qubit q with the given outcome, whose
// probability is p: amplitudes whose bit q differs from the outcome become
// 0, the others are multiplied by 1 / sqrt(p) (renormalised).
void or_collapse(double* state, int n, int q, int outcome, double p) {
  const u64 N = u64(1) << n;
  cplx* a = as_c(state);
  const double s = 1.0 / std::sqrt(p);
  for (u64 x = 0; x < N; ++x) a[x] = ((int)((x >> q) & 1) == outcome) ? a[x] * s : cplx(0.0, 0.0);
}

// Cumulative distribution in index order: F[x] = p_0 + p_1 + ... + p_x,
// one running FP64 sum.
void or_cdf(const double* state, int n, double* F) {
  const u64 N = u64(1) << n;
  const cplx* a = as_c(state);
  double r = 0.0;
  for (u64 x = 0; x < N; ++x) {
    r += prob_of(a[x]);
    F[x] = r;
  }
}

// Sampling by inversion of the cumulative distribution: with F as in or_cdf
// and T = F[N - 1], a uniform u in [0, 1) gives t = u T and the sample is the
// smallest x with F[x] > t.  If rounding leaves no such x, the sample is the
// largest x with p_x > 0.  Returns -1 for a state of zero norm.
int or_sample(const double* state, int n, int nshots, const double* u, u64* out) {
  const u64 N = u64(1) << n;
  const cplx* a = as_c(state);
  std::vector<double> F(N);
  or_cdf(state, n, F.data());
  const double T = F[N - 1];
  if (!(T > 0.0)) return -1;
  u64 last = N - 1;
  while (last > 0 && !(prob_of(a[last]) > 0.0)) --last;
  for (int s = 0; s < nshots; ++s) {
    const double t = u[s] * T;
    const u64 x = (u64)(std::upper_bound(F.begin(), F.end(), t) - F.begin());
    out[s] = x < N ? x : last;
  }
  return 0;
}

}  // extern "C"
