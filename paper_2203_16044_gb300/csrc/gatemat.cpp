// Host-side construction of named gate matrices for the circuit planner.
//
// Definitions (angles in radians; the paper fixes none of them):
//   H = [[1,1],[1,-1]]/sqrt(2); X, Y, Z Pauli; S = diag(1, i); T = diag(1, e^{i pi/4})
//   RX/RY/RZ(t) = exp(-i t P / 2);  P(l) = diag(1, e^{i l})
//   U3(t,p,l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]]
//   CNOT(control = qubits[0], target = qubits[1]); CZ; CP(l) = diag(1,1,1,e^{il}); SWAP
// Matrices are row-major with (re, im) per entry; for two-qubit gates bit 0
// of the 4x4 index is qubits[0].
#include <cmath>

#include "qs_internal.h"

namespace qs {

int gate_arity(int kind) {
  if (kind >= QS_GATE_H && kind <= QS_GATE_U3) return 1;
  if (kind >= QS_GATE_CNOT && kind <= QS_GATE_SWAP) return 2;
  return -1;
}

int gate_nparams(int kind) {
  switch (kind) {
    case QS_GATE_RX: case QS_GATE_RY: case QS_GATE_RZ: case QS_GATE_P: case QS_GATE_CP: return 1;
    case QS_GATE_U3: return 3;
    default: return 0;
  }
}

bool gate_is_diagonal(int kind) {
  switch (kind) {
    case QS_GATE_Z: case QS_GATE_S: case QS_GATE_T: case QS_GATE_RZ: case QS_GATE_P:
    case QS_GATE_CZ: case QS_GATE_CP: return true;
    default: return false;
  }
}

static void set(double* m, int dim, int r, int c, double re, double im) {
  m[2 * (r * dim + c)] = re;
  m[2 * (r * dim + c) + 1] = im;
}

int gate_matrix(int kind, const double* prm, double* m) {
  const int nq = gate_arity(kind);
  if (nq < 0) return -1;
  const int dim = 1 << nq;
  for (int i = 0; i < 2 * dim * dim; ++i) m[i] = 0.0;
  switch (kind) {
    case QS_GATE_H: {
      const double r = 0.70710678118654752440;
      set(m, 2, 0, 0, r, 0); set(m, 2, 0, 1, r, 0); set(m, 2, 1, 0, r, 0); set(m, 2, 1, 1, -r, 0);
    } break;
    case QS_GATE_X: set(m, 2, 0, 1, 1, 0); set(m, 2, 1, 0, 1, 0); break;
    case QS_GATE_Y: set(m, 2, 0, 1, 0, -1); set(m, 2, 1, 0, 0, 1); break;
    case QS_GATE_Z: set(m, 2, 0, 0, 1, 0); set(m, 2, 1, 1, -1, 0); break;
    case QS_GATE_S: set(m, 2, 0, 0, 1, 0); set(m, 2, 1, 1, 0, 1); break;
    case QS_GATE_T: {
      const double r = 0.70710678118654752440;
      set(m, 2, 0, 0, 1, 0); set(m, 2, 1, 1, r, r);
    } break;
    case QS_GATE_RX: {
      const double c = std::cos(0.5 * prm[0]), s = std::sin(0.5 * prm[0]);
      set(m, 2, 0, 0, c, 0); set(m, 2, 0, 1, 0, -s); set(m, 2, 1, 0, 0, -s); set(m, 2, 1, 1, c, 0);
    } break;
    case QS_GATE_RY: {
      const double c = std::cos(0.5 * prm[0]), s = std::sin(0.5 * prm[0]);
      set(m, 2, 0, 0, c, 0); set(m, 2, 0, 1, -s, 0); set(m, 2, 1, 0, s, 0); set(m, 2, 1, 1, c, 0);
    } break;
    case QS_GATE_RZ: {
      const double c = std::cos(0.5 * prm[0]), s = std::sin(0.5 * prm[0]);
      set(m, 2, 0, 0, c, -s); set(m, 2, 1, 1, c, s);
    } break;
    case QS_GATE_P:
      set(m, 2, 0, 0, 1, 0); set(m, 2, 1, 1, std::cos(prm[0]), std::sin(prm[0]));
      break;
    case QS_GATE_U3: {
      const double c = std::cos(0.5 * prm[0]), s = std::sin(0.5 * prm[0]);
      const double ph = prm[1], la = prm[2];
      set(m, 2, 0, 0, c, 0);
      set(m, 2, 0, 1, -std::cos(la) * s, -std::sin(la) * s);
      set(m, 2, 1, 0, std::cos(ph) * s, std::sin(ph) * s);
      set(m, 2, 1, 1, std::cos(ph + la) * c, std::sin(ph + la) * c);
    } break;
    case QS_GATE_CNOT:
      // index r = b0 + 2 b1 with b0 the control: X on b1 when b0 = 1
      set(m, 4, 0, 0, 1, 0); set(m, 4, 2, 2, 1, 0); set(m, 4, 1, 3, 1, 0); set(m, 4, 3, 1, 1, 0);
      break;
    case QS_GATE_CZ:
      set(m, 4, 0, 0, 1, 0); set(m, 4, 1, 1, 1, 0); set(m, 4, 2, 2, 1, 0); set(m, 4, 3, 3, -1, 0);
      break;
    case QS_GATE_CP:
      set(m, 4, 0, 0, 1, 0); set(m, 4, 1, 1, 1, 0); set(m, 4, 2, 2, 1, 0);
      set(m, 4, 3, 3, std::cos(prm[0]), std::sin(prm[0]));
      break;
    case QS_GATE_SWAP:
      set(m, 4, 0, 0, 1, 0); set(m, 4, 1, 2, 1, 0); set(m, 4, 2, 1, 1, 0); set(m, 4, 3, 3, 1, 0);
      break;
    default: return -1;
  }
  return nq;
}

}  // namespace qs
