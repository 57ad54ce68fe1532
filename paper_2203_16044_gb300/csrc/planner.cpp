// Circuits and compiled plans.
//
// A circuit is an ordered gate sequence (§II-A).  qs_plan_build compiles it
// for a qubit count and dtype into a list of HBM passes:
//   QS_PLAN_UNFUSED  one pass per gate, the per-gate traffic model of Eq. (5):
//                    dense one-qubit gates as pair updates (Eq. 4), CNOT as a
//                    controlled update, diagonal gates (RZ, CZ, CP, ...) as
//                    diagonal passes, SWAP as an in-place bit exchange.
//   QS_PLAN_TILED    gates grouped into shared-memory tile passes (tile.cu):
//                    the single-GPU form of applying gates on local qubits
//                    (§III-B) -- a tile of 2^m amplitudes spanning a chosen
//                    qubit set is read once, every gate on those qubits is
//                    applied in shared memory, and the tile is written back.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "qs_internal.h"
#include "planner.h"

using namespace qs;

namespace qs {

// Algorithmic HBM bytes of one unfused step (read + write of what it touches).
double step_bytes(const qs_step& st, int n, int S) {
  const double N = std::ldexp(1.0, n);
  switch (st.type) {
    case qs_step::GATE_1Q: return 2.0 * N * S;
    case qs_step::GATE_CTRL: return 2.0 * N * S / std::ldexp(1.0, st.nq - 1);
    case qs_step::GATE_DIAG: {
      const int k = st.nq, D = 1 << k;
      bool sparse = true;
      for (int r = 0; r < D - 1 && sparse; ++r) sparse = (st.m[2 * r] == 1.0 && st.m[2 * r + 1] == 0.0);
      return sparse ? 2.0 * N * S / D : 2.0 * N * S;
    }
    case qs_step::GATE_SWAP: return N * S;  // half the amplitudes move
    case qs_step::TILE: return 2.0 * N * S;
    case qs_step::BLOCK: return 2.0 * N * S;
    // s disjoint pairs: an amplitude moves unless every pair's two bits
    // agree, a fraction 1 - 2^-s (the fused-swap traffic of §III-D)
    case qs_step::EXCHANGE: return 2.0 * N * S * (1.0 - std::ldexp(1.0, -st.nq));
  }
  return 0.0;
}

qs_step unfused_step(const qs_gate_rec& g) {
  qs_step st{};
  double m[32];
  gate_matrix(g.kind, g.p, m);
  const int arity = gate_arity(g.kind);
  if (arity == 1) {
    st.q[0] = g.q[0];
    if (gate_is_diagonal(g.kind)) {
      st.type = qs_step::GATE_DIAG;
      st.nq = 1;
      st.m[0] = m[0]; st.m[1] = m[1];   // d0 = m00
      st.m[2] = m[6]; st.m[3] = m[7];   // d1 = m11
    } else {
      st.type = qs_step::GATE_1Q;
      st.nq = 1;
      std::memcpy(st.m, m, sizeof(double) * 8);
    }
  } else if (g.kind == QS_GATE_CNOT) {
    st.type = qs_step::GATE_CTRL;
    st.nq = 2;
    st.q[0] = g.q[0];  // control
    st.q[1] = g.q[1];  // target
    double x[8];
    gate_matrix(QS_GATE_X, nullptr, x);
    std::memcpy(st.m, x, sizeof(x));
  } else if (g.kind == QS_GATE_SWAP) {
    st.type = qs_step::GATE_SWAP;
    st.nq = 2;
    st.q[0] = g.q[0];
    st.q[1] = g.q[1];
  } else {  // CZ, CP: diagonal of the 4x4 matrix
    st.type = qs_step::GATE_DIAG;
    st.nq = 2;
    st.q[0] = g.q[0];
    st.q[1] = g.q[1];
    for (int r = 0; r < 4; ++r) {
      st.m[2 * r] = m[2 * (r * 4 + r)];
      st.m[2 * r + 1] = m[2 * (r * 4 + r) + 1];
    }
  }
  return st;
}

qs_status run_exchange(qs_state* s, const std::vector<std::pair<int, int>>& pairs) {
  int a[17], b[17];
  const int np = (int)pairs.size();
  for (int i = 0; i < np; ++i) {
    a[i] = pairs[i].first;
    b[i] = pairs[i].second;
  }
  return run_bitswap(s, a, b, np);
}

qs_status run_step(qs_state* s, qs_plan* p, const qs_step& st) {
  switch (st.type) {
    case qs_step::GATE_1Q: return run_1q(s, st.q[0], st.m);
    case qs_step::GATE_CTRL: return run_controlled(s, &st.q[0], st.nq - 1, st.q[st.nq - 1], st.m);
    case qs_step::GATE_DIAG: return run_diag(s, st.q, st.nq, st.m);
    case qs_step::GATE_SWAP: return run_bitswap(s, &st.q[0], &st.q[1], 1);
    case qs_step::TILE: return run_tile(s, p, st.tile_index, false);
    case qs_step::BLOCK: {
      const qs_block& b = p->blocks[st.tile_index];
      if (b.tc) {  // B uploaded with the plan's other blocks at the start of the run
        const float* bd = static_cast<const float*>(s->scratch) + b.b_off;
        if (s->dtype == QS_C128) return run_dense_tc128_prepared(s, b.q_sorted, b.k, bd, b.f128, false);
        return run_dense_tc_prepared(s, b.q_sorted, b.k, bd, 1);
      }
      return run_dense(s, b.q, b.k, b.M.data(), 1);  // a product of unitary gates
    }
    case qs_step::EXCHANGE: return run_exchange(s, p->exchanges[st.tile_index]);
  }
  return fail(QS_EINVAL, "bad plan step");
}

// The same step on a complex128 state held in double-float storage.
qs_status run_step_dfl(qs_state* s, qs_plan* p, const qs_step& st) {
  switch (st.type) {
    case qs_step::GATE_1Q: return run_controlled_dfl(s, nullptr, 0, st.q[0], st.m);
    case qs_step::GATE_CTRL: return run_controlled_dfl(s, &st.q[0], st.nq - 1, st.q[st.nq - 1], st.m);
    case qs_step::GATE_DIAG: return run_diag_dfl(s, st.q, st.nq, st.m);
    case qs_step::GATE_SWAP: return run_bitswap(s, &st.q[0], &st.q[1], 1);
    case qs_step::TILE: return run_tile(s, p, st.tile_index, true);
    case qs_step::BLOCK: {
      const qs_block& b = p->blocks[st.tile_index];
      if (!b.tc) return fail(QS_EINVAL, "SIMT dense blocks do not run in double-float storage");
      const float* bd = static_cast<const float*>(s->scratch) + b.b_off;
      return run_dense_tc128_prepared(s, b.q_sorted, b.k, bd, b.f128, true);
    }
    case qs_step::EXCHANGE: return run_exchange(s, p->exchanges[st.tile_index]);  // moves whole amplitudes
  }
  return fail(QS_EINVAL, "bad plan step");
}

// Runs every step (optionally recording an event before the first step and
// after each one).  A complex128 state is switched to double-float storage
// for the duration of the plan and switched back even if a step fails.
qs_status run_all_steps(qs_state* s, qs_plan* p, cudaEvent_t* ev) {
  // complex128 plans switch to double-float storage unless they hold SIMT
  // dense blocks (those run on the FP64 layout); the tensor-core blocks take
  // either
  bool dfl = s->dtype == QS_C128;
  for (const qs_block& b : p->blocks) dfl = dfl && b.tc;
  qs_status r = dfl ? run_layout_dfl(s, true) : QS_OK;
  if (r == QS_OK && !p->tc_B.empty()) {
    // every tensor-core block's B in one upload (one synchronisation with
    // earlier work on the stream, not one per block)
    const size_t bytes = p->tc_B.size() * sizeof(float);
    r = ensure_scratch(s, bytes);
    if (r == QS_OK) {
      cudaError_t e = cudaMemcpyAsync(s->scratch, p->tc_B.data(), bytes, cudaMemcpyHostToDevice, s->stream);
      if (e != cudaSuccess) r = cuda_fail(e, "plan: block matrix upload");
    }
  }
  if (ev) cudaEventRecord(ev[0], s->stream);
  for (size_t i = 0; i < p->steps.size() && r == QS_OK; ++i) {
    r = dfl ? run_step_dfl(s, p, p->steps[i]) : run_step(s, p, p->steps[i]);
    if (ev) cudaEventRecord(ev[i + 1], s->stream);
  }
  if (dfl) {
    const qs_status r2 = run_layout_dfl(s, false);
    if (r == QS_OK) r = r2;
  }
  return r;
}

// ---------------------------------------------------------------------------
// QS_PLAN_FUSED: gates multiplied into dense blocks of at most k qubits.
// Each block is a qubit set S and the gates that can move to the front of
// the remaining circuit inside S: scanning in order, a gate joins when its
// qubits are in S and no earlier gate left out of the block touches them;
// a gate left out blocks its qubits for the rest of the scan.  S is chosen
// among the front-greedy set (gates in order join while the set stays within
// k) and every window of k consecutive qubits, as the one that absorbs most
// gates.  The block matrix is built by applying each gate's 2x2 / 4x4 matrix
// to the rows of the running product.
// ---------------------------------------------------------------------------
namespace {
typedef std::complex<double> cd;

// complex multiply-add in plain real arithmetic (std::complex's operator*
// takes the slow Annex G path for infinities and NaNs)
inline cd cmul(cd a, cd b) {
  return cd(a.real() * b.real() - a.imag() * b.imag(), a.real() * b.imag() + a.imag() * b.real());
}

void left_apply(std::vector<cd>& M, int k, const qs_gate_rec& g, const std::vector<int>& bq) {
  const int D = 1 << k;
  auto slot = [&](int q) { return (int)(std::find(bq.begin(), bq.end(), q) - bq.begin()); };
  double m[32];
  const int nq = gate_matrix(g.kind, g.p, m);
  if (nq == 1) {
    const int a = slot(g.q[0]);
    const cd u00(m[0], m[1]), u01(m[2], m[3]), u10(m[4], m[5]), u11(m[6], m[7]);
    for (int r0 = 0; r0 < D; ++r0) {
      if ((r0 >> a) & 1) continue;
      const int r1 = r0 | (1 << a);
      cd* x = &M[(size_t)r0 * D];
      cd* y = &M[(size_t)r1 * D];
      for (int c = 0; c < D; ++c) {
        const cd xv = x[c], yv = y[c];
        x[c] = cmul(u00, xv) + cmul(u01, yv);
        y[c] = cmul(u10, xv) + cmul(u11, yv);
      }
    }
  } else {
    const int a = slot(g.q[0]), b = slot(g.q[1]);
    cd G[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) G[i][j] = cd(m[2 * (i * 4 + j)], m[2 * (i * 4 + j) + 1]);
    // diagonal (CZ, CP): scale rows; a 0/1 permutation (CNOT, SWAP): move rows
    bool diag = true, perm = true;
    int src[4];
    for (int i = 0; i < 4; ++i) {
      int ones = 0;
      for (int j = 0; j < 4; ++j) {
        if (i != j && G[i][j] != cd(0.0)) diag = false;
        if (G[i][j] == cd(1.0)) { ++ones; src[i] = j; }
        else if (G[i][j] != cd(0.0)) perm = false;
      }
      if (ones != 1) perm = false;
    }
    if (diag || perm) {
      std::vector<cd> tmp(4 * (size_t)D);
      for (int base = 0; base < D; ++base) {
        if (((base >> a) & 1) || ((base >> b) & 1)) continue;
        const int idx[4] = {base, base | (1 << a), base | (1 << b), base | (1 << a) | (1 << b)};
        if (diag) {
          for (int i = 0; i < 4; ++i) {
            if (G[i][i] == cd(1.0)) continue;
            cd* row = &M[(size_t)idx[i] * D];
            for (int c = 0; c < D; ++c) row[c] = cmul(G[i][i], row[c]);
          }
        } else {
          for (int i = 0; i < 4; ++i) std::copy_n(&M[(size_t)idx[i] * D], D, &tmp[(size_t)i * D]);
          for (int i = 0; i < 4; ++i) std::copy_n(&tmp[(size_t)src[i] * D], D, &M[(size_t)idx[i] * D]);
        }
      }
      return;
    }
    for (int base = 0; base < D; ++base) {
      if (((base >> a) & 1) || ((base >> b) & 1)) continue;
      const int idx[4] = {base, base | (1 << a), base | (1 << b), base | (1 << a) | (1 << b)};
      for (int c = 0; c < D; ++c) {
        cd v[4];
        for (int j = 0; j < 4; ++j) v[j] = M[(size_t)idx[j] * D + c];
        for (int i = 0; i < 4; ++i) {
          cd w = 0.0;
          for (int j = 0; j < 4; ++j) w += cmul(G[i][j], v[j]);
          M[(size_t)idx[i] * D + c] = w;
        }
      }
    }
  }
}
}  // namespace

// Gates of `remaining` (in order) that a block on the qubit set inS can take
// to the front of the circuit: a gate joins when all its qubits are in the
// set and none is blocked; any other gate blocks its qubits.  The scan stops
// once every qubit of the set is blocked.  Returns the number taken.
int absorb_into(const std::vector<const qs_gate_rec*>& remaining, const std::vector<char>& inS, int nS,
                std::vector<const qs_gate_rec*>* absorbed, std::vector<const qs_gate_rec*>* rest) {
  std::vector<char> blocked(inS.size(), 0);
  int taken = 0, open = nS;
  size_t i = 0;
  for (; i < remaining.size() && open > 0; ++i) {
    const qs_gate_rec* g = remaining[i];
    const int ng = gate_arity(g->kind);
    bool ok = true;
    for (int j = 0; j < ng; ++j) ok &= inS[g->q[j]] && !blocked[g->q[j]];
    if (ok) {
      ++taken;
      if (absorbed) absorbed->push_back(g);
      continue;
    }
    for (int j = 0; j < ng; ++j)
      if (!blocked[g->q[j]]) {
        blocked[g->q[j]] = 1;
        if (inS[g->q[j]]) --open;
      }
    if (rest) rest->push_back(g);
  }
  if (rest) rest->insert(rest->end(), remaining.begin() + i, remaining.end());
  return taken;
}

// The qubits touched by a candidate block's gates.
std::vector<char> touched(const std::vector<const qs_gate_rec*>& gates, int n) {
  std::vector<char> used(n, 0);
  for (const qs_gate_rec* g : gates)
    for (int j = 0; j < gate_arity(g->kind); ++j) used[g->q[j]] = 1;
  return used;
}

// Tensor-core blocks (both dtypes): the qubits a block runs on, given those its
// gates touch.  Idle qubits cost nothing there (a block is one HBM pass
// whatever its width), but the kernel depends on the set's shape: with at
// least 128 groups and at most 5 runs of block and other qubits, a set
// starting with the run 0 .. a-1 (a >= 4; 3 for complex128) moves as
// 128-byte swizzled pieces, any other set with qubit 0 outside it or in the
// run 0, 1 as one TMA box per tile; other sets gather per thread and run at
// about 0.7 of the speed.  The touched qubits are widened to the narrowest window of
// consecutive qubits that holds them (at least 4 qubits, at most kmax;
// starting at 2 or above if possible, else at 0, else at 1); when none
// exists, to at
// least 4 qubits by idle ones next to the touched ones (not qubit 0), so no
// run is added.
uint64_t tc_block_mask(uint64_t used, int n, int kmax) {
  if (!used) return 0;
  const int lo = __builtin_ctzll(used), hi = 63 - __builtin_clzll(used);
  for (int m = std::max(4, hi - lo + 1); m <= kmax && m <= n; ++m) {
    int pick = -1;
    for (int w = std::max(0, hi - m + 1); w <= lo && w + m <= n; ++w) {
      if (w >= 2) { pick = w; break; }
      if (pick < 0 || (w == 0 && pick == 1)) pick = w;  // 0 before 1
    }
    if (pick >= 0) return ((uint64_t(1) << m) - 1) << pick;
  }
  uint64_t u = used;
  for (int pass = 0; pass < 2 && __builtin_popcountll(u) < 4; ++pass)
    for (int q = 0; q < n && __builtin_popcountll(u) < 4; ++q) {
      const bool next_to = (q > 0 && ((u >> (q - 1)) & 1)) || (q + 1 < n && ((u >> (q + 1)) & 1));
      if (!((u >> q) & 1) && (pass == 1 || (q > 0 && next_to))) u |= uint64_t(1) << q;
    }
  return u;
}

// Whether a tensor-core block on `mask` runs near HBM speed: its tiles move
// by TMA (see above) in pieces of at least 64 bytes: a low run 0 .. a-1
// with a >= 4 as 128-byte swizzled pieces, or a set without qubits 0 and 1
// (one holding qubit 1 leaves 16- or 32-byte pieces, 0.6-0.8 of the speed;
// one holding qubit 0 in a run of 1 or 3 gathers).
bool tc_mask_fast(uint64_t mask, int n) {
  const int k = __builtin_popcountll(mask);
  if (n - k < 7) return false;
  int runs = 1;
  for (int q = 1; q < n; ++q) runs += ((mask >> q) & 1) != ((mask >> (q - 1)) & 1);
  if (runs > 5) return false;
  int a = 0;  // the run 0 .. a-1
  while (a < n && ((mask >> a) & 1)) ++a;
  if (a >= 4) return true;    // 128-byte swizzled pieces (qubits 0 .. k-1 among these)
  return (mask & 3) == 0;     // qubit 0 or 1 in the set: gathered, or boxes of 16- or 32-byte pieces
}

std::vector<int> tc_block_qubits(const std::vector<char>& used, int n, int kmax, bool* fast) {
  uint64_t u = 0;
  for (int q = 0; q < n; ++q)
    if (used[q]) u |= uint64_t(1) << q;
  const uint64_t m = tc_block_mask(u, n, kmax);
  *fast = tc_mask_fast(m, n);
  std::vector<int> bq;
  for (int q = 0; q < n; ++q)
    if ((m >> q) & 1) bq.push_back(q);
  return bq;
}

// ---------------------------------------------------------------------------
// The order of the blocks.  A block's set only decides which gates can move
// to the front now; what the next blocks can take depends on it, so taking
// the most gates at every step (the greedy rule) is not the fewest passes:
// on brick circuits a window that advances the qubits' gate frontiers
// unevenly leaves steps that later windows can climb.  The search keeps the
// `beam` best partial schedules (fewest gates left, then lowest cost) and
// extends each by its kBranch best next sets (most gates per unit of cost);
// a beam of 1 is the greedy rule.  Candidate sets: the front-greedy set and
// every window of kmax consecutive qubits.  Cost of a block: 1, or 10/7 for
// a tensor-core block whose qubits must be gathered per thread (the gather
// kernels run at about 0.7 of the TMA kernels' speed).  Qubit sets are
// 64-bit masks (n <= 34); a schedule's gate set is identified by the XOR of
// random 64-bit keys of its gates (SplitMix64 of the gate index), so that
// two orders reaching the same gates count once.
// ---------------------------------------------------------------------------
namespace {
typedef unsigned long long u64m;
constexpr int kBranch = 8;
constexpr int kPlanThreads = 8;  // host threads of the block-order search
}  // namespace

constexpr int kDefaultBeam = 64;  // QS_PLAN_FUSED search width when opts.search is 0

namespace {

struct SchedNode {
  int parent;
  u64m set;
  int nS;
};
struct SchedState {
  std::vector<int> rem;  // gate indices still to apply, in circuit order
  double cost;
  u64m key;
  int node;
};

u64m gate_key(u64m i) {  // SplitMix64 finaliser of the index
  u64m z = (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Gates of rem a block on S (nS qubits) takes (the rule of absorb_into), and
// the qubits they touch.
int take_count(const std::vector<int>& rem, const u64m* gm, u64m S, int nS, u64m* touched_out) {
  u64m blocked = 0, touched = 0;
  int taken = 0, open = nS;
  for (size_t i = 0; i < rem.size() && open > 0; ++i) {
    const u64m m = gm[rem[i]];
    if (!(m & ~S) && !(m & blocked)) {
      ++taken;
      touched |= m;
      continue;
    }
    open -= __builtin_popcountll(m & ~blocked & S);
    blocked |= m;
  }
  *touched_out = touched;
  return taken;
}

// The same scan, splitting rem into the rest (returned) and the key of the
// gates taken.
std::vector<int> take_rest(const std::vector<int>& rem, const u64m* gm, u64m S, int nS, u64m* key) {
  std::vector<int> rest;
  rest.reserve(rem.size());
  u64m blocked = 0, k = 0;
  int open = nS;
  size_t i = 0;
  for (; i < rem.size() && open > 0; ++i) {
    const u64m m = gm[rem[i]];
    if (!(m & ~S) && !(m & blocked)) {
      k ^= gate_key((u64m)rem[i]);
      continue;
    }
    open -= __builtin_popcountll(m & ~blocked & S);
    blocked |= m;
    rest.push_back(rem[i]);
  }
  rest.insert(rest.end(), rem.begin() + i, rem.end());
  *key = k;
  return rest;
}

u64m key_of_taken(const std::vector<int>& rem, const u64m* gm, u64m S, int nS) {
  u64m blocked = 0, k = 0;
  int open = nS;
  for (size_t i = 0; i < rem.size() && open > 0; ++i) {
    const u64m m = gm[rem[i]];
    if (!(m & ~S) && !(m & blocked)) {
      k ^= gate_key((u64m)rem[i]);
      continue;
    }
    open -= __builtin_popcountll(m & ~blocked & S);
    blocked |= m;
  }
  return k;
}
}  // namespace

// Host threads for the search's steps, started once per search: run(count,
// fn) calls fn(0 .. count-1) on the workers and the calling thread (indices
// taken from a shared counter) and returns when all are done.
class WorkPool {
 public:
  explicit WorkPool(int workers) {
    for (int w = 0; w < workers; ++w) th_.emplace_back([this]() { loop(); });
  }
  ~WorkPool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (std::thread& t : th_) t.join();
  }
  void run(int count, const std::function<void(int)>& fn) {
    if (th_.empty() || count <= 1) {
      for (int i = 0; i < count; ++i) fn(i);
      return;
    }
    {
      std::lock_guard<std::mutex> g(mu_);
      fn_ = &fn;
      count_ = count;
      next_.store(0);
      active_ = (int)th_.size();
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> g(mu_);
    done_.wait(g, [this]() { return active_ == 0; });
    fn_ = nullptr;
  }

 private:
  void work() {
    for (int i = next_.fetch_add(1); i < count_; i = next_.fetch_add(1)) (*fn_)(i);
  }
  void loop() {
    long seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> g(mu_);
        cv_.wait(g, [&]() { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
      }
      work();
      std::lock_guard<std::mutex> g(mu_);
      if (--active_ == 0) done_.notify_one();
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* fn_ = nullptr;
  int count_ = 0, active_ = 0;
  long gen_ = 0;
  std::atomic<int> next_{0};
  bool stop_ = false;
};

// Whether a tensor-core block whose gates touch `touched` gets a TMA shape.
bool tc_fast_shape(u64m touched, int n, int kmax) {
  if (!touched) return true;
  return tc_mask_fast(tc_block_mask(touched, n, kmax), n);
}

// The qubit sets of the blocks, in order (masks and sizes), and their cost.
std::vector<std::pair<u64m, int>> search_blocks(const std::vector<qs_gate_rec>& gates, int n, int kmax, bool tc,
                                                int beam, double* cost) {
  const int G = (int)gates.size();
  std::vector<u64m> gm(G);
  for (int i = 0; i < G; ++i) {
    gm[i] = 0;
    for (int j = 0; j < gate_arity(gates[i].kind); ++j) gm[i] |= 1ull << gates[i].q[j];
  }
  std::vector<SchedNode> nodes;
  std::vector<SchedState> cur(1);
  cur[0].rem.resize(G);
  for (int i = 0; i < G; ++i) cur[0].rem[i] = i;
  cur[0].cost = 0.0;
  cur[0].key = 0;
  cur[0].node = -1;
  struct Child {
    int st;
    u64m set;
    int nS, taken;
    double cost, score;
  };
  const int branch = beam > 1 ? kBranch : 1;
  // the states of a step are expanded, and the kept children built, on up
  // to kPlanThreads host threads (each state's work is independent; the
  // merge below runs in state order, so the result does not depend on the
  // thread count)
  const int nthr = beam >= 16 ? std::max(1, std::min<int>(kPlanThreads, (int)std::thread::hardware_concurrency())) : 1;
  WorkPool pool(nthr - 1);
  auto parallel = [&](int count, const std::function<void(int)>& fn) { pool.run(count, fn); };
  for (;;) {
    int done = -1;
    for (int s = 0; s < (int)cur.size(); ++s)
      if (cur[s].rem.empty() && (done < 0 || cur[s].cost < cur[done].cost)) done = s;
    if (done >= 0) {
      std::vector<std::pair<u64m, int>> out;
      for (int v = cur[done].node; v >= 0; v = nodes[v].parent) out.push_back({nodes[v].set, nodes[v].nS});
      std::reverse(out.begin(), out.end());
      *cost = cur[done].cost;
      return out;
    }
    std::vector<std::vector<Child>> per((size_t)cur.size());
    parallel((int)cur.size(), [&](int s) {
      const SchedState& S0 = cur[s];
      std::vector<Child>& mine = per[(size_t)s];
      auto consider = [&](u64m set, int nS) {
        u64m touched = 0;
        const int taken = take_count(S0.rem, gm.data(), set, nS, &touched);
        if (taken == 0) return;
        const double c = tc && !tc_fast_shape(touched, n, kmax) ? 10.0 / 7.0 : 1.0;
        mine.push_back(Child{s, set, nS, taken, S0.cost + c, taken / c});
      };
      {  // the front-greedy set: gates in order join while the set stays within kmax
        u64m inB = 0, blocked = 0;
        for (int idx : S0.rem) {
          const u64m m = gm[idx];
          if (!(m & blocked) && __builtin_popcountll(inB | m) <= kmax) inB |= m;
          else blocked |= m;
        }
        consider(inB, __builtin_popcountll(inB));
      }
      for (int w = 0; w + kmax <= n; ++w) consider(((1ull << kmax) - 1) << w, kmax);
      // most gates per unit of cost first; ties keep the candidate order
      std::stable_sort(mine.begin(), mine.end(), [](const Child& a, const Child& b) { return a.score > b.score; });
      if ((int)mine.size() > branch) mine.resize(branch);
    });
    std::vector<Child> kids;
    for (const std::vector<Child>& mine : per) kids.insert(kids.end(), mine.begin(), mine.end());
    std::stable_sort(kids.begin(), kids.end(), [&](const Child& a, const Child& b) {
      const size_t ra = cur[a.st].rem.size() - a.taken, rb = cur[b.st].rem.size() - b.taken;
      return ra != rb ? ra < rb : a.cost < b.cost;
    });
    // the children's keys (in parallel), then the first `beam` distinct
    // ones in rank order, then their gate lists (in parallel)
    std::vector<u64m> keys(kids.size());
    const size_t nk = std::min(kids.size(), (size_t)beam * (size_t)kBranch);
    parallel((int)nk, [&](int i) {
      const SchedState& S0 = cur[kids[(size_t)i].st];
      keys[(size_t)i] = S0.key ^ key_of_taken(S0.rem, gm.data(), kids[(size_t)i].set, kids[(size_t)i].nS);
    });
    std::vector<int> pick;
    std::vector<u64m> seen;
    for (size_t i = 0; i < nk && (int)pick.size() < beam; ++i) {
      if (std::find(seen.begin(), seen.end(), keys[i]) != seen.end()) continue;
      seen.push_back(keys[i]);
      pick.push_back((int)i);
    }
    std::vector<SchedState> nxt(pick.size());
    parallel((int)pick.size(), [&](int j) {
      const Child& c = kids[(size_t)pick[(size_t)j]];
      const SchedState& S0 = cur[c.st];
      u64m kk = 0;
      nxt[(size_t)j].rem = take_rest(S0.rem, gm.data(), c.set, c.nS, &kk);
      nxt[(size_t)j].cost = c.cost;
      nxt[(size_t)j].key = keys[(size_t)pick[(size_t)j]];
    });
    for (size_t j = 0; j < pick.size(); ++j) {
      const Child& c = kids[(size_t)pick[j]];
      nodes.push_back(SchedNode{cur[c.st].node, c.set, c.nS});
      nxt[j].node = (int)nodes.size() - 1;
    }
    cur.swap(nxt);
  }
}

// The search's schedule, or the greedy one where that costs less (a beam
// can drop the greedy path), so a wider search is never worse.
std::vector<std::pair<u64m, int>> schedule_blocks(const std::vector<qs_gate_rec>& gates, int n, int kmax, bool tc,
                                                  int beam) {
  double cg = 0.0, cb = 0.0;
  std::vector<std::pair<u64m, int>> greedy = search_blocks(gates, n, kmax, tc, 1, &cg);
  if (beam <= 1) return greedy;
  std::vector<std::pair<u64m, int>> found = search_blocks(gates, n, kmax, tc, beam, &cb);
  return cb < cg || (cb == cg && found.size() <= greedy.size()) ? found : greedy;
}

qs_status plan_fused(qs_plan* p) {
  const int n = p->n;
  int kmax = p->opts.fuse_qubits > 0 ? p->opts.fuse_qubits : 5;
  if (kmax < 2 || kmax > 6) return fail(QS_EINVAL, "qs_plan_build: fuse_qubits=%d outside [2, 6]", kmax);
  const int beam = p->opts.search > 0 ? p->opts.search : kDefaultBeam;
  if (beam > 256) return fail(QS_EINVAL, "qs_plan_build: search=%d outside [0, 256]", p->opts.search);
  // complex128 tensor-core blocks exist for k = 4, 5 (six would need 960
  // tensor-memory columns)
  if (p->dtype == QS_C128 && kmax > 5) kmax = 5;
  if (kmax > n) kmax = n;
  const bool tc = kmax >= 4;
  std::vector<const qs_gate_rec*> remaining;
  for (const qs_gate_rec& g : p->gates) remaining.push_back(&g);
  for (const auto& blk : schedule_blocks(p->gates, n, kmax, tc, beam)) {
    std::vector<char> best(n, 0);
    for (int q = 0; q < n; ++q) best[q] = (blk.first >> q) & 1;
    const int best_n = blk.second;
    std::vector<const qs_gate_rec*> absorbed, rest;
    absorb_into(remaining, best, best_n, &absorbed, &rest);
    // the block's qubits: those its gates touch, for complex64 tensor-core
    // blocks widened with idle qubits (identity on them) to a shape that runs
    // at HBM speed, and at least 4 qubits rather than the SIMT dense kernel
    const std::vector<char> used = touched(absorbed, n);
    std::vector<int> bq;
    if (tc) {
      bool fast = false;
      bq = tc_block_qubits(used, n, kmax, &fast);
    } else {
      for (int q = 0; q < n; ++q)
        if (used[q]) bq.push_back(q);
    }
    qs_block b;
    b.k = (int)bq.size();
    for (int i = 0; i < b.k; ++i) b.q[i] = bq[i];
    const int D = 1 << b.k;
    std::vector<cd> M((size_t)D * D, 0.0);
    for (int r = 0; r < D; ++r) M[(size_t)r * D + r] = 1.0;
    for (const qs_gate_rec* g : absorbed) left_apply(M, b.k, *g, bq);
    b.M.resize((size_t)2 * D * D);
    for (size_t i = 0; i < M.size(); ++i) {
      b.M[2 * i] = M[i].real();
      b.M[2 * i + 1] = M[i].imag();
    }
    if (p->dtype == QS_C64 && b.k >= 4) {  // tensor-core launch data, once
      std::vector<float> B;
      qs_status r = tc_prepare(b.q, b.k, b.M.data(), b.q_sorted, B);
      if (r != QS_OK) return r;
      b.tc = true;
      b.b_off = p->tc_B.size();
      p->tc_B.insert(p->tc_B.end(), B.begin(), B.end());
    } else if (p->dtype == QS_C128 && (b.k == 4 || b.k == 5)) {
      std::vector<uint16_t> dig;
      qs_status r = tc128_prepare(b.q, b.k, b.M.data(), b.q_sorted, dig, &b.f128);
      if (r != QS_OK) return r;
      b.tc = true;
      b.b_off = p->tc_B.size();  // a multiple of 4 floats: 16-byte aligned
      p->tc_B.resize(b.b_off + dig.size() / 2);
      std::memcpy(p->tc_B.data() + b.b_off, dig.data(), dig.size() * sizeof(uint16_t));
    }
    p->blocks.push_back(std::move(b));
    qs_step st{};
    st.type = qs_step::BLOCK;
    st.tile_index = (int)p->blocks.size() - 1;
    p->steps.push_back(st);
    remaining.swap(rest);
  }
  return QS_OK;
}

}  // namespace qs

extern "C" {

qs_status qs_circuit_create(qs_circuit** out) {
  if (!out) return fail(QS_EINVAL, "qs_circuit_create: out is NULL");
  *out = new (std::nothrow) qs_circuit();
  return *out ? QS_OK : fail(QS_ENOMEM, "qs_circuit_create");
}

qs_status qs_circuit_destroy(qs_circuit* c) {
  delete c;
  return QS_OK;
}

qs_status qs_circuit_add(qs_circuit* c, int kind, const int* qubits, int nq, const double* params,
                         int param_index) {
  if (!c) return fail(QS_EINVAL, "qs_circuit_add: circuit is NULL");
  const int arity = gate_arity(kind);
  if (arity < 0) return fail(QS_EINVAL, "qs_circuit_add: unknown gate kind %d", kind);
  if (nq != arity || !qubits) return fail(QS_EINVAL, "qs_circuit_add: kind %d takes %d qubits", kind, arity);
  if (qubits[0] < 0 || (arity == 2 && (qubits[1] < 0 || qubits[1] == qubits[0])))
    return fail(QS_EINVAL, "qs_circuit_add: qubits must be distinct and non-negative");
  const int np = gate_nparams(kind);
  if (np > 0 && !params) return fail(QS_EINVAL, "qs_circuit_add: kind %d needs %d params", kind, np);
  if (param_index >= 0 && !(kind == QS_GATE_RX || kind == QS_GATE_RY || kind == QS_GATE_RZ))
    return fail(QS_EINVAL, "qs_circuit_add: only RX/RY/RZ angles can be trainable");
  qs_gate_rec g{};
  g.kind = kind;
  g.q[0] = qubits[0];
  g.q[1] = arity == 2 ? qubits[1] : -1;
  for (int i = 0; i < np; ++i) g.p[i] = params[i];
  g.param_index = param_index < 0 ? -1 : param_index;
  c->gates.push_back(g);
  return QS_OK;
}

qs_status qs_circuit_add_many(qs_circuit* c, int count, const int* kinds, const int* qubits, const double* params,
                              const int* param_index) {
  if (!c || count < 0 || (count > 0 && (!kinds || !qubits || !params)))
    return fail(QS_EINVAL, "qs_circuit_add_many: NULL argument or negative count");
  c->gates.reserve(c->gates.size() + (size_t)count);
  for (int i = 0; i < count; ++i) {
    const int arity = gate_arity(kinds[i]);
    const qs_status st = qs_circuit_add(c, kinds[i], qubits + 2 * (size_t)i, arity < 0 ? 0 : arity,
                                        params + 3 * (size_t)i, param_index ? param_index[i] : -1);
    if (st != QS_OK) {
      const std::string why = qs_last_error();  // copied: fail() rewrites the same buffer
      return fail(st, "qs_circuit_add_many: gate %d: %s", i, why.c_str());
    }
  }
  return QS_OK;
}

qs_status qs_circuit_size(const qs_circuit* c, int* ngates) {
  if (!c || !ngates) return fail(QS_EINVAL, "qs_circuit_size: NULL argument");
  *ngates = (int)c->gates.size();
  return QS_OK;
}

qs_status qs_plan_build(const qs_circuit* c, int n, qs_dtype dtype, const qs_plan_opts* opts, qs_plan** out) {
  if (!c || !out) return fail(QS_EINVAL, "qs_plan_build: NULL argument");
  *out = nullptr;
  if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "qs_plan_build: n=%d outside [1, %d]", n, QS_MAX_QUBITS);
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "qs_plan_build: bad dtype");
  for (size_t i = 0; i < c->gates.size(); ++i) {
    const qs_gate_rec& g = c->gates[i];
    if (g.q[0] >= n || g.q[1] >= n)
      return fail(QS_EINVAL, "qs_plan_build: gate %zu acts on a qubit >= n=%d", i, n);
  }
  qs_plan* p = new (std::nothrow) qs_plan();
  if (!p) return fail(QS_ENOMEM, "qs_plan_build");
  p->n = n;
  p->dtype = dtype;
  if (opts) p->opts = *opts;
  else {
    std::memset(&p->opts, 0, sizeof(p->opts));
    p->opts.mode = QS_PLAN_TILED;
  }
  p->gates = c->gates;
  qs_status st;
  if (p->opts.mode == QS_PLAN_UNFUSED) {
    for (const qs_gate_rec& g : p->gates) p->steps.push_back(unfused_step(g));
    st = QS_OK;
  } else if (p->opts.mode == QS_PLAN_TILED) {
    st = plan_tiled(p);
  } else if (p->opts.mode == QS_PLAN_FUSED) {
    st = plan_fused(p);
  } else if (p->opts.mode == QS_PLAN_SWAP || p->opts.mode == QS_PLAN_PERMUTE) {
    st = plan_routed(p, p->opts.mode == QS_PLAN_PERMUTE);
  } else {
    st = fail(QS_EINVAL, "qs_plan_build: unknown mode %d", p->opts.mode);
  }
  if (st != QS_OK) {
    qs_plan_destroy(p);
    return st;
  }
  const int S = amp_bytes(dtype);
  p->stats.n = n;
  p->stats.dtype = dtype;
  p->stats.gates = (int)p->gates.size();
  p->stats.passes = (int)p->steps.size();
  p->stats.hbm_bytes = 0.0;
  for (const qs_step& s : p->steps) p->stats.hbm_bytes += step_bytes(s, n, S);
  p->stats.stages = tile_stage_count(p, &p->stats.dense_stages);
  p->stats.metric_bytes = 2.0 * std::ldexp(1.0, n) * S * (double)p->gates.size();
  *out = p;
  return QS_OK;
}

qs_status qs_plan_stats_get(const qs_plan* p, qs_plan_stats* out) {
  if (!p || !out) return fail(QS_EINVAL, "qs_plan_stats_get: NULL argument");
  *out = p->stats;
  return QS_OK;
}

qs_status qs_plan_destroy(qs_plan* p) {
  if (!p) return QS_OK;
  for (qs_tile_pass* t : p->tiles) tile_free(t);
  delete p;
  return QS_OK;
}

qs_status qs_run_plan(qs_state* s, qs_plan* p) {
  if (!s || !p) return fail(QS_EINVAL, "qs_run_plan: NULL argument");
  if (s->n != p->n || s->dtype != p->dtype) return fail(QS_EINVAL, "qs_run_plan: plan built for another n/dtype");
  return run_all_steps(s, p, nullptr);
}

qs_status qs_plan_step_info(const qs_plan* p, int i, int* kind, double* hbm_bytes) {
  if (!p || !kind || !hbm_bytes) return fail(QS_EINVAL, "qs_plan_step_info: NULL argument");
  if (i < 0 || i >= (int)p->steps.size()) return fail(QS_EINVAL, "qs_plan_step_info: step %d out of range", i);
  const qs_step& st = p->steps[i];
  switch (st.type) {
    case qs_step::GATE_1Q: *kind = QS_STEP_1Q; break;
    case qs_step::GATE_CTRL: *kind = QS_STEP_CTRL; break;
    case qs_step::GATE_DIAG: *kind = QS_STEP_DIAG; break;
    case qs_step::GATE_SWAP: *kind = QS_STEP_SWAP; break;
    case qs_step::TILE: *kind = QS_STEP_TILE; break;
    case qs_step::BLOCK: *kind = QS_STEP_BLOCK; break;
    case qs_step::EXCHANGE: *kind = QS_STEP_SWAP; break;
  }
  *hbm_bytes = step_bytes(st, p->n, amp_bytes(p->dtype));
  return QS_OK;
}

qs_status qs_plan_step_qubits(const qs_plan* p, int i, int* qubits, int cap, int* count) {
  if (!p || !count || (cap > 0 && !qubits)) return fail(QS_EINVAL, "qs_plan_step_qubits: NULL argument");
  if (i < 0 || i >= (int)p->steps.size()) return fail(QS_EINVAL, "qs_plan_step_qubits: step %d out of range", i);
  const qs_step& st = p->steps[i];
  const int* q = st.q;
  int nq = st.nq;
  int pq[34];
  if (st.type == qs_step::TILE) {
    nq = 0;
  } else if (st.type == qs_step::EXCHANGE) {
    const auto& pr = p->exchanges[st.tile_index];
    nq = 2 * (int)pr.size();
    for (size_t j = 0; j < pr.size(); ++j) {
      pq[2 * j] = pr[j].first;
      pq[2 * j + 1] = pr[j].second;
    }
    q = pq;
  } else if (st.type == qs_step::BLOCK) {
    const qs_block& b = p->blocks[st.tile_index];
    q = b.q;
    nq = b.k;
  }
  if (nq > cap) return fail(QS_EINVAL, "qs_plan_step_qubits: step %d has %d qubits, cap %d", i, nq, cap);
  for (int j = 0; j < nq; ++j) qubits[j] = q[j];
  *count = nq;
  return QS_OK;
}

qs_status qs_plan_step_matrix(const qs_plan* p, int i, double* M, size_t cap, int* k) {
  if (!p || !k) return fail(QS_EINVAL, "qs_plan_step_matrix: NULL argument");
  if (i < 0 || i >= (int)p->steps.size()) return fail(QS_EINVAL, "qs_plan_step_matrix: step %d out of range", i);
  const qs_step& st = p->steps[i];
  if (st.type != qs_step::BLOCK) return fail(QS_EINVAL, "qs_plan_step_matrix: step %d is not a dense block", i);
  const qs_block& b = p->blocks[st.tile_index];
  const size_t need = b.M.size();
  if (cap < need || !M) return fail(QS_EINVAL, "qs_plan_step_matrix: step %d needs %zu doubles, cap %zu", i, need, cap);
  for (size_t j = 0; j < need; ++j) M[j] = b.M[j];
  *k = b.k;
  return QS_OK;
}

qs_status qs_run_plan_profiled(qs_state* s, qs_plan* p, float* step_ms, int nsteps) {
  if (!s || !p || !step_ms) return fail(QS_EINVAL, "qs_run_plan_profiled: NULL argument");
  if (s->n != p->n || s->dtype != p->dtype) return fail(QS_EINVAL, "qs_run_plan_profiled: plan built for another n/dtype");
  if (nsteps != (int)p->steps.size()) return fail(QS_EINVAL, "qs_run_plan_profiled: nsteps != %zu", p->steps.size());
  std::vector<cudaEvent_t> ev(nsteps + 1);
  for (auto& e : ev) {
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return cuda_fail(r, "qs_run_plan_profiled: event");
  }
  qs_status result = run_all_steps(s, p, ev.data());
  cudaError_t r = cudaStreamSynchronize(s->stream);
  if (result == QS_OK && r != cudaSuccess) result = cuda_fail(r, "qs_run_plan_profiled: sync");
  if (result == QS_OK)
    for (int i = 0; i < nsteps; ++i) cudaEventElapsedTime(&step_ms[i], ev[i], ev[i + 1]);
  for (auto& e : ev) cudaEventDestroy(e);
  return result;
}

}  // extern "C"
