// Batched execution: many independent circuits in one persistent launch.
//
// Every circuit is compiled to tile passes (tile.cu).  The batch is a work
// queue of units (circuit c, pass p, a chunk of that pass's tiles) ordered
// pass-major: all first passes (largest circuits first), then all second
// passes, and so on.  A cooperative grid of persistent CTAs takes units from
// an atomic counter; a unit of pass p > 0 first waits until every tile of
// pass p - 1 of its circuit is done (per-circuit completion counters).  The
// wait is bounded (about 2 s of SM clock): then the CTA sets an error flag
// and leaves, the host reports QS_ETIMEOUT and the context stays usable.  Units
// are only ever waited on after they were dequeued by a running CTA, and a
// cooperative launch keeps every CTA resident, so the queue always drains.
//
// Circuits of up to tile_qubits qubits are one tile: loaded once, every gate
// applied in shared memory, stored once.  With init_zero the first pass
// synthesises |0...0> instead of reading the vector.  State loads and stores
// bypass L1 (ld/st.cg): another CTA may have written the lines since this SM
// last saw them.
//
// The launch (counter reset + kernel) is captured in a CUDA graph at
// creation and replayed by qs_batch_run.  The paper mentions running many
// small circuits only for Intel-QS (§II-B); this scheduling is this
// library's own.
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "planner.h"
#include "tilecore.cuh"

namespace qs {
namespace {

// Bound of one dependency wait, in SM clock cycles (about 2 s at 2 GHz).
constexpr long long kSpinCycles = 4000000000LL;
// fused circuits of a batch: tiles per CTA of their block kernels (their
// states are small, and eight of them run at once on side streams)
constexpr int kBatchTilesPerCta = 4;

struct BCircuit {   // device
  void* amp;
  int n, L, m, r;
  int npasses, pass0;   // passes[pass0 .. pass0 + npasses)
  int ntiles;           // tiles per pass, 2^(n - m)
  int pad;
};
struct BPass {      // device
  int nstages, op_off, stage_off, mat_off;
  int H[kMaxR];
  Ins tins;
};
struct BUnit {
  int c, p, tile0, ntiles;
};
struct BatchArgs {
  const BUnit* units;
  int nunits;
  const BCircuit* circuits;
  const BPass* passes;
  const TOp* ops;
  const TStage* stages;
  const float* mats;
  unsigned* counters;   // [0] queue head, [1 + c] tiles done of circuit c
  int* err;
  int init_zero;
  unsigned wait_bias;   // test hook: extra tiles every wait demands (0 in normal use)
};

struct GlobalSrc {
  const TOp* ops;
  const TStage* st;
  const float* mats;
  __device__ __forceinline__ const TStage& stage(int s) const { return st[s]; }
  __device__ __forceinline__ const TOp& op(int o) const { return ops[o]; }
  __device__ __forceinline__ const float* mat(int i) const { return mats + i * kMatFloats; }
};

__device__ __forceinline__ void ldcg16(const float* p, float (&v)[4]) {
  const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ldcg16(const double* p, double (&v)[2]) {
  const double2 t = __ldcg(reinterpret_cast<const double2*>(p));
  v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void stcg16(float* p, const float (&v)[4]) {
  __stcg(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void stcg16(double* p, const double (&v)[2]) {
  __stcg(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
}

// p: packet index (16 bytes: two complex64 or one complex128 amplitude)
template <int MODE>
__device__ __forceinline__ void bload(const float* a, u64 p, float2* t, int la, bool zero) {
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  if (zero) v[0] = p == 0 ? 1.f : 0.f;
  else ldcg16(a + p * 4, v);
  t[swz<MODE>(la)] = make_float2(v[0], v[1]);
  t[swz<MODE>(la + 1)] = make_float2(v[2], v[3]);
}
template <int MODE>
__device__ __forceinline__ void bstore(float* a, u64 p, const float2* t, int la) {
  const float2 x = t[swz<MODE>(la)], y = t[swz<MODE>(la + 1)];
  const float v[4] = {x.x, x.y, y.x, y.y};
  stcg16(a + p * 4, v);
}
template <int MODE>
__device__ __forceinline__ void bload(const double* a, u64 p, cdf* t, int la, bool zero) {
  double v[2] = {0.0, 0.0};
  if (zero) v[0] = p == 0 ? 1.0 : 0.0;
  else ldcg16(a + p * 2, v);
  const dfl r = d2df(v[0]), i = d2df(v[1]);
  t[swz<MODE>(la)] = cdf{r.h, r.l, i.h, i.l};
}
template <int MODE>
__device__ __forceinline__ void bstore(double* a, u64 p, const cdf* t, int la) {
  const cdf x = t[swz<MODE>(la)];
  const double v[2] = {df2d(dfl{x.rh, x.rl}), df2d(dfl{x.ih, x.il})};
  stcg16(a + p * 2, v);
}

template <int MODE, int G, int GPT>
__global__ void __launch_bounds__(kTT) k_batch(const __grid_constant__ BatchArgs A) {
  typedef typename Elem<MODE>::T E;
  typedef typename std::conditional<MODE == 0, float, double>::type R;
  constexpr int APP = MODE == 0 ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem[];
  u64* tab = reinterpret_cast<u64*>(smem);
  E* t = reinterpret_cast<E*>(smem + 2 * 64 * sizeof(u64));
  __shared__ int s_unit, s_abort;
  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = (int)atomicAdd(&A.counters[0], 1u);
      s_abort = 0;
    }
    __syncthreads();
    const int u = s_unit;
    if (u >= A.nunits) return;
    const BUnit unit = A.units[u];
    const BCircuit cd = A.circuits[unit.c];
    const BPass& pd = A.passes[cd.pass0 + unit.p];
    if (unit.p > 0 && threadIdx.x == 0) {
      // every tile of the previous pass of this circuit must be done
      const unsigned need = (unsigned)unit.p * (unsigned)cd.ntiles + A.wait_bias;
      volatile unsigned* done = A.counters + 1 + unit.c;
      const long long t0 = clock64();
      while (*done < need) {
        if (clock64() - t0 > kSpinCycles || *(volatile int*)A.err) {
          atomicExch(A.err, 1);
          s_abort = 1;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    __syncthreads();
    if (s_abort) return;
    build_spread(tab, pd.H, cd.r);
    __syncthreads();
    R* a = static_cast<R*>(cd.amp);
    const int tile = 1 << cd.m;
    const bool zero = A.init_zero && unit.p == 0;
    const GlobalSrc src{A.ops + pd.op_off, A.stages + pd.stage_off, A.mats + pd.mat_off};
    for (int ti = unit.tile0; ti < unit.tile0 + unit.ntiles; ++ti) {
      const u64 F = expand((u64)ti << cd.L, pd.tins);
      for (int e = threadIdx.x; e < tile / APP; e += kTT) {
        const int la = e * APP;
        bload<MODE>(a, tile_global(F, tab, la, cd.L) / APP, t, la, zero);
      }
      __syncthreads();
      run_stages<MODE, G, GPT, MODE == 0 && G == 3>(t, cd.m, F, src, pd.nstages);
      for (int e = threadIdx.x; e < tile / APP; e += kTT) {
        const int la = e * APP;
        bstore<MODE>(a, tile_global(F, tab, la, cd.L) / APP, t, la);
      }
      __syncthreads();
    }
    // publish: every thread's stores are visible before the count moves
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&A.counters[1 + unit.c], (unsigned)unit.ntiles);
  }
}

}  // namespace
}  // namespace qs

struct qs_batch {
  int count = 0;
  qs_dtype dtype = QS_C64;
  int G = 3, gpt = 1;
  cudaStream_t stream = nullptr;
  void* dev = nullptr;          // one device allocation for all tables
  qs::BatchArgs args{};
  size_t smem = 0;
  unsigned grid = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  qs_batch_stats stats{};
  std::vector<qs_plan*> plans;
  // circuits run as fused tensor-core plans (fuse_min_qubits): their plans,
  // states (wrapping the caller's vectors) and block matrices on the device
  int ntiled = 0;                 // circuits in the persistent launch
  std::vector<qs_plan*> fplans;
  std::vector<qs_state*> fstates;
  void* fB = nullptr;             // every fused plan's tc_B, concatenated
  std::vector<size_t> fB_off;     // per fused plan, in floats
  cudaStream_t fs[8] = {};        // streams the fused plans spread over
  cudaEvent_t fork = nullptr, join[8] = {};
};

namespace qs {
namespace {

template <int MODE, int G, int GPT>
qs_status enqueue_batch(qs_batch* b) {
  auto kern = k_batch<MODE, G, GPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  if (e != cudaSuccess) return cuda_fail(e, "batch: smem attribute");
  if (b->grid == 0) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTT, b->smem);
    if (e != cudaSuccess || per_sm < 1) return cuda_fail(e, "batch: occupancy");
    b->grid = (unsigned)(per_sm * sm_count());
  }
  e = cudaMemsetAsync(b->args.counters, 0, sizeof(unsigned) * (1 + b->count), b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch: counter reset");
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(kTT);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, b->args);
  if (e != cudaSuccess) return cuda_fail(e, "batch: cooperative launch");
  return QS_OK;
}

qs_status enqueue_tiled(qs_batch* b) {
  if (b->ntiled == 0) return QS_OK;
  if (b->dtype == QS_C64) {
    if (b->G == 4) return b->gpt == 2 ? enqueue_batch<0, 4, 2>(b) : enqueue_batch<0, 4, 1>(b);
    return b->gpt == 2 ? enqueue_batch<0, 3, 2>(b) : enqueue_batch<0, 3, 1>(b);
  }
  if (b->G == 4) return enqueue_batch<1, 4, 1>(b);
  return b->gpt == 2 ? enqueue_batch<1, 3, 2>(b) : enqueue_batch<1, 3, 1>(b);
}

// The fused circuits: forked from the batch's stream onto the side streams
// (circuit j on stream j mod 8, largest circuits first), each its blocks in
// order, joined back; the persistent launch runs on the batch's stream
// meanwhile.
qs_status enqueue(qs_batch* b) {
  const int nf = (int)b->fplans.size();
  if (nf == 0) return enqueue_tiled(b);
  const int ns = std::min(nf, 8);
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (int i = 0; i < ns && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->fs[i], b->fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch: fork");
  qs_status st = QS_OK;
  for (int j = 0; j < nf && st == QS_OK; ++j) {
    qs_state* s = b->fstates[j];
    s->stream = b->fs[j % ns];
    if (b->args.init_zero) st = run_set_basis(s, 0);
    const qs_plan* p = b->fplans[j];
    const float* B = static_cast<const float*>(b->fB) + b->fB_off[j];
    for (size_t i = 0; i < p->steps.size() && st == QS_OK; ++i) {
      const qs_block& blk = p->blocks[p->steps[i].tile_index];
      st = b->dtype == QS_C64 ? run_dense_tc_prepared(s, blk.q_sorted, blk.k, B + blk.b_off, 1)
                              : run_dense_tc128_prepared(s, blk.q_sorted, blk.k, B + blk.b_off, blk.f128, false);
    }
  }
  if (st == QS_OK) st = enqueue_tiled(b);
  for (int i = 0; i < ns; ++i) {
    e = cudaEventRecord(b->join[i], b->fs[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
    if (e != cudaSuccess && st == QS_OK) st = cuda_fail(e, "batch: join");
  }
  return st;
}

}  // namespace
}  // namespace qs

using namespace qs;

extern "C" {

qs_status qs_batch_create(int count, const int* nq, qs_dtype dtype, void* const* dev_states,
                          const qs_circuit* const* circuits, const qs_plan_opts* opts, void* stream,
                          qs_batch** out) {
  if (!out) return fail(QS_EINVAL, "qs_batch_create: out is NULL");
  *out = nullptr;
  if (count < 1 || !nq || !dev_states || !circuits) return fail(QS_EINVAL, "qs_batch_create: bad arguments");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "qs_batch_create: bad dtype");
  qs_batch* b = new (std::nothrow) qs_batch();
  if (!b) return fail(QS_ENOMEM, "qs_batch_create");
  b->count = count;
  b->dtype = dtype;
  b->stream = static_cast<cudaStream_t>(stream);
  qs_plan_opts o{};
  if (opts) o = *opts;
  o.mode = QS_PLAN_TILED;
  if (o.fuse_min_qubits < 0) {
    qs_batch_destroy(b);
    return fail(QS_EINVAL, "qs_batch_create: fuse_min_qubits=%d < 0", o.fuse_min_qubits);
  }
  // circuits of at least fuse_min_qubits qubits: fused tensor-core plans
  std::vector<int> tiled;
  std::vector<int> fused;
  for (int i = 0; i < count; ++i) (o.fuse_min_qubits > 0 && nq[i] >= o.fuse_min_qubits ? fused : tiled).push_back(i);
  std::stable_sort(fused.begin(), fused.end(), [&](int x, int y) { return nq[x] > nq[y]; });
  double fhbm = 0, fmetric = 0;
  int fpasses = 0;
  if (!fused.empty()) {
    qs_plan_opts fo{};
    fo.mode = QS_PLAN_FUSED;
    fo.fuse_qubits = o.fuse_qubits > 0 ? o.fuse_qubits : (dtype == QS_C64 ? 6 : 5);
    fo.search = o.search;
    std::vector<float> allB;
    for (int i : fused) {
      if (!circuits[i] || !dev_states[i] || (reinterpret_cast<uintptr_t>(dev_states[i]) & 15)) {
        qs_batch_destroy(b);
        return fail(QS_EINVAL, "qs_batch_create: circuit %d: NULL or misaligned state", i);
      }
      qs_plan* p = nullptr;
      qs_status r = qs_plan_build(circuits[i], nq[i], dtype, &fo, &p);
      if (r == QS_OK && (p->steps.empty() || p->tc_B.empty())) {
        qs_plan_destroy(p);
        r = fail(QS_EINVAL, "qs_batch_create: circuit %d gives no tensor-core blocks", i);
      }
      if (r == QS_OK)
        for (const qs_step& st : p->steps)
          if (st.type != qs_step::BLOCK || !p->blocks[st.tile_index].tc)
            r = fail(QS_EINVAL, "qs_batch_create: circuit %d: a fused step is not a tensor-core block", i);
      qs_state* s = nullptr;
      if (r == QS_OK) r = qs_wrap(nq[i], dtype, dev_states[i], &s);
      if (r == QS_OK) s->tiles_per_cta = kBatchTilesPerCta;
      if (r != QS_OK) {
        if (p) qs_plan_destroy(p);
        qs_batch_destroy(b);
        return r;
      }
      b->fplans.push_back(p);
      b->fstates.push_back(s);
      b->fB_off.push_back(allB.size());
      allB.insert(allB.end(), p->tc_B.begin(), p->tc_B.end());
      fhbm += p->stats.hbm_bytes;
      fmetric += p->stats.metric_bytes;
      fpasses += p->stats.passes;
    }
    cudaError_t e = cudaMalloc(&b->fB, allB.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(b->fB, allB.data(), allB.size() * sizeof(float), cudaMemcpyHostToDevice);
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&b->fs[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      qs_batch_destroy(b);
      return cuda_fail(e, "qs_batch_create: fused circuits' set-up");
    }
  }
  b->ntiled = (int)tiled.size();
  if (tiled.empty()) {
    b->stats.circuits = count;
    b->stats.passes = fpasses;
    b->stats.hbm_bytes = fhbm;
    b->stats.metric_bytes = fmetric;
    *out = b;
    return QS_OK;
  }
  const int count_all = count;
  std::vector<int> nq_t;
  std::vector<void*> ds_t;
  std::vector<const qs_circuit*> c_t;
  for (int i : tiled) {
    nq_t.push_back(nq[i]);
    ds_t.push_back(dev_states[i]);
    c_t.push_back(circuits[i]);
  }
  count = (int)tiled.size();
  nq = nq_t.data();
  dev_states = ds_t.data();
  circuits = c_t.data();
  b->count = count;
  std::vector<BCircuit> hc(count);
  std::vector<BPass> hp;
  std::vector<TOp> hops;
  std::vector<TStage> hst;
  std::vector<float> hmat;
  std::vector<BUnit> hu;
  int maxm = 0, maxpasses = 0;
  double hbm = 0, metric = 0;
  qs_status rc = QS_OK;
  for (int i = 0; i < count && rc == QS_OK; ++i) {
    if (!circuits[i] || !dev_states[i] || (reinterpret_cast<uintptr_t>(dev_states[i]) & 15)) {
      rc = fail(QS_EINVAL, "qs_batch_create: circuit %d: NULL or misaligned state", i);
      break;
    }
    if (nq[i] < 4) {
      rc = fail(QS_EINVAL, "qs_batch_create: circuit %d has %d < 4 qubits", i, nq[i]);
      break;
    }
    qs_plan* p = nullptr;
    rc = qs_plan_build(circuits[i], nq[i], dtype, &o, &p);
    if (rc != QS_OK) break;
    b->plans.push_back(p);
    if (i == 0) {
      b->G = p->opts.slot_qubits;
      b->gpt = p->opts.groups_per_thread;
    }
    if (p->tiles.empty()) {
      rc = fail(QS_EINVAL, "qs_batch_create: circuit %d has no gates", i);
      break;
    }
    BCircuit& c = hc[i];
    c.amp = dev_states[i];
    c.n = nq[i];
    const qs_tile_pass& t0 = *p->tiles[0];
    c.L = t0.L;
    c.m = t0.m;
    c.r = t0.r;
    c.npasses = (int)p->tiles.size();
    c.pass0 = (int)hp.size();
    c.ntiles = 1 << (c.n - c.m);
    maxm = std::max(maxm, c.m);
    maxpasses = std::max(maxpasses, c.npasses);
    for (qs_tile_pass* tp : p->tiles) {
      BPass bp{};
      bp.nstages = (int)tp->stages.size();
      bp.op_off = (int)hops.size();
      bp.stage_off = (int)hst.size();
      bp.mat_off = (int)hmat.size();
      hmat.insert(hmat.end(), tp->mats.begin(), tp->mats.end());
      for (int k = 0; k < tp->r; ++k) bp.H[k] = tp->H[k];
      bp.tins.k = tp->r;
      bp.tins.set = 0;
      for (int k = 0; k < tp->r; ++k) bp.tins.pos[k] = tp->H[k];
      hst.insert(hst.end(), tp->stages.begin(), tp->stages.end());
      hops.insert(hops.end(), tp->ops.begin(), tp->ops.end());
      hp.push_back(bp);
    }
    hbm += p->stats.hbm_bytes;
    metric += p->stats.metric_bytes;
  }
  if (rc != QS_OK) {
    qs_batch_destroy(b);
    return rc;
  }
  // work units: pass-major; within a pass, larger circuits first; tiles in
  // chunks of at least one tile and at most 8
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hc[x].n > hc[y].n; });
  for (int pass = 0; pass < maxpasses; ++pass) {
    for (int i : order) {
      const BCircuit& c = hc[i];
      if (pass >= c.npasses) continue;
      const int chunk = std::max(1, std::min(8, c.ntiles / (4 * sm_count()) + 1));
      for (int t0 = 0; t0 < c.ntiles; t0 += chunk) hu.push_back(BUnit{i, pass, t0, std::min(chunk, c.ntiles - t0)});
    }
  }
  // one device allocation: units | circuits | passes | ops | stages | counters | err
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t ou = 0, oc = al(ou + hu.size() * sizeof(BUnit)), op = al(oc + hc.size() * sizeof(BCircuit)),
               oo = al(op + hp.size() * sizeof(BPass)), os = al(oo + hops.size() * sizeof(TOp)),
               om = al(os + hst.size() * sizeof(TStage)), ocnt = al(om + hmat.size() * sizeof(float)),
               oerr = al(ocnt + sizeof(unsigned) * (1 + count)), total = al(oerr + sizeof(int));
  std::vector<unsigned char> host(total, 0);
  std::memcpy(host.data() + ou, hu.data(), hu.size() * sizeof(BUnit));
  std::memcpy(host.data() + oc, hc.data(), hc.size() * sizeof(BCircuit));
  std::memcpy(host.data() + op, hp.data(), hp.size() * sizeof(BPass));
  if (!hops.empty()) std::memcpy(host.data() + oo, hops.data(), hops.size() * sizeof(TOp));
  if (!hst.empty()) std::memcpy(host.data() + os, hst.data(), hst.size() * sizeof(TStage));
  if (!hmat.empty()) std::memcpy(host.data() + om, hmat.data(), hmat.size() * sizeof(float));
  cudaError_t e = cudaMalloc(&b->dev, total);
  if (e != cudaSuccess) {
    qs_batch_destroy(b);
    return fail(QS_ENOMEM, "qs_batch_create: %zu bytes of tables: %s", total, cudaGetErrorString(e));
  }
  e = cudaMemcpy(b->dev, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    qs_batch_destroy(b);
    return cuda_fail(e, "qs_batch_create: upload");
  }
  unsigned char* d = static_cast<unsigned char*>(b->dev);
  b->args.units = reinterpret_cast<const BUnit*>(d + ou);
  b->args.nunits = (int)hu.size();
  b->args.circuits = reinterpret_cast<const BCircuit*>(d + oc);
  b->args.passes = reinterpret_cast<const BPass*>(d + op);
  b->args.ops = reinterpret_cast<const TOp*>(d + oo);
  b->args.stages = reinterpret_cast<const TStage*>(d + os);
  b->args.mats = reinterpret_cast<const float*>(d + om);
  b->args.counters = reinterpret_cast<unsigned*>(d + ocnt);
  b->args.err = reinterpret_cast<int*>(d + oerr);
  b->args.init_zero = 1;
  b->args.wait_bias = (unsigned)std::max(0, o.reserved[0]);
  const size_t esize = dtype == QS_C64 ? sizeof(float2) : sizeof(cdf);
  b->smem = 2 * 64 * sizeof(u64) + (size_t(1) << maxm) * esize;
  b->stats.circuits = count_all;
  b->stats.units = (int)hu.size();
  b->stats.passes = (int)hp.size() + fpasses;
  b->stats.hbm_bytes = hbm + fhbm;
  b->stats.metric_bytes = metric + fmetric;
  *out = b;
  return QS_OK;
}

qs_status qs_batch_run(qs_batch* b, int init_zero) {
  if (!b) return fail(QS_EINVAL, "qs_batch_run: NULL batch");
  init_zero = init_zero ? 1 : 0;
  if (b->exec && b->args.init_zero == init_zero) {
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "qs_batch_run: graph launch");
  }
  // (re)capture the launch for this init mode
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  b->args.init_zero = init_zero;
  qs_status st = enqueue(b);  // first launch outside capture: sets the grid, checks the configuration
  if (st != QS_OK) return st;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qs_batch_run: first launch");
  // a stream that is the legacy default stream cannot be captured: no graph then
  if (b->stream == nullptr) return QS_OK;
  e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "qs_batch_run: begin capture");
  st = enqueue(b);
  e = cudaStreamEndCapture(b->stream, &b->graph);
  if (st != QS_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "qs_batch_run: end capture");
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_fail(e, "qs_batch_run: instantiate");
  }
  return QS_OK;
}

qs_status qs_batch_sync(qs_batch* b) {
  if (!b) return fail(QS_EINVAL, "qs_batch_sync: NULL batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "qs_batch_sync");
  if (!b->fplans.empty()) {
    const qs_status t = b->dtype == QS_C64 ? fused_tc_status() : fused_c128_status();
    if (t != QS_OK) return t;
  }
  if (b->ntiled == 0) return QS_OK;
  int err = 0;
  e = cudaMemcpy(&err, b->args.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "qs_batch_sync: error flag");
  if (err) {
    cudaMemset(b->args.err, 0, sizeof(int));
    return fail(QS_ETIMEOUT, "qs_batch_sync: a pass dependency wait gave up; the states are incomplete");
  }
  return QS_OK;
}

qs_status qs_batch_stats_get(const qs_batch* b, qs_batch_stats* out) {
  if (!b || !out) return fail(QS_EINVAL, "qs_batch_stats_get: NULL argument");
  *out = b->stats;
  out->grid = (int)b->grid;
  out->graph = b->exec != nullptr;
  return QS_OK;
}

qs_status qs_batch_destroy(qs_batch* b) {
  if (!b) return QS_OK;
  if (b->stream || b->dev) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (int i = 0; i < 8; ++i)
    if (b->fs[i]) cudaStreamSynchronize(b->fs[i]);
  if (b->dev) cudaFree(b->dev);
  for (qs_plan* p : b->plans) qs_plan_destroy(p);
  for (qs_plan* p : b->fplans) qs_plan_destroy(p);
  for (qs_state* s : b->fstates) {
    s->stream = nullptr;
    qs_free(s);
  }
  if (b->fB) cudaFree(b->fB);
  for (int i = 0; i < 8; ++i) {
    if (b->fs[i]) cudaStreamDestroy(b->fs[i]);
    if (b->join[i]) cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
  return QS_OK;
}

// Autotuner: times candidate plan shapes on the batch itself and keeps the
// fastest.  Results are cached under a hash of every circuit, the qubit
// counts, the dtype and the GPU (tune.cpp): in memory for the process and in
// the cache file when one is set (qs_tune_cache_file).
qs_status qs_batch_autotune(int count, const int* nq, qs_dtype dtype, void* const* dev_states,
                            const qs_circuit* const* circuits, void* stream, qs_plan_opts* best,
                            double* best_ms) {
  if (!best) return fail(QS_EINVAL, "qs_batch_autotune: best is NULL");
  if (count < 1 || !nq || !circuits) return fail(QS_EINVAL, "qs_batch_autotune: bad arguments");
  qs_status kst = QS_OK;
  const unsigned long long key = batch_tune_key(count, nq, dtype, circuits, &kst);
  if (kst != QS_OK) return kst;
  if (batch_tune_lookup(key, best, best_ms)) return QS_OK;
  const int mcands[] = {11, 12, 13};
  const int gcands[][2] = {{3, 1}, {3, 2}, {4, 1}};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double bestt = 1e30;
  qs_plan_opts bo{};
  qs_status rc = QS_OK;
  for (int m : mcands) {
    for (auto& gg : gcands) {
      if (dtype == QS_C128 && m > 13) continue;
      qs_plan_opts o{};
      o.mode = QS_PLAN_TILED;
      o.tile_qubits = m;
      o.slot_qubits = gg[0];
      o.groups_per_thread = gg[1];
      qs_batch* b = nullptr;
      rc = qs_batch_create(count, nq, dtype, dev_states, circuits, &o, stream, &b);
      if (rc != QS_OK) break;
      rc = qs_batch_run(b, 1);  // warm-up (and graph capture)
      if (rc == QS_OK) rc = qs_batch_sync(b);
      float ms = 0.f;
      if (rc == QS_OK) {
        cudaEventRecord(e0, s);
        rc = qs_batch_run(b, 1);
        cudaEventRecord(e1, s);
        if (rc == QS_OK) rc = qs_batch_sync(b);
        cudaEventElapsedTime(&ms, e0, e1);
      }
      qs_batch_destroy(b);
      if (rc != QS_OK) break;
      if (ms < bestt) {
        bestt = ms;
        bo = o;
      }
    }
    if (rc != QS_OK) break;
  }
  // then circuits from 16, 18 or 20 qubits up as fused tensor-core plans
  const int fmins[] = {16, 18, 20};
  for (int fm : fmins) {
    if (rc != QS_OK) break;
    bool any = false;
    for (int i = 0; i < count; ++i) any |= nq[i] >= fm;
    if (!any) continue;
    qs_plan_opts o = bo;
    o.fuse_min_qubits = fm;
    qs_batch* b = nullptr;
    rc = qs_batch_create(count, nq, dtype, dev_states, circuits, &o, stream, &b);
    if (rc != QS_OK) break;
    rc = qs_batch_run(b, 1);
    if (rc == QS_OK) rc = qs_batch_sync(b);
    float ms = 0.f;
    if (rc == QS_OK) {
      cudaEventRecord(e0, s);
      rc = qs_batch_run(b, 1);
      cudaEventRecord(e1, s);
      if (rc == QS_OK) rc = qs_batch_sync(b);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    qs_batch_destroy(b);
    if (rc == QS_OK && ms < bestt) {
      bestt = ms;
      bo = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != QS_OK) return rc;
  *best = bo;
  if (best_ms) *best_ms = bestt;
  batch_tune_remember(key, bo, bestt);
  return QS_OK;
}

}  // extern "C"
