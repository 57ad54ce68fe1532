/*
 * qs.h -- C ABI of the GB300 state-vector gate engine (libqs.so).
 *
 * The library applies a quantum circuit's gates to a full 2^n-amplitude
 * complex state vector resident in GPU memory (sm_103a, one GPU per process).
 *
 * Conventions shared by every call
 * --------------------------------
 *  State layout (§II-A, Eq. 2): amplitude a_x of basis state |x> is element x;
 *    bit q of x is qubit q (qubit 0 = least significant).  QS_C128 stores
 *    interleaved (re, im) doubles, 16 bytes per amplitude, 2^(n+4) bytes in
 *    total (§I); QS_C64 stores interleaved (re, im) floats, 8 bytes per
 *    amplitude.  These are the numpy/PyTorch complex128 / complex64 layouts.
 *  Matrices are always passed on the host in FP64: a 2x2 matrix is 8 doubles,
 *    row-major, (re, im) per entry; a k-qubit matrix over qubits[0..k-1] is
 *    2^k x 2^k row-major, and bit i of its row/column index r corresponds to
 *    qubits[i].  QS_C64 states round matrices to FP32 once per call.
 *  Host arrays passed in are read before the call returns; the caller keeps
 *    ownership.  Device work is enqueued on the state's stream (qs_set_stream)
 *    and is asynchronous unless the call returns a host value.
 *  Errors: every call returns a qs_status.  Argument errors are detected
 *    synchronously, return QS_EINVAL and leave the state unchanged.  CUDA
 *    launch errors return QS_ECUDA; asynchronous device errors surface on the
 *    next call that synchronises (qs_sync, reductions, copies).  The library
 *    never aborts the process.  qs_last_error() returns a thread-local
 *    description of the most recent failure.
 *  Numerics: QS_C64 computes in FP32; QS_C128 computes with at least 47-bit
 *    significands (FP64, or double-float pairs of FP32 values where the FP64
 *    pipe would be the bottleneck), except dense blocks of 4 or 5 qubits,
 *    which put each group of amplitudes on a fixed-point grid of 43 bits
 *    below the group's largest one (error about 2^-44 of it per block).
 *    Reductions (norm, inner product, expectation values) accumulate in at
 *    least FP64-equivalent precision for both dtypes and are deterministic
 *    (fixed reduction order).
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int qs_status;
enum {
  QS_OK = 0,
  QS_EINVAL = -1,        /* bad argument; nothing was enqueued            */
  QS_ENOMEM = -2,        /* device or host allocation failed              */
  QS_ECUDA = -3,         /* CUDA runtime / launch error                   */
  QS_ETIMEOUT = -4,      /* a bounded device wait gave up                 */
  QS_EUNSUPPORTED = -5   /* valid request this build does not implement   */
};

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

/* Largest qubit count accepted by qs_alloc / qs_wrap (2^34 amplitudes). */
#define QS_MAX_QUBITS 34

typedef struct qs_state qs_state;     /* opaque: one state vector        */
typedef struct qs_circuit qs_circuit; /* opaque: host-side gate list     */
typedef struct qs_plan qs_plan;       /* opaque: compiled pass schedule  */

/* Thread-local text of the last failure ("" if none).  Never NULL. */
const char* qs_last_error(void);
/* Library version string. */
const char* qs_version(void);

/* ---------------------------------------------------------------------- */
/* State lifetime                                                         */
/* ---------------------------------------------------------------------- */

/* Allocate a state of n qubits (1 <= n <= QS_MAX_QUBITS) on the current
 * device, initialised to |0...0>.  The library owns the memory (freed by
 * qs_free).  QS_ENOMEM if the device allocation fails. */
qs_status qs_alloc(int n, qs_dtype dtype, qs_state** out);

/* Wrap caller-owned device memory of 2^n amplitudes of `dtype` (for example
 * a PyTorch tensor's storage).  dev_ptr must be 16-byte aligned and stay
 * valid until qs_free; the contents are not touched; qs_free does not free
 * it. */
qs_status qs_wrap(int n, qs_dtype dtype, void* dev_ptr, qs_state** out);

/* Release the handle (and its memory if it came from qs_alloc) after
 * synchronising its stream.  NULL is accepted. */
qs_status qs_free(qs_state* st);

/* Enqueue all later work of this state on `stream` (a cudaStream_t; NULL is
 * the legacy default stream). */
qs_status qs_set_stream(qs_state* st, void* stream);

/* Wait for all work enqueued on the state's stream; reports any pending
 * asynchronous device error as QS_ECUDA, and QS_ETIMEOUT if a tensor-core
 * block kernel (dense blocks of 4 to 6 qubits on complex64, 4 or 5 on
 * complex128) gave up waiting for its matrix unit or a tile copy since the
 * last qs_sync (bounded wait of about 1 s; the state's contents are then
 * invalid). */
qs_status qs_sync(qs_state* st);

/* Device pointer and size of the amplitude array. */
qs_status qs_data(qs_state* st, void** dev_ptr, size_t* bytes);

/* Set the state to the basis state |x>, x < 2^n (§II-A, Eq. 2). */
qs_status qs_set_basis(qs_state* st, uint64_t x);

/* Copy the whole amplitude array to / from host memory of 2^n amplitudes in
 * the state's dtype layout.  Synchronous with respect to the host.  Pinned
 * host memory gives full link bandwidth; pageable memory also works. */
qs_status qs_copy_to_host(qs_state* st, void* dst);
qs_status qs_copy_from_host(qs_state* st, const void* src);
/* As qs_copy_from_host, but returns once the copy is queued on the state's
 * stream: work queued after it on that stream (a plan run) starts when the
 * data is on the device, and the host can build circuits and plans
 * meanwhile.  src must stay valid and unchanged until the stream has passed
 * the copy (qs_sync, or a later synchronous call on the state); with
 * pageable memory the call may return only after the copy. */
qs_status qs_copy_from_host_async(qs_state* st, const void* src);

/* ---------------------------------------------------------------------- */
/* Gate application (one HBM pass each)                                   */
/* ---------------------------------------------------------------------- */

/* One-qubit gate U on qubit q, Eq. (4) of §II-A: for every x with bit q
 * clear and y = x | 2^q, (a_x, a_y) <- U (a_x, a_y).  U: 8 doubles. */
qs_status qs_apply_1q(qs_state* st, int q, const double U[8]);

/* Controlled one-qubit gate: Eq. (4) applied only where every control bit
 * of x is 1 (CNOT = controlled X, as in the CNOT layers of §IV-F).
 * 0 <= nc <= 8 distinct controls, all different from target. */
qs_status qs_apply_controlled(qs_state* st, const int* controls, int nc, int target,
                              const double U[8]);

/* Diagonal gate on k distinct qubits (1 <= k <= 8): a_x <- d[r(x)] a_x with
 * bit i of r(x) = bit qubits[i] of x.  d: 2^k complex values (2^(k+1)
 * doubles).  RZ, CZ and the controlled phases of the QFT are diagonal. */
qs_status qs_apply_diag(qs_state* st, const int* qubits, int k, const double* d);

/* Dense k-qubit gate (1 <= k <= 6) on distinct qubits: for every base x with
 * the k bits clear, the 2^k amplitudes a[x | spread(r)] are multiplied by
 * the 2^k x 2^k matrix M (2^(2k+1) doubles, row-major, (re, im)).  On the
 * tensor cores for k >= 4 (complex64) and k = 4, 5 (complex128: each group
 * and M on fixed-point grids split into 9-bit integer digits, whose products
 * the MMAs form exactly); M must have finite entries. */
qs_status qs_apply_fused(qs_state* st, const int* qubits, int k, const double* M);

/* Qubit permutation: out[pi(x)] = in[x] where pi moves bit j of x to bit
 * perm[j]; perm is a permutation of 0..n-1.  In place.  The fused swap of
 * §III-D (Listing 1) is the permutation exchanging the disjoint bit fields
 * [p, p+s) and [q, q+s); any permutation runs as at most two in-place passes
 * of disjoint bit-field exchanges. */
qs_status qs_permute_qubits(qs_state* st, const int* perm);

/* fused_swap(p, q, s) of §III-D: swap(p+i, q+i) for i = 0..s-1; the ranges
 * [p, p+s) and [q, q+s) must not overlap.  One in-place pass that moves the
 * 2^n (1 - 2^-s) amplitudes whose two fields differ. */
qs_status qs_fused_swap(qs_state* st, int p, int q, int s);

/* ---------------------------------------------------------------------- */
/* Reductions (return host values; synchronise the state's stream)       */
/* ---------------------------------------------------------------------- */

/* out = sum_x |a_x|^2. */
qs_status qs_norm2(qs_state* st, double* out);

/* out[0] + i out[1] = <a|b> = sum_x conj(a_x) b_x.  Same n and dtype.  When
 * a and b hold the same device vector this is the norm (qs_norm2, one read
 * of the state) with out[1] = 0. */
qs_status qs_inner(qs_state* a, qs_state* b, double out[2]);

/* out = sum_t coeff[t] <psi|P_t|psi> for Pauli strings P_t with X on the
 * qubits set only in xmask[t], Z on those set only in zmask[t], Y on those
 * set in both.  1 <= nterms <= 65536.  Terms sharing an X/Y mask form a
 * group; groups whose X/Y bits fit a tile share tile passes over the
 * state.  Arithmetic: complex128, and complex64 groups of several terms,
 * exact products in double-float summed in FP64 (about 2^-46 of the sum of
 * the term magnitudes); complex64 groups of one term and two-Z-bit classes
 * in tile passes, FP32 products summed in FP32 per thread and tile, then in
 * double-float and FP64 (within about 2^-20 of sum_t |coeff[t]| for a
 * unit-norm state: the complex64 state's own precision). */
qs_status qs_expect_pauli(qs_state* st, int nterms, const uint64_t* xmask,
                          const uint64_t* zmask, const double* coeff, double* out);

/* *passes = the number of reads of the whole state that qs_expect_pauli
 * makes for these terms on an n-qubit state of this dtype: one per tile
 * pass (groups sharing a tile of the 4 lowest qubits plus up to 9, or 8
 * for complex128, higher ones) plus one per group with more X/Y bits above
 * the 4 lowest qubits than a tile holds.  Host only (no device work; no
 * state needed).  QS_EINVAL for n outside 1..34, an unknown dtype, nterms
 * outside 1..65536, NULL arrays, or a term on a qubit >= n. */
qs_status qs_expect_pauli_passes(int n, qs_dtype dtype, int nterms, const uint64_t* xmask,
                                 const uint64_t* zmask, int* passes);

/* ---------------------------------------------------------------------- */
/* Measurement in the computational basis (§II-A: a circuit is a sequence  */
/* of gates, measurements and resets).  Probabilities follow the Born rule, */
/* p_x = |a_x|^2, formed and summed in FP64.                                */
/* ---------------------------------------------------------------------- */

/* Marginal probabilities of k qubits: out[r] (host, 2^k doubles) = sum of
 * p_x over x whose bits at qubits[0..k-1] form r (bit i of r = qubits[i]).
 * 1 <= k <= 6, qubits distinct and < n.  Does not change the state;
 * synchronises its stream. */
qs_status qs_probabilities(qs_state* st, const int* qubits, int k, double* out);

/* Measures qubit q with the caller's uniform u in [0, 1): with p0, p1 the
 * probabilities of 0 and 1 (as qs_probabilities), the outcome is 0 when
 * u (p0 + p1) < p0, else 1 (the other one if the chosen probability is 0).
 * The state collapses onto it: amplitudes of the other outcome become 0,
 * the kept ones are scaled by 1 / sqrt(p_outcome), so the state is
 * renormalised.  *outcome (host) receives 0 or 1; *prob (host, may be NULL)
 * the outcome's probability p_outcome / (p0 + p1).  A reset of qubit q is
 * this followed by an X on q when the outcome is 1.  QS_EINVAL for u outside
 * [0, 1) or a state of zero norm. */
qs_status qs_measure(qs_state* st, int q, double u, int* outcome, double* prob);

/* Samples nshots basis states without changing the state, by inversion of
 * the cumulative distribution in index order, F(x) = p_0 + ... + p_x: for
 * the caller's uniforms u[i] in [0, 1) (host), with T = F(2^n - 1) and
 * t = u[i] T, out[i] (host) is the x with F(x - 1) <= t < F(x); it always has
 * p_x > 0.  The sums are accurate to FP64 level but not taken in index
 * order, so where t lies within their rounding (a few 2^-53 T per term) of
 * a boundary F(x), either neighbour may be returned.  The whole search runs
 * on the GPU (partial sums of 1024- and 32768-amplitude blocks, one warp per
 * shot); the state's scratch buffer grows to about 2^n / 1024 doubles plus
 * 16 bytes per shot (up to 2^20 shots at a time).  QS_EINVAL for a uniform
 * outside [0, 1) or a state of zero norm.  Synchronises the state's stream. */
qs_status qs_sample(qs_state* st, uint64_t nshots, const double* u, uint64_t* out);

/* Allocation-free inner product, for callers that cannot let the library
 * allocate device memory (a framework allocator that owns the GPU's memory,
 * a latency-critical loop where cudaMalloc/cudaFree would synchronise, a
 * host policy that forbids allocations outside its own allocator).  The
 * paper has no counterpart; this is an interface convenience.
 *   a, b:   device pointers to 2^n amplitudes of `dtype` (16-byte aligned),
 *           caller-owned, read only.
 *   stream: cudaStream_t to run on (NULL = legacy default stream).
 *   out:    host array; receives <a|b> = sum_x conj(a_x) b_x (re, im), FP64.
 * Synchronises `stream` before returning.  Allocates nothing: its partial
 * sums live in a fixed 16 KiB (1024 x 16-byte partials + result) static
 * device array that every GPU loading the library keeps until exit.  The
 * first call on a device looks that array's address up (make that first
 * call before any stream capture begins).  All calls share the array:
 * calls that overlap on the GPU race and must be serialised.  Returns
 * QS_EUNSUPPORTED if the reduction would need more than 1024 partials (a
 * device with more than 256 SMs). */
qs_status qs_inner_noalloc(const void* a, const void* b, int n, qs_dtype dtype, void* stream,
                           double out[2]);

/* ---------------------------------------------------------------------- */
/* Circuits and compiled plans                                            */
/* ---------------------------------------------------------------------- */

/* Gate kinds for qs_circuit_add.  Angles in radians.
 *   H, X, Y, Z, S = diag(1, i), T = diag(1, e^{i pi/4})
 *   RX/RY/RZ(t) = exp(-i t P / 2),  P(l) = diag(1, e^{il})
 *   U3(t, p, l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]]
 *   CNOT(control, target), CZ(a, b), CP(a, b; l) = diag(1,1,1,e^{il}), SWAP(a, b)
 */
typedef enum {
  QS_GATE_H = 0, QS_GATE_X, QS_GATE_Y, QS_GATE_Z, QS_GATE_S, QS_GATE_T,
  QS_GATE_RX, QS_GATE_RY, QS_GATE_RZ, QS_GATE_P, QS_GATE_U3,
  QS_GATE_CNOT = 16, QS_GATE_CZ, QS_GATE_CP, QS_GATE_SWAP
} qs_gate_kind;

qs_status qs_circuit_create(qs_circuit** out);
qs_status qs_circuit_destroy(qs_circuit* c);
/* Append one gate.  qubits: 1 or 2 entries by kind; params: 0, 1 or 3 angles
 * by kind (NULL when none).  param_index >= 0 marks the (single) angle of an
 * RX/RY/RZ gate as trainable parameter number param_index (used by
 * qs_adjoint_grad); -1 otherwise. */
qs_status qs_circuit_add(qs_circuit* c, int kind, const int* qubits, int nq,
                         const double* params, int param_index);
/* Append `count` gates at once (the same checks as qs_circuit_add, gate by
 * gate; on an error the gates before the offending one stay appended and
 * the status names its index).  Per gate i: kinds[i]; qubits[2 i], and
 * qubits[2 i + 1] for two-qubit kinds; params[3 i .. 3 i + 2], of which the
 * kind's 0, 1 or 3 angles are read; param_index[i] (NULL: all -1). */
qs_status qs_circuit_add_many(qs_circuit* c, int count, const int* kinds, const int* qubits, const double* params,
                              const int* param_index);
/* Number of gates appended so far. */
qs_status qs_circuit_size(const qs_circuit* c, int* ngates);

/* Plan options.  mode: QS_PLAN_UNFUSED applies every gate with its own pass
 * (one kernel per gate); QS_PLAN_TILED groups gates into shared-memory tile
 * passes; QS_PLAN_FUSED multiplies gates into dense blocks of at most
 * fuse_qubits qubits, each applied as one pass on the tensor cores, as
 * qs_apply_fused (complex64 blocks of 4 to 6 qubits; complex128 blocks of 4
 * or 5, a fuse_qubits of 6 is taken as 5 there; blocks whose gates touch
 * fewer qubits are widened with idle ones to a window of consecutive
 * qubits where one exists).  The order of a fused plan's blocks comes from
 * a search over partial schedules (search: how many are kept at each
 * block; 1 takes, at every block, the qubit set that absorbs the most
 * gates): a block's set decides which gates later blocks can take, so the
 * greedy order is not the fewest passes (a brick circuit of depth 40 on 30
 * qubits: 67 passes greedy, 64 with a width of 16, 63 with the default 64).  QS_PLAN_SWAP and
 * QS_PLAN_PERMUTE apply the
 * gates in tile passes over the tile_qubits lowest physical qubits only and
 * move every other target there first, by in-place bit-pair exchange
 * passes (§III-D): QS_PLAN_SWAP inserts one exchange of one pair (a swap)
 * per target that is not local; QS_PLAN_PERMUTE one exchange of up to
 * tile_qubits pairs (a fused swap) per routing point, for every target the
 * coming gates need; SWAP gates of the circuit only relabel qubits; the
 * state ends in logical order (at most two more exchange passes).  tile_qubits: qubits
 * resident per tile pass (0 = library default
 * for the dtype; at most 14 for QS_C64, 13 for QS_C128); low_qubits: qubits
 * 0..low_qubits-1 kept in every tile for coalesced access (0 = default);
 * slot_qubits: qubits held in registers per stage inside a tile pass, 3 or
 * 4 (0 = default); groups_per_thread: register groups a thread works on at
 * once, 1 or 2 (0 = default; QS_C128 with 4 slots always uses 1); dense:
 * 0 = a stage whose gates all act within its three slot qubits may be fused
 * into one 8x8 matrix when the planner estimates that cheaper (complex64,
 * three slots), -1 = never.  Every field must be zero or valid. */
enum { QS_PLAN_UNFUSED = 0, QS_PLAN_TILED = 1, QS_PLAN_FUSED = 2, QS_PLAN_SWAP = 3, QS_PLAN_PERMUTE = 4 };
typedef struct {
  int mode;
  int tile_qubits;
  int low_qubits;
  int slot_qubits;
  int groups_per_thread;
  int dense;
  int fuse_qubits;    /* QS_PLAN_FUSED: qubits per dense block, 2..6 (0 = 5) */
  int search;         /* QS_PLAN_FUSED: block-order search width, 1..256
                         (1 = greedy; 0 = 64)                           */
  int fuse_min_qubits;/* qs_batch_create: circuits of at least this many
                         qubits run as QS_PLAN_FUSED plans (fuse_qubits,
                         0 = 6 for QS_C64, 5 for QS_C128) on parallel
                         streams; 0 = every circuit as tile passes      */
  int reserved[1];
} qs_plan_opts;

typedef struct {
  int n;              /* qubits                                          */
  int dtype;          /* qs_dtype                                        */
  int gates;          /* logical gates of the circuit                    */
  int passes;         /* HBM passes of the plan (kernel launches)        */
  double hbm_bytes;   /* algorithmic HBM bytes of one run of the plan    */
  double metric_bytes;/* 2 * 2^n * bytes_per_amp * gates (Eq. 5 traffic) */
  int stages;         /* register stages summed over all tile passes     */
  int dense_stages;   /* of which fused into one dense 8x8 matrix        */
} qs_plan_stats;

/* Compile circuit `c` for n qubits and `dtype`.  opts may be NULL
 * (QS_PLAN_TILED with defaults).  The plan keeps its own copy of the gates;
 * device-side gate tables are uploaded on the first qs_run_plan. */
qs_status qs_plan_build(const qs_circuit* c, int n, qs_dtype dtype, const qs_plan_opts* opts,
                        qs_plan** out);
qs_status qs_plan_stats_get(const qs_plan* p, qs_plan_stats* out);
qs_status qs_plan_destroy(qs_plan* p);

/* Apply the whole plan to the state (n and dtype must match). */
qs_status qs_run_plan(qs_state* st, qs_plan* p);

/* Step kinds reported by qs_plan_step_info. */
enum { QS_STEP_1Q = 0, QS_STEP_CTRL = 1, QS_STEP_DIAG = 2, QS_STEP_SWAP = 3, QS_STEP_TILE = 4, QS_STEP_BLOCK = 5 };

/* Kind and algorithmic HBM bytes (read + write of the amplitudes it
 * touches) of plan step i, 0 <= i < passes.  A swap or bit-pair exchange
 * pass (QS_STEP_SWAP) of s pairs moves the 2^n (1 - 2^-s) amplitudes whose
 * index changes. */
qs_status qs_plan_step_info(const qs_plan* p, int i, int* kind, double* hbm_bytes);

/* The qubits plan step i acts on, in the order its matrix uses them (for a
 * dense block, qubit j is bit j of the block matrix's row index; for a gate,
 * controls first, the target last; for a bit-pair exchange pass of
 * QS_PLAN_SWAP / QS_PLAN_PERMUTE, its pairs a0, b0, a1, b1, ... of physical
 * qubit positions): up to `cap` ints written to `qubits`, their number to
 * *count.  Tile passes report 0 qubits.  QS_EINVAL if the
 * step has more than `cap` qubits (nothing written) or i is out of range. */
qs_status qs_plan_step_qubits(const qs_plan* p, int i, int* qubits, int cap, int* count);

/* The 2^k x 2^k complex matrix (row-major, (re, im) per entry, FP64) of a
 * dense-block step i (QS_PLAN_FUSED plans), in the qubit order of
 * qs_plan_step_qubits: bit j of its row and column index is qubit j of
 * that list.  `cap` is the capacity of M in doubles (2 * 4^k needed); *k
 * receives the block's qubit count.  QS_EINVAL for another step kind, a
 * step out of range or too small a buffer. */
qs_status qs_plan_step_matrix(const qs_plan* p, int i, double* M, size_t cap, int* k);

/* As qs_run_plan, and also times every step with CUDA events recorded on the
 * state's stream between launches: step_ms[i] receives the device time of
 * step i (nsteps must equal the plan's pass count).  Synchronises the
 * stream before returning.  Event recording adds a few microseconds per
 * step; use qs_run_plan for throughput. */
qs_status qs_run_plan_profiled(qs_state* st, qs_plan* p, float* step_ms, int nsteps);

/* ---------------------------------------------------------------------- */
/* Batched execution                                                      */
/* ---------------------------------------------------------------------- */

typedef struct qs_batch qs_batch;  /* opaque: many circuits, one launch */

typedef struct {
  int circuits;       /* circuits in the batch                           */
  int units;          /* work units in the queue                         */
  int passes;         /* tile passes summed over circuits                */
  int grid;           /* persistent CTAs (0 before the first run)        */
  int graph;          /* 1 when runs replay a captured CUDA graph        */
  int reserved;
  double hbm_bytes;   /* algorithmic HBM bytes of one run                */
  double metric_bytes;/* 2 * 2^n_i * bytes_per_amp * gates_i, summed     */
} qs_batch_stats;

/* Compile `count` independent circuits (circuit i on n[i] >= 4 qubits,
 * state i at dev_states[i]: 2^n[i] amplitudes of `dtype`, 16-byte aligned,
 * caller-owned) into one batch run on `stream`.  Every circuit becomes tile
 * passes (opts as for qs_plan_build, mode ignored; NULL = defaults); the
 * batch is a work queue of (circuit, pass, tiles) units executed by one
 * persistent cooperative launch.  With opts->fuse_min_qubits > 0, circuits
 * of at least that many qubits instead run as QS_PLAN_FUSED plans (dense
 * blocks of opts->fuse_qubits qubits on the tensor cores, block matrices
 * uploaded once here), spread over 8 streams forked from `stream` and
 * joined back, alongside the persistent launch.  The paper runs circuits
 * one at a time; this is the library's own scheduling.  The first
 * qs_batch_run captures the launches in a CUDA graph (unless `stream` is
 * the legacy default stream).
 * opts->reserved[0] is a test hook and must be 0 in normal use: a positive
 * value makes every wait for a previous pass demand that many tiles more
 * than exist, so the bounded wait runs out (QS_ETIMEOUT from
 * qs_batch_sync, after about 2 s). */
qs_status qs_batch_create(int count, const int* n, qs_dtype dtype, void* const* dev_states,
                          const qs_circuit* const* circuits, const qs_plan_opts* opts, void* stream,
                          qs_batch** out);

/* Enqueue one run of every circuit of the batch (asynchronous).  init_zero:
 * start every circuit from |0...0> (the vectors are not read); otherwise the
 * circuits act on the current contents. */
qs_status qs_batch_run(qs_batch* b, int init_zero);

/* Wait for the batch's stream and check the run: QS_ETIMEOUT if a bounded
 * pass-dependency wait gave up (the states are then incomplete). */
qs_status qs_batch_sync(qs_batch* b);

qs_status qs_batch_stats_get(const qs_batch* b, qs_batch_stats* out);
qs_status qs_batch_destroy(qs_batch* b);

/* Autotuner: builds and times the batch for candidate tile sizes and
 * register slot counts, then, with the best of those, for the qubit counts
 * from which circuits run as fused tensor-core plans (fuse_min_qubits 16,
 * 18, 20 at the dtype's default block width), two runs each, starting from
 * |0...0> (the states are overwritten), and returns the fastest options in
 * *best (and its time in *best_ms if non-NULL).  Cached under a hash of every circuit, the
 * qubit counts, the dtype and the GPU, as for qs_plan_autotune. */
qs_status qs_batch_autotune(int count, const int* n, qs_dtype dtype, void* const* dev_states,
                            const qs_circuit* const* circuits, void* stream, qs_plan_opts* best,
                            double* best_ms);

/* ---------------------------------------------------------------------- */
/* Autotuning                                                             */
/* ---------------------------------------------------------------------- */

/* Picks the fastest plan shape for circuit c on state st by timing
 * candidates on st itself (its contents are overwritten): dense blocks of
 * k = 4, 5, 6 qubits (complex128: 4, 5) and tile passes of 12 to 14 qubits
 * with 3 or 4 register slots.  *best receives options for qs_plan_build,
 * *best_ms (may be NULL) the time of one run of that plan.  The result is
 * cached under a hash of the circuit's gates, n, the dtype and the GPU
 * (name, SM count, compute capability): later calls with the same circuit
 * return at once, also in later processes when a cache file is set. */
qs_status qs_plan_autotune(const qs_circuit* c, qs_state* st, qs_plan_opts* best, double* best_ms);

/* Sets the file that persists autotuning results (one text line per
 * result, appended as results are found) and loads the results it already
 * holds, replacing those in memory.  NULL keeps results in memory only (and
 * clears them).  A file that cannot be written only loses persistence. */
qs_status qs_tune_cache_file(const char* path);

/* 64-bit FNV-1a hash of a circuit's gates (kind, qubits, angle bits,
 * parameter index) with n and dtype: the device-independent part of the
 * autotuner's key. */
qs_status qs_circuit_hash(const qs_circuit* c, int n, qs_dtype dtype, uint64_t* out);

/* ---------------------------------------------------------------------- */
/* Differentiation                                                        */
/* ---------------------------------------------------------------------- */

/* Energies and gradients of E(theta) = <psi(theta)|H|psi(theta)> for `batch`
 * parameter sets, psi(theta) = circuit applied to |0...0>.  The paper has no
 * differentiation; this is the standard adjoint (reverse-sweep) method: one
 * forward run, lambda = H psi, then for each gate from last to first the
 * gradient term Im <lambda|P|psi> of a trainable R_P(theta_j) =
 * exp(-i theta_j P / 2) followed by un-applying the gate to psi and lambda.
 *   st:      state fixing n and dtype; its contents are overwritten.
 *   c:       the circuit; RX/RY/RZ gates added with param_index j >= 0 take
 *            their angle from theta (the stored angle is ignored).
 *   theta:   batch x nparam angles (row-major).
 *   H:       sum_t coeff[t] P_t with Pauli strings as in qs_expect_pauli.
 *   energy:  batch values; grad: batch x nparam, dE/dtheta (row-major).
 * Per-pair gradient products are FP32 (complex64) or double-float
 * (complex128), summed per thread in double-float and across threads in FP64.
 * Parameter sets run in chunks of Bc (a power of two chosen from the state
 * size): psi and lambda of a chunk share one allocation of 2 Bc state
 * vectors, so each fixed gate is one launch for the whole chunk; with Bc = 1
 * the state itself holds psi and one extra vector is allocated.  Allocations
 * (stream-ordered) last for the call; QS_ENOMEM if they fail.  Synchronises
 * the state's stream. */
qs_status qs_adjoint_grad(qs_state* st, const qs_circuit* c, const double* theta, int nparam, int batch,
                          int nterms, const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                          double* energy, double* grad);

#ifdef __cplusplus
}
#endif
#endif /* QS_H */
