// tcgen05 / TMA building blocks shared by the tensor-core block kernels
// (complex64 in fused_tc.cu, complex128 in fused_c128.cu): inline PTX for
// tensor-memory loads and stores, MMA issue, shared-memory matrix and
// instruction descriptors, bounded mbarrier waits and tiled TMA copies.
#pragma once

#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "qs_internal.h"

namespace qs {

constexpr int kUT = 128;  // rows per tile = MMA M = TMEM lanes

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzle:
// start address, lbo = byte distance between core matrices adjacent along
// K, sbo = between core matrices adjacent along M (or N); bits 46-48 hold
// the fixed value 0b001; base offset 0, swizzle mode 0.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* o) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) o[j] = __uint_as_float(r[j]);
}
// mbarrier phase wait with a limit of about 2^31 SM cycles; false on timeout.
// The "memory" clobber keeps the compiler from sinking earlier loads (the
// next tiles' prefetch) below the wait.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const unsigned* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* o) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 8; ++j) o[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const unsigned* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
               "r"(r[2]), "r"(r[3]));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const unsigned* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
}
__device__ __forceinline__ void umma_f16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bd), "r"(idesc), "r"(acc));
}
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// FP16 (bits 7-9, 10-12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at 24.
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(mbar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
               "r"(y), "r"(src)
               : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, const int (&c)[5], uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
          dst),
      "l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, const int (&c)[5], uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(dst),
      "l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const int (&c)[5], uint32_t src) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
               "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, const int (&c)[5], uint32_t src) {
  asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(map),
               "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map), "r"(x),
               "r"(y), "r"(z), "r"(src)
               : "memory");
}

inline qs_status tmap_encoder(PFN_cuTensorMapEncodeTiled_v12000* out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(QS_ECUDA, "fused_tc: cuTensorMapEncodeTiled not available");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *out = encode;
  return QS_OK;
}

// A block's tile as one TMA box of a view of the state with 2 to 5
// dimensions.  The qubits split into maximal runs of block qubits and of
// other qubits; each run is one tensor dimension (2^len entries, stride
// 2^lo amplitudes).  The tile (128 consecutive groups) takes the 7 lowest
// non-block qubits, the box covers them and the block runs whole.  The
// dimensions' order fixes where the box lands in shared memory: element e
// (block index, bit i the i-th block qubit ascending) of tile row r at
// mult_r(r) + pos_e(e), the sums of per-bit multipliers kept in the
// RunBox.  Two orders are used: ascending qubits (long contiguous DRAM
// bursts; a warp's 32 rows are consecutive elements when the lowest run
// holds at least 5 of the tile's qubits, else 2^(5 - t)-way bank conflicts
// for a first run of t tile qubits) when that run holds at least
// kNaturalMinTile of them, else the runs holding tile qubits first (rows
// r at r + 128 e, free of bank conflicts, shorter bursts).  When qubit 0 is
// in the block, its run must be qubits 0 and 1 exactly: that run is
// dimension 0, the contiguous one (32-byte pieces; a run of 1 leaves 16-byte
// pieces and measured slower than gathering), and an element and its
// neighbour in it are adjacent: complex64 reads them as one 16-byte word.
// Needs 2^(n-k) >= 128 and at most 5 runs; false otherwise.  words: 64-bit words per amplitude (1:
// complex64, 2: complex128).  A non-block run's qubits are consecutive
// bits of the group index, so tile g's coordinate along it is
// (g >> gb) & (2^len - 1) (times `words` for d = 0); along block runs 0.
constexpr int kNaturalMinTile = 4;
struct RunBox {
  int8_t gb[5];   // dimension d's coordinate: bits gb .. gb + len - 1 of the group index (gb < 0: a block run)
  int8_t len[5];
  int rank;
  int multr[7];  // position of tile-row bit i (the i-th lowest non-block qubit), in amplitudes
  int multe[6];  // position of block-index bit j (the j-th block qubit), in amplitudes
};
inline bool make_runs_tmap(void* amp, int n, int k, const int* q_sorted, int words, CUtensorMap* map, RunBox* rb,
                           qs_status* st) {
  *st = QS_OK;
  if (n - k < 7 || k > 6) return false;
  if (q_sorted[k - 1] == k - 1) return false;  // qubits 0 .. k-1: the rows form
  if (q_sorted[0] == 0 && !(q_sorted[1] == 1 && q_sorted[2] > 2)) return false;  // qubit 0 in a run other than 2
  uint64_t inb = 0;
  for (int i = 0; i < k; ++i) inb |= uint64_t(1) << q_sorted[i];
  int tilebit[64] = {0};  // 1: one of the 7 lowest non-block qubits
  for (int q = 0, c = 0; q < n && c < 7; ++q)
    if (!((inb >> q) & 1)) { tilebit[q] = 1; ++c; }
  struct Run { int lo, len, tile, block; };
  std::vector<Run> runs;
  for (int q = 0; q < n;) {
    const int b = (int)((inb >> q) & 1);
    int e = q;
    while (e < n && (int)((inb >> e) & 1) == b) ++e;
    int t = 0;
    for (int x = q; x < e; ++x) t += tilebit[x];
    runs.push_back(Run{q, e - q, t, b});
    q = e;
  }
  if (runs.size() > 5) return false;
  std::vector<Run> ord;
  if (runs[0].block) {
    // qubits 0, 1 in the block: that run stays innermost, then
    // the tile's runs, the other block runs and the rest
    ord.push_back(runs[0]);
    for (const Run& r : runs) if (!r.block && r.tile) ord.push_back(r);
    for (size_t i = 1; i < runs.size(); ++i) if (runs[i].block) ord.push_back(runs[i]);
    for (const Run& r : runs) if (!r.block && !r.tile) ord.push_back(r);
  } else if (runs[0].tile >= kNaturalMinTile) {
    ord = runs;
  } else {
    for (const Run& r : runs) if (!r.block && r.tile) ord.push_back(r);
    for (const Run& r : runs) if (r.block) ord.push_back(r);
    for (const Run& r : runs) if (!r.block && !r.tile) ord.push_back(r);
  }
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  *st = tmap_encoder(&encode);
  if (*st != QS_OK) return false;
  const int rank = (int)ord.size();
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  int mult[64] = {0};  // position multiplier of each qubit inside the box (amplitudes)
  int stride_in_box = 1;
  for (int d = 0; d < 5; ++d) {
    rb->gb[d] = -1;
    rb->len[d] = 0;
    if (d >= rank) continue;
    const Run& r = ord[d];
    const int ext = r.block ? r.len : r.tile;  // qubits of the run inside the box
    dims[d] = (cuuint64_t(1) << r.len) * (d == 0 ? words : 1);
    box[d] = (cuuint32_t)((1u << ext) * (d == 0 ? words : 1));
    if (d > 0) strides[d - 1] = (cuuint64_t(1) << r.lo) * 8 * words;
    if (!r.block) {
      int below = 0;  // non-block qubits below the run: its first group-index bit
      for (int x = 0; x < r.lo; ++x) below += !((inb >> x) & 1);
      rb->gb[d] = (int8_t)below;
      rb->len[d] = (int8_t)r.len;
    }
    for (int x = 0; x < ext; ++x) mult[r.lo + x] = stride_in_box << x;
    stride_in_box <<= ext;
  }
  rb->rank = rank;
  for (int i = 0, c = 0; i < n && c < 7; ++i)
    if (tilebit[i]) rb->multr[c++] = mult[i];
  for (int j = 0; j < 6; ++j) rb->multe[j] = j < k ? mult[q_sorted[j]] : 0;
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)rank, amp, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *st = fail(QS_ECUDA, "cuTensorMapEncodeTiled (run box) failed (%d)", (int)r);
    return false;
  }
  return true;
}
// Blocks whose qubits start with a run 0 .. a-1 long enough for 128-byte
// row pieces (2^a amplitudes >= slice_amps: 16 for complex64, 8 for
// complex128), plus any other runs (at most 5 runs in all): the tile moves
// as 2^a / slice_amps boxes, box b holding piece b of the low run (slice_amps
// amplitudes = 128 bytes) for the tile's 128 rows and every value of the
// other block qubits, 128-byte swizzled (16-byte unit c of smem line L at
// c ^ (L mod 8)).  Dimensions: the low run (extent slice_amps), the runs
// holding the tile's qubits, the other block runs, the rest; line
// L = r + 128 e_hi, e_hi the block index above the low run.  Qubits
// 0 .. k-1 are the case without other runs.
struct LowBox {
  int8_t gb[5];   // dimension d's coordinate: group-index bits gb .. gb + len - 1 (gb < 0: none)
  int8_t len[5];
  int rank;
  int nslice;     // boxes per tile (2^a / slice_amps)
  int slice_words;  // 64-bit words of one piece (16)
};
inline bool make_lowrun_tmap(void* amp, int n, int k, const int* q_sorted, int words, int slice_amps,
                             CUtensorMap* map, LowBox* lb, qs_status* st) {
  *st = QS_OK;
  if (n - k < 7 || k > 6) return false;
  int a = 0;
  while (a < k && q_sorted[a] == a) ++a;
  if ((1 << a) < slice_amps) return false;
  uint64_t inb = 0;
  for (int i = 0; i < k; ++i) inb |= uint64_t(1) << q_sorted[i];
  int tilebit[64] = {0};
  for (int q = 0, c = 0; q < n && c < 7; ++q)
    if (!((inb >> q) & 1)) { tilebit[q] = 1; ++c; }
  struct Run { int lo, len, tile, block; };
  std::vector<Run> runs;
  for (int q = 0; q < n;) {
    const int b = (int)((inb >> q) & 1);
    int e = q;
    while (e < n && (int)((inb >> e) & 1) == b) ++e;
    int t = 0;
    for (int x = q; x < e; ++x) t += tilebit[x];
    runs.push_back(Run{q, e - q, t, b});
    q = e;
  }
  if (runs.size() > 5) return false;
  std::vector<Run> ord;
  ord.push_back(runs[0]);  // the low run 0 .. a-1
  for (const Run& r : runs) if (!r.block && r.tile) ord.push_back(r);
  for (size_t i = 1; i < runs.size(); ++i) if (runs[i].block) ord.push_back(runs[i]);
  for (const Run& r : runs) if (!r.block && !r.tile) ord.push_back(r);
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  *st = tmap_encoder(&encode);
  if (*st != QS_OK) return false;
  const int rank = (int)ord.size();
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  for (int d = 0; d < 5; ++d) {
    lb->gb[d] = -1;
    lb->len[d] = 0;
    if (d >= rank) continue;
    const Run& r = ord[d];
    dims[d] = (cuuint64_t(1) << r.len) * (d == 0 ? words : 1);
    box[d] = d == 0 ? (cuuint32_t)(slice_amps * words) : (cuuint32_t)(r.block ? (1u << r.len) : (1u << r.tile));
    if (d > 0) strides[d - 1] = (cuuint64_t(1) << r.lo) * 8 * words;
    if (d > 0 && !r.block) {
      int below = 0;
      for (int x = 0; x < r.lo; ++x) below += !((inb >> x) & 1);
      lb->gb[d] = (int8_t)below;
      lb->len[d] = (int8_t)r.len;
    }
  }
  lb->rank = rank;
  lb->nslice = (1 << a) / slice_amps;  // at most 4: 2^6 / 16 (complex64), 2^5 / 8 (complex128)
  lb->slice_words = slice_amps * words;
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)rank, amp, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *st = fail(QS_ECUDA, "cuTensorMapEncodeTiled (low-run box) failed (%d)", (int)r);
    return false;
  }
  return true;
}
// Every piece of tile g: box b (b < nslice <= 4) at dst0 + b * boxb, its
// coordinates computed once (one thread).
__device__ __forceinline__ void lowrun_coords(uint64_t g, const LowBox& lb, int (&c)[5]) {
  c[0] = 0;
#pragma unroll
  for (int d = 1; d < 5; ++d) c[d] = lb.gb[d] < 0 ? 0 : (int)((g >> lb.gb[d]) & ((uint64_t(1) << lb.len[d]) - 1));
}
__device__ __forceinline__ void lowrun_load(uint32_t dst0, uint32_t boxb, const CUtensorMap* map, uint64_t g,
                                            const LowBox& lb, uint32_t mbar) {
  int c[5];
  lowrun_coords(g, lb, c);
  if (lb.rank == 2) {  // qubits 0 .. k-1
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (b < lb.nslice) tma_load_2d(dst0 + b * boxb, map, b * lb.slice_words, c[1], mbar);
    return;
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    if (b >= lb.nslice) break;
    c[0] = b * lb.slice_words;
    switch (lb.rank) {
      case 3: tma_load_3d(dst0 + b * boxb, map, c[0], c[1], c[2], mbar); break;
      case 4: tma_load_4d(dst0 + b * boxb, map, c, mbar); break;
      default: tma_load_5d(dst0 + b * boxb, map, c, mbar); break;
    }
  }
}
__device__ __forceinline__ void lowrun_store(const CUtensorMap* map, uint64_t g, const LowBox& lb, uint32_t src0,
                                             uint32_t boxb) {
  int c[5];
  lowrun_coords(g, lb, c);
  if (lb.rank == 2) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (b < lb.nslice) tma_store_2d(map, b * lb.slice_words, c[1], src0 + b * boxb);
    return;
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    if (b >= lb.nslice) break;
    c[0] = b * lb.slice_words;
    switch (lb.rank) {
      case 3: tma_store_3d(map, c[0], c[1], c[2], src0 + b * boxb); break;
      case 4: tma_store_4d(map, c, src0 + b * boxb); break;
      default: tma_store_5d(map, c, src0 + b * boxb); break;
    }
  }
}
// The tile's box coordinates (see make_runs_tmap).
__device__ __forceinline__ void run_coords(uint64_t g, const RunBox& rb, int words, int (&c)[5]) {
#pragma unroll
  for (int d = 0; d < 5; ++d)
    c[d] = rb.gb[d] < 0 ? 0 : (int)((g >> rb.gb[d]) & ((uint64_t(1) << rb.len[d]) - 1)) * (d == 0 ? words : 1);
}
// The copy of the box of tile g (its first group) into shared memory at
// dst (one thread).
__device__ __forceinline__ void run_load(uint32_t dst, const CUtensorMap* map, uint64_t g, const RunBox& rb, int words,
                                         uint32_t mbar) {
  int c[5];
  run_coords(g, rb, words, c);
  switch (rb.rank) {
    case 2: tma_load_2d(dst, map, c[0], c[1], mbar); break;
    case 3: tma_load_3d(dst, map, c[0], c[1], c[2], mbar); break;
    case 4: tma_load_4d(dst, map, c, mbar); break;
    default: tma_load_5d(dst, map, c, mbar); break;
  }
}
__device__ __forceinline__ void run_store(const CUtensorMap* map, uint64_t g, const RunBox& rb, int words, uint32_t src) {
  int c[5];
  run_coords(g, rb, words, c);
  switch (rb.rank) {
    case 2: tma_store_2d(map, c[0], c[1], src); break;
    case 3: tma_store_3d(map, c[0], c[1], c[2], src); break;
    case 4: tma_store_4d(map, c, src); break;
    default: tma_store_5d(map, c, src); break;
  }
}
// Position of tile row r in the box (amplitudes).
__device__ __forceinline__ int run_row_pos(const RunBox& rb, int r) {
  int p = 0;
#pragma unroll
  for (int i = 0; i < 7; ++i) p += ((r >> i) & 1) * rb.multr[i];
  return p;
}
// Position of block index e0 + i for a compile-time i below 2^NB, e0 a
// multiple of 2^NB: base (the position of e0) plus the multipliers of i's
// bits, held in m[0 .. NB-1].
template <int NB>
__device__ __forceinline__ int run_elem_pos(int base, const int (&m)[NB], int i) {
  int p = base;
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if ((i >> j) & 1) p += m[j];
  return p;
}

}  // namespace qs
