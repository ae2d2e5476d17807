// Internal definitions shared by the CUDA translation units of libspm.
//
// Terminology used throughout:
//   write      one element write (row, col, value[, seq]) of the input stream
//   key        the paper's linear index row + col * n_rows (Section 3.3); its
//              order is column-major order, so sorting by key and walking the
//              result is the in-order traversal that the paper uses for the
//              conversion to CSC
//   cell       a fixed power-of-two range of keys (level-1 cells of 2^s1 keys;
//              hot cells may be refined into 256 level-2 cells)
//   leaf       a level-1 or level-2 cell that is not refined further; it is
//              split into 2^j equal buckets
//   bucket     an aligned power-of-two key range expected to hold a few
//              thousand writes; the unit of work of the per-bucket kernel
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "spm.h"

namespace spm {

// ---------------------------------------------------------------------------
// Fixed limits
// ---------------------------------------------------------------------------
constexpr int kMaxL1Smem = 12;            // level-1 LUT of at most 4096 cells in shared memory
constexpr int kL2Bits = 8;                // a level-2 table refines one cell into 256 cells
constexpr int kL2Size = 1 << kL2Bits;
constexpr int kMaxL2Tables = 32;          // level-2 tables per matrix
constexpr int kMaxKeyBits = 52;           // n_rows * n_cols <= 2^52
constexpr int kSubBitsMax = 12;           // counting-sort digit inside a bucket: up to 4096 sub-bins
constexpr int64_t kSampleTotal = 1 << 19; // samples drawn per call (spread over the matrices)
constexpr int64_t kSampleMin = 256;       // at least this many per matrix (or all of its writes)
// LUT entry: bit 31 = refers to a level-2 table (bits 0..30 = table id); otherwise bit 30 =
// merged group of 2^x cells, bits 25..29 = x (split exponent j, or group exponent g), bits
// 0..24 = first bucket of the leaf/group (relative to the matrix)
constexpr uint32_t kPtrFlag = 0x80000000u;
constexpr uint32_t kMergeFlag = 0x40000000u;
constexpr int kXShift = 25;
constexpr int kBaseBits = 25;
constexpr uint32_t kBaseMask = (1u << kBaseBits) - 1;
constexpr uint64_t kBadKey = ~0ull;       // sample sentinel for an out-of-range write
constexpr uint64_t kStAgg = 1ull << 62;   // look-back states of a bucket
constexpr uint64_t kStIncl = 2ull << 62;
constexpr uint64_t kStMask = (1ull << 62) - 1;
constexpr int kScanBlock = 1024;          // elements per block of the device-wide scan
constexpr int kLutCapSmem = 12288;        // LUT entries a partition block keeps in shared memory
constexpr int kHistCapSmem = 40960;       // bucket counters a partition block keeps in shared memory

// A partitioned write: key within its bucket, stream position, raw value bits
// (float32 values in the low half).  16 bytes, written with one vector store.
struct __align__(16) Rec {
  uint32_t lkey;
  uint32_t pos;
  uint64_t val;
};

// ---------------------------------------------------------------------------
// Per-matrix metadata (one entry per matrix of a batch; a single matrix is a
// batch of one).  Filled on the device; the host derives the same numbers
// from the same formulas to size the workspace and the launches.
// ---------------------------------------------------------------------------
struct MatMeta {
  int64_t t0;         // first write of this matrix in the concatenated stream
  int64_t m;          // writes of this matrix
  int64_t n_rows, n_cols;
  uint64_t K;         // n_rows * n_cols, the size of the key space
  int32_t bbits;      // smallest b with 2^b >= K
  int32_t L1;         // 2^L1 level-1 cells
  int32_t s1;         // level-1 cell of key = key >> s1
  int32_t H2;         // level-2 tables reserved
  int32_t h2used;     // level-2 tables used (set by the planner)
  int32_t pad;
  int64_t ns;         // samples drawn from this matrix
  int64_t samp_off;   // offset in the sample array
  int64_t lut_len;    // 2^L1 + 256*H2
  int64_t lut_off;    // offset in the LUT arrays
  int64_t l2_off;     // offset in the level-2 cell array
  int64_t col_base;   // offset of this matrix's col_ptr
  int64_t nbcap;      // bound on the number of buckets
  int64_t nbcap_off;
  int64_t nb;         // buckets (planner)
  int64_t bucket_off; // first bucket id (prefix of nb)
  int64_t lut_used_off; // prefix of the used LUT lengths (2^L1 + 256*h2used)
};

struct Derived {
  uint64_t K;
  int32_t bbits, L1, s1, H2;
  int64_t ns, lut_len, nbcap;
};

// Smallest b with 2^b >= x (0 for x <= 1).
__host__ __device__ inline int ceil_log2_u64(uint64_t x) {
  if (x <= 1) return 0;
#ifdef __CUDA_ARCH__
  return 64 - __clzll((long long)(x - 1));
#else
  return 64 - __builtin_clzll(x - 1);
#endif
}

// The sizing formulas (identical on host and device).
__host__ __device__ inline Derived derive(int64_t n_rows, int64_t n_cols, int64_t m, int64_t m_total,
                                          int64_t tgt) {
  Derived d;
  d.K = (uint64_t)n_rows * (uint64_t)n_cols;
  d.bbits = d.K <= 1 ? 0 : ceil_log2_u64(d.K);
  int L1 = 0;
  if (m > tgt) L1 = ceil_log2_u64((uint64_t)((m + tgt - 1) / tgt)) + 3;
  if (L1 > kMaxL1Smem) L1 = kMaxL1Smem;
  if (L1 < d.bbits - 32) L1 = d.bbits - 32;
  if (L1 > d.bbits) L1 = d.bbits;
  d.L1 = L1;
  d.s1 = d.bbits - L1;
  int64_t h = m / (16 * tgt);
  d.H2 = (d.s1 >= kL2Bits) ? (int32_t)(h < kMaxL2Tables ? h : kMaxL2Tables) : 0;
  d.lut_len = (int64_t{1} << L1) + (int64_t)d.H2 * kL2Size;
  if (m <= kSampleMin) {
    d.ns = m;
  } else {
    int64_t mt = m_total > 0 ? m_total : 1;
    int64_t s = (int64_t)(((unsigned long long)kSampleTotal * (unsigned long long)m) / (unsigned long long)mt);
    if (s < kSampleMin) s = kSampleMin;
    if (s > m) s = m;
    d.ns = s;
  }
  d.nbcap = d.lut_len + 4 * ((m + tgt - 1) / tgt) + 8;
  return d;
}

// Hash of one matrix's sizes, summed over the batch (wrapping) to check that
// the device copies of the batch description equal the host copies.
__host__ __device__ inline uint64_t meta_term(int64_t i, int64_t n_rows, int64_t n_cols, int64_t trip_end) {
  uint64_t x = (uint64_t)n_rows * 0x9E3779B97F4A7C15ull ^ (uint64_t)n_cols * 0xC2B2AE3D27D4EB4Full ^
               (uint64_t)trip_end * 0x165667B19E3779F9ull ^ (uint64_t)i * 0x27D4EB2F165667C5ull;
  x ^= x >> 31;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 29;
  return x;
}

// Boundaries of the write chunks handled by the partition blocks: multiples of
// four (vector loads) except the end.
__host__ __device__ inline int64_t chunk_begin(int64_t m_total, int64_t c, int64_t C) {
  if (c >= C) return m_total;
  return (int64_t)((((unsigned long long)m_total * (unsigned long long)c) / (unsigned long long)C) & ~3ull);
}

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
struct Layout {
  // sizes
  int64_t B, m_total, S_total, lut_total, l2_total, nbcap_total, hist_bound, C, scan_blocks;
  int sv;          // value bytes
  bool seq;
  // byte offsets
  size_t meta, scal, cta, samp, cellcnt, lut, l2cell, bk_lo, bk_info, bk_count, bk_start, bk_state,
      scanpart, hist, rec, tmp, rbk, bk_cur, l2h, bk_nnz, bk_out, big_list, total;
  int64_t l2h_len;  // one matrix with level-2 tables: sample counts of all level-2 cells
  bool two_pass;   // writes reach their buckets in two passes (through tmp/rbk)
};

// Device-side scalars block (in the workspace).
struct Scalars {
  uint32_t NB;        // total buckets
  uint32_t ticket;    // persistent-kernel work counter
  uint32_t abort;     // set when a fatal device error was recorded
  uint32_t G;         // two-pass partition: buckets per group (group g = buckets [g*G, (g+1)*G))
  unsigned long long fronts;  // (partition block, bucket) pairs with writes: the scatter's write fronts
  uint32_t ord_ticket;  // ordered single pass: next tile
  uint32_t ord_done;    // ordered single pass: tiles finished
  uint32_t ord_fail;    // ordered single pass: the stream is not in order (the general path runs)
  uint32_t ord_exit;    // ordered single pass: blocks that have left
  uint32_t big_n;       // buckets with more writes than the resolve holds (in big_list)
};

// Per partition block (chunk of writes) information.
struct CtaInfo {
  int64_t e0, e1;     // write range
  int64_t hoff;       // offset of its counters in the hist array
  int64_t l0, l1;     // LUT slice
  uint32_t cb0, cb1;  // bucket range
  int32_t i0, i1;     // matrix range
};

// Arguments of the assembly kernels.
struct Ctx {
  const int32_t* rows;
  const int32_t* cols;
  const void* vals;
  const uint64_t* seq;
  int64_t* col_ptr;
  int32_t* row_idx;
  void* out_vals;
  int64_t* d_nnz;
  int32_t* map;
  int32_t* status;
  // workspace views
  MatMeta* meta;
  Scalars* scal;
  CtaInfo* cta;
  uint64_t* samp;
  uint32_t* cellcnt;
  uint32_t* lut;
  int32_t* l2cell;
  uint64_t* bk_lo;
  uint32_t* bk_info;
  uint32_t* bk_count;
  uint32_t* bk_start;
  uint64_t* bk_state;
  uint32_t* scanpart;
  uint32_t* hist;
  Rec* rec;
  Rec* tmp;           // two-pass partition: records grouped by bucket group
  uint32_t* l2h;      // one matrix: sample counts of every level-2 cell (null: the planner counts)
  uint32_t* rbk;      // two-pass partition: bucket of each tmp record
  uint32_t* bk_cur;   // two-pass partition: next free slot of each bucket in rec
  uint32_t* bk_nnz;   // calls without the map: stored elements per bucket
  uint32_t* bk_out;   // ... their exclusive prefix over all buckets
  uint32_t* big_list; // ... the buckets placed by k_big
  // sizes
  int64_t B, m_total, S_total, lut_total, nbcap_total, hist_bound, C;
  int32_t sum_mode, f64, keep_map, has_seq;
  int64_t tgt;       // planner target (writes per bucket) for this call's mode
  int32_t sub_bits;
  int64_t withhold;   // bucket whose look-back publication is withheld (tests), -1 = none
  int32_t two_pass;   // partition in two passes
  int32_t groups;     // two-pass partition: number of bucket groups aimed at (>= 1)
  int64_t min_fronts; // two-pass partition: used only above this many write fronts
  int32_t keep_zeros; // last-write mode: elements whose value is zero are stored too
};

// Flag bit of the library's own calls (never accepted from the C ABI):
// last-write mode keeps elements whose final value is zero.
constexpr uint32_t kFlagKeepZeros = 1u << 30;

// The per-bucket resolve kernel (resolve.cu): writes a bucket may hold to be
// resolved from shared memory (fewer when the map is kept), its shared-memory
// attributes (set once per device) and its launches: the resolve kernel, then
// (calls without the map, after the scan of the per-bucket counts) the
// placement kernels.
int resolve_capacity(bool map);
void resolve_set_attributes();
void launch_resolve(const Ctx& ctx, int sms, int64_t nbcap, cudaStream_t st);
void launch_place(const Ctx& ctx, int sms, int64_t nbcap, cudaStream_t st);

// Launch counter of the library's kernels (spm_debug_launch_count).
void count_launches(int64_t n);

// Single pass for a stream already in column-major order (one matrix, no
// seq in last-write mode, no map): tiles of the stream, the look-back states
// in c.tmp (ordered_tiles(m) words, zeroed by the caller).
int64_t ordered_tiles(int64_t m);
cudaError_t launch_ordered(const Ctx& c, int64_t n_rows, int64_t n_cols, int sms, cudaStream_t st);

// spm_assemble_csc for the library's own calls: `flags` may hold
// kFlagKeepZeros.
spm_status assemble_internal(int64_t n_rows, int64_t n_cols, int64_t m, const int32_t* rows, const int32_t* cols,
                             const void* vals, const uint64_t* seq, spm_dtype dtype, spm_mode mode, uint32_t flags,
                             int64_t* col_ptr, int32_t* row_idx, void* out_vals, int64_t* d_nnz, int32_t* d_status,
                             void* workspace, size_t ws_bytes, void* stream);

}  // namespace spm
