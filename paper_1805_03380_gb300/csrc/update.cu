// Batch insertion into an existing CSC matrix: Section 3.1 (the elements to
// be inserted are sorted first and then merged with the existing arrays) and
// Section 3.4 (element writes made while the matrix is held in CSC, synced
// back into CSC).
//
// Steps on the GPU, all enqueued on the caller's stream:
//   1. The new writes are assembled on their own into a CSC matrix B (the
//      library's assembly; in last-write mode B keeps elements whose value is
//      zero, because such a write removes an existing element).
//   2. k_check_cp: A's column offsets must run from 0 to nnz_a without
//      decreasing (else SPM_ERR_INVALID_ARG).
//   3. k_split: A and B are both ordered by the linear index
//      row + col * n_rows (Section 3.3), so the result is one merge of two
//      sorted sequences.  The merged sequence is cut into tiles of kTile
//      positions; each cut is found by a binary search over the column starts
//      of the merged sequence (A's start plus B's start of every column)
//      followed by a merge-path search inside the column.  A cut that would
//      separate an element of A from the write to the same element in B
//      moves one position on.
//   4. k_merge: one block per tile (taken in order through a ticket) merges
//      its part of A and B in shared memory -- column by column with 32-bit
//      row compares when the columns starting inside the tile fit a table,
//      else on 64-bit linear indices -- combines an element present in
//      both (last-write mode: B's value; add mode: A's value + B's value),
//      drops zeros, finds the tile's output offset by a bounded decoupled
//      look-back and writes the stored elements and the column offsets of the
//      columns that start inside the tile.  It also checks that A is
//      canonical (rows inside [0, n_rows), strictly increasing inside a
//      column).
//
// The same cuts and tiles compute trace(A^T B) for two CSC matrices of one
// shape (Section 2: the expression is evaluated without forming the
// transpose or the product, by accumulating only the diagonal of A^T B, which
// is the sum over the elements stored in both of A(i,j) * B(i,j); Fig. 1b).
// k_merge in its dot form multiplies the pairs of each tile and writes one
// partial sum per tile; k_dot_sum adds them in tile order.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "spm.h"
#include "spm_common.cuh"

namespace {

constexpr int kMT = 256;                      // threads per merge block
constexpr int kMI = 8;                        // merged positions per thread
constexpr int kTileCap = kMT * kMI;           // positions a block holds
constexpr int64_t kTile = kTileCap - 1;       // nominal positions per tile (a moved cut adds one)
constexpr unsigned kAll = 0xffffffffu;
constexpr uint64_t kAgg = 1ull << 62;         // tile look-back states
constexpr uint64_t kIncl = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr uint64_t kWaitNs = 2000000000ull;   // look-back wait limit
constexpr int kOpSet = 0, kOpSum = 1, kOpDot = 2;

size_t align256(size_t x) { return (x + 255) & ~size_t{255}; }

// A cut of the merged sequence: elements [0, a) of A and [0, b) of B lie
// before it, and j is the first column whose merged start is at or after it.
struct Cut {
  int64_t a, b, j, pad;
};

struct UScal {
  int64_t nnz_b;    // stored elements of B (written by the assembly)
  uint32_t ticket;  // next tile for k_merge
  int32_t go;       // k_merge runs only if nothing failed before it
  int32_t bad_a;    // k_split: two of A's elements out of order across a cut
  int32_t pad;
};

struct UpdateLayout {
  size_t cp_b, row_b, val_b, scal, cuts, state, assembly, total;
  size_t asm_bytes;
  int64_t tiles_max;
};

int64_t tiles_upper(int64_t nnz_a, int64_t m) { return (nnz_a + m) / kTile + 1; }

spm_status update_layout(int64_t n_rows, int64_t n_cols, int64_t nnz_a, int64_t m, spm_dtype dtype, spm_mode mode,
                         uint32_t flags, UpdateLayout& L) {
  if (nnz_a < 0 || m < 0 || n_rows < 0 || n_cols < 0) return SPM_ERR_INVALID_ARG;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  if (mode != SPM_MODE_LAST_WRITE && mode != SPM_MODE_SUM) return SPM_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)(SPM_CHECK_BOUNDS | SPM_SEQ_EXPLICIT)) return SPM_ERR_INVALID_ARG;  // no map
  if (nnz_a > (int64_t)INT32_MAX * 2 || nnz_a + m >= (int64_t{1} << 32) - 64) return SPM_ERR_UNSUPPORTED;
  size_t ab = 0;
  const spm_status s = spm_assemble_csc_workspace(n_rows, n_cols, m, dtype, mode, flags, &ab);
  if (s != SPM_OK) return s;
  const size_t sv = dtype == SPM_F64 ? 8 : 4;
  const size_t mm = (size_t)std::max<int64_t>(m, 1);
  L.tiles_max = tiles_upper(nnz_a, m);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.cp_b = take(8 * ((size_t)n_cols + 1));
  L.row_b = take(4 * mm);
  L.val_b = take(sv * mm);
  L.scal = take(sizeof(UScal));
  L.cuts = take(sizeof(Cut) * ((size_t)L.tiles_max + 1));
  L.state = take(8 * (size_t)L.tiles_max);
  L.assembly = take(ab);
  L.asm_bytes = ab;
  L.total = o;
  return SPM_OK;
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint64_t load_acquire(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void store_release(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void fail(int32_t* status, int code) { atomicCAS(status, 0, code); }

// A's column offsets: 0 at the start, nnz_a at the end, never decreasing.
__global__ void k_check_cp(const int64_t* __restrict__ cp, int64_t n_cols, int64_t nnz_a, int32_t* status) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > n_cols) return;
  const int64_t v = cp[j];
  bool ok = v >= 0 && v <= nnz_a;
  if (j == 0) ok = ok && v == 0;
  if (j == n_cols) ok = ok && v == nnz_a;
  if (j < n_cols) ok = ok && cp[j + 1] >= v;
  if (!ok) fail(status, SPM_ERR_INVALID_ARG);
}

struct MergeArgs {
  int64_t n_rows, n_cols, nnz_a;
  const int64_t* cp_a;
  const int32_t* row_a;
  const void* val_a;
  const int64_t* cp_b;
  const int32_t* row_b;
  const void* val_b;
  UScal* scal;
  Cut* cuts;
  uint64_t* state;
  int64_t* col_ptr;
  int32_t* row_out;
  void* val_out;
  int64_t* d_nnz;
  int32_t* status;
  double* partial;  // trace: one partial sum per tile
  int32_t check_b;  // B is an input (the trace): check that it is canonical too
};

// Merged start of column j: its elements in A before it plus those in B.
__device__ __forceinline__ int64_t merged_start(const MergeArgs& a, int64_t j) { return a.cp_a[j] + a.cp_b[j]; }

// One thread per cut t = 0 .. tiles (tiles = L / kTile + 1, L = nnz_a + nnz_b).
__global__ void k_split(MergeArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (*reinterpret_cast<volatile int32_t*>(a.status) != 0) {  // the assembly of B or the offset check failed
    if (t == 0) a.scal->go = 0;
    return;
  }
  if (t == 0) a.scal->go = 1;
  const int64_t nnz_b = a.cp_b[a.n_cols];
  const int64_t L = a.nnz_a + nnz_b;
  const int64_t tiles = L / kTile + 1;
  if (t > tiles) return;
  const int64_t d = std::min(t * kTile, L);
  int64_t ia = a.nnz_a, ib = nnz_b;
  int64_t jhi = a.n_cols;  // the first column starting at or after the cut is at most this
  if (d < L) {
    // column c holding merged position d: the last column whose merged start is <= d
    int64_t lo = 1, hi = a.n_cols;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (merged_start(a, mid) > d) hi = mid; else lo = mid + 1;
    }
    const int64_t c = lo - 1;
    const int64_t a0 = a.cp_a[c], b0 = a.cp_b[c];
    const int64_t len_a = a.cp_a[c + 1] - a0, len_b = a.cp_b[c + 1] - b0;
    const int64_t off = d - (a0 + b0);
    // merge path inside the column: how many of A's rows come first (A first on equal rows)
    int64_t l2 = std::max<int64_t>(0, off - len_b), h2 = std::min(off, len_a);
    while (l2 < h2) {
      const int64_t mid = (l2 + h2) >> 1;
      if (a.row_a[a0 + mid] <= a.row_b[b0 + off - 1 - mid]) l2 = mid + 1; else h2 = mid;
    }
    ia = a0 + l2;
    ib = b0 + off - l2;
    // keep an element of A and the write to the same element in one tile
    if (l2 > 0 && off - l2 < len_b && a.row_a[ia - 1] == a.row_b[ib]) ++ib;
    // A's elements on either side of the cut, if in one column, must have increasing rows
    // (k_merge checks the pairs inside a tile)
    if (l2 > 0 && l2 < len_a && a.row_a[ia - 1] >= a.row_a[ia]) atomicExch(&a.scal->bad_a, (int)SPM_ERR_INVALID_ARG);
    if (a.check_b && ib > b0 && ib < b0 + len_b && a.row_b[ib - 1] >= a.row_b[ib])
      atomicExch(&a.scal->bad_a, (int)SPM_ERR_INVALID_ARG);
    // column c starts before the cut unless the cut is its start: then the
    // answer is c + 1, else it lies in [0, c]
    jhi = (a0 + b0 < ia + ib) ? c + 1 : c;
  }
  const int64_t cut = ia + ib;
  // first column whose merged start is at or after the cut
  int64_t lo = 0, hi = jhi;
  if (d < L && jhi > 0 && merged_start(a, jhi - 1) < cut) lo = jhi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (merged_start(a, mid) >= cut) hi = mid; else lo = mid + 1;
  }
  a.cuts[t] = Cut{ia, ib, lo, 0};
}

template <typename VT>
__device__ __forceinline__ VT combine_add(VT x, VT y);
template <>
__device__ __forceinline__ uint32_t combine_add<uint32_t>(uint32_t x, uint32_t y) {
  return __float_as_uint(__fadd_rn(__uint_as_float(x), __uint_as_float(y)));
}
template <>
__device__ __forceinline__ uint64_t combine_add<uint64_t>(uint64_t x, uint64_t y) {
  return (uint64_t)__double_as_longlong(__dadd_rn(__longlong_as_double((long long)x), __longlong_as_double((long long)y)));
}

template <typename VT>
__device__ __forceinline__ double as_double(VT bits) {
  return sizeof(VT) == 8 ? __longlong_as_double((long long)bits) : (double)__uint_as_float((uint32_t)bits);
}

template <typename VT>
__device__ __forceinline__ bool nonzero(VT bits) {
  return sizeof(VT) == 8 ? ((uint64_t)bits & 0x7FFFFFFFFFFFFFFFull) != 0 : ((uint32_t)bits & 0x7FFFFFFFu) != 0;
}

template <typename VT>
constexpr size_t merge_smem_bytes() {
  return (size_t)kTileCap * (8 + sizeof(VT) + 4);
}

// OP: kOpSet / kOpSum merge A with the resolved writes B (the update);
// kOpDot accumulates the products of the elements present in both (the trace).
template <typename VT, int OP>
__global__ void __launch_bounds__(kMT, 5) k_merge(MergeArgs a) {
  constexpr bool SUM = OP == kOpSum;
  extern __shared__ __align__(16) unsigned char smem[];
  // key: keys (A's part, then B's part), then the output rows (int32);
  // aux: the column of each element
  uint64_t* key = reinterpret_cast<uint64_t*>(smem);
  VT* val = reinterpret_cast<VT*>(key + kTileCap);
  int32_t* aux = reinterpret_cast<int32_t*>(val + kTileCap);
  __shared__ int32_t s_wtot[kMT / 32];
  __shared__ int64_t s_tile, s_excl;
  __shared__ int32_t s_bad;
  __shared__ int32_t s_ta[kMT], s_tb[kMT];  // column starts inside the tile, relative to A's and B's part
  __shared__ int32_t s_texcl[kMT];          // per thread: output slot of its first kept element
  __shared__ uint32_t s_tmask[kMT];         // per thread: which of its positions are kept

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(&a.scal->ticket, 1u);
    s_bad = 0;
  }
  const int go = *reinterpret_cast<volatile int32_t*>(&a.scal->go);
  const int64_t L = a.nnz_a + a.cp_b[a.n_cols];
  __syncthreads();
  if (!go) return;
  const int64_t tiles = L / kTile + 1;
  const int64_t t = s_tile;
  if (t >= tiles) return;
  const bool last = t == tiles - 1;
  const Cut c0 = a.cuts[t], c1 = a.cuts[t + 1];
  int64_t nA = c1.a - c0.a, nB = c1.b - c0.b;
  if (nA < 0 || nB < 0 || nA + nB > kTileCap) {  // only when A's rows are not sorted
    if (tid == 0) fail(a.status, SPM_ERR_INVALID_ARG);
    nA = nB = 0;
  }
  const int n = (int)(nA + nB);
  const int64_t bd = c0.a + c0.b;  // merged position of the tile's first element
  const int64_t jlo = c0.j, jend = last ? a.n_cols + 1 : c1.j;
  const VT* va = static_cast<const VT*>(a.val_a);
  const VT* vb = static_cast<const VT*>(a.val_b);

  // every global load the tile needs before the merge, issued together: its
  // part of A and B and the column starts inside it
  int32_t lr[kMI];
  VT lv[kMI];
#pragma unroll
  for (int i = 0; i < kMI; ++i) {
    const int k = tid + i * kMT;
    lr[i] = 0;
    lv[i] = 0;
    if (k < nA) {
      lr[i] = __ldg(a.row_a + c0.a + k);
      lv[i] = __ldg(va + c0.a + k);
    } else if (k < n) {
      lr[i] = __ldg(a.row_b + c0.b + (k - nA));
      lv[i] = __ldg(vb + c0.b + (k - nA));
    }
  }
  // the column starts inside the tile (nc of them): a table in shared
  // memory when they are few, else read from global memory
  const int64_t jcap = jend < a.n_cols ? jend : a.n_cols;
  const int nc = (int)(jcap > jlo ? (jcap - jlo < INT_MAX ? jcap - jlo : INT_MAX) : 0);
  const bool table = nc <= kMT;
  const int64_t j0 = jlo + tid;
  int64_t cpa0 = 0, cpb0 = 0;
  if (j0 < jend) {
    cpa0 = a.cp_a[j0];
    cpb0 = a.cp_b[j0];
  }
  auto clamp_rel = [](int64_t v) { return (int32_t)(v < -1 ? -1 : (v > kTileCap + 1 ? kTileCap + 1 : v)); };
  if (table && j0 < jcap) {
    s_ta[tid] = clamp_rel(cpa0 - c0.a);
    s_tb[tid] = clamp_rel(cpb0 - c0.b);
  }
  // values (and, for the column-by-column merge, rows) to shared memory; A
  // (and B when it is an input) must be canonical: rows inside the matrix
  int bad = 0;
#pragma unroll
  for (int i = 0; i < kMI; ++i) {
    const int k = tid + i * kMT;
    if (k < n) {
      val[k] = lv[i];
      if (table) aux[k] = lr[i];
      if ((k < nA || a.check_b) && (lr[i] < 0 || (int64_t)lr[i] >= a.n_rows)) bad = SPM_ERR_INDEX_OUT_OF_RANGE;
    }
  }
  if (bad) atomicMax(&s_bad, bad);
  __syncthreads();

  // each thread merges kMI consecutive positions (A first on equal rows of a column)
  const int p0 = min(tid * kMI, n);
  int32_t orow[kMI];
  VT oval[kMI];
  uint32_t kmask = 0;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kMI; ++k) {
    orow[k] = 0;
    oval[k] = 0;
  }
  if (table) {
    // Column by column: the merged tile is column jlo - 1 (from the tile's
    // start) and then the columns starting inside it, each the merge of its
    // rows in A and in B; rows are compared as 32-bit integers.
    // Segment q = 0 is column jlo - 1; q >= 1 is column jlo + q - 1.
    const int32_t* rowA = aux;
    const int32_t* rowB = aux + nA;
    const int nAi = (int)nA, nBi = (int)nB;
    auto sa = [&](int q) -> int {
      const int v = q == 0 ? 0 : s_ta[q - 1];
      return v < 0 ? 0 : (v > nAi ? nAi : v);
    };
    auto sb = [&](int q) -> int {
      const int v = q == 0 ? 0 : s_tb[q - 1];
      return v < 0 ? 0 : (v > nBi ? nBi : v);
    };
    // the segment holding merged position p0: the last one that starts at or before it
    int lo = 0, hi = nc;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sa(mid) + sb(mid) <= p0) lo = mid; else hi = mid - 1;
    }
    int q = lo;
    int aS = sa(q), bS = sb(q);
    int aE = q < nc ? sa(q + 1) : nAi, bE = q < nc ? sb(q + 1) : nBi;
    aE = aE < aS ? aS : aE;  // (only a malformed A breaks the order)
    bE = bE < bS ? bS : bE;
    int off = p0 - (aS + bS);
    const int seg = (aE - aS) + (bE - bS);
    off = off < 0 ? 0 : (off > seg ? seg : off);
    int l2 = max(0, off - (bE - bS)), h2 = min(off, aE - aS);
    while (l2 < h2) {
      const int mid = (l2 + h2) >> 1;
      if (rowA[aS + mid] <= rowB[bS + off - 1 - mid]) l2 = mid + 1; else h2 = mid;
    }
    int ia = aS + l2, ib = bS + off - l2;
    bool bad_order = false;
#pragma unroll
    for (int k = 0; k < kMI; ++k) {
      if (p0 + k < n) {
        while (ia >= aE && ib >= bE && q < nc) {  // this column is done: the next one
          ++q;
          aS = aE;
          bS = bE;
          aE = q < nc ? sa(q + 1) : nAi;
          bE = q < nc ? sb(q + 1) : nBi;
          aE = aE < aS ? aS : aE;
          bE = bE < bS ? bS : bE;
        }
        if (ia >= aE && ib >= bE) break;  // (only a malformed A)
        const bool take_a = ib >= bE || (ia < aE && rowA[ia] <= rowB[ib]);
        if (take_a) {
          const int32_t r = rowA[ia];
          if (ia > aS && rowA[ia - 1] >= r) bad_order = true;
          const bool pair = ib < bE && rowB[ib] == r;
          if (OP == kOpDot) {
            if (pair) acc = fma(as_double<VT>(val[ia]), as_double<VT>(val[nA + ib]), acc);
          } else {
            VT v = val[ia];
            if (pair) v = SUM ? combine_add<VT>(v, val[nA + ib]) : val[nA + ib];
            orow[k] = r;
            oval[k] = v;
            if (nonzero<VT>(v)) kmask |= 1u << k;
          }
          ++ia;
        } else {
          const int32_t r = rowB[ib];
          if (a.check_b && ib > bS && rowB[ib - 1] >= r) bad_order = true;
          if (OP != kOpDot) {
            const bool tail = ia > aS && rowA[ia - 1] == r;  // B's half of a combined element
            const VT v = val[nA + ib];
            orow[k] = r;
            oval[k] = v;
            if (!tail && nonzero<VT>(v)) kmask |= 1u << k;
          }
          ++ib;
        }
      }
    }
    if (bad_order) atomicMax(&s_bad, (int32_t)SPM_ERR_INVALID_ARG);
  } else {
    // Many columns start inside the tile: the column of every element from a
    // search over the column offsets, then 64-bit linear indices.
    const uint64_t nr = (uint64_t)a.n_rows;
#pragma unroll
    for (int i = 0; i < kMI; ++i) {
      const int k = tid + i * kMT;
      if (k < n) {
        const bool in_a = k < nA;
        const int32_t rel = in_a ? k : k - (int)nA;
        const int64_t* cp = (in_a ? a.cp_a : a.cp_b) + jlo;
        const int64_t base = (in_a ? c0.a : c0.b) + rel;
        int lo = 0, hi = nc;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (cp[mid] <= base) lo = mid + 1; else hi = mid;
        }
        const int32_t col = (int32_t)(jlo - 1 + lo);
        aux[k] = col;
        key[k] = (uint64_t)(uint32_t)col * nr + (uint64_t)(uint32_t)lr[i];
      }
    }
    __syncthreads();
    // strictly increasing linear indices inside A's part of the tile (and
    // B's when it is an input); k_split checks the pairs on either side of each cut
#pragma unroll
    for (int i = 0; i < kMI; ++i) {
      const int k = tid + i * kMT;
      if (k > 0 && k < nA && key[k] <= key[k - 1]) atomicMax(&s_bad, (int32_t)SPM_ERR_INVALID_ARG);
      if (a.check_b && k > nA && k < n && key[k] <= key[k - 1]) atomicMax(&s_bad, (int32_t)SPM_ERR_INVALID_ARG);
    }
    int lo = max(0, p0 - (int)nB), hi = min(p0, (int)nA);
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (key[mid] <= key[nA + p0 - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    int ia = lo, ib = p0 - lo;
#pragma unroll
    for (int k = 0; k < kMI; ++k) {
      if (p0 + k < n) {
        const bool take_a = ib >= nB || (ia < nA && key[ia] <= key[nA + ib]);
        if (take_a) {
          const bool pair = ib < nB && key[nA + ib] == key[ia];
          if (OP == kOpDot) {
            if (pair) acc = fma(as_double<VT>(val[ia]), as_double<VT>(val[nA + ib]), acc);
          } else {
            VT v = val[ia];
            if (pair) v = SUM ? combine_add<VT>(v, val[nA + ib]) : val[nA + ib];
            orow[k] = (int32_t)(key[ia] - (uint64_t)(uint32_t)aux[ia] * nr);
            oval[k] = v;
            if (nonzero<VT>(v)) kmask |= 1u << k;
          }
          ++ia;
        } else {
          const int src = (int)nA + ib;
          if (OP != kOpDot) {
            const bool tail = ia > 0 && key[ia - 1] == key[src];  // B's half of a combined element
            const VT v = val[src];
            orow[k] = (int32_t)(key[src] - (uint64_t)(uint32_t)aux[src] * nr);
            oval[k] = v;
            if (!tail && nonzero<VT>(v)) kmask |= 1u << k;
          }
          ++ib;
        }
      }
    }
  }
  if (OP == kOpDot) {
    // the tile's sum of products
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kAll, acc, o);
    __shared__ double s_part[kMT / 32];
    if (lane == 0) s_part[w] = acc;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int u = 0; u < kMT / 32; ++u) sum += s_part[u];
      a.partial[t] = sum;
      if (s_bad) fail(a.status, s_bad);
    }
    return;
  }
  // exclusive scan of the kept counts over the block
  const int cnt = __popc(kmask);
  int inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kAll, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();  // everyone is done reading the tile (key, val and aux are reused below)
  if (lane == 31) s_wtot[w] = inc;
  __syncthreads();
  int wpre = 0, total = 0;
  for (int u = 0; u < kMT / 32; ++u) {
    if (u < w) wpre += s_wtot[u];
    total += s_wtot[u];
  }
  const int excl_t = wpre + inc - cnt;
  // each thread's first output slot and kept mask (the column offsets read
  // them); the kept elements staged in output order
  s_texcl[tid] = excl_t;
  s_tmask[tid] = kmask;
  int32_t* srow = reinterpret_cast<int32_t*>(key);
#pragma unroll
  for (int k = 0; k < kMI; ++k)
    if (kmask & (1u << k)) {
      const int o = excl_t + __popc(kmask & ((1u << k) - 1u));
      srow[o] = orow[k];
      val[o] = oval[k];
    }

  // the tile's output offset: decoupled look-back over earlier tiles (bounded wait)
  if (w == 0) {
    int64_t excl = 0;
    if (t == 0) {
      if (lane == 0) store_release(&a.state[0], kIncl | (uint64_t)total);
    } else {
      if (lane == 0) store_release(&a.state[t], kAgg | (uint64_t)total);
      __syncwarp();
      int64_t top = t - 1;
      const uint64_t t_start = now_ns();
      uint32_t spins = 0;
      while (true) {
        const int64_t bb = top - lane;
        const uint64_t s = bb >= 0 ? load_acquire(&a.state[bb]) : kIncl;
        const uint64_t flag = s & ~kValMask;
        const unsigned incl = __ballot_sync(kAll, flag == kIncl);
        const unsigned none = __ballot_sync(kAll, flag == 0);
        const int first = incl ? __ffs(incl) - 1 : 32;
        const unsigned upto = first >= 31 ? kAll : ((2u << first) - 1u);
        if ((none & upto) == 0) {
          uint64_t v = lane <= first ? (s & kValMask) : 0ull;
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
          excl += (int64_t)v;
          if (first < 32) break;
          top -= 32;
          continue;
        }
        __nanosleep(64);
        int stop = 0;
        if (lane == 0 && (++spins & 7) == 0 && now_ns() - t_start > kWaitNs) {
          fail(a.status, SPM_ERR_TIMEOUT);
          stop = 1;
        }
        if (__shfl_sync(kAll, stop, 0)) break;
      }
      if (lane == 0) store_release(&a.state[t], kIncl | (uint64_t)(excl + total));
    }
    if (lane == 0) s_excl = excl;
  }
  __syncthreads();
  const int64_t excl = s_excl;
  VT* vo = static_cast<VT*>(a.val_out);
  for (int k = tid; k < total; k += kMT) {
    a.row_out[excl + k] = srow[k];
    vo[excl + k] = val[k];
  }
  // column offsets of the columns that start inside this tile
  for (int64_t j = j0; j < jend; j += kMT) {
    int64_t p = (j == j0 ? cpa0 + cpb0 : merged_start(a, j)) - bd;
    p = p < 0 ? 0 : (p > n ? n : p);
    int before = total;  // elements kept before merged position p of the tile
    if (p < n) {
      const int th = (int)p / kMI, k = (int)p % kMI;
      before = s_texcl[th] + __popc(s_tmask[th] & ((1u << k) - 1u));
    }
    a.col_ptr[j] = excl + before;
  }
  if (last && tid == 0) {
    *a.d_nnz = excl + total;
    if (a.scal->bad_a) fail(a.status, a.scal->bad_a);
  }
  if (tid == 0 && s_bad) fail(a.status, s_bad);
}

// The shared-memory limit of the six k_merge instances, raised once per device.
bool g_merge_ready[64] = {};
std::mutex g_merge_mutex;

cudaError_t merge_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (g_merge_ready[dev]) return cudaSuccess;
  std::lock_guard<std::mutex> lk(g_merge_mutex);
  if (g_merge_ready[dev]) return cudaSuccess;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const int s64 = (int)merge_smem_bytes<uint64_t>(), s32 = (int)merge_smem_bytes<uint32_t>();
  if ((e = cudaFuncSetAttribute(k_merge<uint64_t, kOpSet>, a, s64)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_merge<uint64_t, kOpSum>, a, s64)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_merge<uint64_t, kOpDot>, a, s64)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_merge<uint32_t, kOpSet>, a, s32)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_merge<uint32_t, kOpSum>, a, s32)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_merge<uint32_t, kOpDot>, a, s32)) != cudaSuccess) return e;
  g_merge_ready[dev] = true;
  return cudaSuccess;
}

template <typename VT, int OP>
cudaError_t launch_merge(const MergeArgs& args, int64_t tiles_max, cudaStream_t st) {
  const cudaError_t e = merge_prepare();
  if (e != cudaSuccess) return e;
  k_merge<VT, OP><<<(unsigned)tiles_max, kMT, merge_smem_bytes<VT>(), st>>>(args);
  return cudaGetLastError();
}

// The trace: the sum of the tiles' partial sums, in tile order (one block,
// so the result does not depend on timing), and the checks of k_split.
__global__ void __launch_bounds__(1024) k_dot_sum(MergeArgs a, double* result) {
  __shared__ double s_w[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int go = a.scal->go;
  double acc = 0.0;
  if (go) {
    const int64_t L = a.nnz_a + a.cp_b[a.n_cols];
    const int64_t tiles = L / kTile + 1;
    for (int64_t t = tid; t < tiles; t += blockDim.x) acc += a.partial[t];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kAll, acc, o);
  if (lane == 0) s_w[w] = acc;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int u = 0; u < (int)(blockDim.x / 32); ++u) sum += s_w[u];
    *result = go ? sum : 0.0;
    if (a.scal->bad_a) fail(a.status, a.scal->bad_a);
  }
}

}  // namespace

extern "C" {

spm_status spm_csc_update_workspace(int64_t n_rows, int64_t n_cols, int64_t nnz_a, int64_t m, spm_dtype dtype,
                                    spm_mode mode, uint32_t flags, size_t* bytes) {
  if (!bytes) return SPM_ERR_INVALID_ARG;
  UpdateLayout L;
  const spm_status s = update_layout(n_rows, n_cols, nnz_a, m, dtype, mode, flags, L);
  if (s != SPM_OK) return s;
  *bytes = L.total;
  return SPM_OK;
}

spm_status spm_csc_update(int64_t n_rows, int64_t n_cols, const int64_t* a_col_ptr, const int32_t* a_row_idx,
                          const void* a_vals, int64_t nnz_a, int64_t m, const int32_t* rows, const int32_t* cols,
                          const void* vals, const uint64_t* seq, spm_dtype dtype, spm_mode mode, uint32_t flags,
                          int64_t* col_ptr, int32_t* row_idx, void* out_vals, int64_t* d_nnz, int32_t* d_status,
                          void* workspace, size_t ws_bytes, void* stream) {
  UpdateLayout L;
  spm_status s = update_layout(n_rows, n_cols, nnz_a, m, dtype, mode, flags, L);
  if (s != SPM_OK) return s;
  const bool has_seq = (flags & SPM_SEQ_EXPLICIT) != 0;
  if (has_seq != (seq != nullptr)) return SPM_ERR_INVALID_ARG;
  if (!a_col_ptr || !col_ptr || !d_nnz || !d_status) return SPM_ERR_INVALID_ARG;
  if (nnz_a > 0 && (!a_row_idx || !a_vals)) return SPM_ERR_INVALID_ARG;
  if (m > 0 && (!rows || !cols || !vals)) return SPM_ERR_INVALID_ARG;
  if (nnz_a + m > 0 && (!row_idx || !out_vals)) return SPM_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < L.total) return SPM_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  MergeArgs a = {};
  a.n_rows = n_rows;
  a.n_cols = n_cols;
  a.nnz_a = nnz_a;
  a.cp_a = a_col_ptr;
  a.row_a = a_row_idx;
  a.val_a = a_vals;
  a.cp_b = reinterpret_cast<int64_t*>(ws + L.cp_b);
  a.row_b = reinterpret_cast<int32_t*>(ws + L.row_b);
  a.val_b = ws + L.val_b;
  a.scal = reinterpret_cast<UScal*>(ws + L.scal);
  a.cuts = reinterpret_cast<Cut*>(ws + L.cuts);
  a.state = reinterpret_cast<uint64_t*>(ws + L.state);
  a.col_ptr = col_ptr;
  a.row_out = row_idx;
  a.val_out = out_vals;
  a.d_nnz = d_nnz;
  a.status = d_status;
  cudaMemsetAsync(a.scal, 0, sizeof(UScal), st);
  cudaMemsetAsync(a.state, 0, 8 * (size_t)L.tiles_max, st);
  // 1. B: the new writes on their own (sets d_status to SPM_OK first)
  const uint32_t bflags = flags | (mode == SPM_MODE_LAST_WRITE ? spm::kFlagKeepZeros : 0u);
  s = spm::assemble_internal(n_rows, n_cols, m, rows, cols, vals, seq, dtype, mode, bflags, const_cast<int64_t*>(a.cp_b),
                             const_cast<int32_t*>(a.row_b), const_cast<void*>(a.val_b), &a.scal->nnz_b, d_status,
                             ws + L.assembly, L.asm_bytes, stream);
  if (s != SPM_OK) return s;
  // 2.-4. check A's offsets, cut the merged sequence, merge
  k_check_cp<<<(unsigned)((n_cols + 1 + 255) / 256), 256, 0, st>>>(a_col_ptr, n_cols, nnz_a, d_status);
  k_split<<<(unsigned)((L.tiles_max + 1 + 255) / 256), 256, 0, st>>>(a);
  cudaError_t e;
  if (dtype == SPM_F64)
    e = mode == SPM_MODE_SUM ? launch_merge<uint64_t, kOpSum>(a, L.tiles_max, st)
                             : launch_merge<uint64_t, kOpSet>(a, L.tiles_max, st);
  else
    e = mode == SPM_MODE_SUM ? launch_merge<uint32_t, kOpSum>(a, L.tiles_max, st)
                             : launch_merge<uint32_t, kOpSet>(a, L.tiles_max, st);
  spm::count_launches(3);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return SPM_ERR_CUDA;
  return SPM_OK;
}

namespace {

struct TraceLayout {
  size_t scal, cuts, partial, total;
  int64_t tiles_max;
};

spm_status trace_layout(int64_t n_cols, int64_t nnz_a, int64_t nnz_b, TraceLayout& L) {
  if (n_cols < 0 || nnz_a < 0 || nnz_b < 0) return SPM_ERR_INVALID_ARG;
  if (n_cols > INT32_MAX || nnz_a + nnz_b >= (int64_t{1} << 40)) return SPM_ERR_UNSUPPORTED;
  L.tiles_max = tiles_upper(nnz_a, nnz_b);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.scal = take(sizeof(UScal));
  L.cuts = take(sizeof(Cut) * ((size_t)L.tiles_max + 1));
  L.partial = take(8 * (size_t)L.tiles_max);
  L.total = o;
  return SPM_OK;
}

}  // namespace

spm_status spm_csc_trace_atb_workspace(int64_t n_cols, int64_t nnz_a, int64_t nnz_b, size_t* bytes) {
  if (!bytes) return SPM_ERR_INVALID_ARG;
  TraceLayout L;
  const spm_status s = trace_layout(n_cols, nnz_a, nnz_b, L);
  if (s != SPM_OK) return s;
  *bytes = L.total;
  return SPM_OK;
}

spm_status spm_csc_trace_atb(int64_t n_rows, int64_t n_cols, const int64_t* a_col_ptr, const int32_t* a_row_idx,
                             const void* a_vals, int64_t nnz_a, const int64_t* b_col_ptr, const int32_t* b_row_idx,
                             const void* b_vals, int64_t nnz_b, spm_dtype dtype, double* d_result, int32_t* d_status,
                             void* workspace, size_t ws_bytes, void* stream) {
  TraceLayout L;
  spm_status s = trace_layout(n_cols, nnz_a, nnz_b, L);
  if (s != SPM_OK) return s;
  if (n_rows < 0) return SPM_ERR_INVALID_ARG;
  if (n_rows > INT32_MAX) return SPM_ERR_UNSUPPORTED;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  if (!a_col_ptr || !b_col_ptr || !d_result || !d_status) return SPM_ERR_INVALID_ARG;
  if ((nnz_a > 0 && (!a_row_idx || !a_vals)) || (nnz_b > 0 && (!b_row_idx || !b_vals))) return SPM_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < L.total) return SPM_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  MergeArgs a = {};
  a.n_rows = n_rows;
  a.n_cols = n_cols;
  a.nnz_a = nnz_a;
  a.cp_a = a_col_ptr;
  a.row_a = a_row_idx;
  a.val_a = a_vals;
  a.cp_b = b_col_ptr;
  a.row_b = b_row_idx;
  a.val_b = b_vals;
  a.scal = reinterpret_cast<UScal*>(ws + L.scal);
  a.cuts = reinterpret_cast<Cut*>(ws + L.cuts);
  a.partial = reinterpret_cast<double*>(ws + L.partial);
  a.status = d_status;
  a.check_b = 1;
  cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
  cudaMemsetAsync(a.scal, 0, sizeof(UScal), st);
  const unsigned cblocks = (unsigned)((n_cols + 1 + 255) / 256);
  k_check_cp<<<cblocks, 256, 0, st>>>(a_col_ptr, n_cols, nnz_a, d_status);
  k_check_cp<<<cblocks, 256, 0, st>>>(b_col_ptr, n_cols, nnz_b, d_status);
  k_split<<<(unsigned)((L.tiles_max + 1 + 255) / 256), 256, 0, st>>>(a);
  const cudaError_t e = dtype == SPM_F64 ? launch_merge<uint64_t, kOpDot>(a, L.tiles_max, st)
                                         : launch_merge<uint32_t, kOpDot>(a, L.tiles_max, st);
  k_dot_sum<<<1, 1024, 0, st>>>(a, d_result);
  spm::count_launches(5);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return SPM_ERR_CUDA;
  return SPM_OK;
}

}  // extern "C"
