// libspm: per-bucket resolution of the sync step (sm_103a).
//
// After the partition, the writes of one bucket (an aligned range of the
// paper's linear index row + col * n_rows, Section 3.3) lie contiguously in
// the record array as 16-byte records {key within the bucket, stream
// position, value bits}.  One persistent kernel (one 512-thread block per SM)
// takes the buckets by ticket -- a helper thread fetches the next ticket and
// descriptor and prefetches that bucket into L2 -- and, per bucket:
//
//   load     one bulk copy (cp.async.bulk, completed on an mbarrier, bounded
//            wait) moves the bucket's records into shared memory
//   narrow   a bucket whose keys span at most kDense values is reduced in a
//            key-indexed table with shared-memory atomics, no sort
//            (resolve_dense)
//   sort     otherwise a counting sort on the top key bits (shared-memory
//            atomics give each write its rank in its sub-bin; rows near the
//            diagonal first get an order-preserving narrower key), then
//            sub-bins of 2..8 writes are ordered by a sorting network in one
//            thread's registers and larger ones by warp bitonic networks over
//            windows of whole sub-bins; equal keys may end up in any order,
//            the reduction does not depend on it
//   reduce   the sorted positions are cut into one range per warp at run
//            boundaries, so that no run of equal keys spans two warps; each
//            lane reduces the runs in its strip of the warp's range, and runs
//            that cross lanes are finished with segmented warp scans.
//              add mode: the exact sum of the run (exact_sum.cuh), its binary
//              point set by the run's own largest exponent (found in a first
//              pass); a single write is its own value; runs of several writes
//              are parked and rounded 32 at a time by the whole warp
//              last-write mode: the write with the largest (seq, position)
//   zeros    an element whose value compares equal to zero is dropped (after
//            rounding to the output type), as CSC stores non-zeros only
//            (Section 3.1)
//   out      without the map the stored elements (key, value) are written in
//            key order over the bucket's records with coalesced stores and
//            the bucket's count is recorded; k_place, after a scan of the
//            counts, puts them in the CSC arrays.  With the map the block
//            takes its output offset from a bounded decoupled look-back and
//            places its elements and map entries at once.
//
// A bucket with more writes than fit in shared memory is resolved in windows
// of its key range (records gathered from global memory): with the map at
// once (counted, then written), without it counted here and written by k_big
// once the offsets are known; one key with more writes than a window holds
// is reduced by a streaming pass.
//
// No kernel traps or waits without a bound: an expired wait is reported as
// SPM_ERR_TIMEOUT in the device status word and the call stops.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <type_traits>

#include "device_util.cuh"
#include "exact_sum.cuh"

namespace spm {
namespace {

constexpr int kRT = 512;                    // threads per resolve block (one block per SM)
constexpr int kRW = kRT / 32;               // warps per block
constexpr int kRI = 16;                     // sorted positions per thread at the capacity
constexpr int kRCap = kRT * kRI;            // writes of one bucket resolved in shared memory
constexpr int kRCapNow = kRCap / 2;         // ... when the elements are staged in shared memory
constexpr int kRBins = 1 << kSubBitsMax;    // sub-bins of the counting sort, at most
constexpr uint16_t kKept = 0x8000u;         // perm[] flag: the run ending here is stored
constexpr uint16_t kMulti = 0x4000u;        // perm[] flag: a run of several writes ends here, its
                                            // accumulator is parked (rounded later)
constexpr uint16_t kIdx = 0x1fffu;          // perm[] bits of the record index (< kRCap)

// Dynamic shared memory: records (the upper half doubles as the staging area
// of elements placed at once), sorted keys, sorted record indices, sub-bin
// counters (later the runs' largest exponents).
struct RLay {
  size_t R, stage_key, stage_val, skey, perm, bins, total;
};
__host__ __device__ constexpr RLay rlay() {
  return RLay{0,
              size_t{16} * kRCapNow,
              size_t{16} * kRCapNow + size_t{4} * kRCapNow,
              size_t{16} * kRCap,
              size_t{20} * kRCap,
              size_t{22} * kRCap,
              size_t{22} * kRCap + (((size_t)(kRBins + 1) * 4 + 15) & ~size_t{15})};
}

// ---------------------------------------------------------------------------
// Bulk copies and mbarriers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// the same without the arrival (a later copy of the same phase arrives)
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> own shared memory, 16-byte aligned addresses and a size that is a
// multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for one phase of the mbarrier; false when the limit expired.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  uint64_t t0 = 0;
  for (uint32_t spins = 0;; ++spins) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spins & 63) == 63) {
      const uint64_t t = global_timer_ns();
      if (!t0) t0 = t;
      else if (t - t0 > kWaitLimitNs) return false;
    }
  }
}
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  if (bytes >= 16) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes & ~15u) : "memory");
}

// ---------------------------------------------------------------------------
// Values carried by the segmented warp scans
// ---------------------------------------------------------------------------
template <bool UP>
__device__ __forceinline__ uint32_t sh32(uint32_t x, int o) {
  return UP ? __shfl_up_sync(kFull, x, o) : __shfl_down_sync(kFull, x, o);
}
template <bool UP>
__device__ __forceinline__ uint64_t sh64(uint64_t x, int o) {
  return UP ? __shfl_up_sync(kFull, x, o) : __shfl_down_sync(kFull, x, o);
}

struct EV {  // largest alignment exponent of a run (so far)
  int e;
};
struct AV {  // exact sum (two's complement 128-bit integer) and IEEE special flags
  uint64_t lo, hi;
  uint32_t f;
};
struct WV {  // last-write winner: largest (seq, position), its value
  uint64_t seq, val;
  uint32_t pos, ok;
};
struct OV {  // output index of a run (-2: removed; INT_MIN: none) and its winner's position
  int32_t out;
  uint32_t win;
};

template <bool UP>
__device__ __forceinline__ EV shf(const EV& v, int o) {
  return EV{(int)sh32<UP>((uint32_t)v.e, o)};
}
template <bool UP>
__device__ __forceinline__ AV shf(const AV& v, int o) {
  return AV{sh64<UP>(v.lo, o), sh64<UP>(v.hi, o), sh32<UP>(v.f, o)};
}
template <bool UP>
__device__ __forceinline__ WV shf(const WV& v, int o) {
  return WV{sh64<UP>(v.seq, o), sh64<UP>(v.val, o), sh32<UP>(v.pos, o), sh32<UP>(v.ok, o)};
}
template <bool UP>
__device__ __forceinline__ OV shf(const OV& v, int o) {
  return OV{(int32_t)sh32<UP>((uint32_t)v.out, o), sh32<UP>(v.win, o)};
}

__device__ __forceinline__ AV av_add(const AV& a, const AV& b) {
  const uint64_t lo = a.lo + b.lo;
  return AV{lo, a.hi + b.hi + (lo < a.lo ? 1ull : 0ull), a.f | b.f};
}
__device__ __forceinline__ AV av_of(const Acc& a) { return AV{a.lo, (uint64_t)a.hi, a.flags}; }
__device__ __forceinline__ Acc acc_of(const AV& a) { return Acc{a.lo, (int64_t)a.hi, a.f}; }
__device__ __forceinline__ bool wv_better(const WV& a, const WV& b) {  // is b later than a
  return b.ok && (!a.ok || b.seq > a.seq || (b.seq == a.seq && b.pos > a.pos));
}

struct OpMax {
  __device__ EV operator()(const EV& a, const EV& b) const { return EV{max(a.e, b.e)}; }
};
struct OpAdd {
  __device__ AV operator()(const AV& a, const AV& b) const { return av_add(a, b); }
};
struct OpWin {
  __device__ WV operator()(const WV& a, const WV& b) const { return wv_better(a, b) ? b : a; }
};
struct OpNear {  // the value nearer in the flow direction, unless it is empty
  __device__ OV operator()(const OV& far, const OV& near) const { return near.out == INT_MIN ? far : near; }
};

// Segmented scan over the lanes of a warp in the direction of the flow (FWD:
// from lower to higher lane; otherwise from higher to lower).  Lane l gives
// (reset_l, v_l); out_l = reset_l ? v_l : op(out_prev, v_l) where out_prev is
// the neighbour upstream.  Returns out_prev (ident for the first lane of the
// flow).
template <bool FWD, class T, class Op>
__device__ __forceinline__ T warp_seg_scan(bool reset, const T& v, const T& ident, Op op) {
  const int lane = threadIdx.x & 31;
  bool f = reset;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const bool f2 = sh32<FWD>(f ? 1u : 0u, o) != 0;
    const T x2 = shf<FWD>(x, o);
    if (FWD ? lane >= o : lane + o < 32) {
      if (!f) x = op(x2, x);
      f = f || f2;
    }
  }
  const T xe = shf<FWD>(x, 1);
  return (FWD ? lane == 0 : lane == 31) ? ident : xe;
}

// ---------------------------------------------------------------------------
// Buckets, key ranges and their place in the output
// ---------------------------------------------------------------------------
// Column arithmetic of a key range [klo, klo + span): klo = col0 * n_rows + r0.
struct Range {
  uint64_t klo, span, col0, r0;
  Div32 dv;
  uint32_t fastdiv;  // r0 + span + n_rows < 2^32: 32-bit division by n_rows
};
__device__ __forceinline__ Range make_range(uint64_t nr, uint64_t klo, uint64_t span) {
  Range r;
  r.klo = klo;
  r.span = span;
  r.col0 = klo / nr;
  r.r0 = klo - r.col0 * nr;
  r.fastdiv = (r.r0 + span + nr) < (uint64_t{1} << 32) ? 1u : 0u;
  r.dv = div32_make((uint32_t)nr);
  return r;
}
__device__ __forceinline__ uint64_t col_of(const Range& R, uint64_t x, uint64_t nr) {
  return R.fastdiv ? (uint64_t)div32((uint32_t)x, R.dv) : x / nr;
}

struct Desc {
  uint32_t b, n;      // bucket, its writes
  uint32_t valid;
  int64_t start;      // first record of the bucket
  int64_t mi;         // matrix
  int64_t n_rows, n_cols, col_base, t0, bucket_off;
  uint64_t K;
  Range rg;           // the bucket's key range
};

// Bucket b's descriptor (one thread; reads the bucket tables and the matrix).
// Bucket b's descriptor from its table entries and its matrix.
__device__ __forceinline__ Desc make_desc(uint32_t b, uint32_t n, uint32_t start, uint32_t info, uint64_t klo,
                                          const MatMeta& mm) {
  Desc d;
  d.b = b;
  d.valid = 1;
  d.n = n;
  d.start = start;
  d.mi = info >> 6;
  d.n_rows = mm.n_rows;
  d.n_cols = mm.n_cols;
  d.col_base = mm.col_base;
  d.t0 = mm.t0;
  d.bucket_off = mm.bucket_off;
  d.K = mm.K;
  const uint64_t span = mm.K == 0 ? 0 : min(uint64_t{1} << (info & 63), mm.K - klo);
  d.rg = mm.K == 0 ? Range{0, 0, 0, 0, Div32{0, 0, 0}, 0} : make_range((uint64_t)mm.n_rows, klo, span);
  return d;
}

__device__ __forceinline__ Desc load_desc(const Ctx& c, uint32_t b) {
  const uint32_t info = c.bk_info[b];
  return make_desc(b, c.bk_count[b], c.bk_start[b], info, c.bk_lo[b], c.meta[info >> 6]);
}

// Asynchronous copies of a bucket's table entries into shared memory (the
// helper thread issues them a bucket ahead and waits only when it builds the
// descriptor).
struct DescRaw {
  uint64_t klo;
  uint32_t n, start, info, pad;
};
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void raw_fetch(const Ctx& c, uint32_t b, DescRaw* r) {
  cp_async8(&r->klo, c.bk_lo + b);
  cp_async4(&r->n, c.bk_count + b);
  cp_async4(&r->start, c.bk_start + b);
  cp_async4(&r->info, c.bk_info + b);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

struct RShared {
  Desc cur;           // the bucket being resolved
  Range win;          // window (or single key) being resolved at once
  int64_t base;
  uint32_t wk[32];    // per warp: stored elements
  uint32_t buf[32];
  uint32_t tot, maxbin, nw, taken, abort;
  // single key: result
  uint64_t kbits;
  uint32_t kkeep, kwin;
  int kmax;
  alignas(16) unsigned char parts[kRW * 32];  // per warp partial of a single key
  uint16_t ring[kRW][64];  // per warp: positions of parked runs waiting to be rounded
  uint32_t rb, rb_next;    // first record slot of the current / next bucket in the record area
  uint32_t pre;            // the next bucket's place is set and (part of) its copy in flight
  uint32_t late_off, late_cnt;  // ... the part of it still to copy once this bucket is done
  uint64_t bar;       // mbarrier of the bulk copy
};

__device__ __forceinline__ uint64_t f32_bits_to_f64_bits(uint64_t v) {
  return (uint64_t)__double_as_longlong((double)__uint_as_float((uint32_t)v));
}
template <bool F64>
__device__ __forceinline__ uint64_t wide(uint64_t v) {
  return F64 ? v : f32_bits_to_f64_bits(v);
}
template <bool F64>
__device__ __forceinline__ bool bits_nonzero(uint64_t bits) {
  return F64 ? (bits & 0x7FFFFFFFFFFFFFFFull) != 0 : (bits & 0x7FFFFFFFull) != 0;
}
template <bool F64>
__device__ __forceinline__ int align_exp(uint64_t raw) {
  return max(0, f64_align_exponent(wide<F64>(raw)));
}

// Where the elements of a bucket wait for k_place (calls without the map):
// over the bucket's own records, keys (relative to the bucket) from the first
// record, values from byte 4 * n (rounded up to 8) on.  Both fit: 12 bytes per
// element in the 16 bytes of each record.
__device__ __forceinline__ uint32_t* res_keys(const Ctx& c, int64_t start) {
  return reinterpret_cast<uint32_t*>(c.rec + start);
}
__device__ __forceinline__ uint64_t* res_vals(const Ctx& c, int64_t start, uint32_t n) {
  return reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(c.rec + start) + (((size_t)4 * n + 7) & ~size_t{7}));
}

// acc_add_bits without divergent branches for finite values (the lanes of a
// warp add values of either sign and any exponent): the magnitude is aligned
// and truncated in the same way, then added or, for a negative value,
// subtracted as a two's complement 128-bit integer.  The same sum results.
// The 128-bit two's complement fixed-point value of the finite float64 `bits`
// with the binary point of exponent emax (as acc_add_bits aligns it).
__device__ __forceinline__ void fixed_of(uint64_t bits, int emax, uint64_t& xlo, uint64_t& xhi) {
  const uint32_t e = (uint32_t)(bits >> 52) & 0x7ffu;
  const uint64_t frac = bits & 0xFFFFFFFFFFFFFull;
  const uint64_t mant = e ? (frac | (1ull << 52)) : frac;
  const int sh = (int)max(e, 1u) - (emax - kAlignBits);  // <= kAlignBits
  const uint32_t ls = (uint32_t)max(sh, 0);
  const uint32_t rs = (uint32_t)min(max(-sh, 0), 63);
  const uint64_t tlo = sh >= 0 ? (mant << ls) : (sh > -64 ? (mant >> rs) : 0ull);
  const uint64_t thi = sh > 0 ? (mant >> (64u - ls)) : 0ull;
  const uint64_t neg = (uint64_t)((int64_t)bits >> 63);  // all ones for a negative value
  const uint64_t nlo = tlo ^ neg;
  xlo = nlo + (neg & 1ull);
  xhi = (thi ^ neg) + (xlo < nlo ? 1ull : 0ull);
}

__device__ __forceinline__ void acc_add_fast(Acc& a, uint64_t bits, int emax) {
  const uint32_t e = (uint32_t)(bits >> 52) & 0x7ffu;
  if (e == 0x7ffu) {  // NaN or infinity: a flag
    a.flags |= (bits & 0xFFFFFFFFFFFFFull) ? 1u : ((bits >> 63) ? 4u : 2u);
    return;
  }
  uint64_t xlo, xhi;
  fixed_of(bits, emax, xlo, xhi);
  const uint64_t lo = a.lo + xlo;
  a.hi = (int64_t)((uint64_t)a.hi + xhi + (lo < xlo ? 1ull : 0ull));
  a.lo = lo;
}

// Write the nnz stored elements of the key range R (get(li) gives the key
// relative to R.klo and the value bits of the li-th, in key order) from
// matrix-relative output index base, and the offsets of every column that
// starts inside the range.  Called by the whole block.
template <bool F64, class Get>
__device__ void emit_range(const Ctx& c, const Desc& D, const Range& R, uint32_t nnz, int64_t base, Get get) {
  using VT = typename std::conditional<F64, uint64_t, uint32_t>::type;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint64_t nr = (uint64_t)D.n_rows, col0 = R.col0, r0 = R.r0;
  int64_t* colp = c.col_ptr + D.col_base;
  int32_t* rowp = c.row_idx + D.t0;
  VT* outp = reinterpret_cast<VT*>(c.out_vals) + D.t0;
  const uint64_t jn = col0 + (r0 ? 1u : 0u);                       // first column starting in the range
  const uint64_t je = col0 + col_of(R, r0 + R.span + nr - 1, nr);  // first column starting after it
  uint64_t lastcol = jn - 1;
  // each iteration's element (and, for lane 0, the element before the warp's
  // first) is loaded one iteration ahead, so the loads overlap the stores
  uint32_t nkey = 0, pkey = 0;
  uint64_t nbits = 0, pbits = 0;
  {
    const uint32_t l1 = (tid & ~31u) + lane;
    if (l1 < nnz) get(l1, nkey, nbits);
    if (lane == 0 && l1 > 0 && l1 < nnz) get(l1 - 1, pkey, pbits);
  }
  for (uint32_t li0 = tid & ~31u; li0 < nnz; li0 += blockDim.x) {
    const uint32_t li = li0 + lane;
    const bool have = li < nnz;
    const uint32_t key = nkey, prevkey = pkey;
    const uint64_t bits = nbits;
    {
      const uint32_t ln = li + blockDim.x;
      if (ln < nnz) get(ln, nkey, nbits);
      if (lane == 0 && ln < nnz) get(ln - 1, pkey, pbits);
    }
    uint64_t col = 0;
    if (have) {
      const uint64_t x = r0 + key;
      const uint64_t cr = col_of(R, x, nr);
      col = col0 + cr;
      rowp[base + li] = (int32_t)(x - cr * nr);
      outp[base + li] = (VT)bits;
    }
    uint64_t pc = __shfl_up_sync(kFull, col, 1);
    if (have && lane == 0) pc = li == 0 ? jn - 1 : col0 + col_of(R, r0 + prevkey, nr);
    // offsets of the columns (pc, col]: this element is the first of each
    const uint64_t gap = have ? col - pc : 0;
    if (gap > 0 && gap <= 32)
      for (uint64_t j = pc + 1; j <= col; ++j) colp[j] = base + li;
    unsigned big = __ballot_sync(kFull, gap > 32);
    while (big) {  // long gaps: the warp fills them together
      const int L = __ffs(big) - 1;
      big &= big - 1;
      const uint64_t a = __shfl_sync(kFull, pc, L) + 1, e = __shfl_sync(kFull, col, L);
      const int64_t v = base + (int64_t)__shfl_sync(kFull, li, L);
      for (uint64_t j = a + lane; j <= e; j += 32) colp[j] = v;
    }
  }
  // columns that start after the last element (all of them if there is none)
  if (nnz) {
    uint32_t key;
    uint64_t bits;
    get(nnz - 1, key, bits);
    lastcol = col0 + col_of(R, r0 + key, nr);
  }
  for (uint64_t j = lastcol + 1 + tid; j < je; j += blockDim.x) colp[j] = base + nnz;
}

// Sort k <= 32 (key, index) pairs in shared memory by key with one warp: a
// bitonic network over 32 slots, one per lane (empty slots hold the largest
// value).  Called by all lanes of the warp.
__device__ __forceinline__ void warp_sort32(uint32_t* keys, uint16_t* idx, uint32_t k) {
  const int lane = threadIdx.x & 31;
  uint64_t x = (uint32_t)lane < k ? (((uint64_t)keys[lane] << 16) | idx[lane]) : ~0ull;
#pragma unroll
  for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const uint64_t y = __shfl_xor_sync(kFull, x, j);
      x = (((lane & j) == 0) == ((lane & kk) == 0)) ? min(x, y) : max(x, y);
    }
  }
  if ((uint32_t)lane < k) {
    keys[lane] = (uint32_t)(x >> 16);
    idx[lane] = (uint16_t)x;
  }
}

// Sort k <= 64 (key, index) pairs in shared memory by key with one warp: a
// bitonic network over 64 slots, two per lane (slots lane and lane + 32;
// empty slots hold the largest value).  Called by all lanes of the warp.
__device__ __forceinline__ void warp_sort64(uint32_t* keys, uint16_t* idx, uint32_t k) {
  const int lane = threadIdx.x & 31;
  uint64_t x0 = (uint32_t)lane < k ? (((uint64_t)keys[lane] << 16) | idx[lane]) : ~0ull;
  uint64_t x1 = (uint32_t)lane + 32u < k ? (((uint64_t)keys[lane + 32] << 16) | idx[lane + 32]) : ~0ull;
#pragma unroll
  for (int kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j == 32) {  // the partner is the lane's other slot (kk == 64: ascending)
        const uint64_t lo = min(x0, x1), hi = max(x0, x1);
        x0 = lo;
        x1 = hi;
      } else {
        const uint64_t y0 = __shfl_xor_sync(kFull, x0, j), y1 = __shfl_xor_sync(kFull, x1, j);
        const bool lower = (lane & j) == 0;
        const bool asc0 = (lane & kk) == 0, asc1 = ((lane + 32) & kk) == 0;
        x0 = (lower == asc0) ? min(x0, y0) : max(x0, y0);
        x1 = (lower == asc1) ? min(x1, y1) : max(x1, y1);
      }
    }
  }
  if ((uint32_t)lane < k) {
    keys[lane] = (uint32_t)(x0 >> 16);
    idx[lane] = (uint16_t)x0;
  }
  if ((uint32_t)lane + 32u < k) {
    keys[lane + 32] = (uint32_t)(x1 >> 16);
    idx[lane + 32] = (uint16_t)x1;
  }
}

// ---------------------------------------------------------------------------
// A bucket whose key range is narrow: one table slot per key
// ---------------------------------------------------------------------------
// When a bucket's keys span at most kDense values (the crowded columns of a
// skewed stream, where many writes share few keys), the records are reduced
// into a table indexed by the key itself, with shared-memory atomics, and no
// sort is needed: the table is already in key order.  Sum mode: pass 1 takes
// each key's largest exponent (atomic max), pass 2 adds every write's
// fixed-point value at that binary point into the key's 128-bit slot (four
// 32-bit limbs updated by native shared-memory atomics with exact carries:
// integer addition, so the order of the adds does not matter) -- the same
// integer the run reduction forms, hence the same rounded sum.  Last-write
// mode (positions only): the largest position per key, then its value.  The
// table lies in the shared arrays that the sort would use; the records stay
// untouched, so a sum bucket holding a NaN or an infinity returns kDenseNo
// and is resolved by resolve_tile.
constexpr uint32_t kDense = 3072;      // table slots (20 bytes each in sum mode)
constexpr uint32_t kDenseNo = ~0u;

template <bool F64, bool SUM>
__device__ __noinline__ uint32_t resolve_dense(const Ctx& c, RShared& S, unsigned char* smem, uint32_t n,
                                               const Desc& D, uint32_t rb) {
  constexpr RLay L = rlay();
  const uint4* const R = reinterpret_cast<const uint4*>(smem + L.R) + rb;
  uint32_t* const tag = reinterpret_cast<uint32_t*>(smem + L.skey);  // 1 + largest exponent / 1 + position
  // sum: four 32-bit limbs per slot (the result's bits later in the first
  // two); last write: the value per slot
  uint64_t* const tlo = reinterpret_cast<uint64_t*>(smem + L.skey + 4 * kDense);
  auto slot_val = [&](uint32_t q) -> uint64_t& { return SUM ? tlo[2 * q] : tlo[q]; };
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t span = (uint32_t)D.rg.span;
  for (uint32_t q = tid; q < span; q += kRT) tag[q] = 0u;
  for (uint32_t q = tid; q < (SUM ? 2 * span : span); q += kRT) tlo[q] = 0ull;
  __syncthreads();
  bool odd = false;
  for (uint32_t i = tid; i < n; i += kRT) {
    const uint4 r = R[i];
    if (SUM) {
      const uint64_t w = wide<F64>(((uint64_t)r.w << 32) | r.z);
      odd |= ((w >> 52) & 0x7ffu) == 0x7ffu;
      atomicMax(&tag[r.x], (uint32_t)align_exp<F64>(((uint64_t)r.w << 32) | r.z) + 1u);
    } else {
      atomicMax(&tag[r.x], r.y + 1u);
    }
  }
  if (SUM) {
    if (__syncthreads_or(odd)) return kDenseNo;
  } else {
    __syncthreads();
  }
  if (SUM) {
    // each write's fixed-point value is added to its slot's four 32-bit limbs
    // (native shared-memory atomics): its magnitude, limb by limb from the
    // lowest non-zero one, with the carry (or, for a negative value, the
    // borrow) that each atomic's old value reveals passed to the next limb.
    // Every atomic is exact and the carries are counted exactly, so the slot
    // ends as the two's complement sum of all its writes, whatever the order.
    uint32_t* const limb = reinterpret_cast<uint32_t*>(tlo);  // slot q: limb[4q .. 4q+3], low first
    for (uint32_t i = tid; i < n; i += kRT) {
      const uint4 r = R[i];
      const uint64_t w = wide<F64>(((uint64_t)r.w << 32) | r.z);
      uint64_t xlo, xhi;
      fixed_of(w & 0x7FFFFFFFFFFFFFFFull, max((int)tag[r.x] - 1, 1), xlo, xhi);  // the magnitude
      const bool neg = (w >> 63) != 0;
      const uint32_t m[4] = {(uint32_t)xlo, (uint32_t)(xlo >> 32), (uint32_t)xhi, (uint32_t)(xhi >> 32)};
      uint32_t* const L4 = limb + 4 * r.x;
      uint64_t c = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint64_t add = (uint64_t)m[k] + c;  // 0 .. 2^32
        if (add == 0) continue;                   // (c stays 0)
        if (add >> 32) {                          // 2^32: the limb is unchanged, carry or borrow 1
          c = 1;
          continue;
        }
        if (neg) {
          const uint32_t old = atomicSub(&L4[k], (uint32_t)add);
          c = old < (uint32_t)add ? 1u : 0u;
        } else {
          const uint32_t old = atomicAdd(&L4[k], (uint32_t)add);
          c = ((uint64_t)old + add) >> 32;
        }
      }
    }
  } else {
    for (uint32_t i = tid; i < n; i += kRT) {
      const uint4 r = R[i];
      if (r.y + 1u == tag[r.x]) tlo[r.x] = ((uint64_t)r.w << 32) | r.z;
    }
  }
  __syncthreads();
  // results: each warp a contiguous share of the slots, counted, then written
  // in key order with coalesced stores over the bucket's records
  const bool keep_zeros = !SUM && c.keep_zeros;
  const uint32_t per = ((span + kRW - 1) / kRW + 31) & ~31u;
  const uint32_t s0 = min(span, (uint32_t)wid * per), s1 = min(span, s0 + per);
  uint32_t cnt = 0;
  for (uint32_t q0 = s0; q0 < s1; q0 += 32) {
    const uint32_t q = q0 + lane;
    bool kept = false;
    if (q < s1 && tag[q] != 0u) {
      if (SUM) {
        bool nz;
        const Acc x{tlo[2 * q], (int64_t)tlo[2 * q + 1], 0u};  // (limbs, low first: little-endian words)
        slot_val(q) = acc_round(x, max((int)tag[q] - 1, 1), !F64, &nz);
        kept = nz;
      } else {
        kept = keep_zeros || bits_nonzero<F64>(slot_val(q));
      }
      if (!kept) tag[q] = 0u;
    }
    cnt += __popc(__ballot_sync(kFull, kept));
  }
  if (lane == 0) S.wk[wid] = cnt;
  __syncthreads();
  uint32_t wl = 0, nnz = 0;
#pragma unroll
  for (int w2 = 0; w2 < kRW; ++w2) {
    const uint32_t x = S.wk[w2];
    wl += w2 < wid ? x : 0u;
    nnz += x;
  }
  uint32_t* const dk = res_keys(c, D.start);
  uint64_t* const dv = res_vals(c, D.start, D.n);
  const unsigned lt = (1u << lane) - 1u;
  for (uint32_t q0 = s0; q0 < s1; q0 += 32) {
    const uint32_t q = q0 + lane;
    const bool kept = q < s1 && tag[q] != 0u;
    const unsigned b = __ballot_sync(kFull, kept);
    if (kept) {
      const uint32_t li = wl + __popc(b & lt);
      dk[li] = q;
      dv[li] = slot_val(q);
    }
    wl += __popc(b);
  }
  return nnz;  // (the caller's barrier ends every read of the shared arrays)
}

// ---------------------------------------------------------------------------
// One set of records in shared memory
// ---------------------------------------------------------------------------
// How the stored elements leave resolve_tile.
enum : int {
  kCount = 0,  // only counted
  kDefer = 1,  // written over the bucket's records (res_keys, res_vals), placed by k_place
  kNow = 2     // placed at once (output index from get_base, called by warp 0)
};

// Resolve the n records R[0, n) of bucket D (keys relative to Rg.klo, in
// [0, Rg.span)).  Returns the number of stored elements.  kNow needs
// n <= kRCapNow.  Ends with a barrier, except in kDefer mode (the caller's
// next barrier ends every read of the shared arrays).
template <bool F64, bool SUM, bool SEQ, bool MAP, class GetBase>
__device__ __noinline__ uint32_t resolve_tile(const Ctx& c, RShared& S, unsigned char* smem, uint32_t n, const Desc& D,
                                 const Range& Rg, int mode, GetBase get_base, uint32_t rb = 0) {
  constexpr RLay L = rlay();
  // the records: slots [rb, rb + n) of the record area (rb > 0 only without the map)
  uint4* const R = reinterpret_cast<uint4*>(smem + L.R) + rb;
  const uint64_t* const RV = reinterpret_cast<const uint64_t*>(R);
  uint64_t* const RVw = reinterpret_cast<uint64_t*>(R);
  uint32_t* const skey = reinterpret_cast<uint32_t*>(smem + L.skey);
  uint16_t* const perm = reinterpret_cast<uint16_t*>(smem + L.perm);
  uint32_t* const bins = reinterpret_cast<uint32_t*>(smem + L.bins);
  uint16_t* const rmax = reinterpret_cast<uint16_t*>(smem + L.bins);  // after the sort: largest exponents
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool keep_zeros = !SUM && c.keep_zeros;

  // ---- banded key ranges: when every write's row lies within a band around
  // the diagonal (row - col in [-md, md], as in FEM and stencil matrices) and
  // the bucket spans many columns, the sort uses the order-preserving key
  // (column in the bucket) * W + (row - col + W/2), W = 2^bshift > 2 md + 1,
  // whose range is far narrower than the bucket's: the sub-bins then separate
  // the rows of a column instead of holding whole columns.  The stored keys
  // are mapped back when they are written out (kDefer only).
  uint32_t bshift = 0;
  uint64_t span = Rg.span;
  const uint64_t nr = (uint64_t)D.n_rows;
  if (!MAP && mode == kDefer && n > 64 && Rg.span > (uint64_t)n * 64) {
    uint32_t md = 0;
    for (uint32_t i = tid; i < n; i += kRT) {
      const uint64_t t = Rg.r0 + R[i].x;
      const uint64_t co = col_of(Rg, t, nr);
      const int64_t d = (int64_t)(t - co * nr) - (int64_t)(Rg.col0 + co);
      const int64_t ad = d < 0 ? -d : d;
      md = max(md, (uint32_t)(ad < 0x3fffffff ? ad : 0x3fffffff));
    }
    md = __reduce_max_sync(kFull, md);
    if (lane == 0) S.buf[wid] = md;
    __syncthreads();
    md = 0;
#pragma unroll
    for (int w2 = 0; w2 < kRW; ++w2) md = max(md, S.buf[w2]);
    const uint64_t ncols = col_of(Rg, Rg.r0 + Rg.span - 1, nr) + 1;
    const int sh = ceil_log2_u64(2ull * md + 2ull);
    if ((uint64_t{1} << sh) < nr && (ncols << sh) <= Rg.span / 4 && (ncols << sh) <= (uint64_t{1} << 32)) {
      bshift = (uint32_t)sh;
      span = ncols << sh;
      for (uint32_t i = tid; i < n; i += kRT) {
        const uint64_t t = Rg.r0 + R[i].x;
        const uint64_t co = col_of(Rg, t, nr);
        const int64_t d = (int64_t)(t - co * nr) - (int64_t)(Rg.col0 + co);
        R[i].x = (uint32_t)((co << sh) | (uint64_t)(d + (int64_t{1} << (sh - 1))));
      }
    }
  }
  auto unband = [&](uint32_t k) -> uint32_t {
    if (!bshift) return k;
    const uint64_t co = k >> bshift;
    const int64_t d = (int64_t)(k & ((1u << bshift) - 1u)) - (int64_t{1} << (bshift - 1));
    return (uint32_t)(co * nr + (uint64_t)((int64_t)(Rg.col0 + co) + d) - Rg.r0);
  };

  // ---- counting sort on the top key bits (about one sub-bin per write)
  const int sbits = span <= 1 ? 0 : ceil_log2_u64(span);
  const int bbits = min(c.sub_bits, max(4, n <= 1 ? 0 : ceil_log2_u64(n)));
  const int sshift = sbits > bbits ? sbits - bbits : 0;
  const uint32_t nbins = (uint32_t)(((span - 1) >> sshift) + 1);
  for (uint32_t q = tid; q <= nbins; q += kRT) bins[q] = 0u;
  if (tid == 0) S.maxbin = 0;
  __syncthreads();
  uint32_t rk[kRI / 2] = {};  // rank of each write in its sub-bin (< 2^16), two per word
#pragma unroll
  for (int k = 0; k < kRI; ++k) {
    const uint32_t i = tid + k * kRT;
    if (i < n) rk[k >> 1] |= atomicAdd(&bins[R[i].x >> sshift], 1u) << (16 * (k & 1));
  }
  __syncthreads();
  {
    const uint32_t per = (nbins + kRT - 1) / kRT;
    const uint32_t a = min(nbins, tid * per), e = min(nbins, a + per);
    uint32_t local = 0, mx = 0;
    for (uint32_t q = a; q < e; ++q) {
      const uint32_t x = bins[q];
      local += x;
      mx = max(mx, x);
    }
    mx = __reduce_max_sync(kFull, mx);
    if (lane == 0 && mx) atomicMax(&S.maxbin, mx);
    uint32_t run = block_scan_excl<uint32_t>(local, &S.tot, S.buf);
    for (uint32_t q = a; q < e; ++q) {
      const uint32_t x = bins[q];
      bins[q] = run;
      run += x;
    }
    if (tid == 0) bins[nbins] = n;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kRI; ++k) {
    const uint32_t i = tid + k * kRT;
    if (i < n) {
      const uint32_t kv = R[i].x;
      const uint32_t p = bins[kv >> sshift] + ((rk[k >> 1] >> (16 * (k & 1))) & 0xffffu);
      skey[p] = kv;
      perm[p] = (uint16_t)i;
    }
  }
  __syncthreads();
  // ---- order the keys inside the sub-bins (each holds one key when sshift == 0)
  if (sshift > 0 && n > 1) {
    if (S.maxbin <= 64u) {
      // sub-bins of 2..8 writes: one thread, a sorting network in registers;
      // of 9..64: one warp, a bitonic network over (key, index) in registers
      const uint32_t qa = (uint32_t)(((uint64_t)tid * nbins) / kRT), qb = (uint32_t)(((uint64_t)(tid + 1) * nbins) / kRT);
      for (uint32_t q = qa; q < qb; ++q) {
        const uint32_t a = bins[q], e = bins[q + 1];
        if (e - a < 2u || e - a > 8u) continue;
        // 2..8 writes: an 8-input sorting network in registers (19
        // compare-exchanges; absent inputs are the largest key, ties in any
        // order: equal keys only need to be adjacent)
        const uint32_t k = e - a;
        uint32_t kk[8], pp[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          kk[j] = (uint32_t)j < k ? skey[a + j] : 0xffffffffu;
          pp[j] = (uint32_t)j < k ? perm[a + j] : 0u;
        }
        auto cx = [&](int i, int j) {
          const bool sw = kk[i] > kk[j];
          const uint32_t k0 = sw ? kk[j] : kk[i], k1 = sw ? kk[i] : kk[j];
          const uint32_t p0 = sw ? pp[j] : pp[i], p1 = sw ? pp[i] : pp[j];
          kk[i] = k0, kk[j] = k1, pp[i] = p0, pp[j] = p1;
        };
        cx(0, 2), cx(1, 3), cx(4, 6), cx(5, 7);
        cx(0, 4), cx(1, 5), cx(2, 6), cx(3, 7);
        cx(0, 1), cx(2, 3), cx(4, 5), cx(6, 7);
        cx(2, 4), cx(3, 5);
        cx(1, 4), cx(3, 6);
        cx(1, 2), cx(3, 4), cx(5, 6);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if ((uint32_t)j < k) {
            skey[a + j] = kk[j];
            perm[a + j] = (uint16_t)pp[j];
          }
        }
      }
      // A heavy sub-bin is sorted together with the sub-bins after it, up to
      // 64 positions, as long as those hold at most one write or are heavy
      // too (sub-bins of 2..8 are the threads' above): the sub-bins are in key
      // order, so sorting a window of whole sub-bins sorts each of them.
      for (uint32_t q0 = (uint32_t)wid * 32u; q0 < nbins; q0 += (uint32_t)kRW * 32u) {
        const uint32_t q = q0 + lane;
        const uint32_t qa = q < nbins ? bins[q] : n, qe = q < nbins ? bins[q + 1] : n;
        const uint32_t sz = qe - qa;
        unsigned hv = __ballot_sync(kFull, sz > 8u);
        const unsigned mid = __ballot_sync(kFull, (sz >= 2u && sz <= 8u) || q >= nbins);
        while (hv) {
          const int L = __ffs(hv) - 1;
          const uint32_t P = __shfl_sync(kFull, qa, L);
          // the window ends before the first thread-sorted sub-bin after L or
          // the first sub-bin that ends beyond P + 64
          const unsigned after = ~((2u << L) - 1u);
          const unsigned stop = (mid | __ballot_sync(kFull, qe > P + 64u)) & after;
          const int M = (stop ? __ffs(stop) - 1 : 32) - 1;
          const uint32_t B = __shfl_sync(kFull, qe, M);
          if (B - P <= 32u) warp_sort32(skey + P, perm + P, B - P);
          else warp_sort64(skey + P, perm + P, B - P);
          hv &= M >= 31 ? 0u : ~((2u << M) - 1u);
        }
      }
    } else {
      // a large sub-bin: bitonic sort of the whole set by (key, index)
      uint32_t N = 2;
      while (N < n) N <<= 1;
      for (uint32_t q = n + tid; q < N; q += kRT) {
        skey[q] = 0xffffffffu;
        perm[q] = 0xffffu;
      }
      __syncthreads();
      for (uint32_t k = 2; k <= N; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
          for (uint32_t i = tid; i < N / 2; i += kRT) {
            const uint32_t lo = 2 * j * (i / j) + (i % j), hi = lo + j;
            const bool asc = (lo & k) == 0;
            const uint64_t x = ((uint64_t)skey[lo] << 16) | perm[lo], y = ((uint64_t)skey[hi] << 16) | perm[hi];
            if ((x > y) == asc) {
              skey[lo] = (uint32_t)(y >> 16);
              perm[lo] = (uint16_t)y;
              skey[hi] = (uint32_t)(x >> 16);
              perm[hi] = (uint16_t)x;
            }
          }
          __syncthreads();
        }
      }
    }
    __syncthreads();
  }

  // ---- one range of sorted positions per warp, cut at run heads
  auto run_head_at = [&](uint32_t p) -> uint32_t {  // first run head at or after p
    if (p == 0 || p >= n) return p >= n ? n : 0u;
    const uint32_t k = skey[p - 1];
    if (skey[p] != k) return p;
    uint32_t lo = p + 1, hi = n;  // first position holding a larger key
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (skey[mid] > k) hi = mid;
      else lo = mid + 1;
    }
    return lo;
  };
  const uint32_t A = run_head_at((uint32_t)(((uint64_t)wid * n) / kRW));
  const uint32_t E = wid == kRW - 1 ? n : run_head_at((uint32_t)(((uint64_t)(wid + 1) * n) / kRW));
  // this lane's positions [a, e)
  const uint32_t len = E > A ? E - A : 0u;
  // (an odd strip length: the lanes' loads at the same offset in their
  // strips fall in 32 different banks)
  const uint32_t qn = ((len + 31) >> 5) | 1u;
  const uint32_t a = min(E, A + lane * qn), e = min(E, a + qn);
  const bool have = a < e;
  const bool head_a = have && (a == A || skey[a - 1] != skey[a]);
  const bool tail_e = have && (e == E || skey[e] != skey[e - 1]);
  const bool cont_in = have && !head_a;   // the first run continues from the lane before
  uint32_t ft = ~0u;                      // first tail among the positions
  uint32_t nk = 0;                        // stored elements whose run ends here
  // The value of a run ending at position p goes to the value field of the
  // record perm[p]; kKept marks perm[p] when the element is stored.

  if (SUM) {
    // pass 1: largest exponent of each run piece, at its last position
    int run = 0, vf = 0;
    bool anyhead = false, multi = false;
    if (have) {
      bool h = head_a;
      for (uint32_t p0 = a; p0 < e; p0 += 4) {  // four positions' loads in flight at once
        uint32_t kq[5], iq[4];
        uint64_t vq[4];
#pragma unroll
        for (int i = 0; i < 5; ++i) kq[i] = p0 + i < e ? skey[p0 + i] : 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) iq[i] = p0 + i < e ? perm[p0 + i] : 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) vq[i] = p0 + i < e ? RV[2 * iq[i] + 1] : 0ull;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t p = p0 + i;
          if (p < e) {
            const bool t = p + 1 == e ? tail_e : kq[i + 1] != kq[i];
            const int ex = (h && t) ? 0 : align_exp<F64>(vq[i]);  // (a single write needs none)
            run = h ? ex : max(run, ex);
            if (ft == ~0u) vf = max(vf, ex);
            anyhead = anyhead || h;
            multi = multi || !(h && t);
            if (t) {
              rmax[p] = (uint16_t)run;
              if (ft == ~0u) ft = p;
            }
            h = t;
          }
        }
      }
    }
    if (!__any_sync(kFull, multi)) {
      // every position of the warp is an element of its own: its value is the result
      for (uint32_t p0 = a; p0 < e; p0 += 4) {
        uint32_t iq[4];
        uint64_t vq[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) iq[i] = p0 + i < e ? perm[p0 + i] : 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) vq[i] = p0 + i < e ? RV[2 * iq[i] + 1] : 0ull;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (p0 + i < e && bits_nonzero<F64>(vq[i])) {
            perm[p0 + i] = (uint16_t)(iq[i] | kKept);
            ++nk;
          }
        }
      }
      goto numbered;
    }
    {
    const int inF = warp_seg_scan<true>(!have || anyhead, EV{run}, EV{0}, OpMax()).e;
    const int inB = warp_seg_scan<false>(!have || ft != ~0u, EV{vf}, EV{0}, OpMax()).e;
    // pass 2 (backward): exact sums with each run's own binary point.  A run
    // of several writes leaves its accumulator parked at its last position
    // (the slot of that position's record, or for calls with the map, whose
    // records stay in use, a slot per position in the free upper half of the
    // record area), its binary point and flags in rmax; all lanes round the
    // parked runs together afterwards instead of each at its own time.
    uint4* const park = MAP ? reinterpret_cast<uint4*>(smem + L.stage_key) : R;
    auto park_run = [&](uint32_t pos, const Acc& x, int g) {
      const uint32_t ix = perm[pos];
      park[MAP ? pos : (ix & kIdx)] = make_uint4((uint32_t)x.lo, (uint32_t)(x.lo >> 32), (uint32_t)x.hi,
                                                 (uint32_t)((uint64_t)x.hi >> 32));
      rmax[pos] = (uint16_t)(g | (int)(x.flags << 12));  // g <= 2046
      perm[pos] = (uint16_t)(ix | kMulti);
    };
    Acc acc = acc_zero(), afirst = acc_zero(), alast = acc_zero();
    int G = 1, Gfirst = 1;
    uint32_t pt = 0;  // last position of the piece being summed
    if (have) {
      for (uint32_t p1 = e; p1 > a;) {  // batches [p0, p1), walked backward, loads in flight at once
        const uint32_t p0 = p1 - a >= 4u ? p1 - 4 : a;
        uint32_t kq[6], iq[4];  // kq[i]: key at p0 - 1 + i
        uint64_t vq[4];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const uint32_t q = p0 - 1 + i;
          kq[i] = (i > 0 || p0 > 0) && q < e && q <= p1 ? skey[q] : 0u;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) iq[i] = p0 + i < p1 ? perm[p0 + i] : 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) vq[i] = p0 + i < p1 ? RV[2 * iq[i] + 1] : 0ull;
#pragma unroll
        for (int i = 3; i >= 0; --i) {
          const uint32_t p = p0 + i;
          if (p < p1) {
            const uint32_t kc = kq[i + 1];
            const bool t = p + 1 == e ? tail_e : kq[i + 2] != kc;
            const bool h = p == a ? head_a : kq[i] != kc;
            const uint32_t ix = iq[i];
            const uint64_t raw = vq[i];
            if (p + 1 == e || t) {  // a piece ends at p
              pt = p;
              int pm = t ? (int)rmax[p] : max(run, inB);  // (run: pass 1's largest of the last piece)
              if (cont_in && (t ? p == ft : ft == ~0u)) pm = max(pm, inF);
              G = max(pm, 1);
              acc = acc_zero();
            }
            if (h && t) {  // a single write: its own value (already in place)
              if (bits_nonzero<F64>(raw)) {
                perm[p] = (uint16_t)(ix | kKept);
                ++nk;
              }
            } else {
              acc_add_fast(acc, wide<F64>(raw), G);
              if (h || p == a) {  // the piece's first position
                const bool has_tail = pt + 1 != e || tail_e;
                if (!has_tail) {
                  alast = acc;  // continues in the next lane
                } else if (!h) {
                  afirst = acc;  // continued from the lane before: finished after the scan
                  Gfirst = G;
                } else {
                  park_run(pt, acc, G);
                }
              }
            }
          }
        }
        p1 = p0;
      }
    }
    const AV inA = warp_seg_scan<true>(!have || anyhead, av_of(alast), AV{0, 0, 0}, OpAdd());
    if (cont_in && ft != ~0u) park_run(ft, acc_of(av_add(inA, av_of(afirst))), Gfirst);
    __syncwarp();
    // round the parked runs of the warp's positions, up to 32 at once
    uint16_t* const rq = S.ring[wid];
    uint32_t pend = 0, head = 0, mk = 0;
    const unsigned lt = (1u << lane) - 1u;
    auto round_parked = [&](uint32_t cnt) {
      bool kept = false;
      if ((uint32_t)lane < cnt) {
        const uint32_t p = rq[(head + lane) & 63u];
        const uint32_t ix = perm[p] & kIdx;
        const uint4 sl = park[MAP ? p : ix];
        const uint32_t gf = rmax[p];
        const Acc x{((uint64_t)sl.y << 32) | sl.x, (int64_t)(((uint64_t)sl.w << 32) | sl.z), gf >> 12};
        bool nz;
        RVw[2 * ix + 1] = acc_round(x, (int)(gf & 0xfffu), !F64, &nz);
        perm[p] = (uint16_t)(ix | (nz ? kKept : 0u));
        kept = nz;
      }
      mk += __popc(__ballot_sync(kFull, kept));
      head += cnt;
      pend -= cnt;
      __syncwarp();
    };
    for (uint32_t q0 = A; q0 < E; q0 += 32) {
      const uint32_t p = q0 + lane;
      const bool m = p < E && (perm[p] & kMulti);
      const unsigned bal = __ballot_sync(kFull, m);
      if (m) rq[(head + pend + __popc(bal & lt)) & 63u] = (uint16_t)p;
      pend += __popc(bal);
      __syncwarp();
      if (pend >= 32u) round_parked(32u);
    }
    if (pend) round_parked(pend);
    if (MAP) {
      // the lane's own count, for the positional map below
      nk = 0;
      for (uint32_t p = a; p < e; ++p) nk += (perm[p] & kKept) ? 1u : 0u;
    } else if (lane == 0) {
      nk += mk;  // (only the warp's total is used without the map)
    }
    }
  } else {
    // last write: the largest (seq, position) of each run
    WV w{0, 0, 0, 0}, wfirst{0, 0, 0, 0};
    bool anyhead = false;
    if (have) {
      bool h = head_a;
      for (uint32_t p0 = a; p0 < e; p0 += 4) {  // four positions' loads in flight at once
        uint32_t kq[5], iq[4];
        uint4 rq[4];
#pragma unroll
        for (int i = 0; i < 5; ++i) kq[i] = p0 + i < e ? skey[p0 + i] : 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) iq[i] = p0 + i < e ? perm[p0 + i] : 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) rq[i] = p0 + i < e ? R[iq[i]] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t p = p0 + i;
          if (p < e) {
            const bool t = p + 1 == e ? tail_e : kq[i + 1] != kq[i];
            const uint32_t ix = iq[i];
            const uint4 r = rq[i];
            const uint64_t sq = SEQ ? __ldg(c.seq + r.y) : 0ull;
            if (h) w.ok = 0;
            const WV cand{sq, ((uint64_t)r.w << 32) | r.z, r.y, 1};
            if (wv_better(w, cand)) w = cand;
            anyhead = anyhead || h;
            if (t) {
              if (ft == ~0u && cont_in) {
                wfirst = w;
              } else {
                RVw[2 * ix + 1] = w.val;
                if (MAP) R[ix].x = w.pos;  // (the key field is free after the sort)
                if (keep_zeros || bits_nonzero<F64>(w.val)) {
                  perm[p] = (uint16_t)(ix | kKept);
                  ++nk;
                }
              }
              if (ft == ~0u) ft = p;
            }
            h = t;
          }
        }
      }
    }
    const WV inW = warp_seg_scan<true>(!have || anyhead, w, WV{0, 0, 0, 0}, OpWin());
    if (cont_in && ft != ~0u) {
      const WV r = wv_better(inW, wfirst) ? wfirst : inW;
      const uint32_t it = perm[ft];
      RVw[2 * it + 1] = r.val;
      if (MAP) R[it].x = r.pos;
      if (keep_zeros || bits_nonzero<F64>(r.val)) {
        perm[ft] = (uint16_t)(it | kKept);
        ++nk;
      }
    }
  }

  // ---- number the stored elements: lanes, then warps (in key order)
numbered:
  uint32_t inc = nk;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) S.wk[wid] = inc;
  __syncthreads();
  uint32_t woff = 0, nnz = 0;
#pragma unroll
  for (int w2 = 0; w2 < kRW; ++w2) {
    const uint32_t x = S.wk[w2];
    woff += w2 < wid ? x : 0u;
    nnz += x;
  }
  const uint32_t li0 = woff + inc - nk;
  if (mode == kCount) {
    __syncthreads();
    return nnz;
  }
  if (mode == kDefer) {
    // the warp's positions in lane order (consecutive stored elements go to
    // consecutive words: coalesced stores, conflict-free shared loads)
    uint32_t* const dk = res_keys(c, D.start);
    uint64_t* const dv = res_vals(c, D.start, D.n);
    uint32_t wl = woff;
    for (uint32_t q0 = A; q0 < E; q0 += 64) {  // two positions per lane in flight
      const uint32_t p = q0 + lane, p2 = p + 32;
      const uint32_t ix = p < E ? perm[p] : 0u, ix2 = p2 < E ? perm[p2] : 0u;
      const bool kept = (ix & kKept) != 0, kept2 = (ix2 & kKept) != 0;
      const uint32_t k1 = kept ? unband(skey[p]) : 0u, k2 = kept2 ? unband(skey[p2]) : 0u;
      const uint64_t v1 = kept ? RV[2 * (ix & kIdx) + 1] : 0ull;
      const uint64_t v2 = kept2 ? RV[2 * (ix2 & kIdx) + 1] : 0ull;
      const unsigned b1 = __ballot_sync(kFull, kept), b2 = __ballot_sync(kFull, kept2);
      const unsigned lt = (1u << lane) - 1u;
      if (kept) {
        const uint32_t li = wl + __popc(b1 & lt);
        dk[li] = k1;
        dv[li] = v1;
      }
      wl += __popc(b1);
      if (kept2) {
        const uint32_t li = wl + __popc(b2 & lt);
        dk[li] = k2;
        dv[li] = v2;
      }
      wl += __popc(b2);
    }
    return nnz;  // (the caller's barrier ends every read of the shared arrays)
  }
  // ---- kNow: output index, the map, staging, placement
  OV inO{INT_MIN, 0};
  if (MAP) {
    // output index (local) and winner of the first run ending in this lane,
    // for the positions of a run that ends in a later lane
    OV mine{INT_MIN, 0};
    if (ft != ~0u) {
      const uint32_t it = perm[ft];
      mine.out = (it & kKept) ? (int32_t)li0 : -2;
      mine.win = SUM ? 0u : R[it & kIdx].x;
    }
    inO = warp_seg_scan<false>(!have || ft != ~0u, mine, OV{INT_MIN, 0}, OpNear());
  }
  if (tid < 32) {
    const int64_t b = get_base(nnz);
    if (tid == 0) S.base = b;
  }
  __syncthreads();
  if (S.abort) return 0;
  const int64_t base = S.base;
  if (MAP) {
    // every write of a stored run maps to its element; overwritten writes to -1
    int32_t cur_out = inO.out == INT_MIN ? -2 : (inO.out >= 0 ? (int32_t)(base + inO.out) : inO.out);
    uint32_t cur_win = inO.win;
    uint32_t li = li0 + nk;
    for (uint32_t p = e; p-- > a;) {
      const uint32_t ix = perm[p];
      const bool t = p + 1 == e ? tail_e : skey[p + 1] != skey[p];
      const uint4 r = R[ix & kIdx];
      if (t) {
        if (ix & kKept) {
          --li;
          cur_out = (int32_t)(base + li);
        } else {
          cur_out = -2;
        }
        cur_win = SUM ? 0u : r.x;
      }
      c.map[r.y] = (!SUM && r.y != cur_win) ? -1 : cur_out;
    }
  }
  uint32_t* const sk = reinterpret_cast<uint32_t*>(smem + L.stage_key);
  uint64_t* const sv = reinterpret_cast<uint64_t*>(smem + L.stage_val);
  {
    uint32_t wl = woff;  // the warp's positions in lane order, as in kDefer
    for (uint32_t q0 = A; q0 < E; q0 += 32) {
      const uint32_t p = q0 + lane;
      const uint32_t ix = p < E ? perm[p] : 0u;
      const bool kept = (ix & kKept) != 0;
      const unsigned b1 = __ballot_sync(kFull, kept);
      if (kept) {
        const uint32_t li = wl + __popc(b1 & ((1u << lane) - 1u));
        sk[li] = skey[p];
        sv[li] = RV[2 * (ix & kIdx) + 1];
      }
      wl += __popc(b1);
    }
  }
  __syncthreads();
  emit_range<F64>(c, D, Rg, nnz, base, [&](uint32_t i, uint32_t& k, uint64_t& v) {
    k = sk[i];
    v = sv[i];
  });
  __syncthreads();
  return nnz;
}

// ---------------------------------------------------------------------------
// One key with more writes than a window holds (streaming, records in global
// memory).  Returns 1 if its element is stored.  Ends with a barrier.
// ---------------------------------------------------------------------------
template <bool F64, bool SUM, bool SEQ, bool MAP>
__device__ __noinline__ uint32_t resolve_key(const Ctx& c, RShared& S, unsigned char* smem, const Desc& D,
                                             const uint4* recs, uint32_t lkey, uint64_t kabs, bool emit,
                                             int64_t base) {
  constexpr RLay L = rlay();
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t n = D.n;
  if (tid == 0) S.kmax = 0;
  __syncthreads();
  if (SUM) {
    int e = 0;
    for (uint32_t k = tid; k < n; k += kRT) {
      const uint4 r = __ldcg(recs + k);
      if (r.x == lkey) e = max(e, align_exp<F64>(((uint64_t)r.w << 32) | r.z));
    }
    e = __reduce_max_sync(kFull, e);
    if (lane == 0) atomicMax(&S.kmax, e);
    __syncthreads();
    const int G = max(S.kmax, 1);
    Acc a = acc_zero();
    for (uint32_t k = tid; k < n; k += kRT) {
      const uint4 r = __ldcg(recs + k);
      if (r.x == lkey) acc_add_bits(a, wide<F64>(((uint64_t)r.w << 32) | r.z), G);
    }
    AV v = av_of(a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = av_add(v, AV{__shfl_xor_sync(kFull, v.lo, o), __shfl_xor_sync(kFull, v.hi, o), __shfl_xor_sync(kFull, v.f, o)});
    AV* parts = reinterpret_cast<AV*>(S.parts);
    if (lane == 0) parts[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      AV t{0, 0, 0};
      for (int w = 0; w < kRW; ++w) t = av_add(t, parts[w]);
      bool nz;
      S.kbits = acc_round(acc_of(t), G, !F64, &nz);
      S.kkeep = nz ? 1u : 0u;
      S.kwin = 0;
    }
  } else {
    WV w{0, 0, 0, 0};
    for (uint32_t k = tid; k < n; k += kRT) {
      const uint4 r = __ldcg(recs + k);
      if (r.x != lkey) continue;
      const WV cand{SEQ ? __ldg(c.seq + r.y) : 0ull, ((uint64_t)r.w << 32) | r.z, r.y, 1};
      if (wv_better(w, cand)) w = cand;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const WV x{__shfl_xor_sync(kFull, w.seq, o), __shfl_xor_sync(kFull, w.val, o), __shfl_xor_sync(kFull, w.pos, o),
                 __shfl_xor_sync(kFull, w.ok, o)};
      if (wv_better(w, x)) w = x;
    }
    WV* parts = reinterpret_cast<WV*>(S.parts);
    if (lane == 0) parts[tid >> 5] = w;
    __syncthreads();
    if (tid == 0) {
      WV t{0, 0, 0, 0};
      for (int q = 0; q < kRW; ++q)
        if (wv_better(t, parts[q])) t = parts[q];
      S.kbits = t.val;
      S.kkeep = (c.keep_zeros || bits_nonzero<F64>(t.val)) ? 1u : 0u;
      S.kwin = t.pos;
    }
  }
  __syncthreads();
  const uint32_t keep = S.kkeep;
  if (emit) {
    uint32_t* sk = reinterpret_cast<uint32_t*>(smem + L.stage_key);
    uint64_t* sv = reinterpret_cast<uint64_t*>(smem + L.stage_val);
    if (tid == 0) {
      sk[0] = 0u;
      sv[0] = S.kbits;
      S.win = make_range((uint64_t)D.n_rows, kabs, 1);
    }
    __syncthreads();
    emit_range<F64>(c, D, S.win, keep, base, [&](uint32_t i, uint32_t& k, uint64_t& v) {
      k = sk[i];
      v = sv[i];
    });
    if (MAP) {
      const uint32_t wp = S.kwin;
      for (uint32_t k = tid; k < n; k += kRT) {
        const uint4 r = __ldcg(recs + k);
        if (r.x == lkey) c.map[r.y] = (!SUM && r.y != wp) ? -1 : (keep ? (int32_t)base : -2);
      }
    }
  }
  __syncthreads();
  return keep;
}

// ---------------------------------------------------------------------------
// A bucket with more writes than fit: windows of its key range, each gathered
// into shared memory (at most kRCapNow writes, so that its elements can be
// staged and placed at once).
// ---------------------------------------------------------------------------
template <bool F64, bool SUM, bool SEQ, bool MAP>
__device__ __noinline__ uint32_t resolve_windows(const Ctx& c, RShared& S, unsigned char* smem, const Desc& D,
                                                 bool emit, int64_t base) {
  constexpr RLay L = rlay();
  uint4* const R = reinterpret_cast<uint4*>(smem + L.R);
  uint32_t* const bins = reinterpret_cast<uint32_t*>(smem + L.bins);
  const uint4* recs = reinterpret_cast<const uint4*>(c.rec + D.start);
  const int tid = threadIdx.x;
  const uint32_t n = D.n;
  const uint64_t span = D.rg.span;
  uint32_t running = 0;
  uint64_t wlo = 0;
  while (wlo < span) {
    int hs = (span - wlo <= 1) ? 0 : max(0, ceil_log2_u64(span - wlo) - c.sub_bits);
    uint64_t wend = span, whi = wlo + 1;
    int mode = 0;  // 1 = window, 2 = single key
    while (true) {
      const uint32_t nb = (uint32_t)(((wend - wlo - 1) >> hs) + 1);
      for (uint32_t q = tid; q < nb; q += kRT) bins[q] = 0u;
      __syncthreads();
      for (uint32_t k = tid; k < n; k += kRT) {
        const uint64_t l = __ldcg(&recs[k].x);
        if (l >= wlo && l < wend) atomicAdd(&bins[(uint32_t)((l - wlo) >> hs)], 1u);
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t cum = 0, taken = 0;
        while (taken < nb && cum + bins[taken] <= (uint32_t)kRCapNow) cum += bins[taken++];
        S.taken = taken;
      }
      __syncthreads();
      const uint32_t taken = S.taken;
      __syncthreads();
      if (taken > 0) {
        whi = min(wlo + ((uint64_t)taken << hs), wend);
        mode = 1;
        break;
      }
      if (hs == 0) {
        mode = 2;
        break;
      }
      wend = wlo + (uint64_t{1} << hs);
      hs = max(0, hs - c.sub_bits);
    }
    if (mode == 1) {
      if (tid == 0) {
        S.nw = 0;
        S.win = make_range((uint64_t)D.n_rows, D.rg.klo + wlo, whi - wlo);
      }
      __syncthreads();
      for (uint32_t k = tid; k < n; k += kRT) {
        const uint4 r = __ldcg(recs + k);
        if (r.x >= wlo && r.x < whi) R[atomicAdd(&S.nw, 1u)] = make_uint4(r.x - (uint32_t)wlo, r.y, r.z, r.w);
      }
      __syncthreads();
      const uint32_t nw = S.nw;
      const int64_t b0 = base + running;
      running += resolve_tile<F64, SUM, SEQ, MAP>(c, S, smem, nw, D, S.win, emit ? kNow : kCount,
                                                  [&](uint32_t) { return b0; });
      wlo = whi;
    } else {
      running += resolve_key<F64, SUM, SEQ, MAP>(c, S, smem, D, recs, (uint32_t)wlo, D.rg.klo + wlo, emit,
                                                 base + running);
      wlo += 1;
    }
  }
  return running;
}

// ---------------------------------------------------------------------------
// The kernels
// ---------------------------------------------------------------------------
// Thread kHelper takes the tickets and reads the next bucket's descriptor
// while the block waits for the current bucket's bulk copy.
constexpr int kHelper = kRT - 1;

// Start the bulk copy of bucket D into record slots [rb, rb + D.n) of the
// record area (thread 0; those slots are dead).
__device__ __forceinline__ void start_bucket(const Ctx& c, RShared& S, unsigned char* smem, const Desc& D,
                                             uint32_t cap, uint32_t rb) {
  if (D.n > 0 && D.n <= cap) {
    fence_proxy_async();
    mbar_expect_tx(&S.bar, D.n * 16u);
    bulk_load(smem + rlay().R + (size_t)16 * rb, c.rec + D.start, D.n * 16u, &S.bar);
  }
}

// Copy records [off, off + cnt) of bucket D into slots [dst, dst + cnt)
// (thread 0); `arrive`: this copy completes the barrier's phase, else a later
// one of the same phase does.
__device__ __forceinline__ void copy_part(const Ctx& c, RShared& S, unsigned char* smem, const Desc& D, uint32_t off,
                                          uint32_t cnt, uint32_t dst, bool arrive) {
  fence_proxy_async();
  if (arrive) mbar_expect_tx(&S.bar, cnt * 16u);
  else mbar_expect_tx_only(&S.bar, cnt * 16u);
  bulk_load(smem + rlay().R + (size_t)16 * dst, c.rec + D.start + off, cnt * 16u, &S.bar);
}

// Drop the L2 lines that lie entirely inside [a0, a1) (dead data), so that
// they are never written back to HBM.
__device__ __forceinline__ void discard_lines(const void* p0, const void* p1) {
  const uint64_t a0 = reinterpret_cast<uint64_t>(p0), a1 = reinterpret_cast<uint64_t>(p1);
  const uint64_t l0 = (a0 + 127) & ~127ull, l1 = a1 & ~127ull;
  for (uint64_t a = l0 + (uint64_t)threadIdx.x * 128; a < l1; a += (uint64_t)blockDim.x * 128)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
}

// Output index of a bucket's first element (relative to its matrix), from the
// scan of the per-bucket element counts.
__device__ __forceinline__ int64_t bucket_base(const Ctx& c, const Desc& D) {
  return (int64_t)c.bk_out[D.b] - (int64_t)c.bk_out[D.bucket_off];
}

template <bool F64, bool SUM, bool SEQ, bool MAP>
__global__ void __launch_bounds__(kRT, 1) k_resolve(Ctx c) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ RShared S;
  __shared__ Desc nxt;    // the next bucket's descriptor
  __shared__ DescRaw raw;  // its table entries, fetched asynchronously a bucket earlier
  const int tid = threadIdx.x;
  const uint32_t NB = c.scal->NB;
  const uint32_t cap = MAP ? (uint32_t)kRCapNow : (uint32_t)kRCap;  // writes resolved from shared memory
  // (thread kHelper) the tickets of the next bucket (its entries in flight)
  // and of the one after it, and the matrix of the last descriptor it built
  uint32_t t1 = ~0u, t2 = ~0u;
  int64_t mi_cached = -1;
  MatMeta mm_cached;
  if (tid == 0) {
    mbar_init(&S.bar, 1);
    fence_mbar_init();
    S.abort = 0;
    S.rb = 0;
    S.pre = 0;
    const uint32_t t = is_aborted(c) ? ~0u : atomicAdd(&c.scal->ticket, 1u);
    S.cur.valid = 0;
    S.cur.b = t;
    if (t < NB) {
      S.cur = load_desc(c, t);
      start_bucket(c, S, smem, S.cur, cap, 0);
    }
  }
  __syncthreads();
  if (tid == kHelper && S.cur.valid) {
    t1 = is_aborted(c) ? ~0u : atomicAdd(&c.scal->ticket, 1u);
    if (t1 < NB) {
      raw_fetch(c, t1, &raw);
      t2 = is_aborted(c) ? ~0u : atomicAdd(&c.scal->ticket, 1u);
    }
  }
  uint32_t phase = 0;
  bool copying = false;  // a bulk copy has been started and not yet waited for
  while (true) {
    if (!S.cur.valid) break;
    copying = S.cur.n > 0 && S.cur.n <= cap;
    const Desc& D = S.cur;
    // the next bucket's descriptor, built from its table entries (fetched a
    // bucket earlier) while this bucket's copy is in flight; then the entries
    // of the bucket after it are fetched and the ticket after that taken,
    // both waited for only a bucket later
    if (tid == kHelper) {
      nxt.valid = 0;
      nxt.b = ~0u;
      if (t1 < NB) {
        cp_async_commit_wait();
        const uint32_t mi = raw.info >> 6;
        if ((int64_t)mi != mi_cached) {
          mm_cached = c.meta[mi];
          mi_cached = mi;
        }
        nxt = make_desc(t1, raw.n, raw.start, raw.info, raw.klo, mm_cached);
        // warm L2 with its records, a bucket's time before its bulk copy
        if (nxt.n <= cap) prefetch_l2(c.rec + nxt.start, nxt.n * 16u);
      }
      t1 = t2;
      t2 = ~0u;
      if (t1 < NB) {
        raw_fetch(c, t1, &raw);
        t2 = is_aborted(c) ? ~0u : atomicAdd(&c.scal->ticket, 1u);
      }
    }
    int64_t total = -1;  // set when the bucket is placed here
    const void* dead0 = c.rec + D.start;  // records (or parts) dead after this bucket
    if (D.K == 0) {  // an empty matrix: all offsets are 0
      for (int64_t j = tid; j <= D.n_cols; j += kRT) c.col_ptr[D.col_base + j] = 0;
      if (tid == 0) {
        if (MAP) st_release_u64(&c.bk_state[D.b], kStIncl);
        else c.bk_nnz[D.b] = 0u;
      }
      total = 0;
    } else if (D.n > cap) {
      // more writes than fit: windows of the key range
      const uint32_t cnt = resolve_windows<F64, SUM, SEQ, MAP>(c, S, smem, D, false, 0);
      if (MAP) {
        // resolved twice: counted, then placed after the look-back
        if (tid < 32) {
          int64_t ex = 0;
          if (D.rg.klo == 0) {
            if (tid == 0) st_release_u64(&c.bk_state[D.b], kStIncl | (uint64_t)cnt);
          } else if ((int64_t)D.b != c.withhold) {
            ex = lookback_warp(c, D.b, cnt);
          }
          if (tid == 0) {
            S.base = ex;
            S.abort = is_aborted(c) ? 1u : 0u;
          }
        }
        __syncthreads();
        if (S.abort) break;
        const int64_t base = S.base;
        __syncthreads();
        resolve_windows<F64, SUM, SEQ, MAP>(c, S, smem, D, true, base);
        total = base + cnt;
      } else if (tid == 0) {
        // placed by k_big once the offsets are known
        c.bk_nnz[D.b] = cnt;
        c.big_list[atomicAdd(&c.scal->big_n, 1u)] = D.b;
      }
      dead0 = nullptr;  // (k_big reads the records again)
    } else {
      bool ok = true;
      if (D.n > 0) {
        ok = mbar_wait_bounded(&S.bar, phase);
        phase ^= 1u;
        copying = false;
      }
      if (__syncthreads_or(!ok)) {
        // the copy is still in flight: record the error, give it one more
        // bounded wait, and leave
        if (tid == 0) record_fatal(c, SPM_ERR_TIMEOUT);
        if (!ok) mbar_wait_bounded(&S.bar, phase ^ 1u);
        __syncthreads();
        break;
      }
      if (MAP) {
        const uint32_t b = D.b;
        const bool first = D.rg.klo == 0;
        const uint32_t nnz = resolve_tile<F64, SUM, SEQ, MAP>(c, S, smem, D.n, D, D.rg, kNow, [&](uint32_t cnt) {
          int64_t ex = 0;
          if (first) {
            if ((threadIdx.x & 31) == 0) st_release_u64(&c.bk_state[b], kStIncl | (uint64_t)cnt);
          } else if ((int64_t)b != c.withhold) {
            ex = lookback_warp(c, b, cnt);  // fault injection: a withheld bucket publishes nothing
          }
          if (threadIdx.x == 0 && is_aborted(c)) S.abort = 1;
          return ex;
        });
        if (S.abort) break;
        total = S.base + nnz;
      } else {
        // the next bucket goes to the other end of the record area: the part
        // of its copy that does not land on this bucket's records starts now,
        // while this one is resolved, the rest once it is done
        if (tid == 0 && nxt.valid && nxt.K > 0 && nxt.n > 0 && nxt.n <= cap) {
          const uint32_t n2 = nxt.n;
          const bool top = S.rb == 0;  // this bucket at the bottom: the next one at the top
          const uint32_t r2 = top ? cap - n2 : 0;
          const uint32_t c0 = S.rb, c1 = S.rb + D.n;  // slots in use
          const uint32_t ov = top ? (c1 > r2 ? c1 - r2 : 0u) : (n2 > c0 ? n2 - c0 : 0u);  // overlap
          S.rb_next = r2;
          S.pre = 1;
          S.late_cnt = ov;
          S.late_off = top ? 0u : n2 - ov;
          if (ov < n2) {  // the early part: after the overlap (top) or before it (bottom)
            if (top) copy_part(c, S, smem, nxt, ov, n2 - ov, r2 + ov, ov == 0);
            else copy_part(c, S, smem, nxt, 0, n2 - ov, 0, ov == 0);
          }
        }
        // the elements wait over the bucket's records for k_place
        const uint32_t rb = S.rb;
        uint32_t nnz = kDenseNo;
        if (!SEQ && D.rg.span <= kDense) nnz = resolve_dense<F64, SUM>(c, S, smem, D.n, D, rb);
        if (nnz == kDenseNo) {
          nnz = resolve_tile<F64, SUM, SEQ, MAP>(c, S, smem, D.n, D, D.rg, kDefer, [](uint32_t) {
            return int64_t{0};
          }, rb);
        }
        if (tid == 0) c.bk_nnz[D.b] = nnz;
        dead0 = res_vals(c, D.start, D.n) + nnz;
      }
    }
    if (total >= 0 && tid == 0 && D.rg.klo + D.rg.span == D.K) {
      c.col_ptr[D.col_base + D.n_cols] = total;
      c.d_nnz[D.mi] = total;
    }
    const void* dead1 = c.rec + D.start + D.n;
    fence_proxy_async();  // this thread's writes to the record area come before the next bulk copy
    __syncthreads();      // the record area and the descriptors are free
    if (tid == 0) {
      S.cur = nxt;
      if (S.pre) {
        S.rb = S.rb_next;  // (part of) its copy is in flight already
        if (S.late_cnt) copy_part(c, S, smem, S.cur, S.late_off, S.late_cnt, S.rb + S.late_off, true);
      } else {
        S.rb = 0;
        if (S.cur.valid) start_bucket(c, S, smem, S.cur, cap, 0);
      }
      S.pre = 0;
    }
    if (dead0) discard_lines(dead0, dead1);
    __syncthreads();
  }
  if (copying) mbar_wait_bounded(&S.bar, phase);  // (a call that stopped early)
  if (tid == kHelper) asm volatile("cp.async.wait_all;" ::: "memory");  // (no copy outlives the block)
}

// Calls without the map: every bucket's elements wait over its records, in
// key order (keys relative to the bucket, values); one block per bucket writes
// them to their place in the CSC arrays, with the offsets of the columns that
// start in the bucket.
template <bool F64>
__global__ void __launch_bounds__(256) k_place(Ctx c) {
  __shared__ Desc D;
  __shared__ int64_t s_base;
  __shared__ uint32_t s_nnz, s_skip;
  const uint32_t b = blockIdx.x;
  if (b >= c.scal->NB || is_aborted(c)) return;
  if (threadIdx.x == 0) {
    D = load_desc(c, b);
    s_skip = (D.K == 0 || D.n > (uint32_t)kRCap) ? 1u : 0u;  // (placed by k_resolve / k_big)
    s_nnz = c.bk_nnz[b];
    s_base = bucket_base(c, D);
  }
  __syncthreads();
  if (s_skip) return;
  const uint32_t nnz = s_nnz;
  const int64_t base = s_base;
  const uint32_t* keys = res_keys(c, D.start);
  const uint64_t* vals = res_vals(c, D.start, D.n);
  emit_range<F64>(c, D, D.rg, nnz, base, [&](uint32_t i, uint32_t& k, uint64_t& v) {
    k = __ldcs(keys + i);
    v = __ldcs(reinterpret_cast<const unsigned long long*>(vals) + i);
  });
  if (threadIdx.x == 0 && D.rg.klo + D.rg.span == D.K) {
    c.col_ptr[D.col_base + D.n_cols] = base + nnz;
    c.d_nnz[D.mi] = base + nnz;
  }
}

// Calls without the map: the buckets with more writes than fit (counted by
// k_resolve), resolved again in windows and placed at once.
template <bool F64, bool SUM, bool SEQ>
__global__ void __launch_bounds__(kRT, 1) k_big(Ctx c) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ RShared S;
  const uint32_t nbig = c.scal->big_n;
  if (threadIdx.x == 0) S.abort = 0;
  for (uint32_t i = blockIdx.x; i < nbig && !is_aborted(c); i += gridDim.x) {
    if (threadIdx.x == 0) {
      S.cur = load_desc(c, c.big_list[i]);
      S.base = bucket_base(c, S.cur);
    }
    __syncthreads();
    const Desc& D = S.cur;
    const int64_t base = S.base;
    __syncthreads();
    const uint32_t cnt = resolve_windows<F64, SUM, SEQ, false>(c, S, smem, D, true, base);
    if (threadIdx.x == 0 && D.rg.klo + D.rg.span == D.K) {
      c.col_ptr[D.col_base + D.n_cols] = base + cnt;
      c.d_nnz[D.mi] = base + cnt;
    }
    __syncthreads();
  }
}

template <typename K>
int resident_blocks(K kernel, int sms, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRT, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return sms * per_sm;
}

}  // namespace

int resolve_capacity(bool map) { return map ? kRCapNow : kRCap; }

// Every instantiation: value type x (add mode with or without the map; last
// write with or without seq, with or without the map).
#define SPM_RES_ALL(X) \
  X(true, true, false, false) X(true, true, false, true) X(true, false, false, false) X(true, false, false, true) \
  X(true, false, true, false) X(true, false, true, true) X(false, true, false, false) X(false, true, false, true) \
  X(false, false, false, false) X(false, false, false, true) X(false, false, true, false) X(false, false, true, true)

void resolve_set_attributes() {
  const int bytes = (int)rlay().total;
#define SPM_ATTR(F6, SU, SQ, MP) \
  cudaFuncSetAttribute(k_resolve<F6, SU, SQ, MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); \
  cudaFuncSetAttribute(k_big<F6, SU, SQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  SPM_RES_ALL(SPM_ATTR)
#undef SPM_ATTR
}

void launch_resolve(const Ctx& ctx, int sms, int64_t nbcap, cudaStream_t st) {
  const size_t bytes = rlay().total;
  const int64_t nb = std::max<int64_t>(nbcap, 1);  // (no more blocks than buckets)
  const bool f64 = ctx.f64 != 0, sum = ctx.sum_mode != 0, seq = ctx.has_seq != 0, map = ctx.keep_map != 0;
#define SPM_RES(F6, SU, SQ, MP)                                                                              \
  if (f64 == F6 && sum == SU && seq == SQ && map == MP) {                                                   \
    k_resolve<F6, SU, SQ, MP>                                                                                \
        <<<(unsigned)std::min<int64_t>(resident_blocks(k_resolve<F6, SU, SQ, MP>, sms, bytes), nb), kRT, bytes, \
           st>>>(ctx);                                                                                       \
    return;                                                                                                 \
  }
  SPM_RES_ALL(SPM_RES)
#undef SPM_RES
}

void launch_place(const Ctx& ctx, int sms, int64_t nbcap, cudaStream_t st) {
  const size_t bytes = rlay().total;
  const bool f64 = ctx.f64 != 0, sum = ctx.sum_mode != 0, seq = ctx.has_seq != 0;
  const unsigned blocks = (unsigned)std::max<int64_t>(nbcap, 1);  // one per bucket (NB <= nbcap)
  if (f64) k_place<true><<<blocks, 256, 0, st>>>(ctx);
  else k_place<false><<<blocks, 256, 0, st>>>(ctx);
#define SPM_BIG(F6, SU, SQ, MP)                             \
  if (!MP && f64 == F6 && sum == SU && seq == SQ) {         \
    k_big<F6, SU, SQ><<<(unsigned)std::min<int64_t>(sms, blocks), kRT, bytes, st>>>(ctx); \
    return;                                                 \
  }
  SPM_RES_ALL(SPM_BIG)
#undef SPM_BIG
}
#undef SPM_RES_ALL

}  // namespace spm

