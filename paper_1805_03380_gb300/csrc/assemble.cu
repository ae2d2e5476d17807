// libspm: the sync step of the hybrid sparse matrix class on GB300 (sm_103a).
//
// The paper (Sanderson & Curtin, Section 3.3) converts its red-black tree to
// CSC by an in-order traversal: the tree is keyed by index = row + col*n_rows,
// so the traversal visits elements in column-major order and each index is
// decoded with a division and a modulo.  On the GPU the same result is built
// from an unordered write stream by a bucketed sort over that key:
//
//   sample   -> a few hundred thousand keys drawn at fixed pseudo-random
//               positions give the key distribution (hot columns included)
//   plan     -> per matrix, a two-level lookup table maps a key in O(1) to a
//               bucket: an aligned power-of-two key range expected to hold
//               ~bucket_target writes; hot level-1 cells are refined into 256
//               level-2 cells so that skewed (Zipf) columns still split evenly
//   hist     -> one pass over (row, col) counts writes per (block, bucket)
//   scan     -> per-bucket and per-(block, bucket) offsets
//   scatter  -> one pass over (row, col, value) writes a 16-byte record
//               {key within the bucket, stream position, value} into the
//               bucket's contiguous range (or two passes, through groups of
//               buckets, when one pass would leave too many partly written
//               cache lines)
//   resolve  -> resolve.cu: a persistent kernel loads each bucket into shared
//               memory, sorts it (or reduces it in a key-indexed table when its
//               key range is narrow), resolves repeated writes, drops zeros and
//               writes the bucket's stored elements and count; a scan of the
//               counts and k_place then write the CSC arrays (with the map the
//               resolve kernel places them itself after a decoupled look-back).
//
// No kernel ever traps or spins without a bound: out-of-range indices and
// expired waits are reported in the device status word.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

#include "spm_common.cuh"
#include "device_util.cuh"
#include <climits>

namespace spm {

// ===========================================================================
// Small device helpers
// ===========================================================================
__device__ __forceinline__ uint32_t mix32(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return (uint32_t)x;
}

// Largest i in [lo, hi] with key(i) <= x (requires key(lo) <= x).
template <typename F>
__device__ __forceinline__ int64_t upper_index(int64_t lo, int64_t hi, int64_t x, F key) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo + 1) / 2;
    if (key(mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t isqrt_u32(uint32_t x) {
  uint32_t r = (uint32_t)sqrtf((float)x);
  while ((uint64_t)r * r > x) --r;
  while ((uint64_t)(r + 1) * (r + 1) <= x) ++r;
  return r;
}

// ===========================================================================
// Setup: per-matrix metadata
// ===========================================================================
__global__ void k_setup_single(Ctx c, MatMeta mm) {
  if (threadIdx.x == 0 && blockIdx.x == 0) c.meta[0] = mm;
}

__global__ void k_setup_batched(Ctx c, const int64_t* __restrict__ d_n_rows, const int64_t* __restrict__ d_n_cols,
                                const int64_t* __restrict__ d_trip, int64_t exp_S, int64_t exp_lut, int64_t exp_l2,
                                int64_t exp_nbcap, int64_t exp_cols, unsigned long long exp_hash) {
  __shared__ unsigned long long buf[32];
  __shared__ unsigned long long tot;
  __shared__ unsigned long long hsum;
  __shared__ int bad;
  if (threadIdx.x == 0) {
    bad = 0;
    hsum = 0;
  }
  unsigned long long carry[5] = {0, 0, 0, 0, 0};
  __syncthreads();
  for (int64_t base = 0; base < c.B; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool ok = i < c.B;
    MatMeta mm;
    memset(&mm, 0, sizeof(mm));
    unsigned long long q[5] = {0, 0, 0, 0, 0};
    if (ok) {
      mm.n_rows = d_n_rows[i];
      mm.n_cols = d_n_cols[i];
      mm.t0 = d_trip[i];
      const int64_t t1 = d_trip[i + 1];
      mm.m = t1 - mm.t0;
      atomicAdd(&hsum, (unsigned long long)meta_term(i, mm.n_rows, mm.n_cols, t1));
      if (i == 0 && mm.t0 != 0) atomicExch(&bad, 1);
      bool invalid = mm.n_rows < 0 || mm.n_cols < 0 || mm.n_rows > 0x7fffffffLL || mm.n_cols > 0x7fffffffLL ||
                     mm.m < 0 || mm.t0 < 0 || t1 > c.m_total;
      if (!invalid) {
        Derived d = derive(mm.n_rows, mm.n_cols, mm.m, c.m_total, c.tgt);
        if (d.bbits > kMaxKeyBits) invalid = true;
        mm.K = d.K;
        mm.bbits = d.bbits;
        mm.L1 = d.L1;
        mm.s1 = d.s1;
        mm.H2 = d.H2;
        mm.ns = d.ns;
        mm.lut_len = d.lut_len;
        mm.nbcap = d.nbcap;
        q[0] = (unsigned long long)d.ns;
        q[1] = (unsigned long long)d.lut_len;
        q[2] = (unsigned long long)d.H2;
        q[3] = (unsigned long long)d.nbcap;
        q[4] = (unsigned long long)(mm.n_cols + 1);
      }
      if (invalid) atomicExch(&bad, 1);
    }
    unsigned long long off[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      off[k] = block_scan_excl<unsigned long long>(q[k], &tot, buf) + carry[k];
      carry[k] += tot;
    }
    if (ok) {
      mm.samp_off = (int64_t)off[0];
      mm.lut_off = (int64_t)off[1];
      mm.l2_off = (int64_t)off[2];
      mm.nbcap_off = (int64_t)off[3];
      mm.col_base = (int64_t)off[4];
      c.meta[i] = mm;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bad || hsum != exp_hash || (int64_t)carry[0] != exp_S || (int64_t)carry[1] != exp_lut || (int64_t)carry[2] != exp_l2 ||
        (int64_t)carry[3] != exp_nbcap || (int64_t)carry[4] != exp_cols)
      record_fatal(c, SPM_ERR_INVALID_ARG);
  }
}

// ===========================================================================
// Sampling
// ===========================================================================
// Draw the samples (fixed positions: one per stride of the matrix's writes,
// offset inside the stride by a hash) and count them per level-1 cell.  Lanes
// of a warp that hit the same cell add their count with one atomic.
__global__ void k_sample(Ctx c) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cidx = ~0ull;
  if (g < c.S_total && !is_aborted(c)) {
    const MatMeta* meta = c.meta;
    const int64_t i = upper_index(0, c.B - 1, g, [&](int64_t j) { return meta[j].samp_off; });
    const MatMeta& mm = meta[i];
    const uint64_t k = (uint64_t)(g - mm.samp_off);
    const uint64_t m = (uint64_t)mm.m, ns = (uint64_t)mm.ns;
    uint64_t p;
    if (ns >= m) {
      p = k;
    } else {
      // samples come in groups of eight consecutive writes (one 32-byte
      // sector of rows and of cols per group); group j sits at a hashed
      // offset inside the j-th stretch of m / groups writes
      const uint64_t ng = (ns + 7) / 8, j = k >> 3;
      const uint64_t a = j * m / ng, b = (j + 1) * m / ng;
      const uint64_t room = b - a > 8 ? b - a - 8 : 0;
      const uint64_t off = room ? (mix32(j * 0x9e3779b97f4a7c15ull + (uint64_t)i * 7919 + 17) % room) & ~7ull : 0;
      p = a + off + (k & 7);
      if (p >= m) p = m - 1;
    }
    const int64_t t = mm.t0 + (int64_t)p;
    const int32_t r = c.rows[t], col = c.cols[t];
    uint64_t key = kBadKey;
    if (r >= 0 && (int64_t)r < mm.n_rows && col >= 0 && (int64_t)col < mm.n_cols) {
      key = (uint64_t)col * (uint64_t)mm.n_rows + (uint64_t)r;
      cidx = (unsigned long long)mm.lut_off + (key >> mm.s1);
      // one matrix: also the finer count the planner needs for the cells it
      // refines (a level-2 cell is 2^8 times smaller than a level-1 cell)
      if (c.l2h && mm.H2 > 0) atomicAdd(&c.l2h[key >> (mm.s1 - kL2Bits)], 1u);
    }
    c.samp[g] = key;
  }
  const unsigned peers = __match_any_sync(0xffffffffu, cidx);
  if (cidx != ~0ull && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&c.cellcnt[cidx], (uint32_t)__popc(peers));
}

// ===========================================================================
// Planning: one block per matrix
// ===========================================================================
struct Split {
  int j;
  uint32_t count;
};

// A leaf of 2^shift keys starting at lo, expected to receive `est` writes, is
// split into 2^j equal buckets of at most about tgt writes each; buckets that
// start at or beyond K are not created.
__device__ __forceinline__ Split leaf_split(uint64_t lo, int shift, uint64_t est, uint64_t tgt, uint64_t K) {
  Split s{0, 0};
  if (lo >= K) return s;
  int j = 0;
  if (est > tgt) j = ceil_log2_u64((est + tgt - 1) / tgt);
  if (j > shift) j = shift;
  if (j > 31) j = 31;
  if (j < shift - 32) j = shift - 32;
  const int w = shift - j;
  const uint64_t n = ((K - lo) + ((uint64_t{1} << w) - 1)) >> w;
  const uint64_t full = uint64_t{1} << j;
  s.j = j;
  s.count = (uint32_t)(n < full ? n : full);
  return s;
}

// Writes expected in a region that received `cnt` samples: the count plus a
// one-standard-deviation margin, scaled by writes per sample.
__device__ __forceinline__ uint64_t estimate(uint64_t cnt, const MatMeta& mm) {
  if (mm.ns <= 0) return 0;
  if (mm.ns >= mm.m) return cnt;
  const uint64_t x = cnt + (uint64_t)sqrtf((float)cnt) + 1ull;
  return x * (uint64_t)mm.m / (uint64_t)mm.ns;
}

constexpr int kMergeL1Max = 13;  // cells can be merged when the matrix has at most 2^13 of them
constexpr size_t kPlanSmem = (size_t)kMaxL2Tables * kL2Size * 4 * 2 + ((size_t{1} << kMergeL1Max) + 1) * 8 +
                             ((size_t{1} << kMergeL1Max) + 1) * 2 + 64;

__global__ void __launch_bounds__(1024) k_plan(Ctx c) {
  extern __shared__ __align__(16) unsigned char psm[];
  uint32_t* cnt2 = reinterpret_cast<uint32_t*>(psm);                 // level-2 sample counts
  uint32_t* spl2 = cnt2 + kMaxL2Tables * kL2Size;                    // level-2 splits: j << 27 | count
  uint64_t* P = reinterpret_cast<uint64_t*>(spl2 + kMaxL2Tables * kL2Size);  // prefix of level-1 counts
  uint16_t* T = reinterpret_cast<uint16_t*>(P + (size_t{1} << kMergeL1Max) + 1);  // prefix of table flags
  __shared__ MatMeta mm;
  __shared__ uint32_t buf[32];
  __shared__ unsigned long long buf64[32];
  __shared__ uint32_t s_tot, s_red;
  __shared__ unsigned long long s_tot64;
  __shared__ uint32_t tbl_cell[kMaxL2Tables], tbl_nb[kMaxL2Tables], tbl_base[kMaxL2Tables];
  const int64_t i = blockIdx.x;
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
  if (tid == 0) mm = c.meta[i];
  __syncthreads();
  if (is_aborted(c)) return;
  const uint32_t* cnt = c.cellcnt + mm.lut_off;
  uint32_t* lut = c.lut + mm.lut_off;
  int32_t* l2cell = c.l2cell + mm.l2_off;
  const int64_t L1size = int64_t{1} << mm.L1;
  if (mm.K == 0) {
    if (tid == 0) {
      lut[0] = 0;
      c.meta[i].nb = 1;
      c.meta[i].h2used = 0;
    }
    return;
  }
  const uint64_t* samp = c.samp + mm.samp_off;
  const uint64_t tgt = (uint64_t)c.tgt;
  // ---- level-2 tables for the heaviest cells (at most H2, each worth > 8 buckets)
  uint32_t h = 0;
  if (mm.H2 > 0) {
    const uint64_t thr = 8ull * tgt;
    uint32_t mx = 0;
    for (int64_t cell = tid; cell < L1size; cell += NT) mx = max(mx, cnt[cell]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tid == 0) s_red = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&s_red, mx);
    __syncthreads();
    mx = s_red;
    __syncthreads();
    uint32_t lo = 1, hi = mx + 1;
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo) / 2;
      uint32_t n = 0;
      for (int64_t cell = tid; cell < L1size; cell += NT)
        n += (cnt[cell] >= mid && estimate(cnt[cell], mm) > thr) ? 1u : 0u;
      for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
      if (tid == 0) s_red = 0;
      __syncthreads();
      if (lane == 0) atomicAdd(&s_red, n);
      __syncthreads();
      n = s_red;
      __syncthreads();
      if (n <= (uint32_t)mm.H2) hi = mid; else lo = mid + 1;
    }
    const uint32_t tau = lo;
    uint32_t carry = 0;
    for (int64_t base = 0; base < L1size; base += NT) {
      const int64_t cell = base + tid;
      uint32_t f = 0;
      if (cell < L1size) f = (cnt[cell] >= tau && estimate(cnt[cell], mm) > thr) ? 1u : 0u;
      const uint32_t off = block_scan_excl<uint32_t>(f, &s_tot, buf) + carry;
      if (cell < L1size) {
        lut[cell] = f ? (kPtrFlag | off) : 0u;
        if (f) {
          l2cell[off] = (int32_t)cell;
          tbl_cell[off] = (uint32_t)cell;
        }
      }
      carry += s_tot;
    }
    h = carry;
  } else {
    for (int64_t cell = tid; cell < L1size; cell += NT) lut[cell] = 0u;
  }
  __syncthreads();
  const int s2 = mm.s1 - kL2Bits;
  if (h > 0 && c.l2h) {
    for (uint32_t q = tid; q < h * kL2Size; q += NT)
      cnt2[q] = c.l2h[((uint64_t)tbl_cell[q >> kL2Bits] << kL2Bits) + (q & (kL2Size - 1))];
  } else if (h > 0) {
    for (uint32_t q = tid; q < h * kL2Size; q += NT) cnt2[q] = 0u;
    __syncthreads();
    for (int64_t k = tid; k < mm.ns; k += NT) {
      const uint64_t key = samp[k];
      if (key == kBadKey) continue;
      const uint32_t e = lut[key >> mm.s1];
      if (e & kPtrFlag) atomicAdd(&cnt2[(e & ~kPtrFlag) * kL2Size + ((key >> s2) & (kL2Size - 1))], 1u);
    }
  }
  // ---- prefix sums for merging cold level-1 cells into aligned groups
  const bool merging = mm.L1 <= kMergeL1Max;
  if (merging) {
    unsigned long long carry = 0;
    uint32_t tcarry = 0;
    for (int64_t base = 0; base < L1size; base += NT) {
      const int64_t cell = base + tid;
      const unsigned long long v = cell < L1size ? (unsigned long long)cnt[cell] : 0ull;
      const uint32_t f = (cell < L1size && (lut[cell] & kPtrFlag)) ? 1u : 0u;
      const unsigned long long off = block_scan_excl<unsigned long long>(v, &s_tot64, buf64) + carry;
      const uint32_t toff = block_scan_excl<uint32_t>(f, &s_tot, buf) + tcarry;
      if (cell < L1size) {
        P[cell] = off;
        T[cell] = (uint16_t)toff;
      }
      carry += s_tot64;
      tcarry += s_tot;
    }
    if (tid == 0) {
      P[L1size] = carry;
      T[L1size] = (uint16_t)tcarry;
    }
  }
  __syncthreads();
  const int gcap = min(min(mm.L1, 32 - mm.s1), kMergeL1Max);
  // largest g such that the aligned block of 2^g cells around `cell` has no
  // table and is expected to hold at most tg writes
  auto gmax_of = [&](int64_t cell, uint64_t tg) -> int {
    if (!merging) return 0;
    int g = 0;
    for (int gg = 1; gg <= gcap; ++gg) {
      const int64_t lo_c = (cell >> gg) << gg, hi_c = lo_c + (int64_t{1} << gg);
      if (T[hi_c] != T[lo_c]) break;
      if (estimate(P[hi_c] - P[lo_c], mm) > tg) break;
      g = gg;
    }
    return g;
  };
  // ---- buckets per leaf; retry with a larger target while over the bound
  uint64_t tg = tgt;
  uint32_t nb_total = 0;
  for (int attempt = 0;; ++attempt) {
    for (uint32_t q = tid; q < h * kL2Size; q += NT) {
      const uint32_t tb = q >> kL2Bits, u = q & (kL2Size - 1);
      const uint64_t lo = ((uint64_t)tbl_cell[tb] << mm.s1) + ((uint64_t)u << s2);
      const Split sp = leaf_split(lo, s2, estimate(cnt2[q], mm), tg, mm.K);
      spl2[q] = ((uint32_t)sp.j << 27) | sp.count;
    }
    __syncthreads();
    for (uint32_t tb = warp; tb < h; tb += nwarps) {
      uint32_t sum = 0;
      for (int u = lane; u < kL2Size; u += 32) sum += spl2[tb * kL2Size + u] & 0x7FFFFFFu;
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) tbl_nb[tb] = sum;
    }
    __syncthreads();
    uint32_t total = 0;
    for (int64_t base = 0; base < L1size; base += NT) {
      const int64_t cell = base + tid;
      uint32_t nbc = 0;
      if (cell < L1size) {
        const uint32_t e = lut[cell];
        const uint64_t clo = (uint64_t)cell << mm.s1;
        if (e & kPtrFlag) {
          nbc = tbl_nb[e & ~kPtrFlag];
        } else {
          const int g = gmax_of(cell, tg);
          if (g > 0) nbc = ((cell & ((int64_t{1} << g) - 1)) == 0 && clo < mm.K) ? 1u : 0u;
          else nbc = leaf_split(clo, mm.s1, estimate(cnt[cell], mm), tg, mm.K).count;
        }
      }
      block_scan_excl<uint32_t>(nbc, &s_tot, buf);
      total += s_tot;
    }
    nb_total = total;
    if ((int64_t)nb_total <= mm.nbcap || attempt >= 40) break;
    tg *= 2;
  }
  if ((int64_t)nb_total > mm.nbcap) {
    if (tid == 0) record_fatal(c, SPM_ERR_UNSUPPORTED);
    return;
  }
  // ---- write the entries: level-1 cells (and the bases of the tables)
  uint32_t carry = 0;
  for (int64_t base = 0; base < L1size; base += NT) {
    const int64_t cell = base + tid;
    uint32_t nbc = 0, ent = 0;
    if (cell < L1size) {
      const uint32_t e = lut[cell];
      const uint64_t clo = (uint64_t)cell << mm.s1;
      if (e & kPtrFlag) {
        nbc = tbl_nb[e & ~kPtrFlag];
        ent = e;
      } else {
        const int g = gmax_of(cell, tg);
        if (g > 0) {
          const bool first = (cell & ((int64_t{1} << g) - 1)) == 0;
          const int64_t glo_cell = (cell >> g) << g;
          nbc = (first && clo < mm.K) ? 1u : 0u;
          ent = kMergeFlag | ((uint32_t)g << kXShift);
          // members point at their group's bucket
          ent |= first ? 0u : ((((uint64_t)glo_cell << mm.s1) < mm.K) ? 0x80000000u : 0u);  // marker, fixed below
        } else {
          const Split sp = leaf_split(clo, mm.s1, estimate(cnt[cell], mm), tg, mm.K);
          nbc = sp.count;
          ent = (uint32_t)sp.j << kXShift;
        }
      }
    }
    const uint32_t off = block_scan_excl<uint32_t>(nbc, &s_tot, buf) + carry;
    if (cell < L1size) {
      if (ent & kPtrFlag) {
        if (ent & kMergeFlag) {
          // merged member whose group exists: the group's bucket precedes this cell
          lut[cell] = (ent & ~kPtrFlag) | ((off - 1) & kBaseMask);
        } else {
          tbl_base[ent & ~kPtrFlag] = off;
        }
      } else {
        lut[cell] = ent | (off & kBaseMask);
      }
    }
    carry += s_tot;
  }
  __syncthreads();
  // ---- level-2 entries: base of the table plus the prefix inside it
  for (uint32_t tb = warp; tb < h; tb += nwarps) {
    uint32_t run = tbl_base[tb];
    for (int u0 = 0; u0 < kL2Size; u0 += 32) {
      const uint32_t sp = spl2[tb * kL2Size + u0 + lane];
      const uint32_t cntq = sp & 0x7FFFFFFu;
      uint32_t x = cntq;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const uint32_t excl = run + x - cntq;
      lut[L1size + tb * kL2Size + u0 + lane] = ((sp >> 27) << kXShift) | (excl & kBaseMask);
      run += __shfl_sync(0xffffffffu, x, 31);
    }
  }
  if (tid == 0) {
    c.meta[i].nb = nb_total;
    c.meta[i].h2used = (int32_t)h;
  }
}

// Bucket offsets of the matrices and the ranges of the partition blocks.
__global__ void k_bucket_scan(Ctx c) {
  __shared__ unsigned long long buf[32];
  __shared__ unsigned long long tot;
  if (is_aborted(c)) return;
  unsigned long long carry = 0, lcarry = 0;
  for (int64_t base = 0; base < c.B; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const unsigned long long nb = i < c.B ? (unsigned long long)c.meta[i].nb : 0ull;
    const unsigned long long off = block_scan_excl<unsigned long long>(nb, &tot, buf) + carry;
    if (i < c.B) c.meta[i].bucket_off = (int64_t)off;
    carry += tot;
    const unsigned long long used =
        i < c.B ? (unsigned long long)((int64_t{1} << c.meta[i].L1) + (int64_t)c.meta[i].h2used * kL2Size) : 0ull;
    const unsigned long long loff = block_scan_excl<unsigned long long>(used, &tot, buf) + lcarry;
    if (i < c.B) c.meta[i].lut_used_off = (int64_t)loff;
    lcarry += tot;
  }
  if (threadIdx.x == 0) {
    if (carry > (unsigned long long)c.nbcap_total) record_fatal(c, SPM_ERR_UNSUPPORTED);
    c.scal->NB = (uint32_t)carry;
    const unsigned long long grp = (unsigned long long)max(c.groups, 1);
    c.scal->G = (uint32_t)max(1ull, (carry + grp - 1) / grp);
  }
  __syncthreads();
  const MatMeta* meta = c.meta;
  unsigned long long hcarry = 0;
  for (int64_t base = 0; base < c.C; base += blockDim.x) {
    const int64_t cc = base + threadIdx.x;
    CtaInfo ci;
    memset(&ci, 0, sizeof(ci));
    unsigned long long range = 0;
    if (cc < c.C) {
      ci.e0 = chunk_begin(c.m_total, cc, c.C);
      ci.e1 = chunk_begin(c.m_total, cc + 1, c.C);
      ci.i0 = 0;
      ci.i1 = -1;
      if (ci.e0 < ci.e1) {
        const int64_t i0 = upper_index(0, c.B - 1, ci.e0, [&](int64_t j) { return meta[j].t0; });
        const int64_t i1 = upper_index(0, c.B - 1, ci.e1 - 1, [&](int64_t j) { return meta[j].t0; });
        ci.i0 = (int32_t)i0;
        ci.i1 = (int32_t)i1;
        ci.cb0 = (uint32_t)meta[i0].bucket_off;
        ci.cb1 = (uint32_t)(meta[i1].bucket_off + meta[i1].nb);
        ci.l0 = meta[i0].lut_used_off;
        ci.l1 = meta[i1].lut_used_off + (int64_t{1} << meta[i1].L1) + (int64_t)meta[i1].h2used * kL2Size;
        range = ci.cb1 - ci.cb0;
      }
    }
    const unsigned long long off = block_scan_excl<unsigned long long>(range, &tot, buf) + hcarry;
    if (cc < c.C) {
      ci.hoff = (int64_t)off;
      c.cta[cc] = ci;
    }
    hcarry += tot;
  }
  if (threadIdx.x == 0 && hcarry > (unsigned long long)c.hist_bound) record_fatal(c, SPM_ERR_UNSUPPORTED);
}

// Bucket descriptors (first key and width) from the LUT entries: one warp per
// entry.
__global__ void k_bucket_fill(Ctx c) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= c.lut_total || is_aborted(c)) return;
  const MatMeta* meta = c.meta;
  const int64_t i = upper_index(0, c.B - 1, gw, [&](int64_t j) { return meta[j].lut_off; });
  const MatMeta& mm = meta[i];
  const int64_t e = gw - mm.lut_off;
  if (e >= mm.lut_len) return;
  if (mm.K == 0) {
    if (e == 0 && lane == 0) {
      c.bk_lo[mm.bucket_off] = 0;
      c.bk_info[mm.bucket_off] = ((uint32_t)i << 6) | 0u;
    }
    return;
  }
  const int64_t L1size = int64_t{1} << mm.L1;
  uint64_t lo;
  int shift;
  const uint32_t ent = c.lut[gw];
  if (e < L1size) {
    if (ent & kPtrFlag) return;
    lo = (uint64_t)e << mm.s1;
    shift = mm.s1;
  } else {
    const int64_t tb = (e - L1size) >> kL2Bits;
    const int64_t u = (e - L1size) & (kL2Size - 1);
    if (tb >= mm.h2used) return;
    const int64_t cell = c.l2cell[mm.l2_off + tb];
    shift = mm.s1 - kL2Bits;
    lo = ((uint64_t)cell << mm.s1) + ((uint64_t)u << shift);
  }
  if (lo >= mm.K) return;
  const int x = (ent >> kXShift) & 31;
  const uint32_t base = ent & kBaseMask;
  if (ent & kMergeFlag) {
    if ((e & ((int64_t{1} << x) - 1)) != 0) return;  // not the first cell of its group
    if (lane == 0) {
      const int64_t b = mm.bucket_off + base;
      c.bk_lo[b] = lo;
      c.bk_info[b] = ((uint32_t)i << 6) | (uint32_t)(shift + x);
    }
    return;
  }
  const int w = shift - x;
  const uint64_t n = ((mm.K - lo) + ((uint64_t{1} << w) - 1)) >> w;
  const uint64_t full = uint64_t{1} << x;
  const uint64_t count = n < full ? n : full;
  for (uint64_t q = lane; q < count; q += 32) {
    const int64_t b = mm.bucket_off + base + (int64_t)q;
    c.bk_lo[b] = lo + (q << w);
    c.bk_info[b] = ((uint32_t)i << 6) | (uint32_t)w;
  }
}

// ===========================================================================
// Partition: histogram and scatter
// ===========================================================================
// Current matrix of a thread while it walks its writes in increasing order.
struct MatView {
  int64_t idx, t_end;
  uint64_t n_rows, n_cols;
  int s1;
  int64_t L1size;
  const uint32_t* lut;      // this matrix's LUT (shared or global memory)
  int64_t bucket_rel;       // bucket_off - cb0
};

__device__ __forceinline__ void load_view(const Ctx& c, const CtaInfo& ci, const uint32_t* lut_base, bool lut_smem,
                                          int64_t i, MatView& v) {
  const MatMeta& mm = c.meta[i];
  v.idx = i;
  v.t_end = mm.t0 + mm.m;
  v.n_rows = (uint64_t)mm.n_rows;
  v.n_cols = (uint64_t)mm.n_cols;
  v.s1 = mm.s1;
  v.L1size = int64_t{1} << mm.L1;
  v.lut = lut_smem ? (lut_base + (mm.lut_used_off - ci.l0)) : (c.lut + mm.lut_off);
  v.bucket_rel = mm.bucket_off - (int64_t)ci.cb0;
}

// Classify one write: bucket (relative to the block's range) and key within
// the bucket.  Returns false for an index outside the matrix.
__device__ __forceinline__ bool classify(const MatView& v, int32_t r, int32_t col, uint32_t& brel, uint32_t& lkey) {
  // (n_rows, n_cols < 2^31: one unsigned 32-bit compare per index)
  if ((uint32_t)r >= (uint32_t)v.n_rows || (uint32_t)col >= (uint32_t)v.n_cols) return false;
  const uint64_t key = (uint64_t)col * v.n_rows + (uint64_t)r;
  uint32_t e = v.lut[key >> v.s1];
  int sh = v.s1;
  if (e & kPtrFlag) {
    sh = v.s1 - kL2Bits;
    e = v.lut[v.L1size + (int64_t)(e & ~kPtrFlag) * kL2Size + ((key >> sh) & (kL2Size - 1))];
  }
  const int x = (e >> kXShift) & 31;
  int w;
  uint32_t sub;
  if (e & kMergeFlag) {
    w = sh + x;
    sub = 0;
  } else {
    w = sh - x;
    sub = (uint32_t)((key >> w) & ((uint64_t{1} << x) - 1));
  }
  brel = (uint32_t)(v.bucket_rel + (int64_t)(e & kBaseMask) + sub);
  lkey = (uint32_t)(key & ((uint64_t{1} << w) - 1));
  return true;
}

template <bool BATCHED>
__device__ __forceinline__ void advance_view(const Ctx& c, const CtaInfo& ci, const uint32_t* lut_base, bool lut_smem,
                                             int64_t t, MatView& v) {
  if (BATCHED && t >= v.t_end) {
    const MatMeta* meta = c.meta;
    const int64_t i = upper_index(v.idx + 1, ci.i1, t, [&](int64_t j) { return meta[j].t0; });
    load_view(c, ci, lut_base, lut_smem, i, v);
  }
}

// Shared-memory layout of the partition kernels: [counters | LUT slice];
// `counters` words (at most kHistCapSmem) precede the LUT slice.
__device__ __forceinline__ void partition_prologue(const Ctx& c, const CtaInfo& ci, uint32_t* sm, int64_t counters,
                                                   bool& lut_smem, uint32_t*& lut_base) {
  const int64_t lutn = ci.l1 - ci.l0;
  lut_smem = lutn <= kLutCapSmem;
  const int64_t hwords = (counters + 3) & ~3ll;
  lut_base = sm + hwords;
  if (lut_smem) {
    // per matrix: its level-1 table and the level-2 tables it uses, packed
    for (int64_t i = ci.i0; i <= ci.i1; ++i) {
      const MatMeta& mm = c.meta[i];
      const int64_t len = (int64_t{1} << mm.L1) + (int64_t)mm.h2used * kL2Size;
      uint32_t* dst = lut_base + (mm.lut_used_off - ci.l0);
      const uint32_t* src = c.lut + mm.lut_off;
      for (int64_t k = threadIdx.x; k < len; k += blockDim.x) dst[k] = src[k];
    }
  }
}

template <bool BATCHED, bool VEC>
__global__ void __launch_bounds__(1024) k_hist(Ctx c) {
  extern __shared__ __align__(16) uint32_t sm[];
  const CtaInfo ci = c.cta[blockIdx.x];
  if (is_aborted(c) || ci.e0 >= ci.e1) return;
  bool lut_smem;
  uint32_t* lut_base;
  const int64_t range = (int64_t)ci.cb1 - (int64_t)ci.cb0;
  const bool hist_smem = range <= kHistCapSmem;
  partition_prologue(c, ci, sm, hist_smem ? range : 0, lut_smem, lut_base);
  uint32_t* hist = hist_smem ? sm : (c.hist + ci.hoff);
  for (int64_t k = threadIdx.x; k < range; k += blockDim.x) hist[k] = 0u;
  __syncthreads();
  MatView v;
  load_view(c, ci, lut_base, lut_smem, ci.i0, v);
  bool bad = false;
  auto body = [&](int64_t t, int32_t r, int32_t col) {
    advance_view<BATCHED>(c, ci, lut_base, lut_smem, t, v);
    uint32_t b, lk;
    if (classify(v, r, col, b, lk)) atomicAdd(&hist[b], 1u); else bad = true;
  };
  if (VEC) {
    const int64_t nvec = (ci.e1 - ci.e0) >> 2;
    const int4* r4p = reinterpret_cast<const int4*>(c.rows + ci.e0);
    const int4* c4p = reinterpret_cast<const int4*>(c.cols + ci.e0);
    const int64_t NT = blockDim.x;
    int64_t q = threadIdx.x;
    for (; q + 3 * NT < nvec; q += 4 * NT) {  // four independent 16-byte loads per array in flight
      int4 ra[4], ca[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ra[u] = __ldcs(r4p + q + u * NT);
        ca[u] = __ldcs(c4p + q + u * NT);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t t = ci.e0 + 4 * (q + u * NT);
        body(t, ra[u].x, ca[u].x);
        body(t + 1, ra[u].y, ca[u].y);
        body(t + 2, ra[u].z, ca[u].z);
        body(t + 3, ra[u].w, ca[u].w);
      }
    }
    for (; q < nvec; q += NT) {
      const int4 r4 = __ldcs(r4p + q), c4 = __ldcs(c4p + q);
      const int64_t t = ci.e0 + 4 * q;
      body(t, r4.x, c4.x);
      body(t + 1, r4.y, c4.y);
      body(t + 2, r4.z, c4.z);
      body(t + 3, r4.w, c4.w);
    }
    for (int64_t t = ci.e0 + 4 * nvec + threadIdx.x; t < ci.e1; t += blockDim.x) body(t, c.rows[t], c.cols[t]);
  } else {
    for (int64_t t = ci.e0 + threadIdx.x; t < ci.e1; t += blockDim.x) body(t, c.rows[t], c.cols[t]);
  }
  if (bad) record_error(c, SPM_ERR_INDEX_OUT_OF_RANGE);
  __syncthreads();
  if (hist_smem)
    for (int64_t k = threadIdx.x; k < range; k += blockDim.x) c.hist[ci.hoff + k] = hist[k];
}

// Per bucket: exclusive prefix over the partition blocks (in place) and total.
constexpr int kMaxCtas = 1024;
__global__ void __launch_bounds__(256) k_colscan(Ctx c) {
  __shared__ uint32_t s_cb0[kMaxCtas], s_cb1[kMaxCtas];
  __shared__ int64_t s_hoff[kMaxCtas];
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (is_aborted(c)) return;
  const int C = (int)c.C;
  for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
    const CtaInfo& ci = c.cta[cc];
    const bool nonempty = ci.e0 < ci.e1;
    s_cb0[cc] = nonempty ? ci.cb0 : 1u;
    s_cb1[cc] = nonempty ? ci.cb1 : 0u;
    s_hoff[cc] = ci.hoff;
  }
  __syncthreads();
  if (b >= c.nbcap_total) return;
  const int64_t NB = c.scal->NB;
  if (b >= NB) {
    c.bk_count[b] = 0u;
    return;
  }
  uint32_t running = 0, fronts = 0;
  for (int c0 = 0; c0 < C; c0 += 8) {  // eight independent loads in flight
    uint32_t v[8];
    uint32_t* ptr[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int cc = c0 + u;
      ptr[u] = nullptr;
      v[u] = 0u;
      if (cc < C) {
        const uint32_t cb0 = s_cb0[cc];
        if ((uint32_t)b >= cb0 && (uint32_t)b < s_cb1[cc]) {
          ptr[u] = c.hist + s_hoff[cc] + (b - cb0);
          v[u] = *ptr[u];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (ptr[u]) {
        *ptr[u] = running;
        running += v[u];
        fronts += v[u] != 0u ? 1u : 0u;
      }
    }
  }
  c.bk_count[b] = running;
  const unsigned act = __activemask();
  const uint32_t wsum = __reduce_add_sync(act, fronts);
  if ((threadIdx.x & 31) == __ffs(act) - 1 && wsum) atomicAdd(&c.scal->fronts, (unsigned long long)wsum);
}

// Device-wide exclusive scan of a per-bucket count array (bk_count into
// bk_start; bk_nnz into bk_out) in three kernels.
__global__ void k_scan_reduce(Ctx c, const uint32_t* __restrict__ in) {
  __shared__ uint32_t buf[32];
  __shared__ uint32_t tot;
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const uint32_t v = i < c.nbcap_total && i < (int64_t)c.scal->NB ? in[i] : 0u;
  block_scan_excl<uint32_t>(v, &tot, buf);
  if (threadIdx.x == 0) c.scanpart[blockIdx.x] = tot;
}

__global__ void k_scan_top(Ctx c, int64_t nblk) {
  __shared__ uint32_t buf[32];
  __shared__ uint32_t tot;
  uint32_t carry = 0;
  for (int64_t base = 0; base < nblk; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const uint32_t v = i < nblk ? c.scanpart[i] : 0u;
    const uint32_t off = block_scan_excl<uint32_t>(v, &tot, buf) + carry;
    if (i < nblk) c.scanpart[i] = off;
    carry += tot;
  }
}

// The whole scan in one block when the buckets fit one (small calls: two
// launches fewer than reduce + top + down).
__global__ void k_scan_one(Ctx c, const uint32_t* __restrict__ in, uint32_t* __restrict__ out) {
  __shared__ uint32_t buf[32];
  __shared__ uint32_t tot;
  const int64_t i = threadIdx.x;
  const uint32_t v = i < c.nbcap_total && i < (int64_t)c.scal->NB ? in[i] : 0u;
  const uint32_t off = block_scan_excl<uint32_t>(v, &tot, buf);
  if (i < c.nbcap_total) out[i] = off;
}

__global__ void k_scan_down(Ctx c, const uint32_t* __restrict__ in, uint32_t* __restrict__ out) {
  __shared__ uint32_t buf[32];
  __shared__ uint32_t tot;
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const uint32_t v = i < c.nbcap_total && i < (int64_t)c.scal->NB ? in[i] : 0u;
  const uint32_t off = block_scan_excl<uint32_t>(v, &tot, buf) + c.scanpart[blockIdx.x];
  if (i < c.nbcap_total) out[i] = off;
}

// The two-pass partition runs when the workspace has room for it and the
// one-pass scatter would keep more write fronts open than L2 can hold.
__device__ __forceinline__ bool two_pass_on(const Ctx& c) {
  return c.two_pass != 0 && (int64_t)c.scal->fronts > c.min_fronts;
}

template <bool BATCHED, bool VEC, bool F64>
__global__ void __launch_bounds__(1024) k_scatter(Ctx c) {
  extern __shared__ __align__(16) uint32_t sm[];
  const CtaInfo ci = c.cta[blockIdx.x];
  if (is_aborted(c) || ci.e0 >= ci.e1 || two_pass_on(c)) return;
  bool lut_smem;
  uint32_t* lut_base;
  const int64_t range = (int64_t)ci.cb1 - (int64_t)ci.cb0;
  const bool hist_smem = range <= kHistCapSmem;
  partition_prologue(c, ci, sm, hist_smem ? range : 0, lut_smem, lut_base);
  uint32_t* cur = hist_smem ? sm : (c.hist + ci.hoff);
  for (int64_t k = threadIdx.x; k < range; k += blockDim.x)
    cur[k] = c.bk_start[ci.cb0 + k] + c.hist[ci.hoff + k];
  __syncthreads();
  MatView v;
  load_view(c, ci, lut_base, lut_smem, ci.i0, v);
  using VT = typename std::conditional<F64, uint64_t, uint32_t>::type;
  const VT* vin = reinterpret_cast<const VT*>(c.vals);
  uint64_t keep_policy;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep_policy));
  auto body = [&](int64_t t, int32_t r, int32_t col, VT val) {
    advance_view<BATCHED>(c, ci, lut_base, lut_smem, t, v);
    uint32_t b, lk;
    if (classify(v, r, col, b, lk)) {
      const uint64_t vb = (uint64_t)val;
      const uint32_t slot = atomicAdd(&cur[b], 1u);
      // records are written a few at a time per bucket: ask L2 to keep the
      // partially written lines rather than the streamed inputs
      asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(c.rec + slot), "r"(lk),
                   "r"((uint32_t)t), "r"((uint32_t)vb), "r"((uint32_t)(vb >> 32)), "l"(keep_policy)
                   : "memory");
    }
  };
  if (VEC) {
    const int64_t nvec = (ci.e1 - ci.e0) >> 2;
    const int4* r4p = reinterpret_cast<const int4*>(c.rows + ci.e0);
    const int4* c4p = reinterpret_cast<const int4*>(c.cols + ci.e0);
    auto load_vals = [&](int64_t t, VT& x0, VT& x1, VT& x2, VT& x3) {
      if (F64) {
        const ulonglong2* vp = reinterpret_cast<const ulonglong2*>(vin + t);
        const ulonglong2 a = __ldcs(vp), bq = __ldcs(vp + 1);
        x0 = (VT)a.x; x1 = (VT)a.y; x2 = (VT)bq.x; x3 = (VT)bq.y;
      } else {
        const uint4 a = __ldcs(reinterpret_cast<const uint4*>(vin + t));
        x0 = (VT)a.x; x1 = (VT)a.y; x2 = (VT)a.z; x3 = (VT)a.w;
      }
    };
    const int64_t NT = blockDim.x;
    int64_t q = threadIdx.x;
    for (; q + NT < nvec; q += 2 * NT) {  // two groups of loads in flight per thread
      const int4 ra = __ldcs(r4p + q), ca = __ldcs(c4p + q);
      const int4 rb = __ldcs(r4p + q + NT), cb = __ldcs(c4p + q + NT);
      const int64_t ta = ci.e0 + 4 * q, tb = ci.e0 + 4 * (q + NT);
      VT a0, a1, a2, a3, b0, b1, b2, b3;
      load_vals(ta, a0, a1, a2, a3);
      load_vals(tb, b0, b1, b2, b3);
      body(ta, ra.x, ca.x, a0);
      body(ta + 1, ra.y, ca.y, a1);
      body(ta + 2, ra.z, ca.z, a2);
      body(ta + 3, ra.w, ca.w, a3);
      body(tb, rb.x, cb.x, b0);
      body(tb + 1, rb.y, cb.y, b1);
      body(tb + 2, rb.z, cb.z, b2);
      body(tb + 3, rb.w, cb.w, b3);
    }
    for (; q < nvec; q += NT) {
      const int4 r4 = __ldcs(r4p + q), c4 = __ldcs(c4p + q);
      const int64_t t = ci.e0 + 4 * q;
      VT x0, x1, x2, x3;
      load_vals(t, x0, x1, x2, x3);
      body(t, r4.x, c4.x, x0);
      body(t + 1, r4.y, c4.y, x1);
      body(t + 2, r4.z, c4.z, x2);
      body(t + 3, r4.w, c4.w, x3);
    }
    for (int64_t t = ci.e0 + 4 * nvec + threadIdx.x; t < ci.e1; t += blockDim.x)
      body(t, c.rows[t], c.cols[t], vin[t]);
  } else {
    for (int64_t t = ci.e0 + threadIdx.x; t < ci.e1; t += blockDim.x) body(t, c.rows[t], c.cols[t], vin[t]);
  }
}

// ---------------------------------------------------------------------------
// Two-pass partition.  Buckets are taken in groups of G consecutive buckets
// (group g = buckets [g*G, (g+1)*G), about one group per SM); a group spans
// the same slots of the temporary record array as of the final one.  Pass A
// moves every write to its group, pass B moves the records of one group to
// their buckets.  Both passes first sort each tile of kTileItems x blockDim
// writes by destination in shared memory and then write the tile out in that
// order, so that consecutive threads store to consecutive addresses and the
// records leave as whole cache lines rather than one 16-byte piece per write.
// The loads of the next tile are issued before the current one is sorted.
// ---------------------------------------------------------------------------
constexpr int kTileItems = 4;      // writes per thread per tile
constexpr int kMaxGroupsA = 2048;  // groups one pass-A block may write to
constexpr int kGroupMax = 1024;    // buckets per group, at most

// Shared memory of a tile: T records and their digits (and, in pass A, the
// bucket within the group), then per digit two count buffers (tiles
// alternate between them), the tile's first slot, the tile's first global
// slot and the running global cursor.
__host__ __device__ inline size_t tile_smem_words(int threads, int ndig, bool with_sub) {
  const size_t T = (size_t)kTileItems * threads;
  return 4 * T + T / 2 + (with_sub ? T : 0) + 5 * (size_t)ndig + 4;
}

__host__ __device__ inline size_t part_a_smem_bytes(int threads) {
  return 4 * (tile_smem_words(threads, kMaxGroupsA, true) + (size_t)kLutCapSmem);
}

__host__ __device__ inline size_t part_b_smem_bytes(int threads) { return 4 * tile_smem_words(threads, 2048, false); }

struct TileSmem {
  uint4* stage;
  uint16_t* dig;
  uint32_t* sub;    // pass A: the bucket of each staged record
  uint32_t* cnt0;   // count buffer 0; buffer 1 follows it at cnt0 + ndig
  uint32_t ndig;
  uint32_t* start;  // [ndig + 1]
  uint32_t* gbase;  // first global slot of each digit for the tile being written
  uint32_t* cur;    // next global slot of each digit
  uint32_t* end;    // first word after the tile area
};

__device__ __forceinline__ TileSmem tile_smem(uint32_t* sm, int ndig, bool with_sub) {
  const uint32_t T = kTileItems * blockDim.x;
  TileSmem S;
  S.stage = reinterpret_cast<uint4*>(sm);
  S.dig = reinterpret_cast<uint16_t*>(S.stage + T);
  S.sub = reinterpret_cast<uint32_t*>(S.dig + T);
  uint32_t* w = S.sub + (with_sub ? T : 0);
  S.cnt0 = w;
  S.ndig = (uint32_t)ndig;
  S.start = w + 2 * ndig;
  S.gbase = w + 3 * ndig + 1;
  S.cur = w + 4 * ndig + 1;
  S.end = w + 5 * ndig + 4;
  return S;
}

// One warp: start[] = exclusive prefix sums of this tile's counts,
// gbase[] = cur[], cur[] += counts, and the other count buffer is cleared
// for the next tile.
__device__ __forceinline__ void tile_scan_warp(TileSmem& S, int buf, uint32_t nd) {
  const int lane = threadIdx.x & 31;
  const uint32_t per = (nd + 31) / 32;
  const uint32_t a = min(nd, lane * per), e = min(nd, a + per);
  const uint32_t* cnt = S.cnt0 + (buf ? S.ndig : 0u);
  uint32_t* other = S.cnt0 + (buf ? 0u : S.ndig);
  uint32_t local = 0;
  for (uint32_t q = a; q < e; ++q) local += cnt[q];
  uint32_t inc = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  uint32_t run = inc - local;
  for (uint32_t q = a; q < e; ++q) {
    const uint32_t x = cnt[q];
    S.start[q] = run;
    run += x;
    S.gbase[q] = S.cur[q];
    S.cur[q] += x;
    other[q] = 0u;
  }
  if (lane == 31) S.start[nd] = inc;
}

constexpr uint32_t kNoItem = 0xffffffffu;

// Per tile: count (shared-memory atomics give each item its rank within its
// digit), barrier, one warp scans, barrier, items go to their sorted slots,
// barrier, the sorted tile is written out; the next tile's first barrier
// also ends this write-out.
template <bool BATCHED, bool VEC, bool F64>
__global__ void __launch_bounds__(1024) k_part_a(Ctx c) {
  extern __shared__ __align__(16) uint32_t sm[];
  using VT = typename std::conditional<F64, uint64_t, uint32_t>::type;
  const CtaInfo ci = c.cta[blockIdx.x];
  if (is_aborted(c) || ci.e0 >= ci.e1 || !two_pass_on(c)) return;
  const int tid = threadIdx.x, NT = blockDim.x;
  const uint32_t T = kTileItems * NT;
  const int64_t range = (int64_t)ci.cb1 - (int64_t)ci.cb0;
  const uint32_t G = c.scal->G;
  const Div32 dG = div32_make(G);
  const uint32_t g0 = div32(ci.cb0, dG);
  const uint32_t ngrp = div32(ci.cb1 - 1, dG) - g0 + 1;
  if (ngrp > (uint32_t)kMaxGroupsA) {  // the host keeps the group count below this
    if (tid == 0) record_fatal(c, SPM_ERR_UNSUPPORTED);
    return;
  }
  TileSmem S = tile_smem(sm, kMaxGroupsA, true);
  bool lut_smem;
  uint32_t* lut_base;
  partition_prologue(c, ci, S.end, 0, lut_smem, lut_base);
  // this block's first slot in each group: the writes of the group's buckets
  // that come before its own (earlier matrices, earlier blocks)
  uint32_t* const cnt0 = S.cnt0;
  uint32_t* const cnt1 = S.cnt0 + S.ndig;
  for (uint32_t q = tid; q < ngrp; q += NT) cnt0[q] = cnt1[q] = 0u;
  __syncthreads();
  for (int64_t k = tid; k < range; k += NT)
    atomicAdd(&cnt0[div32(ci.cb0 + (uint32_t)k, dG) - g0], c.hist[ci.hoff + k]);
  __syncthreads();
  for (uint32_t q = tid; q < ngrp; q += NT) {
    S.cur[q] = cnt0[q] + c.bk_start[max((g0 + q) * G, ci.cb0)];
    cnt0[q] = 0u;
  }
  __syncthreads();
  MatView v;
  load_view(c, ci, lut_base, lut_smem, ci.i0, v);
  const VT* vin = reinterpret_cast<const VT*>(c.vals);
  auto tpos = [&](int64_t tb, int u) -> int64_t { return VEC ? tb + 4 * tid + u : tb + tid + (int64_t)u * NT; };
  struct Raw {
    int32_t r[kTileItems], cl[kTileItems];
    VT x[kTileItems];
  };
  auto load_raw = [&](int64_t tb, Raw& R) {
    const int64_t t0 = tb + 4 * tid;
    if (VEC && t0 + 4 <= ci.e1) {
      const int4 a = __ldcs(reinterpret_cast<const int4*>(c.rows + t0));
      const int4 b = __ldcs(reinterpret_cast<const int4*>(c.cols + t0));
      R.r[0] = a.x, R.r[1] = a.y, R.r[2] = a.z, R.r[3] = a.w;
      R.cl[0] = b.x, R.cl[1] = b.y, R.cl[2] = b.z, R.cl[3] = b.w;
      if (F64) {
        const ulonglong2* vp = reinterpret_cast<const ulonglong2*>(vin + t0);
        const ulonglong2 p = __ldcs(vp), q = __ldcs(vp + 1);
        R.x[0] = (VT)p.x, R.x[1] = (VT)p.y, R.x[2] = (VT)q.x, R.x[3] = (VT)q.y;
      } else {
        const uint4 p = __ldcs(reinterpret_cast<const uint4*>(vin + t0));
        R.x[0] = (VT)p.x, R.x[1] = (VT)p.y, R.x[2] = (VT)p.z, R.x[3] = (VT)p.w;
      }
    } else {
#pragma unroll
      for (int u = 0; u < kTileItems; ++u) {
        const int64_t t = tpos(tb, u);
        if (t < ci.e1) {
          R.r[u] = __ldcs(c.rows + t);
          R.cl[u] = __ldcs(c.cols + t);
          R.x[u] = __ldcs(vin + t);
        }
      }
    }
  };
  bool bad = false;
  Raw R;
  load_raw(ci.e0, R);
  uint4* tmp = reinterpret_cast<uint4*>(c.tmp);
  int buf = 0;
  for (int64_t tb = ci.e0; tb < ci.e1; tb += T, buf ^= 1) {
    uint32_t lk[kTileItems], sb[kTileItems], dr[kTileItems];
    uint64_t vv[kTileItems];
#pragma unroll
    for (int u = 0; u < kTileItems; ++u) {
      const int64_t t = tpos(tb, u);
      dr[u] = kNoItem;
      if (t < ci.e1) {
        advance_view<BATCHED>(c, ci, lut_base, lut_smem, t, v);
        uint32_t b;
        if (classify(v, R.r[u], R.cl[u], b, lk[u])) {
          const uint32_t bg = ci.cb0 + b;
          const uint32_t grp = div32(bg, dG);
          const uint32_t d = grp - g0;
          dr[u] = (d << 16) | atomicAdd(&(buf ? cnt1 : cnt0)[d], 1u);
          sb[u] = bg;
          vv[u] = (uint64_t)R.x[u];
        } else {
          bad = true;
        }
      }
    }
    if (tb + T < ci.e1) load_raw(tb + T, R);  // next tile's loads overlap this tile's sort and stores
    __syncthreads();
    if (tid < 32) tile_scan_warp(S, buf, ngrp);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kTileItems; ++u) {
      if (dr[u] != kNoItem) {
        const uint32_t d = dr[u] >> 16;
        const uint32_t p = S.start[d] + (dr[u] & 0xffffu);
        S.stage[p] = make_uint4(lk[u], (uint32_t)tpos(tb, u), (uint32_t)vv[u], (uint32_t)(vv[u] >> 32));
        S.dig[p] = (uint16_t)d;
        S.sub[p] = sb[u];
      }
    }
    __syncthreads();
    const uint32_t nt = S.start[ngrp];
    for (uint32_t i = tid; i < nt; i += NT) {
      const uint32_t d = S.dig[i];
      const uint32_t g = S.gbase[d] + (i - S.start[d]);
      tmp[g] = S.stage[i];
      c.rbk[g] = S.sub[i];
    }
  }
  if (bad) record_error(c, SPM_ERR_INDEX_OUT_OF_RANGE);
}

// Pass B: equal tiles of tmp, spread evenly over the blocks (bucket groups
// differ a lot in size, so a block per group would wait on the largest).
// A tile's records lie in at most a few consecutive groups, so their buckets
// form a short range: the tile is sorted by bucket in shared memory, each
// bucket present reserves its slots in rec with one atomic, and the sorted
// tile is written out.
constexpr int kTileDig = 2048;  // bucket range a tile may span for the shared-memory sort

__global__ void __launch_bounds__(1024) k_part_b(Ctx c) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ uint32_t s_min[32], s_max[32], s_bmin, s_bmax;
  if (is_aborted(c) || !two_pass_on(c)) return;
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, wid = tid >> 5, NWb = NT >> 5;
  const uint32_t T = kTileItems * NT;
  const uint32_t NB = c.scal->NB;
  if (NB == 0) return;
  const uint32_t mtot = c.bk_start[NB - 1] + c.bk_count[NB - 1];
  const uint32_t ntiles = (mtot + T - 1) / T;
  TileSmem S = tile_smem(sm, kTileDig, false);
  uint32_t* const cnt = S.cnt0;
  for (uint32_t q = tid; q < (uint32_t)kTileDig; q += NT) cnt[q] = 0u;
  const uint4* src = reinterpret_cast<const uint4*>(c.tmp);
  uint4* dst = reinterpret_cast<uint4*>(c.rec);
  bool bad = false;
  uint4 r[kTileItems];
  uint32_t bk[kTileItems];
  auto load = [&](uint32_t tile) {
#pragma unroll
    for (int u = 0; u < kTileItems; ++u) {
      const uint32_t k = tile * T + (uint32_t)u * NT + tid;
      bk[u] = ~0u;
      if (k < mtot) {
        r[u] = __ldcs(src + k);
        bk[u] = __ldcs(c.rbk + k);
      }
    }
  };
  uint32_t tile = blockIdx.x;
  if (tile < ntiles) load(tile);
  for (; tile < ntiles; tile += gridDim.x) {
    uint4 rr[kTileItems];
    uint32_t bb[kTileItems];
    uint32_t mn = ~0u, mx = 0u;
#pragma unroll
    for (int u = 0; u < kTileItems; ++u) {
      rr[u] = r[u];
      bb[u] = bk[u];
      if (bb[u] != ~0u) {
        if (bb[u] >= NB) {
          bad = true;
          bb[u] = ~0u;
        } else {
          mn = min(mn, bb[u]);
          mx = max(mx, bb[u]);
        }
      }
    }
    if (tile + gridDim.x < ntiles) load(tile + gridDim.x);  // next tile's loads overlap this one
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) {
      s_min[wid] = mn;
      s_max[wid] = mx;
    }
    __syncthreads();  // (also: the previous tile's write-out is done)
    if (wid == 0) {
      const uint32_t a = __reduce_min_sync(0xffffffffu, lane < NWb ? s_min[lane] : ~0u);
      const uint32_t b = __reduce_max_sync(0xffffffffu, lane < NWb ? s_max[lane] : 0u);
      if (lane == 0) {
        s_bmin = a;
        s_bmax = b;
      }
    }
    __syncthreads();
    const uint32_t bmin = s_bmin;
    if (s_bmin > s_bmax) continue;  // (no records)
    const uint32_t nd = s_bmax - bmin + 1;
    if (nd > (uint32_t)kTileDig) {
      // a tile across many small groups: reserve slot by slot
#pragma unroll
      for (int u = 0; u < kTileItems; ++u)
        if (bb[u] != ~0u) dst[atomicAdd(&c.bk_cur[bb[u]], 1u)] = rr[u];
      continue;
    }
    uint32_t dr[kTileItems];
#pragma unroll
    for (int u = 0; u < kTileItems; ++u) {
      dr[u] = kNoItem;
      if (bb[u] != ~0u) {
        const uint32_t d = bb[u] - bmin;
        dr[u] = (d << 16) | atomicAdd(&cnt[d], 1u);
      }
    }
    __syncthreads();
    // every bucket present reserves its slots; one warp scans the counts
    for (uint32_t d = tid; d < nd; d += NT) {
      const uint32_t x = cnt[d];
      if (x) S.gbase[d] = atomicAdd(&c.bk_cur[bmin + d], x);
    }
    if (wid == 0) {
      const uint32_t per = (nd + 31) / 32;
      const uint32_t a = min(nd, lane * per), e = min(nd, a + per);
      uint32_t local = 0;
      for (uint32_t q = a; q < e; ++q) local += cnt[q];
      uint32_t inc = local;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      uint32_t run = inc - local;
      for (uint32_t q = a; q < e; ++q) {
        S.start[q] = run;
        run += cnt[q];
      }
      if (lane == 31) S.start[nd] = inc;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kTileItems; ++u) {
      if (dr[u] != kNoItem) {
        const uint32_t d = dr[u] >> 16;
        const uint32_t p = S.start[d] + (dr[u] & 0xffffu);
        S.stage[p] = rr[u];
        S.dig[p] = (uint16_t)d;
      }
    }
    for (uint32_t d = tid; d < nd; d += NT) cnt[d] = 0u;  // clean for the next tile
    __syncthreads();
    const uint32_t nt = S.start[nd];
    for (uint32_t i = tid; i < nt; i += NT) {
      const uint32_t d = S.dig[i];
      dst[S.gbase[d] + (i - S.start[d])] = S.stage[i];
    }
  }
  if (bad) record_fatal(c, SPM_ERR_CUDA);
}

// ===========================================================================
// Host side
// ===========================================================================
namespace {

constexpr spm_tuning kDefaultTuning = {6144, 12, 1024, 512, 1 << 22, 1 << 19, 1};
spm_tuning g_tuning = kDefaultTuning;
int64_t g_withhold = -1;
std::mutex g_mutex;

// measurement hooks
constexpr int kStages = 6;
constexpr int kRing = 64;
struct StageRing {
  bool on = false;
  int dev = -1;
  cudaEvent_t ev[kRing][kStages + 1] = {};
  int64_t calls = 0;
};
StageRing g_ring;
std::atomic<int64_t> g_launches{0};

void stage_mark(cudaStream_t st, int64_t call, int boundary) {
  if (call < 0) return;
  cudaEventRecord(g_ring.ev[call % kRing][boundary], st);
}

struct DevState {
  bool init = false;
  int sms = 0;
};
DevState g_dev[64];

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Per-mode parameters: whether the resolve kernel reads stream positions
// (last-write mode, or the map) and seq (last-write mode with seq), the
// number of writes a bucket may hold to be resolved in shared memory, and the
// planner's target.
struct ModeParams {
  bool pos, seq;
  int cap;
  int64_t tgt;
};

ModeParams mode_params(spm_mode mode, uint32_t flags, const spm_tuning& tun) {
  ModeParams p;
  const bool sum = mode == SPM_MODE_SUM;
  p.pos = !sum || (flags & SPM_KEEP_MAP) != 0;
  p.seq = !sum && (flags & SPM_SEQ_EXPLICIT) != 0;
  p.tgt = std::max<int64_t>(256, (int64_t)tun.bucket_target);
  p.cap = resolve_capacity((flags & SPM_KEEP_MAP) != 0);
  return p;
}

size_t partition_smem_bytes() { return (size_t)(kHistCapSmem + kLutCapSmem) * 4; }

// Bucket groups of the two-pass partition: one per SM, or more when needed
// to keep at most kGroupMax buckets in a group.
int64_t two_pass_groups(int sms, int64_t nbcap_total) {
  return std::max<int64_t>((int64_t)sms, (nbcap_total + kGroupMax - 1) / kGroupMax);
}

template <typename K>
void set_smem_attr(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

spm_status device_init(int& dev, DevState*& ds) {
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPM_ERR_CUDA;
  ds = &g_dev[dev];
  if (ds->init) return SPM_OK;
  std::lock_guard<std::mutex> lk(g_mutex);
  if (ds->init) return SPM_OK;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return SPM_ERR_CUDA;
  const size_t ps = partition_smem_bytes();
  set_smem_attr(k_hist<false, false>, ps);
  set_smem_attr(k_hist<false, true>, ps);
  set_smem_attr(k_hist<true, false>, ps);
  set_smem_attr(k_hist<true, true>, ps);
#define SPM_SET_SCATTER(BA, VE)                    \
  set_smem_attr(k_scatter<BA, VE, false>, ps);     \
  set_smem_attr(k_scatter<BA, VE, true>, ps);
  SPM_SET_SCATTER(false, false)
  SPM_SET_SCATTER(false, true)
  SPM_SET_SCATTER(true, false)
  SPM_SET_SCATTER(true, true)
#undef SPM_SET_SCATTER
  resolve_set_attributes();
  {
    set_smem_attr(k_plan, kPlanSmem);
    set_smem_attr(k_part_b, part_b_smem_bytes(1024));
    set_smem_attr(k_part_a<false, false, false>, part_a_smem_bytes(1024));
    set_smem_attr(k_part_a<false, false, true>, part_a_smem_bytes(1024));
    set_smem_attr(k_part_a<false, true, false>, part_a_smem_bytes(1024));
    set_smem_attr(k_part_a<false, true, true>, part_a_smem_bytes(1024));
    set_smem_attr(k_part_a<true, false, false>, part_a_smem_bytes(1024));
    set_smem_attr(k_part_a<true, false, true>, part_a_smem_bytes(1024));
    set_smem_attr(k_part_a<true, true, false>, part_a_smem_bytes(1024));
    set_smem_attr(k_part_a<true, true, true>, part_a_smem_bytes(1024));
  }
  if (cudaGetLastError() != cudaSuccess) return SPM_ERR_CUDA;
  ds->sms = sms;
  ds->init = true;
  return SPM_OK;
}

int num_sms_for_sizing() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (g_dev[dev].init) return g_dev[dev].sms;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return 152;
  }
  return sms;
}

struct HostPlan {
  Layout L;
  MatMeta single;  // B == 1
};

// Validate the sizes and compute the workspace layout.
spm_status host_plan(int64_t B, const int64_t* h_nr, const int64_t* h_nc, const int64_t* h_tp, int sv, bool seq,
                     int64_t tgt, int C, int64_t two_pass_min, HostPlan& hp) {
  if (B < 0 || (B > 0 && (!h_nr || !h_nc || !h_tp))) return SPM_ERR_INVALID_ARG;
  if (B >= (int64_t{1} << 26)) return SPM_ERR_UNSUPPORTED;
  if (B > 0 && h_tp[0] != 0) return SPM_ERR_INVALID_ARG;
  Layout& L = hp.L;
  L.B = B;
  L.sv = sv;
  L.seq = seq;
  L.C = C;
  const int64_t m_total = B > 0 ? h_tp[B] : 0;
  if (m_total < 0 || m_total >= (int64_t{1} << 32) - 64) return m_total < 0 ? SPM_ERR_INVALID_ARG : SPM_ERR_UNSUPPORTED;
  L.m_total = m_total;
  std::vector<int64_t> nbcap_prefix((size_t)B + 1, 0);
  int64_t S = 0, lut = 0, l2 = 0, nbcap = 0, cols = 0;
  for (int64_t i = 0; i < B; ++i) {
    const int64_t nr = h_nr[i], nc = h_nc[i], m = h_tp[i + 1] - h_tp[i];
    if (nr < 0 || nc < 0 || m < 0) return SPM_ERR_INVALID_ARG;
    if (nr > 0x7fffffffLL || nc > 0x7fffffffLL) return SPM_ERR_UNSUPPORTED;
    const Derived d = derive(nr, nc, m, m_total, tgt);
    if (d.bbits > kMaxKeyBits) return SPM_ERR_UNSUPPORTED;
    if (d.nbcap >= (int64_t{1} << kBaseBits)) return SPM_ERR_UNSUPPORTED;
    if (C > kMaxCtas) return SPM_ERR_UNSUPPORTED;
    if (B == 1) {
      MatMeta& mm = hp.single;
      memset(&mm, 0, sizeof(mm));
      mm.t0 = 0;
      mm.m = m;
      mm.n_rows = nr;
      mm.n_cols = nc;
      mm.K = d.K;
      mm.bbits = d.bbits;
      mm.L1 = d.L1;
      mm.s1 = d.s1;
      mm.H2 = d.H2;
      mm.ns = d.ns;
      mm.lut_len = d.lut_len;
      mm.nbcap = d.nbcap;
    }
    S += d.ns;
    lut += d.lut_len;
    l2 += d.H2;
    nbcap += d.nbcap;
    cols += nc + 1;
    nbcap_prefix[(size_t)i + 1] = nbcap;
  }
  L.S_total = S;
  L.lut_total = lut;
  L.l2_total = l2;
  L.nbcap_total = nbcap;
  // bound of the per-block bucket ranges
  int64_t hist = 0;
  auto mat_of = [&](int64_t t) {
    int64_t lo = 0, hi = B - 1;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo + 1) / 2;
      if (h_tp[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  for (int64_t cc = 0; cc < C && B > 0; ++cc) {
    const int64_t e0 = chunk_begin(m_total, cc, C), e1 = chunk_begin(m_total, cc + 1, C);
    if (e0 >= e1) continue;
    const int64_t i0 = mat_of(e0), i1 = mat_of(e1 - 1);
    hist += nbcap_prefix[(size_t)i1 + 1] - nbcap_prefix[(size_t)i0];
  }
  L.hist_bound = hist;
  L.scan_blocks = (nbcap + kScanBlock - 1) / kScanBlock;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L.meta = take(sizeof(MatMeta) * (size_t)std::max<int64_t>(B, 1));
  L.scal = take(sizeof(Scalars));
  L.cta = take(sizeof(CtaInfo) * (size_t)C);
  L.samp = take(8 * (size_t)std::max<int64_t>(S, 1));
  L.cellcnt = take(4 * (size_t)std::max<int64_t>(lut, 1));
  L.lut = take(4 * (size_t)std::max<int64_t>(lut, 1));
  L.l2cell = take(4 * (size_t)std::max<int64_t>(l2, 1));
  L.bk_lo = take(8 * (size_t)std::max<int64_t>(nbcap, 1));
  L.bk_info = take(4 * (size_t)std::max<int64_t>(nbcap, 1));
  L.bk_count = take(4 * (size_t)std::max<int64_t>(nbcap, 1));
  L.bk_start = take(4 * (size_t)std::max<int64_t>(nbcap, 1));
  L.bk_state = take(8 * (size_t)std::max<int64_t>(nbcap, 1));
  L.scanpart = take(4 * (size_t)std::max<int64_t>(L.scan_blocks, 1));
  L.hist = take(4 * (size_t)std::max<int64_t>(hist, 1));
  L.rec = take(sizeof(Rec) * (size_t)(m_total + 4));
  L.two_pass = m_total > 0 && m_total >= two_pass_min && two_pass_groups(C, nbcap) <= kMaxGroupsA;
  // tmp: the first pass's records of the two-pass partition; otherwise only
  // the tile states of the ordered single pass
  L.tmp = take(L.two_pass ? sizeof(Rec) * (size_t)(m_total + 4)
                          : 8 * (size_t)std::max<int64_t>(ordered_tiles(std::max<int64_t>(m_total, 1)), 2));
  L.rbk = L.two_pass ? take(4 * (size_t)(m_total + 4)) : o;
  L.bk_cur = take(4 * (size_t)std::max<int64_t>(nbcap, 1));
  // one matrix with level-2 tables: a sample count per level-2 cell
  L.l2h_len = (B == 1 && hp.single.H2 > 0) ? (int64_t{1} << (hp.single.L1 + kL2Bits)) : 0;
  L.l2h = L.l2h_len ? take(4 * (size_t)L.l2h_len) : o;
  L.bk_nnz = take(4 * (size_t)std::max<int64_t>(nbcap, 1));
  L.bk_out = take(4 * (size_t)std::max<int64_t>(nbcap, 1));
  L.big_list = take(4 * (size_t)std::max<int64_t>(nbcap, 1));
  L.total = o;
  return SPM_OK;
}

// Persistent grid: as many blocks as fit on the SMs at once.
template <typename K>
int resident_grid(K kernel, int sms, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return sms * per_sm;
}

// Exclusive scan of one count per bucket (in -> out).
void launch_bucket_scan(const Ctx& ctx, const Layout& L, const uint32_t* in, uint32_t* out, cudaStream_t st) {
  if (L.scan_blocks == 1) {
    k_scan_one<<<1, kScanBlock, 0, st>>>(ctx, in, out);
    return;
  }
  k_scan_reduce<<<(unsigned)L.scan_blocks, kScanBlock, 0, st>>>(ctx, in);
  k_scan_top<<<1, 1024, 0, st>>>(ctx, L.scan_blocks);
  k_scan_down<<<(unsigned)L.scan_blocks, kScanBlock, 0, st>>>(ctx, in, out);
}

template <bool BATCHED>
void launch_partition(const Ctx& ctx, const Layout& L, bool vec, cudaStream_t st, int threads, int sms,
                      int64_t call) {
  const size_t ps = partition_smem_bytes();
  const int C = (int)L.C;
  if (vec) k_hist<BATCHED, true><<<C, threads, ps, st>>>(ctx);
  else k_hist<BATCHED, false><<<C, threads, ps, st>>>(ctx);
  stage_mark(st, call, 2);
  k_colscan<<<(unsigned)((L.nbcap_total + 255) / 256), 256, 0, st>>>(ctx);
  launch_bucket_scan(ctx, L, ctx.bk_count, ctx.bk_start, st);
  stage_mark(st, call, 3);
  const bool f64 = ctx.f64 != 0;
  if (ctx.two_pass) {  // (the device picks one of the two paths; the other's blocks return at once)
    const size_t pa = part_a_smem_bytes(threads);
    if (vec) {
      if (f64) k_part_a<BATCHED, true, true><<<C, threads, pa, st>>>(ctx);
      else k_part_a<BATCHED, true, false><<<C, threads, pa, st>>>(ctx);
    } else {
      if (f64) k_part_a<BATCHED, false, true><<<C, threads, pa, st>>>(ctx);
      else k_part_a<BATCHED, false, false><<<C, threads, pa, st>>>(ctx);
    }
    cudaMemcpyAsync(ctx.bk_cur, ctx.bk_start, 4 * (size_t)std::max<int64_t>(L.nbcap_total, 1),
                    cudaMemcpyDeviceToDevice, st);
    // (pass B: two 512-thread blocks per SM interleave their tile pipelines)
    const int tb = std::min(threads, 512);
    const size_t pb = part_b_smem_bytes(tb);
    k_part_b<<<resident_grid(k_part_b, sms, tb, pb), tb, pb, st>>>(ctx);
  }
#define SPM_SCATTER(VE, F6) k_scatter<BATCHED, VE, F6><<<C, threads, ps, st>>>(ctx)
  if (vec) {
    if (f64) SPM_SCATTER(true, true); else SPM_SCATTER(true, false);
  } else {
    if (f64) SPM_SCATTER(false, true); else SPM_SCATTER(false, false);
  }
#undef SPM_SCATTER
  stage_mark(st, call, 4);
}


spm_status run_assembly(int64_t B, const int64_t* h_nr, const int64_t* h_nc, const int64_t* h_tp, const int64_t* d_nr,
                        const int64_t* d_nc, const int64_t* d_tp, const int32_t* rows, const int32_t* cols,
                        const void* vals, const uint64_t* seq, spm_dtype dtype, spm_mode mode, uint32_t flags,
                        int64_t* col_ptr, int32_t* row_idx, void* out_vals, int64_t* d_nnz, int32_t* map,
                        int32_t* d_status, void* workspace, size_t ws_bytes, void* stream) {
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  if (mode != SPM_MODE_LAST_WRITE && mode != SPM_MODE_SUM) return SPM_ERR_INVALID_ARG;
  if (flags & ~(7u | kFlagKeepZeros)) return SPM_ERR_INVALID_ARG;
  const bool has_seq = (flags & SPM_SEQ_EXPLICIT) != 0;
  if (has_seq != (seq != nullptr)) return SPM_ERR_INVALID_ARG;
  const bool keep_map = (flags & SPM_KEEP_MAP) != 0;
  if (keep_map && map == nullptr) return SPM_ERR_INVALID_ARG;
  if (!d_status || !d_nnz || !col_ptr) return SPM_ERR_INVALID_ARG;
  int dev;
  DevState* ds;
  spm_status s = device_init(dev, ds);
  if (s != SPM_OK) return s;
  spm_tuning tun;
  int64_t withhold;
  {
    std::lock_guard<std::mutex> lk(g_mutex);
    tun = g_tuning;
    withhold = g_withhold;
  }
  const int sv = dtype == SPM_F64 ? 8 : 4;
  const ModeParams mp = mode_params(mode, flags, tun);
  HostPlan hp;
  s = host_plan(B, h_nr, h_nc, h_tp, sv, mp.seq, mp.tgt, ds->sms, tun.two_pass_min_writes, hp);
  if (s != SPM_OK) return s;
  const Layout& L = hp.L;
  if (L.m_total > 0 && (!rows || !cols || !vals || !row_idx || !out_vals)) return SPM_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < L.total) return SPM_ERR_WORKSPACE_TOO_SMALL;
  if (B == 0) return SPM_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  Ctx ctx;
  memset(&ctx, 0, sizeof(ctx));
  ctx.rows = rows;
  ctx.cols = cols;
  ctx.vals = vals;
  ctx.seq = seq;
  ctx.col_ptr = col_ptr;
  ctx.row_idx = row_idx;
  ctx.out_vals = out_vals;
  ctx.d_nnz = d_nnz;
  ctx.map = map;
  ctx.status = d_status;
  ctx.meta = reinterpret_cast<MatMeta*>(ws + L.meta);
  ctx.scal = reinterpret_cast<Scalars*>(ws + L.scal);
  ctx.cta = reinterpret_cast<CtaInfo*>(ws + L.cta);
  ctx.samp = reinterpret_cast<uint64_t*>(ws + L.samp);
  ctx.cellcnt = reinterpret_cast<uint32_t*>(ws + L.cellcnt);
  ctx.lut = reinterpret_cast<uint32_t*>(ws + L.lut);
  ctx.l2cell = reinterpret_cast<int32_t*>(ws + L.l2cell);
  ctx.bk_lo = reinterpret_cast<uint64_t*>(ws + L.bk_lo);
  ctx.bk_info = reinterpret_cast<uint32_t*>(ws + L.bk_info);
  ctx.bk_count = reinterpret_cast<uint32_t*>(ws + L.bk_count);
  ctx.bk_start = reinterpret_cast<uint32_t*>(ws + L.bk_start);
  ctx.bk_state = reinterpret_cast<uint64_t*>(ws + L.bk_state);
  ctx.scanpart = reinterpret_cast<uint32_t*>(ws + L.scanpart);
  ctx.hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  ctx.rec = reinterpret_cast<Rec*>(ws + L.rec);
  ctx.two_pass = L.two_pass ? 1 : 0;
  ctx.tmp = reinterpret_cast<Rec*>(ws + L.tmp);
  ctx.rbk = L.two_pass ? reinterpret_cast<uint32_t*>(ws + L.rbk) : nullptr;
  ctx.l2h = L.l2h_len ? reinterpret_cast<uint32_t*>(ws + L.l2h) : nullptr;
  ctx.bk_cur = reinterpret_cast<uint32_t*>(ws + L.bk_cur);
  ctx.bk_nnz = reinterpret_cast<uint32_t*>(ws + L.bk_nnz);
  ctx.bk_out = reinterpret_cast<uint32_t*>(ws + L.bk_out);
  ctx.big_list = reinterpret_cast<uint32_t*>(ws + L.big_list);
  ctx.groups = (int32_t)two_pass_groups(ds->sms, L.nbcap_total);
  ctx.min_fronts = tun.two_pass_min_fronts;
  ctx.B = L.B;
  ctx.m_total = L.m_total;
  ctx.S_total = L.S_total;
  ctx.lut_total = L.lut_total;
  ctx.nbcap_total = L.nbcap_total;
  ctx.hist_bound = L.hist_bound;
  ctx.C = L.C;
  ctx.sum_mode = mode == SPM_MODE_SUM;
  ctx.f64 = dtype == SPM_F64;
  ctx.keep_map = keep_map;
  ctx.keep_zeros = (flags & kFlagKeepZeros) != 0 && mode == SPM_MODE_LAST_WRITE && !keep_map;
  ctx.has_seq = mp.seq;
  ctx.tgt = mp.tgt;
  ctx.sub_bits = tun.sub_bits;
  ctx.withhold = withhold;

  int64_t call = -1;
  {
    std::lock_guard<std::mutex> lk(g_mutex);
    if (g_ring.on && g_ring.dev == dev) call = g_ring.calls++;
  }
  stage_mark(st, call, 0);
  cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
  cudaMemsetAsync(ws + L.scal, 0, sizeof(Scalars), st);
  cudaMemsetAsync(ws + L.cellcnt, 0, 4 * (size_t)std::max<int64_t>(L.lut_total, 1), st);
  cudaMemsetAsync(ws + L.bk_state, 0, 8 * (size_t)std::max<int64_t>(L.nbcap_total, 1), st);
  if (L.l2h_len) cudaMemsetAsync(ws + L.l2h, 0, 4 * (size_t)L.l2h_len, st);
  if (tun.ordered_path && B == 1 && d_tp == nullptr && !mp.seq && !keep_map && L.m_total > 0) {
    // a stream already in column-major order is finished in one pass; the
    // kernels below then find the abort flag set and return at once
    cudaMemsetAsync(ws + L.tmp, 0, 8 * (size_t)ordered_tiles(L.m_total), st);
    launch_ordered(ctx, h_nr[0], h_nc[0], ds->sms, st);
    g_launches += 1;
  }
  if (B == 1 && d_tp == nullptr) {
    k_setup_single<<<1, 32, 0, st>>>(ctx, hp.single);
  } else {
    int64_t ncols_total = 0;
    unsigned long long h = 0;
    for (int64_t i = 0; i < B; ++i) {
      ncols_total += h_nc[i] + 1;
      h += (unsigned long long)meta_term(i, h_nr[i], h_nc[i], h_tp[i + 1]);
    }
    k_setup_batched<<<1, 1024, 0, st>>>(ctx, d_nr, d_nc, d_tp, L.S_total, L.lut_total, L.l2_total, L.nbcap_total,
                                        ncols_total, h);
  }
  if (L.S_total > 0) k_sample<<<(unsigned)((L.S_total + 255) / 256), 256, 0, st>>>(ctx);
  k_plan<<<(unsigned)B, 1024, kPlanSmem, st>>>(ctx);
  k_bucket_scan<<<1, 1024, 0, st>>>(ctx);
  k_bucket_fill<<<(unsigned)((L.lut_total * 32 + 255) / 256), 256, 0, st>>>(ctx);
  stage_mark(st, call, 1);
  const bool vec = ((reinterpret_cast<uintptr_t>(rows) | reinterpret_cast<uintptr_t>(cols) |
                     reinterpret_cast<uintptr_t>(vals)) & 15u) == 0;
  const bool batched = B > 1;
  if (batched) launch_partition<true>(ctx, L, vec, st, tun.partition_threads, ds->sms, call);
  else launch_partition<false>(ctx, L, vec, st, tun.partition_threads, ds->sms, call);
  launch_resolve(ctx, ds->sms, L.nbcap_total, st);
  stage_mark(st, call, 5);
  if (!keep_map) {
    // offsets of the buckets' elements, then their placement
    launch_bucket_scan(ctx, L, ctx.bk_nnz, ctx.bk_out, st);
    launch_place(ctx, ds->sms, L.nbcap_total, st);
  }
  stage_mark(st, call, 6);
  // setup, plan, 2 bucket kernels, hist, colscan, scan, scatter (with room for two
  // passes: 2 more), resolve, and without the map a scan and 2 placement kernels
  const int scans = L.scan_blocks == 1 ? 1 : 3;
  g_launches += 8 + scans + (L.S_total > 0 ? 1 : 0) + (L.two_pass ? 2 : 0) + (keep_map ? 0 : 2 + scans);
  if (cudaGetLastError() != cudaSuccess) return SPM_ERR_CUDA;
  return SPM_OK;
}

}  // namespace

void count_launches(int64_t n) { g_launches += n; }

spm_status assemble_internal(int64_t n_rows, int64_t n_cols, int64_t m, const int32_t* rows, const int32_t* cols,
                             const void* vals, const uint64_t* seq, spm_dtype dtype, spm_mode mode, uint32_t flags,
                             int64_t* col_ptr, int32_t* row_idx, void* out_vals, int64_t* d_nnz, int32_t* d_status,
                             void* workspace, size_t ws_bytes, void* stream) {
  if (m < 0 || (flags & SPM_KEEP_MAP)) return SPM_ERR_INVALID_ARG;
  const int64_t tp[2] = {0, m};
  return run_assembly(1, &n_rows, &n_cols, tp, nullptr, nullptr, nullptr, rows, cols, vals, seq, dtype, mode, flags,
                      col_ptr, row_idx, out_vals, d_nnz, nullptr, d_status, workspace, ws_bytes, stream);
}

}  // namespace spm

using namespace spm;

extern "C" {

const char* spm_status_string(spm_status s) {
  switch (s) {
    case SPM_OK: return "SPM_OK";
    case SPM_ERR_INVALID_ARG: return "SPM_ERR_INVALID_ARG";
    case SPM_ERR_INDEX_OUT_OF_RANGE: return "SPM_ERR_INDEX_OUT_OF_RANGE";
    case SPM_ERR_WORKSPACE_TOO_SMALL: return "SPM_ERR_WORKSPACE_TOO_SMALL";
    case SPM_ERR_UNSUPPORTED: return "SPM_ERR_UNSUPPORTED";
    case SPM_ERR_CUDA: return "SPM_ERR_CUDA";
    case SPM_ERR_TIMEOUT: return "SPM_ERR_TIMEOUT";
  }
  return "SPM_ERR_UNKNOWN";
}

int32_t spm_version(void) { return 10000; }

spm_status spm_set_tuning(const spm_tuning* t) {
  std::lock_guard<std::mutex> lk(g_mutex);
  if (!t) {
    g_tuning = kDefaultTuning;
    return SPM_OK;
  }
  if (t->bucket_target < 256 || t->bucket_target > 65536) return SPM_ERR_INVALID_ARG;
  if (t->sub_bits < 8 || t->sub_bits > kSubBitsMax) return SPM_ERR_INVALID_ARG;
  if (t->partition_threads != 256 && t->partition_threads != 512 && t->partition_threads != 1024)
    return SPM_ERR_INVALID_ARG;
  if (t->resolve_threads != 512) return SPM_ERR_INVALID_ARG;
  if (t->two_pass_min_writes < 0 || t->two_pass_min_fronts < 0) return SPM_ERR_INVALID_ARG;
  if (t->ordered_path != 0 && t->ordered_path != 1) return SPM_ERR_INVALID_ARG;
  g_tuning = *t;
  return SPM_OK;
}

spm_status spm_debug_withhold_publication(int64_t bucket) {
  if (bucket < -1) return SPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mutex);
  g_withhold = bucket;
  return SPM_OK;
}

spm_status spm_debug_stage_timing(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_mutex);
  if (enable) {
    if (g_ring.on) return SPM_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPM_ERR_CUDA;
    for (int i = 0; i < kRing; ++i)
      for (int j = 0; j <= kStages; ++j)
        if (cudaEventCreate(&g_ring.ev[i][j]) != cudaSuccess) return SPM_ERR_CUDA;
    g_ring.dev = dev;
    g_ring.calls = 0;
    g_ring.on = true;
  } else if (g_ring.on) {
    for (int i = 0; i < kRing; ++i)
      for (int j = 0; j <= kStages; ++j) cudaEventDestroy(g_ring.ev[i][j]);
    g_ring.on = false;
  }
  return SPM_OK;
}

spm_status spm_debug_stage_times(int32_t back, float* ms, int32_t n) {
  std::lock_guard<std::mutex> lk(g_mutex);
  if (!ms || n < 0 || n > kStages || back < 0 || back >= kRing) return SPM_ERR_INVALID_ARG;
  if (!g_ring.on || back >= g_ring.calls) return SPM_ERR_INVALID_ARG;
  const int64_t call = g_ring.calls - 1 - back;
  for (int j = 0; j < n; ++j) {
    if (cudaEventElapsedTime(&ms[j], g_ring.ev[call % kRing][j], g_ring.ev[call % kRing][j + 1]) != cudaSuccess)
      return SPM_ERR_CUDA;
  }
  return SPM_OK;
}

int64_t spm_debug_launch_count(void) { return g_launches.load(); }

spm_status spm_debug_plan_stats(const void* workspace, size_t ws_bytes, int64_t n_rows, int64_t n_cols, int64_t m,
                                spm_dtype dtype, spm_mode mode, uint32_t flags, int64_t* stats, int32_t n_stats) {
  if (!workspace || !stats || n_stats < 0) return SPM_ERR_INVALID_ARG;
  spm_tuning tun;
  {
    std::lock_guard<std::mutex> lk(g_mutex);
    tun = g_tuning;
  }
  int dev;
  DevState* ds;
  spm_status s = device_init(dev, ds);
  if (s != SPM_OK) return s;
  const int64_t tp[2] = {0, m};
  HostPlan hp;
  const ModeParams mp = mode_params(mode, flags, tun);
  s = host_plan(1, &n_rows, &n_cols, tp, dtype == SPM_F64 ? 8 : 4, mp.seq, mp.tgt, ds->sms, tun.two_pass_min_writes, hp);
  if (s != SPM_OK) return s;
  if (ws_bytes < hp.L.total) return SPM_ERR_WORKSPACE_TOO_SMALL;
  const char* ws = static_cast<const char*>(workspace);
  Scalars sc;
  MatMeta mm;
  if (cudaMemcpy(&sc, ws + hp.L.scal, sizeof(sc), cudaMemcpyDeviceToHost) != cudaSuccess) return SPM_ERR_CUDA;
  if (cudaMemcpy(&mm, ws + hp.L.meta, sizeof(mm), cudaMemcpyDeviceToHost) != cudaSuccess) return SPM_ERR_CUDA;
  std::vector<uint32_t> cnt(sc.NB);
  if (sc.NB && cudaMemcpy(cnt.data(), ws + hp.L.bk_count, 4 * (size_t)sc.NB, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SPM_ERR_CUDA;
  int64_t mx = 0, over = 0, over_w = 0;
  for (uint32_t c : cnt) {
    mx = std::max<int64_t>(mx, c);
    if (c > (uint32_t)mp.cap) {
      ++over;
      over_w += c;
    }
  }
  const bool ordered = m > 0 && sc.ord_fail == 0u && (int64_t)sc.ord_done == ordered_tiles(m);
  const int64_t v[8] = {(int64_t)sc.NB, mx, over, over_w, mp.cap, mm.h2used, mm.nbcap, ordered ? 1 : 0};
  for (int i = 0; i < n_stats && i < 8; ++i) stats[i] = v[i];
  return SPM_OK;
}

spm_status spm_get_tuning(spm_tuning* t) {
  if (!t) return SPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mutex);
  *t = g_tuning;
  return SPM_OK;
}

spm_status spm_assemble_csc_batched_workspace(int64_t batch, const int64_t* h_n_rows, const int64_t* h_n_cols,
                                              const int64_t* h_trip_ptr, spm_dtype dtype, spm_mode mode,
                                              uint32_t flags, size_t* bytes) {
  if (!bytes) return SPM_ERR_INVALID_ARG;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  if (mode != SPM_MODE_LAST_WRITE && mode != SPM_MODE_SUM) return SPM_ERR_INVALID_ARG;
  if (flags & ~7u) return SPM_ERR_INVALID_ARG;
  spm_tuning tun;
  {
    std::lock_guard<std::mutex> lk(g_mutex);
    tun = g_tuning;
  }
  HostPlan hp;
  const ModeParams mp = mode_params(mode, flags, tun);
  const spm_status s = host_plan(batch, h_n_rows, h_n_cols, h_trip_ptr, dtype == SPM_F64 ? 8 : 4, mp.seq, mp.tgt,
                                 num_sms_for_sizing(), tun.two_pass_min_writes, hp);
  if (s != SPM_OK) return s;
  *bytes = hp.L.total;
  return SPM_OK;
}

spm_status spm_assemble_csc_workspace(int64_t n_rows, int64_t n_cols, int64_t m, spm_dtype dtype, spm_mode mode,
                                      uint32_t flags, size_t* bytes) {
  if (m < 0) return SPM_ERR_INVALID_ARG;
  const int64_t tp[2] = {0, m};
  return spm_assemble_csc_batched_workspace(1, &n_rows, &n_cols, tp, dtype, mode, flags, bytes);
}

spm_status spm_assemble_csc(int64_t n_rows, int64_t n_cols, int64_t m, const int32_t* rows, const int32_t* cols,
                            const void* vals, const uint64_t* seq, spm_dtype dtype, spm_mode mode, uint32_t flags,
                            int64_t* col_ptr, int32_t* row_idx, void* out_vals, int64_t* d_nnz, int32_t* map,
                            int32_t* d_status, void* workspace, size_t ws_bytes, void* stream) {
  if (m < 0 || (flags & ~7u)) return SPM_ERR_INVALID_ARG;
  const int64_t tp[2] = {0, m};
  return run_assembly(1, &n_rows, &n_cols, tp, nullptr, nullptr, nullptr, rows, cols, vals, seq, dtype, mode, flags,
                      col_ptr, row_idx, out_vals, d_nnz, map, d_status, workspace, ws_bytes, stream);
}

spm_status spm_assemble_csc_batched(int64_t batch, const int64_t* h_n_rows, const int64_t* h_n_cols,
                                    const int64_t* h_trip_ptr, const int64_t* d_n_rows, const int64_t* d_n_cols,
                                    const int64_t* d_trip_ptr, const int32_t* rows, const int32_t* cols,
                                    const void* vals, const uint64_t* seq, spm_dtype dtype, spm_mode mode,
                                    uint32_t flags, int64_t* col_ptr, int32_t* row_idx, void* out_vals,
                                    int64_t* d_nnz, int32_t* map, int32_t* d_status, void* workspace,
                                    size_t ws_bytes, void* stream) {
  if (batch > 0 && (!d_n_rows || !d_n_cols || !d_trip_ptr)) return SPM_ERR_INVALID_ARG;
  if (flags & ~7u) return SPM_ERR_INVALID_ARG;
  return run_assembly(batch, h_n_rows, h_n_cols, h_trip_ptr, d_n_rows, d_n_cols, d_trip_ptr, rows, cols, vals, seq,
                      dtype, mode, flags, col_ptr, row_idx, out_vals, d_nnz, map, d_status, workspace, ws_bytes,
                      stream);
}

}  // extern "C"
