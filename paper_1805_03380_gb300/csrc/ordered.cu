// Single pass for a write stream that is already in column-major order (the
// paper's quasi-ordered insertion, Section 4: elements inserted in order; the
// tree's append fast path of Section 3.3, which finds the position of an
// element past all previous ones without a search).
//
// When the linear indices row + col * n_rows of the writes never decrease,
// the stream is its own sort: every run of equal indices is one element, in
// CSC order.  k_ordered reads the stream once, tile by tile (tiles taken in
// order through a ticket): it checks the order, reduces every run whose first
// write lies in the tile (the run may continue a little past it), drops
// zeros, finds the tile's output offset with a bounded decoupled look-back and
// writes the stored elements and the column offsets of the columns that start
// inside the tile.  If every tile succeeds, the last one sets the abort flag
// of the call, and the kernels of the general path (which all test it) return
// at once.  A tile that finds two writes out of order, an index outside the
// matrix or a run longer than it can hold stops the pass; the general path
// then runs as usual and overwrites everything (and reports the bad index).
//
// Reduction rules are those of the general path: last-write mode keeps the
// last write of a run; add mode uses one write as it is and otherwise the
// exact fixed-point accumulator (binary point set by the run's largest
// exponent, exact_sum.cuh) rounded once.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include <cuda_runtime.h>

#include "exact_sum.cuh"
#include "spm.h"
#include "spm_common.cuh"

namespace spm {
namespace {

constexpr int kOT = 512;                    // threads per block
constexpr int kOI = 8;                      // positions per thread
constexpr int kOTile = kOT * kOI;           // positions per tile
constexpr int kOExt = 64;                   // positions read past the tile for a run that continues
constexpr int kOBuf = 1 + kOTile + kOExt;   // [previous write, tile, extension]
constexpr unsigned kAll = 0xffffffffu;
constexpr uint64_t kOAgg = 1ull << 62, kOIncl = 2ull << 62, kOMask = (1ull << 62) - 1;
constexpr uint64_t kOWaitNs = 2000000000ull;

__device__ __forceinline__ uint64_t o_now() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint64_t o_ld_acquire(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void o_st_release(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ bool o_failed(const Ctx& c) {
  return *reinterpret_cast<volatile uint32_t*>(&c.scal->ord_fail) != 0u;
}
__device__ __forceinline__ uint64_t o_wide(uint64_t v, bool f64) {
  return f64 ? v : (uint64_t)__double_as_longlong((double)__uint_as_float((uint32_t)v));
}

// Value of one run [j, e) of equal indices and whether it is stored.
template <bool F64, bool SUM>
__device__ uint64_t reduce_run(const uint64_t* val, int j, int e, bool keep_zeros, bool& keep) {
  if (!SUM) {
    const uint64_t b = val[e - 1];
    keep = keep_zeros || (F64 ? (b & 0x7FFFFFFFFFFFFFFFull) != 0 : (b & 0x7FFFFFFFull) != 0);
    return b;
  }
  if (e - j == 1) {
    const uint64_t bits = val[j];
    keep = F64 ? (bits & 0x7FFFFFFFFFFFFFFFull) != 0 : (bits & 0x7FFFFFFFull) != 0;
    return bits;
  }
  if (e - j == 2) {
    // two writes whose exponents lie within the accumulator's window of each
    // other (or a zero, an infinity, a NaN): the accumulator would hold their
    // sum exactly, and one IEEE addition rounds that exact sum correctly --
    // the same bits without the 128-bit path (float32 values: the float64 sum
    // is exact within 28 binades, then rounded once to float32)
    const uint64_t wa = o_wide(val[j], F64), wb = o_wide(val[j + 1], F64);
    const int ea = f64_align_exponent(wa), eb = f64_align_exponent(wb);
    if (ea <= 0 || eb <= 0 || abs(ea - eb) <= (F64 ? kAlignBits : 28)) {
      const double sum = __longlong_as_double((long long)wa) + __longlong_as_double((long long)wb);
      const uint64_t bits = F64 ? (uint64_t)__double_as_longlong(sum) : (uint64_t)__float_as_uint((float)sum);
      keep = F64 ? (bits & 0x7FFFFFFFFFFFFFFFull) != 0 : (bits & 0x7FFFFFFFull) != 0;
      return bits;
    }
  }
  int emax = 1;
  for (int q = j; q < e; ++q) emax = max(emax, f64_align_exponent(o_wide(val[q], F64)));
  Acc acc = acc_zero();
  for (int q = j; q < e; ++q) acc_add_bits(acc, o_wide(val[q], F64), emax);
  bool nz;
  const uint64_t bits = acc_round(acc, emax, !F64, &nz);
  keep = nz;
  return bits;
}

template <bool F64, bool SUM>
__global__ void __launch_bounds__(kOT, 2) k_ordered(Ctx c, int64_t n_rows, int64_t n_cols) {
  extern __shared__ __align__(16) unsigned char o_smem[];
  uint64_t* s_val = reinterpret_cast<uint64_t*>(o_smem);  // [kOBuf]
  int32_t* s_row = reinterpret_cast<int32_t*>(s_val + kOBuf);
  int32_t* s_col = s_row + kOBuf;
  __shared__ int32_t s_cnt[kOI * (kOT / 32)], s_pre[kOI * (kOT / 32)];  // kept per (slot row, warp)
  __shared__ int32_t s_total;
  __shared__ int32_t s_first, s_wait, s_stop;
  __shared__ unsigned long long s_lb_sum;
  __shared__ uint64_t s_lb_t0;
  __shared__ uint32_t s_tile;
  __shared__ int32_t s_bad;
  __shared__ int64_t s_excl;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t m = c.m_total;
  const int64_t tiles = (m + kOTile - 1) / kOTile;
  uint64_t* state = reinterpret_cast<uint64_t*>(c.tmp);
  const bool kz = !SUM && c.keep_zeros;
  using VT = typename std::conditional<F64, uint64_t, uint32_t>::type;
  const VT* vin = static_cast<const VT*>(c.vals);
  VT* vout = static_cast<VT*>(c.out_vals);
  // a probe of 32 writes spread over the stream: most streams that are not
  // in order are turned away here, before any tile is read
  if (w == 0) {
    const int64_t p = m > 1 ? (int64_t)lane * (m - 1) / 31 : 0;
    const int64_t key = (int64_t)c.cols[p] * n_rows + c.rows[p];
    const int64_t prev = __shfl_up_sync(kAll, key, 1);
    const bool any_desc = __any_sync(kAll, lane > 0 && key < prev);
    if (lane == 0) s_bad = any_desc ? 1 : 0;
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) atomicExch(&c.scal->ord_fail, 1u);
    return;
  }
  constexpr int kLoads = (kOBuf + kOT - 1) / kOT;
  __shared__ uint32_t s_done;  // tiles this block finished
  if (tid == 0) s_done = 0;
  while (true) {
    __syncthreads();  // the previous tile is done with the buffers and s_bad
    if (tid == 0) {
      s_tile = o_failed(c) ? ~0u : atomicAdd(&c.scal->ord_ticket, 1u);
      s_bad = 0;
    }
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= tiles) break;
    const int64_t p0 = t * kOTile - 1;  // buffer slot j holds stream position p0 + j
    // load the previous write, the tile and the extension: all loads first
    int32_t lr[kLoads], lc[kLoads];
    VT lv[kLoads];
    bool bad = false;
#pragma unroll
    for (int i = 0; i < kLoads; ++i) {
      const int64_t p = p0 + tid + i * kOT;
      lr[i] = -1;
      lc[i] = -1;
      lv[i] = 0;
      if (tid + i * kOT < kOBuf && p >= 0 && p < m) {
        lr[i] = __ldcs(c.rows + p);
        lc[i] = __ldcs(c.cols + p);
        lv[i] = __ldcs(vin + p);
      }
    }
#pragma unroll
    for (int i = 0; i < kLoads; ++i) {
      const int j = tid + i * kOT;
      if (j < kOBuf) {
        const int64_t p = p0 + j;
        if (p >= 0 && p < m && (lr[i] < 0 || (int64_t)lr[i] >= n_rows || lc[i] < 0 || (int64_t)lc[i] >= n_cols))
          bad = true;
        s_row[j] = lr[i];
        s_col[j] = lc[i];
        s_val[j] = (uint64_t)lv[i];
      }
    }
    __syncthreads();
    // slot k of this thread is j = 1 + tid + k * kOT: neighbouring threads
    // read neighbouring words of the buffers
    // order: every write of the tile is at or before the next write
#pragma unroll
    for (int k = 0; k < kOI; ++k) {
      const int j = 1 + tid + k * kOT;
      if (p0 + j + 1 < m)
        bad |= s_col[j + 1] < s_col[j] || (s_col[j + 1] == s_col[j] && s_row[j + 1] < s_row[j]);
    }
    if (__syncthreads_or(bad)) {
      if (tid == 0) atomicExch(&c.scal->ord_fail, 1u);
      break;
    }
    bad = false;
    // runs whose first write is in one of this thread's slots
    uint32_t kmask = 0;
    int32_t orow[kOI];
    uint64_t oval[kOI];
#pragma unroll
    for (int k = 0; k < kOI; ++k) {
      const int j = 1 + tid + k * kOT;
      orow[k] = 0;
      oval[k] = 0;
      const int64_t p = p0 + j;
      if (p >= m) continue;
      const bool head = p == 0 || s_col[j] != s_col[j - 1] || s_row[j] != s_row[j - 1];
      if (!head) continue;
      int e = j + 1;
      while (e < kOBuf && p0 + e < m && s_col[e] == s_col[j] && s_row[e] == s_row[j]) ++e;
      if (e == kOBuf && p0 + e < m) {  // the run may go on past what the tile read
        bad = true;
        continue;
      }
      bool keep;
      oval[k] = reduce_run<F64, SUM>(s_val, j, e, kz, keep);
      orow[k] = s_row[j];
      if (keep) kmask |= 1u << k;
    }
    // output slot of every kept element: slots are in order row by row (k),
    // warp by warp inside a row, lane by lane inside a warp
    const unsigned lt = (1u << lane) - 1u;
    uint32_t lpre[kOI];
#pragma unroll
    for (int k = 0; k < kOI; ++k) {
      const unsigned bal = __ballot_sync(kAll, (kmask >> k) & 1u);
      lpre[k] = __popc(bal & lt);
      if (lane == 0) s_cnt[k * (kOT / 32) + w] = __popc(bal);
    }
    if (__syncthreads_or(bad)) {
      if (tid == 0) atomicExch(&c.scal->ord_fail, 1u);
      break;
    }
    if (w == 0) {  // exclusive scan of the kOI * (kOT / 32) counts, kPer per lane
      constexpr int kCnt = kOI * (kOT / 32);
      constexpr int kPer = kCnt / 32;
      static_assert(kCnt % 32 == 0, "whole counts per lane");
      int a[kPer];
      int sum = 0;
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        a[u] = s_cnt[kPer * lane + u];
        sum += a[u];
      }
      int inc = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kAll, inc, o);
        if (lane >= o) inc += y;
      }
      int ex = inc - sum;
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        s_pre[kPer * lane + u] = ex;
        ex += a[u];
      }
      if (lane == 31) s_total = inc;
    }
    __syncthreads();
    const int total = s_total;
    // the tile's output offset: decoupled look-back over the earlier tiles,
    // 256 of them per round (one per thread); bounded, gives up if the pass failed
    if (t == 0) {
      if (tid == 0) {
        o_st_release(&state[0], kOIncl | (uint64_t)total);
        s_excl = 0;
      }
    } else {
      if (tid == 0) {
        o_st_release(&state[t], kOAgg | (uint64_t)total);
        s_lb_t0 = o_now();
        s_lb_sum = 0;
      }
      int64_t top = t - 1;
      uint32_t spins = 0;
      while (true) {
        const int64_t bb = top - tid;
        const uint64_t st = bb >= 0 ? o_ld_acquire(&state[bb]) : kOIncl;
        const uint64_t flag = st & ~kOMask;
        __syncthreads();  // everyone has read the previous round's flags
        if (tid == 0) {
          s_first = kOT;
          s_wait = 0;
        }
        __syncthreads();
        if (flag == kOIncl) atomicMin(&s_first, tid);
        __syncthreads();
        const int first = s_first;  // nearest predecessor holding its inclusive prefix (kOT: none)
        if (tid <= first && flag == 0) s_wait = 1;
        __syncthreads();
        if (!s_wait) {
          unsigned long long v = tid <= first ? (st & kOMask) : 0ull;
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
          if (lane == 0 && v) atomicAdd(&s_lb_sum, v);
          top -= kOT;
          if (first < kOT) break;
          continue;
        }
        if (tid == 0) {
          __nanosleep(64);
          s_stop = (o_failed(c) || ((++spins & 7) == 0 && o_now() - s_lb_t0 > kOWaitNs)) ? 1 : 0;
        }
        __syncthreads();
        if (s_stop) break;
      }
      __syncthreads();
      if (tid == 0) {
        const bool fail = s_stop != 0 && s_wait != 0;
        if (fail) {
          atomicExch(&c.scal->ord_fail, 1u);
          s_excl = -1;
        } else {
          s_excl = (int64_t)s_lb_sum;
          o_st_release(&state[t], kOIncl | (uint64_t)(s_lb_sum + (unsigned long long)total));
        }
      }
    }
    __syncthreads();
    const int64_t excl = s_excl;
    if (excl < 0) break;
    // column offsets of the columns whose first write is in one of this thread's slots
#pragma unroll
    for (int k = 0; k < kOI; ++k) {
      const int j = 1 + tid + k * kOT;
      const int64_t p = p0 + j;
      if (p >= m) break;
      const int64_t before = excl + s_pre[k * (kOT / 32) + w] + lpre[k];
      const int64_t cj = s_col[j];
      const int64_t cprev = p == 0 ? -1 : s_col[j - 1];
      for (int64_t q = cprev + 1; q <= cj; ++q) c.col_ptr[q] = before;
      if (p == m - 1) {
        for (int64_t q = cj + 1; q <= n_cols; ++q) c.col_ptr[q] = excl + total;
        *c.d_nnz = excl + total;
      }
    }
    __syncthreads();  // the buffers are reused for the output below
    // stage the stored elements in output order, then write them out
#pragma unroll
    for (int k = 0; k < kOI; ++k)
      if ((kmask >> k) & 1u) {
        const int o = s_pre[k * (kOT / 32) + w] + (int)lpre[k];
        s_row[o] = orow[k];
        s_val[o] = oval[k];
      }
    __syncthreads();
    for (int k = tid; k < total; k += kOT) {
      c.row_idx[excl + k] = s_row[k];
      vout[excl + k] = (VT)s_val[k];
    }
    if (tid == 0) ++s_done;
  }
  // the last block to leave, if every tile was finished and nothing failed,
  // makes the general path stand down
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (s_done) atomicAdd(&c.scal->ord_done, s_done);
    __threadfence();
    const uint32_t left = atomicAdd(&c.scal->ord_exit, 1u) + 1u;
    if (left == gridDim.x && !o_failed(c) && *reinterpret_cast<volatile uint32_t*>(&c.scal->ord_done) == (uint32_t)tiles)
      atomicExch(&c.scal->abort, 1u);
  }
}

constexpr int kOSmem = kOBuf * (8 + 4 + 4);

template <bool F64, bool SUM>
cudaError_t launch_ordered_t(const Ctx& c, int64_t n_rows, int64_t n_cols, unsigned grid, cudaStream_t st) {
  k_ordered<F64, SUM><<<grid, kOT, kOSmem, st>>>(c, n_rows, n_cols);
  return cudaGetLastError();
}

// The shared-memory limit of the four instances, raised once per device (on
// the first call, which comes before any stream capture).
bool g_ord_ready[64] = {};
std::mutex g_ord_mutex;

cudaError_t ordered_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (g_ord_ready[dev]) return cudaSuccess;
  std::lock_guard<std::mutex> lk(g_ord_mutex);
  if (g_ord_ready[dev]) return cudaSuccess;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_ordered<true, true>, a, kOSmem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_ordered<true, false>, a, kOSmem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_ordered<false, true>, a, kOSmem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_ordered<false, false>, a, kOSmem)) != cudaSuccess) return e;
  g_ord_ready[dev] = true;
  return cudaSuccess;
}

}  // namespace

int64_t ordered_tiles(int64_t m) { return (m + kOTile - 1) / kOTile; }

cudaError_t launch_ordered(const Ctx& c, int64_t n_rows, int64_t n_cols, int sms, cudaStream_t st) {
  const cudaError_t e = ordered_prepare();
  if (e != cudaSuccess) return e;
  const int64_t tiles = ordered_tiles(c.m_total);
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)sms * 2);
  if (c.f64)
    return c.sum_mode ? launch_ordered_t<true, true>(c, n_rows, n_cols, grid, st)
                      : launch_ordered_t<true, false>(c, n_rows, n_cols, grid, st);
  return c.sum_mode ? launch_ordered_t<false, true>(c, n_rows, n_cols, grid, st)
                    : launch_ordered_t<false, false>(c, n_rows, n_cols, grid, st);
}

}  // namespace spm
