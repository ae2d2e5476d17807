// Device helpers shared by the assembly kernels (libspm, sm_103a): status
// reporting, bounded waits, block scans, division by an invariant divisor and
// the decoupled look-back over buckets.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "spm_common.cuh"

namespace spm {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // every wait on another block gives up after 2 s

__device__ __forceinline__ void record_error(const Ctx& c, int code) { atomicCAS(c.status, 0, code); }

__device__ __forceinline__ void record_fatal(const Ctx& c, int code) {
  atomicCAS(c.status, 0, code);
  atomicExch(&c.scal->abort, 1u);
}

__device__ __forceinline__ bool is_aborted(const Ctx& c) {
  return *reinterpret_cast<volatile uint32_t*>(&c.scal->abort) != 0u;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive scan of one value per thread over the block (blockDim a multiple
// of 32, at most 1024).  buf needs 32 entries.  Returns the prefix; *total
// receives the block total.  Contains __syncthreads.
template <typename T>
__device__ T block_scan_excl(T v, T* total, T* buf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) buf[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? buf[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    buf[lane] = w;
  }
  __syncthreads();
  T res = (warp ? buf[warp - 1] : T(0)) + x - v;
  if (total) *total = buf[nw - 1];
  __syncthreads();
  return res;
}

// Division of 32-bit integers by an invariant divisor with a multiply and
// shifts (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994, the round-up method of their Fig. 4.1): for
// 1 <= d < 2^32 and l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1 and
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), t = mulhi(m, n).
struct Div32 {
  uint32_t m, s1, s2;
};

__host__ __device__ inline Div32 div32_make(uint32_t d) {
#ifdef __CUDA_ARCH__
  const int l = d > 1 ? 32 - __clz((int)(d - 1)) : 0;
#else
  int l = 0;
  while ((uint64_t{1} << l) < (uint64_t)d) ++l;
#endif
  Div32 r;
  r.m = (uint32_t)(((uint64_t{1} << 32) * ((uint64_t{1} << l) - d)) / d + 1);
  r.s1 = l < 1 ? (uint32_t)l : 1u;
  r.s2 = l > 1 ? (uint32_t)(l - 1) : 0u;
  return r;
}

__device__ __forceinline__ uint32_t div32(uint32_t n, const Div32& D) {
  const uint32_t t = __umulhi(D.m, n);
  return (t + ((n - t) >> D.s1)) >> D.s2;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Wait (bounded) for the look-back chain of bucket b to provide its exclusive
// prefix (the number of stored elements of the same matrix in all earlier
// buckets).  Called by one full warp: each round reads the states of the 128
// nearest predecessors not yet accounted for (four per lane, loads in flight
// together), adds the counts back to the nearest one that holds an inclusive
// value, or waits while one of those nearer ones has published nothing yet.
// Only counts travel through the states, so relaxed loads suffice.  Publishes
// nothing.  Every lane returns the prefix; on an expired wait (SPM_ERR_TIMEOUT
// recorded, abort flag set) or an aborted call the result is meaningless and
// the caller must stop.
__device__ inline int64_t lookback_wait_warp(const Ctx& c, int64_t b) {
  const int lane = threadIdx.x & 31;
  int64_t excl = 0;
  int64_t top = b - 1;  // nearest predecessor not yet accounted for
  const uint64_t t_start = global_timer_ns();
  uint32_t spins = 0;
  while (true) {
    uint64_t s[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t bb = top - (r * 32 + lane);
      s[r] = bb >= 0 ? ld_relaxed_u64(&c.bk_state[bb]) : kStIncl;
    }
    int used = 0;  // groups of 32 fully accounted for
    bool done = false;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (done || used < r) continue;
      const uint64_t flag = s[r] & ~kStMask;
      const unsigned incl = __ballot_sync(kFull, flag == kStIncl);
      const unsigned none = __ballot_sync(kFull, flag == 0);
      const int first_incl = incl ? __ffs(incl) - 1 : 32;
      const unsigned upto = first_incl >= 31 ? kFull : ((2u << first_incl) - 1u);
      if (none & upto) continue;  // a nearer predecessor has not published: wait
      uint64_t v = (lane <= first_incl) ? (s[r] & kStMask) : 0ull;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      excl += (int64_t)v;
      if (first_incl < 32) done = true;
      else used = r + 1;
    }
    if (done) break;
    top -= 32 * used;
    if (used > 0) continue;
    __nanosleep(64);  // leave the issue slots to the other warps meanwhile
    // leave the wait together: lane 0 decides for the warp
    int stop = 0;
    if (lane == 0) {
      if (is_aborted(c)) {
        stop = 1;
      } else if ((++spins & 7) == 0 && global_timer_ns() - t_start > kWaitLimitNs) {
        record_fatal(c, SPM_ERR_TIMEOUT);
        stop = 1;
      }
    }
    if (__shfl_sync(kFull, stop, 0)) break;
  }
  return excl;
}

// Decoupled look-back: publish this bucket's count, wait for the prefix,
// publish the inclusive value.  Called by one full warp.
__device__ inline int64_t lookback_warp(const Ctx& c, int64_t b, uint32_t nnz) {
  if ((threadIdx.x & 31) == 0) st_release_u64(&c.bk_state[b], kStAgg | nnz);
  __syncwarp();
  const int64_t excl = lookback_wait_warp(c, b);
  if ((threadIdx.x & 31) == 0) st_release_u64(&c.bk_state[b], kStIncl | (uint64_t)(excl + nnz));
  return excl;
}

}  // namespace spm
