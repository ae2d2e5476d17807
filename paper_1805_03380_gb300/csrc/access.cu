// Element access on a CSC matrix and its coordinate-list form.
//
// spm_csc_lookup: Section 3.1 -- an element is found (or shown not to be
// stored) by one read of its column's start and end, then a binary search
// among the column's row indices.  One thread per query.
//
// spm_csc_to_coo: Section 3.2 -- the coordinate list holds, for every stored
// element, its row, its column and its value; the CSC arrays already hold the
// rows and the values in column-major order, so the export writes the column
// of every element (and copies the other two arrays when asked).  One block
// per tile of kCooTile elements: two binary searches over the column offsets
// give the columns of the tile's first and last element, the starts of the
// columns in between go to a table in shared memory, and every element's
// column is the tile's first column plus the number of those starts at or
// before it.
#include <climits>
#include <cstdint>

#include <cuda_runtime.h>

#include "spm.h"
#include "spm_common.cuh"

namespace {

constexpr int kCooThreads = 256;
constexpr int kCooItems = 8;
constexpr int kCooTile = kCooThreads * kCooItems;

__device__ __forceinline__ void set_status(int32_t* status, int code) { atomicCAS(status, 0, code); }

// Column offsets of a CSC matrix with nnz elements: 0 first, nnz last, never decreasing.
__global__ void k_check_offsets(const int64_t* __restrict__ cp, int64_t n_cols, int64_t nnz, int32_t* status) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > n_cols) return;
  const int64_t v = cp[j];
  bool ok = v >= 0 && v <= nnz;
  if (j == 0) ok = ok && v == 0;
  if (j == n_cols) ok = ok && v == nnz;
  if (j < n_cols) ok = ok && cp[j + 1] >= v;
  if (!ok) set_status(status, SPM_ERR_INVALID_ARG);
}

template <typename VT>
__global__ void k_lookup(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* __restrict__ cp,
                         const int32_t* __restrict__ ri, const VT* __restrict__ v, int64_t q,
                         const int32_t* __restrict__ qr, const int32_t* __restrict__ qc, VT* __restrict__ out,
                         int64_t* __restrict__ pos, int32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q) return;
  const int32_t r = qr[i], c = qc[i];
  int64_t found = -1;
  if (r < 0 || (int64_t)r >= n_rows || c < 0 || (int64_t)c >= n_cols) {
    set_status(status, SPM_ERR_INDEX_OUT_OF_RANGE);
  } else {
    // the column's elements, clamped to the arrays (malformed offsets read nothing outside them)
    int64_t lo = cp[c], end = cp[c + 1];
    lo = lo < 0 ? 0 : (lo > nnz ? nnz : lo);
    end = end < lo ? lo : (end > nnz ? nnz : end);
    int64_t hi = end;
    while (lo < hi) {  // first row >= r
      const int64_t mid = (lo + hi) >> 1;
      if (__ldg(ri + mid) < r) lo = mid + 1; else hi = mid;
    }
    if (lo < end && __ldg(ri + lo) == r) found = lo;
  }
  out[i] = found >= 0 ? __ldg(v + found) : VT(0);
  if (pos) pos[i] = found;
}

template <typename VT>
__global__ void __launch_bounds__(kCooThreads) k_to_coo(int64_t n_cols, int64_t nnz, const int64_t* __restrict__ cp,
                                                        const int32_t* __restrict__ ri, const VT* __restrict__ v,
                                                        int32_t* __restrict__ o_rows, int32_t* __restrict__ o_cols,
                                                        VT* __restrict__ o_vals) {
  __shared__ int32_t s_start[kCooTile];  // starts of the tile's later columns, relative to the tile
  __shared__ int64_t s_c[2];
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * kCooTile;
  const int64_t e1 = e0 + kCooTile < nnz ? e0 + kCooTile : nnz;
  if (tid < 2) {
    // column of element e: the last column whose start is <= e
    const int64_t e = tid == 0 ? e0 : e1 - 1;
    int64_t lo = 1, hi = n_cols;  // first j in [1, n_cols] with cp[j] > e
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cp[mid] > e) hi = mid; else lo = mid + 1;
    }
    s_c[tid] = lo - 1;
  }
  __syncthreads();
  const int64_t c_first = s_c[0];
  const int64_t c_last = s_c[1] > c_first ? s_c[1] : c_first;
  const int64_t span = c_last - c_first;  // columns starting after c_first, up to c_last
  const bool table = span <= kCooTile;
  if (table)
    for (int64_t k = tid; k < span; k += kCooThreads) {
      const int64_t s = cp[c_first + 1 + k] - e0;
      s_start[k] = (int32_t)(s < -1 ? -1 : (s > kCooTile ? kCooTile : s));
    }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kCooItems; ++i) {
    const int k = tid + i * kCooThreads;
    const int64_t e = e0 + k;
    if (e >= e1) break;
    int64_t lo = 0, hi = span;
    if (table) {
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (s_start[mid] <= k) lo = mid + 1; else hi = mid;
      }
    } else {
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cp[c_first + 1 + mid] <= e) lo = mid + 1; else hi = mid;
      }
    }
    o_cols[e] = (int32_t)(c_first + lo);
    if (o_rows) o_rows[e] = __ldg(ri + e);
    if (o_vals) o_vals[e] = __ldg(v + e);
  }
}

}  // namespace

extern "C" {

spm_status spm_csc_lookup(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* col_ptr, const int32_t* row_idx,
                          const void* vals, spm_dtype dtype, int64_t q, const int32_t* q_rows, const int32_t* q_cols,
                          void* out_vals, int64_t* out_pos, int32_t* d_status, void* stream) {
  if (n_rows < 0 || n_cols < 0 || nnz < 0 || q < 0) return SPM_ERR_INVALID_ARG;
  if (n_rows > INT32_MAX || n_cols > INT32_MAX) return SPM_ERR_UNSUPPORTED;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  if (!col_ptr || !d_status || (nnz > 0 && (!row_idx || !vals))) return SPM_ERR_INVALID_ARG;
  if (q > 0 && (!q_rows || !q_cols || !out_vals)) return SPM_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
  k_check_offsets<<<(unsigned)((n_cols + 1 + 255) / 256), 256, 0, st>>>(col_ptr, n_cols, nnz, d_status);
  if (q > 0) {
    const unsigned blocks = (unsigned)((q + 255) / 256);
    if (dtype == SPM_F64)
      k_lookup<uint64_t><<<blocks, 256, 0, st>>>(n_rows, n_cols, nnz, col_ptr, row_idx,
                                                 static_cast<const uint64_t*>(vals), q, q_rows, q_cols,
                                                 static_cast<uint64_t*>(out_vals), out_pos, d_status);
    else
      k_lookup<uint32_t><<<blocks, 256, 0, st>>>(n_rows, n_cols, nnz, col_ptr, row_idx,
                                                 static_cast<const uint32_t*>(vals), q, q_rows, q_cols,
                                                 static_cast<uint32_t*>(out_vals), out_pos, d_status);
  }
  spm::count_launches(q > 0 ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? SPM_OK : SPM_ERR_CUDA;
}

spm_status spm_csc_to_coo(int64_t n_cols, int64_t nnz, const int64_t* col_ptr, const int32_t* row_idx,
                          const void* vals, spm_dtype dtype, int32_t* out_rows, int32_t* out_cols, void* out_vals,
                          int32_t* d_status, void* stream) {
  if (n_cols < 0 || nnz < 0) return SPM_ERR_INVALID_ARG;
  if (n_cols > INT32_MAX || nnz >= (int64_t{1} << 40)) return SPM_ERR_UNSUPPORTED;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  if (!col_ptr || !d_status) return SPM_ERR_INVALID_ARG;
  if (nnz > 0 && (!out_cols || (out_rows && !row_idx) || (out_vals && !vals))) return SPM_ERR_INVALID_ARG;
  if (nnz > 0 && n_cols == 0) return SPM_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
  k_check_offsets<<<(unsigned)((n_cols + 1 + 255) / 256), 256, 0, st>>>(col_ptr, n_cols, nnz, d_status);
  if (nnz > 0) {
    const unsigned blocks = (unsigned)((nnz + kCooTile - 1) / kCooTile);
    if (dtype == SPM_F64)
      k_to_coo<uint64_t><<<blocks, kCooThreads, 0, st>>>(n_cols, nnz, col_ptr, row_idx,
                                                         static_cast<const uint64_t*>(vals), out_rows, out_cols,
                                                         static_cast<uint64_t*>(out_vals));
    else
      k_to_coo<uint32_t><<<blocks, kCooThreads, 0, st>>>(n_cols, nnz, col_ptr, row_idx,
                                                         static_cast<const uint32_t*>(vals), out_rows, out_cols,
                                                         static_cast<uint32_t*>(out_vals));
  }
  spm::count_launches(nnz > 0 ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? SPM_OK : SPM_ERR_CUDA;
}

}  // extern "C"
