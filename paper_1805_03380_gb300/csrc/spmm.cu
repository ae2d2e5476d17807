// libspm: products with an assembled CSC matrix and the gradient of the
// write values, for the differentiable assemble-then-multiply pattern.
//
//   spm_csc_mm         Y = A X or Y = A^T X with A in CSC (Section 3.1; the
//                      paper's use case (iv), dense times sparse)
//   spm_triplet_dvals  dL/dvals[t] = <dY[rows[t], :], X[cols[t], :]>
//
// Both are bandwidth-bound gathers: a group of k threads (one per column of
// X) walks the stored elements of one CSC column, so that the row of X or dY
// it touches is read as one contiguous k-element segment.

#include <cstdint>

#include "spm_common.cuh"

namespace spm {
void count_launches(int64_t n);
namespace {

// Y = A^T X: output row c gathers the stored elements of column c in storage
// order (deterministic).
template <typename T>
__global__ void k_mm_transposed(int64_t n_cols, const int64_t* __restrict__ col_ptr,
                                const int32_t* __restrict__ row_idx, const T* __restrict__ vals, int64_t k,
                                const T* __restrict__ X, int64_t ldx, T* __restrict__ Y, int64_t ldy) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = g / k, j = g - (g / k) * k;
  if (c >= n_cols) return;
  T acc = T(0);
  const int64_t p1 = col_ptr[c + 1];
  for (int64_t p = col_ptr[c]; p < p1; ++p) acc += vals[p] * X[(int64_t)row_idx[p] * ldx + j];
  Y[c * ldy + j] = acc;
}

template <typename T>
__global__ void k_zero_rows(int64_t n, int64_t k, T* __restrict__ Y, int64_t ldy) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n * k) return;
  const int64_t r = g / k, j = g - r * k;
  Y[r * ldy + j] = T(0);
}

// Y = A X: column c scatters vals * X[c, :] into the rows it holds (atomic adds).
template <typename T>
__global__ void k_mm_scatter(int64_t n_cols, const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                             const T* __restrict__ vals, int64_t k, const T* __restrict__ X, int64_t ldx,
                             T* __restrict__ Y, int64_t ldy) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = g / k, j = g - (g / k) * k;
  if (c >= n_cols) return;
  const T xc = X[c * ldx + j];
  const int64_t p1 = col_ptr[c + 1];
  for (int64_t p = col_ptr[c]; p < p1; ++p) atomicAdd(&Y[(int64_t)row_idx[p] * ldy + j], vals[p] * xc);
}

// dvals[t] = sum_j dY[rows[t], j] * X[cols[t], j]; 0 for overwritten writes.
template <typename T>
__global__ void k_dvals(int64_t m, const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                        const int32_t* __restrict__ map, int64_t k, const T* __restrict__ dY, int64_t lddy,
                        const T* __restrict__ X, int64_t ldx, T* __restrict__ dvals) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  if (map && map[t] == -1) {
    dvals[t] = T(0);
    return;
  }
  const T* a = dY + (int64_t)rows[t] * lddy;
  const T* b = X + (int64_t)cols[t] * ldx;
  T s = T(0);
  for (int64_t j = 0; j < k; ++j) s += a[j] * b[j];
  dvals[t] = s;
}

// Same for k = 16 single precision with 128-bit loads (rows 64 bytes apart).
__global__ void k_dvals_f32_k16(int64_t m, const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                                const int32_t* __restrict__ map, const float* __restrict__ dY, int64_t lddy,
                                const float* __restrict__ X, int64_t ldx, float* __restrict__ dvals) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  if (map && map[t] == -1) {
    dvals[t] = 0.0f;
    return;
  }
  const float4* a = reinterpret_cast<const float4*>(dY + (int64_t)rows[t] * lddy);
  const float4* b = reinterpret_cast<const float4*>(X + (int64_t)cols[t] * ldx);
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 x = a[q], y = b[q];
    s += x.x * y.x;
    s += x.y * y.y;
    s += x.z * y.z;
    s += x.w * y.w;
  }
  dvals[t] = s;
}

}  // namespace
}  // namespace spm

using namespace spm;

extern "C" {

spm_status spm_csc_mm(int64_t n_rows, int64_t n_cols, const int64_t* col_ptr, const int32_t* row_idx,
                      const void* vals, spm_dtype dtype, int32_t transpose, int64_t k, const void* X, int64_t ldx,
                      void* Y, int64_t ldy, void* stream) {
  if (n_rows < 0 || n_cols < 0 || k < 0 || ldx < k || ldy < k) return SPM_ERR_INVALID_ARG;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  if (transpose != 0 && transpose != 1) return SPM_ERR_INVALID_ARG;
  const int64_t out_rows = transpose ? n_cols : n_rows;
  if (k == 0 || out_rows == 0) return SPM_OK;
  if (!col_ptr || !Y || (!X && n_cols > 0) || ((!row_idx || !vals) && n_cols > 0)) return SPM_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int threads = 256;
  const int64_t work = n_cols * k;
  const unsigned grid = (unsigned)((work + threads - 1) / threads);
  count_launches(transpose ? 1 : 2);
  if (dtype == SPM_F32) {
    const float* v = static_cast<const float*>(vals);
    const float* x = static_cast<const float*>(X);
    float* y = static_cast<float*>(Y);
    if (transpose) {
      if (work > 0) k_mm_transposed<float><<<grid, threads, 0, st>>>(n_cols, col_ptr, row_idx, v, k, x, ldx, y, ldy);
    } else {
      k_zero_rows<float><<<(unsigned)((n_rows * k + threads - 1) / threads), threads, 0, st>>>(n_rows, k, y, ldy);
      if (work > 0) k_mm_scatter<float><<<grid, threads, 0, st>>>(n_cols, col_ptr, row_idx, v, k, x, ldx, y, ldy);
    }
  } else {
    const double* v = static_cast<const double*>(vals);
    const double* x = static_cast<const double*>(X);
    double* y = static_cast<double*>(Y);
    if (transpose) {
      if (work > 0) k_mm_transposed<double><<<grid, threads, 0, st>>>(n_cols, col_ptr, row_idx, v, k, x, ldx, y, ldy);
    } else {
      k_zero_rows<double><<<(unsigned)((n_rows * k + threads - 1) / threads), threads, 0, st>>>(n_rows, k, y, ldy);
      if (work > 0) k_mm_scatter<double><<<grid, threads, 0, st>>>(n_cols, col_ptr, row_idx, v, k, x, ldx, y, ldy);
    }
  }
  return cudaGetLastError() == cudaSuccess ? SPM_OK : SPM_ERR_CUDA;
}

spm_status spm_triplet_dvals(int64_t m, const int32_t* rows, const int32_t* cols, const int32_t* map,
                             spm_dtype dtype, int64_t k, const void* dY, int64_t lddy, const void* X, int64_t ldx,
                             void* dvals, void* stream) {
  if (m < 0 || k < 0 || lddy < k || ldx < k) return SPM_ERR_INVALID_ARG;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  if (m == 0) return SPM_OK;
  if (!rows || !cols || !dvals || (k > 0 && (!dY || !X))) return SPM_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int threads = 256;
  const unsigned grid = (unsigned)((m + threads - 1) / threads);
  count_launches(1);
  if (dtype == SPM_F32) {
    const bool fast = k == 16 && (lddy % 4) == 0 && (ldx % 4) == 0 &&
                      ((reinterpret_cast<uintptr_t>(dY) | reinterpret_cast<uintptr_t>(X)) & 15u) == 0;
    if (fast)
      k_dvals_f32_k16<<<grid, threads, 0, st>>>(m, rows, cols, map, static_cast<const float*>(dY), lddy,
                                                static_cast<const float*>(X), ldx, static_cast<float*>(dvals));
    else
      k_dvals<float><<<grid, threads, 0, st>>>(m, rows, cols, map, k, static_cast<const float*>(dY), lddy,
                                               static_cast<const float*>(X), ldx, static_cast<float*>(dvals));
  } else {
    k_dvals<double><<<grid, threads, 0, st>>>(m, rows, cols, map, k, static_cast<const double*>(dY), lddy,
                                              static_cast<const double*>(X), ldx, static_cast<double*>(dvals));
  }
  return cudaGetLastError() == cudaSuccess ? SPM_OK : SPM_ERR_CUDA;
}

}  // extern "C"
