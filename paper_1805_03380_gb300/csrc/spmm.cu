// libspm: products with an assembled CSC matrix, its transpose, and the
// gradient of the write values, for the differentiable
// assemble-then-multiply pattern.
//
//   spm_csc_transpose  CSC of A^T (= CSR of A) from the CSC of A
//   spm_csc_mm         Y = A X or Y = A^T X with A in CSC (Section 3.1; the
//                      paper's use case (iv), dense times sparse)
//   spm_triplet_dvals  dL/dvals[t] = <dY[rows[t], :], X[cols[t], :]>
//
// Every product is a gather: a group of threads (each with 1, 2 or 4
// consecutive columns of X, one vector load) walks the stored elements of
// one column of the matrix it multiplies by in storage order and writes one
// output row, so the sums are taken in a fixed order and repeated calls give
// the same bits.  Y = A^T X gathers over A's own columns.  Y = A X gathers
// over the columns of A^T: the transpose is built in the workspace by the
// assembly path itself (the coordinate list of A with rows and columns
// exchanged, last-write mode with explicit zeros kept: every coordinate
// occurs once, so each value is carried over unchanged).

#include <algorithm>
#include <cstdint>

#include "spm.h"
#include "spm_common.cuh"

namespace spm {
void count_launches(int64_t n);
namespace {

template <typename T, int VW>
struct Vec;
template <>
struct Vec<float, 1> { using type = float; };
template <>
struct Vec<float, 2> { using type = float2; };
template <>
struct Vec<float, 4> { using type = float4; };
template <>
struct Vec<double, 1> { using type = double; };
template <>
struct Vec<double, 2> { using type = double2; };

template <typename V, typename T>
__device__ __forceinline__ void fma_vec(V& acc, T a, const V& x);
template <>
__device__ __forceinline__ void fma_vec<float, float>(float& acc, float a, const float& x) { acc = fmaf(a, x, acc); }
template <>
__device__ __forceinline__ void fma_vec<float2, float>(float2& acc, float a, const float2& x) {
  acc.x = fmaf(a, x.x, acc.x);
  acc.y = fmaf(a, x.y, acc.y);
}
template <>
__device__ __forceinline__ void fma_vec<float4, float>(float4& acc, float a, const float4& x) {
  acc.x = fmaf(a, x.x, acc.x);
  acc.y = fmaf(a, x.y, acc.y);
  acc.z = fmaf(a, x.z, acc.z);
  acc.w = fmaf(a, x.w, acc.w);
}
template <>
__device__ __forceinline__ void fma_vec<double, double>(double& acc, double a, const double& x) {
  acc = fma(a, x, acc);
}
template <>
__device__ __forceinline__ void fma_vec<double2, double>(double2& acc, double a, const double2& x) {
  acc.x = fma(a, x.x, acc.x);
  acc.y = fma(a, x.y, acc.y);
}

// Y[c, :] = sum over the stored elements p of column c (storage order) of
// vals[p] * X[row_idx[p], :].  G = k / VW threads per output row, thread j
// owns columns [j*VW, j*VW + VW) of X and Y.  Two elements are loaded ahead
// of their multiply-adds (independent loads in flight); the sum order is the
// storage order whatever the unrolling.  A row index outside [0, n_in) is
// skipped (X is not read there) and reported in *status when given; offsets
// are clamped to [0, nnz], so a malformed matrix reads no memory outside its
// arrays.  With *status already not SPM_OK on entry (a failed transpose
// before it) the kernel writes zeros and reads nothing else.
template <typename T, int VW>
__global__ void __launch_bounds__(256) k_mm_gather(int64_t n_out, int64_t n_in, int64_t nnz,
                                                   const int64_t* __restrict__ col_ptr,
                                                   const int32_t* __restrict__ row_idx, const T* __restrict__ vals,
                                                   int64_t G, const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                                   int64_t ldy, int32_t* status) {
  using V = typename Vec<T, VW>::type;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = g / G, j = g - c * G;
  if (c >= n_out) return;
  V acc;
  T* a = reinterpret_cast<T*>(&acc);
#pragma unroll
  for (int q = 0; q < VW; ++q) a[q] = T(0);
  const bool failed = status && *reinterpret_cast<volatile int32_t*>(status) != 0;
  int64_t p = failed ? 0 : min(max(col_ptr[c], int64_t{0}), nnz);
  const int64_t p1 = failed ? 0 : min(max(col_ptr[c + 1], p), nnz);
  const T* xb = X + j * VW;
  bool bad = false;
  for (; p + 2 <= p1; p += 2) {
    const int32_t r0 = row_idx[p], r1 = row_idx[p + 1];
    const T v0 = vals[p], v1 = vals[p + 1];
    const bool ok0 = (uint32_t)r0 < (uint64_t)n_in, ok1 = (uint32_t)r1 < (uint64_t)n_in;
    bad |= !(ok0 && ok1);
    const V x0 = *reinterpret_cast<const V*>(xb + (int64_t)(ok0 ? r0 : 0) * ldx);
    const V x1 = *reinterpret_cast<const V*>(xb + (int64_t)(ok1 ? r1 : 0) * ldx);
    if (ok0) fma_vec(acc, v0, x0);
    if (ok1) fma_vec(acc, v1, x1);
  }
  if (p < p1) {
    const int32_t r0 = row_idx[p];
    if ((uint32_t)r0 < (uint64_t)n_in) fma_vec(acc, vals[p], *reinterpret_cast<const V*>(xb + (int64_t)r0 * ldx));
    else bad = true;
  }
  *reinterpret_cast<V*>(Y + c * ldy + j * VW) = acc;
  if (bad && status) atomicCAS(status, 0, (int32_t)SPM_ERR_INDEX_OUT_OF_RANGE);
}

template <typename T>
cudaError_t launch_gather(int64_t n_out, int64_t n_in, int64_t nnz, const int64_t* col_ptr, const int32_t* row_idx,
                          const T* vals, int64_t k, const T* X, int64_t ldx, T* Y, int64_t ldy, int32_t* status,
                          cudaStream_t st) {
  const uintptr_t al = reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y);
  const int vmax = sizeof(T) == 4 ? 4 : 2;
  int vw = 1;
  for (int w = vmax; w > 1; w >>= 1) {
    if (k % w == 0 && ldx % w == 0 && ldy % w == 0 && (al % (w * sizeof(T))) == 0) {
      vw = w;
      break;
    }
  }
  const int64_t G = k / vw;
  const int64_t work = n_out * G;
  if (work == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((work + 255) / 256);
  if constexpr (sizeof(T) == 4) {
    if (vw == 4) k_mm_gather<T, 4><<<grid, 256, 0, st>>>(n_out, n_in, nnz, col_ptr, row_idx, vals, G, X, ldx, Y, ldy, status);
    else if (vw == 2) k_mm_gather<T, 2><<<grid, 256, 0, st>>>(n_out, n_in, nnz, col_ptr, row_idx, vals, G, X, ldx, Y, ldy, status);
    else k_mm_gather<T, 1><<<grid, 256, 0, st>>>(n_out, n_in, nnz, col_ptr, row_idx, vals, G, X, ldx, Y, ldy, status);
  } else {
    if (vw == 2) k_mm_gather<T, 2><<<grid, 256, 0, st>>>(n_out, n_in, nnz, col_ptr, row_idx, vals, G, X, ldx, Y, ldy, status);
    else k_mm_gather<T, 1><<<grid, 256, 0, st>>>(n_out, n_in, nnz, col_ptr, row_idx, vals, G, X, ldx, Y, ldy, status);
  }
  count_launches(1);
  return cudaGetLastError();
}

// A status found by an earlier step (in the workspace) passed on to the
// caller's status word, which the assembly reset.
__global__ void k_pass_status(const int32_t* __restrict__ from, int32_t* to) {
  const int32_t s = *from;
  if (s != 0) atomicCAS(to, 0, s);
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

constexpr size_t kAl = 256;
size_t al_up(size_t x) { return (x + kAl - 1) & ~(kAl - 1); }

// Workspace of spm_csc_transpose: the expanded column indices, two status /
// count words, then the assembly's own workspace.
struct TransposeLayout {
  size_t cols, scal, asm_ws, total, asm_bytes;
};

spm_status transpose_layout(int64_t n_rows, int64_t n_cols, int64_t nnz, spm_dtype dtype, TransposeLayout& L) {
  if (n_rows < 0 || n_cols < 0 || nnz < 0) return SPM_ERR_INVALID_ARG;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  size_t ab = 0;
  const spm_status s = spm_assemble_csc_workspace(n_cols, n_rows, nnz, dtype, SPM_MODE_LAST_WRITE, 0, &ab);
  if (s != SPM_OK) return s;
  L.cols = 0;
  L.scal = al_up((size_t)nnz * 4);
  L.asm_ws = L.scal + kAl;
  L.asm_bytes = ab;
  L.total = L.asm_ws + ab;
  return SPM_OK;
}

spm_status transpose_into(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* col_ptr,
                          const int32_t* row_idx, const void* vals, spm_dtype dtype, int64_t* t_col_ptr,
                          int32_t* t_row_idx, void* t_vals, int32_t* d_status, char* ws, const TransposeLayout& L,
                          cudaStream_t st) {
  int32_t* cexp = reinterpret_cast<int32_t*>(ws + L.cols);
  int32_t* st_coo = reinterpret_cast<int32_t*>(ws + L.scal);
  int64_t* d_nnz_t = reinterpret_cast<int64_t*>(ws + L.scal + 8);
  // the column of every stored element (checks the offsets)
  spm_status s = spm_csc_to_coo(n_cols, nnz, col_ptr, row_idx, vals, dtype, nullptr, nnz > 0 ? cexp : nullptr,
                                nullptr, st_coo, st);
  if (s != SPM_OK) return s;
  // A^T: (column, row) pairs as (row, column) writes; every coordinate once
  s = assemble_internal(n_cols, n_rows, nnz, cexp, row_idx, vals, nullptr, dtype, SPM_MODE_LAST_WRITE,
                        kFlagKeepZeros, t_col_ptr, t_row_idx, t_vals, d_nnz_t, d_status, ws + L.asm_ws, L.asm_bytes,
                        st);
  if (s != SPM_OK) return s;
  k_pass_status<<<1, 1, 0, st>>>(st_coo, d_status);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? SPM_OK : SPM_ERR_CUDA;
}

// Workspace of spm_csc_mm: nothing for A^T X; for A X the CSC of A^T and
// the transpose's workspace.
struct MmLayout {
  size_t t_cp, t_ri, t_v, tr, total;
  TransposeLayout T;
};

spm_status mm_layout(int64_t n_rows, int64_t n_cols, int64_t nnz, spm_dtype dtype, int32_t transpose, MmLayout& L) {
  L = MmLayout{};
  if (transpose) return SPM_OK;
  const spm_status s = transpose_layout(n_rows, n_cols, nnz, dtype, L.T);
  if (s != SPM_OK) return s;
  const size_t sv = dtype == SPM_F64 ? 8 : 4;
  L.t_cp = 0;
  L.t_ri = al_up(8 * (size_t)(n_rows + 1));
  L.t_v = L.t_ri + al_up(4 * (size_t)std::max<int64_t>(nnz, 1));
  L.tr = L.t_v + al_up(sv * (size_t)std::max<int64_t>(nnz, 1));
  L.total = L.tr + L.T.total;
  return SPM_OK;
}

}  // namespace
}  // namespace spm

using namespace spm;

extern "C" {

spm_status spm_csc_transpose_workspace(int64_t n_rows, int64_t n_cols, int64_t nnz, spm_dtype dtype, size_t* bytes) {
  if (!bytes) return SPM_ERR_INVALID_ARG;
  TransposeLayout L;
  const spm_status s = transpose_layout(n_rows, n_cols, nnz, dtype, L);
  if (s != SPM_OK) return s;
  *bytes = L.total;
  return SPM_OK;
}

spm_status spm_csc_transpose(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* col_ptr,
                             const int32_t* row_idx, const void* vals, spm_dtype dtype, int64_t* t_col_ptr,
                             int32_t* t_row_idx, void* t_vals, int32_t* d_status, void* workspace, size_t ws_bytes,
                             void* stream) {
  TransposeLayout L;
  const spm_status s = transpose_layout(n_rows, n_cols, nnz, dtype, L);
  if (s != SPM_OK) return s;
  if (!col_ptr || !t_col_ptr || !d_status) return SPM_ERR_INVALID_ARG;
  if (nnz > 0 && (!row_idx || !vals || !t_row_idx || !t_vals)) return SPM_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < L.total) return SPM_ERR_WORKSPACE_TOO_SMALL;
  return transpose_into(n_rows, n_cols, nnz, col_ptr, row_idx, vals, dtype, t_col_ptr, t_row_idx, t_vals, d_status,
                        static_cast<char*>(workspace), L, reinterpret_cast<cudaStream_t>(stream));
}

spm_status spm_csc_mm_workspace(int64_t n_rows, int64_t n_cols, int64_t nnz, spm_dtype dtype, int32_t transpose,
                                size_t* bytes) {
  if (!bytes || (transpose != 0 && transpose != 1)) return SPM_ERR_INVALID_ARG;
  if (n_rows < 0 || n_cols < 0 || nnz < 0 || (dtype != SPM_F32 && dtype != SPM_F64)) return SPM_ERR_INVALID_ARG;
  MmLayout L;
  const spm_status s = mm_layout(n_rows, n_cols, nnz, dtype, transpose, L);
  if (s != SPM_OK) return s;
  *bytes = L.total;
  return SPM_OK;
}

spm_status spm_csc_mm(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* col_ptr, const int32_t* row_idx,
                      const void* vals, spm_dtype dtype, int32_t transpose, int64_t k, const void* X, int64_t ldx,
                      void* Y, int64_t ldy, int32_t* d_status, void* workspace, size_t ws_bytes, void* stream) {
  if (n_rows < 0 || n_cols < 0 || nnz < 0 || k < 0 || ldx < k || ldy < k) return SPM_ERR_INVALID_ARG;
  if (dtype != SPM_F32 && dtype != SPM_F64) return SPM_ERR_INVALID_ARG;
  if (transpose != 0 && transpose != 1) return SPM_ERR_INVALID_ARG;
  MmLayout L;
  spm_status s = mm_layout(n_rows, n_cols, nnz, dtype, transpose, L);
  if (s != SPM_OK) return s;
  const int64_t out_rows = transpose ? n_cols : n_rows;
  if (k == 0 || out_rows == 0) return SPM_OK;
  if (!col_ptr || !Y || (!X && nnz > 0) || ((!row_idx || !vals) && nnz > 0)) return SPM_ERR_INVALID_ARG;
  if (!transpose && !d_status) return SPM_ERR_INVALID_ARG;
  if (L.total > 0 && (!workspace || ws_bytes < L.total)) return SPM_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t* cp = col_ptr;
  const int32_t* ri = row_idx;
  const void* v = vals;
  if (transpose && d_status) cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
  if (!transpose) {
    char* ws = static_cast<char*>(workspace);
    int64_t* t_cp = reinterpret_cast<int64_t*>(ws + L.t_cp);
    int32_t* t_ri = reinterpret_cast<int32_t*>(ws + L.t_ri);
    void* t_v = ws + L.t_v;
    s = transpose_into(n_rows, n_cols, nnz, col_ptr, row_idx, vals, dtype, t_cp, t_ri, t_v, d_status, ws + L.tr, L.T,
                       st);
    if (s != SPM_OK) return s;
    cp = t_cp;
    ri = t_ri;
    v = t_v;
  }
  // X has n_rows rows for A^T X and n_cols rows for A X
  const int64_t in_rows = transpose ? n_rows : n_cols;
  cudaError_t e;
  if (dtype == SPM_F32)
    e = launch_gather<float>(out_rows, in_rows, nnz, cp, ri, static_cast<const float*>(v), k, static_cast<const float*>(X),
                             ldx, static_cast<float*>(Y), ldy, d_status, st);
  else
    e = launch_gather<double>(out_rows, in_rows, nnz, cp, ri, static_cast<const double*>(v), k,
                              static_cast<const double*>(X), ldx, static_cast<double*>(Y), ldy, d_status, st);
  return e == cudaSuccess ? SPM_OK : SPM_ERR_CUDA;
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
