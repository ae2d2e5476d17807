// libspm: single-matrix assembly for callers that cannot allocate device
// memory.
//
// spm_assemble_csc needs a caller-provided workspace.  Some callers have no
// way to provide one: for example a plugin that runs inside a host
// application which owns every device allocation and hands the plugin only
// its input and output buffers, or a control loop that is not allowed to
// allocate after start-up.  spm_assemble_csc_static serves them by using a
// scratch array that lives in this library's own device image (a file-scope
// __device__ array), so the call itself allocates nothing.
//
// The array is created when the library is loaded on a device and is held by
// that device until the process exits.  Its address is a device address; the
// host-side symbol is only a handle, so the host looks the address up once
// per device with cudaGetSymbolAddress and passes it to the kernels like any
// other workspace pointer.

#include <cstdint>
#include <mutex>

#include "spm_common.cuh"

namespace spm {
namespace {

// 32 MiB of scratch: enough for the workspace of about 1.4 million writes
// (a 16-byte record per write plus the planner's tables; streams that small
// take the one-pass partition, which needs no second copy).
constexpr size_t kStaticScratchBytes = size_t{32} << 20;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mutex;
void* g_static_ptr[64] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
spm_status static_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPM_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return SPM_ERR_CUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return SPM_OK;
}

}  // namespace
}  // namespace spm

extern "C" {

spm_status spm_assemble_csc_static(int64_t n_rows, int64_t n_cols, int64_t m, const int32_t* rows,
                                   const int32_t* cols, const void* vals, const uint64_t* seq, spm_dtype dtype,
                                   spm_mode mode, uint32_t flags, int64_t* col_ptr, int32_t* row_idx,
                                   void* out_vals, int64_t* d_nnz, int32_t* map, int32_t* d_status, void* stream) {
  size_t need = 0;
  spm_status s = spm_assemble_csc_workspace(n_rows, n_cols, m, dtype, mode, flags, &need);
  if (s != SPM_OK) return s;
  if (need > spm::kStaticScratchBytes) return SPM_ERR_WORKSPACE_TOO_SMALL;
  void* scratch = nullptr;
  s = spm::static_scratch(&scratch);
  if (s != SPM_OK) return s;
  return spm_assemble_csc(n_rows, n_cols, m, rows, cols, vals, seq, dtype, mode, flags, col_ptr, row_idx, out_vals,
                          d_nnz, map, d_status, scratch, spm::kStaticScratchBytes, stream);
}

}  // extern "C"
