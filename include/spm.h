/*
 * spm.h -- C ABI of the GB300 (sm_103a) sync-step library.
 *
 * The operation is the "sync" of the hybrid sparse matrix class described by
 * Sanderson & Curtin, "A User-Friendly Hybrid Sparse Matrix Class in C++"
 * (LNCS 10931, 2018): element writes collected outside the compressed format
 * (the red-black-tree / coordinate-list side, Sections 3.2-3.4) are turned into
 * canonical Compressed Sparse Column storage (Section 3.1).  Here the writes
 * arrive as an unordered stream of (row, col, value[, seq]) and the library
 * performs, on the GPU, what the paper's in-order tree traversal performs on
 * the CPU: order the elements by the linear index row + col*n_rows (Section
 * 3.3), resolve repeated writes to one element (element setting "X(r,c) = v"
 * or batch insertion with accumulation "X(r,c) += v", Table 1 and Fig. 2),
 * drop elements that are zero (CSC stores non-zero elements only, Section
 * 3.1) and emit values, row indices and column offsets (c[0] = 0,
 * c[n_cols] = N).
 *
 * Conventions for every call:
 *   - All pointers are DEVICE pointers unless the parameter name starts with
 *     h_ (host memory).  The caller allocates and owns every buffer, including
 *     the workspace; the library never allocates, frees or synchronises.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and returns immediately.  spm_assemble_csc,
 *     spm_assemble_csc_batched, spm_csc_transpose, spm_csc_mm and
 *     spm_triplet_dvals can be
 *     captured in a CUDA graph once a first call on the device has returned
 *     (that first call reads device attributes).
 *   - Host-detectable errors (NULL pointers, negative sizes, index spaces that
 *     are too large, a workspace that is too small) return an error status and
 *     launch nothing.  Errors found by the kernels (an index outside the
 *     matrix, a bounded wait that expired) are written to the device int32
 *     *d_status (0 = SPM_OK) and the call itself returns SPM_OK ("launched");
 *     read *d_status after the stream has completed.  When *d_status is not
 *     SPM_OK the CSC output is unspecified, but no memory outside the given
 *     buffers is touched.
 *   - Sizes: n_rows, n_cols < 2^31 (int32 indices), n_rows * n_cols <= 2^52,
 *     total writes per call m < 2^32 - 64.
 */
#ifndef SPM_H_
#define SPM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPM_OK = 0,
  SPM_ERR_INVALID_ARG = 1,
  SPM_ERR_INDEX_OUT_OF_RANGE = 2,
  SPM_ERR_WORKSPACE_TOO_SMALL = 3,
  SPM_ERR_UNSUPPORTED = 4,
  SPM_ERR_CUDA = 5,
  SPM_ERR_TIMEOUT = 6
} spm_status;

/* Duplicate resolution.  LAST_WRITE: element setting, X(r,c) = v (Table 1);
 * the write with the largest (seq, position) wins and its value is copied
 * bit for bit.  SUM: batch insertion with accumulation, X(r,c) += v (Fig. 2);
 * the exact sum of the writes to one element is rounded once to the output
 * type (round-to-nearest-even), so the result does not depend on the order of
 * the writes or on how the work is split (seq has no effect in this mode).
 * The sum is formed in a 128-bit fixed-point integer whose binary point lies
 * 42 bits below the largest exponent among that element's own writes: the
 * result is the correctly rounded exact sum whenever the element's writes
 * span at most 42 binades; bits of a write lying further down are dropped (less
 * than 2^-94 of the element's largest write per write).  One write is its own
 * value.  NaN and infinities follow IEEE addition. */
typedef enum { SPM_MODE_LAST_WRITE = 0, SPM_MODE_SUM = 1 } spm_mode;

/* Value type of the writes and of the CSC values.  SPM_F32 values are
 * accumulated in double precision in SUM mode; indices are never affected. */
typedef enum { SPM_F32 = 0, SPM_F64 = 1 } spm_dtype;

/* flags */
enum {
  SPM_KEEP_MAP = 1,      /* write map[t] for every write t (see below)               */
  SPM_CHECK_BOUNDS = 2,  /* accepted for compatibility: bounds are always checked    */
  SPM_SEQ_EXPLICIT = 4   /* seq != NULL; must be set when sizing the workspace too   */
};

/* Human-readable name of a status code (static string). */
const char* spm_status_string(spm_status s);

/* Version of this library as major*10000 + minor*100 + patch. */
int32_t spm_version(void);

/*
 * spm_assemble_csc_workspace -- bytes of device workspace that
 * spm_assemble_csc needs for these sizes, dtype, mode and flags.
 * Returns SPM_ERR_INVALID_ARG / SPM_ERR_UNSUPPORTED for sizes the call would
 * reject.  The workspace needs no initialisation and may be reused by
 * successive calls on the same stream.  It is dominated by the 16-byte
 * record of every write in bucket order (which later also holds the
 * per-bucket results), plus 20 bytes per write when the two-pass partition
 * runs (the first pass's records and bucket numbers; from 2^22 writes with
 * the default tuning), plus the planner's tables: about 24 bytes per write
 * at 10^6 writes and 37 at 10^8.  It depends on the tuning (spm_set_tuning).
 */
spm_status spm_assemble_csc_workspace(int64_t n_rows, int64_t n_cols, int64_t m, spm_dtype dtype,
                                      spm_mode mode, uint32_t flags, size_t* bytes);

/*
 * spm_assemble_csc -- canonical CSC of the n_rows x n_cols matrix that the m
 * element writes (rows[t], cols[t], vals[t]) produce, Section 3.1 / 3.3.
 *
 *   rows, cols  int32[m]                zero-based indices; any index outside
 *                                       [0,n_rows) x [0,n_cols) sets
 *                                       *d_status = SPM_ERR_INDEX_OUT_OF_RANGE
 *   vals        float[m] or double[m]   per dtype
 *   seq         NULL, or uint64[m]      order of the writes (larger = later;
 *                                       equal seq keeps stream order); requires
 *                                       SPM_SEQ_EXPLICIT in flags
 *   col_ptr     int64[n_cols+1]         output column offsets, col_ptr[0] = 0,
 *                                       col_ptr[n_cols] = nnz
 *   row_idx     int32[m]                output row indices (first nnz used)
 *   out_vals    float[m] or double[m]   output values (first nnz used)
 *   d_nnz       int64[1]                output number of stored elements
 *   map         NULL, or int32[m]       with SPM_KEEP_MAP: the CSC slot that
 *                                       write t feeds; -1 if the write was
 *                                       overwritten (LAST_WRITE mode); -2 if its
 *                                       element is not stored because its value
 *                                       is zero
 *   d_status    int32[1]                device status, see conventions
 *   workspace   ws_bytes bytes          at least spm_assemble_csc_workspace()
 *
 * Output is canonical: rows strictly increase inside each column and no stored
 * value compares equal to zero (so -0.0 is dropped, NaN is kept).  With m = 0
 * the result is an all-zero col_ptr.
 */
spm_status spm_assemble_csc(int64_t n_rows, int64_t n_cols, int64_t m, const int32_t* rows,
                            const int32_t* cols, const void* vals, const uint64_t* seq, spm_dtype dtype,
                            spm_mode mode, uint32_t flags, int64_t* col_ptr, int32_t* row_idx,
                            void* out_vals, int64_t* d_nnz, int32_t* map, int32_t* d_status,
                            void* workspace, size_t ws_bytes, void* stream);

/*
 * spm_assemble_csc_batched_workspace / spm_assemble_csc_batched -- the same
 * sync step for `batch` independent matrices in one call (one sequence of
 * kernels for the whole batch; no host synchronisation, so the call can be
 * captured in a CUDA graph and replayed).
 *
 *   h_n_rows, h_n_cols  host int64[batch]     matrix sizes
 *   h_trip_ptr          host int64[batch+1]   writes of matrix i are
 *                                             [h_trip_ptr[i], h_trip_ptr[i+1])
 *                                             of the concatenated streams;
 *                                             h_trip_ptr[0] = 0
 *   d_n_rows, d_n_cols, d_trip_ptr            device copies of the same arrays
 *                                             (read by the kernels; a mismatch
 *                                             with the host copies is reported
 *                                             as SPM_ERR_INVALID_ARG in *d_status)
 *   rows, cols, vals, seq                     concatenated as for one matrix
 *   col_ptr   int64[sum_i (n_cols_i + 1)]     matrix i's offsets start at
 *                                             sum_{j<i} (n_cols_j + 1); each
 *                                             matrix's offsets start at 0
 *   row_idx, out_vals  [total writes]         matrix i's elements start at
 *                                             h_trip_ptr[i] (capacity m_i)
 *   d_nnz     int64[batch]                    stored elements per matrix
 *   map       NULL or int32[total writes]     as for one matrix (slots are
 *                                             relative to matrix i's start)
 */
spm_status spm_assemble_csc_batched_workspace(int64_t batch, const int64_t* h_n_rows,
                                              const int64_t* h_n_cols, const int64_t* h_trip_ptr,
                                              spm_dtype dtype, spm_mode mode, uint32_t flags,
                                              size_t* bytes);

spm_status spm_assemble_csc_batched(int64_t batch, const int64_t* h_n_rows, const int64_t* h_n_cols,
                                    const int64_t* h_trip_ptr, const int64_t* d_n_rows,
                                    const int64_t* d_n_cols, const int64_t* d_trip_ptr,
                                    const int32_t* rows, const int32_t* cols, const void* vals,
                                    const uint64_t* seq, spm_dtype dtype, spm_mode mode, uint32_t flags,
                                    int64_t* col_ptr, int32_t* row_idx, void* out_vals, int64_t* d_nnz,
                                    int32_t* map, int32_t* d_status, void* workspace, size_t ws_bytes,
                                    void* stream);

/*
 * spm_assemble_csc_static -- the same assembly as spm_assemble_csc, for
 * callers that cannot allocate device memory and so cannot pass a workspace.
 * The paper has no counterpart; this exists for integration only.  Typical
 * such callers: code running inside a host application that owns every
 * device allocation and gives it nothing but its inputs and outputs, or a
 * loop that must not allocate once it has started.
 *
 * Instead of a workspace the call uses a 32 MiB scratch array that is part of
 * this library's device image: every GPU on which the library is loaded
 * holds that array until the process exits.  The call itself allocates
 * nothing.  Sizes whose workspace (spm_assemble_csc_workspace) exceeds
 * 32 MiB -- about 1.4 million writes -- are rejected with
 * SPM_ERR_WORKSPACE_TOO_SMALL before anything is launched.
 *
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All
 * calls on a device share the one array and it keeps whatever the last call
 * left in it; the call clears the parts that must start at zero itself.  Two
 * calls whose kernels overlap on the GPU (different streams without
 * ordering, or different host threads) race on the array and give wrong
 * results: order them on one stream.
 *
 * Arguments, outputs and errors are exactly those of spm_assemble_csc
 * without `workspace` and `ws_bytes`.
 */
spm_status spm_assemble_csc_static(int64_t n_rows, int64_t n_cols, int64_t m, const int32_t* rows,
                                   const int32_t* cols, const void* vals, const uint64_t* seq, spm_dtype dtype,
                                   spm_mode mode, uint32_t flags, int64_t* col_ptr, int32_t* row_idx,
                                   void* out_vals, int64_t* d_nnz, int32_t* map, int32_t* d_status, void* stream);

/*
 * spm_csc_update_workspace / spm_csc_update -- apply m element writes to an
 * existing n_rows x n_cols matrix A held in canonical CSC and return the
 * updated matrix in canonical CSC: the batch insertion of Section 3.1 (the
 * new elements are sorted first, then merged with the existing arrays) and
 * the sync of Section 3.4 after writes made while A was in compressed form.
 *
 * The writes are first resolved among themselves exactly as spm_assemble_csc
 * resolves them (last write by (seq, position), or the sum of the writes to
 * one element formed as in SUM mode: correctly rounded when they span at
 * most 42 binades); then every element written replaces A's
 * element in SPM_MODE_LAST_WRITE (a final write of zero removes it) and is
 * added to it in SPM_MODE_SUM (one rounding of A's value + that sum; an
 * element whose result is zero is removed).  A's other elements are kept.
 *
 *   a_col_ptr  int64[n_cols+1]       A's column offsets: a_col_ptr[0] = 0,
 *                                    non-decreasing, a_col_ptr[n_cols] = nnz_a;
 *                                    otherwise *d_status = SPM_ERR_INVALID_ARG
 *   a_row_idx  int32[nnz_a]          A's rows, strictly increasing inside each
 *                                    column (else SPM_ERR_INVALID_ARG) and in
 *                                    [0, n_rows) (else SPM_ERR_INDEX_OUT_OF_RANGE)
 *   a_vals     (dtype)[nnz_a]        A's values (zeros are allowed and are
 *                                    removed like any other zero)
 *   rows, cols, vals, seq [m]        the writes, as for spm_assemble_csc
 *   col_ptr    int64[n_cols+1]       output column offsets
 *   row_idx, out_vals  [nnz_a + m]   output elements (first *d_nnz used)
 *   d_nnz, d_status                  as for spm_assemble_csc
 *   workspace  at least spm_csc_update_workspace() bytes: the resolved
 *              writes, the merge's cut table and the assembly's workspace
 *
 * The outputs must not overlap A's arrays or the writes.  When *d_status is
 * not SPM_OK the output is unspecified.  SPM_KEEP_MAP is rejected
 * (SPM_ERR_INVALID_ARG).
 */
spm_status spm_csc_update_workspace(int64_t n_rows, int64_t n_cols, int64_t nnz_a, int64_t m, spm_dtype dtype,
                                    spm_mode mode, uint32_t flags, size_t* bytes);

spm_status spm_csc_update(int64_t n_rows, int64_t n_cols, const int64_t* a_col_ptr, const int32_t* a_row_idx,
                          const void* a_vals, int64_t nnz_a, int64_t m, const int32_t* rows, const int32_t* cols,
                          const void* vals, const uint64_t* seq, spm_dtype dtype, spm_mode mode, uint32_t flags,
                          int64_t* col_ptr, int32_t* row_idx, void* out_vals, int64_t* d_nnz, int32_t* d_status,
                          void* workspace, size_t ws_bytes, void* stream);

/*
 * spm_csc_lookup -- values of q elements of a canonical CSC matrix
 * (Section 3.1: one read of the column's start and end, then a binary search
 * among the column's row indices; an element that is not stored reads 0).
 *
 *   col_ptr int64[n_cols+1], row_idx int32[nnz], vals (dtype)[nnz]   the matrix
 *           (rows strictly increasing inside each column; otherwise the
 *           results are unspecified; offsets that are not 0 .. nnz and
 *           non-decreasing set *d_status = SPM_ERR_INVALID_ARG)
 *   q_rows, q_cols  int32[q]   the elements asked for; one outside the matrix
 *                              sets *d_status = SPM_ERR_INDEX_OUT_OF_RANGE and
 *                              reads 0
 *   out_vals  (dtype)[q]       the values (0 where not stored)
 *   out_pos   NULL or int64[q] the element's index in row_idx / vals, or -1
 *   d_status  int32[1]         set to SPM_OK first, see the conventions
 */
spm_status spm_csc_lookup(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* col_ptr, const int32_t* row_idx,
                          const void* vals, spm_dtype dtype, int64_t q, const int32_t* q_rows, const int32_t* q_cols,
                          void* out_vals, int64_t* out_pos, int32_t* d_status, void* stream);

/*
 * spm_csc_to_coo -- the coordinate list (Section 3.2) of a CSC matrix, in
 * the CSC's order: out_cols[e] is the column of stored element e; with
 * out_rows / out_vals not NULL the row indices and values are copied there
 * too (the CSC arrays already hold them, so they may also be used as they
 * are).  The reverse conversion is spm_assemble_csc.
 *
 *   col_ptr int64[n_cols+1]  offsets 0 .. nnz, non-decreasing (otherwise
 *                            *d_status = SPM_ERR_INVALID_ARG and the output
 *                            is unspecified)
 *   row_idx int32[nnz], vals (dtype)[nnz]   read only for the copies
 *   out_rows NULL or int32[nnz], out_cols int32[nnz], out_vals NULL or (dtype)[nnz]
 *   d_status int32[1]        set to SPM_OK first
 */
spm_status spm_csc_to_coo(int64_t n_cols, int64_t nnz, const int64_t* col_ptr, const int32_t* row_idx,
                          const void* vals, spm_dtype dtype, int32_t* out_rows, int32_t* out_cols, void* out_vals,
                          int32_t* d_status, void* stream);

/*
 * spm_csc_trace_atb_workspace / spm_csc_trace_atb -- trace(A^T B) for two
 * canonical n_rows x n_cols CSC matrices, without forming the transpose or
 * the product (Section 2: only the diagonal of A^T B is accumulated; the
 * paper's second timed workload, Fig. 1b).  It equals the sum, over the
 * elements stored in both matrices, of A(i,j) * B(i,j).
 *
 *   a_col_ptr, a_row_idx, a_vals, nnz_a   A (rows strictly increasing inside
 *   b_col_ptr, b_row_idx, b_vals, nnz_b   each column), B likewise; malformed
 *                                         offsets or rows set *d_status =
 *                                         SPM_ERR_INVALID_ARG, a row outside
 *                                         the matrix SPM_ERR_INDEX_OUT_OF_RANGE
 *   dtype       the value type of both
 *   d_result    double[1]  the trace: products and sums in double precision;
 *               the sum is taken in a fixed order for given nnz_a, nnz_b and
 *               structure, so repeated calls give the same bits
 *   d_status    int32[1]   set to SPM_OK first
 *   workspace   at least spm_csc_trace_atb_workspace() bytes (about 40
 *               bytes per 2047 elements of A and B together)
 */
spm_status spm_csc_trace_atb_workspace(int64_t n_cols, int64_t nnz_a, int64_t nnz_b, size_t* bytes);

spm_status spm_csc_trace_atb(int64_t n_rows, int64_t n_cols, const int64_t* a_col_ptr, const int32_t* a_row_idx,
                             const void* a_vals, int64_t nnz_a, const int64_t* b_col_ptr, const int32_t* b_row_idx,
                             const void* b_vals, int64_t nnz_b, spm_dtype dtype, double* d_result, int32_t* d_status,
                             void* workspace, size_t ws_bytes, void* stream);

/*
 * spm_csc_transpose_workspace / spm_csc_transpose -- the CSC of A^T (an
 * n_cols x n_rows matrix; equivalently the row-major CSR of A) from the CSC
 * of A (Section 3.1's compressed column format; Table 1's transpose X.t(),
 * one of the bulk coordinate transformations of Section 3's use case (iii)).
 * Stored element (i, j, v) of A becomes (j, i, v)
 * of A^T; inside each column of A^T the rows (A's columns) increase.  Built
 * by the assembly path: every coordinate occurs once, so each value, an
 * explicit zero included, is carried over bit for bit, and repeated calls
 * give the same bytes.
 *
 *   col_ptr int64[n_cols+1], row_idx int32[nnz], vals (dtype)[nnz]   A
 *                 (offsets 0 .. nnz and non-decreasing, otherwise *d_status
 *                 = SPM_ERR_INVALID_ARG; a row outside [0, n_rows)
 *                 SPM_ERR_INDEX_OUT_OF_RANGE; the output is then unspecified)
 *   t_col_ptr int64[n_rows+1], t_row_idx int32[nnz], t_vals (dtype)[nnz]
 *                 A^T, written; must not overlap the input
 *   d_status int32[1]   set to SPM_OK first
 *   workspace   at least spm_csc_transpose_workspace() bytes (about the
 *               assembly's workspace for nnz writes, plus 4 bytes per element)
 */
spm_status spm_csc_transpose_workspace(int64_t n_rows, int64_t n_cols, int64_t nnz, spm_dtype dtype, size_t* bytes);

spm_status spm_csc_transpose(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* col_ptr,
                             const int32_t* row_idx, const void* vals, spm_dtype dtype, int64_t* t_col_ptr,
                             int32_t* t_row_idx, void* t_vals, int32_t* d_status, void* workspace, size_t ws_bytes,
                             void* stream);

/*
 * spm_csc_mm_workspace / spm_csc_mm -- Y = A X (transpose = 0) or Y = A^T X
 * (transpose = 1) for A in CSC (Section 3.1; the paper's use cases (iv)
 * "multiplication of dense vectors with sparse matrices", Fig. 2
 * "W = V * X").
 *
 *   col_ptr int64[n_cols+1], row_idx int32[nnz], vals (dtype)[nnz]   A
 *   X   (dtype) row-major, (transpose ? n_rows : n_cols) x k, leading dim ldx
 *   Y   (dtype) row-major, (transpose ? n_cols : n_rows) x k, leading dim ldy;
 *       overwritten.  ldx, ldy >= k.  X and Y must not overlap.
 *   d_status  int32[1], set to SPM_OK first; required for transpose = 0,
 *             optional (NULL) for transpose = 1.  A row index outside the
 *             matrix is skipped and reported as SPM_ERR_INDEX_OUT_OF_RANGE;
 *             the offsets must be well formed for transpose = 1 (they are
 *             checked for transpose = 0).
 *   workspace at least spm_csc_mm_workspace() bytes: none for transpose = 1;
 *             for transpose = 0 the CSC of A^T and the transpose's workspace.
 * Every output row is gathered in a fixed order: Y = A^T X walks column c of
 * A in storage order, Y = A X builds A^T (spm_csc_transpose) and walks its
 * columns, i.e. row r of A in increasing column order.  Products and sums are
 * in the value type with fused multiply-adds; repeated calls give the same
 * bits.  (A caller that multiplies by the same A many times can keep A^T from
 * spm_csc_transpose and call transpose = 1 on it.)
 */
spm_status spm_csc_mm_workspace(int64_t n_rows, int64_t n_cols, int64_t nnz, spm_dtype dtype, int32_t transpose,
                                size_t* bytes);

spm_status spm_csc_mm(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* col_ptr, const int32_t* row_idx,
                      const void* vals, spm_dtype dtype, int32_t transpose, int64_t k, const void* X, int64_t ldx,
                      void* Y, int64_t ldy, int32_t* d_status, void* workspace, size_t ws_bytes, void* stream);

/*
 * spm_triplet_dvals -- gradient of a scalar loss L with respect to the value
 * of every write, given dL/dY for Y = A X with A assembled from the writes:
 *     dvals[t] = sum_j dY[rows[t], j] * X[cols[t], j]
 * except dvals[t] = 0 when map != NULL and map[t] == -1 (a write that was
 * overwritten does not influence A).  A coordinate dropped because its value
 * is zero still passes its gradient (A is continuous there).
 *
 *   rows, cols int32[m]; map NULL or int32[m] (from spm_assemble_csc)
 *   dY  (dtype) row-major n_rows x k, leading dim lddy
 *   X   (dtype) row-major n_cols x k, leading dim ldx
 *   dvals (dtype)[m]  output
 */
spm_status spm_triplet_dvals(int64_t m, const int32_t* rows, const int32_t* cols, const int32_t* map,
                             spm_dtype dtype, int64_t k, const void* dY, int64_t lddy, const void* X,
                             int64_t ldx, void* dvals, void* stream);

/*
 * Tuning parameters of the assembly kernels (process-wide; the autotuner
 * sets them).  A call with NULL restores the defaults.  Changing them changes
 * the workspace size, so query the workspace after setting them.
 *   bucket_target        expected writes per bucket the planner aims for
 *                        (256 .. 65536; default 6144); a bucket may hold up
 *                        to twice the target; at most 8192 writes are
 *                        resolved in shared memory -- larger buckets take a
 *                        slower windowed path
 *   sub_bits             log2 of the largest counting-sort digit used inside
 *                        a bucket (8 .. 12; default 12)
 *   partition_threads    threads per block of the histogram/scatter kernels
 *                        (256, 512 or 1024)
 *   resolve_threads      threads per block of the per-bucket kernel (512: the
 *                        kernel's shared-memory layout is built for it)
 *   two_pass_min_writes  calls with at least this many writes move the
 *                        writes to their buckets in two passes -- first to
 *                        about four groups of buckets per SM, then within
 *                        each group -- which keeps the set of partly written
 *                        cache lines small; the workspace then holds 20 more
 *                        bytes per write (>= 0; default 2^22)
 *   two_pass_min_fronts  ... and only when the one-pass scatter would write
 *                        to more than this many (partition block, bucket)
 *                        pairs, counted on the device after the histogram;
 *                        0 with two_pass_min_writes = 0 forces two passes
 *                        (>= 0)
 *   ordered_path         1: a call on one matrix (no map, no seq in
 *                        last-write mode) first tries a single pass that
 *                        works when the writes are already in column-major
 *                        order (the linear indices never decrease); it gives
 *                        up at the first write out of order and the general
 *                        path runs.  0: never tried.  The result is the same
 *                        either way, bit for bit (both sum each run at its
 *                        own binary point)
 */
typedef struct {
  int32_t bucket_target;
  int32_t sub_bits;
  int32_t partition_threads;
  int32_t resolve_threads;
  int32_t two_pass_min_writes;
  int32_t two_pass_min_fronts;
  int32_t ordered_path;
} spm_tuning;

spm_status spm_set_tuning(const spm_tuning* t);
spm_status spm_get_tuning(spm_tuning* t);

/*
 * spm_debug_withhold_publication -- fault injection for tests of the failure
 * path (the paper has no counterpart).  Calls with SPM_KEEP_MAP place each
 * bucket's elements in the resolving block itself, after a bounded wait for
 * the running element count of the buckets before it (a decoupled look-back);
 * calls without the map place them in a later kernel and no block waits for
 * another.  While set to b >= 0, the block that resolves bucket b of a call
 * with the map publishes no count, so the blocks of the following buckets of
 * the same matrix wait until their bounded wait (about 2 s) expires, record
 * SPM_ERR_TIMEOUT in *d_status and stop.  Nothing traps or hangs.  -1 (the
 * default) switches it off.  Process-wide.
 */
spm_status spm_debug_withhold_publication(int64_t bucket);

/*
 * Measurement hooks for benchmarks (the paper has no counterpart).
 *
 * spm_debug_stage_timing(1) makes every later assembly call on the current
 * device record CUDA events, on the call's stream, at the boundaries of its
 * six stages: 0 planning (sampling, lookup tables, bucket descriptors),
 * 1 histogram pass, 2 bucket offsets, 3 partition into bucket records (one
 * or two kernels), 4 per-bucket resolve (the k_resolve kernel alone),
 * 5 placement of the stored elements: the offset scan over the buckets,
 * k_place and k_big (calls without the map; empty otherwise).
 * Events of the last 64 calls are kept.  spm_debug_stage_timing(0) stops
 * recording.  Not capturable in a CUDA graph while enabled.
 *
 * spm_debug_stage_times(back, ms, n): after the stream has completed, writes
 * the durations in milliseconds of the first n (<= 6) stages of the call made
 * `back` calls ago (0 = the latest).
 *
 * spm_debug_launch_count(): number of kernels this library has launched so
 * far in the process (all entry points).
 */
spm_status spm_debug_stage_timing(int32_t enable);

/*
 * spm_debug_plan_stats -- after a single-matrix assembly call has completed,
 * read back from its workspace (synchronous copies) statistics of the bucket
 * plan: stats[0] buckets, [1] largest bucket, [2] buckets above the
 * in-shared-memory capacity, [3] writes in those buckets, [4] capacity,
 * [5] level-2 tables used, [6] planner's bucket bound, [7] 1 if the call was
 * finished by the single pass for writes in column-major order (the plan
 * statistics are then those of a plan that was not made).  Same sizing arguments
 * as spm_assemble_csc_workspace.  A diagnostic; the paper has no counterpart.
 */
spm_status spm_debug_plan_stats(const void* workspace, size_t ws_bytes, int64_t n_rows, int64_t n_cols, int64_t m,
                                spm_dtype dtype, spm_mode mode, uint32_t flags, int64_t* stats, int32_t n_stats);
spm_status spm_debug_stage_times(int32_t back, float* ms, int32_t n);
int64_t spm_debug_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SPM_H_ */
