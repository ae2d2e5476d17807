// Plain CPU oracle for the "sync" step of the hybrid sparse matrix class
// (Sanderson & Curtin, "A User-Friendly Hybrid Sparse Matrix Class in C++").
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file: only the tests, the smoke check and the benchmark's CPU
// baseline leg use it.  It shares no code, header, table or helper with the
// CUDA library.
//
// What it computes, step by step, in the paper's own terms:
//   * Element writes arrive as (row, col, value) with an optional seq; they
//     are applied in (seq, position) order -- the order in which a user would
//     have written X(row,col) = v (set) or X(row,col) += v (add), Table 1 and
//     Fig. 2.
//   * Each write is keyed by the paper's linear index
//         index = row + col * n_rows                      (Section 3.3)
//     and stored in an ordered red-black tree (std::map is one), exactly the
//     RBT representation of Section 3.3: set mode overwrites the node's value,
//     add mode accumulates into it (in double precision).
//   * The tree is traversed in increasing index order, which is column-major
//     order (Section 3.3); each index is decoded with
//         row = index mod n_rows,  col = floor(index / n_rows)
//     and the non-zero elements are appended to the CSC arrays (values,
//     row indices) while a per-column count is kept.  The column offsets are
//     the exclusive prefix sum of those counts, so c[0] = 0 and
//     c[n_cols] = N (Section 3.1).
//
// Readings where the paper is silent (each also listed in the design notes):
//   * CSC holds only non-zero elements (Section 3.1), so a coordinate whose
//     final value compares equal to 0 (IEEE ==, so -0.0 too) is not stored.
//     NaN is not equal to 0 and is kept.
//   * For single-precision output the accumulated double is rounded to float
//     (round-to-nearest-even) first and the zero test is made on the rounded
//     value.
//   * seq, when given, orders the writes; equal seq values keep stream order
//     (a stable ordering), so the later write wins.
//   * In add mode the first write to a coordinate initialises it (there is no
//     "0.0 +" in front), later writes are added left to right in write order.
//
// Parity status: pinned by brute-force dense matrices, invariants, scipy's
// COO->CSC conversion, numpy.lexsort, exact dyadic sums and closed-form FEM
// matrices (tests/test_oracle_pins.py).

#include <algorithm>
#include <cstdint>
#include <map>
#include <numeric>
#include <vector>

namespace {

struct Node {
  double acc;       // current value of the element (set) or running sum (add)
  int64_t winner;   // position of the write whose value is held (set mode)
  int64_t slot;     // position in the CSC arrays after the traversal, or -2
};

}  // namespace

extern "C" {

// Returns 0 on success, 1 for an invalid argument, 2 for an index outside
// [0, n_rows) x [0, n_cols).
//   rows, cols, vals : m writes (vals already widened to double)
//   seq              : NULL, or m sequence numbers
//   sum_mode         : 0 = element set (last write wins), 1 = add (+=)
//   round_to_f32     : 1 rounds the result to float before the zero test
//   col_ptr          : n_cols + 1 entries
//   row_idx, out_vals: capacity m
//   map_out          : NULL, or m entries: CSC slot of write t, -1 if the
//                      write was overwritten, -2 if its coordinate is not
//                      stored because its value is zero
int oracle_assemble_csc(int64_t n_rows, int64_t n_cols, int64_t m,
                        const int64_t* rows, const int64_t* cols,
                        const double* vals, const uint64_t* seq,
                        int sum_mode, int round_to_f32,
                        int64_t* col_ptr, int64_t* row_idx, double* out_vals,
                        int64_t* nnz_out, int64_t* map_out) {
  if (n_rows < 0 || n_cols < 0 || m < 0) return 1;
  if (m > 0 && (rows == nullptr || cols == nullptr || vals == nullptr)) return 1;
  if (col_ptr == nullptr || nnz_out == nullptr) return 1;

  // Write order: by seq when it is given (stable, so ties keep position).
  std::vector<int64_t> order(static_cast<size_t>(m));
  std::iota(order.begin(), order.end(), int64_t{0});
  if (seq != nullptr) {
    std::stable_sort(order.begin(), order.end(),
                     [seq](int64_t a, int64_t b) { return seq[a] < seq[b]; });
  }

  // The red-black tree of (index, value) nodes, Section 3.3.
  std::map<uint64_t, Node> tree;
  const uint64_t nr = static_cast<uint64_t>(n_rows);
  for (int64_t t : order) {
    const int64_t r = rows[t], c = cols[t];
    if (r < 0 || r >= n_rows || c < 0 || c >= n_cols) return 2;
    const uint64_t index = static_cast<uint64_t>(r) + static_cast<uint64_t>(c) * nr;
    auto it = tree.find(index);
    if (it == tree.end()) {
      tree.emplace(index, Node{vals[t], t, -2});
    } else if (sum_mode) {
      it->second.acc += vals[t];
      it->second.winner = t;
    } else {
      it->second.acc = vals[t];
      it->second.winner = t;
    }
  }

  // In-order traversal = column-major order; decode and emit CSC.
  std::vector<int64_t> count(static_cast<size_t>(n_cols), 0);
  int64_t n = 0;
  for (auto& kv : tree) {
    const uint64_t index = kv.first;
    const int64_t r = static_cast<int64_t>(index % nr);
    const int64_t c = static_cast<int64_t>(index / nr);
    double v = kv.second.acc;
    if (round_to_f32) v = static_cast<double>(static_cast<float>(v));
    if (v != 0.0) {
      if (row_idx) row_idx[n] = r;
      if (out_vals) out_vals[n] = v;
      kv.second.slot = n;
      ++count[static_cast<size_t>(c)];
      ++n;
    }
  }
  col_ptr[0] = 0;
  for (int64_t c = 0; c < n_cols; ++c) col_ptr[c + 1] = col_ptr[c] + count[static_cast<size_t>(c)];
  *nnz_out = n;

  if (map_out != nullptr) {
    for (int64_t t = 0; t < m; ++t) {
      const uint64_t index = static_cast<uint64_t>(rows[t]) + static_cast<uint64_t>(cols[t]) * nr;
      const Node& node = tree.at(index);
      if (!sum_mode && node.winner != t) {
        map_out[t] = -1;
      } else {
        map_out[t] = node.slot;
      }
    }
  }
  return 0;
}

// Y = A * X (transpose = 0; Y is n_rows x k) or Y = A^T * X (transpose = 1;
// Y is n_cols x k), A given in CSC (Section 3.1), X and Y row-major with
// leading dimensions ldx, ldy.  Plain loops over the stored elements of each
// column in storage order, accumulating in double.
int oracle_csc_mm(int64_t n_rows, int64_t n_cols, const int64_t* col_ptr,
                  const int64_t* row_idx, const double* vals, int transpose,
                  int64_t k, const double* X, int64_t ldx, double* Y, int64_t ldy) {
  if (n_rows < 0 || n_cols < 0 || k < 0) return 1;
  const int64_t out_rows = transpose ? n_cols : n_rows;
  for (int64_t i = 0; i < out_rows; ++i)
    for (int64_t j = 0; j < k; ++j) Y[i * ldy + j] = 0.0;
  for (int64_t c = 0; c < n_cols; ++c) {
    for (int64_t p = col_ptr[c]; p < col_ptr[c + 1]; ++p) {
      const int64_t r = row_idx[p];
      const double a = vals[p];
      if (!transpose) {
        for (int64_t j = 0; j < k; ++j) Y[r * ldy + j] += a * X[c * ldx + j];
      } else {
        for (int64_t j = 0; j < k; ++j) Y[c * ldy + j] += a * X[r * ldx + j];
      }
    }
  }
  return 0;
}

// Gradient of <dY, A X> with respect to the value of each write t:
// dvals[t] = sum_j dY[rows[t], j] * X[cols[t], j], or 0 when map[t] == -1
// (an overwritten write has no influence on A).  map may be NULL (add mode:
// every write contributes to its coordinate).
int oracle_dvals(int64_t m, const int64_t* rows, const int64_t* cols,
                 const int64_t* map, int64_t k, const double* dY, int64_t lddy,
                 const double* X, int64_t ldx, double* dvals) {
  for (int64_t t = 0; t < m; ++t) {
    if (map != nullptr && map[t] == -1) {
      dvals[t] = 0.0;
      continue;
    }
    double s = 0.0;
    for (int64_t j = 0; j < k; ++j) s += dY[rows[t] * lddy + j] * X[cols[t] * ldx + j];
    dvals[t] = s;
  }
  return 0;
}

}  // extern "C"
