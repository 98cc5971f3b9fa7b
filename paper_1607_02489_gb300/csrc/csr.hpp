// Host compressed-sparse-row matrices for the hierarchy setup.
//
// Products are structural: the pattern of A*B is the union over k of the
// patterns of B's rows selected by A's row, whatever the values, so an entry
// that cancels numerically stays stored as 0.  Rows keep ascending columns.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <vector>

namespace emin {

struct Csr {
  int nrows = 0, ncols = 0;
  std::vector<int64_t> rowptr{0};
  std::vector<int> col;
  std::vector<double> val;

  int64_t nnz() const { return (int64_t)col.size(); }
  int64_t row_begin(int i) const { return rowptr[i]; }
  int64_t row_end(int i) const { return rowptr[i + 1]; }
  void resize_rows(int n, int m) {
    nrows = n;
    ncols = m;
    rowptr.assign(n + 1, 0);
    col.clear();
    val.clear();
  }
};

// Transpose with ascending columns in every output row.
inline Csr transpose(const Csr& A) {
  Csr T;
  T.resize_rows(A.ncols, A.nrows);
  std::vector<int64_t> cnt(A.ncols + 1, 0);
  for (int64_t t = 0; t < A.nnz(); ++t) cnt[A.col[t] + 1]++;
  for (int j = 0; j < A.ncols; ++j) cnt[j + 1] += cnt[j];
  T.rowptr = cnt;
  T.col.resize(A.nnz());
  T.val.resize(A.nnz());
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  for (int i = 0; i < A.nrows; ++i)
    for (int64_t t = A.row_begin(i); t < A.row_end(i); ++t) {
      int64_t q = pos[A.col[t]]++;
      T.col[q] = i;
      T.val[q] = A.val[t];
    }
  return T;
}

// C = A * B, Gustavson order: row i of C accumulates a_ik * B(k, :) for the
// stored k of A's row i in ascending order.
inline Csr spgemm(const Csr& A, const Csr& B) {
  Csr C;
  C.resize_rows(A.nrows, B.ncols);
  std::vector<int> mark(B.ncols, -1);
  std::vector<double> acc(B.ncols, 0.0);
  std::vector<int> cols;
  for (int i = 0; i < A.nrows; ++i) {
    cols.clear();
    for (int64_t t = A.row_begin(i); t < A.row_end(i); ++t) {
      int k = A.col[t];
      double a = A.val[t];
      for (int64_t u = B.row_begin(k); u < B.row_end(k); ++u) {
        int j = B.col[u];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] = acc[j] + a * B.val[u];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int j : cols) {
      C.col.push_back(j);
      C.val.push_back(acc[j]);
    }
    C.rowptr[i + 1] = (int64_t)C.col.size();
  }
  return C;
}

// Block diagonal I_d (x) M.
inline Csr kron_identity(int d, const Csr& M) {
  Csr K;
  K.resize_rows(d * M.nrows, d * M.ncols);
  K.col.reserve(d * M.nnz());
  K.val.reserve(d * M.nnz());
  for (int c = 0; c < d; ++c)
    for (int i = 0; i < M.nrows; ++i) {
      for (int64_t t = M.row_begin(i); t < M.row_end(i); ++t) {
        K.col.push_back(c * M.ncols + M.col[t]);
        K.val.push_back(M.val[t]);
      }
      K.rowptr[c * M.nrows + i + 1] = (int64_t)K.col.size();
    }
  return K;
}

// Value of A(i, j) (0 when not stored); rows sorted.
inline double lookup(const Csr& A, int i, int j) {
  auto b = A.col.begin() + A.row_begin(i), e = A.col.begin() + A.row_end(i);
  auto it = std::lower_bound(b, e, j);
  if (it != e && *it == j) return A.val[it - A.col.begin()];
  return 0.0;
}

}  // namespace emin
