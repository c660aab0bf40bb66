// rowsop.cuh -- scalar sparse operators of the preconditioner apply, in one of two layouts.
//
// SELL-32 (sliced ELL): rows grouped in slices of 32 consecutive rows; slice s holds W_s slots (its
// longest row) and, for slot j, the 32 rows' column and value at col[(B_s + j) * 32 + t],
// val[(B_s + j) * 32 + t] (t = row within the slice; padding: column = the row, value 0).  One thread
// per row walks its slots; a warp reads one contiguous 128-byte line per slot and array (padding:
// column 0, value 0).
// CSR: kept when the slices would pad more than 30 % above the nonzeros (rows of very different
// lengths side by side); the vector-CSR kernel (TPR lanes per row) runs those.
#pragma once
#include "common.cuh"

namespace mgr {

constexpr int RS_C = 32;
constexpr double RS_MAX_PAD = 1.3;

template <class T>
struct RowsOp {
  int64_t nr = 0, nnz = 0;
  bool sell = false;
  // SELL-32
  int64_t slots = 0;
  DBuf<int64_t> soff;
  DBuf<int32_t> scol;
  DBuf<T> sval;
  // CSR
  DCSR<T> csr;
};

// Build from an FP64 CSR matrix, casting the values to T.
template <class T>
void rowsop_build(Ctx& c, const DCSR<double>& A, RowsOp<T>& op);

}  // namespace mgr
