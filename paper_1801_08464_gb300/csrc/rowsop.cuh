// rowsop.cuh -- scalar sparse operators of the preconditioner apply, in one of two layouts.
//
// SELL-8 (sliced ELL): rows grouped in slices of 8 consecutive rows; slice s holds W_s slots (its
// longest row) and, for slot j, the 8 rows' column and value at col[(B_s + j) * 8 + t],
// val[(B_s + j) * 8 + t] (t = row within the slice; padding: column 0, value 0).  One thread per row
// walks its slots; each slot of a slice is one full 32-byte sector per array and a slice's slots are
// contiguous, so a warp streams 4 slices sector by sector.  Slices of 8 rather than 32 keep the
// padding of the pressure-level operators (rows of 25 to 63 entries side by side) near 10 %.
// CSR: kept when the slices would pad more than 30 % above the nonzeros (rows of very different
// lengths side by side); the vector-CSR kernel (TPR lanes per row) runs those.
#pragma once
#include "common.cuh"

namespace mgr {

constexpr int RS_C = 8;
constexpr double RS_MAX_PAD = 1.3;

template <class T>
struct RowsOp {
  int64_t nr = 0, nnz = 0;
  bool sell = false;
  // SELL-8
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
