// rowsop.cuh -- scalar sparse operators of the preconditioner apply, in one of two layouts.
//
// SELL-8 (sliced ELL) with slots in groups of q (4, or 1 for operators with short rows): rows are
// grouped in slices of 8 consecutive rows; slice s holds W_s slots (its longest row, rounded up to a
// multiple of q) starting at slot B_s (a multiple of q).  Slot j of row t (t = row within the slice)
// is stored at
//   (B_s * 8) + (j / q) * 8q + t * q + (j % q)
// in col[] and val[] (padding: column 0, value 0).  With q = 4 one thread per row reads its slots
// four at a time as one 16-byte load of columns and one 16-byte (FP32) or two 16-byte (FP64) loads
// of values, and the 8 rows of a slice read one contiguous 128-byte line per group: few, wide, fully
// used loads, which keep more bytes in flight per thread than one 4-byte load per slot.  Rows of a
// few entries (transfers, restrictions: 1 to 7 entries) keep q = 1, which pads nothing once the
// rows are ordered by length.  Slices of 8 rather
// than 32 keep the padding of the pressure-level operators (rows of 25 to 63 entries side by side)
// near 10 %.
// Sorted slices: when rows of very different lengths sit side by side (AMG operators and transfers,
// the coarse-level couplings), the rows are first ordered by decreasing length within windows of
// RS_SIGMA consecutive rows (stable), so a slice holds rows of similar length; perm[r] is then the
// operator row stored at slice position r.  Windows keep the rows of a slice close together, so
// their x gathers and outputs stay local.
// Compressed columns: a square operator whose entries use at most 255 distinct offsets col - row is
// stored with one-byte codes into a table of those offsets.  The codes are laid out in groups of 16
// slots (slice widths rounded up to 16, padding code 255): slot j of row t of slice s at
// CB_s * 8 + (j / 16) * 128 + t * 16 + j % 16, so one thread reads the codes of four 4-slot groups as
// one 16-byte load (CB_s: the rounded widths of the slices before s).  Otherwise, when every slice of an
// operator with 4-slot groups spans fewer than 65,536
// columns (the stencil-like operators of this path: a slice holds 8 consecutive rows, or rows of one
// 256-row window), the columns are stored as 16-bit offsets from the slice's smallest column
// (padding slots point at that column with value 0).
// CSR: kept for operators with fewer than RS_MIN_ROWS rows, and when even the sorted slices would pad
// more than 30 % above the nonzeros; the vector-CSR kernel (TPR lanes per row) runs those.
#pragma once
#include "common.cuh"

namespace mgr {

constexpr int RS_C = 8;
constexpr int RS_Q = 4;  // slots per group for operators with long rows
constexpr double RS_QUAD_MIN_AVG = 8.0;  // average row length from which the 4-slot groups pay
constexpr double RS_MAX_PAD = 1.3;
constexpr double RS_SORT_PAD = 1.1;  // above this padding the rows are ordered by length
constexpr int RS_SIGMA = 256;
// one thread per row needs rows to fill the GPU (152 SMs x 2048 threads); smaller operators keep CSR
// and the vector kernel, which puts up to 32 lanes on each row
constexpr int64_t RS_MIN_ROWS = 256 * 1024;

template <class T>
struct RowsOp {
  int64_t nr = 0, nc = 0, nnz = 0;
  bool sell = false;
  // SELL-8 with 4-slot groups
  int64_t slots = 0;
  int q = RS_Q;        // slots per group: RS_Q, or 1 for short rows (where groups of 4 would pad)
  DBuf<int64_t> soff;
  DBuf<int32_t> perm;  // empty when rows keep their order
  DBuf<int32_t> scol;
  DBuf<T> sval;
  // 4-slot groups whose slices span at most 65,536 columns keep 16-bit column offsets from a per-slice
  // base instead of scol (6 bytes per FP32 entry instead of 8)
  bool c16 = false;
  DBuf<uint16_t> scol16;
  DBuf<int32_t> sbase;
  // square operators with 4-slot groups whose entries use at most 255 distinct offsets col - row (the
  // stencil-like operators of the structured levels) keep one byte per entry: a code into the table
  // of those offsets (code 255, offset 0, marks padding); 5 bytes per FP32 entry instead of 8
  bool c8 = false;
  DBuf<uint8_t> scode;
  DBuf<int64_t> coff;  // code slice offsets CB_s (slots)
  DBuf<int32_t> otab;  // 256 offsets
  // CSR
  DCSR<T> csr;
};

// Position of slot j of row t within a slice in the one-byte code layout.
__host__ __device__ __forceinline__ int64_t rs_code_pos(int64_t j, int t) {
  return (j / 16) * 128 + (int64_t)t * 16 + (j % 16);
}

// Hands every buffer of op over to the context c: later releases are ordered on c's stream.
template <class T>
void rowsop_rehome(RowsOp<T>& op, Ctx& c) {
  op.soff.c = &c; op.perm.c = &c; op.scol.c = &c; op.sval.c = &c; op.scol16.c = &c; op.sbase.c = &c;
  op.scode.c = &c; op.coff.c = &c; op.otab.c = &c;
  op.csr.rp.c = &c; op.csr.ci.c = &c; op.csr.v.c = &c;
}

// Build from an FP64 CSR matrix, casting the values to T.
template <class T>
void rowsop_build(Ctx& c, const DCSR<double>& A, RowsOp<T>& op);

// Adds to *bad (device) the number of stored column indices, recomputed as the apply kernels do,
// that fall outside [0, nc), and of offsets, pointers or row permutations out of order or range.
template <class T>
void rowsop_audit(Ctx& c, const RowsOp<T>& op, unsigned long long* bad);

}  // namespace mgr
