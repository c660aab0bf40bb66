// rowsop.cu -- construction of the apply operators in SELL-8 or CSR form (see rowsop.cuh).
#include "rowsop.cuh"

#include <climits>

namespace mgr {

// slice widths (longest row of each slice, rounded up to a multiple of q); rows in slice order are
// perm[r] when perm is given
__global__ void k_rs_width(int64_t nr, const int64_t* rp, const int32_t* perm, int q, int64_t nslices,
                           int64_t* width) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int64_t w = 0, e = (s + 1) * RS_C < nr ? (s + 1) * RS_C : nr;
  for (int64_t r = s * RS_C; r < e; ++r) {
    int64_t o = perm ? perm[r] : r;
    w = max(w, rp[o + 1] - rp[o]);
  }
  width[s] = (w + q - 1) / q * q;
}

// order the rows of each window of RS_SIGMA rows by decreasing length, equal lengths by row index
// (one block per window: bitonic sort of (length, row) keys in shared memory)
__global__ void __launch_bounds__(RS_SIGMA) k_rs_sort(int64_t nr, const int64_t* rp, int32_t* perm) {
  __shared__ unsigned long long key[RS_SIGMA];
  int64_t r0 = (int64_t)blockIdx.x * RS_SIGMA;
  int t = threadIdx.x;
  int64_t r = r0 + t;
  if (r < nr) {
    unsigned long long len = (unsigned long long)(rp[r + 1] - rp[r]);
    // ascending sort of (max_len - len, index) = descending length, ascending index
    key[t] = ((0xFFFFFFFFull - (len > 0xFFFFFFFFull ? 0xFFFFFFFFull : len)) << 32) | (unsigned long long)t;
  } else {
    key[t] = ~0ull;
  }
  __syncthreads();
  for (int k = 2; k <= RS_SIGMA; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      int x = t ^ j;
      if (x > t) {
        bool up = (t & k) == 0;
        unsigned long long a = key[t], b = key[x];
        if ((a > b) == up) { key[t] = b; key[x] = a; }
      }
      __syncthreads();
    }
  if (r < nr) perm[r] = (int32_t)(r0 + (int64_t)(key[t] & 0xFFFFFFFFull));
}

template <class T>
__global__ void k_rs_fill(int64_t nr, int64_t npad, const int64_t* rp, const int32_t* ci, const double* v,
                          const int32_t* perm, int q, const int64_t* soff, int32_t* scol, T* sval) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= npad) return;
  int64_t s = r / RS_C;
  int t = (int)(r - s * RS_C);
  int64_t b0 = soff[s], w = soff[s + 1] - b0;
  int64_t o0 = r < nr ? (perm ? perm[r] : r) : 0;
  int64_t k0 = r < nr ? rp[o0] : 0, len = r < nr ? rp[o0 + 1] - k0 : 0;
  for (int64_t j = 0; j < w; ++j) {
    int64_t o = b0 * RS_C + (j / q) * (q * RS_C) + t * q + (j % q);
    if (j < len) { scol[o] = ci[k0 + j]; sval[o] = (T)v[k0 + j]; }
    else { scol[o] = 0; sval[o] = T(0); }  // column 0 exists in every operator with nonzeros
  }
}

// offsets col - row of the entries: the largest magnitude, then the used ones marked in a window of
// 2 maxd + 1 flags
__global__ void k_rs_offmax(int64_t nr, const int64_t* rp, const int32_t* ci, unsigned long long* maxd) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long m = 0;
  if (r < nr)
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
      long long d = (long long)ci[k] - r;
      m = max(m, (unsigned long long)(d < 0 ? -d : d));
    }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));  // one atomic per warp
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(maxd, m);
}
__global__ void k_rs_offmark(int64_t nr, const int64_t* rp, const int32_t* ci, int64_t maxd, int32_t* flag) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
    int32_t* f = flag + ((int64_t)ci[k] - r + maxd);
    if (*f == 0) *f = 1;  // most offsets repeat: read first, write once
  }
}
__global__ void k_rs_offtab(int64_t nw, const int32_t* flag, const int32_t* code, int64_t maxd, int32_t* otab) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v < nw && flag[v]) otab[code[v]] = (int32_t)(v - maxd);
}
// the slots of row t of each slice as codes (padding: 255)
__global__ void k_rs_cwidth(int64_t ns, const int64_t* soff, int64_t* cw) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s < ns) cw[s] = (soff[s + 1] - soff[s] + 15) / 16 * 16;
}
__global__ void k_rs_pack8(int64_t nr, int64_t npad, const int64_t* rp, const int32_t* perm, const int64_t* soff,
                           const int64_t* coff, const int32_t* scol, const int32_t* code, int64_t maxd,
                           uint8_t* scode) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= npad) return;
  int64_t s = r / RS_C;
  int t = (int)(r - s * RS_C);
  int64_t b0 = soff[s], w = soff[s + 1] - b0;
  int64_t row = r < nr ? (perm ? perm[r] : r) : 0;
  int64_t len = r < nr ? rp[row + 1] - rp[row] : 0;
  const int64_t cb = coff[s] * RS_C, cw = coff[s + 1] - coff[s];
  for (int64_t j = 0; j < cw; ++j) {
    int64_t o = b0 * RS_C + (j / RS_Q) * (RS_Q * RS_C) + t * RS_Q + (j % RS_Q);
    scode[cb + rs_code_pos(j, t)] = (j < w && j < len) ? (uint8_t)code[(int64_t)scol[o] - row + maxd] : (uint8_t)255;
  }
}

// per slice: the smallest column of its rows (base) and a flag when the slice spans more than 65,536
__global__ void k_rs_base(int64_t nr, const int64_t* rp, const int32_t* ci, const int32_t* perm, int64_t nslices,
                          int32_t* base, int* wide) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int32_t lo = INT_MAX, hi = -1;
  int64_t e = (s + 1) * RS_C < nr ? (s + 1) * RS_C : nr;
  for (int64_t r = s * RS_C; r < e; ++r) {
    int64_t o = perm ? perm[r] : r;
    for (int64_t k = rp[o]; k < rp[o + 1]; ++k) {
      lo = min(lo, ci[k]);
      hi = max(hi, ci[k]);
    }
  }
  if (hi < 0) lo = hi = 0;  // an empty slice
  base[s] = lo;
  if ((int64_t)hi - (int64_t)lo > 65535) atomicOr(wide, 1);
}
// the slots of row t of each slice as 16-bit offsets from the slice's base (padding slots, column 0
// below a positive base, become offset 0)
__global__ void k_rs_pack16(int64_t npad, const int64_t* soff, const int32_t* scol, const int32_t* base,
                            uint16_t* scol16) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= npad) return;
  int64_t s = r / RS_C;
  int t = (int)(r - s * RS_C);
  int64_t b0 = soff[s], w = soff[s + 1] - b0;
  const int32_t bs = base[s];
  for (int64_t j = 0; j < w; ++j) {
    int64_t o = b0 * RS_C + (j / RS_Q) * (RS_Q * RS_C) + t * RS_Q + (j % RS_Q);
    int32_t cc = scol[o];
    scol16[o] = (uint16_t)(cc >= bs ? cc - bs : 0);
  }
}

template <class T>
__global__ void k_rs_cast(int64_t n, const double* a, T* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (T)a[i];
}

template <class T>
void rowsop_build(Ctx& c, const DCSR<double>& A, RowsOp<T>& op) {
  op.nr = A.nr;
  op.nc = A.nc;
  op.nnz = A.nnz;
  op.sell = false;
  op.slots = 0;
  if (A.nr >= RS_MIN_ROWS && A.nnz > 0) {
    int64_t ns = (A.nr + RS_C - 1) / RS_C;
    DBuf<int64_t> width(c, ns + 1);
    op.soff.alloc(c, ns + 1);
    op.q = ((double)A.nnz >= RS_QUAD_MIN_AVG * (double)A.nr) ? RS_Q : 1;
    k_rs_width<<<grid_for(ns, 256), 256, 0, c.s>>>(A.nr, A.rp, nullptr, op.q, ns, width.p);
    CU_LAUNCH();
    op.slots = counts_to_rowptr(c, width.p, op.soff.p, ns);
    if ((double)(op.slots * RS_C) > RS_SORT_PAD * (double)A.nnz) {
      op.perm.alloc(c, A.nr);
      k_rs_sort<<<(unsigned)((A.nr + RS_SIGMA - 1) / RS_SIGMA), RS_SIGMA, 0, c.s>>>(A.nr, A.rp, op.perm.p);
      CU_LAUNCH();
      k_rs_width<<<grid_for(ns, 256), 256, 0, c.s>>>(A.nr, A.rp, op.perm.p, op.q, ns, width.p);
      CU_LAUNCH();
      op.slots = counts_to_rowptr(c, width.p, op.soff.p, ns);
    }
    if ((double)(op.slots * RS_C) <= RS_MAX_PAD * (double)A.nnz) {
      op.sell = true;
      op.scol.alloc(c, op.slots * RS_C);
      op.sval.alloc(c, op.slots * RS_C);
      int64_t np = ns * RS_C;
      k_rs_fill<T><<<grid_for(np, 256), 256, 0, c.s>>>(A.nr, np, A.rp, A.ci, A.v, op.perm.p, op.q, op.soff.p,
                                                      op.scol.p, op.sval.p);
      CU_LAUNCH();
      if (op.q == RS_Q && A.nr == A.nc) {
        // one-byte offset codes when at most 255 distinct offsets col - row occur
        DBuf<unsigned long long> md(c, 1);
        CU(cudaMemsetAsync(md.p, 0, sizeof(unsigned long long), c.s));
        k_rs_offmax<<<grid_for(A.nr, 256), 256, 0, c.s>>>(A.nr, A.rp, A.ci, md.p);
        CU_LAUNCH();
        const int64_t maxd = (int64_t)read_scalar(c, md.p);
        if (maxd <= (int64_t(1) << 22)) {
          const int64_t nw = 2 * maxd + 1;
          DBuf<int32_t> flag(c, nw), code(c, nw + 1);
          CU(cudaMemsetAsync(flag.p, 0, sizeof(int32_t) * nw, c.s));
          k_rs_offmark<<<grid_for(A.nr, 256), 256, 0, c.s>>>(A.nr, A.rp, A.ci, maxd, flag.p);
          CU_LAUNCH();
          scan_excl_i32(c, flag.p, code.p, nw);
          const int32_t ncodes = read_scalar(c, code.p + nw);
          if (ncodes <= 255) {
            op.c8 = true;
            op.otab.alloc(c, 256);
            CU(cudaMemsetAsync(op.otab.p, 0, sizeof(int32_t) * 256, c.s));  // code 255 (padding): offset 0
            k_rs_offtab<<<grid_for(nw, 256), 256, 0, c.s>>>(nw, flag.p, code.p, maxd, op.otab.p);
            CU_LAUNCH();
            op.coff.alloc(c, ns + 1);
            k_rs_cwidth<<<grid_for(ns, 256), 256, 0, c.s>>>(ns, op.soff.p, width.p);
            CU_LAUNCH();
            const int64_t cslots = counts_to_rowptr(c, width.p, op.coff.p, ns);
            op.scode.alloc(c, cslots * RS_C);
            k_rs_pack8<<<grid_for(np, 256), 256, 0, c.s>>>(A.nr, np, A.rp, op.perm.p, op.soff.p, op.coff.p,
                                                           op.scol.p, code.p, maxd, op.scode.p);
            CU_LAUNCH();
            op.scol.release();
            return;
          }
        }
      }
      if (op.q == RS_Q) {
        op.sbase.alloc(c, ns);
        DBuf<int> wide(c, 1);
        CU(cudaMemsetAsync(wide.p, 0, sizeof(int), c.s));
        k_rs_base<<<grid_for(ns, 256), 256, 0, c.s>>>(A.nr, A.rp, A.ci, op.perm.p, ns, op.sbase.p, wide.p);
        CU_LAUNCH();
        if (read_scalar(c, wide.p) == 0) {
          op.c16 = true;
          op.scol16.alloc(c, op.slots * RS_C);
          k_rs_pack16<<<grid_for(np, 256), 256, 0, c.s>>>(np, op.soff.p, op.scol.p, op.sbase.p, op.scol16.p);
          CU_LAUNCH();
          op.scol.release();
        } else {
          op.sbase.release();
        }
      }
      return;
    }
    op.soff.release();
    op.perm.release();
  }
  DCSR<T>& B = op.csr;
  B.nr = A.nr; B.nc = A.nc; B.nnz = A.nnz;
  B.rp.alloc(c, A.nr + 1);
  B.ci.alloc(c, A.nnz);
  B.v.alloc(c, A.nnz);
  CU(cudaMemcpyAsync(B.rp.p, A.rp.p, sizeof(int64_t) * (A.nr + 1), cudaMemcpyDeviceToDevice, c.s));
  if (A.nnz) {
    CU(cudaMemcpyAsync(B.ci.p, A.ci.p, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToDevice, c.s));
    k_rs_cast<T><<<grid_for(A.nnz, 256, 8192), 256, 0, c.s>>>(A.nnz, A.v.p, B.v.p);
    CU_LAUNCH();
  }
}

// ---- index audit ---------------------------------------------------------------------------------
// Every column an apply kernel gathers with, recomputed from the stored form the way those kernels
// compute it (32-bit column, slice base + 16-bit offset, row + table[code]), must lie in [0, nc); the
// slice offsets and row pointers must not decrease and the row permutation must stay in [0, nr).
// Each violation adds one to *bad.
__global__ void k_audit_rows_sell(int64_t nr, int64_t nc, int q, const int64_t* soff, const int32_t* perm,
                                  const int32_t* scol, const uint16_t* scol16, const int32_t* sbase,
                                  const uint8_t* scode, const int64_t* coff, const int32_t* otab,
                                  unsigned long long* bad) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  const int64_t s = r / RS_C;
  const int t = (int)(r - s * RS_C);
  const int64_t b0 = soff[s], w = soff[s + 1] - b0;
  unsigned long long nbad = 0;
  const int64_t row = perm ? (int64_t)perm[r] : r;
  if (w < 0 || row < 0 || row >= nr) {
    atomicAdd(bad, 1ull);
    return;
  }
  if (scode) {
    const int64_t cb = coff[s] * RS_C, cw = coff[s + 1] - coff[s];
    if (cw < w) ++nbad;
    for (int64_t j = 0; j < cw; ++j) {
      const int64_t col = row + otab[scode[cb + rs_code_pos(j, t)]];
      nbad += (col < 0 || col >= nc);
    }
  } else {
    for (int64_t j = 0; j < w; ++j) {
      const int64_t o = b0 * RS_C + (j / q) * (q * RS_C) + t * q + (j % q);
      const int64_t col = scol16 ? (int64_t)sbase[s] + scol16[o] : (int64_t)scol[o];
      nbad += (col < 0 || col >= nc);
    }
  }
  if (nbad) atomicAdd(bad, nbad);
}

template <class TI>
__global__ void k_audit_csr(int64_t nr, int64_t nc, int64_t nnz, const int64_t* rp, const TI* ci,
                            unsigned long long* bad) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  const int64_t a = rp[r], b = rp[r + 1];
  if (a < 0 || a > b || b > nnz || (r == 0 && a != 0) || (r == nr - 1 && b != nnz)) {
    atomicAdd(bad, 1ull);
    return;
  }
  unsigned long long nbad = 0;
  for (int64_t k = a; k < b; ++k) nbad += (ci[k] < 0 || (int64_t)ci[k] >= nc);
  if (nbad) atomicAdd(bad, nbad);
}

template <class T>
void rowsop_audit(Ctx& c, const RowsOp<T>& op, unsigned long long* bad) {
  if (op.nr <= 0) return;
  if (op.sell) {
    k_audit_rows_sell<<<grid_for(op.nr, 256), 256, 0, c.s>>>(
        op.nr, op.nc, op.q, op.soff.p, op.perm.p, (op.c8 || op.c16) ? nullptr : op.scol.p,
        op.c16 ? op.scol16.p : nullptr, op.c16 ? op.sbase.p : nullptr, op.c8 ? op.scode.p : nullptr, op.coff.p,
        op.otab.p, bad);
    CU_LAUNCH();
  } else if (op.csr.rp.p) {
    k_audit_csr<int32_t><<<grid_for(op.nr, 256), 256, 0, c.s>>>(op.nr, op.nc, op.csr.nnz, op.csr.rp.p, op.csr.ci.p,
                                                                bad);
    CU_LAUNCH();
  }
}

template void rowsop_audit<float>(Ctx&, const RowsOp<float>&, unsigned long long*);
template void rowsop_audit<double>(Ctx&, const RowsOp<double>&, unsigned long long*);

template void rowsop_build<float>(Ctx&, const DCSR<double>&, RowsOp<float>&);
template void rowsop_build<double>(Ctx&, const DCSR<double>&, RowsOp<double>&);

}  // namespace mgr
