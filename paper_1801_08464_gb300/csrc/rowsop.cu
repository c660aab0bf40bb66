// rowsop.cu -- construction of the apply operators in SELL-8 or CSR form (see rowsop.cuh).
#include "rowsop.cuh"

namespace mgr {

__global__ void k_rs_width(int64_t nr, const int64_t* rp, int64_t nslices, int64_t* width) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int64_t w = 0, e = (s + 1) * RS_C < nr ? (s + 1) * RS_C : nr;
  for (int64_t r = s * RS_C; r < e; ++r) w = max(w, rp[r + 1] - rp[r]);
  width[s] = (w + RS_Q - 1) / RS_Q * RS_Q;
}

template <class T>
__global__ void k_rs_fill(int64_t nr, int64_t npad, const int64_t* rp, const int32_t* ci, const double* v,
                          const int64_t* soff, int32_t* scol, T* sval) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= npad) return;
  int64_t s = r / RS_C;
  int t = (int)(r - s * RS_C);
  int64_t b0 = soff[s], w = soff[s + 1] - b0;
  int64_t k0 = r < nr ? rp[r] : 0, len = r < nr ? rp[r + 1] - k0 : 0;
  for (int64_t j = 0; j < w; ++j) {
    int64_t o = b0 * RS_C + (j / RS_Q) * (RS_Q * RS_C) + t * RS_Q + (j % RS_Q);
    if (j < len) { scol[o] = ci[k0 + j]; sval[o] = (T)v[k0 + j]; }
    else { scol[o] = 0; sval[o] = T(0); }  // column 0 exists in every operator with nonzeros
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
  if (A.nr > 0 && A.nnz > 0) {
    int64_t ns = (A.nr + RS_C - 1) / RS_C;
    DBuf<int64_t> width(c, ns + 1);
    k_rs_width<<<grid_for(ns, 256), 256, 0, c.s>>>(A.nr, A.rp, ns, width.p);
    CU_LAUNCH();
    op.soff.alloc(c, ns + 1);
    op.slots = counts_to_rowptr(c, width.p, op.soff.p, ns);
    if ((double)(op.slots * RS_C) <= RS_MAX_PAD * (double)A.nnz) {
      op.sell = true;
      op.scol.alloc(c, op.slots * RS_C);
      op.sval.alloc(c, op.slots * RS_C);
      int64_t np = ns * RS_C;
      k_rs_fill<T><<<grid_for(np, 256), 256, 0, c.s>>>(A.nr, np, A.rp, A.ci, A.v, op.soff.p, op.scol.p, op.sval.p);
      CU_LAUNCH();
      return;
    }
    op.soff.release();
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

template void rowsop_build<float>(Ctx&, const DCSR<double>&, RowsOp<float>&);
template void rowsop_build<double>(Ctx&, const DCSR<double>&, RowsOp<double>&);

}  // namespace mgr
