// krylov.cu -- FP64 kernels of the flexible GMRES outer iteration (section 6: GMRES around the
// MGR preconditioner) and of the adjoint helpers: BSR SpMV, deterministic multi-dot products with
// warp-shuffle reductions, Gram-Schmidt updates, solution update, block transpose, outer-product
// gradient.  Reductions are two-stage with a fixed grid, so results do not depend on timing.
#include "apply.cuh"

namespace mgr {

// y = A x or y = sub - A x, one thread per block row
__global__ void __launch_bounds__(256) k_bsr3_spmv_f64(int64_t nb, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                       const double* __restrict__ x, const double* __restrict__ sub,
                                                       double* __restrict__ y) {
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  int64_t k1 = rp[I + 1];
  for (int64_t k = rp[I]; k < k1; ++k) {
    int64_t J = ci[k];
    const double* b = v + 9 * k;
    double x0 = __ldg(x + 3 * J), x1 = __ldg(x + 3 * J + 1), x2 = __ldg(x + 3 * J + 2);
    s0 += b[0] * x0 + b[1] * x1 + b[2] * x2;
    s1 += b[3] * x0 + b[4] * x1 + b[5] * x2;
    s2 += b[6] * x0 + b[7] * x1 + b[8] * x2;
  }
  if (sub) { s0 = sub[3 * I] - s0; s1 = sub[3 * I + 1] - s1; s2 = sub[3 * I + 2] - s2; }
  y[3 * I] = s0;
  y[3 * I + 1] = s1;
  y[3 * I + 2] = s2;
}

void launch_bsr3_spmv_f64(Ctx& c, const mgr_bsr3_t& A, const double* x, const double* sub, double* y) {
  k_bsr3_spmv_f64<<<grid_for(A.nb, 256), 256, 0, c.s>>>(A.nb, A.rowptr, A.colind, A.values, x, sub, y);
  CU_LAUNCH();
}

// ---- multi-dot ---------------------------------------------------------------------------------
constexpr int KT = 256;

template <int NA>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NA], int na, double* part) {
  __shared__ double sh[KT / 32][NA];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NA; ++k) {
    if (k < na) {
      double v = warp_sum(acc[k]);
      if (lane == 0) sh[wid][k] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < na) {
    double s = 0.0;
    for (int w = 0; w < KT / 32; ++w) s += sh[w][threadIdx.x];
    part[(int64_t)blockIdx.x * na + threadIdx.x] = s;
  }
}

__global__ void __launch_bounds__(KT) k_mdot(int64_t n, const double* __restrict__ V, int64_t ldv, int nv,
                                             const double* __restrict__ w, int ww, double* __restrict__ part) {
  // acc[0..nv) = V_k . w, acc[KRY_MAXV] = w . w; all indices compile-time after unrolling
  double acc[KRY_MAXV + 1];
#pragma unroll
  for (int k = 0; k <= KRY_MAXV; ++k) acc[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)KT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KT) {
    double wi = w[i];
#pragma unroll
    for (int k = 0; k < KRY_MAXV; ++k)
      if (k < nv) acc[k] += V[k * ldv + i] * wi;
    if (ww) acc[KRY_MAXV] += wi * wi;
  }
  __shared__ double sh[KT / 32][KRY_MAXV + 1];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k <= KRY_MAXV; ++k) {
    if (k < nv || (k == KRY_MAXV && ww)) {
      double v = warp_sum(acc[k]);
      if (lane == 0) sh[wid][k] = v;
    }
  }
  __syncthreads();
  int na = nv + ww;
  if (threadIdx.x < na) {
    int k = (threadIdx.x < nv) ? threadIdx.x : KRY_MAXV;
    double s = 0.0;
    for (int w2 = 0; w2 < KT / 32; ++w2) s += sh[w2][k];
    part[(int64_t)blockIdx.x * na + threadIdx.x] = s;
  }
}

__global__ void k_reduce_final(int nblk, int na, const double* __restrict__ part, double* __restrict__ out) {
  int k = threadIdx.x;
  if (k >= na) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * na + k];
  out[k] = s;
}

void launch_mdot(Ctx& c, int64_t n, const double* V, int64_t ldv, int nv, const double* w, bool want_ww, double* part,
                 double* out) {
  if (nv > KRY_MAXV) throw Error(MGR_ERR_UNSUPPORTED, "multi-dot with more than 32 vectors");
  int ww = want_ww ? 1 : 0;
  k_mdot<<<KRY_GRID, KT, 0, c.s>>>(n, V, ldv, nv, w, ww, part);
  CU_LAUNCH();
  k_reduce_final<<<1, 64, 0, c.s>>>(KRY_GRID, nv + ww, part, out);
  CU_LAUNCH();
}

// w -= sum_k h[k] V_k, then ||w||^2
__global__ void __launch_bounds__(KT) k_mupdate(int64_t n, const double* __restrict__ V, int64_t ldv, int nv,
                                                const double* __restrict__ h, double* __restrict__ w,
                                                double* __restrict__ part) {
  __shared__ double sh_h[KRY_MAXV];
  if (threadIdx.x < nv) sh_h[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)KT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KT) {
    double s = w[i];
#pragma unroll
    for (int k = 0; k < KRY_MAXV; ++k)
      if (k < nv) s -= sh_h[k] * V[k * ldv + i];
    w[i] = s;
    acc[0] += s * s;
  }
  block_reduce_store<1>(acc, 1, part);
}

void launch_mupdate(Ctx& c, int64_t n, const double* V, int64_t ldv, int nv, const double* h, double* w, double* part,
                    double* out) {
  if (nv > KRY_MAXV) throw Error(MGR_ERR_UNSUPPORTED, "update with more than 32 vectors");
  k_mupdate<<<KRY_GRID, KT, 0, c.s>>>(n, V, ldv, nv, h, w, part);
  CU_LAUNCH();
  k_reduce_final<<<1, 64, 0, c.s>>>(KRY_GRID, 1, part, out);
  CU_LAUNCH();
}

__global__ void __launch_bounds__(KT) k_nrm2sq(int64_t n, const double* __restrict__ x, double* __restrict__ part) {
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)KT + threadIdx.x; i < n; i += (int64_t)gridDim.x * KT) acc[0] += x[i] * x[i];
  block_reduce_store<1>(acc, 1, part);
}
void launch_nrm2sq(Ctx& c, int64_t n, const double* x, double* part, double* out) {
  k_nrm2sq<<<KRY_GRID, KT, 0, c.s>>>(n, x, part);
  CU_LAUNCH();
  k_reduce_final<<<1, 64, 0, c.s>>>(KRY_GRID, 1, part, out);
  CU_LAUNCH();
}

__global__ void k_scal(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
void launch_scal(Ctx& c, int64_t n, double alpha, const double* x, double* y) {
  k_scal<<<grid_for(n, 256, 4 * 1024), 256, 0, c.s>>>(n, alpha, x, y);
  CU_LAUNCH();
}

__global__ void k_xupdate(int64_t n, const double* __restrict__ Z, int64_t ldz, int nz, const double* __restrict__ y,
                          double* __restrict__ x) {
  __shared__ double sy[KRY_MAXV];
  if (threadIdx.x < nz) sy[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = x[i];
#pragma unroll
    for (int k = 0; k < KRY_MAXV; ++k)
      if (k < nz) s += sy[k] * Z[k * ldz + i];
    x[i] = s;
  }
}
void launch_xupdate(Ctx& c, int64_t n, const double* Z, int64_t ldz, int nz, const double* y, double* x) {
  for (int k0 = 0; k0 < nz; k0 += KRY_MAXV) {
    int m = nz - k0 < KRY_MAXV ? nz - k0 : KRY_MAXV;
    k_xupdate<<<grid_for(n, 256, 4 * 1024), 256, 0, c.s>>>(n, Z + k0 * ldz, ldz, m, y + k0, x);
    CU_LAUNCH();
  }
}

// ---- adjoint helpers ---------------------------------------------------------------------------
// g[9k + 3p + q] = -lam[3I+p] x[3J+q]
__global__ void k_outer_grad(int64_t nb, const int64_t* rp, const int32_t* ci, const double* lam, const double* x,
                             double* g) {
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  double l0 = lam[3 * I], l1 = lam[3 * I + 1], l2 = lam[3 * I + 2];
  for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
    int64_t J = ci[k];
    double x0 = x[3 * J], x1 = x[3 * J + 1], x2 = x[3 * J + 2];
    double* o = g + 9 * k;
    o[0] = -l0 * x0; o[1] = -l0 * x1; o[2] = -l0 * x2;
    o[3] = -l1 * x0; o[4] = -l1 * x1; o[5] = -l1 * x2;
    o[6] = -l2 * x0; o[7] = -l2 * x1; o[8] = -l2 * x2;
  }
}
void launch_bsr3_outer_grad(Ctx& c, const mgr_bsr3_t& A, const double* lam, const double* x, double* g) {
  k_outer_grad<<<grid_for(A.nb, 256), 256, 0, c.s>>>(A.nb, A.rowptr, A.colind, lam, x, g);
  CU_LAUNCH();
}

__global__ void k_bcol_count(int64_t nnzb, const int32_t* ci, unsigned long long* cnt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnzb; k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[ci[k]], 1ull);
}
__global__ void k_bscatter(int64_t nb, const int64_t* rp, const int32_t* ci, const int64_t* trp, unsigned long long* slot,
                           int32_t* tci, int64_t* src) {
  int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
    int32_t J = ci[k];
    int64_t d = trp[J] + (int64_t)atomicAdd(&slot[J], 1ull);
    tci[d] = (int32_t)I;
    src[d] = k;
  }
}
// sort each transposed block row by column (insertion sort: block rows are short), then copy the
// transposed 3x3 blocks
__global__ void k_bsort_fill(int64_t nb, const int64_t* trp, int32_t* tci, int64_t* src, const double* v, double* vt) {
  int64_t J = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (J >= nb) return;
  int64_t b = trp[J], e = trp[J + 1];
  for (int64_t a = b + 1; a < e; ++a) {
    int32_t key = tci[a];
    int64_t s = src[a];
    int64_t t = a - 1;
    while (t >= b && tci[t] > key) { tci[t + 1] = tci[t]; src[t + 1] = src[t]; --t; }
    tci[t + 1] = key;
    src[t + 1] = s;
  }
  for (int64_t d = b; d < e; ++d) {
    const double* in = v + 9 * src[d];
    double* o = vt + 9 * d;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q) o[3 * p + q] = in[3 * q + p];
  }
}
void launch_bsr3_transpose(Ctx& c, const mgr_bsr3_t& A, int64_t* rpt, int32_t* cit, double* vt) {
  DBuf<unsigned long long> cnt(c, A.nb + 1);
  DBuf<int64_t> src(c, A.nnzb);
  CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (A.nb + 1), c.s));
  k_bcol_count<<<grid_for(A.nnzb, 256, 8192), 256, 0, c.s>>>(A.nnzb, A.colind, cnt.p);
  CU_LAUNCH();
  scan_excl_i64(c, reinterpret_cast<const int64_t*>(cnt.p), rpt, A.nb);
  CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * (A.nb + 1), c.s));
  k_bscatter<<<grid_for(A.nb, 256), 256, 0, c.s>>>(A.nb, A.rowptr, A.colind, rpt, cnt.p, cit, src.p);
  CU_LAUNCH();
  k_bsort_fill<<<grid_for(A.nb, 256), 256, 0, c.s>>>(A.nb, rpt, cit, src.p, A.values, vt);
  CU_LAUNCH();
  CU(cudaStreamSynchronize(c.s));
}

}  // namespace mgr
