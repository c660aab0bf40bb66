// apply.cuh -- launchers of the preconditioner-apply and Krylov kernels.
#pragma once
#include "bsr_sell.cuh"
#include "common.cuh"
#include "rowsop.cuh"

namespace mgr {

template <class T>
struct CSRView {
  int64_t nr = 0, nnz = 0;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const T* v = nullptr;
};
template <class T>
inline CSRView<T> view(const DCSR<T>& m) {
  CSRView<T> r;
  r.nr = m.nr; r.nnz = m.nnz; r.rp = m.rp.p; r.ci = m.ci.p; r.v = m.v.p;
  return r;
}

// ---- level 0 (BSR) ---------------------------------------------------------------------------
// e0 = blockdiag(A)^-1 r (Algorithm step 1); r is the FP64 input.
template <class T>
void launch_global_relax(Ctx& c, int64_t nb, const T* binv, const double* r, T* e0);
// res = r - A e0 over the sliced BSR layout (e0 == nullptr: res = r), routed by map: C dofs to
// rnext[c], F dofs to resF[f].
template <class T>
void launch_bsr_resid_split(Ctx& c, const SellPattern& S, const T* vals, const double* r, const T* e0,
                            const int32_t* map, T* rnext, T* resF);

// ---- reduction levels ------------------------------------------------------------------------
// sweep 1 from e = 0: eF = minv * src, src = r[F[f]] (F != nullptr) or resF[f]
template <class T>
void launch_frelax_first(Ctx& c, int64_t nF, const int32_t* F, const T* src, const T* minv, T* eF);
// later sweeps: eFo = eFi + minv * (src - A_ff eFi)
template <class T>
void launch_frelax_sweep(Ctx& c, const RowsOp<T>& Aff, const int32_t* F, const T* src, const T* minv, const T* eFi,
                         T* eFo, const char* name = "frelax");
// rnext[c] = base_c - A_cf eF with base_c = r[C[c]] (C != nullptr) or rnext[c] (in place)
template <class T>
void launch_restrict(Ctx& c, const RowsOp<T>& Acf, const int32_t* C, const T* r, const T* eF, T* rnext,
                     const char* name = "restrict");
// out[C[c]] = base + ec[c]; out[F[f]] = base + eF[f] + W_p[f,:] ec; base may be nullptr
template <class T, class TO>
void launch_interp(Ctx& c, int64_t nF, const int32_t* F, int64_t nC, const int32_t* C, const RowsOp<T>& Wp,
                   const T* eF, const T* ec, const T* base, TO* out, const char* name = "interp");
template <class T>
void launch_to_f64(Ctx& c, int64_t n, const T* a, double* b);
// pieces of the transposed preconditioner M^-T
template <class T>
void launch_gather_add(Ctx& c, const RowsOp<T>& WpT, const int32_t* C, const T* y, T* out, const char* name);
template <class T>
void launch_scatter_cf(Ctx& c, int64_t nC, const int32_t* C, const T* tc, int64_t nF, const int32_t* F, const T* gF,
                       T* g);
template <class T>
void launch_bsr_grt(Ctx& c, const SellPattern& S, const T* valsT, const double* y, const T* g, const T* bt,
                    double* z);
template <class T>
void launch_transpose_blocks(Ctx& c, int64_t nb, const T* b, T* bt);
void launch_dense_transpose(Ctx& c, int64_t n, const double* a, double* at);
template <class T>
void launch_gather(Ctx& c, int64_t n, const int32_t* idx, const T* src, T* dst);  // dst[f] = src[idx[f]]
template <class T>
void launch_axpy(Ctx& c, int64_t n, const T* x, T* y);                            // y += x
void launch_map_cols(Ctx& c, int64_t nnz, int32_t* ci, const int32_t* map);

// ---- AMG -------------------------------------------------------------------------------------
template <class T>
void launch_scale(Ctx& c, int64_t n, const T* d, const T* b, T* x);                          // x = d * b
template <class T>
void launch_resid(Ctx& c, const RowsOp<T>& A, const T* x, const T* b, T* res,
                  const char* name = "csr_rows");                                           // res = b - A x
template <class T>
void launch_jacobi(Ctx& c, const RowsOp<T>& A, const T* d, const T* b, const T* xi, T* xo,
                   const char* name = "csr_rows");                                          // xo = xi + d (b - A xi)
template <class T>
void launch_spmv(Ctx& c, const RowsOp<T>& A, const T* x, T* y, const char* name = "amg_restrict");  // y = A x
template <class T>
void launch_prolong_add(Ctx& c, const RowsOp<T>& P, const T* xc, T* x, const char* name = "amg_prolong");  // x += P xc
template <class T>
void launch_dense_gemv(Ctx& c, int64_t n, const double* inv, const T* b, T* x);              // x = inv b (FP64)

void launch_cast_f32(Ctx& c, int64_t n, const double* a, float* b);

// ---- Krylov (FP64) ---------------------------------------------------------------------------
void launch_bsr3_spmv_f64(Ctx& c, const mgr_bsr3_t& A, const double* x, const double* sub, double* y);
// the same product over the sliced layout (values filled by sell_fill_values)
void launch_sell_spmv_f64(Ctx& c, const SellPattern& S, const double* vals, const double* x, const double* sub,
                          double* y);
// Deterministic multi-dot: out[k] = V_k . w for k < nv (V_k = V + k ldv, ldv even) and, if
// want_ww, out[nv] = w . w.  `part` must hold KRY_PART doubles.
constexpr int KRY_GRID = 304;
constexpr int KRY_MAXV = 32;
constexpr int KRY_PART = 1216 * (KRY_MAXV + 1);
void launch_mdot(Ctx& c, int64_t n, const double* V, int64_t ldv, int nv, const double* w, bool want_ww, double* part,
                 double* out);
// vout = scale (w - sum_k h[k] V_k) with h and *scale on the device (scale == nullptr: 1); vout may
// alias w; out[0] = ||vout||^2 when out != nullptr
void launch_mupdate(Ctx& c, int64_t n, const double* V, int64_t ldv, int nv, const double* h, const double* scale,
                    const double* w, double* vout, double* part, double* out);
// out[0] = ww - sum h_k^2 and out[1] = 1 / sqrt(out[0]) (0 if out[0] <= 0)
void launch_pyth_scale(Ctx& c, int nv, const double* h, const double* ww, double* out);
// y = alpha x
void launch_scal(Ctx& c, int64_t n, double alpha, const double* x, double* y);
// x += sum_k y[k] Z_k (y on device)
void launch_xupdate(Ctx& c, int64_t n, const double* Z, int64_t ldz, int nz, const double* y, double* x);
// out[0] = x . x
void launch_nrm2sq(Ctx& c, int64_t n, const double* x, double* part, double* out);

// adjoint helpers
void launch_bsr3_outer_grad(Ctx& c, const mgr_bsr3_t& A, const double* lam, const double* x, double* g);
void launch_bsr3_transpose(Ctx& c, const mgr_bsr3_t& A, int64_t* rpt, int32_t* cit, double* vt);
void launch_bsr3_transpose_pattern(Ctx& c, const mgr_bsr3_t& A, int64_t* rpt, int32_t* cit, int64_t* src);

}  // namespace mgr
