// hier.cuh -- device data of the MGR hierarchy and of the AMG coarse solver.
#pragma once
#include <functional>
#include <vector>

#include "common.cuh"
#include "rowsop.cuh"

namespace mgr {

struct AmgLevel {
  int64_t n = 0;
  DCSR<double> A, P, R, S;        // operator, interpolation, restriction = P^T, strength pattern
  DBuf<int8_t> cf;                // 1 = C, -1 = F
  DBuf<double> dinv;              // smoother scaling
  RowsOp<float> A32, P32, R32;    // apply copies (working precision)
  RowsOp<double> A64, P64, R64;
  DBuf<float> dinv32;
  bool cast = false;
  RowsOp<float> AT32;             // A^T for the transposed V-cycle (when built)
  RowsOp<double> AT64;
};

// One reduction level of section 5: F = {marker == l}, C = {marker > l} among the level's dofs.
struct MgrLevel {
  int64_t n = 0, nF = 0, nC = 0;
  DCSR<double> A;                 // level operator A_l (FP64 setup copy)
  DBuf<int8_t> mk;                // markers of the level's dofs
  DBuf<int32_t> F, C, map;        // F / C lists (level-local dof ids); map[d] = c >= 0 or -(f+1)
  DBuf<double> dff, minv;         // diag(A_ff) and the F-relaxation scaling
  int sweeps = 1;
  DCSR<double> Wp, Wr, P, R;      // W_p (nF x nC), W_r (nC x nF), P (n x nC), R (nC x n)
  DCSR<double> Aff, Acf;          // split operators used by the apply (F-local columns)
  // the operators the apply reads, in its working precision (SELL-8 or CSR)
  RowsOp<float> Aff32, Acf32, Wp32;
  RowsOp<double> Aff64, Acf64, Wp64;
  DBuf<float> minv32;
  bool cast = false;              // apply copies built
  // transposed operators of M^-T (built when the handle serves transposed solves): W_p^T with its
  // columns as level dof numbers, A_cf^T, A_ff^T
  RowsOp<float> WpT32, AcfT32, AffT32;
  RowsOp<double> WpT64, AcfT64, AffT64;
  // frelax_type 2 (section 6.2): the F-relaxation is an AMG V(1,1)-cycle on A_ff per sweep; its
  // hierarchy, coarsest inverse (and transpose) and work buffers
  std::vector<AmgLevel> famg;
  DBuf<double> fcinv, fcinvT;
  int64_t fnco = 0;
  std::vector<DBuf<char>> fa_b, fa_xa, fa_xb, fa_res;
  DBuf<char> w_fsrc, w_fres;
};



struct AmgOpts {
  double theta = 0.25;
  int max_levels = 25, max_coarse = 256, smoother = 1, pre = 1, post = 1, pmax = 0;
  double omega = 1.0;
  uint64_t seed = 3;
};

// Builds levels[0..] from A0 (copied, or moved when take is set; its shape stays in A0) and the FP64
// dense inverse of the coarsest operator.  done(level k), when given, is called once level k + 1 has
// been built from level k (level k's matrices are not read again by the build).
void amg_build(Ctx& c, DCSR<double>& A0, bool take, const AmgOpts& o, std::vector<AmgLevel>& levels,
               DBuf<double>& coarse_inv, int64_t& nco, const std::function<void(AmgLevel&)>& done);

// One reduction step at level l: fills L (splitting, W_p, W_r, P, R, split operators, scaling) and
// the coarse operator Anext = R (A P) with the coarse markers.
struct LevelOpts {
  int frelax_type = 0, sweeps = 1, restrict_type = 0;
  double omega = 1.0;
};
void mgr_reduce_level(Ctx& c, MgrLevel& L, int l, const LevelOpts& o, DCSR<double>& Anext, DBuf<int8_t>& mk_next);

// Dense inverse of an n x n matrix given as CSR (n <= 4096), FP64 Gauss-Jordan with partial
// pivoting; sets EBIT_SINGULAR on a zero pivot.
void dense_inverse(Ctx& c, const DCSR<double>& A, DBuf<double>& inv);

}  // namespace mgr
