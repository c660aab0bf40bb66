// mgr.cu -- handle, setup orchestration, preconditioner apply, flexible GMRES and the C ABI.
//
// Setup (sections 4-5 of the paper): validate the BSR input, invert the 3x3 diagonal blocks for the
// global relaxation, form the scalar level-0 operator, run the reduction levels in marker order
// (level l removes the dofs with cf_marker == l), build the AMG hierarchy on the last (pressure)
// level, then cast what the apply reads to the working precision.
// Apply: the presmoothing Algorithm of section 4 recursively over the levels, an AMG V-cycle (or a
// dense inverse) as the coarse solve.
// Solve: right-preconditioned flexible GMRES(m) with classical Gram-Schmidt and selective
// reorthogonalisation, Givens rotations on the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <cstring>
#include <functional>
#include <type_traits>
#include <vector>

#include <thread>

#include "apply.cuh"
#include "hier.cuh"

using namespace mgr;

struct mgr_handle_s {
  Ctx c;
  // second context (own stream and error word): the apply copies of the MGR levels are built on it
  // by a second host thread while the AMG hierarchy is set up on the main stream
  Ctx cw;
  std::mutex acct_mu;
  mgr_options_t o;
  int device = 0;
  bool ready = false;
  int64_t nb = 0, nnzb = 0;
  DBuf<int64_t> rp0;
  DBuf<int32_t> ci0;
  DBuf<double> val64, binv;       // val64 / val32: level-0 values in the sliced layout of `sell`
  DBuf<float> val32, binv32;
  SellPattern sell;               // sliced layout of A's pattern (apply and Krylov products)
  DBuf<double> kry_vals;          // A's values in the sliced layout, refreshed by each fgmres_solve
  int L = 0;
  std::vector<MgrLevel> lev;  // lev[0..L]; lev[L] holds the coarsest operator only
  std::vector<AmgLevel> amg;
  DBuf<double> cinv;
  int64_t nco = 0;
  bool coarse_dense = false;
  // apply work buffers (bytes; element type set by the precision)
  DBuf<char> w_e0, w_resF0, w_tmp_in, w_tmp_out;
  std::vector<DBuf<char>> w_r, w_e, w_eF, w_eF2;
  std::vector<DBuf<char>> a_b, a_xa, a_xb, a_res;
  // Krylov work
  int kry_m = 0;
  int64_t kry_n = 0, kry_ld = 0;
  DBuf<double> V, Z, part, dsc;
  double* hpin = nullptr;  // pinned host scratch
  double setup_ms = 0.0;
  int64_t apply_launches = 0;
  Prof* prof = nullptr;
  // transposed preconditioner M^-T (options.adjoint = 1)
  bool has_t = false;
  SellPattern sellT;              // A^T's pattern in the sliced layout; src holds A's block index
  DBuf<float> valT32, binvT32;
  DBuf<double> valT64, binvT64, kry_valsT, cinvT;
  std::vector<DBuf<char>> w_u;
  // the forward apply as a CUDA graph (options.apply_graph), valid until the next setup
  cudaStream_t gstream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  DBuf<double> g_in, g_out;  // the graph's fixed input and output
  int64_t g_launches = 0;    // kernel launches captured in it
  int applies = 0;           // forward applies since the setup
  bool graph_failed = false;
};

namespace {

mgr_status_t guard_status(const std::exception_ptr& ep, mgr_handle_s* h) {
  try {
    std::rethrow_exception(ep);
  } catch (const Error& e) {
    if (h) cudaGetLastError();
    fprintf(stderr, "[mgr] %s\n", e.what());
    return e.status;
  } catch (const std::bad_alloc&) {
    return MGR_ERR_OOM;
  } catch (...) {
    return MGR_ERR_CUDA;
  }
}

template <class F>
mgr_status_t guarded(mgr_handle_s* h, F&& f) {
  try {
    f();
    return MGR_OK;
  } catch (...) {
    return guard_status(std::current_exception(), h);
  }
}

template <class T>
inline const T* pick_ptr(const DBuf<double>& d, const DBuf<float>& f) {
  if constexpr (std::is_same<T, float>::value) return f.p;
  else return d.p;
}
template <class T>
inline const RowsOp<T>& tv(const RowsOp<double>& d, const RowsOp<float>& f) {
  if constexpr (std::is_same<T, float>::value) return f;
  else return d;
}
template <class T>
inline T* P(DBuf<char>& b) { return reinterpret_cast<T*>(b.p); }

// ---- apply -----------------------------------------------------------------------------------
// timing names per level (levels beyond the table share the last name)
static const char* lvl_name(const char* const* t, int n, int l) { return t[l < n ? l : n - 1]; }
static const char* const kFrelax[] = {"frelax0", "frelax1", "frelax2", "frelax3"};
static const char* const kRestrict[] = {"restrict0", "restrict1", "restrict2", "restrict3"};
static const char* const kInterp[] = {"interp0", "interp1", "interp2", "interp3"};
static const char* const kAmgRows[] = {"amg0_rows", "amg1_rows", "amg2_rows", "amgc_rows"};
static const char* const kAmgRestrict[] = {"amg0_restrict", "amg1_restrict", "amgc_restrict"};
static const char* const kAmgProlong[] = {"amg0_prolong", "amg1_prolong", "amgc_prolong"};

template <class T>
const T* vcycle_ref(mgr_handle_s& h, MgrLevel& L, const T* b, bool transposed);

template <class T>
const T* frelax(mgr_handle_s& h, int l, const T* src, const int32_t* F, bool transposed = false) {
  MgrLevel& L = h.lev[l];
  T* a = P<T>(h.w_eF[l]);
  T* b = P<T>(h.w_eF2[l]);
  if (L.nF == 0) return a;
  if (!L.famg.empty()) {
    // frelax_type 2: e_F = V(src_F), then e_F += V(src_F - A_ff e_F) for further sweeps (with A_ff^T
    // and the transposed cycle in M^-T: the same recurrence, transposed term by term)
    const T* sF = src;
    if (F) {
      T* gsrc = P<T>(L.w_fsrc);
      launch_gather<T>(h.c, L.nF, F, src, gsrc);
      sF = gsrc;
    }
    const T* v = vcycle_ref<T>(h, L, sF, transposed);
    if (L.sweeps <= 1) return v;
    CU(cudaMemcpyAsync(a, v, sizeof(T) * L.nF, cudaMemcpyDeviceToDevice, h.c.s));
    const RowsOp<T>& Aop = transposed ? tv<T>(L.AffT64, L.AffT32) : tv<T>(L.Aff64, L.Aff32);
    T* rres = P<T>(L.w_fres);
    for (int s = 1; s < L.sweeps; ++s) {
      launch_resid<T>(h.c, Aop, a, sF, rres, lvl_name(kFrelax, 4, l));
      const T* dv = vcycle_ref<T>(h, L, rres, transposed);
      launch_axpy<T>(h.c, L.nF, dv, a);
    }
    return a;
  }
  const T* minv = pick_ptr<T>(L.minv, L.minv32);
  launch_frelax_first<T>(h.c, L.nF, F, src, minv, a);
  // the transpose of the sweeps sum_i (I - D^-1 A_ff)^i D^-1 is the same sweeps with A_ff^T
  const RowsOp<T>& Aff = transposed ? tv<T>(L.AffT64, L.AffT32) : tv<T>(L.Aff64, L.Aff32);
  for (int s = 1; s < L.sweeps; ++s) {
    launch_frelax_sweep<T>(h.c, Aff, F, src, minv, a, b, lvl_name(kFrelax, 4, l));
    std::swap(a, b);
  }
  return a;
}

// An AMG hierarchy with its coarsest inverse and work buffers: the coarse-grid solver of the last
// MGR level, or the A_ff solver of an F-relaxation (frelax_type 2).
struct AmgRef {
  std::vector<AmgLevel>* lv;
  const double* cinv;
  const double* cinvT;
  int64_t nco;
  bool dense;
  std::vector<DBuf<char>>* b;
  std::vector<DBuf<char>>* xa;
  std::vector<DBuf<char>>* xb;
  std::vector<DBuf<char>>* res;
  int pre, post;
  bool coarse;  // timing names of the coarse solver (else "famg_*")
};
static AmgRef coarse_ref(mgr_handle_s& h) {
  return {&h.amg, h.cinv.p, h.cinvT.p, h.nco, h.coarse_dense, &h.a_b, &h.a_xa, &h.a_xb, &h.a_res,
          h.o.amg_pre, h.o.amg_post, true};
}
static AmgRef famg_ref(MgrLevel& L) {
  return {&L.famg, L.fcinv.p, L.fcinvT.p, L.fnco, false, &L.fa_b, &L.fa_xa, &L.fa_xb, &L.fa_res, 1, 1, false};
}

// One V(pre, post) cycle from a zero guess on AMG level k.  transposed: the cycle's transpose, i.e.
// V(post, pre) with A_k^T in the smoothing and residual passes, the same transfers (R = P^T) and the
// transposed coarsest inverse.
template <class T>
const T* vcycle(mgr_handle_s& h, const AmgRef& g, int k, const T* b, bool transposed = false) {
  Ctx& c = h.c;
  int last = (int)g.lv->size() - 1;
  if (k == last || g.dense) {
    T* x = P<T>((*g.xa)[k]);
    launch_dense_gemv<T>(c, g.nco, transposed ? g.cinvT : g.cinv, b, x);
    return x;
  }
  // the coarse end of the coarse solver's cycle (levels 3 and below) as one timed scope
  ProfScope tail(c, (g.coarse && k == 3 && !transposed) ? "amg_tail" : nullptr);
  AmgLevel& A = (*g.lv)[k];
  const RowsOp<T>& Av = transposed ? tv<T>(A.AT64, A.AT32) : tv<T>(A.A64, A.A32);
  const int npre = transposed ? g.post : g.pre;
  const int npost = transposed ? g.pre : g.post;
  const T* d = pick_ptr<T>(A.dinv, A.dinv32);
  T* xa = P<T>((*g.xa)[k]);
  T* xb = P<T>((*g.xb)[k]);
  T* res = P<T>((*g.res)[k]);
  const char* nm = g.coarse ? lvl_name(kAmgRows, 4, k) : "famg_rows";
  launch_scale<T>(c, A.n, d, b, xa);
  for (int s = 1; s < npre; ++s) {
    launch_jacobi<T>(c, Av, d, b, xa, xb, nm);
    std::swap(xa, xb);
  }
  launch_resid<T>(c, Av, xa, b, res, nm);
  T* bc = P<T>((*g.b)[k + 1]);
  launch_spmv<T>(c, tv<T>(A.R64, A.R32), res, bc, g.coarse ? lvl_name(kAmgRestrict, 3, k) : "famg_transfer");
  const T* xc = vcycle<T>(h, g, k + 1, bc, transposed);
  launch_prolong_add<T>(c, tv<T>(A.P64, A.P32), xc, xa, g.coarse ? lvl_name(kAmgProlong, 3, k) : "famg_transfer");
  for (int s = 0; s < npost; ++s) {
    launch_jacobi<T>(c, Av, d, b, xa, xb, nm);
    std::swap(xa, xb);
  }
  return xa;
}

template <class T>
const T* vcycle_ref(mgr_handle_s& h, MgrLevel& L, const T* b, bool transposed) {
  return vcycle<T>(h, famg_ref(L), 0, b, transposed);
}

template <class T>
void apply_t(mgr_handle_s& h, const double* r, double* z) {
  Ctx& c = h.c;
  unsigned long long l0 = g_launch_count;
  int L = h.L;
  if (L == 0) {  // the whole system is the coarse system
    T* rin = P<T>(h.w_tmp_in);
    if constexpr (std::is_same<T, float>::value) launch_cast_f32(c, 3 * h.nb, r, rin);
    else CU(cudaMemcpyAsync(rin, r, sizeof(double) * 3 * h.nb, cudaMemcpyDeviceToDevice, c.s));
    const T* e = vcycle<T>(h, coarse_ref(h), 0, rin);
    launch_to_f64<T>(c, 3 * h.nb, e, z);
    h.apply_launches = (int64_t)(g_launch_count - l0);
    return;
  }
  MgrLevel& L0 = h.lev[0];
  const T* binv = pick_ptr<T>(h.binv, h.binv32);
  const T* vals = pick_ptr<T>(h.val64, h.val32);
  T* e0 = h.o.global_relax ? P<T>(h.w_e0) : nullptr;
  if (e0) launch_global_relax<T>(c, h.nb, binv, r, e0);
  T* r1 = P<T>(h.w_r[1]);
  T* resF0 = P<T>(h.w_resF0);
  launch_bsr_resid_split<T>(c, h.sell, vals, r, e0, L0.map.p, r1, resF0);
  std::vector<const T*> eF(L);
  eF[0] = frelax<T>(h, 0, resF0, nullptr);
  launch_restrict<T>(c, tv<T>(L0.Acf64, L0.Acf32), nullptr, nullptr, eF[0], r1, kRestrict[0]);
  for (int l = 1; l < L; ++l) {
    MgrLevel& Ll = h.lev[l];
    const T* rl = P<T>(h.w_r[l]);
    eF[l] = frelax<T>(h, l, rl, Ll.F.p);
    launch_restrict<T>(c, tv<T>(Ll.Acf64, Ll.Acf32), Ll.C.p, rl, eF[l], P<T>(h.w_r[l + 1]),
                       lvl_name(kRestrict, 4, l));
  }
  const T* ec = vcycle<T>(h, coarse_ref(h), 0, P<T>(h.w_r[L]));
  for (int l = L - 1; l >= 1; --l) {
    MgrLevel& Ll = h.lev[l];
    T* el = P<T>(h.w_e[l]);
    launch_interp<T, T>(c, Ll.nF, Ll.F.p, Ll.nC, Ll.C.p, tv<T>(Ll.Wp64, Ll.Wp32), eF[l], ec, nullptr, el,
                        lvl_name(kInterp, 4, l));
    ec = el;
  }
  launch_interp<T, double>(c, L0.nF, L0.F.p, L0.nC, L0.C.p, tv<T>(L0.Wp64, L0.Wp32), eF[0], ec, e0, z, kInterp[0]);
  h.apply_launches = (int64_t)(g_launch_count - l0);
}

// The transposed preconditioner.  With s = (I - A B) r, the apply above is
//   M^-1 = B + [S_F^T Phi S_F + P_0 N_1 (S_C - A_cf Phi S_F)] (I - A B)
// (B the block-diagonal relaxation, Phi the F-relaxation, P_0 = S_C^T + S_F^T W_p, N_1 the map of the
// levels below), so
//   M^-T y = g + B^T (y - A^T g),  g = S_C^T t_C + S_F^T Phi^T (y_F - A_cf^T t_C),  t_C = N_1^T (P_0^T y)
// with P_0^T y = y_C + W_p^T y_F; each level applies the same formula recursively and the last one
// the transposed V-cycle.
template <class T>
const T* level_t(mgr_handle_s& h, int l, const T* y) {
  Ctx& c = h.c;
  if (l == h.L) return vcycle<T>(h, coarse_ref(h), 0, y, true);
  MgrLevel& Lv = h.lev[l];
  T* ecin = P<T>(h.w_r[l + 1]);
  launch_gather_add<T>(c, tv<T>(Lv.WpT64, Lv.WpT32), Lv.C.p, y, ecin, lvl_name(kRestrict, 4, l));
  const T* tc = level_t<T>(h, l + 1, ecin);
  T* u = P<T>(h.w_u[l]);
  launch_restrict<T>(c, tv<T>(Lv.AcfT64, Lv.AcfT32), Lv.F.p, y, tc, u, lvl_name(kRestrict, 4, l));
  const T* gF = frelax<T>(h, l, u, nullptr, true);
  T* g = P<T>(h.w_e[l]);
  launch_scatter_cf<T>(c, Lv.nC, Lv.C.p, tc, Lv.nF, Lv.F.p, gF, g);
  return g;
}

template <class T>
void apply_tt(mgr_handle_s& h, const double* y, double* z) {
  Ctx& c = h.c;
  unsigned long long l0 = g_launch_count;
  int64_t n = 3 * h.nb;
  T* yin = P<T>(h.w_tmp_in);
  if constexpr (std::is_same<T, float>::value) launch_cast_f32(c, n, y, yin);
  else CU(cudaMemcpyAsync(yin, y, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.s));
  const T* g = (h.L == 0) ? vcycle<T>(h, coarse_ref(h), 0, yin, true) : level_t<T>(h, 0, yin);
  if (h.L > 0 && h.o.global_relax) {
    launch_bsr_grt<T>(c, h.sellT, pick_ptr<T>(h.valT64, h.valT32), y, g, pick_ptr<T>(h.binvT64, h.binvT32), z);
  } else {
    launch_to_f64<T>(c, n, g, z);
  }
  h.apply_launches = (int64_t)(g_launch_count - l0);
}

void do_apply_t(mgr_handle_s& h, const double* r, double* z) {
  if (!h.has_t) throw Error(MGR_ERR_STATE, "the handle was set up without options.adjoint");
  if (h.o.precision == MGR_PREC_MIXED) apply_tt<float>(h, r, z);
  else apply_tt<double>(h, r, z);
}

// Systems of at most this many unknowns replay the forward apply as a CUDA graph by default: their
// apply is a chain of small kernels bound by launch overhead.
constexpr int64_t APPLY_GRAPH_AUTO_MAX = int64_t(1) << 21;

void reset_graph(mgr_handle_s& h) {
  if (h.gexec) {
    cudaStreamSynchronize(h.c.s);  // no replay in flight
    cudaGraphExecDestroy(h.gexec);
  }
  h.gexec = nullptr;
  h.g_launches = 0;
  h.applies = 0;
  h.graph_failed = false;
}

bool graph_wanted(const mgr_handle_s& h) {
  if (h.c.prof || h.graph_failed || h.o.apply_graph < 0) return false;
  return h.o.apply_graph > 0 || 3 * h.nb <= APPLY_GRAPH_AUTO_MAX;
}

// Capture one forward apply from g_in to g_out on a private stream (the caller's stream may be the
// legacy default stream, which cannot capture); on any failure the handle keeps launching directly.
template <class T>
void capture_apply(mgr_handle_s& h) {
  Ctx& c = h.c;
  const int64_t n = 3 * h.nb;
  h.g_in.alloc(c, n);
  h.g_out.alloc(c, n);
  if (!h.gstream) CU(cudaStreamCreateWithFlags(&h.gstream, cudaStreamNonBlocking));
  cudaStream_t s0 = c.s;
  const unsigned long long l0 = g_launch_count;
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(h.gstream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  if (ok) {
    c.s = h.gstream;
    try {
      apply_t<T>(h, h.g_in.p, h.g_out.p);
    } catch (...) {
      ok = false;
    }
    c.s = s0;
    ok = (cudaStreamEndCapture(h.gstream, &graph) == cudaSuccess) && ok && graph;
  }
  g_launch_count = l0;  // nothing ran
  if (ok) ok = cudaGraphInstantiate(&h.gexec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    h.gexec = nullptr;
    h.graph_failed = true;
    cudaGetLastError();
    return;
  }
  h.g_launches = h.apply_launches;
}

void do_apply(mgr_handle_s& h, const double* r, double* z) {
  const bool mixed = h.o.precision == MGR_PREC_MIXED;
  ProfScope whole(h.c, "mgr_apply");  // the whole preconditioner application
  // the first apply after a setup runs directly (it also settles the launch-shape caches); the
  // second captures the graph, and later ones replay it
  if (graph_wanted(h) && h.applies++ >= 1) {
    if (!h.gexec) {
      if (mixed) capture_apply<float>(h);
      else capture_apply<double>(h);
    }
    if (h.gexec) {
      Ctx& c = h.c;
      const size_t bytes = sizeof(double) * 3 * h.nb;
      CU(cudaMemcpyAsync(h.g_in.p, r, bytes, cudaMemcpyDeviceToDevice, c.s));
      CU(cudaGraphLaunch(h.gexec, c.s));
      g_launch_count += (unsigned long long)h.g_launches;
      CU(cudaMemcpyAsync(z, h.g_out.p, bytes, cudaMemcpyDeviceToDevice, c.s));
      return;
    }
  }
  if (mixed) apply_t<float>(h, r, z);
  else apply_t<double>(h, r, z);
}

// ---- setup -----------------------------------------------------------------------------------
__global__ void k_max_marker(int64_t n, const int8_t* mk, int* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) atomicMax(out, (int)mk[i]);
}

void alloc_work(mgr_handle_s& h) {
  Ctx& c = h.c;
  size_t es = (h.o.precision == MGR_PREC_MIXED) ? sizeof(float) : sizeof(double);
  int L = h.L;
  h.w_r.clear(); h.w_e.clear(); h.w_eF.clear(); h.w_eF2.clear();
  h.w_r.resize(L + 1); h.w_e.resize(L + 1); h.w_eF.resize(L + 1); h.w_eF2.resize(L + 1);
  h.w_e0.alloc(c, es * 3 * h.nb);
  h.w_tmp_in.alloc(c, es * 3 * h.nb);
  for (int l = 0; l <= L; ++l) {
    int64_t n = h.lev[l].n;
    h.w_r[l].alloc(c, es * n);
    h.w_e[l].alloc(c, es * n);
    if (l < L) {
      h.w_eF[l].alloc(c, es * (h.lev[l].nF + 1));
      h.w_eF2[l].alloc(c, es * (h.lev[l].nF + 1));
    }
  }
  h.w_resF0.alloc(c, es * ((L > 0 ? h.lev[0].nF : 0) + 1));
  for (int l = 0; l < L; ++l) {
    MgrLevel& Lv = h.lev[l];
    size_t nf = Lv.famg.size();
    Lv.fa_b.clear(); Lv.fa_xa.clear(); Lv.fa_xb.clear(); Lv.fa_res.clear();
    if (nf == 0) continue;
    Lv.fa_b.resize(nf); Lv.fa_xa.resize(nf); Lv.fa_xb.resize(nf); Lv.fa_res.resize(nf);
    for (size_t k = 0; k < nf; ++k) {
      int64_t nk = Lv.famg[k].n;
      Lv.fa_b[k].alloc(c, es * nk);
      Lv.fa_xa[k].alloc(c, es * nk);
      Lv.fa_xb[k].alloc(c, es * nk);
      Lv.fa_res[k].alloc(c, es * nk);
    }
    Lv.w_fsrc.alloc(c, es * (Lv.nF + 1));
    Lv.w_fres.alloc(c, es * (Lv.nF + 1));
  }
  h.w_u.clear();
  if (h.o.adjoint) {
    h.w_u.resize(L + 1);
    for (int l = 0; l < L; ++l) h.w_u[l].alloc(c, es * (h.lev[l].nF + 1));
  }
  size_t na = std::max<size_t>(h.amg.size(), 1);
  h.a_b.clear(); h.a_xa.clear(); h.a_xb.clear(); h.a_res.clear();
  h.a_b.resize(na); h.a_xa.resize(na); h.a_xb.resize(na); h.a_res.resize(na);
  for (size_t k = 0; k < na; ++k) {
    int64_t n = h.amg.empty() ? h.nco : h.amg[k].n;
    h.a_b[k].alloc(c, es * n);
    h.a_xa[k].alloc(c, es * n);
    h.a_xb[k].alloc(c, es * n);
    h.a_res[k].alloc(c, es * n);
  }
}

// Frees the buffers of a setup-only matrix; its shape stays for introspection.
void release_csr(DCSR<double>& M) {
  M.rp.release();
  M.ci.release();
  M.v.release();
}

// The apply operators of MGR level l in the working precision (SELL or CSR copies of A_ff, A_cf, W_p).
void cast_mgr_level(mgr_handle_s& h, MgrLevel& L, Ctx& c) {
  if (L.cast) return;
  if (h.o.precision == MGR_PREC_MIXED) {
    rowsop_build<float>(c, L.Aff, L.Aff32);
    rowsop_build<float>(c, L.Acf, L.Acf32);
    rowsop_build<float>(c, L.Wp, L.Wp32);
    L.minv32.alloc(c, L.nF + 1);
    launch_cast_f32(c, L.nF, L.minv.p, L.minv32.p);
  } else {
    rowsop_build<double>(c, L.Aff, L.Aff64);
    rowsop_build<double>(c, L.Acf, L.Acf64);
    rowsop_build<double>(c, L.Wp, L.Wp64);
  }
  if (h.o.adjoint) {
    // W_p^T (its columns renumbered from F positions to level dofs, so it reads the level vector),
    // A_cf^T, A_ff^T
    DCSR<double> WpT, AcfT, AffT;
    transpose(c, L.Wp, WpT);
    launch_map_cols(c, WpT.nnz, WpT.ci.p, L.F.p);
    WpT.nc = L.n;
    transpose(c, L.Acf, AcfT);
    transpose(c, L.Aff, AffT);
    if (h.o.precision == MGR_PREC_MIXED) {
      rowsop_build<float>(c, WpT, L.WpT32);
      rowsop_build<float>(c, AcfT, L.AcfT32);
      rowsop_build<float>(c, AffT, L.AffT32);
    } else {
      rowsop_build<double>(c, WpT, L.WpT64);
      rowsop_build<double>(c, AcfT, L.AcfT64);
      rowsop_build<double>(c, AffT, L.AffT64);
    }
  }
  L.cast = true;
}

void cast_amg_level(mgr_handle_s& h, AmgLevel& G, Ctx& c) {
  if (G.cast) return;
  if (h.o.precision == MGR_PREC_MIXED) {
    rowsop_build<float>(c, G.A, G.A32);
    rowsop_build<float>(c, G.P, G.P32);
    rowsop_build<float>(c, G.R, G.R32);
    G.dinv32.alloc(c, G.n);
    launch_cast_f32(c, G.n, G.dinv.p, G.dinv32.p);
  } else {
    rowsop_build<double>(c, G.A, G.A64);
    rowsop_build<double>(c, G.P, G.P64);
    rowsop_build<double>(c, G.R, G.R64);
  }
  if (h.o.adjoint) {
    DCSR<double> AT;
    transpose(c, G.A, AT);
    if (h.o.precision == MGR_PREC_MIXED) rowsop_build<float>(c, AT, G.AT32);
    else rowsop_build<double>(c, AT, G.AT64);
  }
  G.cast = true;
}

void rehome_amg_level(AmgLevel& G, Ctx& c) {
  rowsop_rehome(G.A32, c); rowsop_rehome(G.P32, c); rowsop_rehome(G.R32, c);
  rowsop_rehome(G.A64, c); rowsop_rehome(G.P64, c); rowsop_rehome(G.R64, c);
  rowsop_rehome(G.AT32, c); rowsop_rehome(G.AT64, c);
  G.dinv32.c = &c;
}

// The apply copies that depend on the MGR levels only: A's values in the sliced layout (and the
// block inverses in FP32) and every MGR level's operators (with the F-relaxation AMG levels).
void cast_mgr_part(mgr_handle_s& h, const mgr_bsr3_t& A, Ctx& c) {
  int64_t nv = 9 * SELL_C * h.sell.slots;
  bool mixed = h.o.precision == MGR_PREC_MIXED;
  if (mixed) {
    h.val32.alloc(c, nv);
    sell_fill_values<double, float>(c, h.sell, A.values, h.val32.p);
    h.binv32.alloc(c, 9 * h.nb);
    launch_cast_f32(c, 9 * h.nb, h.binv.p, h.binv32.p);
  } else {
    h.val64.alloc(c, nv);
    sell_fill_values<double, double>(c, h.sell, A.values, h.val64.p);
  }
  for (int l = 0; l < h.L; ++l) {
    cast_mgr_level(h, h.lev[l], c);
    for (size_t k = 0; k + 1 < h.lev[l].famg.size(); ++k) cast_amg_level(h, h.lev[l].famg[k], c);
  }
}

// Hands the buffers built by cast_mgr_part on context `from` over to the handle's main context.
void rehome_mgr_part(mgr_handle_s& h) {
  Ctx& c = h.c;
  h.val32.c = &c; h.binv32.c = &c; h.val64.c = &c; h.binv.c = &c;
  h.sell.soff.c = &c; h.sell.col.c = &c; h.sell.src.c = &c;
  for (int l = 0; l < h.L; ++l) {
    MgrLevel& L = h.lev[l];
    rowsop_rehome(L.Aff32, c); rowsop_rehome(L.Acf32, c); rowsop_rehome(L.Wp32, c);
    rowsop_rehome(L.Aff64, c); rowsop_rehome(L.Acf64, c); rowsop_rehome(L.Wp64, c);
    rowsop_rehome(L.WpT32, c); rowsop_rehome(L.AcfT32, c); rowsop_rehome(L.AffT32, c);
    rowsop_rehome(L.WpT64, c); rowsop_rehome(L.AcfT64, c); rowsop_rehome(L.AffT64, c);
    L.minv32.c = &c;
    for (size_t k = 0; k + 1 < L.famg.size(); ++k) rehome_amg_level(L.famg[k], c);
  }
}

void cast_hierarchy(mgr_handle_s& h, const mgr_bsr3_t& A, bool mgr_part) {
  Ctx& c = h.c;
  bool mixed = h.o.precision == MGR_PREC_MIXED;
  if (mgr_part) cast_mgr_part(h, A, c);
  for (size_t k = 0; k + 1 < h.amg.size(); ++k) cast_amg_level(h, h.amg[k], c);
  if (h.o.adjoint) {
    // A^T in the sliced layout (its src renumbered to A's blocks, values transposed block by block),
    // the transposed diagonal-block inverses and the transposed coarsest inverse
    DBuf<int64_t> rpt(c, h.nb + 1), srcT(c, h.nnzb);
    DBuf<int32_t> cit(c, h.nnzb);
    launch_bsr3_transpose_pattern(c, A, rpt.p, cit.p, srcT.p);
    sell_build_pattern(c, h.nb, h.nnzb, rpt.p, cit.p, h.sellT);
    sell_compose_src(c, h.sellT, srcT.p);
    int64_t nvt = 9 * SELL_C * h.sellT.slots;
    if (mixed) {
      h.valT32.alloc(c, nvt);
      sell_fill_values_t<double, float>(c, h.sellT, A.values, h.valT32.p);
      h.binvT32.alloc(c, 9 * h.nb);
      launch_transpose_blocks<float>(c, h.nb, h.binv32.p, h.binvT32.p);
    } else {
      h.valT64.alloc(c, nvt);
      sell_fill_values_t<double, double>(c, h.sellT, A.values, h.valT64.p);
      h.binvT64.alloc(c, 9 * h.nb);
      launch_transpose_blocks<double>(c, h.nb, h.binv.p, h.binvT64.p);
    }
    h.cinvT.alloc(c, (size_t)h.nco * h.nco);
    launch_dense_transpose(c, h.nco, h.cinv.p, h.cinvT.p);
    h.has_t = true;
  }
}

AmgOpts amg_opts(const mgr_options_t& o) {
  AmgOpts ao;
  ao.theta = o.amg_theta;
  ao.max_levels = o.amg_max_levels;
  ao.max_coarse = o.amg_max_coarse;
  ao.smoother = o.amg_smoother;
  ao.pre = o.amg_pre;
  ao.post = o.amg_post;
  ao.pmax = o.amg_pmax;
  ao.omega = o.amg_omega;
  ao.seed = o.amg_seed;
  return ao;
}

// frelax_type 2: the AMG hierarchy of the level's A_ff (same settings as the coarse solver, V(1,1),
// PMIS seed amg_seed + 7919 (l + 1)) with its coarsest inverse (and transpose for M^-T)
void build_famg(mgr_handle_s& h, int l) {
  Ctx& c = h.c;
  MgrLevel& L = h.lev[l];
  if (L.nF == 0) return;
  AmgOpts af = amg_opts(h.o);
  af.seed = h.o.amg_seed + 7919ull * (uint64_t)(l + 1);
  af.pre = af.post = 1;
  ProfScope ps(c, "setup_famg");
  if (h.o.lean) {
    amg_build(c, L.Aff, false, af, L.famg, L.fcinv, L.fnco, [&](AmgLevel& G) {
      cast_amg_level(h, G, c);
      release_csr(G.A);
      release_csr(G.P);
      release_csr(G.R);
      release_csr(G.S);
    });
  } else {
    amg_build(c, L.Aff, false, af, L.famg, L.fcinv, L.fnco, nullptr);
  }
  if (h.o.adjoint) {
    L.fcinvT.alloc(c, (size_t)L.fnco * L.fnco);
    launch_dense_transpose(c, L.fnco, L.fcinv.p, L.fcinvT.p);
  }
}

void do_setup(mgr_handle_s& h, const mgr_bsr3_t& A, const int8_t* marker) {
  auto t0 = std::chrono::steady_clock::now();
  Ctx& c = h.c;
  h.ready = false;
  reset_graph(h);
  h.lev.clear();
  h.amg.clear();
  h.cinv.release();
  h.val32.release(); h.val64.release(); h.binv32.release();
  h.has_t = false;
  h.valT32.release(); h.valT64.release(); h.binvT32.release(); h.binvT64.release(); h.cinvT.release();
  h.kry_valsT.release();
  ProfScope ps_all(c, "setup_total");
  // one batch for the products of a mid-size problem; the lean setup keeps the staging small
  c.spgemm_stage = h.o.spgemm_stage > 1024 ? h.o.spgemm_stage : (h.o.lean ? (int64_t(1) << 27) : (int64_t(1) << 29));
  // the pattern and marker checks and the number of reductions (the largest marker) with one wait
  bsr3_validate_launch(c, A, marker);
  int L;
  {
    DBuf<int> mx(c, 1);
    CU(cudaMemsetAsync(mx.p, 0, sizeof(int), c.s));
    k_max_marker<<<grid_for(3 * A.nb, 256), 256, 0, c.s>>>(3 * A.nb, marker, mx.p);
    CU_LAUNCH();
    int err = 0;
    read_back(c, {{c.d_err, &err, sizeof(int)}, {mx.p, &L, sizeof(int)}});
    if (err) check_errors(c, "bsr3_validate");
  }
  h.nb = A.nb;
  h.nnzb = A.nnzb;
  int64_t n = 3 * A.nb;
  // pattern copy (the apply reads the pattern; the caller may free A after setup)
  h.rp0.alloc(c, A.nb + 1);
  h.ci0.alloc(c, A.nnzb);
  CU(cudaMemcpyAsync(h.rp0.p, A.rowptr, sizeof(int64_t) * (A.nb + 1), cudaMemcpyDeviceToDevice, c.s));
  CU(cudaMemcpyAsync(h.ci0.p, A.colind, sizeof(int32_t) * A.nnzb, cudaMemcpyDeviceToDevice, c.s));
  // Without the lean setup the apply copies are built by a second host thread on the second
  // context's stream while this thread carries on with the hierarchy: first those of the MGR levels
  // (and A's sliced values), which depend on nothing the coarse solver builds, then those of each
  // AMG level as soon as the next level has been built from it.  Both threads mostly issue launches
  // and wait for read-backs, which leaves the GPU room for both.  The buffers are handed over to
  // the main context once the thread has joined.
  struct Tasks {
    std::mutex m;
    std::condition_variable cv;
    std::deque<std::function<void()>> q;
    bool closed = false;
  } tasks;
  std::thread caster;
  std::exception_ptr caster_err;
  struct Joiner {
    Tasks& tk;
    std::thread& t;
    ~Joiner() {
      {
        std::lock_guard<std::mutex> g(tk.m);
        tk.closed = true;
      }
      tk.cv.notify_all();
      if (t.joinable()) t.join();
    }
  } joiner{tasks, caster};
  const bool overlap = !h.o.lean;
  // a task for the caster, ordered after everything issued so far on the main stream
  auto post = [&](std::function<void()> fn) {
    cudaEvent_t ev = nullptr;
    CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CU(cudaEventRecord(ev, c.s));
    {
      std::lock_guard<std::mutex> g(tasks.m);
      tasks.q.push_back([&h, ev, fn] {
        CU(cudaStreamWaitEvent(h.cw.s, ev, 0));
        CU(cudaEventDestroy(ev));
        fn();
      });
    }
    tasks.cv.notify_one();
  };
  if (overlap) {
    Ctx& w = h.cw;
    if (!w.s) CU(cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking));
    if (!w.d_err) {
      CU(cudaMalloc(&w.d_err, sizeof(int)));
      CU(cudaMemsetAsync(w.d_err, 0, sizeof(int), c.s));
    }
    w.h_pinned = h.hpin + 512 - PIN_SLOTS;
    w.prof = nullptr;
    w.spgemm_stage = c.spgemm_stage;
    w.num_sms = c.num_sms;
    w.pdl = c.pdl;
    w.acct = &c;
    w.mu = &h.acct_mu;
    c.mu = &h.acct_mu;
    caster = std::thread([&h, &tasks, &caster_err, dev = h.device] {
      try {
        CU(cudaSetDevice(dev));
        for (;;) {
          std::function<void()> fn;
          {
            std::unique_lock<std::mutex> g(tasks.m);
            tasks.cv.wait(g, [&] { return tasks.closed || !tasks.q.empty(); });
            if (tasks.q.empty()) break;
            fn = std::move(tasks.q.front());
            tasks.q.pop_front();
          }
          if (!caster_err) fn();
        }
        CU(cudaStreamSynchronize(h.cw.s));
        check_errors(h.cw, "apply copies");
      } catch (...) {
        caster_err = std::current_exception();
        cudaStreamSynchronize(h.cw.s);
      }
    });
  }
  // the sliced layout of A's pattern and the 3x3 block inverses are read by the apply and the Krylov
  // products only: with the caster they are built on its stream while the MGR levels are set up
  auto build_sell_binv = [&h, &A](Ctx& x) {
    sell_build_pattern(x, A.nb, A.nnzb, A.rowptr, A.colind, h.sell);
    h.binv.alloc(x, 9 * A.nb);
    bsr3_block_inverse(x, A, h.binv.p);
    check_errors(x, "3x3 diagonal blocks");
  };
  if (overlap) post([&h, build_sell_binv] { build_sell_binv(h.cw); });
  else build_sell_binv(c);
  h.L = L;
  h.lev.resize(L + 1);
  h.lev[0].n = n;
  bsr3_to_csr(c, A, h.lev[0].A);
  h.lev[0].mk.alloc(c, n);
  CU(cudaMemcpyAsync(h.lev[0].mk.p, marker, n, cudaMemcpyDeviceToDevice, c.s));
  for (int l = 0; l < L; ++l) {
    LevelOpts lo;
    lo.frelax_type = h.o.frelax_type[l];
    lo.sweeps = h.o.frelax_sweeps[l];
    lo.omega = h.o.frelax_omega[l];
    lo.restrict_type = h.o.restrict_type[l];
    DBuf<int8_t> mk_next;
    ProfScope ps(c, "setup_mgr_level");
    mgr_reduce_level(c, h.lev[l], l, lo, h.lev[l + 1].A, mk_next);
    h.lev[l + 1].n = h.lev[l].nC;
    h.lev[l + 1].mk = std::move(mk_next);
    if (h.o.frelax_type[l] == 2) build_famg(h, l);
    if (h.o.lean) {  // the level's FP64 operators are not read again
      MgrLevel& Lv = h.lev[l];
      cast_mgr_level(h, Lv, c);
      release_csr(Lv.A);
      release_csr(Lv.Wp);
      release_csr(Lv.Wr);
      release_csr(Lv.P);
      release_csr(Lv.R);
      release_csr(Lv.Aff);
      release_csr(Lv.Acf);
    }
  }
  if (overlap) post([&h, &A] { cast_mgr_part(h, A, h.cw); });
  // coarse solve on the last level
  DCSR<double>& Ac = h.lev[L].A;
  if (h.o.coarse_solver == 1) {
    if (Ac.nr > 4096) throw Error(MGR_ERR_UNSUPPORTED, "dense coarse solve limited to 4096 rows");
    h.coarse_dense = true;
    h.nco = Ac.nr;
    dense_inverse(c, Ac, h.cinv);
    check_errors(c, "dense coarse inverse");
  } else {
    h.coarse_dense = false;
    const AmgOpts ao = amg_opts(h.o);
    ProfScope ps(c, "setup_amg");
    if (h.o.lean) {
      // the AMG takes the pressure operator over, and each level's FP64 matrices are freed once the
      // next level is built
      amg_build(c, h.lev[L].A, true, ao, h.amg, h.cinv, h.nco, [&](AmgLevel& G) {
        cast_amg_level(h, G, c);
        release_csr(G.A);
        release_csr(G.P);
        release_csr(G.R);
        release_csr(G.S);
      });
    } else {
      h.amg.reserve(64 + (size_t)std::max(0, h.o.amg_max_levels));  // the caster holds references to levels
      amg_build(c, h.lev[L].A, false, ao, h.amg, h.cinv, h.nco, [&](AmgLevel& G) {
        AmgLevel* g = &G;
        post([&h, g] { cast_amg_level(h, *g, h.cw); });
      });
    }
  }
  if (overlap) {
    {
      std::lock_guard<std::mutex> g(tasks.m);
      tasks.closed = true;
    }
    tasks.cv.notify_all();
    caster.join();
    c.mu = nullptr;
    rehome_mgr_part(h);
    for (AmgLevel& G : h.amg) rehome_amg_level(G, c);
    if (caster_err) std::rethrow_exception(caster_err);
  }
  {
    ProfScope ps(c, "setup_cast_alloc");
    cast_hierarchy(h, A, !overlap);
    alloc_work(h);
  }
  host_wait(c);
  h.ready = true;
  h.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// ---- flexible GMRES ----------------------------------------------------------------------------
// Krylov basis storage: vector k starts at k * ld with ld = n rounded up to 256 doubles plus 160, so
// successive vectors are staggered by 1280 bytes across the HBM channels instead of aliasing at a
// large power-of-two stride; ld is even, so every vector is 16-byte aligned for paired loads.
void ensure_krylov(mgr_handle_s& h, int m, int64_t n) {
  if (h.kry_m == m && h.kry_n == n) return;
  Ctx& c = h.c;
  int64_t ld = ((n + 255) / 256) * 256 + 160;
  h.V.alloc(c, (size_t)(m + 1) * ld);
  h.Z.alloc(c, (size_t)m * ld);
  h.part.alloc(c, (size_t)KRY_PART);
  h.dsc.alloc(c, 256);
  h.kry_m = m;
  h.kry_n = n;
  h.kry_ld = ld;
}

// tr: solve A^T x = b with the transposed preconditioner M^-T, applied from the left: GMRES(m) on
// M^-T A^T x = M^-T b, the transpose of the forward right-preconditioned operator A M^-1 (with M^-T on
// the right, (M^-1 A)^T, restarted GMRES stalls on the layered workloads where the forward solve
// converges).  Each cycle starts from the true residual; the inner iteration stops when the
// preconditioned residual estimate reaches rtol ||b|| scaled by the preconditioned-to-true ratio at
// the cycle start, and the true residual decides convergence.
mgr_status_t do_fgmres(mgr_handle_s& h, const mgr_bsr3_t& A, const double* b, double* x, double rtol, int m, int maxit,
                       mgr_solve_info_t* info, bool tr = false) {
  auto t0 = std::chrono::steady_clock::now();
  Ctx& c = h.c;
  int64_t n = 3 * A.nb;
  ensure_krylov(h, m, n);
  double* hp = h.hpin;  // pinned: [0..63] readbacks
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m);
  mgr_solve_info_t loc;
  memset(&loc, 0, sizeof loc);
  auto rd = [&](const double* d, int cnt) {
    CU(cudaMemcpyAsync(hp, d, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c.s));
    host_wait(c);
  };
  double* V = h.V.p;
  double* Z = h.Z.p;
  const int64_t ld = h.kry_ld;
  // A's (or A^T's) values in the sliced layout (the pattern is the one given to mgr_setup)
  const SellPattern& SP = tr ? h.sellT : h.sell;
  DBuf<double>& KV = tr ? h.kry_valsT : h.kry_vals;
  KV.alloc(c, 9 * SELL_C * SP.slots);
  if (tr) sell_fill_values_t<double, double>(c, SP, A.values, KV.p);
  else sell_fill_values<double, double>(c, SP, A.values, KV.p);
  auto spmv = [&](const double* xx, const double* sub, double* yy) {
    launch_sell_spmv_f64(c, SP, KV.p, xx, sub, yy);
  };
  double* dsc = h.dsc.p;
  mgr_status_t st = MGR_OK;
  launch_nrm2sq(c, n, b, h.part.p, dsc);
  rd(dsc, 1);
  double bnorm = std::sqrt(hp[0]);
  loc.bnorm = bnorm;
  int it = 0;
  if (bnorm == 0.0) {
    CU(cudaMemsetAsync(x, 0, sizeof(double) * n, c.s));
    loc.converged = 1;
  } else {
    spmv(x, b, V);  // r = b - A x
    launch_nrm2sq(c, n, V, h.part.p, dsc);
    rd(dsc, 1);
    double beta = std::sqrt(hp[0]);
    if (info && info->history && info->history_cap > 0) info->history[0] = beta / bnorm;
    loc.relres_true = loc.relres_est = beta / bnorm;
    if (beta <= rtol * bnorm) loc.converged = 1;
    // Re-orthogonalise when ||w - V h|| < eta ||w||.  One classical Gram-Schmidt pass leaves w - V h
    // non-orthogonal to V by about eps ||w|| / ||w - V h||, and the Pythagorean norm ||w||^2 - ||h||^2
    // has relative error about eps ||w||^2 / ||w - V h||^2; eta = 0.3 bounds these by 3.3 eps and
    // 11 eps.  The classical 1/sqrt(2) fires on nearly every step with a strong preconditioner
    // (A M^-1 v_j is close to v_j, inside the basis); below 0.1 the Givens estimate was seen to run
    // ahead of the true residual on a 2-D case and force a restart.
    const double eta = 0.3;
    const bool left = tr;
    while (!loc.converged) {
      double scale = 1.0;  // true / preconditioned residual norm at the cycle start (left)
      double beta_k = beta;
      if (left) {
        CU(cudaMemcpyAsync(Z, V, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.s));
        do_apply_t(h, Z, V);
        launch_nrm2sq(c, n, V, h.part.p, dsc);
        rd(dsc, 1);
        beta_k = std::sqrt(hp[0]);
        if (!(beta_k > 0.0) || !std::isfinite(beta_k)) { st = MGR_ERR_BREAKDOWN; break; }
        scale = beta / beta_k;
      }
      launch_scal(c, n, 1.0 / beta_k, V, V);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta_k;
      int k = 0;
      bool stop = false;
      for (int j = 0; j < m && it < maxit; ++j) {
        double* vj = V + (int64_t)j * ld;
        double* zj = Z + (int64_t)j * ld;
        double* w = V + (int64_t)(j + 1) * ld;
        if (left) {
          spmv(vj, nullptr, Z);  // Z's first column as scratch: the left form needs no Z basis
          do_apply_t(h, Z, w);
        } else {
          do_apply(h, vj, zj);
          spmv(zj, nullptr, w);
        }
        // classical Gram-Schmidt: h = V^T w and w.w in one pass; the norm of w - V h follows from
        // Pythagoras; when it drops below eta ||w|| a second pass re-orthogonalises
        launch_mdot(c, n, V, ld, j + 1, w, true, h.part.p, dsc);
        launch_pyth_scale(c, j + 1, dsc, dsc + j + 1, dsc + 64);
        rd(dsc, 66);
        double hcol[KRY_MAXV + 2];
        for (int i = 0; i <= j; ++i) hcol[i] = hp[i];
        double ww = hp[j + 1], nrm2 = hp[64];
        double nw;
        if (nrm2 >= eta * eta * ww && std::isfinite(nrm2)) {
          launch_mupdate(c, n, V, ld, j + 1, dsc, dsc + 65, w, w, h.part.p, nullptr);
          nw = std::sqrt(nrm2);
        } else {
          launch_mupdate(c, n, V, ld, j + 1, dsc, nullptr, w, w, h.part.p, nullptr);
          launch_mdot(c, n, V, ld, j + 1, w, true, h.part.p, dsc + 96);
          launch_pyth_scale(c, j + 1, dsc + 96, dsc + 96 + j + 1, dsc + 160);
          CU(cudaMemcpyAsync(hp + 96, dsc + 96, sizeof(double) * 66, cudaMemcpyDeviceToHost, c.s));
          host_wait(c);
          for (int i = 0; i <= j; ++i) hcol[i] += hp[96 + i];
          double n2 = hp[96 + 64];
          nw = n2 > 0.0 ? std::sqrt(n2) : 0.0;
          launch_mupdate(c, n, V, ld, j + 1, dsc + 96, dsc + 161, w, w, h.part.p, nullptr);
        }
        if (!std::isfinite(nw)) { st = MGR_ERR_BREAKDOWN; stop = true; break; }
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
        H[(size_t)(j + 1) * m + j] = nw;
        for (int i = 0; i < j; ++i) {
          double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
          H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
        }
        double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
        double den = std::sqrt(a * a + bb * bb);
        if (den == 0.0 || !std::isfinite(den)) { st = MGR_ERR_BREAKDOWN; stop = true; break; }
        cs[j] = a / den;
        sn[j] = bb / den;
        H[(size_t)j * m + j] = den;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++it;
        k = j + 1;
        if (info && info->history && it < info->history_cap) info->history[it] = scale * std::fabs(g[j + 1]) / bnorm;
        if (scale * std::fabs(g[j + 1]) <= rtol * bnorm || nw == 0.0) break;
      }
      if (stop) break;
      for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int t = i + 1; t < k; ++t) s -= H[(size_t)i * m + t] * y[t];
        y[i] = s / H[(size_t)i * m + i];
      }
      if (k > 0) {
        memcpy(hp + 200, y.data(), sizeof(double) * k);
        CU(cudaMemcpyAsync(dsc + 200, hp + 200, sizeof(double) * k, cudaMemcpyHostToDevice, c.s));
        launch_xupdate(c, n, left ? V : Z, ld, k, dsc + 200, x);
      }
      loc.relres_est = (k > 0) ? scale * std::fabs(g[k]) / bnorm : beta / bnorm;
      spmv(x, b, V);
      launch_nrm2sq(c, n, V, h.part.p, dsc);
      rd(dsc, 1);
      beta = std::sqrt(hp[0]);
      loc.relres_true = beta / bnorm;
      if (beta <= rtol * bnorm) { loc.converged = 1; break; }
      if (!std::isfinite(beta)) { st = MGR_ERR_BREAKDOWN; break; }
      if (it >= maxit) { st = MGR_ERR_NOT_CONVERGED; break; }
      loc.restarts++;
    }
  }
  host_wait(c);
  loc.iterations = it;
  loc.status = st;
  loc.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) {
    double* hist = info->history;
    int cap = info->history_cap;
    *info = loc;
    info->history = hist;
    info->history_cap = cap;
  }
  return st;
}

// ---- introspection -----------------------------------------------------------------------------
const DCSR<double>* pick_matrix(mgr_handle_s& h, int kind, int level) {
  if (kind >= 0 && kind <= 4) {
    if (level < 0 || level > h.L || (kind > 0 && level >= h.L)) return nullptr;
    MgrLevel& L = h.lev[level];
    switch (kind) {
      case 0: return &L.A;
      case 1: return &L.Wp;
      case 2: return &L.Wr;
      case 3: return &L.P;
      default: return &L.R;
    }
  }
  int na = (int)h.amg.size();
  if (kind < 5 || kind > 8 || level < 0 || level >= na) return nullptr;
  if (kind > 5 && level >= na - 1) return nullptr;
  AmgLevel& G = h.amg[level];
  switch (kind) {
    case 5: return &G.A;
    case 6: return &G.P;
    case 7: return &G.R;
    default: return &G.S;
  }
}

__global__ void k_fill_one(int64_t n, double* v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] = 1.0;
}
template <class S>
__global__ void k_to_double(int64_t n, const S* a, double* b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

}  // namespace

// =================================== C ABI ======================================================
extern "C" {

const char* mgr_status_string(mgr_status_t s) {
  switch (s) {
    case MGR_OK: return "MGR_OK";
    case MGR_ERR_INVALID_ARG: return "MGR_ERR_INVALID_ARG";
    case MGR_ERR_SINGULAR: return "MGR_ERR_SINGULAR";
    case MGR_ERR_NOT_CONVERGED: return "MGR_ERR_NOT_CONVERGED";
    case MGR_ERR_BREAKDOWN: return "MGR_ERR_BREAKDOWN";
    case MGR_ERR_OOM: return "MGR_ERR_OOM";
    case MGR_ERR_CUDA: return "MGR_ERR_CUDA";
    case MGR_ERR_TIMEOUT: return "MGR_ERR_TIMEOUT";
    case MGR_ERR_STATE: return "MGR_ERR_STATE";
    case MGR_ERR_UNSUPPORTED: return "MGR_ERR_UNSUPPORTED";
  }
  return "MGR_ERR_UNKNOWN";
}

void mgr_options_default(mgr_options_t* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->precision = MGR_PREC_FP64;
  o->global_relax = 1;
  for (int l = 0; l < MGR_MAX_LEVELS; ++l) {
    o->frelax_type[l] = (l == 0) ? 0 : 1;
    o->frelax_sweeps[l] = (l == 0) ? 1 : 2;
    o->frelax_omega[l] = 1.0;
    o->restrict_type[l] = (l == 0) ? 1 : 0;
  }
  o->apply_full_R = 0;
  o->coarse_solver = 0;
  o->amg_theta = 0.25;
  o->amg_max_levels = 25;
  o->amg_max_coarse = 256;
  o->amg_smoother = 1;
  o->amg_pre = 1;
  o->amg_post = 1;
  o->amg_pmax = 0;
  o->amg_omega = 1.0;
  o->amg_seed = 3;
}

static mgr_status_t check_options(const mgr_options_t& o) {
  if (o.precision != MGR_PREC_FP64 && o.precision != MGR_PREC_MIXED) return MGR_ERR_INVALID_ARG;
  for (int l = 0; l < MGR_MAX_LEVELS; ++l) {
    if (o.frelax_sweeps[l] < 1 || o.frelax_sweeps[l] > 64) return MGR_ERR_INVALID_ARG;
    if (o.frelax_type[l] < 0 || o.frelax_type[l] > 2) return MGR_ERR_INVALID_ARG;
    if (o.restrict_type[l] < 0 || o.restrict_type[l] > 1) return MGR_ERR_INVALID_ARG;
  }
  if (o.apply_full_R != 0) return MGR_ERR_UNSUPPORTED;
  if (o.amg_pre < 1 || o.amg_post < 0 || o.amg_max_levels < 1 || o.amg_max_coarse < 1 || o.amg_max_coarse > 4096)
    return MGR_ERR_INVALID_ARG;
  if (o.amg_smoother < 0 || o.amg_smoother > 1 || o.amg_pmax < 0) return MGR_ERR_INVALID_ARG;
  if (o.apply_graph < -1 || o.apply_graph > 1) return MGR_ERR_INVALID_ARG;
  if (o.pdl < -1 || o.pdl > 0) return MGR_ERR_INVALID_ARG;
  return MGR_OK;
}

mgr_status_t mgr_create(mgr_handle_t* out, const mgr_options_t* opt, void* stream) {
  if (!out) return MGR_ERR_INVALID_ARG;
  *out = nullptr;
  mgr_handle_s* h = new (std::nothrow) mgr_handle_s();
  if (!h) return MGR_ERR_OOM;
  if (opt) h->o = *opt; else mgr_options_default(&h->o);
  mgr_status_t st = check_options(h->o);
  if (st != MGR_OK) { delete h; return st; }
  st = guarded(h, [&] {
    CU(cudaGetDevice(&h->device));
    h->c.s = static_cast<cudaStream_t>(stream);
    h->c.pdl = h->o.pdl >= 0;
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    h->c.num_sms = sms;
    cudaMemPool_t pool;
    CU(cudaDeviceGetDefaultMemPool(&pool, h->device));
    uint64_t thr = UINT64_MAX;
    CU(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    CU(cudaMalloc(&h->c.d_err, sizeof(int)));
    CU(cudaMemset(h->c.d_err, 0, sizeof(int)));
    CU(cudaMallocHost(&h->hpin, 512 * sizeof(double)));
    // the last 2 PIN_SLOTS slots: read-backs of the setup (main context, then the second one);
    // the Krylov read-backs use the first 256
    h->c.h_pinned = h->hpin + 512 - 2 * PIN_SLOTS;
  });
  if (st != MGR_OK) {
    if (h->c.d_err) cudaFree(h->c.d_err);
    if (h->hpin) cudaFreeHost(h->hpin);
    delete h;
    return st;
  }
  *out = h;
  return MGR_OK;
}

mgr_status_t mgr_setup(mgr_handle_t h, const mgr_bsr3_t* A, const int8_t* cf_marker) {
  if (!h || !A || !cf_marker) return MGR_ERR_INVALID_ARG;
  return guarded(h, [&] { do_setup(*h, *A, cf_marker); });
}

// ---- index audit -------------------------------------------------------------------------------
__global__ void k_audit_sell32(int64_t nb, const int64_t* soff, const int32_t* col, unsigned long long* bad) {
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nb) return;
  const int64_t s = I / SELL_C;
  const int t = (int)(I - s * SELL_C);
  const int64_t b0 = soff[s], b1 = soff[s + 1];
  unsigned long long nbad = b1 < b0;
  for (int64_t j = b0; j < b1; ++j) {
    const int32_t J = col[j * SELL_C + t];
    nbad += (J < 0 || J >= nb);
  }
  if (nbad) atomicAdd(bad, nbad);
}
__global__ void k_audit_list(int64_t n, const int32_t* a, int64_t hi, unsigned long long* bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && (a[i] < 0 || a[i] >= hi)) atomicAdd(bad, 1ull);
}
// map[d] = c (a C point, c < nC) or -(f + 1) (an F point, f < nF)
__global__ void k_audit_map(int64_t n, const int32_t* map, int64_t nF, int64_t nC, unsigned long long* bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t m = map[i];
  if (m >= 0 ? m >= nC : (-m - 1) >= nF) atomicAdd(bad, 1ull);
}

static void audit_amg(Ctx& c, const std::vector<AmgLevel>& lv, unsigned long long* bad) {
  for (const AmgLevel& G : lv) {
    rowsop_audit(c, G.A32, bad); rowsop_audit(c, G.P32, bad); rowsop_audit(c, G.R32, bad);
    rowsop_audit(c, G.A64, bad); rowsop_audit(c, G.P64, bad); rowsop_audit(c, G.R64, bad);
    rowsop_audit(c, G.AT32, bad); rowsop_audit(c, G.AT64, bad);
  }
}

static void audit_sell(Ctx& c, const SellPattern& S, unsigned long long* bad) {
  if (S.nb <= 0 || !S.col.p) return;
  k_audit_sell32<<<grid_for(S.nb, 256), 256, 0, c.s>>>(S.nb, S.soff.p, S.col.p, bad);
  CU_LAUNCH();
}

mgr_status_t mgr_audit(mgr_handle_t h, int64_t* bad) {
  if (!h || !bad) return MGR_ERR_INVALID_ARG;
  if (!h->ready) return MGR_ERR_STATE;
  return guarded(h, [&] {
    Ctx& c = h->c;
    DBuf<unsigned long long> cnt(c, 1);
    CU(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), c.s));
    audit_sell(c, h->sell, cnt.p);
    if (h->has_t) audit_sell(c, h->sellT, cnt.p);
    for (int l = 0; l < h->L; ++l) {
      const MgrLevel& L = h->lev[l];
      rowsop_audit(c, L.Aff32, cnt.p); rowsop_audit(c, L.Acf32, cnt.p); rowsop_audit(c, L.Wp32, cnt.p);
      rowsop_audit(c, L.Aff64, cnt.p); rowsop_audit(c, L.Acf64, cnt.p); rowsop_audit(c, L.Wp64, cnt.p);
      rowsop_audit(c, L.WpT32, cnt.p); rowsop_audit(c, L.AcfT32, cnt.p); rowsop_audit(c, L.AffT32, cnt.p);
      rowsop_audit(c, L.WpT64, cnt.p); rowsop_audit(c, L.AcfT64, cnt.p); rowsop_audit(c, L.AffT64, cnt.p);
      if (L.nF > 0 && L.F.p) {
        k_audit_list<<<grid_for(L.nF, 256), 256, 0, c.s>>>(L.nF, L.F.p, L.n, cnt.p);
        CU_LAUNCH();
      }
      if (L.nC > 0 && L.C.p) {
        k_audit_list<<<grid_for(L.nC, 256), 256, 0, c.s>>>(L.nC, L.C.p, L.n, cnt.p);
        CU_LAUNCH();
      }
      if (L.n > 0 && L.map.p) {
        k_audit_map<<<grid_for(L.n, 256), 256, 0, c.s>>>(L.n, L.map.p, L.nF, L.nC, cnt.p);
        CU_LAUNCH();
      }
      audit_amg(c, L.famg, cnt.p);
    }
    audit_amg(c, h->amg, cnt.p);
    *bad = (int64_t)read_scalar(c, cnt.p);
  });
}

mgr_status_t mgr_apply(mgr_handle_t h, const double* r, double* z) {
  if (!h || !r || !z) return MGR_ERR_INVALID_ARG;
  if (!h->ready) return MGR_ERR_STATE;
  return guarded(h, [&] { do_apply(*h, r, z); });
}

mgr_status_t fgmres_solve(mgr_handle_t h, const mgr_bsr3_t* A, const double* b, double* x, double rtol, int restart,
                          int maxit, mgr_solve_info_t* info) {
  if (!h || !A || !b || !x || restart < 1 || restart > KRY_MAXV || maxit < 0 || !(rtol >= 0.0))
    return MGR_ERR_INVALID_ARG;
  if (!h->ready) return MGR_ERR_STATE;
  if (A->nb != h->nb || A->nnzb != h->nnzb || !A->rowptr || !A->colind || !A->values) return MGR_ERR_INVALID_ARG;
  mgr_status_t st = MGR_OK;
  mgr_status_t g = guarded(h, [&] { st = do_fgmres(*h, *A, b, x, rtol, restart, maxit, info); });
  return g != MGR_OK ? g : st;
}

mgr_status_t mgr_apply_transpose(mgr_handle_t h, const double* r, double* z) {
  if (!h || !r || !z) return MGR_ERR_INVALID_ARG;
  if (!h->ready || !h->has_t) return MGR_ERR_STATE;
  return guarded(h, [&] { do_apply_t(*h, r, z); });
}

mgr_status_t fgmres_solve_transpose(mgr_handle_t h, const mgr_bsr3_t* A, const double* b, double* x, double rtol,
                                    int restart, int maxit, mgr_solve_info_t* info) {
  if (!h || !A || !b || !x || restart < 1 || restart > KRY_MAXV || maxit < 0 || !(rtol >= 0.0))
    return MGR_ERR_INVALID_ARG;
  if (!h->ready || !h->has_t) return MGR_ERR_STATE;
  if (A->nb != h->nb || A->nnzb != h->nnzb || !A->rowptr || !A->colind || !A->values) return MGR_ERR_INVALID_ARG;
  mgr_status_t st = MGR_OK;
  mgr_status_t g = guarded(h, [&] { st = do_fgmres(*h, *A, b, x, rtol, restart, maxit, info, true); });
  return g != MGR_OK ? g : st;
}

mgr_status_t mgr_destroy(mgr_handle_t h) {
  if (!h) return MGR_OK;
  mgr_status_t st = guarded(h, [&] {
    CU(cudaStreamSynchronize(h->c.s));
    reset_graph(*h);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    h->gstream = nullptr;
    h->lev.clear();
    h->amg.clear();
    rehome_mgr_part(*h);  // buffers a failed setup left on the second context
    if (h->cw.s) {
      CU(cudaStreamSynchronize(h->cw.s));
      cudaStreamDestroy(h->cw.s);
      h->cw.s = nullptr;
    }
    if (h->cw.d_err) cudaFree(h->cw.d_err);
    h->cw.d_err = nullptr;
  });
  {
    // remaining buffers are released by the destructor (stream-ordered frees)
    cudaStream_t s = h->c.s;
    int* e = h->c.d_err;
    double* hp = h->hpin;
    Prof* pr = h->prof;
    h->c.prof = nullptr;
    delete h;
    delete pr;
    cudaStreamSynchronize(s);
    if (e) cudaFree(e);
    if (hp) cudaFreeHost(hp);
  }
  return st;
}

mgr_status_t mgr_get_levels(mgr_handle_t h, int* mgr_levels, int* amg_levels) {
  if (!h || !mgr_levels || !amg_levels) return MGR_ERR_INVALID_ARG;
  if (!h->ready) return MGR_ERR_STATE;
  *mgr_levels = h->L;
  *amg_levels = (int)h->amg.size();
  return MGR_OK;
}

mgr_status_t mgr_matrix_shape(mgr_handle_t h, int kind, int level, int64_t* nr, int64_t* nc, int64_t* nnz) {
  if (!h || !nr || !nc || !nnz) return MGR_ERR_INVALID_ARG;
  if (!h->ready) return MGR_ERR_STATE;
  const DCSR<double>* m = pick_matrix(*h, kind, level);
  if (!m || (m->rp.p == nullptr && !(h->o.lean && m->nr > 0))) return MGR_ERR_INVALID_ARG;
  *nr = m->nr; *nc = m->nc; *nnz = m->nnz;
  return MGR_OK;
}

mgr_status_t mgr_copy_matrix(mgr_handle_t h, int kind, int level, int64_t* rowptr, int32_t* col, double* val) {
  if (!h || !rowptr || !col) return MGR_ERR_INVALID_ARG;
  if (!h->ready) return MGR_ERR_STATE;
  const DCSR<double>* m = pick_matrix(*h, kind, level);
  if (!m) return MGR_ERR_INVALID_ARG;
  if (m->rp.p == nullptr) return (h->o.lean && m->nr > 0) ? MGR_ERR_STATE : MGR_ERR_INVALID_ARG;
  return guarded(h, [&] {
    Ctx& c = h->c;
    CU(cudaMemcpyAsync(rowptr, m->rp.p, sizeof(int64_t) * (m->nr + 1), cudaMemcpyDeviceToDevice, c.s));
    if (m->nnz) CU(cudaMemcpyAsync(col, m->ci.p, sizeof(int32_t) * m->nnz, cudaMemcpyDeviceToDevice, c.s));
    if (val && m->nnz) {
      if (m->v.p) CU(cudaMemcpyAsync(val, m->v.p, sizeof(double) * m->nnz, cudaMemcpyDeviceToDevice, c.s));
      else { k_fill_one<<<grid_for(m->nnz, 256), 256, 0, c.s>>>(m->nnz, val); CU_LAUNCH(); }
    }
    CU(cudaStreamSynchronize(c.s));
  });
}

mgr_status_t mgr_vector_len(mgr_handle_t h, int kind, int level, int64_t* len) {
  if (!h || !len) return MGR_ERR_INVALID_ARG;
  if (!h->ready) return MGR_ERR_STATE;
  int na = (int)h->amg.size();
  switch (kind) {
    case 0: case 3: if (level < 0 || level >= h->L) return MGR_ERR_INVALID_ARG; *len = h->lev[level].nF; return MGR_OK;
    case 4: if (level < 0 || level >= h->L) return MGR_ERR_INVALID_ARG; *len = h->lev[level].nC; return MGR_OK;
    case 1: case 5: if (level < 0 || level >= na - 1) return MGR_ERR_INVALID_ARG; *len = h->amg[level].n; return MGR_OK;
    case 2: *len = 9 * h->nb; return MGR_OK;
  }
  return MGR_ERR_INVALID_ARG;
}

mgr_status_t mgr_copy_vector(mgr_handle_t h, int kind, int level, double* out) {
  int64_t len;
  mgr_status_t st = mgr_vector_len(h, kind, level, &len);
  if (st != MGR_OK) return st;
  if (!out) return MGR_ERR_INVALID_ARG;
  return guarded(h, [&] {
    Ctx& c = h->c;
    if (len > 0) {
      unsigned g = grid_for(len, 256);
      switch (kind) {
        case 0: CU(cudaMemcpyAsync(out, h->lev[level].minv.p, sizeof(double) * len, cudaMemcpyDeviceToDevice, c.s)); break;
        case 1: CU(cudaMemcpyAsync(out, h->amg[level].dinv.p, sizeof(double) * len, cudaMemcpyDeviceToDevice, c.s)); break;
        case 2: CU(cudaMemcpyAsync(out, h->binv.p, sizeof(double) * len, cudaMemcpyDeviceToDevice, c.s)); break;
        case 3: k_to_double<int32_t><<<g, 256, 0, c.s>>>(len, h->lev[level].F.p, out); CU_LAUNCH(); break;
        case 4: k_to_double<int32_t><<<g, 256, 0, c.s>>>(len, h->lev[level].C.p, out); CU_LAUNCH(); break;
        case 5: k_to_double<int8_t><<<g, 256, 0, c.s>>>(len, h->amg[level].cf.p, out); CU_LAUNCH(); break;
      }
    }
    CU(cudaStreamSynchronize(c.s));
  });
}

mgr_status_t mgr_profile(mgr_handle_t h, int enable) {
  if (!h) return MGR_ERR_INVALID_ARG;
  return guarded(h, [&] {
    CU(cudaStreamSynchronize(h->c.s));
    if (enable) {
      if (!h->prof) h->prof = new Prof();
      h->prof->settle();
      h->prof->recs.clear();
      h->c.prof = h->prof;
    } else {
      h->c.prof = nullptr;
    }
  });
}

mgr_status_t mgr_profile_select(mgr_handle_t h, const char* names) {
  if (!h) return MGR_ERR_INVALID_ARG;
  return guarded(h, [&] {
    if (!h->prof) h->prof = new Prof();
    h->prof->only.clear();
    if (!names) return;
    std::string cur;
    for (const char* p = names;; ++p) {
      if (*p == ',' || *p == '\0') {
        if (!cur.empty()) h->prof->only.insert(cur);
        cur.clear();
        if (*p == '\0') break;
      } else if (*p != ' ') {
        cur.push_back(*p);
      }
    }
  });
}

mgr_status_t mgr_kernel_time(mgr_handle_t h, const char* name, int64_t* launches, double* total_ms) {
  if (!h || !name || !launches || !total_ms) return MGR_ERR_INVALID_ARG;
  *launches = 0;
  *total_ms = 0.0;
  if (!h->prof) return MGR_OK;
  return guarded(h, [&] {
    h->prof->settle();
    auto it = h->prof->recs.find(name);
    if (it != h->prof->recs.end()) { *launches = it->second.n; *total_ms = it->second.ms; }
  });
}

mgr_status_t mgr_kernel_bytes(mgr_handle_t h, const char* name, double* bytes) {
  if (!h || !name || !bytes) return MGR_ERR_INVALID_ARG;
  *bytes = 0.0;
  if (!h->prof) return MGR_OK;
  return guarded(h, [&] {
    h->prof->settle();
    auto it = h->prof->recs.find(name);
    if (it != h->prof->recs.end()) *bytes = it->second.bytes;
  });
}

mgr_status_t mgr_kernel_bytes_stored(mgr_handle_t h, const char* name, double* bytes) {
  if (!h || !name || !bytes) return MGR_ERR_INVALID_ARG;
  *bytes = 0.0;
  if (!h->prof) return MGR_OK;
  return guarded(h, [&] {
    h->prof->settle();
    auto it = h->prof->recs.find(name);
    if (it != h->prof->recs.end()) *bytes = it->second.bytes_stored;
  });
}

mgr_status_t mgr_memory_bytes(mgr_handle_t h, int64_t* bytes) {
  if (!h || !bytes) return MGR_ERR_INVALID_ARG;
  *bytes = h->c.bytes;
  return MGR_OK;
}

mgr_status_t mgr_memory_peak_bytes(mgr_handle_t h, int64_t* bytes) {
  if (!h || !bytes) return MGR_ERR_INVALID_ARG;
  *bytes = h->c.peak;
  return MGR_OK;
}

mgr_status_t mgr_get_host_waits(int64_t* waits) {
  if (!waits) return MGR_ERR_INVALID_ARG;
  *waits = (int64_t)g_wait_count;
  return MGR_OK;
}

mgr_status_t mgr_get_stats(mgr_handle_t h, double* setup_ms, int64_t* apply_launches, int64_t* graph_nodes,
                           int64_t* total_launches) {
  if (total_launches) *total_launches = (int64_t)g_launch_count;
  if (!h) return setup_ms || apply_launches || graph_nodes ? MGR_ERR_INVALID_ARG : MGR_OK;
  if (setup_ms) *setup_ms = h->setup_ms;
  if (apply_launches) *apply_launches = h->apply_launches;
  if (graph_nodes) *graph_nodes = h->gexec ? h->g_launches : 0;
  return MGR_OK;
}

static mgr_status_t with_ctx(void* stream, const std::function<void(Ctx&)>& f);

mgr_status_t mgr_bsr3_spmv(const mgr_bsr3_t* A, const double* x, const double* sub, double* y, void* stream) {
  if (!A || !x || !y || A->nb <= 0 || !A->rowptr || !A->colind || !A->values) return MGR_ERR_INVALID_ARG;
  return with_ctx(stream, [&](Ctx& c) { launch_bsr3_spmv_f64(c, *A, x, sub, y); });
}

mgr_status_t mgr_bsr3_transpose(const mgr_bsr3_t* A, int64_t* rpt, int32_t* cit, double* vt, void* stream) {
  if (!A || !rpt || !cit || !vt || A->nb <= 0 || !A->rowptr || !A->colind || !A->values) return MGR_ERR_INVALID_ARG;
  return with_ctx(stream, [&](Ctx& c) { launch_bsr3_transpose(c, *A, rpt, cit, vt); });
}

mgr_status_t mgr_bsr3_outer_grad(const mgr_bsr3_t* A, const double* lam, const double* x, double* g, void* stream) {
  if (!A || !lam || !x || !g || A->nb <= 0 || !A->rowptr || !A->colind) return MGR_ERR_INVALID_ARG;
  return with_ctx(stream, [&](Ctx& c) { launch_bsr3_outer_grad(c, *A, lam, x, g); });
}

}  // extern "C"

static mgr_status_t with_ctx(void* stream, const std::function<void(Ctx&)>& f) {
  Ctx c;
  c.s = static_cast<cudaStream_t>(stream);
  try {
    f(c);
    return MGR_OK;
  } catch (...) {
    return guard_status(std::current_exception(), nullptr);
  }
}
