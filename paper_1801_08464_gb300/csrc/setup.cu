// setup.cu -- MGR reduction levels and the AMG hierarchy (compiled with --fmad=false).
//
// The arithmetic follows a fixed order of IEEE double operations (explicit __dmul_rn, __dadd_rn,
// __ddiv_rn), so every value and every floating-point decision (strength, PMIS weights, lumping)
// is reproducible.
#include <cmath>

#include "hier.cuh"

#include <climits>

namespace mgr {

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dv(double a, double b) { return __ddiv_rn(a, b); }

__device__ __forceinline__ double csr_get(const int64_t* rp, const int32_t* ci, const double* v, int64_t i, int32_t j) {
  int64_t p = find_i32(ci, rp[i], rp[i + 1], j);
  return p >= 0 ? v[p] : 0.0;
}

// ============================== MGR reduction level (sections 4-5) =============================
__global__ void k_level_flags(int64_t n, const int8_t* mk, int l, int32_t* ff, int32_t* cf) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  ff[i] = (mk[i] == l);
  cf[i] = (mk[i] > l);
}
__global__ void k_level_lists(int64_t n, const int8_t* mk, int l, const int32_t* fpre, const int32_t* cpre, int32_t* F,
                              int32_t* C, int32_t* map) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (mk[i] == l) { F[fpre[i]] = (int32_t)i; map[i] = -(fpre[i] + 1); }
  else { C[cpre[i]] = (int32_t)i; map[i] = cpre[i]; }
}

// D_ff = diag(A_ff) and the F-relaxation scaling: omega / d (Jacobi) or 1 / (d + sign(d) l1) with
// l1 = sum of |a_fg| over the off-diagonal F columns of the row, ascending.
__global__ void k_dff_minv(int64_t nF, const int32_t* F, const int64_t* rp, const int32_t* ci, const double* v,
                           const int32_t* map, int type, double omega, double* dff, double* minv, int* err) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nF) return;
  int32_t i = F[f];
  double d = 0.0, l1 = 0.0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
    int32_t j = ci[k];
    if (j == i) d = v[k];
    else if (map[j] < 0) l1 = dd(l1, fabs(v[k]));
  }
  dff[f] = d;
  if (d == 0.0 || !isfinite(d)) { atomicOr(err, EBIT_SINGULAR); minv[f] = 0.0; return; }
  if (type == 1) {
    double den = dd(d, (d >= 0.0) ? l1 : -l1);
    minv[f] = dv(1.0, den);
  } else {
    minv[f] = dv(omega, d);
  }
}

// per-row counts of entries of rows `rows` of A whose column satisfies sel (C: map >= 0, F: map < 0)
template <bool WANT_C>
__global__ void k_count_sel(int64_t nr, const int32_t* rows, const int64_t* rp, const int32_t* ci, const int32_t* map,
                            int64_t* cnt) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  int32_t i = rows[r];
  int64_t s = 0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += WANT_C ? (map[ci[k]] >= 0) : (map[ci[k]] < 0);
  cnt[r] = s;
}

// W_p = -D_ff^-1 A_fc (rows F, coarse columns) and A_ff (rows F, F-local columns); a group of RG
// lanes per F row, entries in row order
__global__ void __launch_bounds__(256) k_fill_wp_aff(int64_t nF, const int32_t* F, const int64_t* rp,
                                                     const int32_t* ci, const double* v, const int32_t* map,
                                                     const double* dff, const int64_t* wrp, int32_t* wci, double* wv,
                                                     const int64_t* frp, int32_t* fci, double* fv) {
  const RowGroup G = row_group();
  const int64_t f = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / RG;
  const bool act = f < nF;
  int64_t k0 = 0, ow = 0, of = 0;
  int len = 0;
  double d = 1.0;
  if (act) {
    const int32_t i = F[f];
    k0 = rp[i];
    len = (int)(rp[i + 1] - k0);
    ow = wrp[f];
    of = frp[f];
    d = dff[f];
  }
  const int rounds = warp_max_int((len + RG - 1) / RG);
  for (int r = 0; r < rounds; ++r) {
    const int t = r * RG + G.g;
    const bool in = act && t < len;
    int32_t m = 0;
    double x = 0.0;
    if (in) {
      m = map[ci[k0 + t]];
      x = v[k0 + t];
    }
    const unsigned bc = __ballot_sync(0xffffffffu, in && m >= 0) & G.gmask;
    const unsigned bf = __ballot_sync(0xffffffffu, in && m < 0) & G.gmask;
    if (in) {
      if (m >= 0) {
        const int64_t o = ow + __popc(bc & G.below);
        wci[o] = m;
        wv[o] = -dv(x, d);
      } else {
        const int64_t o = of + __popc(bf & G.below);
        fci[o] = -m - 1;
        fv[o] = x;
      }
    }
    ow += __popc(bc);
    of += __popc(bf);
  }
}

// A_cf (rows C, F-local columns), and for a non-injective restriction W_r = -A_cf D_ff^-1 and the
// rows of R = [W_r, I] in fine column order (the 1 placed at the C point's own column).  A thread per
// C row: the group-of-lanes form of the other row copies measured slower here (0.72 against 0.48 ms
// per launch at 128^3), its extra ballots and dependent gathers (column, map, D_ff) per round
// outweighing the coalesced writes.
__global__ void k_fill_acf_wr(int64_t nC, const int32_t* C, const int64_t* rp, const int32_t* ci, const double* v,
                              const int32_t* map, const double* dff, int noninj, const int64_t* arp, int32_t* aci,
                              double* av, const int64_t* wrp, int32_t* wci, double* wv, const int64_t* rrp, int32_t* rci,
                              double* rv) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nC) return;
  int32_t i = C[c];
  int64_t oa = arp[c], ow = noninj ? wrp[c] : 0, orr = rrp[c];
  bool placed = false;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
    int32_t j = ci[k], m = map[j];
    if (m >= 0) continue;
    int32_t f = -m - 1;
    aci[oa] = f; av[oa] = v[k]; ++oa;
    if (noninj) {
      double w = -dv(v[k], dff[f]);
      wci[ow] = f; wv[ow] = w; ++ow;
      if (!placed && j > i) { rci[orr] = i; rv[orr] = 1.0; ++orr; placed = true; }
      rci[orr] = j; rv[orr] = w; ++orr;
    }
  }
  if (!placed) { rci[orr] = i; rv[orr] = 1.0; }
}

// P = [W_p; I] in fine row order
__global__ void k_p_count(int64_t n, const int32_t* map, const int64_t* wrp, int64_t* cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t m = map[i];
  cnt[i] = (m >= 0) ? 1 : (wrp[-m] - wrp[-m - 1]);
}
__global__ void k_p_fill(int64_t n, const int32_t* map, const int64_t* wrp, const int32_t* wci, const double* wv,
                         const int64_t* prp, int32_t* pci, double* pv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t m = map[i];
  int64_t o = prp[i];
  if (m >= 0) { pci[o] = m; pv[o] = 1.0; return; }
  int32_t f = -m - 1;
  for (int64_t k = wrp[f]; k < wrp[f + 1]; ++k, ++o) { pci[o] = wci[k]; pv[o] = wv[k]; }
}
__global__ void k_gather_i8(int64_t n, const int32_t* idx, const int8_t* src, int8_t* dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}
__global__ void k_i64_add_one(int64_t n, int64_t* a) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] += 1;
}

// Row pointers from per-row counts, without reading the total (the caller sets M.nnz, from a
// read-back of M.rp[nr] batched with others or from the sizes of other operators), then csr_alloc.
static void csr_rows(Ctx& c, DCSR<double>& M, int64_t nr, int64_t nc, const int64_t* cnt) {
  M.nr = nr;
  M.nc = nc;
  M.rp.alloc(c, nr + 1);
  scan_excl_i64(c, cnt, M.rp.p, nr);
}
static void csr_alloc(Ctx& c, DCSR<double>& M) {
  M.ci.alloc(c, M.nnz);
  M.v.alloc(c, M.nnz);
}
static void alloc_csr(Ctx& c, DCSR<double>& M, int64_t nr, int64_t nc, const int64_t* cnt) {
  M.nr = nr;
  M.nc = nc;
  M.rp.alloc(c, nr + 1);
  M.nnz = counts_to_rowptr(c, cnt, M.rp.p, nr);
  M.ci.alloc(c, M.nnz);
  M.v.alloc(c, M.nnz);
}

void mgr_reduce_level(Ctx& c, MgrLevel& L, int l, const LevelOpts& o, DCSR<double>& Anext, DBuf<int8_t>& mk_next) {
  int64_t n = L.n;
  const DCSR<double>& A = L.A;
  const int B = 256;
  {
    DBuf<int32_t> ff(c, n), cf(c, n), fpre(c, n + 1), cpre(c, n + 1);
    k_level_flags<<<grid_for(n, B), B, 0, c.s>>>(n, L.mk.p, l, ff.p, cf.p);
    CU_LAUNCH();
    scan_excl_i32(c, ff.p, fpre.p, n);
    scan_excl_i32(c, cf.p, cpre.p, n);
    int32_t nf = 0, nc = 0;
    read_back(c, {{fpre.p + n, &nf, sizeof(int32_t)}, {cpre.p + n, &nc, sizeof(int32_t)}});
    L.nF = nf;
    L.nC = nc;
    L.F.alloc(c, L.nF);
    L.C.alloc(c, L.nC);
    L.map.alloc(c, n);
    k_level_lists<<<grid_for(n, B), B, 0, c.s>>>(n, L.mk.p, l, fpre.p, cpre.p, L.F.p, L.C.p, L.map.p);
    CU_LAUNCH();
  }
  if (L.nC == 0) throw Error(MGR_ERR_INVALID_ARG, "cf_marker: a reduction level has no C point");
  int64_t nF = L.nF, nC = L.nC;
  L.sweeps = o.sweeps;
  L.dff.alloc(c, nF);
  L.minv.alloc(c, nF);
  if (nF) {
    k_dff_minv<<<grid_for(nF, B), B, 0, c.s>>>(nF, L.F.p, A.rp.p, A.ci.p, A.v.p, L.map.p, o.frelax_type, o.omega,
                                                L.dff.p, L.minv.p, c.d_err);
    CU_LAUNCH();
  }
  // the sizes of W_p, A_ff and A_cf (and the D_ff check) with one wait; those of W_r, R and P follow
  // from them
  DBuf<int64_t> cw(c, nF + 1), cfcnt(c, nF + 1), ca(c, nC + 1);
  if (nF) {
    k_count_sel<true><<<grid_for(nF, B), B, 0, c.s>>>(nF, L.F.p, A.rp.p, A.ci.p, L.map.p, cw.p);
    CU_LAUNCH();
    k_count_sel<false><<<grid_for(nF, B), B, 0, c.s>>>(nF, L.F.p, A.rp.p, A.ci.p, L.map.p, cfcnt.p);
    CU_LAUNCH();
  }
  k_count_sel<false><<<grid_for(nC, B), B, 0, c.s>>>(nC, L.C.p, A.rp.p, A.ci.p, L.map.p, ca.p);
  CU_LAUNCH();
  csr_rows(c, L.Wp, nF, nC, cw.p);
  csr_rows(c, L.Aff, nF, nF, cfcnt.p);
  csr_rows(c, L.Acf, nC, nF, ca.p);
  {
    int err = 0;
    read_back(c, {{L.Wp.rp.p + nF, &L.Wp.nnz, sizeof(int64_t)}, {L.Aff.rp.p + nF, &L.Aff.nnz, sizeof(int64_t)},
                  {L.Acf.rp.p + nC, &L.Acf.nnz, sizeof(int64_t)}, {c.d_err, &err, sizeof(int)}});
    if (err) check_errors(c, "MGR D_ff");
  }
  csr_alloc(c, L.Wp);
  csr_alloc(c, L.Aff);
  csr_alloc(c, L.Acf);
  // W_p and A_ff
  if (nF) {
    k_fill_wp_aff<<<grid_for(nF * RG, B), B, 0, c.s>>>(nF, L.F.p, A.rp.p, A.ci.p, A.v.p, L.map.p, L.dff.p, L.Wp.rp.p,
                                                  L.Wp.ci.p, L.Wp.v.p, L.Aff.rp.p, L.Aff.ci.p, L.Aff.v.p);
    CU_LAUNCH();
  }
  // A_cf, W_r, R: W_r has A_cf's pattern; R's rows hold one more entry than A_cf's (non-injective)
  // or exactly one (injective)
  {
    bool noninj = o.restrict_type == 1;
    if (noninj) {
      csr_rows(c, L.Wr, nC, nF, ca.p);
      L.Wr.nnz = L.Acf.nnz;
      csr_alloc(c, L.Wr);
      k_i64_add_one<<<grid_for(nC, B), B, 0, c.s>>>(nC, ca.p);
      CU_LAUNCH();
      csr_rows(c, L.R, nC, n, ca.p);
      L.R.nnz = L.Acf.nnz + nC;
    } else {
      L.Wr.nr = nC; L.Wr.nc = nF; L.Wr.nnz = 0;
      L.Wr.rp.alloc(c, nC + 1);
      fill_i64(c, L.Wr.rp.p, 0, nC + 1);
      L.Wr.ci.alloc(c, 0);
      L.Wr.v.alloc(c, 0);
      fill_i64(c, ca.p, 1, nC);
      csr_rows(c, L.R, nC, n, ca.p);
      L.R.nnz = nC;
    }
    csr_alloc(c, L.R);
    k_fill_acf_wr<<<grid_for(nC, B), B, 0, c.s>>>(nC, L.C.p, A.rp.p, A.ci.p, A.v.p, L.map.p, L.dff.p, noninj ? 1 : 0,
                                                   L.Acf.rp.p, L.Acf.ci.p, L.Acf.v.p, L.Wr.rp.p, L.Wr.ci.p, L.Wr.v.p,
                                                   L.R.rp.p, L.R.ci.p, L.R.v.p);
    CU_LAUNCH();
  }
  // P = [W_p; I]
  {
    DBuf<int64_t> cp(c, n + 1);
    k_p_count<<<grid_for(n, B), B, 0, c.s>>>(n, L.map.p, L.Wp.rp.p, cp.p);
    CU_LAUNCH();
    // W_p's entries and one per C point
    csr_rows(c, L.P, n, nC, cp.p);
    L.P.nnz = L.Wp.nnz + nC;
    csr_alloc(c, L.P);
    k_p_fill<<<grid_for(n, B), B, 0, c.s>>>(n, L.map.p, L.Wp.rp.p, L.Wp.ci.p, L.Wp.v.p, L.P.rp.p, L.P.ci.p, L.P.v.p);
    CU_LAUNCH();
  }
  // coarse operator R (A P) and coarse markers.  With an injective R (one 1 per row, at the C point)
  // row c of R (A P) is 0.0 + 1 * (A P)_{C[c]}; a Gustavson sum that starts at +0.0 never ends at -0.0,
  // so that equals (A P)_{C[c]} bit for bit, and only the C rows of A enter the product.
  {
    static const char* const kAP[] = {"rap_mgr0_AP", "rap_mgr1_AP", "rap_mgr2_AP", "rap_mgr3_AP"};
    static const char* const kRAP[] = {"rap_mgr0_RAP", "rap_mgr1_RAP", "rap_mgr2_RAP", "rap_mgr3_RAP"};
    const int li = l < 3 ? l : 3;
    ProfScope ps(c, "setup_mgr_rap");
    if (o.restrict_type == 1) {
      DCSR<double> AP;
      spgemm(c, A, L.P, AP, kAP[li]);
      spgemm(c, L.R, AP, Anext, kRAP[li]);
    } else {
      DCSR<double> AC;
      // the C rows of A hold every entry the F rows (split into W_p and A_ff) do not
      csr_gather_rows(c, A, L.C.p, nC, AC, A.nnz - L.Wp.nnz - L.Aff.nnz);
      spgemm(c, AC, L.P, Anext, kRAP[li], true);
    }
  }
  mk_next.alloc(c, nC);
  k_gather_i8<<<grid_for(nC, B), B, 0, c.s>>>(nC, L.C.p, L.mk.p, mk_next.p);
  CU_LAUNCH();
}

// ===================================== AMG (coarse solve) =====================================
// Strength: with s = +1 if a_ii >= 0 else -1, j != i is strong iff -s a_ij >= theta m where
// m = max(0, max_{k != i} -s a_ik) > 0.  A warp per row; MODE 0 counts, MODE 1 writes in order.
// Everything but theta * m is done on the bit patterns with integer instructions (the FP64 pipe is
// the scarce resource): -s a_ij is a_ij with its sign bit flipped when s = +1, and doubles compare
// like the integers dkey() maps them to (NaN entries are neither strong nor part of the maximum, as
// with IEEE comparisons).  The results are those of the comparisons in FP64 exactly.
constexpr long long DMAG = 0x7FFFFFFFFFFFFFFFLL, DINF = 0x7FF0000000000000LL, DSIGN = (long long)0x8000000000000000ULL;

__device__ __forceinline__ long long dkey(long long b) { return b ^ ((b >> 63) & DMAG); }

// key of -s a for the entry's bits (LLONG_MIN for NaN: never the maximum, never strong)
__device__ __forceinline__ long long strength_key(double a, bool spos) {
  long long b = __double_as_longlong(a);
  if ((b & DMAG) > DINF) return LLONG_MIN;
  return dkey(spos ? (b ^ DSIGN) : b);
}

// s = +1 iff a_ii >= 0 (true for -0.0, false for NaN)
__device__ __forceinline__ bool diag_nonneg(double d) {
  long long b = __double_as_longlong(d);
  return (b & DMAG) == 0 || (b >= 0 && (b & DMAG) <= DINF);
}

__device__ __forceinline__ long long warp_max_ll(long long x) {
  for (int o = 16; o > 0; o >>= 1) {
    long long t = __shfl_xor_sync(0xffffffffu, x, o);
    x = t > x ? t : x;
  }
  return x;
}

// x >= thr for thr = theta * m >= 0 (thr == 0 admits both zeros)
__device__ __forceinline__ bool key_ge_thr(long long kx, long long kthr) {
  return kx >= kthr || (kthr == 0 && kx == -1);
}

template <int MODE>
__global__ void k_strength(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double theta, int64_t* cnt,
                           const int64_t* srp, int32_t* sci) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  int64_t b = rp[i], e = rp[i + 1];
  int64_t count = 0, out = (MODE == 1) ? srp[i] : 0;
  if (e - b <= 64) {
    // the row (at most 64 entries) is read once into registers, two entries per lane
    const int64_t k0 = b + lane, k1 = b + 32 + lane;
    const int32_t c0 = k0 < e ? ci[k0] : -1, c1 = k1 < e ? ci[k1] : -1;
    const double v0 = k0 < e ? v[k0] : 0.0, v1 = k1 < e ? v[k1] : 0.0;
    double d = 0.0;
    const unsigned md0 = __ballot_sync(0xffffffffu, c0 == (int32_t)i), md1 = __ballot_sync(0xffffffffu, c1 == (int32_t)i);
    if (md0) d = __shfl_sync(0xffffffffu, v0, __ffs(md0) - 1);
    else if (md1) d = __shfl_sync(0xffffffffu, v1, __ffs(md1) - 1);
    const bool spos = diag_nonneg(d);
    const long long kx0 = (c0 >= 0 && c0 != (int32_t)i) ? strength_key(v0, spos) : LLONG_MIN;
    const long long kx1 = (c1 >= 0 && c1 != (int32_t)i) ? strength_key(v1, spos) : LLONG_MIN;
    long long km = kx0 > kx1 ? kx0 : kx1;
    km = km > 0 ? km : 0;
    km = warp_max_ll(km);
    if (km > 0) {
      const double thr = dm(theta, __longlong_as_double(km));  // km > 0: the key is the bits
      const long long kthr = dkey(__double_as_longlong(thr));
      const bool st0 = kx0 != LLONG_MIN && key_ge_thr(kx0, kthr);
      const bool st1 = kx1 != LLONG_MIN && key_ge_thr(kx1, kthr);
      const unsigned m0 = __ballot_sync(0xffffffffu, st0), m1 = __ballot_sync(0xffffffffu, st1);
      if (MODE == 1) {
        const unsigned below = (1u << lane) - 1;
        if (st0) sci[out + __popc(m0 & below)] = c0;
        if (st1) sci[out + __popc(m0) + __popc(m1 & below)] = c1;
      }
      count = __popc(m0) + __popc(m1);
    }
    if (MODE == 0 && lane == 0) cnt[i] = count;
    return;
  }
  double d = 0.0;
  for (int64_t k0 = b; k0 < e; k0 += 32) {
    const int64_t k = k0 + lane;
    const bool hit = k < e && ci[k] == i;
    const unsigned mh = __ballot_sync(0xffffffffu, hit);
    if (mh) d = __shfl_sync(0xffffffffu, hit ? v[k] : 0.0, __ffs(mh) - 1);
  }
  const bool spos = diag_nonneg(d);
  long long km = 0;
  for (int64_t k = b + lane; k < e; k += 32)
    if (ci[k] != i) {
      const long long kx = strength_key(v[k], spos);
      km = kx > km ? kx : km;
    }
  km = warp_max_ll(km);
  if (km > 0) {
    const double thr = dm(theta, __longlong_as_double(km));
    const long long kthr = dkey(__double_as_longlong(thr));
    for (int64_t k0 = b; k0 < e; k0 += 32) {
      int64_t k = k0 + lane;
      bool strong = false;
      if (k < e && ci[k] != i) {
        const long long kx = strength_key(v[k], spos);
        strong = kx != LLONG_MIN && key_ge_thr(kx, kthr);
      }
      unsigned msk = __ballot_sync(0xffffffffu, strong);
      if (MODE == 1 && strong) sci[out + __popc(msk & ((1u << lane) - 1))] = ci[k];
      count += __popc(msk);
      out += __popc(msk);
    }
  }
  if (MODE == 0 && lane == 0) cnt[i] = count;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// PMIS weight w_i = |S^T_i| + u_i, u_i = top 53 bits of splitmix64(key ^ i) times 2^-53 with
// key = splitmix64(seed ^ ((level + 1) << 48)); points influencing nobody start as F.
__global__ void k_pmis_init(int64_t n, const int64_t* strp, uint64_t key, double* w, int8_t* st, int* und) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t lam = strp[i + 1] - strp[i];
  double u = (double)(splitmix64(key ^ (uint64_t)i) >> 11) * 0x1.0p-53;
  w[i] = dd((double)lam, u);
  st[i] = lam == 0 ? -1 : 0;
  if (lam) atomicAdd(und, 1);
}
// an undecided point beating every undecided strong neighbour (S and S^T; equal weights -> larger
// index wins) is selected
__global__ void k_pmis_select(int64_t n, const int64_t* srp, const int32_t* sci, const int64_t* trp, const int32_t* tci,
                              const double* w, const int8_t* st, int8_t* nc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  nc[i] = 0;
  if (st[i] != 0) return;
  // the weights are positive doubles, which order like their bit patterns: integer comparisons
  const long long* wb = reinterpret_cast<const long long*>(w);
  const long long wi = wb[i];
  for (int pass = 0; pass < 2; ++pass) {
    const int64_t* rp = pass ? trp : srp;
    const int32_t* ci = pass ? tci : sci;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      int32_t j = ci[k];
      if (j == i || st[j] != 0) continue;
      const long long wj = wb[j];
      if (wj > wi || (wj == wi && j > i)) return;
    }
  }
  nc[i] = 1;
}
// the selected points become C; *ncnt counts the C points (one atomic per warp)
__global__ void k_pmis_mark_c(int64_t n, const int8_t* nc, int8_t* st, int* ncnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool sel = i < n && nc[i];
  if (sel) st[i] = 1;
  const unsigned m = __ballot_sync(0xffffffffu, sel);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(ncnt, __popc(m));
}
// undecided points that strongly depend on a C point become F; count what stays undecided
__global__ void k_pmis_mark_f(int64_t n, const int64_t* srp, const int32_t* sci, int8_t* st, int* und) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || st[i] != 0) return;
  for (int64_t k = srp[i]; k < srp[i + 1]; ++k)
    if (st[sci[k]] == 1) { st[i] = -1; return; }
  atomicAdd(und, 1);
}

// Selection matrices for the extended+i pattern: M row i (F point) = {i} + strong F neighbours,
// T row k = strong C neighbours of k as coarse indices; pattern(P_F) = pattern(M T).
__global__ void k_extpi_sel_count(int64_t n, const int64_t* srp, const int32_t* sci, const int8_t* cf, int64_t* cm,
                                  int64_t* ct) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t a = 0, b = 0;
  for (int64_t k = srp[i]; k < srp[i + 1]; ++k) {
    if (cf[sci[k]] == 1) ++b; else ++a;
  }
  cm[i] = (cf[i] == 1) ? 0 : a + 1;
  ct[i] = b;
}
__global__ void k_extpi_sel_fill(int64_t n, const int64_t* srp, const int32_t* sci, const int8_t* cf, const int32_t* cidx,
                                 const int64_t* mrp, int32_t* mci, const int64_t* trp, int32_t* tci) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t om = mrp[i], ot = trp[i];
  bool fpt = cf[i] != 1, placed = false;
  for (int64_t k = srp[i]; k < srp[i + 1]; ++k) {
    int32_t j = sci[k];
    if (cf[j] == 1) { tci[ot++] = cidx[j]; continue; }
    if (!fpt) continue;
    if (!placed && j > i) { mci[om++] = (int32_t)i; placed = true; }
    mci[om++] = j;
  }
  if (fpt && !placed) mci[om] = (int32_t)i;
}
__global__ void k_cidx(int64_t n, const int8_t* cf, const int32_t* pre, int32_t* cidx, int32_t* cfine) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (cf[i] == 1) { cidx[i] = pre[i]; cfine[pre[i]] = (int32_t)i; }
  else cidx[i] = -1;
}
__global__ void k_flag_c(int64_t n, const int8_t* cf, int32_t* f) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) f[i] = cf[i] == 1;
}
__global__ void k_pfull_count(int64_t n, const int8_t* cf, const int64_t* qrp, int64_t* cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = (cf[i] == 1) ? 1 : qrp[i + 1] - qrp[i];
}
__global__ void k_pfull_fill(int64_t n, const int8_t* cf, const int32_t* cidx, const int64_t* qrp, const int32_t* qci,
                             const int64_t* prp, int32_t* pci) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = prp[i];
  if (cf[i] == 1) { pci[o] = cidx[i]; return; }
  for (int64_t k = qrp[i]; k < qrp[i + 1]; ++k) pci[o++] = qci[k];
}

__device__ __forceinline__ bool opposite(double a, double d) { return (d > 0.0 && a < 0.0) || (d < 0.0 && a > 0.0); }

// opposite() on the bit patterns, with integer instructions: both nonzero, neither NaN, signs differ
__device__ __forceinline__ bool opposite_bits(double a, double d) {
  const long long ia = __double_as_longlong(a), id = __double_as_longlong(d);
  const long long mag = 0x7FFFFFFFFFFFFFFFLL, inf = 0x7FF0000000000000LL;
  const long long ma = ia & mag, md = id & mag;
  return ma != 0 && md != 0 && ma <= inf && md <= inf && (ia ^ id) < 0;
}

// Extended+i weights (De Sterck, Falgout, Nolting & Yang 2008), one warp per F row; the pattern
// (Chat_i, coarse indices, ascending) is already in P.  Per strong F neighbour k (position p in S_i):
//   den_k = sum over l in row k (ascending) with l in Chat_i + {i} and a_kl opposite in sign to a_kk
//   of a_kl; q_k = a_ik / den_k, or a_ik lumped into the diagonal when den_k == 0.
//   at = a_ii + sum(weak neighbours not in Chat_i, ascending) + sum_k (q_k abar_ki or a_ik);
//   w_ij = -(a_ij + sum_k q_k abar_kj) / at.   An F row with at == 0 is flagged empty.
constexpr int EXT_WARPS = 4;
constexpr int EXT_CAP = 256;

__device__ __forceinline__ void extpi_full_row(int64_t i, const int64_t* rp, const int32_t* ci, const double* v,
                                               const int64_t* srp, const int32_t* sci, const int8_t* cf,
                                               const int32_t* cidx, const int32_t* cfine, const int64_t* prp,
                                               const int32_t* pci, double* pv, double* den_g, double* q_g,
                                               int8_t* rowzero, double* s_wt_w, double* s_kt_w, int8_t* s_wf_w,
                                               int8_t* s_kf_w) {
  const int lane = threadIdx.x & 31;
  if (cf[i] == 1) {
    if (lane == 0) { pv[prp[i]] = 1.0; rowzero[i] = 0; }
    return;
  }
  int64_t p0 = prp[i], p1 = prp[i + 1];
  int64_t s0 = srp[i], s1 = srp[i + 1];
  // den_k
  for (int64_t p = s0 + lane; p < s1; p += 32) {
    int32_t k = sci[p];
    if (cf[k] == 1) continue;
    double akk = csr_get(rp, ci, v, k, k), den = 0.0;
    for (int64_t q = rp[k]; q < rp[k + 1]; ++q) {
      int32_t l = ci[q];
      bool in = (l == i) || (cf[l] == 1 && find_i32(pci, p0, p1, cidx[l]) >= 0);
      if (in && opposite(v[q], akk)) den = dd(den, v[q]);
    }
    den_g[p] = den;
  }
  __syncwarp();
  double at = 0.0;
  int64_t r0 = rp[i], len = rp[i + 1] - r0, ns = s1 - s0;
  if (len <= EXT_CAP && ns <= EXT_CAP) {
    // the terms of the diagonal are formed by the lanes in parallel, then added by lane 0 in order
    for (int64_t t = lane; t < len; t += 32) {
      int32_t nn = ci[r0 + t];
      bool lump = nn != i && find_i32(sci, s0, s1, nn) < 0 &&
                  !(cf[nn] == 1 && find_i32(pci, p0, p1, cidx[nn]) >= 0);
      s_wt_w[t] = lump ? v[r0 + t] : 0.0;
      s_wf_w[t] = lump;
    }
    for (int64_t p = s0 + lane; p < s1; p += 32) {
      int32_t k = sci[p];
      int8_t f = 0;
      double term = 0.0;
      if (cf[k] != 1) {
        double aik = csr_get(rp, ci, v, i, k), den = den_g[p];
        if (den != 0.0) {
          double q = dv(aik, den);
          q_g[p] = q;
          double aki = csr_get(rp, ci, v, k, (int32_t)i), akk = csr_get(rp, ci, v, k, k);
          if (opposite(aki, akk)) { term = dm(q, aki); f = 1; }
        } else {
          q_g[p] = 0.0;
          term = aik;
          f = 1;
        }
      }
      s_kt_w[p - s0] = term;
      s_kf_w[p - s0] = f;
    }
    __syncwarp();
    if (lane == 0) {
      at = csr_get(rp, ci, v, i, (int32_t)i);
      for (int64_t t = 0; t < len; ++t)
        if (s_wf_w[t]) at = dd(at, s_wt_w[t]);
      for (int64_t t = 0; t < ns; ++t)
        if (s_kf_w[t]) at = dd(at, s_kt_w[t]);
      rowzero[i] = (at == 0.0);
    }
  } else if (lane == 0) {
    at = csr_get(rp, ci, v, i, (int32_t)i);
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
      int32_t nn = ci[q];
      if (nn == i) continue;
      if (find_i32(sci, s0, s1, nn) >= 0) continue;
      if (cf[nn] == 1 && find_i32(pci, p0, p1, cidx[nn]) >= 0) continue;
      at = dd(at, v[q]);
    }
    for (int64_t p = s0; p < s1; ++p) {
      int32_t k = sci[p];
      if (cf[k] == 1) continue;
      double aik = csr_get(rp, ci, v, i, k), den = den_g[p];
      if (den != 0.0) {
        double q = dv(aik, den);
        q_g[p] = q;
        double aki = csr_get(rp, ci, v, k, (int32_t)i), akk = csr_get(rp, ci, v, k, k);
        if (opposite(aki, akk)) at = dd(at, dm(q, aki));
      } else {
        q_g[p] = 0.0;
        at = dd(at, aik);
      }
    }
    rowzero[i] = (at == 0.0);
  }
  at = __shfl_sync(0xffffffffu, at, 0);
  __syncwarp();
  for (int64_t t = p0 + lane; t < p1; t += 32) {
    int32_t jf = cfine[pci[t]];
    double num = csr_get(rp, ci, v, i, jf);
    for (int64_t p = s0; p < s1; ++p) {
      int32_t k = sci[p];
      if (cf[k] == 1 || den_g[p] == 0.0) continue;
      double akj = csr_get(rp, ci, v, k, jf);
      if (opposite(akj, csr_get(rp, ci, v, k, k))) num = dd(num, dm(q_g[p], akj));
    }
    pv[t] = (at != 0.0) ? -dv(num, at) : 0.0;
  }
}

// The rows listed by the shared-memory kernel, *nrows of them (a count on the device, so the host
// does not wait for it): a warp per listed row, warps striding over the list.
__global__ void __launch_bounds__(32 * EXT_WARPS) k_extpi_weights(const int64_t* rp, const int32_t* ci, const double* v,
                                                                  const int64_t* srp, const int32_t* sci, const int8_t* cf,
                                                                  const int32_t* cidx, const int32_t* cfine,
                                                                  const int64_t* prp, const int32_t* pci, double* pv,
                                                                  double* den_g, double* q_g, int8_t* rowzero,
                                                                  const int32_t* rows, const int* nrows) {
  __shared__ double s_wt[EXT_WARPS][EXT_CAP], s_kt[EXT_WARPS][EXT_CAP];
  __shared__ int8_t s_wf[EXT_WARPS][EXT_CAP], s_kf[EXT_WARPS][EXT_CAP];
  const int w = threadIdx.x >> 5;
  const int nr = *nrows;
  for (int64_t r = (int64_t)blockIdx.x * EXT_WARPS + w; r < nr; r += (int64_t)gridDim.x * EXT_WARPS) {
    extpi_full_row(rows[r], rp, ci, v, srp, sci, cf, cidx, cfine, prp, pci, pv, den_g, q_g, rowzero, s_wt[w], s_kt[w],
                   s_wf[w], s_kf[w]);
    __syncwarp();
  }
}

// The same weights with the row's interpolation columns (fine indices, ascending), its strength
// row, its strong F neighbours with a_ik, and running numerators in shared memory.  One pass over row
// i sets the numerators to a_ij, adds the lumped weak entries to at = a_ii in row order (lane 0, from
// the lanes' shuffled values) and lists the strong F neighbours in ascending order.  The warp then
// walks that list; a neighbour row k of up to 64 entries is loaded once into registers (two per
// lane), its entries are tested against the staged columns in parallel, lane 0 adds den_k's terms
// in row order, and the lanes add q_k a_kl to the numerators of the distinct columns l of row k
// (__syncwarp between successive k).  a_kk comes from the diagonal array.  Every sum is formed in
// the order of k_extpi_weights, so the weights are identical bit for bit.
// It takes the rows that k_extpi_weights_row leaves (rest = 1) within its caps (PCAP interpolation
// columns, KCAP strong neighbours); k_extpi_weights takes the rows beyond those (rest = 2).
constexpr int EXT_PCAP_L = 512, EXT_KCAP_L = 128;

__device__ __forceinline__ int find_sh(const int32_t* a, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && a[lo] == key) ? lo : -1;
}

// lane 0 adds the values x of the lanes in mask m to s, in lane order
__device__ __forceinline__ double ordered_add(unsigned m, double x, double s) {
  const int lane = threadIdx.x & 31;
  while (m) {
    int l = __ffs(m) - 1;
    double y = __shfl_sync(0xffffffffu, x, l);
    if (lane == 0) s = dd(s, y);
    m &= m - 1;
  }
  return s;
}

__global__ void k_diag(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const double* __restrict__ v, double* __restrict__ d) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  d[i] = csr_get(rp, ci, v, i, (int32_t)i);
}

// One thread per row.  The instructions of the FP64 pipe are the scarce resource here (GB300 issues
// about one FP64 warp instruction per 16 SM cycles, whatever its active lanes), and most of the
// arithmetic of a row is sequential (the sums in row order), so each thread takes one row and every
// FP64 warp instruction advances 32 rows.  Membership tests are merge walks of sorted lists (row i
// against its strength row and its interpolation columns; row k against the columns).  The
// interpolation columns and numerators sit in shared memory ([slot][thread]); rows with more than
// EXT_PCAP_T columns are flagged rest = 1 for the warp kernel below.
constexpr int EXT_TPB = 128, EXT_PCAP_T = 8;

// Its loads are one stream per thread, so L1 must hold many rows: the shared stage is kept small
// (EXT_PCAP_T slots per thread; about 3 % of the F rows of a pressure-like operator have more
// interpolation columns and take the warp kernel) and the registers are capped for 12 blocks per SM.
__global__ void __launch_bounds__(EXT_TPB, 12) k_extpi_weights_row(
    int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ v,
    const double* __restrict__ diag, const int64_t* __restrict__ srp, const int32_t* __restrict__ sci,
    const int8_t* __restrict__ cf, const int32_t* __restrict__ cfine, const int64_t* __restrict__ prp,
    const int32_t* __restrict__ pci, double* __restrict__ pv, int8_t* __restrict__ rowzero, int8_t* __restrict__ rest,
    int32_t* __restrict__ over, int* __restrict__ nover) {
  __shared__ int32_t s_pf[EXT_PCAP_T][EXT_TPB];
  __shared__ double s_num[EXT_PCAP_T][EXT_TPB];
  const int64_t i = blockIdx.x * (int64_t)EXT_TPB + threadIdx.x;
  if (i >= n) return;
  const int tx = threadIdx.x;
  if (cf[i] == 1) { pv[prp[i]] = 1.0; rowzero[i] = 0; rest[i] = 0; return; }
  const int64_t p0 = prp[i];
  const int64_t np64 = prp[i + 1] - p0;
  if (np64 > EXT_PCAP_T) { rest[i] = 1; over[atomicAdd(nover, 1)] = (int32_t)i; return; }
  const int np = (int)np64;
  for (int t = 0; t < np; ++t) {
    s_pf[t][tx] = cfine[pci[p0 + t]];
    s_num[t][tx] = 0.0;
  }
  const int64_t r0 = rp[i], r1 = rp[i + 1], s0 = srp[i], s1 = srp[i + 1];
  // row i: numerators a_ij, then at = a_ii plus the lumped weak entries in row order
  double at = diag[i];
  {
    int64_t sp = s0;
    int t = 0;
    for (int64_t q = r0; q < r1; ++q) {
      const int32_t nn = ci[q];
      const double x = v[q];
      while (sp < s1 && sci[sp] < nn) ++sp;
      const bool strong = sp < s1 && sci[sp] == nn;
      while (t < np && s_pf[t][tx] < nn) ++t;
      const bool inp = t < np && s_pf[t][tx] == nn;
      if (inp) s_num[t][tx] = x;
      if (nn != (int32_t)i && !strong && !inp) at = dd(at, x);
    }
  }
  // strong F neighbours k in ascending order (a_ik by a merge walk over row i)
  int64_t q = r0;
  for (int64_t sp = s0; sp < s1; ++sp) {
    const int32_t k = sci[sp];
    while (q < r1 && ci[q] < k) ++q;
    if (cf[k] == 1) continue;
    const double aik = (q < r1 && ci[q] == k) ? v[q] : 0.0;
    const double akk = diag[k];
    const int64_t k0 = rp[k], k1 = rp[k + 1];
    double den = 0.0, aki = 0.0;
    {
      int t = 0;
      for (int64_t u = k0; u < k1; ++u) {
        const int32_t l = ci[u];
        const double x = v[u];
        while (t < np && s_pf[t][tx] < l) ++t;
        const bool inp = t < np && s_pf[t][tx] == l;
        if (l == (int32_t)i) aki = x;
        if ((l == (int32_t)i || inp) && opposite_bits(x, akk)) den = dd(den, x);
      }
    }
    if (den != 0.0) {
      const double qk = dv(aik, den);
      if (opposite_bits(aki, akk)) at = dd(at, dm(qk, aki));
      int t = 0;
      for (int64_t u = k0; u < k1; ++u) {
        const int32_t l = ci[u];
        while (t < np && s_pf[t][tx] < l) ++t;
        if (t < np && s_pf[t][tx] == l) {
          const double x = v[u];
          if (opposite_bits(x, akk)) s_num[t][tx] = dd(s_num[t][tx], dm(qk, x));
        }
      }
    } else {
      at = dd(at, aik);
    }
  }
  rowzero[i] = (at == 0.0);
  rest[i] = 0;
  for (int t = 0; t < np; ++t) pv[p0 + t] = (at != 0.0) ? -dv(s_num[t][tx], at) : 0.0;
}

// pass 1: the rows with rest == 1 (within the caps; others get rest = 2).
template <int PCAP, int KCAP>
__device__ __forceinline__ void extpi_sh_row(
    int64_t i, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ v,
    const double* __restrict__ diag, const int64_t* __restrict__ srp, const int32_t* __restrict__ sci,
    const int8_t* __restrict__ cf, const int32_t* __restrict__ cfine, const int64_t* __restrict__ prp,
    const int32_t* __restrict__ pci, double* __restrict__ pv, int8_t* __restrict__ rowzero, int8_t* __restrict__ rest,
    int32_t* __restrict__ over, int* __restrict__ nover, int32_t* pf, double* num, int32_t* sr, int32_t* s_k_w,
    double* s_aik_w) {
  const int lane = threadIdx.x & 31;
  const int64_t p0 = prp[i], np64 = prp[i + 1] - p0;
  const int64_t s0 = srp[i], ns64 = srp[i + 1] - s0;
  if (np64 > PCAP || ns64 > KCAP) {
    if (lane == 0) { rest[i] = 2; over[atomicAdd(nover, 1)] = (int32_t)i; }
    return;
  }
  const int np = (int)np64, ns = (int)ns64;
  for (int t = lane; t < np; t += 32) {
    pf[t] = cfine[pci[p0 + t]];
    num[t] = 0.0;
  }
  for (int t = lane; t < ns; t += 32) sr[t] = sci[s0 + t];
  __syncwarp();
  // row i: numerators a_ij, lumped weak entries (at = a_ii first), strong F neighbours listed
  const int64_t r0 = rp[i], r1 = rp[i + 1];
  double at = diag[i];
  int nk = 0;
  for (int64_t b = r0; b < r1; b += 32) {
    int64_t q = b + lane;
    bool lump = false, sf = false;
    int32_t nn = -1;
    double val = 0.0;
    if (q < r1) {
      nn = ci[q];
      val = v[q];
      int t = find_sh(pf, np, nn);
      if (t >= 0) num[t] = val;
      bool strong = find_sh(sr, ns, nn) >= 0;
      lump = nn != i && !strong && t < 0;
      sf = strong && cf[nn] != 1;
    }
    at = ordered_add(__ballot_sync(0xffffffffu, lump), val, at);
    unsigned ms = __ballot_sync(0xffffffffu, sf);
    if (sf) {
      int pos = nk + __popc(ms & ((1u << lane) - 1u));
      s_k_w[pos] = nn;
      s_aik_w[pos] = val;
    }
    nk += __popc(ms);
  }
  __syncwarp();
  for (int p = 0; p < nk; ++p) {
    const int32_t k = s_k_w[p];
    const double aik = s_aik_w[p];
    const double akk = diag[k];
    const int64_t k0 = rp[k], k1 = rp[k + 1];
    double den = 0.0, aki = 0.0;
    if (k1 - k0 <= 64) {
      int32_t la = -1, lb = -1;
      double xa = 0.0, xb = 0.0;
      if (k0 + lane < k1) { la = ci[k0 + lane]; xa = v[k0 + lane]; }
      if (k0 + 32 + lane < k1) { lb = ci[k0 + 32 + lane]; xb = v[k0 + 32 + lane]; }
      const int ta = la >= 0 ? find_sh(pf, np, la) : -1;
      const int tb = lb >= 0 ? find_sh(pf, np, lb) : -1;
      const bool oa = opposite(xa, akk), ob = opposite(xb, akk);
      unsigned mi = __ballot_sync(0xffffffffu, la == (int32_t)i);
      if (mi) aki = __shfl_sync(0xffffffffu, xa, __ffs(mi) - 1);
      mi = __ballot_sync(0xffffffffu, lb == (int32_t)i);
      if (mi) aki = __shfl_sync(0xffffffffu, xb, __ffs(mi) - 1);
      den = ordered_add(__ballot_sync(0xffffffffu, (la == (int32_t)i || ta >= 0) && oa), xa, den);
      den = ordered_add(__ballot_sync(0xffffffffu, (lb == (int32_t)i || tb >= 0) && ob), xb, den);
      den = __shfl_sync(0xffffffffu, den, 0);
      if (den != 0.0) {
        const double qk = dv(aik, den);
        if (lane == 0 && opposite(aki, akk)) at = dd(at, dm(qk, aki));
        if (ta >= 0 && oa) num[ta] = dd(num[ta], dm(qk, xa));
        if (tb >= 0 && ob) num[tb] = dd(num[tb], dm(qk, xb));
      } else if (lane == 0) {
        at = dd(at, aik);
      }
    } else {
      for (int64_t b = k0; b < k1; b += 32) {
        int64_t q = b + lane;
        bool in = false;
        double x = 0.0;
        if (q < k1) {
          int32_t l = ci[q];
          x = v[q];
          if (l == (int32_t)i) aki = x;
          in = (l == (int32_t)i || find_sh(pf, np, l) >= 0) && opposite(x, akk);
        }
        den = ordered_add(__ballot_sync(0xffffffffu, in), x, den);
      }
      den = __shfl_sync(0xffffffffu, den, 0);
      unsigned mi = __ballot_sync(0xffffffffu, aki != 0.0);
      aki = mi ? __shfl_sync(0xffffffffu, aki, __ffs(mi) - 1) : 0.0;
      if (den != 0.0) {
        const double qk = dv(aik, den);
        if (lane == 0 && opposite(aki, akk)) at = dd(at, dm(qk, aki));
        for (int64_t b = k0; b < k1; b += 32) {
          int64_t q = b + lane;
          if (q < k1) {
            int32_t l = ci[q];
            double x = v[q];
            int t = find_sh(pf, np, l);
            if (t >= 0 && opposite(x, akk)) num[t] = dd(num[t], dm(qk, x));
          }
        }
      } else if (lane == 0) {
        at = dd(at, aik);
      }
    }
    __syncwarp();
  }
  at = __shfl_sync(0xffffffffu, at, 0);
  if (lane == 0) { rowzero[i] = (at == 0.0); rest[i] = 0; }
  __syncwarp();
  for (int t = lane; t < np; t += 32) pv[p0 + t] = (at != 0.0) ? -dv(num[t], at) : 0.0;
}

// The F rows listed by k_extpi_weights_row, *nrows of them (a count on the device, so the host does
// not wait for it): a warp per listed row, warps striding over the list.
template <int PCAP, int KCAP, int MINB>
__global__ void __launch_bounds__(32 * EXT_WARPS, MINB) k_extpi_weights_sh(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ v,
    const double* __restrict__ diag, const int64_t* __restrict__ srp, const int32_t* __restrict__ sci,
    const int8_t* __restrict__ cf, const int32_t* __restrict__ cfine, const int64_t* __restrict__ prp,
    const int32_t* __restrict__ pci, double* __restrict__ pv, int8_t* __restrict__ rowzero, int8_t* __restrict__ rest,
    const int32_t* __restrict__ rows, const int* __restrict__ nrows, int32_t* __restrict__ over,
    int* __restrict__ nover) {
  __shared__ int32_t s_pf[EXT_WARPS][PCAP];
  __shared__ double s_num[EXT_WARPS][PCAP];
  __shared__ int32_t s_s[EXT_WARPS][KCAP];
  __shared__ int32_t s_k[EXT_WARPS][KCAP];
  __shared__ double s_aik[EXT_WARPS][KCAP];
  const int w = threadIdx.x >> 5;
  const int nr = *nrows;
  for (int64_t r = (int64_t)blockIdx.x * EXT_WARPS + w; r < nr; r += (int64_t)gridDim.x * EXT_WARPS) {
    extpi_sh_row<PCAP, KCAP>(rows[r], rp, ci, v, diag, srp, sci, cf, cfine, prp, pci, pv, rowzero, rest, over, nover,
                             s_pf[w], s_num[w], s_s[w], s_k[w], s_aik[w]);
    __syncwarp();
  }
}

// Keep / truncation: an empty-flagged row keeps nothing; with pmax > 0 a longer F row keeps its pmax
// largest |w| (ties: smaller column) scaled by (sum of all w) / (sum of kept w), sums ascending.
__global__ void k_ptrunc(int64_t n, const int8_t* cf, const int64_t* prp, const double* pv, const int8_t* rowzero,
                         int pmax, int8_t* keep, double* scale, int64_t* cnt) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  int64_t p0 = prp[i], p1 = prp[i + 1];
  int64_t L = p1 - p0;
  bool trunc = cf[i] != 1 && !rowzero[i] && pmax > 0 && L > pmax;
  bool none = cf[i] != 1 && rowzero[i];
  for (int64_t t = p0 + lane; t < p1; t += 32) {
    int8_t k = none ? 0 : 1;
    if (trunc) {
      double a = fabs(pv[t]);
      int64_t rank = 0;
      for (int64_t u = p0; u < p1; ++u) {
        double b = fabs(pv[u]);
        rank += (b > a) || (b == a && u < t);
      }
      k = rank < pmax;
    }
    keep[t] = k;
  }
  __syncwarp();
  if (lane == 0) {
    double f = 1.0;
    if (trunc) {
      double sall = 0.0, skeep = 0.0;
      for (int64_t t = p0; t < p1; ++t) sall = dd(sall, pv[t]);
      for (int64_t t = p0; t < p1; ++t)
        if (keep[t]) skeep = dd(skeep, pv[t]);
      f = (skeep != 0.0) ? dv(sall, skeep) : 1.0;
    }
    scale[i] = f;
    cnt[i] = none ? 0 : (trunc ? pmax : L);
  }
}
__global__ void k_pcompact(int64_t n, const int64_t* prp, const int32_t* pci, const double* pv, const int8_t* keep,
                           const double* scale, bool scaled_rows_only, const int64_t* orp, int32_t* oci, double* ov) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = orp[i];
  double f = scale[i];
  bool full = (orp[i + 1] - o) == (prp[i + 1] - prp[i]);
  for (int64_t t = prp[i]; t < prp[i + 1]; ++t)
    if (keep[t]) { oci[o] = pci[t]; ov[o] = full ? pv[t] : dm(pv[t], f); ++o; }
}

// smoother scaling: l1-Jacobi 1/(a_ii + sign(a_ii) sum_{j!=i}|a_ij|) or omega / a_ii
__global__ void k_smoother_diag(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, int type, double omega,
                                double* dinv, int* err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0, l1 = 0.0;
  // the l1 sum (FP64 additions in row order) only for the l1-Jacobi scaling that uses it
  if (type == 1) {
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] == i) d = v[k];
      else l1 = dd(l1, fabs(v[k]));
    }
  } else {
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) d = v[k];
  }
  double den = (type == 1) ? dd(d, (d >= 0.0) ? l1 : -l1) : d;
  if (den == 0.0 || !isfinite(den)) { atomicOr(err, EBIT_SINGULAR); dinv[i] = 0.0; return; }
  dinv[i] = (type == 1) ? dv(1.0, den) : dv(omega, den);
}

static uint64_t host_splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

static void strength(Ctx& c, const DCSR<double>& A, double theta, DCSR<double>& S) {
  int64_t n = A.nr;
  DBuf<int64_t> cnt(c, n + 1);
  unsigned g = grid_for(n * 32, 256);
  k_strength<0><<<g, 256, 0, c.s>>>(n, A.rp, A.ci, A.v, theta, cnt.p, nullptr, nullptr);
  CU_LAUNCH();
  S.nr = S.nc = n;
  S.rp.alloc(c, n + 1);
  S.nnz = counts_to_rowptr(c, cnt.p, S.rp.p, n);
  S.ci.alloc(c, S.nnz);
  k_strength<1><<<g, 256, 0, c.s>>>(n, A.rp, A.ci, A.v, theta, nullptr, S.rp.p, S.ci.p);
  CU_LAUNCH();
}

// returns the number of C points
static int64_t pmis(Ctx& c, const DCSR<double>& S, uint64_t seed, int lev, DBuf<int8_t>& cf) {
  int64_t n = S.nr;
  DCSR<double> St;
  transpose(c, S, St);
  DBuf<double> w(c, n);
  DBuf<int8_t> nc(c, n);
  DBuf<int> und(c, 2);  // undecided points, C points
  cf.alloc(c, n);
  const int B = 256;
  uint64_t key = host_splitmix64(seed ^ ((uint64_t)(lev + 1) << 48));
  CU(cudaMemsetAsync(und.p, 0, 2 * sizeof(int), c.s));
  k_pmis_init<<<grid_for(n, B), B, 0, c.s>>>(n, St.rp, key, w.p, cf.p, und.p);
  CU_LAUNCH();
  int rounds = 0;
  // the undecided count is read back after every second round, and not before the first: a round
  // after the last decision selects nothing and marks nothing, so the splitting is the same, with
  // fewer host round trips; the C points are counted on the device and read with it
  int left = 1, ncount = 0;
  while (left > 0) {
    for (int r = 0; r < 2; ++r) {
      if (++rounds > 10000) throw Error(MGR_ERR_CUDA, "PMIS did not terminate");
      k_pmis_select<<<grid_for(n, B), B, 0, c.s>>>(n, S.rp, S.ci, St.rp, St.ci, w.p, cf.p, nc.p);
      CU_LAUNCH();
      k_pmis_mark_c<<<grid_for(n, B), B, 0, c.s>>>(n, nc.p, cf.p, und.p + 1);
      CU_LAUNCH();
      CU(cudaMemsetAsync(und.p, 0, sizeof(int), c.s));
      k_pmis_mark_f<<<grid_for(n, B), B, 0, c.s>>>(n, S.rp, S.ci, cf.p, und.p);
      CU_LAUNCH();
    }
    read_back(c, {{und.p, &left, sizeof(int)}, {und.p + 1, &ncount, sizeof(int)}});
  }
  return ncount;
}

static void extpi(Ctx& c, const DCSR<double>& A, const DCSR<double>& S, const DBuf<int8_t>& cf, int64_t nC, int pmax,
                  DCSR<double>& P) {
  int64_t n = A.nr;
  const int B = 256;
  DBuf<int32_t> flag(c, n), pre(c, n + 1), cidx(c, n), cfine(c, nC + 1);
  k_flag_c<<<grid_for(n, B), B, 0, c.s>>>(n, cf.p, flag.p);
  CU_LAUNCH();
  scan_excl_i32(c, flag.p, pre.p, n);
  k_cidx<<<grid_for(n, B), B, 0, c.s>>>(n, cf.p, pre.p, cidx.p, cfine.p);
  CU_LAUNCH();
  // selection matrices and the symbolic product
  DCSR<double> M, T, Q;
  {
    DBuf<int64_t> cm(c, n + 1), ct(c, n + 1);
    k_extpi_sel_count<<<grid_for(n, B), B, 0, c.s>>>(n, S.rp, S.ci, cf.p, cm.p, ct.p);
    CU_LAUNCH();
    M.nr = n; M.nc = n; M.rp.alloc(c, n + 1);
    T.nr = n; T.nc = nC; T.rp.alloc(c, n + 1);
    scan_excl_i64(c, cm.p, M.rp.p, n);
    scan_excl_i64(c, ct.p, T.rp.p, n);
    read_back(c, {{M.rp.p + n, &M.nnz, sizeof(int64_t)}, {T.rp.p + n, &T.nnz, sizeof(int64_t)}});
    M.ci.alloc(c, M.nnz);
    T.ci.alloc(c, T.nnz);
    k_extpi_sel_fill<<<grid_for(n, B), B, 0, c.s>>>(n, S.rp, S.ci, cf.p, cidx.p, M.rp, M.ci, T.rp, T.ci);
    CU_LAUNCH();
  }
  // pattern of M T through the fused product (unit values; only the pattern is used)
  M.v.alloc(c, M.nnz);
  T.v.alloc(c, T.nnz);
  fill_f64(c, M.v.p, 1.0, M.nnz);
  fill_f64(c, T.v.p, 1.0, T.nnz);
  {
    ProfScope ps(c, "extpi_pattern");
    spgemm(c, M, T, Q, "spgemm_extpi");
  }
  DCSR<double> Pf;
  {
    DBuf<int64_t> cnt(c, n + 1);
    k_pfull_count<<<grid_for(n, B), B, 0, c.s>>>(n, cf.p, Q.rp, cnt.p);
    CU_LAUNCH();
    // M has no rows at C points, so Q's F rows hold all its entries: P_full has those and one per C point
    csr_rows(c, Pf, n, nC, cnt.p);
    Pf.nnz = Q.nnz + nC;
    csr_alloc(c, Pf);
    k_pfull_fill<<<grid_for(n, B), B, 0, c.s>>>(n, cf.p, cidx.p, Q.rp, Q.ci, Pf.rp, Pf.ci);
    CU_LAUNCH();
  }
  DBuf<double> den(c, S.nnz + 1), q(c, S.nnz + 1), scale(c, n);
  DBuf<int8_t> rowzero(c, n), keep(c, Pf.nnz + 1), rest(c, n);
  ProfScope psw(c, "extpi_weights");
  DBuf<double> diag(c, n);
  k_diag<<<grid_for(n, B), B, 0, c.s>>>(n, A.rp, A.ci, A.v, diag.p);
  CU_LAUNCH();
  DBuf<int32_t> list1(c, n), list2(c, n);
  DBuf<int> nl(c, 2);
  CU(cudaMemsetAsync(nl.p, 0, 2 * sizeof(int), c.s));
  k_extpi_weights_row<<<grid_for(n, EXT_TPB), EXT_TPB, 0, c.s>>>(n, A.rp, A.ci, A.v, diag.p, S.rp, S.ci, cf.p,
                                                                 cfine.p, Pf.rp, Pf.ci, Pf.v, rowzero.p, rest.p,
                                                                 list1.p, nl.p);
  CU_LAUNCH();
  // the rows with more interpolation columns than the thread-per-row stage holds (a few %), then
  // those beyond the warp kernel's caps (rare): warps stride over their lists, whose lengths stay on
  // the device
  k_extpi_weights_sh<EXT_PCAP_L, EXT_KCAP_L, 1><<<8 * c.num_sms, 32 * EXT_WARPS, 0, c.s>>>(
      A.rp, A.ci, A.v, diag.p, S.rp, S.ci, cf.p, cfine.p, Pf.rp, Pf.ci, Pf.v, rowzero.p, rest.p, list1.p, nl.p, list2.p,
      nl.p + 1);
  CU_LAUNCH();
  k_extpi_weights<<<2 * c.num_sms, 32 * EXT_WARPS, 0, c.s>>>(A.rp, A.ci, A.v, S.rp, S.ci, cf.p, cidx.p, cfine.p, Pf.rp,
                                                              Pf.ci, Pf.v, den.p, q.p, rowzero.p, list2.p, nl.p + 1);
  CU_LAUNCH();
  DBuf<int64_t> cnt(c, n + 1);
  k_ptrunc<<<grid_for(n * 32, 128), 128, 0, c.s>>>(n, cf.p, Pf.rp, Pf.v, rowzero.p, pmax, keep.p, scale.p, cnt.p);
  CU_LAUNCH();
  alloc_csr(c, P, n, nC, cnt.p);
  k_pcompact<<<grid_for(n, B), B, 0, c.s>>>(n, Pf.rp, Pf.ci, Pf.v, keep.p, scale.p, true, P.rp, P.ci, P.v);
  CU_LAUNCH();
}

void amg_build(Ctx& c, DCSR<double>& A0, bool take, const AmgOpts& o, std::vector<AmgLevel>& lv,
               DBuf<double>& cinv, int64_t& nco, const std::function<void(AmgLevel&)>& done) {
  lv.clear();
  lv.emplace_back();
  if (take) {
    DCSR<double>& D = lv[0].A;
    D.nr = A0.nr; D.nc = A0.nc; D.nnz = A0.nnz;
    D.rp = std::move(A0.rp);
    D.ci = std::move(A0.ci);
    D.v = std::move(A0.v);
  } else {
    copy_csr(c, A0, lv[0].A);
  }
  lv[0].n = A0.nr;
  int maxlev = o.max_levels;
  const int B = 256;
  int k = 0;
  while (lv[k].n > o.max_coarse && k < maxlev - 1) {
    AmgLevel& L = lv[k];
    int64_t n = L.n;
    {
      ProfScope ps(c, "setup_amg_strength");
      strength(c, L.A, o.theta, L.S);
    }
    int64_t nC;
    {
      ProfScope ps(c, "setup_amg_pmis");
      nC = pmis(c, L.S, o.seed, k, L.cf);
    }
    if (nC == 0 || nC == n) {
      L.cf.release();
      L.S = DCSR<double>();
      break;
    }
    {
      ProfScope ps(c, "setup_amg_extpi");
      extpi(c, L.A, L.S, L.cf, nC, o.pmax, L.P);
    }
    {
      ProfScope ps(c, "setup_amg_transpose");
      transpose(c, L.P, L.R);
    }
    L.dinv.alloc(c, n);
    // a zero or non-finite diagonal sets the error word, checked once with the coarsest inverse (the
    // scalings are first read by the apply)
    k_smoother_diag<<<grid_for(n, B), B, 0, c.s>>>(n, L.A.rp, L.A.ci, L.A.v, o.smoother, o.omega, L.dinv.p, c.d_err);
    CU_LAUNCH();
    AmgLevel next;
    {
      ProfScope ps(c, "setup_amg_rap");
      DCSR<double> AP;
      static const char* const kAP[] = {"rap_amg0_AP", "rap_amg1_AP", "rap_amgc_AP"};
      static const char* const kPAP[] = {"rap_amg0_PtAP", "rap_amg1_PtAP", "rap_amgc_PtAP"};
      const int ki = k < 2 ? k : 2;
      spgemm(c, L.A, L.P, AP, kAP[ki]);
      spgemm(c, L.R, AP, next.A, kPAP[ki]);
    }
    next.n = nC;
    lv.push_back(std::move(next));
    if (done) done(lv[k]);
    ++k;
  }
  nco = lv.back().n;
  if (nco > 4096) throw Error(MGR_ERR_UNSUPPORTED, "AMG coarsest grid larger than 4096 rows");
  ProfScope ps(c, "setup_dense_inverse");
  dense_inverse(c, lv.back().A, cinv);
  check_errors(c, "AMG smoother diagonal or coarsest inverse");
}

// ===================================== dense inverse ==========================================
__global__ void k_dense_from_csr(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double* M) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* row = M + i * 2 * n;
  for (int64_t j = 0; j < 2 * n; ++j) row[j] = 0.0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) row[ci[k]] = dd(row[ci[k]], v[k]);
  row[n + i] = 1.0;
}
// pivot search on column k (rows k..n-1, largest |.|, first on ties), row swap and row scaling
__global__ void k_gj_pivot(int64_t n, int64_t k, double* M, int* err) {
  __shared__ double bv[1024];
  __shared__ int64_t bi[1024];
  int64_t w = 2 * n;
  double best = -1.0;
  int64_t arg = n;
  for (int64_t i = k + threadIdx.x; i < n; i += blockDim.x) {
    double a = fabs(M[i * w + k]);
    if (a > best) { best = a; arg = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double a = bv[threadIdx.x + s];
      int64_t ia = bi[threadIdx.x + s];
      if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ia < bi[threadIdx.x])) { bv[threadIdx.x] = a; bi[threadIdx.x] = ia; }
    }
    __syncthreads();
  }
  int64_t p = bi[0];
  if (bv[0] == 0.0 || !isfinite(bv[0]) || p >= n) {
    if (threadIdx.x == 0) atomicOr(err, EBIT_SINGULAR);
    return;
  }
  if (p != k)
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) {
      double t = M[k * w + j];
      M[k * w + j] = M[p * w + j];
      M[p * w + j] = t;
    }
  __syncthreads();
  double piv = M[k * w + k];
  __syncthreads();
  for (int64_t j = threadIdx.x; j < w; j += blockDim.x) M[k * w + j] = dv(M[k * w + j], piv);
}
// eliminate column k from every other row (one block per row)
__global__ void k_gj_eliminate(int64_t n, int64_t k, double* M) {
  int64_t i = blockIdx.x;
  if (i == k) return;
  int64_t w = 2 * n;
  __shared__ double f;
  if (threadIdx.x == 0) f = M[i * w + k];
  __syncthreads();
  if (f == 0.0) return;
  for (int64_t j = threadIdx.x; j < w; j += blockDim.x) M[i * w + j] = __dsub_rn(M[i * w + j], dm(f, M[k * w + j]));
}
__global__ void k_dense_right_half(int64_t n, const double* M, double* inv) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  int64_t i = t / n, j = t - i * n;
  inv[t] = M[i * 2 * n + n + j];
}

// The same Gauss-Jordan elimination in one block for n <= GJ_ONE (the coarsest AMG grids): the
// pivot search, the row swap, the scaling and the elimination of each column are separated by block
// barriers instead of kernel boundaries, with the same operations in the same order (the multipliers
// of column k are read before any row is updated), so the inverse is the one of the two-kernel form.
constexpr int64_t GJ_ONE = 1024;
__global__ void __launch_bounds__(1024) k_gj_one(int64_t n, double* M, int* err) {
  __shared__ double bv[1024];
  __shared__ int64_t bi[1024];
  __shared__ double f[GJ_ONE];
  const int64_t w = 2 * n;
  for (int64_t k = 0; k < n; ++k) {
    double best = -1.0;
    int64_t arg = n;
    for (int64_t i = k + threadIdx.x; i < n; i += blockDim.x) {
      double a = fabs(M[i * w + k]);
      if (a > best) { best = a; arg = i; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = arg;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        double a = bv[threadIdx.x + st];
        int64_t ia = bi[threadIdx.x + st];
        if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ia < bi[threadIdx.x])) { bv[threadIdx.x] = a; bi[threadIdx.x] = ia; }
      }
      __syncthreads();
    }
    const int64_t p = bi[0];
    if (bv[0] == 0.0 || !isfinite(bv[0]) || p >= n) {  // uniform over the block
      if (threadIdx.x == 0) atomicOr(err, EBIT_SINGULAR);
      return;
    }
    if (p != k)
      for (int64_t j = threadIdx.x; j < w; j += blockDim.x) {
        double t = M[k * w + j];
        M[k * w + j] = M[p * w + j];
        M[p * w + j] = t;
      }
    __syncthreads();
    const double piv = M[k * w + k];
    __syncthreads();
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) M[k * w + j] = dv(M[k * w + j], piv);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) f[i] = M[i * w + k];
    __syncthreads();
    for (int64_t e = threadIdx.x; e < n * w; e += blockDim.x) {
      const int64_t i = e / w, j = e - i * w;
      if (i != k && f[i] != 0.0) M[e] = __dsub_rn(M[e], dm(f[i], M[k * w + j]));
    }
    __syncthreads();
  }
}

void dense_inverse(Ctx& c, const DCSR<double>& A, DBuf<double>& inv) {
  int64_t n = A.nr;
  inv.alloc(c, n * n);
  if (n == 0) return;
  DBuf<double> M(c, 2 * n * n);
  k_dense_from_csr<<<grid_for(n, 128), 128, 0, c.s>>>(n, A.rp, A.ci, A.v, M.p);
  CU_LAUNCH();
  if (n <= GJ_ONE) {
    k_gj_one<<<1, 1024, 0, c.s>>>(n, M.p, c.d_err);
    CU_LAUNCH();
  } else {
    for (int64_t k = 0; k < n; ++k) {
      k_gj_pivot<<<1, 1024, 0, c.s>>>(n, k, M.p, c.d_err);
      CU_LAUNCH();
      k_gj_eliminate<<<(unsigned)n, 128, 0, c.s>>>(n, k, M.p);
      CU_LAUNCH();
    }
  }
  k_dense_right_half<<<grid_for(n * n, 256), 256, 0, c.s>>>(n, M.p, inv.p);
  CU_LAUNCH();
}

}  // namespace mgr
