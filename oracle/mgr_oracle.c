/*
 * mgr_oracle.c -- TEST INFRASTRUCTURE.  A plain, slow, single-threaded FP64 CPU restatement of
 * MGR-preconditioned flexible GMRES for the 3x3-block NCP Jacobians of Bui, Wang & Osei-Kuffuor.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load it; the GPU library
 * shares no code with it.  Compile with -ffp-contract=off so that no multiply-add is fused: the
 * setup arithmetic (level operators, strength, PMIS weights, interpolation) is written in a fixed
 * order of IEEE operations so that an independent implementation that follows the same order gets
 * the same bits.
 *
 * Passages followed (sections of the paper):
 *   section 4, two-level reduction: C/F splitting, Schur complement S = A_cc - A_cf A_ff^-1 A_fc,
 *     ideal P and R, the MGR identities (additive / multiplicative), approximate operators
 *     P = [W_p; I], R = [W_r, I] with W_p = -D_ff^-1 A_fc and W_r = 0 (injective) or
 *     W_r = -A_cf D_ff^-1 (non-injective), D_ff = diag(A_ff); coarse operator A_c = R A P;
 *   section 4, Algorithm "MGR preconditioner with presmoothing": (1) global relaxation with
 *     blockdiag(A)^-1, (2) F-relaxation e += Q M_ff^-1 Q^T (r - A e), (3) coarse correction
 *     e += P M_c^-1 R_I (r - A e);
 *   section 5, three-level reduction order for the two-phase two-component model: level 1 removes
 *     the constraint rows with nonzero C33 (rho of gas-present cells), level 2 the saturations,
 *     level 3 the constraints with zero diagonal (rho of gas-absent cells), leaving P_l for AMG;
 *   section 6 (experiments): GMRES as the outer Krylov method, AMG for the coarse solve.
 * Components the paper leaves to BoomerAMG are taken from their own publications: PMIS coarsening
 * (De Sterck, Yang & Heys 2006), extended+i interpolation (De Sterck, Falgout, Nolting & Yang 2008),
 * l1-Jacobi smoothing (Baker, Falgout, Kolev & Yang 2011), flexible GMRES (Saad 1993).
 * Readings where the paper is silent are stated at each function.
 * Parity unpinned: the PMIS tie rule between exactly equal weights (the larger index wins).  The
 * weights carry 53 random bits, so ties do not occur in any output a test can observe; every other
 * part is pinned by the CPU tests against closed forms, dense solves and brute force.
 *
 * Sparse matrices are CSR with int64 row pointers, int32 columns sorted ascending, FP64 values.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define O_OK 0
#define O_EINVAL 1
#define O_ESINGULAR 2
#define O_ENOTCONV 3
#define O_EBREAKDOWN 4
#define O_ENOMEM 5

#define MAXLEV 8
#define MAXAMG 32

typedef struct {
  int32_t global_relax;        /* Algorithm step (1) at the finest level */
  int32_t frelax_type[MAXLEV]; /* 0: omega-Jacobi, 1: l1-Jacobi, 2: AMG V(1,1)-cycle on A_ff */
  int32_t frelax_sweeps[MAXLEV];
  double frelax_omega[MAXLEV];
  int32_t restrict_type[MAXLEV]; /* 0: injective W_r = 0; 1: W_r = -A_cf D_ff^-1 */
  int32_t apply_full_R;          /* 0: restrict with R_I (injection) as in the Algorithm; 1: full R */
  int32_t coarse_solver;         /* 0: AMG V-cycle; 1: dense direct solve of the last level */
  double amg_theta;
  int32_t amg_max_levels;
  int32_t amg_max_coarse;
  int32_t amg_smoother;          /* 0: omega-Jacobi, 1: l1-Jacobi */
  int32_t amg_pre, amg_post;
  int32_t amg_pmax;              /* 0: no truncation of interpolation */
  double amg_omega;
  uint64_t amg_seed;
  int32_t ideal;                 /* 1: exact A_ff^-1 in P and in F-relaxation, exact coarse solve */
  int32_t pad_;
} oopts_t;

typedef struct {
  int32_t iterations, restarts, converged, status;
  double relres_true, relres_est, bnorm;
} oinfo_t;

typedef struct {
  int64_t nr, nc, nnz;
  int64_t* rp;
  int32_t* ci;
  double* v;
} csr_t;

static void* xmalloc(size_t n) { return malloc(n ? n : 1); }
static void* xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

static void csr_free(csr_t* a) {
  free(a->rp); free(a->ci); free(a->v);
  memset(a, 0, sizeof *a);
}
static int csr_alloc(csr_t* a, int64_t nr, int64_t nc, int64_t nnz) {
  a->nr = nr; a->nc = nc; a->nnz = nnz;
  a->rp = (int64_t*)xcalloc((size_t)nr + 1, sizeof(int64_t));
  a->ci = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)nnz);
  a->v = (double*)xmalloc(sizeof(double) * (size_t)nnz);
  return (a->rp && a->ci && a->v) ? O_OK : O_ENOMEM;
}
static int csr_copy(const csr_t* s, csr_t* d) {
  if (csr_alloc(d, s->nr, s->nc, s->nnz)) return O_ENOMEM;
  memcpy(d->rp, s->rp, sizeof(int64_t) * (size_t)(s->nr + 1));
  memcpy(d->ci, s->ci, sizeof(int32_t) * (size_t)s->nnz);
  memcpy(d->v, s->v, sizeof(double) * (size_t)s->nnz);
  return O_OK;
}
/* value of entry (i, j), 0 if not stored */
static double csr_get(const csr_t* a, int64_t i, int32_t j) {
  int64_t lo = a->rp[i], hi = a->rp[i + 1] - 1;
  while (lo <= hi) {
    int64_t m = (lo + hi) >> 1;
    if (a->ci[m] == j) return a->v[m];
    if (a->ci[m] < j) lo = m + 1; else hi = m - 1;
  }
  return 0.0;
}
/* y = b - A x (or y = A x when b == NULL), plain row loop */
static void csr_resid(const csr_t* a, const double* x, const double* b, double* y) {
  for (int64_t i = 0; i < a->nr; ++i) {
    double s = 0.0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) s += a->v[k] * x[a->ci[k]];
    y[i] = b ? b[i] - s : s;
  }
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* C = A * B, structural pattern (every product position is stored, no dropping), each entry summed
 * in ascending intermediate index k (Gustavson's row-by-row product). */
static int spgemm(const csr_t* A, const csr_t* B, csr_t* C) {
  int64_t m = A->nr, n = B->nc;
  int64_t* mark = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n);
  double* acc = (double*)xcalloc((size_t)n, sizeof(double));
  if (!mark || !acc) return O_ENOMEM;
  for (int64_t j = 0; j < n; ++j) mark[j] = -1;
  C->nr = m; C->nc = n;
  C->rp = (int64_t*)xcalloc((size_t)m + 1, sizeof(int64_t));
  for (int64_t i = 0; i < m; ++i) {
    int64_t cnt = 0;
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int32_t k = A->ci[p];
      for (int64_t q = B->rp[k]; q < B->rp[k + 1]; ++q) {
        int32_t j = B->ci[q];
        if (mark[j] != i) { mark[j] = i; ++cnt; }
      }
    }
    C->rp[i + 1] = C->rp[i] + cnt;
  }
  C->nnz = C->rp[m];
  C->ci = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)C->nnz);
  C->v = (double*)xmalloc(sizeof(double) * (size_t)C->nnz);
  if (!C->ci || !C->v) return O_ENOMEM;
  for (int64_t j = 0; j < n; ++j) mark[j] = -1;
  for (int64_t i = 0; i < m; ++i) {
    int64_t o = C->rp[i], cnt = 0;
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int32_t k = A->ci[p];
      for (int64_t q = B->rp[k]; q < B->rp[k + 1]; ++q) {
        int32_t j = B->ci[q];
        if (mark[j] != i) { mark[j] = i; C->ci[o + cnt++] = j; }
      }
    }
    qsort(C->ci + o, (size_t)cnt, sizeof(int32_t), cmp_i32);
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int32_t k = A->ci[p];
      double a = A->v[p];
      for (int64_t q = B->rp[k]; q < B->rp[k + 1]; ++q) acc[B->ci[q]] += a * B->v[q];
    }
    for (int64_t t = 0; t < cnt; ++t) { C->v[o + t] = acc[C->ci[o + t]]; acc[C->ci[o + t]] = 0.0; }
  }
  free(mark); free(acc);
  return O_OK;
}

/* B = A^T with rows sorted by column (counting sort keeps ascending order). */
static int transpose(const csr_t* A, csr_t* T) {
  if (csr_alloc(T, A->nc, A->nr, A->nnz)) return O_ENOMEM;
  for (int64_t k = 0; k < A->nnz; ++k) T->rp[A->ci[k] + 1]++;
  for (int64_t j = 0; j < A->nc; ++j) T->rp[j + 1] += T->rp[j];
  int64_t* pos = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)(A->nc + 1));
  memcpy(pos, T->rp, sizeof(int64_t) * (size_t)(A->nc + 1));
  for (int64_t i = 0; i < A->nr; ++i)
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
      int64_t d = pos[A->ci[k]]++;
      T->ci[d] = (int32_t)i;
      T->v[d] = A->v[k];
    }
  free(pos);
  return O_OK;
}

/* ---- dense LU with partial pivoting (row-major), used for the coarsest grid and ideal mode ---- */
static int lu_factor(int64_t n, double* a, int32_t* piv) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    double best = fabs(a[k * n + k]);
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
    piv[k] = (int32_t)p;
    if (best == 0.0) return O_ESINGULAR;
    if (p != k)
      for (int64_t j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
    for (int64_t i = k + 1; i < n; ++i) {
      double l = a[i * n + k] / a[k * n + k];
      a[i * n + k] = l;
      for (int64_t j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return O_OK;
}
static void lu_solve(int64_t n, const double* a, const int32_t* piv, double* x) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = piv[k];
    if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
  }
  for (int64_t i = 0; i < n; ++i) {
    double s = x[i];
    for (int64_t j = 0; j < i; ++j) s -= a[i * n + j] * x[j];
    x[i] = s;
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int64_t j = i + 1; j < n; ++j) s -= a[i * n + j] * x[j];
    x[i] = s / a[i * n + i];
  }
}
static double* csr_to_dense(const csr_t* a) {
  double* d = (double*)xcalloc((size_t)(a->nr * a->nc), sizeof(double));
  for (int64_t i = 0; i < a->nr; ++i)
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) d[i * a->nc + a->ci[k]] += a->v[k];
  return d;
}

/* ---- splitmix64 (Steele, Lea & Flood 2014) for the PMIS tie-breaking weights ----------------- */
static inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
/* u in [0,1) for point i of AMG level lev: key = splitmix64(seed ^ ((lev+1) << 48)),
 * u = top 53 bits of splitmix64(key ^ i) scaled by 2^-53. */
static inline double pmis_u(uint64_t seed, int lev, int64_t i) {
  uint64_t key = splitmix64(seed ^ ((uint64_t)(lev + 1) << 48));
  return (double)(splitmix64(key ^ (uint64_t)i) >> 11) * 0x1.0p-53;
}

/* =============================== AMG (coarse solve M_c^-1) ==================================== */
typedef struct {
  int nlev;
  csr_t A[MAXAMG], P[MAXAMG], R[MAXAMG], S[MAXAMG];
  double* dinv[MAXAMG];
  int8_t* cf[MAXAMG]; /* 1 = C, -1 = F */
  int64_t nco;
  double* lu;
  int32_t* piv;
  int pre, post;
} amg_t;

/* Strength (classical, sign-aware): with s = +1 if a_ii >= 0 else -1, j != i is a strong
 * connection of i iff -s a_ij >= theta * max_{k != i}(-s a_ik) and that maximum is positive. */
static int strength(const csr_t* A, double theta, csr_t* S) {
  int64_t n = A->nr;
  S->nr = n; S->nc = n;
  S->rp = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  S->ci = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)A->nnz);
  S->v = NULL;
  int64_t o = 0;
  for (int64_t i = 0; i < n; ++i) {
    double d = csr_get(A, i, (int32_t)i);
    double s = (d >= 0.0) ? 1.0 : -1.0;
    double m = 0.0;
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
      if (A->ci[k] == i) continue;
      double v = -(s * A->v[k]);
      if (v > m) m = v;
    }
    if (m > 0.0) {
      double thr = theta * m;
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
        if (A->ci[k] == i) continue;
        double v = -(s * A->v[k]);
        if (v >= thr) S->ci[o++] = A->ci[k];
      }
    }
    S->rp[i + 1] = o;
  }
  S->nnz = o;
  return O_OK;
}

/* PMIS C/F splitting.  lambda_i = number of points that strongly depend on i; w_i = lambda_i + u_i.
 * Points with lambda_i = 0 start as F.  Each round, an undecided point whose (w, index) beats every
 * undecided strong neighbour (in S and S^T; larger index wins equal weights) becomes C; then every
 * undecided point that strongly depends on a C point becomes F.  Rounds are synchronous. */
static int pmis(const csr_t* S, uint64_t seed, int lev, int8_t* cf) {
  int64_t n = S->nr;
  csr_t St;
  memset(&St, 0, sizeof St);
  csr_t Sv = *S;
  Sv.v = (double*)xcalloc((size_t)S->nnz, sizeof(double));
  transpose(&Sv, &St);
  free(Sv.v);
  double* w = (double*)xmalloc(sizeof(double) * (size_t)n);
  int8_t* nc = (int8_t*)xcalloc((size_t)n, 1);
  int64_t und = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t lam = St.rp[i + 1] - St.rp[i];
    w[i] = (double)lam + pmis_u(seed, lev, i);
    cf[i] = (lam == 0) ? -1 : 0;
    if (!lam) continue;
    ++und;
  }
  while (und > 0) {
    for (int64_t i = 0; i < n; ++i) {
      nc[i] = 0;
      if (cf[i] != 0) continue;
      int ok = 1;
      for (int pass = 0; pass < 2 && ok; ++pass) {
        const csr_t* G = pass ? &St : S;
        for (int64_t k = G->rp[i]; k < G->rp[i + 1]; ++k) {
          int32_t j = G->ci[k];
          if (j == i || cf[j] != 0) continue;
          if (w[j] > w[i] || (w[j] == w[i] && j > i)) { ok = 0; break; }
        }
      }
      nc[i] = (int8_t)ok;
    }
    for (int64_t i = 0; i < n; ++i) if (nc[i]) { cf[i] = 1; --und; }
    for (int64_t i = 0; i < n; ++i) {
      if (cf[i] != 0) continue;
      for (int64_t k = S->rp[i]; k < S->rp[i + 1]; ++k)
        if (cf[S->ci[k]] == 1) { cf[i] = -1; --und; break; }
    }
  }
  csr_free(&St); free(w); free(nc);
  return O_OK;
}

static inline int opposite(double a, double d) { return (d > 0.0 && a < 0.0) || (d < 0.0 && a > 0.0); }

/* Extended+i interpolation.  For an F point i with strong C neighbours C_i^s and strong F
 * neighbours F_i^s: Chat_i = C_i^s united with C_k^s for k in F_i^s; abar_kl keeps a_kl only when
 * its sign is opposite to a_kk.  For each k in F_i^s, den_k = sum of abar_kl over l in Chat_i + {i}
 * (ascending l); when den_k != 0, q_k = a_ik / den_k distributes a_ik, otherwise a_ik is lumped into
 * the diagonal (reading where the publication leaves the zero case open).  Diagonal:
 *   at = a_ii + sum (weak neighbours not in Chat_i, ascending) a_in
 *        + sum (k in F_i^s, ascending) [den_k != 0 ? q_k abar_ki : a_ik]
 * Weight for j in Chat_i (ascending): num = a_ij + sum_k q_k abar_kj (k ascending), w_ij = -(num/at).
 * A C point interpolates by injection; an F point with at == 0 gets an empty row.
 * With pmax > 0 the row keeps its pmax largest |w| (ties: smaller column) scaled by
 * (sum of all w) / (sum of kept w). */
static int extpi(const csr_t* A, const csr_t* S, const int8_t* cf, int pmax, csr_t* P) {
  int64_t n = A->nr, nC = 0;
  int32_t* cidx = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) cidx[i] = (cf[i] == 1) ? (int32_t)nC++ : -1;
  int32_t* cfine = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)(nC ? nC : 1));
  for (int64_t i = 0; i < n; ++i) if (cidx[i] >= 0) cfine[cidx[i]] = (int32_t)i;
  int32_t* inC = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)(nC ? nC : 1)); /* coarse -> slot */
  for (int64_t c = 0; c < nC; ++c) inC[c] = -1;
  int64_t* smark = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) smark[i] = -1;
  /* worst-case row lengths for allocation */
  int64_t cap = 0;
  int64_t* rb = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    int64_t b = 1;
    if (cf[i] != 1)
      for (int64_t k = S->rp[i]; k < S->rp[i + 1]; ++k) {
        int32_t j = S->ci[k];
        if (cf[j] == 1) ++b; else b += S->rp[j + 1] - S->rp[j];
      }
    rb[i + 1] = rb[i] + b;
    if (b > cap) cap = b;
  }
  int32_t* rowc = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)cap);
  double* roww = (double*)xmalloc(sizeof(double) * (size_t)cap);
  int32_t* fk = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)(cap + 1));
  double* qk = (double*)xmalloc(sizeof(double) * (size_t)(cap + 1));
  int32_t* ord = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)cap);
  csr_t T;
  memset(&T, 0, sizeof T);
  T.nr = n; T.nc = nC;
  T.rp = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  T.ci = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)rb[n]);
  T.v = (double*)xmalloc(sizeof(double) * (size_t)rb[n]);
  int64_t o = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (cf[i] == 1) { T.ci[o] = cidx[i]; T.v[o] = 1.0; ++o; T.rp[i + 1] = o; continue; }
    /* Chat_i */
    int64_t nc_ = 0, nf = 0;
    for (int64_t k = S->rp[i]; k < S->rp[i + 1]; ++k) {
      int32_t j = S->ci[k];
      smark[j] = i;
      if (cf[j] == 1) { if (inC[cidx[j]] < 0) { inC[cidx[j]] = 0; rowc[nc_++] = cidx[j]; } }
      else {
        fk[nf++] = j;
        for (int64_t l = S->rp[j]; l < S->rp[j + 1]; ++l) {
          int32_t c = S->ci[l];
          if (cf[c] == 1 && inC[cidx[c]] < 0) { inC[cidx[c]] = 0; rowc[nc_++] = cidx[c]; }
        }
      }
    }
    qsort(rowc, (size_t)nc_, sizeof(int32_t), cmp_i32);
    for (int64_t t = 0; t < nc_; ++t) inC[rowc[t]] = (int32_t)t;
    /* den_k, q_k */
    for (int64_t t = 0; t < nf; ++t) {
      int32_t k = fk[t];
      double akk = csr_get(A, k, k), den = 0.0;
      for (int64_t p = A->rp[k]; p < A->rp[k + 1]; ++p) {
        int32_t l = A->ci[p];
        int in = (l == i) || (cf[l] == 1 && inC[cidx[l]] >= 0);
        if (in && opposite(A->v[p], akk)) den += A->v[p];
      }
      qk[t] = den;
    }
    double at = 0.0;
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) if (A->ci[p] == i) at = A->v[p];
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int32_t nn = A->ci[p];
      if (nn == i || smark[nn] == i) continue;
      if (cf[nn] == 1 && inC[cidx[nn]] >= 0) continue;
      at += A->v[p];
    }
    for (int64_t t = 0; t < nf; ++t) {
      int32_t k = fk[t];
      double aik = csr_get(A, i, k), den = qk[t];
      if (den != 0.0) {
        double q = aik / den;
        qk[t] = q;
        double aki = csr_get(A, k, (int32_t)i), akk = csr_get(A, k, k);
        if (opposite(aki, akk)) at += q * aki;
      } else {
        qk[t] = 0.0;
        fk[t] = -1 - k; /* marks a lumped connection */
        at += aik;
      }
    }
    int64_t len = 0;
    if (at != 0.0) {
      for (int64_t t = 0; t < nc_; ++t) {
        int32_t jf = cfine[rowc[t]];
        double num = csr_get(A, i, (int32_t)jf);
        for (int64_t u = 0; u < nf; ++u) {
          if (fk[u] < 0) continue;
          int32_t k = fk[u];
          double akj = csr_get(A, k, (int32_t)jf), akk = csr_get(A, k, k);
          if (opposite(akj, akk)) num += qk[u] * akj;
        }
        roww[t] = -(num / at);
      }
      len = nc_;
    }
    if (pmax > 0 && len > pmax) {
      double sall = 0.0, skeep = 0.0;
      for (int64_t t = 0; t < len; ++t) { sall += roww[t]; ord[t] = (int32_t)t; }
      /* selection by |w| descending, ties to the smaller column (insertion sort, short rows) */
      for (int64_t a = 1; a < len; ++a) {
        int32_t x = ord[a];
        int64_t b = a - 1;
        while (b >= 0) {
          double fa = fabs(roww[ord[b]]), fx = fabs(roww[x]);
          if (fa > fx || (fa == fx && ord[b] < x)) break;
          ord[b + 1] = ord[b]; --b;
        }
        ord[b + 1] = x;
      }
      int8_t* keep = (int8_t*)xcalloc((size_t)len, 1);
      for (int64_t t = 0; t < pmax; ++t) keep[ord[t]] = 1;
      for (int64_t t = 0; t < len; ++t) if (keep[t]) skeep += roww[t];
      double f = (skeep != 0.0) ? sall / skeep : 1.0;
      int64_t w = 0;
      for (int64_t t = 0; t < len; ++t)
        if (keep[t]) { rowc[w] = rowc[t]; roww[w] = roww[t] * f; ++w; }
      len = w;
      free(keep);
    }
    for (int64_t t = 0; t < len; ++t) { T.ci[o] = rowc[t]; T.v[o] = roww[t]; ++o; }
    T.rp[i + 1] = o;
    /* rowc may have been compacted by truncation: clear every coarse mark set for this row */
    for (int64_t k = S->rp[i]; k < S->rp[i + 1]; ++k) {
      int32_t j = S->ci[k];
      if (cf[j] == 1) inC[cidx[j]] = -1;
      else for (int64_t l = S->rp[j]; l < S->rp[j + 1]; ++l) if (cf[S->ci[l]] == 1) inC[cidx[S->ci[l]]] = -1;
    }
  }
  T.nnz = o;
  *P = T;
  free(cidx); free(cfine); free(inC); free(smark); free(rb); free(rowc); free(roww); free(fk); free(qk); free(ord);
  return O_OK;
}

/* Smoother scaling: l1-Jacobi 1 / (a_ii + sign(a_ii) sum_{j != i} |a_ij|), or omega / a_ii. */
static int smoother_diag(const csr_t* A, int type, double omega, double* dinv) {
  for (int64_t i = 0; i < A->nr; ++i) {
    double d = 0.0, l1 = 0.0;
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
      if (A->ci[k] == i) d = A->v[k]; else l1 += fabs(A->v[k]);
    }
    double den = (type == 1) ? d + ((d >= 0.0) ? l1 : -l1) : d;
    if (den == 0.0) return O_ESINGULAR;
    dinv[i] = (type == 1) ? 1.0 / den : omega / den;
  }
  return O_OK;
}

static void amg_free(amg_t* g) {
  if (!g) return;
  for (int k = 0; k < MAXAMG; ++k) {
    csr_free(&g->A[k]); csr_free(&g->P[k]); csr_free(&g->R[k]); csr_free(&g->S[k]);
    free(g->dinv[k]); free(g->cf[k]);
  }
  free(g->lu); free(g->piv);
  free(g);
}

static int amg_setup(const csr_t* A0, const oopts_t* o, amg_t** out) {
  amg_t* g = (amg_t*)xcalloc(1, sizeof(amg_t));
  int rc = O_OK, k = 0;
  g->pre = o->amg_pre; g->post = o->amg_post;
  csr_copy(A0, &g->A[0]);
  int maxlev = o->amg_max_levels < MAXAMG ? o->amg_max_levels : MAXAMG;
  while (g->A[k].nr > o->amg_max_coarse && k < maxlev - 1) {
    int64_t n = g->A[k].nr;
    strength(&g->A[k], o->amg_theta, &g->S[k]);
    g->cf[k] = (int8_t*)xmalloc((size_t)n);
    pmis(&g->S[k], o->amg_seed, k, g->cf[k]);
    int64_t nC = 0;
    for (int64_t i = 0; i < n; ++i) nC += (g->cf[k][i] == 1);
    if (nC == 0 || nC == n) { free(g->cf[k]); g->cf[k] = NULL; csr_free(&g->S[k]); break; }
    extpi(&g->A[k], &g->S[k], g->cf[k], o->amg_pmax, &g->P[k]);
    transpose(&g->P[k], &g->R[k]);
    csr_t AP;
    memset(&AP, 0, sizeof AP);
    spgemm(&g->A[k], &g->P[k], &AP);
    spgemm(&g->R[k], &AP, &g->A[k + 1]);
    csr_free(&AP);
    g->dinv[k] = (double*)xmalloc(sizeof(double) * (size_t)n);
    rc = smoother_diag(&g->A[k], o->amg_smoother, o->amg_omega, g->dinv[k]);
    if (rc) { amg_free(g); return rc; }
    ++k;
  }
  g->nlev = k + 1;
  g->nco = g->A[k].nr;
  if (g->nco > 8000) { amg_free(g); return O_EINVAL; }
  g->lu = csr_to_dense(&g->A[k]);
  g->piv = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)(g->nco ? g->nco : 1));
  rc = lu_factor(g->nco, g->lu, g->piv);
  if (rc) { amg_free(g); return rc; }
  *out = g;
  return O_OK;
}

/* One V(pre, post)-cycle from a zero initial guess. */
static void amg_vcycle(const amg_t* g, int k, const double* b, double* x) {
  const csr_t* A = &g->A[k];
  int64_t n = A->nr;
  if (k == g->nlev - 1) {
    memcpy(x, b, sizeof(double) * (size_t)n);
    lu_solve(n, g->lu, g->piv, x);
    return;
  }
  double* res = (double*)xmalloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  for (int s = 0; s < g->pre; ++s) {
    csr_resid(A, x, b, res);
    for (int64_t i = 0; i < n; ++i) x[i] += g->dinv[k][i] * res[i];
  }
  csr_resid(A, x, b, res);
  int64_t nc = g->A[k + 1].nr;
  double* bc = (double*)xmalloc(sizeof(double) * (size_t)nc);
  double* xc = (double*)xmalloc(sizeof(double) * (size_t)nc);
  csr_resid(&g->R[k], res, NULL, bc);
  amg_vcycle(g, k + 1, bc, xc);
  csr_resid(&g->P[k], xc, NULL, res); /* res <- P xc */
  for (int64_t i = 0; i < n; ++i) x[i] += res[i];
  for (int s = 0; s < g->post; ++s) {
    csr_resid(A, x, b, res);
    for (int64_t i = 0; i < n; ++i) x[i] += g->dinv[k][i] * res[i];
  }
  free(res); free(bc); free(xc);
}

/* ================================== MGR hierarchy ============================================== */
typedef struct {
  int64_t n, nF, nC;
  csr_t A;            /* level operator */
  int8_t* mk;         /* markers of this level's dofs */
  int32_t *F, *C, *cidx, *fidx;
  double* minv;       /* F-relaxation scaling */
  int sweeps;
  csr_t Wp, Wr, P, R;
  double* aff_lu;     /* ideal mode: dense LU of A_ff */
  int32_t* aff_piv;
  void* famg;         /* frelax_type 2: AMG hierarchy on A_ff (amg_t) */
} olev_t;

typedef struct {
  oopts_t o;
  int64_t nb;
  double* binv;       /* inverses of the 3x3 diagonal blocks */
  int L;              /* number of reduction levels; level L is the coarse (pressure) system */
  olev_t lev[MAXLEV + 1];
  amg_t* amg;
  double* co_lu;      /* dense coarse solve (coarse_solver == 1 or ideal) */
  int32_t* co_piv;
} omgr_t;

/* Scalar CSR view of the BSR matrix, exact zeros dropped: row 3I+p holds, for each block (I, J) in
 * ascending J and q = 0..2, the nonzero entries (3J+q, B[p][q]). */
static int bsr_to_csr(int64_t nb, const int64_t* rp, const int32_t* ci, const double* v, csr_t* A) {
  int64_t cnt = 0;
  for (int64_t k = 0; k < rp[nb] * 9; ++k) cnt += (v[k] != 0.0);
  if (csr_alloc(A, 3 * nb, 3 * nb, cnt)) return O_ENOMEM;
  int64_t o = 0;
  for (int64_t I = 0; I < nb; ++I)
    for (int p = 0; p < 3; ++p) {
      for (int64_t k = rp[I]; k < rp[I + 1]; ++k)
        for (int q = 0; q < 3; ++q) {
          double x = v[9 * k + 3 * p + q];
          if (x != 0.0) { A->ci[o] = 3 * ci[k] + q; A->v[o] = x; ++o; }
        }
      A->rp[3 * I + p + 1] = o;
    }
  return O_OK;
}

/* Inverse of a 3x3 block by the adjugate: inv = adj(B) / det(B), det expanded along row 0. */
static int inv3(const double* b, double* r) {
  double c00 = b[4] * b[8] - b[5] * b[7];
  double c01 = b[5] * b[6] - b[3] * b[8];
  double c02 = b[3] * b[7] - b[4] * b[6];
  double det = b[0] * c00 + b[1] * c01 + b[2] * c02;
  if (det == 0.0 || !isfinite(det)) return O_ESINGULAR;
  double id = 1.0 / det;
  r[0] = c00 * id;
  r[1] = (b[2] * b[7] - b[1] * b[8]) * id;
  r[2] = (b[1] * b[5] - b[2] * b[4]) * id;
  r[3] = c01 * id;
  r[4] = (b[0] * b[8] - b[2] * b[6]) * id;
  r[5] = (b[2] * b[3] - b[0] * b[5]) * id;
  r[6] = c02 * id;
  r[7] = (b[1] * b[6] - b[0] * b[7]) * id;
  r[8] = (b[0] * b[4] - b[1] * b[3]) * id;
  return O_OK;
}

static void lev_free(olev_t* l) {
  csr_free(&l->A); csr_free(&l->Wp); csr_free(&l->Wr); csr_free(&l->P); csr_free(&l->R);
  free(l->mk); free(l->F); free(l->C); free(l->cidx); free(l->fidx); free(l->minv);
  free(l->aff_lu); free(l->aff_piv);
  amg_free((amg_t*)l->famg);
  memset(l, 0, sizeof *l);
}

void oracle_mgr_free(void* h) {
  omgr_t* m = (omgr_t*)h;
  if (!m) return;
  for (int l = 0; l <= MAXLEV; ++l) lev_free(&m->lev[l]);
  amg_free(m->amg);
  free(m->binv); free(m->co_lu); free(m->co_piv);
  free(m);
}

/* One reduction step at level l (section 4 with the level-l splitting F = {marker == l},
 * C = {marker > l}).  Builds W_p = -D_ff^-1 A_fc (or -A_ff^-1 A_fc in ideal mode), W_r, the
 * interpolation P = [W_p; I], restriction R = [W_r, I] and the coarse operator R (A P). */
static int reduce_level(omgr_t* m, int l) {
  olev_t* L = &m->lev[l];
  olev_t* N = &m->lev[l + 1];
  const oopts_t* o = &m->o;
  const csr_t* A = &L->A;
  int64_t n = L->n, nF = 0, nC = 0;
  L->cidx = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)n);
  L->fidx = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    if (L->mk[i] == l) { L->fidx[i] = (int32_t)nF++; L->cidx[i] = -1; }
    else { L->cidx[i] = (int32_t)nC++; L->fidx[i] = -1; }
  }
  L->nF = nF; L->nC = nC;
  L->F = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)nF);
  L->C = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)nC);
  for (int64_t i = 0; i < n; ++i) { if (L->fidx[i] >= 0) L->F[L->fidx[i]] = (int32_t)i; else L->C[L->cidx[i]] = (int32_t)i; }
  /* D_ff = diag(A_ff) */
  double* dff = (double*)xmalloc(sizeof(double) * (size_t)nF);
  for (int64_t f = 0; f < nF; ++f) {
    dff[f] = csr_get(A, L->F[f], L->F[f]);
    if (dff[f] == 0.0) { free(dff); return O_ESINGULAR; }
  }
  /* F-relaxation scaling over A_ff */
  L->minv = (double*)xmalloc(sizeof(double) * (size_t)nF);
  L->sweeps = o->frelax_sweeps[l];
  for (int64_t f = 0; f < nF; ++f) {
    int64_t i = L->F[f];
    double l1 = 0.0;
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
      if (A->ci[k] != i && L->fidx[A->ci[k]] >= 0) l1 += fabs(A->v[k]);
    double d = dff[f];
    if (o->frelax_type[l] == 1) {
      double den = d + ((d >= 0.0) ? l1 : -l1);
      L->minv[f] = 1.0 / den;
    } else {
      L->minv[f] = o->frelax_omega[l] / d;
    }
  }
  /* frelax_type 2 (section 6.2): the F-relaxation is one AMG V(1,1)-cycle on A_ff (F rows and
   * columns, in F order), built with the same AMG settings and a PMIS seed of its own per level */
  if (o->frelax_type[l] == 2 && !o->ideal && nF > 0) {
    csr_t Aff;
    int64_t cnt = 0;
    for (int64_t f = 0; f < nF; ++f) {
      int64_t i = L->F[f];
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) cnt += (L->fidx[A->ci[k]] >= 0);
    }
    csr_alloc(&Aff, nF, nF, cnt);
    int64_t q = 0;
    for (int64_t f = 0; f < nF; ++f) {
      int64_t i = L->F[f];
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
        int32_t g = L->fidx[A->ci[k]];
        if (g >= 0) { Aff.ci[q] = g; Aff.v[q] = A->v[k]; ++q; }
      }
      Aff.rp[f + 1] = q;
    }
    oopts_t of = *o;
    of.amg_seed = o->amg_seed + 7919ull * (uint64_t)(l + 1);
    of.amg_pre = 1;
    of.amg_post = 1;
    amg_t* g = NULL;
    int rc = amg_setup(&Aff, &of, &g);
    csr_free(&Aff);
    if (rc) { free(dff); return rc; }
    L->famg = g;
  }
  /* W_p (nF x nC) */
  if (!o->ideal) {
    int64_t cnt = 0;
    for (int64_t f = 0; f < nF; ++f) {
      int64_t i = L->F[f];
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) cnt += (L->cidx[A->ci[k]] >= 0);
    }
    csr_alloc(&L->Wp, nF, nC, cnt);
    int64_t q = 0;
    for (int64_t f = 0; f < nF; ++f) {
      int64_t i = L->F[f];
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
        int32_t c = L->cidx[A->ci[k]];
        if (c >= 0) { L->Wp.ci[q] = c; L->Wp.v[q] = -(A->v[k] / dff[f]); ++q; }
      }
      L->Wp.rp[f + 1] = q;
    }
  } else {
    /* ideal: W_p = -A_ff^-1 A_fc, dense (small problems only) */
    if (nF > 6000) { free(dff); return O_EINVAL; }
    double* aff = (double*)xcalloc((size_t)(nF * nF), sizeof(double));
    for (int64_t f = 0; f < nF; ++f) {
      int64_t i = L->F[f];
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
        int32_t g = L->fidx[A->ci[k]];
        if (g >= 0) aff[f * nF + g] = A->v[k];
      }
    }
    L->aff_piv = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)(nF ? nF : 1));
    if (lu_factor(nF, aff, L->aff_piv)) { free(aff); free(dff); return O_ESINGULAR; }
    L->aff_lu = aff;
    csr_alloc(&L->Wp, nF, nC, nF * nC);
    double* col = (double*)xmalloc(sizeof(double) * (size_t)(nF ? nF : 1));
    for (int64_t f = 0; f <= nF; ++f) L->Wp.rp[f] = f * nC;
    for (int64_t c = 0; c < nC; ++c) {
      for (int64_t f = 0; f < nF; ++f) col[f] = csr_get(A, L->F[f], L->C[c]);
      lu_solve(nF, aff, L->aff_piv, col);
      for (int64_t f = 0; f < nF; ++f) { L->Wp.ci[f * nC + c] = (int32_t)c; L->Wp.v[f * nC + c] = -col[f]; }
    }
    free(col);
  }
  /* P (n x nC): C rows inject, F rows carry W_p */
  csr_alloc(&L->P, n, nC, nC + L->Wp.nnz);
  {
    int64_t q = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (L->cidx[i] >= 0) { L->P.ci[q] = L->cidx[i]; L->P.v[q] = 1.0; ++q; }
      else {
        int64_t f = L->fidx[i];
        for (int64_t k = L->Wp.rp[f]; k < L->Wp.rp[f + 1]; ++k) { L->P.ci[q] = L->Wp.ci[k]; L->P.v[q] = L->Wp.v[k]; ++q; }
      }
      L->P.rp[i + 1] = q;
    }
  }
  /* W_r (nC x nF) and R (nC x n) */
  {
    int64_t cnt = 0;
    if (o->restrict_type[l] == 1)
      for (int64_t c = 0; c < nC; ++c) {
        int64_t i = L->C[c];
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) cnt += (L->fidx[A->ci[k]] >= 0);
      }
    csr_alloc(&L->Wr, nC, nF, cnt);
    csr_alloc(&L->R, nC, n, nC + cnt);
    int64_t q = 0, r = 0;
    for (int64_t c = 0; c < nC; ++c) {
      int64_t i = L->C[c];
      int placed = 0;
      if (o->restrict_type[l] == 1)
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
          int32_t j = A->ci[k], f = L->fidx[j];
          if (f < 0) continue;
          double w = -(A->v[k] / dff[f]);
          L->Wr.ci[q] = f; L->Wr.v[q] = w; ++q;
          if (!placed && j > i) { L->R.ci[r] = (int32_t)i; L->R.v[r] = 1.0; ++r; placed = 1; }
          L->R.ci[r] = j; L->R.v[r] = w; ++r;
        }
      if (!placed) { L->R.ci[r] = (int32_t)i; L->R.v[r] = 1.0; ++r; }
      L->Wr.rp[c + 1] = q;
      L->R.rp[c + 1] = r;
    }
  }
  free(dff);
  /* coarse operator R (A P); with injective R this is the C rows of A P */
  csr_t AP;
  memset(&AP, 0, sizeof AP);
  if (spgemm(A, &L->P, &AP)) return O_ENOMEM;
  if (spgemm(&L->R, &AP, &N->A)) return O_ENOMEM;
  csr_free(&AP);
  N->n = nC;
  N->mk = (int8_t*)xmalloc((size_t)(nC ? nC : 1));
  for (int64_t c = 0; c < nC; ++c) N->mk[c] = L->mk[L->C[c]];
  return O_OK;
}

void* oracle_mgr_setup(int64_t nb, const int64_t* rp, const int32_t* ci, const double* v,
                       const int8_t* marker, const oopts_t* o, int* status) {
  *status = O_EINVAL;
  if (nb <= 0 || !rp || !ci || !v || !marker || !o) return NULL;
  omgr_t* m = (omgr_t*)xcalloc(1, sizeof(omgr_t));
  m->o = *o;
  m->nb = nb;
  int L = 0;
  for (int64_t d = 0; d < 3 * nb; ++d) {
    if (marker[d] < 0 || marker[d] >= MAXLEV) { free(m); return NULL; }
    if (marker[d] > L) L = marker[d];
  }
  m->L = L;
  /* global relaxation blocks */
  m->binv = (double*)xmalloc(sizeof(double) * 9 * (size_t)nb);
  for (int64_t I = 0; I < nb; ++I) {
    const double* blk = NULL;
    for (int64_t k = rp[I]; k < rp[I + 1]; ++k) if (ci[k] == I) blk = v + 9 * k;
    if (!blk || inv3(blk, m->binv + 9 * I)) { *status = O_ESINGULAR; oracle_mgr_free(m); return NULL; }
  }
  bsr_to_csr(nb, rp, ci, v, &m->lev[0].A);
  m->lev[0].n = 3 * nb;
  m->lev[0].mk = (int8_t*)xmalloc((size_t)(3 * nb));
  memcpy(m->lev[0].mk, marker, (size_t)(3 * nb));
  for (int l = 0; l < L; ++l) {
    int rc = reduce_level(m, l);
    if (rc) { *status = rc; oracle_mgr_free(m); return NULL; }
  }
  const csr_t* Ac = &m->lev[L].A;
  if (o->ideal || o->coarse_solver == 1) {
    if (Ac->nr > 8000) { oracle_mgr_free(m); return NULL; }
    m->co_lu = csr_to_dense(Ac);
    m->co_piv = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)(Ac->nr ? Ac->nr : 1));
    if (lu_factor(Ac->nr, m->co_lu, m->co_piv)) { *status = O_ESINGULAR; oracle_mgr_free(m); return NULL; }
  } else {
    int rc = amg_setup(Ac, o, &m->amg);
    if (rc) { *status = rc; oracle_mgr_free(m); return NULL; }
  }
  *status = O_OK;
  return m;
}

/* Algorithm step (1), global relaxation: e = blockdiag(A)^-1 r with the 3x3 cell blocks. */
static void global_relax(const omgr_t* m, const double* r, double* e) {
  for (int64_t I = 0; I < m->nb; ++I)
    for (int p = 0; p < 3; ++p) {
      const double* b = m->binv + 9 * I + 3 * p;
      e[3 * I + p] = b[0] * r[3 * I] + b[1] * r[3 * I + 1] + b[2] * r[3 * I + 2];
    }
}
int oracle_global_relax(void* h, const double* r, double* e) {
  omgr_t* m = (omgr_t*)h;
  if (!m || !m->binv) return O_EINVAL;
  global_relax(m, r, e);
  return O_OK;
}

/* Level solve e ~ A_l^-1 r following the Algorithm (global relaxation only at level 0). */
static void level_solve(const omgr_t* m, int l, const double* r, double* e) {
  const olev_t* L = &m->lev[l];
  int64_t n = L->n;
  if (l == m->L) {
    if (m->co_lu) { memcpy(e, r, sizeof(double) * (size_t)n); lu_solve(n, m->co_lu, m->co_piv, e); }
    else amg_vcycle(m->amg, 0, r, e);
    return;
  }
  const csr_t* A = &L->A;
  for (int64_t i = 0; i < n; ++i) e[i] = 0.0;
  if (l == 0 && m->o.global_relax) global_relax(m, r, e);
  /* F-relaxation: e_F += M_ff^-1 (r - A e)_F, Jacobi-type sweeps */
  double* rf = (double*)xmalloc(sizeof(double) * (size_t)(L->nF ? L->nF : 1));
  int sweeps = m->o.ideal ? 1 : L->sweeps;
  for (int s = 0; s < sweeps; ++s) {
    for (int64_t f = 0; f < L->nF; ++f) {
      int64_t i = L->F[f];
      double acc = 0.0;
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) acc += A->v[k] * e[A->ci[k]];
      rf[f] = r[i] - acc;
    }
    if (m->o.ideal) {
      lu_solve(L->nF, L->aff_lu, L->aff_piv, rf);
      for (int64_t f = 0; f < L->nF; ++f) e[L->F[f]] += rf[f];
    } else if (L->famg) {
      double* ef = (double*)xmalloc(sizeof(double) * (size_t)L->nF);
      amg_vcycle((const amg_t*)L->famg, 0, rf, ef);
      for (int64_t f = 0; f < L->nF; ++f) e[L->F[f]] += ef[f];
      free(ef);
    } else {
      for (int64_t f = 0; f < L->nF; ++f) e[L->F[f]] += L->minv[f] * rf[f];
    }
  }
  /* coarse correction: r_c = R_I (r - A e), or full R */
  double* rc = (double*)xmalloc(sizeof(double) * (size_t)(L->nC ? L->nC : 1));
  double* ec = (double*)xmalloc(sizeof(double) * (size_t)(L->nC ? L->nC : 1));
  for (int64_t c = 0; c < L->nC; ++c) {
    int64_t i = L->C[c];
    double acc = 0.0;
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) acc += A->v[k] * e[A->ci[k]];
    rc[c] = r[i] - acc;
  }
  if (m->o.apply_full_R && L->Wr.nnz > 0) {
    for (int64_t f = 0; f < L->nF; ++f) {
      int64_t i = L->F[f];
      double acc = 0.0;
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) acc += A->v[k] * e[A->ci[k]];
      rf[f] = r[i] - acc;
    }
    for (int64_t c = 0; c < L->nC; ++c)
      for (int64_t k = L->Wr.rp[c]; k < L->Wr.rp[c + 1]; ++k) rc[c] += L->Wr.v[k] * rf[L->Wr.ci[k]];
  }
  level_solve(m, l + 1, rc, ec);
  /* interpolation: e_C += e_c, e_F += W_p e_c */
  for (int64_t c = 0; c < L->nC; ++c) e[L->C[c]] += ec[c];
  for (int64_t f = 0; f < L->nF; ++f) {
    double acc = 0.0;
    for (int64_t k = L->Wp.rp[f]; k < L->Wp.rp[f + 1]; ++k) acc += L->Wp.v[k] * ec[L->Wp.ci[k]];
    e[L->F[f]] += acc;
  }
  free(rf); free(rc); free(ec);
}

int oracle_mgr_apply(void* h, const double* r, double* z) {
  omgr_t* m = (omgr_t*)h;
  if (!m || !r || !z) return O_EINVAL;
  level_solve(m, 0, r, z);
  return O_OK;
}

/* ---- BSR SpMV for the Krylov method --------------------------------------------------------- */
static void bsr_mv(int64_t nb, const int64_t* rp, const int32_t* ci, const double* v, const double* x, double* y) {
  for (int64_t I = 0; I < nb; ++I) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t k = rp[I]; k < rp[I + 1]; ++k) {
      const double* b = v + 9 * k;
      const double* xx = x + 3 * (int64_t)ci[k];
      s0 += b[0] * xx[0] + b[1] * xx[1] + b[2] * xx[2];
      s1 += b[3] * xx[0] + b[4] * xx[1] + b[5] * xx[2];
      s2 += b[6] * xx[0] + b[7] * xx[1] + b[8] * xx[2];
    }
    y[3 * I] = s0; y[3 * I + 1] = s1; y[3 * I + 2] = s2;
  }
}
static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Right-preconditioned flexible GMRES(m) (Saad 1993) with modified Gram-Schmidt and Givens
 * rotations.  Stops when |g_{j+1}| <= rtol ||b|| and confirms with the explicit residual
 * ||b - A x|| <= rtol ||b||; a failed confirmation restarts.  h == NULL runs unpreconditioned.
 * If Vout/Zout/Hout are given, the first cycle's basis V (m+1 columns), Z (m columns) and the
 * (m+1) x m Hessenberg matrix are copied out (column-major vectors of length n). */
int oracle_fgmres(void* h, int64_t nb, const int64_t* rp, const int32_t* ci, const double* v,
                  const double* b, double* x, double rtol, int restart, int maxit, oinfo_t* info,
                  double* hist, double* Vout, double* Zout, double* Hout) {
  omgr_t* mg = (omgr_t*)h;
  int64_t n = 3 * nb;
  int m = restart;
  if (m < 1 || maxit < 0 || !b || !x || !info) return O_EINVAL;
  memset(info, 0, sizeof *info);
  double* V = (double*)xmalloc(sizeof(double) * (size_t)(n * (m + 1)));
  double* Z = (double*)xmalloc(sizeof(double) * (size_t)(n * m));
  double* H = (double*)xcalloc((size_t)((m + 1) * m), sizeof(double)); /* H[i*m + j] */
  double* cs = (double*)xmalloc(sizeof(double) * (size_t)m);
  double* sn = (double*)xmalloc(sizeof(double) * (size_t)m);
  double* g = (double*)xmalloc(sizeof(double) * (size_t)(m + 1));
  double* y = (double*)xmalloc(sizeof(double) * (size_t)m);
  double* r = (double*)xmalloc(sizeof(double) * (size_t)n);
  double bnorm = sqrt(dot(n, b, b));
  info->bnorm = bnorm;
  int rc = O_OK, it = 0, first = 1;
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    info->converged = 1;
    goto done;
  }
  bsr_mv(nb, rp, ci, v, x, r);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  double beta = sqrt(dot(n, r, r));
  if (hist) hist[0] = beta / bnorm;
  if (beta <= rtol * bnorm) { info->converged = 1; info->relres_true = info->relres_est = beta / bnorm; goto done; }
  for (;;) {
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int j, k = 0;
    for (j = 0; j < m && it < maxit; ++j) {
      double* vj = V + (int64_t)j * n;
      double* zj = Z + (int64_t)j * n;
      double* w = V + (int64_t)(j + 1) * n;
      if (mg) level_solve(mg, 0, vj, zj); else memcpy(zj, vj, sizeof(double) * (size_t)n);
      bsr_mv(nb, rp, ci, v, zj, w);
      for (int i = 0; i <= j; ++i) {
        double hij = dot(n, w, V + (int64_t)i * n);
        H[i * m + j] = hij;
        for (int64_t t = 0; t < n; ++t) w[t] -= hij * V[(int64_t)i * n + t];
      }
      double hn = sqrt(dot(n, w, w));
      H[(j + 1) * m + j] = hn;
      if (!isfinite(hn)) { rc = O_EBREAKDOWN; goto done; }
      if (hn != 0.0) for (int64_t t = 0; t < n; ++t) w[t] /= hn;
      if (first && Hout) for (int i = 0; i <= j + 1; ++i) Hout[i * m + j] = H[i * m + j];
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double den = sqrt(a * a + c * c);
      if (den == 0.0) { rc = O_EBREAKDOWN; goto done; }
      cs[j] = a / den; sn[j] = c / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      k = j + 1;
      if (hist) hist[it] = fabs(g[j + 1]) / bnorm;
      if (fabs(g[j + 1]) <= rtol * bnorm || hn == 0.0) break;
    }
    if (first && Vout) memcpy(Vout, V, sizeof(double) * (size_t)(n * (k + 1)));
    if (first && Zout) memcpy(Zout, Z, sizeof(double) * (size_t)(n * k));
    first = 0;
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int t = i + 1; t < k; ++t) s -= H[i * m + t] * y[t];
      y[i] = s / H[i * m + i];
    }
    for (int t = 0; t < k; ++t)
      for (int64_t i = 0; i < n; ++i) x[i] += y[t] * Z[(int64_t)t * n + i];
    info->relres_est = (k > 0) ? fabs(g[k]) / bnorm : beta / bnorm;
    bsr_mv(nb, rp, ci, v, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    beta = sqrt(dot(n, r, r));
    info->relres_true = beta / bnorm;
    if (beta <= rtol * bnorm) { info->converged = 1; break; }
    if (it >= maxit) { rc = O_ENOTCONV; break; }
    if (!isfinite(beta)) { rc = O_EBREAKDOWN; break; }
    info->restarts++;
  }
done:
  info->iterations = it;
  info->status = rc;
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(r);
  return rc;
}

/* ---- introspection for the tests ------------------------------------------------------------- */
/* kind: 0 MGR level operator A_l (l = 0..L), 1 W_p(l), 2 W_r(l), 3 P(l), 4 R(l),
 *       5 AMG operator A_k, 6 AMG P_k, 7 AMG R_k, 8 AMG strength S_k (values = 1) */
static const csr_t* pick(const omgr_t* m, int kind, int level) {
  if (kind <= 4) {
    if (level < 0 || level > m->L || (kind > 0 && level >= m->L)) return NULL;
    const olev_t* L = &m->lev[level];
    switch (kind) { case 0: return &L->A; case 1: return &L->Wp; case 2: return &L->Wr; case 3: return &L->P; default: return &L->R; }
  }
  if (!m->amg || level < 0 || level >= m->amg->nlev) return NULL;
  if (kind > 5 && level >= m->amg->nlev - 1) return NULL;
  switch (kind) { case 5: return &m->amg->A[level]; case 6: return &m->amg->P[level]; case 7: return &m->amg->R[level]; case 8: return &m->amg->S[level]; }
  return NULL;
}
int oracle_get_info(void* h, int* L, int* amg_levels) {
  omgr_t* m = (omgr_t*)h;
  if (!m) return O_EINVAL;
  *L = m->L;
  *amg_levels = m->amg ? m->amg->nlev : 0;
  return O_OK;
}
int oracle_mat_shape(void* h, int kind, int level, int64_t* nr, int64_t* nc, int64_t* nnz) {
  const csr_t* a = pick((omgr_t*)h, kind, level);
  if (!a) return O_EINVAL;
  *nr = a->nr; *nc = a->nc; *nnz = a->nnz;
  return O_OK;
}
int oracle_mat_copy(void* h, int kind, int level, int64_t* rp, int32_t* ci, double* v) {
  const csr_t* a = pick((omgr_t*)h, kind, level);
  if (!a) return O_EINVAL;
  memcpy(rp, a->rp, sizeof(int64_t) * (size_t)(a->nr + 1));
  memcpy(ci, a->ci, sizeof(int32_t) * (size_t)a->nnz);
  if (v) {
    if (a->v) memcpy(v, a->v, sizeof(double) * (size_t)a->nnz);
    else for (int64_t k = 0; k < a->nnz; ++k) v[k] = 1.0;
  }
  return O_OK;
}
/* vectors: kind 0 F-relaxation scaling of level l (length nF), 1 AMG smoother scaling of level k,
 * 2 block-diagonal inverses (9 nb), 3 F index list of level l, 4 C index list of level l,
 * 5 AMG C/F split of level k (1 = C, -1 = F) */
int oracle_vec_len(void* h, int kind, int level, int64_t* len) {
  omgr_t* m = (omgr_t*)h;
  if (!m) return O_EINVAL;
  switch (kind) {
    case 0: case 3: if (level < 0 || level >= m->L) return O_EINVAL; *len = m->lev[level].nF; return O_OK;
    case 4: if (level < 0 || level >= m->L) return O_EINVAL; *len = m->lev[level].nC; return O_OK;
    case 1: case 5: if (!m->amg || level < 0 || level >= m->amg->nlev - 1) return O_EINVAL; *len = m->amg->A[level].nr; return O_OK;
    case 2: *len = 9 * m->nb; return O_OK;
  }
  return O_EINVAL;
}
int oracle_vec_copy(void* h, int kind, int level, double* out) {
  omgr_t* m = (omgr_t*)h;
  int64_t len;
  if (oracle_vec_len(h, kind, level, &len)) return O_EINVAL;
  for (int64_t i = 0; i < len; ++i) {
    switch (kind) {
      case 0: out[i] = m->lev[level].minv[i]; break;
      case 1: out[i] = m->amg->dinv[level][i]; break;
      case 2: out[i] = m->binv[i]; break;
      case 3: out[i] = m->lev[level].F[i]; break;
      case 4: out[i] = m->lev[level].C[i]; break;
      case 5: out[i] = m->amg->cf[level][i]; break;
    }
  }
  return O_OK;
}

/* ---- AMG on a scalar CSR matrix alone (textbook Poisson pins) -------------------------------- */
void* oracle_amg_setup_csr(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                           const oopts_t* o, int* status) {
  csr_t A;
  A.nr = n; A.nc = n; A.nnz = rp[n];
  A.rp = (int64_t*)rp; A.ci = (int32_t*)ci; A.v = (double*)v;
  omgr_t* m = (omgr_t*)xcalloc(1, sizeof(omgr_t));
  m->o = *o;
  m->L = 0;
  *status = amg_setup(&A, o, &m->amg);
  if (*status) { free(m); return NULL; }
  csr_copy(&A, &m->lev[0].A);
  m->lev[0].n = n;
  return m;
}
int oracle_amg_vcycle(void* h, const double* b, double* x) {
  omgr_t* m = (omgr_t*)h;
  if (!m || !m->amg) return O_EINVAL;
  amg_vcycle(m->amg, 0, b, x);
  return O_OK;
}

/* ---- stand-alone sparse kernels, exposed so the tests can pin them against a library -------- */
int oracle_spgemm_csr(int64_t m, int64_t k, int64_t n, const int64_t* arp, const int32_t* aci,
                      const double* av, const int64_t* brp, const int32_t* bci, const double* bv,
                      int64_t* nnz_out, int64_t* crp, int32_t* cci, double* cv) {
  csr_t A = {m, k, arp[m], (int64_t*)arp, (int32_t*)aci, (double*)av};
  csr_t B = {k, n, brp[k], (int64_t*)brp, (int32_t*)bci, (double*)bv};
  csr_t C;
  memset(&C, 0, sizeof C);
  if (spgemm(&A, &B, &C)) return O_ENOMEM;
  *nnz_out = C.nnz;
  if (crp) {
    memcpy(crp, C.rp, sizeof(int64_t) * (size_t)(m + 1));
    memcpy(cci, C.ci, sizeof(int32_t) * (size_t)C.nnz);
    memcpy(cv, C.v, sizeof(double) * (size_t)C.nnz);
  }
  csr_free(&C);
  return O_OK;
}

/* Strength + extended+i interpolation for a caller-given C/F split (1 = C, -1 = F), so the tests can
 * pin the interpolation formula on hand-computable cases.  Two calls: first with prp == NULL to get
 * nnz, then with output arrays of that size. */
int oracle_extpi_csr(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double theta,
                     const int8_t* cf, int pmax, int64_t* nnz_out, int64_t* prp, int32_t* pci, double* pv) {
  csr_t A = {n, n, rp[n], (int64_t*)rp, (int32_t*)ci, (double*)v};
  csr_t S, P;
  memset(&S, 0, sizeof S);
  memset(&P, 0, sizeof P);
  strength(&A, theta, &S);
  extpi(&A, &S, cf, pmax, &P);
  *nnz_out = P.nnz;
  if (prp) {
    memcpy(prp, P.rp, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(pci, P.ci, sizeof(int32_t) * (size_t)P.nnz);
    memcpy(pv, P.v, sizeof(double) * (size_t)P.nnz);
  }
  csr_free(&S); csr_free(&P);
  return O_OK;
}

/* Strength + PMIS on a caller-given scalar matrix (AMG level lev's random numbers), so the tests can
 * check the splitting by brute force on small graphs.  cf receives 1 (C) / -1 (F); with srp != NULL
 * the strength graph is returned too (two calls: first srp == NULL for its size). */
int oracle_pmis_csr(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double theta, uint64_t seed,
                    int lev, int8_t* cf, int64_t* snnz_out, int64_t* srp, int32_t* sci) {
  csr_t A = {n, n, rp[n], (int64_t*)rp, (int32_t*)ci, (double*)v};
  csr_t S;
  memset(&S, 0, sizeof S);
  strength(&A, theta, &S);
  *snnz_out = S.nnz;
  if (cf) pmis(&S, seed, lev, cf);
  if (srp) {
    memcpy(srp, S.rp, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(sci, S.ci, sizeof(int32_t) * (size_t)S.nnz);
  }
  csr_free(&S);
  return O_OK;
}
