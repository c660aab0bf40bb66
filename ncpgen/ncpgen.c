/*
 * ncpgen.c -- seeded synthetic Jacobians of the two-phase, two-component (water / hydrogen)
 * porous-media model written as a nonlinear complementarity problem (NCP).
 *
 * This module only manufactures INPUTS (matrix, right-hand side, phase state, cf_marker).  It holds
 * none of the solver's arithmetic and is shared by the CPU oracle and the GPU library tests alike.
 *
 * Physics followed (section 2 of Bui, Wang & Osei-Kuffuor, "Algebraic multigrid preconditioners for
 * multiphase flow in porous media with phase transitions"):
 *   - water and hydrogen mass conservation (section 2.1, the two conservation equations), Darcy-Muskat
 *     velocities and Fick diffusion of dissolved hydrogen, no gravity;
 *   - capillary jump P_g = P_l + P_c(S_l), S_l + S_g = 1, Henry's law rho_l^h = C_h P_g and the ideal
 *     gas law rho_g = C_v P_g (section 2.1);
 *   - the complementarity constraint min(1 - S_l, C_h P_g - rho_l^h) = 0 (section 2.2), linearised
 *     with the active-set rule of the semi-smooth Newton algorithm (section 3.1): rows with
 *     F_j >= G_j take G' (gas present), the others take F' (gas absent);
 *   - power-law (Corey, exponent 2) relative permeabilities (section 2.3) and the linear capillary
 *     pressure P_c = P_r (1 - S_le) (section 2.4); or (closure 1) the Van Genuchten relative
 *     permeabilities and capillary pressure of sections 2.3-2.4, the latter regularised with
 *     epsilon = 1e-5 (section 2.4; the regularisation is read as acting on the gas saturation
 *     S_g = 1 - S_l, see vg_pcap below);
 *   - primary variables u = (P_l, S_l, rho_l^h) per cell, in that order (section 2.5);
 *   - cell-centred two-point finite volumes with phase-potential upwinding and one backward Euler step
 *     (section 3).
 * The paper's physical constants are dimensional and partly garbled; this generator uses
 * non-dimensional stand-ins with the same structure (listed in ncp_constants below).
 *
 * Output: 3x3 block-CSR (BSR) with int64 block-row pointers, int32 block columns sorted ascending,
 * and 9 doubles per block stored row-major (entry (p,q) = d R_p(I) / d u_q(J)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NCP_OK 0
#define NCP_EINVAL 1
#define NCP_ENOMEM 2

typedef struct {
  int32_t nx, ny, nz;         /* grid cells; nz == 1 gives a 2-D 5-point grid */
  double sigma;               /* standard deviation of log-permeability */
  double layer_contrast;      /* 0: no layering; else low-permeability layer multiplier (e.g. 1e-4) */
  double absent_frac;         /* fraction of cells where the gas phase is absent */
  int32_t absent_mode;        /* 0: i.i.d. Bernoulli cells; 1: seeded blob of Gaussian bumps */
  int32_t pad_;
  uint64_t seed;              /* matrix seed */
  double phi;                 /* porosity */
  int32_t closure;            /* 0: Corey n = 2 and linear P_c; 1: Van Genuchten (section 2.3-2.4) */
  int32_t state_mode;         /* 0: seeded linearisation point; 1: two sub-domains x < nx/2 and
                                 x >= nx/2 at S_l = s_l1 / s_l2, P_l = 1, rho on the Henry line
                                 (the initial state of the unsaturated test of section 6.1) */
  double vg_n;                /* Van Genuchten n (m = 1 - 1/n) */
  double s_lr, s_gr;          /* residual saturations (closure 1) */
  double p_r;                 /* entry pressure (closure 1) */
  double s_l1, s_l2;          /* sub-domain saturations (state_mode 1) */
  int32_t closed;             /* 1: no-flow boundary everywhere (no Dirichlet outlet) */
  int32_t pad2_;
} ncp_config_t;

/* Non-dimensional stand-ins for the physical parameters. */
static const double RHO_W = 1.0, MU_L = 1.0, MU_G = 0.05, C_V = 1.0, C_H = 0.02, DIFF = 0.1,
                    P_R = 0.2, S_LR = 0.0, S_GR = 0.0, DT = 1.0, P_OUT = 0.5;

/* ---- counter-based random numbers: splitmix64 (Steele, Lea & Flood 2014) ---------------------- */
static inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
/* Stream key: the (seed, stream) pair hashed once; each index is then hashed against the key. */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return splitmix64(seed ^ (stream << 48));
}
static inline double u01(uint64_t key, uint64_t idx) { /* uniform in [0, 1) with 53 bits */
  return (double)(splitmix64(key ^ idx) >> 11) * 0x1.0p-53;
}
static inline double normal01(uint64_t key, uint64_t idx) { /* Box-Muller on counters 2i, 2i+1 */
  double a = 1.0 - u01(key, 2 * idx), b = u01(key, 2 * idx + 1);
  return sqrt(-2.0 * log(a)) * cos(6.283185307179586 * b);
}

void ncp_normals(uint64_t seed, uint64_t stream, int64_t n, double* out) {
  uint64_t key = stream_key(seed, stream);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = normal01(key, (uint64_t)i);
}
void ncp_uniforms(uint64_t seed, uint64_t stream, int64_t n, double* out) {
  uint64_t key = stream_key(seed, stream);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = u01(key, (uint64_t)i);
}

/* ---- constitutive relations (sections 2.3, 2.4) ------------------------------------------------ */
/* closure 0: Corey (exponent 2) relative permeabilities and the linear capillary pressure */
static inline double s_eff(double s) { return (s - S_LR) / (1.0 - S_LR - S_GR); }
static inline double dse(void) { return 1.0 / (1.0 - S_LR - S_GR); }

/* closure 1: Van Genuchten, m = 1 - 1/n, S_le = (S_l - S_lr) / (1 - S_lr - S_gr) clamped to [0, 1]
 *   k_rl = sqrt(S_le) (1 - (1 - S_le^(1/m))^m)^2,   k_rg = sqrt(1 - S_le) (1 - S_le^(1/m))^(2m).
 * The derivatives are singular at S_le = 0 and 1; S_le is kept in [VG_TINY, 1 - VG_TINY]. */
#define VG_TINY 1e-9
#define VG_EPS 1e-5
static inline double vg_m(const ncp_config_t* c) { return 1.0 - 1.0 / c->vg_n; }
static inline double vg_se(const ncp_config_t* c, double s, double* dsd) {
  double span = 1.0 - c->s_lr - c->s_gr, e = (s - c->s_lr) / span;
  *dsd = 1.0 / span;
  if (e < VG_TINY) { e = VG_TINY; *dsd = 0.0; }
  if (e > 1.0 - VG_TINY) { e = 1.0 - VG_TINY; *dsd = 0.0; }
  return e;
}
static void vg_krl(const ncp_config_t* c, double s, double* kr, double* dkr) {
  double m = vg_m(c), de, e = vg_se(c, s, &de);
  double B = 1.0 - pow(e, 1.0 / m), A = pow(B, m), dA = -pow(B, m - 1.0) * pow(e, 1.0 / m - 1.0);
  *kr = sqrt(e) * (1.0 - A) * (1.0 - A);
  *dkr = (0.5 / sqrt(e) * (1.0 - A) * (1.0 - A) - 2.0 * sqrt(e) * (1.0 - A) * dA) * de;
}
static void vg_krg(const ncp_config_t* c, double s, double* kr, double* dkr) {
  double m = vg_m(c), de, e = vg_se(c, s, &de);
  double B = 1.0 - pow(e, 1.0 / m);
  *kr = sqrt(1.0 - e) * pow(B, 2.0 * m);
  *dkr = (-0.5 / sqrt(1.0 - e) * pow(B, 2.0 * m) - 2.0 * sqrt(1.0 - e) * pow(B, 2.0 * m - 1.0) * pow(e, 1.0 / m - 1.0)) * de;
}
/* Van Genuchten P_c as a function of the gas saturation g: p_r (S_le^(-1/m) - 1)^(1/n) with
 * S_le = (1 - g - s_lr) / span, and its derivative in g. */
static void vg_pc_raw(const ncp_config_t* c, double g, double* pc, double* dpc) {
  double m = vg_m(c), n = c->vg_n, span = 1.0 - c->s_lr - c->s_gr;
  double e = (1.0 - g - c->s_lr) / span, t = pow(e, -1.0 / m) - 1.0;
  *pc = c->p_r * pow(t, 1.0 / n);
  *dpc = c->p_r * (1.0 / n) * pow(t, 1.0 / n - 1.0) * (-1.0 / m) * pow(e, -1.0 / m - 1.0) * (-1.0 / span);
}
/* Regularised P_c (section 2.4, epsilon = 1e-5) read on the gas saturation g = 1 - S_l, whose range
 * is [s_gr, 1 - s_lr]: inside it g is mapped to gt = s_gr + (1 - eps)(g - s_gr) + (eps/2) span, so
 * that S_le stays in [eps/2, 1 - eps/2], and shifted so that P_c(s_gr) = 0; outside it P_c continues
 * linearly with the slope at the nearer end.  Returns P_c and dP_c/dS_l. */
static void vg_pcap(const ncp_config_t* c, double s, double* pc, double* dpc_ds) {
  double span = 1.0 - c->s_lr - c->s_gr, g = 1.0 - s;
  double lo = c->s_gr, hi = 1.0 - c->s_lr, p0, d0;
  vg_pc_raw(c, c->s_gr + 0.5 * VG_EPS * span, &p0, &d0);
  double gc = g < lo ? lo : (g > hi ? hi : g);
  double gt = c->s_gr + (1.0 - VG_EPS) * (gc - c->s_gr) + 0.5 * VG_EPS * span, p, d;
  vg_pc_raw(c, gt, &p, &d);
  double val = p - p0, slope = d * (1.0 - VG_EPS);  /* dP_c/dg */
  val += slope * (g - gc);                          /* linear continuation outside [lo, hi] */
  *pc = val;
  *dpc_ds = -slope;
}

/* the closures used by the assembly: mobilities lam = k_r / mu and P_c, with S_l derivatives */
static inline void clo_lam_l(const ncp_config_t* c, double s, double* v, double* d) {
  if (c->closure == 1) { vg_krl(c, s, v, d); *v /= MU_L; *d /= MU_L; return; }
  double e = s_eff(s);
  *v = e * e / MU_L;
  *d = 2.0 * s_eff(s) * dse() / MU_L;
}
static inline void clo_lam_g(const ncp_config_t* c, double s, double* v, double* d) {
  if (c->closure == 1) { vg_krg(c, s, v, d); *v /= MU_G; *d /= MU_G; return; }
  double e = 1.0 - s_eff(s);
  *v = e * e / MU_G;
  *d = -2.0 * (1.0 - s_eff(s)) * dse() / MU_G;
}
static inline void clo_pcap(const ncp_config_t* c, double s, double* v, double* d) {
  if (c->closure == 1) { vg_pcap(c, s, v, d); return; }
  *v = P_R * (1.0 - s_eff(s));
  *d = -P_R * dse();
}

static int valid_cfg(const ncp_config_t* c) {
  if (!c || c->nx < 1 || c->ny < 1 || c->nz < 1) return 0;
  if (c->absent_frac < 0.0 || c->absent_frac > 1.0) return 0;
  if (c->phi <= 0.0) return 0;
  if (c->closure < 0 || c->closure > 1 || c->state_mode < 0 || c->state_mode > 1) return 0;
  if (c->closure == 1 && (c->vg_n <= 1.0 || c->s_lr < 0.0 || c->s_gr < 0.0 || c->s_lr + c->s_gr >= 1.0))
    return 0;
  return 1;
}

int ncp_count(const ncp_config_t* c, int64_t* nb, int64_t* nnzb) {
  if (!valid_cfg(c) || !nb || !nnzb) return NCP_EINVAL;
  int64_t nx = c->nx, ny = c->ny, nz = c->nz;
  int64_t n = nx * ny * nz;
  int64_t faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1);
  *nb = n;
  *nnzb = n + 2 * faces;
  return NCP_OK;
}

/* Permeability: lognormal times a layer multiplier along the last grid axis. */
static void make_perm(const ncp_config_t* c, double* k) {
  int64_t nx = c->nx, ny = c->ny, nz = c->nz, n = nx * ny * nz;
  uint64_t kkey = stream_key(c->seed, 1);
  int layer_axis_len = (nz > 1) ? (int)nz : (int)ny;
  double* mult = (double*)malloc(sizeof(double) * (size_t)layer_axis_len);
  uint64_t lkey = stream_key(c->seed, 4);
  int cur = (c->layer_contrast > 0.0 && u01(lkey, 0) < 0.5) ? 1 : 0, left = 0;
  uint64_t cnt = 1;
  for (int z = 0; z < layer_axis_len; ++z) {
    if (left == 0) { /* new layer: thickness 1..4 cells, alternating type */
      left = 1 + (int)(4.0 * u01(lkey, cnt++));
      cur ^= 1;
    }
    mult[z] = (c->layer_contrast > 0.0 && cur) ? c->layer_contrast : 1.0;
    --left;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t ax = (nz > 1) ? i / (nx * ny) : (i / nx) % ny;
    k[i] = exp(c->sigma * normal01(kkey, (uint64_t)i)) * mult[ax];
  }
  free(mult);
}

typedef struct { double v; int64_t i; } vi_t;
static int cmp_vi_desc(const void* a, const void* b) {
  const vi_t* x = (const vi_t*)a; const vi_t* y = (const vi_t*)b;
  if (x->v > y->v) return -1;
  if (x->v < y->v) return 1;
  return (x->i < y->i) ? -1 : (x->i > y->i);
}

/* Gas-absent set: i.i.d. Bernoulli cells, or the top absent_frac quantile of a sum of 8 seeded
 * Gaussian bumps (exact count, ties broken by the lower cell index). */
static int make_phase(const ncp_config_t* c, int8_t* gas_present) {
  int64_t nx = c->nx, ny = c->ny, nz = c->nz, n = nx * ny * nz;
  uint64_t pkey = stream_key(c->seed, 5);
  if (c->absent_mode == 0) {
    for (int64_t i = 0; i < n; ++i) gas_present[i] = (u01(pkey, (uint64_t)i) < c->absent_frac) ? 0 : 1;
    return NCP_OK;
  }
  double cx[8], cy[8], cz[8], w[8];
  for (int b = 0; b < 8; ++b) {
    cx[b] = u01(pkey, 4 * b + 0); cy[b] = u01(pkey, 4 * b + 1);
    cz[b] = (nz > 1) ? u01(pkey, 4 * b + 2) : 0.5;
    w[b] = 0.1 + 0.2 * u01(pkey, 4 * b + 3);
  }
  vi_t* a = (vi_t*)malloc(sizeof(vi_t) * (size_t)n);
  if (!a) return NCP_ENOMEM;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
    double px = (x + 0.5) / nx, py = (y + 0.5) / ny, pz = (z + 0.5) / nz;
    double f = 0.0;
    for (int b = 0; b < 8; ++b) {
      double d2 = (px - cx[b]) * (px - cx[b]) + (py - cy[b]) * (py - cy[b]);
      if (nz > 1) d2 += (pz - cz[b]) * (pz - cz[b]);
      f += exp(-d2 / (2.0 * w[b] * w[b]));
    }
    a[i].v = f; a[i].i = i;
  }
  qsort(a, (size_t)n, sizeof(vi_t), cmp_vi_desc);
  int64_t n_absent = (int64_t)llround(c->absent_frac * (double)n);
  for (int64_t i = 0; i < n; ++i) gas_present[i] = 1;
  for (int64_t r = 0; r < n_absent; ++r) gas_present[a[r].i] = 0;
  free(a);
  return NCP_OK;
}

/* Linearisation point (state_mode 0): P_l is a linear drop along x plus noise; gas-present cells
 * carry S_g in U(0.05, 0.4) and rho exactly on the Henry line; gas-absent cells have S_l = 1 and rho
 * below it.  state_mode 1: P_l = 1, S_l = s_l1 for x < nx/2 and s_l2 beyond, rho on the Henry line. */
static void make_state(const ncp_config_t* c, const int8_t* gp, double* u) {
  int64_t nx = c->nx, ny = c->ny, nz = c->nz, n = nx * ny * nz;
  uint64_t key_p = stream_key(c->seed, 3), key_s = stream_key(c->seed, 6), key_r = stream_key(c->seed, 7);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t x = i % nx;
    double p, s, rho, pc, dpc;
    if (c->state_mode == 1) {
      p = 1.0;
      s = (2 * x < nx) ? c->s_l1 : c->s_l2;
      clo_pcap(c, s, &pc, &dpc);
      rho = C_H * (p + pc);
    } else {
      p = 1.0 - 0.5 * (x + 0.5) / nx + 0.01 * normal01(key_p, (uint64_t)i);
      if (gp[i]) {
        s = 1.0 - (0.05 + 0.35 * u01(key_s, (uint64_t)i));
        clo_pcap(c, s, &pc, &dpc);
        rho = C_H * (p + pc);
      } else {
        s = 1.0;
        clo_pcap(c, s, &pc, &dpc);
        rho = 0.9 * u01(key_r, (uint64_t)i) * C_H * (p + pc);
      }
    }
    u[3 * i + 0] = p; u[3 * i + 1] = s; u[3 * i + 2] = rho;
  }
}

/* Flux from cell I into neighbour J (antisymmetric in I, J) and its derivatives with respect to
 * u_I (dI) and u_J (dJ), rows (water, hydrogen), columns (P, S, rho).  If J is the Dirichlet ghost,
 * uJ holds the ghost state and dJ is discarded. */
static void face_flux(const ncp_config_t* c, const double* uI, const double* uJ, double T, double phi,
                      double F[2], double dI[2][3], double dJ[2][3]) {
  double PI = uI[0], SI = uI[1], rI = uI[2];
  double PJ = uJ[0], SJ = uJ[1], rJ = uJ[2];
  double pcI, dpcI, pcJ, dpcJ;
  clo_pcap(c, SI, &pcI, &dpcI);
  clo_pcap(c, SJ, &pcJ, &dpcJ);
  double PgI = PI + pcI, PgJ = PJ + pcJ;
  double dP = PI - PJ, dPg = PgI - PgJ, dr = rI - rJ, sbar = 0.5 * (SI + SJ);
  int upl_I = (PI >= PJ), upg_I = (PgI >= PgJ);
  double Sul = upl_I ? SI : SJ, rul = upl_I ? rI : rJ;
  double Sug = upg_I ? SI : SJ, Pgug = upg_I ? PgI : PgJ;
  double ll, dll, lg, dlg;
  clo_lam_l(c, Sul, &ll, &dll);
  clo_lam_g(c, Sug, &lg, &dlg);
  memset(dI, 0, sizeof(double) * 6);
  memset(dJ, 0, sizeof(double) * 6);
  /* water: rho_w lam_l,up T (P_I - P_J) - phi Sbar D (rho_I - rho_J) */
  F[0] = RHO_W * ll * T * dP - phi * sbar * DIFF * dr;
  dI[0][0] += RHO_W * ll * T;
  dJ[0][0] -= RHO_W * ll * T;
  if (upl_I) dI[0][1] += RHO_W * dll * T * dP; else dJ[0][1] += RHO_W * dll * T * dP;
  dI[0][1] -= 0.5 * phi * DIFF * dr;
  dJ[0][1] -= 0.5 * phi * DIFF * dr;
  dI[0][2] -= phi * sbar * DIFF;
  dJ[0][2] += phi * sbar * DIFF;
  /* hydrogen: rho_up lam_l,up T dP + C_v Pg_up lam_g,up T dPg + phi Sbar D (rho_I - rho_J) */
  F[1] = rul * ll * T * dP + C_V * Pgug * lg * T * dPg + phi * sbar * DIFF * dr;
  dI[1][0] += rul * ll * T;
  dJ[1][0] -= rul * ll * T;
  if (upl_I) { dI[1][2] += ll * T * dP; dI[1][1] += rul * dll * T * dP; }
  else { dJ[1][2] += ll * T * dP; dJ[1][1] += rul * dll * T * dP; }
  {
    double g = C_V * lg * T * dPg;           /* d/dPg_up */
    double gs = C_V * Pgug * dlg * T * dPg;  /* d/dS_up through lam_g */
    if (upg_I) { dI[1][0] += g; dI[1][1] += g * dpcI + gs; }
    else { dJ[1][0] += g; dJ[1][1] += g * dpcJ + gs; }
    double h = C_V * Pgug * lg * T;          /* d/d(dPg) */
    dI[1][0] += h; dI[1][1] += h * dpcI;
    dJ[1][0] -= h; dJ[1][1] -= h * dpcJ;
  }
  dI[1][1] += 0.5 * phi * DIFF * dr;
  dJ[1][1] += 0.5 * phi * DIFF * dr;
  dI[1][2] += phi * sbar * DIFF;
  dJ[1][2] -= phi * sbar * DIFF;
}

static inline double harm(double a, double b) { return 2.0 * a * b / (a + b); }

/* Residual (and optionally the Jacobian in BSR) of one backward Euler step at state u. */
static void assemble(const ncp_config_t* c, const double* k, const double* u, const double* u_old, double* R,
                     const int64_t* rowptr, int32_t* colind, double* val) {
  int64_t nx = c->nx, ny = c->ny, nz = c->nz, n = nx * ny * nz;
  double phi = c->phi;
  const double ghost[3] = {P_OUT, 1.0, 0.0};
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < n; ++I) {
    int64_t x = I % nx, y = (I / nx) % ny, z = I / (nx * ny);
    const double* uI = u + 3 * I;
    double SI = uI[1], rI = uI[2], pcI, dpcI;
    clo_pcap(c, SI, &pcI, &dpcI);
    double PgI = uI[0] + pcI;
    double r[3];
    double D[9];
    memset(D, 0, sizeof D);
    /* accumulation */
    r[0] = phi * RHO_W * SI / DT;
    r[1] = phi * (rI * SI + C_V * PgI * (1.0 - SI)) / DT;
    if (u_old) { /* the previous time level's mass: R = (M(u) - M(u_old)) / dt + fluxes */
      const double* uo = u_old + 3 * I;
      double pco, dpco;
      clo_pcap(c, uo[1], &pco, &dpco);
      r[0] -= phi * RHO_W * uo[1] / DT;
      r[1] -= phi * (uo[2] * uo[1] + C_V * (uo[0] + pco) * (1.0 - uo[1])) / DT;
    }
    D[0 * 3 + 1] += phi * RHO_W / DT;
    D[1 * 3 + 0] += phi * C_V * (1.0 - SI) / DT;
    D[1 * 3 + 1] += phi * (rI + C_V * dpcI * (1.0 - SI) - C_V * PgI) / DT;
    D[1 * 3 + 2] += phi * SI / DT;
    /* complementarity constraint: min(1 - S_l, C_h P_g - rho) with the active-set derivative */
    double Fc = 1.0 - SI, Gc = C_H * PgI - rI;
    r[2] = (Fc < Gc) ? Fc : Gc;
    if (Fc >= Gc) { D[6] = C_H; D[7] = C_H * dpcI; D[8] = -1.0; }
    else { D[6] = 0.0; D[7] = -1.0; D[8] = 0.0; }
    /* neighbours in ascending index order */
    int64_t nbr[6]; int nn = 0;
    if (z > 0) nbr[nn++] = I - nx * ny;
    if (y > 0) nbr[nn++] = I - nx;
    if (x > 0) nbr[nn++] = I - 1;
    int diag_slot = nn;
    if (x < nx - 1) nbr[nn++] = I + 1;
    if (y < ny - 1) nbr[nn++] = I + nx;
    if (z < nz - 1) nbr[nn++] = I + nx * ny;
    double off[6][9];
    for (int t = 0; t < nn; ++t) {
      int64_t J = nbr[t];
      double F[2], dI[2][3], dJ[2][3];
      face_flux(c, uI, u + 3 * J, harm(k[I], k[J]), phi, F, dI, dJ);
      r[0] += F[0]; r[1] += F[1];
      for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 3; ++q) D[p * 3 + q] += dI[p][q];
      memset(off[t], 0, sizeof(off[t]));
      for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 3; ++q) off[t][p * 3 + q] = dJ[p][q];
    }
    if (x == nx - 1 && !c->closed) { /* Dirichlet outlet on the x-max face, half-cell transmissibility */
      double F[2], dI[2][3], dJ[2][3];
      face_flux(c, uI, ghost, 2.0 * k[I], phi, F, dI, dJ);
      r[0] += F[0]; r[1] += F[1];
      for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 3; ++q) D[p * 3 + q] += dI[p][q];
    }
    if (R) { R[3 * I] = r[0]; R[3 * I + 1] = r[1]; R[3 * I + 2] = r[2]; }
    if (val) {
      int64_t b = rowptr[I];
      for (int t = 0; t <= nn; ++t) {
        int64_t slot = b + t;
        if (t < diag_slot) { colind[slot] = (int32_t)nbr[t]; memcpy(val + 9 * slot, off[t], sizeof(double) * 9); }
        else if (t == diag_slot) { colind[slot] = (int32_t)I; memcpy(val + 9 * slot, D, sizeof(double) * 9); }
        else { colind[slot] = (int32_t)nbr[t - 1]; memcpy(val + 9 * slot, off[t - 1], sizeof(double) * 9); }
      }
    }
  }
}

static void make_rowptr(const ncp_config_t* c, int64_t* rowptr) {
  int64_t nx = c->nx, ny = c->ny, nz = c->nz, n = nx * ny * nz;
  rowptr[0] = 0;
  for (int64_t I = 0; I < n; ++I) {
    int64_t x = I % nx, y = (I / nx) % ny, z = I / (nx * ny);
    int cnt = 1 + (x > 0) + (x < nx - 1) + (y > 0) + (y < ny - 1) + (z > 0) + (z < nz - 1);
    rowptr[I + 1] = rowptr[I] + cnt;
  }
}

/* Build the Jacobian.  Outputs (caller-allocated): rowptr[nb+1], colind[nnzb], values[9*nnzb],
 * gas_present[nb], state[3*nb] (may be NULL), perm[nb] (may be NULL). */
int ncp_build(const ncp_config_t* c, int64_t* rowptr, int32_t* colind, double* values,
              int8_t* gas_present, double* state, double* perm) {
  if (!valid_cfg(c) || !rowptr || !colind || !values || !gas_present) return NCP_EINVAL;
  int64_t nb, nnzb;
  ncp_count(c, &nb, &nnzb);
  if (nb > 0x7fffffffLL) return NCP_EINVAL;
  double* k = perm ? perm : (double*)malloc(sizeof(double) * (size_t)nb);
  double* u = state ? state : (double*)malloc(sizeof(double) * 3 * (size_t)nb);
  if (!k || !u) return NCP_ENOMEM;
  make_perm(c, k);
  int rc = make_phase(c, gas_present);
  if (rc == NCP_OK) {
    make_state(c, gas_present, u);
    make_rowptr(c, rowptr);
    assemble(c, k, u, NULL, NULL, rowptr, colind, values);
  }
  if (!perm) free(k);
  if (!state) free(u);
  return rc;
}

/* Jacobian (BSR, same pattern as ncp_build) and optionally the residual at an arbitrary state u,
 * with the permeability of the configuration: the linearisation of one semi-smooth Newton step
 * (section 3.1).  u_old (may be NULL) is the previous time level, whose mass enters R. */
int ncp_jacobian(const ncp_config_t* c, const double* u, const double* u_old, int64_t* rowptr, int32_t* colind,
                 double* values, double* R) {
  if (!valid_cfg(c) || !u || !rowptr || !colind || !values) return NCP_EINVAL;
  int64_t nb, nnzb;
  ncp_count(c, &nb, &nnzb);
  if (nb > 0x7fffffffLL) return NCP_EINVAL;
  double* k = (double*)malloc(sizeof(double) * (size_t)nb);
  if (!k) return NCP_ENOMEM;
  make_perm(c, k);
  make_rowptr(c, rowptr);
  assemble(c, k, u, u_old, R, rowptr, colind, values);
  free(k);
  return NCP_OK;
}

/* Residual R(u) at an arbitrary state with the permeability of the configuration (for
 * finite-difference checks of the Jacobian). */
int ncp_residual(const ncp_config_t* c, const double* u, const double* u_old, double* R) {
  if (!valid_cfg(c) || !u || !R) return NCP_EINVAL;
  int64_t nb, nnzb;
  ncp_count(c, &nb, &nnzb);
  double* k = (double*)malloc(sizeof(double) * (size_t)nb);
  if (!k) return NCP_ENOMEM;
  make_perm(c, k);
  assemble(c, k, u, u_old, R, NULL, NULL, NULL);
  free(k);
  return NCP_OK;
}

/* cf_marker from the phase state: the MGR level at which each dof becomes an F-point.
 *   rho in a gas-present cell -> 0 (first reduction, section 5: constraints with nonzero C33),
 *   S_l in every cell         -> 1 (second reduction: saturation block),
 *   rho in a gas-absent cell  -> 2 (third reduction: constraints with zero diagonal),
 *   P_l                       -> 3 (never F: the pressure system solved by AMG).
 * With the gas phase present in every cell there is no third reduction (the two-level scheme of
 * the unsaturated test, section 6.1) and P_l takes marker 2. */
void ncp_cf_marker(int64_t nb, const int8_t* gas_present, int8_t* marker) {
  int any_absent = 0;
  for (int64_t i = 0; i < nb; ++i) any_absent |= !gas_present[i];
  const int8_t mp = any_absent ? 3 : 2;
  for (int64_t i = 0; i < nb; ++i) {
    marker[3 * i + 0] = mp;
    marker[3 * i + 1] = 1;
    marker[3 * i + 2] = gas_present[i] ? 0 : 2;
  }
}
