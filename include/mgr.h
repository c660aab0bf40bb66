/*
 * mgr.h -- C ABI of the GB300 (sm_103a) library for multigrid-reduction (MGR) preconditioned
 * flexible GMRES on the 3x3-block Jacobians of two-phase, two-component porous-media flow written as
 * a nonlinear complementarity problem (Bui, Wang & Osei-Kuffuor, arXiv 1801.08464).
 *
 * The paper states the problem as A u = f with A the 3N x 3N block system of section 3.2 (one 3x3
 * block per pair of cells, unknowns (P_l, S_l, rho_l^h) per cell, section 2.5) and, after splitting
 * the constraint rows by the phase state, the saddle-point form of section 3.2.  The preconditioner is
 * the "MGR preconditioner with presmoothing" Algorithm of section 4 applied with the three-level
 * reduction order of section 5; the outer Krylov method is GMRES (section 6).
 *
 * Conventions shared by every entry point:
 *  - Pointers are DEVICE pointers unless the comment says "host".  The caller owns all memory it
 *    passes; the library never frees it.  A handle owns the memory of its hierarchy.
 *  - Work is enqueued on the CUDA stream given to mgr_create (NULL = legacy default stream).  Calls
 *    that return sizes or a convergence decision synchronise that stream.
 *  - Every call returns a status; nothing aborts.  A handle is not thread-safe.
 *  - Index types: block-row pointers int64, block columns int32 (so nb < 2^31).
 */
#ifndef MGR_H_
#define MGR_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MGR_MAX_LEVELS 8

typedef enum {
  MGR_OK = 0,
  MGR_ERR_INVALID_ARG = 1,   /* bad pointer, size, pattern or option */
  MGR_ERR_SINGULAR = 2,      /* zero / non-finite pivot: 3x3 diagonal block, D_ff entry, smoother
                                diagonal or coarsest-grid pivot */
  MGR_ERR_NOT_CONVERGED = 3, /* fgmres_solve reached maxit; x holds the last iterate */
  MGR_ERR_BREAKDOWN = 4,     /* NaN/Inf in a norm or Hessenberg entry */
  MGR_ERR_OOM = 5,           /* device allocation failed; the handle stays destroyable */
  MGR_ERR_CUDA = 6,          /* other CUDA runtime error */
  MGR_ERR_TIMEOUT = 7,       /* reserved: no kernel of this library waits on another */
  MGR_ERR_STATE = 8,         /* call order violated (e.g. apply before setup) */
  MGR_ERR_UNSUPPORTED = 9    /* a size beyond a documented limit of a kernel */
} mgr_status_t;

typedef enum { MGR_PREC_FP64 = 0, MGR_PREC_MIXED = 1 } mgr_precision_t;

/* 3x3 block-CSR matrix (device arrays).  rowptr[nb+1] int64 ascending with rowptr[0] = 0;
 * colind[nnzb] int32 strictly ascending within each block row, every block row holding its diagonal
 * block; values[9*nnzb] with block k stored row-major: values[9k + 3p + q] = A(3I+p, 3J+q) for the
 * block (I, J = colind[k]).  Row p of a block is equation p (water, hydrogen, constraint) and column q
 * is unknown q (P_l, S_l, rho_l^h) as in sections 2.5 and 3.2. */
typedef struct {
  int64_t nb;
  int64_t nnzb;
  const int64_t* rowptr;
  const int32_t* colind;
  const double* values;
} mgr_bsr3_t;

/* Solver options.  Levels l = 0, 1, 2 are the three reductions of section 5; index l of the
 * per-level arrays configures the reduction that removes the dofs with cf_marker == l. */
typedef struct {
  int32_t precision;                     /* mgr_precision_t; MIXED = FP32 hierarchy, FP64 Krylov */
  int32_t global_relax;                  /* Algorithm step (1) at the finest level (default 1) */
  int32_t frelax_type[MGR_MAX_LEVELS];   /* 0 omega-Jacobi, 1 l1-Jacobi, 2 one AMG V(1,1)-cycle on
                                            A_ff per sweep (section 6.2; the AMG settings below,
                                            PMIS seed amg_seed + 7919 (l + 1)); defaults 0, 1, 1 */
  int32_t frelax_sweeps[MGR_MAX_LEVELS]; /* F-relaxation sweeps (defaults 1, 2, 2) */
  double frelax_omega[MGR_MAX_LEVELS];   /* Jacobi weight (default 1) */
  int32_t restrict_type[MGR_MAX_LEVELS]; /* 0 injective W_r = 0, 1 W_r = -A_cf D_ff^-1 (eqs.
                                            injective_rp / non_injective_rp); defaults 1, 0, 0 */
  int32_t apply_full_R;                  /* 0: restrict with R_I as in the Algorithm (default) */
  int32_t coarse_solver;                 /* 0: AMG V-cycle on the last level; 1: dense inverse */
  double amg_theta;                      /* strength threshold (default 0.25) */
  int32_t amg_max_levels;                /* default 25 */
  int32_t amg_max_coarse;                /* coarsest AMG size solved densely (default 256, <= 4096) */
  int32_t amg_smoother;                  /* 0 omega-Jacobi, 1 l1-Jacobi (default) */
  int32_t amg_pre, amg_post;             /* V(pre, post), default V(1,1) */
  int32_t amg_pmax;                      /* max interpolation entries per row, 0 = no truncation */
  double amg_omega;                      /* Jacobi weight for amg_smoother = 0 */
  uint64_t amg_seed;                     /* PMIS weight seed (default 3) */
  int32_t lean;                          /* 1: free the setup-only FP64 operators as soon as the setup
                                            no longer needs them (the apply and the solve keep what
                                            they read); their introspection then returns
                                            MGR_ERR_STATE.  Default 0 */
  int32_t spgemm_stage;                  /* SpGEMM products staged per batch of short rows (0 or any
                                            value <= 1024: 2^29, or 2^27 with lean; 12 bytes each) */
  int32_t adjoint;                       /* 1: the setup also builds the transposed operators of the
                                            preconditioner, for mgr_apply_transpose and
                                            fgmres_solve_transpose (default 0) */
  int32_t apply_graph;                   /* the forward apply replayed as a CUDA graph (captured at the
                                            second apply after a setup, on fixed input/output buffers
                                            with device copies around each replay): 0 auto (systems
                                            of at most 2^21 unknowns, where the apply is bound by its
                                            launches), 1 always, -1 never.  Profiling disables it */
  int32_t pdl;                           /* 0: the apply and Krylov kernels use programmatic dependent
                                            launch (each may start while its predecessor drains and
                                            waits for it before touching memory); -1: plain launches */
  int32_t reserved[3];                   /* must be zero */
} mgr_options_t;

typedef struct {
  int32_t iterations;   /* total FGMRES iterations (preconditioner applications) */
  int32_t restarts;
  int32_t converged;
  int32_t status;
  double relres_true;   /* ||b - A x|| / ||b|| at exit, computed explicitly */
  double relres_est;    /* Givens residual estimate at exit */
  double bnorm;
  double solve_ms;      /* wall time of the call, host clock around stream-synchronised work */
  double* history;      /* host, optional: relative residual estimate per iteration */
  int32_t history_cap;  /* capacity of history (entries) */
  int32_t reserved[3];
} mgr_solve_info_t;

typedef struct mgr_handle_s* mgr_handle_t;

/* Human-readable status name (static storage). */
const char* mgr_status_string(mgr_status_t s);

/* Fill *opt (host) with the defaults listed above. */
void mgr_options_default(mgr_options_t* opt);

/* Create a handle bound to the current device and to `cuda_stream` (a cudaStream_t, may be NULL).
 * opt (host) is copied; NULL means defaults.  Errors: INVALID_ARG, OOM, CUDA. */
mgr_status_t mgr_create(mgr_handle_t* h, const mgr_options_t* opt, void* cuda_stream);

/* Build the MGR hierarchy of sections 4-5 for A (device BSR) and cf_marker[3*nb] (device int8):
 * cf_marker[d] is the reduction level at which dof d becomes an F-point (0: rho of a gas-present
 * cell, 1: S_l, 2: rho of a gas-absent cell, 3: P_l, the AMG system).  Level l's F set is
 * {marker == l}, its C set {marker > l}; the coarsest system is {marker == max marker}.
 * Copies or derives everything it needs: A and cf_marker may be freed on return.  A second call
 * rebuilds the hierarchy.  Errors: INVALID_ARG (pattern or marker), SINGULAR, OOM, UNSUPPORTED. */
mgr_status_t mgr_setup(mgr_handle_t h, const mgr_bsr3_t* A, const int8_t* cf_marker);

/* z = M^-1 r: one application of the presmoothing MGR Algorithm (section 4) with an AMG V-cycle as
 * the coarse solve.  r, z: device double[3*nb]; r is not modified; r and z must not overlap.
 * Asynchronous on the handle's stream.  Errors: STATE (no setup), INVALID_ARG. */
mgr_status_t mgr_apply(mgr_handle_t h, const double* r, double* z);

/* Solve A x = b by right-preconditioned flexible GMRES(restart) with M^-1 = mgr_apply, FP64 Krylov
 * vectors.  A must have the pattern given to mgr_setup (its values are read during the call and may
 * differ from the setup values).  x (device) holds x0 on entry and the solution on return.  Stops
 * when the Givens estimate reaches rtol ||b|| and confirms it with ||b - A x|| <= rtol ||b||.
 * info (host) is filled when non-NULL.  Errors: NOT_CONVERGED (x = last iterate), BREAKDOWN,
 * STATE, INVALID_ARG. */
mgr_status_t fgmres_solve(mgr_handle_t h, const mgr_bsr3_t* A, const double* b, double* x, double rtol,
                          int restart, int maxit, mgr_solve_info_t* info);

/* Release the handle and all its device memory (synchronises its stream).  NULL is accepted. */
mgr_status_t mgr_destroy(mgr_handle_t h);

/* ---- transposed solves (adjoint) ----------------------------------------------------------------
 * For a handle set up on A with options.adjoint = 1.  z = M^-T r, the exact transpose of mgr_apply's
 * operator M^-1 (up to rounding): the levels in reverse roles (P_l^T = S_C + W_p^T S_F restricts, the
 * F-relaxation sweeps run with A_ff^T, the coarse residual is formed with A_cf^T, the V-cycle is
 * V(post, pre) with A_k^T, and the global relaxation closes with z = g + B^T (y - A^T g)).
 * MGR_ERR_STATE without options.adjoint. */
mgr_status_t mgr_apply_transpose(mgr_handle_t h, const double* r, double* z);
/* Solves A^T x = b (A the matrix given to mgr_setup, with its values as passed now) by GMRES(m) on
 * M^-T A^T x = M^-T b: the preconditioner on the left makes the operator (A M^-1)^T, the transpose of
 * the forward solve's, which keeps its spectrum and conditioning (with M^-T on the right, restarted
 * GMRES stalls on layered workloads whose forward solve converges).  Each restart cycle begins from
 * the true residual and convergence is declared on ||b - A^T x|| <= rtol ||b||; arguments and
 * statuses as fgmres_solve. */
mgr_status_t fgmres_solve_transpose(mgr_handle_t h, const mgr_bsr3_t* A, const double* b, double* x, double rtol,
                                    int restart, int maxit, mgr_solve_info_t* info);

/* ---- introspection (for parity tests and reporting) ------------------------------------------ */
/* Matrix kinds: 0 level operator A_l (l = 0..L), 1 W_p(l), 2 W_r(l), 3 P(l), 4 R(l) (l < L),
 * 5 AMG operator A_k, 6 AMG P_k, 7 AMG R_k = P_k^T, 8 AMG strength S_k (values 1).
 * All are the FP64 setup copies, CSR with int64 row pointers and ascending int32 columns. */
mgr_status_t mgr_get_levels(mgr_handle_t h, int* mgr_levels, int* amg_levels);
mgr_status_t mgr_matrix_shape(mgr_handle_t h, int kind, int level, int64_t* nrows, int64_t* ncols,
                              int64_t* nnz);
/* Copy a matrix into caller device buffers rowptr[nrows+1], col[nnz], val[nnz] (val may be NULL). */
mgr_status_t mgr_copy_matrix(mgr_handle_t h, int kind, int level, int64_t* rowptr, int32_t* col, double* val);
/* Vector kinds: 0 F-relaxation scaling of level l, 1 AMG smoother scaling of level k, 2 inverses of
 * the 3x3 diagonal blocks (9 nb), 3 F list of level l, 4 C list of level l, 5 AMG C/F split
 * (1 = C, -1 = F).  Copied as doubles into the caller's device buffer. */
mgr_status_t mgr_vector_len(mgr_handle_t h, int kind, int level, int64_t* len);
mgr_status_t mgr_copy_vector(mgr_handle_t h, int kind, int level, double* out);
/* Device bytes held by the handle (host out). */
mgr_status_t mgr_memory_bytes(mgr_handle_t h, int64_t* bytes);
/* Largest number of device bytes the handle has held at once since mgr_create, setup and solve
 * work buffers included (host out). */
mgr_status_t mgr_memory_peak_bytes(mgr_handle_t h, int64_t* bytes);
/* Statistics (host outs, each may be NULL): wall time of the last mgr_setup in milliseconds, kernel
 * launches issued by the last mgr_apply, the kernel launches in the captured apply graph (0 while
 * the apply is launched directly), and the process-wide
 * count of kernel launches issued by this library since load. */
mgr_status_t mgr_get_stats(mgr_handle_t h, double* setup_ms, int64_t* apply_launches, int64_t* graph_nodes,
                           int64_t* total_launches);
/* Process-wide count of host waits on the GPU issued by this library since load (host out): scalar
 * read-backs (sizes of products and coarse grids, PMIS progress, Krylov scalars) and stream
 * synchronisations.  A measurement aid: in the setup each wait leaves the GPU idle until the host
 * has issued the next launch.  NULL: MGR_ERR_INVALID_ARG. */
mgr_status_t mgr_get_host_waits(int64_t* waits);
/* Index audit of a set-up handle (host out, synchronises): on the device, every column index the
 * apply and the Krylov products gather with is recomputed from its stored form (CSR columns, sliced
 * 32-bit columns, slice base + 16-bit offset, row + offset-table code) and checked against the
 * operator's column count, with the slice offsets, row pointers, row permutations and the F/C/map
 * lists of every level; *bad = the number of violations (0 for a sound hierarchy).  A debugging aid
 * that stands in for a memory checker: an index out of range here is an out-of-bounds gather in
 * the apply.  Before mgr_setup: MGR_ERR_STATE. */
mgr_status_t mgr_audit(mgr_handle_t h, int64_t* bad);

/* Per-kernel timing on the handle's stream: enable = 1 starts recording CUDA events around every
 * launch of the named kernels and clears earlier totals, enable = 0 stops.  mgr_kernel_time returns
 * the launches and the summed device milliseconds recorded for `name` (synchronises).  Names:
 *   solve:  "bsr3_spmv_f64" (Krylov SpMV), "mdot", "mupdate" (Arnoldi), "global_relax",
 *           "bsr_resid_split" (level-0 residual); per MGR level l = 0..3: "frelax<l>" (F-relaxation
 *           sweeps), "restrict<l>" (coarse residual r_C - A_cf e_F), "interp<l>" (e = P e_c); per AMG
 *           level: "amg0_rows", "amg1_rows", "amg2_rows", "amgc_rows" (smoothing and residual passes,
 *           levels 3 and coarser together), "amg0_restrict", "amg1_restrict", "amgc_restrict",
 *           "amg0_prolong", "amg1_prolong", "amgc_prolong" (transfers, levels 2 and coarser together);
 *           "mgr_apply" (each whole forward application), "amg_tail" (the coarse solver's cycle from
 *           AMG level 3 down, as one scope);
 *   setup:  "setup_total", "setup_mgr_level", "setup_mgr_rap", "setup_amg", "setup_amg_strength",
 *           "setup_amg_pmis", "setup_amg_extpi", "extpi_pattern", "extpi_weights",
 *           "setup_amg_transpose", "setup_amg_rap", "setup_dense_inverse", "setup_cast_alloc",
 *           "spgemm", "fused_small", "fused_copy", "spgemm_numeric", "sym_ub", "sym_count",
 *           "sym_fill", "sym_block", "sym_bitmap"; per product: "rap_mgr<l>_AP",
 *           "rap_mgr<l>_RAP" (l = 0..2), "rap_amg0_AP", "rap_amg0_PtAP", "rap_amg1_AP", "rap_amg1_PtAP",
 *           "rap_amgc_AP", "rap_amgc_PtAP" (AMG levels 2 and coarser together), "spgemm_extpi".
 * Unknown names report 0 launches. */
mgr_status_t mgr_profile(mgr_handle_t h, int enable);
/* Restrict the recording to a comma-separated list of the names above (NULL or "" records every
 * name); applies to the following mgr_profile(h, 1) session.  Recording fewer names keeps the event
 * overhead out of the timed work. */
mgr_status_t mgr_profile_select(mgr_handle_t h, const char* names);
mgr_status_t mgr_kernel_time(mgr_handle_t h, const char* name, int64_t* launches, double* total_ms);
/* Algorithmic bytes of the launches recorded for `name` since profiling was enabled (host out): for
 * the solve kernels, every input element read once and every output element written once (values,
 * a 4-byte column index per sparse entry, 8-byte row pointers, vectors), whatever form the layout
 * stores; padding and cache re-reads not counted; 0 for the setup scopes.  Divided by
 * mgr_kernel_time's milliseconds it gives the achieved algorithmic bandwidth.
 * mgr_kernel_bytes_stored: the same count with the column indices in the form the sliced layouts
 * store them (one-byte offset codes, 16-bit offsets, or 4-byte indices). */
mgr_status_t mgr_kernel_bytes(mgr_handle_t h, const char* name, double* bytes);
mgr_status_t mgr_kernel_bytes_stored(mgr_handle_t h, const char* name, double* bytes);

/* ---- stand-alone kernels ----------------------------------------------------------------------- */
/* y = A x (sub == NULL) or y = sub - A x, FP64, on `cuda_stream`.  The hot sparse product of the
 * Krylov method (section 6).  x, y: double[3 nb], must not overlap. */
mgr_status_t mgr_bsr3_spmv(const mgr_bsr3_t* A, const double* x, const double* sub, double* y, void* cuda_stream);

/* Block transpose for the adjoint solve: At has block (J, I) = (block (I, J))^T.  Outputs are caller
 * device buffers with the sizes of A (rowptr[nb+1], colind[nnzb], values[9 nnzb]); the columns of
 * each block row come out ascending.  Synchronises the stream. */
mgr_status_t mgr_bsr3_transpose(const mgr_bsr3_t* A, int64_t* rowptr_t, int32_t* colind_t, double* values_t,
                                void* cuda_stream);

/* Adjoint gradient on the pattern of A: grad[9k + 3p + q] = -lambda[3I+p] * x[3J+q] for every
 * stored block k = (I, J) (dL/dA = -lambda x^T restricted to the pattern). */
mgr_status_t mgr_bsr3_outer_grad(const mgr_bsr3_t* A, const double* lambda, const double* x, double* grad,
                                 void* cuda_stream);

/* ---- measurement ---------------------------------------------------------------------------- */
/* FP64 FMA rate of this GPU, the roofline of the FP64-bound Krylov kernels (the 3x3-block SpMV and
 * the Gram-Schmidt multi-dot and update issue FP64 FMAs faster than HBM feeds them on GB300).  Runs
 * one warm-up and `launches` timed launches of a kernel of eight independent FMA chains of
 * `chain_len` (a positive multiple of 4) FMAs per thread over a full-occupancy grid on `cuda_stream`,
 * timed with CUDA events; writes the FMAs per second / 1e9 and the milliseconds per launch (host
 * outs; the latter may be NULL).  Allocates three doubles of scratch; synchronises the stream. */
mgr_status_t mgr_probe_fp64_fma(int64_t chain_len, int launches, void* cuda_stream, double* gfma_per_s,
                                double* ms_per_launch);

/* ---- allocation-free variant ------------------------------------------------------------------
 * The paper has no counterpart to this entry point.
 *
 * mgr_bsr3_transpose_noalloc: the block transpose of mgr_bsr3_transpose (same arguments, same
 * result) for callers that cannot let a library allocate device memory during a call -- code that
 * runs under a device-memory budget or pool the caller owns, latency-critical code that cannot absorb
 * an allocation, or a host application that hands the library only buffers it manages itself.  It
 * calls no cudaMalloc, cudaFree or allocating library routine: its working memory (per-column
 * counters and the source index of every transposed block) is one file-scope device array of about
 * 4.7 MB, which every GPU that loads this library holds until the process exits.
 * Limits: nb <= 65536 block rows and nnzb <= 524288 blocks; larger inputs return
 * MGR_ERR_UNSUPPORTED without touching the GPU.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents (each call clears the counters
 * and the error word it needs): calls that overlap on the GPU -- on other streams or from other
 * threads -- race.
 * The input is checked on the device before anything is written through it: row pointers that do
 * not run from 0 to nnzb without decreasing, or a column outside [0, nb), return MGR_ERR_INVALID_ARG
 * (rowptr_t may then hold partial counts; colind_t and values_t are not written).
 * Enqueued on cuda_stream; the call then synchronises that stream once to read the check. */
mgr_status_t mgr_bsr3_transpose_noalloc(const mgr_bsr3_t* A, int64_t* rowptr_t, int32_t* colind_t, double* values_t,
                                        void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MGR_H_ */
