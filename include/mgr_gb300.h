/*
 * mgr_gb300.h -- C ABI of the GB300 (sm_103a) multigrid-reduction solver.
 *
 * The library applies the multigrid reduction (MGR) preconditioner of Bui,
 * Osei-Kuffuor, Castelletto and White ("A Scalable Multigrid Reduction
 * Framework for Multiphase Poromechanics of Heterogeneous Media") inside a
 * right-preconditioned flexible GMRES solve (Sec. 4) of the fully implicit
 * multiphase-poromechanics Jacobian (Eq. "block_linear_system").  Setup and
 * solve run entirely in CUDA kernels on the device.
 *
 * Conventions shared by every entry point
 *   - Return value: 0 on success, MGR_NOT_CONVERGED (+1) when FGMRES stopped
 *     at max_iter (x then holds the last iterate and info is filled), and a
 *     negative MGR_ERR_* code on failure; mgr_error_string() names it.
 *   - Pointers documented as "device" must point to memory of the current
 *     CUDA device; "host" pointers to ordinary host memory.
 *   - All device work is enqueued on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream).  mgr_setup and fgmres_solve synchronise the
 *     stream before returning; mgr_apply and mgr_vcycle do not.
 *   - Ownership: the caller owns the matrix arrays and all vectors.  mgr_setup
 *     copies what it needs, so the matrix may be freed after it returns, except
 *     that fgmres_solve reads the matrix passed to it.  A handle owns its
 *     hierarchy and workspace (device memory from cudaMallocAsync on the setup
 *     stream) until mgr_destroy.
 *   - A handle is not thread-safe: do not use one handle from two host threads
 *     or two streams at once.
 */
#ifndef MGR_GB300_H
#define MGR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MGR_MAX_LEVELS 8

/* status codes */
#define MGR_SUCCESS 0
#define MGR_NOT_CONVERGED 1
#define MGR_ERR_INVALID_ARG (-1)
#define MGR_ERR_CUDA (-2)
#define MGR_ERR_OOM (-3)
#define MGR_ERR_ZERO_DIAG (-4)   /* zero pivot: D_FF, a smoother block, the coarsest LU */
#define MGR_ERR_BREAKDOWN (-5)   /* NaN/Inf in the Arnoldi process */
#define MGR_ERR_COARSE (-7)      /* coarsest AMG level larger than the dense-LU cap */

/* F-relaxation kinds (per MGR level) */
#define MGR_FRELAX_AMG_VCYCLE 0  /* one AMG V-cycle on A_FF per sweep (Sec. 5.3) */
#define MGR_FRELAX_JACOBI 1      /* z_F += D_FF^-1 (v - A z)_F per sweep (Sec. 5.3) */

/* preconditioner precision */
#define MGR_FP64 0
#define MGR_MIXED 1              /* FP32 hierarchy and MGR/AMG apply; FP64 Krylov */

/*
 * One square sparse matrix in CSR with per-dof grouping (the 3x3 field-block
 * system of Eq. "block_linear_system": three displacement dofs per vertex and
 * saturation/pressure dofs per cell).  All arrays are DEVICE pointers.
 *   row_ptr  [n+1] int64, row_ptr[0] = 0, row_ptr[n] = nnz
 *   col_idx  [nnz] int32, strictly ascending within each row (no duplicates)
 *   val      [nnz] FP64
 *   dof_label[n]   field of each dof (0 = u, 1 = s, 2 = p); the C/F split of
 *                  each MGR level is a set of labels (Sec. 5.1: the user
 *                  chooses the C/F partition)
 *   dof_node [n]   point (vertex or cell) of each dof; the dofs of one point are
 *                  consecutive and at most 4 (the interleaved ordering of the
 *                  Remark in Sec. 5.3), giving the blocks of the global smoother
 *                  and the "diagonals of the sub-blocks" kept by the dropping
 *                  operator G (Eq. "drop_operator")
 *   dof_comp [n]   component within the point (x/y/z or s/p); the AMG of the
 *                  first F-relaxation couples only equal components (the
 *                  "unknown approach" of Sec. 6).  May be NULL (all 0).
 */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
  const int32_t* dof_label;
  const int32_t* dof_node;
  const int32_t* dof_comp;
} mgr_matrix_t;

/*
 * Solver configuration.  mgr_options_default() fills the configuration of
 * Sec. 5.3 / Sec. 6: two reductions (F = {u}, then F = {s}), N_max = 4 at the
 * first and no dropping at the second, one AMG V-cycle as the first
 * F-relaxation, one Jacobi sweep as the second, three cell-block Jacobi sweeps
 * as the second-level global smoother, AMG (theta 0.25, P_max 4, coarsest
 * <= 160 rows, <= 25 levels) on the final pressure system.
 */
typedef struct {
  int32_t num_levels;                       /* number of reductions (0..8) */
  uint32_t f_label_mask[MGR_MAX_LEVELS];    /* bit b set: label b is F at level l */
  int32_t frelax[MGR_MAX_LEVELS];           /* MGR_FRELAX_* */
  int32_t frelax_sweeps[MGR_MAX_LEVELS];
  int32_t nmax_drop[MGR_MAX_LEVELS];        /* N_max of G; < 0: no dropping */
  int32_t global_sweeps[MGR_MAX_LEVELS];    /* point-block Jacobi sweeps; 0 = none */
  double amg_theta;                         /* strength threshold */
  int32_t amg_pmax;                         /* interpolation truncation; 0 = none */
  int32_t amg_max_coarse;                   /* stop coarsening at <= this many rows */
  int32_t amg_max_levels;
  int32_t precision;                        /* MGR_FP64 or MGR_MIXED */
  uint64_t seed;                            /* PMIS weight hash seed */
  /* Operator variants of Sec. 5.1, per level (all 0 in the defaults):
   * restrict_jacobi: restriction R~ = [W_r I] with W_r = -A_CF D_FF^-1
   *   instead of injection; the coarse grid is then the full triple product
   *   A_CC - G(A_cor) with A_cor = A_CC - R~ A P~ = 2 A_CF T - W'(A_FF T),
   *   T = D_FF^-1 A_FC, W' = A_CF D_FF^-1, and r_C = (v - A z)_C + W_r (v - A z)_F;
   * frelax_post: F-relaxation after the coarse-grid correction (Eq.
   *   "MGR-post") instead of before it (Eq. "MGR-pre");
   * dff_block: D_FF = the point-block diagonal of A_FF (runs of F dofs sharing
   *   dof_node, at most 4: the 3x3 nodal blocks of A_uu) instead of
   *   diag(A_FF), in W_p, W_r and the Jacobi F-relaxation. */
  int32_t restrict_jacobi[MGR_MAX_LEVELS];
  int32_t frelax_post[MGR_MAX_LEVELS];
  int32_t dff_block[MGR_MAX_LEVELS];
  /* Global smoother per level (global_sweeps of it): 0 point-block Jacobi;
   * 1 multicolour point-block Gauss-Seidel, the parallel reading of the
   * paper's hybrid block Gauss-Seidel (Sec. 5.3 Remarks, Sec. 6): blocks
   * coloured by Jones-Plassmann rounds on the block graph of A + A^T
   * (weights splitmix64(seed ^ 0xC0 << 56 ^ level << 40 ^ block), ties to
   * the smaller block), each sweep visiting the colours in ascending order
   * and updating every block of a colour from the latest z;
   * 2 pointwise ILU(1) (Sec. 6 uses one sweep of it as the level-2 global
   *   smoother): the exact incomplete factors L U on the level-1 fill pattern
   *   pattern(A) + pattern(L_A U_A) ((L U)_ij = a_ij there), each sweep
   *   z <- z + U^-1 L^-1 (v - A z) with both triangular systems solved by
   *   ilu_solve_sweeps Jacobi iterations (y <- r - (L - I) y from y = r;
   *   w <- D_U^-1 (y - (U - D_U) w) from w = D_U^-1 y). */
  int32_t global_smoother[MGR_MAX_LEVELS];
  /* Aggressive coarsening (Sec. 6 names one level of it for A_uu): the first
   * agg_levels[s] levels of AMG slot s (slot l < num_levels: the F-relaxation
   * AMG of MGR level l; slot num_levels: the coarsest AMG) coarsen in two
   * stages -- PMIS + direct interpolation P1, then the same on P1^T A P1
   * (PMIS weights keyed by level 32 + k), P = P1 P2 truncated to amg_pmax by
   * the direct interpolation's rule.  0 in the defaults. */
  int32_t agg_levels[MGR_MAX_LEVELS];
  /* Jacobi iterations per triangular solve of the ILU(1) global smoother
   * (0..1000; default 3). */
  int32_t ilu_solve_sweeps;
  /* MGR_MIXED only (INVALID_ARG with MGR_FP64): 1 stores the smoother
   * diagonals the FP32 application reads -- the l1-Jacobi inverse diagonals
   * of every AMG level, D_FF^-1 of the Jacobi F-relaxations and the
   * point-block inverses of the global smoother -- in BF16 (each value
   * rounded once from FP64), halving their bytes; every other operator stays
   * FP32.  0 in the defaults. */
  int32_t diag_bf16;
  /* MGR_MIXED only (INVALID_ARG with MGR_FP64): 1 stores the values of the
   * AMG operators that have shared row patterns (the finest operator of each
   * AMG with at least 2^20 non-zeros) in FP16, each row scaled by its largest
   * magnitude (kept in FP32), halving the bytes of the V-cycles' largest
   * products; the products still add in FP32.  0 in the defaults. */
  int32_t values_f16;
} mgr_options_t;

typedef struct {
  int32_t restart;   /* Krylov subspace size m (default 50) */
  int32_t max_iter;  /* total preconditioner applications (default 1000) */
  double rtol;       /* stop when ||b - A x||_2 <= rtol ||b||_2 (default 1e-8) */
  /* Arnoldi orthogonalisation of iteration j, in FP64 (the paper names GMRES
   * without fixing it):
   *   MGR_ORTHO_MGS  -- modified Gram-Schmidt, two projections per launch
   *                     (j/2 + 2 dependent launches; the second projection of
   *                     a pair is corrected by the pair's own basis inner
   *                     product, so every projection is the one-at-a-time
   *                     recurrence's; 2 FMAs and 24 bytes per basis entry,
   *                     memory-bound);
   *   MGR_ORTHO_CGS2 -- classical Gram-Schmidt applied twice: three passes
   *                     over the basis, 4 FMAs per basis entry (FP64-bound on
   *                     GB300, but a fixed handful of launches);
   *   MGR_ORTHO_AUTO -- (default) MGS for systems of at least 2^20 unknowns,
   *                     CGS2 below, where MGS's per-launch latency dominates.
   * Every batch schedule follows the same per-system choice, so batched
   * solutions stay bitwise those of fgmres_solve.  Other values: INVALID_ARG. */
  int32_t ortho;
} fgmres_options_t;

#define MGR_ORTHO_CGS2 0
#define MGR_ORTHO_MGS 1
#define MGR_ORTHO_AUTO 2

typedef struct {
  int32_t iters;         /* preconditioner applications performed */
  int32_t restarts;
  int32_t converged;     /* 1 if the true relative residual met rtol */
  double rel_res_true;   /* ||b - A x|| / ||b|| recomputed in FP64 at the end */
  double setup_s;        /* device time of mgr_setup for this handle */
  double solve_s;        /* device time of this fgmres_solve */
  double* res_hist;      /* host array or NULL: estimated relative residual
                            after each iteration (entry 0 = 1.0) */
  int32_t res_hist_cap;
} fgmres_info_t;

typedef struct mgr_handle_s* mgr_handle_t;

/* Fill `o` with the defaults described above; two_phase = 0 gives the
 * single-reduction u | p configuration. */
void mgr_options_default(mgr_options_t* o, int two_phase);
void fgmres_options_default(fgmres_options_t* o);

/*
 * Build the MGR hierarchy of A (Sec. 5.2-5.3, Eqs. "injective_rp",
 * "drop_operator", "coarse_grid_flow_sparse", "coarse_grid_pressure") and the
 * inner AMG hierarchies (Sec. 6) on the device.  On success *out holds a new
 * handle.  Errors: INVALID_ARG (bad sizes/options, more than 4 dofs per point,
 * an empty F or C set), ZERO_DIAG, COARSE, OOM, CUDA.
 */
int mgr_setup(const mgr_matrix_t* A, const mgr_options_t* o, void* stream, mgr_handle_t* out);

/*
 * z = M^-1 v: one application of the multilevel MGR preconditioner with
 * pre-smoothing F-relaxation (Algorithm 2, Eq. "MGR-pre").  v and z are device
 * FP64 arrays of length n; they must not overlap.  Under MGR_MIXED, v is
 * rounded to FP32 on entry and z computed in FP32, then widened.
 */
int mgr_apply(mgr_handle_t h, const double* v, double* z, void* stream);

/*
 * Solve A x = b by right-preconditioned flexible GMRES(m) with the handle's
 * MGR preconditioner (Sec. 4), x0 = 0, FP64 Arnoldi with classical
 * Gram-Schmidt applied twice, Givens rotations, and the true residual
 * recomputed in FP64 at every restart.  A must be the matrix the handle was set
 * up from; b and x are device FP64 arrays of length n.  info (host) may be
 * NULL.  Returns 0, MGR_NOT_CONVERGED, or an error (BREAKDOWN on NaN/Inf).
 */
int fgmres_solve(mgr_handle_t h, const mgr_matrix_t* A, const double* b, double* x,
                 const fgmres_options_t* o, fgmres_info_t* info, void* stream);

/*
 * The whole path from HOST memory in one call: copies A (row pointers,
 * columns, values, dof_label, dof_node, dof_comp if not NULL) and b to the
 * device, builds the preconditioner (mgr_setup with options o), solves with
 * fgmres_solve (options fo; NULL: defaults), copies x back and frees every
 * device buffer.  All pointers in A and b, x are HOST pointers; pinned host
 * memory gives the full transfer rate (on GB300 ~210 GB/s host to device),
 * pageable memory works at a lower rate.  info (host) may be NULL; its
 * setup_s and solve_s are the device phases, without the transfers.  Returns
 * what mgr_setup or fgmres_solve returns; x is written only on success or
 * MGR_NOT_CONVERGED.  Synchronises the stream.
 */
int mgr_solve_host(const mgr_matrix_t* A, const double* b, double* x, const mgr_options_t* o,
                   const fgmres_options_t* fo, fgmres_info_t* info, void* stream);

/* Release every device allocation of the handle (synchronises the device). */
int mgr_destroy(mgr_handle_t h);

const char* mgr_error_string(int code);

/* ---- inspection (parity checks against an independent implementation) ---- */

/* Hierarchy matrices, copied to HOST buffers.  kind:
 *   0 A_l of MGR level `slot`;   1 W_p of level slot (nF x nC);
 *   2 A_cor before dropping (A_CF D_FF^-1 A_FC, or A_CC - R~ A P~ with the
 *     Jacobi restriction);  3 G(A_cor);
 *   4 the next-level operator S_{slot+1};
 *   5 W_r of level slot (nC x nF; only with restrict_jacobi);
 *   6 D_FF^-1 of level slot as a sparse matrix (nF x nF; only with dff_block);
 *   7 the ILU(1) factors of level slot on one pattern: strict lower part of L
 *     (unit diagonal implied) and U (only with global_smoother 2);
 *   10 AMG operator, 11 strength pattern, 12 interpolation P, 13 R = P^T of
 *   AMG slot `slot` (0..L-1: F-relaxation AMG of MGR level slot; L: the AMG
 *   of the coarsest MGR level), level `lvl`.
 * dims[0..2] receive rows, cols, nnz; row_ptr/col_idx/val are filled when
 * non-NULL (sizes n+1, nnz, nnz).  Synchronises the device. */
int mgr_get_csr(mgr_handle_t h, int kind, int slot, int lvl, int64_t* dims,
                int64_t* row_ptr, int32_t* col_idx, double* val);

/* Number of AMG levels in slot `slot` (0 if that slot has no AMG). */
int mgr_amg_levels(mgr_handle_t h, int slot);

/* Number of shared row patterns of the operator of AMG slot `slot`, level
 * `lvl` (0: the operator is applied as plain CSR).  The finest operator of
 * each AMG with at least 2^20 non-zeros is checked at setup: when its rows
 * share at most 4096 patterns of columns relative to the row -- the stencil
 * rows of a structured mesh -- the application reads a 2-byte pattern id per
 * row and the values, instead of a 4-byte column index per non-zero; the
 * products are the same, summed in the same order.  INVALID_ARG for a bad
 * handle, slot or level.  Host-side query. */
int mgr_row_patterns(mgr_handle_t h, int slot, int lvl);

/* C/F marks (+1 C, -1 F, int8, HOST buffer of length n or NULL) of AMG slot
 * `slot`, level `lvl`; returns n, or a negative error. */
int64_t mgr_get_cf(mgr_handle_t h, int slot, int lvl, int8_t* out);

/* One V-cycle of AMG slot `slot` from a zero guess: x = B b (device FP64
 * arrays of that AMG's size).  Asynchronous on `stream`. */
int mgr_vcycle(mgr_handle_t h, int slot, const double* b, double* x, void* stream);

/* y = A x with the FP64 CSR product that fgmres_solve applies to the Jacobian
 * at every iteration (the "w = A z_j" step of right-preconditioned GMRES,
 * Sec. 4; large systems use the sliced form of mgr_jacobian_product).
 * A's arrays, x and y are DEVICE arrays (n doubles each; y
 * must not overlap x); the grouping arrays of A are not read.  Asynchronous
 * on `stream`.  INVALID_ARG for a NULL or negative-size argument. */
int mgr_spmv(const mgr_matrix_t* A, const double* x, double* y, void* stream);

/* y = A x as fgmres_solve(h, A, ...) forms it.  From 2^24 non-zeros the
 * solve's FP64 products read a sliced (SELL-32) copy of A, rebuilt from A at
 * the start of every solve: rows in slices of 32, a slice's entries stored
 * entry-major, one GPU thread per row (GB300's FP64 pipe is narrow, and this
 * form issues one multiply-add per non-zero with no cross-lane reduction).
 * Each row's sum then runs over its entries in order, so y agrees with
 * mgr_spmv to rounding, not bitwise.  refresh = 1 rebuilds the copy from A
 * first (one pass over A; synchronises `stream`); refresh = 0 reuses the copy
 * of the last solve or refresh of these same arrays -- only for a caller that
 * has not changed A since -- and is asynchronous.  Below 2^24 non-zeros this
 * is mgr_spmv.  Device arrays as for mgr_spmv.  Returns 1 (sliced copy read),
 * 0 (CSR) or a negative error (INVALID_ARG also for refresh other than 0 or
 * 1). */
int mgr_jacobian_product(mgr_handle_t h, const mgr_matrix_t* A, const double* x, double* y,
                         int refresh, void* stream);

/* Splitmix64 (Steele, Lea, Flood 2014) as evaluated on the device, for tests
 * of the PMIS weight hash: out[i] = splitmix64(in[i]) for n values (device). */
int mgr_splitmix64_device(const uint64_t* in, uint64_t* out, int64_t n, void* stream);

/*
 * One V-cycle of AMG slot `slot` from a zero guess, like mgr_vcycle, but
 * allocating nothing and using none of the handle's workspace.  (The paper has
 * no counterpart: this serves callers that cannot allocate device memory where
 * they run, e.g. a program whose device memory is all handed to its own pool up
 * front, or a loop that forbids allocation after start-up.)
 *   b, x: DEVICE FP64 arrays of that AMG's size, supplied by the caller.
 *   Workspace: one fixed 8 MiB buffer compiled into the library
 *   (static __device__, held by every GPU that loads the library until exit).
 *   The CUDA runtime maps it when it loads this part of the library on a
 *   device; under lazy module loading (the CUDA default) that is the first
 *   call of this entry point on the device, which therefore can take device
 *   memory and should be made at start-up, before any stream capture; later
 *   calls take none.
 *   A V-cycle whose level vectors need more than 8 MiB is rejected with
 *   MGR_ERR_INVALID_ARG and a message on stderr; nothing is launched then.
 *   Every call made outside stream capture looks up the buffer's device
 *   address (cudaGetSymbolAddress, with the device current), so a device reset
 *   between calls is harmless; a call on a capturing stream reuses the address
 *   of the last uncaptured call on that device, so make the first call on a
 *   device before any stream capture (a captured first call is rejected with
 *   MGR_ERR_INVALID_ARG), and make an uncaptured call again after a device
 *   reset before capturing.  Every call on a device shares the buffer and it
 *   keeps the last call's contents (each vector in it is written before it is
 *   read, so nothing needs clearing); calls that overlap on the GPU (different
 *   streams, or host threads) race on it and must be serialised by the caller.
 * Asynchronous on `stream`.
 */
int mgr_vcycle_noalloc(mgr_handle_t h, int slot, const double* b, double* x, void* stream);

/*
 * Batched ensemble: nsys independent Jacobians of uneven size (for instance
 * permeability realisations or time steps), each with its own MGR hierarchy,
 * FGMRES iteration and convergence test.  The paper solves one system per
 * run; these entries add nothing to its method (Sec. 5-6): system i's
 * hierarchy is exactly what mgr_setup builds for A[i] alone and its solution
 * exactly what fgmres_solve returns for it alone.  Two schedules:
 *   workers: host worker threads (native, one CUDA stream each) take the
 *     systems largest first, so that the GPU executes several systems'
 *     captured preconditioner graphs, Jacobian products and Gram-Schmidt
 *     kernels at once;
 *   lockstep: every system advances one FGMRES iteration per round, each
 *     phase of the round being one launch for all systems still iterating --
 *     the preconditioner applications as ONE CUDA graph with a conditional
 *     branch per system (its captured application; branches of finished
 *     systems are switched off on the device), the Jacobian products as one
 *     row-binned launch per lanes-per-row group, each Gram-Schmidt launch (a
 *     modified Gram-Schmidt pair of projections, or a classical pass) over all systems'
 *     rows, and one readback of every Hessenberg column.  Each
 *     system's arithmetic is its single-system arithmetic, so its iterations
 *     and solution are bit for bit those of fgmres_solve.
 */
typedef struct mgr_batch_s* mgr_batch_t;

/* Set up nsys systems A[0..nsys) with the same options.  `workers` = number of
 * concurrent workers (1..16) of the worker schedule; -1 selects the lockstep
 * schedule; 0 lets the library choose by timing one round -- one FGMRES
 * iteration of every system: preconditioner application, Jacobian product and
 * the default Gram-Schmidt -- with 1, 2, 4, 8 and 16 workers and with the
 * lockstep schedule (the fastest is kept, the lockstep schedule only when
 * its round takes under 0.8 of the best worker count's, since its rounds
 * keep their cost while systems finish; see mgr_batch_info).  The setups
 * themselves run on up to 16 workers.  Ordered after the caller's earlier work
 * on `stream`; synchronises `stream` before returning.  A[i] is owned by the
 * caller and may be freed afterwards.  Errors: INVALID_ARG (nsys <= 0, workers
 * > 16 or < -1, or any system's mgr_setup argument error), CUDA (workers = -1
 * and the lockstep graph cannot be built; with workers = 0 the worker
 * schedules remain), and every error of mgr_setup (the first one met;
 * nothing is kept then). */
int mgr_setup_batched(int nsys, const mgr_matrix_t* A, const mgr_options_t* o, int workers,
                      void* stream, mgr_batch_t* out);

/* Solve A[i] x[i] = b[i] for every system (device pointers; A[i] the matrices
 * given to mgr_setup_batched, b[i], x[i] of A[i].n doubles; x[i] is
 * overwritten, starting from zero).  info = array of nsys records or NULL.
 * Returns the first negative error of any system (the others still run to
 * their end), else MGR_NOT_CONVERGED if a system missed rtol, else
 * MGR_SUCCESS.  Synchronous: ordered after the caller's work on `stream` and
 * finished when it returns. */
int fgmres_solve_batched(mgr_batch_t bh, const mgr_matrix_t* A, const double* const* b,
                         double* const* x, const fgmres_options_t* o, fgmres_info_t* info,
                         void* stream);

/* Schedule in use (*workers: the worker count, or -1 for lockstep), host wall
 * time of the batched setup (s), and the autotuner's record: tune_workers[6]
 * = the schedules it timed (worker counts 1, 2, 4, 8, 16, each capped at nsys,
 * repeats dropped, then -1 for lockstep; 0 after the last) and tune_ms[6] =
 * their round times in ms (-1 after the last).  Nothing is timed when the
 * schedule was given to mgr_setup_batched.  Any pointer may be NULL. */
int mgr_batch_info(mgr_batch_t bh, int* workers, double* setup_s, int* tune_workers,
                   double* tune_ms);

/* The handle of system i (for the inspection entries above); owned by the
 * batch, valid until mgr_destroy_batched. */
int mgr_batch_handle(mgr_batch_t bh, int i, mgr_handle_t* out);

/* Wait for the batch's streams, free every system and the streams. */
int mgr_destroy_batched(mgr_batch_t bh);

/* Colours of MGR level `level`'s point blocks under the multicolour
 * Gauss-Seidel global smoother, copied to the HOST array out (NULL: size
 * query); *ncolor (may be NULL) receives the colour count.  Returns the number
 * of blocks, MGR_ERR_INVALID_ARG if the level has no such smoother.
 * Synchronises the device. */
int64_t mgr_get_block_colors(mgr_handle_t h, int level, int32_t* out, int32_t* ncolor);

/* Number of CUDA kernels this library has run in this process (all handles,
 * all threads; a graph launch adds the kernels of the graph, those of a
 * lockstep batch graph's active branches).  Lets a caller count the kernels
 * of a region. */
int64_t mgr_launch_count(void);

/* Number of launch calls this library's host code has issued in this process:
 * one per kernel launched directly and one per CUDA graph launched, however
 * many kernels the graph holds. */
int64_t mgr_host_launch_count(void);

/* Identifier of the sources this library was compiled from: the first 16 hex
 * digits of a SHA-256 over the CUDA sources, this header and the compiler
 * flags (the build step passes it in).  Lets a caller check that the loaded
 * library was built from the sources it expects. */
const char* mgr_build_id(void);

/* Bytes of the library's memory pool on the current device: *used = held by
 * live allocations (handle hierarchies and workspaces), *reserved = mapped by
 * the pool, used or kept for reuse.  Either pointer may be NULL.  Host-side
 * query; no device work. */
int mgr_memory_usage(size_t* used, size_t* reserved);

/* Device memory: the library allocates from its own stream-ordered memory
 * pool on each device, which keeps freed blocks mapped so that the next setup
 * reuses them without driver calls.  This entry point synchronises the
 * current device and returns the pool's unused memory to the driver until at
 * most keep_bytes stay reserved (0: all).  Handles stay valid. */
int mgr_trim_memory(size_t keep_bytes);

#ifdef __cplusplus
}
#endif
#endif /* MGR_GB300_H */
