/*
 * mgr_oracle.c -- plain, serial, FP64 CPU oracle of MGR-preconditioned FGMRES.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the GPU library is
 * checked against.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never does.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * It restates, step by step and without any blocking or fusion, the method of
 * Bui, Osei-Kuffuor, Castelletto, White, "A Scalable Multigrid Reduction
 * Framework for Multiphase Poromechanics of Heterogeneous Media":
 *   - C/F splitting by field labels (Sec. 5.1, Sec. 5.3),
 *   - Jacobi interpolation W_p = -D_FF^-1 A_FC, injection restriction W_r = 0
 *     (Sec. 5.1, Eq. "injective_rp"),
 *   - non-Galerkin coarse grid S = A_CC - G(A_CF D_FF^-1 A_FC) with the N_max
 *     dropping operator G (Sec. 5.2, Eq. "drop_operator"),
 *   - the multilevel MGR V-cycle with global smoothing and F-relaxation
 *     (Sec. 5.2, Algorithm 2),
 *   - options of Sec. 5.1: Jacobi restriction W_r = -A_CF D_FF^-1 (full
 *     triple product R~ A P~), F-relaxation after the coarse-grid correction
 *     (Eq. "MGR-post"), and D_FF as the point-block diagonal of A_FF,
 *   - global smoother: point-block Jacobi, multicolour point-block
 *     Gauss-Seidel (the parallel reading of hybrid block Gauss-Seidel), or
 *     ILU(1) with Jacobi iterations for its triangular solves,
 *   - optional aggressive (two-stage) coarsening of the first AMG levels,
 *   - the inner AMG (Sec. 6 solver settings: unknown approach for A_uu, scalar
 *     AMG for the pressure Schur complement, coarsest level by Gaussian
 *     elimination), and
 *   - right-preconditioned flexible GMRES (Sec. 4).
 * Where the paper is silent these readings are taken: strength threshold 0.25
 * on negative couplings, PMIS coarsening
 * with splitmix64 weights, direct interpolation with positive entries lumped,
 * P_max truncation with row-sum rescaling, l1-Jacobi smoothing, 2x2 cell-block
 * Jacobi global smoother, modified Gram-Schmidt Arnoldi; with the Jacobi
 * restriction the dropping G acts on the whole correction A_CC - R~ A P~.
 *
 * Summation order rule: every setup sum runs over ascending column / inner
 * index, starting from 0.0, one rounding per multiply and per add (build with
 * -ffp-contract=off).  Apply-phase arithmetic has no such rule.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-3)
#define ORC_ERR_ZERO_DIAG (-4)
#define ORC_ERR_BREAKDOWN (-5)
#define ORC_ERR_COARSE (-7)
#define ORC_NOT_CONVERGED 1

#define MAXL 8
#define MAXAMG 32
#define LU_CAP 8192

/* -------------------------------------------------------------------------- */
typedef struct {
  int64_t nr, nc, nnz;
  int64_t *rp;
  int32_t *ci;
  double *v;
} ocsr;

typedef struct {
  int32_t num_levels;
  uint32_t f_label_mask[MAXL];
  int32_t frelax[MAXL];          /* 0 = one AMG V-cycle per sweep, 1 = Jacobi */
  int32_t frelax_sweeps[MAXL];
  int32_t nmax_drop[MAXL];       /* < 0: no dropping */
  int32_t global_sweeps[MAXL];   /* block-Jacobi sweeps, 0 = none */
  double amg_theta;
  int32_t amg_pmax, amg_max_coarse, amg_max_levels;
  uint64_t seed;
  /* operator variants of Sec. 5.1 (all 0: the scheme of Sec. 5.3) */
  int32_t restrict_jacobi[MAXL]; /* 1: W_r = -A_CF D_FF^-1 instead of W_r = 0 */
  int32_t frelax_post[MAXL];     /* 1: F-relaxation after the coarse-grid
                                    correction (Eq. MGR-post), else before */
  int32_t dff_block[MAXL];       /* 1: D_FF = point-block diagonal of A_FF
                                    (blocks of F dofs sharing dof_node) */
  int32_t global_smoother[MAXL]; /* 0: point-block Jacobi sweeps; 1: multicolour
                                    point-block Gauss-Seidel sweeps */
  int32_t agg_levels[MAXL];      /* AMG slot s: its first agg_levels[s] levels
                                    are coarsened aggressively (two stages) */
  int32_t ilu_solve_sweeps;      /* global smoother 2 (ILU(1)): Jacobi iterations
                                    per triangular solve */
} orc_opts;

typedef struct {
  ocsr A, S, P, R;
  int32_t *comp;
  int8_t *cf;       /* +1 C, -1 F */
  double *l1;       /* l1-Jacobi diagonal */
} amg_level;

typedef struct {
  int nlev;
  amg_level lev[MAXAMG];
  int64_t ncoarse;
  double *lu;       /* dense LU of the coarsest matrix, row-major, pivots in piv */
  int32_t *piv;
} amg_t;

typedef struct {
  ocsr A;                 /* A_l */
  int32_t *label, *node, *comp;
  int64_t nF, nC;
  int64_t *Fidx, *Cidx;   /* F / C dofs of this level, ascending */
  int64_t *pos;           /* dof -> index within F or within C */
  double *dF;             /* D_FF = diag(A_FF) */
  ocsr W;                 /* W_p = -D_FF^-1 A_FC   (nF x nC) */
  ocsr Acf;               /* A_CF (nC x nF) */
  ocsr Afc;               /* A_FC (nF x nC) */
  ocsr Wr;                /* W_r = -A_CF D_FF^-1 (nC x nF; Jacobi restriction) */
  ocsr Bd;                /* D_FF^-1 as a sparse matrix (nF x nF; point blocks) */
  ocsr cor;               /* A_cor before dropping (nC x nC): A_CF D^-1 A_FC, or
                             with Jacobi restriction A_CC - R~ A P~ */
  ocsr corkept;           /* G(A_cor) */
  amg_t *famg;            /* F-relaxation AMG on A_FF */
  int64_t nblk;           /* global smoother: blocks of equal dof_node */
  int64_t *bstart;
  int32_t *bsize;
  double *binv;           /* 16 doubles per block (row-major, size b) */
  int32_t *bcolor;        /* multicolour Gauss-Seidel: colour of each block */
  int32_t ncolor;
  ocsr ilu;               /* ILU(1) smoother: L (strict, unit diagonal) and U on
                             one pattern, l_ij for i > j, u_ij for i <= j */
} mgr_level;

typedef struct {
  orc_opts o;
  int L;
  mgr_level lev[MAXL];
  ocsr Acoarse;
  int32_t *clabel, *cnode, *ccomp;
  amg_t *camg;
  ocsr Afull;             /* copy of the input, for FGMRES */
} oracle_t;

/* -------------------------------------------------------------------------- */
/* CSR helpers                                                                */
/* -------------------------------------------------------------------------- */
static void *xcalloc(size_t n, size_t s) {
  void *p = calloc(n ? n : 1, s);
  if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
  return p;
}

static void csr_free(ocsr *a) {
  free(a->rp); free(a->ci); free(a->v);
  memset(a, 0, sizeof(*a));
}

static void csr_init(ocsr *a, int64_t nr, int64_t nc, int64_t nnz) {
  a->nr = nr; a->nc = nc; a->nnz = nnz;
  a->rp = xcalloc((size_t)nr + 1, sizeof(int64_t));
  a->ci = xcalloc((size_t)nnz, sizeof(int32_t));
  a->v = xcalloc((size_t)nnz, sizeof(double));
}

static double csr_get(const ocsr *a, int64_t i, int64_t j) {
  for (int64_t k = a->rp[i]; k < a->rp[i + 1]; k++)
    if (a->ci[k] == j) return a->v[k];
  return 0.0;
}

/* Transpose; entries of each output row come out in ascending original row. */
static void csr_transpose(const ocsr *a, ocsr *t) {
  csr_init(t, a->nc, a->nr, a->nnz);
  for (int64_t k = 0; k < a->nnz; k++) t->rp[a->ci[k] + 1]++;
  for (int64_t i = 0; i < a->nc; i++) t->rp[i + 1] += t->rp[i];
  int64_t *fill = xcalloc((size_t)a->nc, sizeof(int64_t));
  for (int64_t i = 0; i < a->nr; i++)
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
      int64_t c = a->ci[k];
      int64_t d = t->rp[c] + fill[c]++;
      t->ci[d] = (int32_t)i;
      t->v[d] = a->v[k];
    }
  free(fill);
}

static int cmp_i32(const void *x, const void *y) {
  int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  return (a > b) - (a < b);
}

/* C = A * B (Gustavson).  Entry (i,j) = sum over ascending k of a_ik * b_kj,
 * accumulated from 0.0 with one rounding per multiply and per add.  Output
 * columns ascending. */
static void csr_matmul(const ocsr *a, const ocsr *b, ocsr *c) {
  double *acc = xcalloc((size_t)b->nc, sizeof(double));
  int64_t *mark = xcalloc((size_t)b->nc, sizeof(int64_t));
  for (int64_t j = 0; j < b->nc; j++) mark[j] = -1;
  int32_t *cols = xcalloc((size_t)b->nc, sizeof(int32_t));
  int64_t cap = a->nnz + 16, nnz = 0;
  int32_t *ci = xcalloc((size_t)cap, sizeof(int32_t));
  double *cv = xcalloc((size_t)cap, sizeof(double));
  int64_t *rp = xcalloc((size_t)a->nr + 1, sizeof(int64_t));
  for (int64_t i = 0; i < a->nr; i++) {
    int64_t nc = 0;
    for (int64_t ka = a->rp[i]; ka < a->rp[i + 1]; ka++) {
      int64_t k = a->ci[ka];
      double aik = a->v[ka];
      for (int64_t kb = b->rp[k]; kb < b->rp[k + 1]; kb++) {
        int64_t j = b->ci[kb];
        double prod = aik * b->v[kb];
        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols[nc++] = (int32_t)j; }
        acc[j] = acc[j] + prod;
      }
    }
    qsort(cols, (size_t)nc, sizeof(int32_t), cmp_i32);
    if (nnz + nc > cap) {
      while (nnz + nc > cap) cap *= 2;
      ci = realloc(ci, (size_t)cap * sizeof(int32_t));
      cv = realloc(cv, (size_t)cap * sizeof(double));
      if (!ci || !cv) abort();
    }
    for (int64_t t = 0; t < nc; t++) { ci[nnz] = cols[t]; cv[nnz] = acc[cols[t]]; nnz++; }
    rp[i + 1] = nnz;
  }
  c->nr = a->nr; c->nc = b->nc; c->nnz = nnz; c->rp = rp; c->ci = ci; c->v = cv;
  free(acc); free(mark); free(cols);
}

/* Sub-matrix A[rows, cols] where colpos[j] >= 0 gives the new column index of
 * column j (ascending with j) and -1 drops it. */
static void csr_extract(const ocsr *a, const int64_t *rows, int64_t nrows,
                        const int64_t *colpos, int64_t ncols, ocsr *out) {
  int64_t nnz = 0;
  for (int64_t r = 0; r < nrows; r++)
    for (int64_t k = a->rp[rows[r]]; k < a->rp[rows[r] + 1]; k++)
      if (colpos[a->ci[k]] >= 0) nnz++;
  csr_init(out, nrows, ncols, nnz);
  nnz = 0;
  for (int64_t r = 0; r < nrows; r++) {
    for (int64_t k = a->rp[rows[r]]; k < a->rp[rows[r] + 1]; k++) {
      int64_t p = colpos[a->ci[k]];
      if (p >= 0) { out->ci[nnz] = (int32_t)p; out->v[nnz] = a->v[k]; nnz++; }
    }
    out->rp[r + 1] = nnz;
  }
}

static void spmv(const ocsr *a, const double *x, double *y) {
  for (int64_t i = 0; i < a->nr; i++) {
    double s = 0.0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; k++) s += a->v[k] * x[a->ci[k]];
    y[i] = s;
  }
}

/* r = b - A x */
static void residual(const ocsr *a, const double *b, const double *x, double *r) {
  for (int64_t i = 0; i < a->nr; i++) {
    double s = 0.0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; k++) s += a->v[k] * x[a->ci[k]];
    r[i] = b[i] - s;
  }
}

/* -------------------------------------------------------------------------- */
/* Dense LU with partial pivoting (coarsest AMG level: Gaussian elimination,  */
/* Sec. 6 solver settings).  Pivot = largest |a|, ties to the smaller row.     */
/* -------------------------------------------------------------------------- */
static int dense_lu(double *a, int32_t *piv, int64_t n) {
  for (int64_t k = 0; k < n; k++) {
    int64_t p = k;
    double best = fabs(a[k * n + k]);
    for (int64_t i = k + 1; i < n; i++)
      if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
    piv[k] = (int32_t)p;
    if (best == 0.0) return ORC_ERR_ZERO_DIAG;
    if (p != k)
      for (int64_t j = 0; j < n; j++) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
    for (int64_t i = k + 1; i < n; i++) {
      double l = a[i * n + k] / a[k * n + k];
      a[i * n + k] = l;
      for (int64_t j = k + 1; j < n; j++) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return ORC_OK;
}

static void dense_lu_solve(const double *lu, const int32_t *piv, int64_t n, const double *b, double *x) {
  for (int64_t i = 0; i < n; i++) x[i] = b[i];
  for (int64_t k = 0; k < n; k++) { int64_t p = piv[k]; if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; } }
  for (int64_t i = 0; i < n; i++) { double s = x[i]; for (int64_t j = 0; j < i; j++) s -= lu[i * n + j] * x[j]; x[i] = s; }
  for (int64_t i = n - 1; i >= 0; i--) { double s = x[i]; for (int64_t j = i + 1; j < n; j++) s -= lu[i * n + j] * x[j]; x[i] = s / lu[i * n + i]; }
}

/* -------------------------------------------------------------------------- */
/* AMG setup                                                                  */
/* -------------------------------------------------------------------------- */

/* splitmix64 (Steele, Lea, Flood 2014): first output of the generator whose
 * state is x.  Used as a counter-based hash for the PMIS random weights. */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Classical strength of connection restricted to equal components (the AMG
 * "unknown approach" for systems, Sec. 6): j in S_i iff j != i,
 * comp_j == comp_i and -a_ij >= theta * max_{k != i, comp_k == comp_i} (-a_ik);
 * S_i is empty when that maximum is <= 0. */
static void amg_strength(const ocsr *a, const int32_t *comp, double theta, ocsr *s) {
  int64_t nnz = 0;
  csr_init(s, a->nr, a->nc, a->nnz);
  for (int64_t i = 0; i < a->nr; i++) {
    double m = 0.0;
    int any = 0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
      int64_t j = a->ci[k];
      if (j == i || comp[j] != comp[i]) continue;
      double neg = -a->v[k];
      if (!any || neg > m) { m = neg; any = 1; }
    }
    if (any && m > 0.0) {
      double thr = theta * m;
      for (int64_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
        int64_t j = a->ci[k];
        if (j == i || comp[j] != comp[i]) continue;
        if (-a->v[k] >= thr) { s->ci[nnz] = (int32_t)j; s->v[nnz] = 1.0; nnz++; }
      }
    }
    s->rp[i + 1] = nnz;
  }
  s->nnz = nnz;
}

/* PMIS coarsening (De Sterck, Yang, Heys 2006; the parallel member of the HMIS
 * family named in Sec. 6).  Weight w_i = |S^T_i| + u_i with u_i from
 * splitmix64.  Synchronous rounds: an undecided i becomes C when its weight
 * beats every undecided neighbour in the symmetrised graph (equal weights: the
 * larger index wins); then every undecided j with a C point in S_j becomes F.
 * Points with no strong connection in either direction are F from the start. */
static void amg_pmis(const ocsr *s, uint64_t seed, int slot, int level, int8_t *cf) {
  int64_t n = s->nr;
  ocsr st;
  csr_transpose(s, &st);
  double *w = xcalloc((size_t)n, sizeof(double));
  int8_t *newc = xcalloc((size_t)n, 1);
  for (int64_t i = 0; i < n; i++) {
    uint64_t key = seed ^ ((uint64_t)slot << 48) ^ ((uint64_t)level << 40) ^ (uint64_t)i;
    double u = (double)(orc_splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
    w[i] = (double)(st.rp[i + 1] - st.rp[i]) + u;
    cf[i] = 0;
    if (s->rp[i + 1] == s->rp[i] && st.rp[i + 1] == st.rp[i]) cf[i] = -1;
  }
  for (;;) {
    int64_t undecided = 0;
    for (int64_t i = 0; i < n; i++) undecided += (cf[i] == 0);
    if (!undecided) break;
    for (int64_t i = 0; i < n; i++) {
      newc[i] = 0;
      if (cf[i] != 0) continue;
      int best = 1;
      for (int pass = 0; pass < 2 && best; pass++) {
        const ocsr *g = pass ? &st : s;
        for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++) {
          int64_t j = g->ci[k];
          if (cf[j] != 0) continue;
          if (!(w[i] > w[j] || (w[i] == w[j] && i > j))) { best = 0; break; }
        }
      }
      newc[i] = (int8_t)best;
    }
    for (int64_t i = 0; i < n; i++) if (newc[i]) cf[i] = 1;
    for (int64_t j = 0; j < n; j++) {
      if (cf[j] != 0) continue;
      for (int64_t k = s->rp[j]; k < s->rp[j + 1]; k++)
        if (cf[s->ci[k]] == 1) { cf[j] = -1; break; }
    }
  }
  free(w); free(newc); csr_free(&st);
}

/* Select the `keep` entries of largest |value| (ties: smaller column); returns
 * a mask over the `m` given entries. */
static void top_abs(const int32_t *col, const double *val, int64_t m, int64_t keep, int8_t *mask) {
  for (int64_t t = 0; t < m; t++) mask[t] = 0;
  for (int64_t r = 0; r < keep && r < m; r++) {
    int64_t best = -1;
    for (int64_t t = 0; t < m; t++) {
      if (mask[t]) continue;
      if (best < 0 || fabs(val[t]) > fabs(val[best]) ||
          (fabs(val[t]) == fabs(val[best]) && col[t] < col[best]))
        best = t;
    }
    mask[best] = 1;
  }
}

/* Direct interpolation (Stueben), restricted to equal components; positive
 * couplings are lumped into the diagonal when no positive strong C neighbour
 * exists; then truncation to the pmax largest |w| with the row sum kept. */
/* P_max truncation of one interpolation row (columns ascending): keep the
 * pmax entries of largest |w| (ties: smaller column) and rescale them by
 * (sum of all w) / (sum of kept w), both sums in row order.  Returns the new
 * length. */
static int64_t truncate_row(int32_t *tc, double *tv, int64_t m, int pmax, int8_t *mask) {
  if (pmax <= 0 || m <= pmax) return m;
  top_abs(tc, tv, m, pmax, mask);
  double sall = 0.0, skept = 0.0;
  for (int64_t t = 0; t < m; t++) sall = sall + tv[t];
  for (int64_t t = 0; t < m; t++) if (mask[t]) skept = skept + tv[t];
  int64_t q = 0;
  for (int64_t t = 0; t < m; t++) {
    if (!mask[t]) continue;
    tc[q] = tc[t];
    tv[q] = (skept != 0.0) ? tv[t] * (sall / skept) : tv[t];
    q++;
  }
  return q;
}

static void amg_interp(const ocsr *a, const ocsr *s, const int32_t *comp, const int8_t *cf,
                       int pmax, ocsr *p, int64_t *nc_out) {
  int64_t n = a->nr;
  int64_t *cmap = xcalloc((size_t)n, sizeof(int64_t));
  int64_t nc = 0;
  for (int64_t i = 0; i < n; i++) cmap[i] = (cf[i] == 1) ? nc++ : -1;
  int8_t *strong = xcalloc((size_t)n, 1);
  int64_t cap = n + 16, nnz = 0;
  csr_init(p, n, nc, 0);
  free(p->ci); free(p->v);
  p->ci = xcalloc((size_t)cap, sizeof(int32_t));
  p->v = xcalloc((size_t)cap, sizeof(double));
  int32_t *tc = xcalloc((size_t)(a->nc + 1), sizeof(int32_t));
  double *tv = xcalloc((size_t)(a->nc + 1), sizeof(double));
  int8_t *mask = xcalloc((size_t)(a->nc + 1), 1);
  for (int64_t i = 0; i < n; i++) {
    int64_t m = 0;
    if (cf[i] == 1) {
      tc[0] = (int32_t)cmap[i]; tv[0] = 1.0; m = 1;
    } else {
      for (int64_t k = s->rp[i]; k < s->rp[i + 1]; k++) strong[s->ci[k]] = 1;
      double sn = 0.0, sp = 0.0, cn = 0.0, cp = 0.0, aii = 0.0;
      for (int64_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
        int64_t j = a->ci[k];
        double v = a->v[k];
        if (j == i) { aii = v; continue; }
        if (comp[j] != comp[i]) continue;
        int sc = strong[j] && cf[j] == 1;
        if (v < 0.0) { sn = sn + v; if (sc) cn = cn + v; }
        else if (v > 0.0) { sp = sp + v; if (sc) cp = cp + v; }
      }
      if (cn != 0.0 || cp != 0.0) {
        double dd = aii;
        if (cp == 0.0) dd = aii + sp;
        double alpha = (cn != 0.0) ? sn / cn : 0.0;
        double beta = (cp != 0.0) ? sp / cp : 0.0;
        for (int64_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
          int64_t j = a->ci[k];
          if (j == i || !(strong[j] && cf[j] == 1)) continue;
          double v = a->v[k];
          double coef = (v < 0.0) ? alpha : beta;
          tc[m] = (int32_t)cmap[j];
          tv[m] = -(coef * v) / dd;
          m++;
        }
      }
      for (int64_t k = s->rp[i]; k < s->rp[i + 1]; k++) strong[s->ci[k]] = 0;
      m = truncate_row(tc, tv, m, pmax, mask);
    }
    if (nnz + m > cap) {
      while (nnz + m > cap) cap *= 2;
      p->ci = realloc(p->ci, (size_t)cap * sizeof(int32_t));
      p->v = realloc(p->v, (size_t)cap * sizeof(double));
      if (!p->ci || !p->v) abort();
    }
    for (int64_t t = 0; t < m; t++) { p->ci[nnz] = tc[t]; p->v[nnz] = tv[t]; nnz++; }
    p->rp[i + 1] = nnz;
  }
  p->nnz = nnz;
  *nc_out = nc;
  free(cmap); free(strong); free(tc); free(tv); free(mask);
}

/* l1-Jacobi diagonal (Baker, Falgout, Kolev, Yang 2011, pointwise member):
 * d_i = a_ii + sum_{j != i} |a_ij| (ascending j). */
static void l1_diag(const ocsr *a, double *d) {
  for (int64_t i = 0; i < a->nr; i++) {
    double off = 0.0, aii = 0.0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; k++) {
      if (a->ci[k] == i) aii = a->v[k];
      else off = off + fabs(a->v[k]);
    }
    d[i] = aii + off;
  }
}

static void csr_copy(const ocsr *a, ocsr *b) {
  csr_init(b, a->nr, a->nc, a->nnz);
  memcpy(b->rp, a->rp, sizeof(int64_t) * (size_t)(a->nr + 1));
  memcpy(b->ci, a->ci, sizeof(int32_t) * (size_t)a->nnz);
  memcpy(b->v, a->v, sizeof(double) * (size_t)a->nnz);
}

static void amg_free(amg_t *g) {
  if (!g) return;
  for (int k = 0; k < g->nlev; k++) {
    amg_level *L = &g->lev[k];
    csr_free(&L->A); csr_free(&L->S); csr_free(&L->P); csr_free(&L->R);
    free(L->comp); free(L->cf); free(L->l1);
  }
  free(g->lu); free(g->piv); free(g);
}

/* Build the AMG hierarchy: coarsen while n > max_coarse and fewer than
 * max_levels levels exist; Galerkin coarse operator R A P with R = P^T,
 * computed as R * (A * P); coarsest level factored by dense LU. */
static int amg_setup(const ocsr *a, const int32_t *comp, const orc_opts *o, int slot, amg_t **out) {
  amg_t *g = xcalloc(1, sizeof(amg_t));
  csr_copy(a, &g->lev[0].A);
  g->lev[0].comp = xcalloc((size_t)a->nr, sizeof(int32_t));
  if (comp) memcpy(g->lev[0].comp, comp, sizeof(int32_t) * (size_t)a->nr);
  int k = 0;
  for (;;) {
    amg_level *L = &g->lev[k];
    int64_t n = L->A.nr;
    L->l1 = xcalloc((size_t)n, sizeof(double));
    l1_diag(&L->A, L->l1);
    if (n <= o->amg_max_coarse || k + 1 >= o->amg_max_levels || k + 1 >= MAXAMG) break;
    amg_strength(&L->A, L->comp, o->amg_theta, &L->S);
    L->cf = xcalloc((size_t)n, 1);
    amg_pmis(&L->S, o->seed, slot, k, L->cf);
    int64_t nc = 0;
    for (int64_t i = 0; i < n; i++) nc += (L->cf[i] == 1);
    if (nc == 0 || nc == n) break;
    amg_interp(&L->A, &L->S, L->comp, L->cf, o->amg_pmax, &L->P, &nc);
    if (slot < MAXL && k < o->agg_levels[slot]) {
      /* Aggressive coarsening, two stages (Sec. 6 names one level of it for
       * A_uu): PMIS and direct interpolation P1 as above, then the same on the
       * Galerkin operator of the first C points (PMIS key level 32 + k), and
       * P = P1 P2 truncated to P_max by the rule of the direct interpolation.
       * If the second stage cannot coarsen, the level stays an ordinary one. */
      ocsr R1, AP1, A1, S1, P2;
      csr_transpose(&L->P, &R1);
      csr_matmul(&L->A, &L->P, &AP1);
      csr_matmul(&R1, &AP1, &A1);
      int32_t *comp1 = xcalloc((size_t)nc + 1, sizeof(int32_t));
      int64_t *cmap1 = xcalloc((size_t)n + 1, sizeof(int64_t));
      for (int64_t i = 0, c = 0; i < n; i++) {
        cmap1[i] = (L->cf[i] == 1) ? c : -1;
        if (L->cf[i] == 1) comp1[c++] = L->comp[i];
      }
      amg_strength(&A1, comp1, o->amg_theta, &S1);
      int8_t *cf2 = xcalloc((size_t)nc + 1, 1);
      amg_pmis(&S1, o->seed, slot, 32 + k, cf2);
      int64_t nc2 = 0;
      for (int64_t c = 0; c < nc; c++) nc2 += (cf2[c] == 1);
      if (nc2 > 0 && nc2 < nc) {
        amg_interp(&A1, &S1, comp1, cf2, o->amg_pmax, &P2, &nc2);
        ocsr PP;
        csr_matmul(&L->P, &P2, &PP);
        int32_t *tc = xcalloc((size_t)nc2 + 1, sizeof(int32_t));
        double *tv = xcalloc((size_t)nc2 + 1, sizeof(double));
        int8_t *mask = xcalloc((size_t)nc2 + 1, 1);
        ocsr Pt;
        csr_init(&Pt, n, nc2, PP.nnz);
        int64_t nz = 0;
        for (int64_t i = 0; i < n; i++) {
          int64_t m = 0;
          for (int64_t q = PP.rp[i]; q < PP.rp[i + 1]; q++) { tc[m] = PP.ci[q]; tv[m] = PP.v[q]; m++; }
          m = truncate_row(tc, tv, m, o->amg_pmax, mask);
          for (int64_t t = 0; t < m; t++) { Pt.ci[nz] = tc[t]; Pt.v[nz] = tv[t]; nz++; }
          Pt.rp[i + 1] = nz;
        }
        Pt.nnz = nz;
        csr_free(&L->P);
        L->P = Pt;
        for (int64_t i = 0; i < n; i++)
          if (L->cf[i] == 1 && cf2[cmap1[i]] != 1) L->cf[i] = -1;
        nc = nc2;
        csr_free(&PP); csr_free(&P2);
        free(tc); free(tv); free(mask);
      }
      csr_free(&R1); csr_free(&AP1); csr_free(&A1); csr_free(&S1);
      free(comp1); free(cmap1); free(cf2);
    }
    csr_transpose(&L->P, &L->R);
    ocsr AP;
    csr_matmul(&L->A, &L->P, &AP);
    amg_level *C = &g->lev[k + 1];
    csr_matmul(&L->R, &AP, &C->A);
    csr_free(&AP);
    C->comp = xcalloc((size_t)nc, sizeof(int32_t));
    for (int64_t i = 0, c = 0; i < n; i++) if (L->cf[i] == 1) C->comp[c++] = L->comp[i];
    k++;
  }
  g->nlev = k + 1;
  amg_level *C = &g->lev[k];
  int64_t n = C->A.nr;
  if (n > LU_CAP) { amg_free(g); return ORC_ERR_COARSE; }
  g->ncoarse = n;
  g->lu = xcalloc((size_t)(n * n), sizeof(double));
  g->piv = xcalloc((size_t)n, sizeof(int32_t));
  for (int64_t i = 0; i < n; i++)
    for (int64_t q = C->A.rp[i]; q < C->A.rp[i + 1]; q++) g->lu[i * n + C->A.ci[q]] = C->A.v[q];
  int st = (n > 0) ? dense_lu(g->lu, g->piv, n) : ORC_OK;
  if (st) { amg_free(g); return st; }
  *out = g;
  return ORC_OK;
}

/* One V-cycle from a zero initial guess: one l1-Jacobi pre-sweep, residual,
 * restriction by R = P^T, recursion, prolongation, one l1-Jacobi post-sweep;
 * the coarsest level is solved exactly. */
static void amg_vcycle(const amg_t *g, int k, const double *b, double *x) {
  const amg_level *L = &g->lev[k];
  int64_t n = L->A.nr;
  if (k == g->nlev - 1) {
    if (n > 0) dense_lu_solve(g->lu, g->piv, n, b, x);
    return;
  }
  const amg_level *C = &g->lev[k + 1];
  int64_t nc = C->A.nr;
  double *r = xcalloc((size_t)n, sizeof(double));
  double *bc = xcalloc((size_t)nc, sizeof(double));
  double *xc = xcalloc((size_t)nc, sizeof(double));
  for (int64_t i = 0; i < n; i++) x[i] = b[i] / L->l1[i];
  residual(&L->A, b, x, r);
  spmv(&L->R, r, bc);
  amg_vcycle(g, k + 1, bc, xc);
  spmv(&L->P, xc, r);
  for (int64_t i = 0; i < n; i++) x[i] += r[i];
  residual(&L->A, b, x, r);
  for (int64_t i = 0; i < n; i++) x[i] += r[i] / L->l1[i];
  free(r); free(bc); free(xc);
}

/* -------------------------------------------------------------------------- */
/* MGR setup (Sec. 5.1-5.3)                                                   */
/* -------------------------------------------------------------------------- */

/* Small dense inverse by Gauss-Jordan with partial pivoting (block smoother). */
static int small_inverse(const double *a, double *inv, int b) {
  double m[4][8];
  for (int i = 0; i < b; i++)
    for (int j = 0; j < 2 * b; j++) m[i][j] = (j < b) ? a[i * b + j] : (j - b == i ? 1.0 : 0.0);
  for (int c = 0; c < b; c++) {
    int p = c;
    for (int i = c + 1; i < b; i++) if (fabs(m[i][c]) > fabs(m[p][c])) p = i;
    if (m[p][c] == 0.0) return ORC_ERR_ZERO_DIAG;
    if (p != c) for (int j = 0; j < 2 * b; j++) { double t = m[c][j]; m[c][j] = m[p][j]; m[p][j] = t; }
    double piv = m[c][c];
    for (int j = 0; j < 2 * b; j++) m[c][j] /= piv;
    for (int i = 0; i < b; i++) {
      if (i == c) continue;
      double f = m[i][c];
      for (int j = 0; j < 2 * b; j++) m[i][j] -= f * m[c][j];
    }
  }
  for (int i = 0; i < b; i++) for (int j = 0; j < b; j++) inv[i * b + j] = m[i][b + j];
  return ORC_OK;
}

static void mgr_level_free(mgr_level *l) {
  csr_free(&l->A); csr_free(&l->W); csr_free(&l->Acf); csr_free(&l->Afc);
  csr_free(&l->Wr); csr_free(&l->Bd); csr_free(&l->ilu);
  csr_free(&l->cor); csr_free(&l->corkept);
  free(l->label); free(l->node); free(l->comp); free(l->Fidx); free(l->Cidx); free(l->pos);
  free(l->dF); free(l->bstart); free(l->bsize); free(l->binv); free(l->bcolor);
  amg_free(l->famg);
  memset(l, 0, sizeof(*l));
}

/* Colouring of the point-block graph for the multicolour block Gauss-Seidel
 * global smoother (the GPU reading of the paper's hybrid block Gauss-Seidel,
 * Sec. 5.3 Remarks / Sec. 6): blocks k and m are adjacent when a row of
 * either has a column in the other (the pattern of A + A^T: S_l is not
 * structurally symmetric after dropping, and two blocks of one colour must not
 * read each other's unknowns).  Jones-Plassmann rounds: block k has the weight
 * w_k = splitmix64(seed ^ 0xC0 << 56 ^ l << 40 ^ k); in round c every block
 * still uncoloured at the start of the round whose (w_k, -k) exceeds that of
 * each neighbour uncoloured at the start of the round takes colour c. */
static void block_coloring(const ocsr *a, const int64_t *bstart, const int32_t *bsize, int64_t nb,
                           uint64_t seed, int l, int32_t *color, int32_t *ncolor) {
  int64_t n = a->nr;
  ocsr at;
  csr_transpose(a, &at);
  int64_t *blk = xcalloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t k = 0; k < nb; k++)
    for (int r = 0; r < bsize[k]; r++) blk[bstart[k] + r] = k;
  uint64_t *w = xcalloc((size_t)nb + 1, sizeof(uint64_t));
  for (int64_t k = 0; k < nb; k++)
    w[k] = orc_splitmix64(seed ^ (0xC0ULL << 56) ^ ((uint64_t)l << 40) ^ (uint64_t)k);
  for (int64_t k = 0; k < nb; k++) color[k] = -1;
  int8_t *win = xcalloc((size_t)nb + 1, 1);
  int64_t left = nb;
  int32_t c = 0;
  while (left > 0) {
    for (int64_t k = 0; k < nb; k++) {
      win[k] = 0;
      if (color[k] != -1) continue;
      int ok = 1;
      for (int pass = 0; pass < 2 && ok; pass++) {
        const ocsr *g = pass ? &at : a;
        for (int r = 0; r < bsize[k] && ok; r++) {
          int64_t i = bstart[k] + r;
          for (int64_t q = g->rp[i]; q < g->rp[i + 1]; q++) {
            int64_t m = blk[g->ci[q]];
            if (m == k || color[m] != -1) continue;
            if (w[m] > w[k] || (w[m] == w[k] && m < k)) { ok = 0; break; }
          }
        }
      }
      win[k] = (int8_t)ok;
    }
    for (int64_t k = 0; k < nb; k++)
      if (win[k]) { color[k] = c; left--; }
    c++;
  }
  *ncolor = c;
  free(blk); free(w); free(win);
  csr_free(&at);
}

/* ILU(1) of A for the global smoother (the paper's processor-local ILU(1),
 * Sec. 6).  Pattern: level-1 fill, pattern(A) + pattern(L_A U_A) with L_A,
 * U_A the strictly lower / upper parts of A (entries (i,j) reached through
 * one k < min(i,j) with a_ik, a_kj in A).  Factors by incomplete row-wise
 * (IKJ) elimination on that pattern: for each row i, for k over its lower
 * entries in ascending order, l_ik = w_ik / u_kk and w_ij -= l_ik u_kj for
 * every j > k that is in both row k and row i; L is unit lower (l_ij, i > j),
 * U upper (u_ij, i <= j), both stored on the pattern. */
static int ilu1_setup(const ocsr *a, ocsr *f) {
  int64_t n = a->nr;
  ocsr lo, up, lu;
  csr_init(&lo, n, n, a->nnz);
  csr_init(&up, n, n, a->nnz);
  int64_t nl = 0, nu = 0;
  for (int64_t i = 0; i < n; i++) {
    for (int64_t q = a->rp[i]; q < a->rp[i + 1]; q++) {
      if (a->ci[q] < i) { lo.ci[nl] = a->ci[q]; lo.v[nl] = 1.0; nl++; }
      else if (a->ci[q] > i) { up.ci[nu] = a->ci[q]; up.v[nu] = 1.0; nu++; }
    }
    lo.rp[i + 1] = nl; up.rp[i + 1] = nu;
  }
  lo.nnz = nl; up.nnz = nu;
  csr_matmul(&lo, &up, &lu);
  /* pattern = A union L_A U_A; values: a_ij or 0 */
  csr_init(f, n, n, a->nnz + lu.nnz);
  int64_t np = 0;
  for (int64_t i = 0; i < n; i++) {
    int64_t p = a->rp[i], pe = a->rp[i + 1], q = lu.rp[i], qe = lu.rp[i + 1];
    while (p < pe || q < qe) {
      int64_t cp = (p < pe) ? a->ci[p] : INT64_MAX, cq = (q < qe) ? lu.ci[q] : INT64_MAX;
      if (cp <= cq) { f->ci[np] = (int32_t)cp; f->v[np] = a->v[p]; p++; if (cp == cq) q++; }
      else { f->ci[np] = (int32_t)cq; f->v[np] = 0.0; q++; }
      np++;
    }
    f->rp[i + 1] = np;
  }
  f->nnz = np;
  csr_free(&lo); csr_free(&up); csr_free(&lu);
  int64_t *dpos = xcalloc((size_t)n, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) {
    int64_t r = f->rp[i];
    while (r < f->rp[i + 1] && f->ci[r] != i) r++;
    if (r == f->rp[i + 1]) { free(dpos); return ORC_ERR_ZERO_DIAG; }
    dpos[i] = r;
  }
  for (int64_t i = 0; i < n; i++) {
    for (int64_t q = f->rp[i]; q < f->rp[i + 1] && f->ci[q] < i; q++) {
      int64_t k = f->ci[q];
      double ukk = f->v[dpos[k]];
      if (ukk == 0.0) { free(dpos); return ORC_ERR_ZERO_DIAG; }
      double lik = f->v[q] / ukk;
      f->v[q] = lik;
      /* w_ij -= l_ik u_kj for j > k in both rows (merge of ascending columns) */
      int64_t pi = q + 1, pk = dpos[k] + 1;
      while (pi < f->rp[i + 1] && pk < f->rp[k + 1]) {
        int64_t ji = f->ci[pi], jk = f->ci[pk];
        if (ji == jk) { f->v[pi] = f->v[pi] - lik * f->v[pk]; pi++; pk++; }
        else if (ji < jk) pi++;
        else pk++;
      }
    }
    if (f->v[dpos[i]] == 0.0) { free(dpos); return ORC_ERR_ZERO_DIAG; }
  }
  free(dpos);
  return ORC_OK;
}

/* One reduction level: C/F split from the labels; D_FF = diag(A_FF);
 * W_p = -D_FF^-1 A_FC (Eq. injective_rp); A_cor = A_CF D_FF^-1 A_FC;
 * S = A_CC - G(A_cor) (Eq. drop_operator), G keeping in each row the entries
 * in columns of the row's own point (the diagonals of the field sub-blocks)
 * plus the nmax others of largest |value| (ties: smaller column). */
static int mgr_level_setup(oracle_t *h, int l, ocsr *Snext) {
  mgr_level *L = &h->lev[l];
  const orc_opts *o = &h->o;
  int64_t n = L->A.nr;
  L->pos = xcalloc((size_t)n, sizeof(int64_t));
  L->Fidx = xcalloc((size_t)n, sizeof(int64_t));
  L->Cidx = xcalloc((size_t)n, sizeof(int64_t));
  int64_t *fpos = xcalloc((size_t)n, sizeof(int64_t));
  int64_t *cpos = xcalloc((size_t)n, sizeof(int64_t));
  L->nF = L->nC = 0;
  for (int64_t i = 0; i < n; i++) {
    int isF = (o->f_label_mask[l] >> L->label[i]) & 1u;
    if (isF) { fpos[i] = L->nF; cpos[i] = -1; L->Fidx[L->nF++] = i; }
    else { cpos[i] = L->nC; fpos[i] = -1; L->Cidx[L->nC++] = i; }
    L->pos[i] = isF ? fpos[i] : cpos[i];
  }
  int64_t nF = L->nF, nC = L->nC;
  if (nF == 0 || nC == 0) { free(fpos); free(cpos); return ORC_ERR_ARG; }
  L->dF = xcalloc((size_t)nF, sizeof(double));
  for (int64_t f = 0; f < nF; f++) {
    L->dF[f] = csr_get(&L->A, L->Fidx[f], L->Fidx[f]);
    if (L->dF[f] == 0.0) { free(fpos); free(cpos); return ORC_ERR_ZERO_DIAG; }
  }
  ocsr Aff, Acc;
  csr_extract(&L->A, L->Fidx, nF, fpos, nF, &Aff);
  csr_extract(&L->A, L->Fidx, nF, cpos, nC, &L->Afc);
  csr_extract(&L->A, L->Cidx, nC, fpos, nF, &L->Acf);
  csr_extract(&L->A, L->Cidx, nC, cpos, nC, &Acc);
  /* T = D_FF^-1 A_FC; W_p = -T (Eq. injective_rp).  Pointwise D_FF: t = a / d.
   * Point-block D_FF (blocks = runs of F dofs sharing dof_node, at most 4):
   * Bd = the block inverses as a sparse matrix, T = Bd A_FC. */
  ocsr T;
  if (o->dff_block[l]) {
    int64_t cap = 0;
    for (int64_t f = 0; f < nF;) {
      int64_t g = f + 1;
      while (g < nF && L->node[L->Fidx[g]] == L->node[L->Fidx[f]]) g++;
      if (g - f > 4) { free(fpos); free(cpos); csr_free(&Aff); csr_free(&Acc); return ORC_ERR_ARG; }
      cap += (g - f) * (g - f);
      f = g;
    }
    csr_init(&L->Bd, nF, nF, cap);
    int64_t nb = 0;
    for (int64_t f = 0; f < nF;) {
      int64_t g = f + 1;
      while (g < nF && L->node[L->Fidx[g]] == L->node[L->Fidx[f]]) g++;
      int b = (int)(g - f);
      double blk[16], inv[16];
      for (int r = 0; r < b; r++)
        for (int c = 0; c < b; c++) blk[r * b + c] = csr_get(&Aff, f + r, f + c);
      if (small_inverse(blk, inv, b) != ORC_OK) {
        free(fpos); free(cpos); csr_free(&Aff); csr_free(&Acc); return ORC_ERR_ZERO_DIAG;
      }
      for (int r = 0; r < b; r++) {
        for (int c = 0; c < b; c++) { L->Bd.ci[nb] = (int32_t)(f + c); L->Bd.v[nb] = inv[r * b + c]; nb++; }
        L->Bd.rp[f + r + 1] = nb;
      }
      f = g;
    }
    csr_matmul(&L->Bd, &L->Afc, &T);
  } else {
    csr_copy(&L->Afc, &T);
    for (int64_t f = 0; f < nF; f++)
      for (int64_t k = T.rp[f]; k < T.rp[f + 1]; k++) T.v[k] = L->Afc.v[k] / L->dF[f];
  }
  csr_copy(&T, &L->W);
  for (int64_t k = 0; k < T.nnz; k++) L->W.v[k] = -T.v[k];
  ocsr C1;
  csr_matmul(&L->Acf, &T, &C1);            /* A_CF D^-1 A_FC */
  if (o->restrict_jacobi[l]) {
    /* U = A_CF D_FF^-1 (pointwise: u = a / d of its column; point-block:
     * U = A_CF Bd); W_r = -U.  R~ A P~ = A_CC + W_r A_FC + A_CF W_p
     * + W_r A_FF W_p = A_CC - [2 A_CF T - U (A_FF T)], and the bracket is
     * the correction that G sparsifies. */
    ocsr U, K, E;
    if (o->dff_block[l]) {
      csr_matmul(&L->Acf, &L->Bd, &U);
    } else {
      csr_copy(&L->Acf, &U);
      for (int64_t k = 0; k < U.nnz; k++) U.v[k] = L->Acf.v[k] / L->dF[L->Acf.ci[k]];
    }
    csr_copy(&U, &L->Wr);
    for (int64_t k = 0; k < U.nnz; k++) L->Wr.v[k] = -U.v[k];
    csr_matmul(&Aff, &T, &K);
    csr_matmul(&U, &K, &E);
    /* cor = 2 C1 - E on the union pattern: (2 c or 0) - (e or 0) */
    csr_init(&L->cor, nC, nC, C1.nnz + E.nnz);
    int64_t nn = 0;
    for (int64_t i = 0; i < nC; i++) {
      int64_t p = C1.rp[i], pe = C1.rp[i + 1], q = E.rp[i], qe = E.rp[i + 1];
      while (p < pe || q < qe) {
        int64_t cp = (p < pe) ? C1.ci[p] : INT64_MAX;
        int64_t cq = (q < qe) ? E.ci[q] : INT64_MAX;
        double a = 0.0, e = 0.0;
        int64_t col;
        if (cp == cq) { col = cp; a = 2.0 * C1.v[p++]; e = E.v[q++]; }
        else if (cp < cq) { col = cp; a = 2.0 * C1.v[p++]; }
        else { col = cq; e = E.v[q++]; }
        L->cor.ci[nn] = (int32_t)col;
        L->cor.v[nn] = a - e;
        nn++;
      }
      L->cor.rp[i + 1] = nn;
    }
    L->cor.nnz = nn;
    csr_free(&U); csr_free(&K); csr_free(&E); csr_free(&C1);
  } else {
    L->cor = C1;
  }
  csr_free(&T);
  /* G: keep own-point columns plus the nmax largest |value| others. */
  int32_t *cnode = xcalloc((size_t)nC, sizeof(int32_t));
  for (int64_t c = 0; c < nC; c++) cnode[c] = L->node[L->Cidx[c]];
  csr_init(&L->corkept, nC, nC, L->cor.nnz);
  int64_t nk = 0;
  int8_t *mask = xcalloc((size_t)nC + 1, 1);
  int32_t *oc = xcalloc((size_t)nC + 1, sizeof(int32_t));
  double *ov = xcalloc((size_t)nC + 1, sizeof(double));
  int64_t *oi = xcalloc((size_t)nC + 1, sizeof(int64_t));
  int nmax = o->nmax_drop[l];
  for (int64_t i = 0; i < nC; i++) {
    int64_t b = L->cor.rp[i], e = L->cor.rp[i + 1], m = 0;
    for (int64_t k = b; k < e; k++) mask[k - b] = 0;
    if (nmax < 0) {
      for (int64_t k = b; k < e; k++) mask[k - b] = 1;
    } else {
      for (int64_t k = b; k < e; k++) {
        if (cnode[L->cor.ci[k]] == cnode[i]) mask[k - b] = 1;
        else { oc[m] = L->cor.ci[k]; ov[m] = L->cor.v[k]; oi[m] = k - b; m++; }
      }
      int8_t *sel = xcalloc((size_t)m + 1, 1);
      top_abs(oc, ov, m, nmax, sel);
      for (int64_t t = 0; t < m; t++) if (sel[t]) mask[oi[t]] = 1;
      free(sel);
    }
    for (int64_t k = b; k < e; k++)
      if (mask[k - b]) { L->corkept.ci[nk] = L->cor.ci[k]; L->corkept.v[nk] = L->cor.v[k]; nk++; }
    L->corkept.rp[i + 1] = nk;
  }
  L->corkept.nnz = nk;
  free(mask); free(oc); free(ov); free(oi); free(cnode);
  /* S = A_CC - G(A_cor) on the union pattern: s = (a or 0) - (cor or 0). */
  csr_init(Snext, nC, nC, Acc.nnz + nk);
  int64_t ns = 0;
  for (int64_t i = 0; i < nC; i++) {
    int64_t p = Acc.rp[i], pe = Acc.rp[i + 1], q = L->corkept.rp[i], qe = L->corkept.rp[i + 1];
    while (p < pe || q < qe) {
      int64_t cp = (p < pe) ? Acc.ci[p] : INT64_MAX;
      int64_t cq = (q < qe) ? L->corkept.ci[q] : INT64_MAX;
      double a = 0.0, c = 0.0;
      int64_t col;
      if (cp == cq) { col = cp; a = Acc.v[p++]; c = L->corkept.v[q++]; }
      else if (cp < cq) { col = cp; a = Acc.v[p++]; }
      else { col = cq; c = L->corkept.v[q++]; }
      Snext->ci[ns] = (int32_t)col;
      Snext->v[ns] = a - c;
      ns++;
    }
    Snext->rp[i + 1] = ns;
  }
  Snext->nnz = ns;
  /* F-relaxation operator. */
  int st = ORC_OK;
  if (o->frelax[l] == 0) {
    int32_t *fcomp = xcalloc((size_t)nF, sizeof(int32_t));
    for (int64_t f = 0; f < nF; f++) fcomp[f] = L->comp[L->Fidx[f]];
    st = amg_setup(&Aff, fcomp, o, l, &L->famg);
    free(fcomp);
  }
  /* Global smoother: blocks of consecutive dofs sharing dof_node. */
  if (st == ORC_OK && o->global_sweeps[l] > 0) {
    L->bstart = xcalloc((size_t)n + 1, sizeof(int64_t));
    L->bsize = xcalloc((size_t)n + 1, sizeof(int32_t));
    int64_t nb = 0;
    for (int64_t i = 0; i < n;) {
      int64_t j = i + 1;
      while (j < n && L->node[j] == L->node[i]) j++;
      if (j - i > 4) st = ORC_ERR_ARG;   /* at most 4 dofs per point */
      L->bstart[nb] = i; L->bsize[nb] = (int32_t)(j - i > 4 ? 4 : j - i); nb++;
      i = j;
    }
    L->nblk = nb;
    L->binv = xcalloc((size_t)nb * 16, sizeof(double));
    for (int64_t bk = 0; bk < nb && st == ORC_OK; bk++) {
      int b = L->bsize[bk];
      double blk[16] = {0};
      for (int r = 0; r < b; r++)
        for (int c = 0; c < b; c++)
          blk[r * b + c] = csr_get(&L->A, L->bstart[bk] + r, L->bstart[bk] + c);
      st = small_inverse(blk, &L->binv[bk * 16], b);
    }
    if (st == ORC_OK && o->global_smoother[l] == 2)
      st = ilu1_setup(&L->A, &L->ilu);
    if (st == ORC_OK && o->global_smoother[l] == 1) {
      L->bcolor = xcalloc((size_t)nb + 1, sizeof(int32_t));
      block_coloring(&L->A, L->bstart, L->bsize, nb, o->seed, l, L->bcolor, &L->ncolor);
    }
  }
  csr_free(&Aff); csr_free(&Acc);
  free(fpos); free(cpos);
  return st;
}

/* -------------------------------------------------------------------------- */
/* MGR apply: Algorithm 2 (multilevel, pre-smoothing F-relaxation)            */
/* -------------------------------------------------------------------------- */
/* Global relaxation z = M_glo^-1 v of level l: sweeps from zero of
 * multicolour point-block Gauss-Seidel (colours in ascending order, each block
 * updated from the latest z) or of point-block Jacobi; r is scratch (n). */
static void global_relax(const mgr_level *L, const orc_opts *o, int l, const double *v, double *z,
                         double *r) {
  int64_t n = L->A.nr;
  for (int64_t i = 0; i < n; i++) z[i] = 0.0;
  if (o->global_smoother[l] == 2) {
    /* ILU(1): z <- z + U^-1 L^-1 (v - A z), each triangular system solved by
     * `ilu_solve_sweeps` Jacobi iterations from y = r and w = D_U^-1 y:
     *   y <- r - (L - I) y;   w <- D_U^-1 (y - (U - D_U) w) */
    const ocsr *F = &L->ilu;
    double *y = xcalloc((size_t)n + 1, sizeof(double));
    double *y2 = xcalloc((size_t)n + 1, sizeof(double));
    double *w = xcalloc((size_t)n + 1, sizeof(double));
    double *w2 = xcalloc((size_t)n + 1, sizeof(double));
    double *du = xcalloc((size_t)n + 1, sizeof(double));
    for (int64_t i = 0; i < n; i++) du[i] = csr_get(F, i, i);
    for (int sw = 0; sw < o->global_sweeps[l]; sw++) {
      residual(&L->A, v, z, r);
      for (int64_t i = 0; i < n; i++) y[i] = r[i];
      for (int it = 0; it < o->ilu_solve_sweeps; it++) {
        for (int64_t i = 0; i < n; i++) {
          double acc = 0.0;
          for (int64_t q = F->rp[i]; q < F->rp[i + 1]; q++)
            if (F->ci[q] < i) acc += F->v[q] * y[F->ci[q]];
          y2[i] = r[i] - acc;
        }
        memcpy(y, y2, sizeof(double) * (size_t)n);
      }
      for (int64_t i = 0; i < n; i++) w[i] = y[i] / du[i];
      for (int it = 0; it < o->ilu_solve_sweeps; it++) {
        for (int64_t i = 0; i < n; i++) {
          double acc = 0.0;
          for (int64_t q = F->rp[i]; q < F->rp[i + 1]; q++)
            if (F->ci[q] > i) acc += F->v[q] * w[F->ci[q]];
          w2[i] = (y[i] - acc) / du[i];
        }
        memcpy(w, w2, sizeof(double) * (size_t)n);
      }
      for (int64_t i = 0; i < n; i++) z[i] += w[i];
    }
    free(y); free(y2); free(w); free(w2); free(du);
    return;
  }
  /* global relaxation: z = M_glo^-1 v, sweeps from zero of multicolour block
   * Gauss-Seidel (colours in ascending order, each block updated from the
   * latest z) or of block Jacobi */
  if (o->global_smoother[l]) {
    for (int sw = 0; sw < o->global_sweeps[l]; sw++)
      for (int32_t c = 0; c < L->ncolor; c++)
        for (int64_t bk = 0; bk < L->nblk; bk++) {
          if (L->bcolor[bk] != c) continue;
          int b = L->bsize[bk];
          int64_t s0 = L->bstart[bk];
          double rb[4], d[4];
          for (int i = 0; i < b; i++) {
            double acc = v[s0 + i];
            for (int64_t q = L->A.rp[s0 + i]; q < L->A.rp[s0 + i + 1]; q++)
              acc -= L->A.v[q] * z[L->A.ci[q]];
            rb[i] = acc;
          }
          for (int i = 0; i < b; i++) {
            double acc = 0.0;
            for (int j = 0; j < b; j++) acc += L->binv[bk * 16 + i * b + j] * rb[j];
            d[i] = acc;
          }
          for (int i = 0; i < b; i++) z[s0 + i] += d[i];
        }
  }
  for (int sw = 0; sw < (o->global_smoother[l] ? 0 : o->global_sweeps[l]); sw++) {
    residual(&L->A, v, z, r);
    for (int64_t bk = 0; bk < L->nblk; bk++) {
      int b = L->bsize[bk];
      int64_t s0 = L->bstart[bk];
      double d[4];
      for (int i = 0; i < b; i++) {
        double acc = 0.0;
        for (int j = 0; j < b; j++) acc += L->binv[bk * 16 + i * b + j] * r[s0 + j];
        d[i] = acc;
      }
      for (int i = 0; i < b; i++) z[s0 + i] += d[i];
    }
  }
}

/* F-relaxation sweeps: z <- z + Q M_FF^-1 Q^T (v - A z), M_FF^-1 one AMG
 * V-cycle or Jacobi with D_FF (pointwise, or the point-block inverse Bd). */
static void mgr_frelax(const oracle_t *h, int l, const double *v, double *z, double *r,
                       double *rf, double *ef) {
  const mgr_level *L = &h->lev[l];
  const orc_opts *o = &h->o;
  int64_t nF = L->nF;
  for (int sw = 0; sw < o->frelax_sweeps[l]; sw++) {
    residual(&L->A, v, z, r);
    for (int64_t f = 0; f < nF; f++) rf[f] = r[L->Fidx[f]];
    if (o->frelax[l] == 0) amg_vcycle(L->famg, 0, rf, ef);
    else if (o->dff_block[l]) spmv(&L->Bd, rf, ef);
    else for (int64_t f = 0; f < nF; f++) ef[f] = rf[f] / L->dF[f];
    for (int64_t f = 0; f < nF; f++) z[L->Fidx[f]] += ef[f];
  }
}

static void mgr_apply_level(const oracle_t *h, int l, const double *v, double *z) {
  if (l == h->L) {           /* coarsest MGR level: one AMG V-cycle */
    amg_vcycle(h->camg, 0, v, z);
    return;
  }
  const mgr_level *L = &h->lev[l];
  const orc_opts *o = &h->o;
  int64_t n = L->A.nr, nF = L->nF, nC = L->nC;
  double *r = xcalloc((size_t)n, sizeof(double));
  double *rf = xcalloc((size_t)nF, sizeof(double));
  double *ef = xcalloc((size_t)nF, sizeof(double));
  double *rc = xcalloc((size_t)nC, sizeof(double));
  double *ec = xcalloc((size_t)nC, sizeof(double));
  global_relax(L, o, l, v, z, r);
  /* F-relaxation before the coarse-grid correction (Eq. MGR-pre) */
  if (!o->frelax_post[l]) mgr_frelax(h, l, v, z, r, rf, ef);
  /* restrict: r_C = R~ (v - A z), R~ = [W_r I]: injection (W_r = 0) or
   * Jacobi restriction r_C += W_r r_F */
  residual(&L->A, v, z, r);
  for (int64_t c = 0; c < nC; c++) rc[c] = r[L->Cidx[c]];
  if (o->restrict_jacobi[l]) {
    double *t = xcalloc((size_t)nC, sizeof(double));
    for (int64_t f = 0; f < nF; f++) rf[f] = r[L->Fidx[f]];
    spmv(&L->Wr, rf, t);
    for (int64_t c = 0; c < nC; c++) rc[c] += t[c];
    free(t);
  }
  /* recursion */
  mgr_apply_level(h, l + 1, rc, ec);
  /* interpolate e = P~ e_C = [W_p e_C; e_C] and correct */
  spmv(&L->W, ec, ef);
  for (int64_t f = 0; f < nF; f++) z[L->Fidx[f]] += ef[f];
  for (int64_t c = 0; c < nC; c++) z[L->Cidx[c]] += ec[c];
  /* F-relaxation after the correction (Eq. MGR-post) */
  if (o->frelax_post[l]) mgr_frelax(h, l, v, z, r, rf, ef);
  free(r); free(rf); free(ef); free(rc); free(ec);
}

/* -------------------------------------------------------------------------- */
/* Public oracle API (ctypes)                                                 */
/* -------------------------------------------------------------------------- */
void orc_free(void *hv) {
  oracle_t *h = hv;
  if (!h) return;
  for (int l = 0; l < MAXL; l++) mgr_level_free(&h->lev[l]);
  csr_free(&h->Acoarse); csr_free(&h->Afull);
  free(h->clabel); free(h->cnode); free(h->ccomp);
  amg_free(h->camg);
  free(h);
}

void *orc_setup(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                const int32_t *label, const int32_t *node, const int32_t *comp,
                const orc_opts *o, int *status) {
  *status = ORC_ERR_ARG;
  if (n <= 0 || o->num_levels < 0 || o->num_levels > MAXL) return NULL;
  oracle_t *h = xcalloc(1, sizeof(oracle_t));
  h->o = *o;
  h->L = o->num_levels;
  csr_init(&h->Afull, n, n, rp[n]);
  memcpy(h->Afull.rp, rp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(h->Afull.ci, ci, sizeof(int32_t) * (size_t)rp[n]);
  memcpy(h->Afull.v, v, sizeof(double) * (size_t)rp[n]);
  csr_copy(&h->Afull, &h->lev[0].A);
  int32_t *lab = xcalloc((size_t)n, sizeof(int32_t));
  int32_t *nod = xcalloc((size_t)n, sizeof(int32_t));
  int32_t *cmp = xcalloc((size_t)n, sizeof(int32_t));
  memcpy(lab, label, sizeof(int32_t) * (size_t)n);
  memcpy(nod, node, sizeof(int32_t) * (size_t)n);
  if (comp) memcpy(cmp, comp, sizeof(int32_t) * (size_t)n);
  int st = ORC_OK;
  for (int l = 0; l < h->L && st == ORC_OK; l++) {
    mgr_level *L = &h->lev[l];
    L->label = lab; L->node = nod; L->comp = cmp;
    ocsr S;
    st = mgr_level_setup(h, l, &S);
    if (st) break;
    int64_t nC = L->nC;
    int32_t *nl = xcalloc((size_t)nC, sizeof(int32_t));
    int32_t *nn = xcalloc((size_t)nC, sizeof(int32_t));
    int32_t *ncmp = xcalloc((size_t)nC, sizeof(int32_t));
    for (int64_t c = 0; c < nC; c++) {
      nl[c] = lab[L->Cidx[c]]; nn[c] = nod[L->Cidx[c]]; ncmp[c] = cmp[L->Cidx[c]];
    }
    lab = nl; nod = nn; cmp = ncmp;
    if (l + 1 < h->L) h->lev[l + 1].A = S;
    else h->Acoarse = S;
  }
  if (st == ORC_OK) {
    if (h->L == 0) csr_copy(&h->Afull, &h->Acoarse);
    h->clabel = lab; h->cnode = nod; h->ccomp = cmp;
    /* the coarsest MGR level is a scalar problem: one component */
    int32_t *zero = xcalloc((size_t)h->Acoarse.nr, sizeof(int32_t));
    st = amg_setup(&h->Acoarse, zero, o, h->L, &h->camg);
    free(zero);
  } else if (h->L == 0 || !h->lev[0].label) {
    free(lab); free(nod); free(cmp);   /* not yet owned by a level */
  }
  *status = st;
  if (st) { orc_free(h); return NULL; }
  return h;
}

int orc_apply(void *hv, const double *v, double *z) {
  oracle_t *h = hv;
  mgr_apply_level(h, 0, v, z);
  return ORC_OK;
}

/* One V-cycle of AMG slot `slot` (0..L-1: F-relaxation AMG of MGR level
 * `slot`; L: coarsest-level AMG). */
int orc_vcycle(void *hv, int slot, const double *b, double *x) {
  oracle_t *h = hv;
  const amg_t *g = (slot == h->L) ? h->camg : (slot >= 0 && slot < h->L ? h->lev[slot].famg : NULL);
  if (!g) return ORC_ERR_ARG;
  amg_vcycle(g, 0, b, x);
  return ORC_OK;
}

static double dot(const double *a, const double *b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

/* Right-preconditioned flexible GMRES(m) (Sec. 4; Saad 1993), x0 = 0,
 * modified Gram-Schmidt Arnoldi, Givens rotations; converged when the true
 * residual ||b - A x|| <= rtol ||b||.  `iters` counts preconditioner
 * applications. */
int orc_fgmres(void *hv, const double *b, double *x, int m, int maxit, double rtol,
               int *iters_out, double *relres_out, double *hist, int histcap) {
  oracle_t *h = hv;
  const ocsr *A = &h->Afull;
  int64_t n = A->nr;
  double *V = xcalloc((size_t)(m + 1) * (size_t)n, sizeof(double));
  double *Z = xcalloc((size_t)m * (size_t)n, sizeof(double));
  double *H = xcalloc((size_t)(m + 1) * (size_t)m, sizeof(double));
  double *cs = xcalloc((size_t)m, sizeof(double)), *sn = xcalloc((size_t)m, sizeof(double));
  double *g = xcalloc((size_t)m + 1, sizeof(double)), *y = xcalloc((size_t)m, sizeof(double));
  double *r = xcalloc((size_t)n, sizeof(double));
  for (int64_t i = 0; i < n; i++) x[i] = 0.0;
  double bnorm = sqrt(dot(b, b, n));
  int iters = 0, st = ORC_NOT_CONVERGED;
  double relres = 1.0;
  if (bnorm == 0.0) { st = ORC_OK; relres = 0.0; goto done; }
  residual(A, b, x, r);
  double beta = sqrt(dot(r, r, n));
  if (hist && histcap > 0) hist[0] = beta / bnorm;
  while (iters < maxit) {
    for (int64_t i = 0; i < n; i++) V[i] = r[i] / beta;
    for (int i = 0; i <= m; i++) g[i] = 0.0;
    g[0] = beta;
    int j, jend = 0;
    for (j = 0; j < m && iters < maxit; j++) {
      double *vj = &V[(size_t)j * n], *zj = &Z[(size_t)j * n], *w = &V[(size_t)(j + 1) * n];
      mgr_apply_level(h, 0, vj, zj);
      spmv(A, zj, w);
      for (int i = 0; i <= j; i++) {
        double hij = dot(w, &V[(size_t)i * n], n);
        H[i * m + j] = hij;
        for (int64_t t = 0; t < n; t++) w[t] -= hij * V[(size_t)i * n + t];
      }
      double hn = sqrt(dot(w, w, n));
      H[(j + 1) * m + j] = hn;
      if (!(hn == hn) || isinf(hn)) { st = ORC_ERR_BREAKDOWN; goto done; }
      if (hn != 0.0) for (int64_t t = 0; t < n; t++) w[t] /= hn;
      for (int i = 0; i < j; i++) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double den = sqrt(a * a + c * c);
      cs[j] = (den == 0.0) ? 1.0 : a / den;
      sn[j] = (den == 0.0) ? 0.0 : c / den;
      H[j * m + j] = cs[j] * a + sn[j] * c;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      iters++;
      jend = j + 1;
      if (hist && iters < histcap) hist[iters] = fabs(g[j + 1]) / bnorm;
      if (fabs(g[j + 1]) <= rtol * bnorm || hn == 0.0) break;
    }
    for (int i = jend - 1; i >= 0; i--) {
      double s = g[i];
      for (int k = i + 1; k < jend; k++) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < jend; i++)
      for (int64_t t = 0; t < n; t++) x[t] += y[i] * Z[(size_t)i * n + t];
    residual(A, b, x, r);
    beta = sqrt(dot(r, r, n));
    relres = beta / bnorm;
    if (relres <= rtol) { st = ORC_OK; break; }
    if (beta == 0.0) { st = ORC_OK; break; }
  }
done:
  *iters_out = iters;
  *relres_out = relres;
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(r);
  return st;
}

/* ---- hierarchy queries (parity dumps) ------------------------------------ */
enum {
  Q_MGR_A = 0,      /* A_l of MGR level l                      */
  Q_MGR_W = 1,      /* W_p of level l (nF x nC)                */
  Q_MGR_COR = 2,    /* A_cor before dropping (nC x nC)         */
  Q_MGR_CORKEPT = 3,/* G(A_cor)                                */
  Q_MGR_S = 4,      /* next level operator S_{l+1}             */
  Q_MGR_WR = 5,     /* W_r of level l (nC x nF; Jacobi restriction) */
  Q_MGR_BD = 6,     /* point-block D_FF^-1 of level l (nF x nF) */
  Q_MGR_ILU = 7,    /* ILU(1) factors of level l (L strict + U, one pattern) */
  Q_AMG_A = 10,     /* AMG slot s, level k operator            */
  Q_AMG_S = 11,     /* strength pattern                        */
  Q_AMG_P = 12,     /* interpolation                           */
  Q_AMG_R = 13
};

static const ocsr *orc_csr_ptr(oracle_t *h, int kind, int slot, int lvl) {
  if (kind < 10) {
    if (slot < 0 || slot >= h->L) return NULL;
    mgr_level *L = &h->lev[slot];
    switch (kind) {
      case Q_MGR_A: return &L->A;
      case Q_MGR_W: return &L->W;
      case Q_MGR_COR: return &L->cor;
      case Q_MGR_CORKEPT: return &L->corkept;
      case Q_MGR_S: return (slot + 1 < h->L) ? &h->lev[slot + 1].A : &h->Acoarse;
      case Q_MGR_WR: return L->Wr.rp ? &L->Wr : NULL;
      case Q_MGR_BD: return L->Bd.rp ? &L->Bd : NULL;
      case Q_MGR_ILU: return L->ilu.rp ? &L->ilu : NULL;
    }
    return NULL;
  }
  const amg_t *g = (slot == h->L) ? h->camg : (slot >= 0 && slot < h->L ? h->lev[slot].famg : NULL);
  if (!g || lvl < 0 || lvl >= g->nlev) return NULL;
  const amg_level *A = &g->lev[lvl];
  switch (kind) {
    case Q_AMG_A: return &A->A;
    case Q_AMG_S: return (lvl < g->nlev - 1) ? &A->S : NULL;
    case Q_AMG_P: return (lvl < g->nlev - 1) ? &A->P : NULL;
    case Q_AMG_R: return (lvl < g->nlev - 1) ? &A->R : NULL;
  }
  return NULL;
}

/* dims[0..2] = rows, cols, nnz.  Arrays are filled when non-NULL. */
int orc_get_csr(void *hv, int kind, int slot, int lvl, int64_t *dims,
                int64_t *rp, int32_t *ci, double *v) {
  const ocsr *a = orc_csr_ptr(hv, kind, slot, lvl);
  if (!a || !a->rp) return ORC_ERR_ARG;
  dims[0] = a->nr; dims[1] = a->nc; dims[2] = a->nnz;
  if (rp) memcpy(rp, a->rp, sizeof(int64_t) * (size_t)(a->nr + 1));
  if (ci) memcpy(ci, a->ci, sizeof(int32_t) * (size_t)a->nnz);
  if (v) memcpy(v, a->v, sizeof(double) * (size_t)a->nnz);
  return ORC_OK;
}

/* Number of AMG levels of slot s (0 if absent). */
int orc_amg_levels(void *hv, int slot) {
  oracle_t *h = hv;
  const amg_t *g = (slot == h->L) ? h->camg : (slot >= 0 && slot < h->L ? h->lev[slot].famg : NULL);
  return g ? g->nlev : 0;
}

/* C/F marks (+1/-1) of AMG slot s, level k; returns the count. */
int64_t orc_get_cf(void *hv, int slot, int lvl, int8_t *out) {
  oracle_t *h = hv;
  const amg_t *g = (slot == h->L) ? h->camg : (slot >= 0 && slot < h->L ? h->lev[slot].famg : NULL);
  if (!g || lvl < 0 || lvl >= g->nlev - 1) return -1;
  int64_t n = g->lev[lvl].A.nr;
  if (out) memcpy(out, g->lev[lvl].cf, (size_t)n);
  return n;
}

/* The global relaxation of MGR level l alone (z = M_glo^-1 v; z = 0 if the
 * level has none), for the smoother's pins. */
int orc_global_relax(void *hv, int l, const double *v, double *z) {
  oracle_t *h = hv;
  if (l < 0 || l >= h->L) return ORC_ERR_ARG;
  double *r = xcalloc((size_t)h->lev[l].A.nr + 1, sizeof(double));
  global_relax(&h->lev[l], &h->o, l, v, z, r);
  free(r);
  return ORC_OK;
}

/* Multicolour Gauss-Seidel colours of MGR level l's point blocks (returns
 * the block count, -1 if the level has none); *ncolor receives the count. */
int64_t orc_get_block_colors(void *hv, int l, int32_t *out, int32_t *ncolor) {
  oracle_t *h = hv;
  if (l < 0 || l >= h->L || !h->lev[l].bcolor) return -1;
  if (out) memcpy(out, h->lev[l].bcolor, sizeof(int32_t) * (size_t)h->lev[l].nblk);
  if (ncolor) *ncolor = h->lev[l].ncolor;
  return h->lev[l].nblk;
}

/* Dense l1 diagonal of AMG slot s, level k. */
int64_t orc_get_l1(void *hv, int slot, int lvl, double *out) {
  oracle_t *h = hv;
  const amg_t *g = (slot == h->L) ? h->camg : (slot >= 0 && slot < h->L ? h->lev[slot].famg : NULL);
  if (!g || lvl < 0 || lvl >= g->nlev) return -1;
  int64_t n = g->lev[lvl].A.nr;
  if (out) memcpy(out, g->lev[lvl].l1, sizeof(double) * (size_t)n);
  return n;
}

/* ---- direct entry to two AMG steps, for their pins ------------------------ */

/* PMIS on a caller-given strength graph S (CSR, n x n, columns ascending):
 * cf[i] = +1 (C) / -1 (F), with the weight key of AMG slot `slot`, level
 * `level`. */
int orc_pmis(int64_t n, const int64_t *srp, const int32_t *sci, uint64_t seed, int slot,
             int level, int8_t *cf) {
  if (n <= 0) return ORC_ERR_ARG;
  ocsr s;
  s.nr = n; s.nc = n; s.nnz = srp[n];
  s.rp = (int64_t *)srp; s.ci = (int32_t *)sci;
  s.v = xcalloc((size_t)s.nnz, sizeof(double));   /* pattern values, as the strength rule writes */
  for (int64_t k = 0; k < s.nnz; k++) s.v[k] = 1.0;
  amg_pmis(&s, seed, slot, level, cf);
  free(s.v);
  return ORC_OK;
}

/* Direct interpolation on caller-given A, strength graph S (it need not come
 * from the strength rule: positive couplings may be strong), components and
 * C/F marks; P (n x nc) is returned through *p_rp, *p_ci, *p_v, allocated here
 * and released with orc_free_buffer. */
int orc_interp(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
               const int64_t *srp, const int32_t *sci, const int32_t *comp, const int8_t *cf,
               int pmax, int64_t *dims, int64_t **p_rp, int32_t **p_ci, double **p_v) {
  if (n <= 0) return ORC_ERR_ARG;
  ocsr a, s, p;
  a.nr = n; a.nc = n; a.nnz = rp[n];
  a.rp = (int64_t *)rp; a.ci = (int32_t *)ci; a.v = (double *)v;
  s.nr = n; s.nc = n; s.nnz = srp[n];
  s.rp = (int64_t *)srp; s.ci = (int32_t *)sci;
  s.v = xcalloc((size_t)s.nnz, sizeof(double));
  for (int64_t k = 0; k < s.nnz; k++) s.v[k] = 1.0;
  int64_t nc = 0;
  amg_interp(&a, &s, comp, cf, pmax, &p, &nc);
  free(s.v);
  dims[0] = p.nr; dims[1] = nc; dims[2] = p.nnz;
  *p_rp = p.rp; *p_ci = p.ci; *p_v = p.v;
  return ORC_OK;
}

void orc_free_buffer(void *q) { free(q); }

/* y = A x with the input matrix (the Jacobian product of the Arnoldi step). */
int orc_matvec(void *hv, const double *x, double *y) {
  oracle_t *h = hv;
  spmv(&h->Afull, x, y);
  return ORC_OK;
}

/* y = A x for a caller-given CSR matrix (same row sums as above: ascending
 * column order from 0.0); usable at any size without a hierarchy. */
int orc_csr_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                 const double *x, double *y) {
  if (n < 0) return ORC_ERR_ARG;
  ocsr a;
  a.nr = n; a.nc = n; a.nnz = n ? rp[n] : 0;
  a.rp = (int64_t *)rp; a.ci = (int32_t *)ci; a.v = (double *)v;
  spmv(&a, x, y);
  return ORC_OK;
}
