// Internal declarations of the GB300 MGR library (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/mgr_gb300.h"

namespace mgr {

// ----------------------------------------------------------------------------
// Errors
// ----------------------------------------------------------------------------
struct Status {
  int code = MGR_SUCCESS;
};

#define MGR_TRY_CUDA(expr)                                                       \
  do {                                                                           \
    cudaError_t _e = (expr);                                                     \
    if (_e != cudaSuccess) {                                                     \
      fprintf(stderr, "mgr_gb300: %s failed: %s (%s:%d)\n", #expr,               \
              cudaGetErrorString(_e), __FILE__, __LINE__);                       \
      return _e == cudaErrorMemoryAllocation ? MGR_ERR_OOM : MGR_ERR_CUDA;       \
    }                                                                            \
  } while (0)

#define MGR_TRY(expr)            \
  do {                           \
    int _s = (expr);             \
    if (_s != MGR_SUCCESS) return _s; \
  } while (0)

// Host-side counts of this library's work: g_launches = kernels executed
// (a graph launch adds its kernel nodes), g_host_launches = launch calls the
// host issued (a graph launch counts once).  Every launch site is written
// `MGR_LAUNCH kernel<<<...>>>(...)`, a comma expression; launches recorded
// into a graph by stream capture on this thread are counted in t_captured
// instead (they run when the graph is launched).
extern std::atomic<long long> g_launches;
extern std::atomic<long long> g_host_launches;
extern thread_local int t_capturing;
extern thread_local long long t_captured;
inline int count_launch() {
  if (t_capturing) {
    ++t_captured;
  } else {
    ++g_launches;
    ++g_host_launches;
  }
  return 0;
}
inline void count_graph_launch(long long kernels) {
  g_launches += kernels;
  ++g_host_launches;
}
#define MGR_LAUNCH (void)mgr::count_launch(),

// device-side error word values (first error wins)
enum DevErr : int { DEV_OK = 0, DEV_ZERO_DIAG = 1, DEV_BAD_ARG = 2, DEV_OVERFLOW = 3 };

// ----------------------------------------------------------------------------
// Device memory owned by a handle (stream-ordered allocations)
// ----------------------------------------------------------------------------
// The library's memory pool on the current device (created on first use; null
// if it cannot be created, and allocations then use the device's default
// pool).  Freed blocks stay mapped in it for the next setup instead of going
// back to the driver at each synchronisation; mgr_trim_memory releases them.
cudaMemPool_t lib_pool();

struct Pool {
  std::vector<void*> ptrs;
  cudaStream_t s = nullptr;
  int err = MGR_SUCCESS;
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    size_t bytes = (n ? n : 1) * sizeof(T);
    cudaMemPool_t mp = lib_pool();
    cudaError_t e = mp ? cudaMallocFromPoolAsync(&p, bytes, mp, s) : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
      err = (e == cudaErrorMemoryAllocation) ? MGR_ERR_OOM : MGR_ERR_CUDA;
      (void)cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  // stream-ordered release of one allocation after the work queued on fs
  void release(void* p, cudaStream_t fs) {
    if (!p) return;
    for (auto& q : ptrs)
      if (q == p) {
        cudaFreeAsync(q, fs);
        q = nullptr;
      }
  }
  void free_all() {
    for (void* p : ptrs)
      if (p) cudaFree(p);
    ptrs.clear();
  }
  // stream-ordered release (no host wait); default: the legacy stream
  void free_all_async(cudaStream_t fs = 0) {
    for (void* p : ptrs)
      if (p) cudaFreeAsync(p, fs);
    ptrs.clear();
  }
};

// ----------------------------------------------------------------------------
// Sparse matrix in CSR on the device
// ----------------------------------------------------------------------------
struct Csr {
  int64_t nr = 0, nc = 0, nnz = 0;
  int64_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* v = nullptr;   // FP64 values (setup, FP64 apply)
  float* vf = nullptr;   // FP32 copy (mixed-precision apply), may be null
  // Shared row patterns (square operators of a structured mesh): row i's
  // columns are i + poff[pstart[pid[i]] + k], k < row length, so the apply
  // reads a 2-byte pattern id per row instead of a 4-byte column per
  // non-zero.  Null when the rows do not share few enough patterns.
  uint16_t* pid = nullptr;
  int32_t* pstart = nullptr;
  int32_t* poff = nullptr;
  int32_t npat = 0;
  // FP32 values of a patterned operator sliced for the apply (SELL-32): the
  // value k of row r at vsell[soff[r / 32] + 32 k + r % 32]; null otherwise
  float* vsell = nullptr;
  int64_t* soff = nullptr;
  // values_f16: the sliced values in FP16 instead (vsell null), row r's
  // values divided by rscale[r] (its largest magnitude)
  __half* vsellh = nullptr;
  float* rscale = nullptr;
  int32_t* sci = nullptr;   // sliced column indices of an operator without row patterns
};

// ----------------------------------------------------------------------------
// Hierarchy
// ----------------------------------------------------------------------------
struct AmgLevel {
  Csr A, S, P, R;
  int8_t* cf = nullptr;      // +1 C, -1 F (levels that were coarsened)
  int32_t* comp = nullptr;
  double* dinv = nullptr;    // 1 / l1-diagonal
  float* dinvf = nullptr;
  __nv_bfloat16* dinvh = nullptr;   // BF16 copy (MGR_MIXED with diag_bf16)
  // apply workspace (value type chosen by the handle precision)
  void* x = nullptr;
  void* b = nullptr;
  void* r = nullptr;
  void* t = nullptr;
};

struct Amg {
  std::vector<AmgLevel> lev;
  bool bf16 = false;         // the FP32 V-cycle reads the BF16 smoother diagonals
  int64_t ncoarse = 0;
  double* inv = nullptr;     // dense inverse of the coarsest operator (row-major)
  float* invf = nullptr;
};

struct MgrLevel {
  Csr A;                         // A_l
  int64_t n = 0, nF = 0, nC = 0;
  int32_t *label = nullptr, *node = nullptr, *comp = nullptr;
  int64_t *Fidx = nullptr, *Cidx = nullptr;   // ascending dof lists
  bool F_is_prefix = false;                  // F = [0, nF), C = [nF, n)
  double* dFinv = nullptr;       // 1 / diag(A_FF)
  float* dFinvf = nullptr;
  __nv_bfloat16* dFinvh = nullptr;   // BF16 copy (diag_bf16)
  Csr W;                         // W_p = -D_FF^-1 A_FC (nF x nC)
  Csr Wr;                        // W_r = -A_CF D_FF^-1 (nC x nF; Jacobi restriction)
  Csr Bd;                        // point-block D_FF^-1 (nF x nF; dff_block)
  bool restrict_jacobi = false, frelax_post = false, dff_block = false;
  Csr Acf;                       // A_CF (nC x nF)
  Csr cor, corkept;              // A_cor before / after G (inspection)
  Amg* famg = nullptr;           // F-relaxation AMG on A_FF
  int frelax = MGR_FRELAX_AMG_VCYCLE, frelax_sweeps = 1, global_sweeps = 0;
  int64_t nblk = 0;
  int64_t* bstart = nullptr;     // block starts (nblk + 1 entries)
  // multicolour point-block Gauss-Seidel global smoother
  bool gs = false;
  int32_t* bcolor = nullptr;     // colour of each block
  int ncolor = 0;
  int64_t* border = nullptr;     // blocks grouped by colour
  std::vector<int64_t> coff;     // colour c's blocks: border[coff[c] .. coff[c+1])
  double* binv = nullptr;        // setup layout: 16 values per block, row-major 4 x 4
  // apply layout: bdim x bdim values per block (bdim = the level's largest
  // block), row-major, so a 2x2 cell block reads 4 values instead of 16
  int bdim = 0;
  double* binvc = nullptr;
  float* binvcf = nullptr;
  __nv_bfloat16* binvch = nullptr;   // BF16 copy (diag_bf16)
  bool bf16 = false;             // FP32 apply reads the BF16 diagonals
  // ILU(1) global smoother: the factors on one pattern (ilu: strict L with
  // unit diagonal implied, plus U), split for the triangular iterations
  bool ilu1 = false;
  int ilu_solve_sweeps = 0;
  Csr ilu, Ilo, Iup;
  double* ilu_dinv = nullptr;    // 1 / u_ii
  float* ilu_dinvf = nullptr;
  void *y1 = nullptr, *y2 = nullptr, *y3 = nullptr;   // apply workspace (n each)
  // apply workspace (precision of the handle), sized n / nF / nC
  void *z = nullptr, *z2 = nullptr, *r = nullptr, *rF = nullptr, *eF = nullptr,
       *rC = nullptr, *eC = nullptr;
};

// Sliced (SELL-32) copy of the Jacobian for the FP64 products of FGMRES:
// entry k of row r at soff[r / 32] + 32 k + r % 32 of sci / sval (padded with
// column r and value 0); row lengths from the CSR row pointers.
static constexpr int64_t JSELL_MIN_NNZ = int64_t(1) << 24;
struct JacobianSell {
  int64_t* soff = nullptr;
  int32_t* sci = nullptr;
  double* sval = nullptr;
  int64_t ns_cap = 0, cap = 0;
  // the matrix the copy was made from, and whether it is current
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* val = nullptr;
  int64_t n = 0, nnz = 0;
  bool valid = false;
};

struct Handle {
  mgr_options_t opt;
  int L = 0;
  int64_t n = 0;
  std::vector<MgrLevel> lev;     // L levels
  Csr Acoarse;                   // operator of the coarsest MGR level
  Amg* camg = nullptr;
  Pool pool;
  double setup_s = 0.0;
  // mixed-precision entry/exit buffers
  float* vin32 = nullptr;
  float* zout32 = nullptr;
  // the whole preconditioner application captured once as a CUDA graph over
  // fixed buffers (FP64: gin/gout; MGR_MIXED: vin32/zout32)
  cudaGraphExec_t apply_exec = nullptr;
  long long apply_nodes = 0;     // kernel nodes per replay
  double* gin = nullptr;
  double* gout = nullptr;
  // FGMRES workspace (lazily sized)
  int64_t kry_n = 0;
  int kry_m = 0;
  double* V = nullptr;           // (m+1) x n
  void* Z = nullptr;             // m x n (FP64, or FP32 under MGR_MIXED)
  double* w = nullptr;
  double* r = nullptr;
  double* part = nullptr;        // partial dot products
  double* hcol = nullptr;        // device Hessenberg column scratch
  double* hred = nullptr;
  double* yv = nullptr;
  unsigned* ticket = nullptr;    // arrival counter of the Gram-Schmidt steps (0 between launches)
  double* gram = nullptr;        // device [m/2 + 2]: V_2k . V_(2k+1) of the current cycle
  // sliced copy of the Jacobian for fgmres_solve's products (from 2^24
  // non-zeros), rebuilt from the solve's matrix at the start of every solve
  JacobianSell jsell;
  int* derr = nullptr;           // device error word
  // the F-relaxation AMG built concurrently with the rest of the setup owns
  // its allocations here (second stream) and reports through derr2
  Pool pool2;
  int* derr2 = nullptr;
};

// ----------------------------------------------------------------------------
// Setup entry points (setup.cu)
// ----------------------------------------------------------------------------
int scan_exclusive(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, Pool& tmp);
int build_mgr_hierarchy(Handle* h, const mgr_matrix_t* A, cudaStream_t s);
int build_amg(Handle* h, Pool& P, int* derr, const Csr& A, bool own_input, const int32_t* comp,
              int slot, Amg** out, cudaStream_t s);
int to_fp32(Handle* h, cudaStream_t s);
int build_row_patterns(Pool& P, Csr& A, cudaStream_t s);
// (Re)build h's sliced copy of A (nnz >= JSELL_MIN_NNZ; synchronises s):
// 1 when built, 0 when A is below the size, < 0 on an error
int jacobian_sell_refresh(Handle* h, const mgr_matrix_t* A, cudaStream_t s);
// y = A x (res: y = b - A x), over h's sliced copy when `sell`, else the CSR
void jacobian_product(Handle* h, const mgr_matrix_t* A, bool sell, const double* x, double* y,
                      const double* b, bool res, cudaStream_t s);

// ----------------------------------------------------------------------------
// Apply entry points (apply.cu)
// ----------------------------------------------------------------------------
int alloc_apply_workspace(Handle* h, cudaStream_t s);
int apply_mgr(Handle* h, const double* v, double* z, cudaStream_t s);
int apply_mgr32(Handle* h, const float* v, float* z, cudaStream_t s);
int apply_mgr_mixed_into(Handle* h, const double* v, float* z, cudaStream_t s);
int capture_apply_graph(Handle* h);
int launch_apply_fixed(Handle* h, cudaStream_t s);
int spmv_lanes(int64_t nnz, int64_t nr);   // lanes per row of the CSR product
int setup_one(const mgr_matrix_t* A, const mgr_options_t* o, cudaStream_t s, Handle** out);
int fgmres_run(Handle* h, const mgr_matrix_t* A, const double* b, double* x,
               const fgmres_options_t* o, fgmres_info_t* info, cudaStream_t s);
int apply_vcycle64(Handle* h, Amg* g, const double* b, double* x, cudaStream_t s);
// V-cycle with a caller-provided workspace of vcycle_ws_bytes() bytes
size_t vcycle_ws_bytes(Handle* h, Amg* g);
int apply_vcycle64_ws(Handle* h, Amg* g, const double* b, double* x, void* ws, cudaStream_t s);
// generic CSR SpMV (FP64): y = A x
void spmv64(const int64_t* rp, const int32_t* ci, const double* v, int64_t nr,
            int64_t nnz, const double* x, double* y, cudaStream_t s);
void spmv64_x32(const int64_t* rp, const int32_t* ci, const double* v, int64_t nr,
                int64_t nnz, const float* x, double* y, cudaStream_t s);
void residual64(const int64_t* rp, const int32_t* ci, const double* v, int64_t nr,
                int64_t nnz, const double* b, const double* x, double* r, cudaStream_t s);

// ----------------------------------------------------------------------------
// Lockstep batch (many systems, one launch per phase; krylov.cu, batched.cu)
// ----------------------------------------------------------------------------
static constexpr int LS_H = 64;   // Hessenberg column stride per system (m <= 60)

struct LsSys {                     // device descriptor of one system
  int64_t n = 0;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* val = nullptr;
  const double* b = nullptr;
  double *x = nullptr, *V = nullptr, *w = nullptr, *r = nullptr;
  void* Z = nullptr;
  float *vin32 = nullptr, *zout32 = nullptr;
  double *gin = nullptr, *gout = nullptr;
  int64_t blk0 = 0;                // first chunk block of this system
  int32_t nb = 0;                  // its chunk blocks
  int32_t ortho = 0;               // this solve's orthogonalisation (MGR_ORTHO_MGS or _CGS2)
  const int64_t* soff = nullptr;   // sliced copy of A (null: the products read the CSR)
  const int32_t* sci = nullptr;
  const double* sval = nullptr;
};

struct Lockstep {
  int nsys = 0;
  bool mixed = false;
  cudaGraphExec_t exec = nullptr;   // one conditional branch per system
  long long graph_nodes = 0;
  std::vector<long long> body_kernels;
  int* flag = nullptr;              // device [nsys]: branch / phase participation
  unsigned long long* cond = nullptr;
  Pool pool;                        // the plan's own device memory
  // per-solve plan (sized at the first solve)
  int m = 0;
  LsSys* dsys = nullptr;            // device [nsys]
  int* jcur = nullptr;              // device [nsys]
  int32_t* blk_sys = nullptr;       // device [total chunk blocks]
  int64_t nblk = 0;
  int64_t* roff = nullptr;          // device [nsys + 1] row offsets of all systems
  int64_t nrows = 0;
  std::vector<int> gl;              // lanes per row of each SpMV group
  std::vector<int*> gsys;           // device: the systems of each group
  std::vector<int64_t*> groff;      // device: row offsets within each group
  std::vector<int64_t> grows;
  std::vector<int> gcnt;
  std::vector<int> lanes, nb;       // per system: lanes per row, chunk blocks
  double *Hc = nullptr, *Yv = nullptr, *red = nullptr, *part = nullptr;
  unsigned* tickets = nullptr;      // device [nsys]: modified Gram-Schmidt arrival counters
  double* gram = nullptr;           // device [nsys * LS_H]: each system's V_2k . V_(2k+1)
  int mgs_gmax = 1;                 // the largest system's modified Gram-Schmidt grid
  std::vector<int> ortho;           // this solve's resolved orthogonalisation per system
  bool any_sell = false;            // some system's products read its sliced copy
  int tune_j = 0;                   // the autotuner's iteration within a cycle
  double* hpin = nullptr;           // pinned host: Hc, red mirrors
  int* ipin = nullptr;              // pinned host: flag, jcur
  ~Lockstep();
};
int lockstep_alloc(Lockstep* L, Handle** hs, const mgr_matrix_t* A, cudaStream_t s);
// The orthogonalisation a solve of n unknowns uses for the option value o
// (MGR_ORTHO_AUTO: modified Gram-Schmidt from 2^20 unknowns), or -1 for an
// unknown value.
static constexpr int64_t MGS_AUTO_MIN_N = int64_t(1) << 20;
inline int resolve_ortho(int o, int64_t n) {
  if (o == MGR_ORTHO_AUTO) return n >= MGS_AUTO_MIN_N ? MGR_ORTHO_MGS : MGR_ORTHO_CGS2;
  return (o == MGR_ORTHO_MGS || o == MGR_ORTHO_CGS2) ? o : -1;
}
int lockstep_tune_round(Lockstep* L, cudaStream_t s);
int lockstep_tune_prepare(Lockstep* L, Handle** hs, const mgr_matrix_t* A, int m, int ortho, int j,
                          cudaStream_t s);
int krylov_tune_iteration(Handle* h, const mgr_matrix_t* A, int m, int ortho, int j, cudaStream_t s);
int fgmres_lockstep(Lockstep* L, Handle** hs, const mgr_matrix_t* A, const double* const* b,
                    double* const* x, const fgmres_options_t* o, fgmres_info_t* info,
                    cudaStream_t s);
int ensure_krylov_ws(Handle* h, int m);

// ----------------------------------------------------------------------------
// Small device helpers
// ----------------------------------------------------------------------------
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  // SplitMix64 (Steele, Lea, Flood 2014): one step from state x.
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

inline unsigned grid_for(int64_t work, int per_block, int cap = 152 * 32) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// Setup phase trace: with the environment variable MGR_TRACE set, phase
// boundaries synchronise the stream and print the elapsed wall time (ms) to
// stderr.  Off by default (no synchronisation added).
struct Trace {
  bool on = false;
  cudaStream_t s = nullptr;
  double t0 = 0.0, last = 0.0;
  void start(cudaStream_t st);
  void mark(const char* what, int a = -1, int b = -1);
};
extern thread_local Trace g_trace;   // per host thread (batched workers)

template <class T>
inline int read_back(T* host, const T* dev, cudaStream_t s) {
  MGR_TRY_CUDA(cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
  MGR_TRY_CUDA(cudaStreamSynchronize(s));
  return MGR_SUCCESS;
}

}  // namespace mgr
