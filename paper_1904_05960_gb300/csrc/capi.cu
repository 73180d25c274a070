// C ABI of the GB300 MGR library (declared in include/mgr_gb300.h).
#include <cuda_runtime.h>

#include <chrono>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "mgr_internal.cuh"

namespace mgr {
std::atomic<long long> g_launches{0};
std::atomic<long long> g_host_launches{0};
thread_local int t_capturing = 0;
thread_local long long t_captured = 0;
thread_local Trace g_trace;

static double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}
void Trace::start(cudaStream_t st) {
  on = getenv("MGR_TRACE") != nullptr;
  s = st;
  if (!on) return;
  cudaStreamSynchronize(s);
  t0 = last = now_ms();
}
void Trace::mark(const char* what, int a, int b) {
  if (!on) return;
  cudaStreamSynchronize(s);
  const double t = now_ms();
  fprintf(stderr, "mgr_trace %-28s %3d %3d  %8.3f ms  (total %8.3f)\n", what, a, b, t - last, t - t0);
  last = t;
}

__global__ void k_splitmix(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = splitmix64(in[i]);
}

static const Csr* find_csr(Handle* h, int kind, int slot, int lvl) {
  if (kind < 10) {
    if (slot < 0 || slot >= h->L) return nullptr;
    MgrLevel& L = h->lev[slot];
    switch (kind) {
      case 0: return &L.A;
      case 1: return &L.W;
      case 2: return &L.cor;
      case 3: return &L.corkept;
      case 4: return (slot + 1 < h->L) ? &h->lev[slot + 1].A : &h->Acoarse;
      case 5: return L.Wr.rp ? &L.Wr : nullptr;
      case 6: return L.Bd.rp ? &L.Bd : nullptr;
      case 7: return L.ilu.rp ? &L.ilu : nullptr;
    }
    return nullptr;
  }
  Amg* g = (slot == h->L) ? h->camg : (slot >= 0 && slot < h->L ? h->lev[slot].famg : nullptr);
  if (!g || lvl < 0 || lvl >= (int)g->lev.size()) return nullptr;
  AmgLevel& A = g->lev[lvl];
  const bool coarsened = lvl + 1 < (int)g->lev.size();
  switch (kind) {
    case 10: return &A.A;
    case 11: return coarsened ? &A.S : nullptr;
    case 12: return coarsened ? &A.P : nullptr;
    case 13: return coarsened ? &A.R : nullptr;
  }
  return nullptr;
}

static Amg* find_amg(Handle* h, int slot) {
  if (slot == h->L) return h->camg;
  if (slot >= 0 && slot < h->L) return h->lev[slot].famg;
  return nullptr;
}

}  // namespace mgr

using namespace mgr;

extern "C" {

void mgr_options_default(mgr_options_t* o, int two_phase) {
  std::memset(o, 0, sizeof(*o));
  o->num_levels = two_phase ? 2 : 1;
  o->f_label_mask[0] = 1u << 0;
  o->f_label_mask[1] = 1u << 1;
  o->frelax[0] = MGR_FRELAX_AMG_VCYCLE;
  o->frelax[1] = MGR_FRELAX_JACOBI;
  for (int l = 0; l < MGR_MAX_LEVELS; l++) o->frelax_sweeps[l] = 1;
  // restrict_jacobi, frelax_post, dff_block: 0 (memset above)
  o->nmax_drop[0] = 4;
  for (int l = 1; l < MGR_MAX_LEVELS; l++) o->nmax_drop[l] = -1;
  o->global_sweeps[0] = 0;
  o->global_sweeps[1] = two_phase ? 3 : 0;
  o->amg_theta = 0.25;
  o->amg_pmax = 4;
  o->amg_max_coarse = 160;
  o->amg_max_levels = 25;
  o->precision = MGR_FP64;
  o->seed = 0;
  o->ilu_solve_sweeps = 3;
}

void fgmres_options_default(fgmres_options_t* o) {
  o->restart = 50;
  o->max_iter = 1000;
  o->rtol = 1e-8;
  o->ortho = MGR_ORTHO_AUTO;
}

const char* mgr_error_string(int code) {
  switch (code) {
    case MGR_SUCCESS: return "success";
    case MGR_NOT_CONVERGED: return "not converged within max_iter";
    case MGR_ERR_INVALID_ARG: return "invalid argument";
    case MGR_ERR_CUDA: return "CUDA error";
    case MGR_ERR_OOM: return "out of device memory";
    case MGR_ERR_ZERO_DIAG: return "zero pivot (D_FF, smoother block or coarsest LU)";
    case MGR_ERR_BREAKDOWN: return "NaN/Inf in the Arnoldi process";
    case MGR_ERR_COARSE: return "coarsest AMG level exceeds the dense-LU cap";
  }
  return "unknown status";
}

int mgr_setup(const mgr_matrix_t* A, const mgr_options_t* o, void* stream, mgr_handle_t* out) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  if (!out) return MGR_ERR_INVALID_ARG;
  *out = nullptr;
  Handle* h = nullptr;
  const int rc = mgr::setup_one(A, o, (cudaStream_t)stream, &h);
  if (rc == MGR_SUCCESS) *out = reinterpret_cast<mgr_handle_t>(h);
  return rc;
}

}  // extern "C"

namespace mgr {
cudaMemPool_t lib_pool() {
  static constexpr int MAX_DEV = 64;
  static std::once_flag once[MAX_DEV];
  static cudaMemPool_t pools[MAX_DEV] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) {
    (void)cudaGetLastError();
    return nullptr;
  }
  std::call_once(once[dev], [dev] {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess) pools[dev] = p;
      else cudaMemPoolDestroy(p);
    }
    (void)cudaGetLastError();
  });
  return pools[dev];
}

// One system's setup (mgr_setup; also run by the batched setup's workers).
int setup_one(const mgr_matrix_t* A, const mgr_options_t* o, cudaStream_t s, Handle** out) {
  if (!A || !o || !out || A->n <= 0 || A->nnz < 0 || !A->row_ptr || !A->col_idx || !A->val ||
      !A->dof_label || !A->dof_node)
    return MGR_ERR_INVALID_ARG;
  if (o->num_levels < 0 || o->num_levels > MGR_MAX_LEVELS || o->amg_max_levels < 1 ||
      o->amg_pmax < 0 || (o->precision != MGR_FP64 && o->precision != MGR_MIXED))
    return MGR_ERR_INVALID_ARG;
  if (A->n > INT32_MAX) return MGR_ERR_INVALID_ARG;
  for (int l = 0; l < MGR_MAX_LEVELS; l++)
    if (o->global_smoother[l] < 0 || o->global_smoother[l] > 2) return MGR_ERR_INVALID_ARG;
  if (o->diag_bf16 != 0 && (o->diag_bf16 != 1 || o->precision != MGR_MIXED)) return MGR_ERR_INVALID_ARG;
  if (o->values_f16 != 0 && (o->values_f16 != 1 || o->precision != MGR_MIXED)) return MGR_ERR_INVALID_ARG;
  if (o->ilu_solve_sweeps < 0 || o->ilu_solve_sweeps > 1000) return MGR_ERR_INVALID_ARG;
  Handle* h = new (std::nothrow) Handle();
  if (!h) return MGR_ERR_OOM;
  h->opt = *o;
  h->L = o->num_levels;
  h->n = A->n;
  h->pool.s = s;
  *out = nullptr;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  int rc = MGR_SUCCESS;
  g_trace.start(s);
  h->derr = h->pool.get<int>(1);
  if (!h->derr) rc = h->pool.err;
  if (!rc && cudaMemsetAsync(h->derr, 0, sizeof(int), s) != cudaSuccess) rc = MGR_ERR_CUDA;
  if (!rc) rc = build_mgr_hierarchy(h, A, s);
  g_trace.mark("hierarchy");
  if (!rc && o->precision == MGR_MIXED) rc = to_fp32(h, s);
  if (!rc) rc = alloc_apply_workspace(h, s);
  if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = MGR_ERR_CUDA;
  g_trace.mark("fp32 copies + workspace");
  if (!rc) rc = capture_apply_graph(h);
  g_trace.mark("apply graph capture");
  cudaEventRecord(e1, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = MGR_ERR_CUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->setup_s = ms * 1e-3;
  if (rc) {
    mgr_destroy(reinterpret_cast<mgr_handle_t>(h));
    return rc;
  }
  *out = h;
  return MGR_SUCCESS;
}
}  // namespace mgr

extern "C" {

int mgr_apply(mgr_handle_t hh, const double* v, double* z, void* stream) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !v || !z) return MGR_ERR_INVALID_ARG;
  return apply_mgr(h, v, z, (cudaStream_t)stream);
}

int fgmres_solve(mgr_handle_t hh, const mgr_matrix_t* A, const double* b, double* x,
                 const fgmres_options_t* o, fgmres_info_t* info, void* stream) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !A || !b || !x || A->n != h->n) return MGR_ERR_INVALID_ARG;
  fgmres_options_t d;
  fgmres_options_default(&d);
  return fgmres_run(h, A, b, x, o ? o : &d, info, (cudaStream_t)stream);
}

int mgr_solve_host(const mgr_matrix_t* A, const double* b, double* x, const mgr_options_t* o,
                   const fgmres_options_t* fo, fgmres_info_t* info, void* stream) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  if (!A || !b || !x || !o || A->n <= 0 || A->nnz < 0 || !A->row_ptr || !A->col_idx || !A->val ||
      !A->dof_label || !A->dof_node)
    return MGR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n, nnz = A->nnz;
  Pool P;
  P.s = s;
  mgr_matrix_t D = *A;
  int64_t* rp = P.get<int64_t>(n + 1);
  int32_t* ci = P.get<int32_t>(nnz);
  double* v = P.get<double>(nnz);
  int32_t* lab = P.get<int32_t>(n);
  int32_t* nod = P.get<int32_t>(n);
  int32_t* cmp = A->dof_comp ? P.get<int32_t>(n) : nullptr;
  double* db = P.get<double>(n);
  double* dx = P.get<double>(n);
  int rc = P.err;
  auto h2d = [&](void* d, const void* hsrc, size_t bytes) {
    if (rc == MGR_SUCCESS && bytes && cudaMemcpyAsync(d, hsrc, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
      rc = MGR_ERR_CUDA;
  };
  h2d(rp, A->row_ptr, sizeof(int64_t) * (n + 1));
  h2d(ci, A->col_idx, sizeof(int32_t) * nnz);
  h2d(v, A->val, sizeof(double) * nnz);
  h2d(lab, A->dof_label, sizeof(int32_t) * n);
  h2d(nod, A->dof_node, sizeof(int32_t) * n);
  if (cmp) h2d(cmp, A->dof_comp, sizeof(int32_t) * n);
  h2d(db, b, sizeof(double) * n);
  D.row_ptr = rp;
  D.col_idx = ci;
  D.val = v;
  D.dof_label = lab;
  D.dof_node = nod;
  D.dof_comp = cmp;
  Handle* h = nullptr;
  if (rc == MGR_SUCCESS) rc = mgr::setup_one(&D, o, s, &h);
  if (rc == MGR_SUCCESS) {
    fgmres_options_t d;
    fgmres_options_default(&d);
    rc = fgmres_run(h, &D, db, dx, fo ? fo : &d, info, s);
    if ((rc == MGR_SUCCESS || rc == MGR_NOT_CONVERGED) &&
        (cudaMemcpyAsync(x, dx, sizeof(double) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
      rc = MGR_ERR_CUDA;
  }
  if (h) mgr_destroy(reinterpret_cast<mgr_handle_t>(h));
  cudaStreamSynchronize(s);
  P.free_all_async(s);
  return rc;
}

int mgr_destroy(mgr_handle_t hh) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return MGR_SUCCESS;
  cudaDeviceSynchronize();
  if (h->apply_exec) cudaGraphExecDestroy(h->apply_exec);
  for (auto& L : h->lev) delete L.famg;
  delete h->camg;
  h->pool.free_all_async();
  h->pool2.free_all_async();
  delete h;
  return MGR_SUCCESS;
}

int mgr_get_csr(mgr_handle_t hh, int kind, int slot, int lvl, int64_t* dims, int64_t* row_ptr,
                int32_t* col_idx, double* val) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !dims) return MGR_ERR_INVALID_ARG;
  const Csr* a = find_csr(h, kind, slot, lvl);
  if (!a || !a->rp) return MGR_ERR_INVALID_ARG;
  MGR_TRY_CUDA(cudaDeviceSynchronize());
  dims[0] = a->nr;
  dims[1] = a->nc;
  dims[2] = a->nnz;
  if (row_ptr) MGR_TRY_CUDA(cudaMemcpy(row_ptr, a->rp, sizeof(int64_t) * (a->nr + 1), cudaMemcpyDeviceToHost));
  if (col_idx && a->nnz) MGR_TRY_CUDA(cudaMemcpy(col_idx, a->ci, sizeof(int32_t) * a->nnz, cudaMemcpyDeviceToHost));
  if (val && a->nnz) {
    if (a->v) MGR_TRY_CUDA(cudaMemcpy(val, a->v, sizeof(double) * a->nnz, cudaMemcpyDeviceToHost));
    else for (int64_t k = 0; k < a->nnz; k++) val[k] = 1.0;   // pattern-only matrix
  }
  return MGR_SUCCESS;
}

int mgr_amg_levels(mgr_handle_t hh, int slot) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return 0;
  Amg* g = find_amg(h, slot);
  return g ? (int)g->lev.size() : 0;
}

int mgr_row_patterns(mgr_handle_t hh, int slot, int lvl) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return MGR_ERR_INVALID_ARG;
  Amg* g = find_amg(h, slot);
  if (!g || lvl < 0 || lvl >= (int)g->lev.size()) return MGR_ERR_INVALID_ARG;
  return g->lev[lvl].A.pid ? g->lev[lvl].A.npat : 0;
}

int mgr_jacobian_product(mgr_handle_t hh, const mgr_matrix_t* A, const double* x, double* y,
                         int refresh, void* stream) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !A || A->n != h->n || A->nnz < 0 || (A->n > 0 && (!A->row_ptr || !x || !y)) ||
      (A->nnz > 0 && (!A->col_idx || !A->val)) || (refresh != 0 && refresh != 1))
    return MGR_ERR_INVALID_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  const JacobianSell& J = h->jsell;
  int sv = 0;
  if (refresh) sv = jacobian_sell_refresh(h, A, s);
  else sv = J.valid && J.rp == A->row_ptr && J.ci == A->col_idx && J.val == A->val &&
            J.n == A->n && J.nnz == A->nnz;
  if (sv < 0) return sv;
  jacobian_product(h, A, sv == 1, x, y, nullptr, false, s);
  MGR_TRY_CUDA(cudaGetLastError());
  return sv;
}

int64_t mgr_get_cf(mgr_handle_t hh, int slot, int lvl, int8_t* out) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return MGR_ERR_INVALID_ARG;
  Amg* g = find_amg(h, slot);
  if (!g || lvl < 0 || lvl + 1 >= (int)g->lev.size()) return MGR_ERR_INVALID_ARG;
  const AmgLevel& L = g->lev[lvl];
  if (out) {
    MGR_TRY_CUDA(cudaDeviceSynchronize());
    MGR_TRY_CUDA(cudaMemcpy(out, L.cf, L.A.nr, cudaMemcpyDeviceToHost));
  }
  return L.A.nr;
}

int mgr_vcycle(mgr_handle_t hh, int slot, const double* b, double* x, void* stream) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !b || !x) return MGR_ERR_INVALID_ARG;
  Amg* g = find_amg(h, slot);
  if (!g) return MGR_ERR_INVALID_ARG;
  return apply_vcycle64(h, g, b, x, (cudaStream_t)stream);
}

int mgr_spmv(const mgr_matrix_t* A, const double* x, double* y, void* stream) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  if (!A || A->n < 0 || A->nnz < 0 || (A->n > 0 && (!A->row_ptr || !x || !y)) ||
      (A->nnz > 0 && (!A->col_idx || !A->val)))
    return MGR_ERR_INVALID_ARG;
  if (A->n == 0) return MGR_SUCCESS;
  spmv64(A->row_ptr, A->col_idx, A->val, A->n, A->nnz, x, y, (cudaStream_t)stream);
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

int mgr_splitmix64_device(const uint64_t* in, uint64_t* out, int64_t n, void* stream) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  if (n < 0 || (n > 0 && (!in || !out))) return MGR_ERR_INVALID_ARG;
  if (n == 0) return MGR_SUCCESS;
  MGR_LAUNCH k_splitmix<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(in, out, n);
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

int64_t mgr_launch_count(void) { return (int64_t)g_launches.load(); }

int64_t mgr_host_launch_count(void) { return (int64_t)g_host_launches.load(); }

#ifndef MGR_BUILD_ID
#define MGR_BUILD_ID "unversioned"
#endif
const char* mgr_build_id(void) { return MGR_BUILD_ID; }

int mgr_memory_usage(size_t* used, size_t* reserved) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  if (used) *used = 0;
  if (reserved) *reserved = 0;
  cudaMemPool_t mp = lib_pool();
  if (!mp) return MGR_SUCCESS;
  uint64_t u = 0, r = 0;
  MGR_TRY_CUDA(cudaMemPoolGetAttribute(mp, cudaMemPoolAttrUsedMemCurrent, &u));
  MGR_TRY_CUDA(cudaMemPoolGetAttribute(mp, cudaMemPoolAttrReservedMemCurrent, &r));
  if (used) *used = (size_t)u;
  if (reserved) *reserved = (size_t)r;
  return MGR_SUCCESS;
}

int mgr_trim_memory(size_t keep_bytes) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  cudaMemPool_t mp = lib_pool();
  if (!mp) return MGR_SUCCESS;
  MGR_TRY_CUDA(cudaDeviceSynchronize());
  MGR_TRY_CUDA(cudaMemPoolTrimTo(mp, keep_bytes));
  return MGR_SUCCESS;
}

int64_t mgr_get_block_colors(mgr_handle_t hh, int level, int32_t* out, int32_t* ncolor) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || level < 0 || level >= h->L || !h->lev[level].gs) return MGR_ERR_INVALID_ARG;
  const MgrLevel& L = h->lev[level];
  if (ncolor) *ncolor = L.ncolor;
  if (out) {
    MGR_TRY_CUDA(cudaDeviceSynchronize());
    MGR_TRY_CUDA(cudaMemcpy(out, L.bcolor, sizeof(int32_t) * L.nblk, cudaMemcpyDeviceToHost));
  }
  return L.nblk;
}

}  // extern "C"
