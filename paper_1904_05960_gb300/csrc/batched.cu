// Batched ensemble: many independent Jacobians of uneven size solved together.
//
// Each system keeps exactly the hierarchy mgr_setup builds for it alone and
// the FGMRES iteration fgmres_solve runs for it alone (own Krylov basis, own
// convergence test), so every system's result equals its single-system
// result.  What batching adds is concurrency: a pool of native host workers,
// each with its own CUDA stream, takes systems largest first, so the GPU runs
// several systems' captured preconditioner graphs, Jacobian products and
// Gram-Schmidt kernels at once; small systems, whose kernels are too short
// to fill the GPU, overlap with large ones.
//
// The lockstep schedule instead advances every system one FGMRES iteration
// per round with one launch per phase for all systems: the preconditioner
// applications as one CUDA graph in which each system's captured application
// is the body of a conditional node (a kernel at the graph's head switches the
// branches of finished systems off), the Jacobian products as one row-binned
// launch per lanes-per-row group, the Gram-Schmidt passes over all systems'
// chunk blocks, and one readback of all Hessenberg columns (krylov.cu).
//
// The schedule autotuner times one round of every system's preconditioner
// application with 1, 2, 4, 8 and 16 workers and with the lockstep graph,
// and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "mgr_internal.cuh"

namespace mgr {

static constexpr int BATCH_MAX_WORKERS = 16;
static constexpr uint32_t BATCH_MAGIC = 0x4d475242u;

struct Batch {
  uint32_t magic = BATCH_MAGIC;
  int nsys = 0;
  int workers = 1;                    // chosen worker count (-1: lockstep)
  Lockstep* ls = nullptr;             // lockstep plan (when built)
  std::vector<Handle*> sys;
  std::vector<int> order;             // systems by decreasing size
  std::vector<cudaStream_t> streams;  // one per worker (BATCH_MAX_WORKERS)
  std::vector<int> tune_workers;      // autotuner: worker counts timed
  std::vector<double> tune_ms;        //   and their round times
  double setup_s = 0.0;
};

// Runs f(system, stream) for every system on `workers` host threads, each
// with its own stream, systems taken in `order`.  Returns the first negative
// status, else the largest non-negative one.
template <class F>
static int run_workers(Batch* B, int workers, F&& f) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<int> next{0};
  std::atomic<int> err{0};
  std::atomic<int> worst{0};
  auto body = [&](int w) {
    cudaSetDevice(dev);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= B->nsys) break;
      const int i = B->order[k];
      const int rc = f(i, B->streams[w]);
      if (rc < 0) {
        int z = 0;
        err.compare_exchange_strong(z, rc);
      } else {
        int cur = worst.load();
        while (rc > cur && !worst.compare_exchange_weak(cur, rc)) {
        }
      }
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < workers; w++) th.emplace_back(body, w);
  body(0);
  for (auto& t : th) t.join();
  return err.load() ? err.load() : worst.load();
}

// Work on the worker streams follows the caller's earlier work on `caller`
// (and, through end_on, the caller's later work follows the batch).
static int begin_on(Batch* B, cudaStream_t caller) {
  cudaEvent_t ev;
  MGR_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  MGR_TRY_CUDA(cudaEventRecord(ev, caller));
  for (cudaStream_t ws : B->streams) MGR_TRY_CUDA(cudaStreamWaitEvent(ws, ev, 0));
  cudaEventDestroy(ev);
  return MGR_SUCCESS;
}
static int end_on(Batch* B, cudaStream_t caller) {
  for (cudaStream_t ws : B->streams) {
    cudaEvent_t ev;
    MGR_TRY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    MGR_TRY_CUDA(cudaEventRecord(ev, ws));
    MGR_TRY_CUDA(cudaStreamWaitEvent(caller, ev, 0));
    cudaEventDestroy(ev);
  }
  return MGR_SUCCESS;
}

// The lockstep graph: a head kernel setting each system's branch condition
// from its flag, then one conditional node per system whose body is that
// system's captured preconditioner application (over its fixed buffers).
__global__ void k_set_branches(const unsigned long long* __restrict__ cond,
                               const int* __restrict__ flag, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) cudaGraphSetConditional(cond[i], flag[i] ? 1u : 0u);
}

static int build_lockstep(Batch* B, const mgr_matrix_t* A, cudaStream_t s) {
  const int ns = B->nsys;
  for (Handle* h : B->sys)
    if (h->opt.precision != B->sys[0]->opt.precision) return MGR_ERR_INVALID_ARG;
  Lockstep* L = new (std::nothrow) Lockstep();
  if (!L) return MGR_ERR_OOM;
  B->ls = L;
  L->nsys = ns;
  L->mixed = B->sys[0]->opt.precision == MGR_MIXED;
  L->pool.s = s;
  L->flag = L->pool.get<int>(ns);
  L->cond = L->pool.get<unsigned long long>(ns);
  if (L->pool.err) return L->pool.err;
  MGR_TRY(lockstep_alloc(L, B->sys.data(), A, s));
  cudaGraph_t g = nullptr;
  MGR_TRY_CUDA(cudaGraphCreate(&g, 0));
  int rc = MGR_SUCCESS;
  std::vector<cudaGraphConditionalHandle> hc(ns);
  for (int i = 0; i < ns && !rc; i++)
    if (cudaGraphConditionalHandleCreate(&hc[i], g, 0, cudaGraphCondAssignDefault) != cudaSuccess)
      rc = MGR_ERR_CUDA;
  cudaGraphNode_t head = nullptr;
  if (!rc) {
    if (cudaMemcpyAsync(L->cond, hc.data(), sizeof(unsigned long long) * ns, cudaMemcpyHostToDevice,
                        s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      rc = MGR_ERR_CUDA;
  }
  if (!rc) {
    cudaKernelNodeParams kp = {};
    int n = ns;
    void* args[] = {&L->cond, &L->flag, &n};
    kp.func = (void*)k_set_branches;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    if (cudaGraphAddKernelNode(&head, g, nullptr, 0, &kp) != cudaSuccess) rc = MGR_ERR_CUDA;
  }
  L->body_kernels.assign(ns, 0);
  cudaStream_t cs = nullptr;
  if (!rc && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rc = MGR_ERR_CUDA;
  for (int i = 0; i < ns && !rc; i++) {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc[i];
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t cn = nullptr;
    if (cudaGraphAddNode(&cn, g, &head, nullptr, 1, &np) != cudaSuccess) {
      rc = MGR_ERR_CUDA;
      break;
    }
    if (cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = MGR_ERR_CUDA;
      break;
    }
    const long long before = t_captured;
    t_capturing++;
    const int rb = launch_apply_fixed(B->sys[i], cs);
    t_capturing--;
    L->body_kernels[i] = t_captured - before;
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(cs, &out) != cudaSuccess || rb != MGR_SUCCESS) rc = MGR_ERR_CUDA;
    L->graph_nodes += L->body_kernels[i];
  }
  if (cs) cudaStreamDestroy(cs);
  if (!rc && cudaGraphInstantiate(&L->exec, g, 0) != cudaSuccess) rc = MGR_ERR_CUDA;
  cudaGraphDestroy(g);
  (void)cudaGetLastError();
  return rc;
}

// Schedule autotuner: time one round -- one FGMRES iteration (preconditioner
// application, Jacobian product, the default Gram-Schmidt at iteration TUNE_J
// of a cycle) of every system -- for each worker count and for the lockstep
// graph, and keep the fastest.
static constexpr int TUNE_M = 50;
// the round timed is iteration TUNE_J of a cycle (half the default restart),
// so that the Gram-Schmidt work of an average iteration is in it
static constexpr int TUNE_J = 24;
static constexpr double LOCKSTEP_MARGIN = 0.8;
static int autotune_workers(Batch* B, const mgr_matrix_t* A, cudaStream_t caller) {
  MGR_TRY_CUDA(cudaStreamSynchronize(caller));
  const int counts[5] = {1, 2, 4, 8, 16};
  double best = 1e300;
  B->tune_workers.clear();
  B->tune_ms.clear();
  for (int c = 0; c < 5; c++) {
    const int w = std::min(counts[c], std::min(B->nsys, BATCH_MAX_WORKERS));
    if (!B->tune_workers.empty() && w == B->tune_workers.back()) continue;
    double t = 0.0;
    for (int rep = 0; rep < 2; rep++) {   // the first round warms up
      MGR_TRY_CUDA(cudaDeviceSynchronize());
      const auto t0 = std::chrono::steady_clock::now();
      const int rc = run_workers(B, w, [&](int i, cudaStream_t s) {
        MGR_TRY(krylov_tune_iteration(B->sys[i], &A[i], TUNE_M, MGR_ORTHO_AUTO, TUNE_J, s));
        MGR_TRY_CUDA(cudaStreamSynchronize(s));
        return MGR_SUCCESS;
      });
      if (rc < 0) return rc;
      t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    B->tune_workers.push_back(w);
    B->tune_ms.push_back(t);
    if (t < best) {
      best = t;
      B->workers = w;
    }
  }
  if (B->ls && B->ls->exec) {
    MGR_TRY(lockstep_tune_prepare(B->ls, B->sys.data(), A, TUNE_M, MGR_ORTHO_AUTO, TUNE_J, caller));
    double t = 0.0;
    for (int rep = 0; rep < 2; rep++) {
      MGR_TRY_CUDA(cudaDeviceSynchronize());
      const auto t0 = std::chrono::steady_clock::now();
      MGR_TRY(lockstep_tune_round(B->ls, caller));
      t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    B->tune_workers.push_back(-1);
    B->tune_ms.push_back(t);
    // a round with every system active flatters the lockstep schedule: its
    // rounds keep their phase structure while the systems finish one by one,
    // where the workers move on to the next system (measured on the
    // 64-system ensemble: the lockstep round 10% faster than 8 workers', the
    // whole solve 8% slower), so it must win the round by more than that
    if (t < LOCKSTEP_MARGIN * best) {
      best = t;
      B->workers = -1;
    }
  }
  return MGR_SUCCESS;
}

}  // namespace mgr

using namespace mgr;

extern "C" {

int mgr_setup_batched(int nsys, const mgr_matrix_t* A, const mgr_options_t* o, int workers,
                      void* stream, mgr_batch_t* out) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  if (!out) return MGR_ERR_INVALID_ARG;
  *out = nullptr;
  if (nsys <= 0 || !A || !o || workers > BATCH_MAX_WORKERS || workers < -1) return MGR_ERR_INVALID_ARG;
  Batch* B = new (std::nothrow) Batch();
  if (!B) return MGR_ERR_OOM;
  B->nsys = nsys;
  B->sys.assign(nsys, nullptr);
  B->order.resize(nsys);
  std::iota(B->order.begin(), B->order.end(), 0);
  std::stable_sort(B->order.begin(), B->order.end(),
                   [&](int a, int b) { return A[a].nnz > A[b].nnz; });
  B->streams.assign(BATCH_MAX_WORKERS, nullptr);
  cudaStream_t caller = (cudaStream_t)stream;
  int rc = MGR_SUCCESS;
  for (auto& ws : B->streams)
    if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) rc = MGR_ERR_CUDA;
  const auto t0 = std::chrono::steady_clock::now();
  if (!rc) rc = begin_on(B, caller);
  const int setup_workers = std::min(nsys, workers > 0 ? workers : BATCH_MAX_WORKERS);
  if (!rc)
    rc = run_workers(B, setup_workers, [&](int i, cudaStream_t s) {
      (void)cudaGetLastError();
      return setup_one(&A[i], o, s, &B->sys[i]);
    });
  if (rc >= 0) rc = end_on(B, caller);
  if (rc >= 0 && cudaStreamSynchronize(caller) != cudaSuccess) rc = MGR_ERR_CUDA;
  B->setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rc >= 0 && workers <= 0) {
    rc = build_lockstep(B, A, caller);
    if (rc < 0 && workers == 0) {   // the worker schedules remain
      delete B->ls;
      B->ls = nullptr;
      rc = MGR_SUCCESS;
    }
  }
  if (rc >= 0) {
    if (workers > 0) B->workers = std::min(workers, nsys);
    else if (workers < 0) B->workers = -1;
    else rc = autotune_workers(B, A, caller);
  }
  if (rc < 0) {
    mgr_destroy_batched(reinterpret_cast<mgr_batch_t>(B));
    return rc;
  }
  *out = reinterpret_cast<mgr_batch_t>(B);
  return MGR_SUCCESS;
}

int fgmres_solve_batched(mgr_batch_t bh, const mgr_matrix_t* A, const double* const* b,
                         double* const* x, const fgmres_options_t* o, fgmres_info_t* info,
                         void* stream) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  Batch* B = reinterpret_cast<Batch*>(bh);
  if (!B || B->magic != BATCH_MAGIC || !A || !b || !x || !o) return MGR_ERR_INVALID_ARG;
  for (int i = 0; i < B->nsys; i++)
    if (A[i].n != B->sys[i]->n || !b[i] || !x[i]) return MGR_ERR_INVALID_ARG;
  cudaStream_t caller = (cudaStream_t)stream;
  if (B->workers < 0) {
    for (Handle* h : B->sys) h->pool.s = caller;
    int rc = fgmres_lockstep(B->ls, B->sys.data(), A, b, x, o, info, caller);
    if (rc >= 0 && cudaStreamSynchronize(caller) != cudaSuccess) rc = MGR_ERR_CUDA;
    return rc;
  }
  MGR_TRY(begin_on(B, caller));
  int rc = run_workers(B, B->workers, [&](int i, cudaStream_t s) {
    (void)cudaGetLastError();
    Handle* h = B->sys[i];
    h->pool.s = s;   // Krylov workspace is allocated on the stream that uses it
    return fgmres_run(h, &A[i], b[i], x[i], o, info ? &info[i] : nullptr, s);
  });
  const int rc2 = end_on(B, caller);
  if (rc >= 0 && rc2 < 0) rc = rc2;
  if (rc >= 0 && cudaStreamSynchronize(caller) != cudaSuccess) rc = MGR_ERR_CUDA;
  return rc;
}

int mgr_batch_info(mgr_batch_t bh, int* workers, double* setup_s, int* tune_workers,
                   double* tune_ms) {
  Batch* B = reinterpret_cast<Batch*>(bh);
  if (!B || B->magic != BATCH_MAGIC) return MGR_ERR_INVALID_ARG;
  if (workers) *workers = B->workers;
  if (setup_s) *setup_s = B->setup_s;
  for (int c = 0; c < 6; c++) {
    const bool have = c < (int)B->tune_ms.size();
    if (tune_workers) tune_workers[c] = have ? B->tune_workers[c] : 0;
    if (tune_ms) tune_ms[c] = have ? B->tune_ms[c] : -1.0;
  }
  return MGR_SUCCESS;
}

int mgr_batch_handle(mgr_batch_t bh, int i, mgr_handle_t* out) {
  Batch* B = reinterpret_cast<Batch*>(bh);
  if (!B || B->magic != BATCH_MAGIC || !out || i < 0 || i >= B->nsys) return MGR_ERR_INVALID_ARG;
  *out = reinterpret_cast<mgr_handle_t>(B->sys[i]);
  return MGR_SUCCESS;
}

int mgr_destroy_batched(mgr_batch_t bh) {
  Batch* B = reinterpret_cast<Batch*>(bh);
  if (!B || B->magic != BATCH_MAGIC) return MGR_ERR_INVALID_ARG;
  for (cudaStream_t ws : B->streams)
    if (ws) cudaStreamSynchronize(ws);
  if (B->ls) {
    cudaDeviceSynchronize();
    delete B->ls;
    B->ls = nullptr;
  }
  for (Handle* h : B->sys)
    if (h) mgr_destroy(reinterpret_cast<mgr_handle_t>(h));
  for (cudaStream_t ws : B->streams)
    if (ws) cudaStreamDestroy(ws);
  B->magic = 0;
  delete B;
  return MGR_SUCCESS;
}

}  // extern "C"
