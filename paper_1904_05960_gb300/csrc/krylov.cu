// Flexible GMRES (Sec. 4: right preconditioning A M^-1 y = b, x = M^-1 y; the
// flexible form keeps the preconditioned vectors z_j = M^-1 v_j so that the
// mixed-precision preconditioner may vary between iterations).  FP64 Arnoldi
// with classical Gram-Schmidt applied twice; Givens rotations and the
// (m+1) x m least-squares problem on the host (a few hundred flops); the
// true residual is recomputed in FP64 on the device at every restart.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <utility>
#include <vector>

#include "mgr_internal.cuh"

namespace mgr {

static constexpr unsigned FULL = 0xffffffffu;
static constexpr int KB = 256;          // threads per block
static constexpr int KGRID = 152 * 6;   // blocks of the multi-vector kernels

__device__ inline double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  }
  __syncthreads();
  return s;
}

// Multi-vector dot products, part[blk * nv + i] = this block's share of
// V_i . w (nv <= 64), in tiles of 16 vectors: each thread forms its partials
// over MD_EPT elements (w kept in registers), stages them in shared memory, and
// each warp then reduces whole vectors in a fixed order.  With UPDATE the block
// first replaces its slice of w by w - sum_i h[i] V_i (classical Gram-Schmidt
// update) and takes the dots with the updated w while V's slice is still in
// cache, so the update and the next projection cost one pass.
static constexpr int MD_EPT = 8;
template <bool UPDATE>
__global__ void __launch_bounds__(KB) k_mdot(const double* __restrict__ V, int64_t ld, int nv,
                                             double* __restrict__ w, int64_t n,
                                             double* __restrict__ part,
                                             const double* __restrict__ h) {
  __shared__ double sh[16][KB];
  __shared__ double hs[64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * (KB * MD_EPT) + threadIdx.x;
  double wr[MD_EPT];
#pragma unroll
  for (int e = 0; e < MD_EPT; e++) {
    const int64_t t = base + (int64_t)e * KB;
    wr[e] = (t < n) ? w[t] : 0.0;
  }
  if (UPDATE) {
    for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
    __syncthreads();
    for (int i = 0; i < nv; i++) {
      const double* vi = V + (int64_t)i * ld;
      const double hi = hs[i];
#pragma unroll
      for (int e = 0; e < MD_EPT; e++) {
        const int64_t t = base + (int64_t)e * KB;
        if (t < n) wr[e] -= hi * vi[t];
      }
    }
#pragma unroll
    for (int e = 0; e < MD_EPT; e++) {
      const int64_t t = base + (int64_t)e * KB;
      if (t < n) w[t] = wr[e];
    }
  }
  for (int i0 = 0; i0 < nv; i0 += 16) {
    const int nq = min(16, nv - i0);
#pragma unroll
    for (int q = 0; q < 16; q++) {
      double acc = 0.0;
      if (q < nq) {
        const double* vi = V + (int64_t)(i0 + q) * ld;
#pragma unroll
        for (int e = 0; e < MD_EPT; e++) {
          const int64_t t = base + (int64_t)e * KB;
          if (t < n) acc += vi[t] * wr[e];
        }
      }
      sh[q][threadIdx.x] = acc;
    }
    __syncthreads();
    for (int q = wid; q < nq; q += KB / 32) {
      double s2 = 0.0;
      for (int k = lane; k < KB; k += 32) s2 += sh[q][k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(FULL, s2, o);
      if (lane == 0) part[(int64_t)blockIdx.x * nv + i0 + q] = s2;
    }
    __syncthreads();
  }
}

static inline int mdot_blocks(int64_t n) { return (int)((n + KB * MD_EPT - 1) / (KB * MD_EPT)); }

// h[i] (+)= sum_blk part[blk * nv + i]: one warp per vector, fixed order.
// With SQRT the sum is replaced by its square root (a norm from partial sums
// of squares) and rinv[0] receives 1/norm (1 if the norm is 0), so the
// scaling kernels multiply instead of dividing per element.
template <bool SQRT>
__global__ void k_mdot_final(const double* __restrict__ part, int nblk, int nv,
                             double* __restrict__ h, int accumulate, double* __restrict__ rinv) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= nv) return;
  double acc = 0.0;
#pragma unroll 4
  for (int b = lane; b < nblk; b += 32) acc += part[(int64_t)b * nv + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
  if (lane == 0) {
    if (SQRT) {
      acc = sqrt(acc);
      rinv[0] = acc > 0.0 ? 1.0 / acc : 1.0;
    }
    h[i] = accumulate ? h[i] + acc : acc;
  }
}

// w -= sum_i h[i] V_i; with NORM, also part[blk] = sum over the block of the
// updated w^2 (fixed order).
template <bool NORM>
__global__ void __launch_bounds__(KB) k_mupdate(const double* __restrict__ V, int64_t ld, int nv,
                                                const double* __restrict__ h, double* __restrict__ w,
                                                int64_t n, double* __restrict__ part) {
  __shared__ double hs[64];
  __shared__ double red[KB / 32];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  double sq = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[t];
    int i = 0;
    // eight loads issued before their multiply-adds: memory-level parallelism
    for (; i + 8 <= nv; i += 8) {
      double x[8];
#pragma unroll
      for (int q = 0; q < 8; q++) x[q] = V[(int64_t)(i + q) * ld + t];
#pragma unroll
      for (int q = 0; q < 8; q++) acc -= hs[i + q] * x[q];
    }
    for (; i < nv; i++) acc -= hs[i] * V[(int64_t)i * ld + t];
    w[t] = acc;
    if (NORM) sq += acc * acc;
  }
  if (NORM) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(FULL, sq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s2 = 0.0;
      for (int q = 0; q < KB / 32; q++) s2 += red[q];
      part[blockIdx.x] = s2;
    }
  }
}

// x += sum_i y[i] Z_i  (Z in FP64 or FP32)
template <class Z>
__global__ void __launch_bounds__(KB) k_xupdate(const Z* __restrict__ Zb, int64_t ld, int nv,
                                                const double* __restrict__ y, double* __restrict__ x,
                                                int64_t n) {
  __shared__ double ys[64];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[t];
    int i = 0;
    for (; i + 8 <= nv; i += 8) {
      double z[8];
#pragma unroll
      for (int q = 0; q < 8; q++) z[q] = (double)Zb[(int64_t)(i + q) * ld + t];
#pragma unroll
      for (int q = 0; q < 8; q++) acc += ys[i + q] * z[q];
    }
    for (; i < nv; i++) acc += ys[i] * (double)Zb[(int64_t)i * ld + t];
    x[t] = acc;
  }
}

// out = a * rinv[0] (rinv on the device, computed once by k_mdot_final)
__global__ void k_scale_by(const double* __restrict__ a, const double* __restrict__ rinv,
                           double* __restrict__ out, int64_t n) {
  const double f = rinv[0];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = a[t] * f;
}

// mixed precision: the preconditioner output z32 is stored as Z_j (FP32) and
// widened once to FP64 for the Jacobian product, in one pass
__global__ void k_widen(const float* __restrict__ z32, float* __restrict__ zj, double* __restrict__ zd,
                        int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const float v = z32[t];
    zj[t] = v;
    zd[t] = (double)v;
  }
}

__global__ void k_fill0(double* p, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    p[t] = 0.0;
}

// ---------------------------------------------------------------------------
static int ensure_krylov(Handle* h, int m, cudaStream_t s) {
  if (h->V && h->kry_m >= m && h->kry_n == h->n) return MGR_SUCCESS;
  Pool& P = h->pool;
  const int64_t n = h->n;
  h->kry_m = m;
  h->kry_n = n;
  h->V = P.get<double>((int64_t)(m + 1) * n);
  if (h->opt.precision == MGR_MIXED) h->Z = P.get<float>((int64_t)m * n);
  else h->Z = P.get<double>((int64_t)m * n);
  h->w = P.get<double>(n);
  h->r = P.get<double>(n);
  h->part = P.get<double>((int64_t)std::max<int64_t>(KGRID, mdot_blocks(n)) * (m + 2));
  h->hcol = P.get<double>(m + 2);
  h->hred = P.get<double>(4);
  h->yv = P.get<double>(m + 2);
  if (P.err) return P.err;
  (void)s;
  return MGR_SUCCESS;
}

// dst[0..nv) = V[0..nv)^T w, computed twice-reduced (fixed order)
static void mdot(Handle* h, const double* V, int64_t ld, int nv, const double* w, int64_t n,
                 double* dst, int accumulate, cudaStream_t s) {
  const int nb = mdot_blocks(n);
  MGR_LAUNCH k_mdot<false><<<nb, KB, 0, s>>>(V, ld, nv, const_cast<double*>(w), n, h->part, nullptr);
  MGR_LAUNCH k_mdot_final<false><<<(nv + 7) / 8, 256, 0, s>>>(h->part, nb, nv, dst, accumulate, nullptr);
}

// Pinned host buffers of 72 doubles (m <= 60) for the Hessenberg readbacks.
// Pinning memory costs far more than a solve step's other host work, so a
// host thread leases one on its first solve and hands it back to a free list
// when it exits (the batched solves run on short-lived worker threads); the
// buffers are never unpinned, their number is bounded by the peak number of
// threads solving at once.
static std::mutex g_pin_mu;
static std::vector<double*> g_pin_free;
struct PinLease {
  double* p = nullptr;
  ~PinLease() {
    if (!p) return;
    std::lock_guard<std::mutex> g(g_pin_mu);
    g_pin_free.push_back(p);
  }
};
static thread_local PinLease t_pin;

static int pinned_scratch(double** out) {
  if (!t_pin.p) {
    {
      std::lock_guard<std::mutex> g(g_pin_mu);
      if (!g_pin_free.empty()) {
        t_pin.p = g_pin_free.back();
        g_pin_free.pop_back();
      }
    }
    if (!t_pin.p) {
      void* q = nullptr;
      MGR_TRY_CUDA(cudaMallocHost(&q, sizeof(double) * 72));
      t_pin.p = static_cast<double*>(q);
    }
  }
  *out = t_pin.p;
  return MGR_SUCCESS;
}

int fgmres_run(Handle* h, const mgr_matrix_t* A, const double* b, double* x,
               const fgmres_options_t* o, fgmres_info_t* info, cudaStream_t s) {
  const int64_t n = h->n;
  const int m = o->restart > 0 ? o->restart : 50;
  if (m > 60) return MGR_ERR_INVALID_ARG;
  const int maxit = o->max_iter > 0 ? o->max_iter : 1000;
  const double rtol = o->rtol > 0 ? o->rtol : 1e-8;
  MGR_TRY(ensure_krylov(h, m, s));
  const bool mixed = h->opt.precision == MGR_MIXED;
  // pinned host mirror for the per-iteration readbacks, leased per host thread
  double* hp = nullptr;
  MGR_TRY(pinned_scratch(&hp));
  // events are destroyed on every return path
  struct Events {
    cudaEvent_t e[7] = {};
    ~Events() {
      for (auto& x : e)
        if (x) cudaEventDestroy(x);
    }
  } ev;
  MGR_TRY_CUDA(cudaEventCreate(&ev.e[0]));
  MGR_TRY_CUDA(cudaEventCreate(&ev.e[1]));
  cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
  MGR_TRY_CUDA(cudaEventRecord(e0, s));

  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m);
  // per-phase device times (MGR_TRACE): apply, A z, Gram-Schmidt, gaps
  const bool tr = g_trace.on || getenv("MGR_TRACE") != nullptr;
  cudaEvent_t* tev = ev.e + 2;   // 5 trace events
  double tsum[4] = {0, 0, 0, 0};
  if (tr)
    for (int q = 0; q < 5; q++) cudaEventCreate(&tev[q]);
  MGR_LAUNCH k_fill0<<<grid_for(n, KB), KB, 0, s>>>(x, n);
  // ||b||
  mdot(h, b, n, 1, b, n, h->hred, 0, s);
  MGR_TRY(read_back(hp, h->hred, s));
  const double bnorm = std::sqrt(hp[0]);
  int iters = 0, restarts = 0, status = MGR_NOT_CONVERGED;
  double relres = 1.0;
  if (info && info->res_hist && info->res_hist_cap > 0) info->res_hist[0] = 1.0;
  if (bnorm == 0.0) {
    status = MGR_SUCCESS;
    relres = 0.0;
  } else {
    // r = b (x0 = 0)
    MGR_TRY_CUDA(cudaMemcpyAsync(h->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    double beta = bnorm;
    while (iters < maxit) {
      // v_0 = r / beta
      {
        const int nb = mdot_blocks(n);
        MGR_LAUNCH k_mdot<false><<<nb, KB, 0, s>>>(h->r, n, 1, h->r, n, h->part, nullptr);
        MGR_LAUNCH k_mdot_final<true><<<1, 32, 0, s>>>(h->part, nb, 1, h->hred, 0, h->hred + 1);
        MGR_LAUNCH k_scale_by<<<grid_for(n, KB), KB, 0, s>>>(h->r, h->hred + 1, h->V, n);
      }
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int jend = 0;
      bool stop = false;
      for (int j = 0; j < m && iters < maxit; j++) {
        double* vj = h->V + (int64_t)j * n;
        double* vnext = h->V + (int64_t)(j + 1) * n;
        if (tr) cudaEventRecord(tev[0], s);
        // z_j = M^-1 v_j ; w = A z_j
        if (mixed) {
          float* zj = (float*)h->Z + (int64_t)j * n;
          MGR_TRY(apply_mgr_mixed_into(h, vj, h->zout32, s));
          MGR_LAUNCH k_widen<<<grid_for(n, KB), KB, 0, s>>>(h->zout32, zj, h->r, n);
          if (tr) cudaEventRecord(tev[1], s);
          spmv64(A->row_ptr, A->col_idx, A->val, n, A->nnz, h->r, h->w, s);
        } else {
          double* zj = (double*)h->Z + (int64_t)j * n;
          MGR_TRY(apply_mgr(h, vj, zj, s));
          if (tr) cudaEventRecord(tev[1], s);
          spmv64(A->row_ptr, A->col_idx, A->val, n, A->nnz, zj, h->w, s);
        }
        if (tr) cudaEventRecord(tev[2], s);
        // classical Gram-Schmidt, twice; the second update also forms ||w||^2
        mdot(h, h->V, n, j + 1, h->w, n, h->hcol, 0, s);                       // h1 = V^T w
        {
          const int nb = mdot_blocks(n);                                        // w -= V h1; h2 = V^T w
          MGR_LAUNCH k_mdot<true><<<nb, KB, 0, s>>>(h->V, n, j + 1, h->w, n, h->part, h->hcol);
          MGR_LAUNCH k_mdot_final<false><<<(j + 1 + 7) / 8, 256, 0, s>>>(h->part, nb, j + 1, h->yv, 0, nullptr);
        }
        MGR_LAUNCH k_mupdate<true><<<KGRID, KB, 0, s>>>(h->V, n, j + 1, h->yv, h->w, n, h->part);   // w -= V h2
        MGR_LAUNCH k_mdot_final<false><<<(j + 1 + 7) / 8, 256, 0, s>>>(h->yv, 1, j + 1, h->hcol, 1, nullptr);   // h += h2
        MGR_LAUNCH k_mdot_final<true><<<1, 32, 0, s>>>(h->part, KGRID, 1, h->hcol + j + 1, 0, h->hred + 1);     // ||w||
        MGR_LAUNCH k_scale_by<<<grid_for(n, KB), KB, 0, s>>>(h->w, h->hred + 1, vnext, n);
        if (tr) cudaEventRecord(tev[3], s);
        MGR_TRY_CUDA(cudaMemcpyAsync(hp, h->hcol, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
        MGR_TRY_CUDA(cudaStreamSynchronize(s));
        if (tr) {
          float a = 0.f, b2 = 0.f, c = 0.f;
          cudaEventElapsedTime(&a, tev[0], tev[1]);
          cudaEventElapsedTime(&b2, tev[1], tev[2]);
          cudaEventElapsedTime(&c, tev[2], tev[3]);
          tsum[0] += a;
          tsum[1] += b2;
          tsum[2] += c;
          if (j > 0) {
            float g = 0.f;
            cudaEventElapsedTime(&g, tev[4], tev[0]);   // previous iteration's end -> this start
            tsum[3] += g;
          }
          std::swap(tev[3], tev[4]);
        }
        MGR_TRY_CUDA(cudaGetLastError());
        for (int i = 0; i <= j + 1; i++) H[(size_t)i * m + j] = hp[i];
        const double hn = hp[j + 1];
        if (!std::isfinite(hn)) {
          status = MGR_ERR_BREAKDOWN;
          stop = true;
          break;
        }
        for (int i = 0; i < j; i++) {
          double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
          H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
        }
        double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
        double den = std::sqrt(a * a + c * c);
        cs[j] = den == 0.0 ? 1.0 : a / den;
        sn[j] = den == 0.0 ? 0.0 : c / den;
        H[(size_t)j * m + j] = cs[j] * a + sn[j] * c;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        iters++;
        jend = j + 1;
        if (info && info->res_hist && iters < info->res_hist_cap)
          info->res_hist[iters] = std::fabs(g[j + 1]) / bnorm;
        if (std::fabs(g[j + 1]) <= rtol * bnorm || hn == 0.0) break;
      }
      if (status == MGR_ERR_BREAKDOWN) break;
      // y = H^-1 g (upper triangular), x += Z y
      for (int i = jend - 1; i >= 0; i--) {
        double t = g[i];
        for (int k = i + 1; k < jend; k++) t -= H[(size_t)i * m + k] * y[k];
        y[i] = t / H[(size_t)i * m + i];
      }
      MGR_TRY_CUDA(cudaMemcpyAsync(h->yv, y.data(), sizeof(double) * jend, cudaMemcpyHostToDevice, s));
      if (mixed)
        MGR_LAUNCH k_xupdate<float><<<KGRID, KB, 0, s>>>((const float*)h->Z, n, jend, h->yv, x, n);
      else
        MGR_LAUNCH k_xupdate<double><<<KGRID, KB, 0, s>>>((const double*)h->Z, n, jend, h->yv, x, n);
      // true residual in FP64
      residual64(A->row_ptr, A->col_idx, A->val, n, A->nnz, b, x, h->r, s);
      mdot(h, h->r, n, 1, h->r, n, h->hred, 0, s);   // ||r||^2
      MGR_TRY(read_back(hp, h->hred, s));
      beta = std::sqrt(hp[0]);
      relres = beta / bnorm;
      if (!std::isfinite(beta)) {
        status = MGR_ERR_BREAKDOWN;
        break;
      }
      if (relres <= rtol || beta == 0.0) {
        status = MGR_SUCCESS;
        break;
      }
      (void)stop;
      restarts++;
    }
  }
  if (tr) {
    fprintf(stderr, "mgr_trace fgmres %d iters: apply %.3f ms, A*z %.3f ms, Gram-Schmidt %.3f ms, "
                    "between iterations %.3f ms (totals)\n", iters, tsum[0], tsum[1], tsum[2], tsum[3]);
  }
  MGR_TRY_CUDA(cudaEventRecord(e1, s));
  MGR_TRY_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  if (info) {
    info->iters = iters;
    info->restarts = restarts;
    info->converged = status == MGR_SUCCESS;
    info->rel_res_true = relres;
    info->setup_s = h->setup_s;
    info->solve_s = ms * 1e-3;
  }
  return status;
}

}  // namespace mgr
