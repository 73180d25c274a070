// Flexible GMRES (Sec. 4: right preconditioning A M^-1 y = b, x = M^-1 y; the
// flexible form keeps the preconditioned vectors z_j = M^-1 v_j so that the
// mixed-precision preconditioner may vary between iterations).  FP64 Arnoldi
// with classical Gram-Schmidt applied twice; Givens rotations and the
// (m+1) x m least-squares problem on the host (a few hundred flops); the
// true residual is recomputed in FP64 on the device at every restart.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <vector>

#include "mgr_internal.cuh"

namespace mgr {

static constexpr unsigned FULL = 0xffffffffu;
static constexpr int KB = 256;          // threads per block
static constexpr int KGRID = 152 * 2;   // blocks of the multi-vector kernels

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

// part[blk * nv + i] = sum over this block's chunk of V_i . w (nv <= 64):
// each warp reduces its partial for vector i into shared memory, one block
// barrier at the end, then a fixed-order sum over the warps.
__global__ void __launch_bounds__(KB) k_mdot(const double* __restrict__ V, int64_t ld, int nv,
                                             const double* __restrict__ w, int64_t n,
                                             double* __restrict__ part) {
  __shared__ double sh[KB / 32][64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(n, b0 + chunk);
  for (int i = 0; i < nv; i++) {
    const double* vi = V + (int64_t)i * ld;
    double acc = 0.0;
    for (int64_t t = b0 + threadIdx.x; t < b1; t += blockDim.x) acc += vi[t] * w[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) sh[wid][i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < KB / 32; q++) s += sh[q][i];
    part[(int64_t)blockIdx.x * nv + i] = s;
  }
}

// h[i] (+)= sum_blk part[blk * nv + i]  (fixed order: deterministic)
__global__ void k_mdot_final(const double* __restrict__ part, int nblk, int nv,
                             double* __restrict__ h, int accumulate) {
  __shared__ double sh[32];
  for (int i = 0; i < nv; i++) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[(int64_t)b * nv + i];
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) h[i] = accumulate ? h[i] + s : s;
  }
}

// w -= sum_i h[i] V_i
__global__ void __launch_bounds__(KB) k_mupdate(const double* __restrict__ V, int64_t ld, int nv,
                                                const double* __restrict__ h, double* __restrict__ w,
                                                int64_t n) {
  __shared__ double hs[64];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[t];
    for (int i = 0; i < nv; i++) acc -= hs[i] * V[(int64_t)i * ld + t];
    w[t] = acc;
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
    for (int i = 0; i < nv; i++) acc += ys[i] * (double)Zb[(int64_t)i * ld + t];
    x[t] = acc;
  }
}

// out = a / sqrt(nrm2[0])  (nrm2 on the device); if nrm2 == 0 copy a
__global__ void k_scale_by_norm(const double* __restrict__ a, const double* __restrict__ nrm2,
                                double* __restrict__ out, int64_t n) {
  const double s = nrm2[0];
  const double f = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = a[t] * f;
}

__global__ void k_sqrt_inplace(double* p) { p[0] = sqrt(p[0]); }

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
  h->part = P.get<double>((int64_t)KGRID * (m + 2));
  h->hcol = P.get<double>(m + 2);
  h->hred = P.get<double>(4);
  h->yv = P.get<double>(m + 2);
  if (P.err) return P.err;
  if (!h->hpinned) MGR_TRY_CUDA(cudaMallocHost(&h->hpinned, sizeof(double) * 72));  // m <= 60
  (void)s;
  return MGR_SUCCESS;
}

// dst[0..nv) = V[0..nv)^T w, computed twice-reduced (fixed order)
static void mdot(Handle* h, const double* V, int64_t ld, int nv, const double* w, int64_t n,
                 double* dst, int accumulate, cudaStream_t s) {
  MGR_LAUNCH k_mdot<<<KGRID, KB, 0, s>>>(V, ld, nv, w, n, h->part);
  MGR_LAUNCH k_mdot_final<<<1, KB, 0, s>>>(h->part, KGRID, nv, dst, accumulate);
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
  double* hp = h->hpinned;
  cudaEvent_t e0, e1;
  MGR_TRY_CUDA(cudaEventCreate(&e0));
  MGR_TRY_CUDA(cudaEventCreate(&e1));
  MGR_TRY_CUDA(cudaEventRecord(e0, s));

  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m);
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
      mdot(h, h->r, n, 1, h->r, n, h->hred, 0, s);
      MGR_LAUNCH k_scale_by_norm<<<grid_for(n, KB), KB, 0, s>>>(h->r, h->hred, h->V, n);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int jend = 0;
      bool stop = false;
      for (int j = 0; j < m && iters < maxit; j++) {
        double* vj = h->V + (int64_t)j * n;
        double* vnext = h->V + (int64_t)(j + 1) * n;
        // z_j = M^-1 v_j ; w = A z_j
        if (mixed) {
          float* zj = (float*)h->Z + (int64_t)j * n;
          MGR_TRY(apply_mgr_mixed_into(h, vj, zj, s));
          spmv64_x32(A->row_ptr, A->col_idx, A->val, n, A->nnz, zj, h->w, s);
        } else {
          double* zj = (double*)h->Z + (int64_t)j * n;
          MGR_TRY(apply_mgr(h, vj, zj, s));
          spmv64(A->row_ptr, A->col_idx, A->val, n, A->nnz, zj, h->w, s);
        }
        // classical Gram-Schmidt, twice
        mdot(h, h->V, n, j + 1, h->w, n, h->hcol, 0, s);
        MGR_LAUNCH k_mupdate<<<KGRID, KB, 0, s>>>(h->V, n, j + 1, h->hcol, h->w, n);
        mdot(h, h->V, n, j + 1, h->w, n, h->yv, 0, s);
        MGR_LAUNCH k_mupdate<<<KGRID, KB, 0, s>>>(h->V, n, j + 1, h->yv, h->w, n);
        MGR_LAUNCH k_mdot_final<<<1, 32, 0, s>>>(h->yv, 1, j + 1, h->hcol, 1);   // h += h2
        mdot(h, h->w, n, 1, h->w, n, h->hcol + j + 1, 0, s);
        MGR_LAUNCH k_scale_by_norm<<<grid_for(n, KB), KB, 0, s>>>(h->w, h->hcol + j + 1, vnext, n);
        MGR_LAUNCH k_sqrt_inplace<<<1, 1, 0, s>>>(h->hcol + j + 1);
        MGR_TRY_CUDA(cudaMemcpyAsync(hp, h->hcol, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
        MGR_TRY_CUDA(cudaStreamSynchronize(s));
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
      mdot(h, h->r, n, 1, h->r, n, h->hred, 0, s);
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
  MGR_TRY_CUDA(cudaEventRecord(e1, s));
  MGR_TRY_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
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
