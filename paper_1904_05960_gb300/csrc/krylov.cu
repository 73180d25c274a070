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
// cache, so the update and the next projection cost one pass.  Block `blk`
// owns the chunk [blk * KB * MD_EPT, (blk + 1) * KB * MD_EPT); the body is
// shared by the single-system kernel and the lockstep (many-system) kernel, so
// both give the same bits.
static constexpr int MD_EPT = 8;
static constexpr int MD_CHUNK = KB * MD_EPT;
template <bool UPDATE>
__device__ __forceinline__ void mdot_body(const double* __restrict__ V, int64_t ld, int nv,
                                          double* __restrict__ w, int64_t n,
                                          double* __restrict__ part, const double* __restrict__ h,
                                          int64_t blk) {
  __shared__ double sh[16][KB];
  __shared__ double hs[64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t base = blk * MD_CHUNK + threadIdx.x;
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
      if (lane == 0) part[blk * nv + i0 + q] = s2;
    }
    __syncthreads();
  }
}

template <bool UPDATE>
__global__ void __launch_bounds__(KB) k_mdot(const double* __restrict__ V, int64_t ld, int nv,
                                             double* __restrict__ w, int64_t n,
                                             double* __restrict__ part,
                                             const double* __restrict__ h) {
  mdot_body<UPDATE>(V, ld, nv, w, n, part, h, blockIdx.x);
}

static inline int mdot_blocks(int64_t n) { return (int)((n + MD_CHUNK - 1) / MD_CHUNK); }

// h[i] (+)= sum_blk part[blk * nv + i]: one block of FIN_T threads per vector,
// each thread adding a strided share of the partials (several loads in
// flight), then a fixed reduction tree.  With SQRT the sum is replaced by its
// square root (a norm from partial sums of squares) and rinv[0] receives
// 1/norm (1 if the norm is 0), so the scaling kernels multiply instead of
// dividing per element.
static constexpr int FIN_T = 256;
template <bool SQRT>
__device__ __forceinline__ void mdot_final_block(const double* __restrict__ part, int nblk, int nv,
                                                 int i, double* __restrict__ h, int accumulate,
                                                 double* __restrict__ rinv) {
  __shared__ double red[FIN_T / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double acc = 0.0;
#pragma unroll 4
  for (int b = threadIdx.x; b < nblk; b += FIN_T) acc += part[(int64_t)b * nv + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < FIN_T / 32; q++) tot += red[q];
    if (SQRT) {
      tot = sqrt(tot);
      rinv[0] = tot > 0.0 ? 1.0 / tot : 1.0;
    }
    h[i] = accumulate ? h[i] + tot : tot;
  }
}

// launched with nv blocks of FIN_T threads
template <bool SQRT>
__global__ void __launch_bounds__(FIN_T) k_mdot_final(const double* __restrict__ part, int nblk,
                                                      int nv, double* __restrict__ h,
                                                      int accumulate, double* __restrict__ rinv) {
  mdot_final_block<SQRT>(part, nblk, nv, blockIdx.x, h, accumulate, rinv);
}

// w -= sum_i h[i] V_i over block blk's chunk (the layout of mdot_body); with
// NORM, also part[blk] = the chunk's sum of the updated w^2 in a fixed order.
template <bool NORM>
__device__ __forceinline__ void mupdate_body(const double* __restrict__ V, int64_t ld, int nv,
                                             const double* __restrict__ h, double* __restrict__ w,
                                             int64_t n, double* __restrict__ part, int64_t blk) {
  __shared__ double hs[64];
  __shared__ double red[KB / 32];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  double sq = 0.0;
  const int64_t base = blk * MD_CHUNK + threadIdx.x;
#pragma unroll 1
  for (int e = 0; e < MD_EPT; e++) {
    const int64_t t = base + (int64_t)e * KB;
    if (t >= n) break;
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
      part[blk] = s2;
    }
  }
}

template <bool NORM>
__global__ void __launch_bounds__(KB) k_mupdate(const double* __restrict__ V, int64_t ld, int nv,
                                                const double* __restrict__ h, double* __restrict__ w,
                                                int64_t n, double* __restrict__ part) {
  mupdate_body<NORM>(V, ld, nv, h, w, n, part, blockIdx.x);
}

// Modified Gram-Schmidt of iteration j, two projections per launch.  Pass p
// (p = 0 .. j/2 + 1) of iteration j:
//   w -= h[2p-2] V_(2p-2) + h[2p-1] V_(2p-1)      (p >= 1; the second term when 2p-1 <= j)
//   h[2p]   = V_2p . w                             (2p <= j)
//   h[2p+1] = V_(2p+1) . w - h[2p] g[p]            (2p+1 <= j)
//   h[j+1] = ||w||, rinv[0] = 1 / ||w|| (1 if ||w|| = 0), and for even j
//   g[j/2] = V_j . w / ||w||                       (the last pass, p = j/2 + 1)
// g[k] = V_2k . V_(2k+1) is the basis's own (rounding-level) inner product,
// formed when V_(2k+1) is: V_(2k+1) . (w - h[2k] V_2k) = V_(2k+1) . w -
// h[2k] g[k], so each projection is the one the one-at-a-time recurrence
// takes, and w is read and written once per two projections (48 bytes per
// entry instead of 64).  G = mgs_grid(n) blocks stride over KB-entry tiles,
// ascending for even p and descending for odd p, so that every pass starts
// where the one before it ended, while that end of w and the last basis
// vectors are still in L2.  Each block stores its two partial sums; the last
// block to arrive (a ticket counter that it resets) adds the partials in block
// order, so the sums do not depend on which block arrives last.  No block
// waits for another.  The body is shared by the single-system kernel and the
// lockstep (many-system) kernel.
static constexpr int MGS_GRID = 152 * 8;
__host__ __device__ inline int mgs_grid(int64_t n) {
  const int64_t t = (n + KB - 1) / KB;
  return (int)(t < 1 ? 1 : (t < MGS_GRID ? t : MGS_GRID));
}
// part holds 2 G partials: [0, G) the first sum, [G, 2G) the second
__device__ __forceinline__ void mgs_pair_body(const double* __restrict__ V, int64_t ld, int p,
                                              int j, double* __restrict__ w, int64_t n,
                                              double* __restrict__ part, double* __restrict__ h,
                                              double* __restrict__ g, double* __restrict__ rinv,
                                              unsigned* __restrict__ ticket, int G, int blk) {
  __shared__ double red[2][KB / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool fin = 2 * p > j;                   // the last pass: ||w||
  const bool upd = p > 0;
  const bool upd2 = upd && 2 * p - 1 <= j;
  // the second sum: V_(2p+1) . w, or at the last pass of an even j, V_j . w
  // (V_j = V_(2p-2), the vector the update reads)
  const bool two = fin ? (j % 2 == 0) : (2 * p + 1 <= j);
  const double ha = upd ? h[2 * p - 2] : 0.0;
  const double hb = upd2 ? h[2 * p - 1] : 0.0;
  const double* va = V + (int64_t)(upd ? 2 * p - 2 : 0) * ld;
  const double* vb = V + (int64_t)(upd2 ? 2 * p - 1 : 0) * ld;
  const double* da = V + (int64_t)(fin ? 0 : 2 * p) * ld;
  const double* db = V + (int64_t)(!fin && two ? 2 * p + 1 : 0) * ld;
  const int64_t ntile = (n + KB - 1) / KB;
  const int64_t nk = blk < ntile ? (ntile - blk + G - 1) / G : 0;
  double acc0 = 0.0, acc1 = 0.0;
#pragma unroll 4
  for (int64_t kk = 0; kk < nk; kk++) {
    const int64_t k = (p & 1) ? nk - 1 - kk : kk;
    const int64_t t = (blk + k * G) * KB + threadIdx.x;
    if (t < n) {
      double x = w[t];
      double a = 0.0;
      if (upd) {
        a = va[t];
        x -= ha * a;
        if (upd2) x -= hb * vb[t];
        w[t] = x;
      }
      if (fin) {
        acc0 += x * x;
        if (two) acc1 += a * x;
      } else {
        acc0 += da[t] * x;
        if (two) acc1 += db[t] * x;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc0 += __shfl_xor_sync(FULL, acc0, o);
    acc1 += __shfl_xor_sync(FULL, acc1, o);
  }
  if (lane == 0) {
    red[0][wid] = acc0;
    red[1][wid] = acc1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < KB / 32; q++) {
      s0 += red[0][q];
      s1 += red[1][q];
    }
    part[blk] = s0;
    part[G + blk] = s1;
    __threadfence();
    last = atomicAdd(ticket, 1u) == (unsigned)(G - 1);
  }
  __syncthreads();
  if (!last) return;
  double s0 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < G; b += KB) {
    s0 += __ldcg(part + b);
    s1 += __ldcg(part + G + b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(FULL, s0, o);
    s1 += __shfl_xor_sync(FULL, s1, o);
  }
  if (lane == 0) {
    red[0][wid] = s0;
    red[1][wid] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int q = 0; q < KB / 32; q++) {
      t0 += red[0][q];
      t1 += red[1][q];
    }
    if (!fin) {
      h[2 * p] = t0;
      if (two) h[2 * p + 1] = t1 - t0 * g[p];
    } else {
      const double nrm = sqrt(t0);
      h[j + 1] = nrm;
      rinv[0] = nrm > 0.0 ? 1.0 / nrm : 1.0;
      if (two) g[j / 2] = nrm > 0.0 ? t1 / nrm : 0.0;
    }
    *ticket = 0u;
  }
}

__global__ void __launch_bounds__(KB) k_mgs_pair(const double* __restrict__ V, int64_t ld, int p,
                                                 int j, double* __restrict__ w, int64_t n,
                                                 double* __restrict__ part, double* __restrict__ h,
                                                 double* __restrict__ g, double* __restrict__ rinv,
                                                 unsigned* __restrict__ ticket) {
  mgs_pair_body(V, ld, p, j, w, n, part, h, g, rinv, ticket, gridDim.x, blockIdx.x);
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
  h->ticket = P.get<unsigned>(1);
  h->gram = P.get<double>(m / 2 + 2);
  if (P.err) return P.err;
  MGR_TRY_CUDA(cudaMemsetAsync(h->ticket, 0, sizeof(unsigned), s));
  // written by the solve before it is read; zeros for the autotuner's
  // iteration over a zero basis
  MGR_TRY_CUDA(cudaMemsetAsync(h->gram, 0, sizeof(double) * (m / 2 + 2), s));
  return MGR_SUCCESS;
}

// dst[0..nv) = V[0..nv)^T w, computed twice-reduced (fixed order)
static void mdot(Handle* h, const double* V, int64_t ld, int nv, const double* w, int64_t n,
                 double* dst, int accumulate, cudaStream_t s) {
  const int nb = mdot_blocks(n);
  MGR_LAUNCH k_mdot<false><<<nb, KB, 0, s>>>(V, ld, nv, const_cast<double*>(w), n, h->part, nullptr);
  MGR_LAUNCH k_mdot_final<false><<<nv, FIN_T, 0, s>>>(h->part, nb, nv, dst, accumulate, nullptr);
}

// ---------------------------------------------------------------------------
// Jacobian product over the sliced copy
// ---------------------------------------------------------------------------
// One thread per row, entry k of row i at soff[i / 32] + 32 k + i % 32: one
// multiply-add per non-zero, summed over k in order (row lengths from the CSR
// row pointers).  RES: y = b - A x.
template <bool RES>
__global__ void __launch_bounds__(256)
k_spmv_sell64(const int64_t* __restrict__ soff, const int64_t* __restrict__ rp,
              const int32_t* __restrict__ sci, const double* __restrict__ sval, int64_t n,
              const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = soff[i >> 5] + (i & 31);
    const int len = (int)(rp[i + 1] - rp[i]);
    double acc = 0.0;
#pragma unroll 4
    for (int k = 0; k < len; k++) acc += sval[o + (int64_t)k * 32] * __ldg(x + sci[o + (int64_t)k * 32]);
    y[i] = RES ? b[i] - acc : acc;
  }
}

void jacobian_product(Handle* h, const mgr_matrix_t* A, bool sell, const double* x, double* y,
                      const double* b, bool res, cudaStream_t s) {
  const int64_t n = A->n, nnz = A->nnz;
  if (!sell || n <= 0) {
    if (res) residual64(A->row_ptr, A->col_idx, A->val, n, nnz, b, x, y, s);
    else spmv64(A->row_ptr, A->col_idx, A->val, n, nnz, x, y, s);
    return;
  }
  const JacobianSell& J = h->jsell;
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 152LL * 64);
  if (res)
    MGR_LAUNCH k_spmv_sell64<true><<<grid, 256, 0, s>>>(J.soff, A->row_ptr, J.sci, J.sval, n, x, y, b);
  else
    MGR_LAUNCH k_spmv_sell64<false><<<grid, 256, 0, s>>>(J.soff, A->row_ptr, J.sci, J.sval, n, x, y, b);
}

// Modified Gram-Schmidt of w against V_0..V_j, two projections per launch
// (j/2 + 2 launches): hcol[0..j] = the projections, hcol[j+1] = ||w||,
// vnext = w / ||w||
static void mgs(Handle* h, int j, double* vnext, cudaStream_t s) {
  const int64_t n = h->n;
  for (int p = 0; p <= j / 2 + 1; p++)
    MGR_LAUNCH k_mgs_pair<<<mgs_grid(n), KB, 0, s>>>(h->V, n, p, j, h->w, n, h->part, h->hcol,
                                                     h->gram, h->hred + 1, h->ticket);
  MGR_LAUNCH k_scale_by<<<grid_for(n, KB), KB, 0, s>>>(h->w, h->hred + 1, vnext, n);
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
  const int ortho = resolve_ortho(o->ortho, n);
  if (m > 60 || ortho < 0) return MGR_ERR_INVALID_ARG;
  const int maxit = o->max_iter > 0 ? o->max_iter : 1000;
  const double rtol = o->rtol > 0 ? o->rtol : 1e-8;
  MGR_TRY(ensure_krylov(h, m, s));
  // large Jacobians: the products read a sliced copy of A made here
  const int sv = jacobian_sell_refresh(h, A, s);
  if (sv < 0) return sv;
  const bool pat = sv == 1;
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
        MGR_LAUNCH k_mdot_final<true><<<1, FIN_T, 0, s>>>(h->part, nb, 1, h->hred, 0, h->hred + 1);
        MGR_LAUNCH k_scale_by<<<grid_for(n, KB), KB, 0, s>>>(h->r, h->hred + 1, h->V, n);
      }
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int jend = 0;
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
          jacobian_product(h, A, pat, h->r, h->w, nullptr, false, s);
        } else {
          double* zj = (double*)h->Z + (int64_t)j * n;
          MGR_TRY(apply_mgr(h, vj, zj, s));
          if (tr) cudaEventRecord(tev[1], s);
          jacobian_product(h, A, pat, zj, h->w, nullptr, false, s);
        }
        if (tr) cudaEventRecord(tev[2], s);
        if (ortho == MGR_ORTHO_MGS) {
          mgs(h, j, vnext, s);   // j + 1 dependent projections, then ||w||
        } else {
          // classical Gram-Schmidt, twice; the second update also forms ||w||^2
          mdot(h, h->V, n, j + 1, h->w, n, h->hcol, 0, s);                     // h1 = V^T w
          const int nb = mdot_blocks(n);                                      // w -= V h1; h2 = V^T w
          MGR_LAUNCH k_mdot<true><<<nb, KB, 0, s>>>(h->V, n, j + 1, h->w, n, h->part, h->hcol);
          MGR_LAUNCH k_mdot_final<false><<<j + 1, FIN_T, 0, s>>>(h->part, nb, j + 1, h->yv, 0, nullptr);
          MGR_LAUNCH k_mupdate<true><<<nb, KB, 0, s>>>(h->V, n, j + 1, h->yv, h->w, n, h->part);   // w -= V h2
          MGR_LAUNCH k_mdot_final<false><<<j + 1, FIN_T, 0, s>>>(h->yv, 1, j + 1, h->hcol, 1, nullptr);   // h += h2
          MGR_LAUNCH k_mdot_final<true><<<1, FIN_T, 0, s>>>(h->part, nb, 1, h->hcol + j + 1, 0, h->hred + 1);   // ||w||
          MGR_LAUNCH k_scale_by<<<grid_for(n, KB), KB, 0, s>>>(h->w, h->hred + 1, vnext, n);
        }
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
      jacobian_product(h, A, pat, x, h->r, b, true, s);
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

// ===========================================================================
// Lockstep batch: every system of an ensemble advances one FGMRES iteration
// per round, and each phase of the round is one launch over all systems that
// take part in it (a device flag per system): the preconditioner applications
// as one CUDA graph with a conditional branch per system, the Jacobian
// products as one row-binned launch per lanes-per-row group, the Gram-Schmidt
// passes as launches over every system's chunk blocks, and one readback of
// all Hessenberg columns.  Each system's arithmetic is that of fgmres_run
// (same kernels' per-element and per-block bodies, same lanes per row, same
// host Givens), so its iterations and solution equal its single-system solve.
// ===========================================================================
namespace mgr {
namespace {

enum { LS_VW = 0, LS_RR = 1, LS_BB = 2 };   // which vectors a dot pass reads

__device__ __forceinline__ int ls_sys_of(const int64_t* __restrict__ off, int cnt, int64_t g) {
  int lo = 0, hi = cnt;   // off[lo] <= g < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Row g of a launch over every system's rows (single < 0: the systems' rows
// concatenated, the system found from the row offsets) or over the rows of
// system `single` alone (a branch of the lockstep graph).
__device__ __forceinline__ int64_t ls_rows(const LsSys* __restrict__ S, int single, int64_t nrows) {
  return single >= 0 ? S[single].n : nrows;
}
__device__ __forceinline__ int ls_row(const int64_t* __restrict__ roff, int nsys, int single,
                                      int64_t g, int64_t* i) {
  if (single >= 0) {
    *i = g;
    return single;
  }
  const int s = ls_sys_of(roff, nsys, g);
  *i = g - roff[s];
  return s;
}

// per row of every flagged system: x = 0 (what 0) or r = b (what 1)
__global__ void k_ls_init(const LsSys* __restrict__ S, const int* __restrict__ flag,
                          const int64_t* __restrict__ roff, int nsys, int64_t nrows, int what) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nrows;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int s = ls_sys_of(roff, nsys, g);
    if (!flag[s]) continue;
    const int64_t i = g - roff[s];
    if (what == 0) S[s].x[i] = 0.0;
    else S[s].r[i] = S[s].b[i];
  }
}

// v_j into the fixed input of the system's preconditioner graph
__global__ void k_ls_gather(const LsSys* __restrict__ S, const int* __restrict__ flag,
                            const int* __restrict__ jcur, const int64_t* __restrict__ roff,
                            int nsys, int64_t nrows, int mixed, int single) {
  const int64_t tot = ls_rows(S, single, nrows);
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < tot;
       g += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    const int s = ls_row(roff, nsys, single, g, &i);
    if (!flag[s]) continue;
    const LsSys& d = S[s];
    const double v = d.V[(int64_t)jcur[s] * d.n + i];
    if (mixed) d.vin32[i] = (float)v;
    else d.gin[i] = v;
  }
}

// z_j from the graph's fixed output: stored as Z_j; under MGR_MIXED also
// widened once into r (the FP64 operand of the Jacobian product)
__global__ void k_ls_scatter(const LsSys* __restrict__ S, const int* __restrict__ flag,
                             const int* __restrict__ jcur, const int64_t* __restrict__ roff,
                             int nsys, int64_t nrows, int mixed, int single) {
  const int64_t tot = ls_rows(S, single, nrows);
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < tot;
       g += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    const int s = ls_row(roff, nsys, single, g, &i);
    if (!flag[s]) continue;
    const LsSys& d = S[s];
    const int64_t at = (int64_t)jcur[s] * d.n + i;
    if (mixed) {
      const float v = d.zout32[i];
      ((float*)d.Z)[at] = v;
      d.r[i] = (double)v;
    } else {
      ((double*)d.Z)[at] = d.gout[i];
    }
  }
}

// FP64 CSR product over the rows of the group's systems, G lanes per row
// (the single-system product's lanes for these matrices, so each row's sum
// is formed in the same order).  RES: r = b - A x; else w = A z_j.
template <int G, bool RES>
__global__ void __launch_bounds__(256)
k_ls_spmv(const LsSys* __restrict__ S, const int* __restrict__ flag, const int* __restrict__ jcur,
          const int* __restrict__ gsys, const int64_t* __restrict__ goff, int cnt, int64_t nrows,
          int mixed, int single) {
  const int lane = threadIdx.x & (G - 1);
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t tot = ls_rows(S, single, nrows);
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; g < tot; g += stride) {
    int s;
    int64_t i;
    if (single >= 0) {
      s = single;
      i = g;
    } else {
      const int q = ls_sys_of(goff, cnt, g);
      s = gsys[q];
      i = g - goff[q];
    }
    if (!flag[s]) continue;
    const LsSys& d = S[s];
    if (d.sval) continue;   // its product reads the sliced copy (k_ls_spmv_sell)
    const double* x = RES ? d.x : (mixed ? d.r : (const double*)d.Z + (int64_t)jcur[s] * d.n);
    const int64_t e0 = d.rp[i], e1 = d.rp[i + 1];
    double acc = 0.0;
    int64_t k = e0 + lane;
#pragma unroll 4
    for (; k < e1; k += G) acc += d.val[k] * __ldg(x + d.ci[k]);
    const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, G);
    if (lane == 0) {
      if (RES) d.r[i] = d.b[i] - acc;
      else d.w[i] = acc;
    }
  }
}

// The product of every flagged system with a sliced copy, one thread per row
// over all systems' rows: k_spmv_sell64's per-row loop.
template <bool RES>
__global__ void __launch_bounds__(256)
k_ls_spmv_sell(const LsSys* __restrict__ S, const int* __restrict__ flag, const int* __restrict__ jcur,
               const int64_t* __restrict__ roff, int nsys, int64_t nrows, int mixed) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nrows;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int s = ls_sys_of(roff, nsys, g);
    if (!flag[s]) continue;
    const LsSys& d = S[s];
    if (!d.sval) continue;
    const int64_t i = g - roff[s];
    const double* x = RES ? d.x : (mixed ? d.r : (const double*)d.Z + (int64_t)jcur[s] * d.n);
    const int64_t o = d.soff[i >> 5] + (i & 31);
    const int len = (int)(d.rp[i + 1] - d.rp[i]);
    double acc = 0.0;
#pragma unroll 4
    for (int k = 0; k < len; k++) acc += d.sval[o + (int64_t)k * 32] * __ldg(x + d.sci[o + (int64_t)k * 32]);
    if (RES) d.r[i] = d.b[i] - acc;
    else d.w[i] = acc;
  }
}

// block -> (system, chunk) for the chunk-block passes (single >= 0: the
// launch covers that system's chunks alone)
__device__ __forceinline__ bool ls_block(const LsSys* __restrict__ S, const int* __restrict__ flag,
                                         const int32_t* __restrict__ blk_sys, int single,
                                         int* s_out, int64_t* c_out) {
  const int s = single >= 0 ? single : blk_sys[blockIdx.x];
  if (!flag[s]) return false;
  *s_out = s;
  *c_out = single >= 0 ? (int64_t)blockIdx.x : (int64_t)blockIdx.x - S[s].blk0;
  return true;
}

template <bool UPDATE>
__global__ void __launch_bounds__(KB)
k_ls_mdot(const LsSys* __restrict__ S, const int* __restrict__ flag, const int* __restrict__ jcur,
          const int32_t* __restrict__ blk_sys, double* __restrict__ part,
          const double* __restrict__ Hc, int which, int single) {
  int s;
  int64_t c;
  if (!ls_block(S, flag, blk_sys, single, &s, &c)) return;
  const LsSys& d = S[s];
  if (which == LS_VW && d.ortho != MGR_ORTHO_CGS2) return;   // a classical Gram-Schmidt pass
  double* ps = part + d.blk0 * LS_H;
  if (which == LS_VW)
    mdot_body<UPDATE>(d.V, d.n, jcur[s] + 1, d.w, d.n, ps, Hc + (int64_t)s * LS_H, c);
  else if (which == LS_RR)
    mdot_body<false>(d.r, d.n, 1, d.r, d.n, ps, nullptr, c);
  else
    mdot_body<false>(d.b, d.n, 1, const_cast<double*>(d.b), d.n, ps, nullptr, c);
}

template <bool NORM>
__global__ void __launch_bounds__(KB)
k_ls_mupdate(const LsSys* __restrict__ S, const int* __restrict__ flag, const int* __restrict__ jcur,
             const int32_t* __restrict__ blk_sys, double* __restrict__ part,
             const double* __restrict__ Yv, int single) {
  int s;
  int64_t c;
  if (!ls_block(S, flag, blk_sys, single, &s, &c)) return;
  const LsSys& d = S[s];
  if (d.ortho != MGR_ORTHO_CGS2) return;   // classical Gram-Schmidt only
  mupdate_body<NORM>(d.V, d.n, jcur[s] + 1, Yv + (int64_t)s * LS_H, d.w, d.n,
                     part + d.blk0 * LS_H, c);
}

// per flagged system, block (blockIdx.x) per vector i < nv (nv = j + 1, or 1
// when `one`), FIN_T threads: dst[s * dstride + (off_j ? j + 1 : 0) + i] (+)=
// the sum of its partials in the single-system order -- the system's chunk
// partials in `part`, or (rows) the one partial row part[s * LS_H ..] -- and
// with SQRT red[s * 4 + 1] = 1/norm.  gs: a classical Gram-Schmidt step,
// skipped by systems that orthogonalise by modified Gram-Schmidt.
template <bool SQRT>
__global__ void __launch_bounds__(FIN_T)
k_ls_final(const LsSys* __restrict__ S, const int* __restrict__ flag, const int* __restrict__ jcur,
           const double* __restrict__ part, int rows, double* __restrict__ dst, int dstride,
           int off_j, int one, int accumulate, double* __restrict__ red, int gs, int single) {
  const int s = single >= 0 ? single : blockIdx.y;
  if (!flag[s]) return;
  const int nv = one ? 1 : jcur[s] + 1;
  const int i = blockIdx.x;
  if (i >= nv) return;
  const LsSys& d = S[s];
  if (gs && d.ortho != MGR_ORTHO_CGS2) return;
  double* h = dst + (int64_t)s * dstride + (off_j ? jcur[s] + 1 : 0);
  if (rows)
    mdot_final_block<SQRT>(part + (int64_t)s * LS_H, 1, nv, i, h, accumulate, red + (int64_t)s * 4 + 1);
  else
    mdot_final_block<SQRT>(part + d.blk0 * LS_H, d.nb, nv, i, h, accumulate, red + (int64_t)s * 4 + 1);
}

// V_(j+1) = w * rinv (what 0), or V_0 = r * rinv (what 1)
__global__ void k_ls_scale(const LsSys* __restrict__ S, const int* __restrict__ flag,
                           const int* __restrict__ jcur, const int64_t* __restrict__ roff,
                           int nsys, int64_t nrows, const double* __restrict__ red, int what,
                           int single) {
  const int64_t tot = ls_rows(S, single, nrows);
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < tot;
       g += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    const int s = ls_row(roff, nsys, single, g, &i);
    if (!flag[s]) continue;
    const LsSys& d = S[s];
    const double f = red[(int64_t)s * 4 + 1];
    if (what == 0) d.V[(int64_t)(jcur[s] + 1) * d.n + i] = d.w[i] * f;
    else d.V[i] = d.r[i] * f;
  }
}

// Modified Gram-Schmidt pass p for every flagged system that orthogonalises
// that way and whose iteration j has p <= j/2 + 1: grid (the largest system's
// mgs_grid, systems); the blocks beyond a system's own mgs_grid return, the
// rest run the single-system body with that system's grid, partial buffer,
// counter, Gram entries and Hessenberg column.
__global__ void __launch_bounds__(KB) k_ls_mgs(const LsSys* __restrict__ S, const int* __restrict__ flag,
                                               const int* __restrict__ jcur, int p,
                                               double* __restrict__ part, double* __restrict__ Hc,
                                               double* __restrict__ gram, double* __restrict__ red,
                                               unsigned* __restrict__ tickets) {
  const int s = blockIdx.y;
  if (!flag[s]) return;
  const LsSys& d = S[s];
  if (d.ortho != MGR_ORTHO_MGS) return;
  const int j = jcur[s];
  if (p > j / 2 + 1) return;
  const int G = mgs_grid(d.n);
  if ((int)blockIdx.x >= G) return;
  mgs_pair_body(d.V, d.n, p, j, d.w, d.n, part + d.blk0 * LS_H, Hc + (int64_t)s * LS_H,
                gram + (int64_t)s * LS_H, red + (int64_t)s * 4 + 1, tickets + s, G, blockIdx.x);
}

// x += sum_{i < jcur+1} y_i Z_i (jcur holds jend - 1 here), as k_xupdate
template <class Z>
__global__ void __launch_bounds__(KB)
k_ls_xupdate(const LsSys* __restrict__ S, const int* __restrict__ flag, const int* __restrict__ jcur,
             const int64_t* __restrict__ roff, int nsys, int64_t nrows, const double* __restrict__ Yv) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nrows;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int s = ls_sys_of(roff, nsys, g);
    if (!flag[s]) continue;
    const LsSys& d = S[s];
    const int64_t t = g - roff[s];
    const int nv = jcur[s] + 1;
    const double* ys = Yv + (int64_t)s * LS_H;
    const Z* Zb = (const Z*)d.Z;
    const int64_t ld = d.n;
    double acc = d.x[t];
    int i = 0;
    for (; i + 8 <= nv; i += 8) {
      double z[8];
#pragma unroll
      for (int q = 0; q < 8; q++) z[q] = (double)Zb[(int64_t)(i + q) * ld + t];
#pragma unroll
      for (int q = 0; q < 8; q++) acc += ys[i + q] * z[q];
    }
    for (; i < nv; i++) acc += ys[i] * (double)Zb[(int64_t)i * ld + t];
    d.x[t] = acc;
  }
}

}  // namespace

int ensure_krylov_ws(Handle* h, int m) {
  MGR_TRY(ensure_krylov(h, m, h->pool.s));
  MGR_TRY_CUDA(cudaStreamSynchronize(h->pool.s));   // the counter reset, before other streams
  return MGR_SUCCESS;
}

// flag / jcur uploads between two host synchronisations each use their own
// pinned slot: an asynchronous copy reads its host source when it runs
static constexpr int LS_SLOTS = 4;

Lockstep::~Lockstep() {
  if (exec) cudaGraphExecDestroy(exec);
  if (hpin) cudaFreeHost(hpin);
  if (ipin) cudaFreeHost(ipin);
  pool.free_all();
}

// Sizes the per-solve plan (descriptors, block map, SpMV groups, reduction
// buffers) for restart m; built once and kept for later solves.
// The plan's device buffers (descriptors, row offsets, chunk-block map, SpMV
// groups, Hessenberg / reduction buffers), sized from the systems alone so
// that the lockstep graph, built at setup, can name them.
int lockstep_alloc(Lockstep* L, Handle** hs, const mgr_matrix_t* A, cudaStream_t s) {
  const int ns = L->nsys;
  Pool& P = L->pool;
  P.s = s;
  L->dsys = P.get<LsSys>(ns);
  L->jcur = P.get<int>(ns);
  L->roff = P.get<int64_t>(ns + 1);
  L->Hc = P.get<double>((int64_t)ns * LS_H);
  L->Yv = P.get<double>((int64_t)ns * LS_H);
  L->red = P.get<double>((int64_t)ns * 4);
  L->tickets = P.get<unsigned>(ns);
  L->gram = P.get<double>((int64_t)ns * LS_H);
  if (P.err) return P.err;
  MGR_TRY_CUDA(cudaMemsetAsync(L->tickets, 0, sizeof(unsigned) * ns, s));
  MGR_TRY_CUDA(cudaMemsetAsync(L->gram, 0, sizeof(double) * ns * LS_H, s));
  MGR_TRY_CUDA(cudaMallocHost(&L->hpin, sizeof(double) * ((size_t)ns * LS_H + (size_t)ns * 4)));
  MGR_TRY_CUDA(cudaMallocHost(&L->ipin, sizeof(int) * 2 * (size_t)ns * LS_SLOTS));
  std::vector<int64_t> roff(ns + 1, 0);
  std::vector<int32_t> bsys;
  L->lanes.assign(ns, 1);
  L->nb.assign(ns, 0);
  for (int q = 0; q < ns; q++) {
    roff[q + 1] = roff[q] + hs[q]->n;
    L->nb[q] = mdot_blocks(hs[q]->n);
    L->mgs_gmax = std::max(L->mgs_gmax, mgs_grid(hs[q]->n));
    for (int k = 0; k < L->nb[q]; k++) bsys.push_back(q);
    L->lanes[q] = spmv_lanes(A[q].nnz, A[q].n);
  }
  L->nrows = roff[ns];
  L->nblk = (int64_t)bsys.size();
  L->blk_sys = P.get<int32_t>(L->nblk);
  L->part = P.get<double>(L->nblk * LS_H);
  if (P.err) return P.err;
  MGR_TRY_CUDA(cudaMemcpyAsync(L->roff, roff.data(), sizeof(int64_t) * (ns + 1),
                               cudaMemcpyHostToDevice, s));
  MGR_TRY_CUDA(cudaMemcpyAsync(L->blk_sys, bsys.data(), sizeof(int32_t) * L->nblk,
                               cudaMemcpyHostToDevice, s));
  // row bins: the systems grouped by their lanes per row
  for (int q = 0; q < ns; q++) {
    size_t gi = 0;
    while (gi < L->gl.size() && L->gl[gi] != L->lanes[q]) gi++;
    if (gi == L->gl.size()) L->gl.push_back(L->lanes[q]);
  }
  for (size_t gi = 0; gi < L->gl.size(); gi++) {
    std::vector<int> sy;
    std::vector<int64_t> off(1, 0);
    for (int q = 0; q < ns; q++)
      if (L->lanes[q] == L->gl[gi]) {
        sy.push_back(q);
        off.push_back(off.back() + hs[q]->n);
      }
    int* gs = P.get<int>(sy.size());
    int64_t* go = P.get<int64_t>(off.size());
    if (P.err) return P.err;
    MGR_TRY_CUDA(cudaMemcpyAsync(gs, sy.data(), sizeof(int) * sy.size(), cudaMemcpyHostToDevice, s));
    MGR_TRY_CUDA(cudaMemcpyAsync(go, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, s));
    MGR_TRY_CUDA(cudaStreamSynchronize(s));   // the host vectors go out of scope
    L->gsys.push_back(gs);
    L->groff.push_back(go);
    L->grows.push_back(off.back());
    L->gcnt.push_back((int)sy.size());
  }
  MGR_TRY_CUDA(cudaStreamSynchronize(s));
  return MGR_SUCCESS;
}

// The row-binned Jacobian products of every flagged system: one launch per
// lanes-per-row group.  RES: r = b - A x; else w = A z_j.
static void ls_spmv_all(Lockstep* L, bool res, cudaStream_t s) {
  const int mixed = L->mixed;
  if (L->any_sell) {
    const unsigned vg = grid_for(L->nrows, 256, 152 * 64);
    if (res)
      MGR_LAUNCH k_ls_spmv_sell<true><<<vg, 256, 0, s>>>(L->dsys, L->flag, L->jcur, L->roff, L->nsys,
                                                         L->nrows, mixed);
    else
      MGR_LAUNCH k_ls_spmv_sell<false><<<vg, 256, 0, s>>>(L->dsys, L->flag, L->jcur, L->roff, L->nsys,
                                                          L->nrows, mixed);
  }
  for (size_t gi = 0; gi < L->gl.size(); gi++) {
    const int G = L->gl[gi];
    const unsigned grid = (unsigned)std::min<int64_t>((L->grows[gi] * G + 255) / 256, 152LL * 64);
#define MGR_LS_CASE(gg)                                                                             \
  case gg:                                                                                          \
    if (res)                                                                                        \
      MGR_LAUNCH k_ls_spmv<gg, true><<<grid, 256, 0, s>>>(L->dsys, L->flag, L->jcur, L->gsys[gi],  \
                                                          L->groff[gi], L->gcnt[gi], L->grows[gi], \
                                                          mixed, -1);                               \
    else                                                                                            \
      MGR_LAUNCH k_ls_spmv<gg, false><<<grid, 256, 0, s>>>(L->dsys, L->flag, L->jcur, L->gsys[gi], \
                                                           L->groff[gi], L->gcnt[gi], L->grows[gi],\
                                                           mixed, -1);                              \
    break;
    switch (G) {
      MGR_LS_CASE(1)
      MGR_LS_CASE(2)
      MGR_LS_CASE(4)
      MGR_LS_CASE(8)
      MGR_LS_CASE(16)
      default: MGR_LS_CASE(32)
    }
#undef MGR_LS_CASE
  }
}

// One FGMRES iteration of every flagged system (flag and jcur already on the
// device), each phase one launch for all of them: v_j into the graph inputs;
// the lockstep graph (the preconditioner application of every flagged system
// as a conditional branch); z_j out; w = A z_j; Gram-Schmidt -- modified
// (one launch per pair of projections up to pass jmax/2 + 1, jmax = the
// largest j of the flagged systems that use it, -1 for none) and classical twice (seven
// launches, when any flagged system uses it); v_(j+1) = w / ||w||.  Every
// per-row, per-chunk and per-element body is the one fgmres_run's kernels
// use, so each system gets the same bits.
static int ls_iterate(Lockstep* L, long long graph_kernels, int jmax, bool cgs, cudaStream_t s) {
  const int ns = L->nsys;
  const int mixed = L->mixed;
  const unsigned vg = grid_for(L->nrows, KB, 152 * 16);
  const int nbk = (int)L->nblk;
  const dim3 fin1(1, ns), finv(LS_H, ns);   // one block per vector and system
  MGR_LAUNCH k_ls_gather<<<vg, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->roff, ns, L->nrows, mixed, -1);
  MGR_TRY_CUDA(cudaGraphLaunch(L->exec, s));
  count_graph_launch(graph_kernels);
  MGR_LAUNCH k_ls_scatter<<<vg, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->roff, ns, L->nrows, mixed, -1);
  ls_spmv_all(L, false, s);
  for (int p = 0; p <= jmax / 2 + 1 && jmax >= 0; p++)
    MGR_LAUNCH k_ls_mgs<<<dim3(L->mgs_gmax, ns), KB, 0, s>>>(L->dsys, L->flag, L->jcur, p, L->part,
                                                             L->Hc, L->gram, L->red, L->tickets);
  if (cgs) {
    MGR_LAUNCH k_ls_mdot<false><<<nbk, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->blk_sys, L->part,
                                                    nullptr, LS_VW, -1);
    MGR_LAUNCH k_ls_final<false><<<finv, FIN_T, 0, s>>>(L->dsys, L->flag, L->jcur, L->part, 0, L->Hc,
                                                        LS_H, 0, 0, 0, L->red, 1, -1);   // h1
    MGR_LAUNCH k_ls_mdot<true><<<nbk, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->blk_sys, L->part,
                                                   L->Hc, LS_VW, -1);
    MGR_LAUNCH k_ls_final<false><<<finv, FIN_T, 0, s>>>(L->dsys, L->flag, L->jcur, L->part, 0, L->Yv,
                                                        LS_H, 0, 0, 0, L->red, 1, -1);   // h2
    MGR_LAUNCH k_ls_mupdate<true><<<nbk, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->blk_sys, L->part,
                                                      L->Yv, -1);
    MGR_LAUNCH k_ls_final<false><<<finv, FIN_T, 0, s>>>(L->dsys, L->flag, L->jcur, L->Yv, 1, L->Hc,
                                                        LS_H, 0, 0, 1, L->red, 1, -1);   // h += h2
    MGR_LAUNCH k_ls_final<true><<<fin1, FIN_T, 0, s>>>(L->dsys, L->flag, L->jcur, L->part, 0, L->Hc,
                                                       LS_H, 1, 1, 0, L->red, 1, -1);    // ||w||
  }
  MGR_LAUNCH k_ls_scale<<<vg, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->roff, ns, L->nrows, L->red, 0,
                                          -1);
  return MGR_SUCCESS;
}

// One lockstep round for the autotuner: every system at the iteration
// lockstep_tune_prepare set up, synchronised.
int lockstep_tune_round(Lockstep* L, cudaStream_t s) {
  std::vector<int> ones(L->nsys, 1);
  MGR_TRY_CUDA(cudaMemcpyAsync(L->flag, ones.data(), sizeof(int) * L->nsys, cudaMemcpyHostToDevice, s));
  long long k = 1;
  for (long long q : L->body_kernels) k += q;
  bool mgs_any = false, cgs_any = false;
  for (int o : L->ortho) (o == MGR_ORTHO_MGS ? mgs_any : cgs_any) = true;
  MGR_TRY(ls_iterate(L, k, mgs_any ? L->tune_j : -1, cgs_any, s));
  MGR_TRY_CUDA(cudaStreamSynchronize(s));
  return MGR_SUCCESS;
}

// One FGMRES iteration (iteration j of a cycle, over a zero basis) of a
// single system with fgmres_run's kernels and no readback: the unit the batch
// schedule autotuner times for the worker schedules.  Allocates the Krylov
// workspace for restart m on `s` if it is not there yet.
int krylov_tune_iteration(Handle* h, const mgr_matrix_t* A, int m, int ortho, int j,
                          cudaStream_t s) {
  h->pool.s = s;
  MGR_TRY(ensure_krylov(h, m, s));
  if (j < 0 || j >= m) return MGR_ERR_INVALID_ARG;
  // the sliced copy of A, made once for all of the autotuner's rounds
  const JacobianSell& J = h->jsell;
  int sv = (J.valid && J.rp == A->row_ptr && J.ci == A->col_idx && J.val == A->val &&
            J.n == A->n && J.nnz == A->nnz) ? 1 : 0;
  if (!sv) sv = jacobian_sell_refresh(h, A, s);
  if (sv < 0) return sv;
  const bool pat = sv == 1;
  const int64_t n = h->n;
  // iteration j of a cycle over a zero basis: the arithmetic of any basis
  MGR_TRY_CUDA(cudaMemsetAsync(h->V, 0, sizeof(double) * n * (j + 1), s));
  double* vj = h->V + (int64_t)j * n;
  double* vnext = h->V + (int64_t)(j + 1) * n;
  if (h->opt.precision == MGR_MIXED) {
    MGR_TRY(apply_mgr_mixed_into(h, vj, h->zout32, s));
    MGR_LAUNCH k_widen<<<grid_for(n, KB), KB, 0, s>>>(h->zout32, (float*)h->Z + (int64_t)j * n, h->r, n);
    jacobian_product(h, A, pat, h->r, h->w, nullptr, false, s);
  } else {
    double* zj = (double*)h->Z + (int64_t)j * n;
    MGR_TRY(apply_mgr(h, vj, zj, s));
    jacobian_product(h, A, pat, zj, h->w, nullptr, false, s);
  }
  if (resolve_ortho(ortho, n) == MGR_ORTHO_MGS) {
    mgs(h, j, vnext, s);
    MGR_TRY_CUDA(cudaGetLastError());
    return MGR_SUCCESS;
  }
  const int nb = mdot_blocks(n);
  mdot(h, h->V, n, j + 1, h->w, n, h->hcol, 0, s);
  MGR_LAUNCH k_mdot<true><<<nb, KB, 0, s>>>(h->V, n, j + 1, h->w, n, h->part, h->hcol);
  MGR_LAUNCH k_mdot_final<false><<<j + 1, FIN_T, 0, s>>>(h->part, nb, j + 1, h->yv, 0, nullptr);
  MGR_LAUNCH k_mupdate<true><<<nb, KB, 0, s>>>(h->V, n, j + 1, h->yv, h->w, n, h->part);
  MGR_LAUNCH k_mdot_final<false><<<j + 1, FIN_T, 0, s>>>(h->yv, 1, j + 1, h->hcol, 1, nullptr);
  MGR_LAUNCH k_mdot_final<true><<<1, FIN_T, 0, s>>>(h->part, nb, 1, h->hcol + j + 1, 0, h->hred + 1);
  MGR_LAUNCH k_scale_by<<<grid_for(n, KB), KB, 0, s>>>(h->w, h->hred + 1, vnext, n);
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

static int lockstep_plan(Lockstep* L, Handle** hs, const mgr_matrix_t* A, const double* const* b,
                         double* const* x, int m, int ortho, cudaStream_t s);

// The lockstep graph's round over valid buffers for the autotuner: every
// system's Krylov workspace for restart m, descriptors, iteration j of a
// cycle over a zero basis (v_0 .. v_j = 0).
int lockstep_tune_prepare(Lockstep* L, Handle** hs, const mgr_matrix_t* A, int m, int ortho, int j,
                          cudaStream_t s) {
  if (j < 0 || j >= m) return MGR_ERR_INVALID_ARG;
  std::vector<const double*> nb(L->nsys, nullptr);
  std::vector<double*> nx(L->nsys, nullptr);
  for (int q = 0; q < L->nsys; q++) hs[q]->pool.s = s;
  MGR_TRY(lockstep_plan(L, hs, A, nb.data(), nx.data(), m, ortho, s));
  for (int q = 0; q < L->nsys; q++)
    MGR_TRY_CUDA(cudaMemsetAsync(hs[q]->V, 0, sizeof(double) * hs[q]->n * (j + 1), s));
  std::vector<int> jv(L->nsys, j);
  MGR_TRY_CUDA(cudaMemcpyAsync(L->jcur, jv.data(), sizeof(int) * L->nsys, cudaMemcpyHostToDevice, s));
  MGR_TRY_CUDA(cudaStreamSynchronize(s));   // jv outlives its copy
  L->tune_j = j;
  return MGR_SUCCESS;
}

// Per solve: every system's Krylov workspace for restart m, its resolved
// orthogonalisation, and the descriptors that point at them.
static int lockstep_plan(Lockstep* L, Handle** hs, const mgr_matrix_t* A, const double* const* b,
                         double* const* x, int m, int ortho, cudaStream_t s) {
  const int ns = L->nsys;
  for (int q = 0; q < ns; q++) MGR_TRY(ensure_krylov_ws(hs[q], m));
  std::vector<LsSys> d(ns);
  L->ortho.assign(ns, MGR_ORTHO_CGS2);
  L->any_sell = false;
  int64_t blk0 = 0;
  for (int q = 0; q < ns; q++) {
    Handle* h = hs[q];
    d[q].n = h->n;
    d[q].rp = A[q].row_ptr;
    d[q].ci = A[q].col_idx;
    d[q].val = A[q].val;
    d[q].b = b[q];
    d[q].x = x[q];
    d[q].V = h->V;
    d[q].w = h->w;
    d[q].r = h->r;
    d[q].Z = h->Z;
    d[q].vin32 = h->vin32;
    d[q].zout32 = h->zout32;
    d[q].gin = h->gin;
    d[q].gout = h->gout;
    d[q].blk0 = blk0;
    d[q].nb = L->nb[q];
    d[q].ortho = L->ortho[q] = resolve_ortho(ortho, h->n);
    if (d[q].ortho < 0) return MGR_ERR_INVALID_ARG;
    // large systems: the products read a sliced copy, as in fgmres_run (the
    // autotuner's plan has no right-hand sides and needs none)
    const int sv = jacobian_sell_refresh(h, &A[q], s);
    if (sv < 0) return sv;
    if (sv == 1) {
      d[q].soff = h->jsell.soff;
      d[q].sci = h->jsell.sci;
      d[q].sval = h->jsell.sval;
      L->any_sell = true;
    }
    blk0 += d[q].nb;
  }
  MGR_TRY_CUDA(cudaMemcpyAsync(L->dsys, d.data(), sizeof(LsSys) * ns, cudaMemcpyHostToDevice, s));
  MGR_TRY_CUDA(cudaStreamSynchronize(s));
  L->m = m;
  return MGR_SUCCESS;
}

int fgmres_lockstep(Lockstep* L, Handle** hs, const mgr_matrix_t* A, const double* const* b,
                    double* const* x, const fgmres_options_t* o, fgmres_info_t* info,
                    cudaStream_t s) {
  const int ns = L->nsys;
  const int m = o->restart > 0 ? o->restart : 50;
  if (m > 60) return MGR_ERR_INVALID_ARG;
  const int maxit = o->max_iter > 0 ? o->max_iter : 1000;
  const double rtol = o->rtol > 0 ? o->rtol : 1e-8;
  MGR_TRY(lockstep_plan(L, hs, A, b, x, m, o->ortho, s));
  const bool mixed = L->mixed;
  struct Events {
    cudaEvent_t e[2] = {};
    ~Events() {
      for (auto& q : e)
        if (q) cudaEventDestroy(q);
    }
  } ev;
  MGR_TRY_CUDA(cudaEventCreate(&ev.e[0]));
  MGR_TRY_CUDA(cudaEventCreate(&ev.e[1]));
  MGR_TRY_CUDA(cudaEventRecord(ev.e[0], s));

  // host state per system, as in fgmres_run
  struct St {
    std::vector<double> H, cs, sn, g, y;
    double bnorm = 0.0, beta = 0.0, relres = 1.0;
    int iters = 0, restarts = 0, status = MGR_NOT_CONVERGED, j = 0, jend = 0;
    bool done = false, cycle_end = false, restart = false;
  };
  std::vector<St> st(ns);
  for (auto& t : st) {
    t.H.assign((size_t)(m + 1) * m, 0.0);
    t.cs.assign(m, 0.0);
    t.sn.assign(m, 0.0);
    t.g.assign(m + 1, 0.0);
    t.y.assign(m, 0.0);
  }
  int slot = 0;
  int* hflag = L->ipin;
  int* hj = L->ipin + ns;
  double* hH = L->hpin;
  double* hred = L->hpin + (size_t)ns * LS_H;
  const unsigned vg = grid_for(L->nrows, KB, 152 * 16);
  const int nbk = (int)L->nblk;
  // the flags / columns written since the last upload go out from the
  // current slot; the host then writes the next slot
  auto upload = [&]() -> int {
    MGR_TRY_CUDA(cudaMemcpyAsync(L->flag, hflag, sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    MGR_TRY_CUDA(cudaMemcpyAsync(L->jcur, hj, sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    if (++slot >= LS_SLOTS) return MGR_ERR_INVALID_ARG;   // more uploads than slots between syncs
    int* nf = L->ipin + (size_t)slot * 2 * ns;
    std::copy(hflag, hflag + ns, nf);
    std::copy(hj, hj + ns, nf + ns);
    hflag = nf;
    hj = nf + ns;
    return MGR_SUCCESS;
  };
  // after a host synchronisation every slot is free again
  auto synced = [&]() {
    if (slot == 0) return;
    int* f0 = L->ipin;
    std::copy(hflag, hflag + ns, f0);
    std::copy(hj, hj + ns, f0 + ns);
    hflag = f0;
    hj = f0 + ns;
    slot = 0;
  };
  const dim3 fin1(1, ns), finv(8, ns);   // one warp / up to 64 warps per system

  // x = 0, ||b||, r = b for every system
  for (int q = 0; q < ns; q++) {
    hflag[q] = 1;
    hj[q] = 0;
  }
  MGR_TRY(upload());
  MGR_LAUNCH k_ls_init<<<vg, KB, 0, s>>>(L->dsys, L->flag, L->roff, ns, L->nrows, 0);
  MGR_LAUNCH k_ls_mdot<false><<<nbk, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->blk_sys, L->part,
                                                  nullptr, LS_BB, -1);
  MGR_LAUNCH k_ls_final<false><<<fin1, FIN_T, 0, s>>>(L->dsys, L->flag, L->jcur, L->part, 0, L->red, 4,
                                                   0, 1, 0, L->red, 0, -1);
  MGR_TRY_CUDA(cudaMemcpyAsync(hred, L->red, sizeof(double) * 4 * ns, cudaMemcpyDeviceToHost, s));
  MGR_TRY_CUDA(cudaStreamSynchronize(s));
  synced();
  bool any_restart = false;
  for (int q = 0; q < ns; q++) {
    St& t = st[q];
    t.bnorm = std::sqrt(hred[(size_t)q * 4]);
    if (info && info[q].res_hist && info[q].res_hist_cap > 0) info[q].res_hist[0] = 1.0;
    if (t.bnorm == 0.0) {
      t.status = MGR_SUCCESS;
      t.relres = 0.0;
      t.done = true;
    } else if (maxit > 0) {
      t.beta = t.bnorm;
      t.restart = true;
      any_restart = true;
    } else {
      t.done = true;
    }
    hflag[q] = t.restart ? 1 : 0;
  }
  if (any_restart) {
    MGR_TRY(upload());
    MGR_LAUNCH k_ls_init<<<vg, KB, 0, s>>>(L->dsys, L->flag, L->roff, ns, L->nrows, 1);
  }
  std::vector<int> ends;
  for (;;) {
    // cycle starts: v_0 = r / ||r||
    any_restart = false;
    for (int q = 0; q < ns; q++) {
      hflag[q] = st[q].restart ? 1 : 0;
      any_restart |= st[q].restart;
    }
    if (any_restart) {
      MGR_TRY(upload());
      MGR_LAUNCH k_ls_mdot<false><<<nbk, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->blk_sys, L->part,
                                                      nullptr, LS_RR, -1);
      MGR_LAUNCH k_ls_final<true><<<fin1, FIN_T, 0, s>>>(L->dsys, L->flag, L->jcur, L->part, 0, L->red, 4,
                                                      0, 1, 0, L->red, 0, -1);
      MGR_LAUNCH k_ls_scale<<<vg, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->roff, ns, L->nrows, L->red, 1,
                                              -1);
      for (int q = 0; q < ns; q++)
        if (st[q].restart) {
          St& t = st[q];
          std::fill(t.g.begin(), t.g.end(), 0.0);
          t.g[0] = t.beta;
          t.j = 0;
          t.jend = 0;
          t.restart = false;
        }
    }
    // one iteration of every system in a cycle
    int active = 0, jmax = -1;
    bool cgs = false;
    long long graph_kernels = 1;
    for (int q = 0; q < ns; q++) {
      const bool a = !st[q].done && !st[q].cycle_end;
      hflag[q] = a ? 1 : 0;
      hj[q] = st[q].j;
      if (a) {
        active++;
        graph_kernels += L->body_kernels[q];
        if (L->ortho[q] == MGR_ORTHO_MGS) jmax = std::max(jmax, st[q].j);
        else cgs = true;
      }
    }
    if (active > 0) {
      MGR_TRY(upload());
      MGR_TRY(ls_iterate(L, graph_kernels, jmax, cgs, s));
      MGR_TRY_CUDA(cudaMemcpyAsync(hH, L->Hc, sizeof(double) * LS_H * ns, cudaMemcpyDeviceToHost, s));
      MGR_TRY_CUDA(cudaStreamSynchronize(s));
      synced();
      MGR_TRY_CUDA(cudaGetLastError());
      for (int q = 0; q < ns; q++) {
        if (!hflag[q]) continue;
        St& t = st[q];
        const int j = t.j;
        const double* hp = hH + (size_t)q * LS_H;
        for (int i = 0; i <= j + 1; i++) t.H[(size_t)i * m + j] = hp[i];
        const double hn = hp[j + 1];
        if (!std::isfinite(hn)) {
          t.status = MGR_ERR_BREAKDOWN;
          t.done = true;
          continue;
        }
        for (int i = 0; i < j; i++) {
          double a = t.H[(size_t)i * m + j], c = t.H[(size_t)(i + 1) * m + j];
          t.H[(size_t)i * m + j] = t.cs[i] * a + t.sn[i] * c;
          t.H[(size_t)(i + 1) * m + j] = -t.sn[i] * a + t.cs[i] * c;
        }
        double a = t.H[(size_t)j * m + j], c = t.H[(size_t)(j + 1) * m + j];
        double den = std::sqrt(a * a + c * c);
        t.cs[j] = den == 0.0 ? 1.0 : a / den;
        t.sn[j] = den == 0.0 ? 0.0 : c / den;
        t.H[(size_t)j * m + j] = t.cs[j] * a + t.sn[j] * c;
        t.H[(size_t)(j + 1) * m + j] = 0.0;
        t.g[j + 1] = -t.sn[j] * t.g[j];
        t.g[j] = t.cs[j] * t.g[j];
        t.iters++;
        t.jend = j + 1;
        if (info && info[q].res_hist && t.iters < info[q].res_hist_cap)
          info[q].res_hist[t.iters] = std::fabs(t.g[j + 1]) / t.bnorm;
        if (std::fabs(t.g[j + 1]) <= rtol * t.bnorm || hn == 0.0 || j + 1 >= m || t.iters >= maxit)
          t.cycle_end = true;
        else
          t.j = j + 1;
      }
    }
    // cycle ends: y = H^-1 g, x += Z y, true residual
    ends.clear();
    for (int q = 0; q < ns; q++)
      if (!st[q].done && st[q].cycle_end) ends.push_back(q);
    if (ends.empty()) {
      bool running = false;
      for (int q = 0; q < ns; q++) running |= !st[q].done;
      if (!running) break;
      continue;
    }
    for (int q = 0; q < ns; q++) {
      hflag[q] = 0;
      hj[q] = 0;
    }
    for (int q : ends) {
      St& t = st[q];
      for (int i = t.jend - 1; i >= 0; i--) {
        double v = t.g[i];
        for (int k = i + 1; k < t.jend; k++) v -= t.H[(size_t)i * m + k] * t.y[k];
        t.y[i] = v / t.H[(size_t)i * m + i];
      }
      std::copy(t.y.begin(), t.y.begin() + t.jend, hH + (size_t)q * LS_H);
      hflag[q] = 1;
      hj[q] = t.jend - 1;
    }
    MGR_TRY_CUDA(cudaMemcpyAsync(L->Yv, hH, sizeof(double) * LS_H * ns, cudaMemcpyHostToDevice, s));
    MGR_TRY(upload());
    if (mixed)
      MGR_LAUNCH k_ls_xupdate<float><<<vg, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->roff, ns, L->nrows,
                                                       L->Yv);
    else
      MGR_LAUNCH k_ls_xupdate<double><<<vg, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->roff, ns,
                                                        L->nrows, L->Yv);
    ls_spmv_all(L, true, s);
    MGR_LAUNCH k_ls_mdot<false><<<nbk, KB, 0, s>>>(L->dsys, L->flag, L->jcur, L->blk_sys, L->part,
                                                    nullptr, LS_RR, -1);
    MGR_LAUNCH k_ls_final<false><<<fin1, FIN_T, 0, s>>>(L->dsys, L->flag, L->jcur, L->part, 0, L->red, 4,
                                                     0, 1, 0, L->red, 0, -1);
    MGR_TRY_CUDA(cudaMemcpyAsync(hred, L->red, sizeof(double) * 4 * ns, cudaMemcpyDeviceToHost, s));
    MGR_TRY_CUDA(cudaStreamSynchronize(s));
    synced();
    for (int q : ends) {
      St& t = st[q];
      t.cycle_end = false;
      t.beta = std::sqrt(hred[(size_t)q * 4]);
      t.relres = t.beta / t.bnorm;
      if (!std::isfinite(t.beta)) {
        t.status = MGR_ERR_BREAKDOWN;
        t.done = true;
      } else if (t.relres <= rtol || t.beta == 0.0) {
        t.status = MGR_SUCCESS;
        t.done = true;
      } else {
        t.restarts++;
        if (t.iters >= maxit) t.done = true;
        else t.restart = true;
      }
    }
  }
  MGR_TRY_CUDA(cudaEventRecord(ev.e[1], s));
  MGR_TRY_CUDA(cudaEventSynchronize(ev.e[1]));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]);
  int first_err = 0, worst = 0;
  for (int q = 0; q < ns; q++) {
    const St& t = st[q];
    if (info) {
      info[q].iters = t.iters;
      info[q].restarts = t.restarts;
      info[q].converged = t.status == MGR_SUCCESS;
      info[q].rel_res_true = t.relres;
      info[q].setup_s = hs[q]->setup_s;
      info[q].solve_s = ms * 1e-3;
    }
    if (t.status < 0 && !first_err) first_err = t.status;
    if (t.status > worst) worst = t.status;
  }
  return first_err ? first_err : worst;
}

}  // namespace mgr
