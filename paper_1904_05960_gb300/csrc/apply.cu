// Device application of the MGR preconditioner (Algorithm 2 of Bui et al.,
// pre-smoothing F-relaxation, Eq. "MGR-pre") and of the inner AMG V-cycles
// (Sec. 6), in FP64 or FP32.
//
// Every kernel here streams a sparse matrix once and gathers vector entries
// through the read-only cache; the work is HBM-bound, so the kernels fuse the
// element-wise smoother / residual / correction arithmetic into the sparse
// product that produces it instead of running separate vector passes.
#include <cuda_runtime.h>

#include <cstdio>
#include <type_traits>
#include <vector>

#include "mgr_internal.cuh"

namespace mgr {

static constexpr unsigned FULL = 0xffffffffu;

template <class T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}

// Smoother diagonals may be stored in BF16 (diag_bf16): widened on load.
__device__ __forceinline__ float dval(float x) { return x; }
__device__ __forceinline__ double dval(double x) { return x; }
__device__ __forceinline__ float dval(__nv_bfloat16 x) { return __bfloat162float(x); }

// ----------------------------------------------------------------------------
// CSR sparse products, G lanes per row (G in 2..32), fused epilogues.
//   MODE_AX     y = A x
//   MODE_RES    y = b - A x
//   MODE_SMOOTH y = xin + dinv .* (b - A xin)          (x = xin)
//   MODE_ADD    y = y + A x
//   MODE_GRES   y[t] = b[rows[t]] - (A x)[t]           (A has one row per t)
//   MODE_RROWS  y[t] = b[rows[t]] - (A x)[rows[t]]     (a subset of A's rows)
//   MODE_RES0   y = b - A (dinv .* b)     (first l1-Jacobi sweep from zero fused in;
//                                          x = b, gathers dinv too)
//   MODE_PROL0  y = dinv .* b + A x       (prolongation onto that first sweep;
//                                          b, dinv are the fine-level vectors)
//   MODE_DRES   y = dinv .* (b - A x)     (Jacobi iteration of a triangular system)
//   MODE_DRES0  y = dinv .* (b - A (dinv .* b))   (its first iteration from
//                                          x = dinv .* b; x = b, gathers dinv)
// ----------------------------------------------------------------------------
enum { MODE_AX = 0, MODE_RES = 1, MODE_SMOOTH = 2, MODE_ADD = 3, MODE_GRES = 4, MODE_RROWS = 5,
       MODE_RES0 = 6, MODE_PROL0 = 7, MODE_DRES = 8, MODE_DRES0 = 9 };

// Lanes of a G-lane group inside its warp (G divides 32; groups are aligned).
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  return (G == 32) ? FULL : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
}

// Grid-stride over rows, one G-lane group per row, one accumulator per lane
// (loads unrolled by four); I is the offset type (int when nnz < 2^31).  All
// lanes of a group always share a row, so the shuffle mask is the group's own
// lanes.  One accumulator rather than two: on GB300 the FP64 products share a
// narrow pipe, and every extra add (merging accumulators) costs a warp
// instruction (measured on the A_uu levels: 7-17% faster).
template <class T, class X, class Y, class I, int G, int MODE, class D>
__global__ void __launch_bounds__(256)
k_spmv(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ val,
       I nr, const X* __restrict__ x, Y* __restrict__ y, const Y* __restrict__ b,
       const D* __restrict__ dinv, const int64_t* __restrict__ rows) {
  const I gid = (I)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & (G - 1);
  const I stride = ((I)gridDim.x * blockDim.x) / G;
  for (I i = gid / G; i < nr; i += stride) {
    const I row = (MODE == MODE_RROWS) ? (I)rows[i] : i;
    const I e0 = (I)rp[row], e1 = (I)rp[row + 1];
    Y acc = 0;
    I k = e0 + lane;
    if (MODE == MODE_RES0 || MODE == MODE_DRES0) {
#pragma unroll 4
      for (; k < e1; k += G) {
        const int32_t c0 = ci[k];
        acc += (Y)val[k] * ((Y)dval(ldg(dinv + c0)) * (Y)ldg(x + c0));
      }
    } else {
#pragma unroll 4
      for (; k < e1; k += G) acc += (Y)val[k] * (Y)ldg(x + ci[k]);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(group_mask<G>(), acc, o, G);
    if (lane == 0) {
      if (MODE == MODE_AX) y[i] = acc;
      else if (MODE == MODE_RES) y[i] = b[i] - acc;
      else if (MODE == MODE_SMOOTH) y[i] = (Y)x[i] + (Y)dval(dinv[i]) * (b[i] - acc);
      else if (MODE == MODE_ADD) y[i] += acc;
      else if (MODE == MODE_GRES) y[i] = b[rows[i]] - acc;
      else if (MODE == MODE_RROWS) y[i] = b[row] - acc;
      else if (MODE == MODE_RES0) y[i] = b[i] - acc;
      else if (MODE == MODE_PROL0) y[i] = (Y)dval(dinv[i]) * b[i] + acc;
      else if (MODE == MODE_DRES || MODE == MODE_DRES0) y[i] = (Y)dval(dinv[i]) * (b[i] - acc);
    }
  }
}

// The same product over an operator with shared row patterns: row i's
// columns are i + poff[pstart[pid[i]] + k], so per non-zero only the value is
// streamed (plus a 2-byte pattern id per row); the pattern table is a few KB
// and stays in cache.  Every row's sum is formed in the order of k_spmv.
template <class T, class X, class Y, class I, int G, int MODE, class D>
__global__ void __launch_bounds__(256)
k_spmv_pat(const int64_t* __restrict__ rp, const uint16_t* __restrict__ pid,
           const int32_t* __restrict__ pstart, const int32_t* __restrict__ poff,
           const T* __restrict__ val, I nr, const X* __restrict__ x, Y* __restrict__ y,
           const Y* __restrict__ b, const D* __restrict__ dinv) {
  const I gid = (I)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & (G - 1);
  const I stride = ((I)gridDim.x * blockDim.x) / G;
  for (I i = gid / G; i < nr; i += stride) {
    const I e0 = (I)rp[i], e1 = (I)rp[i + 1];
    const int32_t* po = poff + pstart[pid[i]];
    Y acc = 0;
    I k = e0 + lane;
    if (MODE == MODE_RES0 || MODE == MODE_DRES0) {
#pragma unroll 4
      for (; k < e1; k += G) {
        const I c0 = i + (I)__ldg(po + (k - e0));
        acc += (Y)val[k] * ((Y)dval(ldg(dinv + c0)) * (Y)ldg(x + c0));
      }
    } else {
#pragma unroll 4
      for (; k < e1; k += G) acc += (Y)val[k] * (Y)ldg(x + (i + (I)__ldg(po + (k - e0))));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(group_mask<G>(), acc, o, G);
    if (lane == 0) {
      if (MODE == MODE_AX) y[i] = acc;
      else if (MODE == MODE_RES) y[i] = b[i] - acc;
      else if (MODE == MODE_SMOOTH) y[i] = (Y)x[i] + (Y)dval(dinv[i]) * (b[i] - acc);
      else if (MODE == MODE_ADD) y[i] += acc;
      else if (MODE == MODE_RES0) y[i] = b[i] - acc;
      else if (MODE == MODE_PROL0) y[i] = (Y)dval(dinv[i]) * b[i] + acc;
      else if (MODE == MODE_DRES || MODE == MODE_DRES0) y[i] = (Y)dval(dinv[i]) * (b[i] - acc);
    }
  }
}

// FP32 product over an operator with shared row patterns whose values are
// also stored sliced (SELL-32): rows in slices of 32, a slice's values
// k-major (value k of the slice's row r at vsell[soff[slice] + 32 k + r],
// zero-padded to the slice's longest row).  One thread per row: a warp's
// value loads are 128 contiguous bytes, its gathers of x follow the rows,
// and each thread has its whole row's loads to issue -- no row-pointer reads
// and no cross-lane reduction.  Each row's sum runs over k in order.
// With FP16 values (VT = __half) each row's sum is multiplied by its scale.
__device__ __forceinline__ float vload(float v) { return v; }
__device__ __forceinline__ double vload(double v) { return v; }
__device__ __forceinline__ float vload(__half v) { return __half2float(v); }
template <class T, class X, class Y, int MODE, class D, class VT = T>
__global__ void __launch_bounds__(256)
k_spmv_sell(const int64_t* __restrict__ soff, const uint16_t* __restrict__ pid,
            const int32_t* __restrict__ pstart, const int32_t* __restrict__ poff,
            const VT* __restrict__ vsell, const float* __restrict__ rscale, int64_t nr,
            const X* __restrict__ x, Y* __restrict__ y, const Y* __restrict__ b,
            const D* __restrict__ dinv) {
  const int64_t npad = (nr + 31) & ~int64_t(31);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i >= nr) continue;
    const int64_t sl = i >> 5;
    const int p = pid[i];
    const int32_t* po = poff + pstart[p];
    const int len = pstart[p + 1] - pstart[p];
    const VT* v = vsell + soff[sl] + (i & 31);
    Y acc = 0;
    if (MODE == MODE_RES0 || MODE == MODE_DRES0) {
#pragma unroll 4
      for (int k = 0; k < len; k++) {
        const int64_t c = i + __ldg(po + k);
        acc += (Y)vload(v[(int64_t)k * 32]) * ((Y)dval(ldg(dinv + c)) * (Y)ldg(x + c));
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < len; k++)
        acc += (Y)vload(v[(int64_t)k * 32]) * (Y)ldg(x + (i + __ldg(po + k)));
    }
    if (std::is_same<VT, __half>::value) acc *= (Y)rscale[i];
    if (MODE == MODE_AX) y[i] = acc;
    else if (MODE == MODE_RES) y[i] = b[i] - acc;
    else if (MODE == MODE_SMOOTH) y[i] = (Y)x[i] + (Y)dval(dinv[i]) * (b[i] - acc);
    else if (MODE == MODE_ADD) y[i] += acc;
    else if (MODE == MODE_RES0) y[i] = b[i] - acc;
    else if (MODE == MODE_PROL0) y[i] = (Y)dval(dinv[i]) * b[i] + acc;
    else if (MODE == MODE_DRES || MODE == MODE_DRES0) y[i] = (Y)dval(dinv[i]) * (b[i] - acc);
  }
}

// The same over a sliced operator without row patterns: the column of each
// entry is stored beside its value (sci).  Row lengths from the row pointers.
// MODE_GRES: y[t] = b[rows[t]] - (A x)[t] (A has one row per t).
template <class T, class X, class Y, int MODE, class D>
__global__ void __launch_bounds__(256)
k_spmv_sellc(const int64_t* __restrict__ soff, const int64_t* __restrict__ rp,
             const int32_t* __restrict__ sci, const T* __restrict__ vsell, int64_t nr,
             const X* __restrict__ x, Y* __restrict__ y, const Y* __restrict__ b,
             const D* __restrict__ dinv, const int64_t* __restrict__ rows) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = soff[i >> 5] + (i & 31);
    const int len = (int)(rp[i + 1] - rp[i]);
    Y acc = 0;
    if (MODE == MODE_RES0 || MODE == MODE_DRES0) {
#pragma unroll 4
      for (int k = 0; k < len; k++) {
        const int32_t c = sci[o + (int64_t)k * 32];
        acc += (Y)vsell[o + (int64_t)k * 32] * ((Y)dval(ldg(dinv + c)) * (Y)ldg(x + c));
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < len; k++)
        acc += (Y)vsell[o + (int64_t)k * 32] * (Y)ldg(x + sci[o + (int64_t)k * 32]);
    }
    if (MODE == MODE_AX) y[i] = acc;
    else if (MODE == MODE_RES) y[i] = b[i] - acc;
    else if (MODE == MODE_SMOOTH) y[i] = (Y)x[i] + (Y)dval(dinv[i]) * (b[i] - acc);
    else if (MODE == MODE_ADD) y[i] += acc;
    else if (MODE == MODE_GRES) y[i] = b[rows[i]] - acc;
    else if (MODE == MODE_RES0) y[i] = b[i] - acc;
    else if (MODE == MODE_PROL0) y[i] = (Y)dval(dinv[i]) * b[i] + acc;
    else if (MODE == MODE_DRES || MODE == MODE_DRES0) y[i] = (Y)dval(dinv[i]) * (b[i] - acc);
  }
}

// Lanes per row from the mean row length (measured on GB300 for FP64 CSR:
// ~19 non-zeros per row run best with 2 lanes, ~34-46 with 4, ~150-210 with
// 8; with 4-byte values rows of 128 and more run best with 16 -- the headline
// A_uu V-cycle's coarse levels of 148-207 non-zeros per row: 2.92 -> 2.85 ms).
static int pick_group(int64_t nnz, int64_t nr, int vbytes = 8) {
  const double avg = nr > 0 ? (double)nnz / (double)nr : 1.0;
  int g;
  if (avg < 6) g = 1;
  else if (avg < 24) g = 2;
  else if (avg < 64) g = 4;
  else if (avg < (vbytes == 4 ? 128 : 256)) g = 8;
  else g = 16;
  // small matrices: latency-bound, so spend more lanes per row (while a row
  // still has entries for them) until about half the GPU's threads are busy
  while (g < 32 && nr * g < 152LL * 1024 && g < avg) g *= 2;
  return g;
}

template <class T, class X, class Y, class I, int MODE, class D>
static void spmv_launch_i(const int64_t* rp, const int32_t* ci, const T* val, int64_t nr,
                          int64_t nnz, const X* x, Y* y, const Y* b, const D* dinv,
                          const int64_t* rows, cudaStream_t s) {
  const int G = pick_group(nnz, nr, (int)sizeof(T));
  const int tpb = 256;
  const int64_t threads = nr * G;
  const unsigned grid = (unsigned)std::min<int64_t>((threads + tpb - 1) / tpb, 152LL * 64);
#define MGR_SPMV_CASE(g)                                                                    \
  case g:                                                                                   \
    MGR_LAUNCH k_spmv<T, X, Y, I, g, MODE, D><<<grid, tpb, 0, s>>>(rp, ci, val, (I)nr, x, y, b, \
                                                                dinv, rows);                \
    break;
  switch (G) {
    MGR_SPMV_CASE(1)
    MGR_SPMV_CASE(2)
    MGR_SPMV_CASE(4)
    MGR_SPMV_CASE(8)
    MGR_SPMV_CASE(16)
    MGR_SPMV_CASE(32)
  }
#undef MGR_SPMV_CASE
}

// D (the storage of dinv) is never deduced: it is T unless given
template <class U>
struct ident {
  using type = U;
};

template <class T, class X, class Y, int MODE, class D = T>
static void spmv_launch(const int64_t* rp, const int32_t* ci, const T* val, int64_t nr, int64_t nnz,
                        const X* x, Y* y, const Y* b, const typename ident<D>::type* dinv,
                        const int64_t* rows, cudaStream_t s) {
  if (nr <= 0) return;
  // 32-bit offsets when every index (rows x lanes, nnz + 2 x lanes) fits
  if (nnz + 64 < INT32_MAX && nr * 16 + 152LL * 64 * 256 < INT32_MAX)
    spmv_launch_i<T, X, Y, int, MODE, D>(rp, ci, val, nr, nnz, x, y, b, dinv, rows, s);
  else
    spmv_launch_i<T, X, Y, int64_t, MODE, D>(rp, ci, val, nr, nnz, x, y, b, dinv, rows, s);
}

template <class T>
static inline const T* vals(const Csr& a);
template <>
inline const double* vals<double>(const Csr& a) { return a.v; }
template <>
inline const float* vals<float>(const Csr& a) { return a.vf; }

template <class T>
static inline const T* pick(const double* d, const float* f);
template <>
inline const double* pick<double>(const double* d, const float*) { return d; }
template <>
inline const float* pick<float>(const double*, const float* f) { return f; }

// a smoother diagonal in its storage type D (FP64, FP32 or BF16)
template <class D>
static inline const D* pickd(const double* d, const float* f, const __nv_bfloat16* h);
template <>
inline const double* pickd<double>(const double* d, const float*, const __nv_bfloat16*) { return d; }
template <>
inline const float* pickd<float>(const double*, const float* f, const __nv_bfloat16*) { return f; }
template <>
inline const __nv_bfloat16* pickd<__nv_bfloat16>(const double*, const float*, const __nv_bfloat16* h) {
  return h;
}

template <class T, int MODE, class D = T>
static void spmv(const Csr& A, const T* x, T* y, const T* b, const typename ident<D>::type* dinv,
                 const int64_t* rows, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (A.vsell && A.sci && MODE != MODE_RROWS && A.nr > 0) {
      const unsigned grid = (unsigned)std::min<int64_t>((A.nr + 255) / 256, 152LL * 64);
      MGR_LAUNCH k_spmv_sellc<T, T, T, MODE, D><<<grid, 256, 0, s>>>(A.soff, A.rp, A.sci, A.vsell,
                                                                    A.nr, x, y, b, dinv, rows);
      return;
    }
    if ((A.vsell || A.vsellh) && MODE != MODE_GRES && MODE != MODE_RROWS && A.nr > 0) {
      const unsigned grid = (unsigned)std::min<int64_t>((A.nr + 255) / 256, 152LL * 64);
      if (A.vsellh)
        MGR_LAUNCH k_spmv_sell<T, T, T, MODE, D, __half><<<grid, 256, 0, s>>>(
            A.soff, A.pid, A.pstart, A.poff, A.vsellh, A.rscale, A.nr, x, y, b, dinv);
      else
        MGR_LAUNCH k_spmv_sell<T, T, T, MODE, D><<<grid, 256, 0, s>>>(
            A.soff, A.pid, A.pstart, A.poff, A.vsell, nullptr, A.nr, x, y, b, dinv);
      return;
    }
  }
  const bool pat = A.pid && MODE != MODE_GRES && MODE != MODE_RROWS && A.nr > 0 &&
                   A.nnz + 64 < INT32_MAX && A.nr * 16 + 152LL * 64 * 256 < INT32_MAX;
  if (!pat) {
    spmv_launch<T, T, T, MODE, D>(A.rp, A.ci, vals<T>(A), A.nr, A.nnz, x, y, b, dinv, rows, s);
    return;
  }
  const int G = pick_group(A.nnz, A.nr, (int)sizeof(T));
  const unsigned grid = (unsigned)std::min<int64_t>((A.nr * G + 255) / 256, 152LL * 64);
#define MGR_SPMV_PAT_CASE(g)                                                                      \
  case g:                                                                                         \
    MGR_LAUNCH k_spmv_pat<T, T, T, int, g, MODE, D><<<grid, 256, 0, s>>>(                         \
        A.rp, A.pid, A.pstart, A.poff, vals<T>(A), (int)A.nr, x, y, b, dinv);                     \
    break;
  switch (G) {
    MGR_SPMV_PAT_CASE(1)
    MGR_SPMV_PAT_CASE(2)
    MGR_SPMV_PAT_CASE(4)
    MGR_SPMV_PAT_CASE(8)
    MGR_SPMV_PAT_CASE(16)
    MGR_SPMV_PAT_CASE(32)
  }
#undef MGR_SPMV_PAT_CASE
}

void spmv64(const int64_t* rp, const int32_t* ci, const double* v, int64_t nr, int64_t nnz,
            const double* x, double* y, cudaStream_t s) {
  spmv_launch<double, double, double, MODE_AX>(rp, ci, v, nr, nnz, x, y, nullptr, nullptr, nullptr, s);
}

void spmv64_x32(const int64_t* rp, const int32_t* ci, const double* v, int64_t nr, int64_t nnz,
                const float* x, double* y, cudaStream_t s) {
  spmv_launch<double, float, double, MODE_AX>(rp, ci, v, nr, nnz, x, y, nullptr, nullptr, nullptr, s);
}

void residual64(const int64_t* rp, const int32_t* ci, const double* v, int64_t nr, int64_t nnz,
                const double* b, const double* x, double* r, cudaStream_t s) {
  spmv_launch<double, double, double, MODE_RES>(rp, ci, v, nr, nnz, x, r, b, nullptr, nullptr, s);
}

// ----------------------------------------------------------------------------
// Vector kernels
// ----------------------------------------------------------------------------
template <class T, class D>
__global__ void k_scale(const D* __restrict__ d, const T* __restrict__ b, T* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (T)dval(d[i]) * b[i];
}

template <class T>
__global__ void k_add(T* __restrict__ z, const T* __restrict__ e, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] += e[i];
}

template <class T>
__global__ void k_gather(const T* __restrict__ src, const int64_t* __restrict__ idx, int64_t n,
                         T* __restrict__ dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = src[idx[t]];
}

// z[idx[t]] += d[t] * e[t]   (d may be null: plain add)
template <class T>
__global__ void k_scatter_add(T* __restrict__ z, const int64_t* __restrict__ idx,
                              const T* __restrict__ e, const T* __restrict__ d, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    z[idx[t]] += d ? d[t] * e[t] : e[t];
}

// x = Ainv b for the dense coarsest inverse: one warp per row.
template <class T>
__global__ void k_dense_gemv(const T* __restrict__ a, int64_t n, const T* __restrict__ b, T* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) / 32) {
    T acc = 0;
    for (int64_t j = lane; j < n; j += 32) acc += a[i * n + j] * b[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) x[i] = acc;
  }
}

template <class A, class B>
__global__ void k_cast(const A* __restrict__ a, B* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (B)a[i];
}

// Point-block Jacobi (global smoother, Sec. 5.3 Remarks).
//   first sweep from zero: z = B^-1 v
//   later sweeps        : zout = zin + B^-1 (v - A zin)
// Each CTA owns BJ_BLOCKS consecutive cell blocks (their rows are consecutive,
// at most 4 per block).  Phase 1: G lanes per row form the residual of those
// rows in shared memory; phase 2: one thread per cell block applies its
// inverse (bd x bd values per block, row-major).
static constexpr int BJ_BLOCKS = 64;
template <class T, int G, bool FIRST, class D>
__global__ void __launch_bounds__(256)
k_block_jacobi(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
               const T* __restrict__ val, const int64_t* __restrict__ bstart,
               const D* __restrict__ binv, int bd, int64_t nblk, const T* __restrict__ v,
               const T* __restrict__ zin, T* __restrict__ zout) {
  __shared__ T rs[4 * BJ_BLOCKS];
  const int64_t k0 = (int64_t)blockIdx.x * BJ_BLOCKS;
  const int64_t k1 = k0 + BJ_BLOCKS < nblk ? k0 + BJ_BLOCKS : nblk;
  const int64_t r0 = bstart[k0];
  const int nrow = (int)(bstart[k1] - r0);
  if (FIRST) {
    for (int q = threadIdx.x; q < nrow; q += blockDim.x) rs[q] = v[r0 + q];
  } else {
    const int lane = threadIdx.x & (G - 1);
    for (int q = threadIdx.x / G; q < nrow; q += blockDim.x / G) {
      const int64_t i = r0 + q;
      const int64_t e1 = rp[i + 1];
      T acc = 0;
#pragma unroll 4
      for (int64_t e = rp[i] + lane; e < e1; e += G) acc += val[e] * ldg(zin + ci[e]);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(group_mask<G>(), acc, o, G);
      if (lane == 0) rs[q] = v[i] - acc;
    }
  }
  __syncthreads();
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int64_t s0 = bstart[k];
    const int b = (int)(bstart[k + 1] - s0);
    const int q0 = (int)(s0 - r0);
    const D* M = binv + (int64_t)bd * bd * k;
    for (int i = 0; i < b; i++) {
      T d = 0;
      for (int j = 0; j < b; j++) d += (T)dval(M[i * bd + j]) * rs[q0 + j];
      zout[s0 + i] = FIRST ? d : zin[s0 + i] + d;
    }
  }
}

// Multicolour point-block Gauss-Seidel: one colour's blocks (list[0..count)),
// z_b += B_b^-1 (v - A z)_b in place.  A warp per block, 8 lanes per row (at
// most 4 rows); blocks of one colour are not adjacent in A + A^T, so a warp
// reads no unknown that another warp of the launch writes.
template <class T, class D>
__global__ void __launch_bounds__(256)
k_block_gs(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ val,
           const int64_t* __restrict__ bstart, const D* __restrict__ binv, int bd,
           const int64_t* __restrict__ list, int64_t count, const T* __restrict__ v, T* z) {
  const int lane = threadIdx.x & 31, g = lane >> 3, sub = lane & 7;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < count; t += nw) {
    const int64_t k = list[t];
    const int64_t s0 = bstart[k];
    const int b = (int)(bstart[k + 1] - s0);
    T acc = 0;
    if (g < b) {
      const int64_t i = s0 + g;
      for (int64_t q = rp[i] + sub; q < rp[i + 1]; q += 8) acc += val[q] * z[ci[q]];
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    const T r = (g < b) ? v[s0 + g] - acc : (T)0;
    T rr[4];
#pragma unroll
    for (int j = 0; j < 4; j++) rr[j] = __shfl_sync(FULL, r, j * 8);
    if (lane < b) {
      const D* M = binv + (int64_t)bd * bd * k;
      T d = 0;
      for (int j = 0; j < b; j++) d += (T)dval(M[lane * bd + j]) * rr[j];
      z[s0 + lane] += d;
    }
  }
}

// Interpolation and correction of Algorithm 2: z_F += W_p e_C, z_C += e_C.
// With base != null the F part of z is zero except base (= e_F of the
// F-relaxation) and C is zero, so z is written instead: z_F = base + W_p e_C,
// z_C = e_C.
template <class T, int G>
__global__ void __launch_bounds__(256)
k_interp_correct(const int64_t* __restrict__ wrp, const int32_t* __restrict__ wci,
                 const T* __restrict__ wv, const int64_t* __restrict__ Fidx,
                 const int64_t* __restrict__ Cidx, int64_t nF, int64_t nC,
                 const T* __restrict__ eC, const T* __restrict__ base, T* __restrict__ z) {
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  const int lane = threadIdx.x & (G - 1);
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t t = gid / G; t < nF + nC; t += stride) {
    if (t < nF) {
      T acc = 0;
      for (int64_t k = wrp[t] + lane; k < wrp[t + 1]; k += G) acc += wv[k] * ldg(eC + wci[k]);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(group_mask<G>(), acc, o, G);
      if (lane == 0) {
        const int64_t d = Fidx ? Fidx[t] : t;
        if (base) z[d] = base[t] + acc;
        else z[d] += acc;
      }
    } else if (lane == 0) {
      const int64_t c = t - nF;
      const int64_t d = Cidx ? Cidx[c] : nF + c;
      if (base) z[d] = eC[c];
      else z[d] += eC[c];
    }
  }
}

static unsigned vgrid(int64_t n) { return grid_for(n, 256, 152 * 16); }

// ----------------------------------------------------------------------------
// Workspace
// ----------------------------------------------------------------------------
template <class T>
static int alloc_amg_ws(Pool& P, Amg* g) {
  if (!g) return MGR_SUCCESS;
  for (size_t k = 0; k < g->lev.size(); k++) {
    AmgLevel& L = g->lev[k];
    int64_t n = L.A.nr;
    if (k > 0) {
      L.x = P.get<T>(n);
      L.b = P.get<T>(n);
    }
    L.r = P.get<T>(n);
    L.t = P.get<T>(n);
  }
  return P.err;
}

template <class T>
static int alloc_ws(Handle* h) {
  Pool& P = h->pool;
  for (auto& L : h->lev) {
    L.z2 = P.get<T>(L.n);
    L.rF = P.get<T>(L.nF);
    L.eF = P.get<T>(L.nF);
    L.rC = P.get<T>(L.nC);
    L.eC = P.get<T>(L.nC);
    if (L.ilu1) {
      L.y1 = P.get<T>(L.n);
      L.y2 = P.get<T>(L.n);
      L.y3 = P.get<T>(L.n);
    }
    MGR_TRY(alloc_amg_ws<T>(P, L.famg));
  }
  MGR_TRY(alloc_amg_ws<T>(P, h->camg));
  return P.err;
}

int alloc_apply_workspace(Handle* h, cudaStream_t s) {
  (void)s;
  if (h->opt.precision == MGR_MIXED) {
    MGR_TRY(alloc_ws<float>(h));
    h->vin32 = h->pool.get<float>(h->n);
    h->zout32 = h->pool.get<float>(h->n);
    return h->pool.err;
  }
  return alloc_ws<double>(h);
}

// ----------------------------------------------------------------------------
// AMG V-cycle from a zero guess (one l1-Jacobi sweep down, one up)
// ----------------------------------------------------------------------------
// Levels with fewer non-zeros fold the first sweep into their sparse products;
// above it the extra gathered multiply per non-zero (FP64 pipe) costs more than
// the separate vector kernel it saves.
static constexpr int64_t FUSE_SCALE_NNZ = 2000000;
template <class T>
struct WsLevel {
  T *b, *x, *t, *r;
};

// One V-cycle on levels k.. of g; W[k'] holds the level vectors (for k' > k:
// b, x; for every non-coarsest level: t, r).  D: storage type of the l1
// diagonals read (T, or BF16 under diag_bf16).
template <class T, class D>
static void vcycle_on(Amg* g, int k, const T* b, T* x, const WsLevel<T>* W, cudaStream_t s) {
  AmgLevel& L = g->lev[k];
  const int64_t n = L.A.nr;
  if (k == (int)g->lev.size() - 1) {
    const T* inv = pick<T>(g->inv, g->invf);
    MGR_LAUNCH k_dense_gemv<T><<<grid_for(n * 32, 256), 256, 0, s>>>(inv, n, b, x);
    return;
  }
  const D* dinv = pickd<D>(L.dinv, L.dinvf, L.dinvh);
  T* t = W[k].t;
  T* r = W[k].r;
  T* cb = W[k + 1].b;
  T* cx = W[k + 1].x;
  if (L.A.nnz < FUSE_SCALE_NNZ) {
    // small level: fold t = dinv .* b into the residual and the prolongation
    spmv<T, MODE_RES0, D>(L.A, b, r, b, dinv, nullptr, s);
    spmv<T, MODE_AX>(L.R, r, cb, nullptr, nullptr, nullptr, s);
    vcycle_on<T, D>(g, k + 1, cb, cx, W, s);
    spmv<T, MODE_PROL0, D>(L.P, cx, t, b, dinv, nullptr, s);
  } else {
    MGR_LAUNCH k_scale<T, D><<<vgrid(n), 256, 0, s>>>(dinv, b, t, n);
    spmv<T, MODE_RES>(L.A, t, r, b, nullptr, nullptr, s);
    spmv<T, MODE_AX>(L.R, r, cb, nullptr, nullptr, nullptr, s);
    vcycle_on<T, D>(g, k + 1, cb, cx, W, s);
    spmv<T, MODE_ADD>(L.P, cx, t, nullptr, nullptr, nullptr, s);
  }
  spmv<T, MODE_SMOOTH, D>(L.A, t, x, b, dinv, nullptr, s);
}

// V-cycle on the level vectors W, with the diagonals in the storage the
// hierarchy was set up with
template <class T>
static void vcycle_ws(Amg* g, int k, const T* b, T* x, const WsLevel<T>* W, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (g->bf16) {
      vcycle_on<float, __nv_bfloat16>(g, k, b, x, W, s);
      return;
    }
  }
  vcycle_on<T, T>(g, k, b, x, W, s);
}

// V-cycle with the handle's level workspace
template <class T>
static void vcycle(Amg* g, int k, const T* b, T* x, cudaStream_t s) {
  WsLevel<T> W[32];
  for (size_t q = 0; q < g->lev.size() && q < 32; q++)
    W[q] = WsLevel<T>{(T*)g->lev[q].b, (T*)g->lev[q].x, (T*)g->lev[q].t, (T*)g->lev[q].r};
  vcycle_ws<T>(g, k, b, x, W, s);
}

// ---- end of the AMG V-cycle: kernels and launch rules above this line ----

// Global relaxation by point-block Jacobi or multicolour point-block
// Gauss-Seidel sweeps from zero (z = M_glo^-1 v), block inverses in storage D.
template <class T, class D>
static void block_sweeps(MgrLevel& L, const D* binv, const T* v, T* z, cudaStream_t s) {
  const int64_t n = L.n;
  const T* Av = vals<T>(L.A);
  const int bd = L.bdim;
  if (L.gs) {
    // multicolour Gauss-Seidel sweeps from zero, in place on z
    cudaMemsetAsync(z, 0, sizeof(T) * n, s);
    for (int sw = 0; sw < L.global_sweeps; sw++)
      for (int c = 0; c < L.ncolor; c++) {
        const int64_t cnt = L.coff[c + 1] - L.coff[c];
        if (cnt == 0) continue;
        const unsigned gg = (unsigned)std::min<int64_t>((cnt + 7) / 8, 152LL * 16);
        MGR_LAUNCH k_block_gs<T, D><<<gg, 256, 0, s>>>(L.A.rp, L.A.ci, Av, L.bstart, binv, bd,
                                                       L.border + L.coff[c], cnt, v, z);
      }
    return;
  }
  T* buf[2] = {((L.global_sweeps - 1) % 2 == 0) ? z : (T*)L.z2,
               ((L.global_sweeps - 1) % 2 == 0) ? (T*)L.z2 : z};
  const unsigned bgrid = (unsigned)((L.nblk + BJ_BLOCKS - 1) / BJ_BLOCKS);
  const int G = pick_group(L.A.nnz, L.A.nr);
  bool first = true;
  for (int sw = 0; sw < L.global_sweeps; sw++, first = false) {
    const T* zi = first ? nullptr : buf[(sw - 1) % 2];
    T* zo = buf[sw % 2];
#define MGR_BJ_CASE(g)                                                                             \
  case g:                                                                                          \
    if (first)                                                                                     \
      MGR_LAUNCH k_block_jacobi<T, g, true, D><<<bgrid, 256, 0, s>>>(L.A.rp, L.A.ci, Av, L.bstart, \
                 binv, bd, L.nblk, v, zi, zo);                                                     \
    else                                                                                           \
      MGR_LAUNCH k_block_jacobi<T, g, false, D><<<bgrid, 256, 0, s>>>(L.A.rp, L.A.ci, Av,          \
                 L.bstart, binv, bd, L.nblk, v, zi, zo);                                           \
    break;
    switch (G) {
      MGR_BJ_CASE(1)
      MGR_BJ_CASE(2)
      MGR_BJ_CASE(4)
      MGR_BJ_CASE(8)
      MGR_BJ_CASE(16)
      default: MGR_BJ_CASE(32)
    }
#undef MGR_BJ_CASE
  }
}

// k_interp_correct over a sliced W (FP32, one thread per F row; the C rows
// copied as there): z_F (+)= base + W e_C, z_C (+)= e_C.
template <class T>
__global__ void __launch_bounds__(256)
k_interp_correct_sell(const int64_t* __restrict__ soff, const int64_t* __restrict__ wrp,
                      const int32_t* __restrict__ sci, const T* __restrict__ sv,
                      const int64_t* __restrict__ Fidx, const int64_t* __restrict__ Cidx,
                      int64_t nF, int64_t nC, const T* __restrict__ eC, const T* __restrict__ base,
                      T* __restrict__ z) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nF + nC;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < nF) {
      const int64_t o = soff[t >> 5] + (t & 31);
      const int len = (int)(wrp[t + 1] - wrp[t]);
      T acc = 0;
#pragma unroll 4
      for (int k = 0; k < len; k++) acc += sv[o + (int64_t)k * 32] * ldg(eC + sci[o + (int64_t)k * 32]);
      const int64_t d = Fidx ? Fidx[t] : t;
      if (base) z[d] = base[t] + acc;
      else z[d] += acc;
    } else {
      const int64_t c = t - nF;
      const int64_t d = Cidx ? Cidx[c] : nF + c;
      if (base) z[d] = eC[c];
      else z[d] += eC[c];
    }
  }
}

// ----------------------------------------------------------------------------
// Algorithm 2 at level l
// ----------------------------------------------------------------------------
template <class T>
static void mgr_level(Handle* h, int l, const T* v, T* z, cudaStream_t s) {
  if (l == h->L) {
    vcycle<T>(h->camg, 0, v, z, s);
    return;
  }
  MgrLevel& L = h->lev[l];
  const int64_t n = L.n, nF = L.nF, nC = L.nC;
  const T* Av = vals<T>(L.A);
  const int64_t* Fi = L.F_is_prefix ? nullptr : L.Fidx;
  const int64_t* Ci = L.F_is_prefix ? nullptr : L.Cidx;
  bool zero = true;             // z == 0 (not materialised)
  // global relaxation z = M_glo^-1 v: sweeps from zero of point-block Jacobi
  // or of multicolour point-block Gauss-Seidel
  if (L.global_sweeps > 0 && L.nblk > 0) {
    if (L.ilu1) {
      // ILU(1) sweeps from zero: r = v - A z; y = L^-1 r and w = U^-1 y by
      // Jacobi iterations; z += w.  The last iteration writes z itself in
      // the first sweep.
      const T* di = pick<T>(L.ilu_dinv, L.ilu_dinvf);
      const int it = L.ilu_solve_sweeps;
      T* ya = (T*)L.y1;
      T* yb = (T*)L.y2;
      T* wb = (T*)L.y3;
      T* z2 = (T*)L.z2;
      for (int sw = 0; sw < L.global_sweeps; sw++) {
        const T* rr = v;
        if (sw > 0) {
          spmv<T, MODE_RES>(L.A, z, wb, v, nullptr, nullptr, s);
          rr = wb;
        }
        const T* y = rr;
        for (int t = 1; t <= it; t++) {
          T* yo = (t % 2) ? ya : yb;
          spmv<T, MODE_RES>(L.Ilo, y, yo, rr, nullptr, nullptr, s);
          y = yo;
        }
        T* last = (sw == 0) ? z : (it == 0 ? z2 : wb);   // never the buffer y is in
        if (it == 0) {
          MGR_LAUNCH k_scale<T, T><<<vgrid(n), 256, 0, s>>>(di, y, last, n);
        }
        const T* w = nullptr;
        for (int t = 1; t <= it; t++) {
          T* wo = ((it - t) % 2 == 0) ? last : z2;
          if (t == 1) spmv<T, MODE_DRES0>(L.Iup, y, wo, y, di, nullptr, s);
          else spmv<T, MODE_DRES>(L.Iup, w, wo, y, di, nullptr, s);
          w = wo;
        }
        if (sw > 0) MGR_LAUNCH k_add<T><<<vgrid(n), 256, 0, s>>>(z, last, n);
      }
    } else {
      bool done = false;
      if constexpr (std::is_same<T, float>::value) {
        if (L.bf16) {
          block_sweeps<float, __nv_bfloat16>(L, L.binvch, v, z, s);
          done = true;
        }
      }
      if (!done) block_sweeps<T, T>(L, pick<T>(L.binvc, L.binvcf), v, z, s);
    }
    zero = false;
  }
  T* rF = (T*)L.rF;
  T* eF = (T*)L.eF;
  const T* zF_only = nullptr;   // z = [e_F at F, 0 at C], not materialised
  // F-relaxation sweeps z <- z + Q M_FF^-1 Q^T (v - A z), M_FF^-1 one AMG
  // V-cycle or Jacobi (pointwise or point-block D_FF): before the coarse-grid
  // correction (Eq. MGR-pre) or after it (Eq. MGR-post)
  auto frelax = [&]() {
    for (int sw = 0; sw < L.frelax_sweeps; sw++) {
      if (zF_only) {
        cudaMemsetAsync(z, 0, sizeof(T) * n, s);
        MGR_LAUNCH k_scatter_add<T><<<vgrid(nF), 256, 0, s>>>(z, L.Fidx, eF, nullptr, nF);
        zF_only = nullptr;
        zero = false;
      }
      const T* rhs;
      if (zero) {
        if (L.F_is_prefix) {
          rhs = v;
        } else {
          MGR_LAUNCH k_gather<T><<<vgrid(nF), 256, 0, s>>>(v, L.Fidx, nF, rF);
          rhs = rF;
        }
      } else {
        spmv_launch<T, T, T, MODE_RROWS>(L.A.rp, L.A.ci, Av, nF, L.A.nnz * nF / (n > 0 ? n : 1), z,
                                         rF, v, nullptr, L.Fidx, s);
        rhs = rF;
      }
      if (L.frelax == MGR_FRELAX_AMG_VCYCLE) vcycle<T>(L.famg, 0, rhs, eF, s);
      else if (L.dff_block) spmv<T, MODE_AX>(L.Bd, rhs, eF, nullptr, nullptr, nullptr, s);
      else if (std::is_same<T, float>::value && L.bf16)
        MGR_LAUNCH k_scale<T, __nv_bfloat16><<<vgrid(nF), 256, 0, s>>>(L.dFinvh, rhs, eF, nF);
      else MGR_LAUNCH k_scale<T, T><<<vgrid(nF), 256, 0, s>>>(pick<T>(L.dFinv, L.dFinvf), rhs, eF, nF);
      if (zero) zF_only = eF;
      else MGR_LAUNCH k_scatter_add<T><<<vgrid(nF), 256, 0, s>>>(z, L.Fidx, eF, nullptr, nF);
    }
  };
  if (!L.frelax_post) frelax();
  // restrict r_C = R~ (v - A z): injection (W_r = 0), plus W_r r_F with the
  // Jacobi restriction
  T* rC = (T*)L.rC;
  T* eC = (T*)L.eC;
  if (L.restrict_jacobi) {
    if (zF_only) {
      cudaMemsetAsync(z, 0, sizeof(T) * n, s);
      MGR_LAUNCH k_scatter_add<T><<<vgrid(nF), 256, 0, s>>>(z, L.Fidx, eF, nullptr, nF);
      zF_only = nullptr;
      zero = false;
    }
    const T* rFsrc = rF;
    if (zero) {
      if (L.F_is_prefix) rFsrc = v;
      else MGR_LAUNCH k_gather<T><<<vgrid(nF), 256, 0, s>>>(v, L.Fidx, nF, rF);
      MGR_LAUNCH k_gather<T><<<vgrid(nC), 256, 0, s>>>(v, L.Cidx, nC, rC);
      cudaMemsetAsync(z, 0, sizeof(T) * n, s);
    } else {
      spmv_launch<T, T, T, MODE_RROWS>(L.A.rp, L.A.ci, Av, nF, L.A.nnz * nF / (n > 0 ? n : 1), z,
                                       rF, v, nullptr, L.Fidx, s);
      spmv_launch<T, T, T, MODE_RROWS>(L.A.rp, L.A.ci, Av, nC, L.A.nnz * nC / (n > 0 ? n : 1), z,
                                       rC, v, nullptr, L.Cidx, s);
    }
    spmv<T, MODE_ADD>(L.Wr, rFsrc, rC, nullptr, nullptr, nullptr, s);
  } else if (zF_only) {
    // z is zero outside F, so (A z)_C = A_CF z_F
    spmv<T, MODE_GRES>(L.Acf, zF_only, rC, v, nullptr, L.Cidx, s);
  } else if (zero) {
    MGR_LAUNCH k_gather<T><<<vgrid(nC), 256, 0, s>>>(v, L.Cidx, nC, rC);
    cudaMemsetAsync(z, 0, sizeof(T) * n, s);
  } else {
    spmv_launch<T, T, T, MODE_RROWS>(L.A.rp, L.A.ci, Av, nC, L.A.nnz * nC / (n > 0 ? n : 1), z,
                                     rC, v, nullptr, L.Cidx, s);
  }
  // coarse-grid correction by recursion
  mgr_level<T>(h, l + 1, rC, eC, s);
  // interpolate e = P~ e_C = [W_p e_C; e_C] and correct
  bool sliced = false;
  if constexpr (std::is_same<T, float>::value) {
    if (L.W.vsell && L.W.sci && L.W.nr == nF) {
      const unsigned g1 = (unsigned)std::min<int64_t>((nF + nC + 255) / 256, 152LL * 64);
      MGR_LAUNCH k_interp_correct_sell<T><<<g1, 256, 0, s>>>(L.W.soff, L.W.rp, L.W.sci, L.W.vsell, Fi,
                                                            Ci, nF, nC, eC, zF_only, z);
      sliced = true;
    }
  }
  const int G = sliced ? 0 : pick_group(L.W.nnz, nF);
  unsigned grid = (unsigned)std::min<int64_t>(((nF + nC) * G + 255) / 256, 152LL * 64);
  const T* wv = vals<T>(L.W);
  switch (G) {
    case 0: break;   // done over the sliced W
    case 1: MGR_LAUNCH k_interp_correct<T, 1><<<grid, 256, 0, s>>>(L.W.rp, L.W.ci, wv, Fi, Ci, nF, nC, eC, zF_only, z); break;
    case 2: MGR_LAUNCH k_interp_correct<T, 2><<<grid, 256, 0, s>>>(L.W.rp, L.W.ci, wv, Fi, Ci, nF, nC, eC, zF_only, z); break;
    case 4: MGR_LAUNCH k_interp_correct<T, 4><<<grid, 256, 0, s>>>(L.W.rp, L.W.ci, wv, Fi, Ci, nF, nC, eC, zF_only, z); break;
    case 8: MGR_LAUNCH k_interp_correct<T, 8><<<grid, 256, 0, s>>>(L.W.rp, L.W.ci, wv, Fi, Ci, nF, nC, eC, zF_only, z); break;
    case 16: MGR_LAUNCH k_interp_correct<T, 16><<<grid, 256, 0, s>>>(L.W.rp, L.W.ci, wv, Fi, Ci, nF, nC, eC, zF_only, z); break;
    default: MGR_LAUNCH k_interp_correct<T, 32><<<grid, 256, 0, s>>>(L.W.rp, L.W.ci, wv, Fi, Ci, nF, nC, eC, zF_only, z); break;
  }
  if (L.frelax_post) {
    // z is materialised by the correction
    zF_only = nullptr;
    zero = false;
    frelax();
  }
}

// Capture mgr_level over the handle's fixed buffers into a graph (once, at
// setup).  On failure the handle keeps launching the kernels directly.
int capture_apply_graph(Handle* h) {
  const bool mixed = h->opt.precision == MGR_MIXED;
  if (!mixed) {
    h->gin = h->pool.get<double>(h->n);
    h->gout = h->pool.get<double>(h->n);
    if (h->pool.err) return h->pool.err;
  }
  cudaStream_t cs;
  MGR_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    t_capturing++;
    if (mixed) mgr_level<float>(h, 0, h->vin32, h->zout32, cs);
    else mgr_level<double>(h, 0, h->gin, h->gout, cs);
    t_capturing--;
    e = cudaStreamEndCapture(cs, &graph);
  }
  if (e == cudaSuccess && graph) {
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    long long kernels = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) kernels++;
    }
    e = cudaGraphInstantiate(&h->apply_exec, graph, 0);
    if (e != cudaSuccess) h->apply_exec = nullptr;
    h->apply_nodes = kernels;
  }
  if (g_trace.on)
    fprintf(stderr, "mgr_trace apply graph: %s (%s, %lld kernel nodes)\n",
            h->apply_exec ? "captured" : "not captured, eager launches", cudaGetErrorString(e),
            (long long)h->apply_nodes);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  (void)cudaGetLastError();
  return MGR_SUCCESS;
}

// Capture one preconditioner application over the handle's fixed buffers
// (FP64: gin -> gout; MGR_MIXED: vin32 -> zout32) into an existing graph (the
// body of a conditional node of the lockstep batch graph).
// One preconditioner application over the handle's fixed buffers (FP64: gin
// -> gout; MGR_MIXED: vin32 -> zout32) launched on `s` -- used inside a
// stream capture (the lockstep batch graph's per-system branches).
int launch_apply_fixed(Handle* h, cudaStream_t s) {
  const bool mixed = h->opt.precision == MGR_MIXED;
  if (!mixed && (!h->gin || !h->gout)) return MGR_ERR_INVALID_ARG;
  if (mixed) mgr_level<float>(h, 0, h->vin32, h->zout32, s);
  else mgr_level<double>(h, 0, h->gin, h->gout, s);
  return MGR_SUCCESS;
}

int spmv_lanes(int64_t nnz, int64_t nr) { return pick_group(nnz, nr); }

int apply_mgr(Handle* h, const double* v, double* z, cudaStream_t s) {
  if (h->opt.precision == MGR_MIXED) {
    MGR_LAUNCH k_cast<double, float><<<vgrid(h->n), 256, 0, s>>>(v, h->vin32, h->n);
    if (h->apply_exec) {
      MGR_TRY_CUDA(cudaGraphLaunch(h->apply_exec, s));
      count_graph_launch(h->apply_nodes);
    } else {
      mgr_level<float>(h, 0, h->vin32, h->zout32, s);
    }
    MGR_LAUNCH k_cast<float, double><<<vgrid(h->n), 256, 0, s>>>(h->zout32, z, h->n);
  } else if (h->apply_exec) {
    MGR_TRY_CUDA(cudaMemcpyAsync(h->gin, v, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s));
    MGR_TRY_CUDA(cudaGraphLaunch(h->apply_exec, s));
    count_graph_launch(h->apply_nodes);
    MGR_TRY_CUDA(cudaMemcpyAsync(z, h->gout, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s));
  } else {
    mgr_level<double>(h, 0, v, z, s);
  }
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

int apply_mgr32(Handle* h, const float* v, float* z, cudaStream_t s) {
  mgr_level<float>(h, 0, v, z, s);
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

int apply_mgr_mixed_into(Handle* h, const double* v, float* z, cudaStream_t s) {
  MGR_LAUNCH k_cast<double, float><<<vgrid(h->n), 256, 0, s>>>(v, h->vin32, h->n);
  if (h->apply_exec) {
    MGR_TRY_CUDA(cudaGraphLaunch(h->apply_exec, s));
    count_graph_launch(h->apply_nodes);
    if (z != h->zout32)
      MGR_TRY_CUDA(cudaMemcpyAsync(z, h->zout32, sizeof(float) * h->n, cudaMemcpyDeviceToDevice, s));
  } else {
    mgr_level<float>(h, 0, h->vin32, z, s);
  }
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

int apply_vcycle64(Handle* h, Amg* g, const double* b, double* x, cudaStream_t s) {
  if (h->opt.precision == MGR_MIXED) {
    int64_t n = g->lev[0].A.nr;
    MGR_LAUNCH k_cast<double, float><<<vgrid(n), 256, 0, s>>>(b, h->vin32, n);
    vcycle<float>(g, 0, h->vin32, h->zout32, s);
    MGR_LAUNCH k_cast<float, double><<<vgrid(n), 256, 0, s>>>(h->zout32, x, n);
  } else {
    vcycle<double>(g, 0, b, x, s);
  }
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}


// ----------------------------------------------------------------------------
// V-cycle with caller-provided workspace (used by the allocation-free entry
// point in noalloc.cu).  The same vcycle_on<T> as mgr_vcycle; the level vectors
// t, r (and b, x below the top level) are carved from `ws`, each 256-byte
// aligned.  Every workspace vector is written before it is read.
// ----------------------------------------------------------------------------
static size_t ws_align(size_t b) { return (b + 255) & ~size_t(255); }

size_t vcycle_ws_bytes(Handle* h, Amg* g) {
  const size_t vb = (h->opt.precision == MGR_MIXED) ? sizeof(float) : sizeof(double);
  size_t total = 0;
  for (size_t k = 0; k < g->lev.size(); k++) {
    const size_t n = (size_t)g->lev[k].A.nr;
    const bool last = k + 1 == g->lev.size();
    if (k > 0) total += 2 * ws_align(n * vb);          // b, x
    if (!last) total += 2 * ws_align(n * vb);          // t, r
  }
  if (h->opt.precision == MGR_MIXED) total += 2 * ws_align((size_t)g->lev[0].A.nr * sizeof(float));
  return total;
}

template <class T>
static void carve(Amg* g, unsigned char*& p, std::vector<WsLevel<T>>& W) {
  W.resize(g->lev.size());
  for (size_t k = 0; k < g->lev.size(); k++) {
    const size_t n = (size_t)g->lev[k].A.nr;
    const bool last = k + 1 == g->lev.size();
    W[k] = WsLevel<T>{nullptr, nullptr, nullptr, nullptr};
    if (k > 0) {
      W[k].b = (T*)p; p += ws_align(n * sizeof(T));
      W[k].x = (T*)p; p += ws_align(n * sizeof(T));
    }
    if (!last) {
      W[k].t = (T*)p; p += ws_align(n * sizeof(T));
      W[k].r = (T*)p; p += ws_align(n * sizeof(T));
    }
  }
}

int apply_vcycle64_ws(Handle* h, Amg* g, const double* b, double* x, void* ws, cudaStream_t s) {
  unsigned char* p = (unsigned char*)ws;
  if (h->opt.precision == MGR_MIXED) {
    std::vector<WsLevel<float>> W;
    carve<float>(g, p, W);
    const int64_t n = g->lev[0].A.nr;
    float* b32 = (float*)p; p += ws_align((size_t)n * sizeof(float));
    float* x32 = (float*)p; p += ws_align((size_t)n * sizeof(float));
    MGR_LAUNCH k_cast<double, float><<<vgrid(n), 256, 0, s>>>(b, b32, n);
    vcycle_ws<float>(g, 0, b32, x32, W.data(), s);
    MGR_LAUNCH k_cast<float, double><<<vgrid(n), 256, 0, s>>>(x32, x, n);
  } else {
    std::vector<WsLevel<double>> W;
    carve<double>(g, p, W);
    vcycle_ws<double>(g, 0, b, x, W.data(), s);
  }
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

}  // namespace mgr
