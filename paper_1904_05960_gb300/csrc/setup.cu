// Device setup of the MGR and AMG hierarchies.
//
// Compiled with -fmad=false, and every product / sum that feeds a later
// integer decision (strength, PMIS, truncation, dropping, sparsity patterns) is
// written with explicit round-to-nearest intrinsics, one rounding per multiply
// and per add, in ascending inner-index order.  With that rule the integer
// outputs of the setup (C/F marks, strength graphs, CSR patterns of P, R, RAP,
// W_p, S_l) are a deterministic function of the input, independent of the
// thread schedule.
//
// Paper map (Bui et al., Sec. 5-6):
//   C/F split per level from field labels ........ Sec. 5.1, Sec. 5.3
//   W_p = -D_FF^-1 A_FC, W_r = 0 .................. Eq. "injective_rp"
//   S = A_CC - G(A_CF D_FF^-1 A_FC) ............... Eq. "drop_operator",
//                                                   Eqs. "coarse_grid_flow_sparse",
//                                                   "coarse_grid_pressure"
//   point-block global smoother blocks ............ Sec. 5.3 Remarks
//   AMG: unknown-approach strength, PMIS, direct
//   interpolation, Galerkin RAP, dense coarsest ... Sec. 6 solver settings
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cmath>
#include <mutex>
#include <thread>

#include "mgr_internal.cuh"

namespace mgr {

static constexpr unsigned FULL = 0xffffffffu;
static constexpr int LU_CAP = 4096;

// ============================================================================
// Exclusive scan (int64): out[i] = sum_{j<i} in[j] for i <= n (out[n] = total)
// ============================================================================
static constexpr int SCAN_TPB = 1024;
static constexpr int SCAN_TILE = 2 * SCAN_TPB;

__device__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t s = (lane < nw) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;
  }
  __syncthreads();
  int64_t pre = (wid > 0 ? wsum[wid - 1] : 0) + x - v;
  *total = wsum[nw - 1];
  __syncthreads();
  return pre;
}

__global__ void k_scan_tile(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ out,
                            int64_t* __restrict__ bsum) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + 2 * threadIdx.x;
  int64_t a = (base < n) ? in[base] : 0;
  int64_t b = (base + 1 < n) ? in[base + 1] : 0;
  int64_t tot;
  int64_t pre = block_excl_scan(a + b, &tot);
  if (base <= n) out[base] = pre;
  if (base + 1 <= n) out[base + 1] = pre + a;
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ off) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + 2 * threadIdx.x;
  int64_t o = off[blockIdx.x];
  if (base <= n) out[base] += o;
  if (base + 1 <= n) out[base + 1] += o;
}

int scan_exclusive(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, Pool& tmp) {
  int64_t m = n + 1;
  int64_t nb = (m + SCAN_TILE - 1) / SCAN_TILE;
  int64_t* bsum = tmp.get<int64_t>(nb);
  if (!bsum) return tmp.err;
  MGR_LAUNCH k_scan_tile<<<(unsigned)nb, SCAN_TPB, 0, s>>>(in, n, out, bsum);
  if (nb > 1) {
    int64_t* boff = tmp.get<int64_t>(nb + 1);
    if (!boff) return tmp.err;
    MGR_TRY(scan_exclusive(bsum, boff, nb, s, tmp));
    MGR_LAUNCH k_scan_add<<<(unsigned)nb, SCAN_TPB, 0, s>>>(out, n, boff);
  }
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

// scan counts -> row pointer, return total on the host
static int rowptr_from_counts(const int64_t* cnt, int64_t* rp, int64_t n, int64_t* total,
                              cudaStream_t s, Pool& tmp) {
  MGR_TRY(scan_exclusive(cnt, rp, n, s, tmp));
  return read_back(total, rp + n, s);
}

__device__ inline void dev_fail(int* err, int code) { atomicCAS(err, DEV_OK, code); }

// Magnitude and sign tests on the IEEE bit pattern (integer pipe; the FP64
// pipe of GB300 is narrow).  For non-NaN x, y: |x| > |y| exactly when
// absbits(x) > absbits(y); x < 0 exactly when the sign bit is set and x != 0.
__device__ __forceinline__ uint64_t absbits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool is_neg(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b >> 63) && (b << 1);
}
__device__ __forceinline__ bool is_pos(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  return !(b >> 63) && b;
}

static int check_dev_err(int* derr, cudaStream_t s) {
  int e = 0;
  MGR_TRY(read_back(&e, derr, s));
  if (e == DEV_ZERO_DIAG) return MGR_ERR_ZERO_DIAG;
  if (e == DEV_BAD_ARG) return MGR_ERR_INVALID_ARG;
  if (e != DEV_OK) return MGR_ERR_CUDA;
  return MGR_SUCCESS;
}

// ============================================================================
// Generic CSR kernels
// ============================================================================
static inline unsigned nblocks(int64_t n, int tpb) {
  int64_t g = (n + tpb - 1) / tpb;
  return (unsigned)(g < 1 ? 1 : g);
}

// Row subset and column relabelling: out = A[rows, cols] with colmap[j] the new
// index of column j (monotone in j) or -1.  Warp per row; ballots keep the
// column order.
template <bool FILL>
__global__ void __launch_bounds__(256)
k_extract(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
          const double* __restrict__ v, const int64_t* __restrict__ rows, int64_t nrows,
          const int32_t* __restrict__ colmap, int64_t* __restrict__ cnt_or_rp,
          int32_t* __restrict__ oci, double* __restrict__ ov) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int64_t t = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); t < nrows;
       t += (int64_t)gridDim.x * wpb) {
    const int64_t r = rows ? rows[t] : t;
    int64_t o = FILL ? cnt_or_rp[t] : 0;
    for (int64_t k0 = rp[r]; k0 < rp[r + 1]; k0 += 32) {
      const int64_t k = k0 + lane;
      int32_t c = -1;
      if (k < rp[r + 1]) c = colmap[ci[k]];
      const unsigned bal = __ballot_sync(FULL, c >= 0);
      if (FILL && c >= 0) {
        const int64_t d = o + __popc(bal & ((1u << lane) - 1u));
        oci[d] = c;
        ov[d] = v[k];
      }
      o += __popc(bal);
    }
    if (!FILL && lane == 0) cnt_or_rp[t] = o;
  }
}

static int csr_alloc(Pool& P, Csr& a, int64_t nr, int64_t nc, int64_t nnz) {
  a.nr = nr;
  a.nc = nc;
  a.nnz = nnz;
  a.rp = P.get<int64_t>(nr + 1);
  a.ci = P.get<int32_t>(nnz);
  a.v = P.get<double>(nnz);
  return P.err;
}

static int extract(Pool& P, Pool& tmp, const Csr& A, const int64_t* rows, int64_t nrows,
                   const int32_t* colmap, int64_t ncols, Csr& out, cudaStream_t s) {
  int64_t* cnt = tmp.get<int64_t>(nrows + 1);
  if (!cnt) return tmp.err;
  out.nr = nrows;
  out.nc = ncols;
  out.rp = P.get<int64_t>(nrows + 1);
  if (!out.rp) return P.err;
  MGR_LAUNCH k_extract<false><<<grid_for(nrows, 8, 152 * 16), 256, 0, s>>>(A.rp, A.ci, A.v, rows, nrows, colmap, cnt,
                                                                  nullptr, nullptr);
  MGR_TRY(rowptr_from_counts(cnt, out.rp, nrows, &out.nnz, s, tmp));
  out.ci = P.get<int32_t>(out.nnz);
  out.v = P.get<double>(out.nnz);
  if (P.err) return P.err;
  MGR_LAUNCH k_extract<true><<<grid_for(nrows, 8, 152 * 16), 256, 0, s>>>(A.rp, A.ci, A.v, rows, nrows, colmap,
                                                                 out.rp, out.ci, out.v);
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

static int copy_csr(Pool& P, const Csr& a, Csr& b, cudaStream_t s) {
  MGR_TRY(csr_alloc(P, b, a.nr, a.nc, a.nnz));
  MGR_TRY_CUDA(cudaMemcpyAsync(b.rp, a.rp, sizeof(int64_t) * (a.nr + 1), cudaMemcpyDeviceToDevice, s));
  MGR_TRY_CUDA(cudaMemcpyAsync(b.ci, a.ci, sizeof(int32_t) * a.nnz, cudaMemcpyDeviceToDevice, s));
  MGR_TRY_CUDA(cudaMemcpyAsync(b.v, a.v, sizeof(double) * a.nnz, cudaMemcpyDeviceToDevice, s));
  return MGR_SUCCESS;
}

// ============================================================================
// Deterministic sparse matrix product C = A * B
//   symbolic: one warp per output row; the candidate columns (union of the B
//   rows selected by the A row) are marked in a shared-memory bitmap window of
//   SPG_WBITS columns and extracted in ascending order.
//   numeric : one warp per output row; the A entries are taken one at a time in
//   ascending order and the lanes add a_ik * b_kj into distinct output slots,
//   so every entry is summed over ascending k from 0.0 exactly as a sequential
//   Gustavson product would.
// ============================================================================
static constexpr int SPG_WARPS = 8;
static constexpr int SPG_WORDS = 1024;                 // 32768 columns per window
static constexpr int64_t SPG_WBITS = 32LL * SPG_WORDS;
static constexpr int SPG_HASH = 2048;                  // hash slots per warp (8 KB)
static constexpr int SPG_HASH_UB = SPG_HASH / 2;       // rows with at most this many products

// Row i of the pattern by bitmap windows: the candidate columns are marked in
// a shared-memory bitmap window of SPG_WBITS columns and extracted in
// ascending order, window by window over the row's column span.
template <bool FILL>
__device__ __forceinline__ int64_t sym_row_bitmap(uint32_t* bm, const int32_t* __restrict__ aci,
                                                  int64_t a0, int64_t a1,
                                                  const int64_t* __restrict__ brp,
                                                  const int32_t* __restrict__ bci,
                                                  int32_t* __restrict__ cci, int64_t out0) {
  const int lane = threadIdx.x & 31;
  int32_t lo = INT32_MAX, hi = -1;
  for (int64_t t = a0 + lane; t < a1; t += 32) {
    int32_t k = (int32_t)aci[t];
    int64_t b0 = brp[k], b1 = brp[k + 1];
    if (b1 > b0) {
      lo = min(lo, bci[b0]);
      hi = max(hi, bci[b1 - 1]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(FULL, lo, o));
    hi = max(hi, __shfl_xor_sync(FULL, hi, o));
  }
  int64_t running = 0;
  for (int64_t w0 = lo; hi >= 0 && w0 <= hi; w0 += SPG_WBITS) {
    int64_t wend = (hi - w0) / 32 + 1;           // words that can hold bits
    if (wend > SPG_WORDS) wend = SPG_WORDS;
    for (int q = lane; q < wend; q += 32) bm[q] = 0u;
    __syncwarp();
    const int64_t w1 = w0 + SPG_WBITS;
    for (int64_t t = a0 + lane; t < a1; t += 32) {
      int32_t k = (int32_t)aci[t];
      for (int64_t e = brp[k]; e < brp[k + 1]; e++) {
        int64_t j = bci[e];
        if (j >= w0 && j < w1) {
          int64_t off = j - w0;
          atomicOr(&bm[off >> 5], 1u << (off & 31));
        }
      }
    }
    __syncwarp();
    for (int64_t q0 = 0; q0 < wend; q0 += 32) {
      int64_t q = q0 + lane;
      uint32_t word = (q < wend) ? bm[q] : 0u;
      int c = __popc(word);
      int x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
      }
      int tot = __shfl_sync(FULL, x, 31);
      if (FILL) {
        int64_t pos = out0 + running + (x - c);
        while (word) {
          int b = __ffs(word) - 1;
          word &= word - 1;
          cci[pos++] = (int32_t)(w0 + 32 * q + b);
        }
      }
      running += tot;
    }
    __syncwarp();
  }
  return running;
}

// Row i of the pattern by a shared-memory hash set (rows with at most
// SPG_HASH_UB products, whose columns may span the whole matrix): insert
// every product's column into an open-addressing table of 2^lg >= 2 ub
// slots, compact the distinct columns to the front and sort them ascending
// (bitonic, in the warp).  The set of columns, hence the pattern, is the one
// the bitmap path finds.
template <bool FILL>
__device__ __forceinline__ int64_t sym_row_hash(int32_t* ht, int lg, const int32_t* __restrict__ aci,
                                                int64_t a0, int64_t a1,
                                                const int64_t* __restrict__ brp,
                                                const int32_t* __restrict__ bci,
                                                int32_t* __restrict__ cci, int64_t out0) {
  const int lane = threadIdx.x & 31;
  const int size = 1 << lg;
  const uint32_t mask = (uint32_t)size - 1u;
  for (int q = lane; q < size; q += 32) ht[q] = -1;
  __syncwarp();
  for (int64_t t = a0 + lane; t < a1; t += 32) {
    const int32_t k = (int32_t)aci[t];
    for (int64_t e = brp[k]; e < brp[k + 1]; e++) {
      const int32_t j = bci[e];
      uint32_t h = ((uint32_t)j * 0x9E3779B1u) >> (32 - lg);
      for (;;) {
        const int32_t old = atomicCAS(&ht[h], -1, j);
        if (old == -1 || old == j) break;
        h = (h + 1u) & mask;
      }
    }
  }
  __syncwarp();
  // compact the occupied slots to the front (in place: every lane reads its
  // slot of a 32-slot chunk before any lane writes, and writes land below)
  int d = 0;
  for (int q0 = 0; q0 < size; q0 += 32) {
    const int32_t v = ht[q0 + lane];
    const unsigned bal = __ballot_sync(FULL, v != -1);
    __syncwarp();
    if (v != -1) ht[d + __popc(bal & ((1u << lane) - 1u))] = v;
    d += __popc(bal);
    __syncwarp();
  }
  if (FILL && d > 0) {
    int P = 1;
    while (P < d) P <<= 1;
    for (int q = d + lane; q < P; q += 32) ht[q] = INT32_MAX;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int i = lane; i < P; i += 32) {
          const int partner = i ^ jj;
          if (partner > i) {
            const int32_t a = ht[i], b = ht[partner];
            const bool up = (i & k) == 0;
            if ((a > b) == up) {
              ht[i] = b;
              ht[partner] = a;
            }
          }
        }
        __syncwarp();
      }
    for (int q = lane; q < d; q += 32) cci[out0 + q] = ht[q];
    __syncwarp();
  }
  return d;
}

// Deterministic sparse matrix product C = A * B, symbolic part: one warp per
// output row, by hash set for rows with few products and by bitmap windows
// otherwise; FILL writes the row's columns at cnt_or_rp[i] (and its length to
// cnt_out[i] if given), else cnt_or_rp[i] = the row's length.
//   numeric : one warp per output row; the A entries are taken one at a time in
//   ascending order and the lanes add a_ik * b_kj into distinct output slots,
//   so every entry is summed over ascending k from 0.0 exactly as a sequential
//   Gustavson product would.
template <bool FILL>
__global__ void __launch_bounds__(SPG_WARPS * 32)
k_spgemm_symbolic(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci, int64_t nr,
                  const int64_t* __restrict__ brp, const int32_t* __restrict__ bci,
                  int64_t* __restrict__ cnt_or_rp, int32_t* __restrict__ cci,
                  int64_t* __restrict__ cnt_out) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* bm = smem + wid * SPG_HASH;
  for (int64_t i = (int64_t)blockIdx.x * SPG_WARPS + wid; i < nr; i += (int64_t)gridDim.x * SPG_WARPS) {
    const int64_t a0 = arp[i], a1 = arp[i + 1];
    int64_t ub = 0;
    for (int64_t t = a0 + lane; t < a1; t += 32) {
      const int32_t k = aci[t];
      ub += brp[k + 1] - brp[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ub += __shfl_xor_sync(FULL, ub, o);
    const int64_t out0 = FILL ? cnt_or_rp[i] : 0;
    int64_t len;
    if (ub <= SPG_HASH_UB) {
      int lg = 6;
      while ((1LL << lg) < 2 * ub) lg++;
      len = sym_row_hash<FILL>((int32_t*)bm, lg, aci, a0, a1, brp, bci, cci, out0);
    } else {
      len = sym_row_bitmap<FILL>(bm, aci, a0, a1, brp, bci, cci, out0);
    }
    if (!FILL && lane == 0) cnt_or_rp[i] = len;
    if (FILL && cnt_out && lane == 0) cnt_out[i] = len;
  }
}

// Product count of each output row, sum over k in A's row of nnz(B_k): an
// upper bound of the row's distinct columns.
__global__ void k_spgemm_ub(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci, int64_t nr,
                            const int64_t* __restrict__ brp, int64_t* __restrict__ ub) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < nr; i += (int64_t)gridDim.x * wpb) {
    int64_t u = 0;
    for (int64_t t = arp[i] + lane; t < arp[i + 1]; t += 32) {
      const int32_t k = aci[t];
      u += brp[k + 1] - brp[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(FULL, u, o);
    if (lane == 0) ub[i] = u;
  }
}

// Rows written at upper-bound offsets, moved to their compact offsets; warp
// per row.
__global__ void k_compact_rows(const int64_t* __restrict__ srp, const int32_t* __restrict__ sci, int64_t nr,
                               const int64_t* __restrict__ drp, int32_t* __restrict__ dci) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < nr; i += (int64_t)gridDim.x * wpb) {
    const int64_t s0 = srp[i], d0 = drp[i], m = drp[i + 1] - d0;
    for (int64_t q = lane; q < m; q += 32) dci[d0 + q] = sci[s0 + q];
  }
}

__device__ inline int64_t lower_bound_i32(const int32_t* a, int64_t n, int32_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256)
k_spgemm_numeric(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                 const double* __restrict__ av, int64_t nr, const int64_t* __restrict__ brp,
                 const int32_t* __restrict__ bci, const double* __restrict__ bv,
                 const int64_t* __restrict__ crp, const int32_t* __restrict__ cci,
                 double* __restrict__ cv) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * wpb + wid; i < nr; i += (int64_t)gridDim.x * wpb) {
    const int64_t c0 = crp[i], m = crp[i + 1] - c0;
    for (int64_t q = lane; q < m; q += 32) cv[c0 + q] = 0.0;
    __syncwarp();
    for (int64_t t = arp[i]; t < arp[i + 1]; t++) {
      const int32_t k = aci[t];
      const double a = av[t];
      for (int64_t e = brp[k] + lane; e < brp[k + 1]; e += 32) {
        int64_t pos = c0 + lower_bound_i32(cci + c0, m, bci[e]);
        cv[pos] = __dadd_rn(cv[pos], __dmul_rn(a, bv[e]));
      }
      __syncwarp();
    }
  }
}

// Thread per output row: the same per-entry order (ascending k) with the A
// row walked sequentially by one thread; used when B's rows are short (fewer
// lanes would be busy in the warp version).
__global__ void __launch_bounds__(256)
k_spgemm_numeric_thread(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                        const double* __restrict__ av, int64_t nr, const int64_t* __restrict__ brp,
                        const int32_t* __restrict__ bci, const double* __restrict__ bv,
                        const int64_t* __restrict__ crp, const int32_t* __restrict__ cci,
                        double* __restrict__ cv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  const int64_t c0 = crp[i], m = crp[i + 1] - c0;
  const int32_t* cols = cci + c0;
  double* out = cv + c0;
  for (int64_t q = 0; q < m; q++) out[q] = 0.0;
  for (int64_t t = arp[i]; t < arp[i + 1]; t++) {
    const int32_t k = aci[t];
    const double a = av[t];
    const int64_t e0 = brp[k], e1 = brp[k + 1];
    if (e0 == e1) continue;
    // B row k and the output row are both ascending: each search starts
    // where the previous one ended
    int64_t pos = 0;
    for (int64_t e = e0; e < e1; e++) {
      pos += lower_bound_i32(cols + pos, m - pos, bci[e]);
      out[pos] = __dadd_rn(out[pos], __dmul_rn(a, bv[e]));
    }
  }
}

// Warp per output row, lane-dense: with LPG = the row's longest B row rounded
// up to a power of two (<= 32), the warp takes 32/LPG consecutive A entries at
// a time, one lane per product.  Products that land on the same output slot in
// one step are found with __match_any_sync and added by the lowest such lane in
// lane order, which is ascending k; every other lane adds its own product.  So
// each entry is the same ascending-k sum from 0.0 as the sequential product,
// and the FP64 adds run on all lanes at once.  The output row is staged in
// shared memory when it has at most GRP_CAP entries; a row whose longest B row
// exceeds 32 takes the one-B-row-at-a-time path.
static constexpr int GRP_CAP = 512;
static constexpr int GRP_WARPS = 4;
struct GrpWarp {
  int32_t cols[GRP_CAP];
  double acc[GRP_CAP];
  double lval[32];
};

__global__ void __launch_bounds__(GRP_WARPS * 32)
k_spgemm_numeric_grp(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                     const double* __restrict__ av, int64_t nr, const int64_t* __restrict__ brp,
                     const int32_t* __restrict__ bci, const double* __restrict__ bv,
                     const int64_t* __restrict__ crp, const int32_t* __restrict__ cci,
                     double* __restrict__ cv) {
  __shared__ GrpWarp sh[GRP_WARPS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  GrpWarp& W = sh[wid];
  for (int64_t i = (int64_t)blockIdx.x * GRP_WARPS + wid; i < nr; i += (int64_t)gridDim.x * GRP_WARPS) {
    const int64_t c0 = crp[i];
    const int m = (int)(crp[i + 1] - c0);
    const int64_t a0 = arp[i], a1 = arp[i + 1];
    int longest = 0;
    for (int64_t t = a0 + lane; t < a1; t += 32) {
      const int32_t k = aci[t];
      longest = max(longest, (int)(brp[k + 1] - brp[k]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) longest = max(longest, __shfl_xor_sync(FULL, longest, o));
    const bool staged = m <= GRP_CAP;
    const int32_t* cols = staged ? W.cols : cci + c0;
    double* acc = staged ? W.acc : cv + c0;
    for (int q = lane; q < m; q += 32) {
      if (staged) W.cols[q] = cci[c0 + q];
      acc[q] = 0.0;
    }
    __syncwarp();
    if (longest > 32) {
      for (int64_t t = a0; t < a1; t++) {
        const int32_t k = aci[t];
        const double a = av[t];
        for (int64_t e = brp[k] + lane; e < brp[k + 1]; e += 32) {
          const int pos = (int)lower_bound_i32(cols, m, bci[e]);
          acc[pos] = __dadd_rn(acc[pos], __dmul_rn(a, bv[e]));
        }
        __syncwarp();
      }
    } else {
      int sh2 = 0;
      while ((1 << sh2) < longest) sh2++;
      const int groups = 32 >> sh2;
      const int g = lane >> sh2, e = lane & ((1 << sh2) - 1);
      for (int64_t t0 = a0; t0 < a1; t0 += groups) {
        const int64_t t = t0 + g;
        bool valid = false;
        int pos = 0;
        double prod = 0.0;
        if (t < a1) {
          const int32_t k = aci[t];
          const int64_t eb = brp[k];
          if (e < brp[k + 1] - eb) {
            prod = __dmul_rn(av[t], bv[eb + e]);
            pos = (int)lower_bound_i32(cols, m, bci[eb + e]);
            valid = true;
          }
        }
        W.lval[lane] = prod;
        const unsigned grp = __match_any_sync(FULL, valid ? pos : -1 - lane);
        __syncwarp();
        if (valid && lane == __ffs(grp) - 1) {
          double x = acc[pos];
          for (unsigned mm = grp; mm; mm &= mm - 1) x = __dadd_rn(x, W.lval[__ffs(mm) - 1]);
          acc[pos] = x;
        }
        __syncwarp();
      }
    }
    if (staged)
      for (int q = lane; q < m; q += 32) cv[c0 + q] = W.acc[q];
    __syncwarp();
  }
}

// Pattern of C = A * B (C.v stays null; A.v and B.v are not read).
static int spgemm_pattern(Pool& P, Pool& tmp, const Csr& A, const Csr& B, Csr& C, cudaStream_t s) {
  C.nr = A.nr;
  C.nc = B.nc;
  C.v = nullptr;
  C.rp = P.get<int64_t>(A.nr + 1);
  int64_t* cnt = tmp.get<int64_t>(A.nr + 1);
  if (P.err || tmp.err) return P.err ? P.err : tmp.err;
  const size_t sm = sizeof(uint32_t) * SPG_HASH * SPG_WARPS;
  // once per process (setups may run concurrently on several host threads)
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&] {
    attr_err = cudaFuncSetAttribute(k_spgemm_symbolic<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(k_spgemm_symbolic<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  MGR_TRY_CUDA(attr_err);
  unsigned g = grid_for(A.nr, SPG_WARPS, 152 * 16);
  // One bitmap pass: rows are written at upper-bound offsets (the product
  // counts) with their exact lengths, then moved to compact offsets.  When the
  // upper bounds would take more than SPG_UB_BYTES, count first and fill
  // exactly (two bitmap passes).
  static constexpr int64_t SPG_UB_BYTES = 2LL << 30;
  int64_t* ubrp = tmp.get<int64_t>(A.nr + 1);
  if (tmp.err) return tmp.err;
  MGR_LAUNCH k_spgemm_ub<<<grid_for(A.nr, 8, 152 * 16), 256, 0, s>>>(A.rp, A.ci, A.nr, B.rp, cnt);
  int64_t ubtot = 0;
  MGR_TRY(rowptr_from_counts(cnt, ubrp, A.nr, &ubtot, s, tmp));
  if (ubtot * (int64_t)sizeof(int32_t) <= SPG_UB_BYTES) {
    int32_t* ubci = tmp.get<int32_t>(ubtot);
    if (tmp.err) return tmp.err;
    MGR_LAUNCH k_spgemm_symbolic<true><<<g, SPG_WARPS * 32, sm, s>>>(A.rp, A.ci, A.nr, B.rp, B.ci, ubrp, ubci, cnt);
    MGR_TRY(rowptr_from_counts(cnt, C.rp, A.nr, &C.nnz, s, tmp));
    C.ci = P.get<int32_t>(C.nnz);
    if (P.err) return P.err;
    MGR_LAUNCH k_compact_rows<<<grid_for(A.nr, 8, 152 * 16), 256, 0, s>>>(ubrp, ubci, A.nr, C.rp, C.ci);
    MGR_TRY_CUDA(cudaGetLastError());
    tmp.release(ubci, s);
    return MGR_SUCCESS;
  }
  MGR_LAUNCH k_spgemm_symbolic<false><<<g, SPG_WARPS * 32, sm, s>>>(A.rp, A.ci, A.nr, B.rp, B.ci, cnt, nullptr,
                                                                    nullptr);
  MGR_TRY(rowptr_from_counts(cnt, C.rp, A.nr, &C.nnz, s, tmp));
  C.ci = P.get<int32_t>(C.nnz);
  if (P.err) return P.err;
  MGR_LAUNCH k_spgemm_symbolic<true><<<g, SPG_WARPS * 32, sm, s>>>(A.rp, A.ci, A.nr, B.rp, B.ci, C.rp, C.ci,
                                                                   nullptr);
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

static int spgemm(Pool& P, Pool& tmp, const Csr& A, const Csr& B, Csr& C, cudaStream_t s) {
  MGR_TRY(spgemm_pattern(P, tmp, A, B, C, s));
  C.v = P.get<double>(C.nnz);
  if (P.err) return P.err;
  if (B.nr > 0 && B.nnz < 12 * B.nr)
    MGR_LAUNCH k_spgemm_numeric_grp<<<grid_for(A.nr, GRP_WARPS, 152 * 32), GRP_WARPS * 32, 0, s>>>(
        A.rp, A.ci, A.v, A.nr, B.rp, B.ci, B.v, C.rp, C.ci, C.v);
  else
    MGR_LAUNCH k_spgemm_numeric<<<grid_for(A.nr, 8, 152 * 16), 256, 0, s>>>(
        A.rp, A.ci, A.v, A.nr, B.rp, B.ci, B.v, C.rp, C.ci, C.v);
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

// ============================================================================
// Transpose with rows ordered by ascending original row index
// ============================================================================
__global__ void k_count_cols(const int32_t* __restrict__ ci, int64_t nnz, int64_t* __restrict__ cnt) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd((unsigned long long*)&cnt[ci[k]], 1ull);
}

__global__ void k_transpose_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ v, int64_t nr,
                                 const int64_t* __restrict__ trp, int64_t* __restrict__ cursor,
                                 int32_t* __restrict__ tci, double* __restrict__ tv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
    int32_t c = ci[k];
    int64_t d = trp[c] + (int64_t)atomicAdd((unsigned long long*)&cursor[c], 1ull);
    tci[d] = (int32_t)i;
    if (tv) tv[d] = v[k];
  }
}

__global__ void k_sort_rows(const int64_t* __restrict__ rp, int64_t nr, int32_t* __restrict__ ci,
                            double* __restrict__ v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  int64_t b = rp[i], e = rp[i + 1];
  for (int64_t k = b + 1; k < e; k++) {
    int32_t c = ci[k];
    double x = v ? v[k] : 0.0;
    int64_t q = k - 1;
    while (q >= b && ci[q] > c) {
      ci[q + 1] = ci[q];
      if (v) v[q + 1] = v[q];
      q--;
    }
    ci[q + 1] = c;
    if (v) v[q + 1] = x;
  }
}

static int transpose(Pool& P, Pool& tmp, const Csr& A, Csr& T, bool values, bool sorted,
                     cudaStream_t s) {
  T.nr = A.nc;
  T.nc = A.nr;
  T.nnz = A.nnz;
  T.rp = P.get<int64_t>(A.nc + 1);
  T.ci = P.get<int32_t>(A.nnz);
  T.v = values ? P.get<double>(A.nnz) : nullptr;
  int64_t* cnt = tmp.get<int64_t>(A.nc + 1);
  int64_t* cur = tmp.get<int64_t>(A.nc + 1);
  if (P.err || tmp.err) return P.err ? P.err : tmp.err;
  MGR_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (A.nc + 1), s));
  MGR_TRY_CUDA(cudaMemsetAsync(cur, 0, sizeof(int64_t) * (A.nc + 1), s));
  MGR_LAUNCH k_count_cols<<<grid_for(A.nnz, 256), 256, 0, s>>>(A.ci, A.nnz, cnt);
  MGR_TRY(scan_exclusive(cnt, T.rp, A.nc, s, tmp));   // total is A.nnz: no readback
  MGR_LAUNCH k_transpose_fill<<<nblocks(A.nr, 256), 256, 0, s>>>(A.rp, A.ci, A.v, A.nr, T.rp, cur, T.ci, T.v);
  if (sorted) MGR_LAUNCH k_sort_rows<<<nblocks(T.nr, 128), 128, 0, s>>>(T.rp, T.nr, T.ci, T.v);
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

// ============================================================================
// MGR reduction level (Sec. 5.1-5.3)
// ============================================================================
__global__ void k_flag_f(const int32_t* __restrict__ label, int64_t n, uint32_t mask,
                         int64_t* __restrict__ flag, int* err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t l = label[i];
  if (l < 0 || l > 31) {
    dev_fail(err, DEV_BAD_ARG);
    flag[i] = 0;
    return;
  }
  flag[i] = (mask >> l) & 1u;
}

__global__ void k_split(const int64_t* __restrict__ fpos, int64_t n, int64_t* __restrict__ Fidx,
                        int64_t* __restrict__ Cidx, int32_t* __restrict__ colF,
                        int32_t* __restrict__ colC) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t f = fpos[i];
  if (fpos[i + 1] != f) {
    Fidx[f] = i;
    colF[i] = (int32_t)f;
    colC[i] = -1;
  } else {
    int64_t c = i - f;
    Cidx[c] = i;
    colC[i] = (int32_t)c;
    colF[i] = -1;
  }
}

// D_FF entries; T = D_FF^-1 A_FC (t = a / d) and W_p = -T on the A_FC pattern.
__global__ void k_dff_and_w(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                            const double* __restrict__ av, const int64_t* __restrict__ Fidx,
                            int64_t nF, const int64_t* __restrict__ frp,
                            const double* __restrict__ fv, double* __restrict__ tv,
                            double* __restrict__ wv, double* __restrict__ dinv,
                            double* __restrict__ dval, int* err) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nF) return;
  int64_t r = Fidx[f];
  double d = 0.0;
  for (int64_t k = arp[r]; k < arp[r + 1]; k++)
    if (aci[k] == r) d = av[k];
  if (d == 0.0) {
    dev_fail(err, DEV_ZERO_DIAG);
    d = 1.0;
  }
  dinv[f] = 1.0 / d;
  dval[f] = d;
  for (int64_t k = frp[f]; k < frp[f + 1]; k++) {
    double t = __ddiv_rn(fv[k], d);
    tv[k] = t;
    wv[k] = -t;
  }
}

// U = A_CF D_FF^-1 for a pointwise D_FF: u = a / d of its column (exact
// division, as T = D^-1 A_FC); W_r = -U.
__global__ void k_acf_dinv(const int32_t* __restrict__ ci, const double* __restrict__ v, int64_t nnz,
                           const double* __restrict__ dval, double* __restrict__ u,
                           double* __restrict__ wr) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const double t = __ddiv_rn(v[k], dval[ci[k]]);
  u[k] = t;
  wr[k] = -t;
}

// point-block D_FF^-1 as a CSR matrix: block k (rows bstart[k] .. +b) holds
// its b x b inverse (binv: 16 per block, row-major 4 x 4)
__global__ void k_bd_counts(const int64_t* __restrict__ bstart, int64_t nblk, int64_t* __restrict__ cnt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nblk) return;
  const int64_t s0 = bstart[k];
  const int b = (int)(bstart[k + 1] - s0);
  for (int r = 0; r < b; r++) cnt[s0 + r] = b;
}
__global__ void k_bd_fill(const int64_t* __restrict__ bstart, int64_t nblk, const double* __restrict__ binv,
                          const int64_t* __restrict__ rp, int32_t* __restrict__ ci, double* __restrict__ v) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nblk) return;
  const int64_t s0 = bstart[k];
  const int b = (int)(bstart[k + 1] - s0);
  for (int r = 0; r < b; r++)
    for (int c = 0; c < b; c++) {
      ci[rp[s0 + r] + c] = (int32_t)(s0 + c);
      v[rp[s0 + r] + c] = binv[k * 16 + r * 4 + c];
    }
}

__global__ void k_neg(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = -a[i];
}
__global__ void k_twice(double* __restrict__ a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = 2.0 * a[i];   // exact
}

// ---- multicolour point-block Gauss-Seidel: colouring of the block graph ----
// Blocks k, m adjacent when a row of either has a column in the other (A and
// A^T).  Jones-Plassmann rounds with w_k = splitmix64(seed ^ 0xC0 << 56 ^
// l << 40 ^ k): in round c a block uncoloured at the start of the round takes
// colour c when its (w_k, -k) beats every neighbour uncoloured at the start of
// the round (colour -1, or c: coloured during this same round).
__global__ void k_blk_of(const int64_t* __restrict__ bstart, int64_t nblk, int64_t* __restrict__ blk) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nblk) return;
  for (int64_t i = bstart[k]; i < bstart[k + 1]; i++) blk[i] = k;
}
__global__ void k_color_init(int64_t nblk, uint64_t seed, int l, uint64_t* __restrict__ w,
                             int32_t* __restrict__ color) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nblk) return;
  w[k] = splitmix64(seed ^ (0xC0ull << 56) ^ ((uint64_t)l << 40) ^ (uint64_t)k);
  color[k] = -1;
}
__global__ void k_color_round(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                              const int64_t* __restrict__ trp, const int32_t* __restrict__ tci,
                              const int64_t* __restrict__ blk, const int64_t* __restrict__ bstart,
                              int64_t nblk, const uint64_t* __restrict__ w, int32_t* color, int c,
                              unsigned long long* __restrict__ left) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nblk || color[k] != -1) return;
  const uint64_t wk = w[k];
  bool win = true;
  for (int pass = 0; pass < 2 && win; pass++) {
    const int64_t* rp = pass ? trp : arp;
    const int32_t* ci = pass ? tci : aci;
    for (int64_t i = bstart[k]; i < bstart[k + 1] && win; i++)
      for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
        const int64_t m = blk[ci[q]];
        if (m == k) continue;
        const int32_t cm = ((volatile int32_t*)color)[m];
        if (cm != -1 && cm != c) continue;
        const uint64_t wm = w[m];
        if (wm > wk || (wm == wk && m < k)) {
          win = false;
          break;
        }
      }
  }
  if (win) color[k] = c;
  else atomicAdd(left, 1ull);
}
__global__ void k_color_count(const int32_t* __restrict__ color, int64_t nblk, int64_t* __restrict__ cnt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nblk) atomicAdd((unsigned long long*)&cnt[color[k]], 1ull);
}
// blocks grouped by colour (order inside a colour is free: its blocks are
// independent)
__global__ void k_color_place(const int32_t* __restrict__ color, int64_t nblk, int64_t* cursor,
                              int64_t* __restrict__ order) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nblk) order[atomicAdd((unsigned long long*)&cursor[color[k]], 1ull)] = k;
}

// G: keep the own-point columns plus the nmax others of largest |value|
// (ties: smaller column); nmax < 0 keeps everything.
__global__ void k_drop_mark(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, int64_t nr,
                            const int32_t* __restrict__ cnode, int nmax,
                            int8_t* __restrict__ keep, int64_t* __restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  int64_t b = rp[i], e = rp[i + 1];
  int64_t kept = 0;
  if (nmax < 0) {
    for (int64_t k = b; k < e; k++) keep[k] = 1;
    kept = e - b;
  } else {
    int32_t own = cnode[i];
    for (int64_t k = b; k < e; k++) {
      int8_t o = (cnode[ci[k]] == own);
      keep[k] = o;
      kept += o;
    }
    for (int r = 0; r < nmax; r++) {
      int64_t best = -1;
      for (int64_t k = b; k < e; k++) {
        if (keep[k]) continue;
        if (best < 0 || absbits(v[k]) > absbits(v[best]) ||
            (absbits(v[k]) == absbits(v[best]) && ci[k] < ci[best]))
          best = k;
      }
      if (best < 0) break;
      keep[best] = 2;     // selected (not own-point)
      kept++;
    }
  }
  cnt[i] = kept;
}

__global__ void k_drop_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, int64_t nr,
                            const int8_t* __restrict__ keep, const int64_t* __restrict__ krp,
                            int32_t* __restrict__ kci, double* __restrict__ kv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  int64_t o = krp[i];
  for (int64_t k = rp[i]; k < rp[i + 1]; k++)
    if (keep[k]) {
      kci[o] = ci[k];
      kv[o] = v[k];
      o++;
    }
}

// S = A_CC - K on the union pattern, s = (a or 0) - (k or 0).
template <bool FILL>
__global__ void k_union_sub(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                            const double* __restrict__ av, const int64_t* __restrict__ krp,
                            const int32_t* __restrict__ kci, const double* __restrict__ kv,
                            int64_t nr, int64_t* __restrict__ cnt_or_rp,
                            int32_t* __restrict__ sci, double* __restrict__ sv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  int64_t p = arp[i], pe = arp[i + 1], q = krp[i], qe = krp[i + 1];
  int64_t o = FILL ? cnt_or_rp[i] : 0;
  while (p < pe || q < qe) {
    int64_t cp = (p < pe) ? aci[p] : INT64_MAX;
    int64_t cq = (q < qe) ? kci[q] : INT64_MAX;
    double a = 0.0, c = 0.0;
    int64_t col;
    if (cp == cq) {
      col = cp;
      a = av[p++];
      c = kv[q++];
    } else if (cp < cq) {
      col = cp;
      a = av[p++];
    } else {
      col = cq;
      c = kv[q++];
    }
    if (FILL) {
      sci[o] = (int32_t)col;
      sv[o] = __dsub_rn(a, c);
    }
    o++;
  }
  if (!FILL) cnt_or_rp[i] = o;
}

__global__ void k_gather3(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                          const int32_t* __restrict__ c, const int64_t* __restrict__ idx,
                          int64_t n, int32_t* __restrict__ oa, int32_t* __restrict__ ob,
                          int32_t* __restrict__ oc) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int64_t i = idx[t];
  oa[t] = a[i];
  ob[t] = b[i];
  oc[t] = c[i];
}

// point blocks: maximal runs of equal dof_node (at most 4 dofs)
__global__ void k_block_heads(const int32_t* __restrict__ node, int64_t n, int64_t* __restrict__ head) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  head[i] = (i == 0 || node[i] != node[i - 1]) ? 1 : 0;
}

__global__ void k_block_starts(const int64_t* __restrict__ hpos, int64_t n,
                               int64_t* __restrict__ bstart, int64_t nblk) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    bstart[nblk] = n;
    return;
  }
  if (hpos[i + 1] != hpos[i]) bstart[hpos[i]] = i;
}

// Inverse of each diagonal point block by Gauss-Jordan with partial pivoting.
__global__ void k_block_inv(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, const int64_t* __restrict__ bstart,
                            int64_t nblk, double* __restrict__ binv, int* err) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nblk) return;
  int64_t s0 = bstart[k];
  int b = (int)(bstart[k + 1] - s0);
  if (b > 4) {
    dev_fail(err, DEV_BAD_ARG);
    return;
  }
  double m[4][8];
  for (int i = 0; i < b; i++)
    for (int j = 0; j < 2 * b; j++) m[i][j] = (j >= b && j - b == i) ? 1.0 : 0.0;
  for (int i = 0; i < b; i++) {
    int64_t r = s0 + i;
    for (int64_t q = rp[r]; q < rp[r + 1]; q++) {
      int64_t c = ci[q] - s0;
      if (c >= 0 && c < b) m[i][c] = v[q];
    }
  }
  for (int c = 0; c < b; c++) {
    int p = c;
    for (int i = c + 1; i < b; i++)
      if (fabs(m[i][c]) > fabs(m[p][c])) p = i;
    if (m[p][c] == 0.0) {
      dev_fail(err, DEV_ZERO_DIAG);
      return;
    }
    if (p != c)
      for (int j = 0; j < 2 * b; j++) {
        double t = m[c][j];
        m[c][j] = m[p][j];
        m[p][j] = t;
      }
    double piv = m[c][c];
    for (int j = 0; j < 2 * b; j++) m[c][j] /= piv;
    for (int i = 0; i < b; i++) {
      if (i == c) continue;
      double f = m[i][c];
      for (int j = 0; j < 2 * b; j++) m[i][j] -= f * m[c][j];
    }
  }
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) binv[k * 16 + i * 4 + j] = (i < b && j < b) ? m[i][b + j] : 0.0;
}

// Largest point block of a level (atomic max over the blocks).
__global__ void k_block_dim_max(const int64_t* __restrict__ bstart, int64_t nblk, int* __restrict__ out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nblk) return;
  atomicMax(out, (int)(bstart[k + 1] - bstart[k]));
}

// Apply layout of the block inverses: bd x bd values per block (row-major),
// taken from the 4 x 4 setup layout.
__global__ void k_compact_binv(const double* __restrict__ binv, int64_t nblk, int bd,
                               double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)bd * bd;
  if (t >= nblk * per) return;
  const int64_t k = t / per;
  const int q = (int)(t - k * per);
  out[t] = binv[k * 16 + (q / bd) * 4 + (q % bd)];
}

// ============================================================================
// AMG setup (Sec. 6 solver settings)
// ============================================================================
// l1-Jacobi diagonal inverse (Baker-Falgout-Kolev-Yang pointwise l1): 1 /
// (a_ii + sum_{j != i} |a_ij|), G lanes per row (G from the mean row length,
// as for the sparse products: FP64 work lane-dense).  Only the smoother uses
// it (no integer decision depends on it), so the sum is a lane tree.
template <int G>
__global__ void __launch_bounds__(256)
k_l1_inv(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
         const double* __restrict__ v, int64_t n, double* __restrict__ dinv, int* err) {
  const int lane = threadIdx.x & (G - 1);
  const unsigned mask = (G == 32) ? FULL : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; i < n; i += stride) {
    double off = 0.0, aii = 0.0;
    for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += G) {
      const double a = v[k];
      if (ci[k] == i) aii = a;
      else off += fabs(a);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      off += __shfl_xor_sync(mask, off, o, G);
      aii += __shfl_xor_sync(mask, aii, o, G);
    }
    if (lane == 0) {
      double d = aii + off;
      if (d == 0.0) {
        dev_fail(err, DEV_ZERO_DIAG);
        d = 1.0;
      }
      dinv[i] = 1.0 / d;
    }
  }
}

static void l1_inv(const Csr& A, double* dinv, int* err, cudaStream_t s) {
  const int64_t n = A.nr;
  if (n <= 0) return;
  const double avg = (double)A.nnz / (double)n;
  const int G = avg < 3 ? 1 : avg < 8 ? 2 : avg < 64 ? 4 : avg < 192 ? 8 : 16;
  const unsigned grid = (unsigned)std::min<int64_t>((n * G + 255) / 256, 152LL * 32);
  switch (G) {
    case 1: MGR_LAUNCH k_l1_inv<1><<<grid, 256, 0, s>>>(A.rp, A.ci, A.v, n, dinv, err); break;
    case 2: MGR_LAUNCH k_l1_inv<2><<<grid, 256, 0, s>>>(A.rp, A.ci, A.v, n, dinv, err); break;
    case 4: MGR_LAUNCH k_l1_inv<4><<<grid, 256, 0, s>>>(A.rp, A.ci, A.v, n, dinv, err); break;
    case 8: MGR_LAUNCH k_l1_inv<8><<<grid, 256, 0, s>>>(A.rp, A.ci, A.v, n, dinv, err); break;
    default: MGR_LAUNCH k_l1_inv<16><<<grid, 256, 0, s>>>(A.rp, A.ci, A.v, n, dinv, err); break;
  }
}

// Strength of connection on negative couplings between equal components.
// Warp per row.  m = max_j (-a_ij) over equal-component off-diagonals; S_i is
// empty unless some such a_ij is negative and non-zero, and then m is the
// largest |a_ij| among the negative ones: an exact integer max over the bit
// patterns (order-free).  Strong entries are compacted with ballots, so S_i
// keeps A's column order.
template <bool FILL>
__global__ void __launch_bounds__(256)
k_strength(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
           const double* __restrict__ v, const int32_t* __restrict__ comp, int64_t n,
           double theta, int64_t* __restrict__ cnt_or_rp, int32_t* __restrict__ sci,
           int64_t* __restrict__ cnt_out) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < n;
       i += (int64_t)gridDim.x * wpb) {
    const int32_t c_i = comp[i];
    const int64_t e0 = rp[i], e1 = rp[i + 1];
    unsigned long long mb = 0;
    for (int64_t k = e0 + lane; k < e1; k += 32) {
      const int32_t j = ci[k];
      const double a = v[k];
      if (j != i && comp[j] == c_i && is_neg(a)) {
        const unsigned long long ab = absbits(a);
        if (ab > mb) mb = ab;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(FULL, mb, o);
      if (y > mb) mb = y;
    }
    int64_t o = FILL ? cnt_or_rp[i] : 0;
    if (mb != 0) {
      const double thr = __dmul_rn(theta, __longlong_as_double((long long)mb));
      const uint64_t tb = absbits(thr);
      for (int64_t k0 = e0; k0 < e1; k0 += 32) {
        const int64_t k = k0 + lane;
        bool strong = false;
        int32_t j = -1;
        if (k < e1) {
          j = ci[k];
          const double a = v[k];
          if (j != i && comp[j] == c_i)
            strong = (tb != 0) ? (is_neg(a) && absbits(a) >= tb) : (-a >= thr);
        }
        const unsigned bal = __ballot_sync(FULL, strong);
        if (FILL && strong) sci[o + __popc(bal & ((1u << lane) - 1u))] = j;
        o += __popc(bal);
      }
    }
    if (!FILL && lane == 0) cnt_or_rp[i] = o;
    if (FILL && cnt_out && lane == 0) cnt_out[i] = o - cnt_or_rp[i];
  }
}

__global__ void k_pmis_init(const int64_t* __restrict__ srp, const int64_t* __restrict__ strp,
                            int64_t n, uint64_t seed, int slot, int level, double* __restrict__ w,
                            int8_t* __restrict__ cf) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t key = seed ^ ((uint64_t)slot << 48) ^ ((uint64_t)level << 40) ^ (uint64_t)i;
  double u = (double)(splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
  int64_t nt = strp[i + 1] - strp[i];
  w[i] = __dadd_rn((double)nt, u);
  cf[i] = (srp[i + 1] == srp[i] && nt == 0) ? (int8_t)-1 : (int8_t)0;
}

__global__ void k_pmis_select(const int64_t* __restrict__ srp, const int32_t* __restrict__ sci,
                              const int64_t* __restrict__ strp, const int32_t* __restrict__ stci,
                              const double* __restrict__ w, const int8_t* __restrict__ cf,
                              int64_t n, int8_t* __restrict__ newc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (cf[i] != 0) {
    newc[i] = 0;
    return;
  }
  const double wi = w[i];
  bool best = true;
  for (int64_t k = srp[i]; k < srp[i + 1] && best; k++) {
    int32_t j = sci[k];
    if (cf[j] != 0) continue;
    double wj = w[j];
    if (!(wi > wj || (wi == wj && i > j))) best = false;
  }
  for (int64_t k = strp[i]; k < strp[i + 1] && best; k++) {
    int32_t j = stci[k];
    if (cf[j] != 0) continue;
    double wj = w[j];
    if (!(wi > wj || (wi == wj && i > j))) best = false;
  }
  newc[i] = best ? 1 : 0;
}

// New C points of the round take C; an undecided point with a strong
// neighbour in C (old or new) becomes F.  A neighbour's mark may change
// during the kernel only from 0 to -1 or, for a new C point, to 1, which the
// newc test already sees, so the outcome does not depend on thread order.
__global__ void k_pmis_apply_mark(const int64_t* __restrict__ srp, const int32_t* __restrict__ sci,
                                  const int8_t* __restrict__ newc, int64_t n, int8_t* cf,
                                  unsigned long long* undecided) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  if (newc[j]) {
    cf[j] = 1;
    return;
  }
  if (cf[j] != 0) return;
  for (int64_t k = srp[j]; k < srp[j + 1]; k++) {
    const int32_t c = sci[k];
    if (newc[c] || cf[c] == 1) {
      cf[j] = -1;
      return;
    }
  }
  atomicAdd(undecided, 1ull);
}

__global__ void k_flag_c(const int8_t* __restrict__ cf, int64_t n, int64_t* __restrict__ flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (cf[i] == 1);
}

// Direct interpolation restricted to equal components with positive couplings
// lumped into the diagonal when no positive strong C neighbour exists, then
// truncation to the pmax entries of largest |w| (ties: smaller column) with the
// row sum kept.  The weights are recomputed where needed instead of stored, so
// a thread needs no per-row scratch.
struct InterpRow {
  double alpha, beta, dd;
  int64_t nsc;   // number of strong C neighbours
};

__device__ inline InterpRow interp_row(const int64_t* rp, const int32_t* ci, const double* v,
                                       const int64_t* srp, const int32_t* sci,
                                       const int32_t* comp, const int8_t* cf, int64_t i) {
  double sn = 0.0, sp = 0.0, cn = 0.0, cp = 0.0, aii = 0.0;
  int64_t nsc = 0;
  int64_t sb = srp[i], se = srp[i + 1], sq = sb;
  for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
    int32_t j = ci[k];
    double a = v[k];
    if (j == i) {
      aii = a;
      continue;
    }
    while (sq < se && sci[sq] < j) sq++;
    bool strong = (sq < se && sci[sq] == j);
    if (comp[j] != comp[i]) continue;
    bool sc = strong && cf[j] == 1;
    if (is_neg(a)) {
      sn = __dadd_rn(sn, a);
      if (sc) cn = __dadd_rn(cn, a);
    } else if (is_pos(a)) {
      sp = __dadd_rn(sp, a);
      if (sc) cp = __dadd_rn(cp, a);
    }
    if (sc) nsc++;
  }
  InterpRow r;
  r.nsc = (cn != 0.0 || cp != 0.0) ? nsc : 0;
  r.dd = (cp == 0.0) ? __dadd_rn(aii, sp) : aii;
  r.alpha = (cn != 0.0) ? __ddiv_rn(sn, cn) : 0.0;
  r.beta = (cp != 0.0) ? __ddiv_rn(sp, cp) : 0.0;
  return r;
}

// Iterates the strong-C entries of row i in ascending column order, calling
// f(col j, weight w) for each.
template <class Fn>
__device__ inline void for_strong_c(const int64_t* rp, const int32_t* ci, const double* v,
                                    const int64_t* srp, const int32_t* sci, const int8_t* cf,
                                    int64_t i, const InterpRow& r, Fn f) {
  int64_t sb = srp[i], se = srp[i + 1], sq = sb;
  for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
    int32_t j = ci[k];
    if (j == i) continue;
    while (sq < se && sci[sq] < j) sq++;
    if (!(sq < se && sci[sq] == j) || cf[j] != 1) continue;
    double a = v[k];
    double coef = is_neg(a) ? r.alpha : r.beta;
    double w = __ddiv_rn(-__dmul_rn(coef, a), r.dd);
    f(j, w);
  }
}

static constexpr int PMAX_CAP = 16;

// Entries of each row of P (the count pass of the interpolation), warp per
// row, without the weights: a C point has 1; an F point has its strong-C
// neighbours of the same component (nsc), capped at pmax, or none when their
// negative and positive sums (cn, cp of the weight formula) are both zero.  A
// sum of same-signed nonzero values is nonzero, so cn != 0 exactly when some
// strong-C entry is negative (the IEEE bit test is_neg), likewise cp; the
// counts are the weight pass's.
__global__ void __launch_bounds__(256)
k_interp_count(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ v,
               const int64_t* __restrict__ srp, const int32_t* __restrict__ sci,
               const int32_t* __restrict__ comp, const int8_t* __restrict__ cf, int64_t n, int pmax,
               int64_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * wpb) {
    if (cf[i] == 1) {
      if (lane == 0) cnt[i] = 1;
      continue;
    }
    const int64_t sb = srp[i], se = srp[i + 1];
    const int32_t c_i = comp[i];
    int nsc = 0;
    bool sign = false;
    for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) {
      const int32_t j = ci[k];
      bool sc = false;
      if (j != i && comp[j] == c_i && cf[j] == 1) {
        int64_t lo = sb, hi = se;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (sci[mid] < j) lo = mid + 1;
          else hi = mid;
        }
        sc = lo < se && sci[lo] == j;
      }
      if (sc) {
        nsc++;
        const double a = v[k];
        sign = sign || is_neg(a) || is_pos(a);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nsc += __shfl_xor_sync(FULL, nsc, o);
    sign = __any_sync(FULL, sign);
    if (lane == 0) {
      const int r = sign ? nsc : 0;
      cnt[i] = (pmax > 0 && r > pmax) ? pmax : r;
    }
  }
}

template <bool FILL>
__device__ void interp_row_seq(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const double* __restrict__ v, const int64_t* __restrict__ srp,
                               const int32_t* __restrict__ sci, const int32_t* __restrict__ comp,
                               const int8_t* __restrict__ cf, const int64_t* __restrict__ cmap,
                               int64_t i, int pmax, int64_t* __restrict__ cnt_or_rp,
                               int32_t* __restrict__ pci, double* __restrict__ pv) {
  if (cf[i] == 1) {
    if (FILL) {
      int64_t o = cnt_or_rp[i];
      pci[o] = (int32_t)cmap[i];
      pv[o] = 1.0;
    } else {
      cnt_or_rp[i] = 1;
    }
    return;
  }
  InterpRow r = interp_row(rp, ci, v, srp, sci, comp, cf, i);
  const bool trunc = pmax > 0 && r.nsc > pmax;
  if (!FILL) {
    cnt_or_rp[i] = trunc ? pmax : r.nsc;
    return;
  }
  if (r.nsc == 0) return;
  int64_t o = cnt_or_rp[i];
  const int64_t oend = cnt_or_rp[i + 1];
  if (!trunc) {
    for_strong_c(rp, ci, v, srp, sci, cf, i, r, [&](int32_t j, double w) {
      if (o < oend) {
        pci[o] = (int32_t)cmap[j];
        pv[o] = w;
      }
      o++;
    });
    return;
  }
  // gather the strong-C (column, weight) pairs once; a row with more than
  // ICAP of them falls back to recomputing the weights on each pass
  constexpr int ICAP = 48;
  int32_t jj[ICAP];
  double ww[ICAP];
  int nloc = 0;
  if (r.nsc <= ICAP) {
    for_strong_c(rp, ci, v, srp, sci, cf, i, r, [&](int32_t j, double w) {
      if (nloc < ICAP) {
        jj[nloc] = j;
        ww[nloc] = w;
        nloc++;
      }
    });
  }
  int32_t sel[PMAX_CAP];
  int ns = 0;
  if (nloc == r.nsc) {
    // select pmax largest |w| (ties: smaller column), repeated max search
    bool taken[ICAP];
    for (int q = 0; q < nloc; q++) taken[q] = false;
    for (int q = 0; q < pmax; q++) {
      int b = -1;
      for (int t = 0; t < nloc; t++) {
        if (taken[t]) continue;
        if (b < 0 || absbits(ww[t]) > absbits(ww[b]) ||
            (absbits(ww[t]) == absbits(ww[b]) && jj[t] < jj[b]))
          b = t;
      }
      if (b >= 0) {
        taken[b] = true;
        ns++;
      }
    }
    double sall = 0.0, skept = 0.0;
    for (int t = 0; t < nloc; t++) {
      sall = __dadd_rn(sall, ww[t]);
      if (taken[t]) skept = __dadd_rn(skept, ww[t]);
    }
    for (int t = 0; t < nloc; t++) {
      if (!taken[t]) continue;
      if (o < oend) {
        pci[o] = (int32_t)cmap[jj[t]];
        pv[o] = (skept != 0.0) ? __dmul_rn(ww[t], __ddiv_rn(sall, skept)) : ww[t];
      }
      o++;
    }
    return;
  }
  // long rows: recompute the weights on each pass
  for (int q = 0; q < pmax; q++) {
    int32_t bj = -1;
    double bw = 0.0;
    for_strong_c(rp, ci, v, srp, sci, cf, i, r, [&](int32_t j, double w) {
      for (int t = 0; t < ns; t++)
        if (sel[t] == j) return;
      if (bj < 0 || absbits(w) > absbits(bw) || (absbits(w) == absbits(bw) && j < bj)) {
        bj = j;
        bw = w;
      }
    });
    if (bj >= 0) sel[ns++] = bj;
  }
  double sall = 0.0, skept = 0.0;
  for_strong_c(rp, ci, v, srp, sci, cf, i, r, [&](int32_t j, double w) {
    sall = __dadd_rn(sall, w);
    for (int t = 0; t < ns; t++)
      if (sel[t] == j) {
        skept = __dadd_rn(skept, w);
        break;
      }
  });
  for_strong_c(rp, ci, v, srp, sci, cf, i, r, [&](int32_t j, double w) {
    for (int t = 0; t < ns; t++)
      if (sel[t] == j) {
        if (o < oend) {
          pci[o] = (int32_t)cmap[j];
          pv[o] = (skept != 0.0) ? __dmul_rn(w, __ddiv_rn(sall, skept)) : w;
        }
        o++;
        break;
      }
  });
}

// Thread per row (lane-dense FP64 sums across 32 rows; for large levels).
template <bool FILL>
__global__ void __launch_bounds__(128)
k_interp_thread(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                const double* __restrict__ v, const int64_t* __restrict__ srp,
                const int32_t* __restrict__ sci, const int32_t* __restrict__ comp,
                const int8_t* __restrict__ cf, const int64_t* __restrict__ cmap, int64_t n, int pmax,
                int64_t* __restrict__ cnt_or_rp, int32_t* __restrict__ pci, double* __restrict__ pv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) interp_row_seq<FILL>(rp, ci, v, srp, sci, comp, cf, cmap, i, pmax, cnt_or_rp, pci, pv);
}

// Warp per row (small levels: few rows, long rows).  Lanes stage the row
// (value, column, flags) in shared memory
// and form the weights (independent divisions) in parallel; lane 0 keeps every
// order-sensitive sum sequential in ascending column order, as the direct
// interpolation definition reads; the P_max largest |w| are picked by an exact
// warp argmax (ties: smaller column).  Rows longer than IW_CAP entries (or S
// rows longer than IW_SCAP) are done by lane 0 with the sequential row code.
static constexpr int IW_CAP = 256;
static constexpr int IW_SCAP = 256;
static constexpr int IW_WARPS = 4;
struct InterpWarp {
  double a[IW_CAP];
  double w[IW_CAP];
  int32_t col[IW_CAP];
  int32_t srow[IW_SCAP];
  uint8_t fl[IW_CAP];     // bit0 diagonal, bit1 same component, bit2 strong C, bit3 selected
  double bc[4];           // dd, alpha, beta, scale
  int flag;
};

template <bool FILL>
__global__ void __launch_bounds__(IW_WARPS * 32)
k_interp(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
         const double* __restrict__ v, const int64_t* __restrict__ srp,
         const int32_t* __restrict__ sci, const int32_t* __restrict__ comp,
         const int8_t* __restrict__ cf, const int64_t* __restrict__ cmap, int64_t n, int pmax,
         int64_t* __restrict__ cnt_or_rp, int32_t* __restrict__ pci, double* __restrict__ pv) {
  __shared__ InterpWarp sh[IW_WARPS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  InterpWarp& W = sh[wid];
  for (int64_t i = (int64_t)blockIdx.x * IW_WARPS + wid; i < n; i += (int64_t)gridDim.x * IW_WARPS) {
    if (cf[i] == 1) {
      if (lane == 0) {
        if (FILL) {
          const int64_t o = cnt_or_rp[i];
          pci[o] = (int32_t)cmap[i];
          pv[o] = 1.0;
        } else {
          cnt_or_rp[i] = 1;
        }
      }
      continue;
    }
    const int64_t e0 = rp[i], e1 = rp[i + 1], sb = srp[i], se = srp[i + 1];
    const int L = (int)(e1 - e0), SL = (int)(se - sb);
    if (L > IW_CAP || SL > IW_SCAP) {
      if (lane == 0)
        interp_row_seq<FILL>(rp, ci, v, srp, sci, comp, cf, cmap, i, pmax, cnt_or_rp, pci, pv);
      __syncwarp();
      continue;
    }
    for (int q = lane; q < SL; q += 32) W.srow[q] = sci[sb + q];
    __syncwarp();
    const int32_t c_i = comp[i];
    int nsc = 0;
    for (int t0 = 0; t0 < L; t0 += 32) {
      const int t = t0 + lane;
      bool sc = false;
      if (t < L) {
        const int32_t j = ci[e0 + t];
        const double a = v[e0 + t];
        int lo = 0, hi = SL;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (W.srow[mid] < j) lo = mid + 1;
          else hi = mid;
        }
        const bool strong = lo < SL && W.srow[lo] == j;
        sc = (j != i) && strong && cf[j] == 1;
        W.a[t] = a;
        W.col[t] = j;
        W.fl[t] = (uint8_t)((j == i ? 1 : 0) | (comp[j] == c_i ? 2 : 0) | (sc ? 4 : 0));
      }
      nsc += __popc(__ballot_sync(FULL, sc));
    }
    const bool trunc = pmax > 0 && nsc > pmax;
    if (!FILL) {
      if (lane == 0) cnt_or_rp[i] = (nsc == 0) ? 0 : (trunc ? pmax : nsc);
      __syncwarp();
      continue;
    }
    if (nsc == 0) {
      __syncwarp();
      continue;
    }
    __syncwarp();
    if (lane == 0) {
      double sn = 0.0, sp = 0.0, cn = 0.0, cp = 0.0, aii = 0.0;
      for (int t = 0; t < L; t++) {
        const uint8_t f = W.fl[t];
        const double a = W.a[t];
        if (f & 1) {
          aii = a;
          continue;
        }
        if (!(f & 2)) continue;
        const bool sc = f & 4;
        if (is_neg(a)) {
          sn = __dadd_rn(sn, a);
          if (sc) cn = __dadd_rn(cn, a);
        } else if (is_pos(a)) {
          sp = __dadd_rn(sp, a);
          if (sc) cp = __dadd_rn(cp, a);
        }
      }
      W.bc[0] = (cp == 0.0) ? __dadd_rn(aii, sp) : aii;
      W.bc[1] = (cn != 0.0) ? __ddiv_rn(sn, cn) : 0.0;
      W.bc[2] = (cp != 0.0) ? __ddiv_rn(sp, cp) : 0.0;
    }
    __syncwarp();
    const double dd = W.bc[0], alpha = W.bc[1], beta = W.bc[2];
    for (int t = lane; t < L; t += 32)
      if (W.fl[t] & 4) {
        const double a = W.a[t];
        W.w[t] = __ddiv_rn(-__dmul_rn(is_neg(a) ? alpha : beta, a), dd);
      }
    __syncwarp();
    int64_t o = cnt_or_rp[i];
    if (!trunc) {
      for (int t0 = 0; t0 < L; t0 += 32) {
        const int t = t0 + lane;
        const bool sc = t < L && (W.fl[t] & 4);
        const unsigned bal = __ballot_sync(FULL, sc);
        if (sc) {
          const int64_t d = o + __popc(bal & ((1u << lane) - 1u));
          pci[d] = (int32_t)cmap[W.col[t]];
          pv[d] = W.w[t];
        }
        o += __popc(bal);
      }
      __syncwarp();
      continue;
    }
    // pmax rounds of an exact warp argmax of |w| (ties: smaller column)
    for (int q = 0; q < pmax; q++) {
      unsigned long long bk = 0;
      int bt = -1;
      for (int t = lane; t < L; t += 32) {
        if ((W.fl[t] & 12) != 4) continue;          // strong C, not yet selected
        const unsigned long long k = absbits(W.w[t]);
        if (bt < 0 || k > bk) {
          bk = k;
          bt = t;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(FULL, bk, off);
        const int ot = __shfl_xor_sync(FULL, bt, off);
        if (ot >= 0 && (bt < 0 || ok > bk || (ok == bk && ot < bt))) {
          bk = ok;
          bt = ot;
        }
      }
      if (lane == 0 && bt >= 0) W.fl[bt] |= 8;
      __syncwarp();
    }
    if (lane == 0) {
      double sall = 0.0, skept = 0.0;
      for (int t = 0; t < L; t++) {
        const uint8_t f = W.fl[t];
        if (!(f & 4)) continue;
        sall = __dadd_rn(sall, W.w[t]);
        if (f & 8) skept = __dadd_rn(skept, W.w[t]);
      }
      W.flag = (skept != 0.0);
      W.bc[3] = (skept != 0.0) ? __ddiv_rn(sall, skept) : 1.0;
    }
    __syncwarp();
    const bool scale = W.flag;
    const double fct = W.bc[3];
    for (int t0 = 0; t0 < L; t0 += 32) {
      const int t = t0 + lane;
      const bool kept = t < L && (W.fl[t] & 8);
      const unsigned bal = __ballot_sync(FULL, kept);
      if (kept) {
        const int64_t d = o + __popc(bal & ((1u << lane) - 1u));
        pci[d] = (int32_t)cmap[W.col[t]];
        pv[d] = scale ? __dmul_rn(W.w[t], fct) : W.w[t];
      }
      o += __popc(bal);
    }
    __syncwarp();
  }
}

__global__ void k_coarse_comp(const int8_t* __restrict__ cf, const int64_t* __restrict__ cmap,
                              const int32_t* __restrict__ comp, int64_t n, int32_t* __restrict__ cc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && cf[i] == 1) cc[cmap[i]] = comp[i];
}

// Coarsest level: dense LU with partial pivoting (ties: smaller row), then the
// explicit inverse (one column per thread), in a single thread block.
__global__ void k_csr_to_dense(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const double* __restrict__ v, int64_t n, double* __restrict__ d) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int64_t k = rp[i]; k < rp[i + 1]; k++) d[i * n + ci[k]] = v[k];
}

__global__ void __launch_bounds__(1024) k_dense_lu_inverse(double* __restrict__ a, int n,
                                                           int32_t* __restrict__ piv,
                                                           double* __restrict__ inv, int* err) {
  __shared__ double sval[1024];
  __shared__ int sidx[1024];
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; k++) {
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += nt) {
      double x = fabs(a[(int64_t)i * n + k]);
      if (x > best || (x == best && i < bi)) {
        best = x;
        bi = i;
      }
    }
    sval[tid] = best;
    sidx[tid] = bi;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s) {
        double x = sval[tid + s];
        int xi = sidx[tid + s];
        if (x > sval[tid] || (x == sval[tid] && xi < sidx[tid])) {
          sval[tid] = x;
          sidx[tid] = xi;
        }
      }
      __syncthreads();
    }
    int p = sidx[0];
    if (tid == 0) {
      piv[k] = p;
      if (sval[0] == 0.0) fail = 1;
    }
    __syncthreads();
    if (fail) break;
    if (p != k)
      for (int j = tid; j < n; j += nt) {
        double t = a[(int64_t)k * n + j];
        a[(int64_t)k * n + j] = a[(int64_t)p * n + j];
        a[(int64_t)p * n + j] = t;
      }
    __syncthreads();
    double akk = a[(int64_t)k * n + k];
    for (int i = k + 1 + tid; i < n; i += nt) a[(int64_t)i * n + k] /= akk;
    __syncthreads();
    int m = n - k - 1;
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
      a[(int64_t)i * n + j] -= a[(int64_t)i * n + k] * a[(int64_t)k * n + j];
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) dev_fail(err, DEV_ZERO_DIAG);
    return;
  }
  for (int c = tid; c < n; c += nt) {
    // column c of the inverse: x = e_c, permute, L solve, U solve
    for (int i = 0; i < n; i++) inv[(int64_t)i * n + c] = (i == c) ? 1.0 : 0.0;
    for (int k = 0; k < n; k++) {
      int p = piv[k];
      if (p != k) {
        double t = inv[(int64_t)k * n + c];
        inv[(int64_t)k * n + c] = inv[(int64_t)p * n + c];
        inv[(int64_t)p * n + c] = t;
      }
    }
    for (int i = 0; i < n; i++) {
      double s = inv[(int64_t)i * n + c];
      for (int j = 0; j < i; j++) s -= a[(int64_t)i * n + j] * inv[(int64_t)j * n + c];
      inv[(int64_t)i * n + c] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
      double s = inv[(int64_t)i * n + c];
      for (int j = i + 1; j < n; j++) s -= a[(int64_t)i * n + j] * inv[(int64_t)j * n + c];
      inv[(int64_t)i * n + c] = s / a[(int64_t)i * n + i];
    }
  }
}

// In-place Gauss-Jordan inversion with partial pivoting (ties: smaller row),
// one thread block: row k is normalised, every other row updated, and the
// recorded row interchanges are undone as column interchanges at the end.
// `a` (n x n, row-major) holds A on entry and A^-1 on exit.  With SMEM the
// matrix is worked on in shared memory (n^2 doubles must fit), else in place.
template <bool SMEM>
__global__ void __launch_bounds__(1024) k_dense_gj_inverse(double* __restrict__ ga, int n,
                                                           int32_t* __restrict__ piv, int* err) {
  extern __shared__ double dyn[];
  double* f;
  if constexpr (SMEM) {
    f = dyn + (size_t)n * n;   // n values after the matrix
  } else {
    __shared__ double fst[1024];
    f = fst;
  }
  __shared__ double wbest[32];
  __shared__ int wbi[32];
  __shared__ int sp;
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  double* a = SMEM ? dyn : ga;
  if (SMEM)
    for (int64_t e = tid; e < (int64_t)n * n; e += nt) a[e] = ga[e];
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; k++) {
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += nt) {
      double x = fabs(a[(int64_t)i * n + k]);
      if (x > best || (x == best && i < bi)) {
        best = x;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      wbest[wid] = best;
      wbi[wid] = bi;
    }
    __syncthreads();
    if (wid == 0) {
      best = (lane < nw) ? wbest[lane] : -1.0;
      bi = (lane < nw) ? wbi[lane] : n;
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        sp = bi;
        piv[k] = bi;
        if (!(best > 0.0)) fail = 1;
      }
    }
    __syncthreads();
    if (fail) break;
    const int p = sp;
    if (p != k)
      for (int j = tid; j < n; j += nt) {
        double t = a[(int64_t)k * n + j];
        a[(int64_t)k * n + j] = a[(int64_t)p * n + j];
        a[(int64_t)p * n + j] = t;
      }
    __syncthreads();
    const double pinv = 1.0 / a[(int64_t)k * n + k];
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      double x = (j == k) ? 1.0 : a[(int64_t)k * n + j];
      a[(int64_t)k * n + j] = x * pinv;
    }
    for (int i = tid; i < n; i += nt) {
      f[i] = (i == k) ? 0.0 : a[(int64_t)i * n + k];
      if (i != k) a[(int64_t)i * n + k] = 0.0;
    }
    __syncthreads();
    const double* rowk = a + (int64_t)k * n;
    for (int i = wid; i < n; i += nw) {
      if (i == k) continue;
      const double fi = f[i];
      double* ri = a + (int64_t)i * n;
      for (int j = lane; j < n; j += 32) ri[j] -= fi * rowk[j];
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) dev_fail(err, DEV_ZERO_DIAG);
    return;
  }
  for (int k = n - 1; k >= 0; k--) {
    const int p = piv[k];
    if (p != k)
      for (int i = tid; i < n; i += nt) {
        double t = a[(int64_t)i * n + k];
        a[(int64_t)i * n + k] = a[(int64_t)i * n + p];
        a[(int64_t)i * n + p] = t;
      }
    __syncthreads();
  }
  if (SMEM)
    for (int64_t e = tid; e < (int64_t)n * n; e += nt) ga[e] = a[e];
}

static constexpr size_t GJ_SMEM_MAX = 220 * 1024;
static int dense_coarsest(Pool& P, int* derr, Amg* g, Pool& tmp, cudaStream_t s) {
  const Csr& A = g->lev.back().A;
  int64_t n = A.nr;
  g->ncoarse = n;
  if (n == 0) return MGR_SUCCESS;
  if (n > LU_CAP) return MGR_ERR_COARSE;
  double* d = tmp.get<double>(n * n);
  int32_t* piv = tmp.get<int32_t>(n);
  g->inv = P.get<double>(n * n);
  if (P.err || tmp.err) return P.err ? P.err : tmp.err;
  if (n <= 1024) {
    MGR_TRY_CUDA(cudaMemsetAsync(g->inv, 0, sizeof(double) * n * n, s));
    MGR_LAUNCH k_csr_to_dense<<<nblocks(n, 256), 256, 0, s>>>(A.rp, A.ci, A.v, n, g->inv);
    const size_t sm = sizeof(double) * ((size_t)n * (size_t)n + (size_t)n);
    if (sm <= GJ_SMEM_MAX) {
      // the attribute is a maximum, set once (setups may run on several threads)
      static std::once_flag gj_once;
      static cudaError_t gj_err = cudaSuccess;
      std::call_once(gj_once, [] {
        gj_err = cudaFuncSetAttribute(k_dense_gj_inverse<true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GJ_SMEM_MAX);
      });
      MGR_TRY_CUDA(gj_err);
      MGR_LAUNCH k_dense_gj_inverse<true><<<1, 1024, sm, s>>>(g->inv, (int)n, piv, derr);
    } else {
      MGR_LAUNCH k_dense_gj_inverse<false><<<1, 1024, 0, s>>>(g->inv, (int)n, piv, derr);
    }
    MGR_TRY_CUDA(cudaGetLastError());
    return check_dev_err(derr, s);
  }
  MGR_TRY_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * n * n, s));
  MGR_LAUNCH k_csr_to_dense<<<nblocks(n, 256), 256, 0, s>>>(A.rp, A.ci, A.v, n, d);
  MGR_LAUNCH k_dense_lu_inverse<<<1, 1024, 0, s>>>(d, (int)n, piv, g->inv, derr);
  MGR_TRY_CUDA(cudaGetLastError());
  return check_dev_err(derr, s);
}

// P_max truncation of the rows of a product interpolation P1 P2 (columns
// ascending): keep the pmax entries of largest |w| (ties: the earlier entry,
// i.e. the smaller column) and rescale them by (sum of all w) / (sum of kept
// w), both sums in row order -- the rule of the direct interpolation.  Thread
// per row; an entry is kept when fewer than pmax entries beat it.
__device__ __forceinline__ uint64_t abs_bits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
template <bool FILL>
__global__ void k_trunc_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, int64_t n, int pmax,
                             int64_t* __restrict__ cnt_or_rp, int32_t* __restrict__ oci,
                             double* __restrict__ ov) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e0 = rp[i], e1 = rp[i + 1], m = e1 - e0;
  if (pmax <= 0 || m <= pmax) {
    if (!FILL) {
      cnt_or_rp[i] = m;
    } else {
      int64_t o = cnt_or_rp[i];
      for (int64_t q = e0; q < e1; q++, o++) {
        oci[o] = ci[q];
        ov[o] = v[q];
      }
    }
    return;
  }
  if (!FILL) {
    cnt_or_rp[i] = pmax;
    return;
  }
  double sall = 0.0, skept = 0.0;
  for (int64_t q = e0; q < e1; q++) sall = __dadd_rn(sall, v[q]);
  for (int64_t q = e0; q < e1; q++) {
    const uint64_t aq = abs_bits(v[q]);
    int r = 0;
    for (int64_t u = e0; u < e1; u++) {
      const uint64_t au = abs_bits(v[u]);
      r += (au > aq || (au == aq && u < q));
    }
    if (r < pmax) skept = __dadd_rn(skept, v[q]);
  }
  const double ratio = (skept != 0.0) ? __ddiv_rn(sall, skept) : 1.0;
  int64_t o = cnt_or_rp[i];
  for (int64_t q = e0; q < e1; q++) {
    const uint64_t aq = abs_bits(v[q]);
    int r = 0;
    for (int64_t u = e0; u < e1; u++) {
      const uint64_t au = abs_bits(v[u]);
      r += (au > aq || (au == aq && u < q));
    }
    if (r < pmax) {
      oci[o] = ci[q];
      ov[o] = (skept != 0.0) ? __dmul_rn(v[q], ratio) : v[q];
      o++;
    }
  }
}

// the aggressive level's C points: first-stage C points that the second stage
// kept C
__global__ void k_agg_cf(int8_t* __restrict__ cf, const int64_t* __restrict__ cmap,
                         const int8_t* __restrict__ cf2, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && cf[i] == 1 && cf2[cmap[i]] != 1) cf[i] = -1;
}

// One coarsening step on (A, comp): strength S (into Ps), PMIS C/F marks
// (weights keyed by `level`; into Ps), coarse numbering cmap (tmp), direct
// interpolation with P_max truncation (into Pi).  *nc = number of C points
// (no interpolation is built when it is 0 or n).
static int coarsen_step(const mgr_options_t& o, Pool& Ps, Pool& Pi, Pool& tmp, const Csr& A,
                        const int32_t* comp, int slot, int level, Csr& S, int8_t** cf_out,
                        int64_t** cmap_out, Csr& Pm, int64_t* nc_out, cudaStream_t s) {
  const int64_t n = A.nr;
  *nc_out = 0;
  int64_t* cnt = tmp.get<int64_t>(n + 1);
  S.nr = S.nc = n;
  S.rp = Ps.get<int64_t>(n + 1);
  if (tmp.err || Ps.err) return tmp.err ? tmp.err : Ps.err;
  // one pass: S is a subset of A's pattern, so each row is written at A's row
  // offset with its exact length, then moved to its compact offset
  int32_t* sfull = tmp.get<int32_t>(A.nnz);
  if (tmp.err) return tmp.err;
  MGR_LAUNCH k_strength<true><<<grid_for(n, 8, 152 * 16), 256, 0, s>>>(A.rp, A.ci, A.v, comp, n,
                                                                      o.amg_theta, A.rp, sfull, cnt);
  MGR_TRY(rowptr_from_counts(cnt, S.rp, n, &S.nnz, s, tmp));
  S.ci = Ps.get<int32_t>(S.nnz);
  if (Ps.err) return Ps.err;
  MGR_LAUNCH k_compact_rows<<<grid_for(n, 8, 152 * 16), 256, 0, s>>>(A.rp, sfull, n, S.rp, S.ci);
  tmp.release(sfull, s);
  g_trace.mark("amg strength", slot, level);
  Csr ST;
  MGR_TRY(transpose(tmp, tmp, S, ST, false, false, s));
  // PMIS
  double* w = tmp.get<double>(n);
  int8_t* newc = tmp.get<int8_t>(n);
  int8_t* cf = Ps.get<int8_t>(n);
  unsigned long long* und = tmp.get<unsigned long long>(4);
  if (tmp.err || Ps.err) return tmp.err ? tmp.err : Ps.err;
  *cf_out = cf;
  MGR_LAUNCH k_pmis_init<<<nblocks(n, 256), 256, 0, s>>>(S.rp, ST.rp, n, o.seed, slot, level, w, cf);
  // synchronous rounds, checked every 4th: a round after the last
  // undecided point is gone changes nothing
  for (int round = 0; round < 100000; round += 4) {
    MGR_TRY_CUDA(cudaMemsetAsync(und, 0, 4 * sizeof(unsigned long long), s));
    for (int q = 0; q < 4; q++) {
      MGR_LAUNCH k_pmis_select<<<nblocks(n, 256), 256, 0, s>>>(S.rp, S.ci, ST.rp, ST.ci, w, cf, n, newc);
      MGR_LAUNCH k_pmis_apply_mark<<<nblocks(n, 256), 256, 0, s>>>(S.rp, S.ci, newc, n, cf, und + q);
    }
    unsigned long long left = 0;
    MGR_TRY(read_back(&left, und + 3, s));
    if (left == 0) break;
  }
  g_trace.mark("amg pmis", slot, level);
  // coarse numbering
  int64_t* flag = tmp.get<int64_t>(n + 1);
  int64_t* cmap = tmp.get<int64_t>(n + 1);
  if (tmp.err) return tmp.err;
  *cmap_out = cmap;
  MGR_LAUNCH k_flag_c<<<nblocks(n, 256), 256, 0, s>>>(cf, n, flag);
  int64_t nc = 0;
  MGR_TRY(rowptr_from_counts(flag, cmap, n, &nc, s, tmp));
  *nc_out = nc;
  if (nc == 0 || nc == n) return MGR_SUCCESS;
  // interpolation
  if (o.amg_pmax > PMAX_CAP) return MGR_ERR_INVALID_ARG;
  Pm.nr = n;
  Pm.nc = nc;
  Pm.rp = Pi.get<int64_t>(n + 1);
  if (Pi.err) return Pi.err;
  // FP64 work is lane-dense in the thread-per-row form; the warp form wins
  // only where a level has too few rows to fill the GPU (measured on GB300:
  // on the 113k-row, 150-non-zero level the warp form took 2.4 ms against
  // 0.8 ms)
  const bool big = n >= 20000;
  MGR_LAUNCH k_interp_count<<<grid_for(n, 8, 152 * 16), 256, 0, s>>>(A.rp, A.ci, A.v, S.rp, S.ci, comp, cf, n,
                                                                   o.amg_pmax, cnt);
  MGR_TRY(rowptr_from_counts(cnt, Pm.rp, n, &Pm.nnz, s, tmp));
  Pm.ci = Pi.get<int32_t>(Pm.nnz);
  Pm.v = Pi.get<double>(Pm.nnz);
  if (Pi.err) return Pi.err;
  if (big)
    MGR_LAUNCH k_interp_thread<true><<<nblocks(n, 128), 128, 0, s>>>(A.rp, A.ci, A.v, S.rp, S.ci, comp, cf,
                                                                    cmap, n, o.amg_pmax, Pm.rp, Pm.ci, Pm.v);
  else
    MGR_LAUNCH k_interp<true><<<grid_for(n, IW_WARPS, 152 * 32), IW_WARPS * 32, 0, s>>>(
        A.rp, A.ci, A.v, S.rp, S.ci, comp, cf, cmap, n, o.amg_pmax, Pm.rp, Pm.ci, Pm.v);
  g_trace.mark("amg interp", slot, level);
  return MGR_SUCCESS;
}

// ============================================================================
// Shared row patterns of a square operator
// ============================================================================
// On a structured mesh most rows of an operator such as A_uu have the same
// columns relative to the row (the interior rows of one displacement
// component), so the columns can be stored once per distinct pattern:
//   1. hash each row's (column - row) sequence;
//   2. insert the hashes into an open-addressing table of PAT_SLOTS slots
//      (the row that claims a slot represents its pattern);
//   3. number the occupied slots, copy each representative's offsets;
//   4. check every row against its pattern (a hash collision or an
//      overfull table leaves the operator without patterns).
static constexpr int PAT_SLOTS = 8192;   // power of two
static constexpr int PAT_MAX = 4096;     // at most this many distinct patterns
static constexpr int64_t PAT_MIN_NNZ = 1 << 20;   // smaller operators keep plain CSR

__device__ __forceinline__ uint64_t pat_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_pat_hash(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n,
                           unsigned long long* __restrict__ hash) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * wpb) {
    const int64_t e0 = rp[i], e1 = rp[i + 1];
    uint64_t acc = 0;
    for (int64_t k = e0 + lane; k < e1; k += 32) {
      const uint32_t off = (uint32_t)((int64_t)ci[k] - i);
      acc ^= pat_mix(((uint64_t)off) | ((uint64_t)(k - e0) << 32));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) {
      uint64_t h = pat_mix(acc + (uint64_t)(e1 - e0) * 0x9E3779B97F4A7C15ull);
      hash[i] = h ? h : 1ull;   // 0 marks an empty slot
    }
  }
}

__global__ void k_pat_insert(const unsigned long long* __restrict__ hash, int64_t n,
                             unsigned long long* keys, int64_t* __restrict__ rep,
                             int32_t* __restrict__ slot_of, int* __restrict__ overflow) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long h = hash[i];
    uint32_t sl = (uint32_t)(h & (PAT_SLOTS - 1));
    int found = -1;
    for (int probe = 0; probe < PAT_SLOTS; probe++) {
      const unsigned long long k = ((volatile unsigned long long*)keys)[sl];
      if (k == h) {
        found = (int)sl;
        break;
      }
      if (k == 0ull) {
        const unsigned long long old = atomicCAS(&keys[sl], 0ull, h);
        if (old == 0ull) {
          rep[sl] = i;
          found = (int)sl;
          break;
        }
        if (old == h) {
          found = (int)sl;
          break;
        }
      }
      sl = (sl + 1) & (PAT_SLOTS - 1);
    }
    slot_of[i] = found;
    if (found < 0) atomicExch(overflow, 1);
  }
}

// one block: number the occupied slots (ascending slot order) and take each
// pattern's length from its representative row
__global__ void __launch_bounds__(1024)
k_pat_number(const unsigned long long* __restrict__ keys, const int64_t* __restrict__ rep,
             const int64_t* __restrict__ rp, int32_t* __restrict__ slot2pid,
             int32_t* __restrict__ plen, int* __restrict__ npat) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int s0 = 0; s0 < PAT_SLOTS; s0 += blockDim.x) {
    const int sl = s0 + threadIdx.x;
    const int occ = (sl < PAT_SLOTS && keys[sl] != 0ull) ? 1 : 0;
    const unsigned bal = __ballot_sync(FULL, occ);
    const int before_in_warp = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; w++) before += wsum[w];
    if (occ) {
      const int id = base + before + before_in_warp;
      slot2pid[sl] = id;
      if (id < PAT_MAX) plen[id] = (int32_t)(rp[rep[sl] + 1] - rp[rep[sl]]);
    } else if (sl < PAT_SLOTS) {
      slot2pid[sl] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += wsum[w];
      base += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *npat = base;
}

// warp per occupied slot: its representative's column offsets
__global__ void k_pat_fill(const unsigned long long* __restrict__ keys, const int64_t* __restrict__ rep,
                           const int32_t* __restrict__ slot2pid, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, const int32_t* __restrict__ pstart,
                           int32_t* __restrict__ poff) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int sl = blockIdx.x * wpb + (threadIdx.x >> 5); sl < PAT_SLOTS; sl += gridDim.x * wpb) {
    if (keys[sl] == 0ull) continue;
    const int p = slot2pid[sl];
    const int64_t r = rep[sl], e0 = rp[r], e1 = rp[r + 1];
    for (int64_t k = e0 + lane; k < e1; k += 32) poff[pstart[p] + (k - e0)] = (int32_t)((int64_t)ci[k] - r);
  }
}

// warp per row: the row against its pattern; pid[i] = the pattern's number
__global__ void k_pat_verify(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n,
                             const int32_t* __restrict__ slot_of, const int32_t* __restrict__ slot2pid,
                             const int32_t* __restrict__ pstart, const int32_t* __restrict__ poff,
                             uint16_t* __restrict__ pid, int* __restrict__ bad) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * wpb) {
    const int p = slot2pid[slot_of[i]];
    const int64_t e0 = rp[i], e1 = rp[i + 1];
    bool ok = (int64_t)(pstart[p + 1] - pstart[p]) == e1 - e0;
    if (ok)
      for (int64_t k = e0 + lane; k < e1; k += 32)
        if ((int64_t)ci[k] - i != (int64_t)poff[pstart[p] + (k - e0)]) ok = false;
    if (__any_sync(FULL, !ok) && lane == 0) atomicExch(bad, 1);
    if (lane == 0) pid[i] = (uint16_t)p;
  }
}

int build_row_patterns(Pool& P, Csr& A, cudaStream_t s) {
  const int64_t n = A.nr;
  if (n <= 0 || A.nr != A.nc) return MGR_SUCCESS;
  Pool tmp;
  tmp.s = s;
  unsigned long long* hash = tmp.get<unsigned long long>(n);
  unsigned long long* keys = tmp.get<unsigned long long>(PAT_SLOTS);
  int64_t* rep = tmp.get<int64_t>(PAT_SLOTS);
  int32_t* slot_of = tmp.get<int32_t>(n);
  int32_t* slot2pid = tmp.get<int32_t>(PAT_SLOTS);
  int32_t* plen = tmp.get<int32_t>(PAT_MAX);
  int* flags = tmp.get<int>(3);   // overflow, npat, bad
  if (tmp.err) {
    tmp.free_all_async(s);
    return tmp.err;
  }
  MGR_TRY_CUDA(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * PAT_SLOTS, s));
  MGR_TRY_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * 3, s));
  MGR_LAUNCH k_pat_hash<<<grid_for(n, 8, 152 * 16), 256, 0, s>>>(A.rp, A.ci, n, hash);
  MGR_LAUNCH k_pat_insert<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(hash, n, keys, rep, slot_of, flags);
  MGR_LAUNCH k_pat_number<<<1, 1024, 0, s>>>(keys, rep, A.rp, slot2pid, plen, flags + 1);
  int hf[3] = {0, 0, 0};
  MGR_TRY_CUDA(cudaMemcpyAsync(hf, flags, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  MGR_TRY_CUDA(cudaStreamSynchronize(s));
  const int npat = hf[1];
  if (hf[0] || npat <= 0 || npat > PAT_MAX) {   // too many patterns: plain CSR
    tmp.free_all_async(s);
    return MGR_SUCCESS;
  }
  std::vector<int32_t> len(npat), start(npat + 1, 0);
  MGR_TRY_CUDA(cudaMemcpyAsync(len.data(), plen, sizeof(int32_t) * npat, cudaMemcpyDeviceToHost, s));
  MGR_TRY_CUDA(cudaStreamSynchronize(s));
  for (int p = 0; p < npat; p++) start[p + 1] = start[p] + len[p];
  A.pstart = P.get<int32_t>(npat + 1);
  A.poff = P.get<int32_t>(start[npat] > 0 ? start[npat] : 1);
  A.pid = P.get<uint16_t>(n);
  if (P.err) {
    tmp.free_all_async(s);
    return P.err;
  }
  MGR_TRY_CUDA(cudaMemcpyAsync(A.pstart, start.data(), sizeof(int32_t) * (npat + 1),
                               cudaMemcpyHostToDevice, s));
  MGR_LAUNCH k_pat_fill<<<grid_for((int64_t)PAT_SLOTS * 32, 256, 152 * 16), 256, 0, s>>>(
      keys, rep, slot2pid, A.rp, A.ci, A.pstart, A.poff);
  MGR_LAUNCH k_pat_verify<<<grid_for(n, 8, 152 * 16), 256, 0, s>>>(A.rp, A.ci, n, slot_of, slot2pid,
                                                                    A.pstart, A.poff, A.pid, flags + 2);
  MGR_TRY_CUDA(cudaMemcpyAsync(hf + 2, flags + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  MGR_TRY_CUDA(cudaStreamSynchronize(s));   // `start` outlives its copy
  tmp.free_all_async(s);
  if (hf[2]) {   // a hash collision: keep plain CSR
    P.release(A.pstart, s);
    P.release(A.poff, s);
    P.release(A.pid, s);
    A.pstart = A.poff = nullptr;
    A.pid = nullptr;
    return MGR_SUCCESS;
  }
  A.npat = npat;
  return MGR_SUCCESS;
}

int build_amg(Handle* h, Pool& P, int* derr, const Csr& A0, bool own_input,
              const int32_t* comp0, int slot, Amg** out, cudaStream_t s) {
  Pool tmp;
  tmp.s = s;
  Amg* g = new Amg();
  *out = g;
  const mgr_options_t& o = h->opt;
  g->lev.emplace_back();
  {
    AmgLevel& L0 = g->lev[0];
    if (own_input && comp0) {
      // A0 and comp0 already belong to P (handed over by the caller)
      L0.A = A0;
      L0.comp = const_cast<int32_t*>(comp0);
    } else {
      int rc = copy_csr(P, A0, L0.A, s);
      if (rc) return rc;
      L0.comp = P.get<int32_t>(A0.nr);
      if (!L0.comp) return P.err;
      if (comp0)
        MGR_TRY_CUDA(cudaMemcpyAsync(L0.comp, comp0, sizeof(int32_t) * A0.nr, cudaMemcpyDeviceToDevice, s));
      else
        MGR_TRY_CUDA(cudaMemsetAsync(L0.comp, 0, sizeof(int32_t) * A0.nr, s));
    }
  }
  int rc = MGR_SUCCESS;
  for (int k = 0;; k++) {
    AmgLevel* L = &g->lev[k];
    const int64_t n = L->A.nr;
    L->dinv = P.get<double>(n);
    if (!L->dinv) { rc = P.err; break; }
    l1_inv(L->A, L->dinv, derr, s);
    if (n <= o.amg_max_coarse || k + 1 >= o.amg_max_levels || k + 1 >= 32) break;
    g_trace.mark("amg l1", slot, k);
    int64_t nc = 0;
    int64_t* cmap = nullptr;
    const bool agg = slot < MGR_MAX_LEVELS && k < o.agg_levels[slot];
    // an aggressive level's first-stage interpolation is scratch
    if ((rc = coarsen_step(o, P, agg ? tmp : P, tmp, L->A, L->comp, slot, k, L->S, &L->cf, &cmap, L->P,
                           &nc, s)))
      break;
    if (nc == 0 || nc == n) break;
    if (agg) {
      // aggressive coarsening, second stage: the same step on the Galerkin
      // operator of the first C points (PMIS weights keyed by level 32 + k),
      // then P = P1 P2 truncated to P_max
      Csr R1, AP1, A1, S1, P2;
      if ((rc = transpose(tmp, tmp, L->P, R1, true, true, s))) break;
      if ((rc = spgemm(tmp, tmp, L->A, L->P, AP1, s))) break;
      if ((rc = spgemm(tmp, tmp, R1, AP1, A1, s))) break;
      int32_t* comp1 = tmp.get<int32_t>(nc);
      if (tmp.err) { rc = tmp.err; break; }
      MGR_LAUNCH k_coarse_comp<<<nblocks(n, 256), 256, 0, s>>>(L->cf, cmap, L->comp, n, comp1);
      int8_t* cf2 = nullptr;
      int64_t* cmap2 = nullptr;
      int64_t nc2 = 0;
      if ((rc = coarsen_step(o, tmp, tmp, tmp, A1, comp1, slot, 32 + k, S1, &cf2, &cmap2, P2, &nc2, s))) break;
      Csr Pfin = L->P;
      if (nc2 > 0 && nc2 < nc) {
        Csr PP;
        if ((rc = spgemm(tmp, tmp, L->P, P2, PP, s))) break;
        int64_t* tcnt = tmp.get<int64_t>(n + 1);
        Pfin.nr = n;
        Pfin.nc = nc2;
        Pfin.rp = P.get<int64_t>(n + 1);
        if (tmp.err || P.err) { rc = tmp.err ? tmp.err : P.err; break; }
        MGR_LAUNCH k_trunc_rows<false><<<nblocks(n, 128), 128, 0, s>>>(PP.rp, PP.ci, PP.v, n, o.amg_pmax,
                                                                       tcnt, nullptr, nullptr);
        if ((rc = rowptr_from_counts(tcnt, Pfin.rp, n, &Pfin.nnz, s, tmp))) break;
        Pfin.ci = P.get<int32_t>(Pfin.nnz);
        Pfin.v = P.get<double>(Pfin.nnz);
        if (P.err) { rc = P.err; break; }
        MGR_LAUNCH k_trunc_rows<true><<<nblocks(n, 128), 128, 0, s>>>(PP.rp, PP.ci, PP.v, n, o.amg_pmax,
                                                                      Pfin.rp, Pfin.ci, Pfin.v);
        MGR_LAUNCH k_agg_cf<<<nblocks(n, 256), 256, 0, s>>>(L->cf, cmap, cf2, n);
        // numbering of the final C points
        int64_t* flag = tmp.get<int64_t>(n + 1);
        cmap = tmp.get<int64_t>(n + 1);
        if (tmp.err) { rc = tmp.err; break; }
        MGR_LAUNCH k_flag_c<<<nblocks(n, 256), 256, 0, s>>>(L->cf, n, flag);
        if ((rc = rowptr_from_counts(flag, cmap, n, &nc, s, tmp))) break;
      } else {
        // the second stage cannot coarsen: an ordinary level (keep P1)
        if ((rc = copy_csr(P, L->P, Pfin, s))) break;
      }
      L->P = Pfin;
      g_trace.mark("amg aggressive stage 2", slot, k);
    }
    if ((rc = transpose(P, tmp, L->P, L->R, true, true, s))) break;
    g_trace.mark("amg transpose P", slot, k);
    Csr AP;
    if ((rc = spgemm(tmp, tmp, L->A, L->P, AP, s))) break;
    g_trace.mark("amg A*P", slot, k);
    g->lev.emplace_back();
    L = &g->lev[k];
    AmgLevel& C = g->lev[k + 1];
    if ((rc = spgemm(P, tmp, L->R, AP, C.A, s))) break;
    C.comp = P.get<int32_t>(nc);
    if (P.err) { rc = P.err; break; }
    MGR_LAUNCH k_coarse_comp<<<nblocks(n, 256), 256, 0, s>>>(L->cf, cmap, L->comp, n, C.comp);
    MGR_TRY_CUDA(cudaGetLastError());
    g_trace.mark("amg R*(AP)", slot, k);
  }
  if (rc == MGR_SUCCESS) rc = check_dev_err(derr, s);
  if (rc == MGR_SUCCESS) rc = dense_coarsest(P, derr, g, tmp, s);
  // shared row patterns of the finest operator (the mesh's own stencil)
  if (rc == MGR_SUCCESS && g->lev[0].A.nnz >= PAT_MIN_NNZ) rc = build_row_patterns(P, g->lev[0].A, s);
  g_trace.mark("amg coarsest inverse", slot, (int)g->lev.size() - 1);
  tmp.free_all_async(s);
  return rc;
}

// ============================================================================
// MGR hierarchy
// ============================================================================
// An F-relaxation AMG whose inputs (A_FF, component ids) are owned by h->pool2,
// to be built by the caller on a second stream.
struct AmgJob {
  Csr A;
  int32_t* comp = nullptr;
  int slot = 0;
  Amg** out = nullptr;
};

// The second stream and host thread of build_mgr_hierarchy.
struct SideBuild {
  bool busy = false;
  std::thread th;
  cudaStream_t ss = nullptr;
  int rc = MGR_SUCCESS;

  cudaStream_t hs = nullptr;   // high-priority stream of the main thread after the fork

  // Starts the side build; *ms becomes the main thread's stream from here on
  // (highest priority, so the main branch's short, host-synchronised kernels
  // get SMs ahead of the side build's long ones).
  int start(Handle* h, const AmgJob& job, cudaStream_t s, cudaStream_t* ms) {
    int dev = 0, lo = 0, hi = 0;
    MGR_TRY_CUDA(cudaGetDevice(&dev));
    MGR_TRY_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    MGR_TRY_CUDA(cudaStreamCreateWithPriority(&ss, cudaStreamNonBlocking, lo));
    MGR_TRY_CUDA(cudaStreamCreateWithPriority(&hs, cudaStreamNonBlocking, hi));
    if (!h->derr2) {
      h->derr2 = h->pool2.get<int>(1);
      if (!h->derr2) return h->pool2.err;
      MGR_TRY_CUDA(cudaMemsetAsync(h->derr2, 0, sizeof(int), s));
    }
    cudaEvent_t fork;
    MGR_TRY_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    MGR_TRY_CUDA(cudaEventRecord(fork, s));
    MGR_TRY_CUDA(cudaStreamWaitEvent(ss, fork, 0));
    MGR_TRY_CUDA(cudaStreamWaitEvent(hs, fork, 0));
    cudaEventDestroy(fork);
    h->pool2.s = ss;   // from here on only the side thread allocates from pool2
    h->pool.s = hs;    // and the main thread allocates in its new stream's order
    g_trace.s = hs;
    *ms = hs;
    busy = true;
    th = std::thread([this, h, job, dev] {
      cudaSetDevice(dev);
      g_trace.start(ss);   // MGR_TRACE: this thread's phases are printed too
      rc = build_amg(h, h->pool2, h->derr2, job.A, true, job.comp, job.slot, job.out, ss);
    });
    return MGR_SUCCESS;
  }
  // join the thread; s then waits for both streams' work and is again the
  // stream of the handle's pool
  int finish(Handle* h, cudaStream_t s) {
    if (!busy) return MGR_SUCCESS;
    th.join();
    busy = false;
    int r = rc;
    for (cudaStream_t x : {ss, hs}) {
      cudaEvent_t join;
      if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess) {
        if (cudaEventRecord(join, x) != cudaSuccess || cudaStreamWaitEvent(s, join, 0) != cudaSuccess)
          r = r ? r : MGR_ERR_CUDA;
        cudaEventDestroy(join);
      } else {
        cudaStreamSynchronize(x);
      }
      cudaStreamDestroy(x);
    }
    ss = hs = nullptr;
    h->pool.s = s;
    g_trace.s = s;
    return r;
  }
  ~SideBuild() {
    if (th.joinable()) th.join();   // every path calls finish(); this is a backstop
  }
};

// ============================================================================
// ILU(1) global smoother (Sec. 6: one sweep of pointwise ILU(1) is the global
// smoother of the second reduction level).  The pattern is level-1 fill:
// pattern(A) + pattern(L_A U_A) with L_A, U_A the strict triangles of A.  The
// factors are the exact incomplete factors on that pattern (the fixed point of
// the fine-grained iteration the paper cites), computed by IKJ elimination:
// rows are grouped by dependency depth and each group is eliminated in one
// launch, every row by one warp in ascending k, so each entry receives the
// same sequence of roundings as sequential elimination.
// ============================================================================
// Strict lower (LOWER) or strict upper triangle of a CSR matrix; values are
// copied when ov is non-null.  Thread per row.
template <bool FILL, bool LOWER>
__global__ void k_tri(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                      const double* __restrict__ v, int64_t n, int64_t* __restrict__ cnt_or_rp,
                      int32_t* __restrict__ oci, double* __restrict__ ov) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = FILL ? cnt_or_rp[i] : 0;
  for (int64_t q = rp[i]; q < rp[i + 1]; q++) {
    const int64_t c = ci[q];
    if (LOWER ? (c < i) : (c > i)) {
      if (FILL) {
        oci[o] = (int32_t)c;
        if (ov) ov[o] = v[q];
      }
      o++;
    }
  }
  if (!FILL) cnt_or_rp[i] = o;
}

static int tri_part(Pool& P, Pool& tmp, const Csr& A, bool lower, bool values, Csr& T,
                    cudaStream_t s) {
  int64_t* cnt = tmp.get<int64_t>(A.nr + 1);
  T.nr = A.nr;
  T.nc = A.nc;
  T.rp = P.get<int64_t>(A.nr + 1);
  if (tmp.err || P.err) return tmp.err ? tmp.err : P.err;
  const unsigned g = nblocks(A.nr, 256);
  if (lower) MGR_LAUNCH k_tri<false, true><<<g, 256, 0, s>>>(A.rp, A.ci, nullptr, A.nr, cnt, nullptr, nullptr);
  else MGR_LAUNCH k_tri<false, false><<<g, 256, 0, s>>>(A.rp, A.ci, nullptr, A.nr, cnt, nullptr, nullptr);
  MGR_TRY(rowptr_from_counts(cnt, T.rp, A.nr, &T.nnz, s, tmp));
  T.ci = P.get<int32_t>(T.nnz);
  T.v = values ? P.get<double>(T.nnz) : nullptr;
  if (P.err) return P.err;
  const double* av = values ? A.v : nullptr;
  if (lower) MGR_LAUNCH k_tri<true, true><<<g, 256, 0, s>>>(A.rp, A.ci, av, A.nr, T.rp, T.ci, T.v);
  else MGR_LAUNCH k_tri<true, false><<<g, 256, 0, s>>>(A.rp, A.ci, av, A.nr, T.rp, T.ci, T.v);
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

// F = pattern(A) + pattern(K) with values a_ij, or +0.0 where A has no entry.
template <bool FILL>
__global__ void k_union_fill0(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                              const double* __restrict__ av, const int64_t* __restrict__ krp,
                              const int32_t* __restrict__ kci, int64_t nr,
                              int64_t* __restrict__ cnt_or_rp, int32_t* __restrict__ fci,
                              double* __restrict__ fv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  int64_t p = arp[i], pe = arp[i + 1], q = krp[i], qe = krp[i + 1];
  int64_t o = FILL ? cnt_or_rp[i] : 0;
  while (p < pe || q < qe) {
    const int64_t cp = (p < pe) ? aci[p] : INT64_MAX;
    const int64_t cq = (q < qe) ? kci[q] : INT64_MAX;
    if (FILL) {
      fci[o] = (int32_t)(cp <= cq ? cp : cq);
      fv[o] = (cp <= cq) ? av[p] : 0.0;
    }
    if (cp <= cq) {
      p++;
      if (cp == cq) q++;
    } else {
      q++;
    }
    o++;
  }
  if (!FILL) cnt_or_rp[i] = o;
}

// position of the diagonal entry of each row (a missing one is a zero pivot)
__global__ void k_diag_pos(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n,
                           int64_t* __restrict__ dpos, int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t r = rp[i];
  while (r < rp[i + 1] && ci[r] != i) r++;
  if (r == rp[i + 1]) {
    dev_fail(err, DEV_ZERO_DIAG);
    r = rp[i];
  }
  dpos[i] = r;
}

// One relaxation pass of depth(i) = max over the lower entries k of row i of
// depth(k) + 1 (0 without lower entries), in place.  Depths only grow and
// never pass the longest dependency chain, so a pass that changes nothing
// has reached the unique solution.
__global__ void k_ilu_depth(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const int64_t* __restrict__ dpos, int64_t n, int32_t* depth,
                            unsigned long long* changed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t m = 0;
  for (int64_t q = rp[i]; q < dpos[i]; q++) {
    const int32_t d = depth[ci[q]] + 1;
    m = d > m ? d : m;
  }
  if (m != depth[i]) {
    depth[i] = m;
    atomicAdd(changed, 1ull);
  }
}

__global__ void k_imax(const int32_t* __restrict__ a, int64_t n, int* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(out, a[i]);
}

// IKJ elimination of the rows of one depth, a warp per row.  Row i takes its
// lower entries in ascending k: l_ik = w_ik / u_kk, then w_ij -= l_ik u_kj for
// every column j > k present in both rows (rows k < i are final: they have a
// smaller depth).  Each lane updates distinct entries of row i.
__global__ void __launch_bounds__(256)
k_ilu_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, double* v,
           const int64_t* __restrict__ dpos, const int64_t* __restrict__ rows, int64_t cnt,
           int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= cnt) return;   // whole warps
  const int64_t i = rows[t];
  const int64_t r1 = rp[i + 1], di = dpos[i];
  for (int64_t q = rp[i]; q < di; q++) {
    const int64_t k = ci[q];
    const int64_t dk = dpos[k];
    const double ukk = v[dk];
    if (ukk == 0.0) {
      if (lane == 0) dev_fail(err, DEV_ZERO_DIAG);
      return;
    }
    const double lik = __ddiv_rn(v[q], ukk);
    __syncwarp();
    if (lane == 0) v[q] = lik;
    const int64_t k1 = rp[k + 1];
    for (int64_t pk = dk + 1 + lane; pk < k1; pk += 32) {
      const int32_t j = ci[pk];
      int64_t lo = q + 1, hi = r1;   // first position in (q, r1) with column >= j
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ci[mid] < j) lo = mid + 1;
        else hi = mid;
      }
      if (lo < r1 && ci[lo] == j) v[lo] = __dsub_rn(v[lo], __dmul_rn(lik, v[pk]));
    }
    __syncwarp();
  }
  if (lane == 0 && v[di] == 0.0) dev_fail(err, DEV_ZERO_DIAG);
}

__global__ void k_diag_inv(const double* __restrict__ v, const int64_t* __restrict__ dpos, int64_t n,
                           double* __restrict__ dinv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dinv[i] = __ddiv_rn(1.0, v[dpos[i]]);
}

static int ilu1_build(Handle* h, Pool& P, Pool& tmp, MgrLevel& L, cudaStream_t s) {
  const Csr& A = L.A;
  const int64_t n = A.nr;
  // level-1 pattern and the values of A on it
  Csr lo, up, lu;
  MGR_TRY(tri_part(tmp, tmp, A, true, false, lo, s));
  MGR_TRY(tri_part(tmp, tmp, A, false, false, up, s));
  MGR_TRY(spgemm_pattern(tmp, tmp, lo, up, lu, s));
  Csr& F = L.ilu;
  F.nr = F.nc = n;
  F.rp = P.get<int64_t>(n + 1);
  int64_t* cnt = tmp.get<int64_t>(n + 1);
  if (P.err || tmp.err) return P.err ? P.err : tmp.err;
  const unsigned g = nblocks(n, 256);
  MGR_LAUNCH k_union_fill0<false><<<g, 256, 0, s>>>(A.rp, A.ci, A.v, lu.rp, lu.ci, n, cnt, nullptr, nullptr);
  MGR_TRY(rowptr_from_counts(cnt, F.rp, n, &F.nnz, s, tmp));
  F.ci = P.get<int32_t>(F.nnz);
  F.v = P.get<double>(F.nnz);
  int64_t* dpos = tmp.get<int64_t>(n);
  int32_t* depth = tmp.get<int32_t>(n);
  if (P.err || tmp.err) return P.err ? P.err : tmp.err;
  MGR_LAUNCH k_union_fill0<true><<<g, 256, 0, s>>>(A.rp, A.ci, A.v, lu.rp, lu.ci, n, F.rp, F.ci, F.v);
  MGR_LAUNCH k_diag_pos<<<g, 256, 0, s>>>(F.rp, F.ci, n, dpos, h->derr);
  MGR_TRY(check_dev_err(h->derr, s));
  // dependency depths: relaxation passes, four per host check, at most n + 1
  // passes (the longest chain has at most n rows)
  static constexpr int PASSES = 4;
  unsigned long long* chg = tmp.get<unsigned long long>(PASSES);
  int* dmax = tmp.get<int>(1);
  if (tmp.err) return tmp.err;
  MGR_TRY_CUDA(cudaMemsetAsync(depth, 0, sizeof(int32_t) * n, s));
  bool done = false;
  for (int64_t p0 = 0; p0 <= n + PASSES && !done; p0 += PASSES) {
    MGR_TRY_CUDA(cudaMemsetAsync(chg, 0, sizeof(unsigned long long) * PASSES, s));
    for (int q = 0; q < PASSES; q++)
      MGR_LAUNCH k_ilu_depth<<<g, 256, 0, s>>>(F.rp, F.ci, dpos, n, depth, chg + q);
    unsigned long long hc[PASSES];
    MGR_TRY_CUDA(cudaMemcpyAsync(hc, chg, sizeof(hc), cudaMemcpyDeviceToHost, s));
    MGR_TRY_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < PASSES; q++) done = done || hc[q] == 0;
  }
  if (!done) return MGR_ERR_CUDA;   // cannot happen: depths are bounded by n
  MGR_TRY_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
  MGR_LAUNCH k_imax<<<g, 256, 0, s>>>(depth, n, dmax);
  int nd = 0;
  MGR_TRY(read_back(&nd, dmax, s));
  nd += 1;
  // rows grouped by depth
  int64_t* dcnt = tmp.get<int64_t>(nd + 1);
  int64_t* order = tmp.get<int64_t>(n);
  if (tmp.err) return tmp.err;
  MGR_TRY_CUDA(cudaMemsetAsync(dcnt, 0, sizeof(int64_t) * (nd + 1), s));
  MGR_LAUNCH k_color_count<<<g, 256, 0, s>>>(depth, n, dcnt);
  std::vector<int64_t> hcnt(nd), off(nd + 1, 0);
  MGR_TRY_CUDA(cudaMemcpyAsync(hcnt.data(), dcnt, sizeof(int64_t) * nd, cudaMemcpyDeviceToHost, s));
  MGR_TRY_CUDA(cudaStreamSynchronize(s));
  for (int d = 0; d < nd; d++) off[d + 1] = off[d] + hcnt[d];
  MGR_TRY_CUDA(cudaMemcpyAsync(dcnt, off.data(), sizeof(int64_t) * nd, cudaMemcpyHostToDevice, s));
  MGR_LAUNCH k_color_place<<<g, 256, 0, s>>>(depth, n, dcnt, order);
  // elimination, one launch per depth
  for (int d = 0; d < nd; d++) {
    const int64_t c = off[d + 1] - off[d];
    if (c == 0) continue;
    MGR_LAUNCH k_ilu_rows<<<nblocks(c * 32, 256), 256, 0, s>>>(F.rp, F.ci, F.v, dpos, order + off[d], c,
                                                                h->derr);
  }
  MGR_TRY(check_dev_err(h->derr, s));
  // split for the triangular iterations
  MGR_TRY(tri_part(P, tmp, F, true, true, L.Ilo, s));
  MGR_TRY(tri_part(P, tmp, F, false, true, L.Iup, s));
  L.ilu_dinv = P.get<double>(n);
  if (P.err) return P.err;
  MGR_LAUNCH k_diag_inv<<<g, 256, 0, s>>>(F.v, dpos, n, L.ilu_dinv);
  MGR_TRY_CUDA(cudaGetLastError());
  L.ilu1 = true;
  return MGR_SUCCESS;
}

// s is the calling thread's stream; it changes (to the main thread's
// high-priority stream) when this level hands its F-relaxation AMG to the
// side build.
static int setup_level(Handle* h, int l, const int32_t* label, const int32_t* node,
                       const int32_t* comp, Pool& tmp, cudaStream_t& s, Csr& Snext,
                       int32_t** nlabel, int32_t** nnode, int32_t** ncomp, SideBuild* side) {
  Pool& P = h->pool;
  MgrLevel& L = h->lev[l];
  const mgr_options_t& o = h->opt;
  const int64_t n = L.A.nr;
  L.n = n;
  L.label = const_cast<int32_t*>(label);
  L.node = const_cast<int32_t*>(node);
  L.comp = const_cast<int32_t*>(comp);
  L.frelax = o.frelax[l];
  L.frelax_sweeps = o.frelax_sweeps[l];
  L.global_sweeps = o.global_sweeps[l];
  L.restrict_jacobi = o.restrict_jacobi[l] != 0;
  L.frelax_post = o.frelax_post[l] != 0;
  L.dff_block = o.dff_block[l] != 0;
  if (L.frelax != MGR_FRELAX_AMG_VCYCLE && L.frelax != MGR_FRELAX_JACOBI) return MGR_ERR_INVALID_ARG;
  if (L.frelax_sweeps < 0 || L.global_sweeps < 0) return MGR_ERR_INVALID_ARG;

  int64_t* flag = tmp.get<int64_t>(n + 1);
  int64_t* fpos = tmp.get<int64_t>(n + 1);
  int32_t* colF = tmp.get<int32_t>(n);
  int32_t* colC = tmp.get<int32_t>(n);
  if (tmp.err) return tmp.err;
  MGR_LAUNCH k_flag_f<<<nblocks(n, 256), 256, 0, s>>>(label, n, o.f_label_mask[l], flag, h->derr);
  MGR_TRY(rowptr_from_counts(flag, fpos, n, &L.nF, s, tmp));
  MGR_TRY(check_dev_err(h->derr, s));
  L.nC = n - L.nF;
  if (L.nF == 0 || L.nC == 0) return MGR_ERR_INVALID_ARG;
  L.Fidx = P.get<int64_t>(L.nF);
  L.Cidx = P.get<int64_t>(L.nC);
  if (P.err) return P.err;
  MGR_LAUNCH k_split<<<nblocks(n, 256), 256, 0, s>>>(fpos, n, L.Fidx, L.Cidx, colF, colC);
  {
    int64_t last_f = -1;
    MGR_TRY(read_back(&last_f, L.Fidx + (L.nF - 1), s));
    L.F_is_prefix = (last_f == L.nF - 1);
  }
  // blocks of A: A_FF (tmp), A_FC (tmp), A_CF, A_CC (tmp)
  Csr Aff, Afc, Acc;
  MGR_TRY(extract(tmp, tmp, L.A, L.Fidx, L.nF, colF, L.nF, Aff, s));
  // F-relaxation AMG on A_FF: handed to the side build (second stream and
  // thread) as soon as A_FF exists, when the side build is free
  if (L.frelax == MGR_FRELAX_AMG_VCYCLE && L.frelax_sweeps > 0) {
    int32_t* fcomp = tmp.get<int32_t>(L.nF);
    int32_t* dummy1 = tmp.get<int32_t>(L.nF);
    int32_t* dummy2 = tmp.get<int32_t>(L.nF);
    if (tmp.err) return tmp.err;
    MGR_LAUNCH k_gather3<<<nblocks(L.nF, 256), 256, 0, s>>>(comp, label, node, L.Fidx, L.nF, fcomp, dummy1, dummy2);
    if (side && !side->busy) {
      // its inputs are copied into the second pool (ordered on s; the side
      // stream waits for s before using them)
      AmgJob job;
      Pool& P2 = h->pool2;
      P2.s = s;
      MGR_TRY(copy_csr(P2, Aff, job.A, s));
      job.comp = P2.get<int32_t>(L.nF);
      if (!job.comp) return P2.err;
      MGR_TRY_CUDA(cudaMemcpyAsync(job.comp, fcomp, sizeof(int32_t) * L.nF, cudaMemcpyDeviceToDevice, s));
      job.slot = l;
      job.out = &L.famg;
      MGR_TRY(side->start(h, job, s, &s));
      tmp.s = s;
    } else {
      MGR_TRY(build_amg(h, P, h->derr, Aff, false, fcomp, l, &L.famg, s));
    }
  }
  MGR_TRY(extract(tmp, tmp, L.A, L.Fidx, L.nF, colC, L.nC, Afc, s));
  MGR_TRY(extract(P, tmp, L.A, L.Cidx, L.nC, colF, L.nF, L.Acf, s));
  MGR_TRY(extract(tmp, tmp, L.A, L.Cidx, L.nC, colC, L.nC, Acc, s));
  // D_FF, T = D^-1 A_FC, W_p = -T (pointwise D_FF: t = a / d)
  L.dFinv = P.get<double>(L.nF);
  double* dval = tmp.get<double>(L.nF);
  Pool& Pw = L.dff_block ? tmp : P;   // the point-block W_p replaces this one
  L.W = Afc;
  L.W.rp = Pw.get<int64_t>(L.nF + 1);
  L.W.ci = Pw.get<int32_t>(Afc.nnz);
  L.W.v = Pw.get<double>(Afc.nnz);
  Csr T = Afc;
  T.v = tmp.get<double>(Afc.nnz);
  if (P.err || tmp.err) return P.err ? P.err : tmp.err;
  MGR_TRY_CUDA(cudaMemcpyAsync(L.W.rp, Afc.rp, sizeof(int64_t) * (L.nF + 1), cudaMemcpyDeviceToDevice, s));
  MGR_TRY_CUDA(cudaMemcpyAsync(L.W.ci, Afc.ci, sizeof(int32_t) * Afc.nnz, cudaMemcpyDeviceToDevice, s));
  MGR_LAUNCH k_dff_and_w<<<nblocks(L.nF, 256), 256, 0, s>>>(L.A.rp, L.A.ci, L.A.v, L.Fidx, L.nF, Afc.rp, Afc.v,
                                                  T.v, L.W.v, L.dFinv, dval, h->derr);
  MGR_TRY(check_dev_err(h->derr, s));
  if (L.dff_block) {
    // point-block D_FF: runs of F dofs sharing dof_node (at most 4), their
    // inverses (Gauss-Jordan, as the global smoother's blocks) as a sparse
    // matrix Bd; T = Bd A_FC, W_p = -T
    int32_t* nodeF = tmp.get<int32_t>(L.nF);
    int32_t* dumA = tmp.get<int32_t>(L.nF);
    int32_t* dumB = tmp.get<int32_t>(L.nF);
    int64_t* head = tmp.get<int64_t>(L.nF + 1);
    int64_t* hpos = tmp.get<int64_t>(L.nF + 1);
    if (tmp.err) return tmp.err;
    MGR_LAUNCH k_gather3<<<nblocks(L.nF, 256), 256, 0, s>>>(node, node, node, L.Fidx, L.nF, nodeF, dumA, dumB);
    MGR_LAUNCH k_block_heads<<<nblocks(L.nF, 256), 256, 0, s>>>(nodeF, L.nF, head);
    int64_t nb = 0;
    MGR_TRY(rowptr_from_counts(head, hpos, L.nF, &nb, s, tmp));
    int64_t* bst = tmp.get<int64_t>(nb + 1);
    double* binv = tmp.get<double>(16 * nb);
    int64_t* cnt = tmp.get<int64_t>(L.nF + 1);
    if (tmp.err) return tmp.err;
    MGR_LAUNCH k_block_starts<<<nblocks(L.nF + 1, 256), 256, 0, s>>>(hpos, L.nF, bst, nb);
    MGR_LAUNCH k_block_inv<<<nblocks(nb, 128), 128, 0, s>>>(Aff.rp, Aff.ci, Aff.v, bst, nb, binv, h->derr);
    MGR_TRY(check_dev_err(h->derr, s));
    MGR_LAUNCH k_bd_counts<<<nblocks(nb, 256), 256, 0, s>>>(bst, nb, cnt);
    L.Bd.nr = L.Bd.nc = L.nF;
    L.Bd.rp = P.get<int64_t>(L.nF + 1);
    if (P.err) return P.err;
    MGR_TRY(rowptr_from_counts(cnt, L.Bd.rp, L.nF, &L.Bd.nnz, s, tmp));
    L.Bd.ci = P.get<int32_t>(L.Bd.nnz);
    L.Bd.v = P.get<double>(L.Bd.nnz);
    if (P.err) return P.err;
    MGR_LAUNCH k_bd_fill<<<nblocks(nb, 256), 256, 0, s>>>(bst, nb, binv, L.Bd.rp, L.Bd.ci, L.Bd.v);
    Csr Tb;
    MGR_TRY(spgemm(tmp, tmp, L.Bd, Afc, Tb, s));
    T = Tb;
    L.W = Tb;
    L.W.rp = P.get<int64_t>(L.nF + 1);
    L.W.ci = P.get<int32_t>(Tb.nnz);
    L.W.v = P.get<double>(Tb.nnz);
    if (P.err) return P.err;
    MGR_TRY_CUDA(cudaMemcpyAsync(L.W.rp, Tb.rp, sizeof(int64_t) * (L.nF + 1), cudaMemcpyDeviceToDevice, s));
    MGR_TRY_CUDA(cudaMemcpyAsync(L.W.ci, Tb.ci, sizeof(int32_t) * Tb.nnz, cudaMemcpyDeviceToDevice, s));
    MGR_LAUNCH k_neg<<<grid_for(Tb.nnz, 256, 152 * 16), 256, 0, s>>>(Tb.v, L.W.v, Tb.nnz);
  }
  g_trace.mark("mgr split/extract/W", l);
  // A_cor = A_CF T
  if (!L.restrict_jacobi) {
    MGR_TRY(spgemm(P, tmp, L.Acf, T, L.cor, s));
  } else {
    // Jacobi restriction: U = A_CF D_FF^-1, W_r = -U; R~ A P~ = A_CC - A_cor
    // with A_cor = 2 A_CF T - U (A_FF T), formed on the union pattern
    Csr C1, U, K, E;
    MGR_TRY(spgemm(tmp, tmp, L.Acf, T, C1, s));
    if (L.dff_block) {
      MGR_TRY(spgemm(tmp, tmp, L.Acf, L.Bd, U, s));
      L.Wr = U;
      L.Wr.rp = P.get<int64_t>(L.nC + 1);
      L.Wr.ci = P.get<int32_t>(U.nnz);
      L.Wr.v = P.get<double>(U.nnz);
      if (P.err) return P.err;
      MGR_TRY_CUDA(cudaMemcpyAsync(L.Wr.rp, U.rp, sizeof(int64_t) * (L.nC + 1), cudaMemcpyDeviceToDevice, s));
      MGR_TRY_CUDA(cudaMemcpyAsync(L.Wr.ci, U.ci, sizeof(int32_t) * U.nnz, cudaMemcpyDeviceToDevice, s));
      MGR_LAUNCH k_neg<<<grid_for(U.nnz, 256, 152 * 16), 256, 0, s>>>(U.v, L.Wr.v, U.nnz);
    } else {
      U = L.Acf;
      U.v = tmp.get<double>(L.Acf.nnz);
      L.Wr = L.Acf;
      L.Wr.v = P.get<double>(L.Acf.nnz);   // shares A_CF's row pointers and columns
      if (P.err || tmp.err) return P.err ? P.err : tmp.err;
      MGR_LAUNCH k_acf_dinv<<<nblocks(L.Acf.nnz, 256), 256, 0, s>>>(L.Acf.ci, L.Acf.v, L.Acf.nnz, dval, U.v, L.Wr.v);
    }
    MGR_TRY(spgemm(tmp, tmp, Aff, T, K, s));
    MGR_TRY(spgemm(tmp, tmp, U, K, E, s));
    MGR_LAUNCH k_twice<<<grid_for(C1.nnz, 256, 152 * 16), 256, 0, s>>>(C1.v, C1.nnz);
    int64_t* ucnt = tmp.get<int64_t>(L.nC + 1);
    L.cor.nr = L.cor.nc = L.nC;
    L.cor.rp = P.get<int64_t>(L.nC + 1);
    if (P.err || tmp.err) return P.err ? P.err : tmp.err;
    MGR_LAUNCH k_union_sub<false><<<nblocks(L.nC, 256), 256, 0, s>>>(C1.rp, C1.ci, C1.v, E.rp, E.ci, E.v,
                                                                   L.nC, ucnt, nullptr, nullptr);
    MGR_TRY(rowptr_from_counts(ucnt, L.cor.rp, L.nC, &L.cor.nnz, s, tmp));
    L.cor.ci = P.get<int32_t>(L.cor.nnz);
    L.cor.v = P.get<double>(L.cor.nnz);
    if (P.err) return P.err;
    MGR_LAUNCH k_union_sub<true><<<nblocks(L.nC, 256), 256, 0, s>>>(C1.rp, C1.ci, C1.v, E.rp, E.ci, E.v,
                                                                  L.nC, L.cor.rp, L.cor.ci, L.cor.v);
  }
  g_trace.mark("mgr A_CF*T", l);
  // next-level labels (needed for G's own-point rule)
  *nlabel = P.get<int32_t>(L.nC);
  *nnode = P.get<int32_t>(L.nC);
  *ncomp = P.get<int32_t>(L.nC);
  if (P.err) return P.err;
  MGR_LAUNCH k_gather3<<<nblocks(L.nC, 256), 256, 0, s>>>(label, node, comp, L.Cidx, L.nC, *nlabel, *nnode, *ncomp);
  // G
  int8_t* keep = tmp.get<int8_t>(L.cor.nnz);
  int64_t* cnt = tmp.get<int64_t>(L.nC + 1);
  if (tmp.err) return tmp.err;
  MGR_LAUNCH k_drop_mark<<<nblocks(L.nC, 128), 128, 0, s>>>(L.cor.rp, L.cor.ci, L.cor.v, L.nC, *nnode,
                                                  o.nmax_drop[l], keep, cnt);
  L.corkept.nr = L.corkept.nc = L.nC;
  L.corkept.rp = P.get<int64_t>(L.nC + 1);
  if (P.err) return P.err;
  MGR_TRY(rowptr_from_counts(cnt, L.corkept.rp, L.nC, &L.corkept.nnz, s, tmp));
  L.corkept.ci = P.get<int32_t>(L.corkept.nnz);
  L.corkept.v = P.get<double>(L.corkept.nnz);
  if (P.err) return P.err;
  MGR_LAUNCH k_drop_fill<<<nblocks(L.nC, 256), 256, 0, s>>>(L.cor.rp, L.cor.ci, L.cor.v, L.nC, keep,
                                                  L.corkept.rp, L.corkept.ci, L.corkept.v);
  // S = A_CC - G(A_cor)
  Snext.nr = Snext.nc = L.nC;
  Snext.rp = P.get<int64_t>(L.nC + 1);
  if (P.err) return P.err;
  MGR_LAUNCH k_union_sub<false><<<nblocks(L.nC, 256), 256, 0, s>>>(Acc.rp, Acc.ci, Acc.v, L.corkept.rp,
                                                       L.corkept.ci, L.corkept.v, L.nC, cnt,
                                                       nullptr, nullptr);
  MGR_TRY(rowptr_from_counts(cnt, Snext.rp, L.nC, &Snext.nnz, s, tmp));
  Snext.ci = P.get<int32_t>(Snext.nnz);
  Snext.v = P.get<double>(Snext.nnz);
  if (P.err) return P.err;
  MGR_LAUNCH k_union_sub<true><<<nblocks(L.nC, 256), 256, 0, s>>>(Acc.rp, Acc.ci, Acc.v, L.corkept.rp,
                                                      L.corkept.ci, L.corkept.v, L.nC, Snext.rp,
                                                      Snext.ci, Snext.v);
  MGR_TRY_CUDA(cudaGetLastError());
  g_trace.mark("mgr drop + S", l);
  // point-block global smoother
  if (L.global_sweeps > 0) {
    int64_t* head = tmp.get<int64_t>(n + 1);
    int64_t* hpos = tmp.get<int64_t>(n + 1);
    if (tmp.err) return tmp.err;
    MGR_LAUNCH k_block_heads<<<nblocks(n, 256), 256, 0, s>>>(node, n, head);
    MGR_TRY(rowptr_from_counts(head, hpos, n, &L.nblk, s, tmp));
    L.bstart = P.get<int64_t>(L.nblk + 1);
    L.binv = P.get<double>(16 * L.nblk);
    if (P.err) return P.err;
    MGR_LAUNCH k_block_starts<<<nblocks(n + 1, 256), 256, 0, s>>>(hpos, n, L.bstart, L.nblk);
    MGR_LAUNCH k_block_inv<<<nblocks(L.nblk, 128), 128, 0, s>>>(L.A.rp, L.A.ci, L.A.v, L.bstart, L.nblk,
                                                      L.binv, h->derr);
    MGR_TRY(check_dev_err(h->derr, s));
    {
      int* dmax = tmp.get<int>(1);
      if (tmp.err) return tmp.err;
      MGR_TRY_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
      MGR_LAUNCH k_block_dim_max<<<nblocks(L.nblk, 256), 256, 0, s>>>(L.bstart, L.nblk, dmax);
      MGR_TRY(read_back(&L.bdim, dmax, s));
      if (L.bdim < 1 || L.bdim > 4) return MGR_ERR_INVALID_ARG;
      L.binvc = P.get<double>((int64_t)L.bdim * L.bdim * L.nblk);
      if (P.err) return P.err;
      MGR_LAUNCH k_compact_binv<<<nblocks((int64_t)L.bdim * L.bdim * L.nblk, 256), 256, 0, s>>>(
          L.binv, L.nblk, L.bdim, L.binvc);
    }
    if (o.global_smoother[l] == 2) {
      L.ilu_solve_sweeps = o.ilu_solve_sweeps;
      MGR_TRY(ilu1_build(h, P, tmp, L, s));
      g_trace.mark("mgr ILU(1)", l);
    } else if (o.global_smoother[l] == 1) {
      // multicolour point-block Gauss-Seidel: colour the block graph, then
      // group the blocks by colour
      L.gs = true;
      Csr AT;
      MGR_TRY(transpose(tmp, tmp, L.A, AT, false, false, s));
      int64_t* blk = tmp.get<int64_t>(n + 1);
      uint64_t* w = tmp.get<uint64_t>(L.nblk);
      static constexpr int MAX_COLORS = 1024;
      unsigned long long* left = tmp.get<unsigned long long>(MAX_COLORS);
      L.bcolor = P.get<int32_t>(L.nblk);
      if (tmp.err || P.err) return tmp.err ? tmp.err : P.err;
      MGR_TRY_CUDA(cudaMemsetAsync(left, 0, sizeof(unsigned long long) * MAX_COLORS, s));
      MGR_LAUNCH k_blk_of<<<nblocks(L.nblk, 256), 256, 0, s>>>(L.bstart, L.nblk, blk);
      MGR_LAUNCH k_color_init<<<nblocks(L.nblk, 256), 256, 0, s>>>(L.nblk, o.seed, l, w, L.bcolor);
      int nc = -1;
      for (int c0 = 0; c0 < MAX_COLORS && nc < 0; c0 += 4) {
        for (int c = c0; c < c0 + 4; c++)
          MGR_LAUNCH k_color_round<<<nblocks(L.nblk, 128), 128, 0, s>>>(L.A.rp, L.A.ci, AT.rp, AT.ci, blk,
                                                                        L.bstart, L.nblk, w, L.bcolor, c,
                                                                        left + c);
        unsigned long long lh[4];
        MGR_TRY_CUDA(cudaMemcpyAsync(lh, left + c0, sizeof(lh), cudaMemcpyDeviceToHost, s));
        MGR_TRY_CUDA(cudaStreamSynchronize(s));
        for (int q = 0; q < 4; q++)
          if (lh[q] == 0) {
            nc = c0 + q + 1;
            break;
          }
      }
      if (nc < 0) return MGR_ERR_INVALID_ARG;   // more than MAX_COLORS colours
      L.ncolor = nc;
      int64_t* cnt = tmp.get<int64_t>(nc + 1);
      L.border = P.get<int64_t>(L.nblk);
      if (tmp.err || P.err) return tmp.err ? tmp.err : P.err;
      MGR_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (nc + 1), s));
      MGR_LAUNCH k_color_count<<<nblocks(L.nblk, 256), 256, 0, s>>>(L.bcolor, L.nblk, cnt);
      std::vector<int64_t> hc(nc);
      MGR_TRY_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(int64_t) * nc, cudaMemcpyDeviceToHost, s));
      MGR_TRY_CUDA(cudaStreamSynchronize(s));
      L.coff.assign(nc + 1, 0);
      for (int c = 0; c < nc; c++) L.coff[c + 1] = L.coff[c] + hc[c];
      MGR_TRY_CUDA(cudaMemcpyAsync(cnt, L.coff.data(), sizeof(int64_t) * nc, cudaMemcpyHostToDevice, s));
      MGR_LAUNCH k_color_place<<<nblocks(L.nblk, 256), 256, 0, s>>>(L.bcolor, L.nblk, cnt, L.border);
      MGR_TRY_CUDA(cudaStreamSynchronize(s));   // coff's host copy outlives the async copy
    }
  }
  return MGR_SUCCESS;
}

int build_mgr_hierarchy(Handle* h, const mgr_matrix_t* A, cudaStream_t s) {
  Pool& P = h->pool;
  const int L = h->L;
  h->lev.resize(L);
  const int64_t n = A->n;
  // own copies of the input
  Csr A0;
  A0.nr = A0.nc = n;
  A0.nnz = A->nnz;
  A0.rp = const_cast<int64_t*>(A->row_ptr);
  A0.ci = const_cast<int32_t*>(A->col_idx);
  A0.v = const_cast<double*>(A->val);
  int32_t* label = P.get<int32_t>(n);
  int32_t* node = P.get<int32_t>(n);
  int32_t* comp = P.get<int32_t>(n);
  if (P.err) return P.err;
  MGR_TRY_CUDA(cudaMemcpyAsync(label, A->dof_label, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  MGR_TRY_CUDA(cudaMemcpyAsync(node, A->dof_node, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  if (A->dof_comp)
    MGR_TRY_CUDA(cudaMemcpyAsync(comp, A->dof_comp, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  else
    MGR_TRY_CUDA(cudaMemsetAsync(comp, 0, sizeof(int32_t) * n, s));
  Csr cur;
  MGR_TRY(copy_csr(P, A0, cur, s));
  // The F-relaxation AMG of the first level that has one (A_uu's, 60% of the
  // setup) depends only on that level's A_FF: it is built on a second stream
  // by a second host thread (own pool and error word) while this thread goes
  // on with the next levels and the coarsest AMG.  Each AMG is built by the
  // same kernels in the same order as when built alone, so the results do not
  // depend on the overlap.
  SideBuild side;
  cudaStream_t ms = s;   // the main thread's stream (changes at the fork)
  int rc = MGR_SUCCESS;
  for (int l = 0; l < L && rc == MGR_SUCCESS; l++) {
    Pool tmp;
    tmp.s = ms;
    h->lev[l].A = cur;
    Csr S;
    int32_t *nl = nullptr, *nn = nullptr, *nc = nullptr;
    rc = setup_level(h, l, label, node, comp, tmp, ms, S, &nl, &nn, &nc, &side);
    tmp.free_all_async(ms);
    if (rc) break;
    cur = S;
    label = nl;
    node = nn;
    comp = nc;
  }
  if (!rc) {
    h->Acoarse = cur;
    // the coarsest MGR level is a scalar problem: one component
    Pool tmp;
    tmp.s = ms;
    int32_t* zero = tmp.get<int32_t>(cur.nr);
    if (!zero) {
      rc = tmp.err;
    } else if (cudaMemsetAsync(zero, 0, sizeof(int32_t) * cur.nr, ms) != cudaSuccess) {
      rc = MGR_ERR_CUDA;
    } else {
      rc = build_amg(h, P, h->derr, cur, false, zero, L, &h->camg, ms);
    }
    tmp.free_all_async(ms);
  }
  const int rc2 = side.finish(h, s);   // always joined, also after an error
  return rc ? rc : rc2;
}

// ============================================================================
// FP32 copies of everything the mixed-precision apply reads
// ============================================================================
__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

static int f32(Pool& P, const double* a, float** b, int64_t n, cudaStream_t s) {
  if (!a || n == 0) return MGR_SUCCESS;
  *b = P.get<float>(n);
  if (!*b) return P.err;
  MGR_LAUNCH k_d2f<<<grid_for(n, 256), 256, 0, s>>>(a, *b, n);
  return MGR_SUCCESS;
}

// BF16 storage of a smoother diagonal: each value rounded once, to nearest
// even, from FP64.
__global__ void k_d2bf(const double* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __double2bfloat16(a[i]);
}

static int bf16(Pool& P, const double* a, __nv_bfloat16** b, int64_t n, cudaStream_t s) {
  if (!a || n == 0) return MGR_SUCCESS;
  *b = P.get<__nv_bfloat16>(n);
  if (!*b) return P.err;
  MGR_LAUNCH k_d2bf<<<grid_for(n, 256), 256, 0, s>>>(a, *b, n);
  return MGR_SUCCESS;
}

// SELL-32 FP32 copy of a patterned operator's values (see Csr::vsell):
// slice lengths (32 x the slice's longest row), their exclusive scan into
// soff, then every value rounded once from FP64 into its slot, zero padding.
__global__ void k_sell_len(const int64_t* __restrict__ rp, int64_t n, int64_t ns,
                           int64_t* __restrict__ cnt) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t m = 0;
    for (int64_t r = q * 32; r < q * 32 + 32 && r < n; r++) m = max(m, rp[r + 1] - rp[r]);
    cnt[q] = 32 * m;
  }
}

__global__ void k_sell_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, int64_t n,
                            const int64_t* __restrict__ soff, float* __restrict__ vs,
                            int32_t* __restrict__ sc) {
  const int64_t npad = (n + 31) & ~int64_t(31);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = i >> 5;
    const int64_t L = (soff[sl + 1] - soff[sl]) >> 5;
    const int64_t len = i < n ? rp[i + 1] - rp[i] : 0;
    const int64_t e0 = i < n ? rp[i] : 0;
    const int64_t o = soff[sl] + (i & 31);
    for (int64_t k = 0; k < L; k++) {
      vs[o + k * 32] = k < len ? (float)v[e0 + k] : 0.0f;
      if (sc) sc[o + k * 32] = k < len ? ci[e0 + k] : 0;
    }
  }
}

// FP16 variant (values_f16): rscale[r] = the row's largest magnitude (1 for
// a zero row), every value divided by it in FP64 and rounded once to FP16.
__global__ void k_sell_fill_h(const int64_t* __restrict__ rp, const double* __restrict__ v, int64_t n,
                              const int64_t* __restrict__ soff, __half* __restrict__ vs,
                              float* __restrict__ rscale) {
  const int64_t npad = (n + 31) & ~int64_t(31);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = i >> 5;
    const int64_t L = (soff[sl + 1] - soff[sl]) >> 5;
    const int64_t len = i < n ? rp[i + 1] - rp[i] : 0;
    const int64_t e0 = i < n ? rp[i] : 0;
    double m = 0.0;
    for (int64_t k = 0; k < len; k++) m = fmax(m, fabs(v[e0 + k]));
    const float sc = m > 0.0 ? (float)m : 1.0f;
    if (i < n) rscale[i] = sc;
    __half* o = vs + soff[sl] + (i & 31);
    for (int64_t k = 0; k < L; k++)
      o[k * 32] = k < len ? __double2half(v[e0 + k] / (double)sc) : __double2half(0.0);
  }
}

// Sliced FP32 copy of an operator: of a patterned operator (values only,
// FP32 or, with f16, FP16), or with `columns` of an unpatterned operator with
// at least SELL_MIN_ROWS rows (one thread per row needs that many rows).  Of
// the unpatterned operators A_CF of the restriction and W of the
// interpolation gain (measured at the headline: the apply 6.82 -> 6.73 ms,
// then 6.66 -> 6.53 ms); the coarse AMG levels, with longer and irregular
// rows, lose (A_uu V-cycle 2.93 -> 3.10 ms).
static constexpr int64_t SELL_MIN_ROWS = int64_t(1) << 18;
static int sell_fp32(Pool& P, Csr& A, cudaStream_t s, bool f16 = false, bool columns = false) {
  const int64_t n = A.nr, ns = (n + 31) / 32;
  if (n <= 0 || !A.v) return MGR_SUCCESS;
  if (!A.pid && !(columns && n >= SELL_MIN_ROWS && A.nnz + 64 < INT32_MAX)) return MGR_SUCCESS;
  if (!A.pid) f16 = false;
  Pool tmp;
  tmp.s = s;
  int64_t* cnt = tmp.get<int64_t>(ns);
  A.soff = P.get<int64_t>(ns + 1);
  if (tmp.err || P.err) {
    tmp.free_all_async(s);
    return tmp.err ? tmp.err : P.err;
  }
  MGR_LAUNCH k_sell_len<<<grid_for(ns, 256), 256, 0, s>>>(A.rp, n, ns, cnt);
  int64_t total = 0;
  int rc = rowptr_from_counts(cnt, A.soff, ns, &total, s, tmp);
  tmp.free_all_async(s);
  MGR_TRY(rc);
  if (f16) {
    A.vsellh = P.get<__half>(total > 0 ? total : 1);
    A.rscale = P.get<float>(n);
    if (!A.vsellh || !A.rscale) return P.err;
    MGR_LAUNCH k_sell_fill_h<<<grid_for((n + 31) & ~int64_t(31), 256), 256, 0, s>>>(
        A.rp, A.v, n, A.soff, A.vsellh, A.rscale);
    return MGR_SUCCESS;
  }
  A.vsell = P.get<float>(total > 0 ? total : 1);
  if (!A.vsell) return P.err;
  if (!A.pid) {
    A.sci = P.get<int32_t>(total > 0 ? total : 1);
    if (!A.sci) return P.err;
  }
  MGR_LAUNCH k_sell_fill<<<grid_for((n + 31) & ~int64_t(31), 256), 256, 0, s>>>(A.rp, A.ci, A.v, n,
                                                                               A.soff, A.vsell, A.sci);
  return MGR_SUCCESS;
}

// ----------------------------------------------------------------------------
// Sliced (SELL-32) copy of the Jacobian for the FP64 products of FGMRES
// ----------------------------------------------------------------------------
// On GB300 the FP64 product is bound by the narrow FP64 pipe as much as by
// HBM: with G lanes per row every row adds log2(G) shuffle-adds and a ragged
// last round of multiply-adds.  One thread per row over a sliced copy (rows
// in slices of 32, a slice's entries k-major: entry k of row r at
// soff[r / 32] + 32 k + r % 32, padded with column r and value 0) issues one
// multiply-add per non-zero and loads 256 contiguous bytes of values per warp
// instruction.  A belongs to the caller and its values may change between
// solves, so the copy is rebuilt from A at the start of every solve.
__global__ void k_jsell_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, int64_t n,
                             const int64_t* __restrict__ soff, int32_t* __restrict__ sci,
                             double* __restrict__ sval) {
  const int64_t npad = (n + 31) & ~int64_t(31);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = i >> 5;
    const int64_t L = (soff[sl + 1] - soff[sl]) >> 5;
    const int64_t len = i < n ? rp[i + 1] - rp[i] : 0;
    const int64_t e0 = i < n ? rp[i] : 0;
    const int32_t self = (int32_t)(i < n ? i : 0);
    const int64_t o = soff[sl] + (i & 31);
    for (int64_t k = 0; k < L; k++) {
      const bool in = k < len;
      sci[o + k * 32] = in ? ci[e0 + k] : self;
      sval[o + k * 32] = in ? v[e0 + k] : 0.0;
    }
  }
}

int jacobian_sell_refresh(Handle* h, const mgr_matrix_t* A, cudaStream_t s) {
  JacobianSell& J = h->jsell;
  J.valid = false;
  if (A->nnz < JSELL_MIN_NNZ || A->n <= 0 || A->n != h->n) return 0;
  const int64_t n = A->n, ns = (n + 31) / 32;
  Pool& P = h->pool;
  if (J.ns_cap < ns + 1) {
    P.release(J.soff, s);
    J.soff = P.get<int64_t>(ns + 1);
    if (!J.soff) return P.err;
    J.ns_cap = ns + 1;
  }
  Pool tmp;
  tmp.s = s;
  int64_t* cnt = tmp.get<int64_t>(ns);
  if (!cnt) {
    tmp.free_all_async(s);
    return tmp.err;
  }
  MGR_LAUNCH k_sell_len<<<grid_for(ns, 256), 256, 0, s>>>(A->row_ptr, n, ns, cnt);
  int64_t total = 0;
  const int rc = rowptr_from_counts(cnt, J.soff, ns, &total, s, tmp);
  tmp.free_all_async(s);
  MGR_TRY(rc);
  if (J.cap < total) {
    P.release(J.sci, s);
    P.release(J.sval, s);
    J.sci = P.get<int32_t>(total);
    J.sval = P.get<double>(total);
    if (!J.sci || !J.sval) return P.err;
    J.cap = total;
  }
  MGR_LAUNCH k_jsell_fill<<<grid_for((n + 31) & ~int64_t(31), 256), 256, 0, s>>>(
      A->row_ptr, A->col_idx, A->val, n, J.soff, J.sci, J.sval);
  MGR_TRY_CUDA(cudaGetLastError());
  J.rp = A->row_ptr;
  J.ci = A->col_idx;
  J.val = A->val;
  J.n = n;
  J.nnz = A->nnz;
  J.valid = true;
  return 1;
}

static int amg_to_fp32(Handle* h, Amg* g, cudaStream_t s) {
  if (!g) return MGR_SUCCESS;
  Pool& P = h->pool;
  for (auto& L : g->lev) {
    MGR_TRY(f32(P, L.A.v, &L.A.vf, L.A.nnz, s));
    MGR_TRY(sell_fp32(P, L.A, s, h->opt.values_f16 != 0));
    MGR_TRY(f32(P, L.P.v, &L.P.vf, L.P.nnz, s));
    MGR_TRY(f32(P, L.R.v, &L.R.vf, L.R.nnz, s));
    MGR_TRY(f32(P, L.dinv, &L.dinvf, L.A.nr, s));
    if (h->opt.diag_bf16) MGR_TRY(bf16(P, L.dinv, &L.dinvh, L.A.nr, s));
  }
  g->bf16 = h->opt.diag_bf16 != 0;
  MGR_TRY(f32(P, g->inv, &g->invf, g->ncoarse * g->ncoarse, s));
  return MGR_SUCCESS;
}

int to_fp32(Handle* h, cudaStream_t s) {
  Pool& P = h->pool;
  for (auto& L : h->lev) {
    MGR_TRY(f32(P, L.A.v, &L.A.vf, L.A.nnz, s));
    MGR_TRY(f32(P, L.W.v, &L.W.vf, L.W.nnz, s));
    MGR_TRY(f32(P, L.Acf.v, &L.Acf.vf, L.Acf.nnz, s));
    MGR_TRY(sell_fp32(P, L.Acf, s, false, true));
    MGR_TRY(sell_fp32(P, L.W, s, false, true));
    MGR_TRY(f32(P, L.dFinv, &L.dFinvf, L.nF, s));
    MGR_TRY(f32(P, L.binvc, &L.binvcf, (int64_t)L.bdim * L.bdim * L.nblk, s));
    if (h->opt.diag_bf16) {
      MGR_TRY(bf16(P, L.dFinv, &L.dFinvh, L.nF, s));
      MGR_TRY(bf16(P, L.binvc, &L.binvch, (int64_t)L.bdim * L.bdim * L.nblk, s));
      L.bf16 = true;
    }
    if (L.Wr.v) MGR_TRY(f32(P, L.Wr.v, &L.Wr.vf, L.Wr.nnz, s));
    if (L.Bd.v) MGR_TRY(f32(P, L.Bd.v, &L.Bd.vf, L.Bd.nnz, s));
    if (L.ilu1) {
      MGR_TRY(f32(P, L.Ilo.v, &L.Ilo.vf, L.Ilo.nnz, s));
      MGR_TRY(f32(P, L.Iup.v, &L.Iup.vf, L.Iup.nnz, s));
      MGR_TRY(f32(P, L.ilu_dinv, &L.ilu_dinvf, L.n, s));
    }
    MGR_TRY(amg_to_fp32(h, L.famg, s));
  }
  MGR_TRY(amg_to_fp32(h, h->camg, s));
  MGR_TRY_CUDA(cudaGetLastError());
  return MGR_SUCCESS;
}

}  // namespace mgr
