// Allocation-free V-cycle entry point (mgr_vcycle_noalloc).
//
// Some callers cannot allocate device memory at the point where they run a
// V-cycle: a host program that hands every byte of device memory to its own
// pool up front (so cudaMalloc would fail or must not be called), or a
// latency-bound loop that forbids allocation after start-up because an
// allocation can synchronise the device and can fail.  For them this entry
// point allocates nothing and uses none of the handle's workspace: the level
// vectors of the V-cycle live in one fixed buffer compiled into the library.
//
// That buffer is a file-scope static __device__ array, so every GPU that loads
// the library holds MGR_NOALLOC_SCRATCH_BYTES of it until the process exits.
// In host code its name is only a host-side stand-in, not a device address; the
// device address is obtained with cudaGetSymbolAddress (with the device
// current) and passed to the kernels.  All calls on a device share
// the buffer, and it keeps the last call's contents.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "mgr_internal.cuh"

#define MGR_NOALLOC_SCRATCH_BYTES (8u << 20)   // 8 MiB
#define MGR_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[MGR_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[MGR_NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch buffer on the current device.  Looked up
// again on every call made outside stream capture (a cheap host-side query), so
// that a device reset or a new primary context never leaves a stale address in
// use; during capture the address of the last uncaptured call on this device
// is used, and without one the call is rejected.
int scratch_address(cudaStream_t s, void** out) {
  int dev = 0;
  MGR_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MGR_NOALLOC_MAX_DEVICES) return MGR_ERR_INVALID_ARG;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    (void)cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "mgr_vcycle_noalloc: cudaGetSymbolAddress failed: %s\n",
              cudaGetErrorString(e));
      return MGR_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  } else if (!g_noalloc_addr[dev]) {
    fprintf(stderr, "mgr_vcycle_noalloc: the first call on a device must come before any "
                    "stream capture\n");
    return MGR_ERR_INVALID_ARG;
  }
  *out = g_noalloc_addr[dev];
  return MGR_SUCCESS;
}
}  // namespace

using namespace mgr;

extern "C" int mgr_vcycle_noalloc(mgr_handle_t hh, int slot, const double* b, double* x,
                                  void* stream) {
  (void)cudaGetLastError();  // errors of earlier calls are not this call's
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !b || !x) return MGR_ERR_INVALID_ARG;
  Amg* g = (slot == h->L) ? h->camg : (slot >= 0 && slot < h->L ? h->lev[slot].famg : nullptr);
  if (!g) return MGR_ERR_INVALID_ARG;
  const size_t need = vcycle_ws_bytes(h, g);
  if (need > MGR_NOALLOC_SCRATCH_BYTES) {
    fprintf(stderr,
            "mgr_vcycle_noalloc: this V-cycle needs %zu bytes of workspace, more than the "
            "fixed %u-byte scratch buffer; use mgr_vcycle instead\n",
            need, (unsigned)MGR_NOALLOC_SCRATCH_BYTES);
    return MGR_ERR_INVALID_ARG;
  }
  void* ws = nullptr;
  MGR_TRY(scratch_address((cudaStream_t)stream, &ws));
  return apply_vcycle64_ws(h, g, b, x, ws, (cudaStream_t)stream);
}
