// maxprod_pnorm_static: the p-norm product for callers that cannot allocate.
//
// Some callers only hold the buffers they were handed -- for example a plugin
// whose host framework owns all device memory and forbids cudaMalloc while it
// runs, or code on a real-time path where an allocation could stall -- and so
// cannot provide the workspace maxprod_pnorm wants.  This entry point runs the
// same computation in a fixed scratch array that lives in this library's own
// device memory (a file-scope __device__ array of PN_STATIC_SCRATCH_BYTES,
// reserved on every GPU that loads the library until the process exits).  It
// calls no cudaMalloc, cudaFree or other allocating routine.
//
// The array's device address is looked up once per device, with that device
// current, on the first call made on it; make that first call before any
// stream capture.  All calls share the one array: calls whose GPU work may
// overlap (different streams, several host threads) race on it and must be
// serialised by the caller.  The part of the scratch that has to start at
// zero is cleared by every call; the rest is fully written before it is read.
#include <mutex>

#include "pn_internal.h"
#include <cuda_runtime.h>

namespace {

static __device__ __align__(256) uint8_t g_static_scratch[PN_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (nullptr if the
// lookup failed).  Looked up once per device and cached.
void* scratch_address() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return nullptr;
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

}  // namespace

extern "C" pn_status maxprod_pnorm_static(int64_t M, int64_t N, int64_t K, const float* A,
                                          int64_t lda, const float* B, int64_t ldb, float* C,
                                          int64_t ldc, uint8_t* p_sel, float* S_sel,
                                          const pn_opts* opts, void* stream) {
  const size_t need = pn_workspace_size(M, N, K, opts);
  if (need == 0) return PN_EINVAL;
  if (need > PN_STATIC_SCRATCH_BYTES) return PN_EWORKSPACE;  // problem too large for the array
  void* ws = scratch_address();
  if (!ws) return PN_ECUDA;
  return maxprod_pnorm(M, N, K, A, lda, B, ldb, C, ldc, p_sel, S_sel, opts, ws,
                       PN_STATIC_SCRATCH_BYTES, stream);
}
