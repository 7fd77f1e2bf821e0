// maxprod_pnorm_static: the p-norm product for callers that cannot allocate.
//
// Some callers only hold the buffers they were handed -- for example a plugin
// whose host framework owns all device memory and forbids cudaMalloc while it
// runs, or code on a real-time path where an allocation could stall -- and so
// cannot provide the workspace maxprod_pnorm wants.  This entry point runs the
// same computation in a fixed scratch array that lives in this library's own
// device memory (a file-scope __device__ array of PN_STATIC_SCRATCH_BYTES).
// CUDA loads a module lazily by default, so the array is reserved on a device
// once this entry point is first used there, and stays reserved until the
// process exits or the device is reset.  The call makes no cudaMalloc,
// cudaFree or other allocating call.
//
// The array's device address is looked up with the device current on every
// call made outside a stream capture, so a device reset (which reloads the
// module and moves the array) is picked up by the next such call.  During a
// capture no lookup is made and the address cached by an earlier call on that
// device is used: make one call on each device before capturing it.  All calls
// share the one array: calls whose GPU work may overlap (different streams,
// several host threads) race on it and must be serialised by the caller.  The
// part of the scratch that has to start at zero is cleared by every call; the
// rest is fully written before it is read.
#include <mutex>

#include "pn_internal.h"
#include <cuda_runtime.h>

namespace {

static __device__ __align__(256) uint8_t g_static_scratch[PN_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, or nullptr.
// Outside a capture of `stream` the address is looked up (and cached); while
// the stream is capturing only the cached address of an earlier call is used.
void* scratch_address(cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t qe = cudaStreamIsCapturing(stream, &cs);
  if (qe != cudaSuccess) (void)cudaGetLastError();  // a failed query counts as capturing
  const bool capturing = qe != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!capturing) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
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
  void* ws = scratch_address(static_cast<cudaStream_t>(stream));
  if (!ws) return PN_ECUDA;
  return maxprod_pnorm(M, N, K, A, lda, B, ldb, C, ldc, p_sel, S_sel, opts, ws,
                       PN_STATIC_SCRATCH_BYTES, stream);
}
