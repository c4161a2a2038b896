// sps_noalloc.cu -- spar_sink_ot_noalloc: Spar-Sink OT that needs no
// caller-provided workspace and allocates nothing.
//
// Who it is for: callers that cannot call cudaMalloc (or any allocator) at
// solve time -- for example a host process whose device memory is owned by
// another allocator (a framework's caching pool or a fixed memory budget
// that must not be bypassed), or an embedding where allocation is only
// allowed at start-up -- and that therefore cannot provide the workspace
// the other entry points ask for.  The paper has no counterpart: it is an
// interface convenience, not part of the method.
//
// How: the workspace is a file-scope device array of SPS_NOALLOC_SCRATCH_BYTES
// bytes.  Every GPU that loads this library's module holds it until the
// process exits.  In host code the array's name is only a host-side stand-in,
// not a device address, so its device address is looked up once per device
// with cudaGetSymbolAddress (with that device current) and then passed to the
// kernels.  All calls share the array and it keeps the last call's contents;
// the solver clears what must start at zero (control block, sums, counters)
// at the start of every call.  Calls whose GPU work overlaps (other streams,
// other host threads, or a second call enqueued before the first finished on
// another stream) race on the array.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "sps_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SPS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; looked up on the
// first call made with that device current.
sps_status scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sps::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    sps::set_error("device ordinal %d out of range for the no-allocation entry point", dev);
    return SPS_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return sps::cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    if (!p) {
      sps::set_error("cudaGetSymbolAddress returned a null scratch address");
      return SPS_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SPS_OK;
}

}  // namespace

extern "C" sps_status spar_sink_ot_noalloc(const sps_problem* prob, const sps_params* prm, void* alpha_out,
                                           void* beta_out, sps_result* res, sps_stream stream) {
  const size_t need = sps_workspace_bytes(prob, prm, SPS_OP_SPAR_SINK);
  if (need == 0) return SPS_ERR_INVALID_ARG;  // message already set by the argument checks
  if (need > (size_t)SPS_NOALLOC_SCRATCH_BYTES) {
    sps::set_error("spar_sink_ot_noalloc: this problem needs %zu bytes of scratch, more than the %zu bytes "
                   "the no-allocation entry point holds; call spar_sink_ot with a caller workspace instead",
                   need, (size_t)SPS_NOALLOC_SCRATCH_BYTES);
    return SPS_ERR_WORKSPACE;
  }
  void* ws = nullptr;
  const sps_status st = scratch_address(&ws);
  if (st != SPS_OK) return st;
  return spar_sink_ot(prob, prm, ws, (size_t)SPS_NOALLOC_SCRATCH_BYTES, alpha_out, beta_out, res, stream);
}
