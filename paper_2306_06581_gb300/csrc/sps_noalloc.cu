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
// not a device address, so its device address is looked up with
// cudaGetSymbolAddress (with the device current) and then passed to the
// kernels.  The lookup is made once per device and CUDA context: the cache
// is keyed by the device ordinal and the current context, because after
// cudaDeviceReset, or under another context of the same device, the module is
// loaded again and the array may sit elsewhere.  All calls share the array and
// it keeps the last call's contents; the solver clears what must start at zero
// (control block, sums, counters) at the start of every call.  Calls whose GPU
// work overlaps (other streams, other host threads, or a second call enqueued
// before the first finished on another stream) race on the array.
#include <cuda.h>   // CUcontext and the cuCtxGetCurrent signature only; no driver library is linked
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "sps_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SPS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
  CUcontext ctx;   // context the address belongs to
  void* addr;
};
Cached g_addr[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// The driver's cuCtxGetCurrent, found through the runtime (so the library
// does not link the driver library itself); null if the driver lacks it.
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  return fn;
}

// Device address of the scratch array on the current device and context;
// looked up on the first call made with that device and context current.
sps_status scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sps::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    sps::set_error("device ordinal %d out of range for the no-allocation entry point", dev);
    return SPS_ERR_INVALID_ARG;
  }
  const CtxGetCurrentFn get = ctx_get_current();
  CUcontext ctx = nullptr;
  if (!get || get(&ctx) != CUDA_SUCCESS) {
    sps::set_error("the no-allocation entry point could not read the current CUDA context");
    return SPS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  Cached& c = g_addr[dev];
  if (!ctx || !c.addr || c.ctx != ctx) {
    // no context current yet on this thread, or a new one: look the address up
    // (the lookup itself makes the device's primary context current)
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return sps::cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    if (!p) {
      sps::set_error("cudaGetSymbolAddress returned a null scratch address");
      return SPS_ERR_CUDA;
    }
    if (get(&ctx) != CUDA_SUCCESS || !ctx) {
      sps::set_error("the no-allocation entry point could not read the current CUDA context");
      return SPS_ERR_CUDA;
    }
    c.ctx = ctx;
    c.addr = p;
  }
  *out = c.addr;
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
