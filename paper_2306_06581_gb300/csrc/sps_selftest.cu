// sps_selftest.cu -- failure-detection self-test of the bounded device waits.
//
// The persistent iteration kernels synchronise their blocks with a counting
// grid barrier whose wait is bounded (kSpinLimit polls): a block that waits
// longer gives up, records wait_timeout in the control block and returns, so
// the solver reports an error instead of hanging and the CUDA context stays
// usable.  This entry point makes that wait run out on purpose, without any
// fault: it launches the same barrier on a two-block grid in which the second
// block returns at once and never arrives, so the count the first block waits
// for is never reached (a flag that nothing sets).  Every wait in it ends:
// the only loop is the barrier's, bounded by kSpinLimit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sps_internal.h"
#include "sps_iterdev.cuh"

namespace {

__global__ void k_barrier_selftest(sps::Ctrl* ctrl) {
  if (blockIdx.x != 0) return;   // this block never arrives
  sps::iterdev::grid_barrier_count(ctrl);
}

}  // namespace

extern "C" sps_status sps_selftest_barrier_timeout(void* ws, size_t ws_bytes, float* wait_ms, sps_stream stream) {
  using namespace sps;
  if (!ws || !wait_ms) { set_error("sps_selftest_barrier_timeout: null workspace or wait_ms"); return SPS_ERR_INVALID_ARG; }
  if (ws_bytes < sizeof(Ctrl) + 256) {
    set_error("sps_selftest_barrier_timeout: workspace of %zu bytes, %zu needed", ws_bytes, sizeof(Ctrl) + 256);
    return SPS_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Ctrl* ctrl = (Ctrl*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SPS_TRY(cuda_fail(cudaEventCreate(&e0), "event create"));
  sps_status s = cuda_fail(cudaEventCreate(&e1), "event create");
  Ctrl h;
  if (s == SPS_OK) s = cuda_fail(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st), "memset");
  if (s == SPS_OK) s = cuda_fail(cudaEventRecord(e0, st), "event record");
  if (s == SPS_OK) {
    k_barrier_selftest<<<2, 32, 0, st>>>(ctrl);
    s = cuda_fail(cudaGetLastError(), "self-test launch");
  }
  if (s == SPS_OK) s = cuda_fail(cudaEventRecord(e1, st), "event record");
  if (s == SPS_OK) s = cuda_fail(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "read back");
  if (s == SPS_OK) s = cuda_fail(cudaStreamSynchronize(st), "synchronize");
  if (s == SPS_OK) s = cuda_fail(cudaEventElapsedTime(wait_ms, e0, e1), "event time");
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s != SPS_OK) return s;
  if (h.wait_timeout) {
    set_error("a device-side grid barrier wait timed out (self-test: one block never arrived)");
    return SPS_ERR_CUDA;
  }
  set_error("self-test: the grid barrier completed although one block never arrived");
  return SPS_OK;
}
