// sps_iterdev.cuh -- device helpers shared by the iteration kernels of the
// plain (sps_iter.cu) and log-domain (sps_logdom.cu) paths.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "sps_internal.h"

namespace sps {
namespace iterdev {

constexpr int kIterThreads = 1024;   // iteration kernels: one or two blocks per SM
constexpr long long kSpinLimit = 20000000;  // grid-barrier wait limit (about 1-2 s)

// Sparse dot product of one row by a segment of LPR lanes (LPR in 4 .. 32).
// A lane takes kU elements of the row per batch: all their index and value
// loads are issued first, then all gathers of x, so a batch costs two memory
// round trips however long it is; a butterfly reduction closes the segment.
// Only the index array is read through the read-only path: the values (which
// the stabilised kernel rewrites) and x (written by other blocks before the
// last grid barrier) use coherent loads.
template <int LPR, typename V, typename T>
__device__ __forceinline__ T seg_row_dot(const int* __restrict__ idx, const V* val, const T* x, int lo, int hi,
                                         int sl) {
  constexpr int kU = sizeof(T) == 8 ? 4 : (LPR >= 32 ? 8 : (LPR == 16 ? 12 : 16));
  T acc = 0;
  for (int k0 = lo + sl; k0 < hi; k0 += LPR * kU) {
    int id[kU];
    T vv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int k = k0 + u * LPR;
      const bool in = k < hi;
      id[u] = in ? __ldg(idx + k) : -1;
      vv[u] = in ? load_as<T>(val + k) : (T)0;
    }
    T xv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) xv[u] = id[u] >= 0 ? x[id[u]] : (T)0;
#pragma unroll
    for (int u = 0; u < kU; ++u) acc += vv[u] * xv[u];
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// The same product with x staged in shared memory: xs holds x[j0 .. j0 + W);
// an index outside the chunk (which a correct segment never holds) adds nothing.
template <int LPR, typename V>
__device__ __forceinline__ float seg_dot_smem(const int* __restrict__ idx, const V* val, const float* xs, int j0,
                                              int W, int lo, int hi, int sl) {
  constexpr int kU = LPR >= 8 ? 8 : 16;
  float acc = 0.0f;
  for (int k0 = lo + sl; k0 < hi; k0 += LPR * kU) {
    int id[kU];
    float vv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int k = k0 + u * LPR;
      const bool in = k < hi;
      id[u] = in ? __ldg(idx + k) - j0 : -1;
      vv[u] = in ? load_as<float>(val + k) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) acc += (unsigned)id[u] < (unsigned)W ? vv[u] * xs[id[u]] : 0.0f;
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

template <typename T> __device__ __forceinline__ T powT(T x, T y);
template <> __device__ __forceinline__ float powT<float>(float x, float y) { return powf(x, y); }
template <> __device__ __forceinline__ double powT<double>(double x, double y) { return pow(x, y); }


// Sum of NV values over the block with one barrier; result in thread 0.
// Accumulations inside a phase use the iterate type: on this GPU the FP64
// pipe is narrow, and only the per-block partials need FP64.
template <int NV, typename R>
__device__ __forceinline__ void block_sum_multi(R (&v)[NV], R* sh /* NV x 32 */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < NV; ++p) v[p] = warp_sum(v[p]);
  if (lane == 0) {
#pragma unroll
    for (int p = 0; p < NV; ++p) sh[p * 32 + w] = v[p];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int p = 0; p < NV; ++p) {
      const R x = lane < (int)(blockDim.x >> 5) ? sh[p * 32 + lane] : (R)0;
      v[p] = warp_sum(x);
    }
  }
  __syncthreads();
}

// Deterministic reduction of NP arrays of block partials (fixed strided
// subsets per thread, fixed tree); result in out[] (shared), valid after return.
template <int NP, typename R>
__device__ void reduce_parts(const double* part, int nblk, double* out) {
  if (threadIdx.x < 32) {
    R s[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) s[p] = (R)0;
#pragma unroll 4
    for (int b = threadIdx.x; b < nblk; b += 32) {
#pragma unroll
      for (int p = 0; p < NP; ++p) s[p] += (R)__ldcg(part + (size_t)p * nblk + b);
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      s[p] = warp_sum(s[p]);
      if (threadIdx.x == 0) out[p] = (double)s[p];
    }
  }
  __syncthreads();
}

// Bulk copies (TMA, non-tensor) into shared memory with an mbarrier.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// dst, src 16-byte aligned; bytes a multiple of 16
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// make an initialised mbarrier visible to the bulk-copy unit
__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// order this thread's earlier generic-proxy accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Grid barrier of the cooperative kernel: arrival counter plus generation;
// the waiting threads spin with a sleep and give up after kSpinLimit polls,
// recording a failure instead of hanging.
__device__ __forceinline__ bool grid_barrier(Ctrl* ctrl) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &ctrl->bar_gen;
    const unsigned int g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&ctrl->bar_count, 1u) == gridDim.x - 1) {
      ctrl->bar_count = 0u;
      __threadfence();
      atomicAdd(&ctrl->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (spins > 4096) __nanosleep(32);
        if (++spins > kSpinLimit) { ok = 0; break; }
      }
    }
    __threadfence();
    if (!ok) { ctrl->wait_timeout = 1; ctrl->done = 1; ctrl->status = SPS_ERR_CUDA; }
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Counting grid barrier: arrivals only ever add to one 64-bit counter (a
// release add), and a block waits until the counter reaches the next multiple
// of the grid (acquire loads).  Arrivals at barrier e + 1 start only after all
// arrivals at barrier e, so the count returned to an arrival fixes its
// barrier.  The counter starts at 0 for each solve and stays a multiple of
// the grid between launches of one solve (same grid).  Bounded wait.
__device__ __forceinline__ bool grid_barrier_count(Ctrl* ctrl) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long prev;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], 1;\n" : "=l"(prev) : "l"(&ctrl->bar_mono) : "memory");
    const unsigned long long target = (prev / gridDim.x + 1) * gridDim.x;
    int ok = 1;
    long long spins = 0;
    for (;;) {
      unsigned long long cur;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];\n" : "=l"(cur) : "l"(&ctrl->bar_mono) : "memory");
      if (cur >= target) break;
      if (++spins > kSpinLimit) { ok = 0; break; }
      if (spins > 256) __nanosleep(32);
    }
    if (!ok) { ctrl->wait_timeout = 1; ctrl->done = 1; ctrl->status = SPS_ERR_CUDA; }
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Blocks of the iteration kernels: all SMs, as many per SM as fit, never more
// than the partial arrays hold.
template <typename K>
int iter_grid(K fn, int cap) {
  int dev = 0, nsm = 152, per_sm = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kIterThreads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  return std::max(1, std::min(cap, nsm * per_sm));
}

}  // namespace iterdev
}  // namespace sps
