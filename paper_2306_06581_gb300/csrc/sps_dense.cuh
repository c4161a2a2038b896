// sps_dense.cuh -- tiling helpers shared by the dense Sinkhorn passes (plain
// scalings and log-sum-exp form): the point / cost view of a pass and the
// split of the column range across blocks.
#pragma once

#include <algorithm>

#include "sps_internal.h"

namespace sps {
namespace dense {

constexpr int kTI = 128;   // threads per block
constexpr int kRPT = 2;    // rows per thread
constexpr int kTJ = 128;   // columns per shared-memory tile

// One pass runs over "rows" p (the original rows, or the original columns
// when transposed) and sums over "columns" q.
struct DenseView {
  const float* P32; const float* Q32;      // row / column points (binary32)
  const double* P64; const double* Q64;    // FP64 points (FP64 problems)
  const float* C32; const double* C64;     // dense raw cost, original orientation n x m
  int transposed;                          // 1: pass rows are the original columns
  int np, nq, d, m_orig;
};

template <typename T>
__device__ __forceinline__ T ldpt(const float* p32, const double* p64, int64_t off) {
  if (sizeof(T) == 8) return (T)(p64 ? p64[off] : (double)p32[off]);
  return (T)p32[off];
}

struct Geo {
  dim3 grid;
  int qchunk;
  int nsplit;
};

// Row blocks of kTI * kRPT rows; the column range is split so that the grid
// holds at least 4 blocks per SM.
inline Geo geometry(int np, int nq) {
  const int gi = (np + kTI * kRPT - 1) / (kTI * kRPT);
  int gs = std::max(1, (152 * 4 + gi - 1) / gi);
  int qchunk = std::max(kTJ, (nq + gs - 1) / gs);
  qchunk = ((qchunk + kTJ - 1) / kTJ) * kTJ;
  gs = (nq + qchunk - 1) / qchunk;
  return Geo{dim3(gi, gs), qchunk, gs};
}

inline DenseView view_rows(const ProbDev& pd) {
  DenseView V;
  V.P32 = pd.cv.x32; V.Q32 = pd.cv.y32; V.P64 = pd.cv.x64; V.Q64 = pd.cv.y64;
  V.C32 = pd.cv.C32; V.C64 = pd.cv.C64; V.transposed = 0; V.np = pd.n; V.nq = pd.m; V.d = pd.d; V.m_orig = pd.m;
  return V;
}

inline DenseView view_cols(const ProbDev& pd) {
  DenseView V = view_rows(pd);
  V.P32 = pd.cv.y32; V.Q32 = pd.cv.x32; V.P64 = pd.cv.y64; V.Q64 = pd.cv.x64;
  V.transposed = 1; V.np = pd.m; V.nq = pd.n;
  return V;
}

// True in the last block of the grid to arrive (after all blocks' writes are visible).
__device__ __forceinline__ bool last_block_d(unsigned int* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  return am_last;
}

// Sums nparts arrays of nblk block partials in a fixed order into out[] (thread 0).
__device__ __forceinline__ void reduce_parts_d(const double* part, int nblk, int nparts, double* out, double* sh) {
  for (int p = 0; p < nparts; ++p) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += __ldcg(part + (size_t)p * nblk + b);
    s = block_sum_d(s, sh);
    if (threadIdx.x == 0) out[p] = s;
    __syncthreads();
  }
}

}  // namespace dense
}  // namespace sps
