// sps_sketch.cu -- construction of the sparse sketch K~ (section 3, Eq. pois).
//
// Pipeline (all on the caller's stream):
//   prepare   binary32 copies of the inputs, weights in the iterate type,
//             input checks, maxima of a and b
//   cost_max  D_max = max_ij raw cost (max is exact and order-free)
//   factors   OT  (Eq. pij-ot):  r_i = (s sqrt(a_i)) / (sum sqrt a sum sqrt b), c_j = sqrt(b_j)
//             UOT (Eq. pij-uot): A_i = a_i^g, B_j = b_j^g, g = lam/(2lam+eps),
//                                Z = sum_ij A_i B_j exp(-D_ij/(Dn (2lam+eps)))
//             with exact order-independent sums rounded once to binary64
//   count     per row: number of kept elements (Philox draw < p*); column counts
//   scan      row_ptr, col_ptr
//   fill      CSR (columns ascending) and an unordered CSC scatter
//   csc_sort  rows ascending inside every column (stable transpose)
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>

#include "sps_internal.h"

namespace sps {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
  atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<long long*>(addr), __double_as_longlong(v));
}

__device__ __forceinline__ bool bad_weight(double w) { return !(w >= 0.0) || isinf(w); }

// ---------------------------------------------------------------------------
// prepare
// ---------------------------------------------------------------------------
__global__ void k_prepare(ProbDev pd, Ctrl* ctrl, SketchScalars* sc, float* x32, float* y32,
                          float* a32, float* b32, float* C32, void* a_it, void* b_it, int it64) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int n = pd.n, m = pd.m, d = pd.d;
  if (pd.in_f64) {
    const double* a = (const double*)pd.a;
    const double* b = (const double*)pd.b;
    for (int64_t k = tid; k < n; k += stride) {
      const double w = a[k];
      if (bad_weight(w)) ctrl->status = SPS_ERR_NUMERIC;
      a32[k] = __double2float_rn(w);
      if (it64) ((double*)a_it)[k] = w; else ((float*)a_it)[k] = __double2float_rn(w);
      atomic_max_nonneg(&sc->maxa, fmaxf(__double2float_rn(w), 0.0f));
    }
    for (int64_t k = tid; k < m; k += stride) {
      const double w = b[k];
      if (bad_weight(w)) ctrl->status = SPS_ERR_NUMERIC;
      b32[k] = __double2float_rn(w);
      if (it64) ((double*)b_it)[k] = w; else ((float*)b_it)[k] = __double2float_rn(w);
      atomic_max_nonneg(&sc->maxb, fmaxf(__double2float_rn(w), 0.0f));
    }
    if (x32) {
      for (int64_t k = tid; k < (int64_t)n * d; k += stride) x32[k] = __double2float_rn(pd.cv.x64[k]);
      for (int64_t k = tid; k < (int64_t)m * d; k += stride) y32[k] = __double2float_rn(pd.cv.y64[k]);
    }
    if (C32) {
      for (int64_t k = tid; k < (int64_t)n * m; k += stride) C32[k] = __double2float_rn(pd.cv.C64[k]);
    }
  } else {
    const float* a = (const float*)pd.a;
    const float* b = (const float*)pd.b;
    for (int64_t k = tid; k < n; k += stride) {
      const float w = a[k];
      if (bad_weight((double)w)) ctrl->status = SPS_ERR_NUMERIC;
      a32[k] = w;
      if (it64) ((double*)a_it)[k] = (double)w; else ((float*)a_it)[k] = w;
      atomic_max_nonneg(&sc->maxa, fmaxf(w, 0.0f));
    }
    for (int64_t k = tid; k < m; k += stride) {
      const float w = b[k];
      if (bad_weight((double)w)) ctrl->status = SPS_ERR_NUMERIC;
      b32[k] = w;
      if (it64) ((double*)b_it)[k] = (double)w; else ((float*)b_it)[k] = w;
      atomic_max_nonneg(&sc->maxb, fmaxf(w, 0.0f));
    }
  }
}

// ---------------------------------------------------------------------------
// cost_max: tiles of kTileI rows (one per thread) against column ranges
// staged in shared memory.  D is the compile-time dimension (0 = runtime d).
// ---------------------------------------------------------------------------
constexpr int kTileI = 128;
constexpr int kTileJ = 256;
constexpr int kMaxDReg = 16;

template <int D>
__global__ void __launch_bounds__(kTileI) k_cost_max(ProbDev pd, SketchScalars* sc, int need64, int jchunk,
                                                     const int* gate) {
  if (gate && *gate == 0) return;   // the pruned maximum already holds the result
  const int n = pd.n, m = pd.m;
  const int d = D > 0 ? D : pd.d;
  extern __shared__ float ys[];  // kTileJ * d
  const int i = blockIdx.x * kTileI + threadIdx.x;
  const int j_begin = blockIdx.y * jchunk;
  const int j_end = min(m, j_begin + jchunk);
  float best = 0.0f;
  double best64 = 0.0;
  if (pd.cv.C32) {
    if (i < n)
      for (int j = j_begin; j < j_end; ++j) best = fmaxf(best, pd.cv.C32[(int64_t)i * m + j]);
  } else {
    float xr[D > 0 ? D : kMaxDReg];
    const bool reg = (D > 0) || d <= kMaxDReg;
    if (i < n && reg) {
#pragma unroll
      for (int k = 0; k < (D > 0 ? D : kMaxDReg); ++k) xr[k] = (k < d) ? pd.cv.x32[(int64_t)i * d + k] : 0.0f;
    }
    for (int j0 = j_begin; j0 < j_end; j0 += kTileJ) {
      const int jn = min(kTileJ, j_end - j0);
      if (reg) {
        __syncthreads();
        for (int t = threadIdx.x; t < jn * d; t += blockDim.x) ys[t] = pd.cv.y32[(int64_t)j0 * d + t];
        __syncthreads();
      }
      if (i < n) {
        if (reg) {
          for (int jj = 0; jj < jn; ++jj) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < (D > 0 ? D : kMaxDReg); ++k) {
              if (D > 0 || k < d) {
                const float t = __fsub_rn(xr[k], ys[jj * d + k]);
                acc = __fmaf_rn(t, t, acc);
              }
            }
            best = fmaxf(best, acc);
          }
        } else {
          for (int jj = 0; jj < jn; ++jj) best = fmaxf(best, raw32(pd.cv, i, j0 + jj));
        }
      }
    }
  }
  if (need64 && i < n)
    for (int j = j_begin; j < j_end; ++j) best64 = fmax(best64, raw64(pd.cv, i, j));
  best = warp_max(best);
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&sc->dmax32, best);
  if (need64) {
    best64 = warp_max(best64);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&sc->dmax64, best64);
  }
}

// ---------------------------------------------------------------------------
// factors
// ---------------------------------------------------------------------------
// OT: exact sums of sqrt(a_i), sqrt(b_j).
__global__ void k_ot_sqrt_sums(ProbDev pd, SketchScalars* sc, const float* a32, const float* b32) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int Ba = exact_floor_for(fmaxf(__fsqrt_rn(sc->maxa), 1e-30f));
  const int Bb = exact_floor_for(fmaxf(__fsqrt_rn(sc->maxb), 1e-30f));
  if (tid == 0) { sc->acc1.B = Ba; sc->acc2.B = Bb; }
  U128 ua{0ull, 0ull}, ub{0ull, 0ull};
  const int64_t lim = (int64_t)max(pd.n, pd.m);
  for (int64_t base = 0; base < lim; base += stride) {
    const int64_t k = base + tid;
    if (k < pd.n) exact_add(ua, &sc->acc1, Ba, __fsqrt_rn(a32[k]));
    if (k < pd.m) exact_add(ub, &sc->acc2, Bb, __fsqrt_rn(b32[k]));
  }
  exact_flush(ua, &sc->acc1);
  exact_flush(ub, &sc->acc2);
}

// Scalars of the decision; stage 0 (before the factors), 1 (OT after sums),
// 2 (UOT after Z).  Binary64 operations are the correctly rounded intrinsics.
__global__ void k_scalars(ProbDev pd, SketchScalars* sc, Ctrl* ctrl, int stage) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (stage == 0) {
    sc->s32 = __double2float_rn(pd.s);
    double dn64 = 1.0;
    float dn32 = 1.0f;
    if (pd.cost_norm == SPS_COST_MAXNORM) {
      if (sc->dmax32 > 0.0f) dn32 = sc->dmax32;
      dn64 = (double)dn32;   // one divisor for both paths: the exact binary32 maximum
    } else if (pd.cost_norm == SPS_COST_SCALE) {
      dn64 = pd.cost_scale;
      dn32 = __double2float_rn(pd.cost_scale);
    }
    sc->dn32 = dn32;
    sc->dn64 = dn64;
    if (pd.cost_kind == SPS_COST_WFR) sc->inv2eta32 = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, pd.eta)));
    if (pd.probs == SPS_PROBS_EQUAL) {
      // equal probabilities p_ij = 1/(n m): r_i = fl(fl(s) fl(1/(n m))), c_j = 1
      sc->scale32 = __double2float_rn(__ddiv_rn(1.0, __dmul_rn((double)pd.n, (double)pd.m)));
    } else if (!pd.is_ot) {
      const double t = __dadd_rn(__dmul_rn(2.0, pd.lam), pd.eps);
      sc->gamma32 = __double2float_rn(__ddiv_rn(pd.lam, t));
      double dn = 1.0;
      if (pd.cost_norm == SPS_COST_MAXNORM && sc->dmax32 > 0.0f) dn = (double)sc->dmax32;
      else if (pd.cost_norm == SPS_COST_SCALE) dn = pd.cost_scale;
      sc->kappa32 = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(dn, t)));
      sc->g2_32 = __double2float_rn(__ddiv_rn(2.0, t));
    }
  } else if (stage == 1) {
    sc->sum1 = exact_round(&sc->acc1);
    sc->sum2 = exact_round(&sc->acc2);
    const double prod = __dmul_rn(sc->sum1, sc->sum2);
    if (!(prod > 0.0) || isinf(prod)) { ctrl->status = SPS_ERR_NUMERIC; sc->scale32 = 0.0f; return; }
    sc->scale32 = __double2float_rn(__ddiv_rn(1.0, prod));
  } else {
    sc->sum1 = exact_round(&sc->acc1);
    if (!(sc->sum1 > 0.0) || isinf(sc->sum1)) { ctrl->status = SPS_ERR_NUMERIC; sc->scale32 = 0.0f; return; }
    sc->scale32 = __double2float_rn(__ddiv_rn(pd.s, sc->sum1));
  }
}

__global__ void k_ot_factors(ProbDev pd, SketchScalars* sc, const float* a32, const float* b32,
                             float* rowf, float* colf) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float s32 = sc->s32, sc32 = sc->scale32;
  for (int64_t i = tid; i < pd.n; i += stride) rowf[i] = __fmul_rn(__fmul_rn(s32, __fsqrt_rn(a32[i])), sc32);
  for (int64_t j = tid; j < pd.m; j += stride) colf[j] = __fsqrt_rn(b32[j]);
}

// Equal probabilities (the Rand-Sink control): r_i = fl(s32 fl(1/(n m))), c_j = 1.
__global__ void k_eq_factors(ProbDev pd, SketchScalars* sc, float* rowf, float* colf) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float r = __fmul_rn(sc->s32, sc->scale32);
  for (int64_t i = tid; i < pd.n; i += stride) rowf[i] = r;
  for (int64_t j = tid; j < pd.m; j += stride) colf[j] = 1.0f;
}

// UOT: A_i = exp(g log a_i), B_j = exp(g log b_j) in the binary32 spec.
__global__ void k_uot_factors(ProbDev pd, SketchScalars* sc, const float* a32, const float* b32,
                              float* rowf, float* colf) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float g = sc->gamma32;
  float ma = 0.0f, mb = 0.0f;
  for (int64_t i = tid; i < pd.n; i += stride) {
    const float a = a32[i];
    const float A = a > 0.0f ? spec_exp(__fmul_rn(g, spec_log(a))) : 0.0f;
    rowf[i] = A;
    ma = fmaxf(ma, A);
  }
  for (int64_t j = tid; j < pd.m; j += stride) {
    const float b = b32[j];
    const float B = b > 0.0f ? spec_exp(__fmul_rn(g, spec_log(b))) : 0.0f;
    colf[j] = B;
    mb = fmaxf(mb, B);
  }
  ma = warp_max(ma);
  mb = warp_max(mb);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&sc->maxa, ma);
    atomic_max_nonneg(&sc->maxb, mb);
  }
}

// ---------------------------------------------------------------------------
// scan: block 0 scans the row counts, block 1 the column counts.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan2(const int* row_cnt, int* row_ptr, int n, const int* col_cnt,
                                                int* col_ptr, int* col_cur, int m, long long cap, Ctrl* ctrl) {
  if (ctrl->status != SPS_OK) return;  // counts were not produced
  const int* cnt = blockIdx.x == 0 ? row_cnt : col_cnt;
  int* ptr = blockIdx.x == 0 ? row_ptr : col_ptr;
  const int len = blockIdx.x == 0 ? n : m;
  __shared__ long long sh[1024];
  const int T = blockDim.x;
  const int t = threadIdx.x;
  const int chunk = (len + T - 1) / T;
  const int lo = min(len, t * chunk), hi = min(len, lo + chunk);
  long long s = 0;
  for (int k = lo; k < hi; ++k) s += cnt[k];
  sh[t] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    const long long v = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  long long run = sh[t] - s;  // exclusive prefix of this thread's chunk
  const long long total = sh[T - 1];
  const bool ok = total <= cap && total <= 0x7fffffffLL;
  for (int k = lo; k < hi; ++k) {
    ptr[k] = ok ? (int)run : 0;
    if (blockIdx.x == 1 && ok) col_cur[k] = (int)run;
    run += cnt[k];
  }
  if (t == T - 1) ptr[len] = ok ? (int)total : 0;
  if (t == 0) {
    if (blockIdx.x == 0) ctrl->nnz = total;
    else ctrl->nnz_cols = total;
    if (!ok) { ctrl->cap_exceeded = 1; ctrl->status = SPS_ERR_CAPACITY; }
  }
}

// ---------------------------------------------------------------------------
// csc_sort: one warp per column; the rank of an element is the number of
// smaller row indices in the column (row indices inside a column are
// distinct), which places it without a comparison sort.
// ---------------------------------------------------------------------------
constexpr int kSortCap = 1024;
constexpr int kSortWarps = 8;

// Gather of the value from its CSR position, bounds-checked against nnz.
template <typename V>
__device__ __forceinline__ V gather_val(const V* val, int src, long long nnz, Ctrl* ctrl) {
  if (src < 0 || (long long)src >= nnz) { ctrl->sketch_fault = 1; return from_d<V>(0.0); }
  return val[src];
}

// Elements off + lane + 32 k (k < Q) of a column staged in sm[0 .. L): each
// one's rank among the column's rows places it.
template <int Q, typename V>
__device__ __forceinline__ void rank_place(const int* sm, int L, int off, int s0, int lane, const int* tmp_src,
                                           const V* val, int* row_idx, int* csr_pos, V* valT,
                                           long long nnz, Ctrl* ctrl, const float* lv, float* lvT) {
  int r[Q], src[Q], rank[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int e = off + lane + 32 * k;
    r[k] = e < L ? sm[e] : 0x7fffffff;
    src[k] = e < L ? tmp_src[s0 + e] : 0;
    rank[k] = 0;
  }
  for (int t = 0; t < L; ++t) {
    const int rt = sm[t];
#pragma unroll
    for (int k = 0; k < Q; ++k) rank[k] += (rt < r[k]) ? 1 : 0;
  }
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int e = off + lane + 32 * k;
    if (e < L) {
      row_idx[s0 + rank[k]] = r[k];
      csr_pos[s0 + rank[k]] = src[k];
      if (val) valT[s0 + rank[k]] = gather_val(val, src[k], nnz, ctrl);
      if (lv) lvT[s0 + rank[k]] = gather_val(lv, src[k], nnz, ctrl);
    }
  }
}

// Eight elements a lane per pass keep the kernel at four or more blocks per SM
// (one 32-element-a-lane variant for long columns had needed 166 registers).
template <typename V>
__global__ void __launch_bounds__(32 * kSortWarps, 4) k_csc_sort(int m, const int* __restrict__ col_ptr,
                                                              const int* __restrict__ tmp_row,
                                                              const int* __restrict__ tmp_src,
                                                              const V* __restrict__ val, int* row_idx,
                                                              int* csr_pos, V* valT, Ctrl* ctrl,
                                                              const float* lv, float* lvT) {
  if (ctrl->status != SPS_OK || ctrl->sketch_fault) return;
  const long long nnz = ctrl->nnz;
  __shared__ int sm_all[kSortWarps][kSortCap];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  int* sm = sm_all[wib];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < m; j += nwarps) {
    const int s0 = col_ptr[j];
    const int L = col_ptr[j + 1] - s0;
    if (L == 0) continue;
    if (L <= kSortCap) {
      __syncwarp();
      for (int e = lane; e < L; e += 32) sm[e] = tmp_row[s0 + e];
      __syncwarp();
      if (L <= 64) {
        rank_place<2>(sm, L, 0, s0, lane, tmp_src, val, row_idx, csr_pos, valT, nnz, ctrl, lv, lvT);
      } else {
        for (int off = 0; off < L; off += 256)
          rank_place<8>(sm, L, off, s0, lane, tmp_src, val, row_idx, csr_pos, valT, nnz, ctrl, lv, lvT);
      }
    } else {
      for (int e = lane; e < L; e += 32) {
        const int re = tmp_row[s0 + e];
        int rank = 0;
        for (int t = 0; t < L; ++t) rank += (tmp_row[s0 + t] < re) ? 1 : 0;
        const int src = tmp_src[s0 + e];
        row_idx[s0 + rank] = re;
        csr_pos[s0 + rank] = src;
        if (val) valT[s0 + rank] = gather_val(val, src, nnz, ctrl);
        if (lv) lvT[s0 + rank] = gather_val(lv, src, nnz, ctrl);
      }
    }
  }
}

int grid_for(int64_t work_items, int per_block) {
  int64_t g = (work_items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
sps_status launch_prepare(const ProbDev& pd, const Layout& L, char* ws, int it64, cudaStream_t st) {
  const int64_t work = std::max<int64_t>(std::max<int64_t>(pd.n, pd.m),
                                         pd.in_f64 ? (int64_t)std::max(pd.n, pd.m) * std::max(pd.d, 1) : 0);
  float* x32 = (pd.in_f64 && pd.cv.x64) ? at<float>(ws, L.x32) : nullptr;
  float* y32 = (pd.in_f64 && pd.cv.y64) ? at<float>(ws, L.y32) : nullptr;
  float* C32 = (pd.in_f64 && pd.cv.C64) ? at<float>(ws, L.C32) : nullptr;
  k_prepare<<<grid_for(work, kThreads), kThreads, 0, st>>>(
      pd, at<Ctrl>(ws, L.ctrl), at<SketchScalars>(ws, L.scal), x32, y32, at<float>(ws, L.a32),
      at<float>(ws, L.b32), C32, ws + L.a_it, ws + L.b_it, it64);
  add_launches(1);
  return cuda_fail(cudaGetLastError(), "prepare");
}

sps_status launch_cost_max(const ProbDev& pd, const Layout& L, char* ws, int need64, cudaStream_t st) {
  const int gi = (pd.n + kTileI - 1) / kTileI;
  int gj = (152 * 8 + gi - 1) / gi;
  if (gj < 1) gj = 1;
  int jchunk = (pd.m + gj - 1) / gj;
  jchunk = std::max(jchunk, 64);
  gj = (pd.m + jchunk - 1) / jchunk;
  dim3 grid(gi, gj);
  const size_t shm = (pd.cv.C32 || pd.d > kMaxDReg) ? 0 : (size_t)kTileJ * pd.d * sizeof(float);
  SketchScalars* sc = at<SketchScalars>(ws, L.scal);
  const int* gate = nullptr;
  if (L.cmx && !need64 && !pd.cv.C32 && pd.cv.x32 && pd.d >= 1 && pd.d <= 16) {
    // bucketed bounds first; the full sweep below then runs only if its pair list overflowed
    SPS_TRY(launch_cost_max_pruned(pd.cv.x32, pd.cv.y32, pd.n, pd.m, pd.d, sc, ws + L.cmx, &gate, st));
  }
  switch (pd.cv.C32 ? 0 : pd.d) {
    case 2: k_cost_max<2><<<grid, kTileI, shm, st>>>(pd, sc, need64, jchunk, gate); break;
    case 3: k_cost_max<3><<<grid, kTileI, shm, st>>>(pd, sc, need64, jchunk, gate); break;
    case 5: k_cost_max<5><<<grid, kTileI, shm, st>>>(pd, sc, need64, jchunk, gate); break;
    case 10: k_cost_max<10><<<grid, kTileI, shm, st>>>(pd, sc, need64, jchunk, gate); break;
    default: k_cost_max<0><<<grid, kTileI, shm, st>>>(pd, sc, need64, jchunk, gate); break;
  }
  add_launches(1);
  return cuda_fail(cudaGetLastError(), "cost_max");
}

// The same maximum for bare binary32 point arrays (the warm start's cost
// divisor); scratch holds one SketchScalars and must start at zero.
sps_status launch_cost_max_points(const float* x, int n, const float* y, int m, int d, void* scratch,
                                  cudaStream_t st) {
  ProbDev pd;
  memset(&pd, 0, sizeof(pd));
  pd.n = n; pd.m = m; pd.d = d;
  pd.cv.x32 = x; pd.cv.y32 = y; pd.cv.n = n; pd.cv.m = m; pd.cv.d = d;
  Layout L;
  memset(&L, 0, sizeof(L));
  L.scal = 0;
  return launch_cost_max(pd, L, (char*)scratch, 0, st);
}

sps_status launch_scalars0(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st) {
  k_scalars<<<1, 32, 0, st>>>(pd, at<SketchScalars>(ws, L.scal), at<Ctrl>(ws, L.ctrl), 0);
  add_launches(1);
  return cuda_fail(cudaGetLastError(), "scalars");
}

sps_status launch_factors(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st) {
  SketchScalars* sc = at<SketchScalars>(ws, L.scal);
  Ctrl* ctrl = at<Ctrl>(ws, L.ctrl);
  const float* a32 = at<float>(ws, L.a32);
  const float* b32 = at<float>(ws, L.b32);
  float* rowf = at<float>(ws, L.rowf);
  float* colf = at<float>(ws, L.colf);
  k_scalars<<<1, 32, 0, st>>>(pd, sc, ctrl, 0);
  const int g = grid_for(std::max(pd.n, pd.m), kThreads);
  if (pd.probs == SPS_PROBS_EQUAL) {
    k_eq_factors<<<g, kThreads, 0, st>>>(pd, sc, rowf, colf);
  } else if (pd.is_ot) {
    k_ot_sqrt_sums<<<g, kThreads, 0, st>>>(pd, sc, a32, b32);
    k_scalars<<<1, 32, 0, st>>>(pd, sc, ctrl, 1);
    k_ot_factors<<<g, kThreads, 0, st>>>(pd, sc, a32, b32, rowf, colf);
  } else {
    cudaMemsetAsync(&sc->maxa, 0, sizeof(float), st);
    cudaMemsetAsync(&sc->maxb, 0, sizeof(float), st);
    k_uot_factors<<<g, kThreads, 0, st>>>(pd, sc, a32, b32, rowf, colf);
    launch_uot_Z(pd, L, ws, st);
    k_scalars<<<1, 32, 0, st>>>(pd, sc, ctrl, 2);
  }
  add_launches(4);
  return cuda_fail(cudaGetLastError(), "factors");
}

template <typename V>
static void csc_sort(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st) {
  const int gs = grid_for((int64_t)pd.m * 32, 32 * kSortWarps);
  // the stabilised solve with binary32 points forms only log K~ in the fill (the
  // absorption writes K' later): no values to transpose then
  const bool vals = !(L.logval && !pd.cv.x64 && !pd.cv.C32 && !pd.cv.C64 && pd.cost_kind != SPS_COST_WFR);
  k_csc_sort<V><<<gs, 32 * kSortWarps, 0, st>>>(pd.m, at<int>(ws, L.col_ptr), at<int>(ws, L.tmp_row),
                                                at<int>(ws, L.tmp_src), vals ? at<V>(ws, L.val) : nullptr,
                                                at<int>(ws, L.row_idx), at<int>(ws, L.csr_pos),
                                                vals ? at<V>(ws, L.valT) : nullptr, at<Ctrl>(ws, L.ctrl),
                                                L.logval ? at<float>(ws, L.logval) : nullptr,
                                                L.logvalT ? at<float>(ws, L.logvalT) : nullptr);
}

// Shared with the batched sketch (one block-diagonal CSR / CSC for all pairs).
void launch_scan_counts(const int* row_cnt, int* row_ptr, int n, const int* col_cnt, int* col_ptr, int* col_cur,
                        int m, long long cap, Ctrl* ctrl, cudaStream_t st) {
  k_scan2<<<2, 1024, 0, st>>>(row_cnt, row_ptr, n, col_cnt, col_ptr, col_cur, m, cap, ctrl);
}

void launch_csc_sort(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st) {
  switch (kd) {
    case SPS_F64: csc_sort<double>(pd, L, ws, st); break;
    case SPS_F32: csc_sort<float>(pd, L, ws, st); break;
    case SPS_BF16: csc_sort<__nv_bfloat16>(pd, L, ws, st); break;
    case SPS_F16: csc_sort<__half>(pd, L, ws, st); break;
  }
}

void launch_csc_sort_f32(int m, const int* col_ptr, const int* tmp_row, const int* tmp_src, const float* val,
                         int* row_idx, int* csr_pos, float* valT, Ctrl* ctrl, cudaStream_t st) {
  const int gs = grid_for((int64_t)m * 32, 32 * kSortWarps);
  k_csc_sort<float><<<gs, 32 * kSortWarps, 0, st>>>(m, col_ptr, tmp_row, tmp_src, val, row_idx, csr_pos, valT, ctrl,
                                                    nullptr, nullptr);
}

sps_status launch_sample(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st) {
  Ctrl* ctrl = at<Ctrl>(ws, L.ctrl);
  int* row_cnt = at<int>(ws, L.row_cnt);
  int* col_cnt = at<int>(ws, L.col_cnt);
  if (L.pad_ofs) {
    // one sweep into padded (row, chunk) slots; compaction gives the two-pass positions
    cudaMemsetAsync(col_cnt, 0, sizeof(int) * (size_t)pd.m, st);
    launch_fused(pd, L, ws, kd, st);
    Ctrl h;
    cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "single-pass sketch");
    if (h.status == SPS_OK && !h.pad_overflow) {
      launch_sum_chunks(pd, L, ws, st);
      k_scan2<<<2, 1024, 0, st>>>(row_cnt, at<int>(ws, L.row_ptr), pd.n, col_cnt, at<int>(ws, L.col_ptr),
                                  at<int>(ws, L.col_cur), pd.m, (long long)L.cap, ctrl);
      launch_compact(pd, L, ws, kd, st);
      switch (kd) {
        case SPS_F64: csc_sort<double>(pd, L, ws, st); break;
        case SPS_F32: csc_sort<float>(pd, L, ws, st); break;
        case SPS_BF16: csc_sort<__nv_bfloat16>(pd, L, ws, st); break;
        case SPS_F16: csc_sort<__half>(pd, L, ws, st); break;
      }
      add_launches(7);
      return cuda_fail(cudaGetLastError(), "single-pass sketch");
    }
    if (h.status != SPS_OK) return SPS_OK;   // the caller reports the status
    // a slot was too small: clear the flag and run the two passes
    cudaMemsetAsync(&ctrl->pad_overflow, 0, sizeof(int), st);
  }
  cudaMemsetAsync(col_cnt, 0, sizeof(int) * (size_t)pd.m, st);
  launch_count(pd, L, ws, st);
  k_scan2<<<2, 1024, 0, st>>>(row_cnt, at<int>(ws, L.row_ptr), pd.n, col_cnt, at<int>(ws, L.col_ptr),
                              at<int>(ws, L.col_cur), pd.m, (long long)L.cap, ctrl);
  launch_fill(pd, L, ws, kd, st);
  switch (kd) {
    case SPS_F64: csc_sort<double>(pd, L, ws, st); break;
    case SPS_F32: csc_sort<float>(pd, L, ws, st); break;
    case SPS_BF16: csc_sort<__nv_bfloat16>(pd, L, ws, st); break;
    case SPS_F16: csc_sort<__half>(pd, L, ws, st); break;
  }
  add_launches(5);
  return cuda_fail(cudaGetLastError(), "sample");
}

}  // namespace sps
