// sps_costmax.cu -- the cost divisor max_ij D_ij (section 5.1 divides the
// squared Euclidean cost by its maximum) without visiting every pair
// (the grid-bucketed bounds below for d <= 4, radial bounds for larger d).
//
// D_ij is the binary32 spec distance (fl(x_ik - y_jk), then fma-accumulated
// in k order: raw32()).  A maximum is exact, so any algorithm that evaluates
// the maximising pair with that formula returns the same number as the full
// n x m sweep.  Here the points of x and of y are bucketed into one grid
// over (up to) three coordinates of largest extent; every cell gets its
// bounding box in all d coordinates; a cell pair's largest possible distance
// is bounded from the boxes, in binary32 with a relative margin of 2^-12 (far
// above the rounding of the spec formula and of the bound itself, at most
// (2d + 4) 2^-24 for d <= 16); the pair of cells with the largest bound is
// evaluated exactly (a lower bound L), then every cell pair whose bound
// reaches L (1 - 2^-12) is evaluated exactly.  A pair outside that list has
// every D_ij below L, so the result is the maximum over all pairs.  If the
// list overflows its capacity, the full sweep runs instead.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "sps_internal.h"

namespace sps {

namespace {

constexpr int kMaxCells = 65536;
constexpr int kMaxPairs = 1 << 20;
constexpr float kMargin = 2.44140625e-04f;   // 2^-12

// Float <-> order-preserving int (for atomic min / max of signed floats).
__device__ __forceinline__ int ord_of(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float float_of(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7fffffff); }

struct CmState {
  int ext_lo[16], ext_hi[16];   // ordered ints of the per-coordinate extent over x and y
  int dims[3], g[3];
  float lo[3], inv[3];
  int ncell;
  int npairs;
  int overflow;
  unsigned long long best;      // (bound bits << 32) | pair index of the largest bound
};

struct CmArgs {
  const float* x;   // n * d
  const float* y;   // m * d
  int n, m, d;
  CmState* st;
  int* cnt;         // [2][kMaxCells + 1]: counts, then offsets (x cells, y cells)
  int* cur;         // [2][kMaxCells]
  int* perm;        // [n + m]: point indices grouped by cell (x, then y)
  float* box;       // [2][kMaxCells][2 d]: per cell min (d) then max (d)
  int* pairs;       // [kMaxPairs][2]
  SketchScalars* sc;
};

__global__ void k_cm_init(CmArgs A) {
  const int t = threadIdx.x;
  if (t < 16) { A.st->ext_lo[t] = 0x7fffffff; A.st->ext_hi[t] = (int)0x80000000; }
  if (t == 0) { A.st->npairs = 0; A.st->overflow = 0; A.st->best = 0ull; }
  for (int c = t; c < 2 * (kMaxCells + 1); c += blockDim.x) A.cnt[c] = 0;
}

__global__ void k_cm_extent(CmArgs A) {
  const int d = A.d;
  for (int k = 0; k < d; ++k) {
    int lo = 0x7fffffff, hi = (int)0x80000000;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.n + A.m;
         p += (long long)gridDim.x * blockDim.x) {
      const float v = p < A.n ? A.x[p * d + k] : A.y[(p - A.n) * d + k];
      const int o = ord_of(v);
      lo = min(lo, o);
      hi = max(hi, o);
    }
    for (int s = 16; s > 0; s >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, s));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, s));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&A.st->ext_lo[k], lo);
      atomicMax(&A.st->ext_hi[k], hi);
    }
  }
}

// Grid: the (up to) three coordinates of largest extent, the same number of
// cells along each, about max(n, m) / 64 cells in all (at most kMaxCells).
__global__ void k_cm_params(CmArgs A) {
  CmState* S = A.st;
  const int d = A.d;
  float ext[16];
  for (int k = 0; k < d; ++k) ext[k] = float_of(S->ext_hi[k]) - float_of(S->ext_lo[k]);
  const int kd = min(3, d);
  for (int r = 0; r < 3; ++r) { S->dims[r] = 0; S->g[r] = 1; S->lo[r] = 0.0f; S->inv[r] = 0.0f; }
  bool used[16] = {false};
  for (int r = 0; r < kd; ++r) {
    int bk = -1;
    for (int k = 0; k < d; ++k)
      if (!used[k] && (bk < 0 || ext[k] > ext[bk])) bk = k;
    used[bk] = true;
    S->dims[r] = bk;
  }
  const double target = fmin((double)kMaxCells, fmax(1.0, (double)max(A.n, A.m) / 64.0));
  const int g = max(1, (int)floor(pow(target, 1.0 / kd) + 1e-9));
  int ncell = 1;
  for (int r = 0; r < kd; ++r) {
    const int k = S->dims[r];
    const float e = ext[k];
    if (e > 0.0f && isfinite(e)) {
      S->g[r] = g;
      S->lo[r] = float_of(S->ext_lo[k]);
      S->inv[r] = (float)g / (e * 1.000001f);
    }
    ncell *= S->g[r];
  }
  S->ncell = ncell;
}

__device__ __forceinline__ int cell_of(const CmState& S, const float* p) {
  int c = 0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    int q = (int)floorf((p[S.dims[r]] - S.lo[r]) * S.inv[r]);
    q = min(max(q, 0), S.g[r] - 1);
    c = c * S.g[r] + q;
  }
  return c;
}

__global__ void k_cm_count(CmArgs A) {
  const CmState S = *A.st;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.n + A.m;
       p += (long long)gridDim.x * blockDim.x) {
    const bool isx = p < A.n;
    const float* pt = isx ? A.x + p * A.d : A.y + (p - A.n) * A.d;
    atomicAdd(&A.cnt[(isx ? 0 : kMaxCells + 1) + cell_of(S, pt)], 1);
  }
}

// Exclusive scans of the two count arrays (block 0: x, block 1: y).
__global__ void __launch_bounds__(1024) k_cm_scan(CmArgs A) {
  __shared__ int sh[1024];
  const int ncell = A.st->ncell;
  int* cnt = A.cnt + blockIdx.x * (kMaxCells + 1);
  int* cur = A.cur + blockIdx.x * kMaxCells;
  const int T = blockDim.x, t = threadIdx.x;
  const int chunk = (ncell + T - 1) / T;
  const int lo = min(ncell, t * chunk), hi = min(ncell, lo + chunk);
  int s = 0;
  for (int c = lo; c < hi; ++c) s += cnt[c];
  sh[t] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    const int v = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  int run = sh[t] - s;
  for (int c = lo; c < hi; ++c) {
    const int k = cnt[c];
    cnt[c] = run;
    cur[c] = run;
    run += k;
  }
  if (t == T - 1) cnt[ncell] = sh[T - 1];
}

__global__ void k_cm_scatter(CmArgs A) {
  const CmState S = *A.st;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.n + A.m;
       p += (long long)gridDim.x * blockDim.x) {
    const bool isx = p < A.n;
    const int idx = isx ? (int)p : (int)(p - A.n);
    const float* pt = isx ? A.x + (long long)idx * A.d : A.y + (long long)idx * A.d;
    const int c = cell_of(S, pt);
    const int pos = atomicAdd(&A.cur[(isx ? 0 : kMaxCells) + c], 1);
    A.perm[(isx ? 0 : A.n) + pos] = idx;
  }
}

// Bounding box of every cell (one warp per cell); empty cells get min > max.
__global__ void k_cm_boxes(CmArgs A) {
  const int ncell = A.st->ncell, d = A.d, lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < 2 * ncell; w += warps) {
    const int side = w >= ncell, c = side ? w - ncell : w;
    const int* off = A.cnt + side * (kMaxCells + 1);
    const int* perm = A.perm + (side ? A.n : 0);
    const float* pts = side ? A.y : A.x;
    float* bx = A.box + ((size_t)side * kMaxCells + c) * 2 * d;
    for (int k = 0; k < d; ++k) {
      float lo = __int_as_float(0x7f800000), hi = __int_as_float(0xff800000);
      for (int q = off[c] + lane; q < off[c + 1]; q += 32) {
        const float v = pts[(long long)perm[q] * d + k];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
      }
      for (int s = 16; s > 0; s >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, s));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, s));
      }
      if (lane == 0) { bx[k] = lo; bx[d + k] = hi; }
    }
  }
}

// Bound of a cell pair (x box bx, y box by): sum over coordinates of the
// largest squared difference, times (1 + margin); -1 when a cell is empty.
__device__ __forceinline__ float pair_bound(const float* bx, const float* by, int d) {
  float u = 0.0f;
  for (int k = 0; k < d; ++k) {
    if (!(bx[k] <= bx[d + k]) || !(by[k] <= by[d + k])) return -1.0f;
    const float t = fmaxf(bx[d + k] - by[k], by[d + k] - bx[k]);
    u = fmaf(t, t, u);
  }
  return u * (1.0f + kMargin);
}

// PASS 0: the pair of largest bound; PASS 1: the list of pairs whose bound
// reaches the exact maximum found so far, less the margin.
template <int PASS>
__global__ void __launch_bounds__(256) k_cm_prune(CmArgs A) {
  const int ncell = A.st->ncell, d = A.d;
  __shared__ float ys[256 * 32];
  const float lb = PASS == 1 ? A.sc->dmax32 * (1.0f - kMargin) : 0.0f;
  unsigned long long best = 0ull;
  for (int cx0 = blockIdx.x * 256; cx0 < ncell; cx0 += gridDim.x * 256) {
    const int cx = cx0 + threadIdx.x;
    float bx[32];
    const bool vx = cx < ncell;
    for (int k = 0; k < 2 * d; ++k) bx[k] = vx ? A.box[(size_t)cx * 2 * d + k] : 0.0f;
    for (int cy0 = blockIdx.y * 256; cy0 < ncell; cy0 += gridDim.y * 256) {
      const int ny = min(256, ncell - cy0);
      __syncthreads();
      for (int t = threadIdx.x; t < ny * 2 * d; t += blockDim.x)
        ys[t] = A.box[((size_t)kMaxCells + cy0) * 2 * d + t];
      __syncthreads();
      if (!vx) continue;
      for (int q = 0; q < ny; ++q) {
        const float u = pair_bound(bx, ys + q * 2 * d, d);
        if (u < 0.0f) continue;
        const int cy = cy0 + q;
        if (PASS == 0) {
          const unsigned long long key =
              ((unsigned long long)__float_as_uint(u) << 32) | ((unsigned)cx * (unsigned)ncell + (unsigned)cy);
          best = key > best ? key : best;
        } else if (u >= lb) {
          const int slot = atomicAdd(&A.st->npairs, 1);
          if (slot < kMaxPairs) {
            A.pairs[2 * slot] = cx;
            A.pairs[2 * slot + 1] = cy;
          } else {
            A.st->overflow = 1;
          }
        }
      }
    }
  }
  if (PASS == 0) {
    for (int s = 16; s > 0; s >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, s);
      best = o > best ? o : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&A.st->best, best);
  }
}

__device__ __forceinline__ void atomic_max_nonneg_f(float* addr, float v) {
  atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
}

// Exact spec distances over the points of one x cell and one y cell.
__device__ void eval_pair(const CmArgs& A, int cx, int cy) {
  const int d = A.d;
  const int* ox = A.cnt;
  const int* oy = A.cnt + kMaxCells + 1;
  const int* px = A.perm;
  const int* py = A.perm + A.n;
  float best = 0.0f;
  for (int qi = ox[cx] + threadIdx.x; qi < ox[cx + 1]; qi += blockDim.x) {
    const float* xi = A.x + (long long)px[qi] * d;
    for (int qj = oy[cy]; qj < oy[cy + 1]; ++qj) {
      const float* yj = A.y + (long long)py[qj] * d;
      float acc = 0.0f;
      for (int k = 0; k < d; ++k) {
        const float t = __fsub_rn(xi[k], yj[k]);
        acc = __fmaf_rn(t, t, acc);
      }
      best = fmaxf(best, acc);
    }
  }
  for (int s = 16; s > 0; s >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, s));
  if ((threadIdx.x & 31) == 0 && best > 0.0f) atomic_max_nonneg_f(&A.sc->dmax32, best);
}

__global__ void k_cm_eval_best(CmArgs A) {
  const unsigned long long key = A.st->best;
  if (!key) return;
  const int ncell = A.st->ncell;
  const unsigned idx = (unsigned)(key & 0xffffffffull);
  eval_pair(A, (int)(idx / (unsigned)ncell), (int)(idx % (unsigned)ncell));
}

__global__ void k_cm_eval_list(CmArgs A) {
  if (A.st->overflow) return;
  const int np = min(A.st->npairs, kMaxPairs);
  for (int p = blockIdx.x; p < np; p += gridDim.x) eval_pair(A, A.pairs[2 * p], A.pairs[2 * p + 1]);
}

// ---------------------------------------------------------------------------
// Radial variant (any d): with c the centre of the bounding box of x and y,
// |x_i - y_j| <= |x_i - c| + |y_j - c|.  A pair whose spec distance reaches
// an exact value L found so far needs |x_i - c| >= sqrt(L) - max_j |y_j - c|
// and |y_j - c| >= sqrt(L) - max_i |x_i - c| (both with a relative margin of
// 2^-10, far above the binary32 rounding of the radii); L is the maximum over
// the farthest x against all y and all x against the farthest y.  Only the
// pairs of the two selected sets are evaluated; if that product exceeds a
// quarter of n m the full sweep runs instead.
// ---------------------------------------------------------------------------
struct NmState {
  int ext_lo[16], ext_hi[16];
  float c[16];
  unsigned long long far_x, far_y;   // (radius bits << 32) | index of the largest radius
  int nx_sel, ny_sel;
  int overflow;
};

struct NmArgs {
  const float* x;
  const float* y;
  int n, m, d;
  NmState* st;
  float* rx;   // [n]
  float* ry;   // [m]
  int* sx;     // [n] selected x
  int* sy;     // [m] selected y
  SketchScalars* sc;
  long long budget;
};

constexpr float kRadMargin = 9.765625e-04f;   // 2^-10

__global__ void k_nm_init(NmArgs A) {
  const int t = threadIdx.x;
  if (t < 16) { A.st->ext_lo[t] = 0x7fffffff; A.st->ext_hi[t] = (int)0x80000000; }
  if (t == 0) { A.st->far_x = 0ull; A.st->far_y = 0ull; A.st->nx_sel = 0; A.st->ny_sel = 0; A.st->overflow = 0; }
}

__global__ void k_nm_extent(NmArgs A) {
  const int d = A.d;
  for (int k = 0; k < d; ++k) {
    int lo = 0x7fffffff, hi = (int)0x80000000;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.n + A.m;
         p += (long long)gridDim.x * blockDim.x) {
      const float v = p < A.n ? A.x[p * d + k] : A.y[(p - A.n) * d + k];
      const int o = ord_of(v);
      lo = min(lo, o);
      hi = max(hi, o);
    }
    for (int s2 = 16; s2 > 0; s2 >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, s2));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, s2));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&A.st->ext_lo[k], lo);
      atomicMax(&A.st->ext_hi[k], hi);
    }
  }
}

__global__ void k_nm_radii(NmArgs A) {
  const int d = A.d;
  float c[16];
  for (int k = 0; k < d; ++k) c[k] = 0.5f * (float_of(A.st->ext_lo[k]) + float_of(A.st->ext_hi[k]));
  if (blockIdx.x == 0 && threadIdx.x < d) A.st->c[threadIdx.x] = c[threadIdx.x];
  unsigned long long bx = 0ull, by = 0ull;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.n + A.m;
       p += (long long)gridDim.x * blockDim.x) {
    const bool isx = p < A.n;
    const int idx = isx ? (int)p : (int)(p - A.n);
    const float* pt = isx ? A.x + (long long)idx * d : A.y + (long long)idx * d;
    float acc = 0.0f;
    for (int k = 0; k < d; ++k) {
      const float t = pt[k] - c[k];
      acc = fmaf(t, t, acc);
    }
    const float r = sqrtf(acc);
    const unsigned long long key = ((unsigned long long)__float_as_uint(r) << 32) | (unsigned)idx;
    if (isx) { A.rx[idx] = r; bx = key > bx ? key : bx; }
    else { A.ry[idx] = r; by = key > by ? key : by; }
  }
  for (int s2 = 16; s2 > 0; s2 >>= 1) {
    const unsigned long long ox = __shfl_xor_sync(0xffffffffu, bx, s2), oy = __shfl_xor_sync(0xffffffffu, by, s2);
    bx = ox > bx ? ox : bx;
    by = oy > by ? oy : by;
  }
  if ((threadIdx.x & 31) == 0) {
    if (bx) atomicMax(&A.st->far_x, bx);
    if (by) atomicMax(&A.st->far_y, by);
  }
}

__device__ __forceinline__ float spec_dist(const float* xi, const float* yj, int d) {
  float acc = 0.0f;
  for (int k = 0; k < d; ++k) {
    const float t = __fsub_rn(xi[k], yj[k]);
    acc = __fmaf_rn(t, t, acc);
  }
  return acc;
}

// The farthest x against all y and all x against the farthest y, exactly.
__global__ void k_nm_lower(NmArgs A) {
  const int d = A.d;
  const int ix = (int)(A.st->far_x & 0xffffffffull), iy = (int)(A.st->far_y & 0xffffffffull);
  const float* xf = A.x + (long long)ix * d;
  const float* yf = A.y + (long long)iy * d;
  float best = 0.0f;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.n + A.m;
       p += (long long)gridDim.x * blockDim.x) {
    best = fmaxf(best, p < A.n ? spec_dist(A.x + p * d, yf, d) : spec_dist(xf, A.y + (p - A.n) * d, d));
  }
  for (int s2 = 16; s2 > 0; s2 >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, s2));
  if ((threadIdx.x & 31) == 0 && best > 0.0f) atomic_max_nonneg_f(&A.sc->dmax32, best);
}

__global__ void k_nm_select(NmArgs A) {
  const float L = sqrtf(A.sc->dmax32) * (1.0f - kRadMargin);
  const float Rx = __uint_as_float((unsigned)(A.st->far_x >> 32)) * (1.0f + kRadMargin);
  const float Ry = __uint_as_float((unsigned)(A.st->far_y >> 32)) * (1.0f + kRadMargin);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.n + A.m;
       p += (long long)gridDim.x * blockDim.x) {
    if (p < A.n) {
      if (A.rx[p] * (1.0f + kRadMargin) >= L - Ry) A.sx[atomicAdd(&A.st->nx_sel, 1)] = (int)p;
    } else {
      const int j = (int)(p - A.n);
      if (A.ry[j] * (1.0f + kRadMargin) >= L - Rx) A.sy[atomicAdd(&A.st->ny_sel, 1)] = j;
    }
  }
}

__global__ void k_nm_pairs(NmArgs A) {
  const int nx = A.st->nx_sel, ny = A.st->ny_sel, d = A.d;
  if ((long long)nx * ny > A.budget) {
    if (blockIdx.x == 0 && threadIdx.x == 0) A.st->overflow = 1;
    return;
  }
  float best = 0.0f;
  const long long tot = (long long)nx * ny;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(q / ny), b = (int)(q % ny);
    best = fmaxf(best, spec_dist(A.x + (long long)A.sx[a] * d, A.y + (long long)A.sy[b] * d, d));
  }
  for (int s2 = 16; s2 > 0; s2 >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, s2));
  if ((threadIdx.x & 31) == 0 && best > 0.0f) atomic_max_nonneg_f(&A.sc->dmax32, best);
}

}  // namespace

size_t cost_max_scratch_bytes(int n, int m, int d) {
  const size_t grid = 1024 + 512 + sizeof(int) * (2 * (size_t)(kMaxCells + 1) + 2 * (size_t)kMaxCells + (size_t)n + m) +
                      sizeof(float) * 2 * (size_t)kMaxCells * 2 * d + sizeof(int) * 2 * (size_t)kMaxPairs;
  const size_t radial = 1024 + 512 + (sizeof(float) + sizeof(int)) * ((size_t)n + m);
  return d > 4 ? radial : grid;
}

// Scratch layout: CmState (padded to 1 KB), counts, cursors, permutation,
// boxes, pair list.  Returns the device flag that is set when the pair list
// overflowed (the caller then runs the full sweep, gated on it).
sps_status launch_cost_max_pruned(const float* x, const float* y, int n, int m, int d, SketchScalars* sc,
                                  char* scratch, const int** overflow_flag, cudaStream_t st) {
  const int gp = (int)std::min<long long>(152 * 8, ((long long)n + m + 255) / 256);
  if (d > 4) {
    NmArgs B;
    B.x = x; B.y = y; B.n = n; B.m = m; B.d = d; B.sc = sc;
    char* q = scratch;
    B.st = reinterpret_cast<NmState*>(q); q += 1024;
    B.rx = reinterpret_cast<float*>(q); q += sizeof(float) * (size_t)n;
    B.ry = reinterpret_cast<float*>(q); q += sizeof(float) * (size_t)m;
    B.sx = reinterpret_cast<int*>(q); q += sizeof(int) * (size_t)n;
    B.sy = reinterpret_cast<int*>(q);
    B.budget = (long long)n * m / 4;
    k_nm_init<<<1, 32, 0, st>>>(B);
    k_nm_extent<<<gp, 256, 0, st>>>(B);
    k_nm_radii<<<gp, 256, 0, st>>>(B);
    k_nm_lower<<<gp, 256, 0, st>>>(B);
    k_nm_select<<<gp, 256, 0, st>>>(B);
    k_nm_pairs<<<152 * 8, 256, 0, st>>>(B);
    add_launches(6);
    *overflow_flag = &B.st->overflow;
    return cuda_fail(cudaGetLastError(), "radial cost max");
  }
  CmArgs A;
  A.x = x; A.y = y; A.n = n; A.m = m; A.d = d;
  A.sc = sc;
  char* p = scratch;
  A.st = reinterpret_cast<CmState*>(p); p += 1024;
  A.cnt = reinterpret_cast<int*>(p); p += sizeof(int) * 2 * (size_t)(kMaxCells + 1);
  A.cur = reinterpret_cast<int*>(p); p += sizeof(int) * 2 * (size_t)kMaxCells;
  A.perm = reinterpret_cast<int*>(p); p += sizeof(int) * ((size_t)n + m);
  p = scratch + ((p - scratch + 255) & ~(size_t)255);
  A.box = reinterpret_cast<float*>(p); p += sizeof(float) * 2 * (size_t)kMaxCells * 2 * d;
  A.pairs = reinterpret_cast<int*>(p);
  k_cm_init<<<1, 1024, 0, st>>>(A);
  k_cm_extent<<<gp, 256, 0, st>>>(A);
  k_cm_params<<<1, 1, 0, st>>>(A);
  k_cm_count<<<gp, 256, 0, st>>>(A);
  k_cm_scan<<<2, 1024, 0, st>>>(A);
  k_cm_scatter<<<gp, 256, 0, st>>>(A);
  k_cm_boxes<<<152 * 4, 256, 0, st>>>(A);
  const dim3 pg(std::max(1, std::min(256, (kMaxCells + 255) / 256)), 16);
  k_cm_prune<0><<<pg, 256, 0, st>>>(A);
  k_cm_eval_best<<<1, 256, 0, st>>>(A);
  k_cm_prune<1><<<pg, 256, 0, st>>>(A);
  k_cm_eval_list<<<152 * 8, 128, 0, st>>>(A);
  add_launches(11);
  *overflow_flag = &A.st->overflow;
  return cuda_fail(cudaGetLastError(), "pruned cost max");
}

}  // namespace sps
