// sps_sweep.cu -- the n x m sweeps of the sketch (section 3, Eq. pois):
//   Z      UOT normaliser Z = sum_ij A_i B_j exp(-D_ij kappa) (Eq. pij-uot), exact
//   COUNT  kept elements per (row, column chunk) and per column
//   FILL   CSR entries (columns ascending) and an unordered CSC scatter
// All three walk the same tiling: a block owns 32 rows (4 per warp) and one
// column chunk; the chunk is cut into tiles of kTJ columns whose decision
// factors c_j and (UOT) binary32 coordinates are staged in shared memory,
// coordinates transposed so that a lane reads the four columns of its Philox
// block with one 128-bit load per coordinate.  Lane l of a warp handles the
// Philox block q = tile_q0 + s*32 + l (columns 4q .. 4q+3) at step s.
// The per-element decision is the binary32 computation of pstar_raw().
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "sps_internal.h"

namespace sps {

namespace {

constexpr int kRW = 4;          // rows per warp
constexpr int kSweepThreads = 256;  // 8 warps
constexpr int kRB = (kSweepThreads / 32) * kRW;  // rows per block
constexpr int kTJ = 512;        // columns per shared-memory tile
constexpr int kSteps = kTJ / 128;
constexpr int kMaxDSmem = 16;   // coordinates staged for d <= 16; larger d reads global memory

enum { SW_Z = 0, SW_COUNT = 1, SW_FILL = 2, SW_FUSED = 3 };

struct SweepArgs {
  ProbDev pd;
  SketchScalars* sc;
  const float* rowf;
  const float* colf;
  int* cnt2;          // [nchunk][n] kept elements per (chunk, row)
  int* col_cnt;       // [m]
  const int* row_ptr;
  int* col_idx;
  void* val;
  int* col_cur;
  const int* col_end;   // col_ptr + 1: end of every column segment
  float* logval;        // log-domain: log K~ of every kept element (or null)
  int* tmp_row;
  int* tmp_src;
  Ctrl* ctrl;
  int chunk;          // columns per chunk (multiple of kTJ)
  int nchunk;
  // single-pass sketch: padded slots per (row, chunk), row-major [i * nchunk + c]
  const int* pad_ofs;   // n * nchunk + 1 offsets
  int* pad_col;
  void* pad_val;
  float* pad_lv;
  float* zsum;          // UOT Z sweep: [nchunk][n] sums of w per (row, chunk) (or null)
  int* cnt_row;         // skip sampler: kept elements per row
};

template <typename V> struct ValMath;
// K~_ij = K_ij / p*_ij of a sampled element; the WFR cost always goes through
// FP64 (its slope grows without bound at the blocking edge d = pi eta).
template <> struct ValMath<double> {
  __device__ static double value(const ProbDev& pd, const SketchScalars& sc, int i, int j, float, float ps) {
    const double C = pd.cost_kind == SPS_COST_WFR ? value_cost64(pd, sc, i, j) : __ddiv_rn(raw64(pd.cv, i, j), sc.dn64);
    return exp(-C / pd.eps) / (double)ps;
  }
};
template <typename V> struct ValMath {
  __device__ static double value(const ProbDev& pd, const SketchScalars& sc, int i, int j, float D, float ps) {
    if (pd.cost_kind == SPS_COST_WFR) return exp(-value_cost64(pd, sc, i, j) / pd.eps) / (double)ps;
    const float C = __fdiv_rn(D, sc.dn32);
    return (double)(expf(-C / (float)pd.eps) / ps);
  }
};

template <int MODE, bool UOT, int D, typename V>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(SweepArgs A) {
  if (A.ctrl->status != SPS_OK) return;
  if (MODE == SW_FUSED && A.ctrl->pad_overflow) return;   // the slots were not laid out: two passes follow
  extern __shared__ __align__(16) float smem[];
  const ProbDev& pd = A.pd;
  const int n = pd.n, m = pd.m;
  const int d = pd.d;
  const bool stage_y = UOT && !pd.cv.C32 && d <= kMaxDSmem;
  float* ct = smem;           // [kTJ]
  float* yT = smem + kTJ;     // [d][kTJ]
  const float kappa = A.sc->kappa32, scale = A.sc->scale32;
  const int wfr = pd.cost_kind == SPS_COST_WFR;
  const float inv2eta = A.sc->inv2eta32, g2 = A.sc->g2_32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y;
  const int jc0 = c * A.chunk;
  const int jc1 = min(m, jc0 + A.chunk);
  U128 acc{0ull, 0ull};
  int Bz = 0;
  if (MODE == SW_Z) {
    Bz = exact_floor_for(fmaxf(__fmul_rn(A.sc->maxa, A.sc->maxb), 1e-30f));
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) A.sc->acc1.B = Bz;
  }
  constexpr int DR = D > 0 ? D : kMaxDSmem;
  if (blockDim.x != kSweepThreads) return;  // the row mapping assumes 8 warps
  // log K~ in binary32 arithmetic when the points are binary32 (no FP64 copy, no dense cost)
  const bool lv32 = (MODE == SW_FILL ? A.logval != nullptr : MODE == SW_FUSED ? A.pad_lv != nullptr : false) &&
                    !pd.cv.x64 && !pd.cv.C32 && !pd.cv.C64 && pd.cost_kind != SPS_COST_WFR;
  float k_hi = 0.0f, k_lo = 0.0f;
  if (lv32) {
    const double k64 = 1.0 / (A.sc->dn64 * pd.eps);   // one division per block
    k_hi = __double2float_rn(k64);
    k_lo = __double2float_rn(k64 - (double)k_hi);
  }
  for (int rb = blockIdx.x * kRB; rb < n; rb += gridDim.x * kRB) {
    // rows rb + warp*kRW + r, r < kRW, handled one after the other on each tile
    int cnt[kRW], pos0[kRW], pend[kRW];
    float zr[kRW];
#pragma unroll
    for (int r = 0; r < kRW; ++r) {
      const int i = rb + warp * kRW + r;
      cnt[r] = 0;
      zr[r] = 0.0f;
      pos0[r] = 0;
      pend[r] = 0;
      if (MODE == SW_FILL && i < n) pend[r] = A.row_ptr[i + 1];
      if (MODE == SW_FILL && i < n && A.rowf[i] > 0.0f) {
        int p = A.row_ptr[i];
        for (int cc = 0; cc < c; ++cc) p += A.cnt2[(size_t)cc * n + i];
        pos0[r] = p;
      }
      if (MODE == SW_FUSED && i < n) {
        pos0[r] = A.pad_ofs[(size_t)i * A.nchunk + c];
        pend[r] = A.pad_ofs[(size_t)i * A.nchunk + c + 1];
      }
    }
    for (int j0 = jc0; j0 < jc1; j0 += kTJ) {
      const int jn = min(kTJ, jc1 - j0);
      __syncthreads();
      for (int t = threadIdx.x; t < kTJ; t += blockDim.x) ct[t] = t < jn ? A.colf[j0 + t] : 0.0f;
      if (stage_y) {
        for (int t = threadIdx.x; t < jn; t += blockDim.x) {
          const float* yr = pd.cv.y32 + (int64_t)(j0 + t) * d;
#pragma unroll
          for (int k = 0; k < DR; ++k)
            if (D > 0 || k < d) yT[k * kTJ + t] = yr[k];
        }
      }
      __syncthreads();
#pragma unroll 1
      for (int r = 0; r < kRW; ++r) {
        const int i = rb + warp * kRW + r;
        const bool rv = i < n;
        const float ri = rv ? A.rowf[i] : 0.0f;
        if (!(rv && ri > 0.0f)) continue;  // uniform over the warp
        float xi[DR];
#pragma unroll
        for (int k = 0; k < DR; ++k) xi[k] = (UOT && stage_y && k < d) ? pd.cv.x32[(int64_t)i * d + k] : 0.0f;
#pragma unroll 1
        for (int s = 0; s < kSteps; ++s) {
          const int jl = 4 * (s * 32 + lane);
          const int j = j0 + jl;
          unsigned mask = 0u;
          float pe[4] = {0.f, 0.f, 0.f, 0.f};
          float Dv[4] = {0.f, 0.f, 0.f, 0.f};
          if (jl < jn) {
            const float4 c4 = *reinterpret_cast<const float4*>(&ct[jl]);
            const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
            if (UOT) {
              if (stage_y) {
#pragma unroll
                for (int k = 0; k < DR; ++k) {
                  if (D > 0 || k < d) {
                    const float4 y4 = *reinterpret_cast<const float4*>(&yT[k * kTJ + jl]);
                    float t;
                    t = __fsub_rn(xi[k], y4.x); Dv[0] = __fmaf_rn(t, t, Dv[0]);
                    t = __fsub_rn(xi[k], y4.y); Dv[1] = __fmaf_rn(t, t, Dv[1]);
                    t = __fsub_rn(xi[k], y4.z); Dv[2] = __fmaf_rn(t, t, Dv[2]);
                    t = __fsub_rn(xi[k], y4.w); Dv[3] = __fmaf_rn(t, t, Dv[3]);
                  }
                }
              } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) Dv[e] = (j + e < jc1) ? raw32(pd.cv, i, j + e) : 0.0f;
              }
            }
            uint4 dr = make_uint4(0u, 0u, 0u, 0u);
            if (MODE != SW_Z) dr = draw4(pd.seed, pd.pid, (uint32_t)i, (uint32_t)(j >> 2));
            const uint32_t dd[4] = {dr.x, dr.y, dr.z, dr.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (j + e < jc1) {
                float p;
                if (UOT) {
                  const float w = __fmul_rn(__fmul_rn(ri, cv[e]), uot_factor(wfr, Dv[e], kappa, inv2eta, g2));
                  if (MODE == SW_Z) { exact_add(acc, &A.sc->acc1, Bz, w); zr[r] += w; continue; }
                  p = __fmul_rn(scale, w);
                } else {
                  p = __fmul_rn(ri, cv[e]);
                }
                pe[e] = p;
                if (keep(dd[e], p)) mask |= 1u << e;
              }
            }
          }
          if (MODE == SW_COUNT || MODE == SW_FUSED) {
            cnt[r] += __popc(mask);
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (mask & (1u << e)) atomicAdd(&A.col_cnt[j + e], 1);
          }
          if (MODE == SW_FILL || MODE == SW_FUSED) {
            // most steps keep nothing anywhere in the warp
            if (__ballot_sync(0xffffffffu, mask != 0u) == 0u) continue;
            // warp prefix of the per-lane counts (0 .. 4) from three bit ballots
            const int cnum = __popc(mask);
            const unsigned c0 = __ballot_sync(0xffffffffu, cnum & 1), c1 = __ballot_sync(0xffffffffu, cnum & 2),
                           c2 = __ballot_sync(0xffffffffu, cnum & 4);
            const unsigned lt = (1u << lane) - 1u;
            const int excl = __popc(c0 & lt) + 2 * __popc(c1 & lt) + 4 * __popc(c2 & lt);
            const int total = __popc(c0) + 2 * __popc(c1) + 4 * __popc(c2);
            int pos = pos0[r] + excl;
            if (mask) {
              const SketchScalars& sc = *A.sc;
              V* val = (V*)(MODE == SW_FUSED ? A.pad_val : A.val);
              int* cidx = MODE == SW_FUSED ? A.pad_col : A.col_idx;
              float* lvo = MODE == SW_FUSED ? A.pad_lv : A.logval;
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                if (mask & (1u << e)) {
                  const int jj = j + e;
                  const float ps = pe[e] < 1.0f ? pe[e] : 1.0f;
                  // bounds checks: never written out of range.  FILL: a count/fill mismatch
                  // (a fault); FUSED: the padded slot was too small (the two-pass sweep reruns).
                  if (pos >= pend[r]) {
                    if (MODE == SW_FUSED) A.ctrl->pad_overflow = 1;
                    else A.ctrl->sketch_fault = 1;
                    ++pos;
                    continue;
                  }
                  cidx[pos] = jj;
                  if (lv32) {
                    // stabilised iterations: the absorption writes K' later; only log K~ = -C/eps - log p*
                    const float ce = cost_over_eps_df(pd.cv.x32 + (int64_t)i * d, pd.cv.y32 + (int64_t)jj * d, d,
                                                      k_hi, k_lo);
                    lvo[pos] = __fsub_rn(-ce, logf(ps));
                  } else {
                    const float Dd = UOT ? Dv[e] : raw32(pd.cv, i, jj);
                    val[pos] = from_d<V>(ValMath<V>::value(pd, sc, i, jj, Dd, ps));
                    if (lvo) {
                      // log K~ = -C/eps - log p*, C from the FP64 distance of the points
                      const double C64 = value_cost64(pd, sc, i, jj);
                      lvo[pos] = (float)(-C64 / pd.eps - (double)logf(ps));
                    }
                  }
                  if (MODE == SW_FILL) {
                    const int slot = atomicAdd(&A.col_cur[jj], 1);
                    if (slot < A.col_end[jj]) {
                      A.tmp_row[slot] = i;
                      A.tmp_src[slot] = pos;
                    } else {
                      A.ctrl->sketch_fault = 1;
                    }
                  }
                  ++pos;
                }
              }
            }
            pos0[r] += total;
          }
        }
      }
    }
    if (MODE == SW_COUNT || MODE == SW_FUSED) {
#pragma unroll
      for (int r = 0; r < kRW; ++r) {
        const int i = rb + warp * kRW + r;
        const int cs = warp_sum(cnt[r]);
        if (lane == 0 && i < n) A.cnt2[(size_t)c * n + i] = cs;
      }
    }
    if (MODE == SW_Z && A.zsum) {
#pragma unroll
      for (int r = 0; r < kRW; ++r) {
        const int i = rb + warp * kRW + r;
        const float zs = warp_sum(zr[r]);
        if (lane == 0 && i < n) A.zsum[(size_t)c * n + i] = zs;
      }
    }
  }
  if (MODE == SW_Z) exact_flush(acc, &A.sc->acc1);
}

// Row counts: sum of the per-chunk counts in chunk order.
__global__ void k_sum_chunks(int n, int nchunk, const int* cnt2, int* row_cnt, const Ctrl* ctrl) {
  if (ctrl->status != SPS_OK) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int s = 0;
    for (int c = 0; c < nchunk; ++c) s += cnt2[(size_t)c * n + i];
    row_cnt[i] = s;
  }
}


// ---------------------------------------------------------------------------
// Single-pass sketch.  The expected number of kept elements of (row i, chunk
// c) is bounded by mu = sum_j p_ij before clipping: OT r_i sum_{j in c} c_j,
// UOT fl32(s/Z) sum_{j in c} w_ij (from the Z sweep).  A slot of
// mu + 8 sqrt(mu) + 16 entries (at most the chunk's width) holds the pair's
// elements unless the count lies ~8 standard deviations above its mean; then
// the two-pass sweep runs instead, so the result never depends on the slots.
// ---------------------------------------------------------------------------
__global__ void k_chunk_csum(int m, int chunk, int nchunk, const float* colf, float* csum) {
  __shared__ float sh[32];
  for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const int j0 = c * chunk, j1 = min(m, j0 + chunk);
    float s = 0.0f;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) s += colf[j];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
      csum[c] = t;
    }
    __syncthreads();
  }
}

__global__ void k_pad_caps(int n, int m, int chunk, int nchunk, int uot, const float* rowf, const float* csum,
                           const float* zsum, const SketchScalars* sc, int* caps) {
  const float scale = sc->scale32;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < (long long)n * nchunk;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k / nchunk), c = (int)(k % nchunk);
    const float mu = uot ? scale * zsum[(size_t)c * n + i] : rowf[i] * csum[c];
    const int width = min(m, (c + 1) * chunk) - c * chunk;
    float cap = mu + 8.0f * sqrtf(fmaxf(mu, 0.0f)) + 16.0f;
    if (!(cap < (float)width)) cap = (float)width;   // also catches NaN
    caps[k] = (int)ceilf(cap);
  }
}

// Exclusive scan of len counts into ofs[0 .. len] by one block; a total above
// limit sets the overflow flag (the two-pass sweep then runs).
__global__ void __launch_bounds__(1024) k_pad_scan(const int* caps, int* ofs, long long len, long long limit,
                                                   Ctrl* ctrl) {
  __shared__ long long sh[1024];
  const int T = blockDim.x, t = threadIdx.x;
  const long long per = (len + T - 1) / T;
  const long long lo = min(len, (long long)t * per), hi = min(len, lo + per);
  long long s = 0;
  for (long long k = lo; k < hi; ++k) s += caps[k];
  sh[t] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    const long long v = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  const long long total = sh[T - 1];
  const bool over = total > limit;
  if (over && t == 0) ctrl->pad_overflow = 1;
  // offsets are always written (all zero when the slots do not fit), so that no
  // kernel can read an undefined value; the fused sweep skips on the flag
  long long run = sh[t] - s;
  for (long long k = lo; k < hi; ++k) {
    ofs[k] = over ? 0 : (int)run;
    run += caps[k];
  }
  if (t == T - 1) ofs[len] = over ? 0 : (int)total;
}

// Copy every (row, chunk) slot to its CSR position (row_ptr[i] plus the earlier
// chunks' counts: the positions of the two-pass fill) and scatter the CSC.
template <typename V>
__global__ void k_compact(int n, int nchunk, const int* pad_ofs, const int* cnt2, const int* row_ptr,
                          const int* pad_col, const V* pad_val, const float* pad_lv, int* col_idx, V* val,
                          float* logval, int* col_cur, const int* col_end, int* tmp_row, int* tmp_src, Ctrl* ctrl) {
  // pad_val is null when the sweep formed only log K~ (the absorption writes K' later)
  if (ctrl->status != SPS_OK || ctrl->pad_overflow) return;
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
    int dst = row_ptr[i];
    const int end = row_ptr[i + 1];
    for (int c = 0; c < nchunk; ++c) {
      const int src = pad_ofs[(size_t)i * nchunk + c];
      const int len = cnt2[(size_t)c * n + i];
      for (int e = lane; e < len; e += 32) {
        const int q = dst + e;
        if (q >= end) { ctrl->sketch_fault = 1; continue; }
        const int j = pad_col[src + e];
        col_idx[q] = j;
        if (pad_val) val[q] = pad_val[src + e];
        if (pad_lv) logval[q] = pad_lv[src + e];
        const int slot = atomicAdd(&col_cur[j], 1);
        if (slot < col_end[j]) {
          tmp_row[slot] = i;
          tmp_src[slot] = q;
        } else {
          ctrl->sketch_fault = 1;
        }
      }
      dst += len;
    }
  }
}

template <int MODE, bool UOT, int D, typename V>
void launch_sweep_d(const SweepArgs& A, dim3 grid, cudaStream_t st) {
  const bool stage = UOT && !A.pd.cv.C32 && A.pd.d <= kMaxDSmem;
  const size_t shm = (size_t)kTJ * sizeof(float) * (1 + (stage ? A.pd.d : 0));
  k_sweep<MODE, UOT, D, V><<<grid, kSweepThreads, shm, st>>>(A);
}

template <int MODE, bool UOT, typename V>
void launch_sweep(const SweepArgs& A, dim3 grid, cudaStream_t st) {
  if (!UOT) { launch_sweep_d<MODE, false, 1, V>(A, grid, st); return; }
  switch (A.pd.cv.C32 ? 0 : A.pd.d) {
    case 2: launch_sweep_d<MODE, true, 2, V>(A, grid, st); break;
    case 3: launch_sweep_d<MODE, true, 3, V>(A, grid, st); break;
    case 5: launch_sweep_d<MODE, true, 5, V>(A, grid, st); break;
    case 10: launch_sweep_d<MODE, true, 10, V>(A, grid, st); break;
    default: launch_sweep_d<MODE, true, 0, V>(A, grid, st); break;
  }
}

}  // namespace

// Geometry: row groups of 8 and column chunks (multiples of kTJ) chosen so
// that the grid holds at least four waves of 1216 blocks when n is small.
SweepGeo sweep_geometry(int n, int m) {
  const int groups = (n + kRB - 1) / kRB;
  int nchunk = (4 * 1216 + groups - 1) / groups;
  const int max_chunks = (m + kTJ - 1) / kTJ;
  nchunk = std::max(1, std::min(nchunk, std::min(max_chunks, 16)));
  int chunk = (m + nchunk - 1) / nchunk;
  chunk = ((chunk + kTJ - 1) / kTJ) * kTJ;
  nchunk = (m + chunk - 1) / chunk;
  SweepGeo g;
  g.nchunk = nchunk;
  g.chunk = chunk;
  g.row_blocks = std::min(groups, 152 * 64);
  return g;
}

// ---------------------------------------------------------------------------
// Skip sampler: the law of one Bernoulli(p*_ij) decision per element
// (Eq. pois) with work proportional to the sampled count.  Row i bounds every
// p_ij by q_i: OT (Eq. pij-ot) p_ij = fl(r_i c_j), q_i = min(1, fl(r_i cmax));
// UOT (Eq. pij-uot) p_ij = fl(scale fl(fl(A_i B_j) F(D_ij))) with F the
// decision factor of the cost (E(-D_ij kappa), or the WFR cos power), q_i =
// min(1, fl(scale fl(A_i cmax))) (F <= 1; rounding is monotone), cmax =
// max_j of the column factors.  Candidates form a Bernoulli(q_i) process generated by
// geometric gaps G = floor(log U / log(1 - q_i)), U = ((w >> 8) + 1) 2^-24
// on (0, 1]; a candidate j is kept when V < fl(p_ij / q_i), V = (w' >> 8)
// 2^-24.  Candidate t of row i reads Philox at counter (t >> 1, i, pid,
// 0x5B1E), words 2 (t & 1) and 2 (t & 1) + 1.  COUNT writes the row counts
// and the column counts, FILL the CSR entries and the CSC scatter.
// ---------------------------------------------------------------------------
enum { SK_COUNT = 0, SK_FILL = 1 };

__global__ void k_colf_max(const float* __restrict__ colf, int m, SketchScalars* sc) {
  float c = 0.0f;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) c = fmaxf(c, colf[j]);
  c = warp_max(c);
  if ((threadIdx.x & 31) == 0 && c > 0.0f) atomicMax(reinterpret_cast<int*>(&sc->cmax32), __float_as_int(c));
}

// One warp per row.  The gaps of a row's candidates depend only on their
// draws, so a warp computes 64 candidates at a time (lane l: candidates
// base + 2l and base + 2l + 1, which share one Philox call) and places them by
// a prefix sum of (1 + G); the row's candidate sequence, its stop and the
// order of the kept elements are those of the one-at-a-time definition.
template <int MODE, bool UOT, typename V>
__global__ void __launch_bounds__(256) k_skip(SweepArgs A) {
  if (A.ctrl->status != SPS_OK) return;
  const ProbDev& pd = A.pd;
  const int n = pd.n, m = pd.m, d = pd.d;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const float cmax = A.sc->cmax32;
  const float kappa = A.sc->kappa32, scale = A.sc->scale32;
  const int wfr = pd.cost_kind == SPS_COST_WFR;
  const float inv2eta = A.sc->inv2eta32, g2 = A.sc->g2_32;
  const bool lv32 = MODE == SK_FILL && A.logval != nullptr && !pd.cv.x64 && !pd.cv.C32 && !pd.cv.C64 && !wfr;
  float k_hi = 0.0f, k_lo = 0.0f;
  if (lv32) {
    const double k64 = 1.0 / (A.sc->dn64 * pd.eps);
    k_hi = __double2float_rn(k64);
    k_lo = __double2float_rn(k64 - (double)k_hi);
  }
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const float r = A.rowf[i];
    const float q = UOT ? __fmul_rn(scale, __fmul_rn(r, cmax)) : __fmul_rn(r, cmax);
    int cnt = 0;
    int pos = 0, pend = 0;
    if (MODE == SK_FILL) { pos = A.row_ptr[i]; pend = A.row_ptr[i + 1]; }
    if (q > 0.0f) {
      const bool full = q >= 1.0f;
      const float L = full ? 0.0f : spec_log1m(q);
      long long jprev = -1;
      for (uint32_t call0 = 0;; call0 += 32) {
        const uint4 w4 = skip_words4(pd.seed, pd.pid, (uint32_t)i, call0 + (uint32_t)lane);
        // gaps of the lane's two candidates; an invalid gap ends the row there
        bool ok0 = true, ok1 = true;
        long long st0 = 1, st1 = 1;
        if (!full) {
          const float r0 = __fdiv_rn(spec_log(__fmul_rn(__uint2float_rn((w4.x >> 8) + 1u), 5.9604644775390625e-08f)), L);
          const float r1 = __fdiv_rn(spec_log(__fmul_rn(__uint2float_rn((w4.z >> 8) + 1u), 5.9604644775390625e-08f)), L);
          ok0 = r0 < (float)m;
          ok1 = r1 < (float)m;
          st0 = ok0 ? 1 + (long long)floorf(r0) : 0;
          st1 = ok1 ? 1 + (long long)floorf(r1) : 0;
        }
        // first invalid candidate of the 64 (64: none)
        const unsigned bad = __ballot_sync(0xffffffffu, !ok0 || !ok1);
        int tstop = 64;
        if (bad) {
          const int fl = __ffs(bad) - 1;
          const bool b0 = __shfl_sync(0xffffffffu, !ok0, fl);
          tstop = 2 * fl + (b0 ? 0 : 1);
        }
        // positions: jprev + inclusive prefix of the steps in candidate order
        const long long tot = st0 + st1;
        long long inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        const long long j0 = jprev + (inc - tot) + st0;
        const long long j1 = j0 + st1;
        const bool in0 = 2 * lane < tstop && j0 < m;
        const bool in1 = 2 * lane + 1 < tstop && j1 < m;
        bool acc[2] = {false, false};
        float pv[2] = {0.0f, 0.0f}, Dv[2] = {0.0f, 0.0f};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const bool in = e == 0 ? in0 : in1;
          if (!in) continue;
          const int jj = (int)(e == 0 ? j0 : j1);
          float p;
          if (UOT) {
            Dv[e] = raw32(pd.cv, i, jj);
            p = __fmul_rn(scale, __fmul_rn(__fmul_rn(r, A.colf[jj]), uot_factor(wfr, Dv[e], kappa, inv2eta, g2)));
          } else {
            p = __fmul_rn(r, A.colf[jj]);
          }
          const float a_ = full ? p : __fdiv_rn(p, q);
          const uint32_t h = e == 0 ? w4.y : w4.w;
          acc[e] = __fmul_rn(__uint2float_rn(h >> 8), 5.9604644775390625e-08f) < a_;
          pv[e] = p;
        }
        const unsigned m0 = __ballot_sync(0xffffffffu, acc[0]), m1 = __ballot_sync(0xffffffffu, acc[1]);
        if (MODE == SK_COUNT) {
          cnt += __popc(m0) + __popc(m1);
#pragma unroll
          for (int e = 0; e < 2; ++e)
            if (acc[e]) atomicAdd(&A.col_cnt[(int)(e == 0 ? j0 : j1)], 1);
        } else {
          int wpos = pos + __popc(m0 & lt) + __popc(m1 & lt);
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            if (!acc[e]) continue;
            const int jj = (int)(e == 0 ? j0 : j1);
            if (wpos >= pend) {   // count and fill disagree: never write out of range
              A.ctrl->sketch_fault = 1;
              continue;
            }
            const float ps = pv[e] < 1.0f ? pv[e] : 1.0f;
            A.col_idx[wpos] = jj;
            if (lv32) {
              const float ce =
                  cost_over_eps_df(pd.cv.x32 + (int64_t)i * d, pd.cv.y32 + (int64_t)jj * d, d, k_hi, k_lo);
              A.logval[wpos] = __fsub_rn(-ce, logf(ps));
            } else {
              reinterpret_cast<V*>(A.val)[wpos] =
                  from_d<V>(ValMath<V>::value(pd, *A.sc, i, jj, UOT ? Dv[e] : raw32(pd.cv, i, jj), ps));
              if (A.logval) {
                const double C64 = value_cost64(pd, *A.sc, i, jj);
                A.logval[wpos] = (float)(-C64 / pd.eps - (double)logf(ps));
              }
            }
            const int slot = atomicAdd(&A.col_cur[jj], 1);
            if (slot < A.col_end[jj]) {
              A.tmp_row[slot] = i;
              A.tmp_src[slot] = wpos;
            } else {
              A.ctrl->sketch_fault = 1;
            }
            ++wpos;
          }
          pos += __popc(m0) + __popc(m1);
        }
        // the row ends at an invalid gap or once a position reaches m
        const long long jlast = __shfl_sync(0xffffffffu, j1, 31);
        if (tstop < 64 || jlast >= m) break;
        jprev = jlast;
      }
    }
    if (lane == 0) {
      if (MODE == SK_COUNT) A.cnt_row[i] = cnt;
      else if (pos != pend) A.ctrl->sketch_fault = 1;
    }
  }
}

static SweepArgs base_args(const ProbDev& pd, const Layout& L, char* ws) {
  SweepArgs A;
  memset(&A, 0, sizeof(A));
  A.pd = pd;
  A.sc = at<SketchScalars>(ws, L.scal);
  A.rowf = at<float>(ws, L.rowf);
  A.colf = at<float>(ws, L.colf);
  A.ctrl = at<Ctrl>(ws, L.ctrl);
  const SweepGeo g = sweep_geometry(pd.n, pd.m);
  A.chunk = g.chunk;
  A.nchunk = g.nchunk;
  A.cnt2 = at<int>(ws, L.cnt2);
  return A;
}

void launch_uot_Z(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st) {
  SweepArgs A = base_args(pd, L, ws);
  A.zsum = L.zsum ? at<float>(ws, L.zsum) : nullptr;
  const SweepGeo g = sweep_geometry(pd.n, pd.m);
  launch_sweep<SW_Z, true, float>(A, dim3(g.row_blocks, g.nchunk), st);
}

void launch_count(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st) {
  SweepArgs A = base_args(pd, L, ws);
  A.col_cnt = at<int>(ws, L.col_cnt);
  const SweepGeo g = sweep_geometry(pd.n, pd.m);
  const dim3 grid(g.row_blocks, g.nchunk);
  if (pd.sep) launch_sweep<SW_COUNT, false, float>(A, grid, st);
  else launch_sweep<SW_COUNT, true, float>(A, grid, st);
  k_sum_chunks<<<std::max(1, std::min(1216, (pd.n + 255) / 256)), 256, 0, st>>>(pd.n, g.nchunk, A.cnt2,
                                                                                 at<int>(ws, L.row_cnt), A.ctrl);
}

template <typename V>
static void fill_v(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st) {
  SweepArgs A = base_args(pd, L, ws);
  A.row_ptr = at<int>(ws, L.row_ptr);
  A.col_idx = at<int>(ws, L.col_idx);
  A.val = ws + L.val;
  A.col_cur = at<int>(ws, L.col_cur);
  A.col_end = at<int>(ws, L.col_ptr) + 1;
  A.logval = L.logval ? at<float>(ws, L.logval) : nullptr;
  A.tmp_row = at<int>(ws, L.tmp_row);
  A.tmp_src = at<int>(ws, L.tmp_src);
  const SweepGeo g = sweep_geometry(pd.n, pd.m);
  const dim3 grid(g.row_blocks, g.nchunk);
  if (pd.sep) launch_sweep<SW_FILL, false, V>(A, grid, st);
  else launch_sweep<SW_FILL, true, V>(A, grid, st);
}

void launch_fill(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st) {
  switch (kd) {
    case SPS_F64: fill_v<double>(pd, L, ws, st); break;
    case SPS_F32: fill_v<float>(pd, L, ws, st); break;
    case SPS_BF16: fill_v<__nv_bfloat16>(pd, L, ws, st); break;
    case SPS_F16: fill_v<__half>(pd, L, ws, st); break;
  }
}

template <typename V>
static void fused_v(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st) {
  SweepArgs A = base_args(pd, L, ws);
  const SweepGeo g = sweep_geometry(pd.n, pd.m);
  const long long len = (long long)pd.n * g.nchunk;
  int* caps = at<int>(ws, L.pad_ofs) + len + 1;   // scratch after the offsets
  if (pd.sep)
    k_chunk_csum<<<std::min(g.nchunk, 1024), 256, 0, st>>>(pd.m, g.chunk, g.nchunk, A.colf, at<float>(ws, L.csum));
  const int gc = (int)std::max<long long>(1, std::min<long long>(4096, (len + 255) / 256));
  k_pad_caps<<<gc, 256, 0, st>>>(pd.n, pd.m, g.chunk, g.nchunk, pd.sep ? 0 : 1, A.rowf, at<float>(ws, L.csum),
                                 L.zsum ? at<float>(ws, L.zsum) : nullptr, A.sc, caps);
  k_pad_scan<<<1, 1024, 0, st>>>(caps, at<int>(ws, L.pad_ofs), len, (long long)L.pad_cap, A.ctrl);
  A.col_cnt = at<int>(ws, L.col_cnt);
  A.pad_ofs = at<int>(ws, L.pad_ofs);
  A.pad_col = at<int>(ws, L.pad_col);
  A.pad_val = ws + L.pad_val;
  A.pad_lv = L.pad_lv ? at<float>(ws, L.pad_lv) : nullptr;
  const dim3 grid(g.row_blocks, g.nchunk);
  if (pd.sep) launch_sweep<SW_FUSED, false, V>(A, grid, st);
  else launch_sweep<SW_FUSED, true, V>(A, grid, st);
}

void launch_fused(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st) {
  switch (kd) {
    case SPS_F64: fused_v<double>(pd, L, ws, st); break;
    case SPS_F32: fused_v<float>(pd, L, ws, st); break;
    case SPS_BF16: fused_v<__nv_bfloat16>(pd, L, ws, st); break;
    case SPS_F16: fused_v<__half>(pd, L, ws, st); break;
  }
}

template <typename V>
static void compact_v(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st) {
  const SweepGeo g = sweep_geometry(pd.n, pd.m);
  const int gb = std::max(1, std::min(152 * 32, (pd.n * 32 + 255) / 256));
  // the same condition as the sweep's binary32 log K~ (then no plain values were written)
  const bool lv32 = L.pad_lv && !pd.cv.x64 && !pd.cv.C32 && !pd.cv.C64;
  k_compact<V><<<gb, 256, 0, st>>>(pd.n, g.nchunk, at<int>(ws, L.pad_ofs), at<int>(ws, L.cnt2), at<int>(ws, L.row_ptr),
                                   at<int>(ws, L.pad_col), lv32 ? nullptr : at<V>(ws, L.pad_val),
                                   L.pad_lv ? at<float>(ws, L.pad_lv) : nullptr, at<int>(ws, L.col_idx),
                                   at<V>(ws, L.val), L.logval ? at<float>(ws, L.logval) : nullptr,
                                   at<int>(ws, L.col_cur), at<int>(ws, L.col_ptr) + 1, at<int>(ws, L.tmp_row),
                                   at<int>(ws, L.tmp_src), at<Ctrl>(ws, L.ctrl));
}

void launch_sum_chunks(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st) {
  k_sum_chunks<<<std::max(1, std::min(1216, (pd.n + 255) / 256)), 256, 0, st>>>(
      pd.n, sweep_geometry(pd.n, pd.m).nchunk, at<int>(ws, L.cnt2), at<int>(ws, L.row_cnt), at<Ctrl>(ws, L.ctrl));
}

void launch_compact(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st) {
  switch (kd) {
    case SPS_F64: compact_v<double>(pd, L, ws, st); break;
    case SPS_F32: compact_v<float>(pd, L, ws, st); break;
    case SPS_BF16: compact_v<__nv_bfloat16>(pd, L, ws, st); break;
    case SPS_F16: compact_v<__half>(pd, L, ws, st); break;
  }
}

template <typename V>
static void skip_fill_v(const ProbDev& pd, const Layout& L, char* ws, int grid, cudaStream_t st) {
  SweepArgs A = base_args(pd, L, ws);
  A.row_ptr = at<int>(ws, L.row_ptr);
  A.col_idx = at<int>(ws, L.col_idx);
  A.val = ws + L.val;
  A.col_cur = at<int>(ws, L.col_cur);
  A.col_end = at<int>(ws, L.col_ptr) + 1;
  A.logval = L.logval ? at<float>(ws, L.logval) : nullptr;
  A.tmp_row = at<int>(ws, L.tmp_row);
  A.tmp_src = at<int>(ws, L.tmp_src);
  if (pd.sep) k_skip<SK_FILL, false, V><<<grid, 256, 0, st>>>(A);
  else k_skip<SK_FILL, true, V><<<grid, 256, 0, st>>>(A);
}

sps_status launch_skip_sample(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st) {
  SweepArgs A = base_args(pd, L, ws);
  A.col_cnt = at<int>(ws, L.col_cnt);
  A.cnt_row = at<int>(ws, L.row_cnt);
  const int grid = std::max(1, std::min(152 * 8, (pd.n + 7) / 8));   // one warp per row
  cudaMemsetAsync(A.col_cnt, 0, sizeof(int) * (size_t)pd.m, st);
  k_colf_max<<<std::max(1, std::min(1024, (pd.m + 255) / 256)), 256, 0, st>>>(A.colf, pd.m, A.sc);
  if (pd.sep) k_skip<SK_COUNT, false, float><<<grid, 256, 0, st>>>(A);
  else k_skip<SK_COUNT, true, float><<<grid, 256, 0, st>>>(A);
  launch_scan_counts(A.cnt_row, at<int>(ws, L.row_ptr), pd.n, A.col_cnt, at<int>(ws, L.col_ptr),
                     at<int>(ws, L.col_cur), pd.m, (long long)L.cap, A.ctrl, st);
  switch (kd) {
    case SPS_F64: skip_fill_v<double>(pd, L, ws, grid, st); break;
    case SPS_F32: skip_fill_v<float>(pd, L, ws, grid, st); break;
    case SPS_BF16: skip_fill_v<__nv_bfloat16>(pd, L, ws, grid, st); break;
    case SPS_F16: skip_fill_v<__half>(pd, L, ws, grid, st); break;
  }
  launch_csc_sort(pd, L, ws, kd, st);
  add_launches(5);
  return cuda_fail(cudaGetLastError(), "skip sample");
}

}  // namespace sps
