// sps_batch.cu -- Spar-Sink for a batch of problems over shared point sets.
//
// Pair p transports set src[p] to set dst[p].  Every pair is sketched exactly
// as a single problem (Eq. pois with Eq. pij-ot or Eq. pij-uot, the binary32
// decision rule, Philox problem id = base + p), into one block-diagonal CSR /
// CSC with pair-local indices.  The scaling iterations (Alg. 3 / Alg. 4 in
// the stabilised form: exact log-sum-exp first iteration, absorbed potentials,
// K' stored per row / column with a power-of-two scale) then run in ONE
// persistent launch: a block takes a pair from a queue (largest first),
// keeps u~ (two buffers) and v~ in shared memory, iterates with block-local
// barriers until the pair's own stopping rule holds, and forms the pair's
// objective terms before taking the next pair.  No block ever waits for
// another.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sps_internal.h"
#include "sps_iterdev.cuh"

namespace sps {
namespace batch {

using namespace iterdev;

struct PairDesc {
  int n, m;            // source / target sizes
  int src, dst;        // set indices
  long long xo, yo;    // first point of the source / target set
  long long ro, co;    // first global row / column of the pair
  double s;            // sample budget
  unsigned pid;        // Philox problem id
  int pad;
};

struct PairScal {
  float s32, scale32, kappa32, dn32;
  double dn64;
  unsigned dmax_bits;  // per-pair maximum of the binary32 distances (cost_norm = maxnorm)
  int pad;
  ExactAcc acc;        // UOT normaliser Z
};

struct PairOut {
  int status, iters, n_absorb, nnz;
  double residual, transport, neg_entropy, logp, mass, kl_a, kl_b, unreach_a, unreach_b;
};

struct SetScal {
  unsigned fmax_bits;  // maximum decision factor of the set (binary32 bits, values >= 0)
  int pad;
  ExactAcc sq;         // OT: exact sum of sqrt(mass)
};

struct BatchDev {
  int n_pairs, n_sets, d, uot;
  int cost_norm, kd;
  double cost_scale, eps, lam, tol;
  float gamma32, phi, inv_phi, inv_eps, eps32, inv_lam, tau;
  int max_iter;
  int skip;                       // sketch by the skip sampler (else one decision per element)
  uint64_t seed;
  long long R, M, P;              // total rows, columns, set points
  const PairDesc* pairs;
  const long long* ro_tab;        // n_pairs + 1 row offsets
  PairScal* ps;
  PairOut* out;
  SetScal* ss;
  const long long* set_off;       // n_sets + 1
  const float* x32;               // P x d
  const double* x64;              // FP64 points or null
  const float* w32;               // P masses
  float* fac;                     // P decision factors
  Ctrl* ctrl;
  unsigned* queue;                // work counters
  const int* order;               // pairs, largest first
  int* row_cnt; int* row_ptr; int* col_cnt; int* col_ptr; int* col_cur;
  int* col_idx; float* logval; int* row_idx; float* logvalT; int* csr_pos; int* tmp_row; int* tmp_src;
  void* val; void* valT;
  float *alpha, *beta, *ahat, *bhat, *erow, *ecol;
  const float *init_alpha, *init_beta;
  float *alpha_out, *beta_out;
};

constexpr int kBT = 256;          // threads of the sketch kernels
constexpr int kGrabRows = 16;     // rows a warp takes from the queue at a time
enum { Q_MAX = 0, Q_Z = 1, Q_COUNT = 2, Q_FILL = 3, Q_ITER = 4, Q_N = 8 };
enum { SW_MAX = 0, SW_Z = 1, SW_COUNT = 2, SW_FILL = 3 };

__device__ __forceinline__ float ninf() { return __int_as_float(0xff800000); }

__device__ __forceinline__ int pair_of_row(const BatchDev& B, long long r) {
  int lo = 0, hi = B.n_pairs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.ro_tab[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ----------------------------------------------------------------------------
// Set preparation: binary32 masses (and points for FP64 inputs), decision
// factors (OT: sqrt(mass); UOT: exp(gamma log mass) in the binary32 spec),
// per-set maxima and (OT) exact sums of sqrt(mass).
// ----------------------------------------------------------------------------
template <typename T>
__global__ void k_b_prepare(BatchDev B, const T* pts, const T* mass, float* x32w, float* w32w) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long st = (long long)gridDim.x * blockDim.x;
  for (long long k = tid; k < B.P; k += st) {
    const float w = (float)mass[k];
    w32w[k] = w;
    bool bad = !(w >= 0.0f) || isinf(w);
    for (int c = 0; c < B.d; ++c) {
      const float xc = (float)pts[k * B.d + c];
      if (x32w) x32w[k * B.d + c] = xc;
      bad |= !isfinite(xc);
    }
    if (bad) B.ctrl->status = SPS_ERR_NUMERIC;
  }
}

__global__ void k_b_set_factors(BatchDev B) {
  // one block per set
  const int sset = blockIdx.x;
  const long long lo = B.set_off[sset], hi = B.set_off[sset + 1];
  float mx = 0.0f;
  for (long long k = lo + threadIdx.x; k < hi; k += blockDim.x) {
    const float w = B.w32[k];
    float F;
    if (B.uot) {
      F = w > 0.0f ? spec_exp(__fmul_rn(B.gamma32, spec_log(w))) : 0.0f;
    } else {
      F = __fsqrt_rn(w);
      exact_slow_add(&B.ss[sset].sq, F);
    }
    B.fac[k] = F;
    mx = fmaxf(mx, F);
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) atomicMax(&B.ss[sset].fmax_bits, __float_as_uint(mx));
}

// Per-pair scalars.  stage 0: divisor, kappa, OT scale, Z window base;
// stage 1 (UOT): scale = fl32(s / Z).
__global__ void k_b_scalars(BatchDev B, int stage) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B.n_pairs) return;
  const PairDesc P = B.pairs[p];
  PairScal* S = B.ps + p;
  if (stage == 0) {
    S->s32 = __double2float_rn(P.s);
    double dn64 = 1.0;
    float dn32 = 1.0f;
    if (B.cost_norm == SPS_COST_MAXNORM) {
      const float dm = __uint_as_float(S->dmax_bits);
      if (dm > 0.0f) dn32 = dm;
      dn64 = (double)dn32;
    } else if (B.cost_norm == SPS_COST_SCALE) {
      dn64 = B.cost_scale;
      dn32 = __double2float_rn(B.cost_scale);
    }
    S->dn32 = dn32;
    S->dn64 = dn64;
    if (B.uot) {
      const double t = __dadd_rn(__dmul_rn(2.0, B.lam), B.eps);
      S->kappa32 = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(dn64, t)));
      const float fa = __uint_as_float(B.ss[P.src].fmax_bits), fb = __uint_as_float(B.ss[P.dst].fmax_bits);
      S->acc.B = exact_floor_for(fmaxf(__fmul_rn(fa, fb), 1e-30f));
    } else {
      const double sa = exact_round(&B.ss[P.src].sq), sb = exact_round(&B.ss[P.dst].sq);
      const double prod = __dmul_rn(sa, sb);
      if (!(prod > 0.0) || isinf(prod)) { S->scale32 = 0.0f; B.out[p].status = SPS_ERR_NUMERIC; }
      else S->scale32 = __double2float_rn(__ddiv_rn(1.0, prod));
    }
  } else {
    const double Z = exact_round(&S->acc);
    if (!(Z > 0.0) || isinf(Z)) { S->scale32 = 0.0f; B.out[p].status = SPS_ERR_NUMERIC; }
    else S->scale32 = __double2float_rn(__ddiv_rn(P.s, Z));
  }
}

// Binary32 spec distance (k ascending, no contraction) of source point xi to target point yj.
template <int DM>
__device__ __forceinline__ float spec_dist(const float (&xi)[DM], const float* yj, int d) {
  float acc = 0.0f;
#pragma unroll
  for (int k = 0; k < DM; ++k) {
    if (k < d) {
      const float t = __fsub_rn(xi[k], yj[k]);
      acc = __fmaf_rn(t, t, acc);
    }
  }
  return acc;
}

__device__ __forceinline__ double dist64(const BatchDev& B, long long xk, long long yk) {
  double acc = 0.0;
  for (int k = 0; k < B.d; ++k) {
    const double a = B.x64 ? B.x64[xk * B.d + k] : (double)B.x32[xk * B.d + k];
    const double b = B.x64 ? B.x64[yk * B.d + k] : (double)B.x32[yk * B.d + k];
    const double t = __dsub_rn(a, b);
    acc = __fma_rn(t, t, acc);
  }
  return acc;
}

// ----------------------------------------------------------------------------
// Sketch sweeps: a warp per row, all m_p columns of the row's pair, rows taken
// from a queue kGrabRows at a time.
//   SW_MAX   per-pair maximum of the binary32 distances
//   SW_Z     per-pair exact Z = sum_ij A_i B_j E(-D_ij kappa)        (UOT)
//   SW_COUNT per-row counts, per-column counts
//   SW_FILL  columns and log K~ at the CSR positions, CSC scatter
// ----------------------------------------------------------------------------
template <int MODE, bool UOT, int DM>
__global__ void __launch_bounds__(kBT) k_b_sweep(BatchDev B) {
  if (B.ctrl->status != SPS_OK) return;
  const int lane = threadIdx.x & 31;
  for (;;) {
    long long r0 = 0;
    if (lane == 0) r0 = (long long)atomicAdd(&B.queue[MODE == SW_MAX ? Q_MAX : MODE == SW_Z ? Q_Z : MODE == SW_COUNT ? Q_COUNT : Q_FILL], 1u) * kGrabRows;
    r0 = __shfl_sync(0xffffffffu, r0, 0);
    if (r0 >= B.R) break;
    const long long r1 = min(B.R, r0 + kGrabRows);
    int p = pair_of_row(B, r0);
    U128 zacc{0ull, 0ull};
    int zp = p;
    float dmax = 0.0f;
    for (long long r = r0; r < r1; ++r) {
      while (r >= B.ro_tab[p + 1]) ++p;
      if (MODE == SW_Z && p != zp) {
        exact_flush(zacc, &B.ps[zp].acc);
        zacc = U128{0ull, 0ull};
        zp = p;
      }
      if (MODE == SW_MAX && p != zp) {
        dmax = warp_max(dmax);
        if (lane == 0 && dmax > 0.0f) atomicMax(&B.ps[zp].dmax_bits, __float_as_uint(dmax));
        dmax = 0.0f;
        zp = p;
      }
      const PairDesc P = B.pairs[p];
      const int i = (int)(r - P.ro);
      if (B.out[p].status != SPS_OK) {   // the pair's scalars failed: no elements
        if (MODE == SW_COUNT && lane == 0) B.row_cnt[r] = 0;
        continue;
      }
      const long long xk = P.xo + i;
      float xi[DM];
#pragma unroll
      for (int k = 0; k < DM; ++k) xi[k] = k < B.d ? B.x32[xk * B.d + k] : 0.0f;
      const PairScal* S = B.ps + p;
      float ri = B.fac[xk];
      if (!UOT) ri = __fmul_rn(__fmul_rn(S->s32, ri), S->scale32);
      if (MODE != SW_MAX && !(ri > 0.0f)) {
        if (MODE == SW_COUNT && lane == 0) B.row_cnt[r] = 0;
        continue;
      }
      const float kappa = S->kappa32, scale = S->scale32;
      const int Bz = UOT ? S->acc.B : 0;
      float k_hi = 0.0f, k_lo = 0.0f;
      if (MODE == SW_FILL) {
        const double k64 = 1.0 / (S->dn64 * B.eps);
        k_hi = __double2float_rn(k64);
        k_lo = __double2float_rn(k64 - (double)k_hi);
      }
      int cnt = 0;
      int pos = MODE == SW_FILL ? B.row_ptr[r] : 0;
      const int pend = MODE == SW_FILL ? B.row_ptr[r + 1] : 0;
      for (int j0 = 0; j0 < P.m; j0 += 128) {
        const int j = j0 + 4 * lane;
        unsigned mask = 0u;
        float pe[4] = {0.f, 0.f, 0.f, 0.f};
        if (j < P.m) {
          uint4 dr = make_uint4(0u, 0u, 0u, 0u);
          if (MODE == SW_COUNT || MODE == SW_FILL) dr = draw4(B.seed, P.pid, (uint32_t)i, (uint32_t)(j >> 2));
          const uint32_t dd[4] = {dr.x, dr.y, dr.z, dr.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int jj = j + e;
            if (jj < P.m) {
              const long long yk = P.yo + jj;
              if (MODE == SW_MAX) {
                dmax = fmaxf(dmax, spec_dist<DM>(xi, B.x32 + yk * B.d, B.d));
                continue;
              }
              float pr;
              if (UOT) {
                const float D = spec_dist<DM>(xi, B.x32 + yk * B.d, B.d);
                const float w = __fmul_rn(__fmul_rn(ri, B.fac[yk]), spec_exp(-__fmul_rn(D, kappa)));
                if (MODE == SW_Z) { exact_add(zacc, &B.ps[p].acc, Bz, w); continue; }
                pr = __fmul_rn(scale, w);
              } else {
                pr = __fmul_rn(ri, B.fac[yk]);
              }
              pe[e] = pr;
              if (keep(dd[e], pr)) mask |= 1u << e;
            }
          }
        }
        if (MODE == SW_COUNT) {
          cnt += __popc(mask);
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (mask & (1u << e)) atomicAdd(&B.col_cnt[P.co + j + e], 1);
        } else if (MODE == SW_FILL) {
          if (__ballot_sync(0xffffffffu, mask != 0u) == 0u) continue;
          const int cnum = __popc(mask);
          const unsigned c0 = __ballot_sync(0xffffffffu, cnum & 1), c1 = __ballot_sync(0xffffffffu, cnum & 2),
                         c2 = __ballot_sync(0xffffffffu, cnum & 4);
          const unsigned lt = (1u << lane) - 1u;
          int q = pos + __popc(c0 & lt) + 2 * __popc(c1 & lt) + 4 * __popc(c2 & lt);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (mask & (1u << e)) {
              const int jj = j + e;
              if (q >= pend) { B.ctrl->sketch_fault = 1; ++q; continue; }
              const float ps = pe[e] < 1.0f ? pe[e] : 1.0f;
              B.col_idx[q] = jj;
              if (B.x64) {
                const double C = dist64(B, xk, P.yo + jj) / S->dn64;
                B.logval[q] = (float)(-C / B.eps - (double)logf(ps));
              } else {
                // binary32 double-float C/eps (the FP64 pipe is narrow on this GPU)
                B.logval[q] = __fsub_rn(-cost_over_eps_df(xi, B.x32 + (P.yo + jj) * B.d, B.d, k_hi, k_lo), logf(ps));
              }
              const int slot = atomicAdd(&B.col_cur[P.co + jj], 1);
              if (slot < B.col_ptr[P.co + jj + 1]) {
                B.tmp_row[slot] = i;
                B.tmp_src[slot] = q;
              } else {
                B.ctrl->sketch_fault = 1;
              }
              ++q;
            }
          }
          pos += __popc(c0) + 2 * __popc(c1) + 4 * __popc(c2);
        }
      }
      if (MODE == SW_COUNT) {
        cnt = warp_sum(cnt);
        if (lane == 0) B.row_cnt[r] = cnt;
      }
    }
    if (MODE == SW_Z) exact_flush(zacc, &B.ps[zp].acc);
    if (MODE == SW_MAX) {
      dmax = warp_max(dmax);
      if (lane == 0 && dmax > 0.0f) atomicMax(&B.ps[zp].dmax_bits, __float_as_uint(dmax));
    }
  }
}

// ----------------------------------------------------------------------------
// Skip sampler for the batch (sampler = SPS_SAMPLER_SKIP): per row the stream
// of the single-problem skip sampler (k_skip in sps_sweep.cu) with the pair's
// problem id, so every pair's sketch is the one a single solve with that id
// draws.  Row i of pair p bounds every p_ij by q_i: OT q_i = min(1,
// fl(r_i cmax)), UOT q_i = min(1, fl(scale fl(A_i cmax))), cmax the largest
// decision factor of the target set.  Candidates are a Bernoulli(q_i) process
// of geometric gaps G = floor(log U / log(1 - q_i)), U = ((w >> 8) + 1) 2^-24;
// candidate j is kept when V < fl(p_ij / q_i), V = (w' >> 8) 2^-24; candidate t
// of row i reads Philox at counter (t >> 1, i, pid, 0x5B1E).  A warp takes 64
// candidates at a time (lane l: candidates 2l and 2l + 1 of the round, one
// Philox call) and places them by a prefix sum of the steps 1 + G.
// ----------------------------------------------------------------------------
enum { BK_COUNT = 0, BK_FILL = 1 };

template <int MODE, bool UOT, int DM>
__global__ void __launch_bounds__(kBT) k_b_skip(BatchDev B) {
  if (B.ctrl->status != SPS_OK) return;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (;;) {
    long long r0 = 0;
    if (lane == 0) r0 = (long long)atomicAdd(&B.queue[MODE == BK_COUNT ? Q_COUNT : Q_FILL], 1u) * kGrabRows;
    r0 = __shfl_sync(0xffffffffu, r0, 0);
    if (r0 >= B.R) break;
    const long long r1 = min(B.R, r0 + kGrabRows);
    int p = pair_of_row(B, r0);
    for (long long r = r0; r < r1; ++r) {
      while (r >= B.ro_tab[p + 1]) ++p;
      const PairDesc P = B.pairs[p];
      const int i = (int)(r - P.ro);
      const int m = P.m;
      if (B.out[p].status != SPS_OK) {   // the pair's scalars failed: no elements
        if (MODE == BK_COUNT && lane == 0) B.row_cnt[r] = 0;
        continue;
      }
      const long long xk = P.xo + i;
      const PairScal* S = B.ps + p;
      float ri = B.fac[xk];
      if (!UOT) ri = __fmul_rn(__fmul_rn(S->s32, ri), S->scale32);
      const float cmax = __uint_as_float(B.ss[P.dst].fmax_bits);
      const float kappa = S->kappa32, scale = S->scale32;
      const float q = UOT ? __fmul_rn(scale, __fmul_rn(ri, cmax)) : __fmul_rn(ri, cmax);
      float xi[DM];
#pragma unroll
      for (int k = 0; k < DM; ++k) xi[k] = k < B.d ? B.x32[xk * B.d + k] : 0.0f;
      float k_hi = 0.0f, k_lo = 0.0f;
      if (MODE == BK_FILL) {
        const double k64 = 1.0 / (S->dn64 * B.eps);
        k_hi = __double2float_rn(k64);
        k_lo = __double2float_rn(k64 - (double)k_hi);
      }
      int cnt = 0;
      int pos = MODE == BK_FILL ? B.row_ptr[r] : 0;
      const int pend = MODE == BK_FILL ? B.row_ptr[r + 1] : 0;
      if (q > 0.0f) {
        const bool full = q >= 1.0f;
        const float L = full ? 0.0f : spec_log1m(q);
        long long jprev = -1;
        for (uint32_t call0 = 0;; call0 += 32) {
          const uint4 w4 = skip_words4(B.seed, P.pid, (uint32_t)i, call0 + (uint32_t)lane);
          // gaps of the lane's two candidates; an invalid gap ends the row there
          bool ok0 = true, ok1 = true;
          long long st0 = 1, st1 = 1;
          if (!full) {
            const float g0 = __fdiv_rn(spec_log(__fmul_rn(__uint2float_rn((w4.x >> 8) + 1u), 5.9604644775390625e-08f)), L);
            const float g1 = __fdiv_rn(spec_log(__fmul_rn(__uint2float_rn((w4.z >> 8) + 1u), 5.9604644775390625e-08f)), L);
            ok0 = g0 < (float)m;
            ok1 = g1 < (float)m;
            st0 = ok0 ? 1 + (long long)floorf(g0) : 0;
            st1 = ok1 ? 1 + (long long)floorf(g1) : 0;
          }
          const unsigned bad = __ballot_sync(0xffffffffu, !ok0 || !ok1);
          int tstop = 64;
          if (bad) {
            const int fl = __ffs(bad) - 1;
            const bool b0 = __shfl_sync(0xffffffffu, !ok0, fl);
            tstop = 2 * fl + (b0 ? 0 : 1);
          }
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
          bool keep_[2] = {false, false};
          float pv[2] = {0.0f, 0.0f};
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const bool in = e == 0 ? in0 : in1;
            if (!in) continue;
            const long long yk = P.yo + (e == 0 ? j0 : j1);
            float pr;
            if (UOT) {
              const float D = spec_dist<DM>(xi, B.x32 + yk * B.d, B.d);
              pr = __fmul_rn(scale, __fmul_rn(__fmul_rn(ri, B.fac[yk]), spec_exp(-__fmul_rn(D, kappa))));
            } else {
              pr = __fmul_rn(ri, B.fac[yk]);
            }
            const float a_ = full ? pr : __fdiv_rn(pr, q);
            const uint32_t h = e == 0 ? w4.y : w4.w;
            keep_[e] = __fmul_rn(__uint2float_rn(h >> 8), 5.9604644775390625e-08f) < a_;
            pv[e] = pr;
          }
          const unsigned m0 = __ballot_sync(0xffffffffu, keep_[0]), m1 = __ballot_sync(0xffffffffu, keep_[1]);
          if (MODE == BK_COUNT) {
            cnt += __popc(m0) + __popc(m1);
#pragma unroll
            for (int e = 0; e < 2; ++e)
              if (keep_[e]) atomicAdd(&B.col_cnt[P.co + (e == 0 ? j0 : j1)], 1);
          } else {
            int wpos = pos + __popc(m0 & lt) + __popc(m1 & lt);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              if (!keep_[e]) continue;
              const int jj = (int)(e == 0 ? j0 : j1);
              if (wpos >= pend) {   // count and fill disagree: never write out of range
                B.ctrl->sketch_fault = 1;
                continue;
              }
              const float ps = pv[e] < 1.0f ? pv[e] : 1.0f;
              B.col_idx[wpos] = jj;
              if (B.x64) {
                const double C = dist64(B, xk, P.yo + jj) / S->dn64;
                B.logval[wpos] = (float)(-C / B.eps - (double)logf(ps));
              } else {
                B.logval[wpos] =
                    __fsub_rn(-cost_over_eps_df(xi, B.x32 + (P.yo + jj) * B.d, B.d, k_hi, k_lo), logf(ps));
              }
              const int slot = atomicAdd(&B.col_cur[P.co + jj], 1);
              if (slot < B.col_ptr[P.co + jj + 1]) {
                B.tmp_row[slot] = i;
                B.tmp_src[slot] = wpos;
              } else {
                B.ctrl->sketch_fault = 1;
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
      if (MODE == BK_COUNT && lane == 0) B.row_cnt[r] = cnt;   // cnt is the same on every lane (ballot counts)
    }
  }
}

// ----------------------------------------------------------------------------
// Persistent per-pair iterations.
// ----------------------------------------------------------------------------
struct IterShape {
  int n_limit;      // pairs taken from the queue (autotuning runs a prefix)
  int max_iter;     // iteration cap of this launch
  double tol;       // < 0: never stop early (autotuning)
  int absorb;       // 0: no absorption (autotuning)
  int objective;    // 1: objective terms and potentials
  int nmax, mmax;   // shared-memory vector sizes
};

__device__ __forceinline__ float warp_lse_b(const int* idx, const float* logv, const float* pot, float inv_eps,
                                            int lo, int hi, int lane) {
  float mx = ninf();
  for (int k = lo + lane; k < hi; k += 32) {
    const float o = pot[idx[k]];
    if (o != ninf()) mx = fmaxf(mx, logv[k] + o * inv_eps);
  }
  mx = warp_max(mx);
  if (mx == ninf()) return mx;
  float s = 0.0f;
  for (int k = lo + lane; k < hi; k += 32) {
    const float o = pot[idx[k]];
    if (o != ninf()) s += expf(logv[k] + o * inv_eps - mx);
  }
  s = warp_sum(s);
  return mx + logf(s);
}

// K' of one row (or column) scaled by 2^-e with e = floor(log2 of its largest value).
template <typename V>
__device__ __forceinline__ void absorb_seg_b(int lo, int hi, const int* idx, const float* logv, float pi,
                                             const float* other, float inv_eps, V* out, float* e_out, int lane) {
  constexpr float kLog2e = 1.4426950408889634f;
  float mx = ninf();
  if (pi != ninf())
    for (int k = lo + lane; k < hi; k += 32) {
      const float o = other[idx[k]];
      if (o != ninf()) mx = fmaxf(mx, logv[k] + (pi + o) * inv_eps);
    }
  mx = warp_max(mx);
  const float e = mx == ninf() ? 0.0f : floorf(mx * kLog2e);
  for (int k = lo + lane; k < hi; k += 32) {
    const float o = other[idx[k]];
    float z = ninf();
    if (pi != ninf() && o != ninf()) z = logv[k] + (pi + o) * inv_eps;
    out[k] = from_d<V>((double)exp2f(z * kLog2e - e));
  }
  if (lane == 0) *e_out = e;
}

template <typename V>
__device__ void absorb_pair(const BatchDev& B, const PairDesc& P, const int* rp, const int* cp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float* al = B.alpha + P.ro;
  float* be = B.beta + P.co;
  for (int i = warp; i < P.n; i += nw)
    absorb_seg_b<V>(rp[i], rp[i + 1], B.col_idx, B.logval, al[i], be, B.inv_eps, (V*)B.val, B.erow + P.ro + i, lane);
  for (int j = warp; j < P.m; j += nw)
    absorb_seg_b<V>(cp[j], cp[j + 1], B.row_idx, B.logvalT, be[j], al, B.inv_eps, (V*)B.valT, B.ecol + P.co + j,
                    lane);
}

template <int NV>
__device__ __forceinline__ void block_sums_f(float (&v)[NV], float* sh) {
  block_sum_multi<NV, float>(v, sh);
  // thread 0 holds the totals; broadcast
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) sh[96 + k] = v[k];
  __syncthreads();
  for (int k = 0; k < NV; ++k) v[k] = sh[96 + k];
  __syncthreads();
}

__device__ __forceinline__ float block_max_f(float v, float* sh) {
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) sh[64 + (threadIdx.x >> 5)] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float x = threadIdx.x < (blockDim.x >> 5) ? sh[64 + threadIdx.x] : 0.0f;
    x = warp_max(x);
    if (threadIdx.x == 0) sh[100] = x;
  }
  __syncthreads();
  const float r = sh[100];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double kl_d(double x, double y) {
  if (x == 0.0) return y;
  if (y == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  return x * log(x / y) - x + y;
}

template <int LPR, typename V, bool UOT>
__device__ void solve_pair(const BatchDev& B, const IterShape& I, int p, float* sm, float* sh, double* shd) {
  const PairDesc P = B.pairs[p];
  PairOut* O = B.out + p;
  const int n = P.n, m = P.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int* rp = B.row_ptr + P.ro;
  const int* cp = B.col_ptr + P.co;
  const float* a = B.w32 + P.xo;
  const float* b = B.w32 + P.yo;
  float* al = B.alpha + P.ro;
  float* be = B.beta + P.co;
  float* ah = B.ahat + P.ro;
  float* bh = B.bhat + P.co;
  const float* er = B.erow + P.ro;
  const float* ec = B.ecol + P.co;
  float* U0 = sm;
  float* U1 = sm + I.nmax;
  float* Vs = sm + 2 * I.nmax;
  const float eps = B.eps32, inv_eps = B.inv_eps, phi = B.phi;
  if (O->status != SPS_OK) {   // a numeric failure in the sketch scalars: NaN potentials
    if (I.objective) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) B.alpha_out[P.ro + i] = __int_as_float(0x7fc00000);
      for (int j = threadIdx.x; j < m; j += blockDim.x) B.beta_out[P.co + j] = __int_as_float(0x7fc00000);
    }
    return;
  }

  // exact first iteration in the log domain: alpha from beta^0, then beta
  for (int j = threadIdx.x; j < m; j += blockDim.x) be[j] = B.init_beta ? B.init_beta[P.co + j] : 0.0f;
  __syncthreads();
  for (int i = warp; i < n; i += nw) {
    const float L = warp_lse_b(B.col_idx, B.logval, be, inv_eps, rp[i], rp[i + 1], lane);
    if (lane == 0) al[i] = (L == ninf() || !(a[i] > 0.0f)) ? ninf() : phi * eps * (logf(a[i]) - L);
  }
  __syncthreads();
  for (int j = warp; j < m; j += nw) {
    const float L = warp_lse_b(B.row_idx, B.logvalT, al, inv_eps, cp[j], cp[j + 1], lane);
    if (lane == 0) be[j] = (L == ninf() || !(b[j] > 0.0f)) ? ninf() : phi * eps * (logf(b[j]) - L);
  }
  __syncthreads();
  absorb_pair<V>(B, P, rp, cp);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float x = al[i];
    U1[i] = x == ninf() ? 0.0f : 1.0f;
    ah[i] = (UOT && x != ninf()) ? a[i] * expf(-x * B.inv_lam) : a[i];
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const float x = be[j];
    Vs[j] = x == ninf() ? 0.0f : 1.0f;
    bh[j] = (UOT && x != ninf()) ? b[j] * expf(-x * B.inv_lam) : b[j];
  }
  __syncthreads();

  constexpr int RPW = 32 / LPR;
  const int sl = lane & (LPR - 1);
  int t = 1, done = 0, status = SPS_NOT_CONVERGED, n_abs = 0;
  float res = 0.0f, unr = 0.0f, unb = 0.0f;
  for (;;) {
    float* uo = (t & 1) ? U1 : U0;
    float* un = (t & 1) ? U0 : U1;
    // row pass: residual of the pair t, u~ of the pair t+1
    float r_res = 0.0f, r_unr = 0.0f, r_ml = 0.0f;
    for (int base = warp * RPW; base < n; base += nw * RPW) {
      const int i = base + lane / LPR;
      const bool ok = i < n;
      const int lo = ok ? rp[i] : 0, hi = ok ? rp[i + 1] : 0;
      const float qs = seg_dot_smem<LPR, V>(B.col_idx, (const V*)B.val, Vs, 0, m, lo, hi, sl);
      if (ok && sl == 0) {
        const float q = qs * exp2f(er[i]);
        const float ahi = ah[i], ai = a[i];
        float u;
        if (q > 0.0f) {
          u = UOT ? powf(ahi / q, phi) : ahi / q;
          const float lhs = (UOT ? powf(uo[i], B.inv_phi) : uo[i]) * q;
          const float w = UOT ? (ahi > 0.0f ? ai / ahi : 1.0f) : 1.0f;
          r_res += w * fabsf(lhs - ahi);
          if (u > 0.0f) r_ml = fmaxf(r_ml, fabsf(logf(u)));
        } else {
          u = 0.0f;
          r_unr += ai;
        }
        un[i] = u;
      }
    }
    float s2[2] = {r_res, r_unr};
    block_sums_f<2>(s2, sh);
    res = s2[0];
    unr = s2[1];
    if (!isfinite(res)) { status = SPS_ERR_NUMERIC; done = 1; }
    else if (res <= I.tol) { status = SPS_OK; done = 1; }
    else if (t >= I.max_iter) { status = SPS_NOT_CONVERGED; done = 1; }
    if (done) break;
    const float mlu = block_max_f(r_ml, sh);
    // column pass: v~ of the pair t+1 (in place)
    float c_unb = 0.0f, c_ml = 0.0f;
    for (int base = warp * RPW; base < m; base += nw * RPW) {
      const int j = base + lane / LPR;
      const bool ok = j < m;
      const int lo = ok ? cp[j] : 0, hi = ok ? cp[j + 1] : 0;
      const float rs = seg_dot_smem<LPR, V>(B.row_idx, (const V*)B.valT, un, 0, n, lo, hi, sl);
      if (ok && sl == 0) {
        const float r = rs * exp2f(ec[j]);
        float v;
        if (r > 0.0f) {
          v = UOT ? powf(bh[j] / r, phi) : bh[j] / r;
          if (v > 0.0f) c_ml = fmaxf(c_ml, fabsf(logf(v)));
        } else {
          v = 0.0f;
          c_unb += b[j];
        }
        Vs[j] = v;
      }
    }
    float s1[1] = {c_unb};
    block_sums_f<1>(s1, sh);
    unb = s1[0];
    const float mlv = block_max_f(c_ml, sh);
    ++t;
    if (I.absorb && fmaxf(mlu, mlv) > B.tau) {
      // fold the scalings of the new pair into the potentials and rewrite K'
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float u = un[i];
        if (u > 0.0f) {
          const float x = al[i] + eps * logf(u);
          al[i] = x;
          un[i] = 1.0f;
          ah[i] = UOT ? a[i] * expf(-x * B.inv_lam) : a[i];
        }
      }
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const float v = Vs[j];
        if (v > 0.0f) {
          const float x = be[j] + eps * logf(v);
          be[j] = x;
          Vs[j] = 1.0f;
          bh[j] = UOT ? b[j] * expf(-x * B.inv_lam) : b[j];
        }
      }
      __syncthreads();
      absorb_pair<V>(B, P, rp, cp);
      __syncthreads();
      ++n_abs;
    }
  }
  if (!I.objective) return;

  // potentials of the returned pair (u~^t, v~^t): A = alpha + eps log u~, B = beta + eps log v~
  float* uo = (t & 1) ? U1 : U0;
  float* Apot = (t & 1) ? U0 : U1;   // the other buffer is free
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float x = uo[i] > 0.0f ? al[i] + eps * logf(uo[i]) : ninf();
    Apot[i] = x;
    B.alpha_out[P.ro + i] = x;
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const float x = Vs[j] > 0.0f ? be[j] + eps * logf(Vs[j]) : ninf();
    Vs[j] = x;
    B.beta_out[P.co + j] = x;
  }
  __syncthreads();
  // objective terms over the support (binary32 per row, FP64 totals)
  const PairScal* S = B.ps + p;
  double tr = 0.0, ne = 0.0, lp = 0.0, ms = 0.0, kla = 0.0, klb = 0.0;
  for (int i = warp; i < n; i += nw) {
    const float Ai = Apot[i];
    float rtr = 0.f, rne = 0.f, rlp = 0.f, rs = 0.f;
    const long long xk = P.xo + i;
    if (Ai != ninf()) {
      float ri = B.fac[xk];
      if (!UOT) ri = __fmul_rn(__fmul_rn(S->s32, ri), S->scale32);
      for (int k = rp[i] + lane; k < rp[i + 1]; k += 32) {
        const int j = B.col_idx[k];
        const float Bj = Vs[j];
        if (Bj == ninf()) continue;
        const float z = B.logval[k] + (Ai + Bj) * inv_eps;
        const float T = expf(z);
        if (!(T > 0.0f)) continue;
        const long long yk = P.yo + j;
        float D = 0.0f;
        for (int c = 0; c < B.d; ++c) {
          const float d0 = __fsub_rn(B.x32[xk * B.d + c], B.x32[yk * B.d + c]);
          D = __fmaf_rn(d0, d0, D);
        }
        float pr;
        if (UOT) pr = __fmul_rn(S->scale32, __fmul_rn(__fmul_rn(ri, B.fac[yk]), spec_exp(-__fmul_rn(D, S->kappa32))));
        else pr = __fmul_rn(ri, B.fac[yk]);
        const float psv = pr < 1.0f ? pr : 1.0f;
        rtr += T * __fdiv_rn(D, S->dn32);
        rne += T * (z - 1.0f);
        rlp += T * logf(psv);
        rs += T;
      }
    }
    rtr = warp_sum(rtr); rne = warp_sum(rne); rlp = warp_sum(rlp); rs = warp_sum(rs);
    if (lane == 0) {
      tr += rtr; ne += rne; lp += rlp; ms += rs;
      kla += kl_d((double)rs, (double)a[i]);
    }
  }
  for (int j = warp; j < m; j += nw) {
    const float Bj = Vs[j];
    float cs = 0.f;
    if (Bj != ninf())
      for (int k = cp[j] + lane; k < cp[j + 1]; k += 32) {
        const float Ai = Apot[B.row_idx[k]];
        if (Ai != ninf()) cs += expf(B.logvalT[k] + (Ai + Bj) * inv_eps);
      }
    cs = warp_sum(cs);
    if (lane == 0) klb += kl_d((double)cs, (double)b[j]);
  }
  const double vals[6] = {tr, ne, lp, ms, kla, klb};
  double tot[6];
  for (int k = 0; k < 6; ++k) {
    tot[k] = block_sum_d(vals[k], shd);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    O->status = status;
    O->iters = t;
    O->n_absorb = n_abs;
    O->nnz = rp[n] - rp[0];
    O->residual = res;
    O->unreach_a = unr;
    O->unreach_b = unb;
    O->transport = tot[0]; O->neg_entropy = tot[1]; O->logp = tot[2]; O->mass = tot[3];
    O->kl_a = tot[4]; O->kl_b = tot[5];
  }
  __syncthreads();
}

template <int LPR, typename V, bool UOT>
__global__ void __launch_bounds__(1024) k_b_iterate(BatchDev B, IterShape I) {
  extern __shared__ __align__(16) float bsm[];
  __shared__ float sh[128];
  __shared__ double shd[32];
  __shared__ int pair_sh;
  if (B.ctrl->status != SPS_OK || B.ctrl->sketch_fault || B.ctrl->nnz != B.ctrl->nnz_cols) return;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned q = atomicAdd(&B.queue[Q_ITER], 1u);
      pair_sh = q < (unsigned)I.n_limit ? B.order[q] : -1;
    }
    __syncthreads();
    const int p = pair_sh;
    if (p < 0) break;
    solve_pair<LPR, V, UOT>(B, I, p, bsm, sh, shd);
  }
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
struct Plan {
  size_t ctrl, queue, pairs, ro_tab, order, ps, out, ss, set_off, x32, w32, fac;
  size_t row_cnt, row_ptr, col_cnt, col_ptr, col_cur;
  size_t col_idx, logval, row_idx, logvalT, csr_pos, tmp_row, tmp_src, val, valT;
  size_t alpha, beta, ahat, bhat, erow, ecol;
  size_t total;
  long long R, M, P, cap;
  int nmax, mmax;
};

bool plan(const sps_batch* Bt, const sps_params* Q, Plan* L, std::vector<PairDesc>* descs) {
  memset(L, 0, sizeof(*L));
  const int np = Bt->n_pairs, ns = Bt->n_sets, d = Bt->d;
  const long long P = Bt->set_off[ns];
  long long R = 0, M = 0;
  double cap = 0.0;
  int nmax = 0, mmax = 0;
  if (descs) descs->resize(np);
  for (int p = 0; p < np; ++p) {
    const int sa = Bt->src[p], sb = Bt->dst[p];
    const int n = (int)(Bt->set_off[sa + 1] - Bt->set_off[sa]);
    const int m = (int)(Bt->set_off[sb + 1] - Bt->set_off[sb]);
    if (descs) {
      PairDesc& D = (*descs)[p];
      memset(&D, 0, sizeof(D));
      D.n = n; D.m = m; D.src = sa; D.dst = sb;
      D.xo = Bt->set_off[sa]; D.yo = Bt->set_off[sb];
      D.ro = R; D.co = M; D.s = Bt->s[p]; D.pid = Q->problem_id + (uint32_t)p;
    }
    R += n;
    M += m;
    const double nm = (double)n * (double)m;
    cap += std::min(nm, ceil(Bt->s[p] + 8.0 * sqrt(Bt->s[p]) + 64.0));
    nmax = std::max(nmax, n);
    mmax = std::max(mmax, m);
  }
  if (cap > 2147483000.0) return false;
  const size_t vb = dtype_bytes(Q->kdtype);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  L->ctrl = take(sizeof(Ctrl));
  L->queue = take(sizeof(unsigned) * Q_N);
  L->pairs = take(sizeof(PairDesc) * np);
  L->ro_tab = take(sizeof(long long) * (np + 1));
  L->order = take(sizeof(int) * np);
  L->ps = take(sizeof(PairScal) * np);
  L->out = take(sizeof(PairOut) * np);
  L->ss = take(sizeof(SetScal) * ns);
  L->set_off = take(sizeof(long long) * (ns + 1));
  L->x32 = Bt->dtype == SPS_F64 ? take(sizeof(float) * P * d) : 0;
  L->w32 = take(sizeof(float) * P);
  L->fac = take(sizeof(float) * P);
  L->row_cnt = take(4 * (size_t)R);
  L->row_ptr = take(4 * (size_t)(R + 1));
  L->col_cnt = take(4 * (size_t)M);
  L->col_ptr = take(4 * (size_t)(M + 1));
  L->col_cur = take(4 * (size_t)M);
  const size_t c = (size_t)cap;
  L->col_idx = take(4 * c);
  L->logval = take(4 * c);
  L->row_idx = take(4 * c);
  L->logvalT = take(4 * c);
  L->csr_pos = take(4 * c);
  L->tmp_row = take(4 * c);
  L->tmp_src = take(4 * c);
  L->val = take(vb * c);
  L->valT = take(vb * c);
  L->alpha = take(4 * (size_t)R);
  L->beta = take(4 * (size_t)M);
  L->ahat = take(4 * (size_t)R);
  L->bhat = take(4 * (size_t)M);
  L->erow = take(4 * (size_t)R);
  L->ecol = take(4 * (size_t)M);
  L->total = off + 256;
  L->R = R; L->M = M; L->P = P; L->cap = (long long)cap;
  L->nmax = nmax; L->mmax = mmax;
  return true;
}

sps_status validate_batch(const sps_batch* Bt, const sps_params* Q) {
  if (!Bt || !Q) { set_error("null batch or params"); return SPS_ERR_INVALID_ARG; }
  if (Bt->n_sets < 1 || Bt->n_pairs < 1) { set_error("empty batch"); return SPS_ERR_INVALID_ARG; }
  if (Q->sampler != SPS_SAMPLER_ELEMENT && Q->sampler != SPS_SAMPLER_SKIP) { set_error("unknown sampler %d", Q->sampler); return SPS_ERR_INVALID_ARG; }
  if (Q->probs != SPS_PROBS_PAPER) { set_error("the batched solver samples with Eq. (pij-ot) / Eq. (pij-uot) only (probs 0)"); return SPS_ERR_INVALID_ARG; }
  if (Bt->d < 1 || Bt->d > 16) { set_error("batch points need 1 <= d <= 16 (d=%d)", Bt->d); return SPS_ERR_INVALID_ARG; }
  if (!Bt->set_off || !Bt->pts || !Bt->mass || !Bt->src || !Bt->dst || !Bt->s) { set_error("null batch array"); return SPS_ERR_INVALID_ARG; }
  if (Bt->dtype != SPS_F32 && Bt->dtype != SPS_F64) { set_error("batch inputs are F32 or F64"); return SPS_ERR_INVALID_ARG; }
  if (Bt->cost_norm < SPS_COST_RAW || Bt->cost_norm > SPS_COST_SCALE) { set_error("unknown cost_norm"); return SPS_ERR_INVALID_ARG; }
  if (Bt->cost_norm == SPS_COST_SCALE && !(Bt->cost_scale > 0.0 && isfinite(Bt->cost_scale))) {
    set_error("cost_scale must be finite and > 0"); return SPS_ERR_INVALID_ARG;
  }
  if (Bt->set_off[0] != 0) { set_error("set_off[0] must be 0"); return SPS_ERR_INVALID_ARG; }
  for (int k = 0; k < Bt->n_sets; ++k)
    if (Bt->set_off[k + 1] <= Bt->set_off[k]) { set_error("set %d is empty or offsets decrease", k); return SPS_ERR_INVALID_ARG; }
  for (int p = 0; p < Bt->n_pairs; ++p) {
    const int a = Bt->src[p], b = Bt->dst[p];
    if (a < 0 || a >= Bt->n_sets || b < 0 || b >= Bt->n_sets) { set_error("pair %d names a set out of range", p); return SPS_ERR_INVALID_ARG; }
    if (!(Bt->s[p] > 0.0) || !isfinite(Bt->s[p])) { set_error("pair %d: budget must be > 0", p); return SPS_ERR_INVALID_ARG; }
    const long long n = Bt->set_off[a + 1] - Bt->set_off[a], m = Bt->set_off[b + 1] - Bt->set_off[b];
    if (2 * n + m > SPS_BATCH_MAX_SMEM_ENTRIES) {
      set_error("pair %d: 2 n + m = %lld exceeds %d (the scaling vectors live in shared memory)", p, 2 * n + m,
                SPS_BATCH_MAX_SMEM_ENTRIES);
      return SPS_ERR_INVALID_ARG;
    }
  }
  if (!(Q->eps > 0.0) || !isfinite(Q->eps)) { set_error("eps must be > 0"); return SPS_ERR_INVALID_ARG; }
  if (!(Q->lambda > 0.0)) { set_error("lambda must be > 0 (+inf for OT)"); return SPS_ERR_INVALID_ARG; }
  if (Q->max_iter < 1) { set_error("max_iter must be >= 1"); return SPS_ERR_INVALID_ARG; }
  if (!(Q->tol >= 0.0)) { set_error("tol must be >= 0"); return SPS_ERR_INVALID_ARG; }
  if (Q->kdtype != SPS_F32 && Q->kdtype != SPS_BF16 && Q->kdtype != SPS_F16) { set_error("batched K' is stored in F32, BF16 or F16"); return SPS_ERR_INVALID_ARG; }
  if (Q->stop_rule != SPS_STOP_RESIDUAL) { set_error("the batched solver stops on the residual rule"); return SPS_ERR_INVALID_ARG; }
  if (!(Q->absorb_tau >= 0.0 && isfinite(Q->absorb_tau))) {
    set_error("absorb_tau must be finite and >= 0 (0 = default)"); return SPS_ERR_INVALID_ARG;
  }
  Plan L;
  if (!plan(Bt, Q, &L, nullptr)) { set_error("the batch's total sample capacity exceeds 2^31 elements"); return SPS_ERR_CAPACITY; }
  return SPS_OK;
}

BatchDev make_dev(const sps_batch* Bt, const sps_params* Q, const Plan& L, char* ws) {
  BatchDev B;
  memset(&B, 0, sizeof(B));
  B.n_pairs = Bt->n_pairs; B.n_sets = Bt->n_sets; B.d = Bt->d;
  B.uot = isinf(Q->lambda) ? 0 : 1;
  B.cost_norm = Bt->cost_norm; B.kd = Q->kdtype; B.cost_scale = Bt->cost_scale;
  B.eps = Q->eps; B.lam = B.uot ? Q->lambda : 0.0; B.tol = Q->tol;
  const double phi = B.uot ? Q->lambda / (Q->lambda + Q->eps) : 1.0;
  B.phi = (float)phi; B.inv_phi = (float)(1.0 / phi);
  B.eps32 = (float)Q->eps; B.inv_eps = (float)(1.0 / Q->eps);
  B.inv_lam = B.uot ? (float)(1.0 / Q->lambda) : 0.0f;
  B.tau = (float)(Q->absorb_tau > 0.0 ? Q->absorb_tau : 12.0);
  if (B.uot) B.gamma32 = (float)(Q->lambda / (2.0 * Q->lambda + Q->eps));   // the same rounding as the device
  B.max_iter = Q->max_iter;
  B.seed = Q->seed;
  B.skip = Q->sampler == SPS_SAMPLER_SKIP ? 1 : 0;
  B.R = L.R; B.M = L.M; B.P = L.P;
  B.pairs = at<PairDesc>(ws, L.pairs);
  B.ro_tab = at<long long>(ws, L.ro_tab);
  B.ps = at<PairScal>(ws, L.ps);
  B.out = at<PairOut>(ws, L.out);
  B.ss = at<SetScal>(ws, L.ss);
  B.set_off = at<long long>(ws, L.set_off);
  B.x32 = Bt->dtype == SPS_F64 ? at<float>(ws, L.x32) : (const float*)Bt->pts;
  B.x64 = Bt->dtype == SPS_F64 ? (const double*)Bt->pts : nullptr;
  B.w32 = at<float>(ws, L.w32);
  B.fac = at<float>(ws, L.fac);
  B.ctrl = at<Ctrl>(ws, L.ctrl);
  B.queue = at<unsigned>(ws, L.queue);
  B.order = at<int>(ws, L.order);
  B.row_cnt = at<int>(ws, L.row_cnt); B.row_ptr = at<int>(ws, L.row_ptr);
  B.col_cnt = at<int>(ws, L.col_cnt); B.col_ptr = at<int>(ws, L.col_ptr); B.col_cur = at<int>(ws, L.col_cur);
  B.col_idx = at<int>(ws, L.col_idx); B.logval = at<float>(ws, L.logval);
  B.row_idx = at<int>(ws, L.row_idx); B.logvalT = at<float>(ws, L.logvalT);
  B.csr_pos = at<int>(ws, L.csr_pos); B.tmp_row = at<int>(ws, L.tmp_row); B.tmp_src = at<int>(ws, L.tmp_src);
  B.val = ws + L.val; B.valT = ws + L.valT;
  B.alpha = at<float>(ws, L.alpha); B.beta = at<float>(ws, L.beta);
  B.ahat = at<float>(ws, L.ahat); B.bhat = at<float>(ws, L.bhat);
  B.erow = at<float>(ws, L.erow); B.ecol = at<float>(ws, L.ecol);
  B.init_alpha = (const float*)Q->init_alpha;
  B.init_beta = (const float*)Q->init_beta;
  return B;
}

int sweep_grid() { return 152 * 16; }

template <int MODE, bool UOT>
void sweep(const BatchDev& B, cudaStream_t st) {
  const int g = sweep_grid();
  switch (B.d) {
    case 1: k_b_sweep<MODE, UOT, 1><<<g, kBT, 0, st>>>(B); break;
    case 2: k_b_sweep<MODE, UOT, 2><<<g, kBT, 0, st>>>(B); break;
    case 3: k_b_sweep<MODE, UOT, 3><<<g, kBT, 0, st>>>(B); break;
    default:
      if (B.d <= 4) k_b_sweep<MODE, UOT, 4><<<g, kBT, 0, st>>>(B);
      else if (B.d <= 8) k_b_sweep<MODE, UOT, 8><<<g, kBT, 0, st>>>(B);
      else k_b_sweep<MODE, UOT, 16><<<g, kBT, 0, st>>>(B);
  }
}

template <int MODE, bool UOT>
void skip(const BatchDev& B, cudaStream_t st) {
  const int g = sweep_grid();
  switch (B.d) {
    case 1: k_b_skip<MODE, UOT, 1><<<g, kBT, 0, st>>>(B); break;
    case 2: k_b_skip<MODE, UOT, 2><<<g, kBT, 0, st>>>(B); break;
    case 3: k_b_skip<MODE, UOT, 3><<<g, kBT, 0, st>>>(B); break;
    default:
      if (B.d <= 4) k_b_skip<MODE, UOT, 4><<<g, kBT, 0, st>>>(B);
      else if (B.d <= 8) k_b_skip<MODE, UOT, 8><<<g, kBT, 0, st>>>(B);
      else k_b_skip<MODE, UOT, 16><<<g, kBT, 0, st>>>(B);
  }
}

template <bool UOT>
void sweeps_t(const BatchDev& B, const Plan& L, cudaStream_t st) {
  if (B.cost_norm == SPS_COST_MAXNORM) sweep<SW_MAX, UOT>(B, st);
  k_b_scalars<<<(B.n_pairs + 127) / 128, 128, 0, st>>>(B, 0);
  if (UOT) {
    sweep<SW_Z, UOT>(B, st);
    k_b_scalars<<<(B.n_pairs + 127) / 128, 128, 0, st>>>(B, 1);
  }
  if (B.skip) skip<BK_COUNT, UOT>(B, st);
  else sweep<SW_COUNT, UOT>(B, st);
  launch_scan_counts(B.row_cnt, B.row_ptr, (int)B.R, B.col_cnt, B.col_ptr, B.col_cur, (int)B.M, L.cap, B.ctrl, st);
  if (B.skip) skip<BK_FILL, UOT>(B, st);
  else sweep<SW_FILL, UOT>(B, st);
  launch_csc_sort_f32((int)B.M, B.col_ptr, B.tmp_row, B.tmp_src, B.logval, B.row_idx, B.csr_pos, B.logvalT, B.ctrl,
                      st);
}

// The whole device work of a batched solve (capturable: no host transfers).
template <typename T>
void enqueue_sketch(const BatchDev& B, const Plan& L, char* ws, const void* pts, const void* mass, cudaStream_t st) {
  cudaMemsetAsync(ws + L.ctrl, 0, sizeof(Ctrl), st);
  cudaMemsetAsync(ws + L.queue, 0, sizeof(unsigned) * Q_N, st);
  cudaMemsetAsync(ws + L.ps, 0, sizeof(PairScal) * B.n_pairs, st);
  cudaMemsetAsync(ws + L.out, 0, sizeof(PairOut) * B.n_pairs, st);
  cudaMemsetAsync(ws + L.ss, 0, sizeof(SetScal) * B.n_sets, st);
  cudaMemsetAsync(ws + L.col_cnt, 0, 4 * (size_t)B.M, st);
  const int g = (int)std::min<long long>(4096, (B.P + 255) / 256);
  k_b_prepare<T><<<std::max(g, 1), 256, 0, st>>>(B, (const T*)pts, (const T*)mass,
                                                  L.x32 ? at<float>(ws, L.x32) : nullptr, at<float>(ws, L.w32));
  k_b_set_factors<<<B.n_sets, 256, 0, st>>>(B);
  if (B.uot) sweeps_t<true>(B, L, st);
  else sweeps_t<false>(B, L, st);
}

template <int LPR, typename V, bool UOT>
bool launch_iter_t(const BatchDev& B, const IterShape& I, int threads, cudaStream_t st) {
  auto fn = k_b_iterate<LPR, V, UOT>;
  const size_t smem = sizeof(float) * (size_t)(2 * I.nmax + I.mmax);
  if (cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess || per < 1) {
    cudaGetLastError();
    return false;
  }
  const int grid = std::min(nsm * per, std::max(1, I.n_limit));
  fn<<<grid, threads, smem, st>>>(B, I);
  return cudaGetLastError() == cudaSuccess;
}

template <typename V, bool UOT>
bool launch_iter_v(const BatchDev& B, const IterShape& I, int lpr, int threads, cudaStream_t st) {
  switch (lpr) {
    case 4: return launch_iter_t<4, V, UOT>(B, I, threads, st);
    case 8: return launch_iter_t<8, V, UOT>(B, I, threads, st);
    case 16: return launch_iter_t<16, V, UOT>(B, I, threads, st);
    default: return launch_iter_t<32, V, UOT>(B, I, threads, st);
  }
}

bool launch_iter(const BatchDev& B, const IterShape& I, int lpr, int threads, cudaStream_t st) {
  if (B.uot) {
    switch (B.kd) {
      case SPS_BF16: return launch_iter_v<__nv_bfloat16, true>(B, I, lpr, threads, st);
      case SPS_F16: return launch_iter_v<__half, true>(B, I, lpr, threads, st);
      default: return launch_iter_v<float, true>(B, I, lpr, threads, st);
    }
  }
  switch (B.kd) {
    case SPS_BF16: return launch_iter_v<__nv_bfloat16, false>(B, I, lpr, threads, st);
    case SPS_F16: return launch_iter_v<__half, false>(B, I, lpr, threads, st);
    default: return launch_iter_v<float, false>(B, I, lpr, threads, st);
  }
}

// Autotuner cache: batch shape -> (lanes per row, block threads).
struct TuneKey {
  int n_pairs, kd, uot;
  long long R, nnz_bucket;
  bool operator<(const TuneKey& o) const {
    if (n_pairs != o.n_pairs) return n_pairs < o.n_pairs;
    if (kd != o.kd) return kd < o.kd;
    if (uot != o.uot) return uot < o.uot;
    if (R != o.R) return R < o.R;
    return nnz_bucket < o.nnz_bucket;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;

struct GraphEntry {
  cudaGraphExec_t exec;
  int lpr, threads;
};
std::mutex g_graph_mu;
std::map<std::string, GraphEntry> g_graphs;

}  // namespace batch

using namespace batch;

static sps_status batch_fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }

}  // namespace sps

using namespace sps;
using namespace sps::batch;

extern "C" {

size_t sps_batch_workspace_bytes(const sps_batch* batch, const sps_params* prm) {
  if (validate_batch(batch, prm) != SPS_OK) return 0;
  Plan L;
  if (!plan(batch, prm, &L, nullptr)) return 0;
  return L.total;
}

sps_status spar_sink_batched(const sps_batch* Bt, const sps_params* Q, sps_batch_opts* opts, void* wsv,
                             size_t ws_bytes, void* alpha_out, void* beta_out, sps_result* res, sps_stream stream) {
  SPS_TRY(validate_batch(Bt, Q));
  if (!wsv || !alpha_out || !beta_out) { set_error("null workspace or output"); return SPS_ERR_INVALID_ARG; }
  sps_batch_opts dflt;
  memset(&dflt, 0, sizeof(dflt));
  sps_batch_opts* O = opts ? opts : &dflt;
  if (O->lanes_per_row != 0 && O->lanes_per_row != 4 && O->lanes_per_row != 8 && O->lanes_per_row != 16 &&
      O->lanes_per_row != 32) { set_error("lanes_per_row must be 0, 4, 8, 16 or 32"); return SPS_ERR_INVALID_ARG; }
  if (O->block_threads != 0 && O->block_threads != 256 && O->block_threads != 512 && O->block_threads != 1024) {
    set_error("block_threads must be 0, 256, 512 or 1024");
    return SPS_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (O->use_graph && st == nullptr) { set_error("use_graph needs a stream other than the legacy default stream"); return SPS_ERR_INVALID_ARG; }
  Plan L;
  std::vector<PairDesc> descs;
  if (!plan(Bt, Q, &L, &descs)) { set_error("capacity"); return SPS_ERR_CAPACITY; }
  if (ws_bytes < L.total) { set_error("workspace too small: %zu < %zu", ws_bytes, L.total); return SPS_ERR_WORKSPACE; }
  char* ws = (char*)(((uintptr_t)wsv + 255) & ~(uintptr_t)255);
  const int np = Bt->n_pairs;
  // host tables: descriptors, row offsets, schedule (largest budget first), set offsets
  std::vector<long long> ro(np + 1);
  for (int p = 0; p < np; ++p) ro[p] = descs[p].ro;
  ro[np] = L.R;
  std::vector<int> order(np);
  for (int p = 0; p < np; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return Bt->s[x] > Bt->s[y]; });
  SPS_TRY(batch_fail(cudaMemcpyAsync(ws + L.pairs, descs.data(), sizeof(PairDesc) * np, cudaMemcpyHostToDevice, st), "descriptors"));
  SPS_TRY(batch_fail(cudaMemcpyAsync(ws + L.ro_tab, ro.data(), sizeof(long long) * (np + 1), cudaMemcpyHostToDevice, st), "row offsets"));
  SPS_TRY(batch_fail(cudaMemcpyAsync(ws + L.order, order.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st), "schedule"));
  SPS_TRY(batch_fail(cudaMemcpyAsync(ws + L.set_off, Bt->set_off, sizeof(long long) * (Bt->n_sets + 1), cudaMemcpyHostToDevice, st), "set offsets"));
  SPS_TRY(batch_fail(cudaStreamSynchronize(st), "table upload"));

  BatchDev B = make_dev(Bt, Q, L, ws);
  B.alpha_out = (float*)alpha_out;
  B.beta_out = (float*)beta_out;
  IterShape I;
  I.n_limit = np; I.max_iter = Q->max_iter; I.tol = Q->tol; I.absorb = 1; I.objective = 1;
  I.nmax = L.nmax; I.mmax = L.mmax;

  cudaEvent_t ev[4];
  for (auto& e : ev) cudaEventCreate(&e);
  auto cleanup = [&]() { for (auto& e : ev) cudaEventDestroy(e); };
  auto enqueue_sk = [&]() {
    if (Bt->dtype == SPS_F64) enqueue_sketch<double>(B, L, ws, Bt->pts, Bt->mass, st);
    else enqueue_sketch<float>(B, L, ws, Bt->pts, Bt->mass, st);
  };

  // launch shape: given, cached, or tuned now on this batch
  int lpr = O->lanes_per_row, thr = O->block_threads;
  O->tune_ms = 0.0f;
  std::string gkey;
  GraphEntry* cached = nullptr;
  if (O->use_graph) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%p|%p|%p|%p|%p|%d|%lld|%lld|%lld|%lld|%d|%d|%d|%d|%.17g|%.17g|%.17g|%.17g|%d|%llu|%u|%d|%g|%d|%d|%d",
             wsv, alpha_out, beta_out, Bt->pts, Bt->mass, np, L.R, L.M, L.P, L.cap, L.nmax, L.mmax, Q->kdtype,
             Bt->cost_norm, Bt->cost_scale, Q->eps, Q->lambda, Q->tol, Q->max_iter, (unsigned long long)Q->seed,
             Q->problem_id, Bt->d, Q->absorb_tau, O->lanes_per_row, O->block_threads, Q->sampler);
    gkey = buf;
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto it = g_graphs.find(gkey);
    if (it != g_graphs.end()) cached = &it->second;
  }
  if (cached) {
    lpr = cached->lpr;
    thr = cached->threads;
  } else if (lpr == 0 || thr == 0) {
    TuneKey key{np, Q->kdtype, B.uot, L.R, 0};
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) { if (!lpr) lpr = it->second.first; if (!thr) thr = it->second.second; }
    }
    if (lpr == 0 || thr == 0) {
      // time each candidate for a few iterations on a prefix of the schedule
      cudaEventRecord(ev[0], st);
      enqueue_sk();
      SPS_TRY(batch_fail(cudaStreamSynchronize(st), "autotune sketch"));
      IterShape T = I;
      int dev = 0, nsm = 152;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      T.n_limit = std::min(np, 2 * nsm);
      T.max_iter = 6; T.tol = -1.0; T.absorb = 0; T.objective = 0;
      const int lprs[4] = {4, 8, 16, 32}, thrs[3] = {256, 512, 1024};
      float best = 1e30f;
      int bl = 8, bt = 512;
      for (int li = 0; li < 4; ++li) {
        if (O->lanes_per_row && lprs[li] != O->lanes_per_row) continue;
        for (int ti = 0; ti < 3; ++ti) {
          if (O->block_threads && thrs[ti] != O->block_threads) continue;
          float ms = 0.0f;
          bool ok = true;
          for (int rep = 0; rep < 2 && ok; ++rep) {
            cudaMemsetAsync(ws + L.queue + sizeof(unsigned) * Q_ITER, 0, sizeof(unsigned), st);
            cudaEventRecord(ev[1], st);
            ok = launch_iter(B, T, lprs[li], thrs[ti], st);
            cudaEventRecord(ev[2], st);
            if (cudaEventSynchronize(ev[2]) != cudaSuccess) ok = false;
            if (ok) cudaEventElapsedTime(&ms, ev[1], ev[2]);
          }
          if (ok && ms < best) { best = ms; bl = lprs[li]; bt = thrs[ti]; }
        }
      }
      cudaEventRecord(ev[3], st);
      cudaEventSynchronize(ev[3]);
      cudaEventElapsedTime(&O->tune_ms, ev[0], ev[3]);
      lpr = bl;
      thr = bt;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = {lpr, thr};
    }
  }
  O->chosen_lanes = lpr;
  O->chosen_threads = thr;

  auto enqueue_all = [&](bool timed) -> bool {
    if (timed) cudaEventRecord(ev[0], st);
    enqueue_sk();
    if (timed) cudaEventRecord(ev[1], st);
    cudaMemsetAsync(ws + L.queue + sizeof(unsigned) * Q_ITER, 0, sizeof(unsigned), st);
    const bool ok = launch_iter(B, I, lpr, thr, st);
    if (timed) cudaEventRecord(ev[2], st);
    return ok;
  };
  bool ok = true;
  bool timed = true;
  if (O->use_graph) {
    timed = false;
    if (!cached) {
      cudaGraph_t g;
      SPS_TRY(batch_fail(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture"));
      ok = enqueue_all(false);
      cudaError_t e = cudaStreamEndCapture(st, &g);
      if (!ok || e != cudaSuccess) { cleanup(); set_error("capturing the batched solve failed"); return SPS_ERR_CUDA; }
      cudaGraphExec_t exec;
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "graph instantiate"); }
      std::lock_guard<std::mutex> lk(g_graph_mu);
      g_graphs[gkey] = GraphEntry{exec, lpr, thr};
      cached = &g_graphs[gkey];
    }
    cudaEventRecord(ev[0], st);
    SPS_TRY(batch_fail(cudaGraphLaunch(cached->exec, st), "graph launch"));
    cudaEventRecord(ev[2], st);
  } else {
    ok = enqueue_all(true);
  }
  if (!ok) { cleanup(); set_error("the batched iteration kernel could not be launched"); return SPS_ERR_CUDA; }
  std::vector<PairOut> outs(np);
  Ctrl h;
  SPS_TRY(batch_fail(cudaMemcpyAsync(outs.data(), ws + L.out, sizeof(PairOut) * np, cudaMemcpyDeviceToHost, st), "results"));
  SPS_TRY(batch_fail(cudaMemcpyAsync(&h, ws + L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "control"));
  SPS_TRY(batch_fail(cudaStreamSynchronize(st), "stream synchronize"));
  float ms_sk = 0.f, ms_it = 0.f;
  if (timed) {
    cudaEventElapsedTime(&ms_sk, ev[0], ev[1]);
    cudaEventElapsedTime(&ms_it, ev[1], ev[2]);
  } else {
    cudaEventElapsedTime(&ms_it, ev[0], ev[2]);
  }
  cleanup();
  if (h.status != SPS_OK) { set_error("batched sketch failed (status %d)", h.status); return (sps_status)h.status; }
  if (h.sketch_fault || h.nnz != h.nnz_cols) { set_error("batched sketch: count / fill mismatch"); return SPS_ERR_CUDA; }
  sps_status total = SPS_OK;
  for (int p = 0; p < np; ++p) {
    const PairOut& o = outs[p];
    if (res) {
      sps_result& r = res[p];
      memset(&r, 0, sizeof(r));
      r.status = o.status;
      r.iters = o.iters;
      r.residual = o.residual;
      r.transport = o.transport; r.neg_entropy = o.neg_entropy; r.logp = o.logp; r.mass = o.mass;
      r.kl_a = o.kl_a; r.kl_b = o.kl_b;
      r.obj = o.transport + Q->eps * o.neg_entropy;
      if (!isinf(Q->lambda)) r.obj += Q->lambda * (o.kl_a + o.kl_b);
      r.obj_sparse = r.obj + Q->eps * o.logp;
      r.unreach_a = o.unreach_a; r.unreach_b = o.unreach_b;
      r.nnz = o.nnz; r.n_absorb = o.n_absorb;
      r.ms_sketch = ms_sk; r.ms_iter = ms_it; r.ms_obj = 0.0f;
      r.launches = 0;
      r.iters_enqueued = o.iters;
    }
    if (o.status == SPS_ERR_NUMERIC) total = SPS_ERR_NUMERIC;
    else if (o.status != SPS_OK && total == SPS_OK) total = SPS_NOT_CONVERGED;
  }
  if (total == SPS_ERR_NUMERIC) set_error("non-finite value in a pair's iterates or scalars");
  return total;
}

}  // extern "C"
