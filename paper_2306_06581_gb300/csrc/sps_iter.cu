// sps_iter.cu -- Sinkhorn scaling iterations on the sketch (Alg. 1 / Alg. 2
// run on K~, as Alg. 3 / Alg. 4 prescribe) and the objective of their
// output line.
//
// Iteration t -> t+1 has two phases:
//   row phase  q = K~ v^t (CSR), u^{t+1} = (a / q)^phi, and
//              -- fused, at no extra pass -- the stopping residual of the pair
//              (u^t, v^t):
//                  rho_t = sum over reachable i of | (u^t_i)^{1/phi} q_i - a_i |
//              (the column side of that pair is zero up to rounding because
//              v^t was computed from u^t);
//   col phase  r = K~^T u^{t+1} (CSC), v^{t+1} = (b / r)^phi.
// u and v are double-buffered by the parity of t, so the pair (u^t, v^t)
// survives the phase that follows it and the convergence decision may lag
// half an iteration.  Rows (columns) whose product is zero get u_i = 0
// (v_j = 0): they carry mass no plan on the sketch can move, are left out of
// the residual, and their mass is reported.
//
// Three executions of the same phases:
//   - k_iterate_units: a persistent cooperative kernel over fixed nnz-balanced
//     work units (element rings filled by bulk copies, the gathered vector
//     staged in shared memory, a counting grid barrier; warp 0 of block 0
//     reduces the block partials in a fixed order and decides) -- the path a
//     solve takes;
//   - k_iterate: a persistent cooperative kernel with LPR lanes per row, two
//     grid barriers per iteration (bounded spin waits), block 0 deciding --
//     used when the unit kernel's launch is refused;
//   - one kernel per phase (the last block to finish reduces the partials),
//     used for the final residual and when no cooperative launch is possible.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "sps_internal.h"
#include "sps_iterdev.cuh"

namespace sps {

namespace {

using namespace iterdev;

constexpr int kThreads = 256;        // objective and set-up kernels
constexpr int kWarps = kThreads / 32;

struct IterArgs {
  int n, m;
  const int *row_ptr, *col_idx, *col_ptr, *row_idx;
  const void *val, *valT;
  void* ubuf;          // u buffers (2 x n), parity of t
  void* vbuf;          // v buffers (2 x m), parity of t
  const void* a;       // iterate type
  const void* b;
  double phi, inv_phi, tol;
  int stop_rule;
  Ctrl* ctrl;
  double* part;        // kPartSlots x nblk
  int nblk;
  const int *unit_r, *unit_c;   // work units of the persistent kernel (null: none)
  int ring;                     // ring elements per slot of the unit kernel
};

// Row phase of iteration t -> t+1 for the rows of this block; returns the
// block sums (thread 0) of residual, unreachable a-mass and |u^{t+1} - u^t|.
template <int LPR, typename V, typename T, bool UOT>
__device__ __forceinline__ void row_phase(const IterArgs& A, int t, double (&out)[3], T* sh) {
  const T* v = (const T*)A.vbuf + (size_t)(t & 1) * A.m;
  const T* uold = (const T*)A.ubuf + (size_t)(t & 1) * A.n;
  T* unew = (T*)A.ubuf + (size_t)((t + 1) & 1) * A.n;
  const T* a = (const T*)A.a;
  const V* val = (const V*)A.val;
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31, sl = lane & (LPR - 1);
  const T phi = (T)A.phi, inv_phi = (T)A.inv_phi;
  T res = 0, unr = 0, dl = 0;
  const int nw = blockDim.x >> 5;
  const int wg = blockIdx.x * nw + (threadIdx.x >> 5);
  for (int base = wg * RPW; base < A.n; base += gridDim.x * nw * RPW) {
    const int i = base + lane / LPR;
    const bool ok = i < A.n;
    const int lo = ok ? __ldg(A.row_ptr + i) : 0, hi = ok ? __ldg(A.row_ptr + i + 1) : 0;
    T ai = 0, uo = 0;
    if (ok && sl == 0) { ai = a[i]; uo = uold[i]; }  // issued before the dot product
    const T q = seg_row_dot<LPR, V, T>(A.col_idx, val, v, lo, hi, sl);
    if (ok && sl == 0) {
      T un;
      if (q > (T)0) {
        un = UOT ? powT<T>(ai / q, phi) : ai / q;
        const T lhs = (UOT ? powT<T>(uo, inv_phi) : uo) * q;
        res += fabs(lhs - ai);
      } else {
        un = (T)0;
        unr += ai;
      }
      dl += fabs(un - uo);
      unew[i] = un;
    }
  }
  T o[3] = {res, unr, dl};
  block_sum_multi<3, T>(o, sh);
  out[0] = (double)o[0]; out[1] = (double)o[1]; out[2] = (double)o[2];
}

// Column phase: v^{t+1} from u^{t+1}; block sums of unreachable b-mass and |v^{t+1} - v^t|.
template <int LPR, typename V, typename T, bool UOT>
__device__ __forceinline__ void col_phase(const IterArgs& A, int t, double (&out)[2], T* sh) {
  const T* u = (const T*)A.ubuf + (size_t)((t + 1) & 1) * A.n;
  const T* vold = (const T*)A.vbuf + (size_t)(t & 1) * A.m;
  T* vnew = (T*)A.vbuf + (size_t)((t + 1) & 1) * A.m;
  const T* b = (const T*)A.b;
  const V* val = (const V*)A.valT;
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31, sl = lane & (LPR - 1);
  const T phi = (T)A.phi;
  T unb = 0, dl = 0;
  const int nw = blockDim.x >> 5;
  const int wg = blockIdx.x * nw + (threadIdx.x >> 5);
  for (int base = wg * RPW; base < A.m; base += gridDim.x * nw * RPW) {
    const int j = base + lane / LPR;
    const bool ok = j < A.m;
    const int lo = ok ? __ldg(A.col_ptr + j) : 0, hi = ok ? __ldg(A.col_ptr + j + 1) : 0;
    T bj = 0, vo = 0;
    if (ok && sl == 0) { bj = b[j]; vo = vold[j]; }
    const T r = seg_row_dot<LPR, V, T>(A.row_idx, val, u, lo, hi, sl);
    if (ok && sl == 0) {
      T vn;
      if (r > (T)0) {
        vn = UOT ? powT<T>(bj / r, phi) : bj / r;
      } else {
        vn = (T)0;
        unb += bj;
      }
      dl += fabs(vn - vo);
      vnew[j] = vn;
    }
  }
  T o[2] = {unb, dl};
  block_sum_multi<2, T>(o, sh);
  out[0] = (double)o[0]; out[1] = (double)o[1];
}

// Decision state of the solve.  The persistent kernel keeps it in block 0's
// shared memory across iterations (only written to the control block); the
// per-phase kernels load it from the control block.
struct DecState {
  int done;
  double delta_u, delta_v;
};

// Decisions taken by one thread from the reduced partials.  Only the row
// phase of iteration t -> t+1 stops a solve, and always on the pair
// (u^t, v^t), whose buffers that iteration does not overwrite:
//   residual rule:  rho_t (this row phase) <= tol;
//   paper's rule:   ||u^t - u^{t-1}||_1 (row phase of iteration t, stored) +
//                   ||v^t - v^{t-1}||_1 (column phase of iteration t, stored) <= tol.
__device__ __forceinline__ void decide_row(Ctrl* ctrl, DecState& S, const IterArgs& A, int t, const double* tot) {
  ctrl->last_residual = tot[0];
  ctrl->last_unreach_a = tot[1];
  if (!S.done) {
    int stop = 0, numeric = 0;
    double r = tot[0];
    if (A.stop_rule == SPS_STOP_RESIDUAL) {
      numeric = !isfinite(r);
      stop = numeric || (t >= 1 && r <= A.tol);
    } else if (t >= 1) {
      r = S.delta_u + S.delta_v;
      numeric = !isfinite(r);
      stop = numeric || r <= A.tol;
    }
    if (stop) {
      S.done = 1;
      ctrl->iters = t;
      ctrl->residual = r;
      ctrl->unreach_a = tot[1];
      if (numeric) ctrl->status = SPS_ERR_NUMERIC;
      __threadfence();
      ctrl->done = 1;
    }
  }
  S.delta_u = tot[2];   // ||u^{t+1} - u^t||_1, judged with the next column phase
  ctrl->delta_u = tot[2];
}

__device__ __forceinline__ void decide_col(Ctrl* ctrl, DecState& S, int t, const double* tot) {
  ctrl->unreach_b = tot[0];
  S.delta_v = tot[1];
  ctrl->delta_v = tot[1];
  ctrl->t = t + 1;
}

__device__ __forceinline__ DecState load_state(const Ctrl* ctrl) {
  DecState S;
  S.done = ctrl->done;
  S.delta_u = ctrl->delta_u;
  S.delta_v = ctrl->delta_v;
  return S;
}

// Thread 0 publishes the block's partials, fences, and counts the block in;
// the block that arrives last sees every partial.
__device__ __forceinline__ bool publish_and_check_last(unsigned int* counter, double* part, int nblk,
                                                       const double* vals, int nvals, int slot0) {
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    for (int k = 0; k < nvals; ++k) part[(size_t)(slot0 + k) * nblk + blockIdx.x] = vals[k];
    __threadfence();
    am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  return am_last;
}

template <int LR, int LC, typename V, typename T, bool UOT>
__global__ void __launch_bounds__(kIterThreads) k_iterate(IterArgs A, int iters) {
  __shared__ T sh[3 * 32];
  __shared__ double tot[3];
  __shared__ DecState S;   // block 0's decision state
  Ctrl* ctrl = A.ctrl;
  if (ctrl->done) return;
  int t = ctrl->t;
  if (blockIdx.x == 0 && threadIdx.x == 0) S = load_state(ctrl);
  for (int k = 0; k < iters; ++k) {
    double r3[3];
    row_phase<LR, V, T, UOT>(A, t, r3, sh);
    if (threadIdx.x == 0) {
      A.part[0 * (size_t)A.nblk + blockIdx.x] = r3[0];
      A.part[1 * (size_t)A.nblk + blockIdx.x] = r3[1];
      A.part[2 * (size_t)A.nblk + blockIdx.x] = r3[2];
    }
    if (!grid_barrier(ctrl)) return;
    if (blockIdx.x == 0) {
      reduce_parts<3, T>(A.part, A.nblk, tot);
      if (threadIdx.x == 0) decide_row(ctrl, S, A, t, tot);
    }
    double c2[2];
    col_phase<LC, V, T, UOT>(A, t, c2, sh);
    if (threadIdx.x == 0) {
      A.part[3 * (size_t)A.nblk + blockIdx.x] = c2[0];
      A.part[4 * (size_t)A.nblk + blockIdx.x] = c2[1];
    }
    if (!grid_barrier(ctrl)) return;
    if (*(volatile int*)&ctrl->done) return;
    if (blockIdx.x == 0) {
      reduce_parts<2, T>(A.part + 3 * (size_t)A.nblk, A.nblk, tot);
      if (threadIdx.x == 0) decide_col(ctrl, S, t, tot);
    }
    ++t;
  }
}

// ---------------------------------------------------------------------------
// Persistent iterations over fixed work units.
//
// The rows (columns) are cut once per solve into contiguous units of at most
// kUnitRows rows whose element counts are close to T = ceil(nnz / W), W the
// number of working warps: a unit holds the rows whose first element falls
// into one bucket [b T, (b + 1) T) of the element range, split every
// kUnitRows rows.  Working warp w owns units w, w + W, ... for the whole
// solve, so the bounds, the weights and the current iterate values of its
// first unit stay in registers across iterations, and a phase reads only the
// unit's elements and the gathered vector.  The unit's index and value
// arrays stream through a two-slot ring of the warp in shared memory, filled
// by bulk copies (TMA) one slot ahead of the one being read, so the copies in
// flight hold no registers; the warp reads the elements in order with all 32
// lanes and closes each row with a butterfly.
// Warp 0 of block 0 takes no unit: it reduces the block partials of the
// phase just finished while the other warps run the next phase.
// With STAGE, every block first copies the whole gathered vector into shared
// memory (one bulk copy): scattered reads of one vector make each warp-wide
// gather touch up to 32 cache lines, so served from L1 they cost about one
// cycle per element per SM, while shared memory serves them at the rate of
// its bank conflicts.
// ---------------------------------------------------------------------------
constexpr int kUnitRows = 16;
constexpr int kUnitThreads = 512;            // 16 warps per block, one block per SM: up to 128 registers a thread
constexpr int kUnitWarps = kUnitThreads / 32;
constexpr size_t kStageBudget = 160 * 1024;   // largest staged vector (bytes)

template <typename T>
struct UnitCache {   // one unit of one warp, in shared memory
  int r0, nr;        // rows r0 .. r0 + nr - 1 (nr = 0: none)
  int p[kUnitRows + 1];   // ptr[r0 .. r0 + nr]
  T w[kUnitRows];    // weights of the rows
  T x[kUnitRows];    // current iterate values of the rows
};

// Shared memory of the unit kernel: the vector copy's barrier, two ring
// barriers per warp, three unit caches per warp (first row unit, first
// column unit, scratch), the rings (ring elements per slot, a multiple of
// 16) and the staged vector, each part 128-byte aligned.
template <typename T>
__host__ __device__ constexpr size_t unit_head_bytes() {
  return (64 + kUnitWarps * 16 + 3 * kUnitWarps * sizeof(UnitCache<T>) + 127) / 128 * 128;
}
template <typename V>
__host__ __device__ constexpr size_t ring_bytes(int ring) {
  return (size_t)kUnitWarps * 2 * ring * (sizeof(int) + sizeof(V));
}

// Unit starts: ustart[0 .. U] (ustart[U] = n) and U in ustart[n + 1].  One
// block; each thread scans a contiguous range of rows, so only the first row
// of a range needs a binary search for the start of its bucket.
__global__ void __launch_bounds__(1024) k_units(const int* __restrict__ ptr, int n, int W, int* __restrict__ ustart) {
  __shared__ int wtot[32];
  __shared__ int total;
  const long long nnz = ptr[n];
  const long long T = max(32LL, (nnz + W - 1) / W);
  const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
  const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
  auto walk = [&](auto&& emit) {
    if (lo >= hi) return;
    long long bprev = lo > 0 ? (long long)ptr[lo - 1] / T : -1;
    int first = lo;
    for (int i = lo; i < hi; ++i) {
      const long long b = (long long)ptr[i] / T;
      if (b != bprev) {
        first = i;
      } else if (i == lo) {   // the bucket started before this range
        const long long key = b * T;
        int l = 0, h = lo;
        while (l < h) {
          const int mid = (l + h) >> 1;
          if ((long long)ptr[mid] < key) l = mid + 1;
          else h = mid;
        }
        first = l;
      }
      if (b != bprev || (i - first) % kUnitRows == 0) emit(i);
      bprev = b;
    }
  };
  int cnt = 0;
  walk([&](int) { ++cnt; });
  // exclusive scan of the counts over the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wtot[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int nw = (int)(blockDim.x >> 5);
    int x = lane < nw ? wtot[lane] : 0, xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    if (lane < nw) wtot[lane] = xi - x;
    if (lane == 31) total = xi;
  }
  __syncthreads();
  int pos = wtot[w] + inc - cnt;
  walk([&](int i) { ustart[pos++] = i; });
  if (threadIdx.x == 0) {
    ustart[total] = n;
    ustart[n + 1] = total;
  }
}

// Unit u (or none: nr = 0) into the warp's cache c.
template <typename T>
__device__ __forceinline__ void load_unit(UnitCache<T>* c, const int* ustart, int U, const int* ptr, const T* wgt,
                                          const T* xcur, int u) {
  const int lane = threadIdx.x & 31;
  const int r0 = u < U ? ustart[u] : 0;
  const int nr = u < U ? ustart[u + 1] - r0 : 0;
  if (lane == 0) { c->r0 = r0; c->nr = nr; }
  if (lane <= nr) c->p[lane] = __ldg(ptr + r0 + lane);
  if (lane < nr) { c->w[lane] = wgt[r0 + lane]; c->x[lane] = xcur[r0 + lane]; }
  __syncwarp();
}

// q_i = sum_k val[k] x[idx[k]] for the rows of one unit, returned on lane
// i - r0 (lanes >= nr: 0).  Slot h of the ring holds `ring` elements of the
// index array (ridx) and of the value array (rval); chunk c of the unit's
// 16-element aligned range goes to slot c & 1 and the warp's barrier bars[h]
// completes when it has landed; `par` holds the two barriers' phase bits.
// Element k of a row goes to lane (k - start of the row's piece in the chunk)
// mod 32; a lane's partial sum carries over chunk boundaries.
// Chunk ch of a unit's aligned element range [kA, kE) into ring slot ch & 1 (lane 0).
template <typename V>
__device__ __forceinline__ void ring_issue(const int* idx, const V* val, int kA, int kE, int ch, int* ridx, V* rval,
                                           uint64_t* bars, int ring) {
  const int cs = kA + ch * ring;
  const unsigned cnt = (unsigned)(min(cs + ring, kE) - cs);
  const int h = ch & 1;
  fence_proxy_async_shared();
  mbar_arrive_expect_tx(bars + h, cnt * (unsigned)(sizeof(int) + sizeof(V)));
  bulk_copy_g2s(ridx + h * ring, idx + cs, cnt * (unsigned)sizeof(int), bars + h);
  bulk_copy_g2s(rval + h * ring, val + cs, cnt * (unsigned)sizeof(V), bars + h);
}

template <typename T>
__device__ __forceinline__ int ring_chunks(const UnitCache<T>* c, int ring) {
  const int kA = c->p[0] & ~15, kE = (c->p[c->nr] + 15) & ~15;
  return (kE - kA + ring - 1) / ring;
}

// The unit's first two chunks, issued ahead (the ring must be free).
template <typename V, typename T>
__device__ __forceinline__ void ring_start(const UnitCache<T>* c, const int* idx, const V* val, int* ridx, V* rval,
                                           uint64_t* bars, int ring) {
  if ((threadIdx.x & 31) == 0) {
    const int kA = c->p[0] & ~15, kE = (c->p[c->nr] + 15) & ~15;
    const int nch = (kE - kA + ring - 1) / ring;
    if (nch > 0) ring_issue<V>(idx, val, kA, kE, 0, ridx, rval, bars, ring);
    if (nch > 1) ring_issue<V>(idx, val, kA, kE, 1, ridx, rval, bars, ring);
  }
}

// Bounded wait for chunk ch's slot; false when it gave up.
__device__ __forceinline__ bool ring_wait(uint64_t* bars, unsigned& par, int ch) {
  const int h = ch & 1;
  bool ok = true;
  long long polls = 0;
  while (!mbar_try_wait(bars + h, (par >> h) & 1u)) {
    if (++polls > kSpinLimit) { ok = false; break; }
  }
  par ^= 1u << h;
  return __all_sync(0xffffffffu, ok);
}

// Wait for the chunks ring_start issued and use none of them (before an exit).
template <typename T>
__device__ __forceinline__ void ring_drain(const UnitCache<T>* c, uint64_t* bars, unsigned& par, int ring) {
  const int nch = min(ring_chunks(c, ring), 2);
  for (int ch = 0; ch < nch; ++ch) ring_wait(bars, par, ch);
}

template <typename V, typename T>
__device__ __forceinline__ bool unit_products(const UnitCache<T>* c, int nr, const int* __restrict__ idx,
                                              const V* val, const T* x, int* ridx, V* rval, uint64_t* bars,
                                              unsigned& par, int ring, bool started, T* q_out) {
  const int lane = threadIdx.x & 31;
  const int k0 = c->p[0], k1 = c->p[nr];
  const int kA = k0 & ~15, kE = (k1 + 15) & ~15;
  const int nch = (kE - kA + ring - 1) / ring;
  if (!started) ring_start<V, T>(c, idx, val, ridx, rval, bars, ring);
  int i = 0, re = c->p[1];
  T acc = 0, mine = 0;
  for (int ch = 0; ch < nch; ++ch) {
    const int h = ch & 1;
    if (!ring_wait(bars, par, ch)) return false;
    const int cs = kA + ch * ring;
    const int* si = ridx + h * ring - cs;
    const V* sv = rval + h * ring - cs;
    const int kend = min(cs + ring, k1);
    int k = max(cs, k0);
    while (k < kend) {
      const int pe = min(re, kend);
#pragma unroll 4
      for (int kk = k + lane; kk < pe; kk += 32) acc += load_as<T>(sv + kk) * x[si[kk]];
      k = pe;
      if (k == re) {   // the row ends here (an empty row ends at once)
        acc = warp_sum(acc);
        if (lane == i) mine = acc;
        acc = (T)0;
        ++i;
        re = c->p[min(i + 1, nr)];
      }
    }
    __syncwarp();   // slot h is read
    if (lane == 0 && ch + 2 < nch) ring_issue<V>(idx, val, kA, kE, ch + 2, ridx, rval, bars, ring);
  }
  *q_out = mine;   // rows left open are empty: 0
  return true;
}

// Row phase (ROW: u^{t+1} = (a / q)^phi with the residual terms of (u^t, v^t))
// or column phase (v^{t+1} = (b / r)^phi) over this warp's units.
// s[] gathers: ROW residual, unreachable a-mass, |u^{t+1} - u^t|;
//              column: unreachable b-mass, |v^{t+1} - v^t|.
template <typename V, typename T, bool UOT, bool ROW>
__device__ __forceinline__ bool unit_phase(const int* ustart, int U, const int* ptr, const int* idx, const V* val,
                                           const T* x, const T* wgt, const T* xcur, T* xnew, UnitCache<T>* c0,
                                           UnitCache<T>* scratch, int worker, int W, T phi, T inv_phi, T (&s)[3],
                                           int* ridx, V* rval, uint64_t* bars, unsigned& par, int ring,
                                           bool first_started) {
  const int lane = threadIdx.x & 31;
  int k = 0;
  for (int u = worker; u < U; u += W, ++k) {
    UnitCache<T>* c = c0;
    if (k > 0) {
      load_unit(scratch, ustart, U, ptr, wgt, xcur, u);
      c = scratch;
    }
    const int nr = c->nr;
    T q;
    if (!unit_products<V, T>(c, nr, idx, val, x, ridx, rval, bars, par, ring, k == 0 && first_started, &q))
      return false;
    if (lane < nr) {
      const T wi = c->w[lane], xo = c->x[lane];
      T xn;
      if (q > (T)0) {
        xn = UOT ? powT<T>(wi / q, phi) : wi / q;
        if (ROW) {
          const T lhs = (UOT ? powT<T>(xo, inv_phi) : xo) * q;
          s[0] += fabs(lhs - wi);
        }
      } else {
        xn = (T)0;
        s[ROW ? 1 : 0] += wi;
      }
      s[ROW ? 2 : 1] += fabs(xn - xo);
      xnew[c->r0 + lane] = xn;
      c->x[lane] = xn;
    }
    __syncwarp();
  }
  return true;
}

// The block partials reduced by one warp, in the order reduce_parts uses.
template <int NP, typename R>
__device__ __forceinline__ void reduce_parts_warp(const double* part, int nblk, double* out) {
  const int lane = threadIdx.x & 31;
  R s[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) s[p] = (R)0;
#pragma unroll 4
  for (int b = lane; b < nblk; b += 32) {
#pragma unroll
    for (int p = 0; p < NP; ++p) s[p] += (R)__ldcg(part + (size_t)p * nblk + b);
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) out[p] = (double)warp_sum(s[p]);
}

// A bounded wait gave up: the solve stops with an error.
__device__ __forceinline__ void wait_failed(Ctrl* ctrl) {
  ctrl->wait_timeout = 1;
  ctrl->status = SPS_ERR_CUDA;
  __threadfence();
  ctrl->done = 1;
}

// The whole vector x[0 .. len) into shared memory: one bulk copy (TMA) of
// its 16-byte aligned body when x is 16-byte aligned, plain loads otherwise
// and for the tail.  x was written by other blocks before the last grid
// barrier; the copy is ordered after that barrier by a proxy fence.  The
// wait is bounded: false (and the error recorded) when it gives up.
template <typename T>
__device__ __forceinline__ bool stage_vector(T* xs, const T* x, int len, uint64_t* bar, unsigned& parity,
                                             Ctrl* ctrl) {
  const size_t bytes = (size_t)len * sizeof(T);
  const bool bulk = ((uintptr_t)x & 15) == 0 && bytes >= 16;
  const unsigned body = bulk ? (unsigned)(bytes & ~(size_t)15) : 0u;
  if (bulk && threadIdx.x == 0) {
    fence_proxy_async_global();
    fence_proxy_async_shared();
    mbar_arrive_expect_tx(bar, body);
    bulk_copy_g2s(xs, x, body, bar);
  }
  for (int j = (int)(body / sizeof(T)) + (int)threadIdx.x; j < len; j += kUnitThreads) xs[j] = __ldcg(x + j);
  int ok = 1;
  if (bulk) {
    long long polls = 0;
    while (!mbar_try_wait(bar, parity)) {
      if (++polls > kSpinLimit) { ok = 0; break; }
    }
    parity ^= 1u;
  }
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) wait_failed(ctrl);
    return false;
  }
  return true;
}

template <typename V, typename T, bool UOT, bool STAGE>
__global__ void __launch_bounds__(kUnitThreads, 1) k_iterate_units(IterArgs A, int iters) {
  __shared__ T sh[3 * 32];
  __shared__ DecState S;   // block 0's decision state
  extern __shared__ __align__(128) char udyn[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ring = A.ring;
  uint64_t* bar = reinterpret_cast<uint64_t*>(udyn);               // STAGE: the vector copy's barrier
  uint64_t* bars = reinterpret_cast<uint64_t*>(udyn + 64) + 2 * warp;
  UnitCache<T>* ucache = reinterpret_cast<UnitCache<T>*>(udyn + 64 + kUnitWarps * 16) + 3 * warp;
  char* rings = udyn + unit_head_bytes<T>();
  int* ridx = reinterpret_cast<int*>(rings) + (size_t)warp * 2 * ring;
  V* rval = reinterpret_cast<V*>(rings + (size_t)kUnitWarps * 2 * ring * sizeof(int)) + (size_t)warp * 2 * ring;
  T* xs = reinterpret_cast<T*>(rings + ring_bytes<V>(ring));        // STAGE: the gathered vector
  Ctrl* ctrl = A.ctrl;
  if (ctrl->done) return;
  int t = ctrl->t;
  const bool reducer = blockIdx.x == 0 && warp == 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) S = load_state(ctrl);
  unsigned parity = 0, par = 0;
  if (threadIdx.x == 0 && STAGE) mbar_init(bar, 1);
  if (lane == 0) {
    mbar_init(bars + 0, 1);
    mbar_init(bars + 1, 1);
    fence_mbarrier_init();
  }
  __syncthreads();
  const int W = (int)gridDim.x * kUnitWarps - 1;
  const int worker = (int)blockIdx.x * kUnitWarps + warp - 1;
  const int Ur = A.unit_r[A.n + 1], Uc = A.unit_c[A.m + 1];
  const T* a = (const T*)A.a;
  const T* b = (const T*)A.b;
  const V* val = (const V*)A.val;
  const V* valT = (const V*)A.valT;
  const T phi = (T)A.phi, inv_phi = (T)A.inv_phi;
  if (!reducer) {
    load_unit(ucache + 0, A.unit_r, Ur, A.row_ptr, a, (const T*)A.ubuf + (size_t)(t & 1) * A.n, worker);
    load_unit(ucache + 1, A.unit_c, Uc, A.col_ptr, b, (const T*)A.vbuf + (size_t)(t & 1) * A.m, worker);
  }
  // The index and value arrays do not change: the first chunks of a warp's
  // next unit are issued before the grid barrier that precedes its phase.
  const bool has_r = !reducer && worker < Ur, has_c = !reducer && worker < Uc;
  int pre = 0;   // 1: row unit started, 2: column unit started
  auto bail = [&]() {
    if (pre) ring_drain(ucache + (pre - 1), bars, par, ring);
  };
  if (has_r) {
    ring_start<V, T>(ucache + 0, A.col_idx, val, ridx, rval, bars, ring);
    pre = 1;
  }
  for (int k = 0; k < iters; ++k) {
    const T* v = (const T*)A.vbuf + (size_t)(t & 1) * A.m;
    const T* uold = (const T*)A.ubuf + (size_t)(t & 1) * A.n;
    T* unew = (T*)A.ubuf + (size_t)((t + 1) & 1) * A.n;
    T* vnew = (T*)A.vbuf + (size_t)((t + 1) & 1) * A.m;
    T s3[3] = {(T)0, (T)0, (T)0};
    if (STAGE && !stage_vector<T>(xs, v, A.m, bar, parity, ctrl)) { bail(); return; }
    if (!reducer &&
        !unit_phase<V, T, UOT, true>(A.unit_r, Ur, A.row_ptr, A.col_idx, val, STAGE ? (const T*)xs : v, a, uold,
                                     unew, ucache + 0, ucache + 2, worker, W, phi, inv_phi, s3, ridx, rval, bars, par,
                                     ring, pre == 1))
      wait_failed(ctrl);
    pre = 0;
    if (has_c) {
      ring_start<V, T>(ucache + 1, A.row_idx, valT, ridx, rval, bars, ring);
      pre = 2;
    }
    block_sum_multi<3, T>(s3, sh);
    if (threadIdx.x == 0) {
      A.part[0 * (size_t)A.nblk + blockIdx.x] = (double)s3[0];
      A.part[1 * (size_t)A.nblk + blockIdx.x] = (double)s3[1];
      A.part[2 * (size_t)A.nblk + blockIdx.x] = (double)s3[2];
    }
    if (!grid_barrier_count(ctrl)) { bail(); return; }
    if (reducer) {
      double tot[3];
      reduce_parts_warp<3, T>(A.part, A.nblk, tot);
      if (lane == 0) decide_row(ctrl, S, A, t, tot);
    }
    T s2[3] = {(T)0, (T)0, (T)0};
    if (STAGE && !stage_vector<T>(xs, unew, A.n, bar, parity, ctrl)) { bail(); return; }
    if (!reducer &&
        !unit_phase<V, T, UOT, false>(A.unit_c, Uc, A.col_ptr, A.row_idx, valT, STAGE ? (const T*)xs : unew, b,
                                      (const T*)A.vbuf + (size_t)(t & 1) * A.m, vnew, ucache + 1, ucache + 2, worker,
                                      W, phi, inv_phi, s2, ridx, rval, bars, par, ring, pre == 2))
      wait_failed(ctrl);
    pre = 0;
    if (has_r && k + 1 < iters) {
      ring_start<V, T>(ucache + 0, A.col_idx, val, ridx, rval, bars, ring);
      pre = 1;
    }
    T c2[2] = {s2[0], s2[1]};
    block_sum_multi<2, T>(c2, sh);
    if (threadIdx.x == 0) {
      A.part[3 * (size_t)A.nblk + blockIdx.x] = (double)c2[0];
      A.part[4 * (size_t)A.nblk + blockIdx.x] = (double)c2[1];
    }
    if (!grid_barrier_count(ctrl)) { bail(); return; }
    if (*(volatile int*)&ctrl->done) { bail(); return; }
    if (reducer) {
      double tot[2];
      reduce_parts_warp<2, T>(A.part + 3 * (size_t)A.nblk, A.nblk, tot);
      if (lane == 0) decide_col(ctrl, S, t, tot);
    }
    ++t;
  }
}

template <int LPR, typename V, typename T, bool UOT>
__global__ void __launch_bounds__(kIterThreads) k_row_pass(IterArgs A) {
  __shared__ T sh[3 * 32];
  __shared__ double tot[3];
  Ctrl* ctrl = A.ctrl;
  if (ctrl->done) return;
  const int t = ctrl->t;
  double r3[3];
  row_phase<LPR, V, T, UOT>(A, t, r3, sh);
  if (!publish_and_check_last(&ctrl->blocks_a, A.part, A.nblk, r3, 3, 0)) return;
  reduce_parts<3, T>(A.part, A.nblk, tot);
  if (threadIdx.x == 0) {
    DecState S = load_state(ctrl);
    decide_row(ctrl, S, A, t, tot);
    ctrl->blocks_a = 0u;
  }
}

template <int LPR, typename V, typename T, bool UOT>
__global__ void __launch_bounds__(kIterThreads) k_col_pass(IterArgs A) {
  __shared__ T sh[3 * 32];
  __shared__ double tot[3];
  Ctrl* ctrl = A.ctrl;
  if (ctrl->done) return;
  const int t = ctrl->t;
  double c2[2];
  col_phase<LPR, V, T, UOT>(A, t, c2, sh);
  if (!publish_and_check_last(&ctrl->blocks_b, A.part, A.nblk, c2, 2, 3)) return;
  reduce_parts<2, T>(A.part + 3 * (size_t)A.nblk, A.nblk, tot);
  if (threadIdx.x == 0) {
    DecState S = load_state(ctrl);
    decide_col(ctrl, S, t, tot);
    ctrl->blocks_b = 0u;
  }
}

// u^0 = exp(alpha0/eps) (or 1), v^0 = exp(beta0/eps) (or 1), in buffer 0.
template <typename T>
__global__ void k_iter_init(int n, int m, T* u0, T* v0, const T* al, const T* be, double eps, Ctrl* ctrl) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) u0[i] = al ? (T)exp((double)al[i] / eps) : (T)1;
  for (int64_t j = tid; j < m; j += stride) v0[j] = be ? (T)exp((double)be[j] / eps) : (T)1;
  if (tid == 0) {
    ctrl->t = 0; ctrl->done = 0; ctrl->iters = 0;
    ctrl->blocks_a = ctrl->blocks_b = ctrl->blocks_c = 0u;
    ctrl->bar_count = 0u;
    ctrl->bar_mono = 0ull;
    if (ctrl->status != SPS_OK) { ctrl->done = 1; }
  }
}

// ---------------------------------------------------------------------------
// Objective (output line of Alg. 3 / Alg. 4) over the support of
// T~ = diag(u) K~ diag(v): per-element terms in the iterate type, FP64
// accumulation, deterministic block partials.
//   part slots: 0 transport, 1 neg_entropy, 2 logp, 3 mass, 4 KL(T1||a), 5 KL(T^T1||b)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double kl_term(double x, double y) {
  if (x == 0.0) return y;
  if (y == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  return x * log(x / y) - x + y;
}

__device__ __forceinline__ int returned_iter(const Ctrl* c) { return c->done ? c->iters : c->t; }

template <typename V, typename T, bool UOT>
__global__ void __launch_bounds__(kThreads) k_obj_rows(ProbDev pd, const SketchScalars* __restrict__ scp,
                                                       const float* __restrict__ rowf,
                                                       const float* __restrict__ colf, const int* ptr,
                                                       const int* idx, const V* val, const T* ubuf,
                                                       const T* vbuf, const T* a, const Ctrl* ctrl,
                                                       double* part, int nblk) {
  __shared__ double sh[32];
  const SketchScalars sc = *scp;
  const int it = returned_iter(ctrl);
  const T* u = ubuf + (size_t)(it & 1) * pd.n;
  const T* v = vbuf + (size_t)(it & 1) * pd.m;
  const int lane = threadIdx.x & 31;
  // per-element terms and per-row sums in the iterate type, FP64 across rows
  double tr = 0.0, ne = 0.0, lp = 0.0, ms = 0.0, kla = 0.0;
  for (int i = blockIdx.x * kWarps + (threadIdx.x >> 5); i < pd.n; i += gridDim.x * kWarps) {
    const T ui = u[i];
    T rtr = 0, rne = 0, rlp = 0, rs = 0;
    if (ui > (T)0) {
      const float ri = rowf[i];
      for (int k = ptr[i] + lane; k < ptr[i + 1]; k += 32) {
        const int j = idx[k];
        const T Tij = ui * load_as<T>(val + k) * v[j];
        if (!(Tij > (T)0)) continue;
        float D = 0.0f;
        const float p = pstar_raw<UOT>(pd, sc, ri, colf, i, j, &D);
        const T ps = p < 1.0f ? (T)p : (T)1;
        T C;
        if (pd.cost_kind == SPS_COST_WFR) C = (T)value_cost64(pd, sc, i, j);
        else if (sizeof(T) == 8) C = (T)(raw64(pd.cv, i, j) / sc.dn64);
        else C = (T)__fdiv_rn(UOT ? D : raw32(pd.cv, i, j), sc.dn32);
        rtr += Tij * C;
        rne += Tij * (log(Tij) - (T)1);
        rlp += Tij * log(ps);
        rs += Tij;
      }
    }
    rtr = warp_sum(rtr); rne = warp_sum(rne); rlp = warp_sum(rlp); rs = warp_sum(rs);
    if (lane == 0) {
      tr += (double)rtr; ne += (double)rne; lp += (double)rlp;
      ms += (double)rs;
      kla += kl_term((double)rs, (double)a[i]);
    }
  }
  const double vals[5] = {tr, ne, lp, ms, kla};
  for (int p = 0; p < 5; ++p) {
    const double s = block_sum_d(vals[p], sh);
    if (threadIdx.x == 0) part[(size_t)p * nblk + blockIdx.x] = s;
    __syncthreads();
  }
}

template <typename V, typename T>
__global__ void __launch_bounds__(kThreads) k_obj_cols(int m, const int* ptr, const int* idx, const V* valT,
                                                       const T* ubuf, const T* vbuf, const T* b, int n,
                                                       const Ctrl* ctrl, double* part, int nblk) {
  __shared__ double sh[32];
  const int it = returned_iter(ctrl);
  const T* u = ubuf + (size_t)(it & 1) * n;
  const T* v = vbuf + (size_t)(it & 1) * m;
  const int lane = threadIdx.x & 31;
  double klb = 0.0;
  for (int j = blockIdx.x * kWarps + (threadIdx.x >> 5); j < m; j += gridDim.x * kWarps) {
    const T vj = v[j];
    double cs = 0.0;
    if (vj > (T)0)
      for (int k = ptr[j] + lane; k < ptr[j + 1]; k += 32) cs += (double)(u[idx[k]] * load_as<T>(valT + k) * vj);
    cs = warp_sum(cs);
    if (lane == 0) klb += kl_term(cs, (double)b[j]);
  }
  const double s = block_sum_d(klb, sh);
  if (threadIdx.x == 0) part[5 * (size_t)nblk + blockIdx.x] = s;
}

template <typename T>
__global__ void k_obj_final(const double* part, int nblk, DevResult* out, const Ctrl* ctrl) {
  __shared__ double sh[32];
  double r[6];
  for (int p = 0; p < 6; ++p) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(size_t)p * nblk + b];
    s = block_sum_d(s, sh);
    __syncthreads();
    r[p] = s;
  }
  if (threadIdx.x == 0) {
    out->transport = r[0]; out->neg_entropy = r[1]; out->logp = r[2]; out->mass = r[3];
    out->kl_a = r[4]; out->kl_b = r[5];
    out->residual = ctrl->done ? ctrl->residual : ctrl->last_residual;
    out->unreach_a = ctrl->done ? ctrl->unreach_a : ctrl->last_unreach_a;
    out->unreach_b = ctrl->unreach_b;
  }
}

// Potentials alpha = eps log u, beta = eps log v of the returned pair.
template <typename T>
__global__ void k_potentials(int n, int m, const T* ubuf, const T* vbuf, double eps, const Ctrl* ctrl, T* al, T* be) {
  const int it = returned_iter(ctrl);
  const T* u = ubuf + (size_t)(it & 1) * n;
  const T* v = vbuf + (size_t)(it & 1) * m;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) al[i] = (T)(eps * log((double)u[i]));
  for (int64_t j = tid; j < m; j += stride) be[j] = (T)(eps * log((double)v[j]));
}

IterArgs make_args(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic) {
  IterArgs A;
  A.n = pd.n; A.m = pd.m;
  A.row_ptr = at<int>(ws, L.row_ptr); A.col_idx = at<int>(ws, L.col_idx);
  A.col_ptr = at<int>(ws, L.col_ptr); A.row_idx = at<int>(ws, L.row_idx);
  A.val = ws + L.val; A.valT = ws + L.valT;
  A.ubuf = ws + L.u; A.vbuf = ws + L.v; A.a = ws + L.a_it; A.b = ws + L.b_it;
  A.phi = ic.phi; A.inv_phi = 1.0 / ic.phi; A.tol = ic.tol; A.stop_rule = ic.stop_rule;
  A.ctrl = at<Ctrl>(ws, L.ctrl); A.part = at<double>(ws, L.part); A.nblk = L.nblk_rows;
  A.unit_r = L.unit_r ? at<int>(ws, L.unit_r) : nullptr;
  A.unit_c = L.unit_c ? at<int>(ws, L.unit_c) : nullptr;
  return A;
}

template <int LPR, typename V, typename T>
void pass_lpr(IterArgs A, bool uot, bool row, cudaStream_t st) {
  if (row) {
    if (uot) { auto f = k_row_pass<LPR, V, T, true>; A.nblk = iter_grid(f, A.nblk); f<<<A.nblk, kIterThreads, 0, st>>>(A); }
    else { auto f = k_row_pass<LPR, V, T, false>; A.nblk = iter_grid(f, A.nblk); f<<<A.nblk, kIterThreads, 0, st>>>(A); }
  } else {
    if (uot) { auto f = k_col_pass<LPR, V, T, true>; A.nblk = iter_grid(f, A.nblk); f<<<A.nblk, kIterThreads, 0, st>>>(A); }
    else { auto f = k_col_pass<LPR, V, T, false>; A.nblk = iter_grid(f, A.nblk); f<<<A.nblk, kIterThreads, 0, st>>>(A); }
  }
}

template <typename V, typename T>
void one_pass(const IterArgs& A, bool uot, bool row, int lpr, cudaStream_t st) {
  if (lpr >= 32) pass_lpr<32, V, T>(A, uot, row, st);
  else if (lpr >= 16) pass_lpr<16, V, T>(A, uot, row, st);
  else if (lpr >= 8) pass_lpr<8, V, T>(A, uot, row, st);
  else pass_lpr<4, V, T>(A, uot, row, st);
}

// Cooperative launch of the persistent kernel; false when the device refuses it
// (then the per-phase kernels are used).
template <int LR, int LC, typename V, typename T, bool UOT>
bool coop_launch(IterArgs A, int iters, cudaStream_t st) {
  auto fn = k_iterate<LR, LC, V, T, UOT>;
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kIterThreads, 0) != cudaSuccess || per_sm < 1) return false;
  const int grid = std::min(A.nblk, nsm * per_sm);
  A.nblk = grid;
  void* args[] = {(void*)&A, (void*)&iters};
  if (cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kIterThreads), args, 0, st) != cudaSuccess) {
    cudaGetLastError();  // clear the refusal
    return false;
  }
  return true;
}

template <int LR, typename V, typename T, bool UOT>
bool coop_lc(const IterArgs& A, int lc, int iters, cudaStream_t st) {
  if (lc >= 32) return coop_launch<LR, 32, V, T, UOT>(A, iters, st);
  if (lc >= 16) return coop_launch<LR, 16, V, T, UOT>(A, iters, st);
  if (lc >= 8) return coop_launch<LR, 8, V, T, UOT>(A, iters, st);
  return coop_launch<LR, 4, V, T, UOT>(A, iters, st);
}

// Instantiated lane pairs: equal lanes for rows and columns, or neighbours.
template <typename V, typename T, bool UOT>
bool coop(const IterArgs& A, int lr, int lc, int iters, cudaStream_t st) {
  if (lr >= 32) return coop_lc<32, V, T, UOT>(A, lc, iters, st);
  if (lr >= 16) return coop_lc<16, V, T, UOT>(A, lc, iters, st);
  if (lr >= 8) return coop_lc<8, V, T, UOT>(A, lc, iters, st);
  return coop_lc<4, V, T, UOT>(A, lc, iters, st);
}

// Shared memory plan of the unit kernel: the gathered vector staged when it
// fits beside rings of at least 128 elements a slot (rings of up to 512).
struct UnitPlan {
  bool stage;
  int ring;
  size_t smem;
};

template <typename V, typename T>
UnitPlan unit_plan(int n, int m) {
  const size_t limit = 227 * 1024 - 2048;   // dynamic part (the static arrays take under 1 KB)
  const size_t head = unit_head_bytes<T>();
  const size_t per16 = ring_bytes<V>(16);
  auto ring_for = [&](size_t room) { return (int)std::min<size_t>(512, room / per16 * 16); };
  const size_t sb = ((size_t)std::max(n, m) * sizeof(T) + 15) / 16 * 16;
  if (sb <= kStageBudget && head + sb < limit) {
    const int r = ring_for(limit - head - sb);
    if (r >= 128) return {true, r, head + ring_bytes<V>(r) + sb};
  }
  const int r = ring_for(limit - head);
  return {false, r, head + ring_bytes<V>(r)};
}

// Grid of the unit kernel (all SMs, as many blocks per SM as fit, at most
// cap); false when the device refuses a cooperative launch of it.
template <typename V, typename T, bool UOT, bool STAGE>
bool units_grid(int cap, size_t smem, int* grid_out) {
  auto fn = k_iterate_units<V, T, UOT, STAGE>;
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  if (cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kUnitThreads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  *grid_out = std::max(1, std::min(cap, nsm * per_sm));
  return true;
}

template <typename V, typename T, bool UOT, bool STAGE>
bool coop_units_s(IterArgs A, const UnitPlan& pl, int iters, cudaStream_t st) {
  int grid = 0;
  if (!units_grid<V, T, UOT, STAGE>(A.nblk, pl.smem, &grid)) return false;
  A.nblk = grid;
  A.ring = pl.ring;
  void* args[] = {(void*)&A, (void*)&iters};
  if (cudaLaunchCooperativeKernel((const void*)k_iterate_units<V, T, UOT, STAGE>, dim3(grid), dim3(kUnitThreads),
                                  args, pl.smem, st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

template <typename V, typename T, bool UOT>
bool coop_units(const IterArgs& A, int iters, cudaStream_t st) {
  const UnitPlan pl = unit_plan<V, T>(A.n, A.m);
  return pl.stage ? coop_units_s<V, T, UOT, true>(A, pl, iters, st) : coop_units_s<V, T, UOT, false>(A, pl, iters, st);
}

template <typename V, typename T, bool UOT>
int units_grid_u(int n, int m, int cap) {
  int g = 0;
  const UnitPlan pl = unit_plan<V, T>(n, m);
  const bool ok = pl.stage ? units_grid<V, T, UOT, true>(cap, pl.smem, &g) : units_grid<V, T, UOT, false>(cap, pl.smem, &g);
  return ok ? g : 0;
}

template <typename V, typename T>
int units_grid_vt(const IterCfg& ic, int n, int m, int cap) {
  return ic.uot ? units_grid_u<V, T, true>(n, m, cap) : units_grid_u<V, T, false>(n, m, cap);
}

int units_grid_dispatch(const IterCfg& ic, int n, int m, int cap) {
  switch (ic.kd) {
    case SPS_F64: return units_grid_vt<double, double>(ic, n, m, cap);
    case SPS_F32: return units_grid_vt<float, float>(ic, n, m, cap);
    case SPS_BF16: return units_grid_vt<__nv_bfloat16, float>(ic, n, m, cap);
    default: return units_grid_vt<__half, float>(ic, n, m, cap);
  }
}

// Set by launch_iter_init when it enqueued this solve's work units (the unit
// kernel runs only on a partition of the current sketch).
thread_local bool g_units_ready = false;

// Enqueue `iters` iterations; returns the number of kernels launched.
template <typename V, typename T>
int iterate_vt(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters, cudaStream_t st) {
  const IterArgs A = make_args(pd, L, ws, ic);
  if (ic.persistent && A.unit_r && A.unit_c && g_units_ready) {
    const bool ok = ic.uot ? coop_units<V, T, true>(A, iters, st) : coop_units<V, T, false>(A, iters, st);
    if (ok) return 1;
  }
  if (ic.persistent) {
    const bool ok = ic.uot ? coop<V, T, true>(A, ic.lpr_rows, ic.lpr_cols, iters, st)
                           : coop<V, T, false>(A, ic.lpr_rows, ic.lpr_cols, iters, st);
    if (ok) return 1;
  }
  for (int k = 0; k < iters; ++k) {
    one_pass<V, T>(A, ic.uot, true, ic.lpr_rows, st);
    one_pass<V, T>(A, ic.uot, false, ic.lpr_cols, st);
  }
  return 2 * iters;
}

int iterate_dispatch(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters, cudaStream_t st) {
  switch (ic.kd) {
    case SPS_F64: return iterate_vt<double, double>(pd, L, ws, ic, iters, st);
    case SPS_F32: return iterate_vt<float, float>(pd, L, ws, ic, iters, st);
    case SPS_BF16: return iterate_vt<__nv_bfloat16, float>(pd, L, ws, ic, iters, st);
    default: return iterate_vt<__half, float>(pd, L, ws, ic, iters, st);
  }
}

void row_only_dispatch(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, cudaStream_t st) {
  const IterArgs A = make_args(pd, L, ws, ic);
  switch (ic.kd) {
    case SPS_F64: one_pass<double, double>(A, ic.uot, true, ic.lpr_rows, st); break;
    case SPS_F32: one_pass<float, float>(A, ic.uot, true, ic.lpr_rows, st); break;
    case SPS_BF16: one_pass<__nv_bfloat16, float>(A, ic.uot, true, ic.lpr_rows, st); break;
    default: one_pass<__half, float>(A, ic.uot, true, ic.lpr_rows, st); break;
  }
}

template <typename V, typename T>
void objective_vt(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, void* al, void* be, cudaStream_t st) {
  const SketchScalars* sc = at<SketchScalars>(ws, L.scal);
  const Ctrl* ctrl = at<Ctrl>(ws, L.ctrl);
  double* part = at<double>(ws, L.part);
  const T* u = at<T>(ws, L.u);
  const T* v = at<T>(ws, L.v);
  const int nb = L.nblk_rows;
  if (!pd.sep)   // the template selects the decision rule of p* (Eq. pij-uot or separable)
    k_obj_rows<V, T, true><<<nb, kThreads, 0, st>>>(pd, sc, at<float>(ws, L.rowf), at<float>(ws, L.colf),
        at<int>(ws, L.row_ptr), at<int>(ws, L.col_idx), at<V>(ws, L.val), u, v, at<T>(ws, L.a_it), ctrl, part, nb);
  else
    k_obj_rows<V, T, false><<<nb, kThreads, 0, st>>>(pd, sc, at<float>(ws, L.rowf), at<float>(ws, L.colf),
        at<int>(ws, L.row_ptr), at<int>(ws, L.col_idx), at<V>(ws, L.val), u, v, at<T>(ws, L.a_it), ctrl, part, nb);
  k_obj_cols<V, T><<<nb, kThreads, 0, st>>>(pd.m, at<int>(ws, L.col_ptr), at<int>(ws, L.row_idx),
      at<V>(ws, L.valT), u, v, at<T>(ws, L.b_it), pd.n, ctrl, part, nb);
  k_obj_final<T><<<1, kThreads, 0, st>>>(part, nb, at<DevResult>(ws, L.res), ctrl);
  const int g = (int)std::min<int64_t>(4096, (std::max(pd.n, pd.m) + kThreads - 1) / kThreads);
  if (al && be) k_potentials<T><<<std::max(g, 1), kThreads, 0, st>>>(pd.n, pd.m, u, v, ic.eps, ctrl, (T*)al, (T*)be);
}

}  // namespace

sps_status launch_iter_init(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                            const void* init_alpha, const void* init_beta, cudaStream_t st) {
  const int g = (int)std::min<int64_t>(4096, (std::max(pd.n, pd.m) + kThreads - 1) / kThreads);
  if (ic.it64)
    k_iter_init<double><<<std::max(g, 1), kThreads, 0, st>>>(pd.n, pd.m, at<double>(ws, L.u), at<double>(ws, L.v),
        (const double*)init_alpha, (const double*)init_beta, ic.eps, at<Ctrl>(ws, L.ctrl));
  else
    k_iter_init<float><<<std::max(g, 1), kThreads, 0, st>>>(pd.n, pd.m, at<float>(ws, L.u), at<float>(ws, L.v),
        (const float*)init_alpha, (const float*)init_beta, ic.eps, at<Ctrl>(ws, L.ctrl));
  add_launches(1);
  g_units_ready = false;
  if (ic.persistent && L.unit_r && L.unit_c) {
    // work units for the grid the persistent kernel will get
    const int grid = units_grid_dispatch(ic, pd.n, pd.m, L.nblk_rows);
    if (grid > 0) {
      g_units_ready = true;
      const int W = grid * kUnitWarps - 1;
      k_units<<<1, 1024, 0, st>>>(at<int>(ws, L.row_ptr), pd.n, W, at<int>(ws, L.unit_r));
      k_units<<<1, 1024, 0, st>>>(at<int>(ws, L.col_ptr), pd.m, W, at<int>(ws, L.unit_c));
      add_launches(2);
    }
  }
  return cuda_fail(cudaGetLastError(), "iter_init");
}

sps_status launch_sparse_iterations(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters,
                                    cudaStream_t st) {
  add_launches(iterate_dispatch(pd, L, ws, ic, iters, st));
  return cuda_fail(cudaGetLastError(), "sparse iterations");
}

sps_status launch_sparse_row_only(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, cudaStream_t st) {
  row_only_dispatch(pd, L, ws, ic, st);
  add_launches(1);
  return cuda_fail(cudaGetLastError(), "sparse row pass");
}

sps_status launch_sparse_objective(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                   void* alpha_out, void* beta_out, cudaStream_t st) {
  switch (ic.kd) {
    case SPS_F64: objective_vt<double, double>(pd, L, ws, ic, alpha_out, beta_out, st); break;
    case SPS_F32: objective_vt<float, float>(pd, L, ws, ic, alpha_out, beta_out, st); break;
    case SPS_BF16: objective_vt<__nv_bfloat16, float>(pd, L, ws, ic, alpha_out, beta_out, st); break;
    case SPS_F16: objective_vt<__half, float>(pd, L, ws, ic, alpha_out, beta_out, st); break;
  }
  add_launches((alpha_out && beta_out) ? 4 : 3);
  return cuda_fail(cudaGetLastError(), "objective");
}

}  // namespace sps
