// sps_iter.cu -- Sinkhorn scaling iterations on the sketch (Alg. 1 / Alg. 2
// run on K~, as Alg. 3 / Alg. 4 prescribe) and the objective of their
// output line.
//
// Iteration t -> t+1 has two phases:
//   row phase  q = K~ v^t (CSR; LPR lanes per row), u^{t+1} = (a / q)^phi, and
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
// Two executions of the same phases:
//   - a persistent cooperative kernel that runs a whole chunk of iterations in
//     one launch, with two grid barriers per iteration (bounded spin waits);
//     block 0 reduces the block partials in a fixed order and decides;
//   - one kernel per phase (the last block to finish reduces the partials),
//     used for the final residual and when a cooperative launch is refused.
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
        if (sizeof(T) == 8) C = (T)(raw64(pd.cv, i, j) / sc.dn64);
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

// Enqueue `iters` iterations; returns the number of kernels launched.
template <typename V, typename T>
int iterate_vt(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters, cudaStream_t st) {
  const IterArgs A = make_args(pd, L, ws, ic);
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
  if (ic.uot)
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
