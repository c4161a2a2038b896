// sps_iter.cu -- Sinkhorn scaling iterations on the sketch (Alg. 1 / Alg. 2
// run on K~, as Alg. 3 / Alg. 4 prescribe) and the objective of their
// output line.
//
// One iteration t -> t+1 is two kernels:
//   row pass  q = K~ v^t (CSR, one warp per row), u^{t+1} = (a / q)^phi into
//             the other u buffer, and -- fused, at no extra pass -- the
//             stopping residual of the pair (u^t, v^t):
//                 rho_t = sum over reachable i of | (u^t_i)^{1/phi} q_i - a_i |
//             (the column side of that pair is zero up to rounding because
//             v^t was computed from u^t).  The last block to finish reduces
//             the block partials in a fixed order and sets the stop flag.
//   col pass  r = K~^T u^{t+1} (CSC), v^{t+1} = (b / r)^phi in place; the last
//             block advances the iteration counter.
// Both kernels return at once when the stop flag is set, so any number of
// iterations can be enqueued ahead of the convergence read-back.
// Rows (columns) whose product is zero get u_i = 0 (v_j = 0): they carry
// mass no plan on the sketch can move, are left out of the residual, and
// their mass is reported.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "sps_internal.h"

namespace sps {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Warp-cooperative sparse dot product of one row: four independent chains
// per lane so that index and value loads of several strides are in flight.
template <typename V, typename T>
__device__ __forceinline__ T warp_row_dot(const int* __restrict__ idx, const V* __restrict__ val,
                                          const T* __restrict__ x, int lo, int hi, int lane) {
  T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  int k = lo + lane;
  for (; k + 96 < hi; k += 128) {
    const int i0 = __ldg(idx + k), i1 = __ldg(idx + k + 32), i2 = __ldg(idx + k + 64), i3 = __ldg(idx + k + 96);
    const T v0 = load_as<T>(val + k), v1 = load_as<T>(val + k + 32), v2 = load_as<T>(val + k + 64),
            v3 = load_as<T>(val + k + 96);
    a0 += v0 * __ldg(x + i0);
    a1 += v1 * __ldg(x + i1);
    a2 += v2 * __ldg(x + i2);
    a3 += v3 * __ldg(x + i3);
  }
  for (; k < hi; k += 32) a0 += load_as<T>(val + k) * __ldg(x + __ldg(idx + k));
  return warp_sum((a0 + a1) + (a2 + a3));
}

template <typename T> __device__ __forceinline__ T powT(T x, T y);
template <> __device__ __forceinline__ float powT<float>(float x, float y) { return powf(x, y); }
template <> __device__ __forceinline__ double powT<double>(double x, double y) { return pow(x, y); }

struct HalfArgs {
  int rows;            // rows of this pass (n for CSR, m for CSC)
  const int* ptr;
  const int* idx;
  const void* val;
  const void* xin;     // gathered vector (v for the row pass; unused for the col pass)
  void* ubuf;          // u buffers (2 x n)
  void* vbuf;          // v (m)
  const void* marg;    // a (row pass) or b (col pass), iterate type
  int n;               // length of one u buffer
  double phi, inv_phi, tol;
  int stop_rule;
  Ctrl* ctrl;
  double* part;        // kPartSlots x nblk
  int nblk;
};

// Deterministic reduction of `nparts` arrays of block partials by the last block.
__device__ void reduce_parts(const double* part, int nblk, int nparts, double* out, double* sh) {
  for (int p = 0; p < nparts; ++p) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += __ldcg(part + (size_t)p * nblk + b);
    s = block_sum_d(s, sh);
    if (threadIdx.x == 0) out[p] = s;
    __syncthreads();
  }
}

__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  return am_last;
}

template <typename V, typename T, bool UOT>
__global__ void __launch_bounds__(kThreads) k_row_pass(HalfArgs A) {
  Ctrl* ctrl = A.ctrl;
  if (ctrl->done) return;
  __shared__ double sh[32];
  const int t = ctrl->t;
  const T* v = (const T*)A.xin;
  const T* uold = (const T*)A.ubuf + (size_t)(t & 1) * A.n;
  T* unew = (T*)A.ubuf + (size_t)((t + 1) & 1) * A.n;
  const T* a = (const T*)A.marg;
  const V* val = (const V*)A.val;
  const int lane = threadIdx.x & 31;
  const T phi = (T)A.phi, inv_phi = (T)A.inv_phi;
  double res = 0.0, unr = 0.0, dl = 0.0;
  for (int i = blockIdx.x * kWarps + (threadIdx.x >> 5); i < A.rows; i += gridDim.x * kWarps) {
    const T q = warp_row_dot<V, T>(A.idx, val, v, A.ptr[i], A.ptr[i + 1], lane);
    if (lane == 0) {
      const T ai = a[i], uo = uold[i];
      T un;
      if (q > (T)0) {
        un = UOT ? powT<T>(ai / q, phi) : ai / q;
        const T lhs = (UOT ? powT<T>(uo, inv_phi) : uo) * q;
        res += fabs((double)lhs - (double)ai);
      } else {
        un = (T)0;
        unr += (double)ai;
      }
      dl += fabs((double)un - (double)uo);
      unew[i] = un;
    }
  }
  res = block_sum_d(res, sh);
  __syncthreads();
  unr = block_sum_d(unr, sh);
  __syncthreads();
  dl = block_sum_d(dl, sh);
  if (threadIdx.x == 0) {
    A.part[0 * A.nblk + blockIdx.x] = res;
    A.part[1 * A.nblk + blockIdx.x] = unr;
    A.part[2 * A.nblk + blockIdx.x] = dl;
  }
  if (!last_block(&ctrl->blocks_a)) return;
  double tot[3];
  __shared__ double outv[3];
  reduce_parts(A.part, A.nblk, 3, outv, sh);
  if (threadIdx.x == 0) {
    tot[0] = outv[0]; tot[1] = outv[1]; tot[2] = outv[2];
    ctrl->last_residual = tot[0];
    ctrl->last_unreach_a = tot[1];
    ctrl->delta_u = tot[2];
    if (A.stop_rule == SPS_STOP_RESIDUAL) {
      if (!isfinite(tot[0])) {
        ctrl->done = 1; ctrl->status = SPS_ERR_NUMERIC; ctrl->iters = t; ctrl->residual = tot[0];
      } else if (t >= 1 && tot[0] <= A.tol) {
        ctrl->done = 1; ctrl->iters = t; ctrl->residual = tot[0]; ctrl->unreach_a = tot[1];
      }
    }
    ctrl->blocks_a = 0u;
  }
}

template <typename V, typename T, bool UOT>
__global__ void __launch_bounds__(kThreads) k_col_pass(HalfArgs A) {
  Ctrl* ctrl = A.ctrl;
  if (ctrl->done) return;
  __shared__ double sh[32];
  const int t = ctrl->t;
  const T* u = (const T*)A.ubuf + (size_t)((t + 1) & 1) * A.n;
  T* v = (T*)A.vbuf;
  const T* b = (const T*)A.marg;
  const V* val = (const V*)A.val;
  const int lane = threadIdx.x & 31;
  const T phi = (T)A.phi;
  double unb = 0.0, dl = 0.0;
  for (int j = blockIdx.x * kWarps + (threadIdx.x >> 5); j < A.rows; j += gridDim.x * kWarps) {
    const T r = warp_row_dot<V, T>(A.idx, val, u, A.ptr[j], A.ptr[j + 1], lane);
    if (lane == 0) {
      const T bj = b[j], vo = v[j];
      T vn;
      if (r > (T)0) {
        vn = UOT ? powT<T>(bj / r, phi) : bj / r;
      } else {
        vn = (T)0;
        unb += (double)bj;
      }
      dl += fabs((double)vn - (double)vo);
      v[j] = vn;
    }
  }
  unb = block_sum_d(unb, sh);
  __syncthreads();
  dl = block_sum_d(dl, sh);
  if (threadIdx.x == 0) {
    A.part[3 * A.nblk + blockIdx.x] = unb;
    A.part[4 * A.nblk + blockIdx.x] = dl;
  }
  if (!last_block(&ctrl->blocks_b)) return;
  __shared__ double outv[2];
  reduce_parts(A.part + 3 * (size_t)A.nblk, A.nblk, 2, outv, sh);
  if (threadIdx.x == 0) {
    ctrl->unreach_b = outv[0];
    const int tn = t + 1;
    ctrl->t = tn;
    if (A.stop_rule == SPS_STOP_DELTA_UV) {
      const double tot = ctrl->delta_u + outv[1];
      if (!isfinite(tot)) {
        ctrl->done = 1; ctrl->status = SPS_ERR_NUMERIC; ctrl->iters = tn; ctrl->residual = tot;
      } else if (tot <= A.tol) {
        ctrl->done = 1; ctrl->iters = tn; ctrl->residual = tot; ctrl->unreach_a = ctrl->last_unreach_a;
      }
    }
    ctrl->blocks_b = 0u;
  }
}

// u^0 = exp(alpha0/eps) (or 1) in buffer 0, v^0 = exp(beta0/eps) (or 1).
template <typename T>
__global__ void k_iter_init(int n, int m, T* u0, T* v0, const T* al, const T* be, double eps, Ctrl* ctrl) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) u0[i] = al ? (T)exp((double)al[i] / eps) : (T)1;
  for (int64_t j = tid; j < m; j += stride) v0[j] = be ? (T)exp((double)be[j] / eps) : (T)1;
  if (tid == 0) {
    ctrl->t = 0; ctrl->done = 0; ctrl->iters = 0;
    ctrl->blocks_a = ctrl->blocks_b = ctrl->blocks_c = 0u;
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

template <typename V, typename T, bool UOT>
__global__ void __launch_bounds__(kThreads) k_obj_rows(ProbDev pd, const SketchScalars* __restrict__ scp,
                                                       const float* __restrict__ rowf,
                                                       const float* __restrict__ colf, const int* ptr,
                                                       const int* idx, const V* val, const T* ubuf,
                                                       const T* v, const T* a, const Ctrl* ctrl,
                                                       double* part, int nblk) {
  __shared__ double sh[32];
  const SketchScalars sc = *scp;
  const int it = ctrl->done ? ctrl->iters : ctrl->t;
  const T* u = ubuf + (size_t)(it & 1) * pd.n;
  const int lane = threadIdx.x & 31;
  double tr = 0.0, ne = 0.0, lp = 0.0, ms = 0.0, kla = 0.0;
  for (int i = blockIdx.x * kWarps + (threadIdx.x >> 5); i < pd.n; i += gridDim.x * kWarps) {
    const T ui = u[i];
    double rs = 0.0;
    if (ui > (T)0) {
      const float ri = rowf[i];
      for (int k = ptr[i] + lane; k < ptr[i + 1]; k += 32) {
        const int j = idx[k];
        const T Tij = ui * load_as<T>(val + k) * v[j];
        if (!(Tij > (T)0)) continue;
        float D = 0.0f;
        const float p = pstar_raw<UOT>(pd, sc, ri, colf, i, j, &D);
        const double ps = p < 1.0f ? (double)p : 1.0;
        double C;
        if (sizeof(T) == 8) C = raw64(pd.cv, i, j) / sc.dn64;
        else C = (double)__fdiv_rn(UOT ? D : raw32(pd.cv, i, j), sc.dn32);
        const double td = (double)Tij;
        tr += td * C;
        ne += td * ((double)log(Tij) - 1.0);
        lp += td * log(ps);
        rs += td;
      }
    }
    rs = warp_sum(rs);
    if (lane == 0) {
      ms += rs;
      kla += kl_term(rs, (double)a[i]);
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
                                                       const T* ubuf, const T* v, const T* b, int n,
                                                       const Ctrl* ctrl, double* part, int nblk) {
  __shared__ double sh[32];
  const int it = ctrl->done ? ctrl->iters : ctrl->t;
  const T* u = ubuf + (size_t)(it & 1) * n;
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

// Final reduction, potentials alpha = eps log u, beta = eps log v.
template <typename T>
__global__ void k_obj_final(const double* part, int nblk_r, int nblk_c, DevResult* out, const Ctrl* ctrl) {
  __shared__ double sh[32];
  double r[6];
  for (int p = 0; p < 6; ++p) {
    const int nb = p == 5 ? nblk_c : nblk_r;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(size_t)p * nblk_r + b];
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

template <typename T, typename O>
__global__ void k_potentials(int n, int m, const T* ubuf, const T* v, double eps, const Ctrl* ctrl, O* al, O* be) {
  const int it = ctrl->done ? ctrl->iters : ctrl->t;
  const T* u = ubuf + (size_t)(it & 1) * n;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) al[i] = (O)(eps * log((double)u[i]));
  for (int64_t j = tid; j < m; j += stride) be[j] = (O)(eps * log((double)v[j]));
}

template <typename V, typename T>
HalfArgs row_args(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic) {
  HalfArgs A;
  A.rows = pd.n; A.ptr = at<int>(ws, L.row_ptr); A.idx = at<int>(ws, L.col_idx); A.val = ws + L.val;
  A.xin = ws + L.v; A.ubuf = ws + L.u; A.vbuf = ws + L.v; A.marg = ws + L.a_it; A.n = pd.n;
  A.phi = ic.phi; A.inv_phi = 1.0 / ic.phi; A.tol = ic.tol; A.stop_rule = ic.stop_rule;
  A.ctrl = at<Ctrl>(ws, L.ctrl); A.part = at<double>(ws, L.part); A.nblk = L.nblk_rows;
  return A;
}

template <typename V, typename T>
HalfArgs col_args(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic) {
  HalfArgs A = row_args<V, T>(pd, L, ws, ic);
  A.rows = pd.m; A.ptr = at<int>(ws, L.col_ptr); A.idx = at<int>(ws, L.row_idx); A.val = ws + L.valT;
  A.marg = ws + L.b_it; A.nblk = L.nblk_cols;
  return A;
}

template <typename V, typename T>
void iteration_vt(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, bool row_only, cudaStream_t st) {
  const HalfArgs R = row_args<V, T>(pd, L, ws, ic);
  if (ic.uot) k_row_pass<V, T, true><<<L.nblk_rows, kThreads, 0, st>>>(R);
  else k_row_pass<V, T, false><<<L.nblk_rows, kThreads, 0, st>>>(R);
  if (row_only) return;
  const HalfArgs Cc = col_args<V, T>(pd, L, ws, ic);
  if (ic.uot) k_col_pass<V, T, true><<<L.nblk_cols, kThreads, 0, st>>>(Cc);
  else k_col_pass<V, T, false><<<L.nblk_cols, kThreads, 0, st>>>(Cc);
}

void iteration_dispatch(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, bool row_only, cudaStream_t st) {
  switch (ic.kd) {
    case SPS_F64: iteration_vt<double, double>(pd, L, ws, ic, row_only, st); break;
    case SPS_F32: iteration_vt<float, float>(pd, L, ws, ic, row_only, st); break;
    case SPS_BF16: iteration_vt<__nv_bfloat16, float>(pd, L, ws, ic, row_only, st); break;
    case SPS_F16: iteration_vt<__half, float>(pd, L, ws, ic, row_only, st); break;
  }
}

template <typename V, typename T>
void objective_vt(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, void* al, void* be, cudaStream_t st) {
  const SketchScalars* sc = at<SketchScalars>(ws, L.scal);
  const Ctrl* ctrl = at<Ctrl>(ws, L.ctrl);
  double* part = at<double>(ws, L.part);
  const T* u = at<T>(ws, L.u);
  const T* v = at<T>(ws, L.v);
  if (ic.uot)
    k_obj_rows<V, T, true><<<L.nblk_rows, kThreads, 0, st>>>(pd, sc, at<float>(ws, L.rowf), at<float>(ws, L.colf),
        at<int>(ws, L.row_ptr), at<int>(ws, L.col_idx), at<V>(ws, L.val), u, v, at<T>(ws, L.a_it), ctrl, part, L.nblk_rows);
  else
    k_obj_rows<V, T, false><<<L.nblk_rows, kThreads, 0, st>>>(pd, sc, at<float>(ws, L.rowf), at<float>(ws, L.colf),
        at<int>(ws, L.row_ptr), at<int>(ws, L.col_idx), at<V>(ws, L.val), u, v, at<T>(ws, L.a_it), ctrl, part, L.nblk_rows);
  k_obj_cols<V, T><<<L.nblk_cols, kThreads, 0, st>>>(pd.m, at<int>(ws, L.col_ptr), at<int>(ws, L.row_idx),
      at<V>(ws, L.valT), u, v, at<T>(ws, L.b_it), pd.n, ctrl, part, L.nblk_rows);
  k_obj_final<T><<<1, kThreads, 0, st>>>(part, L.nblk_rows, L.nblk_cols, at<DevResult>(ws, L.res), ctrl);
  const int g = (int)std::min<int64_t>(4096, (std::max(pd.n, pd.m) + kThreads - 1) / kThreads);
  if (al && be)
    k_potentials<T, T><<<std::max(g, 1), kThreads, 0, st>>>(pd.n, pd.m, u, v, ic.eps, ctrl, (T*)al, (T*)be);
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

sps_status launch_sparse_iteration(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, cudaStream_t st) {
  iteration_dispatch(pd, L, ws, ic, false, st);
  add_launches(2);
  return cuda_fail(cudaGetLastError(), "sparse iteration");
}

sps_status launch_sparse_row_only(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, cudaStream_t st) {
  iteration_dispatch(pd, L, ws, ic, true, st);
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
