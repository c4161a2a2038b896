// sps_dense.cu -- dense Sinkhorn (Alg. 1 / Alg. 2, section 2) with the Gibbs
// kernel K_ij = exp(-C_ij/eps) recomputed from the points in every pass and
// never stored.
//
// A pass is a tiled kernel over (row block, column range): a block owns
// kRPT * kTI rows (kRPT per thread, coordinates in registers) and stages the
// coordinates and the scaling of kTJ columns at a time in shared memory.
// Each column range writes its own partial vector; the update kernels add the
// partials in a fixed order, so results are deterministic.  The update
// kernels carry the stopping logic of the sparse path: the row update forms
// the residual of the incoming pair, the column update advances the counter.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "sps_dense.cuh"
#include "sps_internal.h"

namespace sps {

namespace {

using namespace dense;

struct PassArgs {
  DenseView V;
  const SketchScalars* sc;
  double eps;
  const void* w;        // explicit column scaling (wsel == 0)
  const void* ubuf;     // u buffers (2 x n_u)
  int n_u;
  int wsel;             // 0: w; 1: u^{t+1} (column pass of an iteration); 2: returned u
  const void* v;        // mode 1: column scaling
  void* out;            // mode 0: partial vectors [split][np]
  int qchunk;
  int gate;             // 1: skip when the solve has stopped
  const Ctrl* ctrl;
  double* part;         // mode 1: 3 x nblk_total block partials
  int nblk_total;
};

__device__ __forceinline__ int returned_iter(const Ctrl* c) { return c->done ? c->iters : c->t; }

template <typename T> __device__ __forceinline__ T gibbs(T D, T k2);
// exp(-D / (dn eps)) = exp2(-D * k2), k2 = log2(e) / (dn eps)
template <> __device__ __forceinline__ float gibbs<float>(float D, float k2) { return exp2f(-D * k2); }
template <> __device__ __forceinline__ double gibbs<double>(double D, double k2) { return exp(-D * k2); }

// mode 0: out[split][p] = sum_{q in range} K_pq w_q
// mode 1: block partials of transport, neg_entropy, mass over the range
template <typename T, int DM, bool EXACT, int MODE>
__global__ void __launch_bounds__(kTI) k_dense_pass(PassArgs A) {
  if (A.gate && A.ctrl->done) return;
  __shared__ T qs[kTJ * DM];
  __shared__ T ws[kTJ];
  __shared__ T lws[kTJ];   // mode 1: log of the column scaling
  __shared__ double sh[32];
  const DenseView& V = A.V;
  const int d = V.d;
  const bool dense_cost = V.C32 || V.C64;
  const double dn = sizeof(T) == 8 ? A.sc->dn64 : (double)A.sc->dn32;
  const T k2 = (T)((sizeof(T) == 8 ? 1.0 : 1.4426950408889634) / (dn * A.eps));
  const T inv_dn = (T)(1.0 / dn), inv_eps = (T)(1.0 / A.eps);
  const T* w = (const T*)A.w;
  if (A.wsel == 1) w = (const T*)A.ubuf + (size_t)((A.ctrl->t + 1) & 1) * A.n_u;
  if (A.wsel == 2) w = (const T*)A.ubuf + (size_t)(returned_iter(A.ctrl) & 1) * A.n_u;
  const T* urow = (const T*)A.ubuf + (size_t)(returned_iter(A.ctrl) & 1) * A.n_u;
  const int p0 = blockIdx.x * (kTI * kRPT);
  const int q_begin = blockIdx.y * A.qchunk;
  const int q_end = min(V.nq, q_begin + A.qchunk);
  T pr[kRPT][DM];
  T acc[kRPT];
  T lu[kRPT];
  double tr = 0.0, ne = 0.0, ms = 0.0;
#pragma unroll
  for (int r = 0; r < kRPT; ++r) {
    const int p = p0 + threadIdx.x + r * kTI;
    acc[r] = 0;
    lu[r] = 0;
#pragma unroll
    for (int k = 0; k < DM; ++k) pr[r][k] = (p < V.np && k < d && !dense_cost) ? ldpt<T>(V.P32, V.P64, (int64_t)p * d + k) : (T)0;
    if (MODE == 1 && p < V.np) lu[r] = urow[p];
  }
  T llu[kRPT];
#pragma unroll
  for (int r = 0; r < kRPT; ++r) llu[r] = (MODE == 1 && lu[r] > (T)0) ? log(lu[r]) : (T)0;
  for (int q0 = q_begin; q0 < q_end; q0 += kTJ) {
    const int qn = min(kTJ, q_end - q0);
    __syncthreads();
    if (!dense_cost)
      for (int t = threadIdx.x; t < qn * d; t += kTI) {
        const int qq = t / d, k = t - qq * d;
        qs[qq * DM + k] = ldpt<T>(V.Q32, V.Q64, (int64_t)(q0 + qq) * d + k);
      }
    for (int t = threadIdx.x; t < qn; t += kTI) {
      const T wv = (MODE == 0) ? w[q0 + t] : ((const T*)A.v)[q0 + t];
      ws[t] = wv;
      if (MODE == 1) lws[t] = wv > (T)0 ? log(wv) : (T)0;
    }
    __syncthreads();
    T ttr = 0, tne = 0, tms = 0;   // per-tile sums (mode 1), added to FP64 per tile
    for (int qq = 0; qq < qn; ++qq) {
      const T wq = ws[qq];
#pragma unroll
      for (int r = 0; r < kRPT; ++r) {
        const int p = p0 + threadIdx.x + r * kTI;
        T D = 0;
        if (dense_cost) {
          if (p < V.np) {
            const int64_t off = V.transposed ? (int64_t)(q0 + qq) * V.m_orig + p : (int64_t)p * V.m_orig + q0 + qq;
            D = ldpt<T>(V.C32, V.C64, off);
          }
        } else {
#pragma unroll
          for (int k = 0; k < DM; ++k) {
            if (EXACT || k < d) {
              const T t = pr[r][k] - qs[qq * DM + k];
              D = fma(t, t, D);
            }
          }
        }
        const T K = gibbs<T>(D, k2);
        if (MODE == 0) {
          acc[r] = fma(K, wq, acc[r]);
        } else if (p < V.np) {
          const T Tpq = lu[r] * K * wq;
          if (Tpq > (T)0) {
            const T C = D * inv_dn;
            ttr += Tpq * C;
            tne += Tpq * (llu[r] + lws[qq] - C * inv_eps - (T)1);
            tms += Tpq;
          }
        }
      }
    }
    if (MODE == 1) { tr += (double)ttr; ne += (double)tne; ms += (double)tms; }
  }
  if (MODE == 0) {
    T* out = (T*)A.out;
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
      const int p = p0 + threadIdx.x + r * kTI;
      if (p < V.np) out[(size_t)blockIdx.y * V.np + p] = acc[r];
    }
  } else {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    const double vals[3] = {tr, ne, ms};
    for (int k = 0; k < 3; ++k) {
      const double s = block_sum_d(vals[k], sh);
      if (threadIdx.x == 0) A.part[(size_t)k * A.nblk_total + b] = s;
      __syncthreads();
    }
  }
}

template <typename T> __device__ __forceinline__ T powD(T x, T y);
template <> __device__ __forceinline__ float powD<float>(float x, float y) { return powf(x, y); }
template <> __device__ __forceinline__ double powD<double>(double x, double y) { return pow(x, y); }

// Row update: q = sum of split partials; residual of (u^t, v^t); u^{t+1}.
template <typename T, bool UOT>
__global__ void k_dense_row_update(int n, int nsplit, const T* qpart, T* ubuf, const T* a, double phi_d,
                                   double tol, int stop_rule, Ctrl* ctrl, double* part, int nblk) {
  if (ctrl->done) return;
  __shared__ double sh[32];
  const int t = ctrl->t;
  const T* uold = ubuf + (size_t)(t & 1) * n;
  T* unew = ubuf + (size_t)((t + 1) & 1) * n;
  const T phi = (T)phi_d, inv_phi = (T)(1.0 / phi_d);
  double res = 0.0, unr = 0.0, dl = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T q = 0;
    for (int s = 0; s < nsplit; ++s) q += qpart[(size_t)s * n + i];
    const T ai = a[i], uo = uold[i];
    T un;
    if (q > (T)0) {
      un = UOT ? powD<T>(ai / q, phi) : ai / q;
      res += fabs((double)((UOT ? powD<T>(uo, inv_phi) : uo) * q) - (double)ai);
    } else {
      un = 0;
      unr += (double)ai;
    }
    dl += fabs((double)un - (double)uo);
    unew[i] = un;
  }
  res = block_sum_d(res, sh);
  __syncthreads();
  unr = block_sum_d(unr, sh);
  __syncthreads();
  dl = block_sum_d(dl, sh);
  if (threadIdx.x == 0) {
    part[0 * (size_t)nblk + blockIdx.x] = res;
    part[1 * (size_t)nblk + blockIdx.x] = unr;
    part[2 * (size_t)nblk + blockIdx.x] = dl;
  }
  if (!last_block_d(&ctrl->blocks_a)) return;
  __shared__ double outv[3];
  reduce_parts_d(part, nblk, 3, outv, sh);
  if (threadIdx.x == 0) {
    ctrl->last_residual = outv[0];
    ctrl->last_unreach_a = outv[1];
    ctrl->delta_u = outv[2];
    if (stop_rule == SPS_STOP_RESIDUAL) {
      if (!isfinite(outv[0])) { ctrl->done = 1; ctrl->status = SPS_ERR_NUMERIC; ctrl->iters = t; ctrl->residual = outv[0]; }
      else if (t >= 1 && outv[0] <= tol) { ctrl->done = 1; ctrl->iters = t; ctrl->residual = outv[0]; ctrl->unreach_a = outv[1]; }
    }
    ctrl->blocks_a = 0u;
  }
}

template <typename T, bool UOT>
__global__ void k_dense_col_update(int m, int nsplit, const T* rpart, T* v, const T* b, double phi_d,
                                   double tol, int stop_rule, Ctrl* ctrl, double* part, int nblk) {
  if (ctrl->done) return;
  __shared__ double sh[32];
  const T phi = (T)phi_d;
  double unb = 0.0, dl = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    T r = 0;
    for (int s = 0; s < nsplit; ++s) r += rpart[(size_t)s * m + j];
    const T bj = b[j], vo = v[j];
    T vn;
    if (r > (T)0) vn = UOT ? powD<T>(bj / r, phi) : bj / r;
    else { vn = 0; unb += (double)bj; }
    dl += fabs((double)vn - (double)vo);
    v[j] = vn;
  }
  unb = block_sum_d(unb, sh);
  __syncthreads();
  dl = block_sum_d(dl, sh);
  if (threadIdx.x == 0) {
    part[3 * (size_t)nblk + blockIdx.x] = unb;
    part[4 * (size_t)nblk + blockIdx.x] = dl;
  }
  if (!last_block_d(&ctrl->blocks_b)) return;
  __shared__ double outv[2];
  reduce_parts_d(part + 3 * (size_t)nblk, nblk, 2, outv, sh);
  if (threadIdx.x == 0) {
    ctrl->unreach_b = outv[0];
    const int tn = ctrl->t + 1;
    ctrl->t = tn;
    if (stop_rule == SPS_STOP_DELTA_UV) {
      const double tot = ctrl->delta_u + outv[1];
      if (!isfinite(tot)) { ctrl->done = 1; ctrl->status = SPS_ERR_NUMERIC; ctrl->iters = tn; ctrl->residual = tot; }
      else if (tot <= tol) { ctrl->done = 1; ctrl->iters = tn; ctrl->residual = tot; ctrl->unreach_a = ctrl->last_unreach_a; }
    }
    ctrl->blocks_b = 0u;
  }
}

__device__ __forceinline__ double kl_elem(double x, double y) {
  if (x == 0.0) return y;
  if (y == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  return x * log(x / y) - x + y;
}

// Totals of the objective: terms from the mode-1 partials; KL terms from the
// row sums u_i (K v)_i and column sums v_j (K^T u)_j.
template <typename T>
__global__ void k_dense_final(const double* part, int nblk_pass, DevResult* out, const Ctrl* ctrl, const T* ubuf,
                              const T* v, const T* qrow, const T* rcol, int nsr, int nsc, int n, int m, const T* a,
                              const T* b) {
  __shared__ double sh[32];
  const T* u = ubuf + (size_t)(returned_iter(ctrl) & 1) * n;
  double r3[3];
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int bb = threadIdx.x; bb < nblk_pass; bb += blockDim.x) s += part[(size_t)k * nblk_pass + bb];
    s = block_sum_d(s, sh);
    __syncthreads();
    r3[k] = s;
  }
  double kla = 0.0, klb = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T q = 0;
    for (int s = 0; s < nsr; ++s) q += qrow[(size_t)s * n + i];
    kla += kl_elem((double)u[i] * (double)q, (double)a[i]);
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    T r = 0;
    for (int s = 0; s < nsc; ++s) r += rcol[(size_t)s * m + j];
    klb += kl_elem((double)v[j] * (double)r, (double)b[j]);
  }
  kla = block_sum_d(kla, sh);
  __syncthreads();
  klb = block_sum_d(klb, sh);
  if (threadIdx.x == 0) {
    out->transport = r3[0]; out->neg_entropy = r3[1]; out->mass = r3[2]; out->logp = 0.0;
    out->kl_a = kla; out->kl_b = klb;
    out->residual = ctrl->done ? ctrl->residual : ctrl->last_residual;
    out->unreach_a = ctrl->done ? ctrl->unreach_a : ctrl->last_unreach_a;
    out->unreach_b = ctrl->unreach_b;
  }
}

template <typename T>
__global__ void k_dense_potentials(int n, int m, const T* ubuf, const T* v, double eps, const Ctrl* ctrl, T* al, T* be) {
  const T* u = ubuf + (size_t)(returned_iter(ctrl) & 1) * n;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) al[i] = (T)(eps * log((double)u[i]));
  for (int64_t j = tid; j < m; j += stride) be[j] = (T)(eps * log((double)v[j]));
}

PassArgs base_args(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic) {
  PassArgs A{};
  A.sc = at<SketchScalars>(ws, L.scal);
  A.eps = ic.eps;
  A.ubuf = ws + L.u;
  A.n_u = pd.n;
  A.ctrl = at<Ctrl>(ws, L.ctrl);
  A.part = at<double>(ws, L.part);
  return A;
}

template <typename T, int DM, int MODE>
void pass(const PassArgs& A, const Geo& g, cudaStream_t st) {
  if (A.V.d == DM || A.V.C32 || A.V.C64) k_dense_pass<T, DM, true, MODE><<<g.grid, kTI, 0, st>>>(A);
  else k_dense_pass<T, DM, false, MODE><<<g.grid, kTI, 0, st>>>(A);
}

template <typename T, int DM>
void dense_iteration_t(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, bool row_only, cudaStream_t st) {
  Ctrl* ctrl = at<Ctrl>(ws, L.ctrl);
  double* part = at<double>(ws, L.part);
  const int nb = L.nblk_rows;
  const Geo gr = geometry(pd.n, pd.m), gc = geometry(pd.m, pd.n);
  PassArgs A = base_args(pd, L, ws, ic);
  A.V = view_rows(pd); A.w = ws + L.v; A.wsel = 0; A.out = ws + L.qpart; A.qchunk = gr.qchunk; A.gate = 1;
  pass<T, DM, 0>(A, gr, st);
  if (ic.uot) k_dense_row_update<T, true><<<nb, 256, 0, st>>>(pd.n, gr.nsplit, at<T>(ws, L.qpart), at<T>(ws, L.u), at<T>(ws, L.a_it), ic.phi, ic.tol, ic.stop_rule, ctrl, part, nb);
  else k_dense_row_update<T, false><<<nb, 256, 0, st>>>(pd.n, gr.nsplit, at<T>(ws, L.qpart), at<T>(ws, L.u), at<T>(ws, L.a_it), ic.phi, ic.tol, ic.stop_rule, ctrl, part, nb);
  if (row_only) return;
  PassArgs B = base_args(pd, L, ws, ic);
  B.V = view_cols(pd); B.wsel = 1; B.out = ws + L.rpart; B.qchunk = gc.qchunk; B.gate = 1;
  pass<T, DM, 0>(B, gc, st);
  if (ic.uot) k_dense_col_update<T, true><<<nb, 256, 0, st>>>(pd.m, gc.nsplit, at<T>(ws, L.rpart), at<T>(ws, L.v), at<T>(ws, L.b_it), ic.phi, ic.tol, ic.stop_rule, ctrl, part, nb);
  else k_dense_col_update<T, false><<<nb, 256, 0, st>>>(pd.m, gc.nsplit, at<T>(ws, L.rpart), at<T>(ws, L.v), at<T>(ws, L.b_it), ic.phi, ic.tol, ic.stop_rule, ctrl, part, nb);
}

template <typename T, int DM>
void dense_objective_t(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, void* al, void* be, cudaStream_t st) {
  const Geo gr = geometry(pd.n, pd.m), gc = geometry(pd.m, pd.n);
  PassArgs A = base_args(pd, L, ws, ic);
  A.V = view_rows(pd); A.w = ws + L.v; A.wsel = 0; A.out = ws + L.qpart; A.qchunk = gr.qchunk; A.gate = 0;
  pass<T, DM, 0>(A, gr, st);                     // (K v)_i with the returned v
  PassArgs B = base_args(pd, L, ws, ic);
  B.V = view_cols(pd); B.wsel = 2; B.out = ws + L.rpart; B.qchunk = gc.qchunk; B.gate = 0;
  pass<T, DM, 0>(B, gc, st);                     // (K^T u)_j with the returned u
  PassArgs M = base_args(pd, L, ws, ic);
  M.V = view_rows(pd); M.v = ws + L.v; M.qchunk = gr.qchunk; M.gate = 0; M.nblk_total = gr.grid.x * gr.grid.y;
  pass<T, DM, 1>(M, gr, st);                     // transport, neg_entropy, mass
  k_dense_final<T><<<1, 256, 0, st>>>(at<double>(ws, L.part), M.nblk_total, at<DevResult>(ws, L.res),
                                      at<Ctrl>(ws, L.ctrl), at<T>(ws, L.u), at<T>(ws, L.v), at<T>(ws, L.qpart),
                                      at<T>(ws, L.rpart), gr.nsplit, gc.nsplit, pd.n, pd.m, at<T>(ws, L.a_it),
                                      at<T>(ws, L.b_it));
  if (al && be) {
    const int g = (int)std::min<int64_t>(4096, (std::max(pd.n, pd.m) + 255) / 256);
    k_dense_potentials<T><<<std::max(g, 1), 256, 0, st>>>(pd.n, pd.m, at<T>(ws, L.u), at<T>(ws, L.v), ic.eps,
                                                          at<Ctrl>(ws, L.ctrl), (T*)al, (T*)be);
  }
}

template <typename T>
void dense_dispatch(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int what, void* al, void* be,
                    cudaStream_t st) {
  const int d = (pd.cv.C32 || pd.cv.C64) ? 1 : pd.d;
#define SPS_DENSE_CASE(DMV)                                              \
  if (what == 0) dense_iteration_t<T, DMV>(pd, L, ws, ic, false, st);    \
  else if (what == 1) dense_iteration_t<T, DMV>(pd, L, ws, ic, true, st); \
  else dense_objective_t<T, DMV>(pd, L, ws, ic, al, be, st);
  if (d <= 2) { SPS_DENSE_CASE(2) }
  else if (d == 3) { SPS_DENSE_CASE(3) }
  else if (d <= 4) { SPS_DENSE_CASE(4) }
  else if (d == 5) { SPS_DENSE_CASE(5) }
  else if (d <= 8) { SPS_DENSE_CASE(8) }
  else if (d == 10) { SPS_DENSE_CASE(10) }
  else { SPS_DENSE_CASE(16) }
#undef SPS_DENSE_CASE
}

}  // namespace

// Split-partial buffer sizes (elements of the iterate type) for the layout.
size_t dense_qpart_elems(int n, int m) { return (size_t)geometry(n, m).nsplit * (size_t)n; }
size_t dense_rpart_elems(int n, int m) { return (size_t)geometry(m, n).nsplit * (size_t)m; }
int dense_pass_blocks(int n, int m) {
  const Geo a = geometry(n, m), b = geometry(m, n);
  return std::max((int)(a.grid.x * a.grid.y), (int)(b.grid.x * b.grid.y));
}

sps_status launch_dense_iterations(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters,
                                   cudaStream_t st) {
  for (int k = 0; k < iters; ++k) {
    if (ic.it64) dense_dispatch<double>(pd, L, ws, ic, 0, nullptr, nullptr, st);
    else dense_dispatch<float>(pd, L, ws, ic, 0, nullptr, nullptr, st);
  }
  add_launches(4 * iters);
  return cuda_fail(cudaGetLastError(), "dense iteration");
}

sps_status launch_dense_row_only(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, cudaStream_t st) {
  if (ic.it64) dense_dispatch<double>(pd, L, ws, ic, 1, nullptr, nullptr, st);
  else dense_dispatch<float>(pd, L, ws, ic, 1, nullptr, nullptr, st);
  add_launches(2);
  return cuda_fail(cudaGetLastError(), "dense row pass");
}

sps_status launch_dense_objective(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, void* alpha_out,
                                  void* beta_out, cudaStream_t st) {
  if (ic.it64) dense_dispatch<double>(pd, L, ws, ic, 2, alpha_out, beta_out, st);
  else dense_dispatch<float>(pd, L, ws, ic, 2, alpha_out, beta_out, st);
  add_launches((alpha_out && beta_out) ? 5 : 4);
  return cuda_fail(cudaGetLastError(), "dense objective");
}

}  // namespace sps
