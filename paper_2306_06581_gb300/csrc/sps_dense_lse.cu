// sps_dense_lse.cu -- dense Sinkhorn in log-sum-exp form (log_domain = 1),
// for the small eps at which exp(-C/eps) leaves the binary32 range.
//
// The iterates are the potentials alpha = eps log u, beta = eps log v of
// Alg. 1 / Alg. 2 (binary32).  A row pass computes, for every row i,
//   log r_i = LSE_j ((alpha_i / phi + beta_j - C_ij) / eps)
// = log (u_i^{1/phi} (K v)_i), the quantity of the stopping residual, with an
// online maximum (one rescale whenever a larger exponent appears) and
// per-tile partial sums.  The update is then
//   alpha_i <- alpha_i + phi eps (log a_i - log r_i),
// which is Alg. 2's u = (a / K v)^phi written in potentials (phi = 1: Alg. 1),
// and the residual of the incoming pair is sum_i |r_i - a_i|.  The exponent
// is formed as (alpha_i/phi + beta_j - C_ij) * log2(e)/eps with the cost
// subtracted by one fused multiply-add first, so that the terms that matter
// (exponent near 0) carry no large rounding error.  Columns are symmetric.
// K is recomputed from the points in every pass and never stored.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "sps_dense.cuh"
#include "sps_internal.h"

namespace sps {

namespace {

using namespace dense;

constexpr float kLn2F = 0.6931471805599453f;
constexpr float kNegBig = -1.0e30f;   // initial running maximum (finite, so -inf exponents give 0 terms)

struct LseArgs {
  DenseView V;
  const SketchScalars* sc;
  float eps;
  float shift_mul;        // 1/phi in an iteration, 1 for the plan's own sums
  const float* abuf;      // alpha of two pairs (2 x n), by the parity of t
  int n;
  const float* beta;      // beta (m)
  int asel;               // alpha of 0: pair t, 1: pair t+1, 2: the returned pair
  float* out;             // [2][nsplit][np]: running maximum (log2 units), then scaled sum
  int qchunk, nsplit;
  int gate;               // 1: skip when the solve has stopped
  const Ctrl* ctrl;
  double* part;           // objective pass: 3 x nblk_total block partials
  int nblk_total;
};

__device__ __forceinline__ int returned_pair(const Ctrl* c) { return c->done ? c->iters : c->t; }

__device__ __forceinline__ const float* alpha_of(const LseArgs& A) {
  const int t = A.asel == 2 ? returned_pair(A.ctrl) : A.ctrl->t + A.asel;
  return A.abuf + (size_t)(t & 1) * A.n;
}

// Distance of pass row p (coordinates in registers) to staged column qq.
template <int DM, bool EXACT>
__device__ __forceinline__ float pass_dist(const DenseView& V, const float (&pr)[DM], const float* qs, int p, int q,
                                           int qq, bool dense_cost) {
  float D = 0.0f;
  if (dense_cost) {
    if (p < V.np) {
      const int64_t off = V.transposed ? (int64_t)q * V.m_orig + p : (int64_t)p * V.m_orig + q;
      D = ldpt<float>(V.C32, V.C64, off);
    }
  } else {
#pragma unroll
    for (int k = 0; k < DM; ++k) {
      if (EXACT || k < V.d) {
        const float t = pr[k] - qs[qq * DM + k];
        D = fmaf(t, t, D);
      }
    }
  }
  return D;
}

// MODE 0: per (row, column split) running maximum and sum of
//         exp2((shift_p * shift_mul + other_q - C_pq) * log2(e)/eps).
// MODE 1: block partials of transport, neg_entropy and mass of
//         T_pq = exp((alpha_p + beta_q - C_pq)/eps) (rows of the original problem).
template <int DM, bool EXACT, int MODE>
__global__ void __launch_bounds__(kTI) k_lse_pass(LseArgs A) {
  if (A.gate && A.ctrl->done) return;
  __shared__ float qs[kTJ * DM];
  __shared__ float ws[kTJ];
  __shared__ double sh[32];
  const DenseView& V = A.V;
  const int d = V.d;
  const bool dense_cost = V.C32 || V.C64;
  const float* al = alpha_of(A);
  const float* shift = V.transposed ? A.beta : al;
  const float* other = V.transposed ? al : A.beta;
  const float inv_dn = (float)(1.0 / (double)A.sc->dn32);
  const float k2 = (float)(1.4426950408889634 / (double)A.eps);
  const int p0 = blockIdx.x * (kTI * kRPT);
  const int q_begin = blockIdx.y * A.qchunk;
  const int q_end = min(V.nq, q_begin + A.qchunk);
  float pr[kRPT][DM];
  float sp[kRPT], mx[kRPT], sm[kRPT];
#pragma unroll
  for (int r = 0; r < kRPT; ++r) {
    const int p = p0 + threadIdx.x + r * kTI;
#pragma unroll
    for (int k = 0; k < DM; ++k)
      pr[r][k] = (p < V.np && k < d && !dense_cost) ? ldpt<float>(V.P32, V.P64, (int64_t)p * d + k) : 0.0f;
    sp[r] = p < V.np ? shift[p] * (MODE == 0 ? A.shift_mul : 1.0f) : 0.0f;
    mx[r] = kNegBig;
    sm[r] = 0.0f;
  }
  double tr = 0.0, ne = 0.0, ms = 0.0;
  for (int q0 = q_begin; q0 < q_end; q0 += kTJ) {
    const int qn = min(kTJ, q_end - q0);
    __syncthreads();
    if (!dense_cost)
      for (int t = threadIdx.x; t < qn * d; t += kTI) {
        const int qq = t / d, k = t - qq * d;
        qs[qq * DM + k] = ldpt<float>(V.Q32, V.Q64, (int64_t)(q0 + qq) * d + k);
      }
    for (int t = threadIdx.x; t < qn; t += kTI) ws[t] = other[q0 + t];
    __syncthreads();
    float ts[kRPT], ttr = 0.0f, tne = 0.0f, tms = 0.0f;
#pragma unroll
    for (int r = 0; r < kRPT; ++r) ts[r] = 0.0f;
    for (int qq = 0; qq < qn; ++qq) {
      const float wq = ws[qq];
#pragma unroll
      for (int r = 0; r < kRPT; ++r) {
        const int p = p0 + threadIdx.x + r * kTI;
        const float D = pass_dist<DM, EXACT>(V, pr[r], qs, p, q0 + qq, qq, dense_cost);
        const float z = fmaf(-D, inv_dn, sp[r] + wq) * k2;   // log2 of the term
        if (MODE == 0) {
          if (z > mx[r]) {
            const float c = exp2f(mx[r] - z);
            sm[r] *= c;
            ts[r] *= c;
            mx[r] = z;
          }
          ts[r] += exp2f(z - mx[r]);
        } else if (p < V.np) {
          const float T = exp2f(z);
          if (T > 0.0f) {
            ttr += T * (D * inv_dn);
            tne += T * fmaf(z, kLn2F, -1.0f);
            tms += T;
          }
        }
      }
    }
    if (MODE == 0) {
#pragma unroll
      for (int r = 0; r < kRPT; ++r) sm[r] += ts[r];
    } else {
      tr += (double)ttr; ne += (double)tne; ms += (double)tms;
    }
  }
  if (MODE == 0) {
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
      const int p = p0 + threadIdx.x + r * kTI;
      if (p < V.np) {
        A.out[(size_t)blockIdx.y * V.np + p] = mx[r];
        A.out[(size_t)(A.nsplit + blockIdx.y) * V.np + p] = sm[r];
      }
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

// log2 of the total of one row over the column splits (fixed order); -inf if empty.
__device__ __forceinline__ float combine_splits(const float* out, int nsplit, int np, int i) {
  float M = kNegBig;
  for (int s = 0; s < nsplit; ++s) M = fmaxf(M, out[(size_t)s * np + i]);
  float S = 0.0f;
  for (int s = 0; s < nsplit; ++s) S += out[(size_t)(nsplit + s) * np + i] * exp2f(out[(size_t)s * np + i] - M);
  return S > 0.0f ? M + log2f(S) : __int_as_float(0xff800000);
}

// Row update: residual of the pair t and alpha of the pair t+1.
__global__ void k_lse_row_update(int n, int nsplit, const float* qpart, float* abuf, const float* a, float phi,
                                 float eps, double tol, Ctrl* ctrl, double* part, int nblk) {
  if (ctrl->done) return;
  __shared__ double sh[32];
  const int t = ctrl->t;
  const float* aold = abuf + (size_t)(t & 1) * n;
  float* anew = abuf + (size_t)((t + 1) & 1) * n;
  double res = 0.0, unr = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float l2 = combine_splits(qpart, nsplit, n, i);
    const float ai = a[i];
    float an;
    if (l2 != __int_as_float(0xff800000)) {
      const float lr = l2 * kLn2F;
      res += fabs((double)expf(lr) - (double)ai);
      an = ai > 0.0f ? aold[i] + phi * eps * (logf(ai) - lr) : __int_as_float(0xff800000);
    } else {
      an = __int_as_float(0xff800000);
      unr += (double)ai;
    }
    anew[i] = an;
  }
  res = block_sum_d(res, sh);
  __syncthreads();
  unr = block_sum_d(unr, sh);
  if (threadIdx.x == 0) {
    part[0 * (size_t)nblk + blockIdx.x] = res;
    part[1 * (size_t)nblk + blockIdx.x] = unr;
  }
  if (!last_block_d(&ctrl->blocks_a)) return;
  __shared__ double outv[2];
  reduce_parts_d(part, nblk, 2, outv, sh);
  if (threadIdx.x == 0) {
    ctrl->last_residual = outv[0];
    ctrl->last_unreach_a = outv[1];
    if (!isfinite(outv[0])) { ctrl->done = 1; ctrl->status = SPS_ERR_NUMERIC; ctrl->iters = t; ctrl->residual = outv[0]; }
    else if (t >= 1 && outv[0] <= tol) { ctrl->done = 1; ctrl->iters = t; ctrl->residual = outv[0]; ctrl->unreach_a = outv[1]; }
    ctrl->blocks_a = 0u;
  }
}

// Column update: beta of the pair t+1 (in place); advances t.
__global__ void k_lse_col_update(int m, int nsplit, const float* rpart, float* beta, const float* b, float phi,
                                 float eps, Ctrl* ctrl, double* part, int nblk) {
  if (ctrl->done) return;
  __shared__ double sh[32];
  double unb = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const float l2 = combine_splits(rpart, nsplit, m, j);
    const float bj = b[j];
    float bn;
    if (l2 != __int_as_float(0xff800000)) {
      bn = bj > 0.0f ? beta[j] + phi * eps * (logf(bj) - l2 * kLn2F) : __int_as_float(0xff800000);
    } else {
      bn = __int_as_float(0xff800000);
      unb += (double)bj;
    }
    beta[j] = bn;
  }
  unb = block_sum_d(unb, sh);
  if (threadIdx.x == 0) part[3 * (size_t)nblk + blockIdx.x] = unb;
  if (!last_block_d(&ctrl->blocks_b)) return;
  __shared__ double outv[1];
  reduce_parts_d(part + 3 * (size_t)nblk, nblk, 1, outv, sh);
  if (threadIdx.x == 0) {
    ctrl->unreach_b = outv[0];
    ctrl->t = ctrl->t + 1;
    ctrl->blocks_b = 0u;
  }
}

__global__ void k_lse_init(int n, int m, float* abuf, float* beta, const float* al0, const float* be0, Ctrl* ctrl) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) abuf[i] = al0 ? al0[i] : 0.0f;
  for (int64_t j = tid; j < m; j += stride) beta[j] = be0 ? be0[j] : 0.0f;
  if (tid == 0) {
    ctrl->t = 0; ctrl->done = 0; ctrl->iters = 0;
    ctrl->blocks_a = ctrl->blocks_b = ctrl->blocks_c = 0u;
    if (ctrl->status != SPS_OK) ctrl->done = 1;
  }
}

__device__ __forceinline__ double kl_elem_l(double x, double y) {
  if (x == 0.0) return y;
  if (y == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  return x * log(x / y) - x + y;
}

// Totals: transport, neg_entropy, mass from the objective pass; KL terms from
// the plan's row and column sums (log2 form, split partials).
__global__ void k_lse_final(const double* part, int nblk_pass, DevResult* out, const Ctrl* ctrl, const float* qrow,
                            const float* rcol, int nsr, int nsc, int n, int m, const float* a, const float* b) {
  __shared__ double sh[32];
  double r3[3];
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int bb = threadIdx.x; bb < nblk_pass; bb += blockDim.x) s += part[(size_t)k * nblk_pass + bb];
    s = block_sum_d(s, sh);
    __syncthreads();
    r3[k] = s;
  }
  double kla = 0.0, klb = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    kla += kl_elem_l(exp2((double)combine_splits(qrow, nsr, n, i)), (double)a[i]);
  for (int j = threadIdx.x; j < m; j += blockDim.x)
    klb += kl_elem_l(exp2((double)combine_splits(rcol, nsc, m, j)), (double)b[j]);
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

__global__ void k_lse_potentials(int n, int m, const float* abuf, const float* beta, const Ctrl* ctrl, float* al,
                                 float* be) {
  const float* a = abuf + (size_t)(returned_pair(ctrl) & 1) * n;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) al[i] = a[i];
  for (int64_t j = tid; j < m; j += stride) be[j] = beta[j];
}

template <int DM, int MODE>
void lse_pass(const LseArgs& A, const Geo& g, cudaStream_t st) {
  if (A.V.d == DM || A.V.C32 || A.V.C64) k_lse_pass<DM, true, MODE><<<g.grid, kTI, 0, st>>>(A);
  else k_lse_pass<DM, false, MODE><<<g.grid, kTI, 0, st>>>(A);
}

LseArgs base_lse(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic) {
  LseArgs A{};
  A.sc = at<SketchScalars>(ws, L.scal);
  A.eps = (float)ic.eps;
  A.abuf = at<float>(ws, L.u);
  A.n = pd.n;
  A.beta = at<float>(ws, L.v);
  A.ctrl = at<Ctrl>(ws, L.ctrl);
  A.part = at<double>(ws, L.part);
  return A;
}

template <int DM>
void lse_iteration(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, bool row_only, cudaStream_t st) {
  Ctrl* ctrl = at<Ctrl>(ws, L.ctrl);
  double* part = at<double>(ws, L.part);
  const int nb = L.nblk_rows;
  const Geo gr = geometry(pd.n, pd.m), gc = geometry(pd.m, pd.n);
  LseArgs A = base_lse(pd, L, ws, ic);
  A.V = view_rows(pd); A.shift_mul = (float)(1.0 / ic.phi); A.asel = 0; A.out = at<float>(ws, L.qpart);
  A.qchunk = gr.qchunk; A.nsplit = gr.nsplit; A.gate = 1;
  lse_pass<DM, 0>(A, gr, st);
  k_lse_row_update<<<nb, 256, 0, st>>>(pd.n, gr.nsplit, at<float>(ws, L.qpart), at<float>(ws, L.u),
                                       at<float>(ws, L.a_it), (float)ic.phi, (float)ic.eps, ic.tol, ctrl, part, nb);
  if (row_only) return;
  LseArgs B = base_lse(pd, L, ws, ic);
  B.V = view_cols(pd); B.shift_mul = (float)(1.0 / ic.phi); B.asel = 1; B.out = at<float>(ws, L.rpart);
  B.qchunk = gc.qchunk; B.nsplit = gc.nsplit; B.gate = 1;
  lse_pass<DM, 0>(B, gc, st);
  k_lse_col_update<<<nb, 256, 0, st>>>(pd.m, gc.nsplit, at<float>(ws, L.rpart), at<float>(ws, L.v),
                                       at<float>(ws, L.b_it), (float)ic.phi, (float)ic.eps, ctrl, part, nb);
}

template <int DM>
void lse_objective(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, void* al, void* be,
                   cudaStream_t st) {
  const Geo gr = geometry(pd.n, pd.m), gc = geometry(pd.m, pd.n);
  LseArgs A = base_lse(pd, L, ws, ic);
  A.V = view_rows(pd); A.shift_mul = 1.0f; A.asel = 2; A.out = at<float>(ws, L.qpart);
  A.qchunk = gr.qchunk; A.nsplit = gr.nsplit; A.gate = 0;
  lse_pass<DM, 0>(A, gr, st);                       // row sums of the returned plan
  LseArgs B = base_lse(pd, L, ws, ic);
  B.V = view_cols(pd); B.shift_mul = 1.0f; B.asel = 2; B.out = at<float>(ws, L.rpart);
  B.qchunk = gc.qchunk; B.nsplit = gc.nsplit; B.gate = 0;
  lse_pass<DM, 0>(B, gc, st);                       // column sums
  LseArgs M = base_lse(pd, L, ws, ic);
  M.V = view_rows(pd); M.asel = 2; M.qchunk = gr.qchunk; M.nsplit = gr.nsplit; M.gate = 0;
  M.nblk_total = gr.grid.x * gr.grid.y;
  lse_pass<DM, 1>(M, gr, st);                       // transport, neg_entropy, mass
  k_lse_final<<<1, 256, 0, st>>>(at<double>(ws, L.part), M.nblk_total, at<DevResult>(ws, L.res), at<Ctrl>(ws, L.ctrl),
                                 at<float>(ws, L.qpart), at<float>(ws, L.rpart), gr.nsplit, gc.nsplit, pd.n, pd.m,
                                 at<float>(ws, L.a_it), at<float>(ws, L.b_it));
  if (al && be) {
    const int g = (int)std::min<int64_t>(4096, (std::max(pd.n, pd.m) + 255) / 256);
    k_lse_potentials<<<std::max(g, 1), 256, 0, st>>>(pd.n, pd.m, at<float>(ws, L.u), at<float>(ws, L.v),
                                                     at<Ctrl>(ws, L.ctrl), (float*)al, (float*)be);
  }
}

void lse_dispatch(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int what, void* al, void* be,
                  cudaStream_t st) {
  const int d = (pd.cv.C32 || pd.cv.C64) ? 1 : pd.d;
#define SPS_LSE_CASE(DMV)                                              \
  if (what == 0) lse_iteration<DMV>(pd, L, ws, ic, false, st);         \
  else if (what == 1) lse_iteration<DMV>(pd, L, ws, ic, true, st);     \
  else lse_objective<DMV>(pd, L, ws, ic, al, be, st);
  if (d <= 2) { SPS_LSE_CASE(2) }
  else if (d == 3) { SPS_LSE_CASE(3) }
  else if (d <= 4) { SPS_LSE_CASE(4) }
  else if (d == 5) { SPS_LSE_CASE(5) }
  else if (d <= 8) { SPS_LSE_CASE(8) }
  else if (d == 10) { SPS_LSE_CASE(10) }
  else { SPS_LSE_CASE(16) }
#undef SPS_LSE_CASE
}

}  // namespace

sps_status launch_dense_lse_init(const ProbDev& pd, const Layout& L, char* ws, const void* init_alpha,
                                 const void* init_beta, cudaStream_t st) {
  const int g = (int)std::min<int64_t>(4096, (std::max(pd.n, pd.m) + 255) / 256);
  k_lse_init<<<std::max(g, 1), 256, 0, st>>>(pd.n, pd.m, at<float>(ws, L.u), at<float>(ws, L.v),
                                             (const float*)init_alpha, (const float*)init_beta,
                                             at<Ctrl>(ws, L.ctrl));
  add_launches(1);
  return cuda_fail(cudaGetLastError(), "dense log-domain init");
}

sps_status launch_dense_lse_iterations(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters,
                                       cudaStream_t st) {
  for (int k = 0; k < iters; ++k) lse_dispatch(pd, L, ws, ic, 0, nullptr, nullptr, st);
  add_launches(4 * iters);
  return cuda_fail(cudaGetLastError(), "dense log-domain iteration");
}

sps_status launch_dense_lse_row_only(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                     cudaStream_t st) {
  lse_dispatch(pd, L, ws, ic, 1, nullptr, nullptr, st);
  add_launches(2);
  return cuda_fail(cudaGetLastError(), "dense log-domain row pass");
}

sps_status launch_dense_lse_objective(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                      void* alpha_out, void* beta_out, cudaStream_t st) {
  lse_dispatch(pd, L, ws, ic, 2, alpha_out, beta_out, st);
  add_launches((alpha_out && beta_out) ? 5 : 4);
  return cuda_fail(cudaGetLastError(), "dense log-domain objective");
}

}  // namespace sps
