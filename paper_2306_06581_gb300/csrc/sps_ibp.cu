// sps_ibp.cu -- Spar-IBP: fixed-support Wasserstein barycenters by iterative
// Bregman projections on sketched kernels (the paper's appendix on
// barycenters; IBP after Benamou et al. 2015).
//
// The M sketches are drawn by the library's own sparsifier (sparsify_kernel:
// Eq. (pois) with Eq. (pij-ot) for a = 1/n and b = b_k, Philox problem id
// problem_id + k), each in its own slice of the caller's workspace.  The
// iterations run in one persistent cooperative kernel with two grid barriers
// per iteration:
//   phase 1 (columns of every sketch): v_k = b_k / (K~_k^T u_k), a warp per
//           (k, column);
//   phase 2 (rows): a warp per row i forms (K~_k v_k)_i for every k, then
//           q_i = prod_k (K~_k v_k)_i^{w_k} (0 if a factor is 0), then
//           u_{k,i} = q_i / (K~_k v_k)_i, and adds |q_i - q_i^{prev}| to the
//           block's partial of ||q^t - q^{t-1}||_1.
// After the second barrier every block sums the same partials and takes the
// same stopping decision (||q^t - q^{t-1}||_1 <= tol).  Accumulations run in
// the iterate type (FP64 for F64 values, else FP32); the block partials and
// the stopping sum are FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sps_internal.h"
#include "sps_iterdev.cuh"

namespace sps {
namespace {

using namespace iterdev;

constexpr int kIbpThreads = 256;
constexpr int kIbpMaxMeasures = 64;

// One sketch's arrays (views into its workspace slice).
template <typename V>
struct IbpSk {
  const int *rp, *ci, *cp, *ri;
  const V *val, *valT;
};

template <typename V, typename T>
struct IbpArgs {
  int n, M;
  const IbpSk<V>* sk;   // M sketches (device)
  const T* b;           // M x n measures in the iterate type
  const double* w;      // M weights
  T* u;                 // M x n
  T* v;                 // M x n
  T* q;                 // 2 x n: q^t at (t & 1)
  double* part;         // block partials of ||q^t - q^{t-1}||_1
  Ctrl* ctrl;
  double tol;
  int nblk;
};

// Byte offsets of the Spar-IBP workspace: header, then one slice per sketch.
struct IbpLayout {
  size_t ctrl, a, w, sk, b, u, v, q, part, sub0, sub_bytes, total;
};

template <typename V, typename T>
__device__ __forceinline__ T seg_dot(const int* idx, const V* val, const T* x, int lo, int hi, int lane) {
  T acc = (T)0;
  for (int e = lo + lane; e < hi; e += 32) acc += load_as<T>(val + e) * x[idx[e]];
  return warp_sum(acc);
}

template <typename V, typename T>
__global__ void __launch_bounds__(kIbpThreads) k_ibp(IbpArgs<V, T> A, int iters) {
  __shared__ double sh[32];
  __shared__ int stop_sh;
  Ctrl* ctrl = A.ctrl;
  if (ctrl->done) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int n = A.n, M = A.M;
  int t = ctrl->t;
  for (int it = 0; it < iters; ++it) {
    // phase 1: v_k = b_k / (K~_k^T u_k)
    for (int c = gw; c < M * n; c += nw) {
      const int k = c / n, j = c - k * n;
      const IbpSk<V> s = A.sk[k];
      const T r = seg_dot<V, T>(s.ri, s.valT, A.u + (size_t)k * n, s.cp[j], s.cp[j + 1], lane);
      if (lane == 0) A.v[(size_t)k * n + j] = r > (T)0 ? A.b[(size_t)k * n + j] / r : (T)0;
    }
    if (!grid_barrier(ctrl)) return;
    // phase 2: q = prod_k (K~_k v_k)^{w_k}, u_k = q / (K~_k v_k)
    const T* qold = A.q + (size_t)(t & 1) * n;
    T* qnew = A.q + (size_t)((t + 1) & 1) * n;
    double dsum = 0.0;
    for (int i = gw; i < n; i += nw) {
      T logq = (T)0;
      bool zero = false;
      for (int k = 0; k < M; ++k) {
        const IbpSk<V> s = A.sk[k];
        const T kv = seg_dot<V, T>(s.ci, s.val, A.v + (size_t)k * n, s.rp[i], s.rp[i + 1], lane);
        if (lane == 0) A.u[(size_t)k * n + i] = kv;   // u_k is free after phase 1: hold K~_k v_k there
        if (kv > (T)0) logq += (T)A.w[k] * log(kv);
        else zero = true;
      }
      const T qi = zero ? (T)0 : exp(logq);
      if (lane == 0) {
        qnew[i] = qi;
        dsum += fabs((double)qi - (double)qold[i]);
        for (int k = 0; k < M; ++k) {
          const T kv = A.u[(size_t)k * n + i];
          A.u[(size_t)k * n + i] = kv > (T)0 ? qi / kv : (T)0;
        }
      }
    }
    const double bs = block_sum_d(dsum, sh);
    if (threadIdx.x == 0) A.part[blockIdx.x] = bs;
    if (!grid_barrier(ctrl)) return;
    // every block sums the same partials in the same order and takes the same decision
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int b = threadIdx.x; b < A.nblk; b += 32) s += __ldcg(A.part + b);
      s = warp_sum(s);
      if (threadIdx.x == 0) {
        const int numeric = !isfinite(s);
        stop_sh = (numeric || s <= A.tol) ? 1 : 0;
        if (blockIdx.x == 0) {
          ctrl->last_residual = s;
          ctrl->t = t + 1;
          if (stop_sh) {
            ctrl->iters = t + 1;
            ctrl->residual = s;
            if (numeric) ctrl->status = SPS_ERR_NUMERIC;
            __threadfence();
            ctrl->done = 1;
          }
        }
      }
    }
    __syncthreads();
    ++t;
    if (stop_sh) return;
  }
}

// u = 1, q^0 = 1/n, the measures in the iterate type, the uniform source weight.
template <typename T>
__global__ void k_ibp_init(int n, int M, const void* b_in, int in64, T* b, T* u, T* q, void* a_unif, Ctrl* ctrl) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = tid; e < (int64_t)M * n; e += st) {
    b[e] = in64 ? (T) static_cast<const double*>(b_in)[e] : (T) static_cast<const float*>(b_in)[e];
    u[e] = (T)1;
  }
  for (int64_t i = tid; i < n; i += st) {
    q[i] = (T)(1.0 / (double)n);
    if (in64) static_cast<double*>(a_unif)[i] = 1.0 / (double)n;
    else static_cast<float*>(a_unif)[i] = (float)(1.0 / (double)n);
  }
  if (tid == 0) {
    const Ctrl zero = {};
    *ctrl = zero;
  }
}

// The sketch problem of measure k: a = 1/n (uniform) to b_k on the shared support.
sps_problem sub_problem(const sps_barycenter* B, const void* a_unif, int k) {
  sps_problem P;
  memset(&P, 0, sizeof(P));
  const size_t eb = B->dtype == SPS_F64 ? 8 : 4;
  P.n = B->n; P.m = B->n; P.d = B->d;
  P.x = B->x; P.y = B->x; P.C = nullptr;
  P.cost_norm = B->cost_norm; P.cost_scale = B->cost_scale;
  P.a = a_unif;
  P.b = static_cast<const char*>(B->b) + (size_t)k * B->n * eb;
  P.dtype = B->dtype;
  P.cost_kind = SPS_COST_SQEUCLID;
  return P;
}

sps_params sub_params(const sps_params* Q, int k) {
  sps_params R = *Q;
  R.problem_id = Q->problem_id + (uint32_t)k;
  return R;
}

sps_status validate_ibp(const sps_barycenter* B, const sps_params* Q) {
  if (!B || !Q) { set_error("null barycenter problem or params"); return SPS_ERR_INVALID_ARG; }
  if (B->n < 1 || B->d < 1) { set_error("support size n and dimension d must be >= 1"); return SPS_ERR_INVALID_ARG; }
  if (B->n_measures < 1 || B->n_measures > kIbpMaxMeasures) {
    set_error("n_measures must be in 1 .. %d (got %d)", kIbpMaxMeasures, B->n_measures); return SPS_ERR_INVALID_ARG;
  }
  if (!B->x || !B->b || !B->w) { set_error("support x, measures b and weights w are required"); return SPS_ERR_INVALID_ARG; }
  if (B->dtype != SPS_F32 && B->dtype != SPS_F64) { set_error("barycenter dtype must be F32 or F64"); return SPS_ERR_INVALID_ARG; }
  double sw = 0.0;
  for (int k = 0; k < B->n_measures; ++k) {
    if (!(B->w[k] >= 0.0) || !isfinite(B->w[k])) { set_error("weight w[%d] must be finite and >= 0", k); return SPS_ERR_INVALID_ARG; }
    sw += B->w[k];
  }
  if (!(fabs(sw - 1.0) <= 1e-9)) { set_error("the weights must sum to 1 (sum %.17g)", sw); return SPS_ERR_INVALID_ARG; }
  if (!isinf(Q->lambda) || Q->lambda < 0) { set_error("Spar-IBP sketches balanced-OT kernels: lambda must be +inf"); return SPS_ERR_INVALID_ARG; }
  if (Q->log_domain) { set_error("Spar-IBP iterates in the plain domain (log_domain 0)"); return SPS_ERR_INVALID_ARG; }
  if (Q->probs != SPS_PROBS_PAPER) { set_error("Spar-IBP samples with Eq. (pij-ot) (probs 0)"); return SPS_ERR_INVALID_ARG; }
  if (Q->stop_rule != SPS_STOP_RESIDUAL) { set_error("Spar-IBP stops on ||q^t - q^{t-1}||_1 (stop_rule 0)"); return SPS_ERR_INVALID_ARG; }
  if (Q->max_iter < 1) { set_error("max_iter must be >= 1"); return SPS_ERR_INVALID_ARG; }
  return SPS_OK;
}

bool plan_ibp(const sps_barycenter* B, const sps_params* Q, IbpLayout* L) {
  memset(L, 0, sizeof(*L));
  const int n = B->n, M = B->n_measures;
  const size_t it = Q->kdtype == SPS_F64 ? 8 : 4;
  const size_t eb = B->dtype == SPS_F64 ? 8 : 4;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  L->ctrl = take(sizeof(Ctrl));
  L->a = take((size_t)n * eb);
  L->w = take((size_t)M * sizeof(double));
  L->sk = take((size_t)M * sizeof(IbpSk<double>));
  L->b = take((size_t)M * n * it);
  L->u = take((size_t)M * n * it);
  L->v = take((size_t)M * n * it);
  L->q = take((size_t)2 * n * it);
  L->part = take((size_t)kMaxBlocks * sizeof(double));
  // every sketch slice has the size of one sparsify_kernel workspace (the same for all k)
  const sps_problem P0 = sub_problem(B, B->x /* any non-null pointer: sizes only */, 0);
  const sps_params Q0 = sub_params(Q, 0);
  const size_t sub = sps_workspace_bytes(&P0, &Q0, SPS_OP_SPARSIFY);
  if (sub == 0) return false;
  L->sub_bytes = (sub + 255) & ~(size_t)255;
  L->sub0 = off;
  L->total = off + (size_t)M * L->sub_bytes + 256;
  return true;
}

template <typename V, typename T>
bool coop_ibp(IbpArgs<V, T> A, int iters, cudaStream_t st) {
  auto fn = k_ibp<V, T>;
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kIbpThreads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  const int want = (int)std::max<int64_t>(1, ((int64_t)A.M * A.n * 32 + kIbpThreads - 1) / kIbpThreads);
  A.nblk = std::min(std::min(nsm * per_sm, kMaxBlocks), want);
  void* args[] = {(void*)&A, (void*)&iters};
  if (cudaLaunchCooperativeKernel((const void*)fn, dim3(A.nblk), dim3(kIbpThreads), args, 0, st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

struct Ev2 {
  cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
  Ev2() { for (auto& x : e) cudaEventCreate(&x); }
  ~Ev2() { for (auto& x : e) if (x) cudaEventDestroy(x); }
  float ms(int a, int b) const {
    float v = 0.0f;
    return cudaEventElapsedTime(&v, e[a], e[b]) == cudaSuccess ? v : 0.0f;
  }
};

template <typename V, typename T>
sps_status ibp_run(const sps_barycenter* B, const sps_params* Q, const IbpLayout& L, char* ws, void* q_out,
                   sps_result* res, cudaStream_t st) {
  const int n = B->n, M = B->n_measures;
  Ev2 ev;
  cudaEventRecord(ev.e[0], st);
  // uniform source weight, measures in the iterate type, u = 1, q^0 = 1/n
  k_ibp_init<T><<<std::max(1, std::min(2048, (int)(((int64_t)M * n + 255) / 256))), 256, 0, st>>>(
      n, M, B->b, B->dtype == SPS_F64, at<T>(ws, L.b), at<T>(ws, L.u), at<T>(ws, L.q), ws + L.a, at<Ctrl>(ws, L.ctrl));
  add_launches(1);
  SPS_TRY(cuda_fail(cudaGetLastError(), "barycenter init"));
  // the M sketches, each by the library's sparsifier in its own workspace slice
  std::vector<IbpSk<V>> sk(M);
  int64_t nnz = 0;
  for (int k = 0; k < M; ++k) {
    const sps_problem P = sub_problem(B, ws + L.a, k);
    const sps_params R = sub_params(Q, k);
    sps_sketch out;
    SPS_TRY(sparsify_kernel(&P, &R, ws + L.sub0 + (size_t)k * L.sub_bytes, L.sub_bytes, &out, (sps_stream)st));
    sk[k] = IbpSk<V>{out.row_ptr, out.col_idx, out.col_ptr, out.row_idx, static_cast<const V*>(out.val),
                     static_cast<const V*>(out.valT)};
    nnz += out.nnz;
  }
  SPS_TRY(cuda_fail(cudaMemcpyAsync(ws + L.sk, sk.data(), sizeof(IbpSk<V>) * M, cudaMemcpyHostToDevice, st), "sketch table"));
  SPS_TRY(cuda_fail(cudaMemcpyAsync(ws + L.w, B->w, sizeof(double) * M, cudaMemcpyHostToDevice, st), "weights"));
  cudaEventRecord(ev.e[1], st);
  IbpArgs<V, T> A;
  A.n = n; A.M = M;
  A.sk = at<IbpSk<V>>(ws, L.sk);
  A.b = at<T>(ws, L.b);
  A.w = at<double>(ws, L.w);
  A.u = at<T>(ws, L.u);
  A.v = at<T>(ws, L.v);
  A.q = at<T>(ws, L.q);
  A.part = at<double>(ws, L.part);
  A.ctrl = at<Ctrl>(ws, L.ctrl);
  A.tol = Q->tol;
  A.nblk = 0;
  Ctrl h;
  int launched = 0, chunk = Q->check_every > 0 ? Q->check_every : 32;
  for (;;) {
    const int k = std::min(chunk, Q->max_iter - launched);
    if (k <= 0) break;
    if (!coop_ibp<V, T>(A, k, st)) {
      set_error("the device refused the cooperative launch of the Spar-IBP iterations");
      return SPS_ERR_CUDA;
    }
    add_launches(1);
    launched += k;
    SPS_TRY(cuda_fail(cudaMemcpyAsync(&h, ws + L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "ctrl read-back"));
    SPS_TRY(cuda_fail(cudaStreamSynchronize(st), "stream synchronize"));
    if (h.done || launched >= Q->max_iter) break;
    if (Q->check_every <= 0) chunk = std::min(chunk * 2, 4096);
  }
  cudaEventRecord(ev.e[2], st);
  const int T_ = h.done ? h.iters : h.t;
  if (q_out)
    SPS_TRY(cuda_fail(cudaMemcpyAsync(q_out, ws + L.q + (size_t)(T_ & 1) * n * sizeof(T), sizeof(T) * n,
                                      cudaMemcpyDeviceToDevice, st), "barycenter copy"));
  SPS_TRY(cuda_fail(cudaStreamSynchronize(st), "stream synchronize"));
  if (h.wait_timeout) { set_error("a device-side grid barrier of the Spar-IBP kernel timed out"); return SPS_ERR_CUDA; }
  sps_result r;
  memset(&r, 0, sizeof(r));
  r.iters = T_;
  r.residual = h.done ? h.residual : h.last_residual;
  r.nnz = nnz;
  r.ms_sketch = ev.ms(0, 1);
  r.ms_iter = ev.ms(1, 2);
  r.iters_enqueued = launched;
  r.status = h.status != SPS_OK ? h.status : (h.done ? SPS_OK : SPS_NOT_CONVERGED);
  if (res) *res = r;
  if (r.status == SPS_ERR_NUMERIC) set_error("non-finite value in the Spar-IBP iterates");
  return (sps_status)r.status;
}

}  // namespace
}  // namespace sps

using namespace sps;

extern "C" size_t sps_ibp_workspace_bytes(const sps_barycenter* bar, const sps_params* prm) {
  if (validate_ibp(bar, prm) != SPS_OK) return 0;
  IbpLayout L;
  if (!plan_ibp(bar, prm, &L)) return 0;
  return L.total;
}

extern "C" sps_status spar_ibp(const sps_barycenter* bar, const sps_params* prm, void* wsv, size_t ws_bytes,
                               void* q_out, sps_result* res, sps_stream stream) {
  SPS_TRY(validate_ibp(bar, prm));
  if (!wsv) { set_error("null workspace"); return SPS_ERR_INVALID_ARG; }
  IbpLayout L;
  if (!plan_ibp(bar, prm, &L)) return SPS_ERR_INVALID_ARG;   // message set by the sketch's checks
  if (ws_bytes < L.total) { set_error("workspace too small: %zu < %zu", ws_bytes, L.total); return SPS_ERR_WORKSPACE; }
  char* ws = (char*)(((uintptr_t)wsv + 255) & ~(uintptr_t)255);
  cudaStream_t st = (cudaStream_t)stream;
  switch (prm->kdtype) {
    case SPS_F64: return ibp_run<double, double>(bar, prm, L, ws, q_out, res, st);
    case SPS_BF16: return ibp_run<__nv_bfloat16, float>(bar, prm, L, ws, q_out, res, st);
    case SPS_F16: return ibp_run<__half, float>(bar, prm, L, ws, q_out, res, st);
    default: return ibp_run<float, float>(bar, prm, L, ws, q_out, res, st);
  }
}
