// sps_logdom.cu -- stabilised iterations for small eps (log_domain = 1).
//
// With eps = 0.01 the sketch values K~_ij = exp(-C_ij/eps)/p*_ij span more
// than the binary32 range, and so do the scalings u, v.  The solve keeps
//   - absorbed potentials alpha_i, beta_j (binary32),
//   - stored kernel values K'_ij = K~_ij exp((alpha_i + beta_j)/eps), written
//     per row (CSR) and per column (CSC) with a power-of-two scale 2^-e so that
//     the largest stored value of every row / column lies in [1, 2) (this keeps
//     BF16 and FP16 storage from flushing a whole row or column to zero),
//   - scalings u~ = u e^{-alpha/eps}, v~ = v e^{-beta/eps} around 1.
// In these variables Alg. 2 reads u~ = (a^ / (K' v~))^phi with
// a^_i = a_i e^{-alpha_i/lam} (a^ = a for OT), and the stopping residual of a
// pair is sum_i (a_i / a^_i) | u~_i^{1/phi} (K' v~)_i - a^_i |.
// log K~_ij = -C_ij/eps - log p*_ij is the sparse cost C~ = C + eps log p* of
// the UOT iteration lemma's proof divided by -eps; it is stored in binary32.
//
// The first iteration is done exactly in the log domain (log-sum-exp over
// the support, rows then columns), which gives (alpha, beta) of the pair
// (u^1, v^1); an absorb pass then writes K' and sets u~ = v~ = 1.  Later
// iterations run in a persistent cooperative kernel; when max |log u~| or
// max |log v~| exceeds tau, every block folds its scalings into alpha / beta
// and rewrites its rows and columns of K' (two extra grid barriers).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "sps_internal.h"
#include "sps_iterdev.cuh"

namespace sps {

namespace {

using namespace iterdev;

constexpr int kT = 256;
constexpr float kLog2e = 1.4426950408889634f;

struct LogArgs {
  int n, m;
  const int *row_ptr, *col_idx, *col_ptr, *row_idx;
  void *val, *valT;                // K' storage (scaled)
  const float *logval, *logvalT;   // log K~ (CSR / CSC order)
  float *ubuf, *vbuf;              // u~ (2 x n), v~ (2 x m), parity of t
  float *alpha, *beta;             // absorbed potentials
  float *ahat, *bhat;
  float *erow, *ecol;              // power-of-two exponents of stored rows / columns
  const float *a, *b;
  float eps, inv_eps, lam, inv_lam, phi, inv_phi, tol, tau;
  int uot;
  Ctrl* ctrl;
  double* part;
  int nblk;
  // staged gathers (large problems): the gathered vector passes through shared
  // memory in chunks of W entries; block b owns rows [b rows_pb, (b+1) rows_pb)
  // and columns [b cols_pb, (b+1) cols_pb); seg_r[c n + i] is the first CSR
  // position of row i with column >= c W (c = 0 .. Jr), seg_c likewise for CSC.
  int stage, W, Jr, Jc, rows_pb, cols_pb;
  const int *seg_r, *seg_c;
  // grouped copies for the staged passes (side 0: rows over the CSR, 1:
  // columns over the CSC; layout in sps_internal.h): the warp slices, the
  // parts' byte offsets, the copies themselves and, per CSR / CSC position,
  // the value slot its K' goes to.  K' is stored there instead of val / valT
  // unless ctrl->ell_overflow is set (a sketch too large for the planned copy),
  // in which case the passes gather directly.
  int sblk;                        // blocks of the staged kernel (one per SM)
  int* el_slice[2];
  long long* el_pbytes[2];
  long long* el_poff[2];
  int* el_tmp[2];
  unsigned char* el_pack[2];
  float* el_logk[2];               // log K~ by value slot of the grouped copy (-inf in padding)
  long long pack_lim;              // bytes of one grouped copy
  long long nnz_lim;               // elements of the CSR / CSC arrays (bounds checks)
};

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

// A refused access: record where (first one wins) and skip it.
__device__ __forceinline__ void oob(Ctrl* ctrl, int code, long long index) {
  if (atomicCAS(&ctrl->oob_code, 0, code) == 0) ctrl->oob_index = index;
}

// log-sum-exp over one row (or column) by a whole warp: max, then sum.
__device__ __forceinline__ float warp_lse(const int* idx, const float* logv, const float* pot, float inv_eps,
                                          int lo, int hi, int lane) {
  float mx = neg_inf();
  for (int k = lo + lane; k < hi; k += 32) mx = fmaxf(mx, logv[k] + pot[idx[k]] * inv_eps);
  mx = warp_max(mx);
  if (mx == neg_inf()) return mx;
  float s = 0.0f;
  for (int k = lo + lane; k < hi; k += 32) s += expf(logv[k] + pot[idx[k]] * inv_eps - mx);
  s = warp_sum(s);
  return mx + logf(s);
}

// One exact log-domain half-iteration: pot_i = phi (eps log marg_i - eps LSE_j(logK~_ij + other_j/eps)).
__global__ void __launch_bounds__(kT) k_lse_half(int rows, const int* ptr, const int* idx, const float* logv,
                                                  const float* other, const float* marg, float* pot, float eps,
                                                  float phi) {
  const int lane = threadIdx.x & 31;
  const float inv_eps = 1.0f / eps;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += (gridDim.x * blockDim.x) >> 5) {
    const float L = warp_lse(idx, logv, other, inv_eps, ptr[i], ptr[i + 1], lane);
    if (lane == 0) {
      const float mi = marg[i];
      pot[i] = (L == neg_inf() || !(mi > 0.0f)) ? neg_inf() : phi * eps * (logf(mi) - L);
    }
  }
}

// The stored kernel value, step by step with explicit rounding (no
// contraction into fused multiply-adds), so that both absorption paths (by
// CSR / CSC segment and in grouped-copy order) store the same bits:
// z = logK~ + (pot_i + other_j)/eps, e = floor(log2 of the row's largest
// exp(z)), K' = 2^(z log2(e) - e).
__device__ __forceinline__ float absorbed_z(float lk, float pi, float o, float inv_eps) {
  return __fadd_rn(lk, __fmul_rn(__fadd_rn(pi, o), inv_eps));
}
__device__ __forceinline__ float absorbed_exponent(float zmax) {
  return zmax == neg_inf() ? 0.0f : floorf(__fmul_rn(zmax, kLog2e));
}
__device__ __forceinline__ float absorbed_value(float z, float e) {
  return exp2f(__fsub_rn(__fmul_rn(z, kLog2e), e));
}

// Write one row (CSR) or column (CSC) of K' = exp(logK~ + (pot_i + other_j)/eps)
// scaled by 2^-e, e = floor(log2 of the largest value).
template <typename V>
__device__ __forceinline__ void absorb_segment(int lo, int hi, const int* idx, const float* logv, float pot_i,
                                               const float* other, float inv_eps, V* out, float* e_out, int lane,
                                               const int* perm = nullptr, long long limit = 0,
                                               Ctrl* ctrl = nullptr) {
  float mx = neg_inf();
  if (pot_i != neg_inf())
    for (int k = lo + lane; k < hi; k += 32) {
      const float o = other[idx[k]];
      if (o != neg_inf()) mx = fmaxf(mx, absorbed_z(logv[k], pot_i, o, inv_eps));
    }
  mx = warp_max(mx);
  const float e = absorbed_exponent(mx);
  for (int k = lo + lane; k < hi; k += 32) {
    const float o = other[idx[k]];
    float z = neg_inf();
    if (pot_i != neg_inf() && o != neg_inf()) z = absorbed_z(logv[k], pot_i, o, inv_eps);
    const int dst = perm ? perm[k] : k;
    if (perm && (dst < 0 || (long long)dst >= limit)) { oob(ctrl, 1, dst); continue; }
    out[dst] = from_d<V>((double)absorbed_value(z, e));
  }
  if (lane == 0) *e_out = e;
}

// Where K' of one side goes when it is absorbed in CSR / CSC order: val /
// valT (the grouped copies are absorbed in copy order, by ell_absorb).
template <typename V>
struct AbsorbOut {
  V* out;
  const int* perm;
  long long limit;
};
template <typename V>
__device__ __forceinline__ AbsorbOut<V> absorb_out(const LogArgs& A, int side) {
  return {reinterpret_cast<V*>(side ? A.valT : A.val), nullptr, A.nnz_lim};
}
__device__ __forceinline__ bool grouped_copies(const LogArgs& A) {
  return A.stage && !*(volatile int*)&A.ctrl->ell_overflow;
}

template <typename V>
__global__ void __launch_bounds__(kT) k_absorb_all(LogArgs A, int t) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const AbsorbOut<V> R = absorb_out<V>(A, 0), C = absorb_out<V>(A, 1);
  const bool grouped = grouped_copies(A);   // the grouped copies were written by k_absorb_pack
  for (int i = gw; i < A.n && !grouped; i += nw)
    absorb_segment<V>(A.row_ptr[i], A.row_ptr[i + 1], A.col_idx, A.logval, A.alpha[i], A.beta, A.inv_eps, R.out,
                      A.erow + i, lane, R.perm, R.limit, A.ctrl);
  for (int j = gw; j < A.m && !grouped; j += nw)
    absorb_segment<V>(A.col_ptr[j], A.col_ptr[j + 1], A.row_idx, A.logvalT, A.beta[j], A.alpha, A.inv_eps, C.out,
                      A.ecol + j, lane, C.perm, C.limit, A.ctrl);
  // scalings of the pair t: 1 where the potential is finite, 0 where the row / column is unreachable
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  float* u = A.ubuf + (size_t)(t & 1) * A.n;
  float* v = A.vbuf + (size_t)(t & 1) * A.m;
  for (int i = tid; i < A.n; i += st) {
    const float al = A.alpha[i];
    u[i] = al == neg_inf() ? 0.0f : 1.0f;
    A.ahat[i] = A.uot && al != neg_inf() ? A.a[i] * expf(-al * A.inv_lam) : A.a[i];
  }
  for (int j = tid; j < A.m; j += st) {
    const float be = A.beta[j];
    v[j] = be == neg_inf() ? 0.0f : 1.0f;
    A.bhat[j] = A.uot && be != neg_inf() ? A.b[j] * expf(-be * A.inv_lam) : A.b[j];
  }
  if (tid == 0) A.ctrl->t = t;
}

template <typename T>
__global__ void k_log_init(int n, int m, float* alpha, float* beta, const T* al0, const T* be0, Ctrl* ctrl) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) alpha[i] = al0 ? (float)al0[i] : 0.0f;
  for (int64_t j = tid; j < m; j += stride) beta[j] = be0 ? (float)be0[j] : 0.0f;
  if (tid == 0) {
    ctrl->t = 0; ctrl->done = 0; ctrl->iters = 0;
    ctrl->blocks_a = ctrl->blocks_b = ctrl->blocks_c = 0u;
    ctrl->bar_count = 0u;
    ctrl->ell_overflow = 0;
    ctrl->ell_bytes[0] = ctrl->ell_bytes[1] = 0;
    if (ctrl->status != SPS_OK) ctrl->done = 1;
  }
}

// ----------------------------------------------------------------------------
// Phases of the stabilised iteration.
// ----------------------------------------------------------------------------

// Row update from q' = (K' v~)_i (scale applied): u~ = (a^/q')^phi; residual
// term (a/a^)|u~_old^{1/phi} q' - a^|; an empty row is unreachable (u~ = 0).
template <bool UOT>
__device__ __forceinline__ float row_math(const LogArgs& A, float q, float ah, float ai, float uo, float& res,
                                          float& unr, float& mlog) {
  float un;
  if (q > 0.0f) {
    un = UOT ? powf(ah / q, A.phi) : ah / q;
    const float lhs = (UOT ? powf(uo, A.inv_phi) : uo) * q;
    const float w = UOT ? (ah > 0.0f ? ai / ah : 1.0f) : 1.0f;
    res += w * fabsf(lhs - ah);
    if (un > 0.0f) mlog = fmaxf(mlog, fabsf(logf(un)));
  } else {
    un = 0.0f;
    unr += ai;
  }
  return un;
}

// Column update from r' = (K'^T u~)_j: v~ = (b^/r')^phi.
template <bool UOT>
__device__ __forceinline__ float col_math(const LogArgs& A, float r, float bh, float bj, float& unb, float& mlog) {
  float vn;
  if (r > 0.0f) {
    vn = UOT ? powf(bh / r, A.phi) : bh / r;
    if (vn > 0.0f) mlog = fmaxf(mlog, fabsf(logf(vn)));
  } else {
    vn = 0.0f;
    unb += bj;
  }
  return vn;
}

// Block totals of a phase: sums of NV values (thread 0) and the block maximum
// of mlog (thread 0).
template <int NV>
__device__ __forceinline__ float finish_phase(float (&s)[NV], float mlog, float* sh) {
  block_sum_multi<NV, float>(s, sh);
  const float mw = warp_max(mlog);
  if ((threadIdx.x & 31) == 0) sh[64 + (threadIdx.x >> 5)] = mw;
  __syncthreads();
  float mm = 0.0f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, sh[64 + w]);
  __syncthreads();
  return mm;
}

template <int LPR, typename V, bool UOT>
__device__ __forceinline__ void log_row_phase(const LogArgs& A, int t, float (&o)[3], float* sh) {
  const float* v = A.vbuf + (size_t)(t & 1) * A.m;
  const float* uold = A.ubuf + (size_t)(t & 1) * A.n;
  float* unew = A.ubuf + (size_t)((t + 1) & 1) * A.n;
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31, sl = lane & (LPR - 1);
  float res = 0.0f, unr = 0.0f, mlog = 0.0f;
  const int nw = blockDim.x >> 5;
  const int wg = blockIdx.x * nw + (threadIdx.x >> 5);
  for (int base = wg * RPW; base < A.n; base += gridDim.x * nw * RPW) {
    const int i = base + lane / LPR;
    const bool ok = i < A.n;
    const int lo = ok ? __ldg(A.row_ptr + i) : 0, hi = ok ? __ldg(A.row_ptr + i + 1) : 0;
    float ah = 0.f, ai = 0.f, uo = 0.f, er = 0.f;
    if (ok && sl == 0) { ah = A.ahat[i]; ai = A.a[i]; uo = uold[i]; er = A.erow[i]; }
    const float qs = seg_row_dot<LPR, V, float>(A.col_idx, (const V*)A.val, v, lo, hi, sl);
    if (ok && sl == 0) unew[i] = row_math<UOT>(A, qs * exp2f(er), ah, ai, uo, res, unr, mlog);
  }
  float s2[2] = {res, unr};
  o[2] = finish_phase<2>(s2, mlog, sh);
  o[0] = s2[0]; o[1] = s2[1];
}

template <int LPR, typename V, bool UOT>
__device__ __forceinline__ void log_col_phase(const LogArgs& A, int t, float (&o)[2], float* sh) {
  const float* u = A.ubuf + (size_t)((t + 1) & 1) * A.n;
  float* vnew = A.vbuf + (size_t)((t + 1) & 1) * A.m;
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31, sl = lane & (LPR - 1);
  float unb = 0.0f, mlog = 0.0f;
  const int nw = blockDim.x >> 5;
  const int wg = blockIdx.x * nw + (threadIdx.x >> 5);
  for (int base = wg * RPW; base < A.m; base += gridDim.x * nw * RPW) {
    const int j = base + lane / LPR;
    const bool ok = j < A.m;
    const int lo = ok ? __ldg(A.col_ptr + j) : 0, hi = ok ? __ldg(A.col_ptr + j + 1) : 0;
    float bh = 0.f, bj = 0.f, ec = 0.f;
    if (ok && sl == 0) { bh = A.bhat[j]; bj = A.b[j]; ec = A.ecol[j]; }
    const float rs = seg_row_dot<LPR, V, float>(A.row_idx, (const V*)A.valT, u, lo, hi, sl);
    if (ok && sl == 0) vnew[j] = col_math<UOT>(A, rs * exp2f(ec), bh, bj, unb, mlog);
  }
  float s1[1] = {unb};
  o[1] = finish_phase<1>(s1, mlog, sh);
  o[0] = s1[0];
}

// 16-byte asynchronous copy global -> shared through L2 (cp.async.cg), and the
// wait for all of this thread's copies.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ----------------------------------------------------------------------------
// Staged passes over the grouped copy (its layout is described with kEllWarps).
// ----------------------------------------------------------------------------

constexpr int kEllWins = kEllRing / kEllWin;   // windows a ring holds

// Wait until at most n of this thread's cp.async groups are pending (n is
// clamped to 0 .. kEllWins - 1; the instruction takes an immediate).
__device__ __forceinline__ void cp_async_wait_n(int n) {
  switch (n <= 0 ? 0 : n >= kEllWins - 1 ? kEllWins - 1 : n) {
    case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
  }
}
static_assert(kEllWins >= 2 && kEllWins <= 8, "cp_async_wait_n covers up to eight windows");
static_assert(kEllWin % (32 * 16) == 0, "a window is a whole number of 16-byte copies per lane");

template <typename V> __device__ __forceinline__ float ring_val(const unsigned char* p);
template <> __device__ __forceinline__ float ring_val<float>(const unsigned char* p) {
  return *reinterpret_cast<const float*>(p);
}
template <> __device__ __forceinline__ float ring_val<__nv_bfloat16>(const unsigned char* p) {
  return __uint_as_float((unsigned)*reinterpret_cast<const unsigned short*>(p) << 16);
}
template <> __device__ __forceinline__ float ring_val<__half>(const unsigned char* p) {
  return __half2float(*reinterpret_cast<const __half*>(p));
}

// One warp's stream of the grouped copy: the bytes [s0, s1) of the pack, at
// positions relative to a0 (s0 rounded down to a window), pass through the
// warp's ring; relative byte r sits at ring[r mod kEllRing] while resident.
// Window k is the relative bytes [k kEllWin, (k + 1) kEllWin), clipped to the
// stream; lane l copies its 16-byte pieces l, l + 32, ... of each window
// (cp.async through L2) and commits one group per window, so window k has landed for the lane once at
// most (issued - 1 - k) of its groups are pending.  Window k is issued once
// every byte of window k - kEllWins has been read by the whole warp.
struct EllRing {
  const unsigned char* src;   // pack + a0
  unsigned char* ring;
  unsigned r0, r1;            // the stream, relative
  unsigned issued, nwin;
  unsigned pf;                // windows below pf have been issued or prefetched into L2
};

// Bulk prefetch of [g, g + bytes) into L2 (16-byte aligned address, size a
// multiple of 16); a hint with no completion and no shared-memory effect.
__device__ __forceinline__ void prefetch_l2_bulk(const void* g, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(g), "r"(bytes) : "memory");
}

// Make the relative bytes below `end` readable by the warp: issue the windows
// that the read position `cons` allows (every byte below it has been read by
// every lane), wait for the window holding byte end - 1, then a warp barrier.
// end - cons <= kEllRing - kEllWin, so that window has been issued.
__device__ __forceinline__ void ell_need(EllRing& R, unsigned cons, unsigned end) {
  __syncwarp();
  const unsigned lim = min(R.nwin, cons / kEllWin + kEllWins);
  const unsigned l16 = 16u * (threadIdx.x & 31);
  while (R.issued < lim) {
#pragma unroll
    for (int j = 0; j < kEllWin / 512; ++j) {
      const unsigned r = R.issued * kEllWin + 512u * j + l16;
      if (r >= R.r0 && r < R.r1) cp_async16(R.ring + (r & (kEllRing - 1)), R.src + r);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    ++R.issued;
  }
  if (kEllPrefetch > 0) {
    // the next kEllPrefetch windows start their way from DRAM into L2, so that a
    // window's copy into the ring mostly waits for L2 rather than DRAM: the bytes
    // in flight are no longer bounded by the ring
    const unsigned from = max(R.pf, R.issued), plim = min(R.nwin, R.issued + kEllPrefetch);
    if (from < plim) {
      const unsigned b0 = max(from * kEllWin, R.r0), b1 = min(plim * kEllWin, R.r1);
      if ((threadIdx.x & 31) == 0 && b1 > b0) prefetch_l2_bulk(R.src + b0, b1 - b0);
      R.pf = plim;
    }
  }
  cp_async_wait_n((int)R.issued - 1 - (int)((end - 1) / kEllWin));
  __syncwarp();
}

// One staged pass of this block: acc[r] += sum over the block's row r of
// K'_rj x_j (rows local to the block, nr of them), x of length nx passing
// through shared memory (xs) in J chunks of W entries.  Warp w streams its
// slice's groups (one contiguous byte range over all chunks) through its ring
// and walks them chunk by chunk; lane l of a group continues its row's sum
// with run l, one multiply-add per step in column order, so every row's sum is
// one sequential chain over its columns and no two lanes of the block ever
// hold the same row at once (a row belongs to one slice and appears once in a
// chunk's groups): plain loads and stores of acc, no atomics.  A group's
// header names the next group's height, so one wait covers a whole group (up
// to KB steps).  The stream runs ahead across chunk boundaries.  The chunk of
// x arrives by one bulk copy on its own mbarrier (when x is 16-byte aligned):
// every warp counts itself done with chunk c in shared memory, the warp that
// completes the count issues chunk c + 1 into the same buffer, and all wait for
// that phase only, so the stream's windows in flight are not drained at a
// switch.  Otherwise by cp.async between two block barriers.
__device__ __forceinline__ void mbar_arrive_plain(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

// Chunk c of x into xs, issued by one thread: the whole 16-byte part by a bulk
// copy, the last (at most 3) entries by plain stores made before the arrive
// (whose release makes them visible to the phase's waiters).
__device__ __forceinline__ void ell_issue_chunk(const float* x, int nx, int W, int c, float* xs, uint64_t* bar) {
  const int j0 = c * W;
  const int jn = min(W, nx - j0);
  const int n4 = jn & ~3;
  for (int k = n4; k < jn; ++k) xs[k] = __ldcg(x + j0 + k);
  if (n4 > 0) {
    mbar_arrive_expect_tx(bar, (unsigned)n4 * 4u);
    bulk_copy_g2s(xs, x + j0, (unsigned)n4 * 4u, bar);
  } else {
    mbar_arrive_plain(bar);
  }
}

// Bounded wait for a phase of the chunk barrier by every thread; a wait that
// gives up records the failure (the solve then reports it) instead of hanging.
__device__ __forceinline__ void ell_wait_chunk(uint64_t* bar, unsigned parity, Ctrl* ctrl) {
  long long polls = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++polls > kSpinLimit) {
      ctrl->wait_timeout = 1;
      ctrl->status = SPS_ERR_CUDA;
      ctrl->done = 1;
      break;
    }
  }
}

template <typename V>
__device__ __forceinline__ void ell_pass(const unsigned char* __restrict__ pack, const long long* __restrict__ poff,
                                         const float* x, int nx, int nr, int W, int J, float* xs, float* acc,
                                         unsigned char* rings, long long pack_lim, Ctrl* ctrl) {
  constexpr int vb = (int)sizeof(V);
  constexpr unsigned st = (unsigned)ell_step_bytes(vb);
  constexpr unsigned M = kEllRing - 1;
  constexpr int KB = (int)((kEllRing - kEllWin - kEllHdr) / st);   // steps one wait covers
  const int T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const long long* po = poff + ((size_t)blockIdx.x * kEllWarps + warp) * J;
  long long s0 = __ldg(po), s1 = __ldg(po + J);
  if (s0 < 0 || s1 < s0 || s1 > pack_lim || (s0 & 15) || (s1 & 15) || s1 - s0 > (1LL << 30)) {
    if (lane == 0) oob(ctrl, 2, s1);   // inconsistent slice bounds: skip the slice
    s1 = s0 = 0;
  }
  const long long a0 = s0 & ~(long long)(kEllWin - 1);
  EllRing R;
  R.src = pack + a0;
  R.ring = rings + (size_t)warp * kEllRing;
  R.r0 = (unsigned)(s0 - a0);
  R.r1 = (unsigned)(s1 - a0);
  R.nwin = R.r1 > R.r0 ? (R.r1 - 1) / kEllWin + 1 : 0;
  R.issued = 0;
  R.pf = 0;
  ell_need(R, R.r0, R.r0 + 16);   // the first windows (the wait is for the first one only)
  const unsigned l2 = 2u * lane, lv = 64u + (unsigned)vb * lane;
  unsigned p = R.r0;   // read position (uniform over the warp)
  int Hc = -1;         // height of the group at p, when known from the previous header
  __shared__ __align__(8) uint64_t xbar;   // chunk barrier (one phase a chunk)
  __shared__ int xdone;                     // warps done with the current chunk, counted over the pass
  const bool bulk = (((uintptr_t)x) & 15) == 0;   // chunk starts c W are multiples of 1024 entries
  if (bulk) {
    if (t == 0) {
      mbar_init(&xbar, 1);
      fence_mbarrier_init();
      xdone = 0;
    }
    __syncthreads();   // the barrier is set (and acc is initialised)
    if (t == 0) {
      fence_proxy_async_global();   // x was written by ordinary stores before the last grid barrier
      ell_issue_chunk(x, nx, W, 0, xs, &xbar);
    }
  }
  for (int c = 0; c < J; ++c) {
    const int j0 = c * W;
    const int jn = min(W, nx - j0);
    const long long e1 = __ldg(po + c + 1);
    const unsigned pe = (unsigned)(min(max(e1, a0 + (long long)p), s1) - a0);   // end of this part
    if (bulk) {
      ell_wait_chunk(&xbar, (unsigned)(c & 1), ctrl);
    } else {
      __syncthreads();   // the previous chunk is no longer read (and acc is initialised)
      if ((((uintptr_t)(x + j0)) & 15) == 0) {
        const int n4 = jn >> 2;
        for (int k = t; k < n4; k += T) cp_async16(xs + 4 * k, x + j0 + 4 * k);
        for (int k = 4 * n4 + t; k < jn; k += T) xs[k] = __ldcg(x + j0 + k);
      } else {
        for (int k = t; k < jn; k += T) xs[k] = __ldcg(x + j0 + k);
      }
      cp_async_wait_all();   // also lands the stream windows issued so far
      __syncthreads();
    }
    while (p < pe) {
      if (Hc < 0) {
        ell_need(R, p, min(p + kEllHdr, pe));
        Hc = *reinterpret_cast<const int*>(R.ring + ((p + 64) & M));
      }
      if (Hc < 1 || (long long)p + ell_group_bytes(Hc, vb) > pe) {   // inconsistent group: skip the rest of the part
        if (lane == 0) oob(ctrl, 4, a0 + p);
        p = pe;
        Hc = -1;
        break;
      }
      const int H = Hc;
      int n = min(H, KB);
      ell_need(R, p, p + kEllHdr + n * st);
      const unsigned row = *reinterpret_cast<const unsigned short*>(R.ring + ((p + l2) & M));
      const int Hn = *reinterpret_cast<const int*>(R.ring + ((p + 68) & M));
      if (*reinterpret_cast<const int*>(R.ring + ((p + 64) & M)) != H) {
        if (lane == 0) oob(ctrl, 4, a0 + p);
        p = pe;
        Hc = -1;
        break;
      }
      const bool mine = row < (unsigned)nr;
      if (!mine && row != 0xFFFFu) oob(ctrl, 5, row);
      float s = mine ? acc[row] : 0.0f;
      unsigned q = p + kEllHdr;
      for (int k = 0;;) {
#pragma unroll 4
        for (int u = 0; u < n; ++u) {
          const unsigned o = q + u * st;
          const unsigned iq = *reinterpret_cast<const unsigned short*>(R.ring + ((o + l2) & M));
          const float w = ring_val<V>(R.ring + ((o + lv) & M));
          // a padding step adds 0 x xs[0] (x is finite); an index past the chunk
          // (only in an inconsistent copy) reads inside xs
          s = fmaf(w, xs[min(iq, (unsigned)(W - 1))], s);
        }
        q += n * st;
        k += n;
        if (k >= H) break;
        n = min(KB, H - k);
        ell_need(R, q, q + n * st);
      }
      if (mine) acc[row] = s;
      p = q;
      Hc = Hn > 0 ? Hn : -1;
    }
    p = max(p, pe);
    if (bulk) {   // this warp is done with chunk c; the last one to finish issues chunk c + 1
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();   // the warp's reads of xs precede the count
        const int prev = atomicAdd(&xdone, 1);
        if (prev == kEllWarps * (c + 1) - 1 && c + 1 < J) {
          fence_proxy_async_shared();   // those reads precede the bulk copy's writes
          ell_issue_chunk(x, nx, W, c + 1, xs, &xbar);
        }
      }
    }
  }
  cp_async_wait_all();   // nothing of the stream stays in flight
  __syncthreads();
}

// Staged row pass: u~ of this block's rows from the grouped copy of the CSR.
template <typename V, bool UOT>
__device__ __forceinline__ void log_row_phase_staged(const LogArgs& A, int t, float (&o)[3], float* sh, float* dsm) {
  const float* v = A.vbuf + (size_t)(t & 1) * A.m;
  const float* uold = A.ubuf + (size_t)(t & 1) * A.n;
  float* unew = A.ubuf + (size_t)((t + 1) & 1) * A.n;
  const int r0 = blockIdx.x * A.rows_pb;
  const int nr = max(0, min(A.n, r0 + A.rows_pb) - r0);
  float* acc = dsm + A.W;
  for (int k = threadIdx.x; k < nr; k += blockDim.x) acc[k] = 0.0f;
  unsigned char* rings = reinterpret_cast<unsigned char*>(dsm) + ell_ring_offset(A.W, max(A.rows_pb, A.cols_pb));
  ell_pass<V>(A.el_pack[0], A.el_poff[0], v, A.m, nr, A.W, A.Jr, dsm, acc, rings, A.pack_lim, A.ctrl);
  float res = 0.0f, unr = 0.0f, mlog = 0.0f;
  for (int k = threadIdx.x; k < nr; k += blockDim.x) {
    const int i = r0 + k;
    unew[i] = row_math<UOT>(A, acc[k] * exp2f(A.erow[i]), A.ahat[i], A.a[i], uold[i], res, unr, mlog);
  }
  float s2[2] = {res, unr};
  o[2] = finish_phase<2>(s2, mlog, sh);
  o[0] = s2[0]; o[1] = s2[1];
}

// Staged column pass: v~ of this block's columns from the grouped copy of the CSC.
template <typename V, bool UOT>
__device__ __forceinline__ void log_col_phase_staged(const LogArgs& A, int t, float (&o)[2], float* sh, float* dsm) {
  const float* u = A.ubuf + (size_t)((t + 1) & 1) * A.n;
  float* vnew = A.vbuf + (size_t)((t + 1) & 1) * A.m;
  const int c0 = blockIdx.x * A.cols_pb;
  const int nc = max(0, min(A.m, c0 + A.cols_pb) - c0);
  float* acc = dsm + A.W;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) acc[k] = 0.0f;
  unsigned char* rings = reinterpret_cast<unsigned char*>(dsm) + ell_ring_offset(A.W, max(A.rows_pb, A.cols_pb));
  ell_pass<V>(A.el_pack[1], A.el_poff[1], u, A.n, nc, A.W, A.Jc, dsm, acc, rings, A.pack_lim, A.ctrl);
  float unb = 0.0f, mlog = 0.0f;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const int j = c0 + k;
    vnew[j] = col_math<UOT>(A, acc[k] * exp2f(A.ecol[j]), A.bhat[j], A.b[j], unb, mlog);
  }
  float s1[1] = {unb};
  o[1] = finish_phase<1>(s1, mlog, sh);
  o[0] = s1[0];
}

// seg[c * ld + i] for c = 0 .. J: the first position of segment i (a CSR row
// or a CSC column) whose index is >= c W; lane c of the segment's warp finds it
// by binary search over the sorted indices.
__global__ void k_chunk_ptrs(int rows, const int* __restrict__ ptr, const int* __restrict__ idx, int W, int J,
                             int* __restrict__ seg) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += (gridDim.x * blockDim.x) >> 5) {
    const int lo0 = ptr[i], hi0 = ptr[i + 1];
    for (int c = lane; c <= J; c += 32) {
      int lo = lo0, hi = hi0;
      if (c == 0) hi = lo0;
      else if (c == J) lo = hi0;
      else {
        const int key = c * W;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (idx[mid] < key) lo = mid + 1; else hi = mid;
        }
      }
      seg[(size_t)c * rows + i] = lo;
    }
  }
}

// ----------------------------------------------------------------------------
// Building the grouped copies (once a solve, after the sketch).
// ----------------------------------------------------------------------------

// Warp slices: slice w of block b is the block-local rows [S[w], S[w + 1]),
// cut where the elements before it reach w / kEllWarps of the block's (block b
// owns rows [b R, (b + 1) R) of the rows).
__global__ void k_el_slices(int rows, int R, int nblk, const int* __restrict__ ptr, int* __restrict__ S) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= nblk * (kEllWarps + 1)) return;
  const int b = tid / (kEllWarps + 1), w = tid % (kEllWarps + 1);
  const int r0 = (int)min((long long)rows, (long long)b * R), r1 = (int)min((long long)rows, (long long)r0 + R);
  const long long e0 = ptr[r0], E = (long long)ptr[r1] - e0;
  const long long target = e0 + E * w / kEllWarps;
  int lo = r0, hi = r1;   // the first row i of [r0, r1] with ptr[i] >= target
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ptr[mid] < target) lo = mid + 1; else hi = mid;
  }
  S[tid] = w == kEllWarps ? r1 - r0 : lo - r0;
}

// Run lengths of one part, the rows [g0, g1) in chunk c (one warp):
// len = seg[(c + 1) rows + r] - seg[c rows + r], counted in hist by bin
// min(len, kEllBins - 1) (rows without a run are left out).  Returns the
// longest run of the last bin (0 if it is empty) on every lane; a negative
// length (inconsistent chunk pointers) sets *bad.
__device__ __forceinline__ int ell_hist(const int* __restrict__ seg, int rows, int c, int g0, int g1, int* hist,
                                        int* bad) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k < kEllBins; k += 32) hist[k] = 0;
  __syncwarp();
  const int* s0 = seg + (size_t)c * rows;
  const int* s1 = s0 + rows;
  unsigned lump = 0u;
  for (int r = g0 + lane; r < g1; r += 32) {
    const int len = s1[r] - s0[r];
    if (len < 0) *bad = 1;
    if (len > 0) {
      atomicAdd(&hist[min(len, kEllBins - 1)], 1);
      if (len >= kEllBins - 1) lump = max(lump, (unsigned)len);
    }
  }
  __syncwarp();
  return (int)__reduce_max_sync(0xffffffffu, lump);
}

// The sorted order of a part (longest runs first): start[k] = runs in bins
// above k (if start is given), *bytes = the part's bytes (every group takes
// the height of its first run; the last bin's groups take the longest run).
// Lane l handles bins 8 l .. 8 l + 7.  Returns the part's runs on every lane.
__device__ __forceinline__ int ell_order(const int* hist, int* start, int lump, int vb, long long* bytes) {
  const int lane = threadIdx.x & 31;
  int cnt[8], tot = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    cnt[u] = hist[8 * lane + u];
    tot += cnt[u];
  }
  int suf = tot;   // runs in the bins of this lane and the lanes above
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_down_sync(0xffffffffu, suf, o);
    if (lane + o < 32) suf += y;
  }
  int pos = suf - tot;
  long long by = 0;
#pragma unroll
  for (int u = 7; u >= 0; --u) {
    const int k = 8 * lane + u;
    if (start) start[k] = pos;
    const int C = cnt[u];
    if (C > 0) {
      const int h = k < kEllBins - 1 ? k : lump;
      const int groups = (pos + C + 31) / 32 - (pos + 31) / 32;   // groups whose first run is in bin k
      by += (long long)groups * ell_group_bytes(h, vb);
    }
    pos += C;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) by += __shfl_xor_sync(0xffffffffu, by, o);
  *bytes = by;
  __syncwarp();
  return __shfl_sync(0xffffffffu, suf, 0);
}

// Bytes of every part: one warp a slice, chunk by chunk.
__global__ void __launch_bounds__(256) k_el_size(int rows, int R, int nblk, int J, const int* __restrict__ seg,
                                                 const int* __restrict__ S, int vb, long long* __restrict__ pbytes,
                                                 Ctrl* ctrl) {
  __shared__ int hist_sh[8][kEllBins];
  __shared__ int bad_sh[8];
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sl = blockIdx.x * 8 + wl;   // b kEllWarps + w
  if (sl >= nblk * kEllWarps) return;
  const int b = sl / kEllWarps, w = sl % kEllWarps;
  const int r0 = (int)min((long long)rows, (long long)b * R);
  const int* Sb = S + (size_t)b * (kEllWarps + 1);
  const int g0 = r0 + Sb[w], g1 = r0 + Sb[w + 1];
  if (lane == 0) bad_sh[wl] = 0;
  __syncwarp();
  for (int c = 0; c < J; ++c) {
    const int lump = ell_hist(seg, rows, c, g0, g1, hist_sh[wl], &bad_sh[wl]);
    long long by = 0;
    ell_order(hist_sh[wl], nullptr, lump, vb, &by);
    if (lane == 0) pbytes[(size_t)sl * J + c] = by;
  }
  __syncwarp();
  if (lane == 0 && bad_sh[wl]) {
    oob(ctrl, 6, sl);
    ctrl->ell_overflow = 1;
  }
}

// Exclusive prefix sums of the parts' bytes (one block); a total above the
// planned copy, or with more value slots than an int counts, sets
// ell_overflow (the passes then gather directly).
__global__ void __launch_bounds__(1024) k_el_scan(long long P, const long long* __restrict__ pbytes,
                                                  long long* __restrict__ poff, long long cap_bytes, int vb,
                                                  Ctrl* ctrl, int side) {
  __shared__ long long sh[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const long long per = (P + T - 1) / T;
  const long long lo = min(P, (long long)t * per), hi = min(P, lo + per);
  long long s = 0;
  for (long long i = lo; i < hi; ++i) s += pbytes[i];
  sh[t] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    const long long y = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += y;
    __syncthreads();
  }
  long long run = sh[t] - s;
  for (long long i = lo; i < hi; ++i) {
    poff[i] = run;
    run += pbytes[i];
  }
  if (t == T - 1) {
    const long long tot = sh[T - 1];
    poff[P] = tot;
    ctrl->ell_bytes[side] = tot;
    if (tot > cap_bytes || tot / vb > 0x7fffffffLL) ctrl->ell_overflow = 1;
  }
}

// The grouped copy of every part (one warp a slice, chunk by chunk): the runs
// in sorted order (a bin's runs in row order) go to the slice's scratch as
// (block-local row, length, first CSR position), then each group of 32 is
// written: header, indices (padding 0), padding values 0 and log K~ by value
// slot (absorption writes K' over every slot, in copy order).  A part whose bytes
// disagree with k_el_size sets ell_overflow.
template <typename V>
__global__ void __launch_bounds__(256) k_el_fill(int rows, int R, int nblk, int J, int W, const int* __restrict__ seg,
                                                 const int* __restrict__ idx, const int* __restrict__ S,
                                                 const long long* __restrict__ poff, int* __restrict__ tmp,
                                                 unsigned char* __restrict__ pack, const float* __restrict__ logv,
                                                 float* __restrict__ logk,
                                                 long long nnz_lim, long long pack_lim, Ctrl* ctrl) {
  constexpr int vb = (int)sizeof(V);
  __shared__ int hist_sh[8][kEllBins];
  __shared__ int start_sh[8][kEllBins];
  __shared__ int bad_sh[8];
  if (*(volatile int*)&ctrl->ell_overflow) return;
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sl = blockIdx.x * 8 + wl;
  if (sl >= nblk * kEllWarps) return;
  const int b = sl / kEllWarps, w = sl % kEllWarps;
  const int r0 = (int)min((long long)rows, (long long)b * R);
  const int* Sb = S + (size_t)b * (kEllWarps + 1);
  const int g0 = r0 + Sb[w], g1 = r0 + Sb[w + 1];
  int* cur = start_sh[wl];
  if (lane == 0) bad_sh[wl] = 0;
  __syncwarp();
  long long prev = -1;   // header of the slice's previous group (its next-height field is set here)
  for (int c = 0; c < J; ++c) {
    const int lump = ell_hist(seg, rows, c, g0, g1, hist_sh[wl], &bad_sh[wl]);
    long long by = 0;
    const int runs = ell_order(hist_sh[wl], cur, lump, vb, &by);
    const long long p0 = poff[(size_t)sl * J + c], p1 = poff[(size_t)sl * J + c + 1];
    if (p1 - p0 != by || p0 < 0 || p1 > pack_lim || runs > g1 - g0) {
      if (lane == 0) {
        oob(ctrl, 7, p0);
        ctrl->ell_overflow = 1;
      }
      return;
    }
    // sorted positions: within a bin, runs keep their row order
    for (int base = g0; base < g1; base += 32) {
      const int r = base + lane;
      int len = 0, src = 0;
      if (r < g1) {
        src = seg[(size_t)c * rows + r];
        len = seg[(size_t)(c + 1) * rows + r] - src;
      }
      const int bin = len > 0 ? min(len, kEllBins - 1) : -1;
      const unsigned same = __match_any_sync(0xffffffffu, bin);
      const int rank = __popc(same & ((1u << lane) - 1u));
      const int pos = bin > 0 ? cur[bin] + rank : 0;
      __syncwarp();
      if (bin > 0 && rank == 0) cur[bin] += __popc(same);
      __syncwarp();
      if (bin > 0) {
        int* e = tmp + 3 * ((size_t)g0 + pos);
        e[0] = r - r0;
        e[1] = len;
        e[2] = src;
      }
    }
    __syncwarp();
    long long off = p0;
    const int G = (runs + 31) / 32;
    for (int g = 0; g < G; ++g) {
      const int pos = 32 * g + lane;
      int row = 0xFFFF, len = 0, src = 0;
      if (pos < runs) {
        const int* e = tmp + 3 * ((size_t)g0 + pos);
        row = e[0];
        len = e[1];
        src = e[2];
      }
      const int l0 = __shfl_sync(0xffffffffu, len, 0);
      const int h = l0 < kEllBins - 1 ? l0 : lump;
      if (off + ell_group_bytes(h, vb) > p1) {
        if (lane == 0) {
          oob(ctrl, 8, off);
          ctrl->ell_overflow = 1;
        }
        return;
      }
      unsigned char* gp = pack + off;
      reinterpret_cast<unsigned short*>(gp)[lane] = (unsigned short)row;
      if (lane < 4) reinterpret_cast<int*>(gp + 64)[lane] = lane == 0 ? h : 0;
      if (lane == 0 && prev >= 0) reinterpret_cast<int*>(pack + prev + 68)[0] = h;
      prev = off;
      constexpr long long st = ell_step_bytes(vb);
      // eight steps at a time: the run's indices and log K~ are loaded first
      // (every lane reads its own row's run), then the steps are written
      for (int k0 = 0; k0 < h; k0 += 8) {
        int qv[8];
        float lv[8];
        bool okv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = k0 + u;
          const long long e = (long long)src + k;
          okv[u] = k < h && k < len && e >= 0 && e < nnz_lim;
          qv[u] = okv[u] ? idx[e] : 0;
          lv[u] = okv[u] ? logv[e] : neg_inf();
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = k0 + u;
          if (k >= h) break;
          unsigned char* sp = gp + kEllHdr + k * st;   // step k: 32 indices, then 32 values
          const long long slot = (off + kEllHdr + k * st + 64) / vb + lane;
          unsigned short q = 0;
          float lk = neg_inf();
          if (k < len) {
            const long long e = (long long)src + k;
            if (okv[u]) {
              q = (unsigned short)(qv[u] - c * W);
              lk = lv[u];
            } else {
              oob(ctrl, 9, e);
              ctrl->ell_overflow = 1;
            }
          } else {
            reinterpret_cast<V*>(sp + 64)[lane] = from_d<V>(0.0);
          }
          logk[slot] = lk;
          reinterpret_cast<unsigned short*>(sp)[lane] = q;
        }
      }
      off += ell_group_bytes(h, vb);
    }
    if (off != p1) {
      if (lane == 0) {
        oob(ctrl, 8, off);
        ctrl->ell_overflow = 1;
      }
      return;
    }
  }
  __syncwarp();
  if (lane == 0 && bad_sh[wl]) {
    oob(ctrl, 6, sl);
    ctrl->ell_overflow = 1;
  }
}

// Absorption in copy order, one side (0: rows over the CSR copy, 1: columns
// over the CSC copy) of this block's rows:
// K' = exp(logK~ + (pot_i + other_j)/eps) 2^-e_i, e_i = floor(log2 of row i's
// largest value), the formula of absorb_segment element for element, so the
// stored values are the same.  Pass 1 takes each row's maximum (lane l of a
// group holds row l, and a slice's rows belong to one warp, so mx needs no
// atomics), pass 2 writes the values over the groups' value steps, every
// write a whole 32-lane row of a step.  The other side's potentials pass
// through shared memory (xs) chunk by chunk, as the gathered vector does in
// ell_pass.  mx: shared scratch of the block's rows.
template <typename V, int NB>
__device__ void ell_absorb(const LogArgs& A, int side, float* xs, float* mx) {
  constexpr int vb = (int)sizeof(V);
  constexpr long long st = ell_step_bytes(vb);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int R = side ? A.cols_pb : A.rows_pb;
  const int rows = side ? A.m : A.n;
  const int r0 = blockIdx.x * R;
  const int nr = max(0, min(rows, r0 + R) - r0);
  const int J = side ? A.Jc : A.Jr;
  const int nx = side ? A.n : A.m;
  const float* pot = side ? A.beta : A.alpha;
  const float* oth = side ? A.alpha : A.beta;
  float* e_out = side ? A.ecol : A.erow;
  const unsigned char* pack = A.el_pack[side];
  V* val = reinterpret_cast<V*>(A.el_pack[side]);
  const float* logk = A.el_logk[side];
  const long long* po = A.el_poff[side] + ((size_t)blockIdx.x * kEllWarps + warp) * J;
  for (int k = threadIdx.x; k < nr; k += blockDim.x) mx[k] = neg_inf();
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    long long off = __ldg(po);
    long long s1 = __ldg(po + J);
    if (off < 0 || s1 < off || s1 > A.pack_lim) {   // inconsistent slice bounds: skip the slice
      if (lane == 0) oob(A.ctrl, 2, s1);
      off = s1 = 0;
    }
    for (int c = 0; c < J; ++c) {
      const long long pe = min(max(__ldg(po + c + 1), off), s1);
      const int j0 = c * A.W, jn = min(A.W, nx - j0);
      __syncthreads();   // the previous chunk is no longer read
      if ((((uintptr_t)(oth + j0)) & 15) == 0) {   // 16-byte copies, all in flight at once
        const int n4 = jn >> 2;
        for (int k = threadIdx.x; k < n4; k += blockDim.x) cp_async16(xs + 4 * k, oth + j0 + 4 * k);
        for (int k = 4 * n4 + threadIdx.x; k < jn; k += blockDim.x) xs[k] = __ldcg(oth + j0 + k);
      } else {
        for (int k = threadIdx.x; k < jn; k += blockDim.x) xs[k] = __ldcg(oth + j0 + k);
      }
      cp_async_wait_all();
      __syncthreads();
      while (off < pe) {
        const int H = __ldg(reinterpret_cast<const int*>(pack + off + 64));
        const unsigned row = __ldg(reinterpret_cast<const unsigned short*>(pack + off) + lane);
        if (H < 1 || off + ell_group_bytes(H, vb) > pe) {
          if (lane == 0) oob(A.ctrl, 4, off);
          off = pe;
          break;
        }
        const bool mine = row < (unsigned)nr;
        const float pi = mine ? __ldcg(pot + r0 + row) : neg_inf();
        const float ei = (pass == 1 && mine) ? mx[row] : 0.0f;
        float m = neg_inf();
        // NB steps at a time: their indices and log K~, then the staged
        // potentials, then the values (loads first: the stores go to the
        // same buffer as the indices)
        for (int k0 = 0; k0 < H; k0 += NB) {
          const int nk = min(NB, H - k0);
          unsigned q[NB];
          float lk[NB], o[NB];
#pragma unroll
          for (int u = 0; u < NB; ++u) {
            q[u] = 0u;
            lk[u] = neg_inf();
            if (u < nk) {
              const long long so = off + kEllHdr + (long long)(k0 + u) * st;
              q[u] = __ldg(reinterpret_cast<const unsigned short*>(pack + so) + lane);
              lk[u] = __ldg(logk + (so + 64) / vb + lane);
            }
          }
#pragma unroll
          for (int u = 0; u < NB; ++u) o[u] = u < nk ? xs[min(q[u], (unsigned)(jn - 1))] : neg_inf();
#pragma unroll
          for (int u = 0; u < NB; ++u) {
            if (u < nk) {
              float z = neg_inf();
              if (pi != neg_inf() && o[u] != neg_inf()) z = absorbed_z(lk[u], pi, o[u], A.inv_eps);
              if (pass == 0) {
                m = fmaxf(m, z);
              } else {
                const long long so = off + kEllHdr + (long long)(k0 + u) * st;
                val[(so + 64) / vb + lane] = from_d<V>((double)absorbed_value(z, ei));
              }
            }
          }
        }
        if (pass == 0 && mine) mx[row] = fmaxf(mx[row], m);
        off += ell_group_bytes(H, vb);
      }
      off = max(off, pe);
    }
    __syncthreads();
    if (pass == 0) {
      for (int k = threadIdx.x; k < nr; k += blockDim.x) {
        const float e = absorbed_exponent(mx[k]);
        mx[k] = e;
        e_out[r0 + k] = e;
      }
      __syncthreads();
    }
  }
}

// The first absorption of a staged solve, in copy order (block b of the
// staged kernel's grid owns the same rows and columns here).
template <typename V>
__global__ void __launch_bounds__(kStgThreads, 1) k_absorb_pack(LogArgs A) {
  extern __shared__ __align__(16) float absorb_sh[];   // W entries of the other side's potentials, then rows
  if (*(volatile int*)&A.ctrl->ell_overflow) return;
  ell_absorb<V, 16>(A, 0, absorb_sh, absorb_sh + A.W);
  ell_absorb<V, 16>(A, 1, absorb_sh, absorb_sh + A.W);
}

// Fold the scalings of the pair t into the potentials (this block's rows and
// columns) and reset them to 1.
__device__ __forceinline__ void fold_scalings(const LogArgs& A, int t) {
  float* u = A.ubuf + (size_t)(t & 1) * A.n;
  float* v = A.vbuf + (size_t)(t & 1) * A.m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
    const float ui = u[i];
    if (ui > 0.0f) {
      const float al = A.alpha[i] + A.eps * logf(ui);
      A.alpha[i] = al;
      u[i] = 1.0f;
      A.ahat[i] = A.uot ? A.a[i] * expf(-al * A.inv_lam) : A.a[i];
    }
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < A.m; j += gridDim.x * blockDim.x) {
    const float vj = v[j];
    if (vj > 0.0f) {
      const float be = A.beta[j] + A.eps * logf(vj);
      A.beta[j] = be;
      v[j] = 1.0f;
      A.bhat[j] = A.uot ? A.b[j] * expf(-be * A.inv_lam) : A.b[j];
    }
  }
}

template <typename V>
__device__ __forceinline__ void rewrite_block(const LogArgs& A) {
  const int lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const int gw = blockIdx.x * nw + (threadIdx.x >> 5);
  const int tw = gridDim.x * nw;
  const AbsorbOut<V> R = absorb_out<V>(A, 0), C = absorb_out<V>(A, 1);
  for (int i = gw; i < A.n; i += tw)
    absorb_segment<V>(A.row_ptr[i], A.row_ptr[i + 1], A.col_idx, A.logval, A.alpha[i], A.beta, A.inv_eps, R.out,
                      A.erow + i, lane, R.perm, R.limit, A.ctrl);
  for (int j = gw; j < A.m; j += tw)
    absorb_segment<V>(A.col_ptr[j], A.col_ptr[j + 1], A.row_idx, A.logvalT, A.beta[j], A.alpha, A.inv_eps, C.out,
                      A.ecol + j, lane, C.perm, C.limit, A.ctrl);
}

// Persistent stabilised iterations.  Partial slots: 0 residual, 1 unreachable
// a-mass, 3 unreachable b-mass, 5 / 7 max |log u~| (by the parity of t: the
// row phase of the next iteration writes it before any barrier while slower
// blocks may still read this iteration's values), 6 max |log v~|.
template <int LR, int LC, typename V, bool UOT, bool STG>
__global__ void __launch_bounds__(STG ? kStgThreads : kIterThreads, 1) k_iterate_log(LogArgs A, int iters, int row_only) {
  __shared__ float sh[3 * 32 + 64];
  __shared__ int absorb_now;
  extern __shared__ __align__(16) float dsm[];   // staged chunk of the gathered vector, then row sums
  Ctrl* ctrl = A.ctrl;
  if (ctrl->done) return;
  // staged launches read the grouped copies unless the sketch did not fit them
  const bool grp = STG && !*(volatile int*)&ctrl->ell_overflow;
  int t = ctrl->t;
  for (int k = 0; k < iters; ++k) {
    float r3[3];
    if constexpr (STG) {
      if (grp) log_row_phase_staged<V, UOT>(A, t, r3, sh, dsm);
      else log_row_phase<LR, V, UOT>(A, t, r3, sh);
    } else {
      log_row_phase<LR, V, UOT>(A, t, r3, sh);
    }
    if (threadIdx.x == 0) {
      A.part[0 * (size_t)A.nblk + blockIdx.x] = r3[0];
      A.part[1 * (size_t)A.nblk + blockIdx.x] = r3[1];
      A.part[(size_t)(5 + 2 * (t & 1)) * A.nblk + blockIdx.x] = r3[2];
    }
    if (!grid_barrier(ctrl)) return;
    if (blockIdx.x == 0) {
      if (threadIdx.x < 32) {
        float s0 = 0.f, s1 = 0.f;
        for (int b = threadIdx.x; b < A.nblk; b += 32) {
          s0 += (float)__ldcg(A.part + b);
          s1 += (float)__ldcg(A.part + (size_t)A.nblk + b);
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        if (threadIdx.x == 0) {
          const double res = (double)s0, unr = (double)s1;
          ctrl->last_residual = res;
          ctrl->last_unreach_a = unr;
          if (!ctrl->done) {
            const int numeric = !isfinite(res);
            if (numeric || (t >= 1 && res <= A.tol)) {
              ctrl->iters = t; ctrl->residual = res; ctrl->unreach_a = unr;
              if (numeric) ctrl->status = SPS_ERR_NUMERIC;
              __threadfence();
              ctrl->done = 1;
            }
          }
        }
      }
      __syncthreads();
    }
    if (row_only) return;
    float c2[2];
    if constexpr (STG) {
      if (grp) log_col_phase_staged<V, UOT>(A, t, c2, sh, dsm);
      else log_col_phase<LC, V, UOT>(A, t, c2, sh);
    } else {
      log_col_phase<LC, V, UOT>(A, t, c2, sh);
    }
    if (threadIdx.x == 0) {
      A.part[3 * (size_t)A.nblk + blockIdx.x] = c2[0];
      A.part[6 * (size_t)A.nblk + blockIdx.x] = c2[1];
    }
    if (!grid_barrier(ctrl)) return;
    if (*(volatile int*)&ctrl->done) return;
    // every block takes the same absorption decision from the same partials
    if (threadIdx.x < 32) {
      float mu = 0.f, mv = 0.f, ub = 0.f;
      for (int b = threadIdx.x; b < A.nblk; b += 32) {
        mu = fmaxf(mu, (float)__ldcg(A.part + (size_t)(5 + 2 * (t & 1)) * A.nblk + b));
        mv = fmaxf(mv, (float)__ldcg(A.part + 6 * (size_t)A.nblk + b));
        if (blockIdx.x == 0) ub += (float)__ldcg(A.part + 3 * (size_t)A.nblk + b);
      }
      mu = warp_max(mu);
      mv = warp_max(mv);
      ub = warp_sum(ub);
      if (threadIdx.x == 0) {
        absorb_now = (fmaxf(mu, mv) > A.tau) ? 1 : 0;
        if (blockIdx.x == 0) {
          ctrl->unreach_b = (double)ub;
          ctrl->t = t + 1;
          ctrl->max_logu = mu;
          ctrl->max_logv = mv;
        }
      }
    }
    __syncthreads();
    if (absorb_now) {
      fold_scalings(A, t + 1);
      if (!grid_barrier(ctrl)) return;
      if constexpr (STG) {
        if (grp) {
          ell_absorb<V, 8>(A, 0, dsm, dsm + A.W);   // inside the persistent kernel: its register budget
          ell_absorb<V, 8>(A, 1, dsm, dsm + A.W);
        } else {
          rewrite_block<V>(A);
        }
      } else {
        rewrite_block<V>(A);
      }
      if (!grid_barrier(ctrl)) return;
      if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->n_absorb += 1;
    }
    ++t;
  }
}

template <int LR, int LC, typename V, bool UOT, bool STG>
bool coop_log(LogArgs A, int iters, int row_only, cudaStream_t st) {
  auto fn = k_iterate_log<LR, LC, V, UOT, STG>;
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  size_t smem = 0;
  if (STG) {
    // one block per SM owns a fixed row range and column range
    smem = ell_smem_bytes(A.W, std::max(A.rows_pb, A.cols_pb));
    if (cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
  }
  const int threads = STG ? kStgThreads : kIterThreads;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  if (STG) {
    // the grouped copies were laid out for one block per SM of this device
    if ((int64_t)A.rows_pb * nsm < A.n || (int64_t)A.cols_pb * nsm < A.m || A.sblk != nsm) return false;
    A.nblk = nsm;
  } else {
    A.nblk = std::min(A.nblk, nsm * per_sm);
  }
  void* args[] = {(void*)&A, (void*)&iters, (void*)&row_only};
  if (cudaLaunchCooperativeKernel((const void*)fn, dim3(A.nblk), dim3(threads), args, smem, st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

template <int LR, typename V, bool UOT>
bool coop_log_lc(const LogArgs& A, int lc, int iters, int row_only, cudaStream_t st) {
  if (lc >= 32) return coop_log<LR, 32, V, UOT, false>(A, iters, row_only, st);
  if (lc >= 16) return coop_log<LR, 16, V, UOT, false>(A, iters, row_only, st);
  return coop_log<LR, 8, V, UOT, false>(A, iters, row_only, st);
}

template <typename V, bool UOT>
bool coop_log_dispatch(const LogArgs& A, int lr, int lc, int iters, int row_only, cudaStream_t st) {
  if (A.stage) {
    // staged segments are a row's share of one chunk: one lane count for both passes
    if (lr >= 32) return coop_log<32, 32, V, UOT, true>(A, iters, row_only, st);
    if (lr >= 16) return coop_log<16, 16, V, UOT, true>(A, iters, row_only, st);
    if (lr >= 8) return coop_log<8, 8, V, UOT, true>(A, iters, row_only, st);
    return coop_log<4, 4, V, UOT, true>(A, iters, row_only, st);
  }
  if (lr >= 32) return coop_log_lc<32, V, UOT>(A, lc, iters, row_only, st);
  if (lr >= 16) return coop_log_lc<16, V, UOT>(A, lc, iters, row_only, st);
  return coop_log_lc<8, V, UOT>(A, lc, iters, row_only, st);
}

LogArgs make_log_args(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic) {
  LogArgs A;
  A.n = pd.n; A.m = pd.m;
  A.row_ptr = at<int>(ws, L.row_ptr); A.col_idx = at<int>(ws, L.col_idx);
  A.col_ptr = at<int>(ws, L.col_ptr); A.row_idx = at<int>(ws, L.row_idx);
  A.val = ws + L.val; A.valT = ws + L.valT;
  A.logval = at<float>(ws, L.logval); A.logvalT = at<float>(ws, L.logvalT);
  A.ubuf = at<float>(ws, L.u); A.vbuf = at<float>(ws, L.v);
  A.alpha = at<float>(ws, L.alpha); A.beta = at<float>(ws, L.beta);
  A.ahat = at<float>(ws, L.ahat); A.bhat = at<float>(ws, L.bhat);
  A.erow = at<float>(ws, L.erow); A.ecol = at<float>(ws, L.ecol);
  A.a = at<float>(ws, L.a_it); A.b = at<float>(ws, L.b_it);
  A.eps = (float)ic.eps; A.inv_eps = (float)(1.0 / ic.eps);
  A.lam = ic.uot ? (float)(ic.phi * ic.eps / (1.0 - ic.phi)) : 0.0f;
  A.inv_lam = ic.uot ? (float)((1.0 - ic.phi) / (ic.phi * ic.eps)) : 0.0f;
  A.phi = (float)ic.phi; A.inv_phi = (float)(1.0 / ic.phi); A.tol = (float)ic.tol; A.tau = (float)ic.tau;
  A.uot = ic.uot;
  A.ctrl = at<Ctrl>(ws, L.ctrl); A.part = at<double>(ws, L.part); A.nblk = L.nblk_rows;
  A.stage = L.stage_w > 0 ? 1 : 0;
  A.W = L.stage_w; A.Jr = L.stage_jr; A.Jc = L.stage_jc;
  A.rows_pb = L.stage_nsm > 0 ? (pd.n + L.stage_nsm - 1) / L.stage_nsm : 0;
  A.cols_pb = L.stage_nsm > 0 ? (pd.m + L.stage_nsm - 1) / L.stage_nsm : 0;
  A.seg_r = A.stage ? at<int>(ws, L.seg_r) : nullptr;
  A.seg_c = A.stage ? at<int>(ws, L.seg_c) : nullptr;
  A.sblk = L.stage_nsm;
  for (int s = 0; s < 2; ++s) {
    A.el_slice[s] = A.stage ? at<int>(ws, L.el_slice[s]) : nullptr;
    A.el_pbytes[s] = A.stage ? at<long long>(ws, L.el_pbytes[s]) : nullptr;
    A.el_poff[s] = A.stage ? at<long long>(ws, L.el_poff[s]) : nullptr;
    A.el_tmp[s] = A.stage ? at<int>(ws, L.el_tmp[s]) : nullptr;
    A.el_pack[s] = A.stage ? at<unsigned char>(ws, L.el_pack[s]) : nullptr;
    A.el_logk[s] = A.stage ? at<float>(ws, L.el_logk[s]) : nullptr;
  }
  A.pack_lim = A.stage ? L.el_pack_cap : 0;
  A.nnz_lim = L.cap;
  return A;
}

template <typename V>
void log_iterate_v(const LogArgs& A, const IterCfg& ic, int iters, int row_only, cudaStream_t st, bool* ok) {
  *ok = ic.uot ? coop_log_dispatch<V, true>(A, ic.lpr_rows, ic.lpr_cols, iters, row_only, st)
               : coop_log_dispatch<V, false>(A, ic.lpr_rows, ic.lpr_cols, iters, row_only, st);
}

// ----------------------------------------------------------------------------
// Objective over the support with T~_ij = exp(logK~_ij + (A_i + B_j)/eps),
// A = alpha + eps log u~, B = beta + eps log v~ of the returned pair.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double kl_term_d(double x, double y) {
  if (x == 0.0) return y;
  if (y == 0.0) return __longlong_as_double(0x7ff0000000000000LL);
  return x * log(x / y) - x + y;
}

__global__ void k_log_potentials(LogArgs A, float* al_out, float* be_out) {
  const Ctrl* ctrl = A.ctrl;
  const int it = ctrl->done ? ctrl->iters : ctrl->t;
  const float* u = A.ubuf + (size_t)(it & 1) * A.n;
  const float* v = A.vbuf + (size_t)(it & 1) * A.m;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  for (int i = tid; i < A.n; i += st) al_out[i] = u[i] > 0.0f ? A.alpha[i] + A.eps * logf(u[i]) : neg_inf();
  for (int j = tid; j < A.m; j += st) be_out[j] = v[j] > 0.0f ? A.beta[j] + A.eps * logf(v[j]) : neg_inf();
}

template <bool UOT>
__global__ void __launch_bounds__(kT) k_log_obj_rows(ProbDev pd, const SketchScalars* __restrict__ scp, LogArgs A,
                                                     const float* __restrict__ rowf, const float* __restrict__ colf,
                                                     const float* Apot, const float* Bpot, double* part, int nblk) {
  __shared__ double sh[32];
  const SketchScalars sc = *scp;
  const int lane = threadIdx.x & 31;
  double tr = 0.0, ne = 0.0, lp = 0.0, ms = 0.0, kla = 0.0;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < pd.n; i += (gridDim.x * blockDim.x) >> 5) {
    const float Ai = Apot[i];
    float rtr = 0.f, rne = 0.f, rlp = 0.f, rs = 0.f;
    if (Ai != neg_inf()) {
      const float ri = rowf[i];
      for (int k = A.row_ptr[i] + lane; k < A.row_ptr[i + 1]; k += 32) {
        const int j = A.col_idx[k];
        const float Bj = Bpot[j];
        if (Bj == neg_inf()) continue;
        const float z = A.logval[k] + (Ai + Bj) * A.inv_eps;   // log T~_ij
        const float T = expf(z);
        if (!(T > 0.0f)) continue;
        float D = 0.0f;
        const float p = pstar_raw<UOT>(pd, sc, ri, colf, i, j, &D);
        const float ps = p < 1.0f ? p : 1.0f;
        const float C = pd.cost_kind == SPS_COST_WFR ? (float)value_cost64(pd, sc, i, j)
                                                     : __fdiv_rn(UOT ? D : raw32(pd.cv, i, j), sc.dn32);
        rtr += T * C;
        rne += T * (z - 1.0f);
        rlp += T * logf(ps);
        rs += T;
      }
    }
    rtr = warp_sum(rtr); rne = warp_sum(rne); rlp = warp_sum(rlp); rs = warp_sum(rs);
    if (lane == 0) {
      tr += rtr; ne += rne; lp += rlp; ms += rs;
      kla += kl_term_d((double)rs, (double)A.a[i]);
    }
  }
  const double vals[5] = {tr, ne, lp, ms, kla};
  for (int p = 0; p < 5; ++p) {
    const double s = block_sum_d(vals[p], sh);
    if (threadIdx.x == 0) part[(size_t)p * nblk + blockIdx.x] = s;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kT) k_log_obj_cols(LogArgs A, const float* Apot, const float* Bpot, double* part,
                                                     int nblk) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31;
  double klb = 0.0;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < A.m; j += (gridDim.x * blockDim.x) >> 5) {
    const float Bj = Bpot[j];
    float cs = 0.f;
    if (Bj != neg_inf())
      for (int k = A.col_ptr[j] + lane; k < A.col_ptr[j + 1]; k += 32) {
        const float Ai = Apot[A.row_idx[k]];
        if (Ai != neg_inf()) cs += expf(A.logvalT[k] + (Ai + Bj) * A.inv_eps);
      }
    cs = warp_sum(cs);
    if (lane == 0) klb += kl_term_d((double)cs, (double)A.b[j]);
  }
  const double s = block_sum_d(klb, sh);
  if (threadIdx.x == 0) part[5 * (size_t)nblk + blockIdx.x] = s;
}

__global__ void k_log_obj_final(const double* part, int nblk, DevResult* out, const Ctrl* ctrl) {
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

int grid1(int64_t items, int per_block) {
  int64_t g = (items + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

template <typename V>
void first_iteration_v(const LogArgs& A, const IterCfg& ic, const void* al0, const void* be0, cudaStream_t st) {
  k_log_init<float><<<grid1(std::max(A.n, A.m), kT), kT, 0, st>>>(A.n, A.m, A.alpha, A.beta, (const float*)al0,
                                                                   (const float*)be0, A.ctrl);
  k_lse_half<<<grid1((int64_t)A.n * 32, kT), kT, 0, st>>>(A.n, A.row_ptr, A.col_idx, A.logval, A.beta, A.a,
                                                         A.alpha, A.eps, A.phi);
  k_lse_half<<<grid1((int64_t)A.m * 32, kT), kT, 0, st>>>(A.m, A.col_ptr, A.row_idx, A.logvalT, A.alpha, A.b,
                                                         A.beta, A.eps, A.phi);
  if (A.stage) {
    // chunk pointers, then the grouped copies (the absorption below writes K' in copy order)
    k_chunk_ptrs<<<grid1((int64_t)A.n * 32, kT), kT, 0, st>>>(A.n, A.row_ptr, A.col_idx, A.W, A.Jr, (int*)A.seg_r);
    k_chunk_ptrs<<<grid1((int64_t)A.m * 32, kT), kT, 0, st>>>(A.m, A.col_ptr, A.row_idx, A.W, A.Jc, (int*)A.seg_c);
    for (int side = 0; side < 2; ++side) {
      const int rows = side ? A.m : A.n, R = side ? A.cols_pb : A.rows_pb, J = side ? A.Jc : A.Jr;
      const int* ptr = side ? A.col_ptr : A.row_ptr;
      const int* idx = side ? A.row_idx : A.col_idx;
      const int* seg = side ? A.seg_c : A.seg_r;
      const long long P = (long long)A.sblk * kEllWarps * J;
      const int slices = A.sblk * kEllWarps;
      k_el_slices<<<(A.sblk * (kEllWarps + 1) + 255) / 256, 256, 0, st>>>(rows, R, A.sblk, ptr, A.el_slice[side]);
      k_el_size<<<(slices + 7) / 8, 256, 0, st>>>(rows, R, A.sblk, J, seg, A.el_slice[side], (int)sizeof(V),
                                                  A.el_pbytes[side], A.ctrl);
      k_el_scan<<<1, 1024, 0, st>>>(P, A.el_pbytes[side], A.el_poff[side], A.pack_lim, (int)sizeof(V), A.ctrl,
                                    side);
      k_el_fill<V><<<(slices + 7) / 8, 256, 0, st>>>(rows, R, A.sblk, J, A.W, seg, idx, A.el_slice[side],
                                                     A.el_poff[side], A.el_tmp[side], A.el_pack[side],
                                                     side ? A.logvalT : A.logval,
                                                     A.el_logk[side], A.nnz_lim, A.pack_lim, A.ctrl);
    }
  }
  if (A.stage) {
    // a refused attribute makes the launch fail, and the caller reports it
    const size_t sm = sizeof(float) * ((size_t)A.W + std::max(A.rows_pb, A.cols_pb));
    cudaFuncSetAttribute((const void*)k_absorb_pack<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_absorb_pack<V><<<A.sblk, kStgThreads, sm, st>>>(A);
  }
  k_absorb_all<V><<<grid1((int64_t)std::max(A.n, A.m) * 32, kT), kT, 0, st>>>(A, 1);
  (void)ic;
}

}  // namespace

sps_status launch_log_first_iteration(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                      const void* init_alpha, const void* init_beta, cudaStream_t st) {
  const LogArgs A = make_log_args(pd, L, ws, ic);
  switch (ic.kd) {
    case SPS_BF16: first_iteration_v<__nv_bfloat16>(A, ic, init_alpha, init_beta, st); break;
    case SPS_F16: first_iteration_v<__half>(A, ic, init_alpha, init_beta, st); break;
    default: first_iteration_v<float>(A, ic, init_alpha, init_beta, st); break;
  }
  add_launches(A.stage ? 15 : 4);
  return cuda_fail(cudaGetLastError(), "log-domain first iteration");
}

static sps_status log_coop(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters, int row_only,
                           cudaStream_t st) {
  const LogArgs A = make_log_args(pd, L, ws, ic);
  bool ok = false;
  switch (ic.kd) {
    case SPS_BF16: log_iterate_v<__nv_bfloat16>(A, ic, iters, row_only, st, &ok); break;
    case SPS_F16: log_iterate_v<__half>(A, ic, iters, row_only, st, &ok); break;
    default: log_iterate_v<float>(A, ic, iters, row_only, st, &ok); break;
  }
  if (!ok) {
    set_error("the device refused the cooperative launch of the stabilised iterations");
    return SPS_ERR_CUDA;
  }
  add_launches(1);
  return cuda_fail(cudaGetLastError(), "log-domain iterations");
}

sps_status launch_log_iterations(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters,
                                 cudaStream_t st) {
  return log_coop(pd, L, ws, ic, iters, 0, st);
}

sps_status launch_log_row_only(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, cudaStream_t st) {
  return log_coop(pd, L, ws, ic, 1, 1, st);
}

sps_status launch_log_objective(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, void* alpha_out,
                                void* beta_out, cudaStream_t st) {
  const LogArgs A = make_log_args(pd, L, ws, ic);
  float* Ap = at<float>(ws, L.pot_a);
  float* Bp = at<float>(ws, L.pot_b);
  k_log_potentials<<<grid1(std::max(A.n, A.m), kT), kT, 0, st>>>(A, Ap, Bp);
  double* part = at<double>(ws, L.part);
  const int nb = L.nblk_rows;
  const SketchScalars* sc = at<SketchScalars>(ws, L.scal);
  if (!pd.sep)   // the template selects the decision rule of p* (Eq. pij-uot or separable)
    k_log_obj_rows<true><<<nb, kT, 0, st>>>(pd, sc, A, at<float>(ws, L.rowf), at<float>(ws, L.colf), Ap, Bp, part, nb);
  else
    k_log_obj_rows<false><<<nb, kT, 0, st>>>(pd, sc, A, at<float>(ws, L.rowf), at<float>(ws, L.colf), Ap, Bp, part, nb);
  k_log_obj_cols<<<nb, kT, 0, st>>>(A, Ap, Bp, part, nb);
  k_log_obj_final<<<1, kT, 0, st>>>(part, nb, at<DevResult>(ws, L.res), A.ctrl);
  int launches = 4;
  if (alpha_out && beta_out) {
    cudaMemcpyAsync(alpha_out, Ap, sizeof(float) * (size_t)pd.n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(beta_out, Bp, sizeof(float) * (size_t)pd.m, cudaMemcpyDeviceToDevice, st);
  }
  add_launches(launches);
  return cuda_fail(cudaGetLastError(), "log-domain objective");
}

}  // namespace sps
