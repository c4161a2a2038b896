// sps_internal.h -- internal declarations of the Spar-Sink CUDA library:
// device control block, workspace layout and the host launchers of each
// kernel family.  Not part of the public ABI (include/sparsink.h).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sparsink.h"
#include "sps_device.cuh"

namespace sps {

// Device-resident control block of one solve.  The iteration kernels read and
// update it, so a chunk of iterations needs no host involvement; the host
// reads it back between chunks.
struct Ctrl {
  int t;                 // completed iterations (pairs (u^t, v^t) formed)
  int done;              // 1: stop (converged or numeric failure)
  int status;            // SPS_OK / SPS_ERR_NUMERIC / SPS_ERR_CAPACITY
  int iters;             // iterations of the returned pair
  unsigned int blocks_a; // last-block counters of the two half-iteration kernels
  unsigned int blocks_b;
  unsigned int blocks_c;
  int n_absorb;          // absorptions performed
  int absorb_req;        // 1: the next absorption step runs
  int cap_exceeded;      // sampled nnz above capacity
  long long nnz;         // sampled nnz
  long long nnz_cols;    // the same counted by columns (must agree)
  double residual;       // residual of the returned pair
  double last_residual;  // residual of the most recent pair evaluated
  double last_unreach_a; // unreachable a-mass of that pair
  double unreach_a;      // of the returned pair
  double unreach_b;      // unreachable b-mass of the current v
  double delta_u;        // ||u^t - u^{t-1}||_1 of the current iteration
  double delta_v;        // ||v^t - v^{t-1}||_1 of the current iteration
  float max_logu;        // max |log u~| over the last row pass (absorbing mode)
  float max_logv;
  unsigned int bar_count; // grid barrier of the persistent iteration kernel: arrivals
  unsigned int bar_gen;   //   and generation
  unsigned long long bar_mono;  // arrivals at the counting grid barrier (a multiple of the grid between launches)
  int wait_timeout;       // a bounded device wait gave up
  int sketch_fault;       // fill disagreed with count (write skipped instead of out of range)
  int pad_overflow;       // single-pass sketch: a padded (row, chunk) slot was too small
  int oob_code;           // a bounds check skipped an access (code of the place; 0: none)
  int ell_overflow;       // staged layout: the grouped copy would not fit its planned space (direct gathers instead)
  long long ell_bytes[2]; // staged layout: bytes of the grouped copies (row pass, column pass)
  long long oob_index;    //   and the index it refused
};

// Scalars of the sampling decision, computed on the device.
struct SketchScalars {
  float dmax32;       // max raw binary32 cost
  float maxa, maxb;   // max of the row / column factor bases
  float s32;          // fl32(s)
  double dmax64;      // max raw FP64 cost (FP64 value path)
  double sum1, sum2;  // OT: exact sum sqrt(a), sqrt(b); UOT: exact Z in sum1
  float scale32;      // OT: fl32(1/(sum1 sum2)); UOT: fl32(s/Z)
  float gamma32;      // UOT exponent lam/(2 lam + eps)
  float kappa32;      // UOT: fl32(1/(Dnorm (2 lam + eps)))
  float dn32;         // value path: cost normaliser (binary32)
  double dn64;        // value path: cost normaliser (FP64)
  float cmax32;       // skip sampler: max_j of the column factors (exact)
  float inv2eta32;    // WFR: fl32(1/(2 eta))
  float g2_32;        // WFR UOT decision: fl32(2/(2 lam + eps)), K^{eps/(2 lam + eps)} = cos^{g2}
  ExactAcc acc1, acc2;
};

// Result record assembled on the device at the end of a solve.
struct DevResult {
  double residual, obj, obj_sparse, transport, neg_entropy, logp, mass, kl_a, kl_b;
  double unreach_a, unreach_b;
};

enum IterType { IT_F32 = 0, IT_F64 = 1 };

// Byte offsets of every buffer inside the caller's workspace.
struct Layout {
  size_t ctrl, scal, res;
  size_t x32, y32, a32, b32, C32;   // binary32 copies for the decision
  size_t a_it, b_it;                // weights in the iterate type
  size_t rowf, colf;                // decision factors
  size_t row_cnt, row_ptr, col_cnt, col_ptr, col_cur, cnt2;
  size_t col_idx, val, row_idx, valT, csr_pos, tmp_row, tmp_src;
  size_t u, v, alpha, beta, ahat;   // iterates (u: two buffers)
  size_t qpart, rpart;              // dense: split partial vectors
  size_t logval, logvalT;           // log-domain: log K~ in CSR / CSC order (binary32)
  size_t bhat, erow, ecol, pot_a, pot_b;
  size_t seg_r, seg_c;              // staged gathers: chunk pointers of the CSR rows / CSC columns
  // staged gathers, per side (0: row pass over the CSR, 1: column pass over the CSC): the grouped copy
  size_t el_slice[2];               //   warp slices of every block: block-local row bounds [nblk][kEllWarps + 1]
  size_t el_pbytes[2];              //   bytes of every part (block, slice, chunk)
  size_t el_poff[2];                //   their exclusive prefix sums [parts + 1]
  size_t el_tmp[2];                 //   layout scratch: (row, length, start) of every run of one slice
  size_t el_pack[2];                //   the grouped copy
  size_t el_logk[2];                //   log K~ by value slot (-inf in padding), for absorptions in copy order
  int64_t el_pack_cap;              //   bytes planned for one grouped copy
  size_t pad_ofs, pad_col, pad_val, pad_lv, zsum, csum;   // single-pass sketch (0: two passes)
  size_t unit_r, unit_c;            // persistent iterations: unit starts over rows [n + 2] / columns [m + 2]
  size_t cmx;                       // pruned cost maximum: scratch (0: the full sweep only)
  int64_t pad_cap;
  int stage_w, stage_jr, stage_jc;  // staged gathers: chunk width, chunks over columns / rows (0: off)
  int stage_nsm;                    // SM count the staging was planned for (one block per SM)
  int stage_vb;                     // bytes of a stored value of the grouped copy
  size_t part;                      // block partials
  size_t total;
  int64_t cap;                      // sketch capacity (elements)
  int nblk_rows, nblk_cols;         // grid sizes of the half-iteration kernels
  int vbytes, ibytes;               // value / iterate element sizes
};

// Staged stabilised passes (sps_logdom.cu).  Block b (one per SM) owns a row
// range; warp w of the block owns a slice of those rows (slices hold about
// equal element counts).  A part is (block, slice, chunk of W columns): the
// runs of the slice's rows inside the chunk.  Each part is stored as groups
// of 32 runs sorted by run length (longest first), lane l of the warp walking
// run l:
//   bytes [0, 64)        32 block-local rows (u16; 0xFFFF: no run),
//   bytes [64, 68)       the group's height h (int), the length of its first run,
//   bytes [68, 72)       the height of the next group of the slice's stream (0: none),
//   bytes [72, 80)       zero,
//   then h steps of 32 x (2 + vb) bytes: 32 chunk-local indices (u16), then
//   32 values (V); step k holds element k of every run of the group, a run
//   shorter than h padded with index 0 and value 0.
// Parts follow each other in (block, slice, chunk) order, so that a warp's
// pass over its slice is one contiguous byte range; the warp streams it
// through a ring of kEllRing bytes of shared memory in windows of kEllWin.
constexpr int kEllWarps = 16;                      // warps (slices) of the staged kernel's block
constexpr int kStgThreads = 32 * kEllWarps;        // its threads
constexpr int kEllHdr = 80;                        // bytes of a group header
constexpr int kEllBins = 256;                      // run-length bins of the sort (the last one holds >= 255)
constexpr int kEllRing = 4096;                     // ring of one warp (a power of two)
constexpr int kEllWin = 1024;                      // window: two 16-byte copies per lane
constexpr int kEllPrefetch = 8;                    // windows of a warp's stream prefetched into L2 beyond its ring
__host__ __device__ constexpr long long ell_step_bytes(int vb) { return 32LL * (2 + vb); }
__host__ __device__ constexpr long long ell_group_bytes(int h, int vb) { return kEllHdr + (long long)h * ell_step_bytes(vb); }
// Dynamic shared memory of the staged kernel: the chunk of the gathered
// vector (W entries), the block's row sums (128-byte aligned), the rings.
__host__ __device__ constexpr size_t ell_acc_offset(int W) { return (size_t)W * 4; }
__host__ __device__ constexpr size_t ell_ring_offset(int W, int rows) { return ((size_t)W * 4 + (size_t)rows * 4 + 127) & ~(size_t)127; }
__host__ __device__ constexpr size_t ell_smem_bytes(int W, int rows) { return ell_ring_offset(W, rows) + (size_t)kEllWarps * kEllRing; }

constexpr int kPartSlots = 8;      // partial arrays of nblk doubles each
constexpr int kMaxBlocks = 4096;

bool plan_layout(const sps_problem* P, const sps_params* Q, int op, Layout* L);

inline size_t dtype_bytes(sps_dtype t) {
  switch (t) {
    case SPS_F64: return 8;
    case SPS_F32: return 4;
    default: return 2;
  }
}

#define SPS_TRY(x)                     \
  do {                                 \
    sps_status _s = (x);               \
    if (_s != SPS_OK) return _s;       \
  } while (0)

// ---- error reporting and launch accounting ----
void add_launches(int k);
void set_error(const char* fmt, ...);
sps_status cuda_fail(cudaError_t e, const char* what);

// Kernel argument bundles -----------------------------------------------------
struct ProbDev {
  int n, m, d;
  CostView cv;
  const void* a;       // input weights (dtype)
  const void* b;
  int in_f64;          // 1: inputs FP64
  int cost_norm;
  double cost_scale;
  double eps, lam, s;
  int is_ot;           // balanced OT (lam = +inf): Alg. 1 iterations
  int sep;             // the decision factors as r_i c_j: Eq. (pij-ot), or the equal probabilities
  int probs;           // SPS_PROBS_*
  int cost_kind;       // SPS_COST_SQEUCLID / SPS_COST_WFR
  double eta;          // WFR length scale
  uint64_t seed;
  uint32_t pid;
};

// Sweep geometry (sps_sweep.cu): column chunks of the n x m sweeps.
struct SweepGeo { int nchunk, chunk, row_blocks; };
SweepGeo sweep_geometry(int n, int m);
void launch_uot_Z(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st);
void launch_count(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st);
void launch_fill(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st);
// Single pass: padded slots from the expected counts, then the sweep (counts and
// entries together); the caller reads pad_overflow and either compacts or
// falls back to launch_count / launch_fill.
void launch_fused(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st);
void launch_compact(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st);
void launch_sum_chunks(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st);

// Host launchers (sps_sketch.cu)
sps_status launch_prepare(const ProbDev& pd, const Layout& L, char* ws, int it64, cudaStream_t st);
sps_status launch_cost_max(const ProbDev& pd, const Layout& L, char* ws, int need64, cudaStream_t st);
sps_status launch_factors(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st);
sps_status launch_sample(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st);
sps_status launch_scalars0(const ProbDev& pd, const Layout& L, char* ws, cudaStream_t st);

// Host launchers (sps_iter.cu)
struct IterCfg {
  int it64;            // iterate in FP64
  sps_dtype kd;        // value dtype
  int uot;             // Alg. 2 exponent
  double phi, eps, tol;
  int stop_rule;
  int max_iter;
  int lpr_rows = 32;   // lanes per row of the row pass (8, 16, 32)
  int lpr_cols = 32;   // lanes per column of the column pass
  int persistent = 1;  // run chunks of iterations in one cooperative launch
  int log_domain = 0;  // stabilised iterations with absorption
  double tau = 12.0;   // absorption threshold on max |log u~|, |log v~|
  int dense = 0;       // dense Sinkhorn (log_domain: log-sum-exp form)
};
sps_status launch_iter_init(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                            const void* init_alpha, const void* init_beta, cudaStream_t st);
sps_status launch_sparse_iterations(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                    int iters, cudaStream_t st);
sps_status launch_log_first_iteration(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                      const void* init_alpha, const void* init_beta, cudaStream_t st);
sps_status launch_log_iterations(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters,
                                 cudaStream_t st);
sps_status launch_log_row_only(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, cudaStream_t st);
sps_status launch_log_objective(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, void* alpha_out,
                                void* beta_out, cudaStream_t st);
sps_status launch_sparse_row_only(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                  cudaStream_t st);
sps_status launch_sparse_objective(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                   void* alpha_out, void* beta_out, cudaStream_t st);

// Host launchers (sps_dense.cu)
sps_status launch_dense_iterations(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                   int iters, cudaStream_t st);
sps_status launch_dense_row_only(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                 cudaStream_t st);
size_t dense_qpart_elems(int n, int m);
size_t dense_rpart_elems(int n, int m);
int dense_pass_blocks(int n, int m);
sps_status launch_dense_objective(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                  void* alpha_out, void* beta_out, cudaStream_t st);
// Dense log-sum-exp form (sps_dense_lse.cu)
sps_status launch_dense_lse_init(const ProbDev& pd, const Layout& L, char* ws, const void* init_alpha,
                                 const void* init_beta, cudaStream_t st);
sps_status launch_dense_lse_iterations(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, int iters,
                                       cudaStream_t st);
sps_status launch_dense_lse_row_only(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                     cudaStream_t st);
sps_status launch_dense_lse_objective(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic,
                                      void* alpha_out, void* beta_out, cudaStream_t st);

// Skip sampler (balanced OT): count, scan, fill and CSC of the sketch (sps_sweep.cu).
sps_status launch_skip_sample(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st);
void launch_csc_sort(const ProbDev& pd, const Layout& L, char* ws, sps_dtype kd, cudaStream_t st);
// Cost divisor by bucketed bounds (sps_costmax.cu); *overflow_flag gates the full sweep.
size_t cost_max_scratch_bytes(int n, int m, int d);
sps_status launch_cost_max_pruned(const float* x, const float* y, int n, int m, int d, SketchScalars* sc,
                                  char* scratch, const int** overflow_flag, cudaStream_t st);
sps_status launch_cost_max_points(const float* x, int n, const float* y, int m, int d, void* scratch,
                                  cudaStream_t st);
// Shared with the batched path (sps_sketch.cu)
void launch_scan_counts(const int* row_cnt, int* row_ptr, int n, const int* col_cnt, int* col_ptr, int* col_cur,
                        int m, long long cap, Ctrl* ctrl, cudaStream_t st);
void launch_csc_sort_f32(int m, const int* col_ptr, const int* tmp_row, const int* tmp_src, const float* val,
                         int* row_idx, int* csr_pos, float* valT, Ctrl* ctrl, cudaStream_t st);

template <typename T> T* at(char* ws, size_t off) { return reinterpret_cast<T*>(ws + off); }

// The binary32 decision factor K_ij^{eps/(2 lam + eps)} = exp(-C_ij/(2 lam + eps))
// of Eq. (pij-uot) from the raw squared distance D.  Squared Euclidean:
// E(-fl(D kappa)).  WFR (section 2.2): with z = fl(fl(sqrt D) fl(1/(2 eta))),
// 0 for z >= fl(pi/2) (transport blocked), else cos_+^2 to the power
// 1/(2 lam + eps) = E(fl(g2 L(cos z))), 0 when the spec cos is not positive.
__device__ __forceinline__ float uot_factor(int wfr, float D, float kappa, float inv2eta, float g2) {
  if (!wfr) return spec_exp(-__fmul_rn(D, kappa));
  const float z = __fmul_rn(__fsqrt_rn(D), inv2eta);
  if (!(z < (float)(0.5 * 3.14159265358979323846))) return 0.0f;
  const float c = spec_cos(z);
  if (!(c > 0.0f)) return 0.0f;
  return spec_exp(__fmul_rn(g2, spec_log(c)));
}

// The Wasserstein-Fisher-Rao cost (section 2.2) of the value path from the
// FP64 squared distance: -2 log cos(sqrt(D) / (2 eta)), +inf where the angle
// reaches pi/2.
__device__ __forceinline__ double wfr_cost64(double D, double eta) {
  const double z = sqrt(D) / (2.0 * eta);
  if (z >= 0.5 * 3.14159265358979323846) return __longlong_as_double(0x7ff0000000000000LL);
  return -2.0 * log(cos(z));
}

// p*_ij before clipping at 1, in the binary32 decision spec.
//   separable (Eq. pij-ot, or equal probabilities): fl(r_i c_j)
//   UOT (Eq. pij-uot): fl(scale fl(fl(A_i B_j) F(D_ij))), F = uot_factor
// D receives the binary32 raw cost when it is computed (UOT).
template <bool UOT>
__device__ __forceinline__ float pstar_raw(const ProbDev& pd, const SketchScalars& sc, float ri,
                                           const float* colf, int i, int j, float* D) {
  if (!UOT) return __fmul_rn(ri, colf[j]);
  const float Dij = raw32(pd.cv, i, j);
  *D = Dij;
  const float f = uot_factor(pd.cost_kind == SPS_COST_WFR, Dij, sc.kappa32, sc.inv2eta32, sc.g2_32);
  const float w = __fmul_rn(__fmul_rn(ri, colf[j]), f);
  return __fmul_rn(sc.scale32, w);
}

// The cost of the value path at a sampled element, C_ij in FP64: the WFR cost
// of the FP64 distance, or the raw FP64 cost over its divisor.
__device__ __forceinline__ double value_cost64(const ProbDev& pd, const SketchScalars& sc, int i, int j) {
  const double D = raw64(pd.cv, i, j);
  return pd.cost_kind == SPS_COST_WFR ? wfr_cost64(D, pd.eta) : D / sc.dn64;
}

}  // namespace sps
