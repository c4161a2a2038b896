// sps_api.cu -- the C ABI (include/sparsink.h): argument checks, workspace
// planning and the host orchestration of the sketch, the iterations and the
// objective.  Nothing here allocates device memory; every buffer is a slice
// of the caller's workspace.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "sps_internal.h"

namespace sps {

static thread_local char g_err[512] = "";
static thread_local int g_launches = 0;

void add_launches(int k) { g_launches += k; }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

sps_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SPS_OK;
  set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return SPS_ERR_CUDA;
}

static int64_t sketch_capacity(const sps_problem* P, const sps_params* Q) {
  const double nm = (double)P->n * (double)P->m;
  double cap = ceil(Q->s + 8.0 * sqrt(Q->s) + 1024.0);
  if (cap > nm) cap = nm;
  if (cap > 2147483647.0) cap = 2147483647.0;
  return (int64_t)cap;
}

// Staged gathers for the stabilised iterations: when both scaling vectors are
// too long to stay in L1 (2^16 entries and more), every block streams the
// gathered vector through shared memory in chunks of W entries, one block per
// SM.  W is the largest multiple of 1024 (at most 48K entries) that leaves room
// for the block's own row sums and its warps' stream rings, balanced over the
// chunks.  The sketch is read
// from a grouped copy per pass (runs of 32 rows sorted by length, 16-bit
// chunk-local indices); its size depends on the run lengths, so it is planned
// generously and, when a sketch does not fit, the passes gather directly.
constexpr int kStageMin = 1 << 16;
constexpr int kStageWMax = 48 * 1024;
constexpr size_t kStageSmem = 227 * 1024 - 1024;   // dynamic shared memory of one block

template <typename Take>
static void plan_staging(int n, int m, int mode, int kd, Layout* L, Take& take) {
  if (mode == SPS_GATHER_DIRECT) return;
  if (mode == SPS_GATHER_AUTO && (n < kStageMin || m < kStageMin)) return;
  if (L->cap <= 0) return;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      nsm < 1) {
    cudaGetLastError();
    return;
  }
  const int big = std::max(n, m);
  const size_t acc = (size_t)((big + nsm - 1) / nsm);   // row sums of one block
  if (ell_smem_bytes(8192, (int)acc) > kStageSmem) return;
  if (acc >= 65535) return;   // the grouped copy names block-local rows in 16 bits (0xFFFF: none)
  const size_t fixed = ell_smem_bytes(0, (int)acc) + 128;   // row sums, rings, alignment
  const int wcap = std::min<int>(kStageWMax, (int)(((kStageSmem - fixed) / 4) / 1024 * 1024));
  int J = (big + wcap - 1) / wcap;
  if (mode == SPS_GATHER_STAGED) J = std::max(J, std::min(4, (big + 1023) / 1024));   // forced: several chunks
  const int W = (int)(((big + J - 1) / J + 1023) / 1024 * 1024);
  L->stage_w = W;
  L->stage_jr = (m + W - 1) / W;
  L->stage_jc = (n + W - 1) / W;
  L->stage_nsm = nsm;
  const int vb = (kd == SPS_BF16 || kd == SPS_F16) ? 2 : 4;   // the stabilised passes store K' in 16 or 32 bits
  L->stage_vb = vb;
  L->seg_r = take((size_t)(L->stage_jr + 1) * n * 4);
  L->seg_c = take((size_t)(L->stage_jc + 1) * m * 4);
  const size_t parts[2] = {(size_t)nsm * kEllWarps * L->stage_jr, (size_t)nsm * kEllWarps * L->stage_jc};
  const int rows[2] = {n, m};
  // A part's groups are sorted, so each group's height is at most the shortest
  // run of the group before it: a part holds at most its elements plus 32 x
  // its longest run h0 of (2 + vb)-byte steps, and a header per 32 runs plus
  // one.  The plan takes h0 <= 3 x the mean run + 16 (sketches of independent
  // inclusions stay far below; a sketch that does not fit falls back to
  // direct gathers).
  int64_t need = 0;
  for (int s = 0; s < 2; ++s) {
    const int J = s ? L->stage_jc : L->stage_jr;
    const int64_t h0 = 3 * ((L->cap + (int64_t)rows[s] * J - 1) / ((int64_t)rows[s] * J)) + 16;
    need = std::max<int64_t>(need, (int64_t)(2 + vb + 3) * L->cap + (int64_t)parts[s] * (kEllHdr + 32 * (2 + vb) * h0));
  }
  L->el_pack_cap = (need + 15) & ~(int64_t)15;
  for (int s = 0; s < 2; ++s) {
    L->el_slice[s] = take((size_t)nsm * (kEllWarps + 1) * 4);
    L->el_pbytes[s] = take(parts[s] * 8);
    L->el_poff[s] = take((parts[s] + 1) * 8);
    L->el_tmp[s] = take((size_t)rows[s] * 12);
    L->el_pack[s] = take((size_t)L->el_pack_cap);
    L->el_logk[s] = take((size_t)(L->el_pack_cap / vb) * 4);
  }
}

bool plan_layout(const sps_problem* P, const sps_params* Q, int op, Layout* L) {
  memset(L, 0, sizeof(*L));
  const int n = P->n, m = P->m, d = P->d;
  const bool it64 = Q->kdtype == SPS_F64;
  const size_t ib = it64 ? 8 : 4;
  const size_t vb = dtype_bytes(Q->kdtype);
  const bool in64 = P->dtype == SPS_F64;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  L->ctrl = take(sizeof(Ctrl));
  L->scal = take(sizeof(SketchScalars));
  L->res = take(sizeof(DevResult));
  if (in64 && !P->C) {
    L->x32 = take((size_t)n * d * 4);
    L->y32 = take((size_t)m * d * 4);
  }
  if (in64 && P->C) L->C32 = take((size_t)n * m * 4);
  L->a32 = take((size_t)n * 4);
  L->b32 = take((size_t)m * 4);
  L->a_it = take((size_t)n * ib);
  L->b_it = take((size_t)m * ib);
  L->rowf = take((size_t)n * 4);
  L->colf = take((size_t)m * 4);
  int nb = (int)std::min<int64_t>(152 * 8, std::max<int64_t>(1, ((int64_t)std::max(n, m) + 7) / 8));
  if (op == SPS_OP_SPARSIFY || op == SPS_OP_SPAR_SINK) {
    const int64_t cap = sketch_capacity(P, Q);
    L->cap = cap;
    L->row_cnt = take((size_t)n * 4);
    L->row_ptr = take((size_t)(n + 1) * 4);
    L->col_cnt = take((size_t)m * 4);
    L->col_ptr = take((size_t)(m + 1) * 4);
    L->col_cur = take((size_t)m * 4);
    L->cnt2 = take((size_t)sweep_geometry(n, m).nchunk * n * 4);
    // pruned cost maximum for large point problems (below 1e8 pairs the full sweep is short)
    if (P->cost_norm == SPS_COST_MAXNORM && !P->C && P->d >= 1 && P->d <= 16 && (double)n * (double)m > 1e8)
      L->cmx = take(cost_max_scratch_bytes(n, m, P->d));
    // + 16: staged passes read aligned groups of 8, the ring copies aligned groups of 16
    L->col_idx = take(((size_t)cap + 16) * 4);
    L->val = take(((size_t)cap + 16) * vb);
    L->row_idx = take(((size_t)cap + 16) * 4);
    L->valT = take(((size_t)cap + 16) * vb);
    L->csr_pos = take((size_t)cap * 4);
    L->tmp_row = take((size_t)cap * 4);
    L->tmp_src = take((size_t)cap * 4);
    if (Q->log_domain && op == SPS_OP_SPAR_SINK) {   // sparsify_kernel returns K~ itself
      L->logval = take((size_t)cap * 4);
      L->logvalT = take((size_t)cap * 4);
    }
    // single-pass sketch: padded slots of ceil(mu + 8 sqrt(mu) + 16) per (row, chunk); by Cauchy-Schwarz
    // their total is at most s + 8 sqrt(cells s) + 17 cells (cells = n x chunks; one more per cell for
    // the rounding up), plus a margin for the binary32 sums behind mu
    const SweepGeo g = sweep_geometry(n, m);
    const double cells = (double)n * g.nchunk;
    double pcap = ceil(1.001 * Q->s + 8.0 * sqrt(cells * Q->s) + 17.0 * cells + 1024.0);
    pcap = std::min(pcap, (double)n * (double)m);
    if (Q->sketch_mode == SPS_SKETCH_SINGLE && Q->sampler == SPS_SAMPLER_ELEMENT && pcap < 2147483000.0 &&
        cells * 2.0 + 1.0 < 2147483000.0) {
      L->pad_cap = (int64_t)pcap;
      L->pad_ofs = take((size_t)(2 * cells + 1) * 4);
      L->pad_col = take((size_t)pcap * 4);
      L->pad_val = take((size_t)pcap * vb);   // written unless log K~ is formed in binary32
      if (Q->log_domain && op == SPS_OP_SPAR_SINK) L->pad_lv = take((size_t)pcap * 4);
      if (!isinf(Q->lambda)) L->zsum = take((size_t)cells * 4);
      L->csum = take((size_t)g.nchunk * 4);
    }
  }
  int part_blocks = nb;
  if (op == SPS_OP_DENSE) {
    nb = (int)std::min<int64_t>(152 * 8, std::max<int64_t>(1, ((int64_t)std::max(n, m) + 255) / 256));
    part_blocks = std::max(nb, dense_pass_blocks(n, m));
    // log_domain: a running maximum and a scaled sum per element
    const size_t lf = Q->log_domain ? 2 : 1;
    L->qpart = take(dense_qpart_elems(n, m) * ib * lf);
    L->rpart = take(dense_rpart_elems(n, m) * ib * lf);
  }
  if (op == SPS_OP_SPAR_SINK || op == SPS_OP_DENSE) {
    L->u = take((size_t)2 * n * ib);
    L->v = take((size_t)2 * m * ib);
    L->alpha = take((size_t)n * 4);
    L->beta = take((size_t)m * 4);
    L->ahat = take((size_t)n * 4);
    if (op == SPS_OP_SPAR_SINK && !Q->log_domain) {
      L->unit_r = take((size_t)(n + 2) * 4);
      L->unit_c = take((size_t)(m + 2) * 4);
    }
    if (Q->log_domain) {
      L->bhat = take((size_t)m * 4);
      L->erow = take((size_t)n * 4);
      L->ecol = take((size_t)m * 4);
      L->pot_a = take((size_t)n * 4);
      L->pot_b = take((size_t)m * 4);
      if (op == SPS_OP_SPAR_SINK) plan_staging(n, m, Q->gather_mode, Q->kdtype, L, take);
    }
  }
  L->nblk_rows = nb;
  L->nblk_cols = nb;
  L->part = take((size_t)kPartSlots * part_blocks * sizeof(double));
  L->total = off + 256;
  L->vbytes = (int)vb;
  L->ibytes = (int)ib;
  return true;
}

static bool valid_dtype(int t) { return t >= SPS_F64 && t <= SPS_F16; }

static sps_status validate(const sps_problem* P, const sps_params* Q, int op) {
  if (!P || !Q) { set_error("null problem or params"); return SPS_ERR_INVALID_ARG; }
  if (P->n < 1 || P->m < 1) { set_error("n and m must be >= 1 (n=%d m=%d)", P->n, P->m); return SPS_ERR_INVALID_ARG; }
  if ((double)P->n * (double)P->m >= 4.6e18) { set_error("n*m too large"); return SPS_ERR_INVALID_ARG; }
  if (P->dtype != SPS_F32 && P->dtype != SPS_F64) { set_error("problem dtype must be F32 or F64"); return SPS_ERR_INVALID_ARG; }
  if (!P->C && (!P->x || !P->y || P->d < 1)) { set_error("points x, y (d >= 1) or a cost matrix C are required"); return SPS_ERR_INVALID_ARG; }
  if (!P->a || !P->b) { set_error("weights a and b are required"); return SPS_ERR_INVALID_ARG; }
  if (P->cost_norm < SPS_COST_RAW || P->cost_norm > SPS_COST_SCALE) { set_error("bad cost_norm"); return SPS_ERR_INVALID_ARG; }
  if (P->cost_norm == SPS_COST_SCALE && !(P->cost_scale > 0.0 && isfinite(P->cost_scale))) { set_error("cost_scale must be > 0"); return SPS_ERR_INVALID_ARG; }
  if (!(Q->eps > 0.0) || !isfinite(Q->eps)) { set_error("eps must be > 0 and finite (eps=%g)", Q->eps); return SPS_ERR_INVALID_ARG; }
  if (!(Q->lambda > 0.0)) { set_error("lambda must be > 0 (use +inf for balanced OT)"); return SPS_ERR_INVALID_ARG; }
  if (op != SPS_OP_DENSE && (!(Q->s > 0.0) || !isfinite(Q->s))) { set_error("sample budget s must be > 0 (s=%g)", Q->s); return SPS_ERR_INVALID_ARG; }
  if (!(Q->tol >= 0.0)) { set_error("tol must be >= 0"); return SPS_ERR_INVALID_ARG; }
  if (op != SPS_OP_SPARSIFY && Q->max_iter < 1) { set_error("max_iter must be >= 1"); return SPS_ERR_INVALID_ARG; }
  if (Q->stop_rule != SPS_STOP_RESIDUAL && Q->stop_rule != SPS_STOP_DELTA_UV) { set_error("bad stop_rule"); return SPS_ERR_INVALID_ARG; }
  if (!valid_dtype(Q->kdtype)) { set_error("bad kdtype"); return SPS_ERR_INVALID_ARG; }
  if (op == SPS_OP_DENSE && Q->kdtype != SPS_F64 && Q->kdtype != SPS_F32) { set_error("dense Sinkhorn iterates in F64 or F32"); return SPS_ERR_INVALID_ARG; }
  if (op == SPS_OP_DENSE && !P->C && P->d > 16) { set_error("dense Sinkhorn on points supports d <= 16 (d=%d)", P->d); return SPS_ERR_INVALID_ARG; }
  if (Q->log_domain && op == SPS_OP_DENSE && Q->kdtype != SPS_F32) { set_error("dense log_domain iterates in F32"); return SPS_ERR_INVALID_ARG; }
  if (Q->log_domain && Q->kdtype == SPS_F64) { set_error("log_domain stores K' in F32, BF16 or F16"); return SPS_ERR_INVALID_ARG; }
  if (Q->log_domain && Q->stop_rule != SPS_STOP_RESIDUAL) { set_error("log_domain stops on the residual rule"); return SPS_ERR_INVALID_ARG; }
  if (Q->log_domain && !(Q->absorb_tau >= 0.0 && isfinite(Q->absorb_tau))) {
    set_error("absorb_tau must be finite and >= 0 (0 = default)"); return SPS_ERR_INVALID_ARG;
  }
  if (Q->check_every < 0) { set_error("check_every must be >= 0 (0 = automatic)"); return SPS_ERR_INVALID_ARG; }
  if (Q->gather_mode < SPS_GATHER_AUTO || Q->gather_mode > SPS_GATHER_STAGED) { set_error("unknown gather_mode %d", Q->gather_mode); return SPS_ERR_INVALID_ARG; }
  if (Q->sketch_mode != SPS_SKETCH_SINGLE && Q->sketch_mode != SPS_SKETCH_TWO_PASS) { set_error("unknown sketch_mode %d", Q->sketch_mode); return SPS_ERR_INVALID_ARG; }
  if (Q->sampler != SPS_SAMPLER_ELEMENT && Q->sampler != SPS_SAMPLER_SKIP) { set_error("unknown sampler %d", Q->sampler); return SPS_ERR_INVALID_ARG; }
  if (Q->probs != SPS_PROBS_PAPER && Q->probs != SPS_PROBS_EQUAL) { set_error("unknown probs %d", Q->probs); return SPS_ERR_INVALID_ARG; }
  if (P->cost_kind != SPS_COST_SQEUCLID && P->cost_kind != SPS_COST_WFR) {
    set_error("unknown cost_kind %d", P->cost_kind); return SPS_ERR_INVALID_ARG;
  }
  if (P->cost_kind == SPS_COST_WFR) {
    if (P->C) { set_error("the WFR cost is defined from points: give x, y and no cost matrix"); return SPS_ERR_INVALID_ARG; }
    if (P->cost_norm != SPS_COST_RAW) { set_error("the WFR cost takes cost_norm = SPS_COST_RAW"); return SPS_ERR_INVALID_ARG; }
    if (!(P->eta > 0.0) || !isfinite(P->eta)) { set_error("WFR eta must be > 0 and finite (eta=%g)", P->eta); return SPS_ERR_INVALID_ARG; }
    if (op == SPS_OP_DENSE) { set_error("sinkhorn_dense takes the squared Euclidean cost only"); return SPS_ERR_INVALID_ARG; }
  }

  if (op != SPS_OP_DENSE && (double)Q->s + 8.0 * sqrt(Q->s) + 1024.0 > 2147483647.0 &&
      (double)P->n * (double)P->m > 2147483647.0) {
    set_error("sample budget too large for int32 indices"); return SPS_ERR_CAPACITY;
  }
  return SPS_OK;
}

// The sampling probabilities a solve uses (dense Sinkhorn samples nothing).
static int op_probs(const sps_params* Q) { return Q->probs == SPS_PROBS_EQUAL ? SPS_PROBS_EQUAL : SPS_PROBS_PAPER; }

static ProbDev make_probdev(const sps_problem* P, const sps_params* Q, const Layout& L, char* ws) {
  ProbDev pd;
  memset(&pd, 0, sizeof(pd));
  pd.n = P->n; pd.m = P->m; pd.d = P->C ? 0 : P->d;
  const bool in64 = P->dtype == SPS_F64;
  pd.in_f64 = in64;
  if (P->C) {
    pd.cv.C64 = in64 ? (const double*)P->C : nullptr;
    pd.cv.C32 = in64 ? at<float>(ws, L.C32) : (const float*)P->C;
  } else {
    pd.cv.x64 = in64 ? (const double*)P->x : nullptr;
    pd.cv.y64 = in64 ? (const double*)P->y : nullptr;
    pd.cv.x32 = in64 ? at<float>(ws, L.x32) : (const float*)P->x;
    pd.cv.y32 = in64 ? at<float>(ws, L.y32) : (const float*)P->y;
  }
  pd.cv.n = P->n; pd.cv.m = P->m; pd.cv.d = pd.d;
  pd.a = P->a; pd.b = P->b;
  pd.cost_norm = P->cost_norm; pd.cost_scale = P->cost_scale;
  pd.eps = Q->eps; pd.lam = Q->lambda; pd.s = Q->s;
  pd.is_ot = isinf(Q->lambda) ? 1 : 0;
  pd.probs = op_probs(Q);
  pd.sep = (pd.is_ot || pd.probs == SPS_PROBS_EQUAL) ? 1 : 0;
  pd.cost_kind = P->cost_kind;
  pd.eta = P->cost_kind == SPS_COST_WFR ? P->eta : 0.0;
  pd.seed = Q->seed; pd.pid = Q->problem_id;
  return pd;
}

static sps_status read_ctrl(const Layout& L, char* ws, Ctrl* h, cudaStream_t st) {
  sps_status s = cuda_fail(cudaMemcpyAsync(h, ws + L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "ctrl read-back");
  if (s != SPS_OK) return s;
  return cuda_fail(cudaStreamSynchronize(st), "stream synchronize");
}


struct Events {
  cudaEvent_t e[5];   // start, sketch done, iterations done, objective done; 4: iteration setup done
  bool ok = false;
  Events() { ok = true; for (auto& x : e) if (cudaEventCreate(&x) != cudaSuccess) ok = false; }
  ~Events() { for (auto& x : e) cudaEventDestroy(x); }
  void rec(int k, cudaStream_t st) { if (ok) cudaEventRecord(e[k], st); }
  float ms(int a, int b) {
    float t = 0.0f;
    if (ok && cudaEventElapsedTime(&t, e[a], e[b]) == cudaSuccess) return t;
    return 0.0f;
  }
};

// Enqueue the sketch; return after reading back its status and nnz.
static sps_status run_sketch(const sps_problem* P, const sps_params* Q, const Layout& L, char* ws, ProbDev& pd,
                             cudaStream_t st, Ctrl* hctrl) {
  SPS_TRY(cuda_fail(cudaMemsetAsync(ws + L.ctrl, 0, sizeof(Ctrl), st), "memset ctrl"));
  SPS_TRY(cuda_fail(cudaMemsetAsync(ws + L.scal, 0, sizeof(SketchScalars), st), "memset scalars"));
  const int it64 = Q->kdtype == SPS_F64;
  SPS_TRY(launch_prepare(pd, L, ws, it64, st));
  if (P->cost_norm == SPS_COST_MAXNORM) SPS_TRY(launch_cost_max(pd, L, ws, 0, st));
  SPS_TRY(launch_factors(pd, L, ws, st));
  if (Q->sampler == SPS_SAMPLER_SKIP) SPS_TRY(launch_skip_sample(pd, L, ws, Q->kdtype, st));
  else SPS_TRY(launch_sample(pd, L, ws, Q->kdtype, st));
  SPS_TRY(read_ctrl(L, ws, hctrl, st));
  if (hctrl->status == SPS_OK && hctrl->nnz != hctrl->nnz_cols) {
    set_error("internal error: row and column counts of the sketch disagree (%lld vs %lld)",
              (long long)hctrl->nnz, (long long)hctrl->nnz_cols);
    return SPS_ERR_CUDA;
  }
  if (hctrl->sketch_fault) {
    set_error("internal error: the fill pass disagreed with the count pass (writes skipped)");
    return SPS_ERR_CUDA;
  }
  if (hctrl->status == SPS_ERR_NUMERIC) {
    set_error("non-finite or negative input weights, or a zero normaliser");
    return SPS_ERR_NUMERIC;
  }
  if (hctrl->status == SPS_ERR_CAPACITY || hctrl->cap_exceeded) {
    set_error("sampled nnz %lld exceeds the workspace capacity %lld", (long long)hctrl->nnz, (long long)L.cap);
    return SPS_ERR_CAPACITY;
  }
  if (hctrl->status != SPS_OK) {
    set_error("non-finite or negative input weights, or a zero normaliser");
    return (sps_status)hctrl->status;
  }
  return SPS_OK;
}

// The iteration driver: chunks of iterations are enqueued back to back; the
// device-side stop flag turns the rest of a chunk into no-ops.
typedef sps_status (*IterFn)(const ProbDev&, const Layout&, char*, const IterCfg&, int, cudaStream_t);
typedef sps_status (*RowFn)(const ProbDev&, const Layout&, char*, const IterCfg&, cudaStream_t);

static thread_local int g_iters_enqueued = 0;

static sps_status run_iterations(const ProbDev& pd, const Layout& L, char* ws, const IterCfg& ic, const sps_params* Q,
                                 IterFn full, RowFn row_only, cudaStream_t st, Ctrl* h, Events* ev) {
  int launched = 0;
  if (ic.log_domain && ic.dense) {
    SPS_TRY(launch_dense_lse_init(pd, L, ws, Q->init_alpha, Q->init_beta, st));
  } else if (ic.log_domain) {
    // the first iteration runs exactly in the log domain and forms the pair (u^1, v^1)
    SPS_TRY(launch_log_first_iteration(pd, L, ws, ic, Q->init_alpha, Q->init_beta, st));
    launched = 1;
    g_iters_enqueued = 1;
  } else {
    SPS_TRY(launch_iter_init(pd, L, ws, ic, Q->init_alpha, Q->init_beta, st));
  }
  ev->rec(4, st);   // the setup before the iteration kernels (a first exact iteration in the log domain)
  if (launched >= ic.max_iter) {
    SPS_TRY(read_ctrl(L, ws, h, st));
  }
  int chunk = Q->check_every > 0 ? Q->check_every : (ic.persistent ? 32 : 4);
  for (;;) {
    const int k = std::min(chunk, ic.max_iter - launched);
    if (k <= 0) break;
    SPS_TRY(full(pd, L, ws, ic, k, st));
    launched += k;
    g_iters_enqueued = launched;
    SPS_TRY(read_ctrl(L, ws, h, st));
    if (h->done || launched >= ic.max_iter) break;
    if (Q->check_every <= 0) chunk = std::min(chunk * 2, ic.persistent ? 4096 : 64);
  }
  if (!h->done) {
    SPS_TRY(row_only(pd, L, ws, ic, st));  // residual of the final pair
    SPS_TRY(read_ctrl(L, ws, h, st));
  }
  return SPS_OK;
}

// Lanes that share one row of the sparse product, by the mean row length:
// long rows a whole warp, shorter rows a half, quarter or eighth of one, so
// that a row fits one load batch of its segment (measured on the 20000-point
// UOT workload: 16 lanes beat 4, 8 and 32 for 158 elements per row).
static int lanes_per_row(double mean_nnz, int rows) {
  (void)rows;
  if (mean_nnz >= 192.0) return 32;
  if (mean_nnz >= 48.0) return 16;
  if (mean_nnz >= 12.0) return 8;
  return 4;
}

static void fill_result(sps_result* res, const DevResult& dr, const Ctrl& h, const sps_params* Q, int64_t nnz) {
  memset(res, 0, sizeof(*res));
  res->iters = h.done ? h.iters : h.t;
  res->residual = dr.residual;
  res->transport = dr.transport;
  res->neg_entropy = dr.neg_entropy;
  res->logp = dr.logp;
  res->mass = dr.mass;
  res->kl_a = dr.kl_a;
  res->kl_b = dr.kl_b;
  res->obj = dr.transport + Q->eps * dr.neg_entropy;
  if (!isinf(Q->lambda)) res->obj += Q->lambda * (dr.kl_a + dr.kl_b);
  res->obj_sparse = res->obj + Q->eps * dr.logp;
  res->unreach_a = dr.unreach_a;
  res->unreach_b = dr.unreach_b;
  res->nnz = nnz;
  res->n_absorb = h.n_absorb;
  res->launches = g_launches;
  res->iters_enqueued = g_iters_enqueued;
  if (h.status != SPS_OK) res->status = h.status;
  else res->status = h.done ? SPS_OK : SPS_NOT_CONVERGED;
}

static sps_status spar_sink_impl(const sps_problem* P, const sps_params* Q, void* wsv, size_t ws_bytes,
                                 void* alpha_out, void* beta_out, sps_result* res, cudaStream_t st, int want_uot) {
  SPS_TRY(validate(P, Q, SPS_OP_SPAR_SINK));
  if (want_uot && isinf(Q->lambda)) { set_error("spar_sink_uot needs a finite lambda"); return SPS_ERR_INVALID_ARG; }
  if (!want_uot && !isinf(Q->lambda)) { set_error("spar_sink_ot needs lambda = +inf"); return SPS_ERR_INVALID_ARG; }
  if (!wsv) { set_error("null workspace"); return SPS_ERR_INVALID_ARG; }
  Layout L;
  plan_layout(P, Q, SPS_OP_SPAR_SINK, &L);
  if (ws_bytes < L.total) { set_error("workspace too small: %zu < %zu", ws_bytes, L.total); return SPS_ERR_WORKSPACE; }
  char* ws = (char*)(((uintptr_t)wsv + 255) & ~(uintptr_t)255);
  ProbDev pd = make_probdev(P, Q, L, ws);
  g_launches = 0;
  g_iters_enqueued = 0;
  Events ev;
  ev.rec(0, st);
  Ctrl h;
  SPS_TRY(run_sketch(P, Q, L, ws, pd, st, &h));
  const int64_t nnz = h.nnz;
  ev.rec(1, st);
  IterCfg ic;
  ic.it64 = Q->kdtype == SPS_F64;
  ic.kd = Q->kdtype;
  ic.uot = want_uot;
  ic.phi = want_uot ? Q->lambda / (Q->lambda + Q->eps) : 1.0;
  ic.eps = Q->eps;
  ic.tol = Q->tol;
  ic.stop_rule = Q->stop_rule;
  ic.max_iter = Q->max_iter;
  ic.lpr_rows = lanes_per_row((double)nnz / P->n, P->n);
  ic.lpr_cols = lanes_per_row((double)nnz / P->m, P->m);
  ic.log_domain = Q->log_domain ? 1 : 0;
  ic.tau = Q->absorb_tau > 0.0 ? Q->absorb_tau : 12.0;
  if (ic.log_domain && L.stage_w > 0) {
    // staged passes work on a row's share of one chunk: lanes x 16 (4 lanes) or
    // x 8 (more lanes) elements per load batch, sized to the mean share
    const double seg = (double)nnz / ((double)P->n * L.stage_jr);
    ic.lpr_rows = seg <= 64.0 ? 4 : seg <= 128.0 ? 8 : seg <= 256.0 ? 16 : 32;
    ic.lpr_cols = ic.lpr_rows;
  }
  if (ic.log_domain) {
    SPS_TRY(run_iterations(pd, L, ws, ic, Q, launch_log_iterations, launch_log_row_only, st, &h, &ev));
    ev.rec(2, st);
    SPS_TRY(launch_log_objective(pd, L, ws, ic, alpha_out, beta_out, st));
  } else {
    SPS_TRY(run_iterations(pd, L, ws, ic, Q, launch_sparse_iterations, launch_sparse_row_only, st, &h, &ev));
    ev.rec(2, st);
    SPS_TRY(launch_sparse_objective(pd, L, ws, ic, alpha_out, beta_out, st));
  }
  ev.rec(3, st);
  DevResult dr;
  SPS_TRY(cuda_fail(cudaMemcpyAsync(&dr, ws + L.res, sizeof(dr), cudaMemcpyDeviceToHost, st), "result read-back"));
  SPS_TRY(cuda_fail(cudaStreamSynchronize(st), "stream synchronize"));
  sps_result r;
  fill_result(&r, dr, h, Q, nnz);
  r.gather = (ic.log_domain && L.stage_w > 0) ? (h.ell_overflow ? SPS_PASS_STAGED_FALLBACK : SPS_PASS_STAGED)
                                              : SPS_PASS_DIRECT;
  if (r.gather == SPS_PASS_STAGED) r.stream_bytes = h.ell_bytes[0] + h.ell_bytes[1];
  r.ms_sketch = ev.ms(0, 1);
  r.ms_iter = ev.ms(1, 2);
  r.ms_setup = ev.ms(1, 4);
  r.ms_obj = ev.ms(2, 3);
  if (res) *res = r;
  if (r.status == SPS_ERR_NUMERIC) set_error("non-finite value in the iterates");
  if (h.wait_timeout) set_error("a device-side grid barrier of the iteration kernel timed out");
  if (h.oob_code) {
    set_error("a device-side bounds check refused an access (place %d, index %lld)", h.oob_code, h.oob_index);
    if (res) res->status = SPS_ERR_CUDA;
    return SPS_ERR_CUDA;
  }
  return (sps_status)r.status;
}

}  // namespace sps

using namespace sps;

extern "C" {

const char* sps_last_error(void) { return g_err; }

const char* sps_version(void) { return "sparsink-gb300 0.1 (sm_103a)"; }

size_t sps_workspace_bytes(const sps_problem* prob, const sps_params* prm, int32_t op) {
  if (op < SPS_OP_SPARSIFY || op > SPS_OP_DENSE) return 0;
  if (validate(prob, prm, op) != SPS_OK) return 0;
  Layout L;
  plan_layout(prob, prm, op, &L);
  return L.total;
}

sps_status sparsify_kernel(const sps_problem* prob, const sps_params* prm, void* wsv, size_t ws_bytes,
                           sps_sketch* out, sps_stream stream) {
  SPS_TRY(validate(prob, prm, SPS_OP_SPARSIFY));
  if (!wsv || !out) { set_error("null workspace or output"); return SPS_ERR_INVALID_ARG; }
  Layout L;
  plan_layout(prob, prm, SPS_OP_SPARSIFY, &L);
  if (ws_bytes < L.total) { set_error("workspace too small: %zu < %zu", ws_bytes, L.total); return SPS_ERR_WORKSPACE; }
  char* ws = (char*)(((uintptr_t)wsv + 255) & ~(uintptr_t)255);
  cudaStream_t st = (cudaStream_t)stream;
  ProbDev pd = make_probdev(prob, prm, L, ws);
  Ctrl h;
  SPS_TRY(run_sketch(prob, prm, L, ws, pd, st, &h));
  out->n = prob->n;
  out->m = prob->m;
  out->nnz = h.nnz;
  out->capacity = L.cap;
  out->kdtype = prm->kdtype;
  out->row_ptr = at<int32_t>(ws, L.row_ptr);
  out->col_idx = at<int32_t>(ws, L.col_idx);
  out->val = ws + L.val;
  out->col_ptr = at<int32_t>(ws, L.col_ptr);
  out->row_idx = at<int32_t>(ws, L.row_idx);
  out->valT = ws + L.valT;
  out->csr_pos = at<int32_t>(ws, L.csr_pos);
  SketchScalars sc;
  SPS_TRY(cuda_fail(cudaMemcpyAsync(&sc, ws + L.scal, sizeof(sc), cudaMemcpyDeviceToHost, st), "scalars read-back"));
  SPS_TRY(cuda_fail(cudaStreamSynchronize(st), "stream synchronize"));
  const bool equal = prm->probs == SPS_PROBS_EQUAL;
  out->sum1 = equal ? 0.0 : sc.sum1;
  out->sum2 = equal || !isinf(prm->lambda) ? 0.0 : sc.sum2;
  return SPS_OK;
}

sps_status spar_sink_ot(const sps_problem* prob, const sps_params* prm, void* ws, size_t ws_bytes, void* alpha_out,
                        void* beta_out, sps_result* res, sps_stream stream) {
  return spar_sink_impl(prob, prm, ws, ws_bytes, alpha_out, beta_out, res, (cudaStream_t)stream, 0);
}

sps_status spar_sink_uot(const sps_problem* prob, const sps_params* prm, void* ws, size_t ws_bytes, void* alpha_out,
                         void* beta_out, sps_result* res, sps_stream stream) {
  return spar_sink_impl(prob, prm, ws, ws_bytes, alpha_out, beta_out, res, (cudaStream_t)stream, 1);
}

sps_status sinkhorn_dense(const sps_problem* prob, const sps_params* prm, void* wsv, size_t ws_bytes,
                          void* alpha_out, void* beta_out, sps_result* res, sps_stream stream) {
  SPS_TRY(validate(prob, prm, SPS_OP_DENSE));
  if (!wsv) { set_error("null workspace"); return SPS_ERR_INVALID_ARG; }
  Layout L;
  plan_layout(prob, prm, SPS_OP_DENSE, &L);
  if (ws_bytes < L.total) { set_error("workspace too small: %zu < %zu", ws_bytes, L.total); return SPS_ERR_WORKSPACE; }
  char* ws = (char*)(((uintptr_t)wsv + 255) & ~(uintptr_t)255);
  cudaStream_t st = (cudaStream_t)stream;
  ProbDev pd = make_probdev(prob, prm, L, ws);
  g_launches = 0;
  g_iters_enqueued = 0;
  Events ev;
  ev.rec(0, st);
  SPS_TRY(cuda_fail(cudaMemsetAsync(ws + L.ctrl, 0, sizeof(Ctrl), st), "memset ctrl"));
  SPS_TRY(cuda_fail(cudaMemsetAsync(ws + L.scal, 0, sizeof(SketchScalars), st), "memset scalars"));
  const int it64 = prm->kdtype == SPS_F64;
  SPS_TRY(launch_prepare(pd, L, ws, it64, st));
  if (prob->cost_norm == SPS_COST_MAXNORM) SPS_TRY(launch_cost_max(pd, L, ws, 0, st));
  SPS_TRY(launch_scalars0(pd, L, ws, st));
  ev.rec(1, st);
  IterCfg ic;
  ic.it64 = it64;
  ic.kd = prm->kdtype;
  ic.uot = isinf(prm->lambda) ? 0 : 1;
  ic.phi = ic.uot ? prm->lambda / (prm->lambda + prm->eps) : 1.0;
  ic.eps = prm->eps;
  ic.tol = prm->tol;
  ic.stop_rule = prm->stop_rule;
  ic.max_iter = prm->max_iter;
  Ctrl h;
  ic.persistent = 0;
  ic.dense = 1;
  ic.log_domain = prm->log_domain ? 1 : 0;
  if (ic.log_domain) {
    SPS_TRY(run_iterations(pd, L, ws, ic, prm, launch_dense_lse_iterations, launch_dense_lse_row_only, st, &h, &ev));
    ev.rec(2, st);
    SPS_TRY(launch_dense_lse_objective(pd, L, ws, ic, alpha_out, beta_out, st));
  } else {
    SPS_TRY(run_iterations(pd, L, ws, ic, prm, launch_dense_iterations, launch_dense_row_only, st, &h, &ev));
    ev.rec(2, st);
    SPS_TRY(launch_dense_objective(pd, L, ws, ic, alpha_out, beta_out, st));
  }
  ev.rec(3, st);
  DevResult dr;
  SPS_TRY(cuda_fail(cudaMemcpyAsync(&dr, ws + L.res, sizeof(dr), cudaMemcpyDeviceToHost, st), "result read-back"));
  SPS_TRY(cuda_fail(cudaStreamSynchronize(st), "stream synchronize"));
  sps_result r;
  fill_result(&r, dr, h, prm, (int64_t)prob->n * prob->m);
  r.ms_sketch = ev.ms(0, 1);
  r.ms_iter = ev.ms(1, 2);
  r.ms_setup = ev.ms(1, 4);
  r.ms_obj = ev.ms(2, 3);
  if (res) *res = r;
  if (r.status == SPS_ERR_NUMERIC) set_error("non-finite value in the iterates");
  return (sps_status)r.status;
}

}  // extern "C"
