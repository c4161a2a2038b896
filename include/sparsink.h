/*
 * sparsink.h -- C ABI of the GB300 (sm_103a) Spar-Sink library.
 *
 * Spar-Sink (Li, Yu, Li & Meng, "Importance Sparsification for Sinkhorn
 * Algorithm", JMLR 24, 2023) approximates entropic optimal transport by
 * sampling the Gibbs kernel K = exp(-C/eps) element-wise with importance
 * probabilities and running the Sinkhorn scaling iterations on the sparse,
 * reweighted sketch K~.
 *
 * Conventions shared by every entry point:
 *  - Memory.  Every pointer in sps_problem / sps_params, the workspace and the
 *    potential outputs are DEVICE pointers owned by the caller.  The library
 *    never allocates device memory: it writes only into the caller's
 *    workspace (size from sps_workspace_bytes) and outputs.  `res` is a HOST
 *    pointer (or NULL).
 *  - Streams.  All work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 *    default stream).  The solvers read convergence flags back between chunks
 *    of iterations and synchronise `stream` before returning.
 *  - Errors.  Functions return an sps_status; nothing throws across the ABI.
 *    Argument errors are detected before any launch.  sps_last_error()
 *    returns a thread-local message for the last failure on this thread.
 *    SPS_NOT_CONVERGED still writes valid potentials and results.
 *  - Layout.  Points are row-major (n x d, m x d); a dense cost is row-major
 *    n x m; indices are int32.  Potentials are returned in log form
 *    alpha = eps log u, beta = eps log v (-inf marks an unreachable row or
 *    column: one with no sampled element carrying mass).
 *  - Shapes.  n != m is allowed (the paper takes n = m only for brevity,
 *    section 2.1).  n*m < 2^62, nnz < 2^31.
 */
#ifndef SPARSINK_H
#define SPARSINK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sps_stream;  /* same type as cudaStream_t */

typedef enum {
  SPS_OK = 0,
  SPS_NOT_CONVERGED = 1,   /* max_iter reached; outputs hold the last pair */
  SPS_ERR_INVALID_ARG = 2, /* bad sizes, eps <= 0, negative weights, ... (no launch made) */
  SPS_ERR_WORKSPACE = 3,   /* ws_bytes smaller than sps_workspace_bytes() */
  SPS_ERR_CAPACITY = 4,    /* sampled nnz above the workspace capacity or INT32_MAX */
  SPS_ERR_NUMERIC = 5,     /* NaN/Inf met in the inputs or the iterates */
  SPS_ERR_CUDA = 6         /* a CUDA call failed; see sps_last_error() */
} sps_status;

typedef enum { SPS_F64 = 0, SPS_F32 = 1, SPS_BF16 = 2, SPS_F16 = 3 } sps_dtype;

/* cost_norm */
#define SPS_COST_RAW 0     /* C = raw cost */
#define SPS_COST_MAXNORM 1 /* C = raw / max over all (i, j) of raw */
#define SPS_COST_SCALE 2   /* C = raw / cost_scale */

/* stop_rule */
#define SPS_STOP_RESIDUAL 0 /* sum_i |u_i^{1/phi} (K~v)_i - a_i| <= tol (row side; see below) */
#define SPS_STOP_DELTA_UV 1 /* ||u^t - u^{t-1}||_1 + ||v^t - v^{t-1}||_1 <= tol (Alg. 1 / 2) */

/* One OT/UOT problem (section 2): measures a (n) and b (m) on points x, y,
 * with the squared Euclidean raw cost ||x_i - y_j||^2 (section 5.1), a given
 * raw cost matrix, or the Wasserstein-Fisher-Rao cost of section 2.2. */
typedef struct {
  int32_t n, m, d;
  const void* x;      /* device, n*d, dtype; may be NULL when C is given (then ignored) */
  const void* y;      /* device, m*d, dtype; may be NULL when C is given (then ignored) */
  const void* C;      /* device, n*m raw cost, dtype; NULL = squared Euclidean */
  int32_t cost_norm;  /* SPS_COST_* */
  double cost_scale;  /* divisor for SPS_COST_SCALE (finite, > 0) */
  const void* a;      /* device, n, dtype, a_i >= 0 */
  const void* b;      /* device, m, dtype, b_j >= 0 */
  sps_dtype dtype;    /* SPS_F32 or SPS_F64: type of x, y, C, a, b */
  int32_t cost_kind;  /* SPS_COST_SQEUCLID (0): the raw cost above, normalised by cost_norm.
                         SPS_COST_WFR (1): C_ij = -log cos_+^2(d_ij / (2 eta)) with d_ij the
                         Euclidean distance of the points (section 2.2): K_ij = cos^2 where
                         d_ij < pi eta, 0 (transport blocked) beyond.  Needs points (C = NULL)
                         and cost_norm = SPS_COST_RAW; sinkhorn_dense and the batched solver
                         take SPS_COST_SQEUCLID only.  Other values: SPS_ERR_INVALID_ARG. */
  double eta;         /* SPS_COST_WFR: the length scale eta (finite, > 0); ignored otherwise */
} sps_problem;

#define SPS_COST_SQEUCLID 0
#define SPS_COST_WFR 1

/* Parameters of a solve. */
typedef struct {
  double eps;          /* entropic regularisation, > 0 */
  double lambda;       /* KL marginal penalty (Eq. ruot); +INFINITY = balanced OT */
  double s;            /* sample budget: E nnz(K~) <= s (Eq. pois), > 0 */
  double tol;          /* stopping tolerance */
  int32_t max_iter;    /* iteration cap (>= 1) */
  int32_t check_every; /* iterations enqueued between convergence read-backs (0 = auto;
                          negative: SPS_ERR_INVALID_ARG) */
  int32_t stop_rule;   /* SPS_STOP_* */
  uint64_t seed;       /* Philox key of the sampling stream */
  uint32_t problem_id; /* third Philox counter word (distinct streams per problem) */
  sps_dtype kdtype;    /* storage of K~ values: F64, F32, BF16 or F16.  F64 iterates in
                          FP64; the others iterate in FP32 */
  int32_t log_domain;  /* 1: stabilised (absorbing) iterations for small eps */
  double absorb_tau;   /* absorb when max |log u~| or |log v~| exceeds this (0 = default 12;
                          with log_domain, NaN, infinite or negative: SPS_ERR_INVALID_ARG) */
  const void* init_alpha; /* optional device warm start (n), iterate type, or NULL */
  const void* init_beta;  /* optional device warm start (m), iterate type, or NULL */
  int32_t gather_mode; /* stabilised iterations only: how the sparse products read the
                          gathered scaling vector.  SPS_GATHER_AUTO (0) stages it through
                          shared memory in column chunks when n and m are both >= 65536,
                          SPS_GATHER_DIRECT (1) never does, SPS_GATHER_STAGED (2) always does
                          (with at least four chunks when n or m exceeds 3072).
                          The results agree to rounding; the choice is a performance one. */
  int32_t sketch_mode; /* SPS_SKETCH_SINGLE (0): one n x m sweep writes every kept element
                          into a padded slot per (row, column chunk) sized from its expected
                          count, then a compaction places it; if a slot overflows (a count
                          about 8 standard deviations above its mean) the two passes run
                          instead.  SPS_SKETCH_TWO_PASS (1): count, then fill.  Both give the
                          same sketch bit for bit. */
  int32_t sampler;     /* How the sketch draws Eq. (pois).  SPS_SAMPLER_ELEMENT (0): one
                          Philox decision per element (n m work; every (i, j) tested).
                          SPS_SAMPLER_SKIP (1): every row draws its kept columns by geometric
                          gaps over a row bound q_i >= p_ij (OT: r_i max_j c_j; UOT:
                          (s/Z) A_i max_j B_j, since the exponential factor is at most 1)
                          followed by thinning with p_ij / q_i -- the same law (each element
                          kept independently with probability p*_ij) from a different random
                          stream, with work proportional to the sampled count (the UOT
                          normaliser Z is still an exact sum over all pairs).  sketch_mode
                          does not apply to it.  spar_sink_batched takes both; with either,
                          pair p's sketch is the one a single solve with problem id
                          problem_id + p draws (its row bound takes the largest factor of the
                          pair's target set). */
  int32_t probs;       /* Sampling probabilities of Eq. (pois).  SPS_PROBS_PAPER (0):
                          Eq. (pij-ot) for OT, Eq. (pij-uot) for UOT.  SPS_PROBS_EQUAL (1):
                          p_ij = 1/(n m) for every element, p*_ij = min(1, s/(n m)) -- the
                          equal-probability control (Rand-Sink) of section 5, for OT and UOT;
                          the decision is then r_i c_j with r_i = fl(fl(s) fl(1/(n m))), c_j = 1.
                          spar_sink_batched takes SPS_PROBS_PAPER only.  Other values:
                          SPS_ERR_INVALID_ARG. */
} sps_params;

#define SPS_PROBS_PAPER 0
#define SPS_PROBS_EQUAL 1

#define SPS_SKETCH_SINGLE 0
#define SPS_SKETCH_TWO_PASS 1

#define SPS_SAMPLER_ELEMENT 0
#define SPS_SAMPLER_SKIP 1

#define SPS_GATHER_AUTO 0
#define SPS_GATHER_DIRECT 1
#define SPS_GATHER_STAGED 2

/* Results of a solve (host struct). */
typedef struct {
  int32_t status;      /* sps_status of the solve */
  int32_t iters;       /* iterations of the returned pair (u^t, v^t) */
  double residual;     /* stopping residual of the returned pair */
  double obj;          /* <T,C> - eps H(T) (+ lam KL(T1||a) + lam KL(T^T1||b)), output line of Alg. 3/4 */
  double obj_sparse;   /* obj + eps sum T log p*: the value of the sparse problem (cost C + eps log p*) */
  double transport;    /* <T, C> */
  double neg_entropy;  /* sum T (log T - 1) = -H(T) */
  double logp;         /* sum T log p* (0 for dense) */
  double mass;         /* sum T */
  double kl_a, kl_b;   /* KL(T1 || a), KL(T^T 1 || b), section 2 definition */
  double unreach_a;    /* mass of a on rows with (K~v)_i = 0 */
  double unreach_b;    /* mass of b on columns with (K~^T u)_j = 0 */
  int64_t nnz;         /* elements of K~ */
  int32_t n_absorb;    /* absorptions performed (log_domain) */
  float ms_sketch, ms_iter, ms_obj; /* device time of the three phases */
  int32_t launches;    /* kernels this call launched (including iterations enqueued after the stop flag) */
  int32_t iters_enqueued; /* iterations enqueued (>= iters; the surplus returned at once) */
  int32_t gather;      /* how the iterations read the sketch: SPS_PASS_* below */
  float ms_setup;      /* device time of the part of ms_iter before the iteration kernels: the
                          initial pair, and in the log domain the exact first iteration, the
                          absorption and the staged passes' grouped copies */
  int64_t stream_bytes; /* gather == STAGED: bytes of the two grouped copies, which one iteration
                           reads once each (0 otherwise) */
} sps_result;

/* sps_result.gather.  DIRECT: every product gathers the scaling vector from
   global memory (CSR / CSC order).  STAGED (log_domain, long vectors): the
   vector passes through shared memory chunk by chunk and the sketch is read
   from a copy grouped by chunk (runs of 32 rows sorted by length, 16-bit
   chunk-local indices).  STAGED_FALLBACK: staging was planned but the grouped
   copy did not fit its planned space (a sketch with very uneven runs), so the
   products gathered directly; the results are the same up to rounding. */
#define SPS_PASS_DIRECT 0
#define SPS_PASS_STAGED 1
#define SPS_PASS_STAGED_FALLBACK 2

/* Views of a sketch inside the workspace (filled by sparsify_kernel). */
typedef struct {
  int32_t n, m;
  int64_t nnz, capacity;
  sps_dtype kdtype;
  int32_t* row_ptr;   /* n+1 */
  int32_t* col_idx;   /* nnz, ascending inside each row */
  void* val;          /* nnz, K~_ij = K_ij / p*_ij in kdtype */
  int32_t* col_ptr;   /* m+1 */
  int32_t* row_idx;   /* nnz, ascending inside each column (stable transpose) */
  void* valT;         /* nnz, values in CSC order */
  int32_t* csr_pos;   /* nnz, CSR position of each CSC entry */
  double sum1, sum2;  /* the exact sums of the sampling probabilities, rounded to binary64 once:
                         OT (Eq. pij-ot) sum_i sqrt(a_i) and sum_j sqrt(b_j); UOT (Eq. pij-uot) the
                         normaliser Z = sum_ij A_i B_j F(C_ij) in sum1 (sum2 = 0); equal
                         probabilities: 0 */
} sps_sketch;

/* Operation codes for sps_workspace_bytes. */
#define SPS_OP_SPARSIFY 0
#define SPS_OP_SPAR_SINK 1
#define SPS_OP_DENSE 2

/* Bytes of device workspace an operation needs for this problem and these
 * parameters (0 on invalid arguments).  The sketch capacity is
 * min(n*m, s + 8 sqrt(s) + 1024) elements: E nnz = sum p* <= s (section 3.1),
 * and Var nnz <= s, so the capacity is exceeded with probability < 1e-15. */
size_t sps_workspace_bytes(const sps_problem* prob, const sps_params* prm, int32_t op);

/* Dense Sinkhorn, Alg. 1 (lambda = +INFINITY) or Alg. 2 (finite lambda), on
 * K = exp(-C/eps) computed on the fly (never stored), section 2; points need
 * d <= 16 (SPS_ERR_INVALID_ARG otherwise).  Writes
 * alpha_out (n) and beta_out (m) in the iterate type (FP64 if kdtype = F64,
 * else FP32).  Stopping: see SPS_STOP_*; the residual of a pair (u^t, v^t)
 * is its row side because v^t = (b / K^T u^t)^phi makes the column side zero
 * up to rounding. */
sps_status sinkhorn_dense(const sps_problem* prob, const sps_params* prm, void* ws,
                          size_t ws_bytes, void* alpha_out, void* beta_out, sps_result* res,
                          sps_stream stream);

/* Importance sparsification of K (section 3.1, Eq. pois): element (i, j) is
 * kept with probability p*_ij = min(1, s p_ij), p_ij from Eq. (pij-ot) when
 * lambda = +INFINITY and Eq. (pij-uot) otherwise, and stored as K_ij / p*_ij.
 * The keep/drop decision is a fixed binary32 computation on a Philox4x32-10
 * stream (counter (j>>2, i, problem_id, 0x5A17), key = seed), so the pattern
 * is reproducible bit for bit.  Fills `out` with views into `ws`. */
sps_status sparsify_kernel(const sps_problem* prob, const sps_params* prm, void* ws,
                           size_t ws_bytes, sps_sketch* out, sps_stream stream);

/* Spar-Sink for OT, Alg. 3 (section 3.2): sparsify with Eq. (pij-ot), run
 * Alg. 1 on K~, evaluate the objective terms.  Requires lambda = +INFINITY. */
sps_status spar_sink_ot(const sps_problem* prob, const sps_params* prm, void* ws,
                        size_t ws_bytes, void* alpha_out, void* beta_out, sps_result* res,
                        sps_stream stream);

/* Spar-Sink for UOT, Alg. 4 (section 3.3): sparsify with Eq. (pij-uot), run
 * Alg. 2 (exponent lambda/(lambda+eps)) on K~.  Requires 0 < lambda < inf. */
sps_status spar_sink_uot(const sps_problem* prob, const sps_params* prm, void* ws,
                         size_t ws_bytes, void* alpha_out, void* beta_out, sps_result* res,
                         sps_stream stream);

/* Spar-Sink OT (as spar_sink_ot) for callers that cannot allocate device
 * memory at solve time -- e.g. a process whose device memory belongs to
 * another allocator (a framework's caching pool, a fixed budget) or an
 * embedding that only allocates at start-up -- and so cannot supply a
 * workspace.  The paper has no counterpart; this is an interface convenience.
 *
 * The workspace is a file-scope device array of SPS_NOALLOC_SCRATCH_BYTES
 * bytes, held by every GPU that loads the library until the process exits.
 * The call makes no device allocation (no cudaMalloc / cudaFree, no
 * allocating library routine); like every solver entry point it creates the
 * CUDA events that time its phases.  The first call made on a device in a
 * CUDA context (with that device current) looks up the array's device address
 * with cudaGetSymbolAddress; later calls in the same context reuse it, and a
 * new context (after cudaDeviceReset, say) gets its own lookup.  Like
 * spar_sink_ot, the call waits for its stream and reads the result back
 * before it returns.
 * Problems whose sps_workspace_bytes(..., SPS_OP_SPAR_SINK) exceeds the array
 * are rejected with SPS_ERR_WORKSPACE before any launch.  All calls share the
 * array, which keeps the last call's contents (each call clears what must
 * start at zero); calls whose GPU work overlaps race on it.  Inputs and
 * outputs are the caller's device buffers, as for spar_sink_ot. */
#define SPS_NOALLOC_SCRATCH_BYTES (16u << 20)
sps_status spar_sink_ot_noalloc(const sps_problem* prob, const sps_params* prm, void* alpha_out,
                                void* beta_out, sps_result* res, sps_stream stream);

/* ---------------- batches of problems over shared point sets ----------------
 * Many independent problems whose points come from a few shared sets, e.g.
 * all pairs of frames of an image sequence: pair p transports set src[p]
 * (weights a = mass of that set) to set dst[p] (b = its mass), with its own
 * budget s[p] and its own sampling stream (Philox problem id
 * prm->problem_id + p).  Every pair is sketched as in Eq. (pois) with
 * Eq. (pij-ot) or Eq. (pij-uot) and solved by Alg. 3 (lambda = +inf) or
 * Alg. 4 with the stabilised iterations (log-domain first iteration and
 * absorption, the form used for small eps), then its objective terms.
 * There is no batched counterpart in the paper: the batch is a throughput
 * form of the same per-pair computation, and each pair's pattern, iteration
 * count and objective equal those of a single spar_sink_ot / spar_sink_uot
 * call with log_domain = 1 and the same problem id (to rounding).
 *
 * The sketches of all pairs live in one block-diagonal CSR / CSC in the
 * workspace; the iterations of all pairs run in ONE persistent launch whose
 * blocks take pairs from a queue (largest first) and iterate each pair to its
 * own stopping rule with block-local barriers only, the scaling vectors in
 * shared memory.  Hence a support limit: 2 n_p + m_p <= SPS_BATCH_MAX_SMEM_ENTRIES
 * for every pair.
 */
typedef struct {
  int32_t n_sets;          /* number of point sets */
  int32_t d;               /* dimension of the points, 1 .. 16 */
  const int64_t* set_off;  /* HOST, n_sets + 1 offsets: set k holds points set_off[k] .. set_off[k+1]-1 */
  const void* pts;         /* DEVICE, set_off[n_sets] x d row-major, dtype */
  const void* mass;        /* DEVICE, set_off[n_sets] weights >= 0, dtype */
  int32_t n_pairs;         /* number of problems */
  const int32_t* src;      /* HOST, n_pairs source set indices */
  const int32_t* dst;      /* HOST, n_pairs target set indices */
  const double* s;         /* HOST, n_pairs sample budgets (> 0) */
  int32_t cost_norm;       /* SPS_COST_RAW, SPS_COST_MAXNORM (max over the pair) or SPS_COST_SCALE */
  double cost_scale;       /* divisor for SPS_COST_SCALE (finite, > 0) */
  sps_dtype dtype;         /* F32 or F64 points and weights */
} sps_batch;

#define SPS_BATCH_MAX_SMEM_ENTRIES 49152

/* Launch shape of the persistent iteration kernel.  Zero fields are chosen
 * by the library's autotuner: it times every candidate (lanes per row 4, 8,
 * 16, 32 x block threads 256, 512, 1024) on the batch itself for a few
 * iterations and caches the winner per batch shape for the process. */
typedef struct {
  int32_t lanes_per_row;   /* lanes sharing one row / column segment: 4, 8, 16, 32, or 0 */
  int32_t block_threads;   /* 256, 512, 1024, or 0 */
  int32_t use_graph;       /* 1: capture the enqueued device work in a CUDA graph on the first
                              call with this workspace and batch shape, and replay it after
                              (needs a stream other than the legacy default stream) */
  int32_t chosen_lanes;    /* out: the shape used */
  int32_t chosen_threads;  /* out */
  float tune_ms;           /* out: time spent autotuning in this call (0 if cached or fixed) */
} sps_batch_opts;

/* Workspace bytes for spar_sink_batched, or 0 on invalid arguments. */
size_t sps_batch_workspace_bytes(const sps_batch* batch, const sps_params* prm);

/* Solves every pair.  alpha_out: DEVICE, sum_p n_p floats (pair p's source
 * potentials at offset sum_{q<p} n_q); beta_out likewise with m_p.  res:
 * HOST array of n_pairs results (ms_* fields hold the whole batch's phase
 * times).  Returns SPS_OK when every pair converged, SPS_NOT_CONVERGED if
 * any did not (see res[p].status), or an error.  prm: eps, lambda, tol,
 * max_iter, seed, problem_id, kdtype (F32, BF16 or F16), absorb_tau;
 * init_alpha / init_beta (DEVICE, same layout as the outputs) may be given. */
sps_status spar_sink_batched(const sps_batch* batch, const sps_params* prm, sps_batch_opts* opts, void* ws,
                             size_t ws_bytes, void* alpha_out, void* beta_out, sps_result* res,
                             sps_stream stream);

/* ---------------- Wasserstein barycenters (Spar-IBP) ----------------
 * The fixed-support barycenter q of M measures b_1 .. b_M on one support x
 * (n points): the minimiser of sum_k w_k OT_eps(q, b_k), by the iterative
 * Bregman projections (IBP) of the paper's appendix run on sketches.  Spar-IBP
 * (the appendix's algorithm): every Gibbs kernel K_k = exp(-C / eps) of the
 * shared cost C (squared Euclidean on x, normalised by cost_norm) is replaced
 * by its sketch of Eq. (pois) with p_{k,ij} = sqrt(b_{k,j}) / (n sum_j
 * sqrt(b_{k,j})) -- Eq. (pij-ot) with the uniform source a = 1/n -- drawn
 * with Philox problem id prm->problem_id + k.  From q^0 = 1/n and u_k = 1,
 * every iteration forms v_k = b_k / (K~_k^T u_k), then q = prod_k (K~_k
 * v_k)^{w_k}, then u_k = q / (K~_k v_k) (the order of the cited IBP: as
 * printed, the listing forms u_k from the previous q, which leaves a common
 * scale of the u_k oscillating), and stops when ||q^t - q^{t-1}||_1 <= tol.
 * An empty row of a sketch gives q_i = 0 and u_{k,i} = 0; an empty column gives
 * v_{k,j} = 0.  A budget s at least 1 / min p_ij keeps every element and the
 * iterations are those of IBP on the dense kernels. */
typedef struct {
  int32_t n, d;         /* support size and dimension */
  int32_t n_measures;   /* M, 1 .. 64 */
  const void* x;        /* device, n*d row-major, dtype: the shared support */
  const void* b;        /* device, M*n, dtype: measure k in b[k n .. (k+1) n), b >= 0 */
  const double* w;      /* host, M weights: finite, >= 0, summing to 1 within 1e-9 */
  int32_t cost_norm;    /* SPS_COST_*: of the squared Euclidean cost on x */
  double cost_scale;    /* divisor for SPS_COST_SCALE */
  sps_dtype dtype;      /* SPS_F32 or SPS_F64: type of x and b */
} sps_barycenter;

/* Workspace bytes of spar_ibp (0 and an error message on invalid arguments).
 * prm: eps, s (the budget of every sketch), tol, max_iter, seed, problem_id,
 * kdtype (F64 iterates in FP64, F32 / BF16 / F16 values iterate in FP32) and
 * sampler are used; lambda must be +INFINITY, log_domain 0, probs
 * SPS_PROBS_PAPER, stop_rule SPS_STOP_RESIDUAL (here: the ||q^t - q^{t-1}||_1
 * rule of the appendix). */
size_t sps_ibp_workspace_bytes(const sps_barycenter* bar, const sps_params* prm);

/* Spar-IBP (the appendix's Spar-IBP algorithm, after Benamou et al. 2015):
 * writes the barycenter q (n, iterate type: double for kdtype F64, else
 * float) to q_out (device).  res (host, optional): iters, residual =
 * ||q^t - q^{t-1}||_1 of the returned q, nnz = total elements of the M
 * sketches, ms_sketch / ms_iter, status (SPS_OK or SPS_NOT_CONVERGED; other
 * fields 0).  Synchronises the stream.  Errors as for spar_sink_ot. */
sps_status spar_ibp(const sps_barycenter* bar, const sps_params* prm, void* ws, size_t ws_bytes, void* q_out,
                    sps_result* res, sps_stream stream);

/* ---------------- learned warm start ----------------
 * The paper starts the scaling iterations from u = v = 1 (Alg. 1, Alg. 2).
 * These entry points predict starting potentials instead, with one small
 * network per side: for source point i,
 *   f_i = [x_i / sqrt(cost_max), n a_i],  P = sum_j b_j relu(We [y_j / sqrt(cost_max), m b_j] + ce) / sum_j b_j,
 *   alpha^_i = w3 . relu(W2 relu(W1 [f_i, P] + b1) + b2) + b3
 * (hidden width SPS_MLP_HIDDEN, embedding SPS_MLP_EMB), and symmetrically
 * beta^_j.  Potentials are in units of the normalised cost C = D / cost_max,
 * ready for sps_params.init_alpha / init_beta with
 * cost_norm = SPS_COST_SCALE, cost_scale = cost_max (which reproduces
 * SPS_COST_MAXNORM exactly when cost_max comes from sps_cost_max).  The
 * forward pass reads BF16 weights and accumulates in FP32; training keeps
 * FP32 master weights and Adam moments.  The fixed point, stopping rule and
 * result of the solve do not depend on the start; only the iteration count
 * does.
 *
 * Parameter vectors: FP32 (sps_mlp_param_count(d) floats) and a BF16 copy of
 * the same length; layout per side: We (EMB x (d+1)), ce, W1 (HIDDEN x
 * (d+1+EMB)), b1, W2 (HIDDEN x HIDDEN), b2, w3, b3; the source side first.
 * All pointers are DEVICE pointers; ws holds sps_mlp_workspace_bytes(). */
#define SPS_MLP_HIDDEN 128
#define SPS_MLP_EMB 16

typedef struct {
  const float* x; const float* y;   /* DEVICE points, n x d and m x d, binary32 */
  const float* a; const float* b;   /* DEVICE weights */
  int32_t n, m, d;                  /* 1 <= d <= 16 */
  double cost_max;                  /* the cost divisor (sps_cost_max) */
  double eps;                       /* training loss scale (finite, > 0): errors are measured in units of eps */
} sps_mlp_instance;

/* Length of each parameter vector (FP32 and BF16 copies) for points of dimension d (both sides);
 * 0 unless 1 <= d <= 16. */
size_t sps_mlp_param_count(int32_t d);
/* Bytes of the scratch `ws` that sps_cost_max, sps_mlp_infer, sps_mlp_gauge_fix and sps_mlp_grad take
 * (caller-allocated device memory, independent of the instance size). */
size_t sps_mlp_workspace_bytes(void);
/* He-uniform initialisation from the Philox stream of `seed`; fills both copies. */
sps_status sps_mlp_init(float* params, void* params_bf16, int32_t d, uint64_t seed, sps_stream stream);
sps_status sps_mlp_sync_bf16(const float* params, void* params_bf16, int32_t d, sps_stream stream);
/* Exact maximum over all pairs of the binary32 squared distance (the divisor
 * of SPS_COST_MAXNORM), read back to the host. */
sps_status sps_cost_max(const float* x, int32_t n, const float* y, int32_t m, int32_t d, double* cost_max,
                        void* ws, sps_stream stream);
/* The same maximum, bit for bit, with a caller workspace (device memory) of
 * sps_cost_max_workspace_bytes(n, m, d) bytes (0: invalid sizes; 1 <= d <= 16).
 * Above 1e8 pairs it evaluates only the pairs that can reach the maximum, as
 * the solver's own sketch does (grid cells bounded by their boxes for d <= 4,
 * radial bounds about the bounding-box centre for d > 4; the full sweep after
 * an overflowing candidate list), instead of all n m of them.  A smaller
 * workspace returns SPS_ERR_WORKSPACE; the call synchronises its stream. */
size_t sps_cost_max_workspace_bytes(int32_t n, int32_t m, int32_t d);
sps_status sps_cost_max_ws(const float* x, int32_t n, const float* y, int32_t m, int32_t d, double* cost_max,
                           void* ws, size_t ws_bytes, sps_stream stream);
/* Predicted potentials alpha^ (n) and beta^ (m). */
sps_status sps_mlp_infer(const void* params_bf16, const sps_mlp_instance* inst, float* alpha_out,
                         float* beta_out, void* ws, sps_stream stream);
/* Shift a potential pair (in place) so that sum a alpha = sum b beta over the
 * finite entries (the OT gauge: (alpha + c, beta - c) is the same plan). */
sps_status sps_mlp_gauge_fix(const sps_mlp_instance* inst, float* alpha, float* beta, void* ws,
                             sps_stream stream);
/* Gradient of the loss sum_i a_i ((alpha^_i - alpha_i)/eps)^2 / sum a + (same for beta)
 * with respect to the BF16 forward's weights, into grad (param count floats);
 * the loss value goes to *loss_out (HOST, may be NULL; non-NULL synchronises). */
sps_status sps_mlp_grad(const float* params, const void* params_bf16, const sps_mlp_instance* inst,
                        const float* alpha_target, const float* beta_target, float* grad, float* loss_out,
                        void* ws, sps_stream stream);
/* One Adam step (bias-corrected, step >= 1) on the FP32 master weights; refreshes the BF16 copy.
 * lr must be finite and >= 0, beta1 and beta2 in [0, 1), eps finite and > 0 (else SPS_ERR_INVALID_ARG). */
sps_status sps_mlp_adam(float* params, void* params_bf16, float* m1, float* m2, const float* grad, int32_t d,
                        int32_t step, float lr, float beta1, float beta2, float eps, sps_stream stream);

/* Thread-local message describing the last error on this thread (valid until the next call
 * on this thread that fails). */
const char* sps_last_error(void);

/* Library version string. */
const char* sps_version(void);

/* Failure-detection self-test of the bounded device waits (the paper has no
 * counterpart: its algorithms have no device waits).  The persistent
 * iteration kernels synchronise their blocks with a grid barrier whose wait
 * gives up after a fixed number of polls (about a second or more), records
 * the timeout in the solve's control block and returns, so that a solve
 * reports an error instead of hanging and the CUDA context stays usable.
 * This call makes that wait run out, without any fault: it runs the same
 * barrier on a two-block grid in which one block never arrives.
 * ws: DEVICE, at least 1024 bytes (caller-owned scratch, contents
 * overwritten).  *wait_ms (HOST) receives the duration of the launch.
 * Synchronises `stream`.  Returns SPS_ERR_CUDA with the message "... timed
 * out ..." when the device recorded the timeout (the expected outcome),
 * SPS_OK if the barrier completed anyway, SPS_ERR_INVALID_ARG /
 * SPS_ERR_WORKSPACE for bad arguments (before any launch). */
sps_status sps_selftest_barrier_timeout(void* ws, size_t ws_bytes, float* wait_ms, sps_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SPARSINK_H */
