/*
 * sparsink_oracle.h -- plain, slow FP64 CPU oracle for Spar-Sink.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  The product path never links, loads or calls it,
 * and it shares no source with the CUDA library.
 *
 * What it follows (Li, Yu, Li & Meng, "Importance Sparsification for
 * Sinkhorn Algorithm", JMLR 24, 2023):
 *   - Alg. 1 (SinkhornOT) and Alg. 2 (SinkhornUOT), section 2;
 *   - Eq. (pois): Poisson (independent Bernoulli) element-wise sampling,
 *     K~_ij = K_ij / p*_ij with probability p*_ij = min(1, s p_ij), section 3.1;
 *   - Eq. (pij-ot): p_ij proportional to sqrt(a_i b_j), section 3.2;
 *   - Eq. (pij-uot): p_ij proportional to (a_i b_j)^{lam/(2lam+eps)}
 *     K_ij^{eps/(2lam+eps)}, section 3.3;
 *   - Alg. 3 / Alg. 4 (Spar-Sink OT / UOT) and their objectives;
 *   - KL and entropy H as defined in section 2 (0 log 0 = 0);
 *   - the sparse cost C~ = C + eps log p* used in the proof of the UOT
 *     iteration lemma (appendix), which gives the log-domain form.
 *
 * The sampling decision (include or not) is computed in a fixed sequence of
 * correctly rounded IEEE binary32 operations so that any other
 * implementation of the same written rule reproduces the sparsity pattern
 * bit for bit.  Everything else is FP64.
 *
 * Parity pins: every function here is checked by the CPU tests against
 * something other than itself (closed forms, linear programming, a library
 * routine, an independent Philox implementation, Monte Carlo laws).
 */
#ifndef SPARSINK_ORACLE_H
#define SPARSINK_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- counter-based random numbers ---------------- */

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).  out = Philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The 24-bit uniform draw U_ij of element (i, j) of problem `pid`:
 * counter (j >> 2, i, pid, 0x5A17), key (seed low word, seed high word),
 * word j & 3 of the output, shifted right by 8. */
uint32_t orc_draw24(uint64_t seed, uint32_t pid, uint32_t i, uint32_t j);

/* ---------------- binary32 spec arithmetic ---------------- */

/* exp(x) in binary32: Cody-Waite reduction by ln 2 and a degree-7 Taylor
 * polynomial on [-ln2/2, ln2/2]. */
float orc_exp32(float x);
/* log(x) in binary32 for x > 0: exponent split, mantissa in
 * [sqrt(1/2), sqrt(2)], 2 atanh((m-1)/(m+1)) series. */
float orc_log32(float x);
/* vectorised forms for tests */
void orc_exp32_vec(const float* x, float* y, int64_t n);
/* binary32 spec cos on [0, pi/2] (Taylor series in z^2 to z^14, Horner form). */
float orc_cos32(float z);
void orc_cos32_vec(const float* z, float* y, int64_t n);
void orc_log32_vec(const float* x, float* y, int64_t n);

/* Exact sum of non-negative finite binary32 values, rounded once to the
 * nearest binary64 (ties to even).  Fixed-point accumulation over the whole
 * binary32 range (Collange, Defour, Graillat & Iakymchuk 2015 "superaccumulator"). */
double orc_exact_sum_f32(const float* x, int64_t n);

/* ---------------- sampling (Eq. pois with Eq. pij-ot / pij-uot) ---------------- */

typedef struct {
  int32_t n, m, d;
  const double* x;      /* n*d row-major, or NULL when C is given */
  const double* y;      /* m*d row-major, or NULL when C is given */
  const double* C;      /* n*m raw cost, or NULL (then squared Euclidean) */
  int32_t cost_norm;    /* 1: divide the raw cost by the max of its binary32 values over all pairs;
                           2: divide by cost_scale; 0: raw */
  double cost_scale;
  const double* a;      /* n */
  const double* b;      /* m */
  double eps;
  double lambda;        /* +INFINITY: balanced OT */
  double s;             /* expected sample budget */
  uint64_t seed;
  uint32_t pid;         /* problem id: third Philox counter word */
  int32_t cost_kind;    /* 0: squared Euclidean (or C); 1: Wasserstein-Fisher-Rao
                           C_ij = -log cos_+^2(d_ij / (2 eta)), d_ij the Euclidean distance of
                           the points (section 2.2); needs points and cost_norm = 0 */
  double eta;           /* WFR: eta > 0 (transport blocked where d_ij >= pi eta) */
  int32_t probs;        /* 0: Eq. (pij-ot) / Eq. (pij-uot); 1: equal probabilities p_ij = 1/(n m)
                           for every element (the Rand-Sink control of section 5), any lambda */
} orc_problem;

/* Scalars shared by every element's decision and value. */
typedef struct {
  double dmax64;     /* max raw cost, FP64 (value path) */
  float dmax32;      /* max raw cost, binary32 spec (decision path) */
  double sum1;       /* OT: exact sum sqrt(a); UOT: exact Z */
  double sum2;       /* OT: exact sum sqrt(b); UOT: unused */
  float scale32;     /* OT: invS = 1/(Sa Sb); UOT: fl32(s/Z) */
  float s32;         /* fl32(s) */
  float gamma32;     /* UOT exponent lam/(2lam+eps) */
  float kappa32;     /* UOT: 1/(Dnorm (2lam+eps)) */
  float inv2eta32;   /* WFR: fl32(1/(2 eta)) */
  float g2_32;       /* WFR UOT: fl32(2/(2lam+eps)), K^{eps/(2lam+eps)} = cos^{g2} */
} orc_scalars;

/* Row and column factors of the decision.  OT: r[i], c[j] with
 * p*_ij = min(1, r_i c_j).  Equal probabilities (probs = 1, OT or UOT):
 * r_i = fl(fl(s) fl(1/(n m))), c_j = 1, with the same rule.  UOT: A[i], B[j] with w_ij = A_i B_j E(-D_ij kappa)
 * and p*_ij = min(1, scale32 w_ij).  Returns 0 on success, <0 on bad input. */
int orc_factors(const orc_problem* P, float* rowf, float* colf, orc_scalars* S);

/* p*_ij (before the min with 1) as the binary32 spec computes it. */
float orc_pstar_raw(const orc_problem* P, const float* rowf, const float* colf,
                    const orc_scalars* S, int32_t i, int32_t j);

/* Count the sampled elements of every row (row_cnt[n]); returns total nnz. */
int64_t orc_count(const orc_problem* P, const float* rowf, const float* colf,
                  const orc_scalars* S, int32_t* row_cnt);

/* Sample one row: writes its columns (ascending), values K~ = K/p*,
 * log K~ = -C/eps - log p*, p* and C for each sampled element; returns the
 * row's count.  Arrays must hold m entries. */
int32_t orc_sample_row(const orc_problem* P, const float* rowf, const float* colf,
                       const orc_scalars* S, int32_t i, int32_t* cols, double* val,
                       double* logval, float* pstar, double* cost);

/* Full sketch: CSR (row_ptr n+1, col_idx, val, logval, pstar, cost; nnz
 * entries) and its stable transpose CSC (col_ptr m+1, row_idx, valT, perm
 * with perm[k] = CSR position of CSC entry k).  Arrays sized by the caller
 * from orc_count.  Returns nnz. */
int64_t orc_sparsify(const orc_problem* P, int32_t* row_ptr, int32_t* col_idx, double* val,
                     double* logval, float* pstar, double* cost, int32_t* col_ptr,
                     int32_t* row_idx, double* valT, int32_t* perm, orc_scalars* S);

/* Skip sampler (OT and UOT): the same law as orc_sample_row's per-element
 * decisions through a different random stream, with work proportional to
 * the sampled count (see the comment in the source). */
float orc_log1m32(float q);                      /* log(1 - q), 0 < q < 1, binary32 spec */
void orc_log1m32_vec(const float* q, float* y, int64_t n);
void orc_skip_words(uint64_t seed, uint32_t pid, uint32_t i, uint32_t t, uint32_t w[2]);
float orc_colf_max(const float* colf, int32_t m);
int32_t orc_skip_row(const orc_problem* P, const float* rowf, const float* colf, const orc_scalars* S,
                     float cmax, int32_t i, int32_t* cols, double* val, double* logval, float* pstar,
                     double* cost);
int64_t orc_skip_count(const orc_problem* P, const float* rowf, const float* colf, const orc_scalars* S,
                       int32_t* row_cnt);
int64_t orc_sparsify_skip(const orc_problem* P, int32_t* row_ptr, int32_t* col_idx, double* val,
                          double* logval, float* pstar, double* cost, int32_t* col_ptr,
                          int32_t* row_idx, double* valT, int32_t* perm, orc_scalars* S);

/* Dense kernel K_ij = exp(-C_ij/eps) and the normalised cost C_ij (n*m). */
int orc_dense_kernel(const orc_problem* P, double* K, double* Cn);

/* ---------------- scaling iterations (Alg. 1 / Alg. 2) ---------------- */

/* Result record of a solve. */
typedef struct {
  int32_t iters;          /* completed iterations of the returned pair */
  int32_t status;         /* 0 converged, 1 max_iter reached, 5 numeric */
  double residual;        /* stopping residual of the returned pair */
  double unreach_a;       /* sum of a_i over rows with (K~v)_i = 0 */
  double unreach_b;       /* sum of b_j over columns with (K~^T u)_j = 0 */
} orc_solve_info;

/* Stopping rules. */
#define ORC_STOP_RESIDUAL 0  /* ||u^{1/phi} (K~v) - a||_1 over reachable rows */
#define ORC_STOP_DELTA_UV 1  /* ||u^t-u^{t-1}||_1 + ||v^t-v^{t-1}||_1 (Alg. 1/2) */

/* Plain-domain Sinkhorn on a CSR/CSC pair (the dense case is a CSR holding
 * every element).  u, v: in = initial scalings (or NULL for all ones), out =
 * returned pair.  lambda = +INFINITY gives Alg. 1, otherwise Alg. 2. */
int orc_sinkhorn_sparse(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                        const double* val, const int32_t* col_ptr, const int32_t* row_idx,
                        const double* valT, const double* a, const double* b, double eps,
                        double lambda, double tol, int32_t max_iter, int32_t stop_rule,
                        const double* u0, const double* v0, double* u, double* v,
                        orc_solve_info* info);

/* Dense plain-domain Sinkhorn with K stored n*m (row-major). */
int orc_sinkhorn_dense(int32_t n, int32_t m, const double* K, const double* a, const double* b,
                       double eps, double lambda, double tol, int32_t max_iter,
                       int32_t stop_rule, const double* u0, const double* v0, double* u,
                       double* v, orc_solve_info* info);

/* Log-domain Sinkhorn on the support: potentials alpha = eps log u,
 * beta = eps log v, using logval = log K~ (CSR and CSC order).  Empty rows
 * get alpha = -inf.  alpha0/beta0 may be NULL (zeros). */
int orc_sinkhorn_log_sparse(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                            const double* logval, const int32_t* col_ptr, const int32_t* row_idx,
                            const double* logvalT, const double* a, const double* b, double eps,
                            double lambda, double tol, int32_t max_iter, int32_t stop_rule,
                            const double* alpha0, const double* beta0, double* alpha,
                            double* beta, orc_solve_info* info);

/* ---------------- objective (Alg. 3 / Alg. 4, output line) ---------------- */

/* Terms over the support of T~ = diag(u) K~ diag(v), given log T~_ij via
 * logT[k] = log u_i + log K~_ij + log v_j (or -inf).  cost[k] = C_ij,
 * pstar[k] = p*_ij (1 for dense).  out[0..6] = transport <T,C>,
 * neg_entropy sum T (log T - 1), logp sum T log p*, mass sum T,
 * KL(T1 || a), KL(T^T 1 || b), and unused. */
int orc_objective_terms(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                        const double* logT, const double* cost, const float* pstar,
                        const double* a, const double* b, double* out);

#ifdef __cplusplus
}
#endif
#endif
