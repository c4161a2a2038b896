/*
 * sparsink_oracle.c -- plain, slow FP64 CPU oracle for Spar-Sink.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  Parity of
 * every function is pinned by the CPU tests (see each function's comment).
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off [-fopenmp].  The flag
 * -ffp-contract=off matters: the binary32 decision spec is a fixed sequence
 * of individually rounded operations, and a fused multiply-add that the
 * compiler invented would change it.  Explicit fmaf() calls are part of the
 * spec and stay fused.
 */
#define _DEFAULT_SOURCE
#include "sparsink_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ======================================================================
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, section 4.2).
 * One round: two 32x32->64 products of counter words 0 and 2 with the
 * round multipliers; the high halves are xor-ed with the other counter
 * words and the round key; words are permuted.  The key is bumped by the
 * Weyl constants (golden ratio and sqrt(3)-1 in 0.32 fixed point) between
 * rounds.
 * Pinned by tests/test_oracle_rng.py against an independent Philox
 * implementation and by uniformity tests.
 * ====================================================================== */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint32_t orc_draw24(uint64_t seed, uint32_t pid, uint32_t i, uint32_t j) {
  uint32_t ctr[4] = {j >> 2, i, pid, 0x5A17u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[j & 3u] >> 8;
}

/* ======================================================================
 * binary32 spec arithmetic: exp and log written from their series.
 * Pinned against libm FP64 exp/log (error bound in ulps) by
 * tests/test_oracle_specmath.py.
 * ====================================================================== */
typedef union { float f; uint32_t u; } f32bits;

/* ln 2 split for Cody-Waite: LN2_HI is ln 2 truncated to 16 significant
 * bits (45426 / 65536), so e * LN2_HI is exact for |e| < 256; LN2_LO is the
 * binary32 rounding of ln 2 - LN2_HI. */
static const float LN2_HI = 0.693145751953125f;
static const float LN2_LO = 1.42860677e-06f;
static const float LOG2E_F = 1.44269502e+00f;   /* binary32 rounding of 1/ln 2 */
static const float SQRT2_F = 1.41421354e+00f;   /* binary32 rounding of sqrt 2 */

static float pow2_small(int k) { /* 2^k for -126 <= k <= 127 */
  f32bits t;
  t.u = (uint32_t)(k + 127) << 23;
  return t.f;
}

float orc_exp32(float x) {
  if (x != x) return x;
  if (x > 88.75f) return INFINITY;
  if (x < -104.0f) return 0.0f;
  /* x = k ln2 + r, |r| <= ln2/2 (plus rounding) */
  float k = rintf(x * LOG2E_F);
  float r = fmaf(-k, LN2_HI, x);
  r = fmaf(-k, LN2_LO, r);
  /* e^r by its Taylor series to degree 7, Horner form */
  float p = (float)(1.0 / 5040.0);
  p = fmaf(p, r, (float)(1.0 / 720.0));
  p = fmaf(p, r, (float)(1.0 / 120.0));
  p = fmaf(p, r, (float)(1.0 / 24.0));
  p = fmaf(p, r, (float)(1.0 / 6.0));
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  /* scale by 2^k in two exact power-of-two steps */
  int ki = (int)k;
  int k1 = ki / 2;
  int k2 = ki - k1;
  return (p * pow2_small(k1)) * pow2_small(k2);
}

float orc_log32(float x) {
  if (x != x) return x;
  if (x < 0.0f) return NAN;
  if (x == 0.0f) return -INFINITY;
  if (isinf(x)) return x;
  f32bits t;
  t.f = x;
  int e = 0;
  if (t.u < 0x00800000u) { /* subnormal: scale into the normal range exactly */
    t.f = x * 16777216.0f;
    e = -24;
  }
  e += (int)((t.u >> 23) & 0xffu) - 127;
  t.u = (t.u & 0x007fffffu) | 0x3f800000u; /* mantissa m in [1, 2) */
  float m = t.f;
  if (m > SQRT2_F) {
    m = m * 0.5f;
    e += 1;
  }
  /* log m = 2 atanh(z), z = (m-1)/(m+1), |z| <= 0.1716 */
  float f = m - 1.0f;
  float z = f / (m + 1.0f);
  float w = z * z;
  float P = (float)(1.0 / 11.0);
  P = fmaf(P, w, (float)(1.0 / 9.0));
  P = fmaf(P, w, (float)(1.0 / 7.0));
  P = fmaf(P, w, 0.2f);
  P = fmaf(P, w, (float)(1.0 / 3.0));
  float q = w * P;
  float z2 = z + z;
  float lm = fmaf(z2, q, z2);
  float fe = (float)e;
  float r = fmaf(fe, LN2_LO, lm);
  return fmaf(fe, LN2_HI, r);
}

void orc_exp32_vec(const float* x, float* y, int64_t n) {
  for (int64_t k = 0; k < n; ++k) y[k] = orc_exp32(x[k]);
}
/* cos z for 0 <= z <= pi/2: 1 - z^2/2! + z^4/4! - ... to z^14/14! in w = z^2
 * (the next term is below 7e-11 at z = pi/2), Horner form. */
float orc_cos32(float z) {
  const float w = z * z;
  float p = (float)(-1.0 / 87178291200.0);
  p = fmaf(p, w, (float)(1.0 / 479001600.0));
  p = fmaf(p, w, (float)(-1.0 / 3628800.0));
  p = fmaf(p, w, (float)(1.0 / 40320.0));
  p = fmaf(p, w, (float)(-1.0 / 720.0));
  p = fmaf(p, w, (float)(1.0 / 24.0));
  p = fmaf(p, w, -0.5f);
  return fmaf(p, w, 1.0f);
}

void orc_cos32_vec(const float* z, float* y, int64_t n) {
  for (int64_t k = 0; k < n; ++k) y[k] = orc_cos32(z[k]);
}

void orc_log32_vec(const float* x, float* y, int64_t n) {
  for (int64_t k = 0; k < n; ++k) y[k] = orc_log32(x[k]);
}

/* ======================================================================
 * Exact summation: a non-negative binary32 value is an integer times
 * 2^-149.  The accumulator keeps that integer in 32-bit digits held in
 * 64-bit words (carry-save), so any order of additions gives the same
 * integer; the result is rounded once to binary64.
 * Pinned against Python's math.fsum (a correctly rounded sum) by
 * tests/test_oracle_specmath.py.
 * ====================================================================== */
#define SA_DIGITS 12
typedef struct {
  uint64_t d[SA_DIGITS];
  uint64_t pending;
} superacc;

static void sa_norm(superacc* A) {
  uint64_t carry = 0;
  for (int k = 0; k < SA_DIGITS; ++k) {
    uint64_t t = A->d[k] + carry;
    A->d[k] = t & 0xffffffffull;
    carry = t >> 32;
  }
  A->pending = 0;
}

static void sa_add(superacc* A, float x) {
  f32bits t;
  t.f = x;
  uint32_t ex = (t.u >> 23) & 0xffu, man = t.u & 0x7fffffu;
  uint64_t M;
  int off;
  if (ex == 0) { M = man; off = 0; }
  else { M = (uint64_t)(man | 0x800000u); off = (int)ex - 1; }
  int k = off >> 5, sh = off & 31;
  uint64_t v = M << sh;
  A->d[k] += v & 0xffffffffull;
  A->d[k + 1] += v >> 32;
  if (++A->pending == (1ull << 30)) sa_norm(A);
}

static void sa_merge(superacc* A, superacc* B) {
  sa_norm(A);
  sa_norm(B);
  for (int k = 0; k < SA_DIGITS; ++k) A->d[k] += B->d[k];
  sa_norm(A);
}

static int sa_bit(const superacc* A, int pos) {
  if (pos < 0) return 0;
  return (int)((A->d[pos >> 5] >> (pos & 31)) & 1u);
}

static double sa_round(superacc* A) {
  sa_norm(A);
  int top = SA_DIGITS - 1;
  while (top >= 0 && A->d[top] == 0) --top;
  if (top < 0) return 0.0;
  int hb = 32 * top;
  for (int b = 31; b >= 0; --b)
    if ((A->d[top] >> b) & 1u) { hb += b; break; }
  if (hb < 53) {
    uint64_t v = 0;
    for (int p = hb; p >= 0; --p) v = (v << 1) | (uint64_t)sa_bit(A, p);
    return ldexp((double)v, -149);
  }
  uint64_t mant = 0;
  for (int p = hb; p > hb - 53; --p) mant = (mant << 1) | (uint64_t)sa_bit(A, p);
  int round_bit = sa_bit(A, hb - 53);
  int sticky = 0;
  for (int p = hb - 54; p >= 0 && !sticky; --p) sticky = sa_bit(A, p);
  if (round_bit && (sticky || (mant & 1u))) {
    mant += 1;
    if (mant == (1ull << 53)) { mant >>= 1; hb += 1; }
  }
  return ldexp((double)mant, hb - 52 - 149);
}

double orc_exact_sum_f32(const float* x, int64_t n) {
  superacc A;
  memset(&A, 0, sizeof(A));
  for (int64_t k = 0; k < n; ++k) {
    if (!(x[k] >= 0.0f) || isinf(x[k])) return NAN;
    sa_add(&A, x[k]);
  }
  return sa_round(&A);
}

/* ======================================================================
 * Sampling: Eq. (pois) with the probabilities of Eq. (pij-ot) / (pij-uot).
 * ====================================================================== */

/* Raw cost of element (i, j) in the binary32 decision spec: the squared
 * Euclidean distance accumulated in ascending coordinate order with one
 * fused multiply-add per coordinate (section 5.1 uses squared Euclidean
 * cost), or the given cost matrix rounded to binary32. */
static float raw_cost32(const orc_problem* P, int32_t i, int32_t j) {
  if (P->C) return (float)P->C[(int64_t)i * P->m + j];
  float acc = 0.0f;
  for (int k = 0; k < P->d; ++k) {
    float t = (float)P->x[(int64_t)i * P->d + k] - (float)P->y[(int64_t)j * P->d + k];
    acc = fmaf(t, t, acc);
  }
  return acc;
}

/* The same in FP64 for the value path. */
static double raw_cost64(const orc_problem* P, int32_t i, int32_t j) {
  if (P->C) return P->C[(int64_t)i * P->m + j];
  double acc = 0.0;
  for (int k = 0; k < P->d; ++k) {
    double t = P->x[(int64_t)i * P->d + k] - P->y[(int64_t)j * P->d + k];
    acc = fma(t, t, acc);
  }
  return acc;
}

static int is_ot(const orc_problem* P) { return isinf(P->lambda) && P->lambda > 0; }

/* Probabilities that factor as p*_ij = min(1, r_i c_j): Eq. (pij-ot), or the
 * equal probabilities of the Rand-Sink control. */
static int separable(const orc_problem* P) { return is_ot(P) || P->probs == 1; }

/* Divisor of the raw cost: C = D / divisor.  With cost_norm = 1 it is the
 * maximum of the binary32 raw costs over all pairs (a maximum is exact, so
 * every implementation of the spec finds the same number); with cost_norm = 2
 * the given cost_scale; otherwise 1.  Both the decision and the value path
 * use it. */
static double cost_divisor(const orc_problem* P, const orc_scalars* S) {
  if (P->cost_norm == 1 && S->dmax32 > 0.0f) return (double)S->dmax32;
  if (P->cost_norm == 2 && P->cost_scale > 0.0) return P->cost_scale;
  return 1.0;
}

static int is_wfr(const orc_problem* P) { return P->cost_kind == 1; }

/* Wasserstein-Fisher-Rao cost (section 2.2) from the squared distance D:
 * C = -log cos_+^2(sqrt(D) / (2 eta)), +inf where sqrt(D) / (2 eta) >= pi/2. */
static double wfr_cost64(const orc_problem* P, double D) {
  const double z = sqrt(D) / (2.0 * P->eta);
  if (z >= 0.5 * M_PI) return INFINITY;
  return -2.0 * log(cos(z));
}

/* The cost of the value path: WFR, or the raw cost over its divisor. */
static double cost64(const orc_problem* P, const orc_scalars* S, int32_t i, int32_t j) {
  const double d = raw_cost64(P, i, j);
  return is_wfr(P) ? wfr_cost64(P, d) : d / cost_divisor(P, S);
}

/* binary32 decision factor K_ij^{eps/(2lam+eps)} = exp(-C_ij/(2lam+eps)).
 * Squared Euclidean: E(-D kappa).  WFR: with z = fl(fl(sqrt D) inv2eta),
 * 0 for z >= fl(pi/2), else E(fl(g2 L(cos z))) (cos^2 to the power
 * 1/(2lam+eps)), 0 when the spec cos is not positive. */
static float uot_factor(const orc_problem* P, const orc_scalars* S, float dd) {
  if (!is_wfr(P)) return orc_exp32(-(dd * S->kappa32));
  const float z = sqrtf(dd) * S->inv2eta32;
  if (!(z < (float)(0.5 * M_PI))) return 0.0f;
  const float c = orc_cos32(z);
  if (!(c > 0.0f)) return 0.0f;
  return orc_exp32(S->g2_32 * orc_log32(c));
}

/* UOT weight w_ij = (A_i B_j) E(-D_ij kappa): the numerator of Eq. (pij-uot),
 * since K_ij^{eps/(2lam+eps)} = exp(-C_ij/(2lam+eps)). */
static float uot_weight(const orc_problem* P, const float* rowf, const float* colf,
                        const orc_scalars* S, int32_t i, int32_t j) {
  const float e = uot_factor(P, S, raw_cost32(P, i, j));
  return (rowf[i] * colf[j]) * e;
}

float orc_pstar_raw(const orc_problem* P, const float* rowf, const float* colf,
                    const orc_scalars* S, int32_t i, int32_t j) {
  if (separable(P)) return rowf[i] * colf[j];
  return S->scale32 * uot_weight(P, rowf, colf, S, i, j);
}

static int check_problem(const orc_problem* P) {
  if (P->n < 1 || P->m < 1) return -1;
  if (!P->C && (P->d < 1 || !P->x || !P->y)) return -1;
  if (!(P->eps > 0.0) || !(P->s > 0.0) || !(P->lambda > 0.0)) return -1;
  if (P->cost_norm == 2 && !(P->cost_scale > 0.0)) return -1;
  if (P->cost_kind != 0 && P->cost_kind != 1) return -1;
  if (is_wfr(P) && (P->C || P->cost_norm != 0 || !(P->eta > 0.0))) return -1;
  if (P->probs != 0 && P->probs != 1) return -1;
  if (!P->a || !P->b) return -1;
  for (int32_t i = 0; i < P->n; ++i) if (!(P->a[i] >= 0.0) || isinf(P->a[i])) return -1;
  for (int32_t j = 0; j < P->m; ++j) if (!(P->b[j] >= 0.0) || isinf(P->b[j])) return -1;
  return 0;
}

int orc_factors(const orc_problem* P, float* rowf, float* colf, orc_scalars* S) {
  if (check_problem(P)) return -1;
  const int32_t n = P->n, m = P->m;
  memset(S, 0, sizeof(*S));
  /* maximum raw cost over all pairs, in both precisions (max is exact); it is
     the divisor of the max-normalised cost only, so other normalisations skip it */
  float dmax32 = 0.0f;
  double dmax64 = 0.0;
#pragma omp parallel for reduction(max : dmax32, dmax64) schedule(static)
  for (int32_t i = 0; i < (P->cost_norm == 1 ? n : 0); ++i) {
    for (int32_t j = 0; j < m; ++j) {
      float d32 = raw_cost32(P, i, j);
      double d64 = raw_cost64(P, i, j);
      if (d32 > dmax32) dmax32 = d32;
      if (d64 > dmax64) dmax64 = d64;
    }
  }
  S->dmax32 = dmax32;
  S->dmax64 = dmax64;
  S->s32 = (float)P->s;
  if (P->probs == 1) {
    /* Rand-Sink: p_ij = 1/(n m) for every element; p*_ij = min(1, s p_ij) */
    S->scale32 = (float)(1.0 / ((double)n * (double)m));
    for (int32_t i = 0; i < n; ++i) rowf[i] = S->s32 * S->scale32;
    for (int32_t j = 0; j < m; ++j) colf[j] = 1.0f;
    return 0;
  }
  if (is_ot(P)) {
    /* Eq. (pij-ot): p_ij = sqrt(a_i) sqrt(b_j) / (sum sqrt(a) sum sqrt(b)) */
    float* sa = (float*)malloc(sizeof(float) * (size_t)n);
    float* sb = (float*)malloc(sizeof(float) * (size_t)m);
    for (int32_t i = 0; i < n; ++i) sa[i] = sqrtf((float)P->a[i]);
    for (int32_t j = 0; j < m; ++j) sb[j] = sqrtf((float)P->b[j]);
    S->sum1 = orc_exact_sum_f32(sa, n);
    S->sum2 = orc_exact_sum_f32(sb, m);
    double prod = S->sum1 * S->sum2;
    if (!(prod > 0.0)) { free(sa); free(sb); return -2; }
    S->scale32 = (float)(1.0 / prod);
    for (int32_t i = 0; i < n; ++i) rowf[i] = (S->s32 * sa[i]) * S->scale32;
    for (int32_t j = 0; j < m; ++j) colf[j] = sb[j];
    free(sa);
    free(sb);
    return 0;
  }
  /* Eq. (pij-uot) */
  double t = 2.0 * P->lambda + P->eps;
  S->gamma32 = (float)(P->lambda / t);
  S->kappa32 = (float)(1.0 / (cost_divisor(P, S) * t));
  S->inv2eta32 = is_wfr(P) ? (float)(1.0 / (2.0 * P->eta)) : 0.0f;
  S->g2_32 = (float)(2.0 / t);
  for (int32_t i = 0; i < n; ++i) {
    float a32 = (float)P->a[i];
    rowf[i] = a32 > 0.0f ? orc_exp32(S->gamma32 * orc_log32(a32)) : 0.0f;
  }
  for (int32_t j = 0; j < m; ++j) {
    float b32 = (float)P->b[j];
    colf[j] = b32 > 0.0f ? orc_exp32(S->gamma32 * orc_log32(b32)) : 0.0f;
  }
  /* Z = sum_ij w_ij, exactly */
  superacc total;
  memset(&total, 0, sizeof(total));
#pragma omp parallel
  {
    superacc part;
    memset(&part, 0, sizeof(part));
#pragma omp for schedule(static)
    for (int32_t i = 0; i < n; ++i)
      for (int32_t j = 0; j < m; ++j) sa_add(&part, uot_weight(P, rowf, colf, S, i, j));
#pragma omp critical
    sa_merge(&total, &part);
  }
  S->sum1 = sa_round(&total);
  if (!(S->sum1 > 0.0)) return -2;
  S->scale32 = (float)(P->s / S->sum1);
  return 0;
}

/* One element's decision and value.  Returns 1 if sampled. */
static int sample_elem(const orc_problem* P, const float* rowf, const float* colf,
                       const orc_scalars* S, int32_t i, int32_t j, float* ps) {
  float praw = orc_pstar_raw(P, rowf, colf, S, i, j);
  uint32_t U = orc_draw24(P->seed, P->pid, (uint32_t)i, (uint32_t)j);
  float u = (float)U * 0x1p-24f;
  *ps = praw < 1.0f ? praw : 1.0f;
  return u < praw;
}

int64_t orc_count(const orc_problem* P, const float* rowf, const float* colf,
                  const orc_scalars* S, int32_t* row_cnt) {
  int64_t total = 0;
#pragma omp parallel for reduction(+ : total) schedule(dynamic, 8)
  for (int32_t i = 0; i < P->n; ++i) {
    int32_t c = 0;
    float ps;
    for (int32_t j = 0; j < P->m; ++j) c += sample_elem(P, rowf, colf, S, i, j, &ps);
    row_cnt[i] = c;
    total += c;
  }
  return total;
}

/* Value of a sampled element (i, j) with p* = ps, written at position c. */
static void emit_elem(const orc_problem* P, const orc_scalars* S, int32_t i, int32_t j, float ps, int32_t c,
                      int32_t* cols, double* val, double* logval, float* pstar, double* cost) {
  double Cn = cost64(P, S, i, j);
  double Kij = exp(-Cn / P->eps);
  if (cols) cols[c] = j;
  if (val) val[c] = Kij / (double)ps;
  if (logval) logval[c] = -Cn / P->eps - log((double)ps);
  if (pstar) pstar[c] = ps;
  if (cost) cost[c] = Cn;
}

int32_t orc_sample_row(const orc_problem* P, const float* rowf, const float* colf,
                       const orc_scalars* S, int32_t i, int32_t* cols, double* val,
                       double* logval, float* pstar, double* cost) {
  int32_t c = 0;
  for (int32_t j = 0; j < P->m; ++j) {
    float ps;
    if (!sample_elem(P, rowf, colf, S, i, j, &ps)) continue;
    emit_elem(P, S, i, j, ps, c, cols, val, logval, pstar, cost);
    ++c;
  }
  return c;
}

/* ======================================================================
 * Skip sampler: the same law as one Bernoulli(p*_ij) decision per element,
 * with work proportional to the sampled count instead of n m.  Thinning
 * construction with a row bound q_i >= p_ij for every j: OT p_ij =
 * fl(r_i c_j), q_i = min(1, fl(r_i cmax)); UOT p_ij = fl(scale fl(fl(A_i B_j)
 * E(-D_ij kappa))), q_i = min(1, fl(scale fl(A_i cmax))) (E <= 1 and
 * rounding is monotone), cmax = max_j of the column factors.  Candidates form a Bernoulli(q_i) process
 * over j = 0 .. m-1, generated by geometric gaps: with U uniform on (0, 1],
 * G = floor(log U / log(1 - q_i)) has P(G >= k) = P(U <= (1 - q_i)^k) =
 * (1 - q_i)^k.  A candidate j is kept when V < fl(p_ij / q_i), V uniform on
 * [0, 1), so j is kept with probability q_i (p_ij / q_i) = p_ij,
 * independently of every other element (to the 2^-24 resolution of U, V).
 * Draws: candidate t of row i reads Philox4x32-10 at counter (t >> 1, i,
 * pid, 0x5B1E) under key (seed), words 2(t & 1) (gap) and 2(t & 1) + 1
 * (acceptance); U = ((w >> 8) + 1) 2^-24, V = (w >> 8) 2^-24.  Every step is
 * the binary32 operation written here (log1m and log are the spec's).
 * Pinned by tests/test_oracle_skip.py (inclusion frequencies, pairwise
 * independence, expected count, degenerate rows).
 * ====================================================================== */

/* log(1 - q) for 0 < q < 1: the spec log of 1 - q for q >= 1/4; below, 2
 * atanh(z) with z = -q / (2 - q) (|z| <= 1/7) by its series to z^13. */
float orc_log1m32(float q) {
  if (q >= 0.25f) return orc_log32(1.0f - q);
  float z = -q / (2.0f - q);
  float w = z * z;
  float P = (float)(1.0 / 13.0);
  P = fmaf(P, w, (float)(1.0 / 11.0));
  P = fmaf(P, w, (float)(1.0 / 9.0));
  P = fmaf(P, w, (float)(1.0 / 7.0));
  P = fmaf(P, w, 0.2f);
  P = fmaf(P, w, (float)(1.0 / 3.0));
  float z2 = z + z;
  return fmaf(z2, w * P, z2);
}

void orc_log1m32_vec(const float* q, float* y, int64_t n) {
  for (int64_t k = 0; k < n; ++k) y[k] = orc_log1m32(q[k]);
}

void orc_skip_words(uint64_t seed, uint32_t pid, uint32_t i, uint32_t t, uint32_t w[2]) {
  uint32_t ctr[4] = {t >> 1, i, pid, 0x5B1Eu};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  w[0] = out[2u * (t & 1u)];
  w[1] = out[2u * (t & 1u) + 1u];
}

/* The largest column factor (a maximum is exact). */
float orc_colf_max(const float* colf, int32_t m) {
  float c = 0.0f;
  for (int32_t j = 0; j < m; ++j) if (colf[j] > c) c = colf[j];
  return c;
}

int32_t orc_skip_row(const orc_problem* P, const float* rowf, const float* colf, const orc_scalars* S,
                     float cmax, int32_t i, int32_t* cols, double* val, double* logval, float* pstar,
                     double* cost) {
  const float r = rowf[i];
  const float q = separable(P) ? r * cmax : S->scale32 * (r * cmax);
  if (!(q > 0.0f)) return 0;
  const int full = q >= 1.0f;
  const float L = full ? 0.0f : orc_log1m32(q);
  int64_t j = -1;
  int32_t c = 0;
  for (uint32_t t = 0;; ++t) {
    uint32_t w[2];
    orc_skip_words(P->seed, P->pid, (uint32_t)i, t, w);
    if (full) {
      j += 1;
    } else {
      const float U = (float)((w[0] >> 8) + 1u) * 0x1p-24f;
      const float ratio = orc_log32(U) / L;
      if (!(ratio < (float)P->m)) break;
      j += 1 + (int64_t)floorf(ratio);
    }
    if (j >= P->m) break;
    const float p = orc_pstar_raw(P, rowf, colf, S, i, (int32_t)j);
    const float acc = full ? p : p / q;
    const float V = (float)(w[1] >> 8) * 0x1p-24f;
    if (V < acc) {
      emit_elem(P, S, i, (int32_t)j, p < 1.0f ? p : 1.0f, c, cols, val, logval, pstar, cost);
      ++c;
    }
  }
  return c;
}

/* Row counts of the skip sampler's sketch (row_cnt[n]); returns the total. */
int64_t orc_skip_count(const orc_problem* P, const float* rowf, const float* colf, const orc_scalars* S,
                       int32_t* row_cnt) {
  const float cmax = orc_colf_max(colf, P->m);
  int64_t nnz = 0;
#pragma omp parallel for reduction(+ : nnz) schedule(dynamic, 64)
  for (int32_t i = 0; i < P->n; ++i) {
    row_cnt[i] = orc_skip_row(P, rowf, colf, S, cmax, i, NULL, NULL, NULL, NULL, NULL);
    nnz += row_cnt[i];
  }
  return nnz;
}

static int64_t sparsify_impl(const orc_problem* P, int skip, int32_t* row_ptr, int32_t* col_idx, double* val,
                             double* logval, float* pstar, double* cost, int32_t* col_ptr,
                             int32_t* row_idx, double* valT, int32_t* perm, orc_scalars* S) {
  const int32_t n = P->n, m = P->m;
  float* rowf = (float*)malloc(sizeof(float) * (size_t)n);
  float* colf = (float*)malloc(sizeof(float) * (size_t)m);
  if (orc_factors(P, rowf, colf, S)) { free(rowf); free(colf); return -1; }
  const float cmax = skip ? orc_colf_max(colf, m) : 0.0f;
  int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t nnz = 0;
  if (skip) {
    nnz = orc_skip_count(P, rowf, colf, S, cnt);
  } else {
    nnz = orc_count(P, rowf, colf, S, cnt);
  }
  row_ptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + cnt[i];
#pragma omp parallel for schedule(dynamic, 8)
  for (int32_t i = 0; i < n; ++i) {
    int64_t o = row_ptr[i];
    if (skip)
      orc_skip_row(P, rowf, colf, S, cmax, i, col_idx + o, val ? val + o : NULL, logval ? logval + o : NULL,
                   pstar ? pstar + o : NULL, cost ? cost + o : NULL);
    else
      orc_sample_row(P, rowf, colf, S, i, col_idx + o, val ? val + o : NULL,
                     logval ? logval + o : NULL, pstar ? pstar + o : NULL, cost ? cost + o : NULL);
  }
  /* stable transpose: rows ascending inside every column */
  if (col_ptr) {
    int32_t* cur = (int32_t*)calloc((size_t)m + 1, sizeof(int32_t));
    for (int64_t k = 0; k < nnz; ++k) cur[col_idx[k] + 1] += 1;
    col_ptr[0] = 0;
    for (int32_t j = 0; j < m; ++j) col_ptr[j + 1] = col_ptr[j] + cur[j + 1];
    for (int32_t j = 0; j < m; ++j) cur[j] = col_ptr[j];
    for (int32_t i = 0; i < n; ++i) {
      for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
        int32_t pos = cur[col_idx[k]]++;
        if (row_idx) row_idx[pos] = i;
        if (valT && val) valT[pos] = val[k];
        if (perm) perm[pos] = k;
      }
    }
    free(cur);
  }
  free(cnt);
  free(rowf);
  free(colf);
  return nnz;
}

int64_t orc_sparsify(const orc_problem* P, int32_t* row_ptr, int32_t* col_idx, double* val,
                     double* logval, float* pstar, double* cost, int32_t* col_ptr,
                     int32_t* row_idx, double* valT, int32_t* perm, orc_scalars* S) {
  return sparsify_impl(P, 0, row_ptr, col_idx, val, logval, pstar, cost, col_ptr, row_idx, valT, perm, S);
}

int64_t orc_sparsify_skip(const orc_problem* P, int32_t* row_ptr, int32_t* col_idx, double* val,
                          double* logval, float* pstar, double* cost, int32_t* col_ptr,
                          int32_t* row_idx, double* valT, int32_t* perm, orc_scalars* S) {
  return sparsify_impl(P, 1, row_ptr, col_idx, val, logval, pstar, cost, col_ptr, row_idx, valT, perm, S);
}

int orc_dense_kernel(const orc_problem* P, double* K, double* Cn) {
  if (check_problem(P)) return -1;
  orc_scalars S;
  memset(&S, 0, sizeof(S));
  for (int32_t i = 0; i < P->n; ++i)
    for (int32_t j = 0; j < P->m; ++j) {
      float d = raw_cost32(P, i, j);
      if (d > S.dmax32) S.dmax32 = d;
    }
  for (int32_t i = 0; i < P->n; ++i)
    for (int32_t j = 0; j < P->m; ++j) {
      double c = cost64(P, &S, i, j);
      if (Cn) Cn[(int64_t)i * P->m + j] = c;
      if (K) K[(int64_t)i * P->m + j] = exp(-c / P->eps);
    }
  return 0;
}

/* ======================================================================
 * Scaling iterations: Alg. 1 (phi = 1) and Alg. 2 (phi = lam/(lam+eps)).
 * Iteration t computes u^t from v^{t-1}, then v^t from u^t (u^0 = v^0 = 1).
 * Because v^t is computed from u^t, the column condition of Eq. (first-order
 * conditions) holds for the pair (u^t, v^t) up to rounding; the stopping
 * residual of that pair is therefore its row side
 *     rho_t = sum over reachable i of | (u^t_i)^{1/phi} (K~ v^t)_i - a_i |,
 * which the row pass of iteration t+1 obtains from K~ v^t.  The solver
 * returns the first pair with rho_t <= tol (t >= 1).  Rows whose (K~v)_i is
 * zero get u_i = 0 and are unreachable (their mass is reported), likewise
 * columns.
 * Pinned in tests/test_oracle_sinkhorn.py (LP limit, closed forms, dual
 * maximisation by a generic optimiser, marginals, duality gap).
 * ====================================================================== */
typedef struct {
  int dense;
  int32_t n, m;
  const double* K;  /* dense */
  const int32_t *row_ptr, *col_idx, *col_ptr, *row_idx;
  const double *val, *valT;
} kop;

static void kop_rows(const kop* O, const double* v, double* q) { /* q = K v */
  for (int32_t i = 0; i < O->n; ++i) {
    double acc = 0.0;
    if (O->dense) {
      const double* Ki = O->K + (int64_t)i * O->m;
      for (int32_t j = 0; j < O->m; ++j) acc += Ki[j] * v[j];
    } else {
      for (int32_t k = O->row_ptr[i]; k < O->row_ptr[i + 1]; ++k) acc += O->val[k] * v[O->col_idx[k]];
    }
    q[i] = acc;
  }
}

static void kop_cols(const kop* O, const double* u, double* r) { /* r = K^T u */
  if (O->dense) {
    for (int32_t j = 0; j < O->m; ++j) {
      double acc = 0.0;
      for (int32_t i = 0; i < O->n; ++i) acc += O->K[(int64_t)i * O->m + j] * u[i];
      r[j] = acc;
    }
  } else {
    for (int32_t j = 0; j < O->m; ++j) {
      double acc = 0.0;
      for (int32_t k = O->col_ptr[j]; k < O->col_ptr[j + 1]; ++k) acc += O->valT[k] * u[O->row_idx[k]];
      r[j] = acc;
    }
  }
}

static double row_residual(int32_t n, const double* u, const double* q, const double* a, double phi,
                           double* unreach) {
  double res = 0.0, un = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    if (q[i] > 0.0) {
      double ui = (phi == 1.0) ? u[i] : pow(u[i], 1.0 / phi);
      res += fabs(ui * q[i] - a[i]);
    } else {
      un += a[i];
    }
  }
  if (unreach) *unreach = un;
  return res;
}

static double col_unreach(int32_t m, const double* r, const double* b) {
  double un = 0.0;
  for (int32_t j = 0; j < m; ++j) if (!(r[j] > 0.0)) un += b[j];
  return un;
}

static int sinkhorn_plain(const kop* O, const double* a, const double* b, double eps, double lambda,
                          double tol, int32_t max_iter, int32_t stop_rule, const double* u0,
                          const double* v0, double* u, double* v, orc_solve_info* info) {
  const int32_t n = O->n, m = O->m;
  const double phi = isinf(lambda) ? 1.0 : lambda / (lambda + eps);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  double* r = (double*)calloc((size_t)m, sizeof(double));
  double* up = (double*)malloc(sizeof(double) * (size_t)n);
  double* vp = (double*)malloc(sizeof(double) * (size_t)m);
  for (int32_t i = 0; i < n; ++i) u[i] = u0 ? u0[i] : 1.0;
  for (int32_t j = 0; j < m; ++j) v[j] = v0 ? v0[j] : 1.0;
  memset(info, 0, sizeof(*info));
  int done = 0;
  for (int32_t t = 1; t <= max_iter && !done; ++t) {
    kop_rows(O, v, q);
    if (t >= 2 && stop_rule == ORC_STOP_RESIDUAL) {
      double un;
      double res = row_residual(n, u, q, a, phi, &un);
      if (!isfinite(res)) { info->status = 5; info->iters = t - 1; info->residual = res; done = 1; break; }
      if (res <= tol) {
        info->iters = t - 1;
        info->residual = res;
        info->unreach_a = un;
        info->unreach_b = col_unreach(m, r, b);
        info->status = 0;
        done = 1;
        break;
      }
    }
    memcpy(up, u, sizeof(double) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) u[i] = q[i] > 0.0 ? pow(a[i] / q[i], phi) : 0.0;
    kop_cols(O, u, r);
    memcpy(vp, v, sizeof(double) * (size_t)m);
    for (int32_t j = 0; j < m; ++j) v[j] = r[j] > 0.0 ? pow(b[j] / r[j], phi) : 0.0;
    if (stop_rule == ORC_STOP_DELTA_UV) {
      double dl = 0.0;
      for (int32_t i = 0; i < n; ++i) dl += fabs(u[i] - up[i]);
      for (int32_t j = 0; j < m; ++j) dl += fabs(v[j] - vp[j]);
      if (!isfinite(dl)) { info->status = 5; info->iters = t; info->residual = dl; done = 1; break; }
      if (dl <= tol) {
        info->iters = t;
        info->residual = dl;
        double un;
        kop_rows(O, v, q);
        row_residual(n, u, q, a, phi, &un);
        info->unreach_a = un;
        info->unreach_b = col_unreach(m, r, b);
        info->status = 0;
        done = 1;
        break;
      }
    }
  }
  if (!done) {
    double un;
    kop_rows(O, v, q);
    double res = row_residual(n, u, q, a, phi, &un);
    info->iters = max_iter;
    if (stop_rule == ORC_STOP_RESIDUAL) info->residual = res;
    info->unreach_a = un;
    info->unreach_b = col_unreach(m, r, b);
    info->status = !isfinite(res) ? 5 : (stop_rule == ORC_STOP_RESIDUAL && res <= tol ? 0 : 1);
  }
  free(q); free(r); free(up); free(vp);
  return info->status;
}

int orc_sinkhorn_sparse(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                        const double* val, const int32_t* col_ptr, const int32_t* row_idx,
                        const double* valT, const double* a, const double* b, double eps,
                        double lambda, double tol, int32_t max_iter, int32_t stop_rule,
                        const double* u0, const double* v0, double* u, double* v,
                        orc_solve_info* info) {
  kop O = {0, n, m, NULL, row_ptr, col_idx, col_ptr, row_idx, val, valT};
  return sinkhorn_plain(&O, a, b, eps, lambda, tol, max_iter, stop_rule, u0, v0, u, v, info);
}

int orc_sinkhorn_dense(int32_t n, int32_t m, const double* K, const double* a, const double* b,
                       double eps, double lambda, double tol, int32_t max_iter,
                       int32_t stop_rule, const double* u0, const double* v0, double* u,
                       double* v, orc_solve_info* info) {
  kop O = {1, n, m, K, NULL, NULL, NULL, NULL, NULL, NULL};
  return sinkhorn_plain(&O, a, b, eps, lambda, tol, max_iter, stop_rule, u0, v0, u, v, info);
}

/* ----------------------------------------------------------------------
 * Log domain: alpha = eps log u, beta = eps log v.  With log K~_ij =
 * -C~_ij/eps (C~ = C + eps log p*, the sparse cost of the UOT iteration
 * lemma's proof), the u-update of Alg. 2 reads
 *     alpha_i = phi (eps log a_i - eps LSE_{j in S_i}(beta_j/eps + log K~_ij)),
 * where LSE is log-sum-exp over the sampled support S_i of row i; the
 * v-update is symmetric.  Same iteration order and stopping residual as
 * the plain form.
 * ---------------------------------------------------------------------- */
static double lse_row(int32_t lo, int32_t hi, const int32_t* idx, const double* logval,
                      const double* pot, double inv_eps) {
  double mx = -INFINITY;
  for (int32_t k = lo; k < hi; ++k) {
    double z = pot[idx[k]] * inv_eps + logval[k];
    if (z > mx) mx = z;
  }
  if (mx == -INFINITY) return -INFINITY;
  double acc = 0.0;
  for (int32_t k = lo; k < hi; ++k) acc += exp(pot[idx[k]] * inv_eps + logval[k] - mx);
  return mx + log(acc);
}

int orc_sinkhorn_log_sparse(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                            const double* logval, const int32_t* col_ptr, const int32_t* row_idx,
                            const double* logvalT, const double* a, const double* b, double eps,
                            double lambda, double tol, int32_t max_iter, int32_t stop_rule,
                            const double* alpha0, const double* beta0, double* alpha,
                            double* beta, orc_solve_info* info) {
  const double phi = isinf(lambda) ? 1.0 : lambda / (lambda + eps);
  const double ie = 1.0 / eps;
  double* L = (double*)malloc(sizeof(double) * (size_t)n);
  double* M = (double*)malloc(sizeof(double) * (size_t)m);
  double* ap = (double*)malloc(sizeof(double) * (size_t)n);
  double* bp = (double*)malloc(sizeof(double) * (size_t)m);
  for (int32_t i = 0; i < n; ++i) alpha[i] = alpha0 ? alpha0[i] : 0.0;
  for (int32_t j = 0; j < m; ++j) { beta[j] = beta0 ? beta0[j] : 0.0; M[j] = 0.0; }
  memset(info, 0, sizeof(*info));
  int done = 0;
  for (int32_t t = 1; t <= max_iter && !done; ++t) {
    for (int32_t i = 0; i < n; ++i) L[i] = lse_row(row_ptr[i], row_ptr[i + 1], col_idx, logval, beta, ie);
    if (t >= 2 && stop_rule == ORC_STOP_RESIDUAL) {
      double res = 0.0, un = 0.0;
      for (int32_t i = 0; i < n; ++i) {
        if (L[i] > -INFINITY) res += fabs(exp(alpha[i] * ie / phi + L[i]) - a[i]);
        else un += a[i];
      }
      if (!isfinite(res)) { info->status = 5; info->iters = t - 1; info->residual = res; done = 1; break; }
      if (res <= tol) {
        double ub = 0.0;
        for (int32_t j = 0; j < m; ++j) if (!(M[j] > -INFINITY)) ub += b[j];
        info->iters = t - 1; info->residual = res; info->unreach_a = un; info->unreach_b = ub;
        info->status = 0; done = 1; break;
      }
    }
    memcpy(ap, alpha, sizeof(double) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
      alpha[i] = L[i] > -INFINITY ? phi * (eps * log(a[i]) - eps * L[i]) : -INFINITY;
    for (int32_t j = 0; j < m; ++j) M[j] = lse_row(col_ptr[j], col_ptr[j + 1], row_idx, logvalT, alpha, ie);
    memcpy(bp, beta, sizeof(double) * (size_t)m);
    for (int32_t j = 0; j < m; ++j)
      beta[j] = M[j] > -INFINITY ? phi * (eps * log(b[j]) - eps * M[j]) : -INFINITY;
    if (stop_rule == ORC_STOP_DELTA_UV) {
      double dl = 0.0;
      for (int32_t i = 0; i < n; ++i) dl += fabs(exp(alpha[i] * ie) - exp(ap[i] * ie));
      for (int32_t j = 0; j < m; ++j) dl += fabs(exp(beta[j] * ie) - exp(bp[j] * ie));
      if (dl <= tol) {
        info->iters = t; info->residual = dl; info->status = 0; done = 1;
        double un = 0.0, ub = 0.0;
        for (int32_t i = 0; i < n; ++i) if (!(lse_row(row_ptr[i], row_ptr[i + 1], col_idx, logval, beta, ie) > -INFINITY)) un += a[i];
        for (int32_t j = 0; j < m; ++j) if (!(M[j] > -INFINITY)) ub += b[j];
        info->unreach_a = un; info->unreach_b = ub;
        break;
      }
    }
  }
  if (!done) {
    double res = 0.0, un = 0.0, ub = 0.0;
    for (int32_t i = 0; i < n; ++i) {
      L[i] = lse_row(row_ptr[i], row_ptr[i + 1], col_idx, logval, beta, ie);
      if (L[i] > -INFINITY) res += fabs(exp(alpha[i] * ie / phi + L[i]) - a[i]);
      else un += a[i];
    }
    for (int32_t j = 0; j < m; ++j) if (!(M[j] > -INFINITY)) ub += b[j];
    info->iters = max_iter;
    if (stop_rule == ORC_STOP_RESIDUAL) info->residual = res;
    info->unreach_a = un; info->unreach_b = ub;
    info->status = !isfinite(res) ? 5 : (stop_rule == ORC_STOP_RESIDUAL && res <= tol ? 0 : 1);
  }
  free(L); free(M); free(ap); free(bp);
  return info->status;
}

/* ======================================================================
 * Objective terms of Alg. 3 / Alg. 4 (output line), with KL and H of
 * section 2 (0 log 0 = 0).  Pinned against scipy.special.kl_div / entr.
 * ====================================================================== */
static double kl_term(double x, double y) {
  if (x == 0.0) return y;
  if (y == 0.0) return INFINITY;
  return x * log(x / y) - x + y;
}

int orc_objective_terms(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                        const double* logT, const double* cost, const float* pstar,
                        const double* a, const double* b, double* out) {
  double* rs = (double*)calloc((size_t)n, sizeof(double));
  double* cs = (double*)calloc((size_t)m, sizeof(double));
  double tr = 0.0, ne = 0.0, lp = 0.0, mass = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      double lt = logT[k];
      if (lt == -INFINITY) continue;
      double T = exp(lt);
      if (T == 0.0) continue;
      tr += T * cost[k];
      ne += T * (lt - 1.0);
      lp += T * log((double)pstar[k]);
      mass += T;
      rs[i] += T;
      cs[col_idx[k]] += T;
    }
  }
  double kla = 0.0, klb = 0.0;
  for (int32_t i = 0; i < n; ++i) kla += kl_term(rs[i], a[i]);
  for (int32_t j = 0; j < m; ++j) klb += kl_term(cs[j], b[j]);
  out[0] = tr; out[1] = ne; out[2] = lp; out[3] = mass; out[4] = kla; out[5] = klb; out[6] = 0.0;
  free(rs);
  free(cs);
  return 0;
}
