// sps_device.cuh -- device helpers shared by the Spar-Sink kernels (sm_103a).
//
// - Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) for the per-element
//   Bernoulli draws of Eq. (pois);
// - the binary32 decision arithmetic (exp, log, squared distance) written with
//   explicitly rounded intrinsics so that no contraction or approximation
//   changes a keep/drop decision;
// - exact order-independent accumulation of non-negative binary32 terms
//   (fixed-point superaccumulator, after Collange, Defour, Graillat &
//   Iakymchuk 2015), used for the normalisers of Eq. (pij-ot) / (pij-uot);
// - warp / block reductions.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace sps {

// ---------------------------------------------------------------------------
// Philox4x32-10.  Round: multiply counter words 0 and 2 by the round
// multipliers, xor the high halves with the other words and the round key,
// permute; bump the key by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The four 24-bit draws of columns 4q .. 4q+3 of row i: counter (q, i, pid, 0x5A17).
__device__ __forceinline__ uint4 draw4(uint64_t seed, uint32_t pid, uint32_t i, uint32_t q) {
  uint4 w = philox4x32_10(make_uint4(q, i, pid, 0x5A17u), (uint32_t)seed, (uint32_t)(seed >> 32));
  return make_uint4(w.x >> 8, w.y >> 8, w.z >> 8, w.w >> 8);
}

// U = draw * 2^-24 (exact); keep iff U < p (p before clipping at 1).
__device__ __forceinline__ bool keep(uint32_t d24, float p) {
  return __fmul_rn(__uint2float_rn(d24), 5.9604644775390625e-08f) < p;
}

// ---------------------------------------------------------------------------
// binary32 spec exp / log.
// exp: x = k ln2 + r with k = rint(x / ln2) (ln 2 split in a 16-bit head and
// a binary32 tail so that k * head is exact), e^r by its degree-7 Taylor
// polynomial in Horner form, then two exact power-of-two scalings.
// log: x = 2^e m with m in [sqrt(1/2), sqrt(2)], log m = 2 atanh(z),
// z = (m-1)/(m+1), odd series to z^11.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pow2f_small(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }

__device__ __forceinline__ float spec_exp(float x) {
  if (x != x) return x;
  if (x > 88.75f) return __int_as_float(0x7f800000);
  if (x < -104.0f) return 0.0f;
  const float k = rintf(__fmul_rn(x, 1.44269502e+00f));
  float r = __fmaf_rn(-k, 0.693145751953125f, x);
  r = __fmaf_rn(-k, 1.42860677e-06f, r);
  float p = (float)(1.0 / 5040.0);
  p = __fmaf_rn(p, r, (float)(1.0 / 720.0));
  p = __fmaf_rn(p, r, (float)(1.0 / 120.0));
  p = __fmaf_rn(p, r, (float)(1.0 / 24.0));
  p = __fmaf_rn(p, r, (float)(1.0 / 6.0));
  p = __fmaf_rn(p, r, 0.5f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  const int ki = (int)k;
  const int k1 = ki / 2;
  const int k2 = ki - k1;
  // p lies in [1/2, 2): for -125 <= k <= 126 both scalings below are exact
  // and the result is normal, so adding k to p's exponent gives the same bits
  if (ki >= -125 && ki <= 126) return __int_as_float(__float_as_int(p) + (ki << 23));
  return __fmul_rn(__fmul_rn(p, pow2f_small(k1)), pow2f_small(k2));
}

// cos z for 0 <= z <= pi/2 in the binary32 spec: the Taylor series
// 1 - z^2/2! + z^4/4! - ... to z^14/14! in w = z^2 (the next term is below
// 7e-11 at pi/2), Horner form with fused multiply-adds; the coefficients are
// 1/k! rounded once to binary32.
__device__ __forceinline__ float spec_cos(float z) {
  const float w = __fmul_rn(z, z);
  float p = (float)(-1.0 / 87178291200.0);
  p = __fmaf_rn(p, w, (float)(1.0 / 479001600.0));
  p = __fmaf_rn(p, w, (float)(-1.0 / 3628800.0));
  p = __fmaf_rn(p, w, (float)(1.0 / 40320.0));
  p = __fmaf_rn(p, w, (float)(-1.0 / 720.0));
  p = __fmaf_rn(p, w, (float)(1.0 / 24.0));
  p = __fmaf_rn(p, w, -0.5f);
  return __fmaf_rn(p, w, 1.0f);
}

__device__ __forceinline__ float spec_log(float x) {
  if (x != x) return x;
  if (x < 0.0f) return __int_as_float(0x7fc00000);
  if (x == 0.0f) return __int_as_float(0xff800000);
  if (x == __int_as_float(0x7f800000)) return x;
  uint32_t u = __float_as_uint(x);
  int e = 0;
  if (u < 0x00800000u) {
    u = __float_as_uint(__fmul_rn(x, 16777216.0f));
    e = -24;
  }
  e += (int)((u >> 23) & 0xffu) - 127;
  float m = __uint_as_float((u & 0x007fffffu) | 0x3f800000u);
  if (m > 1.41421354e+00f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float f = __fsub_rn(m, 1.0f);
  const float z = __fdiv_rn(f, __fadd_rn(m, 1.0f));
  const float w = __fmul_rn(z, z);
  float P = (float)(1.0 / 11.0);
  P = __fmaf_rn(P, w, (float)(1.0 / 9.0));
  P = __fmaf_rn(P, w, (float)(1.0 / 7.0));
  P = __fmaf_rn(P, w, 0.2f);
  P = __fmaf_rn(P, w, (float)(1.0 / 3.0));
  const float q = __fmul_rn(w, P);
  const float z2 = __fadd_rn(z, z);
  const float lm = __fmaf_rn(z2, q, z2);
  const float fe = (float)e;
  const float r = __fmaf_rn(fe, 1.42860677e-06f, lm);
  return __fmaf_rn(fe, 0.693145751953125f, r);
}

// log(1 - q) for 0 < q < 1 (the skip sampler's gap rate): spec_log(1 - q)
// for q >= 1/4; below, 2 atanh(z) with z = -q / (2 - q), |z| <= 1/7, by its
// odd series to z^13.
__device__ __forceinline__ float spec_log1m(float q) {
  if (q >= 0.25f) return spec_log(__fsub_rn(1.0f, q));
  const float z = __fdiv_rn(-q, __fsub_rn(2.0f, q));
  const float w = __fmul_rn(z, z);
  float P = (float)(1.0 / 13.0);
  P = __fmaf_rn(P, w, (float)(1.0 / 11.0));
  P = __fmaf_rn(P, w, (float)(1.0 / 9.0));
  P = __fmaf_rn(P, w, (float)(1.0 / 7.0));
  P = __fmaf_rn(P, w, 0.2f);
  P = __fmaf_rn(P, w, (float)(1.0 / 3.0));
  const float z2 = __fadd_rn(z, z);
  return __fmaf_rn(z2, __fmul_rn(w, P), z2);
}

// The words of skip-sampler candidates 2c and 2c + 1 of row i: counter
// (c, i, pid, 0x5B1E); candidate 2c uses (x, y), 2c + 1 uses (z, w), the
// first word of a pair for the gap and the second for the acceptance.
__device__ __forceinline__ uint4 skip_words4(uint64_t seed, uint32_t pid, uint32_t i, uint32_t c) {
  return philox4x32_10(make_uint4(c, i, pid, 0x5B1Eu), (uint32_t)seed, (uint32_t)(seed >> 32));
}

// ---------------------------------------------------------------------------
// Cost access.  Decision path: binary32 squared distance accumulated in
// ascending coordinate order, one fused multiply-add per coordinate; or the
// given cost rounded to binary32.  Value path: the same in the value type.
// ---------------------------------------------------------------------------
struct CostView {
  const float* x32;   // n*d
  const float* y32;   // m*d
  const double* x64;  // n*d (FP64 problems)
  const double* y64;
  const float* C32;   // n*m raw cost (binary32 copy)
  const double* C64;  // n*m raw cost (FP64 problems)
  int n, m, d;
};

__device__ __forceinline__ float raw32(const CostView& cv, int i, int j) {
  if (cv.C32) return cv.C32[(int64_t)i * cv.m + j];
  const float* xi = cv.x32 + (int64_t)i * cv.d;
  const float* yj = cv.y32 + (int64_t)j * cv.d;
  float acc = 0.0f;
  for (int k = 0; k < cv.d; ++k) {
    const float t = __fsub_rn(xi[k], yj[k]);
    acc = __fmaf_rn(t, t, acc);
  }
  return acc;
}

__device__ __forceinline__ double raw64(const CostView& cv, int i, int j) {
  if (cv.C64) return cv.C64[(int64_t)i * cv.m + j];
  if (cv.C32) return (double)cv.C32[(int64_t)i * cv.m + j];
  double acc = 0.0;
  if (cv.x64) {
    const double* xi = cv.x64 + (int64_t)i * cv.d;
    const double* yj = cv.y64 + (int64_t)j * cv.d;
    for (int k = 0; k < cv.d; ++k) {
      const double t = __dsub_rn(xi[k], yj[k]);
      acc = __fma_rn(t, t, acc);
    }
  } else {
    const float* xi = cv.x32 + (int64_t)i * cv.d;
    const float* yj = cv.y32 + (int64_t)j * cv.d;
    for (int k = 0; k < cv.d; ++k) {
      const double t = __dsub_rn((double)xi[k], (double)yj[k]);
      acc = __fma_rn(t, t, acc);
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Value storage conversions.
// ---------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ float to_f(V v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

template <typename V> __device__ __forceinline__ V from_d(double v);
template <> __device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }
template <> __device__ __forceinline__ __half from_d<__half>(double v) { return __float2half_rn((float)v); }

template <typename T, typename V> __device__ __forceinline__ T load_as(const V* p) { return (T)to_f<V>(*p); }
template <> __device__ __forceinline__ double load_as<double, double>(const double* p) { return *p; }

// ---------------------------------------------------------------------------
// Reductions.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block sum of a double, result valid in thread 0.  Fixed tree: deterministic.
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// ---------------------------------------------------------------------------
// Exact accumulation of non-negative binary32 terms.
//
// A term t = M 2^E (M the 24-bit significand incl. the hidden bit, E its
// exponent) whose E is at least the window floor B is added exactly to a
// per-thread 128-bit integer counting units of 2^B; B = eW - 104 where all
// terms are known to be below 2^eW, so a term fits in 80+24 bits and a thread
// can add 2^24 terms.  Any other term (below the floor, or unexpectedly above
// the bound) takes the slow path: 32-bit digits of a full-range integer in
// units of 2^-149, added with global atomics.  Integer addition is
// associative, so the result does not depend on the order of the terms.
// ---------------------------------------------------------------------------
struct ExactAcc {            // device-resident, zero-initialised
  unsigned long long win[3];  // sum of window parts, units of 2^B (192 bits)
  unsigned long long full[12];// slow path: 32-bit digits, units of 2^-149
  int B;                      // window floor exponent
  int pad;
};

struct U128 { unsigned long long lo, hi; };

__device__ __forceinline__ void u128_add(U128& a, unsigned long long lo, unsigned long long hi) {
  const unsigned long long s = a.lo + lo;
  a.hi += hi + (s < a.lo ? 1ull : 0ull);
  a.lo = s;
}

__device__ __forceinline__ void exact_slow_add(ExactAcc* acc, float t) {
  const uint32_t u = __float_as_uint(t);
  const uint32_t ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
  unsigned long long M;
  int off;
  if (ex == 0) { M = man; off = 0; }
  else { M = (unsigned long long)(man | 0x800000u); off = (int)ex - 1; }
  const int k = off >> 5, sh = off & 31;
  const unsigned long long v = M << sh;
  atomicAdd(&acc->full[k], v & 0xffffffffull);
  atomicAdd(&acc->full[k + 1], v >> 32);
}

// Add term t >= 0 (finite) to the thread accumulator, or to the slow path.
__device__ __forceinline__ void exact_add(U128& a, ExactAcc* acc, int B, float t) {
  const uint32_t u = __float_as_uint(t);
  if (u == 0u) return;
  const uint32_t ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
  unsigned long long M;
  int E;
  if (ex == 0) { M = man; E = -149; }
  else { M = (unsigned long long)(man | 0x800000u); E = (int)ex - 150; }
  const int p = E - B;
  if (p < 0 || p > 80) { exact_slow_add(acc, t); return; }
  if (p < 64) {
    const unsigned long long lo = M << p;
    const unsigned long long hi = (p > 40) ? (M >> (64 - p)) : 0ull;
    u128_add(a, lo, hi);
  } else {
    u128_add(a, 0ull, M << (p - 64));
  }
}

// Warp-reduce the thread accumulators into 192 bits and add them to the
// global window sum (multi-word atomic add with carry propagation).
__device__ __forceinline__ void exact_flush(const U128& a, ExactAcc* acc) {
  unsigned long long l0 = a.lo, l1 = a.hi, l2 = 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long r0 = __shfl_xor_sync(0xffffffffu, l0, o);
    const unsigned long long r1 = __shfl_xor_sync(0xffffffffu, l1, o);
    const unsigned long long r2 = __shfl_xor_sync(0xffffffffu, l2, o);
    const unsigned long long s0 = l0 + r0;
    const unsigned long long c0 = s0 < l0 ? 1ull : 0ull;
    const unsigned long long t1 = l1 + r1;
    const unsigned long long c1 = t1 < l1 ? 1ull : 0ull;
    const unsigned long long s1 = t1 + c0;
    const unsigned long long c1b = s1 < t1 ? 1ull : 0ull;
    l0 = s0;
    l1 = s1;
    l2 = l2 + r2 + c1 + c1b;
  }
  if ((threadIdx.x & 31) == 0 && (l0 | l1 | l2)) {
    const unsigned long long o0 = atomicAdd(&acc->win[0], l0);
    const unsigned long long c0 = (o0 + l0 < o0) ? 1ull : 0ull;
    const unsigned long long a1 = l1 + c0;
    const unsigned long long c1a = (a1 < l1) ? 1ull : 0ull;
    const unsigned long long o1 = atomicAdd(&acc->win[1], a1);
    const unsigned long long c1b = (o1 + a1 < o1) ? 1ull : 0ull;
    atomicAdd(&acc->win[2], l2 + c1a + c1b);
  }
}

// Round the exact sum (window part * 2^B + slow part * 2^-149) to the nearest
// binary64, ties to even.  Single-thread helper.
__device__ inline double exact_round(const ExactAcc* acc) {
  // big integer in units of 2^-149, 32-bit digits
  const int ND = 16;
  unsigned long long dig[ND];
  for (int k = 0; k < ND; ++k) dig[k] = 0ull;
  for (int k = 0; k < 12; ++k) dig[k] += acc->full[k];
  const int sh = acc->B + 149;  // >= 0 by construction
  // add the 192-bit window value shifted left by sh bits
  for (int w = 0; w < 6; ++w) {
    const unsigned long long part = (acc->win[w >> 1] >> (32 * (w & 1))) & 0xffffffffull;
    if (!part) continue;
    const int pos = sh + 32 * w;
    const int k = pos >> 5, s = pos & 31;
    const unsigned long long v = part << s;
    dig[k] += v & 0xffffffffull;
    dig[k + 1] += v >> 32;
  }
  unsigned long long carry = 0ull;
  for (int k = 0; k < ND; ++k) {
    const unsigned long long t = dig[k] + carry;
    dig[k] = t & 0xffffffffull;
    carry = t >> 32;
  }
  int top = ND - 1;
  while (top >= 0 && dig[top] == 0ull) --top;
  if (top < 0) return 0.0;
  const int hb = 32 * top + 31 - __clzll(dig[top] << 32);
  auto bit = [&](int p) -> unsigned long long {
    return p < 0 ? 0ull : ((dig[p >> 5] >> (p & 31)) & 1ull);
  };
  if (hb < 53) {
    unsigned long long v = 0ull;
    for (int p = hb; p >= 0; --p) v = (v << 1) | bit(p);
    return ldexp((double)v, -149);
  }
  unsigned long long mant = 0ull;
  for (int p = hb; p > hb - 53; --p) mant = (mant << 1) | bit(p);
  const unsigned long long rb = bit(hb - 53);
  unsigned long long sticky = 0ull;
  for (int p = hb - 54; p >= 0 && !sticky; --p) sticky = bit(p);
  int e = hb;
  if (rb && (sticky || (mant & 1ull))) {
    mant += 1ull;
    if (mant == (1ull << 53)) { mant >>= 1; e += 1; }
  }
  return ldexp((double)mant, e - 52 - 149);
}

// Window floor for terms bounded above by `bound` (> 0 finite): B = eW - 104
// with bound < 2^eW, clamped to >= -149.
__device__ __forceinline__ int exact_floor_for(float bound) {
  const uint32_t u = __float_as_uint(bound);
  const int ex = (int)((u >> 23) & 0xffu);
  const int eW = (ex == 0) ? -126 : ex - 126;   // bound < 2^(ex-126)
  const int B = eW - 104;
  return B < -149 ? -149 : B;
}

// C_ij / eps for log K~ without the FP64 pipe (narrow on this GPU): the
// squared distance of the binary32 points in double-float arithmetic (exact
// differences by TwoSum, squares by an FMA error term), times 1/(dn eps) held
// as a binary32 pair.  The result is within about one binary32 ulp of the
// FP64 value.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float cost_over_eps_df(const float* xi, const float* yj, int d, float k_hi, float k_lo) {
  float hi = 0.0f, lo = 0.0f;
  for (int k = 0; k < d; ++k) {
    float t, te;
    two_sum(xi[k], -yj[k], t, te);
    const float p = __fmul_rn(t, t);
    const float pe = __fmaf_rn(t, t, -p);                 // exact error of t*t
    const float q = __fmaf_rn(__fmul_rn(2.0f, t), te, pe);  // 2 t te + error (te^2 below ulp)
    float s, se;
    two_sum(hi, p, s, se);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(se, q));
  }
  const float ph = __fmul_rn(hi, k_hi);
  const float pe = __fmaf_rn(hi, k_hi, -ph);
  return __fadd_rn(ph, __fmaf_rn(hi, k_lo, __fmaf_rn(lo, k_hi, pe)));
}

}  // namespace sps
