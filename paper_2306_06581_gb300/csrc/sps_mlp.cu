// sps_mlp.cu -- learned warm start for the scaling iterations.
//
// The paper starts Alg. 1 / Alg. 2 from u = v = 1.  This library can start
// from predicted potentials instead: for each side (source rows -> alpha,
// target columns -> beta) a small network reads one point and a summary of
// the OTHER measure,
//   f_i  = [x_i / sqrt(Dmax), n a_i]                    (point features, F = d + 1)
//   P    = sum_j b_j relu(We f_j + ce) / sum_j b_j      (pooled embedding of the other side, E)
//   h1   = relu(W1 [f_i, P] + b1),  h2 = relu(W2 h1 + b2),  alpha^_i = w3 . h2 + b3
// with hidden width H = 128, weights stored in BF16 for the forward pass and
// FP32 accumulation; the FP32 master weights are trained by Adam on the
// potentials the solver itself returns (gauge-fixed: sum a alpha = sum b beta),
// with the loss sum_i a_i ((alpha^_i - alpha_i)/eps)^2 / sum a (and the same
// for beta).  Only the warm start changes: the solver's fixed point and
// stopping rule are those of the cold start.
//
// Kernels: pooled embedding (forward / backward), a fused tile kernel that
// runs the forward pass of 32 points and, for training, their backward pass
// with the weight gradients accumulated in shared memory by persistent
// blocks, Adam, the BF16 refresh, initialisation and the gauge fix.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "sps_internal.h"

namespace sps {
namespace mlp {

constexpr int E = SPS_MLP_EMB;
constexpr int H = SPS_MLP_HIDDEN;
constexpr int TP = 32;          // points per tile
constexpr int NT = 256;         // threads of the tile kernel
constexpr int HP = H + 1;       // padded row stride of W2 in shared memory
constexpr int HB = H + 8;       // row stride (BF16 elements) of the split h1 copies: conflict-free fragment loads
constexpr int PB = TP + 8;      // row stride (BF16) of the point-contiguous copies of the backward

struct Off {                    // offsets (floats) of one side's parameters
  int F, D0, We, ce, W1, b1, W2, b2, w3, b3, size;
};

__host__ __device__ inline Off offsets(int d) {
  Off o;
  o.F = d + 1;
  o.D0 = o.F + E;
  o.We = 0;
  o.ce = o.We + E * o.F;
  o.W1 = o.ce + E;
  o.b1 = o.W1 + H * o.D0;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + H * H;
  o.w3 = o.b2 + H;
  o.b3 = o.w3 + H;
  o.size = o.b3 + 1;
  return o;
}

// One side: the points whose potentials are predicted ("self") and the
// measure that is pooled ("other").
struct Side {
  const float* sp; const float* sw; int sn;   // self points (sn x d), weights
  const float* op; const float* ow; int on;   // other points, weights
  const float* target;                        // gauge-fixed target potentials (train) or null
  float* out;                                 // predictions (infer) or null
  const __nv_bfloat16* wb;                    // BF16 weights of this side
  const float* wf;                            // FP32 master weights of this side (backward)
  float* grad;                                // gradient of this side (train)
  float* pool;                                // [E + 1]: sum_j b_j e_j, sum_j b_j
  float* dpool;                               // [E]: dL/dP
  float* loss;                                // accumulated loss
  int d;
  float inv_s;                                // 1 / sqrt(Dmax)
  float inv_eps2;                             // 1 / eps^2
};

__device__ __forceinline__ float bf(const __nv_bfloat16* w, int k) { return __bfloat162float(w[k]); }

__device__ __forceinline__ void features(const float* p, const float* w, int cnt, int i, int d, float inv_s,
                                         float* f) {
  for (int c = 0; c < d; ++c) f[c] = p[(size_t)i * d + c] * inv_s;
  f[d] = (float)cnt * w[i];
}

// pooled embedding of the other measure: pool[e] += sum_j b_j relu(We f_j + ce)_e, pool[E] += sum_j b_j
__global__ void k_pool_fwd(Side S) {
  const Off o = offsets(S.d);
  __shared__ float acc[E + 1];
  if (threadIdx.x <= E) acc[threadIdx.x] = 0.0f;
  __syncthreads();
  float loc[E + 1];
  for (int e = 0; e <= E; ++e) loc[e] = 0.0f;
  float f[17];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.on; j += gridDim.x * blockDim.x) {
    features(S.op, S.ow, S.on, j, S.d, S.inv_s, f);
    const float bj = S.ow[j];
    for (int e = 0; e < E; ++e) {
      float z = bf(S.wb, o.ce + e);
      for (int c = 0; c < o.F; ++c) z = fmaf(bf(S.wb, o.We + e * o.F + c), f[c], z);
      loc[e] += bj * fmaxf(z, 0.0f);
    }
    loc[E] += bj;
  }
  for (int e = 0; e <= E; ++e) {
    const float v = warp_sum(loc[e]);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[e], v);
  }
  __syncthreads();
  if (threadIdx.x <= E) atomicAdd(&S.pool[threadIdx.x], acc[threadIdx.x]);
}

// backward of the pool: dWe, dce from dL/dP
__global__ void k_pool_bwd(Side S) {
  const Off o = offsets(S.d);
  __shared__ float acc[E * 17 + E];
  for (int k = threadIdx.x; k < E * o.F + E; k += blockDim.x) acc[k] = 0.0f;
  __syncthreads();
  const float wsum = S.pool[E];
  float f[17];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.on; j += gridDim.x * blockDim.x) {
    features(S.op, S.ow, S.on, j, S.d, S.inv_s, f);
    const float bj = wsum > 0.0f ? S.ow[j] / wsum : 0.0f;
    for (int e = 0; e < E; ++e) {
      float z = bf(S.wb, o.ce + e);
      for (int c = 0; c < o.F; ++c) z = fmaf(bf(S.wb, o.We + e * o.F + c), f[c], z);
      if (z > 0.0f) {
        const float g = bj * S.dpool[e];
        for (int c = 0; c < o.F; ++c) atomicAdd(&acc[e * o.F + c], g * f[c]);
        atomicAdd(&acc[E * o.F + e], g);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < E * o.F; k += blockDim.x) atomicAdd(&S.grad[o.We + k], acc[k]);
  for (int k = threadIdx.x; k < E; k += blockDim.x) atomicAdd(&S.grad[o.ce + k], acc[E * o.F + k]);
}

// Shared memory of the tile kernel (floats).
struct TileMem {
  int W1, b1, W2, b2, w3, h0, h1, h1b, h2, dh1, h1T, dh2b, dh2T, outv, dout, P, dW1, db1, db2, dw3, misc, total;
};

__host__ __device__ inline TileMem tile_mem(int D0, int train) {
  TileMem m;
  int k = 0;
  m.W1 = k; k += H * D0;
  m.b1 = k; k += H;
  m.W2 = k; k += H * HB / 2;        // W2 in BF16 (exact), rows of HB
  m.b2 = k; k += H;
  m.w3 = k; k += H;
  m.h0 = k; k += TP * D0;
  m.h1 = k; k += TP * H;
  m.h1b = k; k += 3 * TP * HB / 2;   // h1 as three BF16 parts (hi, mid, lo), TP rows of HB
  m.h2 = k; k += TP * H;
  m.dh1 = k; k += train ? TP * H : 0;
  m.h1T = k; k += train ? 2 * H * PB / 2 : 0;    // h1 (hi, mid) point-contiguous: [part][unit][point]
  m.dh2b = k; k += train ? 2 * TP * HB / 2 : 0;  // dh2 (hi, mid): [part][point][unit]
  m.dh2T = k; k += train ? 2 * H * PB / 2 : 0;   // dh2 (hi, mid) point-contiguous
  m.outv = k; k += TP * 4;
  m.dout = k; k += TP;
  m.P = k; k += E;
  m.dW1 = k; k += train ? H * D0 : 0;
  m.db1 = k; k += train ? H : 0;
  m.db2 = k; k += train ? H : 0;
  m.dw3 = k; k += train ? H : 0;
  m.misc = k; k += 8 + E;
  m.total = k;
  return m;
}

// ---------------------------------------------------------------------------
// Tensor-core tiles (mma.sync m16n8k16, BF16 operands, FP32 accumulation).
// Fragment ownership follows the PTX definition of the shape: with g = lane / 4
// and q = lane % 4, A (16 x 16, row-major) registers hold (g, 2q..2q+1),
// (g + 8, 2q..), (g, 2q + 8..), (g + 8, 2q + 8..); B (16 x 8, column-major)
// holds rows 2q..2q+1 and 2q + 8..2q + 9 of column g; C holds (g, 2q..2q+1) and
// (g + 8, 2q..2q+1).  An FP32 activation x enters as three BF16 parts
// hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid), whose sum carries
// its 24 significant bits; the weights are BF16 already, so every product is
// exact and the three MMAs give the layer to FP32 accumulation accuracy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  const float r1 = __fsub_rn(x, __bfloat162float(hi));
  mid = __float2bfloat16_rn(r1);
  lo = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(mid)));
}

// Forward (and for TRAIN the backward) of tiles of TP points; persistent
// blocks take tiles round-robin and keep their weight gradients in shared
// memory until the end.
template <bool TRAIN>
__global__ void __launch_bounds__(NT) k_mlp_tile(Side S) {
  extern __shared__ __align__(16) float sm[];
  const Off o = offsets(S.d);
  const TileMem M = tile_mem(o.D0, TRAIN);
  const int t = threadIdx.x;
  // weights into shared memory (FP32 from the BF16 copy)
  for (int k = t; k < H * o.D0; k += NT) sm[M.W1 + k] = bf(S.wb, o.W1 + k);
  __nv_bfloat16* w2s = reinterpret_cast<__nv_bfloat16*>(sm + M.W2);
  for (int k = t; k < H * H; k += NT) w2s[(k / H) * HB + (k % H)] = S.wb[o.W2 + k];
  for (int k = t; k < H; k += NT) {
    sm[M.b1 + k] = bf(S.wb, o.b1 + k);
    sm[M.b2 + k] = bf(S.wb, o.b2 + k);
    sm[M.w3 + k] = bf(S.wb, o.w3 + k);
  }
  const float wsum = S.pool[E];
  for (int e = t; e < E; e += NT) sm[M.P + e] = wsum > 0.0f ? S.pool[e] / wsum : 0.0f;
  if (TRAIN) {
    for (int k = t; k < H * o.D0; k += NT) sm[M.dW1 + k] = 0.0f;
    for (int k = t; k < H; k += NT) { sm[M.db1 + k] = 0.0f; sm[M.db2 + k] = 0.0f; sm[M.dw3 + k] = 0.0f; }
    if (t < 8 + E) sm[M.misc + t] = 0.0f;   // [0] db3, [1] loss, [8..] dpool
  }
  const float b3 = bf(S.wb, o.b3);
  // the self side's total weight over points with a finite target (loss normaliser)
  float wtot = 0.0f;
  if (TRAIN) wtot = S.pool[E + 1];
  const int hh = t & (H - 1), g = t >> 7;   // hidden unit, point half
  const int warp = t >> 5, lane = t & 31, gq = lane >> 2, tq = lane & 3;
  // W2 as MMA B fragments, kept in registers for every tile: warp w computes
  // output units [16 w, 16 w + 16) (two n-tiles of 8) over the 8 k-steps.
  // Read from the shared BF16 copy (rows of HB, an even stride, so every pair
  // is 4-byte aligned; a side's weights in global memory may start at an odd
  // BF16 offset).
  __syncthreads();
  uint32_t Bw[H / 16][2][2];
#pragma unroll
  for (int ks = 0; ks < H / 16; ++ks)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int n = 16 * warp + 8 * nt + gq, k = 16 * ks + 2 * tq;
      Bw[ks][nt][0] = *reinterpret_cast<const uint32_t*>(w2s + n * HB + k);
      Bw[ks][nt][1] = *reinterpret_cast<const uint32_t*>(w2s + n * HB + k + 8);
    }
  // TRAIN: W2 as the B operand of dh1 = dh2 W2 (B element (j, k) = W2[j][k],
  // two units j a register), and the warp's 16 rows of dW2 in registers
  uint32_t BwT[TRAIN ? H / 16 : 1][2][2];
  float dw2[TRAIN ? H / 8 : 1][4];
  if (TRAIN) {
#pragma unroll
    for (int ks = 0; ks < H / 16; ++ks)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int k = 16 * warp + 8 * nt + gq, j = 16 * ks + 2 * tq;
        const auto pk = [&](int jj) {
          return (uint32_t)__bfloat16_as_ushort(w2s[jj * HB + k]) |
                 ((uint32_t)__bfloat16_as_ushort(w2s[(jj + 1) * HB + k]) << 16);
        };
        BwT[ks][nt][0] = pk(j);
        BwT[ks][nt][1] = pk(j + 8);
      }
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) dw2[nt][0] = dw2[nt][1] = dw2[nt][2] = dw2[nt][3] = 0.0f;
  }
  __nv_bfloat16* h1b = reinterpret_cast<__nv_bfloat16*>(sm + M.h1b);
  __nv_bfloat16* h1T = reinterpret_cast<__nv_bfloat16*>(sm + M.h1T);
  __nv_bfloat16* dh2b = reinterpret_cast<__nv_bfloat16*>(sm + M.dh2b);
  __nv_bfloat16* dh2T = reinterpret_cast<__nv_bfloat16*>(sm + M.dh2T);
  const int ntiles = (S.sn + TP - 1) / TP;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int p0 = tile * TP;
    __syncthreads();
    // h0 = [f_i, P]
    for (int k = t; k < TP * o.D0; k += NT) {
      const int p = k / o.D0, c = k % o.D0, i = p0 + p;
      float v = 0.0f;
      if (i < S.sn) {
        if (c < S.d) v = S.sp[(size_t)i * S.d + c] * S.inv_s;
        else if (c == S.d) v = (float)S.sn * S.sw[i];
        else v = sm[M.P + (c - o.F)];
      }
      sm[M.h0 + k] = v;
    }
    __syncthreads();
    // h1 = relu(W1 h0 + b1): thread (hh, g) for points g, g+2, ...
    {
      float acc[TP / 2];
#pragma unroll
      for (int q = 0; q < TP / 2; ++q) acc[q] = sm[M.b1 + hh];
      for (int c = 0; c < o.D0; ++c) {
        const float w = sm[M.W1 + hh * o.D0 + c];
#pragma unroll
        for (int q = 0; q < TP / 2; ++q) acc[q] = fmaf(w, sm[M.h0 + (2 * q + g) * o.D0 + c], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < TP / 2; ++q) {
        const int p = 2 * q + g;
        const float v = fmaxf(acc[q], 0.0f);
        sm[M.h1 + p * H + hh] = v;
        __nv_bfloat16 hi, mid, lo;
        split3(v, hi, mid, lo);
        h1b[(0 * TP + p) * HB + hh] = hi;
        h1b[(1 * TP + p) * HB + hh] = mid;
        h1b[(2 * TP + p) * HB + hh] = lo;
        if (TRAIN) {
          h1T[(0 * H + hh) * PB + p] = hi;
          h1T[(1 * H + hh) * PB + p] = mid;
        }
      }
    }
    __syncthreads();
    // h2 = relu(W2 h1 + b2) on the tensor cores: the tile's 32 points are two
    // m-tiles; each of the three parts of h1 meets the warp's W2 fragments
    {
      float acc[2][2][4];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int n = 16 * warp + 8 * nt + 2 * tq;
        const float c0 = sm[M.b2 + n], c1 = sm[M.b2 + n + 1];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          acc[mt][nt][0] = c0; acc[mt][nt][1] = c1; acc[mt][nt][2] = c0; acc[mt][nt][3] = c1;
        }
      }
#pragma unroll
      for (int ks = 0; ks < H / 16; ++ks)
#pragma unroll
        for (int part = 0; part < 3; ++part)
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            const __nv_bfloat16* r0 = h1b + (part * TP + 16 * mt + gq) * HB + 16 * ks + 2 * tq;
            const __nv_bfloat16* r8 = r0 + 8 * HB;
            const uint32_t a[4] = {*reinterpret_cast<const uint32_t*>(r0), *reinterpret_cast<const uint32_t*>(r8),
                                   *reinterpret_cast<const uint32_t*>(r0 + 8), *reinterpret_cast<const uint32_t*>(r8 + 8)};
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_bf16(acc[mt][nt], a, Bw[ks][nt][0], Bw[ks][nt][1]);
          }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int p = 16 * mt + gq, n = 16 * warp + 8 * nt + 2 * tq;
          sm[M.h2 + p * H + n] = fmaxf(acc[mt][nt][0], 0.0f);
          sm[M.h2 + p * H + n + 1] = fmaxf(acc[mt][nt][1], 0.0f);
          sm[M.h2 + (p + 8) * H + n] = fmaxf(acc[mt][nt][2], 0.0f);
          sm[M.h2 + (p + 8) * H + n + 1] = fmaxf(acc[mt][nt][3], 0.0f);
        }
    }
    __syncthreads();
    // out = w3 . h2 + b3: partial sums over hidden units per warp (warps 0-3: g = 0, warps 4-7: g = 1)
    {
#pragma unroll
      for (int q = 0; q < TP / 2; ++q) {
        const int p = 2 * q + g;
        float v = sm[M.w3 + hh] * sm[M.h2 + p * H + hh];
        v = warp_sum(v);
        if (lane == 0) sm[M.outv + p * 4 + (warp & 3)] = v;
      }
    }
    __syncthreads();
    if (t < TP) {
      const int i = p0 + t;
      const float out = b3 + sm[M.outv + t * 4] + sm[M.outv + t * 4 + 1] + sm[M.outv + t * 4 + 2] +
                        sm[M.outv + t * 4 + 3];
      float dout = 0.0f;
      if (i < S.sn) {
        if (!TRAIN) S.out[i] = out;
        else {
          const float tg = S.target[i];
          if (isfinite(tg) && wtot > 0.0f) {
            const float wi = S.sw[i] / wtot;
            const float r = out - tg;
            dout = 2.0f * wi * r * S.inv_eps2;
            atomicAdd(&sm[M.misc + 1], wi * r * r * S.inv_eps2);
          }
        }
      }
      if (TRAIN) {
        sm[M.dout + t] = dout;
        atomicAdd(&sm[M.misc + 0], dout);
      }
    }
    if (!TRAIN) continue;
    __syncthreads();
    // dw3 += sum_p dout_p h2_p ; dh2 = dout w3 [h2 > 0] (in place of h2 after use) ; db2
    {
      float s3 = 0.0f, s2 = 0.0f;
#pragma unroll
      for (int q = 0; q < TP / 2; ++q) {
        const int p = 2 * q + g;
        const float h = sm[M.h2 + p * H + hh];
        const float dp = sm[M.dout + p];
        s3 += dp * h;
        const float d2 = h > 0.0f ? dp * sm[M.w3 + hh] : 0.0f;
        sm[M.h2 + p * H + hh] = d2;
        const __nv_bfloat16 dhi = __float2bfloat16_rn(d2);
        const __nv_bfloat16 dmid = __float2bfloat16_rn(__fsub_rn(d2, __bfloat162float(dhi)));
        dh2b[(0 * TP + p) * HB + hh] = dhi;
        dh2b[(1 * TP + p) * HB + hh] = dmid;
        dh2T[(0 * H + hh) * PB + p] = dhi;
        dh2T[(1 * H + hh) * PB + p] = dmid;
        s2 += d2;
      }
      atomicAdd(&sm[M.dw3 + hh], s3);
      atomicAdd(&sm[M.db2 + hh], s2);
    }
    __syncthreads();
    // dW2[hh][k] += sum_p dh2[p][hh] h1[p][k] on the tensor cores, a contraction
    // over the tile's 32 points: warp w owns rows hh of [16 w, 16 w + 16) in
    // registers (dw2) for every tile; both operands enter as two BF16 parts
    // (hi hi + hi mid + mid hi: relative error near 2^-16)
#pragma unroll
    for (int ks = 0; ks < TP / 16; ++ks) {
      uint32_t a[2][4];
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        const __nv_bfloat16* r0 = dh2T + (part * H + 16 * warp + gq) * PB + 16 * ks + 2 * tq;
        const __nv_bfloat16* r8 = r0 + 8 * PB;
        a[part][0] = *reinterpret_cast<const uint32_t*>(r0);
        a[part][1] = *reinterpret_cast<const uint32_t*>(r8);
        a[part][2] = *reinterpret_cast<const uint32_t*>(r0 + 8);
        a[part][3] = *reinterpret_cast<const uint32_t*>(r8 + 8);
      }
#pragma unroll
      for (int nt = 0; nt < H / 8; ++nt) {
        uint32_t bq[2][2];
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const __nv_bfloat16* q0 = h1T + (part * H + 8 * nt + gq) * PB + 16 * ks + 2 * tq;
          bq[part][0] = *reinterpret_cast<const uint32_t*>(q0);
          bq[part][1] = *reinterpret_cast<const uint32_t*>(q0 + 8);
        }
        mma_bf16(dw2[nt], a[0], bq[0][0], bq[0][1]);
        mma_bf16(dw2[nt], a[0], bq[1][0], bq[1][1]);
        mma_bf16(dw2[nt], a[1], bq[0][0], bq[0][1]);
      }
    }
    // dh1[p][k] = [h1 > 0] sum_j dh2[p][j] W2[j][k] on the tensor cores: warp w
    // computes units k of [16 w, 16 w + 16) for the tile's two m-tiles of points
    {
      float acc[2][2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < H / 16; ++ks)
#pragma unroll
        for (int part = 0; part < 2; ++part)
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            const __nv_bfloat16* r0 = dh2b + (part * TP + 16 * mt + gq) * HB + 16 * ks + 2 * tq;
            const __nv_bfloat16* r8 = r0 + 8 * HB;
            const uint32_t a[4] = {*reinterpret_cast<const uint32_t*>(r0), *reinterpret_cast<const uint32_t*>(r8),
                                   *reinterpret_cast<const uint32_t*>(r0 + 8), *reinterpret_cast<const uint32_t*>(r8 + 8)};
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_bf16(acc[mt][nt], a, BwT[ks][nt][0], BwT[ks][nt][1]);
          }
      float s1[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};   // [nt][unit k or k + 1]: this thread's points
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int p = 16 * mt + gq, k = 16 * warp + 8 * nt + 2 * tq;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int pp = p + (e >> 1) * 8, kk = k + (e & 1);
            const float d1 = sm[M.h1 + pp * H + kk] > 0.0f ? acc[mt][nt][e] : 0.0f;
            sm[M.dh1 + pp * H + kk] = d1;
            s1[nt][e & 1] += d1;
          }
        }
      // db1: the eight lanes of a column pair (same q) hold the other points
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          float v = s1[nt][e];
          v += __shfl_xor_sync(0xffffffffu, v, 4);
          v += __shfl_xor_sync(0xffffffffu, v, 8);
          v += __shfl_xor_sync(0xffffffffu, v, 16);
          if (gq == 0) atomicAdd(&sm[M.db1 + 16 * warp + 8 * nt + 2 * tq + e], v);
        }
    }
    __syncthreads();
    // dW1[k][c] += sum_p dh1[p][k] h0[p][c]; dP[e] += sum_p sum_k W1[k][F+e] dh1[p][k]
    for (int idx = t; idx < H * o.D0; idx += NT) {
      const int k = idx / o.D0, c = idx % o.D0;
      float a = 0.0f;
#pragma unroll 4
      for (int p = 0; p < TP; ++p) a = fmaf(sm[M.dh1 + p * H + k], sm[M.h0 + p * o.D0 + c], a);
      sm[M.dW1 + idx] += a;
    }
    if (t < E * 8) {
      const int e = t >> 3, part = t & 7;   // 8 threads per pooled dimension
      float a = 0.0f;
      for (int k = part; k < H; k += 8) {
        const float w = sm[M.W1 + k * o.D0 + o.F + e];
        float s = 0.0f;
        for (int p = 0; p < TP; ++p) s += sm[M.dh1 + p * H + k];
        a = fmaf(w, s, a);
      }
      atomicAdd(&sm[M.misc + 8 + e], a);
    }
  }
  if (!TRAIN) return;
  __syncthreads();
  for (int k = t; k < H * o.D0; k += NT) atomicAdd(&S.grad[o.W1 + k], sm[M.dW1 + k]);
#pragma unroll
  for (int nt = 0; nt < H / 8; ++nt) {   // this warp's rows of dW2, from registers
    const int hr = 16 * warp + gq, k = 8 * nt + 2 * tq;
    atomicAdd(&S.grad[o.W2 + hr * H + k], dw2[nt][0]);
    atomicAdd(&S.grad[o.W2 + hr * H + k + 1], dw2[nt][1]);
    atomicAdd(&S.grad[o.W2 + (hr + 8) * H + k], dw2[nt][2]);
    atomicAdd(&S.grad[o.W2 + (hr + 8) * H + k + 1], dw2[nt][3]);
  }
  for (int k = t; k < H; k += NT) {
    atomicAdd(&S.grad[o.b1 + k], sm[M.db1 + k]);
    atomicAdd(&S.grad[o.b2 + k], sm[M.db2 + k]);
    atomicAdd(&S.grad[o.w3 + k], sm[M.dw3 + k]);
  }
  if (t == 0) {
    atomicAdd(&S.grad[o.b3], sm[M.misc + 0]);
    atomicAdd(S.loss, sm[M.misc + 1]);
  }
  for (int e = t; e < E; e += NT) atomicAdd(&S.dpool[e], sm[M.misc + 8 + e]);
}

// total weight of the self side over points with a finite target
__global__ void k_target_weight(Side S) {
  float s = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.sn; i += gridDim.x * blockDim.x)
    if (isfinite(S.target[i])) s += S.sw[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(&S.pool[E + 1], s);
}

// Gauge fix: c = (sum b beta - sum a alpha) / (sum a + sum b) over finite
// entries; alpha += c, beta -= c.
__global__ void k_gauge_sums(const float* a, const float* al, int n, const float* b, const float* be, int m,
                             double* acc) {
  double s[4] = {0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (isfinite(al[i])) { s[0] += (double)a[i] * al[i]; s[1] += a[i]; }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    if (isfinite(be[j])) { s[2] += (double)b[j] * be[j]; s[3] += b[j]; }
  for (int k = 0; k < 4; ++k) {
    const double v = warp_sum(s[k]);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[k], v);
  }
}

__global__ void k_gauge_apply(float* al, int n, float* be, int m, const double* acc) {
  const double c = (acc[2] - acc[0]) / (acc[1] + acc[3]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (isfinite(al[i])) al[i] = (float)((double)al[i] + c);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    if (isfinite(be[j])) be[j] = (float)((double)be[j] - c);
}

// Adam on the FP32 master weights, then the BF16 copy.
__global__ void k_adam(float* w, __nv_bfloat16* wb, float* m1, float* m2, const float* g, int count, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float a = b1 * m1[k] + (1.0f - b1) * gk;
    const float v = b2 * m2[k] + (1.0f - b2) * gk * gk;
    m1[k] = a;
    m2[k] = v;
    const float x = w[k] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    w[k] = x;
    wb[k] = __float2bfloat16_rn(x);
  }
}

__global__ void k_to_bf16(const float* w, __nv_bfloat16* wb, int count) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x)
    wb[k] = __float2bfloat16_rn(w[k]);
}

// He-uniform initialisation from the Philox stream (key = seed, counter = (k, 0xC0FFEE, 0, 0)).
__global__ void k_init(float* w, int d, uint64_t seed) {
  const Off o = offsets(d);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 2 * o.size; k += gridDim.x * blockDim.x) {
    const int r = k % o.size;
    float fan = 0.0f;
    if (r < o.ce) fan = (float)o.F;
    else if (r >= o.W1 && r < o.b1) fan = (float)o.D0;
    else if (r >= o.W2 && r < o.b2) fan = (float)H;
    else if (r >= o.w3 && r < o.b3) fan = (float)H;
    float v = 0.0f;
    if (fan > 0.0f) {
      const uint4 q = philox4x32_10(make_uint4((uint32_t)k, 0xC0FFEEu, 0u, 0u), (uint32_t)seed, (uint32_t)(seed >> 32));
      const float u = (float)(q.x >> 8) * 5.9604644775390625e-08f;   // [0, 1)
      const float lim = sqrtf(6.0f / fan) * (r >= o.w3 ? 0.1f : 1.0f);
      v = (2.0f * u - 1.0f) * lim;
    }
    w[k] = v;
  }
}

Side make_side(const float* sp, const float* sw, int sn, const float* op, const float* ow, int on, int d,
               float inv_s, float eps, const float* target, float* out, const __nv_bfloat16* wb, const float* wf,
               float* grad, float* pool, float* dpool, float* loss) {
  Side S;
  S.sp = sp; S.sw = sw; S.sn = sn; S.op = op; S.ow = ow; S.on = on;
  S.target = target; S.out = out; S.wb = wb; S.wf = wf; S.grad = grad; S.pool = pool; S.dpool = dpool;
  S.loss = loss; S.d = d; S.inv_s = inv_s; S.inv_eps2 = (float)(1.0 / ((double)eps * eps));
  return S;
}

int nsm_now() {
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  return nsm;
}

template <bool TRAIN>
sps_status tile(const Side& S, cudaStream_t st) {
  const Off o = offsets(S.d);
  const size_t smem = sizeof(float) * (size_t)tile_mem(o.D0, TRAIN).total;
  auto fn = k_mlp_tile<TRAIN>;
  SPS_TRY(cuda_fail(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "mlp shared memory"));
  const int ntiles = (S.sn + TP - 1) / TP;
  const int grid = std::max(1, std::min(ntiles, nsm_now()));
  fn<<<grid, NT, smem, st>>>(S);
  return cuda_fail(cudaGetLastError(), "mlp tile");
}

int grid_pts(int n) { return std::max(1, std::min(4 * 152, (n + 255) / 256)); }

// workspace: per side pool[E + 2], dpool[E], loss, gauge acc (4 doubles)
struct MlpWs {
  float* pool[2];
  float* dpool[2];
  float* loss;
  double* gauge;
};
constexpr size_t kWsBytes = 4096;

MlpWs ws_split(void* ws) {
  char* p = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  MlpWs W;
  float* f = (float*)p;
  W.pool[0] = f; W.pool[1] = f + 32;
  W.dpool[0] = f + 64; W.dpool[1] = f + 96;
  W.loss = f + 128;
  W.gauge = (double*)(p + 1024);
  return W;
}

sps_status check_inputs(const sps_mlp_instance* I) {
  if (!I || !I->x || !I->y || !I->a || !I->b) { set_error("null warm-start instance"); return SPS_ERR_INVALID_ARG; }
  if (I->n < 1 || I->m < 1 || I->d < 1 || I->d > 16) { set_error("warm start needs n, m >= 1 and 1 <= d <= 16"); return SPS_ERR_INVALID_ARG; }
  if (!(I->cost_max > 0.0) || !isfinite(I->cost_max)) { set_error("cost_max must be > 0"); return SPS_ERR_INVALID_ARG; }
  return SPS_OK;
}

}  // namespace mlp
}  // namespace sps

using namespace sps;
using namespace sps::mlp;

extern "C" {

size_t sps_mlp_param_count(int32_t d) {
  if (d < 1 || d > 16) return 0;
  return 2 * (size_t)offsets(d).size;
}

size_t sps_mlp_workspace_bytes(void) { return kWsBytes; }

sps_status sps_mlp_init(float* params, void* params_bf16, int32_t d, uint64_t seed, sps_stream stream) {
  if (!params || !params_bf16 || d < 1 || d > 16) { set_error("bad warm-start init arguments"); return SPS_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const int count = 2 * offsets(d).size;
  k_init<<<grid_pts(count), 256, 0, st>>>(params, d, seed);
  k_to_bf16<<<grid_pts(count), 256, 0, st>>>(params, (__nv_bfloat16*)params_bf16, count);
  return cuda_fail(cudaGetLastError(), "mlp init");
}

sps_status sps_mlp_sync_bf16(const float* params, void* params_bf16, int32_t d, sps_stream stream) {
  if (!params || !params_bf16 || d < 1 || d > 16) { set_error("bad arguments"); return SPS_ERR_INVALID_ARG; }
  const int count = 2 * offsets(d).size;
  k_to_bf16<<<grid_pts(count), 256, 0, (cudaStream_t)stream>>>(params, (__nv_bfloat16*)params_bf16, count);
  return cuda_fail(cudaGetLastError(), "mlp bf16 copy");
}

sps_status sps_cost_max(const float* x, int32_t n, const float* y, int32_t m, int32_t d, double* cost_max,
                        void* ws, sps_stream stream) {
  if (!x || !y || !cost_max || !ws || n < 1 || m < 1 || d < 1 || d > 16) { set_error("bad cost_max arguments"); return SPS_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  SketchScalars* sc = (SketchScalars*)(((uintptr_t)ws + 2048 + 255) & ~(uintptr_t)255);
  SPS_TRY(cuda_fail(cudaMemsetAsync(sc, 0, sizeof(SketchScalars), st), "memset"));
  SPS_TRY(launch_cost_max_points(x, n, y, m, d, sc, st));   // the sketch's own tiled kernel
  float f = 0.0f;
  SPS_TRY(cuda_fail(cudaMemcpyAsync(&f, &sc->dmax32, sizeof(f), cudaMemcpyDeviceToHost, st), "read back"));
  SPS_TRY(cuda_fail(cudaStreamSynchronize(st), "synchronize"));
  *cost_max = (double)f;
  return SPS_OK;
}

// The same maximum with a caller workspace sized for the pruned search of the
// solver's sketch (sps_costmax.cu): above 1e8 pairs only the cell pairs (d <= 4)
// or radial candidate sets (d > 4) that can reach the maximum are evaluated,
// the full sweep running only when the candidate list overflowed.
constexpr double kPrunePairs = 1e8;
constexpr size_t kCmScalBytes = 4096;   // SketchScalars at offset 0, then the scratch
static_assert(sizeof(SketchScalars) <= kCmScalBytes, "cost max scalars");

size_t sps_cost_max_workspace_bytes(int32_t n, int32_t m, int32_t d) {
  if (n < 1 || m < 1 || d < 1 || d > 16) return 0;
  const bool prune = (double)n * (double)m > kPrunePairs;
  return 256 + kCmScalBytes + (prune ? cost_max_scratch_bytes(n, m, d) : 0);
}

sps_status sps_cost_max_ws(const float* x, int32_t n, const float* y, int32_t m, int32_t d, double* cost_max,
                           void* ws, size_t ws_bytes, sps_stream stream) {
  if (!x || !y || !cost_max || !ws || n < 1 || m < 1 || d < 1 || d > 16) { set_error("bad cost_max arguments"); return SPS_ERR_INVALID_ARG; }
  const size_t need = sps_cost_max_workspace_bytes(n, m, d);
  if (ws_bytes < need) { set_error("cost_max workspace too small: %zu < %zu", ws_bytes, need); return SPS_ERR_WORKSPACE; }
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  SketchScalars* sc = (SketchScalars*)base;
  SPS_TRY(cuda_fail(cudaMemsetAsync(sc, 0, sizeof(SketchScalars), st), "memset"));
  bool full = true;
  if ((double)n * (double)m > kPrunePairs) {
    const int* overflow = nullptr;
    SPS_TRY(launch_cost_max_pruned(x, y, n, m, d, sc, base + kCmScalBytes, &overflow, st));
    int ov = 1;
    SPS_TRY(cuda_fail(cudaMemcpyAsync(&ov, overflow, sizeof(int), cudaMemcpyDeviceToHost, st), "read back"));
    SPS_TRY(cuda_fail(cudaStreamSynchronize(st), "synchronize"));
    full = ov != 0;
  }
  if (full) SPS_TRY(launch_cost_max_points(x, n, y, m, d, sc, st));
  float f = 0.0f;
  SPS_TRY(cuda_fail(cudaMemcpyAsync(&f, &sc->dmax32, sizeof(f), cudaMemcpyDeviceToHost, st), "read back"));
  SPS_TRY(cuda_fail(cudaStreamSynchronize(st), "synchronize"));
  *cost_max = (double)f;
  return SPS_OK;
}

sps_status sps_mlp_infer(const void* params_bf16, const sps_mlp_instance* I, float* alpha_out, float* beta_out,
                         void* ws, sps_stream stream) {
  SPS_TRY(check_inputs(I));
  if (!params_bf16 || !alpha_out || !beta_out || !ws) { set_error("null argument"); return SPS_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const Off o = offsets(I->d);
  const __nv_bfloat16* wb = (const __nv_bfloat16*)params_bf16;
  MlpWs W = ws_split(ws);
  SPS_TRY(cuda_fail(cudaMemsetAsync(W.pool[0], 0, 1024, st), "memset"));
  const float inv_s = (float)(1.0 / sqrt(I->cost_max));
  Side A = make_side(I->x, I->a, I->n, I->y, I->b, I->m, I->d, inv_s, 1.0f, nullptr, alpha_out, wb, nullptr, nullptr,
                     W.pool[0], W.dpool[0], W.loss);
  Side B = make_side(I->y, I->b, I->m, I->x, I->a, I->n, I->d, inv_s, 1.0f, nullptr, beta_out, wb + o.size, nullptr,
                     nullptr, W.pool[1], W.dpool[1], W.loss);
  k_pool_fwd<<<grid_pts(I->m), 256, 0, st>>>(A);
  k_pool_fwd<<<grid_pts(I->n), 256, 0, st>>>(B);
  SPS_TRY(tile<false>(A, st));
  SPS_TRY(tile<false>(B, st));
  add_launches(4);
  return cuda_fail(cudaGetLastError(), "mlp inference");
}

sps_status sps_mlp_gauge_fix(const sps_mlp_instance* I, float* alpha, float* beta, void* ws, sps_stream stream) {
  SPS_TRY(check_inputs(I));
  if (!alpha || !beta || !ws) { set_error("null argument"); return SPS_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  MlpWs W = ws_split(ws);
  SPS_TRY(cuda_fail(cudaMemsetAsync(W.gauge, 0, 4 * sizeof(double), st), "memset"));
  const int g = grid_pts(std::max(I->n, I->m));
  k_gauge_sums<<<g, 256, 0, st>>>(I->a, alpha, I->n, I->b, beta, I->m, W.gauge);
  k_gauge_apply<<<g, 256, 0, st>>>(alpha, I->n, beta, I->m, W.gauge);
  return cuda_fail(cudaGetLastError(), "gauge fix");
}

sps_status sps_mlp_grad(const float* params, const void* params_bf16, const sps_mlp_instance* I,
                        const float* alpha_target, const float* beta_target, float* grad, float* loss_out,
                        void* ws, sps_stream stream) {
  SPS_TRY(check_inputs(I));
  if (!params || !params_bf16 || !alpha_target || !beta_target || !grad || !ws) { set_error("null argument"); return SPS_ERR_INVALID_ARG; }
  if (!(I->eps > 0.0) || !isfinite(I->eps)) { set_error("eps must be finite and > 0"); return SPS_ERR_INVALID_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const Off o = offsets(I->d);
  const __nv_bfloat16* wb = (const __nv_bfloat16*)params_bf16;
  MlpWs W = ws_split(ws);
  SPS_TRY(cuda_fail(cudaMemsetAsync(W.pool[0], 0, 1024, st), "memset"));
  SPS_TRY(cuda_fail(cudaMemsetAsync(grad, 0, sizeof(float) * 2 * (size_t)o.size, st), "memset grad"));
  const float inv_s = (float)(1.0 / sqrt(I->cost_max));
  Side A = make_side(I->x, I->a, I->n, I->y, I->b, I->m, I->d, inv_s, (float)I->eps, alpha_target, nullptr, wb,
                     params, grad, W.pool[0], W.dpool[0], W.loss);
  Side B = make_side(I->y, I->b, I->m, I->x, I->a, I->n, I->d, inv_s, (float)I->eps, beta_target, nullptr,
                     wb + o.size, params + o.size, grad + o.size, W.pool[1], W.dpool[1], W.loss);
  k_pool_fwd<<<grid_pts(I->m), 256, 0, st>>>(A);
  k_pool_fwd<<<grid_pts(I->n), 256, 0, st>>>(B);
  k_target_weight<<<grid_pts(I->n), 256, 0, st>>>(A);
  k_target_weight<<<grid_pts(I->m), 256, 0, st>>>(B);
  SPS_TRY(tile<true>(A, st));
  SPS_TRY(tile<true>(B, st));
  k_pool_bwd<<<grid_pts(I->m), 256, 0, st>>>(A);
  k_pool_bwd<<<grid_pts(I->n), 256, 0, st>>>(B);
  add_launches(8);
  if (loss_out) {
    SPS_TRY(cuda_fail(cudaMemcpyAsync(loss_out, W.loss, sizeof(float), cudaMemcpyDeviceToHost, st), "loss"));
    SPS_TRY(cuda_fail(cudaStreamSynchronize(st), "synchronize"));
  }
  return cuda_fail(cudaGetLastError(), "mlp gradient");
}

sps_status sps_mlp_adam(float* params, void* params_bf16, float* m1, float* m2, const float* grad, int32_t d,
                        int32_t step, float lr, float beta1, float beta2, float eps, sps_stream stream) {
  if (!params || !params_bf16 || !m1 || !m2 || !grad || d < 1 || d > 16 || step < 1) { set_error("bad Adam arguments"); return SPS_ERR_INVALID_ARG; }
  // the bias corrections 1 - beta^step must be positive and the denominator sqrt(v) + eps non-zero
  if (!(lr >= 0.0f) || !isfinite(lr) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
      !(eps > 0.0f) || !isfinite(eps)) {
    set_error("Adam needs a finite lr >= 0, 0 <= beta1, beta2 < 1 and a finite eps > 0");
    return SPS_ERR_INVALID_ARG;
  }
  const int count = 2 * offsets(d).size;
  const float c1 = (float)(1.0 - pow((double)beta1, step)), c2 = (float)(1.0 - pow((double)beta2, step));
  k_adam<<<grid_pts(count), 256, 0, (cudaStream_t)stream>>>(params, (__nv_bfloat16*)params_bf16, m1, m2, grad, count,
                                                             lr, beta1, beta2, eps, c1, c2);
  add_launches(1);
  return cuda_fail(cudaGetLastError(), "adam");
}

}  // extern "C"
