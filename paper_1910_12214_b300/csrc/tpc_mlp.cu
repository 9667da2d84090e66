// BF16 MLP surrogate of the space-point correction: training, evaluation and
// inference kernels.
//
// The paper asks for a location-dependent calibration of the cluster positions
// during the online reconstruction (Abstract; online calibration, Sec. 3).  The
// plain method is a per-sector trilinear grid (k_correct_grid).  This file
// replaces the grid by a small network per sector, trained on samples of that
// grid: 3 -> 64 -> 64 -> 3 with SiLU, inputs the measured position normalised to
// [-1, 1]^3 by the grid's bounds, output the correction / 10 cm.  Operands
// (inputs, weights, activations) are BF16 (round to nearest even), sums FP32.
//
//  - k_mlp_grad: forward and backward of one training batch, one CTA per 128
//    samples of a sector, FP32 arithmetic on BF16-rounded operands; per-CTA
//    gradient partials (fixed summation order, so training is deterministic).
//  - k_mlp_adam: sums the partials in a fixed order and takes an Adam step
//    (cosine learning rate) on the FP32 master weights.
//  - k_correct_mlp: inference inside tracking.  A warp handles 16 clusters: the
//    64x64 layer runs on the tensor cores (mma.sync m16n8k16, BF16 inputs, FP32
//    accumulators); the 3-wide layers on the FMA pipes.
//
// Training samples and initial weights come from a counter-based generator
// (splitmix64, Steele, Lea and Flood 2014) keyed by (seed, sector, step, index).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "tpc.h"
#include "tpc_internal.cuh"

namespace {

constexpr int H = 64;
constexpr int OW1 = 0, OB1 = 192, OW2 = 256, OB2 = 4352, OW3 = 4416, OB3 = 4608, NP = 4611;
constexpr int NPP = 4616;     // padded parameter stride per sector
constexpr int TB = 128;       // samples per training CTA
constexpr float OUT_SCALE = 10.0f;

__device__ __forceinline__ uint64_t sm64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// uniform in [0, 1) with 24 bits: exact in FP32
__device__ __forceinline__ float counter_uniform(uint64_t seed, uint64_t a, uint64_t b, uint64_t k) {
  return (float)(sm64(sm64(sm64(seed + a) + b) + k) >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
// logistic function with the hardware exponential and reciprocal (a few ulp;
// training only: its gradients are compared with the FP64 oracle at 2e-2)
__device__ __forceinline__ float sigm(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }

// SiLU of the deployed network (inference and its residual evaluation):
// z * sigmoid(z) = h + h tanh(h) with h = z / 2 and the hardware tanh (relative
// error about 2^-11, below the BF16 rounding that follows); one special-function
// operation instead of an exponential and a division.  (The BF16x2 form of the
// hardware tanh was measured too coarse: trained-network residual 0.61 cm rms
// instead of 0.02 cm.)
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float silu_fast(float z) {
  const float hz = 0.5f * z;
  return fmaf(hz, tanh_hw(hz), hz);
}
// the same SiLU from h = z / 2
__device__ __forceinline__ float silu_of_half(float hz) { return fmaf(hz, tanh_hw(hz), hz); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = sigm(z);
  return s * (1.0f + z * (1.0f - s));
}

// trilinear (dy, dz) of a sector grid at index-space coordinates t (clamped)
__device__ __forceinline__ float2 grid_at(const float2* G, int nx, int ny, int nz, float tx, float ty, float tz) {
  const float t[3] = {tx, ty, tz};
  const int dims[3] = {nx, ny, nz};
  int lo[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float u = fminf(fmaxf(t[a], 0.0f), (float)(dims[a] - 1));
    int k = (int)floorf(u);
    k = min(max(k, 0), dims[a] - 2);
    lo[a] = k;
    f[a] = u - k;
  }
  const size_t sy = nz, sx = (size_t)ny * nz;
  const float2* g0 = G + lo[0] * sx + lo[1] * sy + lo[2];
  float dy = 0.f, dz = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float2 c = g0[(k >> 2) * sx + ((k >> 1) & 1) * sy + (k & 1)];
    const float w = ((k >> 2) ? f[0] : 1.f - f[0]) * (((k >> 1) & 1) ? f[1] : 1.f - f[1]) * ((k & 1) ? f[2] : 1.f - f[2]);
    dy += w * c.x;
    dz += w * c.y;
  }
  return make_float2(dy, dz);
}

}  // namespace

// ---------------------------------------------------------------------------- training
// Training clock on the device: the step and its Adam scalars, advanced by the
// last block of every step's Adam kernel, so that a CUDA graph of K steps
// replays the next K steps without arguments from the host.
struct MlpClock {
  unsigned long long step, T;
  float lr;                 // base learning rate
  float lr_t, c1, c2;       // cosine-decayed rate and the bias corrections 1 - b^(t+1) of this step
};

__device__ __forceinline__ void clock_scalars(MlpClock* c) {
  const double t = (double)c->step;
  c->lr_t = (float)(c->lr * 0.5 * (1.0 + cos(M_PI * t / (double)c->T)));
  c->c1 = (float)(1.0 - pow(0.9, t + 1.0));
  c->c2 = (float)(1.0 - pow(0.999, t + 1.0));
}

__global__ void k_mlp_clock_set(MlpClock* c, unsigned long long step, unsigned long long T, float lr) {
  c->step = step;
  c->T = T;
  c->lr = lr;
  clock_scalars(c);
}

struct StagedW;

struct MlpTrain {
  const MlpClock* clock;  // the step comes from here when set, else from `step`
  const StagedW* staged;  // [S] the step's weights as the CTAs read them
  float* partial;       // [S][nblk][NPP]
  float* loss;          // [S][nblk]
  const float2* grid;   // [S][nx][ny][nz]
  int nx, ny, nz;
  uint64_t seed, step;
  int batch;            // samples per sector and step (multiple of TB)
};

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// four 8x8 BF16 matrices from shared memory; lanes 8j..8j+7 give the row
// addresses of matrix j.  Plain: lane l receives row l/4, columns 2(l%4) and
// 2(l%4)+1 of each; transposed: rows 2(l%4), 2(l%4)+1 at column l/4.
__device__ __forceinline__ void ldmatrix_x4(uint32_t* r, const void* smem_row) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldmatrix_x4_t(uint32_t* r, const void* smem_row) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// D += A B, m16n8k16, BF16 operands, FP32 accumulators.  Fragments (lane =
// 4 g + q): A rows g and g+8 at columns 2q, 2q+1 and +8; B column g at rows
// 2q, 2q+1 and +8; D rows g and g+8 at columns 2q, 2q+1.
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int TS = 72;  // padded row stride (BF16 elements) of the training tiles: conflict-free ldmatrix

// The weights of one sector as a training CTA reads them: W2 and W2^T as BF16
// tiles with padded rows, the 3-wide layers rounded to BF16 (held as floats),
// the biases FP32.  Staged in global memory once per step (by k_mlp_stage, and
// by the Adam step for the next step) and copied into shared memory by every
// CTA with 16-byte loads.
struct __align__(16) StagedW {
  __nv_bfloat16 w2[H * TS];   // W2 [out j][in i]: B of the forward layer 2
  __nv_bfloat16 w2t[H * TS];  // W2^T [in i][out j]: B of the backward layer 2
  float w1[192], b1[64], b2[64], w3[192], b3[4];
};
static_assert(sizeof(StagedW) % 16 == 0, "staged weights are copied in 16-byte units");

// Shared memory of one training CTA: the staged weights, then the sample tiles
// [sample][column]: A1x and A2x hold the hidden activations with a column of
// ones at 64 (the bias gradients come out of the same products), GZ1 and GZ2
// the gradients of the pre-activations, INx the inputs with a one at 3, GOx the
// output gradients (columns 0..2).
struct __align__(16) TrainSmem : StagedW {
  __nv_bfloat16 a1x[TB * TS], a2x[TB * TS], gz1[TB * TS], gz2[TB * TS];
  __nv_bfloat16 inx[TB * 8], gox[TB * 16];
  float loss[TB / 32];
};

// parameter p of a sector with value v, staged
__device__ __forceinline__ void stage_param(StagedW* W, int p, float v) {
  if (p < OB1) {
    W->w1[p - OW1] = bf(v);
  } else if (p < OW2) {
    W->b1[p - OB1] = v;
  } else if (p < OB2) {
    const int r = (p - OW2) / H, c = (p - OW2) % H;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    W->w2[r * TS + c] = h;
    W->w2t[c * TS + r] = h;
  } else if (p < OW3) {
    W->b2[p - OB2] = v;
  } else if (p < OB3) {
    W->w3[p - OW3] = bf(v);
  } else {
    W->b3[p - OB3] = v;
  }
}

// every weight of a sector staged from its FP32 master M, and the padding
__global__ void __launch_bounds__(256) k_mlp_stage(const float* master, StagedW* staged) {
  const float* M = master + (size_t)blockIdx.x * NPP;
  StagedW* W = staged + blockIdx.x;
  for (int p = threadIdx.x; p < NP; p += blockDim.x) stage_param(W, p, M[p]);
  for (int p = threadIdx.x; p < H * (TS - H); p += blockDim.x) {
    const int r = p / (TS - H), c = H + p % (TS - H);
    W->w2[r * TS + c] = __float2bfloat16_rn(0.0f);
    W->w2t[r * TS + c] = __float2bfloat16_rn(0.0f);
  }
  if (threadIdx.x == 0) W->b3[3] = 0.0f;
}

// One CTA per TB = 128 samples of a sector (four warps of 32 samples, two
// 16-sample tiles each).  Forward and backward of a tile run on the tensor
// cores with the fragments kept in registers (each layer's accumulators,
// after SiLU and BF16 rounding, become the next product's A fragments):
//   z1 = W1 in + b1 (K padded 3 -> 16), a1 = bf(silu(z1));
//   z2 = W2 a1 + b2, a2 = bf(silu(z2)); o = W3 a2 + b3 (N padded 3 -> 8);
//   go = 2 (o - target) / batch; ga2 = W3^T go (three FMAs per element);
//   gz2 = ga2 silu'(z2); ga1 = W2^T gz2 (tensor cores); gz1 = ga1 silu'(z1).
// The sums over the CTA's samples are products over the staged tiles:
//   [gW2 | gb2] = gz2^T [a1 | 1], [gW1 | gb1] = gz1^T [in | 1],
//   [gW3 | gb3] = go^T [a2 | 1]  (BF16 operands, FP32 accumulation),
// written to the CTA's partial in a fixed layout (deterministic training).
__global__ void __launch_bounds__(TB) k_mlp_grad(const __grid_constant__ MlpTrain a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int s = blockIdx.y, blk = blockIdx.x, t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5, g = lane >> 2, q = lane & 3;
  {
    const int4* src = reinterpret_cast<const int4*>(a.staged + s);
    int4* dst = reinterpret_cast<int4*>(static_cast<StagedW*>(&S));
    for (int p = t; p < (int)(sizeof(StagedW) / 16); p += TB) dst[p] = __ldg(src + p);
  }
  // the columns beyond the data: ones at 64 (bias column), zeros after
  for (int r = t; r < TB; r += TB) {
    for (int c = H; c < TS; ++c) {
      S.a1x[r * TS + c] = __float2bfloat16_rn(c == H ? 1.0f : 0.0f);
      S.a2x[r * TS + c] = __float2bfloat16_rn(c == H ? 1.0f : 0.0f);
      S.gz1[r * TS + c] = __float2bfloat16_rn(0.0f);
      S.gz2[r * TS + c] = __float2bfloat16_rn(0.0f);
    }
  }
  __syncthreads();
  // per-lane B fragments of layers 1 and 3 (constant over the CTA)
  uint32_t B1[8];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int n = 8 * nt + g;
    B1[nt] = q == 0 ? pack_bf2(S.w1[3 * n], S.w1[3 * n + 1]) : q == 1 ? pack_bf2(S.w1[3 * n + 2], 0.0f) : 0u;
  }
  uint32_t B3[4][2];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int k0 = 16 * ks + 2 * q;
    B3[ks][0] = g < 3 ? pack_bf2(S.w3[64 * g + k0], S.w3[64 * g + k0 + 1]) : 0u;
    B3[ks][1] = g < 3 ? pack_bf2(S.w3[64 * g + k0 + 8], S.w3[64 * g + k0 + 9]) : 0u;
  }
  const float2* G = a.grid + (size_t)s * a.nx * a.ny * a.nz;
  const float inv_batch = 2.0f / (float)a.batch;
  const uint64_t step = a.clock ? a.clock->step : a.step;
  float lsum = 0.f;
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = 32 * warp + 16 * mt;  // first sample (CTA row) of the tile
    // inputs and targets of rows g and g + 8
    float in[2][3], tgt[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t k = (uint64_t)blk * TB + r0 + g + 8 * h;
      float u[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        u[c] = counter_uniform(a.seed, (uint64_t)s, step, 3ull * k + c);
        in[h][c] = bf(2.0f * u[c] - 1.0f);
      }
      const float2 tg = grid_at(G, a.nx, a.ny, a.nz, u[0] * (a.nx - 1), u[1] * (a.ny - 1), u[2] * (a.nz - 1));
      tgt[h][0] = tg.x / OUT_SCALE;
      tgt[h][1] = tg.y / OUT_SCALE;
      if (q == 0) {  // [in | 1] row
        uint32_t* row = reinterpret_cast<uint32_t*>(S.inx + (r0 + g + 8 * h) * 8);
        row[0] = pack_bf2(in[h][0], in[h][1]);
        row[1] = pack_bf2(in[h][2], 1.0f);
        row[2] = 0u;
        row[3] = 0u;
      }
    }
    // layer 1 (K padded 3 -> 16): z1 accumulators, a1 fragments
    uint32_t A1in[4];
    A1in[0] = q == 0 ? pack_bf2(in[0][0], in[0][1]) : q == 1 ? pack_bf2(in[0][2], 0.0f) : 0u;
    A1in[1] = q == 0 ? pack_bf2(in[1][0], in[1][1]) : q == 1 ? pack_bf2(in[1][2], 0.0f) : 0u;
    A1in[2] = 0u;
    A1in[3] = 0u;
    float z1[8][4];
    uint32_t A[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float2 bb = *reinterpret_cast<const float2*>(S.b1 + 8 * nt + 2 * q);
      z1[nt][0] = bb.x;
      z1[nt][1] = bb.y;
      z1[nt][2] = bb.x;
      z1[nt][3] = bb.y;
      mma_bf16(z1[nt], A1in, B1[nt], 0u);
      const float a0 = bf(silu(z1[nt][0])), a1 = bf(silu(z1[nt][1]));
      const float a2 = bf(silu(z1[nt][2])), a3 = bf(silu(z1[nt][3]));
      const int ks = nt >> 1, half = nt & 1;
      A[ks][2 * half] = pack_bf2(a0, a1);
      A[ks][2 * half + 1] = pack_bf2(a2, a3);
      *reinterpret_cast<uint32_t*>(S.a1x + (r0 + g) * TS + 8 * nt + 2 * q) = A[ks][2 * half];
      *reinterpret_cast<uint32_t*>(S.a1x + (r0 + g + 8) * TS + 8 * nt + 2 * q) = A[ks][2 * half + 1];
    }
    // layer 2: z2 accumulators, a2 fragments
    float z2[8][4];
    uint32_t A3[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float2 bb = *reinterpret_cast<const float2*>(S.b2 + 8 * nt + 2 * q);
      z2[nt][0] = bb.x;
      z2[nt][1] = bb.y;
      z2[nt][2] = bb.x;
      z2[nt][3] = bb.y;
#pragma unroll
      for (int ks = 0; ks < 4; ks += 2) {
        uint32_t b4[4];
        const int j = lane >> 3;
        ldmatrix_x4(b4, S.w2 + (8 * nt + (lane & 7)) * TS + 16 * (ks + (j >> 1)) + 8 * (j & 1));
        mma_bf16(z2[nt], A[ks], b4[0], b4[1]);
        mma_bf16(z2[nt], A[ks + 1], b4[2], b4[3]);
      }
      const float a0 = bf(silu(z2[nt][0])), a1 = bf(silu(z2[nt][1]));
      const float a2 = bf(silu(z2[nt][2])), a3 = bf(silu(z2[nt][3]));
      const int ks3 = nt >> 1, half = nt & 1;
      A3[ks3][2 * half] = pack_bf2(a0, a1);
      A3[ks3][2 * half + 1] = pack_bf2(a2, a3);
      *reinterpret_cast<uint32_t*>(S.a2x + (r0 + g) * TS + 8 * nt + 2 * q) = A3[ks3][2 * half];
      *reinterpret_cast<uint32_t*>(S.a2x + (r0 + g + 8) * TS + 8 * nt + 2 * q) = A3[ks3][2 * half + 1];
    }
    // layer 3 (N padded 3 -> 8): outputs at columns 0..2
    float o[4] = {q == 0 ? S.b3[0] : q == 1 ? S.b3[2] : 0.f, q == 0 ? S.b3[1] : 0.f,
                  q == 0 ? S.b3[0] : q == 1 ? S.b3[2] : 0.f, q == 0 ? S.b3[1] : 0.f};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) mma_bf16(o, A3[ks], B3[ks][0], B3[ks][1]);
    // output gradients: lane q = 0 holds outputs 0, 1 (x, dy), lane q = 1 output 2 (dz)
    float go[4] = {0.f, 0.f, 0.f, 0.f};
    if (q == 0) {
      const float r[4] = {o[0], o[1] - tgt[0][0], o[2], o[3] - tgt[1][0]};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        go[e] = inv_batch * r[e];
        lsum += r[e] * r[e];
      }
    } else if (q == 1) {
      const float r0v = o[0] - tgt[0][1], r1v = o[2] - tgt[1][1];
      go[0] = inv_batch * r0v;
      go[2] = inv_batch * r1v;
      lsum += r0v * r0v + r1v * r1v;
    }
    {  // [go] rows: columns 0..2, zeros to 15
      uint32_t* row_g = reinterpret_cast<uint32_t*>(S.gox + (r0 + g) * 16);
      uint32_t* row_h = reinterpret_cast<uint32_t*>(S.gox + (r0 + g + 8) * 16);
      row_g[q] = q < 2 ? pack_bf2(go[0], go[1]) : 0u;
      row_h[q] = q < 2 ? pack_bf2(go[2], go[3]) : 0u;
      row_g[4 + q] = 0u;
      row_h[4 + q] = 0u;
    }
    // the three output gradients of rows g and g + 8 in every lane of the quad
    const int base = lane & ~3;
    const float g0a = __shfl_sync(0xffffffffu, go[0], base), g1a = __shfl_sync(0xffffffffu, go[1], base);
    const float g2a = __shfl_sync(0xffffffffu, go[0], base + 1);
    const float g0b = __shfl_sync(0xffffffffu, go[2], base), g1b = __shfl_sync(0xffffffffu, go[3], base);
    const float g2b = __shfl_sync(0xffffffffu, go[2], base + 1);
    // gz2 = (W3^T go) silu'(z2): fragments of the backward product, and the tile
    uint32_t GZ[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = 8 * nt + 2 * q + (e & 1);
        const float ga = e < 2 ? g0a * S.w3[j] + g1a * S.w3[64 + j] + g2a * S.w3[128 + j]
                               : g0b * S.w3[j] + g1b * S.w3[64 + j] + g2b * S.w3[128 + j];
        v[e] = ga * dsilu(z2[nt][e]);
      }
      const int ks = nt >> 1, half = nt & 1;
      GZ[ks][2 * half] = pack_bf2(v[0], v[1]);
      GZ[ks][2 * half + 1] = pack_bf2(v[2], v[3]);
      *reinterpret_cast<uint32_t*>(S.gz2 + (r0 + g) * TS + 8 * nt + 2 * q) = GZ[ks][2 * half];
      *reinterpret_cast<uint32_t*>(S.gz2 + (r0 + g + 8) * TS + 8 * nt + 2 * q) = GZ[ks][2 * half + 1];
    }
    // ga1 = W2^T gz2 on the tensor cores, gz1 = ga1 silu'(z1)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < 4; ks += 2) {
        uint32_t b4[4];
        const int j = lane >> 3;
        ldmatrix_x4(b4, S.w2t + (8 * nt + (lane & 7)) * TS + 16 * (ks + (j >> 1)) + 8 * (j & 1));
        mma_bf16(d, GZ[ks], b4[0], b4[1]);
        mma_bf16(d, GZ[ks + 1], b4[2], b4[3]);
      }
      const float v0 = d[0] * dsilu(z1[nt][0]), v1 = d[1] * dsilu(z1[nt][1]);
      const float v2 = d[2] * dsilu(z1[nt][2]), v3 = d[3] * dsilu(z1[nt][3]);
      *reinterpret_cast<uint32_t*>(S.gz1 + (r0 + g) * TS + 8 * nt + 2 * q) = pack_bf2(v0, v1);
      *reinterpret_cast<uint32_t*>(S.gz1 + (r0 + g + 8) * TS + 8 * nt + 2 * q) = pack_bf2(v2, v3);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if (lane == 0) S.loss[warp] = lsum;
  __syncthreads();
  float* P = a.partial + ((size_t)s * gridDim.x + blk) * NPP;
  // sums over the CTA's 128 samples (K = samples, 8 steps of 16).  A = a
  // gradient tile transposed, B = an activation tile with its ones column;
  // both through transposed ldmatrix (matrix j of an x4: rows 8 (j & 1) and
  // columns 8 (j >> 1) of the 16 x 16 block for A; k rows 8 (j & 1), n tile
  // j >> 1 for B).
  const int mj = lane >> 3, mr = lane & 7;
  {  // [gW2 | gb2]: warp w takes output units 16w .. 16w + 15, all 9 n-tiles
    float acc[9][4];
#pragma unroll
    for (int nt = 0; nt < 9; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    for (int kk = 0; kk < TB; kk += 16) {
      uint32_t af[4];
      // A[m = j][k = sample] from gz2[sample][j]: matrix j's rows are samples
      ldmatrix_x4_t(af, S.gz2 + (kk + 8 * (mj >> 1) + mr) * TS + 16 * warp + 8 * (mj & 1));
#pragma unroll
      for (int nt = 0; nt < 9; nt += 2) {
        uint32_t bfr[4];
        const int ntb = nt + (mj >> 1) < 9 ? nt + (mj >> 1) : nt;  // the odd last tile reads tile 8 twice
        ldmatrix_x4_t(bfr, S.a1x + (kk + 8 * (mj & 1) + mr) * TS + 8 * ntb);
        mma_bf16(acc[nt], af, bfr[0], bfr[1]);
        if (nt + 1 < 9) mma_bf16(acc[nt + 1], af, bfr[2], bfr[3]);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 9; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = 16 * warp + g + 8 * (e >> 1), i = 8 * nt + 2 * q + (e & 1);
        if (i < H) P[OW2 + H * j + i] = acc[nt][e];
        else if (i == H) P[OB2 + j] = acc[nt][e];
      }
  }
  {  // [gW1 | gb1]: warp w takes hidden units 16w .. 16w + 15; B = [in | 1] (one n tile)
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kk = 0; kk < TB; kk += 16) {
      uint32_t af[4], bfr[4];
      ldmatrix_x4_t(af, S.gz1 + (kk + 8 * (mj >> 1) + mr) * TS + 16 * warp + 8 * (mj & 1));
      // matrices 0, 1: k rows 0-7 and 8-15 of the [in | 1] tile (2, 3 repeat them)
      ldmatrix_x4_t(bfr, S.inx + (kk + 8 * (mj & 1) + mr) * 8);
      mma_bf16(acc, af, bfr[0], bfr[1]);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 16 * warp + g + 8 * (e >> 1), c = 2 * q + (e & 1);
      if (c < 3) P[OW1 + 3 * j + c] = acc[e];
      else if (c == 3) P[OB1 + j] = acc[e];
    }
  }
  {  // [gW3 | gb3]: A = go^T (rows 0..2 of 16), B = [a2 | 1]; warp w takes n tiles w, w + 4 (and 8)
    for (int nt = warp; nt < 9; nt += 4) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int kk = 0; kk < TB; kk += 16) {
        uint32_t af[4], bfr[4];
        ldmatrix_x4_t(af, S.gox + (kk + 8 * (mj >> 1) + mr) * 16 + 8 * (mj & 1));
        ldmatrix_x4_t(bfr, S.a2x + (kk + 8 * (mj & 1) + mr) * TS + 8 * nt);
        mma_bf16(acc, af, bfr[0], bfr[1]);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = g + 8 * (e >> 1), j = 8 * nt + 2 * q + (e & 1);
        if (c < 3) {
          if (j < H) P[OW3 + H * c + j] = acc[e];
          else if (j == H) P[OB3 + c] = acc[e];
        }
      }
    }
  }
  if (t == 0) a.loss[(size_t)s * gridDim.x + blk] = ((S.loss[0] + S.loss[1]) + S.loss[2]) + S.loss[3];
}

struct MlpAdam {
  MlpClock* clock;  // lr_t, c1, c2 of the step; advanced by the step's last block
  float* master;
  float* m;
  float* v;
  const float* partial;
  StagedW* staged;  // the next step's weights
  unsigned* done;   // blocks finished with the step (zero between steps)
  int nblk;
  float b1, b2, eps;
};

// one thread per parameter: the CTA partials summed in a fixed order, then
// one Adam step on the FP32 master weights and their staged copy; the last
// block to finish advances the clock
__global__ void __launch_bounds__(256) k_mlp_adam(const __grid_constant__ MlpAdam a) {
  const int s = blockIdx.y, p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NP) {
    float g = 0.f;
    for (int k = 0; k < a.nblk; ++k) g += a.partial[((size_t)s * a.nblk + k) * NPP + p];
    const size_t q = (size_t)s * NPP + p;
    const float m = a.b1 * a.m[q] + (1.0f - a.b1) * g;
    const float v = a.b2 * a.v[q] + (1.0f - a.b2) * g * g;
    a.m[q] = m;
    a.v[q] = v;
    const float w = a.master[q] - a.clock->lr_t * (m / a.clock->c1) / (sqrtf(v / a.clock->c2) + a.eps);
    a.master[q] = w;
    stage_param(a.staged + s, p, w);
  }
  __syncthreads();  // every thread of the block has read the clock
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.done, 1u) == gridDim.x * gridDim.y - 1) {
      *a.done = 0u;
      a.clock->step += 1;
      clock_scalars(a.clock);
    }
  }
}

// Xavier-uniform initial weights (stream b = 0x5EED00000000, index = parameter)
__global__ void k_mlp_init(float* master, float* m, float* v, uint64_t seed) {
  const int s = blockIdx.x;
  for (int p = threadIdx.x; p < NPP; p += blockDim.x) {
    float lim = 0.f;
    if (p < OB1) lim = sqrtf(6.0f / (3 + H));
    else if (p >= OW2 && p < OB2) lim = sqrtf(6.0f / (H + H));
    else if (p >= OW3 && p < OB3) lim = sqrtf(6.0f / (H + 3));
    const size_t q = (size_t)s * NPP + p;
    master[q] = (p < NP && lim > 0.f)
                    ? (2.0f * counter_uniform(seed, (uint64_t)s, 0x5EED00000000ull, (uint64_t)p) - 1.0f) * lim
                    : 0.f;
    m[q] = 0.f;
    v[q] = 0.f;
  }
}

// residual |network - grid| (dy, dz) in cm at held-out points
struct MlpEval {
  const float* master;
  const float2* grid;
  int nx, ny, nz;
  uint64_t seed;
  float* out;  // [S][nblk][2]: max, sum of squares
};

__global__ void __launch_bounds__(TB) k_mlp_eval(const __grid_constant__ MlpEval a) {
  __shared__ float W[NPP];
  __shared__ float red[2][TB];
  const int s = blockIdx.y, blk = blockIdx.x, t = threadIdx.x;
  const float* M = a.master + (size_t)s * NPP;
  for (int p = t; p < NP; p += TB) {
    const bool bias = (p >= OB1 && p < OW2) || (p >= OB2 && p < OW3) || p >= OB3;
    W[p] = bias ? M[p] : bf(M[p]);
  }
  __syncthreads();
  float u[3], in[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u[c] = counter_uniform(a.seed, (uint64_t)s, 0xE7A100000000ull + blk, 3ull * t + c);
    in[c] = bf(2.0f * u[c] - 1.0f);
  }
  float a1[H];
#pragma unroll
  for (int j = 0; j < H; ++j)
    a1[j] = bf(silu_fast(W[OB1 + j] + W[OW1 + 3 * j] * in[0] + W[OW1 + 3 * j + 1] * in[1] + W[OW1 + 3 * j + 2] * in[2]));
  float o[3] = {W[OB3], W[OB3 + 1], W[OB3 + 2]};
  for (int j = 0; j < H; ++j) {
    float z2 = W[OB2 + j];
#pragma unroll
    for (int i = 0; i < H; ++i) z2 += W[OW2 + H * j + i] * a1[i];
    const float a2 = bf(silu_fast(z2));
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] += W[OW3 + H * c + j] * a2;
  }
  const float2* G = a.grid + (size_t)s * a.nx * a.ny * a.nz;
  const float2 tg = grid_at(G, a.nx, a.ny, a.nz, u[0] * (a.nx - 1), u[1] * (a.ny - 1), u[2] * (a.nz - 1));
  const float r = hypotf(OUT_SCALE * o[1] - tg.x, OUT_SCALE * o[2] - tg.y);
  red[0][t] = r;
  red[1][t] = r * r;
  __syncthreads();
  for (int off = TB / 2; off > 0; off >>= 1) {
    if (t < off) {
      red[0][t] = fmaxf(red[0][t], red[0][t + off]);
      red[1][t] += red[1][t + off];
    }
    __syncthreads();
  }
  if (t == 0) {
    a.out[((size_t)s * gridDim.x + blk) * 2] = red[0][0];
    a.out[((size_t)s * gridDim.x + blk) * 2 + 1] = red[1][0];
  }
}

// ---------------------------------------------------------------------------- inference
// Per-sector inference copy: W2 in BF16 with padded rows (16-byte aligned rows
// for ldmatrix, conflict-free), the other parameters as floats (weights
// BF16-rounded, biases FP32).  Layers 1 and 2 are stored halved (weights and
// biases x 0.5): their accumulators are then h = z / 2, the argument of the
// SiLU form h + h tanh(h), with no multiply.  Scaling by a power of two is
// exact in the BF16 operands, their products and the FP32 sums, so every
// output equals that of the unscaled network.
constexpr int W2S = 72;  // padded row stride of W2 in BF16 elements
struct __align__(16) MlpInfer {
  __nv_bfloat16 w2[H * W2S];
  float w1[192], b1[64], b2[64], w3[192], b3[4];
  float bounds[8];
};
static_assert(sizeof(MlpInfer) % 16 == 0, "16-byte copies");

__global__ void k_mlp_prepare(const float* master, const float* bounds, MlpInfer* inf) {
  const int s = blockIdx.x;
  const float* M = master + (size_t)s * NPP;
  MlpInfer& I = inf[s];
  for (int p = threadIdx.x; p < H * W2S; p += blockDim.x) {
    const int j = p / W2S, i = p % W2S;
    I.w2[p] = __float2bfloat16_rn(i < H ? 0.5f * bf(M[OW2 + H * j + i]) : 0.0f);
  }
  for (int p = threadIdx.x; p < 192; p += blockDim.x) {
    I.w1[p] = 0.5f * bf(M[OW1 + p]);
    I.w3[p] = bf(M[OW3 + p]);
  }
  for (int p = threadIdx.x; p < 64; p += blockDim.x) {
    I.b1[p] = 0.5f * M[OB1 + p];
    I.b2[p] = 0.5f * M[OB2 + p];
  }
  if (threadIdx.x < 3) I.b3[threadIdx.x] = M[OB3 + threadIdx.x];
  if (threadIdx.x < 6) I.bounds[threadIdx.x] = bounds[6 * s + threadIdx.x];
}

// One CTA per cluster chunk (one item): the sector's network in shared memory;
// each warp takes 16 clusters at a time and runs all three layers on the
// tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulators starting
// from the FP32 biases): layer 1 with K padded from 3 to 16, layer 3 with N
// padded from 3 to 8; each layer's accumulators become the next layer's A
// fragments in registers (after SiLU and BF16 rounding).  Fragment layout
// (lane = 4 g + q): A rows g and g+8, columns 2q, 2q+1 and +8; B column g, rows
// 2q, 2q+1 and +8; accumulators rows g and g+8, columns 2q, 2q+1.  The kernel
// is bound by instruction issue (two per SiLU: tanh and one FMA, on halved
// layers), so it is held to 80 registers for 6 CTAs per SM (measured 10%
// faster than 4 CTAs at 98 registers, despite a few spilled values).
__global__ void __launch_bounds__(128, 6) k_correct_mlp(const __grid_constant__ Buffers b) {
  __shared__ __align__(16) MlpInfer S;
  __shared__ float s_x[TPC_MAX_ROWS];  // row positions (lanes read different rows)
  const DevParams& P = b.par;
  const Chunk ch = b.chunks[blockIdx.x];
  const int sector = b.item_sector ? (int)b.item_sector[ch.item] : 0;
  if (sector >= b.mlp_sectors) {
    if (threadIdx.x == 0 && ch.end > ch.begin) atomicOr(b.err, TPC_DERR_BAD_INPUT);
    return;
  }
  {
    const int4* src = reinterpret_cast<const int4*>(reinterpret_cast<const MlpInfer*>(b.mlp) + sector);
    int4* dst = reinterpret_cast<int4*>(&S);
    for (int p = threadIdx.x; p < (int)(sizeof(MlpInfer) / 16); p += blockDim.x) dst[p] = src[p];
    for (int r = threadIdx.x; r < P.n_rows; r += blockDim.x) s_x[r] = P.x[r];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  // per-lane B fragments of layers 1 and 3 (constant over the chunk)
  uint32_t B1[8];  // n-tile t: rows 2q, 2q+1 of W1^T at unit 8t + g (inputs x, v | z, 0 | 0)
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int n = 8 * t + g;
    B1[t] = q == 0 ? pack_bf2(S.w1[3 * n], S.w1[3 * n + 1]) : q == 1 ? pack_bf2(S.w1[3 * n + 2], 0.0f) : 0u;
  }
  uint32_t B3[4][2];  // k-step ks: output g (< 3) at hidden units 16 ks + 2q, +1 and +8, +9
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int k0 = 16 * ks + 2 * q;
    B3[ks][0] = g < 3 ? pack_bf2(S.w3[64 * g + k0], S.w3[64 * g + k0 + 1]) : 0u;
    B3[ks][1] = g < 3 ? pack_bf2(S.w3[64 * g + k0 + 8], S.w3[64 * g + k0 + 9]) : 0u;
  }
  // layer-3 accumulator start: the output biases at columns 2q, 2q+1 (3 outputs)
  const float c3a = q == 0 ? S.b3[0] : q == 1 ? S.b3[2] : 0.0f;
  const float c3b = q == 0 ? S.b3[1] : 0.0f;
  const float sx = 2.0f / (S.bounds[1] - S.bounds[0]), sv = 2.0f / (S.bounds[3] - S.bounds[2]);
  const float sz = 2.0f / (S.bounds[5] - S.bounds[4]);
  // the cluster inputs of the two rows a lane touches are fetched one
  // iteration ahead
  int r_nx[2];
  float y_nx[2], z_nx[2];
  auto fetch = [&](int base) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = base + g + 8 * h;
      r_nx[h] = -1;
      y_nx[h] = 0.f;
      z_nx[h] = 0.f;
      if (i < ch.end) {
        r_nx[h] = __ldg(b.row + i);
        y_nx[h] = __ldg(b.y + i);
        z_nx[h] = __ldg(b.z + i);
      }
    }
  };
  fetch(ch.begin + warp * 16);
  for (int base = ch.begin + warp * 16; base < ch.end; base += 64) {
    const int r_cur[2] = {r_nx[0], r_nx[1]};
    const float y_cur[2] = {y_nx[0], y_nx[1]}, z_cur[2] = {z_nx[0], z_nx[1]};
    fetch(base + 64);
    // normalised inputs of the two rows this lane touches
    float in[2][3];
    int idx[2];
    bool ok[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = base + g + 8 * h;
      idx[h] = i;
      const int r = r_cur[h];
      ok[h] = i < ch.end && r >= 0 && r < P.n_rows;
      float x = 0.f, y = 0.f, z = 0.f;
      if (ok[h]) {
        x = s_x[r];
        y = y_cur[h];
        z = z_cur[h];
      }
      const float v = y / (x > 0.f ? x * P.tan_half : 1.0f);
      in[h][0] = (x - S.bounds[0]) * sx - 1.0f;
      in[h][1] = (v - S.bounds[2]) * sv - 1.0f;
      in[h][2] = (z - S.bounds[4]) * sz - 1.0f;
    }
    // layer 1: A = inputs (row g: x, v at q = 0, z at q = 1), K padded to 16
    uint32_t A1[4];
    A1[0] = q == 0 ? pack_bf2(in[0][0], in[0][1]) : q == 1 ? pack_bf2(in[0][2], 0.0f) : 0u;
    A1[1] = q == 0 ? pack_bf2(in[1][0], in[1][1]) : q == 1 ? pack_bf2(in[1][2], 0.0f) : 0u;
    A1[2] = 0u;
    A1[3] = 0u;
    uint32_t A[4][4];  // layer-2 A fragments
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const float2 bb = *reinterpret_cast<const float2*>(S.b1 + 8 * t + 2 * q);
      float d[4] = {bb.x, bb.y, bb.x, bb.y};
      mma_bf16(d, A1, B1[t], 0u);
      const int ks = t >> 1, half = t & 1;
      A[ks][2 * half] = pack_bf2(silu_of_half(d[0]), silu_of_half(d[1]));      // row g
      A[ks][2 * half + 1] = pack_bf2(silu_of_half(d[2]), silu_of_half(d[3]));  // row g + 8
    }
    // layer 2: B fragments of two k-steps per ldmatrix (matrix j = lane / 8 is
    // rows 8nt..8nt+7 of W2 at columns 16 (ks + j/2) + 8 (j%2))
    uint32_t A3[4][4];  // layer-3 A fragments
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float2 bb = *reinterpret_cast<const float2*>(S.b2 + 8 * nt + 2 * q);
      float d[4] = {bb.x, bb.y, bb.x, bb.y};
#pragma unroll
      for (int ks = 0; ks < 4; ks += 2) {
        uint32_t bf4[4];
        const int j = lane >> 3;
        ldmatrix_x4(bf4, S.w2 + (8 * nt + (lane & 7)) * W2S + 16 * (ks + (j >> 1)) + 8 * (j & 1));
        mma_bf16(d, A[ks], bf4[0], bf4[1]);
        mma_bf16(d, A[ks + 1], bf4[2], bf4[3]);
      }
      const int ks3 = nt >> 1, half = nt & 1;
      A3[ks3][2 * half] = pack_bf2(silu_of_half(d[0]), silu_of_half(d[1]));
      A3[ks3][2 * half + 1] = pack_bf2(silu_of_half(d[2]), silu_of_half(d[3]));
    }
    // layer 3: outputs 0..2 in columns 0..2 (column 1 = dy, column 2 = dz)
    float o[4] = {c3a, c3b, c3a, c3b};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) mma_bf16(o, A3[ks], B3[ks][0], B3[ks][1]);
    // dy sits in lane q = 0 (column 1), dz in lane q = 1 (column 0 + 2)
    if (q < 2) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = idx[h];
        if (i >= ch.end) continue;
        const float corr = q == 0 ? o[2 * h + 1] : o[2 * h];
        if (q == 0) b.cy[i] = y_cur[h] + (ok[h] ? OUT_SCALE * corr : 0.0f);
        else b.cz[i] = z_cur[h] + (ok[h] ? OUT_SCALE * corr : 0.0f);
      }
    }
  }
}

cudaError_t tpc_launch_mlp_correction(const Buffers& b, cudaStream_t s) {
  k_correct_mlp<<<b.n_chunks, 128, 0, s>>>(b);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------- host side
size_t tpc_mlp_infer_bytes() { return sizeof(MlpInfer); }
int tpc_mlp_nparams() { return NP; }
int tpc_mlp_stride() { return NPP; }

cudaError_t tpc_mlp_init(float* master, float* m, float* v, int S, uint64_t seed, cudaStream_t s) {
  k_mlp_init<<<S, 256, 0, s>>>(master, m, v, seed);
  return cudaGetLastError();
}

// Training workspace of S sectors: the clock and the step counter, then the
// staged weights of every sector.
namespace {
struct __align__(16) MlpWorkHead {
  MlpClock clock;
  unsigned done;
};
StagedW* staged_of(void* work) {
  return reinterpret_cast<StagedW*>(static_cast<char*>(work) + sizeof(MlpWorkHead));
}
}  // namespace
static_assert(sizeof(MlpWorkHead) % 16 == 0, "staged weights follow at a 16-byte boundary");

size_t tpc_mlp_work_bytes(int S) { return sizeof(MlpWorkHead) + sizeof(StagedW) * (size_t)S; }

cudaError_t tpc_mlp_train_steps(void* work, uint64_t first, uint64_t T, float lr, uint64_t n_steps, float* master,
                                float* m, float* v, float* partial, float* loss, const float2* grid, int nx, int ny,
                                int nz, int S, int batch, uint64_t seed, bool graph, cudaStream_t s) {
  // an attribute of the current device: set per call (a process may train on several devices)
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TrainSmem));
  if (e != cudaSuccess) return e;
  MlpWorkHead* w = static_cast<MlpWorkHead*>(work);
  MlpClock* ck = &w->clock;
  StagedW* staged = staged_of(work);
  k_mlp_clock_set<<<1, 1, 0, s>>>(ck, first, T, lr);
  if ((e = cudaMemsetAsync(&w->done, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  k_mlp_stage<<<S, 256, 0, s>>>(master, staged);
  const int nblk = batch / TB;
  MlpTrain a{ck, staged, partial, loss, grid, nx, ny, nz, seed, 0, batch};
  MlpAdam ad{ck, master, m, v, partial, staged, &w->done, nblk, 0.9f, 0.999f, 1e-8f};
  auto one = [&]() {
    k_mlp_grad<<<dim3(nblk, S), TB, sizeof(TrainSmem), s>>>(a);
    k_mlp_adam<<<dim3((NP + 255) / 256, S), 256, 0, s>>>(ad);
  };
  // K steps captured once and replayed: no host work between steps
  constexpr uint64_t K = 64;
  uint64_t done = 0;
  if (graph && n_steps >= 2 * K) {  // (the legacy default stream cannot be captured)
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (uint64_t k = 0; k < K; ++k) one();
    cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    for (; done + K <= n_steps && e == cudaSuccess; done += K) e = cudaGraphLaunch(ge, s);
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) return e;
  }
  for (; done < n_steps; ++done) one();
  return cudaGetLastError();
}

cudaError_t tpc_mlp_grad_only(void* work, const float* master, float* partial, float* loss, const float2* grid,
                              int nx, int ny, int nz, int S, int batch, uint64_t seed, uint64_t step, cudaStream_t s) {
  const size_t smem = sizeof(TrainSmem);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  StagedW* staged = staged_of(work);
  k_mlp_stage<<<S, 256, 0, s>>>(master, staged);
  MlpTrain a{nullptr, staged, partial, loss, grid, nx, ny, nz, seed, step, batch};
  k_mlp_grad<<<dim3(batch / TB, S), TB, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t tpc_mlp_eval(const float* master, const float2* grid, int nx, int ny, int nz, int S, int nblk,
                         uint64_t seed, float* out, cudaStream_t s) {
  MlpEval a{master, grid, nx, ny, nz, seed, out};
  k_mlp_eval<<<dim3(nblk, S), TB, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t tpc_mlp_prepare(const float* master, const float* bounds, void* infer, int S, cudaStream_t s) {
  k_mlp_prepare<<<S, 256, 0, s>>>(master, bounds, reinterpret_cast<MlpInfer*>(infer));
  return cudaGetLastError();
}
