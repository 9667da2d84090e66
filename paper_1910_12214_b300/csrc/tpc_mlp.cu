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
constexpr int WS = 516;       // per-warp slots: 192 gW3, 3 gb3, 64 gb2, 192 gW1, 64 gb1, loss

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
__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

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
__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
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
struct MlpTrain {
  const float* master;  // [S][NPP]
  float* partial;       // [S][nblk][NPP]
  float* loss;          // [S][nblk]
  const float2* grid;   // [S][nx][ny][nz]
  int nx, ny, nz;
  uint64_t seed, step;
  int batch;            // samples per sector and step (multiple of TB)
};

__global__ void __launch_bounds__(TB) k_mlp_grad(const __grid_constant__ MlpTrain a) {
  extern __shared__ float smem[];
  float* W = smem;                 // rounded weights and FP32 biases [NPP]
  float* A1 = W + NPP;             // [H][TB] first hidden activations (BF16 values)
  float* Z2 = A1 + H * TB;         // [H][TB] second pre-activations, then their gradients
  float* WP = Z2 + H * TB;         // [4 warps][WS] per-warp gradient sums
  const int s = blockIdx.y, blk = blockIdx.x, t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const float* M = a.master + (size_t)s * NPP;
  for (int p = t; p < NP; p += TB) {
    const bool bias = (p >= OB1 && p < OW2) || (p >= OB2 && p < OW3) || p >= OB3;
    W[p] = bias ? M[p] : bf(M[p]);
  }
  __syncthreads();
  // sample and target
  const uint64_t k = (uint64_t)blk * TB + t;
  float in[3], u[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u[c] = counter_uniform(a.seed, (uint64_t)s, a.step, 3ull * k + c);
    in[c] = bf(2.0f * u[c] - 1.0f);
  }
  const float2* G = a.grid + (size_t)s * a.nx * a.ny * a.nz;
  const float2 tg = grid_at(G, a.nx, a.ny, a.nz, u[0] * (a.nx - 1), u[1] * (a.ny - 1), u[2] * (a.nz - 1));
  const float tgt[3] = {0.0f, tg.x / OUT_SCALE, tg.y / OUT_SCALE};
  // forward
  for (int j = 0; j < H; ++j) {
    const float z1 = W[OB1 + j] + W[OW1 + 3 * j] * in[0] + W[OW1 + 3 * j + 1] * in[1] + W[OW1 + 3 * j + 2] * in[2];
    A1[j * TB + t] = bf(silu(z1));
  }
  float o[3] = {W[OB3], W[OB3 + 1], W[OB3 + 2]};
  for (int j = 0; j < H; ++j) {
    float z2 = W[OB2 + j];
    const float* w2 = W + OW2 + H * j;
    for (int i = 0; i < H; ++i) z2 += w2[i] * A1[i * TB + t];
    Z2[j * TB + t] = z2;
    const float a2 = bf(silu(z2));
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] += W[OW3 + H * c + j] * a2;
  }
  float go[3], l = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float r = o[c] - tgt[c];
    l += r * r;
    go[c] = 2.0f * r / (float)a.batch;
  }
  // backward through layer 3: per-warp sums of the 3-wide gradients
  auto wsum = [&](float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
  };
  float* wp = WP + warp * WS;  // 192 gW3 | 3 gb3 | 64 gb2 | 192 gW1 | 64 gb1 | loss
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float v = wsum(go[c]);
    if (lane == 0) wp[192 + c] = v;
  }
  {
    const float lv = wsum(l);
    if (lane == 0) wp[515] = lv;
  }
  for (int j = 0; j < H; ++j) {
    const float z2 = Z2[j * TB + t];
    const float a2 = bf(silu(z2));
    float ga2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ga2 += W[OW3 + H * c + j] * go[c];
      const float v = wsum(go[c] * a2);
      if (lane == 0) wp[H * c + j] = v;
    }
    const float gz2 = ga2 * dsilu(z2);
    Z2[j * TB + t] = gz2;
    const float v = wsum(gz2);
    if (lane == 0) wp[195 + j] = v;
  }
  __syncthreads();
  float* P = a.partial + ((size_t)s * gridDim.x + blk) * NPP;
  // gW2[j][i] = sum over samples of gz2[j] a1[i]
  for (int e = t; e < H * H; e += TB) {
    const int j = e / H, i = e % H;
    const float* gz = Z2 + j * TB;
    const float* a1 = A1 + i * TB;
    float acc = 0.f;
    for (int b = 0; b < TB; ++b) acc += gz[b] * a1[b];
    P[OW2 + e] = acc;
  }
  // layer 1
  for (int i = 0; i < H; ++i) {
    float ga1 = 0.f;
    for (int j = 0; j < H; ++j) ga1 += W[OW2 + H * j + i] * Z2[j * TB + t];
    const float z1 = W[OB1 + i] + W[OW1 + 3 * i] * in[0] + W[OW1 + 3 * i + 1] * in[1] + W[OW1 + 3 * i + 2] * in[2];
    const float gz1 = ga1 * dsilu(z1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float v = wsum(gz1 * in[c]);
      if (lane == 0) wp[259 + 3 * i + c] = v;
    }
    const float v = wsum(gz1);
    if (lane == 0) wp[451 + i] = v;
  }
  __syncthreads();
  // fixed-order sum of the four warps
  for (int q = t; q < WS; q += TB) {
    const float v = ((WP[q] + WP[WS + q]) + WP[2 * WS + q]) + WP[3 * WS + q];
    if (q < 192) P[OW3 + q] = v;
    else if (q < 195) P[OB3 + q - 192] = v;
    else if (q < 259) P[OB2 + q - 195] = v;
    else if (q < 451) P[OW1 + q - 259] = v;
    else if (q < 515) P[OB1 + q - 451] = v;
    else a.loss[(size_t)s * gridDim.x + blk] = v;
  }
}

struct MlpAdam {
  float* master;
  float* m;
  float* v;
  const float* partial;
  int nblk;
  float lr_t, b1, b2, c1, c2, eps;  // c1 = 1 - b1^t, c2 = 1 - b2^t
};

__global__ void __launch_bounds__(256) k_mlp_adam(const __grid_constant__ MlpAdam a) {
  const int s = blockIdx.x;
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    float g = 0.f;
    for (int k = 0; k < a.nblk; ++k) g += a.partial[((size_t)s * a.nblk + k) * NPP + p];
    const size_t q = (size_t)s * NPP + p;
    const float m = a.b1 * a.m[q] + (1.0f - a.b1) * g;
    const float v = a.b2 * a.v[q] + (1.0f - a.b2) * g * g;
    a.m[q] = m;
    a.v[q] = v;
    a.master[q] -= a.lr_t * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
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
// BF16-rounded, biases FP32).
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
    I.w2[p] = __float2bfloat16_rn(i < H ? M[OW2 + H * j + i] : 0.0f);
  }
  for (int p = threadIdx.x; p < 192; p += blockDim.x) {
    I.w1[p] = bf(M[OW1 + p]);
    I.w3[p] = bf(M[OW3 + p]);
  }
  for (int p = threadIdx.x; p < 64; p += blockDim.x) {
    I.b1[p] = M[OB1 + p];
    I.b2[p] = M[OB2 + p];
  }
  if (threadIdx.x < 3) I.b3[threadIdx.x] = M[OB3 + threadIdx.x];
  if (threadIdx.x < 6) I.bounds[threadIdx.x] = bounds[6 * s + threadIdx.x];
}

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// four 8x8 BF16 matrices from shared memory (rows given by lanes 8j..8j+7 for
// matrix j); lane l receives row l/4, columns 2(l%4) and 2(l%4)+1 of each
__device__ __forceinline__ void ldmatrix_x4(uint32_t* r, const void* smem_row) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One CTA per cluster chunk (one item): the sector's network in shared memory;
// each warp takes 16 clusters at a time and runs all three layers on the
// tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulators starting
// from the FP32 biases): layer 1 with K padded from 3 to 16, layer 3 with N
// padded from 3 to 8; each layer's accumulators become the next layer's A
// fragments in registers (after SiLU and BF16 rounding).  Fragment layout
// (lane = 4 g + q): A rows g and g+8, columns 2q, 2q+1 and +8; B column g, rows
// 2q, 2q+1 and +8; accumulators rows g and g+8, columns 2q, 2q+1.
__global__ void __launch_bounds__(128) k_correct_mlp(const __grid_constant__ Buffers b) {
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
      A[ks][2 * half] = pack_bf2(silu_fast(d[0]), silu_fast(d[1]));      // row g
      A[ks][2 * half + 1] = pack_bf2(silu_fast(d[2]), silu_fast(d[3]));  // row g + 8
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
      A3[ks3][2 * half] = pack_bf2(silu_fast(d[0]), silu_fast(d[1]));
      A3[ks3][2 * half + 1] = pack_bf2(silu_fast(d[2]), silu_fast(d[3]));
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

cudaError_t tpc_mlp_step(float* master, float* m, float* v, float* partial, float* loss, const float2* grid, int nx,
                         int ny, int nz, int S, int batch, uint64_t seed, uint64_t step, float lr_t, float c1, float c2,
                         cudaStream_t s) {
  const size_t smem = sizeof(float) * (NPP + 2 * H * TB + 4 * WS);
  // an attribute of the current device: set per call (a process may train on several devices)
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  MlpTrain a{master, partial, loss, grid, nx, ny, nz, seed, step, batch};
  const int nblk = batch / TB;
  k_mlp_grad<<<dim3(nblk, S), TB, smem, s>>>(a);
  MlpAdam ad{master, m, v, partial, nblk, lr_t, 0.9f, 0.999f, c1, c2, 1e-8f};
  k_mlp_adam<<<S, 256, 0, s>>>(ad);
  return cudaGetLastError();
}

cudaError_t tpc_mlp_grad_only(const float* master, float* partial, float* loss, const float2* grid, int nx, int ny,
                              int nz, int S, int batch, uint64_t seed, uint64_t step, cudaStream_t s) {
  const size_t smem = sizeof(float) * (NPP + 2 * H * TB + 4 * WS);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  MlpTrain a{master, partial, loss, grid, nx, ny, nz, seed, step, batch};
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
