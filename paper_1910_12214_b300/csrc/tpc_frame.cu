// Continuous read-out time frames (the paper's Abstract and Sec. 2: 50 kHz
// Pb-Pb with continuous read-out, no a-priori vertex, so that cluster z carries
// the drift-time offset of its collision) cut into overlapping slices on the
// device, so that every slice is an ordinary tracker item.
//
// Each frame item (normally a sector) is cut along z into cores
// [c0 + k core, c0 + (k + 1) core), k = 0 .. K-1, with c0 = floor(zmin / core)
// core and K the number of cores up to zmax; slice k holds every cluster of the
// item with c0 + k core - overlap <= z < c0 + (k + 1) core + overlap.  The
// ranges are decided exactly as in FP64: the bounds are rounded up to the next
// float, which makes the FP32 comparison of a float z equal to the FP64 one.
// Inside a slice the clusters keep the frame's order (a stable scatter), so the
// slice's cluster ids order them as the frame's indices do and every id
// tie-break of the tracker decides as on the unsliced frame.  A track is
// reported by the slice whose core holds its innermost cluster (item_core).
#include "tpc_internal.cuh"

namespace {

__device__ __forceinline__ int f2ord(float f) {  // order-preserving float -> int
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

// smallest float >= d
__device__ __forceinline__ float ceil_float(double d) {
  float f = (float)d;
  if ((double)f < d) f = nextafterf(f, INFINITY);
  return f;
}

__global__ void __launch_bounds__(256) k_tf_init(const __grid_constant__ FrameArgs a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.F; i += gridDim.x * blockDim.x) {
    a.ext[2 * i] = 0x7FFFFFFF;
    a.ext[2 * i + 1] = (int)0x80000000;
  }
}

// z extent of every item (chunk-parallel, ordered-integer atomics); a
// non-finite z flags the frame as bad input
__global__ void __launch_bounds__(256) k_tf_extent(const __grid_constant__ FrameArgs a) {
  const Chunk ch = a.chunks[blockIdx.x];
  int lo = 0x7FFFFFFF, hi = (int)0x80000000;
  bool bad = false;
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) {
    const float z = a.z[i];
    if (!(fabsf(z) <= 1e6f)) {
      bad = true;
      continue;
    }
    const int o = f2ord(z);
    lo = min(lo, o);
    hi = max(hi, o);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(a.err, TPC_DERR_BAD_INPUT);
  if ((threadIdx.x & 31) == 0 && lo <= hi) {
    atomicMin(&a.ext[2 * ch.item], lo);
    atomicMax(&a.ext[2 * ch.item + 1], hi);
  }
}

// per item: first core c0, slice count K and the exact float bounds of every
// slice's extended range (one thread per item; the only FP64 work)
__global__ void __launch_bounds__(64) k_tf_slices(const __grid_constant__ FrameArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.F) return;
  const int lo = a.ext[2 * i], hi = a.ext[2 * i + 1];
  int K = 0;
  double c0 = 0.0;
  if (lo <= hi) {
    const double zmin = ord2f(lo), zmax = ord2f(hi);
    c0 = floor(zmin / a.core) * a.core;
    K = (int)floor((zmax - c0) / a.core) + 1;
    if (K > TF_KMAX) {
      atomicOr(a.err, TPC_DERR_CAPACITY);
      K = 0;
    }
  }
  a.c0[i] = c0;
  a.nslice[i] = K;
  for (int k = 0; k < K; ++k) {
    const double c = c0 + k * a.core;
    a.bounds[i * TF_KMAX + k] = make_float2(ceil_float(c - a.overlap), ceil_float(c + a.core + a.overlap));
  }
}

// the slices [k0, k1] of the item that contain z (k1 < k0: none)
__device__ __forceinline__ void tf_members(const FrameArgs& a, const float2* bnd, float c0, int K, float z, int* k0,
                                           int* k1) {
  const int ke = (int)floorf((z - c0) / a.core);
  int lo = 1 << 30, hi = -1;
  for (int k = max(0, ke - a.W); k <= min(K - 1, ke + a.W); ++k) {
    const float2 b = bnd[k];
    if (z >= b.x && z < b.y) {
      lo = min(lo, k);
      hi = k;
    }
  }
  *k0 = lo;
  *k1 = hi;
}

// memberships per (chunk, slice): cnt[chunk][k]
__global__ void __launch_bounds__(256) k_tf_count(const __grid_constant__ FrameArgs a) {
  __shared__ float2 s_b[TF_KMAX];
  __shared__ int s_cnt[TF_KMAX];
  const Chunk ch = a.chunks[blockIdx.x];
  const int K = a.nslice[ch.item];
  const float c0 = (float)a.c0[ch.item];
  for (int k = threadIdx.x; k < TF_KMAX; k += blockDim.x) {
    s_cnt[k] = 0;
    if (k < K) s_b[k] = a.bounds[ch.item * TF_KMAX + k];
  }
  __syncthreads();
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) {
    const float z = a.z[i];
    if (!(fabsf(z) <= 1e6f)) continue;
    int k0, k1;
    tf_members(a, s_b, c0, K, z, &k0, &k1);
    for (int k = k0; k <= k1; ++k) atomicAdd(&s_cnt[k], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < TF_KMAX; k += blockDim.x) a.cnt[(size_t)blockIdx.x * TF_KMAX + k] = s_cnt[k];
}

// per item and slice: exclusive scan of the counts over the item's chunks (in
// place: cnt becomes each chunk's base inside the slice) and the slice sizes
__global__ void __launch_bounds__(TF_KMAX) k_tf_scan(const __grid_constant__ FrameArgs a) {
  const int i = blockIdx.x, k = threadIdx.x;
  int run = 0;
  for (int c = a.chunk_first[i]; c < a.chunk_first[i + 1]; ++c) {
    int* p = a.cnt + (size_t)c * TF_KMAX + k;
    const int v = *p;
    *p = run;
    run += v;
  }
  a.size[i * TF_KMAX + k] = run;
}

// stable scatter of every chunk's clusters into its slices of the sliced batch
__global__ void __launch_bounds__(256) k_tf_scatter(const __grid_constant__ FrameArgs a) {
  __shared__ float2 s_b[TF_KMAX];
  __shared__ long long s_run[TF_KMAX];
  __shared__ int s_wt[8][TF_KMAX];
  const Chunk ch = a.chunks[blockIdx.x];
  const int K = a.nslice[ch.item];
  const float c0 = (float)a.c0[ch.item];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    s_b[k] = a.bounds[ch.item * TF_KMAX + k];
    s_run[k] = (long long)a.slice_off[a.slice_first[ch.item] + k] + a.cnt[(size_t)blockIdx.x * TF_KMAX + k];
  }
  __syncthreads();
  for (int base = ch.begin; base < ch.end; base += blockDim.x) {  // block-uniform rounds, frame order
    const int i = base + threadIdx.x;
    int k0 = 1 << 30, k1 = -1;
    float z = 0.f;
    if (i < ch.end) {
      z = a.z[i];
      if (fabsf(z) <= 1e6f) tf_members(a, s_b, c0, K, z, &k0, &k1);
    }
    int pre[2 * TF_WMAX + 1];  // rank among the earlier lanes of the warp, per own slice
    for (int k = 0; k < K; ++k) {
      const unsigned bal = __ballot_sync(0xffffffffu, k >= k0 && k <= k1);
      if (k >= k0 && k <= k1) pre[k - k0] = __popc(bal & ((1u << lane) - 1u));
      if (lane == 0) s_wt[w][k] = __popc(bal);
    }
    __syncthreads();
    if (i < ch.end && k1 >= k0) {
      const float x = a.x[i], y = a.y[i];
      const int r = a.row[i];
      for (int k = k0; k <= k1; ++k) {
        long long pos = s_run[k] + pre[k - k0];
        for (int v = 0; v < w; ++v) pos += s_wt[v][k];
        a.ox[pos] = x;
        a.oy[pos] = y;
        a.oz[pos] = z;
        a.orow[pos] = r;
        a.src[pos] = i;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      int t = 0;
      for (int v = 0; v < (int)(blockDim.x >> 5); ++v) t += s_wt[v][k];
      s_run[k] += t;
    }
    __syncthreads();
  }
}

// output cluster ids of the sliced batch -> frame indices
__global__ void __launch_bounds__(256) k_tf_map_ids(const uint32_t* in, const int* src, uint32_t* out,
                                                    const unsigned long long* counts) {
  const unsigned long long n = counts[1];
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
       j += (unsigned long long)gridDim.x * blockDim.x)
    out[j] = (uint32_t)src[in[j]];
}

}  // namespace

cudaError_t tpc_frame_count(const FrameArgs& a, cudaStream_t s) {
  if (a.F == 0) return cudaSuccess;
  k_tf_init<<<(a.F + 255) / 256, 256, 0, s>>>(a);
  if (a.n_chunks) k_tf_extent<<<a.n_chunks, 256, 0, s>>>(a);
  k_tf_slices<<<(a.F + 63) / 64, 64, 0, s>>>(a);
  if (a.n_chunks) k_tf_count<<<a.n_chunks, 256, 0, s>>>(a);
  k_tf_scan<<<a.F, TF_KMAX, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t tpc_frame_scatter(const FrameArgs& a, cudaStream_t s) {
  if (a.n_chunks) k_tf_scatter<<<a.n_chunks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t tpc_frame_map_ids(const uint32_t* in, const int* src, uint32_t* out, const unsigned long long* counts,
                              int blocks, cudaStream_t s) {
  k_tf_map_ids<<<blocks, 256, 0, s>>>(in, src, out, counts);
  return cudaGetLastError();
}
