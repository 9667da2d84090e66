// tpc_bin_sector_noalloc: the binning step for one sector without any device
// allocation.
//
// Who needs this: callers that must not allocate GPU memory while they run --
// for example code inside a real-time readout loop with a fixed memory budget
// set up at start, a plug-in that runs under a host framework which owns all
// device memory, or code that must not call cudaMalloc/cudaFree because those
// calls synchronise the device and would stall other work.  They pass their own
// input and output buffers; the temporary storage the step needs lives in a
// fixed, file-scope device array that is part of the loaded library.
//
// The scratch array is shared by every call in the process on a given GPU and
// keeps the previous call's contents.  Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on it: run them one after another.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "tpc.h"

namespace {

constexpr int NA_THREADS = 1024;
constexpr int NA_MAX_ROWS = 256;

// Scratch of one call: grouped (row-contiguous, in input order) hits and
// their ids, the slot of every hit in its bin, and an error word.  Every call
// writes each entry it later reads, except the error word, which the kernel
// clears first.  Size: 16 bytes per cluster (1 MiB) plus 256 bytes.
struct __align__(16) NoAllocScratch {
  int2 g_q[TPC_NOALLOC_MAX_CLUSTERS];
  int g_id[TPC_NOALLOC_MAX_CLUSTERS];
  int slot[TPC_NOALLOC_MAX_CLUSTERS];
  unsigned int err;
  unsigned int pad[63];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ int na_block_excl_scan(int v, int* sm, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sm[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    const int s = lane < nw ? sm[lane] : 0;
    int si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += t;
    }
    if (lane < nw) sm[lane] = si - s;
    if (lane == 31) sm[32] = si;
  }
  __syncthreads();
  const int r = sm[w] + inc - v;
  *total = sm[32];
  __syncthreads();
  return r;
}

// Stable ranks for one chunk of blockDim.x items, one per thread in thread
// order: each valid item gets counters[key] plus the number of valid items of
// the same key in earlier threads of the chunk, and counters[key] grows by the
// chunk's count of that key.  Within a warp the lanes of one key are found by
// match_any (the lowest lane adds the warp's count); the warps add in warp
// order, one per barrier.  The whole block must call it (uniform control flow).
__device__ __forceinline__ int na_stable_rank(int key, bool valid, int* counters) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // invalid lanes share a key no valid lane has (keys are >= 0)
  const unsigned peers = __match_any_sync(0xffffffffu, valid ? key : -1);
  const int leader = __ffs(peers) - 1;
  const int before = __popc(peers & ((1u << lane) - 1u));
  int base = 0;
  for (int k = 0; k < nw; ++k) {
    if (w == k && valid && lane == leader) {
      base = counters[key];
      counters[key] = base + __popc(peers);
    }
    __syncthreads();
  }
  return __shfl_sync(0xffffffffu, base, leader) + before;
}

// One CTA bins the whole sector: quantise y, z to 2^-10 cm (round half to
// even; the scale is exact in FP32), per-row counts and extents, bin edge 2^s
// quanta with s the smallest s >= 10 such that n*4^s >= Ly*Lz and
// ny*nz <= 2n+2, a stable counting sort into rows (input order kept inside a
// row), then per row a bin histogram, scan and stable scatter, so that a bin
// holds its hits in input order (the canonical order: row, bin, original
// index) without a sort.  The output layout equals the one of the tracker's
// own binning step for a single item.
__global__ void __launch_bounds__(NA_THREADS) k_bin_sector_noalloc(NoAllocScratch* sc, const float* y, const float* z,
                                                                   const int* row, int n, int n_rows, int4* sorted,
                                                                   int* rows_out, int* first_out) {
  __shared__ int s_cnt[NA_MAX_ROWS], s_min[4][NA_MAX_ROWS], s_fill[NA_MAX_ROWS];
  __shared__ int s_pos0[NA_MAX_ROWS], s_shift[NA_MAX_ROWS], s_ny[NA_MAX_ROWS], s_nz[NA_MAX_ROWS], s_bin0[NA_MAX_ROWS];
  __shared__ int sm[33];
  __shared__ unsigned int s_err;
  if (threadIdx.x == 0) s_err = 0;
  for (int r = threadIdx.x; r < n_rows; r += blockDim.x) {
    s_cnt[r] = 0;
    s_fill[r] = 0;
    s_min[0][r] = s_min[1][r] = s_min[2][r] = s_min[3][r] = 0x7F7F7F7F;
  }
  __syncthreads();
  // counts and extents
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float yv = y[i], zv = z[i];
    const int r = row[i];
    if (!(r >= 0 && r < n_rows && fabsf(yv) <= 1e6f && fabsf(zv) <= 1e6f)) {
      atomicOr(&s_err, 1u);
      continue;
    }
    const int qy = __float2int_rn(yv * 1024.0f), qz = __float2int_rn(zv * 1024.0f);
    atomicAdd(&s_cnt[r], 1);
    atomicMin(&s_min[0][r], qy);
    atomicMin(&s_min[1][r], -qy);
    atomicMin(&s_min[2][r], qz);
    atomicMin(&s_min[3][r], -qz);
  }
  __syncthreads();
  // grid of every row
  const int r = threadIdx.x;
  int cnt = 0, nb = 0;
  if (r < n_rows) {
    cnt = s_cnt[r];
    int s = 10, ny = 0, nz = 0;
    if (cnt > 0) {
      const long long dy = (long long)(-s_min[1][r]) - s_min[0][r];
      const long long dz = (long long)(-s_min[3][r]) - s_min[2][r];
      const long long need = ((dy + 1) * (dz + 1) + cnt - 1) / cnt;
      for (;; ++s) {
        const long long nyy = (dy >> s) + 1, nzz = (dz >> s) + 1;
        if ((2 * s >= 63 || (1ll << (2 * s)) >= need) && nyy * nzz <= 2ll * cnt + 2) {
          ny = (int)nyy;
          nz = (int)nzz;
          break;
        }
      }
      nb = ny * nz;
    } else {
      s_min[0][r] = 0;
      s_min[2][r] = 0;
    }
    s_shift[r] = s;
    s_ny[r] = ny;
    s_nz[r] = nz;
  }
  int tot;
  const int pos_ex = na_block_excl_scan(cnt, sm, &tot);
  const int bin_ex = na_block_excl_scan(r < n_rows ? nb + 1 : 0, sm, &tot);
  if (r < n_rows) {
    s_pos0[r] = pos_ex;
    s_bin0[r] = bin_ex;
    int* o = rows_out + 8 * r;
    o[0] = pos_ex;
    o[1] = cnt;
    o[2] = s_min[0][r];
    o[3] = s_min[2][r];
    o[4] = s_shift[r];
    o[5] = s_ny[r];
    o[6] = s_nz[r];
    o[7] = bin_ex;
  }
  __syncthreads();
  // stable counting sort into rows: chunks of the input in index order
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    float yv = 0.f, zv = 0.f;
    int rr = -1;
    if (i < n) {
      yv = y[i];
      zv = z[i];
      rr = row[i];
    }
    const bool ok = i < n && rr >= 0 && rr < n_rows && fabsf(yv) <= 1e6f && fabsf(zv) <= 1e6f;
    const int rank = na_stable_rank(ok ? rr : 0, ok, s_fill);
    if (ok) {
      const int gp = s_pos0[rr] + rank;
      sc->g_q[gp] = make_int2(__float2int_rn(yv * 1024.0f), __float2int_rn(zv * 1024.0f));
      sc->g_id[gp] = i;
    }
  }
  __syncthreads();
  // per row: bin histogram (in first_out), exclusive scan, stable scatter
  for (int rr = 0; rr < n_rows; ++rr) {
    const int cn = s_cnt[rr], p0 = s_pos0[rr], b0 = s_bin0[rr];
    const int nbr = cn > 0 ? s_ny[rr] * s_nz[rr] : 0;
    int* hist = first_out + b0;
    for (int j = threadIdx.x; j <= nbr; j += blockDim.x) hist[j] = 0;
    __syncthreads();
    const int sh = s_shift[rr], ymin = s_min[0][rr], zmin = s_min[2][rr], nzr = s_nz[rr];
    for (int base = 0; base < cn; base += blockDim.x) {  // block-uniform loop
      const int j = base + threadIdx.x;
      int bin = 0;
      if (j < cn) {
        const int2 q = sc->g_q[p0 + j];
        bin = ((q.x - ymin) >> sh) * nzr + ((q.y - zmin) >> sh);
      }
      const int slot = na_stable_rank(bin, j < cn, hist);
      if (j < cn) sc->slot[p0 + j] = slot;
    }
    __syncthreads();
    int carry = 0;
    for (int base = 0; base <= nbr; base += blockDim.x) {
      const int j = base + threadIdx.x;
      const int v = j <= nbr ? hist[j] : 0;
      int t2;
      const int ex = na_block_excl_scan(v, sm, &t2);
      if (j <= nbr) hist[j] = carry + ex;
      carry += t2;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cn; j += blockDim.x) {
      const int2 q = sc->g_q[p0 + j];
      const int bin = ((q.x - ymin) >> sh) * nzr + ((q.y - zmin) >> sh);
      sorted[p0 + hist[bin] + sc->slot[p0 + j]] = make_int4(q.x, q.y, sc->g_id[p0 + j], rr);
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= nbr; j += blockDim.x) hist[j] += p0;
    __syncthreads();
  }
  if (threadIdx.x == 0) sc->err = s_err;
}

}  // namespace

extern "C" tpc_status tpc_bin_sector_noalloc(const float* y, const float* z, const int32_t* row, uint32_t n, int n_rows,
                                             int32_t* sorted, int32_t* rows_out, int32_t* first_out, void* stream) {
  if (n > TPC_NOALLOC_MAX_CLUSTERS || n_rows < 1 || n_rows > NA_MAX_ROWS) return TPC_ERR_CAPACITY;
  if ((n > 0 && (!y || !z || !row || !sorted)) || !rows_out || !first_out) return TPC_ERR_INVALID_ARG;
  // The array's host-side name is not a device address: look the address up
  // in the current context on every call (it allocates nothing).  An address
  // kept from an earlier call could belong to another context of the device
  // (a caller's own context, or one made after cudaDeviceReset).
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return TPC_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  k_bin_sector_noalloc<<<1, NA_THREADS, 0, s>>>(static_cast<NoAllocScratch*>(ptr), y, z, row, (int)n, n_rows,
                                                reinterpret_cast<int4*>(sorted), rows_out, first_out);
  if (cudaGetLastError() != cudaSuccess) return TPC_ERR_CUDA;
  unsigned int err = 0;
  if (cudaMemcpyAsync(&err, &static_cast<NoAllocScratch*>(ptr)->err, sizeof(err), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return TPC_ERR_CUDA;
  }
  return err ? TPC_ERR_BAD_INPUT : TPC_OK;
}
