// CUDA kernels of the TPC sector tracker (sm_103a).
//
// Steps (one kernel each in plain mode; see tpc_capi.cu for the launch order):
//   k_row_stats      quantise y,z to Q = 2^-10 cm, validate, per-(item,row) count
//                    and extents (global atomics)
//   k_row_setup      bin size, grid dims, row and bin offsets (block scans)
//   k_group_scatter  counting sort of clusters into row-contiguous order
//   k_row_sort_warp  per row (a warp each): bin histogram, scan, scatter, in-bin sort
//                    by id (canonical order row, bin, original id) and first[] starts
//   k_row_sort       the same per CTA: rows too large for a warp's shared memory, and
//                    every row of batches with dense rows (time-frame slices)
//   k_links          per hit of an inner row: best (up, down) pair (integer metric)
//   k_clean_start    mutual-link cleaning and start-hit flags
//   k_scan_*         device-wide exclusive scans (reduce-then-scan, fixed grid)
//   k_tracklets_up   FP32 Kalman tracklet per start hit: chain fit and outward
//                    extension; each tracklet claims its outermost hit
//   k_tracklets_down inward refit with hit re-picking, one per outermost hit
//   k_select_max/own shared-cluster resolution by 64-bit atomicMax keys
//   k_output         track and cluster-id compaction
// Batched form (S9 below): the same steps, the tracklet passes as persistent
// kernels fed by work queues (k_chain_walk, k_queue_items, k_tracklets_up_p,
// k_down_order, k_tracklets_down_p).  Space-point correction: k_correct_grid
// (S11; the MLP in tpc_mlp.cu).
//
// The method follows the paper's TPC tracking (Sec. 3: cellular-automaton track
// finding derived from the Run 2 HLT tracker, followed by a Kalman fit) under
// the conditions of the Abstract (continuous read-out, no vertex constraint).
// All discrete decisions before the fit are exact integer arithmetic on
// quantised coordinates, so the result does not depend on thread order
// (the ordering and rounding effects discussed in Sec. 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "tpc.h"
#include "tpc_internal.cuh"


namespace {

constexpr float CHI2_CUT = 16.0f;
constexpr float WIN_MIN = 0.5f;
constexpr int MAX_MISS = 5;
constexpr float SIN_MAX = 0.93969262f;  // sin 70 deg: steeper segments are not fitted (Sec. 4)
constexpr float SNP_LIMIT = 0.9999f;
constexpr int MIN_HITS = 10;
constexpr int SHIFT_MIN = 10;
constexpr long long LINK_D = 512;       // 0.5 cm chord deviation
constexpr float INFLATE = 100.0f;       // refit prior: outward variances x100 (at most C0)
constexpr int JOSEPH_UPDATES = 3;       // first updates of a fit done in the Joseph form
constexpr int LINK_THREADS = 256;
constexpr int LINK_MAXC_STAGED = 8;     // the same in k_links (overflow: direct enumeration)
constexpr int LINK_STAGE_MAX = 160 * 1024;  // shared-memory staging of k_links

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan64(unsigned long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan over the block; sm needs 33 ints.  All threads must call it.
__device__ __forceinline__ int block_excl_scan(int v, int* sm, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const int inc = warp_incl_scan(v);
  if (lane == 31) sm[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int s = lane < nw ? sm[lane] : 0;
    const int si = warp_incl_scan(s);
    if (lane < nw) sm[lane] = si - s;
    if (lane == 31) sm[32] = si;
  }
  __syncthreads();
  const int r = sm[w] + inc - v;
  *total = sm[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ unsigned long long block_excl_scan64(unsigned long long v, unsigned long long* sm,
                                                                unsigned long long* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const unsigned long long inc = warp_incl_scan64(v);
  if (lane == 31) sm[w] = inc;
  __syncthreads();
  if (w == 0) {
    const unsigned long long s = lane < nw ? sm[lane] : 0ull;
    const unsigned long long si = warp_incl_scan64(s);
    if (lane < nw) sm[lane] = si - s;
    if (lane == 31) sm[32] = si;
  }
  __syncthreads();
  const unsigned long long r = sm[w] + inc - v;
  *total = sm[32];
  __syncthreads();
  return r;
}

}  // namespace

// ============================================================================ S1
// Quantise and validate; per-(item,row) count and extents.  A CTA handles one
// chunk of one item and aggregates in shared memory first (one global atomic
// per row and statistic per CTA).  rs_min holds four planes: ymin, -ymax, zmin,
// -zmax (atomicMin, initialised to 0x7F7F7F7F).
__global__ void __launch_bounds__(256) k_row_stats(const __grid_constant__ Buffers b) {
  const DevParams& P = b.par;
  __shared__ int s_cnt[TPC_MAX_ROWS], s_min[4][TPC_MAX_ROWS];
  const Chunk ch = b.chunks[blockIdx.x];
  const int NR = P.n_rows;
  const int M = b.I * NR;
  for (int r = threadIdx.x; r < NR; r += blockDim.x) {
    s_cnt[r] = 0;
    s_min[0][r] = s_min[1][r] = s_min[2][r] = s_min[3][r] = 0x7F7F7F7F;
  }
  __syncthreads();
  // one cluster: validation, quantisation (y*1024 is exact in FP32; round half
  // to even), the row's count and extents; returns the key (-1: rejected)
  auto one = [&](float xv, float yv, float zv, int r, int2* q) {
    const bool ok = r >= 0 && r < NR && fabsf(xv) < INFINITY && fabsf(yv) <= 1e6f && fabsf(zv) <= 1e6f;
    if (!ok) {
      atomicOr(b.err, TPC_DERR_BAD_INPUT);
      *q = make_int2(0, 0);
      return -1;
    }
    const int qy = __float2int_rn(yv * TPC_QSCALE);
    const int qz = __float2int_rn(zv * TPC_QSCALE);
    *q = make_int2(qy, qz);
    atomicAdd(&s_cnt[r], 1);
    atomicMin(&s_min[0][r], qy);
    atomicMin(&s_min[1][r], -qy);
    atomicMin(&s_min[2][r], qz);
    atomicMin(&s_min[3][r], -qz);
    return ch.item * NR + r;
  };
  auto scalar = [&](int i) {
    int2 q;
    const int key = one(b.x[i], b.y[i], b.z[i], b.row[i], &q);
    b.cl_key[i] = key;
    if (key >= 0) b.cl_q[i] = q;
  };
  const bool vec = ((reinterpret_cast<uintptr_t>(b.x) | reinterpret_cast<uintptr_t>(b.y) |
                     reinterpret_cast<uintptr_t>(b.z) | reinterpret_cast<uintptr_t>(b.row)) & 15) == 0;
  if (vec) {
    // four consecutive clusters per thread with one 16-byte load per array
    // (and 16-byte stores), the unaligned head and tail of the chunk alone
    const int a4 = min(ch.end, (ch.begin + 3) & ~3), e4 = max(a4, ch.end & ~3);
    for (int i = ch.begin + threadIdx.x; i < a4; i += blockDim.x) scalar(i);
    for (int i = e4 + threadIdx.x; i < ch.end; i += blockDim.x) scalar(i);
    for (int v = a4 + 4 * threadIdx.x; v < e4; v += 4 * blockDim.x) {
      const float4 X = __ldg(reinterpret_cast<const float4*>(b.x + v));
      const float4 Y = __ldg(reinterpret_cast<const float4*>(b.y + v));
      const float4 Z = __ldg(reinterpret_cast<const float4*>(b.z + v));
      const int4 R = __ldg(reinterpret_cast<const int4*>(b.row + v));
      int2 q0, q1, q2, q3;
      const int k0 = one(X.x, Y.x, Z.x, R.x, &q0), k1 = one(X.y, Y.y, Z.y, R.y, &q1);
      const int k2 = one(X.z, Y.z, Z.z, R.z, &q2), k3 = one(X.w, Y.w, Z.w, R.w, &q3);
      *reinterpret_cast<int4*>(b.cl_key + v) = make_int4(k0, k1, k2, k3);
      int4* qv = reinterpret_cast<int4*>(b.cl_q + v);
      qv[0] = make_int4(q0.x, q0.y, q1.x, q1.y);
      qv[1] = make_int4(q2.x, q2.y, q3.x, q3.y);
    }
  } else {
    for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) scalar(i);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < NR; r += blockDim.x) {
    if (s_cnt[r] == 0) continue;
    const int k = ch.item * NR + r;
    atomicAdd(&b.rs_cnt[k], s_cnt[r]);
#pragma unroll
    for (int j = 0; j < 4; ++j) atomicMin(&b.rs_min[j * M + k], s_min[j][r]);
  }
}

// ============================================================================ S2a
// Per row: bin edge 2^s quanta with s the smallest s >= 10 such that
// n*4^s >= Ly*Lz (about one hit per bin) and ny*nz <= 2n+2 (bounded grid).
// Row and bin offsets inside the item come from block scans; the item's bin
// space starts at 2*item_off + 3*n_rows*item (closed form of the bound).
__global__ void __launch_bounds__(256) k_row_setup(const __grid_constant__ Buffers b) {
  const DevParams& P = b.par;
  __shared__ int sm[33];
  const int item = blockIdx.x, NR = P.n_rows, M = b.I * NR;
  const int r = threadIdx.x;
  int n = 0, ymin = 0, zmin = 0, s = SHIFT_MIN, ny = 0, nz = 0;
  if (r < NR) {
    const int k = item * NR + r;
    n = b.rs_cnt[k];
    if (n > 0) {
      ymin = b.rs_min[k];
      const int ymax = -b.rs_min[M + k];
      zmin = b.rs_min[2 * M + k];
      const int zmax = -b.rs_min[3 * M + k];
      const long long dy = (long long)ymax - ymin, dz = (long long)zmax - zmin;
      const long long area = (dy + 1) * (dz + 1);
      const long long need = (area + n - 1) / n;  // n*4^s >= area  <=>  4^s >= ceil(area/n)
      for (;; ++s) {
        const long long nyy = (dy >> s) + 1, nzz = (dz >> s) + 1;
        const bool dense = (2 * s >= 63) || ((1ll << (2 * s)) >= need);
        if (dense && nyy * nzz <= 2ll * n + 2) {
          ny = (int)nyy;
          nz = (int)nzz;
          break;
        }
      }
    }
  }
  const int nb = n > 0 ? ny * nz : 0;
  int tot;
  const int pos_ex = block_excl_scan(n, sm, &tot);
  const int bin_ex = block_excl_scan(r < NR ? nb + 1 : 0, sm, &tot);
  if (r < NR) {
    const long long off = (long long)b.item_off[item];
    RowInfo ri;
    ri.pos0 = (int)off + pos_ex;
    ri.n = n;
    ri.ymin = ymin;
    ri.zmin = zmin;
    ri.shift = s;
    ri.ny = ny;
    ri.nz = nz;
    ri.bin0 = (int)(2 * off) + 3 * NR * item + bin_ex;
    b.rows[item * NR + r] = ri;
  }
}

// ============================================================================ S2b
// Counting sort into row-contiguous order (order inside a row is arbitrary here;
// k_row_sort makes it canonical).  The CTA counts its chunk per row in shared
// memory, reserves one contiguous range per row with a single global atomic, and
// places clusters at local slots inside it.
__global__ void __launch_bounds__(256) k_group_scatter(const __grid_constant__ Buffers b) {
  const DevParams& P = b.par;
  __shared__ int s_cnt[TPC_MAX_ROWS], s_base[TPC_MAX_ROWS];
  const Chunk ch = b.chunks[blockIdx.x];
  const int NR = P.n_rows;
  for (int r = threadIdx.x; r < NR; r += blockDim.x) s_cnt[r] = 0;
  __syncthreads();
  constexpr int PER = 1024 / 256;  // chunks hold <= 1024 clusters
  int key[PER], slot[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int i = ch.begin + threadIdx.x + u * 256;
    key[u] = i < ch.end ? b.cl_key[i] : -1;
    slot[u] = key[u] >= 0 ? atomicAdd(&s_cnt[key[u] - ch.item * NR], 1) : 0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < NR; r += blockDim.x) {
    const int k = ch.item * NR + r;
    s_base[r] = s_cnt[r] ? b.rows[k].pos0 + atomicAdd(&b.row_fill[k], s_cnt[r]) : 0;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    if (key[u] < 0) continue;
    const int i = ch.begin + threadIdx.x + u * 256;
    const int gp = s_base[key[u] - ch.item * NR] + slot[u];
    b.g_q[gp] = b.cl_q[i];
    b.g_id[gp] = i;
  }
}

// ============================================================================ S2c
// One CTA per (item,row).  Rows that fit the dynamic shared-memory budget are
// sorted in shared memory; larger rows use the same code on global scratch
// (tq/tid/tslot) with the row's own first[] entries as the histogram.
// Rows sorted by one warp each (8 rows per CTA, no block barriers): the counting
// sort of k_row_sort below, hits by bin and, inside a bin, by original id, for
// rows whose scratch fits the warp's slice of shared memory (RS_WARP_BYTES);
// larger rows are listed in b.rs_big for k_row_sort.  Empty rows get their one
// bin start here.
// bin of quantised hit q in row ri (y-major cells of 2^shift quanta)
__device__ __forceinline__ int rs_bin(const int2& q, const RowInfo& ri) {
  return ((q.x - ri.ymin) >> ri.shift) * ri.nz + ((q.y - ri.zmin) >> ri.shift);
}

// hits [a, e) of one bin put in original-id order (insertion sort: bins hold a few hits)
__device__ __forceinline__ void rs_bin_sort(int2* q2, int* id2, int a, int e) {
  for (int i = a + 1; i < e; ++i) {
    const int2 qv = q2[i];
    const int iv = id2[i];
    int j = i - 1;
    while (j >= a && id2[j] > iv) {
      q2[j + 1] = q2[j];
      id2[j + 1] = id2[j];
      --j;
    }
    q2[j + 1] = qv;
    id2[j + 1] = iv;
  }
}

constexpr int RS_WARPS = 8;
constexpr int RS_WARP_BYTES = 4096;

__device__ __forceinline__ bool rs_fits_warp(int n, int nb) { return 16ll * n + 4ll * (nb + 1) <= RS_WARP_BYTES; }

__global__ void __launch_bounds__(32 * RS_WARPS) k_row_sort_warp(const __grid_constant__ Buffers b, int M) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * RS_WARPS + w;
  if (k >= M) return;  // warp-uniform
  const RowInfo ri = b.rows[k];
  const int n = ri.n;
  if (n == 0) {
    if (lane == 0) b.first[ri.bin0] = ri.pos0;
    return;
  }
  const int nb = ri.ny * ri.nz;
  if (!rs_fits_warp(n, nb)) {
    if (lane == 0) b.rs_big[atomicAdd(b.rs_big + M, 1)] = k;
    return;
  }
  int2* q2 = reinterpret_cast<int2*>(smem_raw + (size_t)w * RS_WARP_BYTES);
  int* id2 = reinterpret_cast<int*>(q2 + n);
  int* slot = id2 + n;
  int* hist = slot + n;
  for (int j = lane; j <= nb; j += 32) hist[j] = 0;
  __syncwarp();
  for (int j = lane; j < n; j += 32) slot[j] = atomicAdd(&hist[rs_bin(b.g_q[ri.pos0 + j], ri)], 1);
  __syncwarp();
  int carry = 0;  // exclusive scan of hist[0..nb], 32 entries at a time
  for (int j0 = 0; j0 <= nb; j0 += 32) {
    const int j = j0 + lane;
    const int v = j <= nb ? hist[j] : 0;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (j <= nb) hist[j] = carry + inc - v;
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();
  for (int j = lane; j < n; j += 32) {
    const int2 q = b.g_q[ri.pos0 + j];
    const int p = hist[rs_bin(q, ri)] + slot[j];
    q2[p] = q;
    id2[p] = b.g_id[ri.pos0 + j];
  }
  __syncwarp();
  for (int bin = lane; bin < nb; bin += 32) rs_bin_sort(q2, id2, hist[bin], hist[bin + 1]);
  __syncwarp();
  for (int j = lane; j < n; j += 32) b.s_hit[ri.pos0 + j] = make_int4(q2[j].x, q2[j].y, id2[j], k);
  for (int j = lane; j <= nb; j += 32) b.first[ri.bin0 + j] = ri.pos0 + hist[j];
}

// The same sort by a CTA per row: every row (listed = 0, one CTA each), or the
// rows listed by k_row_sort_warp (listed = 1, a grid-stride loop over the
// list).  Scratch in shared memory when it fits `smem_bytes`, else in the
// global scratch arrays tq, tid_buf, tslot at the row's positions.
__global__ void __launch_bounds__(128) k_row_sort(const __grid_constant__ Buffers b, int smem_bytes, int2* tq, int* tid_buf, int* tslot, int M, int listed) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sm[33];
  const int n_here = listed ? b.rs_big[M] : M;
  for (int ib = blockIdx.x; ib < n_here; ib += gridDim.x) {  // block-uniform loop
    const int k = listed ? b.rs_big[ib] : ib;
    const RowInfo ri = b.rows[k];
    const int n = ri.n;
    if (n == 0) {  // (rows of the unlisted form only)
      if (threadIdx.x == 0) b.first[ri.bin0] = ri.pos0;
      continue;
    }
    const int nb = ri.ny * ri.nz;
    const long long need = 12ll * n + 4ll * n + 4ll * (nb + 1);
    int2* q2;
    int* id2;
    int* slot;
    int* hist;
    if (need <= smem_bytes) {
      q2 = reinterpret_cast<int2*>(smem_raw);
      id2 = reinterpret_cast<int*>(q2 + n);
      slot = id2 + n;
      hist = slot + n;
    } else {
      q2 = tq + ri.pos0;
      id2 = tid_buf + ri.pos0;
      slot = tslot + ri.pos0;
      hist = b.first + ri.bin0;
    }
    for (int j = threadIdx.x; j <= nb; j += blockDim.x) hist[j] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) slot[j] = atomicAdd(&hist[rs_bin(b.g_q[ri.pos0 + j], ri)], 1);
    __syncthreads();
    // exclusive scan of hist[0..nb] in place, chunk by chunk
    int carry = 0;
    for (int base = 0; base <= nb; base += blockDim.x) {
      const int j = base + threadIdx.x;
      const int v = j <= nb ? hist[j] : 0;
      int tot;
      const int ex = block_excl_scan(v, sm, &tot);
      if (j <= nb) hist[j] = carry + ex;
      carry += tot;
      __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int2 q = b.g_q[ri.pos0 + j];
      const int p = hist[rs_bin(q, ri)] + slot[j];
      q2[p] = q;
      id2[p] = b.g_id[ri.pos0 + j];
    }
    __syncthreads();
    // canonical order inside a bin: original id
    for (int bin = threadIdx.x; bin < nb; bin += blockDim.x) rs_bin_sort(q2, id2, hist[bin], hist[bin + 1]);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) b.s_hit[ri.pos0 + j] = make_int4(q2[j].x, q2[j].y, id2[j], k);
    if (hist != b.first + ri.bin0) {
      for (int j = threadIdx.x; j <= nb; j += blockDim.x) b.first[ri.bin0 + j] = ri.pos0 + hist[j];
    } else {
      __syncthreads();
      for (int j = threadIdx.x; j <= nb; j += blockDim.x) b.first[ri.bin0 + j] += ri.pos0;
    }
    __syncthreads();  // the scratch is reused by the next listed row
  }
}

// ============================================================================ S3
namespace {
// bin range of [lo, hi] along one axis; empty if hi < lo
__device__ __forceinline__ void bin_range(long long lo, long long hi, int vmin, int shift, int nbin, int* a,
                                          int* e) {
  if (hi < vmin || nbin == 0) {
    *a = 0;
    *e = -1;
    return;
  }
  const long long vmax = (long long)vmin + ((long long)nbin << shift) - 1;
  if (lo > vmax) {
    *a = 0;
    *e = -1;
    return;
  }
  *a = lo <= vmin ? 0 : (int)((lo - vmin) >> shift);
  const long long t = (hi - vmin) >> shift;
  *e = t < nbin - 1 ? (int)t : nbin - 1;
}
}  // namespace

// For every hit h of an inner row: the pair (u on r+1, d on r-1) inside the
// windows |dqy| <= 11*dqx/4, |dqz| <= 16*dqx/5 that minimises m = dY^2 + dZ^2,
// dY = (qy_u-qy_h)*dx_dn - (qy_h-qy_d)*dx_up (int64), accepted if
// m <= ((dx_up+dx_dn)*512)^2; ties: smaller id_u, then smaller id_d.  Rows 0 and
// n_rows-1 get no links (targets only).
namespace {
// Sorted hits and bin index entries, read from global memory or from the rows
// of one item staged in shared memory (positions offset by p_lo, bins by f_lo).
struct GlobalSrc {
  const int4* h;
  const int* f;
  __device__ __forceinline__ int4 hit(int p) const { return h[p]; }
  __device__ __forceinline__ int first(int i) const { return f[i]; }
};

struct StageSrc {
  const int2* q;   // (qy, qz)
  const int* id;   // original id
  const int* f;
  int p_lo, f_lo;
  __device__ __forceinline__ int4 hit(int p) const {
    const int2 v = q[p - p_lo];
    return make_int4(v.x, v.y, id[p - p_lo], 0);
  }
  __device__ __forceinline__ int first(int i) const { return f[i - f_lo]; }
};

// m of one (u, d) pair given the window offsets ey = qy_u - qy_h, ez, fy =
// qy_h - qy_d, fz; false if m > cut^2.  With W32 the factors are 32-bit integers
// (exact for a row pitch of at most 2^14 quanta, checked on the host) squared by
// widening multiplies; |dY| > cut or |dZ| > cut already implies m > cut^2.
template <bool W32>
__device__ __forceinline__ bool link_metric(int ey, int ez, int fy, int fz, int dxu, int dxd, long long cut,
                                            long long cut2, long long* m) {
  if constexpr (W32) {
    const int dY = ey * dxd - fy * dxu;
    const int dZ = ez * dxd - fz * dxu;
    if (dY > cut || -dY > cut || dZ > cut || -dZ > cut) return false;
    *m = (long long)dY * dY + (long long)dZ * dZ;
  } else {
    const long long dY = (long long)ey * dxd - (long long)fy * dxu;
    const long long dZ = (long long)ez * dxd - (long long)fz * dxu;
    *m = dY * dY + dZ * dZ;
  }
  return *m <= cut2;
}

// Neighbour search of one hit at sorted position pos on inner row r of an item
// (rows[r - lo] is row r): the window candidates of each side go to this
// thread's lists s_cu / s_cd (MAXC entries), then every pair is scored; with
// more candidates than the lists hold, the pairs are enumerated directly.
template <int W, int MAXC, bool W32, class Src>
__device__ __forceinline__ void link_hit(const Buffers& b, const Src& S, const RowInfo* rows, int lo, int pos,
                                         int4 qh, int r, int (*s_cu)[W], int (*s_cd)[W], int t) {
  const DevParams& P = b.par;
  const RowInfo U = rows[r + 1 - lo], D = rows[r - 1 - lo];
  const int dxu = P.qx[r + 1] - P.qx[r];
  const int dxd = P.qx[r] - P.qx[r - 1];
  const int wyu = dxu * 11 / 4, wzu = dxu * 16 / 5;
  const int wyd = dxd * 11 / 4, wzd = dxd * 16 / 5;
  const long long cut = (long long)(dxu + dxd) * LINK_D;
  const long long cut2 = cut * cut;
  const int yh = qh.x, zh = qh.y;
  int uy0, uy1, uz0, uz1, dy0, dy1, dz0, dz1;
  bin_range((long long)yh - wyu, (long long)yh + wyu, U.ymin, U.shift, U.ny, &uy0, &uy1);
  bin_range((long long)zh - wzu, (long long)zh + wzu, U.zmin, U.shift, U.nz, &uz0, &uz1);
  bin_range((long long)yh - wyd, (long long)yh + wyd, D.ymin, D.shift, D.ny, &dy0, &dy1);
  bin_range((long long)zh - wzd, (long long)zh + wzd, D.zmin, D.shift, D.nz, &dz0, &dz1);
  // candidates of each side: hits inside the window, from one contiguous hit
  // range per y-bin row (the z-bins of a y-bin row are adjacent)
  int nu = 0, nd = 0;
  bool ovf = false;
  if (uz1 >= uz0 && dz1 >= dz0) {
    for (int iy = uy0; iy <= uy1; ++iy) {
      const int b0 = U.bin0 + iy * U.nz + uz0;
      const int e_ = S.first(b0 + uz1 - uz0 + 1);
      for (int pu = S.first(b0); pu < e_; ++pu) {
        const int4 q = S.hit(pu);
        const int ey = q.x - yh, ez = q.y - zh;
        if (ey > wyu || -ey > wyu || ez > wzu || -ez > wzu) continue;
        if (nu < MAXC) s_cu[nu++][t] = pu; else ovf = true;
      }
    }
    if (nu > 0)
      for (int iy = dy0; iy <= dy1; ++iy) {
        const int b0 = D.bin0 + iy * D.nz + dz0;
        const int e_ = S.first(b0 + dz1 - dz0 + 1);
        for (int pd = S.first(b0); pd < e_; ++pd) {
          const int4 q = S.hit(pd);
          const int fy = yh - q.x, fz = zh - q.y;
          if (fy > wyd || -fy > wyd || fz > wzd || -fz > wzd) continue;
          if (nd < MAXC) s_cd[nd++][t] = pd; else ovf = true;
        }
      }
  }
  long long best = -1;
  int bu = -1, bd = -1, bid_u = 0, bid_d = 0;
  auto pair = [&](int pu, const int4& qu, int pd, const int4& qd) {
    long long m;
    if (!link_metric<W32>(qu.x - yh, qu.y - zh, yh - qd.x, zh - qd.y, dxu, dxd, cut, cut2, &m)) return;
    bool better = best < 0 || m < best;
    if (!better && m == best) better = qu.z < bid_u || (qu.z == bid_u && qd.z < bid_d);
    if (better) {
      best = m;
      bu = pu;
      bd = pd;
      bid_u = qu.z;
      bid_d = qd.z;
    }
  };
  if (!ovf) {
    for (int iu = 0; iu < nu; ++iu) {
      const int pu = s_cu[iu][t];
      const int4 qu = S.hit(pu);
      for (int id = 0; id < nd; ++id) {
        const int pd = s_cd[id][t];
        pair(pu, qu, pd, S.hit(pd));
      }
    }
  } else {
    // more candidates than the lists hold (very dense rows): direct enumeration
    for (int iy = uy0; iy <= uy1; ++iy) {
      const int bu0 = U.bin0 + iy * U.nz + uz0;
      const int ue = S.first(bu0 + uz1 - uz0 + 1);
      for (int pu = S.first(bu0); pu < ue; ++pu) {
        const int4 qu = S.hit(pu);
        const int ey = qu.x - yh, ez = qu.y - zh;
        if (ey > wyu || -ey > wyu || ez > wzu || -ez > wzu) continue;
        for (int jy = dy0; jy <= dy1; ++jy) {
          const int bd0 = D.bin0 + jy * D.nz + dz0;
          const int de = S.first(bd0 + dz1 - dz0 + 1);
          for (int pd = S.first(bd0); pd < de; ++pd) {
            const int4 qd = S.hit(pd);
            const int fy = yh - qd.x, fz = zh - qd.y;
            if (fy > wyd || -fy > wyd || fz > wzd || -fz > wzd) continue;
            pair(pu, qu, pd, qd);
          }
        }
      }
    }
  }
  b.up_raw[pos] = bu;
  b.dn_raw[pos] = bd;
}
}  // namespace

// One CTA per block of `rows_per_cta` consecutive rows of one item (their hits
// are contiguous in sorted order, so the threads take a flat range of them).
// The block's rows and the rows on either side are staged in shared memory
// (sorted hits and bin index, at most `stage_bytes`); a block that does not fit
// reads global memory instead.
template <bool W32>
__global__ void __launch_bounds__(LINK_THREADS) k_links(const __grid_constant__ Buffers b, int rows_per_cta,
                                                        int stage_bytes) {
  const DevParams& P = b.par;
  extern __shared__ int2 s_stage[];
  __shared__ RowInfo s_rows[TPC_MAX_ROWS + 2];
  __shared__ int s_cu[LINK_MAXC_STAGED][LINK_THREADS], s_cd[LINK_MAXC_STAGED][LINK_THREADS];
  const int NR = P.n_rows;
  const int nrb = (NR + rows_per_cta - 1) / rows_per_cta;
  const int item = blockIdx.x / nrb;
  const int r_begin = (blockIdx.x - item * nrb) * rows_per_cta;
  const int r_end = min(NR, r_begin + rows_per_cta);
  const int lo = max(0, r_begin - 1), hi = min(NR - 1, r_end);
  for (int r = lo + threadIdx.x; r <= hi; r += blockDim.x) s_rows[r - lo] = b.rows[item * NR + r];
  __syncthreads();
  const int p_begin = s_rows[r_begin - lo].pos0;
  const int p_end = s_rows[r_end - 1 - lo].pos0 + s_rows[r_end - 1 - lo].n;
  const RowInfo& rl = s_rows[0];
  const RowInfo& rh = s_rows[hi - lo];
  const int p_lo = rl.pos0, p_hi = rh.pos0 + rh.n;
  const int f_lo = rl.bin0, f_hi = rh.bin0 + (rh.n > 0 ? rh.ny * rh.nz : 0) + 1;
  const int nh = p_hi - p_lo, nf = f_hi - f_lo;
  // staged layout: (qy, qz) int2 [nh], id int [nh], bin index int [nf]
  const bool staged = (long long)nh * 12 + (long long)nf * 4 <= stage_bytes;
  int* sid = reinterpret_cast<int*>(s_stage + (staged ? nh : 0));
  int* sf = sid + (staged ? nh : 0);
  if (staged) {
    for (int i = threadIdx.x; i < nh; i += blockDim.x) {
      const int4 v = __ldg(b.s_hit + p_lo + i);
      s_stage[i] = make_int2(v.x, v.y);
      sid[i] = v.z;
    }
    for (int i = threadIdx.x; i < nf; i += blockDim.x) sf[i] = __ldg(b.first + f_lo + i);
  }
  __syncthreads();
  const int t = threadIdx.x;
  const StageSrc SS{s_stage, sid, sf, p_lo, f_lo};
  const GlobalSrc GS{b.s_hit, b.first};
  for (int pos = p_begin + t; pos < p_end; pos += blockDim.x) {
    const int4 qh = __ldg(b.s_hit + pos);
    const int r = qh.w - item * NR;
    if (r == 0 || r == NR - 1) {
      b.up_raw[pos] = -1;
      b.dn_raw[pos] = -1;
      continue;
    }
    if (staged)
      link_hit<LINK_THREADS, LINK_MAXC_STAGED, W32>(b, SS, s_rows, lo, pos, qh, r, s_cu, s_cd, t);
    else
      link_hit<LINK_THREADS, LINK_MAXC_STAGED, W32>(b, GS, s_rows, lo, pos, qh, r, s_cu, s_cd, t);
  }
}

// ============================================================================ S4+S5
// Mutual links only (reads the raw arrays only); start hit = clean up link, no
// clean down link, chain of >= 3 hits.
__global__ void __launch_bounds__(256) k_clean_start(const __grid_constant__ Buffers b) {
  for (int pos = blockIdx.x * blockDim.x + threadIdx.x; pos < b.N; pos += gridDim.x * blockDim.x) {
    const int u = b.up_raw[pos], d = b.dn_raw[pos];
    const int cu = (u >= 0 && b.dn_raw[u] == pos) ? u : -1;
    const int cd = (d >= 0 && b.up_raw[d] == pos) ? d : -1;
    b.up[pos] = cu;
    b.dn[pos] = cd;
    int start = 0;
    if (cu >= 0 && cd < 0) {
      const int u2 = b.up_raw[cu];
      start = (u2 >= 0 && b.dn_raw[u2] == cu) ? 1 : 0;
    }
    b.flags[pos] = start;
  }
}

// ============================================================================ scans
// Reduce-then-scan over n values (n from the host or from a device word) with a
// fixed grid: block g owns a contiguous range; bsum gets per-block totals.
template <typename T>
__global__ void __launch_bounds__(256) k_scan_reduce(const T* in, const int* n_dev, long long n_host, T* bsum) {
  const long long n = n_dev ? (long long)*n_dev : n_host;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long a = blockIdx.x * per, e = a + per < n ? a + per : n;
  T s = 0;
  for (long long i = a + threadIdx.x; i < e; i += blockDim.x) s += in[i];
  __shared__ T red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = red[0];
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_bsums(T* bsum, int nb) {
  // nb <= 1024: one element per thread; exclusive, total in bsum[nb]
  __shared__ T sm[1024];
  const int t = threadIdx.x;
  sm[t] = t < nb ? bsum[t] : 0;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const T v = t >= o ? sm[t - o] : 0;
    __syncthreads();
    sm[t] += v;
    __syncthreads();
  }
  if (t < nb) bsum[t] = t ? sm[t - 1] : 0;
  if (t == nb - 1) bsum[nb] = sm[t];
}

__global__ void __launch_bounds__(256) k_scan_final_i32(const int* in, int* out, const int* n_dev, long long n_host,
                                                        const unsigned long long* bsum) {
  __shared__ int sm[33];
  const long long n = n_dev ? (long long)*n_dev : n_host;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long a = blockIdx.x * per, e = a + per < n ? a + per : n;
  int carry = (int)bsum[blockIdx.x];
  for (long long base = a; base < e; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    const int v = i < e ? in[i] : 0;
    int tot;
    const int ex = block_excl_scan(v, sm, &tot);
    if (i < e) out[i] = carry + ex;
    carry += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (int)bsum[gridDim.x];
}

__global__ void __launch_bounds__(256) k_scan_final_u64(const unsigned long long* in, unsigned long long* out,
                                                        const int* n_dev, long long n_host,
                                                        const unsigned long long* bsum) {
  __shared__ unsigned long long sm[33];
  const long long n = n_dev ? (long long)*n_dev : n_host;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long a = blockIdx.x * per, e = a + per < n ? a + per : n;
  unsigned long long carry = bsum[blockIdx.x];
  for (long long base = a; base < e; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    const unsigned long long v = i < e ? in[i] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan64(v, sm, &tot);
    if (i < e) out[i] = carry + ex;
    carry += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = bsum[gridDim.x];
}

// int flags summed into 64-bit block sums
__global__ void __launch_bounds__(256) k_scan_reduce_i32(const int* in, long long n, unsigned long long* bsum) {
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long a = blockIdx.x * per, e = a + per < n ? a + per : n;
  unsigned long long s = 0;
  for (long long i = a + threadIdx.x; i < e; i += blockDim.x) s += (unsigned long long)in[i];
  __shared__ unsigned long long red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = red[0];
}

template __global__ void k_scan_reduce<unsigned long long>(const unsigned long long*, const int*, long long,
                                                           unsigned long long*);
template __global__ void k_scan_bsums<unsigned long long>(unsigned long long*, int);

__global__ void __launch_bounds__(256) k_starts(const __grid_constant__ Buffers b) {
  for (int pos = blockIdx.x * blockDim.x + threadIdx.x; pos < b.N; pos += gridDim.x * blockDim.x)
    if (b.flags[pos]) b.starts[b.start_ex[pos]] = pos;
}

// ============================================================================ S6
namespace {
// packed lower triangle index
__device__ __forceinline__ constexpr int ix(int i, int j) { return i * (i + 1) / 2 + j; }

// a*b + c*d with the rounding fixed (the first product fused, the second
// rounded): left to itself the compiler may fuse either product, and its choice
// can differ between the kernels this code is inlined into.
__device__ __forceinline__ float fma2(float a, float b, float c, float d) { return __fmaf_rn(a, b, __fmul_rn(c, d)); }

// square root of x > 0 from the hardware reciprocal square root (a few ulp;
// one multiply instead of the correctly rounded sequence)
__device__ __forceinline__ float sqrt_pos(float x) { return x * rsqrtf(x); }

__device__ __forceinline__ float asin_over_u(float u) {
  if (fabsf(u) < 0.1f) {
    const float u2 = u * u;
    return 1.0f + u2 * (1.0f / 6.0f + u2 * (3.0f / 40.0f + u2 * (5.0f / 112.0f)));
  }
  return asinf(u) / u;
}

__device__ __forceinline__ float d_asin_over_u(float u) {
  if (fabsf(u) < 0.1f) {
    const float u2 = u * u;
    return u * (1.0f / 3.0f + u2 * (3.0f / 10.0f + u2 * (15.0f / 56.0f + u2 * (35.0f / 144.0f))));
  }
  return (u / sqrtf(1.0f - u * u) - asinf(u)) / (u * u);
}

// Helix step of (y, z, sinphi, tanlambda, q/pT) and covariance transport C <- F C F^T.
// F differs from the identity in F02, F04, F12, F13, F14, F24 only.
struct Jac {
  float a, bq, c, d, e, g;  // F02, F04, F12, F13, F14, F24
};

__device__ __forceinline__ bool kf_step_state(const DevParams& P, float* p, float x1, float x2, Jac* J) {
  const float kB = P.kB;
  const float dx = x2 - x1;
  const float s1 = p[2];
  const float kappa = kB * p[4];
  const float s2 = s1 - kappa * dx;
  if (!(fabsf(s1) < SNP_LIMIT) || !(fabsf(s2) < SNP_LIMIT)) return false;
  const float c1 = sqrt_pos((1.0f - s1) * (1.0f + s1));
  const float c2 = sqrt_pos((1.0f - s2) * (1.0f + s2));
  // fast reciprocals (2 ulp): the Jacobian only feeds the covariance
  const float cc = c1 + c2;
  const float inv_cc = __fdividef(1.0f, cc);
  const float T = (s1 + s2) * inv_cc;
  const float w = sqrt_pos(1.0f + T * T);
  const float adx = fabsf(dx);
  const float u = 0.5f * kappa * adx * w;
  if (!(fabsf(u) < 1.0f)) return false;
  const float f = asin_over_u(u);
  const float fp = d_asin_over_u(u);
  const float ell = dx * w * f;
  const float A = (1.0f + c1 * c2 + s1 * s2) * inv_cc * inv_cc;
  const float A1 = __fdividef(A, c1), A2 = __fdividef(A, c2);
  const float dT_ds = A1 + A2;
  const float dT_dq = -A2 * kB * dx;
  const float dg_dT = __fdividef(T, w) * (f + u * fp);
  const float dg_dk = 0.5f * w * w * adx * fp;
  const float tgl = p[3];
  J->a = dx * dT_ds;                                  // F02
  J->bq = dx * dT_dq;                                 // F04
  J->c = tgl * dx * dg_dT * dT_ds;                    // F12
  J->d = ell;                                         // F13
  J->e = tgl * dx * fma2(dg_dT, dT_dq, dg_dk, kB);    // F14
  J->g = -kB * dx;                                    // F24
  p[0] += dx * T;
  p[1] += tgl * ell;
  p[2] = s2;
  return true;
}

__device__ __forceinline__ void kf_transport(float* C, const Jac& J) {
  const float a = J.a, bq = J.bq, c = J.c, d = J.d, e = J.e, g = J.g;
  // full symmetric copy
  float M[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      M[i][j] = C[ix(i, j)];
      M[j][i] = C[ix(i, j)];
    }
  // v_j = C F_j^T for the three non-trivial rows of F
  float v0[5], v1[5], v2[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    v0[i] = M[i][0] + a * M[i][2] + bq * M[i][4];
    v1[i] = M[i][1] + c * M[i][2] + d * M[i][3] + e * M[i][4];
    v2[i] = M[i][2] + g * M[i][4];
  }
  C[ix(0, 0)] = v0[0] + a * v0[2] + bq * v0[4];
  C[ix(1, 0)] = v0[1] + c * v0[2] + d * v0[3] + e * v0[4];
  C[ix(1, 1)] = v1[1] + c * v1[2] + d * v1[3] + e * v1[4];
  C[ix(2, 0)] = v0[2] + g * v0[4];
  C[ix(2, 1)] = v1[2] + g * v1[4];
  C[ix(2, 2)] = v2[2] + g * v2[4];
  C[ix(3, 0)] = v0[3];
  C[ix(3, 1)] = v1[3];
  C[ix(3, 2)] = v2[3];
  C[ix(4, 0)] = v0[4];
  C[ix(4, 1)] = v1[4];
  C[ix(4, 2)] = v2[4];
  // (3,3), (4,3), (4,4) unchanged
}

__device__ __forceinline__ bool kf_propagate(const DevParams& P, float* p, float* C, float x1, float x2) {
  Jac J;
  if (!kf_step_state(P, p, x1, x2, &J)) return false;
  kf_transport(C, J);
  return true;
}

// Search window of the predicted state: the innovation covariance S = C_yz + V,
// its inverse determinant and the half-widths max(0.5 cm, 4 sqrt(S_ii)).
struct Win {
  float S00, S01, S11, inv_det, wy, wz;
};

__device__ __forceinline__ Win make_win(const DevParams& P, const float* C) {
  Win w;
  w.S00 = C[ix(0, 0)] + P.vy;
  w.S01 = C[ix(1, 0)];
  w.S11 = C[ix(1, 1)] + P.vz;
  w.inv_det = 1.0f / fma2(w.S00, w.S11, -w.S01, w.S01);
  // window only: the 2-quantum margin of the box covers the approximation
  w.wy = fmaxf(WIN_MIN, 4.0f * sqrt_pos(w.S00));
  w.wz = fmaxf(WIN_MIN, 4.0f * sqrt_pos(w.S11));
  return w;
}

// Kalman update with H = [I2 0] and the innovation covariance of `w` (made
// from the same predicted C); residuals (r0, r1); returns the chi2 increment.
__device__ __forceinline__ float kf_update(const Win& w, float* p, float* C, float r0, float r1) {
  const float I00 = w.S11 * w.inv_det, I01 = -w.S01 * w.inv_det, I11 = w.S00 * w.inv_det;
  // columns 0 and 1 of the symmetric covariance
  float c0[5], c1[5], K0[5], K1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) c0[i] = C[ix(i, 0)];
  c1[0] = C[ix(1, 0)];
#pragma unroll
  for (int i = 1; i < 5; ++i) c1[i] = C[ix(i, 1)];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    K0[i] = fma2(c0[i], I00, c1[i], I01);
    K1[i] = fma2(c0[i], I01, c1[i], I11);
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] += fma2(K0[i], r0, K1[i], r1);
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) C[ix(i, j)] -= fma2(K0[i], c0[j], K1[i], c1[j]);
  return fma2(r0, fma2(I00, r0, I01, r1), r1, fma2(I01, r0, I11, r1));
}

// The same update with the covariance in the Joseph form
//   C <- (I - K H) C (I - K H)^T + K V K^T,   V = diag(vy, vz):
// algebraically equal to kf_update's C - K H C, but a sum of symmetric
// positive terms instead of a difference.  A fit that starts from C0 (angle
// variances 1, q/pT variance 100 against 0.01 cm^2 measurements) cancels most
// digits of the small covariance entries in its first updates: in FP32 the
// difference form lost up to 4% in q/pT on short low-pT tracks refitted from
// C0, this form keeps them within 1e-3 of the FP64 filter.  Every product and
// sum is an explicit fused operation, so every kernel that inlines this
// rounds alike.
__device__ __forceinline__ float kf_update_joseph(const Win& w, float vy, float vz, float* p, float* C, float r0,
                                                  float r1) {
  const float I00 = w.S11 * w.inv_det, I01 = -w.S01 * w.inv_det, I11 = w.S00 * w.inv_det;
  float M[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      M[i][j] = C[ix(i, j)];
      M[j][i] = C[ix(i, j)];
    }
  float K0[5], K1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    K0[i] = fma2(M[i][0], I00, M[i][1], I01);
    K1[i] = fma2(M[i][0], I01, M[i][1], I11);
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] += fma2(K0[i], r0, K1[i], r1);
  // T = (I - K H) C (rows 0..4; columns 0, 1 and the lower triangle are used)
  float T[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) T[i][j] = __fmaf_rn(-K0[i], M[0][j], __fmaf_rn(-K1[i], M[1][j], M[i][j]));
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float a0 = __fmul_rn(vy, K0[i]), a1 = __fmul_rn(vz, K1[i]);
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float v = __fmaf_rn(-T[i][0], K0[j], T[i][j]);
      v = __fmaf_rn(-T[i][1], K1[j], v);
      v = __fmaf_rn(a0, K0[j], v);
      C[ix(i, j)] = __fmaf_rn(a1, K1[j], v);
    }
  }
  return fma2(r0, fma2(I00, r0, I01, r1), r1, fma2(I01, r0, I11, r1));
}

__device__ __forceinline__ bool cov_ok(const float* C) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 15; ++i) ok &= fabsf(C[i]) < INFINITY;
  ok &= C[ix(0, 0)] > 0.f && C[ix(1, 1)] > 0.f && C[ix(2, 2)] > 0.f && C[ix(3, 3)] > 0.f && C[ix(4, 4)] > 0.f;
  return ok;
}

__device__ __forceinline__ void set_c0(const DevParams& P, float* C) {
#pragma unroll
  for (int i = 0; i < 15; ++i) C[i] = 0.f;
  C[ix(0, 0)] = P.vy;
  C[ix(1, 1)] = P.vz;
  C[ix(2, 2)] = 1.0f;
  C[ix(3, 3)] = 1.0f;
  C[ix(4, 4)] = 100.0f;
}

// Group helpers: a tracklet is handled by a group of G consecutive lanes
// (G = 1, 2, 4, 8, 16 or 32).  All lanes of a group hold the same state and take
// the same branches; they split the chain loads and the hit search of a row.
template <int G>
struct Grp {
  int gl;        // lane inside the group
  unsigned mask; // lanes of the group
  __device__ __forceinline__ Grp() {
    const int lane = threadIdx.x & 31;
    gl = lane & (G - 1);
    mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  }
  template <class T>
  __device__ __forceinline__ T shfl(T v, int src) const {
    if constexpr (G == 1) return v;
    else return __shfl_sync(mask, v, src, G);
  }
  __device__ __forceinline__ int incl_scan(int v) const {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const int t = __shfl_up_sync(mask, v, o, G);
      if (gl >= o) v += t;
    }
    return v;
  }
  // minimum of a 64-bit key over the group: two warp reductions (high word,
  // then low word among the lanes holding the smallest high word)
  __device__ __forceinline__ unsigned long long min64(unsigned long long v) const {
    if constexpr (G == 1) {
      return v;
    } else {
      const unsigned hi = __reduce_min_sync(mask, (unsigned)(v >> 32));
      const unsigned lo = __reduce_min_sync(mask, (unsigned)(v >> 32) == hi ? (unsigned)v : 0xFFFFFFFFu);
      return ((unsigned long long)hi << 32) | lo;
    }
  }
  __device__ __forceinline__ void sync() const {
    if constexpr (G > 1) __syncwarp(mask);
  }
};

// Read-only loads: through the non-coherent path where the data was written by
// an earlier launch (NC = true); plain loads for data of the same launch and
// for shared memory.
template <bool NC, class T>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

template <bool NC>
__device__ __forceinline__ RowInfo load_row(const RowInfo* p) {
  if constexpr (NC) {
    const int4 a = __ldg(reinterpret_cast<const int4*>(p));
    const int4 c = __ldg(reinterpret_cast<const int4*>(p) + 1);
    RowInfo r;
    r.pos0 = a.x;
    r.n = a.y;
    r.ymin = a.z;
    r.zmin = a.w;
    r.shift = c.x;
    r.ny = c.y;
    r.nz = c.z;
    r.bin0 = c.w;
    return r;
  } else {
    return *p;
  }
}

// Where a tracklet reads its item's row table, bin index, sorted hits and clean
// up-links.  `r` is the pad row of the position read (unused by these global
// sources; a source that splits an item's rows over several places needs it).
template <bool NC>
struct GSrc {  // global memory; NC: data written by an earlier launch
  // candidates per round of the single-lane search
  static constexpr int kRound = 8;
  const Buffers* b;
  const RowInfo* rows;  // the item's row table (global, or shared memory)
  __device__ __forceinline__ RowInfo row(int r) const { return load_row<NC>(rows + r); }
  __device__ __forceinline__ int first(int, int f) const { return ld<NC>(b->first + f); }
  __device__ __forceinline__ int4 hit(int, int p) const { return ld<NC>(b->s_hit + p); }
  __device__ __forceinline__ int up(int, int p) const { return ld<NC>(b->up + p); }
};


// Bins [iy0, iy1] x [iz0, iz1] of a row's grid covered by the box
// yc +- wy, zc +- wz (cm, z relative to z_base) widened by 2 quanta; empty
// (iy1 < iy0 or iz1 < iz0) if it misses the grid or the row has no hits.
struct Box {
  int iy0, iy1, iz0, iz1;
  int qy0, qy1, qz0, qz1;  // the box itself in quanta (absolute z)
};

__device__ __forceinline__ Box row_box(const RowInfo& ri, float yc, float zc, float wy, float wz, int z_base) {
  Box x;
  // 32-bit conversions (values clamped to +-1e9): 64-bit ones run on the FP64 pipe
  const float lim = 1.0e9f;
  const long long ylo = (long long)(int)floorf(fmaxf(-lim, (yc - wy) * TPC_QSCALE)) - 2;
  const long long yhi = (long long)(int)ceilf(fminf(lim, (yc + wy) * TPC_QSCALE)) + 2;
  const long long zlo = (long long)(int)floorf(fmaxf(-lim, (zc - wz) * TPC_QSCALE)) - 2 + z_base;
  const long long zhi = (long long)(int)ceilf(fminf(lim, (zc + wz) * TPC_QSCALE)) + 2 + z_base;
  bin_range(ylo, yhi, ri.ymin, ri.shift, ri.ny, &x.iy0, &x.iy1);
  bin_range(zlo, zhi, ri.zmin, ri.shift, ri.nz, &x.iz0, &x.iz1);
  if (ri.n == 0) x.iy1 = -1;
  // within int range: |float bounds| <= 1e9 + 2 quanta, |z_base| < 1.03e9
  x.qy0 = (int)ylo;
  x.qy1 = (int)yhi;
  x.qz0 = (int)zlo;
  x.qz1 = (int)zhi;
  return x;
}

__device__ __forceinline__ bool box_empty(const Box& x) { return x.iy1 < x.iy0 || x.iz1 < x.iz0; }

// chi2 of hit q against the predicted (y, z) = (p[0], p[1]); the selection key
// (chi2 bit pattern, original id) if chi2 <= 16, else ~0.
__device__ __forceinline__ unsigned long long hit_key(const int4& q, const float* p, const Win& w, int z_base) {
  const float Q = 1.0f / TPC_QSCALE;
  const float dy = (float)q.x * Q - p[0];
  const float dz = (float)(q.y - z_base) * Q - p[1];
  const float quad = __fmaf_rn(w.S00 * dz, dz, fma2(w.S11 * dy, dy, -2.0f * w.S01 * dy, dz));
  const float chi2 = fmaxf(0.0f, quad * w.inv_det);
  return chi2 <= CHI2_CUT ? ((unsigned long long)__float_as_uint(chi2) << 32) | (unsigned)q.z : ~0ull;
}

// Best hit of the row described by `ri` inside box `bx` for the predicted
// state: the smallest chi2 <= 16, ties to the smaller original id (a 64-bit key
// of the chi2 bit pattern and the id, minimised over the group).  The search box
// (max(0.5 cm, 4 sigma) plus 2 quanta) contains every hit with chi2 <= 16, so
// the box never changes the result.  Every lane of the group returns the same
// position and the hit's (qy, qz, id, key) in *qout.
template <int G, class Src>
__device__ __forceinline__ int pick_box(const Src& S, const Grp<G>& g, int r, const RowInfo& ri, const Box& bx,
                                        const float* p, const Win& w, int z_base, int4* qout) {
  if (box_empty(bx)) return -1;
  // the bins (iy, iz0..iz1) of one y-bin row are contiguous: one hit range each
  const int nyb = bx.iy1 - bx.iy0 + 1;
  const int span = bx.iz1 - bx.iz0 + 1;
  unsigned long long best = ~0ull;
  int best_pos = -1;
  int4 best_q = make_int4(0, 0, 0, 0);
  auto consider = [&](int h, const int4& q) {
    const unsigned long long key = hit_key(q, p, w, z_base);
    if (key < best) {
      best = key;
      best_pos = h;
      best_q = q;
    }
  };
  if constexpr (G == 1) {
    // one lane: the hit ranges of the first two y-bin rows (windows rarely
    // cover more), then the candidates four at a time: four loads in flight,
    // four keys formed independently and reduced by a tree before the one
    // compare with the running best (short dependency chains: the step's
    // time is issue latency more than memory latency)
    const int b0 = ri.bin0 + bx.iy0 * ri.nz + bx.iz0;
    const int a0 = S.first(r, b0), e0 = S.first(r, b0 + span);
    int a1 = 0, e1 = 0;
    if (nyb > 1) {
      a1 = S.first(r, b0 + ri.nz);
      e1 = S.first(r, b0 + ri.nz + span);
    }
    const int n0 = e0 - a0, total = n0 + (e1 - a1);
    // candidates CB at a time (the warp runs as many rounds as its lane with
    // the most candidates: a wide round keeps that count at one); keys of
    // four slots at a time reduced by a tree, one compare with the running best
    constexpr int CB = Src::kRound;
    const int off1 = a1 - n0;  // candidate j is at a0 + j below n0, else at off1 + j
    for (int j0 = 0; j0 < total; j0 += CB) {
      int pos[CB];
      int4 qk[CB];
#pragma unroll
      for (int k = 0; k < CB; ++k) {
        const int j = j0 + k;
        pos[k] = j + (j < n0 ? a0 : off1);
        if (j < total) qk[k] = S.hit(r, pos[k]);
      }
      // a hit with chi2 <= 16 lies inside the box (|dy| <= 4 sqrt(S_yy) <= wy,
      // likewise z), so an integer box test rejects most candidates of the
      // bins; only the survivors (typically the one hit of the track) get a
      // chi2 key, their record read again from the first-level cache
      unsigned live = 0;
#pragma unroll
      for (int k = 0; k < CB; ++k)
        if (j0 + k < total && qk[k].x >= bx.qy0 && qk[k].x <= bx.qy1 && qk[k].y >= bx.qz0 && qk[k].y <= bx.qz1)
          live |= 1u << k;
      while (live) {
        const int k = __ffs(live) - 1;
        live &= live - 1;
        const int j = j0 + k;
        const int ps = j + (j < n0 ? a0 : off1);
        const int4 q = S.hit(r, ps);
        const unsigned long long key = hit_key(q, p, w, z_base);
        if (key < best) {
          best = key;
          best_pos = ps;
          best_q = q;
        }
      }
    }
    for (int iy = bx.iy0 + 2; iy <= bx.iy1; ++iy) {  // wider windows (rare)
      const int b1 = ri.bin0 + iy * ri.nz + bx.iz0;
      const int a = S.first(r, b1), e = S.first(r, b1 + span);
      for (int h = a; h < e; ++h) consider(h, S.hit(r, h));
    }
    *qout = best_q;
    return best_pos;
  } else if (nyb == 1) {
    // one y-bin row (the usual case): every lane reads its hit range (one
    // address for the group) and takes hits gl and gl + G of each 2G
    const int b0 = ri.bin0 + bx.iy0 * ri.nz + bx.iz0;
    const int a = S.first(r, b0);
    const int total = S.first(r, b0 + span) - a;
    for (int kk = g.gl; kk < total; kk += 2 * G) {
      const int h0 = a + kk, h1 = a + kk + G;
      const bool two = kk + G < total;
      const int4 q0 = S.hit(r, h0);
      int4 q1 = q0;
      if (two) q1 = S.hit(r, h1);
      const unsigned long long k0 = hit_key(q0, p, w, z_base);
      const unsigned long long k1 = two ? hit_key(q1, p, w, z_base) : ~0ull;
      const bool second = k1 < k0;
      const unsigned long long km = second ? k1 : k0;
      if (km < best) {
        best = km;
        best_pos = second ? h1 : h0;
        best_q = second ? q1 : q0;
      }
    }
  } else {
    for (int base = 0; base < nyb; base += G) {  // group-uniform loop
      // one y-bin row per lane: its hit range [a, a + cnt)
      const int j = base + g.gl;
      int a = 0, cnt = 0;
      if (j < nyb) {
        const int b0 = ri.bin0 + (bx.iy0 + j) * ri.nz + bx.iz0;
        a = S.first(r, b0);
        cnt = S.first(r, b0 + span) - a;
      }
      const int inc = g.incl_scan(cnt);
      const int ex = inc - cnt;
      const int total = g.shfl(inc, G - 1);
      for (int kk = 0; kk < total; kk += 2 * G) {  // group-uniform loop, two hits per lane
        int h2[2];
        int4 q2[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int k = kk + t * G + g.gl;
          // lane holding candidate k: the first lane whose inclusive count exceeds k
          int lo = 0;
          int hi = G - 1;
#pragma unroll
          for (int step = 1; step < G; step <<= 1) {
            const int mid = (lo + hi) >> 1;
            const int v = g.shfl(inc, mid);
            if (v > k) hi = mid; else lo = mid + 1;
          }
          const int a_src = g.shfl(a, lo);
          const int ex_src = g.shfl(ex, lo);
          h2[t] = k < total ? a_src + (k - ex_src) : -1;
          if (h2[t] >= 0) q2[t] = S.hit(r, h2[t]);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t)
          if (h2[t] >= 0) consider(h2[t], q2[t]);
      }
    }
  }
  if constexpr (G > 1) {
    const unsigned long long gbest = g.min64(best);
    if (gbest == ~0ull) return -1;
    const unsigned who = __ballot_sync(g.mask, best == gbest) & g.mask;
    const int src = (__ffs(who) - 1) & (G - 1);
    qout->x = g.shfl(best_q.x, src);
    qout->y = g.shfl(best_q.y, src);
    qout->z = g.shfl(best_q.z, src);
    qout->w = g.shfl(best_q.w, src);
    return g.shfl(best_pos, src);
  }
  return -1;  // not reached: every branch above returns
}

template <int G, class Src>
__device__ __forceinline__ int pick_hit(const Src& S, const Grp<G>& g, int r, const RowInfo& ri, const float* p,
                                        const Win& w, int z_base, int4* qout) {
  const Box bx = row_box(ri, p[0], p[1], w.wy, w.wz, z_base);
  return pick_box<G>(S, g, r, ri, bx, p, w, z_base, qout);
}

}  // namespace

// One group of G lanes per tracklet; all lanes of a group run the same Kalman
// arithmetic on the same values and split the hit search of every row.
//  (i)   circle through the first, middle and last chain hits -> initial state;
//        Kalman fit along the chain (chain hits accepted without a chi2 test);
//  (ii)  outward extension: best hit with chi2 <= 16, 5 consecutive misses end it;
//  (iii) inward refit from the outermost hit (its y, z; outward sinphi,
//        tanlambda, q/pT with variances inflated 100-fold), re-picking hits
//        down to row 0.
// The first JOSEPH_UPDATES updates of each fit use the Joseph form (FP32
// conditioning of a fit from a wide prior).
// Guards end a pass: |sinphi| >= sin 70 deg, |y| > x tan(half angle), invalid
// step.  A non-finite or non-positive covariance diagonal drops the tracklet.
// z is carried relative to the start hit (z_base) so that FP32 keeps its
// precision for time-frame z' of thousands of cm.

// State of the outward passes of one tracklet.
struct UpFit {
  float p[5], C[15], x;
  float out_p[5], ov2, ov3, ov4;  // state and variances at the outermost hit
  int out_row, out_hit;
  int hn, hn2;                    // the next chain hit and the one after it
  int4 qn;                        // coordinates of the next chain hit
  int misses, n_upd, L, r0, z_base;
  bool dead;
};

// (i) start: the chain (walked here, or by an earlier kernel with PRE) and the
// initial state from the circle through its first, middle and last hits.
template <int G, bool PRE, class Src>
__device__ __forceinline__ void up_begin(const Buffers& b, const Grp<G>& g, const Src& S, const float* xr, int start,
                                         int4 hs, int tl, UpFit& f) {
  const DevParams& P = b.par;
  const int NR = P.n_rows;
  const float Q = 1.0f / TPC_QSCALE;
  const int key = hs.w;
  const int item = key / NR;
  const int r0 = key - item * NR;
  const int z_base = hs.y;
  int* hl = b.tl_hits + (size_t)tl * NR;
  // chain walk (pointer chasing; every lane of the group loads the same
  // address), or the chain a previous kernel walked (PRE)
  int L = 0, last = start;
  if constexpr (PRE) {
    L = __ldg(b.chain_len + tl);
    last = __ldcg(hl + L - 1);
  } else {
    for (int h = start; h >= 0 && L < NR; h = S.up(r0 + L - 1, h)) {
      if (g.gl == 0) hl[L] = h;
      last = h;
      ++L;
    }
  }
  g.sync();
  const int hmid = hl[L / 2];
  const int hn0 = L > 1 ? hl[1] : start, hn1 = L > 2 ? hl[2] : start;
  const int4 qa = hs, qm = S.hit(r0 + L / 2, hmid), qc = S.hit(r0 + L - 1, last);
  const float x1 = xr[r0], x2 = xr[r0 + L / 2], x3 = xr[r0 + L - 1];
  const float y1 = qa.x * Q, y2 = qm.x * Q, y3 = qc.x * Q;
  const float z3 = (float)(qc.y - z_base) * Q;
  const float dx13 = x3 - x1, dy13 = y3 - y1;
  const float d13 = sqrtf(fma2(dx13, dx13, dy13, dy13));
  const float d12 = sqrtf(fma2(x2 - x1, x2 - x1, y2 - y1, y2 - y1));
  const float d23 = sqrtf(fma2(x3 - x2, x3 - x2, y3 - y2, y3 - y2));
  const float cross = fma2(x2 - x1, y3 - y1, -(y2 - y1), x3 - x1);
  const float kappa = -2.0f * cross / (d12 * d23 * d13);
  const float u = fminf(1.0f, fmaxf(-1.0f, 0.5f * kappa * d13));
  const float phi1 = atan2f(dy13, dx13) + asinf(u);
  const float arc = d13 * asin_over_u(u);
  f.p[0] = y1;
  f.p[1] = 0.0f;
  f.p[2] = sinf(phi1);
  f.p[3] = z3 / arc;
  f.p[4] = kappa / P.kB;
  set_c0(P, f.C);
  f.x = x1;
  f.out_row = r0;
  f.out_hit = start;
#pragma unroll
  for (int m = 0; m < 5; ++m) f.out_p[m] = f.p[m];
  f.ov2 = f.C[ix(2, 2)];
  f.ov3 = f.C[ix(3, 3)];
  f.ov4 = f.C[ix(4, 4)];
  f.dead = false;
  // the next chain hit (position and coordinates) and the one after it are
  // fetched one row ahead of their use
  f.hn = hn0;
  f.hn2 = hn1;
  f.qn = S.hit(L > 1 ? r0 + 1 : r0, f.hn);
  f.misses = 0;
  f.n_upd = 0;
  f.L = L;
  f.r0 = r0;
  f.z_base = z_base;
}

// Row r of the outward passes: the chain hit while the chain lasts, else (ii)
// the best hit of the row.  false ends the pass (f.dead set if the covariance
// failed); a row without a hit counts a miss.
template <int G, class Src>
__device__ __forceinline__ bool up_row(const DevParams& P, const Grp<G>& g, const Src& S, const float* xr,
                                       const int* hl, int r, UpFit& f) {
  const float Q = 1.0f / TPC_QSCALE;
  const int i = r - f.r0;  // chain index of row r
  const bool chain = i < f.L;
  int h = -1;
  int4 q = make_int4(0, 0, 0, 0);
  // the row table entry is fetched for every row (one 32-byte load, off the
  // dependency chain) so that it lives in registers
  const RowInfo ri = S.row(r);
  if (chain) {
    h = f.hn;
    q = f.qn;
    f.hn = f.hn2;
    if (i + 1 < f.L) f.qn = S.hit(r + 1, f.hn);
    if (i + 2 < f.L) f.hn2 = hl[i + 2];
  }
  const float xn = xr[r];
  if (!kf_propagate(P, f.p, f.C, f.x, xn)) return false;
  f.x = xn;
  if (!(fabsf(f.p[2]) < SIN_MAX) || fabsf(f.p[0]) > f.x * P.tan_half) return false;
  const Win w = make_win(P, f.C);
  if (!chain) h = pick_hit<G>(S, g, r, ri, f.p, w, f.z_base, &q);
  if (!chain && h < 0) {
    ++f.misses;
    return true;
  }
  if (f.n_upd < JOSEPH_UPDATES)
    kf_update_joseph(w, P.vy, P.vz, f.p, f.C, q.x * Q - f.p[0], (float)(q.y - f.z_base) * Q - f.p[1]);
  else
    kf_update(w, f.p, f.C, q.x * Q - f.p[0], (float)(q.y - f.z_base) * Q - f.p[1]);
  ++f.n_upd;
  if (!cov_ok(f.C)) {
    f.dead = true;
    return false;
  }
  f.misses = 0;
  f.out_row = r;
  f.out_hit = h;
#pragma unroll
  for (int m = 0; m < 5; ++m) f.out_p[m] = f.p[m];
  f.ov2 = f.C[ix(2, 2)];
  f.ov3 = f.C[ix(3, 3)];
  f.ov4 = f.C[ix(4, 4)];
  return true;
}

// End of the outward passes: the record goes to b.tlu[tl] and the tracklet
// claims its outermost hit (smallest tracklet index wins).
template <int G>
__device__ __forceinline__ void up_end(const Buffers& b, const Grp<G>& g, int tl, int item, int local,
                                       const UpFit& f) {
  if (g.gl == 0) {
    TrackletUp u;
    u.out_hit = f.dead ? -1 : f.out_hit;
    u.out_row = f.out_row;
    u.snp = f.out_p[2];
    u.tgl = f.out_p[3];
    u.qpt = f.out_p[4];
    u.v2 = f.ov2;
    u.v3 = f.ov3;
    u.v4 = f.ov4;
    u.z_base = f.z_base;
    u.item = item;
    u.local = local;
    u.pad = 0;
    b.tlu[tl] = u;
    if (!f.dead) atomicMin(&b.out_owner[f.out_hit], tl);
  }
  g.sync();
}

// Outward passes (i) and (ii) of the tracklet with start hit `start`: one loop
// over the rows above the start row, taking the chain hit while the chain lasts
// and searching afterwards (so that lanes of a warp in different phases run the
// same propagation and update code together).  `local` is the item-local id,
// `xr` the row positions.
template <int G, bool PRE, class Src>
__device__ __forceinline__ void tracklet_up(const Buffers& b, const Grp<G>& g, const Src& S, const float* xr,
                                            int start, int4 hs, int tl, int local) {
  const int NR = b.par.n_rows;
  const int* hl = b.tl_hits + (size_t)tl * NR;
  UpFit f;
  up_begin<G, PRE>(b, g, S, xr, start, hs, tl, f);
  for (int r = f.r0 + 1; r < NR && f.misses < MAX_MISS; ++r)
    if (!up_row<G>(b.par, g, S, xr, hl, r, f)) break;
  up_end<G>(b, g, tl, hs.w / NR, local, f);
}

// Inward refit (iii): the state of one refit and its three steps, shared by the
// per-tracklet loop below and the refilling kernel of the batched form.
struct DownFit {
  float q5[5], C[15];        // running state and covariance
  float x, chi2sum, in_x;    // current x; chi2 sum; x of the innermost hit
  float in_p[5], in_C[15];   // state at the innermost hit so far
  int n, in_z, misses;
  bool dead;
};

// Start of the refit of tracklet tl, only if it is the smallest tracklet that
// reached its outermost hit (the others are dropped): that hit's y, z and the
// outward direction and curvature with variances inflated 100-fold (capped at
// the initial ones).
template <int G, class Src>
__device__ __forceinline__ void down_begin(const Buffers& b, const Grp<G>& g, const Src& S, const float* xr, int tl,
                                           const TrackletUp& u, int* hl, DownFit& f) {
  const DevParams& P = b.par;
  const float Q = 1.0f / TPC_QSCALE;
  // claims of other threads of the previous launch: read from L2
  f.dead = u.out_hit < 0 || __ldcg(b.out_owner + u.out_hit) != tl;
  f.x = xr[u.out_row];
  f.n = 0;
  f.chi2sum = 0.f;
  f.in_x = f.x;
  f.in_z = 0;
  f.misses = 0;
#pragma unroll
  for (int m = 0; m < 5; ++m) f.in_p[m] = 0.f;
#pragma unroll
  for (int m = 0; m < 15; ++m) f.in_C[m] = 0.f;
  if (!f.dead) {
    const int4 qo = S.hit(u.out_row, u.out_hit);
    f.q5[0] = qo.x * Q;
    f.q5[1] = (float)(qo.y - u.z_base) * Q;
    f.q5[2] = u.snp;
    f.q5[3] = u.tgl;
    f.q5[4] = u.qpt;
    set_c0(P, f.C);
    f.C[ix(2, 2)] = fminf(1.0f, INFLATE * u.v2);
    f.C[ix(3, 3)] = fminf(1.0f, INFLATE * u.v3);
    f.C[ix(4, 4)] = fminf(100.0f, INFLATE * u.v4);
    g.sync();
    if (g.gl == 0) hl[0] = u.out_hit;
    f.n = 1;
    f.in_z = qo.y;
#pragma unroll
    for (int m = 0; m < 5; ++m) f.in_p[m] = f.q5[m];
#pragma unroll
    for (int m = 0; m < 15; ++m) f.in_C[m] = f.C[m];
  }
}

// Row r of the refit: propagate, pick the best hit, update.  false ends the
// pass (f.dead set if the covariance failed); a row without a hit counts a miss.
template <int G, class Src>
__device__ __forceinline__ bool down_row(const DevParams& P, const Grp<G>& g, const Src& S, const float* xr, int r,
                                         int z_base, int* hl, DownFit& f) {
  const float Q = 1.0f / TPC_QSCALE;
  const RowInfo ri = S.row(r);  // independent of the state: in flight during the step
  const float xn = xr[r];
  if (!kf_propagate(P, f.q5, f.C, f.x, xn)) return false;
  f.x = xn;
  if (!(fabsf(f.q5[2]) < SIN_MAX) || fabsf(f.q5[0]) > f.x * P.tan_half) return false;
  int4 q;
  const Win w = make_win(P, f.C);
  const int h = pick_hit<G>(S, g, r, ri, f.q5, w, z_base, &q);
  if (h < 0) {
    ++f.misses;
    return true;
  }
  const float e0 = q.x * Q - f.q5[0], e1 = (float)(q.y - z_base) * Q - f.q5[1];
  f.chi2sum += f.n <= JOSEPH_UPDATES ? kf_update_joseph(w, P.vy, P.vz, f.q5, f.C, e0, e1)
                                     : kf_update(w, f.q5, f.C, e0, e1);
  if (!cov_ok(f.C)) {
    f.dead = true;
    return false;
  }
  f.misses = 0;
  if (g.gl == 0) hl[f.n] = h;
  ++f.n;
  f.in_z = q.y;
  f.in_x = f.x;
#pragma unroll
  for (int m = 0; m < 5; ++m) f.in_p[m] = f.q5[m];
#pragma unroll
  for (int m = 0; m < 15; ++m) f.in_C[m] = f.C[m];
  return true;
}

// End of the refit: the 112-byte record of tracklet tl (n = 0 if dropped or
// short), fields split over the lanes of the group.
template <int G>
__device__ __forceinline__ void down_end(const Buffers& b, const Grp<G>& g, int tl, int item, int local, int z_base,
                                         DownFit& f) {
  if (f.dead || f.n < MIN_HITS) f.n = 0;
  float* rf = reinterpret_cast<float*>(b.tl + tl);
  int* ri_ = reinterpret_cast<int*>(b.tl + tl);
  const int z_in = f.n ? f.in_z : 0;
  for (int fld = g.gl; fld < 27; fld += G) {
    float fv = 0.f;
#pragma unroll
    for (int m = 0; m < 5; ++m) fv = (fld == m) ? f.in_p[m] : fv;
#pragma unroll
    for (int m = 0; m < 15; ++m) fv = (fld == 5 + m) ? f.in_C[m] : fv;
    if (fld < 20) rf[fld] = fv;
    else if (fld == 20) rf[20] = f.chi2sum;
    else if (fld == 21) rf[21] = f.in_x;
    else if (fld == 22) ri_[22] = f.n;
    else if (fld == 23) ri_[23] = z_base;
    else if (fld == 24) ri_[24] = z_in;
    else if (fld == 25) ri_[25] = item;
    else ri_[26] = local;
  }
  g.sync();
}

// Inward refit (iii) of tracklet tl by a group of G lanes: the record goes to
// b.tl[tl] and the hit list to b.tl_hits[tl * n_rows ...].
template <int G, class Src>
__device__ __forceinline__ void tracklet_down(const Buffers& b, const Grp<G>& g, const Src& S, const float* xr,
                                              int tl) {
  const TrackletUp u = b.tlu[tl];
  int* hl = b.tl_hits + (size_t)tl * b.par.n_rows;
  DownFit f;
  down_begin<G>(b, g, S, xr, tl, u, hl, f);
  if (!f.dead)
    for (int r = u.out_row - 1; r >= 0 && f.misses < MAX_MISS; --r)
      if (!down_row<G>(b.par, g, S, xr, r, u.z_base, hl, f)) break;
  down_end<G>(b, g, tl, u.item, u.local, u.z_base, f);
}

template <int G>
__global__ void __launch_bounds__(128) k_tracklets_up(const __grid_constant__ Buffers b) {
  __shared__ float s_x[TPC_MAX_ROWS];
  for (int r = threadIdx.x; r < b.par.n_rows; r += blockDim.x) s_x[r] = b.par.x[r];
  __syncthreads();
  const Grp<G> g;
  const int T = b.start_ex[b.N];
  const int NR = b.par.n_rows;
  const int grp = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int ngrp = (gridDim.x * blockDim.x) / G;
  for (int t = grp; t < T; t += ngrp) {
    const int start = b.starts[t];
    const int4 hs = __ldg(b.s_hit + start);
    const int item = hs.w / NR;
    const GSrc<true> S{&b, b.rows + (size_t)item * NR};
    tracklet_up<G, false>(b, g, S, s_x, start, hs, t, t - b.start_ex[b.item_off[item]]);
  }
}

template <int G>
__global__ void __launch_bounds__(128) k_tracklets_down(const __grid_constant__ Buffers b) {
  __shared__ float s_x[TPC_MAX_ROWS];
  for (int r = threadIdx.x; r < b.par.n_rows; r += blockDim.x) s_x[r] = b.par.x[r];
  __syncthreads();
  const Grp<G> g;
  const int T = b.start_ex[b.N];
  const int grp = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int ngrp = (gridDim.x * blockDim.x) / G;
  for (int t = grp; t < T; t += ngrp) {
    const GSrc<true> S{&b, b.rows + (size_t)b.tlu[t].item * b.par.n_rows};
    tracklet_down<G>(b, g, S, s_x, t);
  }
}


cudaError_t tpc_launch_tracklets(const Buffers& b, const LaunchCfg& c, cudaStream_t s) {
  cudaMemsetAsync(b.out_owner, 0x7F, sizeof(int) * (size_t)b.N, s);
  const int grid = c.grid_tl, block = c.block_tl;
  switch (c.tl_group) {
#define TPC_TL(GG)                                        \
  case GG:                                                \
    k_tracklets_up<GG><<<grid, block, 0, s>>>(b);         \
    k_tracklets_down<GG><<<grid, block, 0, s>>>(b);       \
    break;
    TPC_TL(1)
    TPC_TL(2)
    TPC_TL(4)
    TPC_TL(8)
    TPC_TL(16)
    default:
      k_tracklets_up<32><<<grid, block, 0, s>>>(b);
      k_tracklets_down<32><<<grid, block, 0, s>>>(b);
      break;
#undef TPC_TL
  }
  return cudaGetLastError();
}

// ============================================================================ S7
__device__ __forceinline__ unsigned long long tl_key(int n, int local) {
  return ((unsigned long long)(unsigned)n << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)local);
}

namespace {
// Ownership bid of tracklet tl: one 64-bit atomicMax per hit (key: more hits,
// then smaller item-local id), lanes of a warp over the hits.
__device__ __forceinline__ void select_max_warp(const Buffers& b, int tl, int lane) {
  const int n = b.tl[tl].n;
  if (n < MIN_HITS) return;
  const unsigned long long key = tl_key(n, b.tl[tl].local);
  const int* hl = b.tl_hits + (size_t)tl * b.par.n_rows;
  for (int k = lane; k < n; k += 32) atomicMax(&b.hit_key[hl[k]], key);
}

// Hits owned by tracklet tl; a track if >= 10 (and, with slices, if its innermost
// hit lies in the item's core).  Returns (1 << 32 | owned) or 0, in every lane.
__device__ __forceinline__ unsigned long long select_own_warp(const Buffers& b, int tl, int lane) {
  const TrackletRec& r = b.tl[tl];
  const int n = r.n;
  if (n < MIN_HITS) return 0;
  const unsigned long long key = tl_key(n, r.local);
  const int* hl = b.tl_hits + (size_t)tl * b.par.n_rows;
  int own = 0;
  for (int k = lane; k < n; k += 32) own += b.hit_key[hl[k]] == key;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) own += __shfl_xor_sync(0xffffffffu, own, o);
  bool keep = own >= MIN_HITS;
  if (keep && b.item_core) keep = r.z_in >= b.item_core[2 * r.item] && r.z_in < b.item_core[2 * r.item + 1];
  return keep ? ((1ull << 32) | (unsigned long long)own) : 0ull;
}

// Track record of tracklet tl (first_cluster = io) and its owned cluster ids,
// innermost first, at ids[io ...]; a warp per tracklet.
__device__ __forceinline__ void emit_warp(const Buffers& b, int tl, unsigned long long cnt, unsigned io,
                                          tpc_track_t* dst, uint32_t* ids, int lane) {
  const TrackletRec& r = b.tl[tl];
  // the 112-byte record, one 32-bit word per lane (words 0-4 params, 5-19
  // covariance, 20 chi2, 21 ndf, 22 item, 23 sector, 24 event, 25 first
  // cluster, 26 cluster count, with x_ref first: the tpc_track_t layout)
  if (lane < 28) {
    const float* rf = reinterpret_cast<const float*>(&r);
    uint32_t v = 0;
    if (lane == 0) v = __float_as_uint(r.x_ref);
    else if (lane == 2) v = __float_as_uint(r.p[1] + (float)r.z_base * (1.0f / TPC_QSCALE));
    else if (lane <= 5) v = __float_as_uint(rf[lane - 1]);           // y, (z), snp, tgl, qpt
    else if (lane <= 20) v = __float_as_uint(rf[lane - 1]);          // cov[0..14]
    else if (lane == 21) v = __float_as_uint(r.chi2);
    else if (lane == 22) v = (uint32_t)(2 * r.n - 5);
    else if (lane == 23) v = (uint32_t)r.item;
    else if (lane == 24) v = b.item_sector ? b.item_sector[r.item] : 0u;
    else if (lane == 25) v = b.item_event ? b.item_event[r.item] : 0u;
    else if (lane == 26) v = io;
    else v = (uint32_t)(cnt & 0xFFFFFFFFull);
    reinterpret_cast<uint32_t*>(dst)[lane] = v;
  }
  const unsigned long long key = tl_key(r.n, r.local);
  const int* hl = b.tl_hits + (size_t)tl * b.par.n_rows;
  unsigned done = 0;
  for (int base = 0; base < r.n; base += 32) {
    const int k = r.n - 1 - (base + lane);
    int h = -1;
    bool own = false;
    if (k >= 0) {
      h = hl[k];
      own = b.hit_key[h] == key;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, own);
    if (own) ids[done + __popc(bal & ((1u << lane) - 1))] = (uint32_t)b.s_hit[h].z;
    done += __popc(bal);
  }
}
}  // namespace

__global__ void __launch_bounds__(256) k_select_max(const __grid_constant__ Buffers b) {
  const int T = b.start_ex[b.N];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t = warp; t < T; t += nwarps) select_max_warp(b, t, lane);
}

__global__ void __launch_bounds__(256) k_select_own(const __grid_constant__ Buffers b) {
  const int T = b.start_ex[b.N];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t = warp; t < T; t += nwarps) {
    const unsigned long long out = select_own_warp(b, t, lane);
    if (lane == 0) b.tl_cnt[t] = out;
  }
}

// ============================================================================ S8
__global__ void __launch_bounds__(256) k_output(const __grid_constant__ Buffers b) {
  const int T = b.start_ex[b.N];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  tpc_track_t* trk = reinterpret_cast<tpc_track_t*>(b.trk);
  for (int t = warp; t < T; t += nwarps) {
    const unsigned long long cnt = b.tl_cnt[t];
    if (cnt == 0) continue;
    const unsigned long long ex = b.tl_ex[t];
    const unsigned ti = (unsigned)(ex >> 32);
    const unsigned io = (unsigned)(ex & 0xFFFFFFFFull);
    emit_warp(b, t, cnt, io, trk + ti, b.trk_ids + io, lane);
    if (lane == 0) b.trk_tl[ti] = t;
  }
}

__global__ void k_counts(const __grid_constant__ Buffers b) {
  const int T = b.start_ex[b.N];
  const unsigned long long tot = b.tl_ex[T];
  b.counts[0] = tot >> 32;
  b.counts[1] = tot & 0xFFFFFFFFull;
  b.counts[2] = (unsigned long long)T;
}


// ============================================================================ S9
// Batched form: the stages of the plain form over all items of the batch
// (events, sectors, time slices) in one captured graph, with the tracklet
// passes as persistent kernels that refill their lanes from work queues (below).
// A warp runs as long as its slowest lane; a lane costs about 900 cycles per
// chain row and 3,400 per searched row, and tracklets run from a few rows to
// 300.  The queues change no result: a tracklet's outputs go to its canonical
// index.  Each queue keeps an item's tracklets together, so that the lanes of
// an SM keep reading a few items' rows, bins and hits (a global order mixed
// items in every warp and cost more in cache misses than it saved).
//   k_chain_walk:  every start hit's chain (hits kept for the outward pass);
//   k_queue_items: per item (one CTA), a counting sort of its tracklets by chain
//                  length in shared memory, shortest chains first: their long
//                  searches start first, and lanes that switch from chain to
//                  search at the same row share a warp;
//   k_down_order:  the inward pass's order (by outermost row, per segment).
// The non-persistent k_tracklets_up_q<G> serves groups of G > 1 lanes.
__global__ void __launch_bounds__(256) k_chain_walk(const __grid_constant__ Buffers b) {
  const int T = b.start_ex[b.N];
  const int NR = b.par.n_rows;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    int* hl = b.tl_hits + (size_t)t * NR;
    int L = 0;
    for (int h = b.starts[t]; h >= 0 && L < NR; h = __ldg(b.up + h)) hl[L++] = h;
    b.chain_len[t] = L;
  }
}

__global__ void __launch_bounds__(256) k_queue_items(const __grid_constant__ Buffers b) {
  __shared__ int s_cnt[TPC_MAX_ROWS + 2];
  __shared__ int sm[33];
  const int item = blockIdx.x;
  const int t0 = b.start_ex[b.item_off[item]], t1 = b.start_ex[b.item_off[item + 1]];
  const int nb = b.par.n_rows + 1;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) s_cnt[k] = 0;
  __syncthreads();
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) atomicAdd(&s_cnt[b.chain_len[t]], 1);
  __syncthreads();
  int carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {  // block-uniform loop
    const int k = base + threadIdx.x;
    const int v = k < nb ? s_cnt[k] : 0;
    int tot;
    const int ex = block_excl_scan(v, sm, &tot);
    if (k < nb) s_cnt[k] = carry + ex;
    carry += tot;
  }
  __syncthreads();
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) b.tl_order[t0 + atomicAdd(&s_cnt[b.chain_len[t]], 1)] = t;
}

template <int G>
__global__ void __launch_bounds__(128) k_tracklets_up_q(const __grid_constant__ Buffers b) {
  __shared__ float s_x[TPC_MAX_ROWS];
  for (int r = threadIdx.x; r < b.par.n_rows; r += blockDim.x) s_x[r] = b.par.x[r];
  __syncthreads();
  const Grp<G> g;
  const int T = b.start_ex[b.N];
  const int NR = b.par.n_rows;
  const int grp = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int ngrp = (gridDim.x * blockDim.x) / G;
  for (int i = grp; i < T; i += ngrp) {
    const int t = __ldg(b.tl_order + i);
    const int start = __ldg(b.starts + t);
    const int4 hs = __ldg(b.s_hit + start);
    const int item = hs.w / NR;
    const GSrc<true> S{&b, b.rows + (size_t)item * NR};
    tracklet_up<G, true>(b, g, S, s_x, start, hs, t, t - b.start_ex[b.item_off[item]]);
  }
}

// Persistent tracklet kernels of the batched form: one CTA per SM with
// TL_WARPS warps; the tracklets (in the order b.tl_order) are cut into one
// contiguous segment per CTA, and a lane takes the next tracklet as soon as it
// finishes one, so that a warp stays full until the work runs out.  A warp
// takes from its own CTA's segment (whose items' rows, bins and hits stay in
// the SM's L1) and, once that is empty, from the following segments (work per
// segment differs by up to 1.5x across a batch of uneven events).
constexpr int TL_WARPS = 16;

// segment c of T tracklets cut into n: [i0, i0 + len)
__device__ __forceinline__ void tl_segment(int T, int n, int c, int* i0, int* len) {
  const int seg = (T + n - 1) / n;
  const int a = min(T, c * seg);
  *i0 = a;
  *len = min(T, a + seg) - a;
}

// Called by all lanes of a warp: the lanes with `need` get the next tracklets
// of the order, or -1 when none is left.  Lane 0 claims them with one atomic on
// the counter b.seg_next of segment *cs (its CTA's first, then the following
// ones as they run empty; *tried counts the empty ones, so the search ends).
__device__ __forceinline__ int take_tracklet(const Buffers& b, int T, bool need, int* cs, int* tried) {
  const unsigned m = __ballot_sync(0xffffffffu, need);
  if (!m) return -1;
  const int lane = threadIdx.x & 31, nseg = gridDim.x;
  int base = -1, i0 = 0, len = 0;
  if (lane == 0) {
    while (*tried < nseg) {
      tl_segment(T, nseg, *cs, &i0, &len);
      if (__ldcg(b.seg_next + *cs) < len) {
        base = atomicAdd(b.seg_next + *cs, __popc(m));
        if (base < len) break;
      }
      *cs = *cs + 1 == nseg ? 0 : *cs + 1;
      ++*tried;
      base = -1;
    }
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  i0 = __shfl_sync(0xffffffffu, i0, 0);
  len = __shfl_sync(0xffffffffu, len, 0);
  const int k = base + __popc(m & ((1u << lane) - 1u));
  return (need && base >= 0 && k < len) ? __ldg(b.tl_order + i0 + k) : -1;
}

__global__ void __launch_bounds__(32 * TL_WARPS, 1) k_tracklets_up_p(const __grid_constant__ Buffers b) {
  __shared__ float s_x[TPC_MAX_ROWS];
  for (int r = threadIdx.x; r < b.par.n_rows; r += blockDim.x) s_x[r] = b.par.x[r];
  __syncthreads();
  const Grp<1> g;
  const int NR = b.par.n_rows;
  const int T = b.start_ex[b.N];
  int cs = blockIdx.x, tried = 0;
  int tl = -1, r = 0, item = 0, local = 0;
  UpFit f;
  while (true) {
    const int got = take_tracklet(b, T, tl < 0, &cs, &tried);
    if (tl < 0 && got >= 0) {
      tl = got;
      const int start = __ldg(b.starts + tl);
      const int4 hs = __ldg(b.s_hit + start);
      item = hs.w / NR;
      local = tl - b.start_ex[b.item_off[item]];
      const GSrc<true> S{&b, b.rows + (size_t)item * NR};
      up_begin<1, true>(b, g, S, s_x, start, hs, tl, f);
      r = f.r0 + 1;
    }
    if (!__any_sync(0xffffffffu, tl >= 0)) break;
    if (tl >= 0) {
      bool more = r < NR && f.misses < MAX_MISS;
      if (more) {
        const GSrc<true> S{&b, b.rows + (size_t)item * NR};
        more = up_row<1>(b.par, g, S, s_x, b.tl_hits + (size_t)tl * NR, r, f);
        ++r;
        more = more && r < NR && f.misses < MAX_MISS;
      }
      if (!more) {
        up_end<1>(b, g, tl, item, local, f);
        tl = -1;
      }
    }
  }
}

// Inward refits of the batched form, persistent as above.  With a tracklet per
// lane a warp runs as long as its longest refit, and refits run from a few to
// 150 rows.  k_down_order sorts every segment by outermost row, highest first
// (the refit runs from there towards row 0, so that row bounds its length):
// the long refits start first and a segment ends on short ones; dropped
// tracklets go last.  It also resets the segment counters.  The order changes
// no result: every tracklet writes its own record.
__device__ __forceinline__ int down_key(const Buffers& b, int t, int NR) {
  const TrackletUp u = b.tlu[t];
  const bool dropped = u.out_hit < 0 || __ldcg(b.out_owner + u.out_hit) != t;
  return dropped ? NR : NR - 1 - u.out_row;
}

__global__ void __launch_bounds__(256) k_down_order(const __grid_constant__ Buffers b) {
  __shared__ int s_cnt[TPC_MAX_ROWS + 2];
  __shared__ int sm[33];
  const int T = b.start_ex[b.N];
  int i0, len;
  tl_segment(T, gridDim.x, blockIdx.x, &i0, &len);
  const int i1 = i0 + len;
  const int NR = b.par.n_rows, nb = NR + 1;
  if (threadIdx.x == 0) b.seg_next[blockIdx.x] = 0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) s_cnt[k] = 0;
  __syncthreads();
  for (int t = i0 + threadIdx.x; t < i1; t += blockDim.x) atomicAdd(&s_cnt[down_key(b, t, NR)], 1);
  __syncthreads();
  int carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {  // block-uniform loop
    const int k = base + threadIdx.x;
    const int v = k < nb ? s_cnt[k] : 0;
    int tot;
    const int ex = block_excl_scan(v, sm, &tot);
    if (k < nb) s_cnt[k] = carry + ex;
    carry += tot;
  }
  __syncthreads();
  for (int t = i0 + threadIdx.x; t < i1; t += blockDim.x)
    b.tl_order[i0 + atomicAdd(&s_cnt[down_key(b, t, NR)], 1)] = t;
}

__global__ void __launch_bounds__(32 * TL_WARPS, 1) k_tracklets_down_p(const __grid_constant__ Buffers b) {
  __shared__ float s_x[TPC_MAX_ROWS];
  for (int r = threadIdx.x; r < b.par.n_rows; r += blockDim.x) s_x[r] = b.par.x[r];
  __syncthreads();
  const Grp<1> g;
  const int NR = b.par.n_rows;
  const int T = b.start_ex[b.N];
  int cs = blockIdx.x, tried = 0;
  int tl = -1, r = 0, item = 0, local = 0, z_base = 0;
  DownFit f;
  while (true) {
    const int got = take_tracklet(b, T, tl < 0, &cs, &tried);
    if (tl < 0 && got >= 0) {
      tl = got;
      const TrackletUp u = b.tlu[tl];
      item = u.item;
      local = u.local;
      z_base = u.z_base;
      r = u.out_row - 1;
      const GSrc<true> S{&b, b.rows + (size_t)item * NR};
      down_begin<1>(b, g, S, s_x, tl, u, b.tl_hits + (size_t)tl * NR, f);
    }
    if (!__any_sync(0xffffffffu, tl >= 0)) break;
    if (tl >= 0) {
      bool more = !f.dead && r >= 0 && f.misses < MAX_MISS;
      if (more) {
        const GSrc<true> S{&b, b.rows + (size_t)item * NR};
        more = down_row<1>(b.par, g, S, s_x, r, z_base, b.tl_hits + (size_t)tl * NR, f);
        --r;
        more = more && r >= 0 && f.misses < MAX_MISS;
      }
      if (!more) {
        down_end<1>(b, g, tl, item, local, z_base, f);
        tl = -1;
      }
    }
  }
}

cudaError_t tpc_launch_tracklets_queued(const Buffers& b, const LaunchCfg& c, cudaStream_t s) {
  cudaMemsetAsync(b.out_owner, 0x7F, sizeof(int) * (size_t)b.N, s);
  k_chain_walk<<<c.num_sms * 8, 256, 0, s>>>(b);
  k_queue_items<<<b.I, 256, 0, s>>>(b);
  const int grid = c.grid_tl, block = c.block_tl;
  switch (c.batch_group) {
#define TPC_TLQ(GG)                                       \
  case GG:                                                \
    k_tracklets_up_q<GG><<<grid, block, 0, s>>>(b);       \
    k_tracklets_down<GG><<<grid, block, 0, s>>>(b);       \
    break;
    case 1:
    {
      const int nseg = std::min(c.num_sms, TPC_MAX_SEGS);
      cudaMemsetAsync(b.seg_next, 0, sizeof(int) * nseg, s);
      k_tracklets_up_p<<<nseg, 32 * TL_WARPS, 0, s>>>(b);
      k_down_order<<<nseg, 256, 0, s>>>(b);
      k_tracklets_down_p<<<nseg, 32 * TL_WARPS, 0, s>>>(b);
    }
      break;
    TPC_TLQ(2)
    default:
      k_tracklets_up_q<4><<<grid, block, 0, s>>>(b);
      k_tracklets_down<4><<<grid, block, 0, s>>>(b);
      break;
#undef TPC_TLQ
  }
  return cudaGetLastError();
}


// ============================================================================ S11
// Space-point correction by a per-sector grid (location-dependent calibration,
// Abstract; online calibration, Sec. 3): trilinear interpolation of (dy, dz)
// nodes over (x, v = y / (x tan_half), z), coordinates clamped to the grid, at
// the pad row's radius (the row fixes x).  Writes corrected y, z.
__global__ void __launch_bounds__(256) k_correct_grid(const __grid_constant__ Buffers b) {
  const DevParams& P = b.par;
  const Chunk ch = b.chunks[blockIdx.x];
  const int sector = b.item_sector ? (int)b.item_sector[ch.item] : 0;
  if (sector >= b.grid_sectors) {
    if (threadIdx.x == 0 && ch.end > ch.begin) atomicOr(b.err, TPC_DERR_BAD_INPUT);
    return;
  }
  __shared__ float s_x[TPC_MAX_ROWS];  // row positions (lanes read different rows)
  for (int r = threadIdx.x; r < P.n_rows; r += blockDim.x) s_x[r] = P.x[r];
  __syncthreads();
  const float* B = b.grid_bounds + 6 * sector;
  const float bx0 = B[0], sx = (b.grid_nx - 1) / (B[1] - B[0]);
  const float bv0 = B[2], sv = (b.grid_ny - 1) / (B[3] - B[2]);
  const float bz0 = B[4], sz = (b.grid_nz - 1) / (B[5] - B[4]);
  const float2* G = b.grid + (size_t)sector * b.grid_nx * b.grid_ny * b.grid_nz;
  for (int i = ch.begin + threadIdx.x; i < ch.end; i += blockDim.x) {
    const int r = b.row[i];
    const float y = b.y[i], z = b.z[i];
    if (r < 0 || r >= P.n_rows) {  // rejected later by validation
      b.cy[i] = y;
      b.cz[i] = z;
      continue;
    }
    const float x = s_x[r];
    const float v = y / (x * P.tan_half);
    float u[3] = {(x - bx0) * sx, (v - bv0) * sv, (z - bz0) * sz};
    const int dims[3] = {b.grid_nx, b.grid_ny, b.grid_nz};
    int lo[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float t = fminf(fmaxf(u[a], 0.0f), (float)(dims[a] - 1));  // NaN stays NaN, caught later
      int k = (int)floorf(t);
      k = min(max(k, 0), dims[a] - 2);
      lo[a] = k;
      f[a] = t - k;
    }
    const size_t sy_ = b.grid_nz, sx_ = (size_t)b.grid_ny * b.grid_nz;
    const float2* g0 = G + lo[0] * sx_ + lo[1] * sy_ + lo[2];
    float2 c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = g0[(k >> 2) * sx_ + ((k >> 1) & 1) * sy_ + (k & 1)];
    float dy = 0.f, dz = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = ((k >> 2) ? f[0] : 1.f - f[0]) * (((k >> 1) & 1) ? f[1] : 1.f - f[1]) * ((k & 1) ? f[2] : 1.f - f[2]);
      dy += w * c[k].x;
      dz += w * c[k].y;
    }
    b.cy[i] = y + dy;
    b.cz[i] = z + dz;
  }
}

cudaError_t tpc_launch_grid_correction(const Buffers& b, cudaStream_t s) {
  k_correct_grid<<<b.n_chunks, 256, 0, s>>>(b);
  return cudaGetLastError();
}
// ============================================================================ host launchers
cudaError_t tpc_configure_kernels(int sort_smem, int link_smem) {
  (void)link_smem;
  cudaError_t e = cudaFuncSetAttribute(k_row_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, sort_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_row_sort_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_WARPS * RS_WARP_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_links<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, LINK_STAGE_MAX);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_links<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, LINK_STAGE_MAX);
  return e;
}

static void scan_i32(const int* in, int* out, long long n, unsigned long long* bsum, int G, cudaStream_t s) {
  k_scan_reduce_i32<<<G, 256, 0, s>>>(in, n, bsum);
  k_scan_bsums<unsigned long long><<<1, 1024, 0, s>>>(bsum, G);
  k_scan_final_i32<<<G, 256, 0, s>>>(in, out, nullptr, n, bsum);
}

static void scan_u64_dev(const unsigned long long* in, unsigned long long* out, const int* n_dev,
                         unsigned long long* bsum, int G, cudaStream_t s) {
  k_scan_reduce<unsigned long long><<<G, 256, 0, s>>>(in, n_dev, 0, bsum);
  k_scan_bsums<unsigned long long><<<1, 1024, 0, s>>>(bsum, G);
  k_scan_final_u64<<<G, 256, 0, s>>>(in, out, n_dev, 0, bsum);
}

// Plain mode: one launch per step over all items.  ev (nullable) receives
// TPC_N_STAGES+1 events around the steps.
namespace {
cudaError_t launch_stages(const Buffers& b, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev, bool queued) {
  const int NR = c.n_rows;
  const int M = b.I * NR;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(ev[i], s);
  };
  mark(0);
  cudaMemsetAsync(b.rs_cnt, 0, sizeof(int) * M, s);
  cudaMemsetAsync(b.rs_min, 0x7F, sizeof(int) * 4 * (size_t)M, s);
  cudaMemsetAsync(b.row_fill, 0, sizeof(int) * M, s);
  cudaMemsetAsync(b.hit_key, 0, sizeof(unsigned long long) * (size_t)b.N, s);
  k_row_stats<<<b.n_chunks, 256, 0, s>>>(b);
  mark(1);
  k_row_setup<<<b.I, 256, 0, s>>>(b);
  mark(2);
  k_group_scatter<<<b.n_chunks, 256, 0, s>>>(b);
  mark(3);
  // rows of at most 256 hits on average (events, sectors): a warp per row, the
  // few larger rows by CTAs; denser rows (time-frame slices): a CTA per row
  if (M && (long long)b.N <= 256ll * M) {
    cudaMemsetAsync(b.rs_big + M, 0, sizeof(int), s);
    k_row_sort_warp<<<(M + RS_WARPS - 1) / RS_WARPS, 32 * RS_WARPS, RS_WARPS * RS_WARP_BYTES, s>>>(b, M);
    k_row_sort<<<c.num_sms * 16, 128, c.sort_smem, s>>>(b, c.sort_smem, b.cl_q, b.cl_key, b.up_raw, M, 1);
  } else if (M) {
    k_row_sort<<<M, 128, c.sort_smem, s>>>(b, c.sort_smem, b.cl_q, b.cl_key, b.up_raw, M, 0);
  }
  mark(4);
  // positions left unwritten by rejected clusters must read as "no link"
  cudaMemsetAsync(b.up_raw, 0xFF, sizeof(int) * (size_t)b.N, s);
  cudaMemsetAsync(b.dn_raw, 0xFF, sizeof(int) * (size_t)b.N, s);
  {
    // default: 8 rows per CTA (measured best between 4 for one event and 16 for 64 events)
    const int rpc = c.link_rows > 0 ? std::min(c.link_rows, NR) : std::min(8, NR);
    const int nrb = (NR + rpc - 1) / rpc;
    // staging room for the block's rows at up to 1.25 times the mean row
    // occupancy (hits 12 B; bin index about one entry per hit, at most 2n + 3);
    // blocks with denser rows read global memory
    const long long avg = (b.N + (long long)b.I * NR - 1) / std::max(1LL, (long long)b.I * NR);
    const long long n125 = (5 * avg + 3) / 4;
    long long stage = (long long)(rpc + 2) * (12 * n125 + 4 * (n125 + 4)) + 64;
    stage = std::min<long long>(LINK_STAGE_MAX, std::max<long long>(4096, (stage + 15) / 16 * 16));
    int max_dx = 0;
    for (int r = 0; r + 1 < NR; ++r) max_dx = std::max(max_dx, b.par.qx[r + 1] - b.par.qx[r]);
    if (max_dx <= 16384)
      k_links<true><<<b.I * nrb, LINK_THREADS, stage, s>>>(b, rpc, (int)stage);
    else
      k_links<false><<<b.I * nrb, LINK_THREADS, stage, s>>>(b, rpc, (int)stage);
  }
  mark(5);
  const int gN = (int)((b.N + 255) / 256) < c.num_sms * 8 ? (int)((b.N + 255) / 256) : c.num_sms * 8;
  k_clean_start<<<gN > 0 ? gN : 1, 256, 0, s>>>(b);
  scan_i32(b.flags, b.start_ex, b.N, b.scan_tmp, c.grid_scan, s);
  k_starts<<<gN > 0 ? gN : 1, 256, 0, s>>>(b);
  mark(6);
  if (queued)
    tpc_launch_tracklets_queued(b, c, s);
  else
    tpc_launch_tracklets(b, c, s);
  mark(7);
  // a warp per tracklet: enough blocks for every resident warp slot
  k_select_max<<<c.num_sms * 8, 256, 0, s>>>(b);
  k_select_own<<<c.num_sms * 8, 256, 0, s>>>(b);
  scan_u64_dev(b.tl_cnt, b.tl_ex, b.start_ex + b.N, b.scan_tmp, c.grid_scan, s);
  mark(8);
  k_output<<<c.num_sms * 8, 256, 0, s>>>(b);
  k_counts<<<1, 1, 0, s>>>(b);
  mark(9);
  return cudaGetLastError();
}
}  // namespace

cudaError_t tpc_launch_plain(const Buffers& b, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev) {
  return launch_stages(b, c, s, ev, false);
}

cudaError_t tpc_launch_batched(const Buffers& b, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev) {
  return launch_stages(b, c, s, ev, true);
}
