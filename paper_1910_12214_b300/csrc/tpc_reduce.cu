// Data-reduction kernels (Sec. 4): the cluster codec (step 2).
//
// The codec is a pure stream: 28 bytes of float/int32 properties in, 13 bytes
// of codes out per cluster, no reuse.  It is bound by HBM bandwidth, so the
// design is about moving bytes: each thread converts four consecutive clusters
// with 16-byte loads of every input array and one vector store per output array
// (8-, 16- or 4-byte wide), in a grid sized to the SM count; unaligned arrays
// take a scalar path with the same arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "tpc_internal.cuh"

namespace {

// Fixed point: nearest integer of v * scale (an exact product for a power-of-two
// scale), ties to even, saturated to [lo, hi]; NaN -> 0.
__device__ __forceinline__ int fix_sat(float v, float scale, int lo, int hi) {
  const float s = rintf(v * scale);
  if (s != s) return 0;
  if (s <= (float)lo) return lo;
  if (s >= (float)hi) return hi;
  return (int)s;
}

// Dynamic precision: keep the leading one of v and the n bits after it, round
// the dropped bits half upward, clamp to `top` (the largest value of the field
// with n bits after its leading one).  v = 0 has no leading one: __clz gives 32
// and nothing is dropped.
__device__ __forceinline__ unsigned dyn_prec(unsigned v, int n, unsigned top) {
  const int drop = (31 - __clz(v)) - n;
  if (drop > 0) v = ((v + (1u << (drop - 1))) >> drop) << drop;
  return min(v, top);
}

__device__ __forceinline__ int row_code(int row, int n_rows) { return (row >= 0 && row < n_rows) ? row : 0; }
__device__ __forceinline__ int charge(float q) { return (int)dyn_prec((unsigned)fix_sat(q, 1.f, 0, 65535), 4, 0xF800u); }
__device__ __forceinline__ int size(float s) { return (int)dyn_prec((unsigned)fix_sat(s, 128.f, 0, 255), 3, 0xF0u); }
__device__ __forceinline__ unsigned pack16(int a, int b) { return (unsigned)(a & 0xffff) | ((unsigned)b << 16); }
__device__ __forceinline__ unsigned pack8(int a, int b, int c, int d) {
  return (unsigned)a | ((unsigned)b << 8) | ((unsigned)c << 16) | ((unsigned)d << 24);
}
__device__ __forceinline__ bool finite4(float4 v) { return isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w); }

// Bad clusters of a quad (row out of range or a non-finite value).
__device__ __forceinline__ int bad_count(float4 y, float4 z, int4 r, float4 qt, float4 qm, float4 sy, float4 sz,
                                         int n_rows) {
  auto ok = [&](int row, float a, float b, float c, float d, float e, float f) {
    return row >= 0 && row < n_rows && isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d) && isfinite(e) &&
           isfinite(f);
  };
  if (finite4(y) && finite4(z) && finite4(qt) && finite4(qm) && finite4(sy) && finite4(sz) &&
      (unsigned)r.x < (unsigned)n_rows && (unsigned)r.y < (unsigned)n_rows && (unsigned)r.z < (unsigned)n_rows &&
      (unsigned)r.w < (unsigned)n_rows)
    return 0;
  return (int)!ok(r.x, y.x, z.x, qt.x, qm.x, sy.x, sz.x) + (int)!ok(r.y, y.y, z.y, qt.y, qm.y, sy.y, sz.y) +
         (int)!ok(r.z, y.z, z.z, qt.z, qm.z, sy.z, sz.z) + (int)!ok(r.w, y.w, z.w, qt.w, qm.w, sy.w, sz.w);
}

struct Codes {
  int y, z, row, qt, qm, sy, sz;
};

__device__ __forceinline__ Codes encode_one(float y, float z, int row, float qt, float qm, float sy, float sz,
                                            int n_rows, bool& bad) {
  bad = !(row >= 0 && row < n_rows && isfinite(y) && isfinite(z) && isfinite(qt) && isfinite(qm) &&
          isfinite(sy) && isfinite(sz));
  Codes c;
  c.y = fix_sat(y, 64.f, -32768, 32767);
  c.z = fix_sat(z, 64.f, INT32_MIN, INT32_MAX);
  c.row = row_code(row, n_rows);
  c.qt = charge(qt);
  c.qm = charge(qm);
  c.sy = size(sy);
  c.sz = size(sz);
  return c;
}

// One warp-aggregated add of the warp's bad clusters.
__device__ __forceinline__ void count_bad(int nbad, unsigned long long* n_bad) {
  const unsigned m = __ballot_sync(0xffffffffu, nbad != 0);
  if (!m) return;
  int s = nbad;
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(n_bad, (unsigned long long)s);
}

// Vector path: quads [0, nq) with 16-byte loads; the tail (n % 4 clusters) is
// done by the first threads of the grid.
__global__ void __launch_bounds__(256, 4) k_encode_vec(CodecIn in, CodecOut out, long long n, int n_rows,
                                                    unsigned long long* n_bad) {
  const long long nq = n >> 2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long iters = (nq + stride - 1) / stride;  // uniform trip count: every lane reaches the ballot
  int nbad = 0;
  for (long long it = 0; it < iters; ++it) {
    const long long q = i0 + it * stride;
    if (q < nq) {
      const float4 y = __ldcs(reinterpret_cast<const float4*>(in.y) + q);
      const float4 z = __ldcs(reinterpret_cast<const float4*>(in.z) + q);
      const int4 r = __ldcs(reinterpret_cast<const int4*>(in.row) + q);
      const float4 qt = __ldcs(reinterpret_cast<const float4*>(in.qt) + q);
      const float4 qm = __ldcs(reinterpret_cast<const float4*>(in.qm) + q);
      const float4 sy = __ldcs(reinterpret_cast<const float4*>(in.sy) + q);
      const float4 sz = __ldcs(reinterpret_cast<const float4*>(in.sz) + q);
      // one output field at a time keeps few values live
      nbad += bad_count(y, z, r, qt, qm, sy, sz, n_rows);
      __stcs(reinterpret_cast<uint2*>(out.y) + q,
             make_uint2(pack16(fix_sat(y.x, 64.f, -32768, 32767), fix_sat(y.y, 64.f, -32768, 32767)),
                        pack16(fix_sat(y.z, 64.f, -32768, 32767), fix_sat(y.w, 64.f, -32768, 32767))));
      __stcs(reinterpret_cast<int4*>(out.z) + q,
             make_int4(fix_sat(z.x, 64.f, INT32_MIN, INT32_MAX), fix_sat(z.y, 64.f, INT32_MIN, INT32_MAX),
                       fix_sat(z.z, 64.f, INT32_MIN, INT32_MAX), fix_sat(z.w, 64.f, INT32_MIN, INT32_MAX)));
      __stcs(reinterpret_cast<unsigned*>(out.row) + q,
             pack8(row_code(r.x, n_rows), row_code(r.y, n_rows), row_code(r.z, n_rows), row_code(r.w, n_rows)));
      __stcs(reinterpret_cast<uint2*>(out.qt) + q, make_uint2(pack16(charge(qt.x), charge(qt.y)),
                                                              pack16(charge(qt.z), charge(qt.w))));
      __stcs(reinterpret_cast<uint2*>(out.qm) + q, make_uint2(pack16(charge(qm.x), charge(qm.y)),
                                                              pack16(charge(qm.z), charge(qm.w))));
      __stcs(reinterpret_cast<unsigned*>(out.sy) + q, pack8(size(sy.x), size(sy.y), size(sy.z), size(sy.w)));
      __stcs(reinterpret_cast<unsigned*>(out.sz) + q, pack8(size(sz.x), size(sz.y), size(sz.z), size(sz.w)));
    }
  }
  const long long t = 4 * nq + i0;  // tail: at most 3 clusters
  if (t < n) {
    bool b;
    const Codes c = encode_one(in.y[t], in.z[t], in.row[t], in.qt[t], in.qm[t], in.sy[t], in.sz[t], n_rows, b);
    nbad += (int)b;
    out.y[t] = (int16_t)c.y;
    out.z[t] = c.z;
    out.row[t] = (uint8_t)c.row;
    out.qt[t] = (uint16_t)c.qt;
    out.qm[t] = (uint16_t)c.qm;
    out.sy[t] = (uint8_t)c.sy;
    out.sz[t] = (uint8_t)c.sz;
  }
  count_bad(nbad, n_bad);
}

// Scalar path for arrays without the vector alignment.
__global__ void __launch_bounds__(256) k_encode_scalar(CodecIn in, CodecOut out, long long n, int n_rows,
                                                       unsigned long long* n_bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long iters = (n + stride - 1) / stride;
  int nbad = 0;
  for (long long it = 0; it < iters; ++it) {
    const long long t = i0 + it * stride;
    if (t < n) {
      bool b;
      const Codes c = encode_one(in.y[t], in.z[t], in.row[t], in.qt[t], in.qm[t], in.sy[t], in.sz[t], n_rows, b);
      nbad += (int)b;
      out.y[t] = (int16_t)c.y;
      out.z[t] = c.z;
      out.row[t] = (uint8_t)c.row;
      out.qt[t] = (uint16_t)c.qt;
      out.qm[t] = (uint16_t)c.qm;
      out.sy[t] = (uint8_t)c.sy;
      out.sz[t] = (uint8_t)c.sz;
    }
  }
  count_bad(nbad, n_bad);
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace

bool codec_vector_ok(const CodecIn& in, const CodecOut& out) {
  return aligned(in.y, 16) && aligned(in.z, 16) && aligned(in.row, 16) && aligned(in.qt, 16) &&
         aligned(in.qm, 16) && aligned(in.sy, 16) && aligned(in.sz, 16) && aligned(out.z, 16) &&
         aligned(out.y, 8) && aligned(out.qt, 8) && aligned(out.qm, 8) && aligned(out.row, 4) &&
         aligned(out.sy, 4) && aligned(out.sz, 4);
}

cudaError_t launch_encode(const CodecIn& in, const CodecOut& out, long long n, int n_rows,
                          unsigned long long* n_bad, int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const bool vec = codec_vector_ok(in, out);
  const long long work = vec ? (n >> 2) : n;
  long long blocks = (work + threads - 1) / threads;
  blocks = blocks < 1 ? 1 : blocks;
  const long long cap = (long long)num_sms * (vec ? 4 : 8);  // one resident wave (vector path: <= 64 registers)
  if (blocks > cap) blocks = cap;
  if (vec)
    k_encode_vec<<<(unsigned)blocks, threads, 0, s>>>(in, out, n, n_rows, n_bad);
  else
    k_encode_scalar<<<(unsigned)blocks, threads, 0, s>>>(in, out, n, n_rows, n_bad);
  return cudaGetLastError();
}

// ============================================================================
// Cluster association, protection and removal masks (Sec. 4, cluster removal).
//
// Pass 1 (k_mask_assoc), one warp per track: every candidate (track, cluster)
// pair bids the 64-bit key (~bits(|q/pT|) << 32 | ~track) into the cluster's
// word with atomicMax, so the highest pT wins and equal pT goes to the smaller
// track index whatever the order of the bids.  The lanes first bid for the
// track's own clusters (attachment), then take one pad row each of the track's
// row span, place the track on the row, and scan the bins of the tracker's
// y-z grid that overlap the tube's bounding box, bidding for every hit inside
// the tube (adjacency).  Pass 2 (k_mask_final), one thread per cluster: the
// winning track's pT, leg and local inclination at the cluster's row decide
// protection and the two strategies; the word is cleared for the next call.
#include <climits>

#include "tpc.h"

namespace {

constexpr float MASK_SNP_LIMIT = 0.9999f;  // the tracker's propagation validity
enum : uint8_t { M_ASSOC = 1, M_PROT = 2, M_REMOVE_A = 4, M_REMOVE_B = 8 };

// (y, z) where the track crosses the plane x = X (helix model of the tracker:
// sin phi linear in x, chord slope (s1 + s2) / (c1 + c2), arc length from
// asin); false where the track does not reach X.
__device__ __forceinline__ bool track_at(const tpc_track_t& t, float kB, float X, float* yo, float* zo) {
  const float dx = X - t.x_ref;
  const float kappa = kB * t.qpt;
  const float s1 = t.snp, s2 = s1 - kappa * dx;
  if (!(fabsf(s1) < MASK_SNP_LIMIT) || !(fabsf(s2) < MASK_SNP_LIMIT)) return false;
  const float c1 = sqrtf(1.0f - s1 * s1), c2 = sqrtf(1.0f - s2 * s2);
  const float T = (s1 + s2) / (c1 + c2);
  const float w = sqrtf(1.0f + T * T);
  const float u = 0.5f * kappa * fabsf(dx) * w;
  if (!(fabsf(u) < 1.0f)) return false;
  float f;
  if (fabsf(u) < 0.1f) {
    const float u2 = u * u;
    f = 1.0f + u2 * (1.0f / 6.0f + u2 * (3.0f / 40.0f + u2 * (5.0f / 112.0f)));
  } else {
    f = asinf(u) / u;
  }
  *yo = t.y + dx * T;
  *zo = t.z + t.tgl * (dx * w * f);
  return true;
}

// bins [a, e] of the values [lo, hi] along one axis of a row grid; e < a if none
__device__ __forceinline__ void axis_bins(long long lo, long long hi, int vmin, int shift, int nbin, int* a, int* e) {
  const long long vmax = (long long)vmin + ((long long)nbin << shift) - 1;
  if (nbin == 0 || hi < vmin || lo > vmax) {
    *a = 0;
    *e = -1;
    return;
  }
  *a = lo <= vmin ? 0 : (int)((lo - vmin) >> shift);
  const long long t = (hi - vmin) >> shift;
  *e = t < nbin - 1 ? (int)t : nbin - 1;
}

// Bids `key` for every hit of grid row `ri` inside the tube around (yt, zt).
__device__ __forceinline__ void scan_row(const MaskArgs& a, const RowInfo& ri, float yt, float zt, float tube2,
                                         unsigned long long key) {
  const float Q = 1.0f / TPC_QSCALE;
  // the tube's bounding box in quanta (2 quanta of margin) and its bins
  const int qy0 = (int)floorf((yt - a.tube) * TPC_QSCALE) - 2, qy1 = (int)ceilf((yt + a.tube) * TPC_QSCALE) + 2;
  const int qz0 = (int)floorf((zt - a.tube) * TPC_QSCALE) - 2, qz1 = (int)ceilf((zt + a.tube) * TPC_QSCALE) + 2;
  int iy0, iy1, iz0, iz1;
  axis_bins(qy0, qy1, ri.ymin, ri.shift, ri.ny, &iy0, &iy1);
  axis_bins(qz0, qz1, ri.zmin, ri.shift, ri.nz, &iz0, &iz1);
  if (iz1 < iz0 || iy1 < iy0) return;
  for (int iy = iy0; iy <= iy1; iy += 2) {
    // the hit ranges of two y-bin rows at once (bins iz0..iz1 of a y-bin row are contiguous)
    const int b0 = ri.bin0 + iy * ri.nz;
    const bool two = iy + 1 <= iy1;
    const int a0 = a.first[b0 + iz0], e0 = a.first[b0 + iz1 + 1];
    const int a1 = two ? a.first[b0 + ri.nz + iz0] : 0, e1 = two ? a.first[b0 + ri.nz + iz1 + 1] : 0;
    const int n0 = e0 - a0, total = n0 + (e1 - a1);
    // candidates four at a time: four independent loads in flight, an integer
    // test against the box, then the distance of the survivors
    for (int j0 = 0; j0 < total; j0 += 4) {
      int4 q[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = j0 + k;
        q[k] = j < total ? a.s_hit[j < n0 ? a0 + j : a1 + (j - n0)] : make_int4(INT_MIN, INT_MIN, 0, 0);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (q[k].x < qy0 || q[k].x > qy1 || q[k].y < qz0 || q[k].y > qz1) continue;
        const float dy = (float)q[k].x * Q - yt, dz = (float)q[k].y * Q - zt;
        if (dy * dy + dz * dz <= tube2) atomicMax(a.assoc + q[k].z, key);
      }
    }
  }
}

__global__ void k_mask_assoc(const __grid_constant__ MaskArgs a, const __grid_constant__ DevParams par) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long n_trk = a.counts ? (long long)a.counts[0] : a.n_trk;
  const long long n_ids = a.counts ? (long long)a.counts[1] : a.n_ids;
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const float tube2 = a.tube * a.tube;
  const int NR = par.n_rows;
  for (long long t = warp; t < n_trk; t += n_warps) {
    const tpc_track_t T = trk[t];
    const long long first = T.first_cluster, cnt = T.n_clusters;
    if (T.item >= (uint32_t)a.I || first + cnt > n_ids) {
      if (lane == 0) atomicOr(a.err, TPC_DERR_BAD_TRACK);
      continue;
    }
    if (cnt == 0) continue;
    const unsigned long long key =
        ((unsigned long long)(~__float_as_uint(fabsf(T.qpt))) << 32) | (0xFFFFFFFFull - (unsigned long long)t);
    // attachment: the track's own clusters
    bool bad = false;
    for (long long j = lane; j < cnt; j += 32) {
      const uint32_t id = a.ids[first + j];
      if (id < (uint32_t)a.N)
        atomicMax(a.assoc + id, key);
      else
        bad = true;
    }
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) atomicOr(a.err, TPC_DERR_BAD_TRACK);
      continue;
    }
    // adjacency: the tube on every row of the span
    const int ra = a.row[a.ids[first]], rb = a.row[a.ids[first + cnt - 1]];
    const int lo = max(0, min(ra, rb)), hi = min(NR - 1, max(ra, rb));
    // one row per lane; the next row's crossing point and grid record are
    // requested before the current row's bins are scanned (software pipeline)
    int r = lo + lane;
    bool ok = false;
    float yt = 0.f, zt = 0.f;
    RowInfo ri{};
    if (r <= hi && (ok = track_at(T, par.kB, par.x[r], &yt, &zt))) ri = a.rows[(long long)T.item * NR + r];
    while (r <= hi) {
      const int rn = r + 32;
      bool okn = false;
      float ytn = 0.f, ztn = 0.f;
      RowInfo rin{};
      if (rn <= hi && (okn = track_at(T, par.kB, par.x[rn], &ytn, &ztn))) rin = a.rows[(long long)T.item * NR + rn];
      if (ok && ri.n > 0) {
        yt = fminf(1.0e6f, fmaxf(-1.0e6f, yt));  // keeps the box arithmetic in range (NaN: no hit passes)
        zt = fminf(1.0e6f, fmaxf(-1.0e6f, zt));
        scan_row(a, ri, yt, zt, tube2, key);
      }
      r = rn;
      ok = okn;
      yt = ytn;
      zt = ztn;
      ri = rin;
    }
  }
}

// Mask and owner of one cluster from its association word.
__device__ __forceinline__ void final_one(const MaskArgs& a, const DevParams& par, const tpc_track_t* trk,
                                          unsigned long long key, int r, uint8_t* m, int* w) {
  *m = M_REMOVE_B;
  *w = -1;
  if (!key) return;
  const int t = (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
  const float x_ref = trk[t].x_ref, snp = trk[t].snp, qpt = trk[t].qpt;
  const float X = (r >= 0 && r < par.n_rows) ? par.x[r] : x_ref;
  const float s = fabsf(snp - par.kB * qpt * (X - x_ref));
  const bool prot = fabsf(qpt) < a.max_qpt && (!a.leg || a.leg[t] == 0) && s < a.max_snp;
  *m = prot ? (M_ASSOC | M_PROT) : (M_ASSOC | M_REMOVE_A | M_REMOVE_B);
  *w = t;
}

// VEC: four clusters per thread with 16-byte loads of the words and rows and
// vector stores of masks and owners (row 16-, mask 4-, owner 16-byte aligned);
// the words are cleared for the next call.
template <bool VEC>
__global__ void k_mask_final(const __grid_constant__ MaskArgs a, const __grid_constant__ DevParams par) {
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long done = 0;
  if constexpr (VEC) {
    const long long nq = (long long)a.N >> 2;
    ulonglong2* w2 = reinterpret_cast<ulonglong2*>(a.assoc);
    for (long long q = i0; q < nq; q += stride) {
      const ulonglong2 k01 = w2[2 * q], k23 = w2[2 * q + 1];
      const int4 r = reinterpret_cast<const int4*>(a.row)[q];
      if (k01.x | k01.y) w2[2 * q] = make_ulonglong2(0, 0);
      if (k23.x | k23.y) w2[2 * q + 1] = make_ulonglong2(0, 0);
      uint8_t m0, m1, m2, m3;
      int o0, o1, o2, o3;
      final_one(a, par, trk, k01.x, r.x, &m0, &o0);
      final_one(a, par, trk, k01.y, r.y, &m1, &o1);
      final_one(a, par, trk, k23.x, r.z, &m2, &o2);
      final_one(a, par, trk, k23.y, r.w, &m3, &o3);
      reinterpret_cast<unsigned*>(a.mask)[q] =
          (unsigned)m0 | ((unsigned)m1 << 8) | ((unsigned)m2 << 16) | ((unsigned)m3 << 24);
      if (a.owner) reinterpret_cast<int4*>(a.owner)[q] = make_int4(o0, o1, o2, o3);
    }
    done = 4 * nq;
  }
  for (long long c = done + i0; c < a.N; c += stride) {
    const unsigned long long key = a.assoc[c];
    if (key) a.assoc[c] = 0;
    uint8_t m;
    int o;
    final_one(a, par, trk, key, a.row[c], &m, &o);
    a.mask[c] = m;
    if (a.owner) a.owner[c] = o;
  }
}

}  // namespace

cudaError_t launch_masks(const MaskArgs& a, const DevParams& par, int num_sms, cudaStream_t s, cudaEvent_t* ev) {
  if (a.N <= 0) return cudaSuccess;
  // grid-stride kernels sized to one resident wave
  static int per_sm[3] = {0, 0, 0};
  if (!per_sm[0]) {
    cudaError_t e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_mask_assoc, 256, 0)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_mask_final<true>, 256, 0)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], k_mask_final<false>, 256, 0)) != cudaSuccess) {
      per_sm[0] = 0;
      return e;
    }
    for (int& v : per_sm) v = v < 1 ? 1 : v;
  }
  auto al = [](const void* p, uintptr_t n) { return (reinterpret_cast<uintptr_t>(p) & (n - 1)) == 0; };
  const bool vec = al(a.row, 16) && al(a.mask, 4) && (!a.owner || al(a.owner, 16)) && al(a.assoc, 16);
  if (ev) cudaEventRecord(ev[0], s);
  k_mask_assoc<<<num_sms * per_sm[0], 256, 0, s>>>(a, par);
  if (ev) cudaEventRecord(ev[1], s);
  long long blocks = (((long long)a.N >> (vec ? 2 : 0)) + 255) / 256;
  const long long cap = (long long)num_sms * per_sm[vec ? 1 : 2];
  blocks = blocks < 1 ? 1 : (blocks > cap ? cap : blocks);
  if (vec)
    k_mask_final<true><<<(unsigned)blocks, 256, 0, s>>>(a, par);
  else
    k_mask_final<false><<<(unsigned)blocks, 256, 0, s>>>(a, par);
  if (ev) cudaEventRecord(ev[2], s);
  return cudaGetLastError();
}

// ============================================================================
// Cluster compression (Sec. 4, steps 3 and 4).
//
// Entropy reduction: clusters not attached to a track are taken in the
// tracker's canonical order (the cells of each pad row's y-z grid, y-major,
// then the cluster index) and stored as zigzag differences of their y and z
// codes to the previous unattached cluster of the row; attached clusters are
// stored track by track as the row increment and the residuals of their codes
// to the track's prediction.  The prediction is a fixed sequence of correctly
// rounded float32 operations (explicit _rn intrinsics: no contraction into
// fused multiply-adds), so any decoder that performs the same sequence
// reproduces it bit for bit.
//
// Entropy coding: each symbol stream is split into byte planes, each plane is
// coded by rANS (32-bit states, 16-bit renormalisation, frequencies scaled to
// 2^12) in chunks of 8192 symbols, one warp per chunk with symbol i of the
// chunk on lane i mod 32.  Encoding runs backwards; at every step the lanes
// that renormalise place their 16-bit word by a ballot and a population count,
// so the words land in exactly the order a decoder warp reads them.
namespace {

enum { C_UNATT_N, C_DY, C_DZ, C_DROW, C_RY, C_RZ, C_QT, C_QM, C_SY, C_SZ, C_TRK_N };
constexpr int SCAN_TILE = 8192;  // elements per block of the scans (1024 threads x 8)

__device__ __forceinline__ unsigned long long zigzag(long long v) {
  return v >= 0 ? (unsigned long long)v << 1 : (((unsigned long long)(-(v + 1))) << 1) | 1ull;
}

// code (step 2^-6 cm) of a predicted coordinate; 0 where it is not finite or out of reach
__device__ __forceinline__ long long pred_code(float v) {
  if (!(fabsf(v) < 1.0e17f)) return 0;
  return __double2ll_rn((double)v * 64.0);
}

// The track model's (y, z) codes at pad-row radius X.
__device__ void predict_codes(const tpc_track_t& t, float kB, float X, long long* py, long long* pz) {
  const float dx = __fsub_rn(X, t.x_ref);
  const float kappa = __fmul_rn(kB, t.qpt);
  const float s2 = fminf(fmaxf(__fsub_rn(t.snp, __fmul_rn(kappa, dx)), -0.9999f), 0.9999f);
  const float s1 = fminf(fmaxf(t.snp, -0.9999f), 0.9999f);
  const float c1 = __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(s1, s1)));
  const float c2 = __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(s2, s2)));
  const float T = __fdiv_rn(__fadd_rn(s1, s2), __fadd_rn(c1, c2));
  const float y = __fadd_rn(t.y, __fmul_rn(dx, T));
  const float chord = __fmul_rn(dx, __fsqrt_rn(__fadd_rn(1.0f, __fmul_rn(T, T))));
  const float a = fminf(fabsf(__fmul_rn(__fmul_rn(0.5f, kappa), chord)), 1.0f);
  float g = 1.0f;  // asin(a) / a by two half-angle steps and a series to a^8
  if (a > 1e-6f) {
    const float a1 =
        __fdiv_rn(a, __fsqrt_rn(__fmul_rn(2.0f, __fadd_rn(1.0f, __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(a, a)))))));
    const float a2 =
        __fdiv_rn(a1, __fsqrt_rn(__fmul_rn(2.0f, __fadd_rn(1.0f, __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(a1, a1)))))));
    const float t2 = __fmul_rn(a2, a2);
    float ser = __fmul_rn(t2, 35.0f / 1152.0f);
    ser = __fmul_rn(t2, __fadd_rn(5.0f / 112.0f, ser));
    ser = __fmul_rn(t2, __fadd_rn(3.0f / 40.0f, ser));
    ser = __fmul_rn(t2, __fadd_rn(1.0f / 6.0f, ser));
    ser = __fadd_rn(1.0f, ser);
    g = __fdiv_rn(__fmul_rn(__fmul_rn(4.0f, a2), ser), a);
  }
  const float z = __fadd_rn(t.z, __fmul_rn(t.tgl, __fmul_rn(chord, g)));
  *py = pred_code(y);
  *pz = pred_code(z);
}

// ---- exclusive scan of int32 values in place; a[n] receives the total
__global__ void __launch_bounds__(1024) k_scan_reduce(const int* a, long long n, int* partial) {
  __shared__ int ws[32];
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  int s = 0;
  for (int k = 0; k < 8; ++k) {
    const long long i = base + (long long)k * 1024 + threadIdx.x;
    if (i < n) s += a[i];
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = ws[threadIdx.x];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// block-wide exclusive scan of one value per thread (1024 threads)
__device__ __forceinline__ int block_exscan(int v, int* total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  __syncthreads();
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  if (w == 0) {
    int x = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    ws[lane] = x;
  }
  __syncthreads();
  *total = ws[31];
  return inc - v + (w ? ws[w - 1] : 0);
}

__global__ void __launch_bounds__(1024) k_scan_partials(int* partial, int nb) {
  int carry = 0;
  for (int b0 = 0; b0 < nb; b0 += 1024) {
    const int i = b0 + threadIdx.x;
    const int v = i < nb ? partial[i] : 0;
    int tot;
    const int ex = block_exscan(v, &tot);
    if (i < nb) partial[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) partial[nb] = carry;
}

__global__ void __launch_bounds__(1024) k_scan_apply(int* a, long long n, const int* partial, int nb) {
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  int carry = partial[blockIdx.x];
  for (int k = 0; k < 8; ++k) {
    const long long i = base + (long long)k * 1024 + threadIdx.x;
    const int v = i < n ? a[i] : 0;
    int tot;
    const int ex = block_exscan(v, &tot);
    if (i < n) a[i] = carry + ex;
    carry += tot;
  }
  if (blockIdx.x == nb - 1 && threadIdx.x == 0) a[n] = partial[nb];
}

cudaError_t scan_i32(int* a, long long n, int* tmp, cudaStream_t s) {
  const int nb = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
  if (nb == 0) return cudaMemsetAsync(a, 0, 4, s);
  k_scan_reduce<<<nb, 1024, 0, s>>>(a, n, tmp);
  k_scan_partials<<<1, 1024, 0, s>>>(tmp, nb);
  k_scan_apply<<<nb, 1024, 0, s>>>(a, n, tmp, nb);
  return cudaGetLastError();
}

// ---- symbols
__device__ __forceinline__ long long n_tracks_of(const CmpArgs& a) { return a.counts ? (long long)a.counts[0] : a.n_trk; }

// attachment flags and per-track cluster counts (one warp per track); a track
// outside the batch raises the error bit
__global__ void k_cmp_attach(const __grid_constant__ CmpArgs a, const __grid_constant__ DevParams par) {
  const int lane = threadIdx.x & 31;
  const long long n_trk = n_tracks_of(a);
  const long long n_ids = a.counts ? (long long)a.counts[1] : a.n_ids;
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_trk; t += nw) {
    const long long first = trk[t].first_cluster, cnt = trk[t].n_clusters;
    bool bad = trk[t].item >= (uint32_t)a.I || first + cnt > n_ids;
    int kept = 0;
    if (!bad)
      for (long long j = lane; j < cnt; j += 32) {
        const uint32_t c = a.ids[first + j];
        if (c >= (uint32_t)a.N) {
          bad = true;
        } else {
          a.attached[c] = 1;
          kept += (!a.keep || a.keep[c]) ? 1 : 0;
        }
      }
    bad = __any_sync(0xffffffffu, bad);
    for (int o = 16; o; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if (lane == 0) {
      a.trk_n[t] = bad ? 0 : kept;  // the clusters the track stores
      if (bad) atomicOr(a.err, TPC_DERR_BAD_TRACK);
    }
  }
}

// the codes of every cluster packed in one 16-byte record, in the input order
// (coalesced), so that the symbol kernels gather one sector per cluster
__global__ void k_cmp_records(const __grid_constant__ CmpArgs a, int n_rows) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += stride) {
    const int r = a.row[c];
    const unsigned ry = (unsigned)fix_sat(a.y[c], 64.f, -32768, 32767) & 0xffffu;
    a.rec[c] = make_int4(fix_sat(a.z[c], 64.f, INT32_MIN, INT32_MAX), (int)(ry | ((unsigned)charge(a.qt[c]) << 16)),
                         (int)((unsigned)charge(a.qm[c]) | ((unsigned)(r >= 0 && r < n_rows ? r : 0xffff) << 16)),
                         (int)((unsigned)size(a.sy[c]) | ((unsigned)size(a.sz[c]) << 8)));
  }
}
__device__ __forceinline__ int rec_y(const int4& q) { return (int)(int16_t)(q.y & 0xffff); }
__device__ __forceinline__ int rec_row(const int4& q) { return (int)((unsigned)q.z >> 16); }  // 0xffff = out of range

// unattached flags of the binned clusters, one warp per (item, row); the
// positions between items' binned ranges (clusters left out of the binning)
// keep the zero the array was cleared to
__global__ void k_cmp_flags(const __grid_constant__ CmpArgs a, int n_rows) {
  const int lane = threadIdx.x & 31;
  const long long G = (long long)a.I * n_rows;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
    const RowInfo ri = a.rows[g];
    for (int p = ri.pos0 + lane; p < ri.pos0 + ri.n; p += 32) {
      const int c = a.s_hit[p].z;
      a.kpos[p] = (a.attached[c] || (a.keep && !a.keep[c])) ? 0 : 1;
    }
  }
}

// compaction of the unattached clusters; the row's first one is marked
__global__ void k_cmp_unatt(const __grid_constant__ CmpArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < a.P; p += stride) {
    const int k = a.kpos[p];
    if (a.kpos[p + 1] == k) continue;  // attached
    const int4 h = a.s_hit[p];
    a.unatt_id[k] = h.z;
    a.unatt_first[k] = (uint8_t)(k == a.kpos[a.rows[h.w].pos0]);
  }
}

// Statistics of the symbol values, gathered by the kernels that produce them
// (so that no pass reads the values back): per block, the histograms of byte
// planes 0 and 1 of every stream in shared memory, flushed to a.hist, and per
// thread the largest value of each stream it writes, reduced per warp into
// a.vmax.  Planes 2..7 follow in k_cmp_hist_high where the largest value
// needs them.
constexpr int CMP_STAT_WORDS = TPC_CMP_STREAMS * 512;

__device__ __forceinline__ void stats_clear(unsigned* h) {
  for (int i = threadIdx.x; i < CMP_STAT_WORDS; i += blockDim.x) h[i] = 0u;
  __syncthreads();
}

__device__ __forceinline__ void stats_add(unsigned* h, int s, unsigned long long x, unsigned long long* mx) {
  atomicAdd(&h[s * 512 + (int)(x & 255u)], 1u);
  atomicAdd(&h[s * 512 + 256 + (int)((x >> 8) & 255u)], 1u);
  *mx = x > *mx ? x : *mx;
}

// every thread of the block calls it once, after its last value
template <int K>
__device__ __forceinline__ void stats_flush(const CmpArgs& a, const unsigned* h, const int (&streams)[K],
                                            unsigned long long (&mx)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    unsigned long long m = mx[k];
    for (int o = 16; o; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, m, o);
      m = u > m ? u : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(a.vmax + streams[k], m);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < CMP_STAT_WORDS; i += blockDim.x) {
    const unsigned c = h[i];
    if (c) atomicAdd(a.hist + (long long)(i >> 9) * 2048 + (i & 511), (unsigned long long)c);
  }
}

__global__ void __launch_bounds__(256) k_cmp_rowcounts(const __grid_constant__ CmpArgs a, int n_rows) {
  __shared__ unsigned h[CMP_STAT_WORDS];
  stats_clear(h);
  const int st[1] = {C_UNATT_N};
  unsigned long long mx[1] = {0ull};
  const long long G = (long long)a.I * n_rows;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += stride) {
    const RowInfo ri = a.rows[g];
    const unsigned long long v = ri.n > 0 ? (unsigned long long)(a.kpos[ri.pos0 + ri.n] - a.kpos[ri.pos0]) : 0ull;
    a.val[C_UNATT_N][g] = v;
    stats_add(h, C_UNATT_N, v, &mx[0]);
  }
  stats_flush(a, h, st, mx);
}

// the four property codes of a stored cluster (record q) at position k of the
// property streams; mx[0..3] are their running maxima
__device__ __forceinline__ void put_props(const CmpArgs& a, long long k, const int4& q, unsigned* h,
                                          unsigned long long* mx) {
  const unsigned long long qt = (unsigned)q.y >> 16, qm = (unsigned)q.z & 0xffffu;
  const unsigned long long sy = (unsigned)q.w & 0xffu, sz = ((unsigned)q.w >> 8) & 0xffu;
  a.val[C_QT][k] = qt;
  a.val[C_QM][k] = qm;
  a.val[C_SY][k] = sy;
  a.val[C_SZ][k] = sz;
  stats_add(h, C_QT, qt, mx + 0);
  stats_add(h, C_QM, qm, mx + 1);
  stats_add(h, C_SY, sy, mx + 2);
  stats_add(h, C_SZ, sz, mx + 3);
}

__global__ void __launch_bounds__(256) k_cmp_unatt_symbols(const __grid_constant__ CmpArgs a) {
  __shared__ unsigned h[CMP_STAT_WORDS];
  stats_clear(h);
  const int st[6] = {C_QT, C_QM, C_SY, C_SZ, C_DY, C_DZ};
  unsigned long long mx[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  const long long n_un = a.kpos[a.P];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_un; k += stride) {
    const int4 q = a.rec[a.unatt_id[k]];
    long long yp = 0, zp = 0;
    if (!a.unatt_first[k]) {
      const int4 b = a.rec[a.unatt_id[k - 1]];
      yp = rec_y(b);
      zp = b.x;
    }
    const unsigned long long dy = zigzag((long long)rec_y(q) - yp), dz = zigzag((long long)q.x - zp);
    a.val[C_DY][k] = dy;
    a.val[C_DZ][k] = dz;
    stats_add(h, C_DY, dy, &mx[4]);
    stats_add(h, C_DZ, dz, &mx[5]);
    put_props(a, k, q, h, mx);
  }
  stats_flush(a, h, st, mx);
}

// one warp per track: row increments, residuals to the prediction, charges
__global__ void __launch_bounds__(256) k_cmp_track_symbols(const __grid_constant__ CmpArgs a,
                                                            const __grid_constant__ DevParams par) {
  __shared__ unsigned h[CMP_STAT_WORDS];
  stats_clear(h);
  const int st[8] = {C_QT, C_QM, C_SY, C_SZ, C_DROW, C_RY, C_RZ, C_TRK_N};
  unsigned long long mx[8] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  const int lane = threadIdx.x & 31;
  const long long n_trk = n_tracks_of(a);
  const long long n_un = a.kpos[a.P];
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_trk; t += nw) {
    const tpc_track_t T = trk[t];
    const long long base = a.trk_n[t], stored = a.trk_n[t + 1] - base;
    // the track's clusters (all of them when it stores any; a bad track stores none)
    const long long cnt = stored > 0 ? (long long)T.n_clusters : 0;
    if (lane == 0) {
      a.val[C_TRK_N][t] = (unsigned long long)stored;
      stats_add(h, C_TRK_N, (unsigned long long)stored, &mx[7]);
    }
    int carry = 0;        // row of the previous stored cluster (0 before the first)
    long long done = 0;   // stored clusters of the previous rounds
    for (long long j0 = 0; j0 < cnt; j0 += 32) {
      const long long j = j0 + lane;
      const uint32_t c = j < cnt ? a.ids[T.first_cluster + j] : 0u;
      const bool act = j < cnt && (!a.keep || a.keep[c]);
      const int4 q = act ? a.rec[c] : make_int4(0, 0, 0, 0);
      const int r = rec_row(q);
      // the stored clusters of this round: rank among them, row of the previous one
      const unsigned m = __ballot_sync(0xffffffffu, act);
      const unsigned below = m & ((1u << lane) - 1u);
      const int src = below ? 31 - __clz(below) : 0;
      const int rsrc = __shfl_sync(0xffffffffu, r, src);
      const int rp = below ? rsrc : carry;
      const int last = m ? 31 - __clz(m) : 0;
      const int rlast = __shfl_sync(0xffffffffu, r, last);
      const long long pos = done + __popc(below);
      done += __popc(m);
      if (m) carry = rlast;
      if (!act) continue;
      if (r >= par.n_rows) {  // a cluster with a pad row out of range: the track cannot be stored
        atomicOr(a.err, TPC_DERR_BAD_TRACK);
        continue;
      }
      long long py, pz;
      predict_codes(T, par.kB, par.x[r], &py, &pz);
      const unsigned long long drow = zigzag((long long)(r - rp));
      const unsigned long long ry = zigzag((long long)rec_y(q) - py), rz = zigzag((long long)q.x - pz);
      a.val[C_DROW][base + pos] = drow;
      a.val[C_RY][base + pos] = ry;
      a.val[C_RZ][base + pos] = rz;
      stats_add(h, C_DROW, drow, &mx[4]);
      stats_add(h, C_RY, ry, &mx[5]);
      stats_add(h, C_RZ, rz, &mx[6]);
      put_props(a, n_un + base + pos, q, h, mx);
    }
  }
  stats_flush(a, h, st, mx);
}

// length of stream s from the device-side totals
__device__ __forceinline__ long long stream_len(const CmpArgs& a, int s, int n_rows) {
  const long long n_un = a.kpos[a.P], n_att = a.trk_n[n_tracks_of(a)];
  switch (s) {
    case C_UNATT_N: return (long long)a.I * n_rows;
    case C_DY: case C_DZ: return n_un;
    case C_DROW: case C_RY: case C_RZ: return n_att;
    case C_TRK_N: return n_tracks_of(a);
    default: return n_un + n_att;
  }
}

// histograms of byte planes 2 .. n_planes-1 of stream s
__global__ void __launch_bounds__(256) k_cmp_hist_high(const __grid_constant__ CmpArgs a, int n_rows, int s,
                                                        int n_planes) {
  __shared__ unsigned int h[6][256];
  const long long n = stream_len(a, s, n_rows);
  for (int i = threadIdx.x; i < 6 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const unsigned long long* v = a.val[s];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long x = v[i];
    for (int p = 2; p < n_planes; ++p) atomicAdd(&h[p - 2][(x >> (8 * p)) & 255], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 6 * 256; i += blockDim.x) {
    const unsigned int c = (&h[0][0])[i];
    if (c) atomicAdd(a.hist + (long long)s * 2048 + 512 + i, (unsigned long long)c);
  }
}

// ---- coding
// index of the largest f (smallest index on ties) over a block of 256 threads
__device__ __forceinline__ int block_argmax256(unsigned f) {
  __shared__ unsigned long long red[8];
  unsigned long long key = ((unsigned long long)f << 32) | (255u - threadIdx.x);  // larger f, then smaller index
  for (int o = 16; o; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, key, o);
    key = u > key ? u : key;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = key;
  __syncthreads();
  unsigned long long m = red[0];
  for (int w = 1; w < 8; ++w) m = red[w] > m ? red[w] : m;
  return 255 - (int)(m & 0xffffffffu);
}

// frequencies of one (stream, plane), one block of 256 threads (one per byte
// value): the scaling rule of the format; the excess is removed one unit at a
// time from the current largest frequency, as the rule states
__global__ void __launch_bounds__(256) k_cmp_norm(const CmpPlane* planes, const unsigned long long* hist,
                                                  const int* plane_stream, uint16_t* ftab) {
  __shared__ unsigned long long s_tot;
  __shared__ int s_sum;
  const int q = blockIdx.x, b = threadIdx.x;
  const unsigned long long cnt = hist[(long long)plane_stream[q] * 2048 + 256 * planes[q].plane + b];
  if (b == 0) {
    s_tot = 0;
    s_sum = 0;
  }
  __syncthreads();
  atomicAdd(&s_tot, cnt);
  __syncthreads();
  const unsigned long long total = s_tot;
  unsigned f = cnt ? (unsigned)((cnt * 4096ull) / total) : 0u;
  if (cnt && f == 0) f = 1;
  atomicAdd(&s_sum, (int)f);
  __syncthreads();
  int sum = s_sum;
  if (total) {
    while (sum > 4096) {  // at most one unit per byte value raised to 1: <= 256 rounds
      const int m = block_argmax256(f);
      if (b == m) f -= 1;
      --sum;
    }
    if (sum < 4096) {
      const int m = block_argmax256(f);
      if (b == m) f += (unsigned)(4096 - sum);
    }
  }
  // cumulative frequencies: exclusive scan over the 256 byte values
  __shared__ unsigned ws[8];
  const int lane = b & 31, w = b >> 5;
  unsigned inc = f;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  __syncthreads();
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  unsigned base = 0;
  for (int k = 0; k < w; ++k) base += ws[k];
  ftab[512 * q + b] = (uint16_t)f;
  ftab[512 * q + 256 + b] = (uint16_t)(base + inc - f);
}

// one warp per chunk: interleaved rANS, words written backwards from the end
// of the chunk's scratch region (64 + n words), states last
__global__ void __launch_bounds__(128) k_cmp_rans(const CmpPlane* planes, const int* chunk_plane, int n_chunks,
                                                   const uint16_t* ftab, uint16_t* scratch, long long* chunk_ptr,
                                                   int* chunk_len) {
  // per warp and byte value: (f | c << 16, m), m the multiplier of the exact
  // division by f through a multiply-high (Granlund and Montgomery, "Division
  // by invariant integers using multiplication", 1994: for l = ceil(log2 f),
  // m = floor(2^32 (2^l - f) / f) + 1, x / f = (t + ((x - t) >> 1)) >> (l - 1)
  // with t = mulhi(m, x); f = 1 divides trivially)
  __shared__ uint2 tab[4][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ch = blockIdx.x * 4 + w;
  const bool live = ch < n_chunks;
  const int q = live ? chunk_plane[ch] : 0;
  const CmpPlane P = planes[q];
  for (int s = lane; s < 256; s += 32) {
    const uint32_t f = live ? ftab[512 * q + s] : 0u, c = live ? ftab[512 * q + 256 + s] : 0u;
    uint32_t m = 0;
    if (f >= 2) {
      const int l = 32 - __clz(f - 1);
      m = (uint32_t)((((1ull << 32) * ((1ull << l) - f)) / f) + 1);
    }
    tab[w][s] = make_uint2(f | (c << 16), m);
  }
  __syncwarp();
  if (!live) return;
  const long long c0 = ch - P.chunk0;
  const long long a0 = c0 * TPC_CMP_CHUNK;
  const int n = (int)min((long long)TPC_CMP_CHUNK, P.n - a0);
  uint16_t* buf = scratch + P.scratch0 + c0 * (TPC_CMP_CHUNK + 64);
  long long ptr = 64 + n;
  uint32_t x = 1u << 16;
  const int sh = 8 * P.plane;
  for (int k = (n + 31) / 32 - 1; k >= 0; --k) {
    const int i = k * 32 + lane;
    const bool act = i < n;
    const uint32_t sym = act ? (uint32_t)((P.v[a0 + i] >> sh) & 255ull) : 0u;
    const uint2 e = tab[w][sym];
    const uint32_t fs = e.x & 0xffffu, cs = e.x >> 16;
    const bool emit = act && (unsigned long long)x >= ((unsigned long long)fs << 20);
    const unsigned m = __ballot_sync(0xffffffffu, emit);
    ptr -= __popc(m);
    if (emit) {
      buf[ptr + __popc(m & ((1u << lane) - 1u))] = (uint16_t)(x & 0xffffu);
      x >>= 16;
    }
    if (act) {
      uint32_t qt = x;
      if (fs >= 2) {
        const uint32_t t = __umulhi(e.y, x);
        qt = (t + ((x - t) >> 1)) >> (31 - __clz(fs - 1));  // l - 1
      }
      x = (qt << 12) + (x - qt * fs) + cs;
    }
  }
  ptr -= 64;
  buf[ptr + 2 * lane] = (uint16_t)(x & 0xffffu);
  buf[ptr + 2 * lane + 1] = (uint16_t)(x >> 16);
  if (lane == 0) {
    chunk_ptr[ch] = P.scratch0 + c0 * (TPC_CMP_CHUNK + 64) + ptr;
    chunk_len[ch] = (int)(64 + n - ptr);
  }
}

// ---- blob assembly
__device__ __forceinline__ void put16(uint8_t* o, long long at, unsigned v) {
  *reinterpret_cast<uint16_t*>(o + at) = (uint16_t)v;
}
__device__ __forceinline__ void put32(uint8_t* o, long long at, unsigned v) {
  put16(o, at, v & 0xffffu);
  put16(o, at + 2, v >> 16);
}
__device__ __forceinline__ void put64(uint8_t* o, long long at, unsigned long long v) {
  put32(o, at, (unsigned)v);
  put32(o, at + 4, (unsigned)(v >> 32));
}

// One block: the header, every stream's and plane's fixed fields, each chunk's
// destination, the offset of the track table (written to out_size[1]) and the
// blob's size (out_size[0]).
__global__ void __launch_bounds__(1024) k_cmp_layout(const CmpPlane* planes, int n_planes, const int* stream_planes,
                                                      const long long* stream_n, const uint16_t* ftab,
                                                      const int* chunk_len, long long n_trk, uint32_t kB_bits,
                                                      unsigned long long xb0, unsigned long long xb1, int n_items,
                                                      int n_rows, long long n_unatt, long long n_att, uint8_t* out,
                                                      long long* out_size, long long* chunk_dst) {
  __shared__ long long at_s;
  if (threadIdx.x == 0) {
    put32(out, 0, 0x5A435054u);
    put32(out, 4, 1u);
    put32(out, 8, (unsigned)n_items);
    put32(out, 12, (unsigned)n_rows);
    put32(out, 16, (unsigned)n_trk);
    put32(out, 20, kB_bits);
    put64(out, 24, xb0);
    put64(out, 32, xb1);
    put64(out, 40, (unsigned long long)n_unatt);
    put64(out, 48, (unsigned long long)n_att);
    at_s = 56;
  }
  __syncthreads();
  int q = 0;
  for (int s = 0; s < TPC_CMP_STREAMS; ++s) {
    if (threadIdx.x == 0) {
      put64(out, at_s, (unsigned long long)stream_n[s]);
      put32(out, at_s + 8, (unsigned)stream_planes[s]);
      at_s += 12;
    }
    __syncthreads();
    for (int p = 0; p < stream_planes[s]; ++p, ++q) {
      const CmpPlane P = planes[q];
      const int nch = (int)((P.n + TPC_CMP_CHUNK - 1) / TPC_CMP_CHUNK);
      long long at = at_s;
      for (int i = threadIdx.x; i < 256; i += blockDim.x) put16(out, at + 2 * i, ftab[512 * q + i]);
      at += 512;
      if (threadIdx.x == 0) put32(out, at, (unsigned)nch);
      at += 4;
      for (int i = threadIdx.x; i < nch; i += blockDim.x) put32(out, at + 4 * i, (unsigned)chunk_len[P.chunk0 + i]);
      at += 4ll * nch;
      // destinations of the chunks' words: a block scan of their lengths
      long long carry = at;
      for (int b0 = 0; b0 < nch; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const int len = i < nch ? chunk_len[P.chunk0 + i] : 0;
        int tot;
        const int ex = block_exscan(len, &tot);
        if (i < nch) chunk_dst[P.chunk0 + i] = carry + 2ll * ex;
        carry += 2ll * tot;
      }
      __syncthreads();
      if (threadIdx.x == 0) at_s = carry;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    out_size[1] = at_s;
    out_size[0] = at_s + 28ll * n_trk;
  }
}

__global__ void k_cmp_copy(const uint16_t* scratch, const long long* chunk_ptr, const int* chunk_len,
                           const long long* chunk_dst, int n_chunks, uint8_t* out) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int ch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < n_chunks; ch += nw) {
    const uint16_t* src = scratch + chunk_ptr[ch];
    uint16_t* dst = reinterpret_cast<uint16_t*>(out + chunk_dst[ch]);
    for (int i = lane; i < chunk_len[ch]; i += 32) dst[i] = src[i];
  }
}

__global__ void k_cmp_tracks(const void* trk_v, long long n_trk, const long long* out_size, uint8_t* out) {
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(trk_v);
  const long long at0 = out_size[1];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_trk; t += stride) {
    const tpc_track_t& T = trk[t];
    const long long at = at0 + 28 * t;
    put32(out, at, __float_as_uint(T.x_ref));
    put32(out, at + 4, __float_as_uint(T.y));
    put32(out, at + 8, __float_as_uint(T.z));
    put32(out, at + 12, __float_as_uint(T.snp));
    put32(out, at + 16, __float_as_uint(T.tgl));
    put32(out, at + 20, __float_as_uint(T.qpt));
    put32(out, at + 24, T.item);
  }
}

}  // namespace

cudaError_t cmp_symbols(const CmpArgs& a, const DevParams& par, int num_sms, cudaStream_t s) {
  cudaError_t e;
  const int g = num_sms * 8;
  if ((e = cudaMemsetAsync(a.attached, 0, (size_t)a.N, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(a.vmax, 0, 8 * TPC_CMP_STREAMS, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(a.hist, 0, 8ull * TPC_CMP_STREAMS * 2048, s)) != cudaSuccess)
    return e;
  k_cmp_records<<<g, 256, 0, s>>>(a, par.n_rows);
  k_cmp_attach<<<g, 256, 0, s>>>(a, par);
  // the track counts' scan needs their number on the host side: own tracks are
  // counted on the device, so scan the capacity (unused entries are zero)
  if ((e = cudaMemsetAsync(a.kpos, 0, 4 * ((size_t)a.P + 1), s)) != cudaSuccess) return e;
  k_cmp_flags<<<g, 256, 0, s>>>(a, par.n_rows);
  if ((e = scan_i32(a.kpos, a.P, a.scan_tmp, s)) != cudaSuccess) return e;
  if ((e = scan_i32(a.trk_n, a.n_trk, a.scan_tmp + (a.P / SCAN_TILE + 2), s)) != cudaSuccess) return e;
  k_cmp_unatt<<<g, 256, 0, s>>>(a);
  k_cmp_rowcounts<<<g, 256, 0, s>>>(a, par.n_rows);
  k_cmp_unatt_symbols<<<g, 256, 0, s>>>(a);
  k_cmp_track_symbols<<<g, 256, 0, s>>>(a, par);
  return cudaGetLastError();
}

cudaError_t cmp_hist_high(const CmpArgs& a, const DevParams& par, int num_sms, const int* stream_planes,
                          cudaStream_t s) {
  for (int st = 0; st < TPC_CMP_STREAMS; ++st)
    if (stream_planes[st] > 2) k_cmp_hist_high<<<num_sms * 2, 256, 0, s>>>(a, par.n_rows, st, stream_planes[st]);
  return cudaGetLastError();
}

cudaError_t cmp_encode(const CmpPlane* planes, int n_planes, int n_chunks_total, const unsigned long long* hist,
                       const int* plane_stream, uint16_t* ftab, uint16_t* scratch, long long* chunk_ptr, int* chunk_len,
                       const int* chunk_plane, cudaStream_t s) {
  if (n_planes == 0) return cudaSuccess;
  k_cmp_norm<<<n_planes, 256, 0, s>>>(planes, hist, plane_stream, ftab);
  if (n_chunks_total) k_cmp_rans<<<(n_chunks_total + 3) / 4, 128, 0, s>>>(planes, chunk_plane, n_chunks_total, ftab, scratch, chunk_ptr, chunk_len);
  return cudaGetLastError();
}

cudaError_t cmp_layout(const CmpPlane* planes, int n_planes, const int* stream_planes, const long long* stream_n,
                       const uint16_t* ftab, const uint16_t* scratch, const long long* chunk_ptr, const int* chunk_len,
                       int n_chunks_total, const void* trk, long long n_trk, uint32_t kB_bits, double x_min,
                       double x_max, int n_items, int n_rows, long long n_unatt, long long n_att, uint8_t* out,
                       long long* out_size, long long* chunk_dst, cudaStream_t s) {
  unsigned long long xb0, xb1;
  memcpy(&xb0, &x_min, 8);
  memcpy(&xb1, &x_max, 8);
  k_cmp_layout<<<1, 1024, 0, s>>>(planes, n_planes, stream_planes, stream_n, ftab, chunk_len, n_trk, kB_bits, xb0, xb1,
                                  n_items, n_rows, n_unatt, n_att, out, out_size, chunk_dst);
  if (n_chunks_total) k_cmp_copy<<<(n_chunks_total + 7) / 8, 256, 0, s>>>(scratch, chunk_ptr, chunk_len, chunk_dst, n_chunks_total, out);
  if (n_trk) k_cmp_tracks<<<(int)std::min<long long>((n_trk + 255) / 256, 4096), 256, 0, s>>>(trk, n_trk, out_size, out);
  return cudaGetLastError();
}

// ============================================================================
// Sector-track merger (Sec. 4: the pieces of one track found in neighbouring
// sectors are joined, and the merged track is refitted).
//
// Every track gets its circle in the global frame (FP64, with FP32 and
// float-float copies); the tracks of each event and side are sorted by
// tan(lambda).  One warp per track finds, among the tracks of sectors k+1 and
// k-1 inside its tan(lambda) window, the compatible candidate of smallest
// score (a curvature chi2, the continuation on the better-measured circle,
// tan(lambda), z along the arc): FP32 prefilters with safe margins, then the
// tests in float-float.  A link joins two tracks that are each other's best
// in opposite directions.  Links are mutual and one per direction, so every
// group is a path through neighbouring sectors: a bounded walk labels it by
// its smallest index.  One warp per group then refits the group's clusters in
// the global frame (algebraic circle fit, then z against the arc): per-cluster
// sums in float-float, the solves in FP64 one group per thread.
namespace {

constexpr double MRG_WEDGE = 2.0 * 3.14159265358979323846 / 18.0;
constexpr int MRG_FIT_NACC = 14;                        // float-float sums of the refit
constexpr int MRG_FIT_SUMS = 4 + 2 * MRG_FIT_NACC + 2;  // floats per group record: n, members, mean, sums

// Float-float ("double-float") numbers for the compatibility tests and the
// refit's per-cluster sums: a value is hi + lo with |lo| <= ulp(hi) / 2, a
// 48-bit significand computed on
// the FP32 pipe, which the B300 has about 60 times wider than the FP64 one.
// The error-free transformations are Knuth's TwoSum, Dekker's Fast2Sum (valid
// for |a| >= |b|) and the fused-multiply-add TwoProduct; the additions are the
// "sloppy" form (absolute error a few 2^-46 of |a| + |b|, like an FP64 sum's
// 2^-53 of its terms).  Explicit _rn intrinsics keep the compiler from fusing
// or reordering any of it.
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const F2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ F2 f2_neg(F2 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ F2 f2_mul_f(F2 a, float b) {  // times a float
  const float p = __fmul_rn(a.hi, b);
  return fast_two_sum(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}

// square root by one Newton correction of the correctly rounded FP32 root
// (x + (a - x^2) / 2x, the residual a - x^2 formed exactly by TwoProduct)
__device__ __forceinline__ F2 f2_sqrt(F2 a) {
  if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
  const float x = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(x, x);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), __fmaf_rn(x, x, -p)), a.lo);
  return fast_two_sum(x, __fmul_rn(r, __fdividef(0.5f, x)));
}

// float-float form of a double known at compile time
struct F2c {
  float hi, lo;
  constexpr F2c(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};
constexpr F2c kF2_002(0.02), kF2_1em30(1e-30);

__device__ __forceinline__ F2 f2c(F2c c) { return {c.hi, c.lo}; }

__device__ __forceinline__ F2 f2_from(double v) {
  const float hi = (float)v;
  return {hi, (float)(v - (double)hi)};
}

__device__ __forceinline__ bool f2_less(F2 a, F2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

__device__ __forceinline__ bool f2_le(F2 a, F2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

__device__ __forceinline__ F2 f2_abs(F2 a) { return a.hi < 0.0f ? f2_neg(a) : a; }

// quotient by long division: q1 = a / b in FP32, the remainder a - q1 b formed
// in float-float, q2 = remainder / b
__device__ __forceinline__ F2 f2_div(F2 a, F2 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const F2 r = f2_add(a, f2_neg(f2_mul_f(b, q1)));
  return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

__device__ __forceinline__ F2 warp_sum(F2 v) {
  for (int o = 16; o; o >>= 1) {
    const F2 w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = f2_add(v, w);
  }
  return v;
}

enum { G_OK, G_XC, G_YC, G_R, G_X, G_Y, G_RAD, G_Z, G_TGL, G_QPT, G_VQ, G_SIGN, G_N };

__global__ void k_mrg_geom(const __grid_constant__ MrgArgs a) {
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_trk; t += stride) {
    const tpc_track_t T = trk[t];
    double* g = a.geo + G_N * t;
    const bool range_ok = T.item < (uint32_t)a.I && (long long)T.first_cluster + T.n_clusters <= a.n_ids;
    if (!range_ok || (t > 0 && trk[t - 1].item > T.item)) atomicOr(a.err, TPC_DERR_BAD_TRACK);
    const bool ok = fabsf(T.qpt) >= 1e-4f && range_ok;
    g[G_OK] = ok ? 1.0 : 0.0;
    a.pre[t] = make_float4(ok ? T.tgl : __int_as_float(0x7fc00000), T.qpt, sqrtf(fmaxf(T.cov[14], 0.f)),
                           T.qpt > 0.f ? 1.f : -1.f);
    if (!ok) {
      a.geo32[2 * t] = make_float4(0.f, 0.f, 0.f, 0.f);
      a.geo32[2 * t + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int k = 0; k < 4; ++k) a.geof2[4 * t + k] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const int s = (int)a.item_sector[T.item];
    const double ang = (double)(s % 18) * MRG_WEDGE, ca = cos(ang), sa = sin(ang);
    const double kap = a.kB * (double)T.qpt;
    const double snp = T.snp, csp = sqrt(fmax(0.0, 1.0 - snp * snp));
    const double lx = (double)T.x_ref + snp / kap, ly = (double)T.y - csp / kap;
    g[G_XC] = lx * ca - ly * sa;
    g[G_YC] = lx * sa + ly * ca;
    g[G_R] = 1.0 / fabs(kap);
    const double X = (double)T.x_ref * ca - (double)T.y * sa, Y = (double)T.x_ref * sa + (double)T.y * ca;
    g[G_X] = X;
    g[G_Y] = Y;
    g[G_RAD] = hypot(X, Y);
    g[G_Z] = T.z;
    g[G_TGL] = T.tgl;
    g[G_QPT] = T.qpt;
    g[G_VQ] = fmax(0.0, (double)T.cov[14]);
    g[G_SIGN] = T.qpt > 0.f ? 1.0 : -1.0;
    // the same quantities rounded to FP32 (var q/pT is a float: exact) for the prefilters
    a.geo32[2 * t] = make_float4((float)g[G_XC], (float)g[G_YC], (float)g[G_R], (float)g[G_VQ]);
    a.geo32[2 * t + 1] = make_float4((float)X, (float)Y, T.z, (float)g[G_RAD]);
    // and as float-float (z, tan lambda, q/pT and var q/pT are floats)
    const F2 fxc = f2_from(g[G_XC]), fyc = f2_from(g[G_YC]), fr = f2_from(g[G_R]), fx = f2_from(X), fy = f2_from(Y);
    a.geof2[4 * t] = make_float4(fxc.hi, fxc.lo, fyc.hi, fyc.lo);
    a.geof2[4 * t + 1] = make_float4(fr.hi, fr.lo, fx.hi, fx.lo);
    a.geof2[4 * t + 2] = make_float4(fy.hi, fy.lo, T.z, T.tgl);
    a.geof2[4 * t + 3] = make_float4(T.qpt, fmaxf(0.f, T.cov[14]), 0.f, 0.f);
  }
}

// first track of every item (tracks are sorted by item)
__global__ void k_mrg_item_first(const __grid_constant__ MrgArgs a) {
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= a.I; i += stride) {
    long long lo = 0, hi = a.n_trk;  // first t with item >= i
    while (lo < hi) {
      const long long m = (lo + hi) >> 1;
      if (trk[m].item < (uint32_t)i)
        lo = m + 1;
      else
        hi = m;
    }
    a.item_first[i] = (int)lo;
  }
}

// a non-negative score as an integer key: the bits of a non-negative double
// order like its value, and integer compares keep the reductions off the FP64 pipe
__device__ __forceinline__ unsigned long long score_key(double sc) { return (unsigned long long)__double_as_longlong(sc); }

// the same for a non-negative float-float score: the bits of hi, then lo's bits
// mapped to an order-preserving unsigned integer (hi, lo) compare like the value
__device__ __forceinline__ unsigned long long score_key(F2 sc) {
  const unsigned lo = __float_as_uint(sc.lo);
  return ((unsigned long long)__float_as_uint(sc.hi) << 32) | ((lo & 0x80000000u) ? ~lo : (lo | 0x80000000u));
}

// The merger's compatibility tests (curvature chi2, the reference point on the
// better-measured circle, tan(lambda), z continuity) and the score of a compatible pair, in
// float-float on the per-track records (geof2): a few 2^-46 relative, so every
// decision equals the exact one except within about 1e-13 of a limit.
struct TrkF2 {
  F2 xc, yc, r, x, y;
  float z, tgl, qpt, vq;
};

__device__ __forceinline__ TrkF2 load_trk_f2(const float4* g) {
  const float4 g0 = g[0], g1 = g[1], g2 = g[2], g3 = g[3];
  return {{g0.x, g0.y}, {g0.z, g0.w}, {g1.x, g1.y}, {g1.z, g1.w}, {g2.x, g2.y}, g2.z, g2.w, g3.x, g3.y};
}

__device__ __forceinline__ F2 f2_hypot(F2 dx, F2 dy) { return f2_sqrt(f2_add(f2_mul(dx, dx), f2_mul(dy, dy))); }

__device__ __forceinline__ bool mrg_compatible(const TrkF2& A, const TrkF2& B, bool a_inner, F2 kB3,
                                               unsigned long long* score) {
  // the cheap tests first (they reject almost every wrong pair): tan(lambda), then the curvature chi2
  const F2 dt = f2_abs(two_sum(A.tgl, -B.tgl));
  if (!f2_le(dt, f2c(kF2_002))) return false;
  const F2 dq = two_sum(A.qpt, -B.qpt);
  F2 vsum = two_sum(A.vq, B.vq);
  if (f2_less(vsum, f2c(kF2_1em30))) vsum = f2c(kF2_1em30);
  const F2 dq2 = f2_mul(dq, dq);
  if (!f2_le(dq2, f2_mul_f(vsum, 16.0f))) return false;
  const F2 chi2 = f2_div(dq2, vsum);
  const TrkF2& ref = A.vq <= B.vq ? A : B;
  const TrkF2& oth = A.vq <= B.vq ? B : A;
  const F2 L = f2_hypot(f2_add(oth.x, f2_neg(ref.x)), f2_add(oth.y, f2_neg(ref.y)));
  const F2 d = f2_abs(f2_add(f2_hypot(f2_add(oth.x, f2_neg(ref.xc)), f2_add(oth.y, f2_neg(ref.yc))), f2_neg(ref.r)));
  const F2 dlim = f2_add({1.0f, 0.0f}, f2_mul(f2_mul(kB3, f2_sqrt({ref.vq, 0.0f})), f2_mul(L, L)));
  const TrkF2& in = a_inner ? A : B;
  const TrkF2& out = a_inner ? B : A;
  const F2 c = f2_hypot(f2_add(out.x, f2_neg(in.x)), f2_add(out.y, f2_neg(in.y)));
  const F2 Rb = f2_mul_f(f2_add(A.r, B.r), 0.5f);
  const F2 arc = f2_mul(c, f2_add({1.0f, 0.0f}, f2_div(f2_mul(c, c), f2_mul_f(f2_mul(Rb, Rb), 24.0f))));
  const F2 dz = f2_abs(f2_add({out.z, 0.0f}, f2_neg(f2_add({in.z, 0.0f}, f2_mul_f(arc, in.tgl)))));
  const F2 sc = f2_add(f2_add(f2_add(f2_mul_f(chi2, 0.0625f), f2_div(d, dlim)), f2_div(dt, f2c(kF2_002))),
                       f2_mul_f(dz, 0.5f));
  *score = score_key(sc);
  return f2_le(d, dlim) && f2_le(dz, {2.0f, 0.0f});
}

// FP32 form of the continuity and dz tests of mrg_compatible that never rejects
// a pair the FP64 tests accept.  Inputs are the FP64 values rounded to FP32
// (relative error u = 2^-24 each).  With M the sum of the magnitudes entering a
// difference, a rounded difference is off by at most 2u M, a rounded hypot by
// 5u M, and the distance |h - R| by 7u (M + R); the limit 1 + 3 kB sqrt(V) L^2
// by 8u of its value plus 8u kB sqrt(V) M^2; dz by 8u times the magnitudes of
// its terms.  The margins below are about 20 times these bounds.  The reference
// (smaller var q/pT) is chosen alike in both precisions because the variance is
// a float; the inner track (smaller radius) too unless the rounded radii are
// equal, where the dz test is left to FP64.  A NaN or infinity passes.
__device__ __forceinline__ bool mrg_maybe_compatible(const float4* A32, const float4* B32, float tgl_a,
                                                     float tgl_b, float kB) {
  constexpr float e = 1e-5f;
  const float4 a0 = A32[0], a1 = A32[1], b0 = B32[0], b1 = B32[1];
  const bool a_ref = a0.w <= b0.w;
  const float4 r0 = a_ref ? a0 : b0, r1 = a_ref ? a1 : b1, o1 = a_ref ? b1 : a1;
  const float dxl = o1.x - r1.x, dyl = o1.y - r1.y;
  const float L2 = fmaf(dxl, dxl, dyl * dyl);
  const float ex = o1.x - r0.x, ey = o1.y - r0.y;
  const float d = fabsf(sqrtf(fmaf(ex, ex, ey * ey)) - r0.z);
  const float kv = 3.0f * kB * sqrtf(r0.w);
  const float Q = fabsf(o1.x) + fabsf(o1.y) + fabsf(r1.x) + fabsf(r1.y);
  const float Mc = fabsf(o1.x) + fabsf(o1.y) + fabsf(r0.x) + fabsf(r0.y) + r0.z;
  const float dlim = fmaf(kv, L2, 1.0f);
  if (d > dlim * (1.0f + e) + e * (kv * Q * Q + Mc) + 1e-6f) return false;
  if (a1.w == b1.w) return true;
  const bool a_in = a1.w < b1.w;
  const float4 in1 = a_in ? a1 : b1, out1 = a_in ? b1 : a1;
  const float tin = a_in ? tgl_a : tgl_b;
  const float cx = out1.x - in1.x, cy = out1.y - in1.y;
  const float c = sqrtf(fmaf(cx, cx, cy * cy));
  const float Rb = 0.5f * (a0.z + b0.z);
  const float t = c * c / (24.0f * Rb * Rb);
  const float arc = c * (1.0f + t);
  const float dz = fabsf(out1.z - fmaf(tin, arc, in1.z));
  const float Qz = fabsf(in1.x) + fabsf(in1.y) + fabsf(out1.x) + fabsf(out1.y);
  return !(dz > 2.0f + e * (fabsf(out1.z) + fabsf(in1.z) + fabsf(tin) * (arc + Qz) * (2.0f + 4.0f * t)) + 1e-6f);
}

// Tan(lambda)-sorted candidate lists, one per segment (the items of one event
// and side): every prefilter asks for |tan(lambda_a) -+ tan(lambda_b)| <= 0.0201,
// so a window of the sorted list holds every candidate that can pass, and the
// scans visit a few percent of the segment's tracks.  The selections are minima
// of (score, index), so the order of the visits does not change them.
constexpr int MRG_SORT_CAP = 16384;  // tracks of a segment sorted in shared memory (more: item-by-item scans)

__device__ __forceinline__ unsigned tgl_key(float v) {  // order-preserving bits; every NaN last
  const unsigned u = __float_as_uint(v);
  if (v != v) return 0xffffffffu;
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_mrg_seg_count(const __grid_constant__ MrgArgs a) {
  const int stride = gridDim.x * blockDim.x;
  for (int sg = blockIdx.x * blockDim.x + threadIdx.x; sg < a.S; sg += stride) {
    const int* it = a.seg_items + 19 * (long long)sg;
    int n = 0;
    for (int k = 0; k < 18; ++k)
      if (it[k] >= 0) n += a.item_first[it[k] + 1] - a.item_first[it[k]];
    a.seg_n[sg] = n;
  }
}

__global__ void __launch_bounds__(1024) k_mrg_seg_scan(const __grid_constant__ MrgArgs a) {
  __shared__ int wsum[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < a.S; base += 1024) {
    const int i = base + (int)threadIdx.x;
    const int v = i < a.S ? a.seg_n[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const int incl = x + (wid ? wsum[wid - 1] : 0) + carry;
    if (i < a.S) a.seg_off[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) a.seg_off[a.S] = carry;
}

// one block per segment: (key, track) pairs sorted ascending by a bitonic network in shared memory
__global__ void __launch_bounds__(1024) k_mrg_seg_sort(const __grid_constant__ MrgArgs a) {
  extern __shared__ unsigned long long sk[];
  __shared__ int s_first[18], s_pos[19];
  const int sg = blockIdx.x;
  const int* it = a.seg_items + 19 * (long long)sg;
  const int n = a.seg_n[sg];
  const bool ok = n <= min(a.sort_cap, MRG_SORT_CAP) && it[18] <= 18;
  if (threadIdx.x == 0) a.seg_ok[sg] = ok ? 1 : 0;
  if (!ok || n == 0) return;
  if (threadIdx.x < 32) {  // the listed items' track ranges and their offsets in the list
    const int k = threadIdx.x;
    const int item = k < 18 ? it[k] : -1;
    const int f = item >= 0 ? a.item_first[item] : 0, cnt = item >= 0 ? a.item_first[item + 1] - f : 0;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (k >= o) incl += y;
    }
    if (k < 18) {
      s_first[k] = f;
      s_pos[k] = incl - cnt;
    }
    if (k == 17) s_pos[18] = incl;
  }
  __syncthreads();
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 0; k < 18; ++k) {
    const int f = s_first[k], pos = s_pos[k], cnt = s_pos[k + 1] - pos;
    for (int j = threadIdx.x; j < cnt; j += blockDim.x)
      sk[pos + j] = ((unsigned long long)tgl_key(a.pre[f + j].x) << 32) | (unsigned)(f + j);
  }
  for (int p = n + threadIdx.x; p < P; p += blockDim.x) sk[p] = ~0ull;
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      __syncthreads();
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long x = sk[i], y = sk[l];
          if ((x > y) == ((i & k) == 0)) {
            sk[i] = y;
            sk[l] = x;
          }
        }
      }
    }
  __syncthreads();
  const int off = a.seg_off[sg];
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const unsigned long long x = sk[p];
    a.skey[off + p] = (unsigned)(x >> 32);
    a.sidx[off + p] = (int)(unsigned)x;
  }
}

// first position of keys[0, n) (ascending) holding a key >= target, found by the
// whole warp 32 ways at a time
__device__ __forceinline__ int warp_lower_bound(const unsigned* keys, int n, unsigned target) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) >> 5;
    const int p = lo + lane * step;
    const int c = __popc(__ballot_sync(0xffffffffu, p < hi && keys[p] < target));
    if (c == 0) return lo;
    const int nlo = lo + (c - 1) * step + 1;
    hi = min(hi, lo + c * step);
    lo = nlo;
  }
  const int p = lo + lane;
  return lo + __popc(__ballot_sync(0xffffffffu, p < hi && keys[p] < target));
}

// lane-local then warp-wide minimum of (score key, index)
__device__ __forceinline__ void keep_best(unsigned long long sc, long long b, unsigned long long* bs, long long* bi) {
  if (*bi < 0 || sc < *bs || (sc == *bs && b < *bi)) {
    *bs = sc;
    *bi = b;
  }
}

__device__ __forceinline__ long long warp_best(unsigned long long bs, long long bi) {
  for (int o = 16; o; o >>= 1) {
    const unsigned long long os = __shfl_xor_sync(0xffffffffu, bs, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oi >= 0) keep_best(os, oi, &bs, &bi);
  }
  return bi;
}

// one warp per track: the best compatible candidate in sector k+1 (d = 0) and k-1 (d = 1)
__global__ void k_mrg_best(const __grid_constant__ MrgArgs a) {
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const float kBf = (float)a.kB;
  for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < a.n_trk; t += nw) {
    const double* A = a.geo + G_N * t;
    const bool ok = __double_as_longlong(A[G_OK]) != 0;  // 1.0 or 0.0
    const int item = (int)trk[t].item;
    const float4 pa = a.pre[t];
    const int nb0 = ok ? a.nb_item[2 * item] : -1, nb1 = ok ? a.nb_item[2 * item + 1] : -1;
    unsigned long long bs[2] = {0, 0};
    long long bi[2] = {-1, -1};
    const TrkF2 TA = load_trk_f2(a.geof2 + 4 * t);
    const F2 kB3 = {a.kB3_hi, a.kB3_lo};
    // the tests of candidate b of direction d (the FP32 prefilter with margins wider
    // than any FP32 rounding of the FP64 tests; a NaN tan lambda fails every comparison)
    auto consider = [&](long long b, int d) {
      const float4 pb = a.pre[b];
      if (!(fabsf(pa.x - pb.x) <= 0.0201f) || pa.w != pb.w) return;
      const float dq = pa.y - pb.y, sq = pa.z * pa.z + pb.z * pb.z;
      if (!(dq * dq <= 16.2f * sq + 1e-28f)) return;
      if (!mrg_maybe_compatible(a.geo32 + 2 * t, a.geo32 + 2 * b, pa.x, pb.x, kBf)) return;
      // a track without a circle has a NaN tan lambda and the same sign test as G_SIGN: both were checked
      const TrkF2 B = load_trk_f2(a.geof2 + 4 * b);
      unsigned long long sc;
      if (mrg_compatible(TA, B, A[G_RAD] <= a.geo[G_N * b + G_RAD], kB3, &sc)) keep_best(sc, b, &bs[d], &bi[d]);
    };
    const int sg = (nb0 >= 0 || nb1 >= 0) ? a.item_seg[item] : -1;
    if (sg >= 0 && a.seg_ok[sg]) {
      if (pa.x == pa.x) {  // the window |tan(lambda_b) - tan(lambda_a)| <= 0.0202 (+ the rounding of large values)
        const float wd = 0.0202f + 1e-6f * fabsf(pa.x);
        const unsigned lo_key = tgl_key(pa.x - wd), hi_key = tgl_key(pa.x + wd);
        const unsigned* keys = a.skey + a.seg_off[sg];
        const int* idx = a.sidx + a.seg_off[sg];
        const int n = a.seg_n[sg];
        const int f0 = nb0 >= 0 ? a.item_first[nb0] : 0, e0 = nb0 >= 0 ? a.item_first[nb0 + 1] : 0;
        const int f1 = nb1 >= 0 ? a.item_first[nb1] : 0, e1 = nb1 >= 0 ? a.item_first[nb1 + 1] : 0;
        for (int i0 = warp_lower_bound(keys, n, lo_key);; i0 += 32) {
          const int i = i0 + lane;
          const bool in = i < n && keys[i] <= hi_key;
          if (in) {
            const int b = idx[i];  // in the item of sector k+1 or k-1?
            if (b >= f0 && b < e0) consider(b, 0);
            else if (b >= f1 && b < e1) consider(b, 1);
          }
          if (__ballot_sync(0xffffffffu, in) != 0xffffffffu) break;
        }
      }
    } else {
      for (int d = 0; d < 2; ++d) {
        const int nb = d ? nb1 : nb0;
        if (nb >= 0)
          for (long long b = a.item_first[nb] + lane; b < a.item_first[nb + 1]; b += 32) consider(b, d);
      }
    }
    for (int d = 0; d < 2; ++d) {
      const long long b = warp_best(bs[d], bi[d]);
      if (lane == 0) a.best[2 * t + d] = (int)b;
    }
  }
}

__global__ void k_mrg_link(const __grid_constant__ MrgArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_trk; t += stride)
    for (int d = 0; d < 2; ++d) {
      const int b = a.best[2 * t + d];
      a.link[2 * t + d] = (b >= 0 && a.best[2 * b + (1 - d)] == (int)t) ? b : -1;
    }
}

// the group of a track: the smallest index on its path of links (at most 18
// steps each way: one track per sector of a side)
__global__ void k_mrg_group(const __grid_constant__ MrgArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_trk; t += stride) {
    int m = (int)t;
    for (int d = 0; d < 2; ++d) {
      int cur = (int)t;
      for (int step = 0; step < 18; ++step) {
        const int nxt = a.link[2 * cur + d];
        if (nxt < 0) break;
        m = min(m, nxt);
        cur = nxt;
      }
    }
    a.group[t] = m;
  }
}

// Refit of every group in the global frame, in two kernels.  k_mrg_fit (one warp
// per group root) takes the clusters twice: the mean and the innermost cluster,
// then every sum the fits need, in float-float.  The arc length from the
// innermost cluster, s = c (1 + k c^2) with chord c and k = 1 / (24 R^2), is a
// polynomial in c, so the sums over s, s^2 and s z follow from sums of powers of
// c before R is known.  k_mrg_fit_solve (one thread per group) then solves the
// circle (algebraic fit on the centred moments) and the line z = z0 + tan(lambda) s
// in FP64.
__global__ void __launch_bounds__(128) k_mrg_fit(const __grid_constant__ MrgArgs a,
                                                  const __grid_constant__ DevParams par) {
  __shared__ int mem[4][40];
  __shared__ F2 rot[4][40][2];  // cos and sin of each member's sector angle
  __shared__ F2 sec_rot[18][2];  // cos and sin of the 18 sector angles, once per block
  if (threadIdx.x < 18) {
    const double ang = (double)threadIdx.x * MRG_WEDGE;
    sec_rot[threadIdx.x][0] = f2_from(cos(ang));
    sec_rot[threadIdx.x][1] = f2_from(sin(ang));
  }
  __syncthreads();
  constexpr int STAGE = 384;    // clusters of a group kept in shared memory (larger groups re-gather)
  __shared__ F2 sX[4][STAGE], sY[4][STAGE];
  __shared__ float sZ[4][STAGE];
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < a.n_trk; t += nw) {
    double* o = a.fit + 7 * t;
    if (lane < 7) o[lane] = 0.0;
    float* out = a.fit_sums + (long long)MRG_FIT_SUMS * t;
    if (lane == 0) out[0] = 0.0f;  // no fit unless written below
    if (a.group[t] != (int)t) continue;
    if (__double_as_longlong(a.geo[G_N * t + G_OK]) == 0) continue;  // 0.0: no circle
    // members in index order (the root is the smallest)
    int nm = 0;
    if (lane == 0) {
      mem[w][nm++] = (int)t;
      for (int d = 0; d < 2; ++d) {
        int cur = (int)t;
        for (int step = 0; step < 18; ++step) {
          const int nxt = a.link[2 * cur + d];
          if (nxt < 0) break;
          mem[w][nm++] = nxt;
          cur = nxt;
        }
      }
      for (int i = 1; i < nm; ++i)  // insertion sort (at most 37 members)
        for (int j = i; j > 0 && mem[w][j - 1] > mem[w][j]; --j) {
          const int x = mem[w][j];
          mem[w][j] = mem[w][j - 1];
          mem[w][j - 1] = x;
        }
    }
    nm = __shfl_sync(0xffffffffu, nm, 0);
    __syncwarp();
    for (int m = lane; m < nm; m += 32) {
      const int k = (int)(a.item_sector[trk[mem[w][m]].item] % 18u);
      rot[w][m][0] = sec_rot[k][0];
      rot[w][m][1] = sec_rot[k][1];
    }
    __syncwarp();
    long long n_all = 0;
    for (int m = 0; m < nm; ++m) n_all += trk[mem[w][m]].n_clusters;
    const bool staged = n_all <= STAGE;
    // global position of cluster j of member m: x_row cos - y sin, x_row sin + y cos
    auto gather = [&](int m, long long j, F2* X, F2* Y, float* Z) {
      const tpc_track_t& T = trk[mem[w][m]];
      const F2 ca = rot[w][m][0], sa = rot[w][m][1];
      uint32_t c = a.ids[T.first_cluster + j];
      int r = c < (uint32_t)a.N ? a.row[c] : -1;
      if (r < 0 || r >= par.n_rows) {  // reported as an error (the results are then not used); read cluster 0
        atomicOr(a.err, TPC_DERR_BAD_TRACK);
        c = 0;
        r = 0;
      }
      const float lx = par.x[r], ly = a.N > 0 ? a.y[c] : 0.0f;
      *X = f2_add(f2_mul_f(ca, lx), f2_neg(f2_mul_f(sa, ly)));
      *Y = f2_add(f2_mul_f(sa, lx), f2_mul_f(ca, ly));
      *Z = a.N > 0 ? a.z[c] : 0.0f;
    };
    if (staged) {
      long long base = 0;
      for (int m = 0; m < nm; ++m) {
        const long long cnt = trk[mem[w][m]].n_clusters;
        for (long long j = lane; j < cnt; j += 32) gather(m, j, &sX[w][base + j], &sY[w][base + j], &sZ[w][base + j]);
        base += cnt;
      }
      __syncwarp();
    }
    // cluster j of member m (p = its position over the group): from shared memory or gathered again
    auto cluster_at = [&](int m, long long j, long long p, F2* X, F2* Y, float* Z) {
      if (staged) {
        *X = sX[w][p];
        *Y = sY[w][p];
        *Z = sZ[w][p];
      } else {
        gather(m, j, X, Y, Z);
      }
    };
    // pass 1: mean, count and the innermost cluster (smallest radius, first in order on ties)
    F2 sx = {0.f, 0.f}, sy = {0.f, 0.f}, rmin = {INFINITY, 0.f}, xin = {0.f, 0.f}, yin = {0.f, 0.f};
    long long pin = -1, n = 0, pos = 0;
    for (int m = 0; m < nm; ++m) {
      const long long cnt = trk[mem[w][m]].n_clusters;
      for (long long j = lane; j < cnt; j += 32) {
        F2 X, Y;
        float Z;
        cluster_at(m, j, pos + j, &X, &Y, &Z);
        sx = f2_add(sx, X);
        sy = f2_add(sy, Y);
        const F2 rr = f2_add(f2_mul(X, X), f2_mul(Y, Y));  // ordering by the squared radius
        if (f2_less(rr, rmin)) {  // a lane sees its positions in increasing order
          rmin = rr;
          pin = pos + j;
          xin = X;
          yin = Y;
        }
      }
      pos += cnt;
      n += cnt;
    }
    for (int off = 16; off; off >>= 1) {
      const F2 orr = {__shfl_xor_sync(0xffffffffu, rmin.hi, off), __shfl_xor_sync(0xffffffffu, rmin.lo, off)};
      const long long op = __shfl_xor_sync(0xffffffffu, pin, off);
      const F2 ox = {__shfl_xor_sync(0xffffffffu, xin.hi, off), __shfl_xor_sync(0xffffffffu, xin.lo, off)};
      const F2 oy = {__shfl_xor_sync(0xffffffffu, yin.hi, off), __shfl_xor_sync(0xffffffffu, yin.lo, off)};
      if (op >= 0 && (pin < 0 || f2_less(orr, rmin) || (orr.hi == rmin.hi && orr.lo == rmin.lo && op < pin))) {
        rmin = orr;
        pin = op;
        xin = ox;
        yin = oy;
      }
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if (n < 3) continue;
    const F2 fn = {(float)n, 0.0f};  // n < 2^24
    const F2 mx = f2_div(sx, fn), my = f2_div(sy, fn);
    const F2 nmx = f2_neg(mx), nmy = f2_neg(my), nxin = f2_neg(xin), nyin = f2_neg(yin);
    // pass 2: centred moments of the circle fit and powers of the chord from the innermost cluster
    F2 acc[MRG_FIT_NACC];
#pragma unroll
    for (int k = 0; k < MRG_FIT_NACC; ++k) acc[k] = {0.f, 0.f};
    pos = 0;
    for (int m = 0; m < nm; ++m) {
      const long long cnt = trk[mem[w][m]].n_clusters;
      for (long long j = lane; j < cnt; j += 32) {
        F2 X, Y;
        float Z;
        cluster_at(m, j, pos + j, &X, &Y, &Z);
        const F2 u = f2_add(X, nmx), v = f2_add(Y, nmy);
        const F2 uu = f2_mul(u, u), vv = f2_mul(v, v), ww = f2_add(uu, vv);
        acc[0] = f2_add(acc[0], uu);
        acc[1] = f2_add(acc[1], f2_mul(u, v));
        acc[2] = f2_add(acc[2], vv);
        acc[3] = f2_add(acc[3], f2_mul(u, ww));
        acc[4] = f2_add(acc[4], f2_mul(v, ww));
        acc[5] = f2_add(acc[5], ww);
        const F2 cx = f2_add(X, nxin), cy = f2_add(Y, nyin);
        const F2 c2 = f2_add(f2_mul(cx, cx), f2_mul(cy, cy));
        const F2 c = f2_sqrt(c2), c3 = f2_mul(c, c2), c4 = f2_mul(c2, c2);
        acc[6] = f2_add(acc[6], c);
        acc[7] = f2_add(acc[7], c2);
        acc[8] = f2_add(acc[8], c3);
        acc[9] = f2_add(acc[9], c4);
        acc[10] = f2_add(acc[10], f2_mul(c4, c2));
        acc[11] = f2_add(acc[11], {Z, 0.0f});
        acc[12] = f2_add(acc[12], f2_mul_f(c, Z));
        acc[13] = f2_add(acc[13], f2_mul_f(c3, Z));
      }
      pos += cnt;
    }
    // the sums over the warp: accumulators 0..11 through the staging area (free now; lanes 2k and
    // 2k + 1 add the two halves of accumulator k and join them), 12 and 13 by shuffles
    static_assert(12 * 32 <= STAGE && MRG_FIT_NACC == 14, "reduction layout");
    __syncwarp();
    F2* red = sX[w];
#pragma unroll
    for (int k = 0; k < 12; ++k) red[k * 32 + lane] = acc[k];
    __syncwarp();
    F2 part = {0.f, 0.f};
    if ((lane >> 1) < 12) {
      const F2* src = red + (lane >> 1) * 32 + (lane & 1) * 16;
#pragma unroll 4
      for (int j = 0; j < 16; ++j) part = f2_add(part, src[j]);
    }
    part = f2_add(part, {__shfl_xor_sync(0xffffffffu, part.hi, 1), __shfl_xor_sync(0xffffffffu, part.lo, 1)});
    const F2 a12 = warp_sum(acc[12]), a13 = warp_sum(acc[13]);
    // record: n, members, then the mean (x, y) and the sums, each as (hi, lo): lane l writes float 2 + l
    const int ka = (lane - 4) >> 1;  // the accumulator of lane l >= 4
    const int from = lane < 4 ? 0 : 2 * ka;
    const F2 got = {__shfl_sync(0xffffffffu, part.hi, from & 31), __shfl_sync(0xffffffffu, part.lo, from & 31)};
    float v;
    if (lane < 4) {
      v = lane == 0 ? mx.hi : (lane == 1 ? mx.lo : (lane == 2 ? my.hi : my.lo));
    } else {
      const F2 val = ka < 12 ? got : (ka == 12 ? a12 : a13);
      v = ((lane - 4) & 1) ? val.lo : val.hi;
    }
    out[2 + lane] = v;
    if (lane == 0) {
      out[1] = (float)nm;
      out[0] = (float)n;
    }
  }
}

// one thread per group root: the circle from the centred moments (algebraic
// fit u^2 + v^2 + D u + E v + F = 0), then the line z = z0 + tan(lambda) s from
// the sums of powers of the chord (s = c + k c^3), in FP64
__global__ void k_mrg_fit_solve(const __grid_constant__ MrgArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_trk; t += stride) {
    const float* r = a.fit_sums + (long long)MRG_FIT_SUMS * t;
    const double n = r[0];
    if (n < 3.0) continue;
    auto val = [&](int k) { return (double)r[2 + 2 * k] + (double)r[3 + 2 * k]; };
    const double mx = val(0), my = val(1);
    const double Suu = val(2), Suv = val(3), Svv = val(4), Su3 = val(5), Sv3 = val(6), Sw = val(7);
    const double det = Suu * Svv - Suv * Suv;
    if (!(fabs(det) > 0.0)) continue;
    const double inv_det = 1.0 / det, inv_n = 1.0 / n;
    const double D = (-Su3 * Svv + Sv3 * Suv) * inv_det, E = (-Sv3 * Suu + Su3 * Suv) * inv_det, F = -Sw * inv_n;
    const double R = sqrt(0.25 * (D * D + E * E) - F);
    const double k = 1.0 / (24.0 * R * R);
    const double Sc = val(8), Sc2 = val(9), Sc3 = val(10), Sc4 = val(11), Sc6 = val(12);
    const double Sz = val(13), Scz = val(14), Sc3z = val(15);
    const double Ss = Sc + k * Sc3, Sss = Sc2 + k * (2.0 * Sc4 + k * Sc6), Ssz = Scz + k * Sc3z;
    const double den = n * Sss - Ss * Ss;
    const double tgl = den > 0.0 ? (n * Ssz - Ss * Sz) / den : 0.0;
    double* o = a.fit + 7 * t;
    o[0] = mx - 0.5 * D;
    o[1] = my - 0.5 * E;
    o[2] = R;
    o[3] = tgl;
    o[4] = (Sz - tgl * Ss) * inv_n;
    o[5] = n;
    o[6] = r[1];
  }
}

// Looper legs, one warp per track that can turn inside a sector (R < 250 cm):
// the best candidate of opposite q/pT and tan(lambda) sign on the same circle
// among the tracks of the same event and side.
__global__ void k_mrg_legs(const __grid_constant__ MrgArgs a) {
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const float kBf = (float)a.kB;
  for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < a.n_trk; t += nw) {
    const double* A = a.geo + G_N * t;
    unsigned long long bs = 0;
    long long bi = -1;
    if (A[G_OK] != 0.0 && A[G_R] < 250.0) {
      const float4 pa = a.pre[t];
      const float4 ga = a.geo32[2 * t];
      auto consider = [&](long long b) {
        // FP32 prefilter (margins wider than FP32 rounding; R < 250 cm <=> |q/pT| > 2.668 c/GeV at 0.5 T)
        const float4 pb = a.pre[b];
        if (pb.w == pa.w || !((pa.x > 0.f) != (pb.x > 0.f)) || !(fabsf(pa.x + pb.x) <= 0.0201f)) return;
        const float dq = fabsf(pa.y) - fabsf(pb.y), sq = pa.z * pa.z + pb.z * pb.z;
        if (!(dq * dq <= 16.2f * sq + 1e-28f)) return;
        {  // the centre distance in FP32, margins as in mrg_maybe_compatible
          const float4 gb = a.geo32[2 * b];
          const float ex = ga.x - gb.x, ey = ga.y - gb.y;
          const float Rm = fmaxf(ga.z, gb.z);
          const float kv = 3.0f * kBf * sqrtf(ga.w + gb.w);
          const float dl = fmaf(kv * Rm, Rm, 1.0f);
          const float M = fabsf(ga.x) + fabsf(ga.y) + fabsf(gb.x) + fabsf(gb.y);
          if (sqrtf(fmaf(ex, ex, ey * ey)) > dl * (1.0f + 1e-5f) + 1e-5f * (kv * Rm * Rm + M) + 1e-6f) return;
        }
        const double* B = a.geo + G_N * b;
        if (B[G_OK] == 0.0 || !(B[G_R] < 250.0)) return;
        const double qa = fabs(A[G_QPT]), qb = fabs(B[G_QPT]);
        const double vs = fmax(A[G_VQ] + B[G_VQ], 1e-30);
        const double chi2 = (qa - qb) * (qa - qb) / vs;
        const double Rm = fmax(A[G_R], B[G_R]);
        const double dlim = 1.0 + 3.0 * a.kB * sqrt(A[G_VQ] + B[G_VQ]) * Rm * Rm;
        const double dc = hypot(A[G_XC] - B[G_XC], A[G_YC] - B[G_YC]);
        const double st = fabs(A[G_TGL] + B[G_TGL]);
        if (!(chi2 <= 16.0 && dc <= dlim && st <= 0.02)) return;
        keep_best(score_key(chi2 / 16.0 + dc / dlim + st / 0.02), b, &bs, &bi);
      };
      const int sg = a.item_seg[trk[t].item];
      if (sg >= 0 && a.seg_ok[sg]) {
        if (pa.x == pa.x) {  // the window |tan(lambda_b) + tan(lambda_a)| <= 0.0202 (+ rounding)
          const float wd = 0.0202f + 1e-6f * fabsf(pa.x);
          const unsigned lo_key = tgl_key(-pa.x - wd), hi_key = tgl_key(-pa.x + wd);
          const unsigned* keys = a.skey + a.seg_off[sg];
          const int* idx = a.sidx + a.seg_off[sg];
          const int n = a.seg_n[sg];
          for (int i0 = warp_lower_bound(keys, n, lo_key);; i0 += 32) {
            const int i = i0 + lane;
            const bool in = i < n && keys[i] <= hi_key;
            if (in) consider(idx[i]);
            if (__ballot_sync(0xffffffffu, in) != 0xffffffffu) break;
          }
        }
      } else if (sg >= 0) {
        const int* items = a.seg_items + 19 * (long long)sg;
        for (int k = 0; k < 18; ++k) {
          const int it = items[k];
          if (it < 0) continue;
          for (long long b = a.item_first[it] + lane; b < a.item_first[it + 1]; b += 32) consider(b);
        }
      }
    }
    const long long b = warp_best(bs, bi);
    if (lane == 0) a.lbest[t] = (int)b;
  }
}

__global__ void k_mrg_legs_final(const __grid_constant__ MrgArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_trk; t += stride) {
    const int p = a.lbest[t];
    const bool mutual = p >= 0 && a.lbest[p] == (int)t;
    a.partner[t] = mutual ? p : -1;
    if (a.leg) {
      const double zt = fabs(a.geo[G_N * t + G_Z]), zp = mutual ? fabs(a.geo[G_N * (long long)p + G_Z]) : 0.0;
      a.leg[t] = (mutual && (zt > zp || (zt == zp && (int)t > p))) ? 1 : 0;
    }
  }
}

}  // namespace

// ============================================================================ looper legs joined
// The groups of the merger joined through every mutual leg pair into one
// track each (Sec. 4: the legs of a looper, found separately, are merged into
// one track), and each joined track refitted over the clusters of both legs:
// the algebraic circle as for the groups, then z = z0 + tan(lambda) s with
// s = R dtheta, the turning angle from the primary legs' innermost cluster in
// the particle's sense of rotation (clockwise for q/pT > 0 of the primary leg
// with the smallest index), taken in [-0.1, 2 pi - 0.1).  FP64 throughout:
// loopers are few.
namespace {
constexpr int JN_MAXG = 16;    // groups of one joined track
constexpr int JN_MAXM = 96;    // tracks of one joined track

__device__ __forceinline__ bool jn_pair(const JoinArgs& a, int t, int* p) {
  const int q = a.partner[t];
  if (q < 0 || q >= a.n_trk) return false;
  const int back = a.partner[q];
  *p = q;
  return back == t;
}

// the primary legs of mutual pairs (order of arrival: every use below is
// order-independent); input values out of range are flagged and skipped
__global__ void k_join_pairs(const __grid_constant__ JoinArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_trk; t += stride) {
    a.glab[t] = (int)t;
    const int g = a.group[t], q = a.partner[t];
    if (g < 0 || g >= a.n_trk || q < -1 || q >= a.n_trk || a.group[g] != g) {
      atomicOr(a.err, TPC_DERR_BAD_TRACK);
      continue;
    }
    int p;
    if (jn_pair(a, (int)t, &p) && a.leg[t] == 0) a.plist[atomicAdd(a.n_pairs, 1)] = (int)t;
  }
}

// one round of min-label propagation over the pairs (between group roots)
__global__ void k_join_union(const __grid_constant__ JoinArgs a, int final_check) {
  const int np = *a.n_pairs;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += stride) {
    const int t = a.plist[i];
    const int ga = a.group[t], gb = a.group[a.partner[t]];
    if (gb < 0 || gb >= a.n_trk) continue;
    const int la = a.glab[ga], lb = a.glab[gb];
    if (final_check) {
      if (la != lb) atomicOr(a.err, TPC_DERR_BAD_TRACK);  // a chain of joins longer than the rounds
      continue;
    }
    const int m = min(la, lb);
    atomicMin(&a.glab[ga], m);
    atomicMin(&a.glab[gb], m);
  }
}

__global__ void k_join_label(const __grid_constant__ JoinArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n_trk; t += stride) {
    const int g = a.group[t];
    a.joined[t] = (g >= 0 && g < a.n_trk) ? a.glab[g] : (int)t;
    double* o = a.jfit + 7 * t;
#pragma unroll
    for (int k = 0; k < 7; ++k) o[k] = 0.0;
  }
}

__device__ __forceinline__ double jn_wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// one warp per pair; the pair with the smallest primary index of its joined
// track refits it
__global__ void __launch_bounds__(128) k_join_fit(const __grid_constant__ JoinArgs a,
                                                   const __grid_constant__ DevParams par) {
  __shared__ int s_grp[4][JN_MAXG], s_prim[4][JN_MAXG], s_mem[4][JN_MAXM], s_off[4][JN_MAXM + 1];
  const tpc_track_t* trk = static_cast<const tpc_track_t*>(a.trk);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int np = *a.n_pairs;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < np; i += nw) {
    const int t = a.plist[i];
    const int root = a.glab[a.group[t]];
    // the representative: no pair of the same joined track with a smaller primary
    bool rep = true;
    for (int j = lane; j < np; j += 32) {
      const int u = a.plist[j];
      if (u < t && a.glab[a.group[u]] == root) rep = false;
    }
    if (!__all_sync(0xffffffffu, rep)) continue;
    // groups of the joined track (primary groups flagged) and their members
    int ng = 0, nm = 0;
    bool ok = true;
    if (lane == 0) {
      auto add_group = [&](int g, int prim) {
        if (g < 0 || g >= a.n_trk) {
          ok = false;
          return;
        }
        for (int k = 0; k < ng; ++k)
          if (s_grp[w][k] == g) {
            s_prim[w][k] |= prim;
            return;
          }
        if (ng == JN_MAXG) {
          ok = false;
          return;
        }
        s_grp[w][ng] = g;
        s_prim[w][ng] = prim;
        ++ng;
      };
      for (int j = 0; j < np; ++j) {
        const int u = a.plist[j];
        if (a.glab[a.group[u]] != root) continue;
        add_group(a.group[u], 1);
        add_group(a.group[a.partner[u]], 0);
      }
      for (int k = 0; k < ng && ok; ++k) {  // members of group k: the root and its link paths
        const int g = s_grp[w][k];
        if (nm == JN_MAXM) {
          ok = false;
          break;
        }
        s_mem[w][nm++] = g;
        for (int d = 0; d < 2 && ok; ++d) {
          int cur = g;
          for (int step = 0; step < 18; ++step) {
            const int nxt = a.link[2 * cur + d];
            if (nxt < 0 || nxt >= a.n_trk) break;
            if (nm == JN_MAXM) {
              ok = false;
              break;
            }
            s_mem[w][nm++] = nxt;
            cur = nxt;
          }
        }
      }
      for (int x = 1; x < nm; ++x)  // index order
        for (int y = x; y > 0 && s_mem[w][y - 1] > s_mem[w][y]; --y) {
          const int v = s_mem[w][y];
          s_mem[w][y] = s_mem[w][y - 1];
          s_mem[w][y - 1] = v;
        }
      s_off[w][0] = 0;
      for (int m = 0; m < nm; ++m) s_off[w][m + 1] = s_off[w][m] + (int)trk[s_mem[w][m]].n_clusters;
      if (!ok) atomicOr(a.err, TPC_DERR_BAD_TRACK);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    nm = __shfl_sync(0xffffffffu, nm, 0);
    ng = __shfl_sync(0xffffffffu, ng, 0);
    __syncwarp();
    if (!ok) continue;
    const int m_all = s_off[w][nm];
    // cluster k of the concatenation (members in index order, clusters in track order)
    auto cluster = [&](int k, double* X, double* Y, double* Z, bool* prim) {
      int m = 0;
      while (s_off[w][m + 1] <= k) ++m;
      const tpc_track_t& T = trk[s_mem[w][m]];
      const long long pos = (long long)T.first_cluster + (k - s_off[w][m]);
      const uint32_t c = pos < a.n_ids ? a.ids[pos] : 0xffffffffu;
      const int r = c < (uint32_t)a.N ? a.row[c] : -1;
      const bool good = T.item < (uint32_t)a.I && r >= 0 && r < par.n_rows;
      const double ang = good ? (double)(a.item_sector[T.item] % 18u) * MRG_WEDGE : 0.0;
      const double lx = good ? (double)par.x[r] : 0.0, ly = good ? (double)a.y[c] : 0.0;
      *X = lx * cos(ang) - ly * sin(ang);
      *Y = lx * sin(ang) + ly * cos(ang);
      *Z = good ? (double)a.z[c] : 0.0;
      if (!good) atomicOr(a.err, TPC_DERR_BAD_TRACK);
      int g = s_mem[w][m];
      g = a.group[g];
      bool p = false;
      for (int q = 0; q < ng; ++q) p |= s_grp[w][q] == g && s_prim[w][q];
      *prim = p;
    };
    if (m_all < 3) continue;
    double sx = 0, sy = 0;
    for (int k = lane; k < m_all; k += 32) {
      double X, Y, Z;
      bool p;
      cluster(k, &X, &Y, &Z, &p);
      sx += X;
      sy += Y;
    }
    const double mx = jn_wsum(sx) / m_all, my = jn_wsum(sy) / m_all;
    double suu = 0, suv = 0, svv = 0, su3 = 0, sv3 = 0, sw = 0;
    double rmin = 1e300;
    int kref = m_all;
    for (int k = lane; k < m_all; k += 32) {
      double X, Y, Z;
      bool p;
      cluster(k, &X, &Y, &Z, &p);
      const double u = X - mx, v = Y - my, q = u * u + v * v;
      suu += u * u;
      suv += u * v;
      svv += v * v;
      su3 += u * q;
      sv3 += v * q;
      sw += q;
      const double rr = hypot(X, Y);
      if (p && rr < rmin) {  // lanes visit k in increasing order: the first of equal radii stays
        rmin = rr;
        kref = k;
      }
    }
    suu = jn_wsum(suu);
    suv = jn_wsum(suv);
    svv = jn_wsum(svv);
    su3 = jn_wsum(su3);
    sv3 = jn_wsum(sv3);
    sw = jn_wsum(sw);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {  // innermost primary cluster: smallest radius, then smallest k
      const double r2 = __shfl_xor_sync(0xffffffffu, rmin, o);
      const int k2 = __shfl_xor_sync(0xffffffffu, kref, o);
      if (r2 < rmin || (r2 == rmin && k2 < kref)) {
        rmin = r2;
        kref = k2;
      }
    }
    const double det = suu * svv - suv * suv;
    if (!(fabs(det) > 0) || kref >= m_all) continue;
    const double D = (-su3 * svv + sv3 * suv) / det, E = (-sv3 * suu + su3 * suv) / det, F = -sw / m_all;
    const double xc = mx - 0.5 * D, yc = my - 0.5 * E;
    const double R = sqrt(0.25 * (D * D + E * E) - F);
    double Xr, Yr, Zr;
    bool pr;
    cluster(kref, &Xr, &Yr, &Zr, &pr);
    const double th0 = atan2(Yr - yc, Xr - xc);
    const bool cw = trk[t].qpt > 0.0f;  // the smallest primary leg of the joined track
    const double two_pi = 2.0 * 3.14159265358979323846;
    double ss = 0, sz = 0, sss = 0, ssz = 0;
    for (int k = lane; k < m_all; k += 32) {
      double X, Y, Z;
      bool p;
      cluster(k, &X, &Y, &Z, &p);
      const double th = atan2(Y - yc, X - xc);
      double d = cw ? th0 - th : th - th0;
      d -= two_pi * floor((d + 0.1) / two_pi);
      const double sv = R * d;
      ss += sv;
      sz += Z;
      sss += sv * sv;
      ssz += sv * Z;
    }
    ss = jn_wsum(ss);
    sz = jn_wsum(sz);
    sss = jn_wsum(sss);
    ssz = jn_wsum(ssz);
    if (lane == 0) {
      const double den = m_all * sss - ss * ss;
      const double tgl = den > 0 ? (m_all * ssz - ss * sz) / den : 0.0;
      double* o = a.jfit + 7 * (long long)root;
      o[0] = xc;
      o[1] = yc;
      o[2] = R;
      o[3] = tgl;
      o[4] = (sz - tgl * ss) / m_all;
      o[5] = (double)m_all;
      o[6] = (double)nm;
    }
  }
}
}  // namespace

cudaError_t launch_join(const JoinArgs& a, const DevParams& par, int num_sms, cudaStream_t s) {
  const int g = num_sms * 8;
  cudaMemsetAsync(a.n_pairs, 0, sizeof(int), s);
  if (a.n_trk > 0) {
    k_join_pairs<<<g, 256, 0, s>>>(a);
    for (int r = 0; r < 4; ++r) k_join_union<<<g, 256, 0, s>>>(a, 0);
    k_join_union<<<g, 256, 0, s>>>(a, 1);
    k_join_label<<<g, 256, 0, s>>>(a);
    k_join_fit<<<num_sms * 4, 128, 0, s>>>(a, par);
  }
  return cudaGetLastError();
}

cudaError_t launch_merge(const MrgArgs& a, const DevParams& par, int num_sms, cudaStream_t s) {
  const int g = num_sms * 8;
  k_mrg_item_first<<<(a.I + 256) / 256, 256, 0, s>>>(a);
  if (a.n_trk > 0) {
    k_mrg_geom<<<g, 256, 0, s>>>(a);
    if (a.S > 0) {
      // the sort's shared memory above the default 48 KB (an attribute of the current device: set per call)
      const cudaError_t e = cudaFuncSetAttribute(k_mrg_seg_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 8 * MRG_SORT_CAP);
      if (e != cudaSuccess) return e;
      k_mrg_seg_count<<<(a.S + 255) / 256, 256, 0, s>>>(a);
      k_mrg_seg_scan<<<1, 1024, 0, s>>>(a);
      k_mrg_seg_sort<<<a.S, 1024, 8 * MRG_SORT_CAP, s>>>(a);
    }
    k_mrg_best<<<g, 256, 0, s>>>(a);
    k_mrg_link<<<g, 256, 0, s>>>(a);
    k_mrg_group<<<g, 256, 0, s>>>(a);
    k_mrg_fit<<<num_sms * 16, 128, 0, s>>>(a, par);
    k_mrg_fit_solve<<<g, 256, 0, s>>>(a);
    if (a.legs) {
      k_mrg_legs<<<g, 256, 0, s>>>(a);
      k_mrg_legs_final<<<g, 256, 0, s>>>(a);
    }
  }
  return cudaGetLastError();
}
