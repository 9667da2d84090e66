// Data-reduction kernels (Sec. 4): the cluster codec (step 2).
//
// The codec is a pure stream: 28 bytes of float/int32 properties in, 13 bytes
// of codes out per cluster, no reuse.  It is bound by HBM bandwidth, so the
// design is about moving bytes: each thread converts four consecutive clusters
// with 16-byte loads of every input array and one vector store per output array
// (8-, 16- or 4-byte wide), in a grid sized to the SM count; unaligned arrays
// take a scalar path with the same arithmetic.
#include <cuda_runtime.h>

#include <cstdint>

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
