// CPU oracle of the TPC cluster compression chain after the integer
// conversion: entropy reduction (Sec. 4, step 3) and entropy coding with ANS
// (Sec. 4, step 4), encoder and decoder.
//
// Test infrastructure only: tests, smoke() and the CPU baseline of the
// benchmark use it; the library never does.  It shares no code with the CUDA
// path.
//
// What the paper fixes: clusters not assigned to tracks are ordered in y and z
// and stored as differences to the previous cluster; clusters assigned to
// tracks are stored as residuals to the extrapolated track (track-model
// compression); an ANS entropy coder compresses the result.
//
// Readings (the paper names the steps, not their formats):
//  - integer codes of the clusters: the cluster codec (codec_oracle.cpp);
//  - "ordered in y and z": the tracker's canonical order inside a pad row,
//    i.e. the cells of its y-z grid, y-major, then the cluster index; per
//    (item, row) the number of unattached clusters, then per cluster zigzag
//    differences of the y and z codes to the previous unattached cluster of
//    the row (the first one to 0);
//  - track model: per track its float32 state (x_ref, y, z, sin phi,
//    tan lambda, q/pT) and item stored raw, its cluster count, then per
//    cluster (innermost first) the zigzag row increment (the first to row 0)
//    and the zigzag residuals of the y and z codes to the track's prediction
//    at that row; the prediction is a fixed sequence of correctly rounded
//    float32 operations (no fused multiply-add) so that encoder and decoder
//    agree bit for bit: the helix of the tracker, with the arc length's
//    asin(a)/a from two half-angle reductions and a series to a^8;
//  - charges and sizes: their codes, in the order the positions are stored;
//  - removal (Sec. 4, step 5: clusters not used for physics are discarded):
//    with a keep mask, a cluster with keep = 0 is stored neither as an
//    unattached cluster nor in its track (a track keeps its place with the
//    clusters left; its row increments refer to its previous kept cluster);
//  - every symbol stream is split into byte planes (as many as its largest
//    value needs, at least one) and each plane is coded by rANS: 32-bit
//    states, 16-bit renormalisation, frequencies scaled to 2^12, chunks of
//    8192 symbols each coded by 32 interleaved states (symbol i of a chunk by
//    state i mod 32); a chunk is its 32 final states (two 16-bit words each,
//    low first) followed by the renormalisation words in decoding order;
//  - frequency scaling: f = max(1, floor(count * 4096 / total)) for every
//    present symbol; while the sum exceeds 4096 the largest f (smallest
//    symbol on ties) loses one; a shortfall goes to the largest f;
//  - blob: little-endian; header (magic "TPCZ", version 1, n_items, n_rows,
//    n_tracks, kB bits, x of the first and last pad row as float64 bits,
//    unattached count, attached count), then for each of
//    the 11 streams: value count (u64), plane count (u32), and per plane the
//    256 frequencies (u16), the chunk count (u32), each chunk's length in
//    words (u32) and the words; then the raw track table (7 x u32 per track).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

extern "C" int64_t orc_encode_clusters(int64_t n, int n_rows, const float* y, const float* z, const int32_t* row,
                                       const float* q_tot, const float* q_max, const float* sigma_y,
                                       const float* sigma_z, int16_t* cy, int32_t* cz, uint8_t* crow, uint16_t* cqt,
                                       uint16_t* cqm, uint8_t* csy, uint8_t* csz);

namespace {

enum { S_UNATT_N, S_DY, S_DZ, S_DROW, S_RY, S_RZ, S_QT, S_QM, S_SY, S_SZ, S_TRK_N, N_STREAMS };
const int CHUNK = 8192, LANES = 32, SCALE_BITS = 12, M = 1 << SCALE_BITS;
const uint32_t RANS_L = 1u << 16;

uint64_t zigzag(int64_t v) { return v >= 0 ? (uint64_t)v << 1 : (((uint64_t)(-(v + 1))) << 1) | 1; }
int64_t unzigzag(uint64_t u) { return (u & 1) ? -(int64_t)(u >> 1) - 1 : (int64_t)(u >> 1); }

// Track prediction of the (y, z) codes at pad-row radius X (step 2^-6 cm).
void predict(const float* st, float kB, float X, int64_t* py, int64_t* pz) {
  const float x_ref = st[0], y0 = st[1], z0 = st[2], snp = st[3], tgl = st[4], qpt = st[5];
  const float dx = X - x_ref;
  const float kappa = kB * qpt;
  float s2 = snp - kappa * dx;
  s2 = std::fmin(std::fmax(s2, -0.9999f), 0.9999f);
  const float s1 = std::fmin(std::fmax(snp, -0.9999f), 0.9999f);
  const float c1 = std::sqrt(1.0f - s1 * s1), c2 = std::sqrt(1.0f - s2 * s2);
  const float T = (s1 + s2) / (c1 + c2);
  const float y = y0 + dx * T;
  const float chord = dx * std::sqrt(1.0f + T * T);
  const float a = std::fmin(std::fabs(0.5f * kappa * chord), 1.0f);  // sin of half the turning angle
  float g = 1.0f;  // asin(a) / a: two half-angle steps asin(a) = 2 asin(a / sqrt(2 (1 + sqrt(1 - a^2)))),
  if (a > 1e-6f) {  // then the series to a^8 on the reduced argument (below 0.383)
    const float a1 = a / std::sqrt(2.0f * (1.0f + std::sqrt(1.0f - a * a)));
    const float a2 = a1 / std::sqrt(2.0f * (1.0f + std::sqrt(1.0f - a1 * a1)));
    const float t = a2 * a2;
    const float ser = 1.0f + t * (1.0f / 6.0f + t * (3.0f / 40.0f + t * (5.0f / 112.0f + t * (35.0f / 1152.0f))));
    g = 4.0f * a2 * ser / a;
  }
  const float z = z0 + tgl * (chord * g);
  // code of a prediction; 0 where it is not finite or beyond the codes' reach
  *py = std::fabs(y) < 1.0e17f ? (int64_t)std::nearbyint((double)y * 64.0) : 0;
  *pz = std::fabs(z) < 1.0e17f ? (int64_t)std::nearbyint((double)z * 64.0) : 0;
}

void scale_freqs(const uint64_t* cnt, uint16_t* f) {
  uint64_t total = 0;
  for (int s = 0; s < 256; ++s) total += cnt[s];
  int64_t sum = 0;
  for (int s = 0; s < 256; ++s) {
    uint64_t v = cnt[s] ? (cnt[s] * (uint64_t)M) / total : 0;
    if (cnt[s] && v == 0) v = 1;
    f[s] = (uint16_t)v;
    sum += (int64_t)v;
  }
  if (!total) return;
  auto largest = [&]() {
    int b = 0;
    for (int s = 1; s < 256; ++s)
      if (f[s] > f[b]) b = s;
    return b;
  };
  while (sum > M) {
    f[largest()] -= 1;
    --sum;
  }
  if (sum < M) f[largest()] += (uint16_t)(M - sum);
}

struct Writer {
  std::vector<uint8_t> b;
  void u16(uint32_t v) {
    b.push_back(v & 0xff);
    b.push_back((v >> 8) & 0xff);
  }
  void u32(uint32_t v) {
    u16(v & 0xffff);
    u16(v >> 16);
  }
  void u64(uint64_t v) {
    u32((uint32_t)v);
    u32((uint32_t)(v >> 32));
  }
};

// One chunk of n <= 8192 symbols: returns its words (final states, then the
// renormalisation words in the order the decoder reads them).
std::vector<uint16_t> rans_chunk(const uint8_t* sym, int n, const uint16_t* f, const uint16_t* c) {
  const int K = (n + LANES - 1) / LANES;
  std::vector<uint16_t> buf(2 * LANES + n);
  size_t ptr = buf.size();  // filled backwards
  uint32_t x[LANES];
  for (int j = 0; j < LANES; ++j) x[j] = RANS_L;
  for (int k = K - 1; k >= 0; --k) {
    bool emit[LANES] = {};
    int n_emit = 0;
    for (int j = 0; j < LANES; ++j) {
      const int i = k * LANES + j;
      if (i >= n) continue;
      emit[j] = (uint64_t)x[j] >= ((uint64_t)f[sym[i]] << 20);  // x_max = ((L >> 12) << 16) * f
      n_emit += emit[j];
    }
    ptr -= n_emit;
    size_t w = ptr;
    for (int j = 0; j < LANES; ++j)
      if (emit[j]) {
        buf[w++] = (uint16_t)(x[j] & 0xffff);
        x[j] >>= 16;
      }
    for (int j = 0; j < LANES; ++j) {
      const int i = k * LANES + j;
      if (i >= n) continue;
      const uint32_t fs = f[sym[i]];
      x[j] = ((x[j] / fs) << SCALE_BITS) + (x[j] % fs) + c[sym[i]];
    }
  }
  ptr -= 2 * LANES;
  for (int j = 0; j < LANES; ++j) {
    buf[ptr + 2 * j] = (uint16_t)(x[j] & 0xffff);
    buf[ptr + 2 * j + 1] = (uint16_t)(x[j] >> 16);
  }
  return std::vector<uint16_t>(buf.begin() + ptr, buf.end());
}

void put_stream(Writer& W, const std::vector<uint64_t>& v) {
  uint64_t mx = 0;
  for (uint64_t a : v) mx = a > mx ? a : mx;
  int planes = 1;
  while (planes < 8 && (mx >> (8 * planes))) ++planes;
  W.u64(v.size());
  W.u32((uint32_t)planes);
  std::vector<uint8_t> sym(v.size());
  for (int p = 0; p < planes; ++p) {
    uint64_t cnt[256] = {};
    for (size_t i = 0; i < v.size(); ++i) {
      sym[i] = (uint8_t)(v[i] >> (8 * p));
      ++cnt[sym[i]];
    }
    uint16_t f[256], c[256];
    scale_freqs(cnt, f);
    uint32_t acc = 0;
    for (int s = 0; s < 256; ++s) {
      c[s] = (uint16_t)acc;
      acc += f[s];
    }
    for (int s = 0; s < 256; ++s) W.u16(f[s]);
    const size_t n_chunks = (v.size() + CHUNK - 1) / CHUNK;
    W.u32((uint32_t)n_chunks);
    std::vector<std::vector<uint16_t>> words(n_chunks);
    for (size_t ch = 0; ch < n_chunks; ++ch) {
      const size_t a = ch * CHUNK, e = std::min(v.size(), a + CHUNK);
      words[ch] = rans_chunk(sym.data() + a, (int)(e - a), f, c);
    }
    for (auto& w : words) W.u32((uint32_t)w.size());
    for (auto& w : words)
      for (uint16_t x : w) W.u16(x);
  }
}

struct Reader {
  const uint8_t* p;
  size_t n, at = 0;
  bool ok = true;
  uint32_t u16() {
    if (at + 2 > n) {
      ok = false;
      return 0;
    }
    const uint32_t v = p[at] | (p[at + 1] << 8);
    at += 2;
    return v;
  }
  uint32_t u32() {
    const uint32_t lo = u16();
    return lo | (u16() << 16);
  }
  uint64_t u64() {
    const uint64_t lo = u32();
    return lo | ((uint64_t)u32() << 32);
  }
};

bool get_stream(Reader& R, std::vector<uint64_t>& v) {
  const uint64_t n = R.u64();
  const uint32_t planes = R.u32();
  if (!R.ok || planes < 1 || planes > 8 || n > (1ull << 36)) return false;
  v.assign(n, 0);
  for (uint32_t p = 0; p < planes; ++p) {
    uint16_t f[256], c[256];
    uint32_t acc = 0;
    for (int s = 0; s < 256; ++s) {
      f[s] = (uint16_t)R.u16();
      c[s] = (uint16_t)acc;
      acc += f[s];
    }
    if (n && acc != (uint32_t)M) return false;
    std::vector<uint8_t> slot(M);
    for (int s = 0; s < 256; ++s)
      for (uint32_t k = 0; k < f[s]; ++k) slot[c[s] + k] = (uint8_t)s;
    const uint32_t n_chunks = R.u32();
    if (!R.ok || n_chunks != (n + CHUNK - 1) / CHUNK) return false;
    std::vector<uint32_t> len(n_chunks);
    for (auto& l : len) l = R.u32();
    for (uint32_t ch = 0; ch < n_chunks; ++ch) {
      const size_t a = (size_t)ch * CHUNK, m = std::min<size_t>(n - a, CHUNK);
      const size_t start = R.at;
      uint32_t x[LANES];
      for (int j = 0; j < LANES; ++j) x[j] = R.u32();
      const int K = (int)((m + LANES - 1) / LANES);
      for (int k = 0; k < K; ++k) {
        for (int j = 0; j < LANES; ++j) {
          const size_t i = (size_t)k * LANES + j;
          if (i >= m) continue;
          const uint32_t sl = x[j] & (M - 1);
          const uint8_t s = slot[sl];
          x[j] = f[s] * (x[j] >> SCALE_BITS) + sl - c[s];
          v[a + i] |= (uint64_t)s << (8 * p);
        }
        for (int j = 0; j < LANES; ++j) {
          const size_t i = (size_t)k * LANES + j;
          if (i < m && x[j] < RANS_L) x[j] = (x[j] << 16) | R.u16();
        }
      }
      for (int j = 0; j < LANES; ++j)
        if (x[j] != RANS_L) return false;  // every state returns to its initial value
      if (!R.ok || R.at - start != 2 * (size_t)len[ch]) return false;
    }
  }
  return R.ok;
}

}  // namespace

extern "C" {

// Encodes the clusters of a tracked batch.  order/seg_off: the canonical
// order of the binned clusters (original indices) and its (item, row)
// segments (n_items * n_rows + 1 offsets).  Tracks: trk_f [n][6] float32,
// trk_i [n][3] (item, first, count) into ids.  Writes at most cap bytes to out
// and returns the blob's size (negative on bad input).
int64_t orc_compress(int n_rows, double x_min, double x_max, float kB, int64_t n, const float* y, const float* z,
                     const int32_t* row, const float* q_tot, const float* q_max, const float* sigma_y,
                     const float* sigma_z, int64_t n_items, const int32_t* order, const int64_t* seg_off,
                     int64_t n_trk, const float* trk_f, const int64_t* trk_i, const uint32_t* ids,
                     const uint8_t* keep, uint8_t* out, int64_t cap) {
  std::vector<int16_t> cy(n);
  std::vector<int32_t> cz(n);
  std::vector<uint8_t> crow(n), csy(n), csz(n);
  std::vector<uint16_t> cqt(n), cqm(n);
  orc_encode_clusters(n, n_rows, y, z, row, q_tot, q_max, sigma_y, sigma_z, cy.data(), cz.data(), crow.data(),
                      cqt.data(), cqm.data(), csy.data(), csz.data());
  std::vector<float> xr(n_rows);
  for (int r = 0; r < n_rows; ++r)
    xr[r] = (float)(std::nearbyint((x_min + r * ((x_max - x_min) / (n_rows - 1))) * 1024.0) / 1024.0);
  std::vector<uint8_t> attached(n, 0);
  for (int64_t t = 0; t < n_trk; ++t)
    for (int64_t j = 0; j < trk_i[3 * t + 2]; ++j) {
      const uint32_t c = ids[trk_i[3 * t + 1] + j];
      if (c >= (uint64_t)n) return -1;
      attached[c] = 1;
    }
  std::vector<std::vector<uint64_t>> S(N_STREAMS);
  auto props = [&](uint32_t c) {
    S[S_QT].push_back(cqt[c]);
    S[S_QM].push_back(cqm[c]);
    S[S_SY].push_back(csy[c]);
    S[S_SZ].push_back(csz[c]);
  };
  uint64_t n_unatt = 0, n_att = 0;
  for (int64_t g = 0; g < n_items * n_rows; ++g) {
    int64_t prev_y = 0, prev_z = 0, cnt = 0;
    for (int64_t p = seg_off[g]; p < seg_off[g + 1]; ++p) {
      const uint32_t c = (uint32_t)order[p];
      if (attached[c] || (keep && !keep[c])) continue;
      S[S_DY].push_back(zigzag((int64_t)cy[c] - prev_y));
      S[S_DZ].push_back(zigzag((int64_t)cz[c] - prev_z));
      prev_y = cy[c];
      prev_z = cz[c];
      props(c);
      ++cnt;
    }
    S[S_UNATT_N].push_back((uint64_t)cnt);
    n_unatt += cnt;
  }
  for (int64_t t = 0; t < n_trk; ++t) {
    const int64_t first = trk_i[3 * t + 1], cnt = trk_i[3 * t + 2];
    int64_t kept = 0;
    for (int64_t j = 0; j < cnt; ++j) kept += (!keep || keep[ids[first + j]]) ? 1 : 0;
    S[S_TRK_N].push_back((uint64_t)kept);
    int64_t prev_row = 0;
    for (int64_t j = 0; j < cnt; ++j) {
      const uint32_t c = ids[first + j];
      const int r = row[c];
      if (r < 0 || r >= n_rows) return -1;
      if (keep && !keep[c]) continue;
      S[S_DROW].push_back(zigzag(r - prev_row));
      prev_row = r;
      int64_t py, pz;
      predict(trk_f + 6 * t, kB, xr[r], &py, &pz);
      S[S_RY].push_back(zigzag((int64_t)cy[c] - py));
      S[S_RZ].push_back(zigzag((int64_t)cz[c] - pz));
      props(c);
      ++n_att;
    }
  }
  Writer W;
  W.u32(0x5A435054u);
  W.u32(1);
  W.u32((uint32_t)n_items);
  W.u32((uint32_t)n_rows);
  W.u32((uint32_t)n_trk);
  uint32_t kb;
  std::memcpy(&kb, &kB, 4);
  W.u32(kb);
  uint64_t xb;
  std::memcpy(&xb, &x_min, 8);
  W.u64(xb);
  std::memcpy(&xb, &x_max, 8);
  W.u64(xb);
  W.u64(n_unatt);
  W.u64(n_att);
  for (int s = 0; s < N_STREAMS; ++s) put_stream(W, S[s]);
  for (int64_t t = 0; t < n_trk; ++t) {
    for (int k = 0; k < 6; ++k) {
      uint32_t b;
      std::memcpy(&b, trk_f + 6 * t + k, 4);
      W.u32(b);
    }
    W.u32((uint32_t)trk_i[3 * t]);
  }
  if ((int64_t)W.b.size() <= cap && out) std::memcpy(out, W.b.data(), W.b.size());
  return (int64_t)W.b.size();
}

// Decodes a blob.  Per stored cluster (unattached ones in stored order, then
// attached ones track by track): item, row, y code, z code, q_tot, q_max,
// sigma_y, sigma_z codes and the track (-1 = unattached), written to the
// arrays when their capacity `cap` suffices.  Returns the number of stored
// clusters, or -1 if the blob is malformed.
int64_t orc_decompress(const uint8_t* blob, int64_t size, int64_t cap, int32_t* item, int32_t* row, int32_t* y,
                       int32_t* z, int32_t* qt, int32_t* qm, int32_t* sy, int32_t* sz, int32_t* track) {
  Reader R{blob, (size_t)size};
  if (R.u32() != 0x5A435054u || R.u32() != 1) return -1;
  const uint32_t n_items = R.u32(), n_rows = R.u32(), n_trk = R.u32(), kb = R.u32();
  const uint64_t xb0 = R.u64(), xb1 = R.u64();
  const uint64_t n_unatt = R.u64(), n_att = R.u64();
  if (!R.ok || n_rows < 2 || n_rows > 256) return -1;
  double x_min, x_max;
  std::memcpy(&x_min, &xb0, 8);
  std::memcpy(&x_max, &xb1, 8);
  float kB;
  std::memcpy(&kB, &kb, 4);
  std::vector<std::vector<uint64_t>> S(N_STREAMS);
  for (int s = 0; s < N_STREAMS; ++s)
    if (!get_stream(R, S[s])) return -1;
  std::vector<float> tf(6 * (size_t)n_trk);
  std::vector<uint32_t> titem(n_trk);
  for (uint32_t t = 0; t < n_trk; ++t) {
    for (int k = 0; k < 6; ++k) {
      const uint32_t b = R.u32();
      std::memcpy(&tf[6 * t + k], &b, 4);
    }
    titem[t] = R.u32();
  }
  if (!R.ok || R.at != (size_t)size) return -1;
  if (S[S_UNATT_N].size() != (size_t)n_items * n_rows || S[S_DY].size() != n_unatt || S[S_RY].size() != n_att ||
      S[S_TRK_N].size() != n_trk || S[S_QT].size() != n_unatt + n_att)
    return -1;
  const int64_t total = (int64_t)(n_unatt + n_att);
  if (total > cap) return total;
  int64_t k = 0, u = 0;
  for (uint64_t g = 0; g < (uint64_t)n_items * n_rows; ++g) {
    int64_t py = 0, pz = 0;
    for (uint64_t j = 0; j < S[S_UNATT_N][g]; ++j, ++u, ++k) {
      py += unzigzag(S[S_DY][u]);
      pz += unzigzag(S[S_DZ][u]);
      item[k] = (int32_t)(g / n_rows);
      row[k] = (int32_t)(g % n_rows);
      y[k] = (int32_t)py;
      z[k] = (int32_t)pz;
      track[k] = -1;
    }
  }
  if ((uint64_t)u != n_unatt) return -1;
  std::vector<float> xr(n_rows);  // pad-row radii, as the encoder placed them
  for (uint32_t r = 0; r < n_rows; ++r)
    xr[r] = (float)(std::nearbyint((x_min + r * ((x_max - x_min) / (n_rows - 1))) * 1024.0) / 1024.0);
  int64_t a = 0;
  for (uint32_t t = 0; t < n_trk; ++t) {
    int64_t prev_row = 0;
    for (uint64_t j = 0; j < S[S_TRK_N][t]; ++j, ++a, ++k) {
      if ((uint64_t)a >= n_att) return -1;
      prev_row += unzigzag(S[S_DROW][a]);
      if (prev_row < 0 || prev_row >= (int64_t)n_rows) return -1;
      int64_t py, pz;
      predict(&tf[6 * t], kB, xr[prev_row], &py, &pz);
      item[k] = (int32_t)titem[t];
      row[k] = (int32_t)prev_row;
      y[k] = (int32_t)(py + unzigzag(S[S_RY][a]));
      z[k] = (int32_t)(pz + unzigzag(S[S_RZ][a]));
      track[k] = (int32_t)t;
    }
  }
  for (int64_t i = 0; i < total; ++i) {
    qt[i] = (int32_t)S[S_QT][i];
    qm[i] = (int32_t)S[S_QM][i];
    sy[i] = (int32_t)S[S_SY][i];
    sz[i] = (int32_t)S[S_SZ][i];
  }
  return total;
}

// One symbol stream coded as in a blob (value count, planes, tables, chunks).
int64_t orc_code_stream(const uint64_t* v, int64_t n, uint8_t* out, int64_t cap) {
  Writer W;
  put_stream(W, std::vector<uint64_t>(v, v + n));
  if ((int64_t)W.b.size() <= cap && out) std::memcpy(out, W.b.data(), W.b.size());
  return (int64_t)W.b.size();
}

// Decodes one coded stream; returns its value count (-1 if malformed).
int64_t orc_decode_stream(const uint8_t* in, int64_t size, uint64_t* v, int64_t cap) {
  Reader R{in, (size_t)size};
  std::vector<uint64_t> d;
  if (!get_stream(R, d) || R.at != (size_t)size) return -1;
  if ((int64_t)d.size() <= cap && v) std::memcpy(v, d.data(), 8 * d.size());
  return (int64_t)d.size();
}

// The track model's (y, z) codes at pad-row radius X.
void orc_predict(const float* state6, float kB, float X, int64_t* py, int64_t* pz) { predict(state6, kB, X, py, pz); }

}  // extern "C"
