// FP64 CPU oracle of cluster-to-track association (attachment and
// adjacency), protection, and the cluster-removal masks of strategies A and B
// (Sec. 4, "TPC Data Reduction", the removal steps).
//
// Test infrastructure only: tests, smoke() and the CPU baseline of the
// benchmark use it; the library never does.  It shares no code with the CUDA
// path; the track model is the oracle's own propagation (tpc_oracle.cpp).
//
// What the paper fixes (Sec. 4): tracking attaches clusters to tracks, and an
// ambiguous cluster goes to the track of higher momentum; clusters inside a
// tube of 1.5 cm around a track are adjacent to it, ambiguity again going to
// the higher-momentum track; clusters adjacent to the primary leg of a track
// with pT > 50 MeV/c and a local inclination |phi| < 70 degrees are protected.
// Strategy B removes every cluster that is not protected; strategy A removes
// the clusters that are not protected and are attached or adjacent to a track
// with pT <= 50 MeV/c, to a secondary leg, or to a track with |phi| >= 70.
//
// Readings (the paper gives the rule, not its geometry):
//  - candidates of a cluster: the tracks whose cluster list holds it
//    (attachment) and the tracks of its work item whose tube holds it
//    (adjacency); it goes to the candidate with the highest pT, i.e. the
//    smallest |q/pT| of the float32 track state, ties to the smaller track
//    index.  "Attached or adjacent" = it has a candidate;
//  - tube: in the cluster's pad-row plane, the distance between the cluster
//    (its quantised coordinates, 2^-10 cm) and the point where the track
//    crosses that plane is at most the tube radius; only rows from the
//    track's innermost to its outermost cluster row count, and only rows the
//    track reaches (the tracker's propagation is valid there);
//  - local inclination: sin(phi) of the winning track at the cluster's row,
//    linear in x (Bz fixed); |phi| < 70 deg <=> |sin phi| < fl32(sin 70 deg);
//  - pT > 50 MeV/c <=> |q/pT| < fl32(1 / 0.05 GeV) = 20 c/GeV;
//  - the leg of a track is an input (0 = primary); a sector tracker without
//    a merger makes every track its own primary leg;
//  - a cluster is flagged ambiguous when rounding could change its result: a
//    tube distance within 1e-3 cm of the radius, a |sin phi| within 1e-5 of
//    the propagation limit, or the winner's |sin phi| within 1e-5 of the
//    inclination limit.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

extern "C" int orc_propagate(const double* p_in, double x1, double x2, double bz, double* p_out, double* F);

namespace {

const double KB_PER_TESLA = 0.299792458e-2;
const double SNP_LIMIT = 0.9999;

enum : uint8_t { ASSOCIATED = 1, PROTECTED = 2, REMOVE_A = 4, REMOVE_B = 8 };

struct Trk {
  double x_ref, y, z, snp, tgl;
  float qpt;
  int64_t item, first, count;
};

// a better than b: higher pT (smaller |q/pT|), ties to the smaller index; b < 0 = none
bool better(const std::vector<Trk>& T, int64_t a, int64_t b) {
  if (b < 0) return true;
  const float qa = std::fabs(T[a].qpt), qb = std::fabs(T[b].qpt);
  return qa < qb || (qa == qb && a < b);
}

}  // namespace

extern "C" int64_t orc_cluster_masks(int n_rows, double x_min, double x_max, double bz, int64_t n, const float* y,
                                     const float* z, const int32_t* row, const uint64_t* item_off, int64_t n_items,
                                     int64_t n_trk, const float* trk_f, const int64_t* trk_i, const uint32_t* ids,
                                     const uint8_t* leg, double tube, float max_qpt, float max_snp, uint8_t* mask,
                                     int32_t* owner, uint8_t* ambiguous) {
  // pad-row radii (quantised to 2^-10 cm, as the tracker places its rows)
  std::vector<double> xr(n_rows);
  for (int r = 0; r < n_rows; ++r)
    xr[r] = std::nearbyint((x_min + r * ((x_max - x_min) / (n_rows - 1))) * 1024.0) / 1024.0;
  std::vector<Trk> T(n_trk);
  for (int64_t t = 0; t < n_trk; ++t) {
    const float* f = trk_f + 6 * t;
    T[t] = Trk{f[0], f[1], f[2], f[3], f[4], f[5], trk_i[3 * t], trk_i[3 * t + 1], trk_i[3 * t + 2]};
  }
  // attachment: the best track among those holding each cluster
  std::vector<int64_t> best(n, -1);
  for (int64_t t = 0; t < n_trk; ++t)
    for (int64_t j = 0; j < T[t].count; ++j) {
      const int64_t c = ids[T[t].first + j];
      if (better(T, t, best[c])) best[c] = t;
    }
  std::vector<std::vector<int64_t>> of_item(n_items);
  for (int64_t t = 0; t < n_trk; ++t)
    if (T[t].item >= 0 && T[t].item < n_items) of_item[T[t].item].push_back(t);
  for (int64_t c = 0; c < n; ++c) ambiguous[c] = 0;

  for (int64_t it = 0; it < n_items; ++it) {
    // every track of the item at every row of its span: position, or unreachable
    struct Pos {
      bool ok;
      double y, z;
    };
    const auto& tr = of_item[it];
    std::vector<int> lo(tr.size()), hi(tr.size());
    std::vector<std::vector<Pos>> pos(tr.size());
    for (size_t k = 0; k < tr.size(); ++k) {
      const Trk& t = T[tr[k]];
      if (t.count <= 0) {
        lo[k] = 1;
        hi[k] = 0;
        continue;
      }
      const int ra = row[ids[t.first]], rb = row[ids[t.first + t.count - 1]];
      lo[k] = std::min(ra, rb);
      hi[k] = std::max(ra, rb);
      for (int r = lo[k]; r <= hi[k]; ++r) {
        const double p[5] = {t.y, t.z, t.snp, t.tgl, (double)t.qpt};
        double q[5];
        Pos P{false, 0, 0};
        if (orc_propagate(p, t.x_ref, xr[r], bz, q, nullptr)) P = Pos{true, q[0], q[1]};
        pos[k].push_back(P);
      }
    }
    for (uint64_t c = item_off[it]; c < item_off[it + 1]; ++c) {
      const int r = row[c];
      if (r < 0 || r >= n_rows || !std::isfinite(y[c]) || !std::isfinite(z[c])) continue;  // never binned
      const double cy = std::nearbyint((double)y[c] * 1024.0) / 1024.0;
      const double cz = std::nearbyint((double)z[c] * 1024.0) / 1024.0;
      for (size_t k = 0; k < tr.size(); ++k) {
        if (r < lo[k] || r > hi[k]) continue;
        const Trk& t = T[tr[k]];
        const double s2 = t.snp - KB_PER_TESLA * bz * (double)t.qpt * (xr[r] - t.x_ref);
        if (std::fabs(std::fabs(s2) - SNP_LIMIT) < 1e-5) ambiguous[c] = 1;
        const Pos& P = pos[k][r - lo[k]];
        if (!P.ok) continue;
        const double d = std::hypot(cy - P.y, cz - P.z);
        if (std::fabs(d - tube) < 1e-3) ambiguous[c] = 1;
        if (d <= tube && better(T, tr[k], best[c])) best[c] = tr[k];
      }
    }
  }

  int64_t n_amb = 0;
  for (int64_t c = 0; c < n; ++c) {
    const int64_t w = best[c];
    owner[c] = (int32_t)w;
    if (w < 0) {
      mask[c] = REMOVE_B;
    } else {
      const Trk& t = T[w];
      const int r = row[c];
      const double xc = (r >= 0 && r < n_rows) ? xr[r] : t.x_ref;
      const double s = std::fabs(t.snp - KB_PER_TESLA * bz * (double)t.qpt * (xc - t.x_ref));
      if (std::fabs(s - (double)max_snp) < 1e-5) ambiguous[c] = 1;
      const bool prot = std::fabs(t.qpt) < max_qpt && (!leg || leg[w] == 0) && s < (double)max_snp;
      mask[c] = prot ? (ASSOCIATED | PROTECTED) : (ASSOCIATED | REMOVE_A | REMOVE_B);
    }
    n_amb += ambiguous[c];
  }
  return n_amb;
}
