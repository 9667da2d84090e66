// FP64 CPU oracle of the sector-track merger (Sec. 4: the tracker finds the
// pieces of one track in neighbouring sectors separately and merges them; the
// removal of clusters depends on the merging working).
//
// Test infrastructure only: tests, smoke() and the CPU baseline of the
// benchmark use it; the library never does.  It shares no code with the CUDA
// path.
//
// Readings (the paper states the need for merging, not an algorithm):
//  - geometry: 36 sectors, 18 per side (sectors 0-17 z >= 0, 18-35 z < 0),
//    sector k = s mod 18 centred at azimuth k * 20 degrees; local (x, y) ->
//    global (x cos a - y sin a, x sin a + y cos a);
//  - a track's circle: curvature kappa = 0.299792458e-2 * Bz * q/pT, centre
//    (x_ref + sinphi / kappa, y - cosphi / kappa) in its sector frame, radius
//    1 / |kappa|; tracks with |q/pT| < 1e-4 c/GeV (straight) are not merged;
//  - candidates: tracks of the same event and side in the sectors k + 1 and
//    k - 1 (mod 18), same sign of q/pT; compatible if
//      (a) the curvatures agree: (q/pT_A - q/pT_B)^2 <= 16 (var_A + var_B);
//      (b) the pieces continue each other: the reference point of one lies on
//          the circle of the better measured one (smaller q/pT variance, A on
//          ties) within 1 cm + 3 kB sqrt(var) L^2, L the chord between the two
//          reference points (the sagitta error of a curvature error grows as
//          L^2);
//      (c) |d tan(lambda)| <= 0.02;
//      (d) the outer reference point's z lies within 2 cm of the inner track's
//          z + tan(lambda) * arc, the arc from the chord c between the
//          reference points as c (1 + c^2 / (24 R^2)), R the mean radius;
//          "outer" = larger distance from the beam axis;
//  - score = chi2(a) / 16 + distance(b) / its limit + |d tan(lambda)| / 0.02 +
//    |dz| / 2 cm; per direction the compatible candidate with the smallest
//    score (ties: smaller index); a link joins two tracks that are each
//    other's best in opposite directions;
//  - groups = connected components of the links, labelled by the smallest
//    track index; each group is refitted: the clusters of its tracks in global
//    coordinates (the pad row fixes x), a circle by the algebraic least-squares
//    fit of x^2 + y^2 + D x + E y + F (coordinates centred on their mean), then
//    z = z0 + tan(lambda) s by least squares, s the chord-series arc from the
//    innermost cluster (smallest radius);
//  - looper legs: a helix with radius R < 250 cm can turn inside a sector and
//    comes back inward; the tracker fits the returning (secondary) leg as a
//    track of opposite q/pT and tan(lambda) sign on the same circle (the
//    centre does not change when the direction is reversed).  Candidates:
//    tracks with R < 250 cm of the same event and side, opposite signs of q/pT
//    and of tan(lambda); compatible if (|q/pT_A| - |q/pT_B|)^2 <= 16 (var_A +
//    var_B), the centres lie within 1 cm + 3 kB sqrt(var_A + var_B) R^2, and
//    |tan(lambda)_A + tan(lambda)_B| <= 0.02; score = chi2 / 16 + centre
//    distance / its limit + |sum of tan(lambda)| / 0.02; mutual best pairs are
//    the two legs of one looper; the leg whose reference z is farther from 0
//    (the vertex of an event) is the secondary one (ties: the larger index);
//  - ambiguous: a compatibility quantity within 1e-6 (relative) of its bound,
//    or best and second-best scores within 1e-9: the test then checks only
//    validity for that track.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <tuple>
#include <utility>
#include <vector>

namespace {

struct G {
  bool ok;          // has a circle
  double xc, yc, R;  // global centre and radius
  double X, Y, r;   // global reference point and its distance from the axis
  double z, tgl, qpt, vq;  // vq: variance of q/pT
  int k, side, sign;
  int64_t event;
};

// compatibility of a with b; score and a closeness-to-threshold flag
bool compatible(const G& a, const G& b, double kB, double* score, bool* near) {
  const double chi2 = (a.qpt - b.qpt) * (a.qpt - b.qpt) / std::max(a.vq + b.vq, 1e-30);
  const G& ref = a.vq <= b.vq ? a : b;
  const G& oth = a.vq <= b.vq ? b : a;
  const double L = std::hypot(oth.X - ref.X, oth.Y - ref.Y);
  const double d = std::fabs(std::hypot(oth.X - ref.xc, oth.Y - ref.yc) - ref.R);
  const double dlim = 1.0 + 3.0 * kB * std::sqrt(ref.vq) * L * L;
  const double dt = std::fabs(a.tgl - b.tgl);
  const G& in = a.r <= b.r ? a : b;
  const G& out = a.r <= b.r ? b : a;
  const double c = std::hypot(out.X - in.X, out.Y - in.Y);
  const double Rb = 0.5 * (a.R + b.R);
  const double arc = c * (1.0 + c * c / (24.0 * Rb * Rb));
  const double dz = std::fabs(out.z - (in.z + in.tgl * arc));
  auto close = [](double v, double lim) { return std::fabs(v - lim) <= 1e-6 * std::max(1.0, lim); };
  *near = close(chi2, 16.0) || close(d, dlim) || close(dt, 0.02) || close(dz, 2.0);
  *score = chi2 / 16.0 + d / dlim + dt / 0.02 + dz / 2.0;
  return chi2 <= 16.0 && d <= dlim && dt <= 0.02 && dz <= 2.0;
}

}  // namespace

// trk_f: [n][7] x_ref, y, z, sinphi, tanlambda, q/pT, variance of q/pT;
// trk_i: [n][3] item, first, count into ids.  partner (nullable): the other
// leg of a looper, -1 none; leg (nullable): 1 for a secondary leg, else 0.
extern "C" int64_t orc_merge(int n_rows, double x_min, double x_max, double bz, int64_t n, const float* y,
                             const float* z, const int32_t* row, int64_t n_items, const uint32_t* item_sector,
                             const uint32_t* item_event, int64_t n_trk, const float* trk_f, const int64_t* trk_i,
                             const uint32_t* ids, int32_t* link, int32_t* group, uint8_t* amb, double* fit,
                             int32_t* partner, uint8_t* leg) {
  const double kB = 0.299792458e-2 * bz;
  const double wedge = 2.0 * M_PI / 18.0;
  std::vector<double> xr(n_rows);
  for (int r = 0; r < n_rows; ++r)
    xr[r] = std::nearbyint((x_min + r * ((x_max - x_min) / (n_rows - 1))) * 1024.0) / 1024.0;
  std::vector<G> g(n_trk);
  for (int64_t t = 0; t < n_trk; ++t) {
    const float* f = trk_f + 7 * t;
    const int64_t it = trk_i[3 * t];
    G& q = g[t];
    q.ok = std::fabs(f[5]) >= 1e-4f && it >= 0 && it < n_items;
    if (!q.ok) continue;
    const int s = (int)item_sector[it];
    q.k = s % 18;
    q.side = s / 18;
    q.event = item_event[it];
    const double a = q.k * wedge, ca = std::cos(a), sa = std::sin(a);
    const double kap = kB * f[5];
    const double snp = f[3], csp = std::sqrt(std::max(0.0, 1.0 - snp * snp));
    const double lx = f[0] + snp / kap, ly = f[1] - csp / kap;
    q.xc = lx * ca - ly * sa;
    q.yc = lx * sa + ly * ca;
    q.R = 1.0 / std::fabs(kap);
    q.X = f[0] * ca - f[1] * sa;
    q.Y = f[0] * sa + f[1] * ca;
    q.r = std::hypot(q.X, q.Y);
    q.z = f[2];
    q.tgl = f[4];
    q.vq = std::max(0.0, (double)f[6]);
    q.qpt = f[5];
    q.sign = f[5] > 0 ? 1 : -1;
  }
  // tracks bucketed by (event, side, sector) in index order
  std::map<std::tuple<int64_t, int, int>, std::vector<int64_t>> bucket;
  for (int64_t t = 0; t < n_trk; ++t)
    if (g[t].ok) bucket[std::make_tuple(g[t].event, g[t].side, g[t].k)].push_back(t);
  // best compatible candidate per direction (0: sector k + 1, 1: sector k - 1)
  std::vector<int64_t> best(2 * n_trk, -1);
  for (int64_t t = 0; t < n_trk; ++t) amb[t] = 0;
  for (int64_t a = 0; a < n_trk; ++a) {
    if (!g[a].ok) continue;
    for (int d = 0; d < 2; ++d) {
      const int kb = (g[a].k + (d == 0 ? 1 : 17)) % 18;
      double bs = 0, second = 1e300;
      int64_t bi = -1;
      const auto hit = bucket.find(std::make_tuple(g[a].event, g[a].side, kb));
      if (hit == bucket.end()) continue;
      for (int64_t b : hit->second) {
        if (b == a || g[b].sign != g[a].sign) continue;
        double sc;
        bool near;
        const bool ok = compatible(g[a], g[b], kB, &sc, &near);
        if (near) amb[a] = 1;
        if (!ok) continue;
        if (bi < 0 || sc < bs) {
          if (bi >= 0) second = std::min(second, bs);
          bs = sc;
          bi = b;
        } else {
          second = std::min(second, sc);
        }
      }
      if (bi >= 0 && second - bs <= 1e-9 * std::max(1.0, bs)) amb[a] = 1;
      best[2 * a + d] = bi;
    }
  }
  // mutual links and connected components (label = smallest index)
  std::vector<int64_t> lab(n_trk);
  for (int64_t t = 0; t < n_trk; ++t) {
    lab[t] = t;
    for (int d = 0; d < 2; ++d) {
      const int64_t b = best[2 * t + d];
      link[2 * t + d] = (b >= 0 && best[2 * b + (1 - d)] == t) ? (int32_t)b : -1;
    }
  }
  for (bool changed = true; changed;) {
    changed = false;
    for (int64_t t = 0; t < n_trk; ++t)
      for (int d = 0; d < 2; ++d) {
        const int32_t b = link[2 * t + d];
        if (b >= 0 && lab[b] < lab[t]) {
          lab[t] = lab[b];
          changed = true;
        }
      }
  }
  for (int64_t t = 0; t < n_trk; ++t) group[t] = (int32_t)lab[t];
  // looper legs
  {
    std::map<std::pair<int64_t, int>, std::vector<int64_t>> loopers;  // (event, side) -> tracks with R < 250 cm
    for (int64_t t = 0; t < n_trk; ++t)
      if (g[t].ok && g[t].R < 250.0) loopers[std::make_pair(g[t].event, g[t].side)].push_back(t);
    std::vector<int64_t> lbest(n_trk, -1);
    for (auto& kv : loopers) {
      const auto& v = kv.second;
      for (int64_t a : v) {
        double bs = 0, second = 1e300;
        int64_t bi = -1;
        for (int64_t b : v) {
          if (b == a || g[b].sign == g[a].sign || (g[a].tgl > 0) == (g[b].tgl > 0)) continue;
          const double qa = std::fabs(g[a].qpt), qb = std::fabs(g[b].qpt);
          const double chi2 = (qa - qb) * (qa - qb) / std::max(g[a].vq + g[b].vq, 1e-30);
          const double Rm = std::max(g[a].R, g[b].R);
          const double dlim = 1.0 + 3.0 * kB * std::sqrt(g[a].vq + g[b].vq) * Rm * Rm;
          const double dc = std::hypot(g[a].xc - g[b].xc, g[a].yc - g[b].yc);
          const double st = std::fabs(g[a].tgl + g[b].tgl);
          auto close = [](double x, double lim) { return std::fabs(x - lim) <= 1e-6 * std::max(1.0, lim); };
          if (close(chi2, 16.0) || close(dc, dlim) || close(st, 0.02)) amb[a] = 1;
          if (!(chi2 <= 16.0 && dc <= dlim && st <= 0.02)) continue;
          const double sc = chi2 / 16.0 + dc / dlim + st / 0.02;
          if (bi < 0 || sc < bs) {
            if (bi >= 0) second = std::min(second, bs);
            bs = sc;
            bi = b;
          } else {
            second = std::min(second, sc);
          }
        }
        if (bi >= 0 && second - bs <= 1e-9 * std::max(1.0, bs)) amb[a] = 1;
        lbest[a] = bi;
      }
    }
    for (int64_t t = 0; t < n_trk; ++t) {
      const int64_t p = lbest[t];
      const bool mutual = p >= 0 && lbest[p] == t;
      if (partner) partner[t] = mutual ? (int32_t)p : -1;
      if (leg) {
        const double zt = std::fabs(g[t].z), zp = mutual ? std::fabs(g[p].z) : 0.0;
        leg[t] = (mutual && (zt > zp || (zt == zp && t > p))) ? 1 : 0;
      }
    }
  }
  // refit of every group: fit[root] = (xc, yc, R, tgl, z0, n_clusters, n_tracks)
  std::vector<std::vector<int64_t>> members(n_trk);
  for (int64_t t = 0; t < n_trk; ++t) members[lab[t]].push_back(t);
  for (int64_t t = 0; t < 7 * n_trk; ++t) fit[t] = 0.0;
  for (int64_t root = 0; root < n_trk; ++root) {
    if (members[root].empty() || !g[root].ok) continue;
    std::vector<double> X, Y, Z;
    for (int64_t t : members[root]) {
      const int s = (int)item_sector[trk_i[3 * t]];
      const double a = (s % 18) * wedge, ca = std::cos(a), sa = std::sin(a);
      for (int64_t j = 0; j < trk_i[3 * t + 2]; ++j) {
        const uint32_t c = ids[trk_i[3 * t + 1] + j];
        if (c >= (uint64_t)n || row[c] < 0 || row[c] >= n_rows) return -1;
        const double lx = xr[row[c]], ly = y[c];
        X.push_back(lx * ca - ly * sa);
        Y.push_back(lx * sa + ly * ca);
        Z.push_back(z[c]);
      }
    }
    const size_t m = X.size();
    if (m < 3) continue;
    double mx = 0, my = 0;
    for (size_t i = 0; i < m; ++i) {
      mx += X[i];
      my += Y[i];
    }
    mx /= m;
    my /= m;
    double suu = 0, suv = 0, svv = 0, su3 = 0, sv3 = 0, sw = 0;
    for (size_t i = 0; i < m; ++i) {
      const double u = X[i] - mx, v = Y[i] - my, w = u * u + v * v;
      suu += u * u;
      suv += u * v;
      svv += v * v;
      su3 += u * w;
      sv3 += v * w;
      sw += w;
    }
    const double det = suu * svv - suv * suv;
    if (!(std::fabs(det) > 0)) continue;
    const double D = (-su3 * svv + sv3 * suv) / det, E = (-sv3 * suu + su3 * suv) / det, F = -sw / m;
    const double xc = mx - 0.5 * D, yc = my - 0.5 * E;
    const double R = std::sqrt(0.25 * (D * D + E * E) - F);
    size_t in = 0;
    for (size_t i = 1; i < m; ++i)
      if (std::hypot(X[i], Y[i]) < std::hypot(X[in], Y[in])) in = i;
    double ss = 0, sz = 0, sss = 0, ssz = 0;
    for (size_t i = 0; i < m; ++i) {
      const double c = std::hypot(X[i] - X[in], Y[i] - Y[in]);
      const double s = c * (1.0 + c * c / (24.0 * R * R));
      ss += s;
      sz += Z[i];
      sss += s * s;
      ssz += s * Z[i];
    }
    const double den = m * sss - ss * ss;
    const double tgl = den > 0 ? (m * ssz - ss * sz) / den : 0.0;
    const double z0 = (sz - tgl * ss) / m;
    double* o = fit + 7 * root;
    o[0] = xc;
    o[1] = yc;
    o[2] = R;
    o[3] = tgl;
    o[4] = z0;
    o[5] = (double)m;
    o[6] = (double)members[root].size();
  }
  return 0;
}

// Looper legs joined into one track (Sec. 4: the tracker finds the legs of a
// looping track separately and merges them into one track).  Reading:
//  - components: the groups of the merger joined through every mutual leg
//    pair (union of the two legs' groups), labelled by their smallest track
//    index; tracks of other groups keep their group label;
//  - refit of every component that contains a pair: the clusters of all its
//    tracks in the global frame, the algebraic circle as for the groups, then
//    z = z0 + tan(lambda) s by least squares, s = R dtheta the arc along the
//    circle from the innermost cluster of the primary legs (the first leg from
//    the vertex, leg = 0; ties: the first cluster in track-index order), dtheta
//    the turning angle in the particle's sense of rotation (clockwise for
//    q/pT > 0 of the primary leg with the smallest index: its centre lies to
//    the right of its direction) taken in [-0.1, 2 pi - 0.1).  The chord from
//    the innermost cluster cannot be used: the returning leg passes the same
//    radii again.
//  joined: [n] component label; jfit: [n][7] at each joined component's label:
//  centre x, y, radius, tan(lambda), z0 (at the reference cluster), clusters,
//  tracks; zero elsewhere.  Returns the number of joined components, -1 on bad
//  input.
extern "C" int64_t orc_join_loopers(int n_rows, double x_min, double x_max, double bz, int64_t n, const float* y,
                                    const float* z, const int32_t* row, int64_t n_items, const uint32_t* item_sector,
                                    int64_t n_trk, const float* trk_f, const int64_t* trk_i, const uint32_t* ids,
                                    const int32_t* group, const int32_t* partner, const uint8_t* leg, int32_t* joined,
                                    double* jfit) {
  (void)bz;
  const double wedge = 2.0 * M_PI / 18.0;
  std::vector<double> xr(n_rows);
  for (int r = 0; r < n_rows; ++r)
    xr[r] = std::nearbyint((x_min + r * ((x_max - x_min) / (n_rows - 1))) * 1024.0) / 1024.0;
  // union of groups through the pairs: lab[g] of every group root g ends as the
  // smallest root of its component (= its smallest track index)
  std::vector<int64_t> lab(n_trk);
  for (int64_t t = 0; t < n_trk; ++t) lab[t] = group[t];
  std::vector<char> paired(n_trk, 0);
  for (bool changed = true; changed;) {
    changed = false;
    for (int64_t t = 0; t < n_trk; ++t) {
      const int64_t p = partner[t];
      if (p < 0 || p >= n_trk || partner[p] != t) continue;
      paired[t] = 1;
      const int64_t m = std::min(lab[group[t]], lab[group[p]]);
      if (lab[group[t]] != m) lab[group[t]] = m, changed = true;
      if (lab[group[p]] != m) lab[group[p]] = m, changed = true;
    }
  }
  for (int64_t t = 0; t < n_trk; ++t) joined[t] = (int32_t)lab[group[t]];
  for (int64_t t = 0; t < 7 * n_trk; ++t) jfit[t] = 0.0;
  std::vector<std::vector<int64_t>> members(n_trk);
  std::vector<char> has_pair(n_trk, 0);
  for (int64_t t = 0; t < n_trk; ++t) {
    members[joined[t]].push_back(t);
    if (paired[t]) has_pair[joined[t]] = 1;
  }
  int64_t n_joined = 0;
  for (int64_t root = 0; root < n_trk; ++root) {
    if (!has_pair[root]) continue;
    // the primary legs' groups and the sense of rotation
    std::vector<char> prim_group(n_trk, 0);
    int64_t first_prim = -1;
    for (int64_t t : members[root])
      if (paired[t] && leg[t] == 0) {
        prim_group[group[t]] = 1;
        if (first_prim < 0) first_prim = t;
      }
    if (first_prim < 0) continue;
    std::vector<double> X, Y, Z;
    std::vector<char> P;
    for (int64_t t : members[root]) {
      if (trk_i[3 * t] < 0 || trk_i[3 * t] >= n_items) return -1;
      const int s = (int)item_sector[trk_i[3 * t]];
      const double a = (s % 18) * wedge, ca = std::cos(a), sa = std::sin(a);
      for (int64_t j = 0; j < trk_i[3 * t + 2]; ++j) {
        const uint32_t c = ids[trk_i[3 * t + 1] + j];
        if (c >= (uint64_t)n || row[c] < 0 || row[c] >= n_rows) return -1;
        const double lx = xr[row[c]], ly = y[c];
        X.push_back(lx * ca - ly * sa);
        Y.push_back(lx * sa + ly * ca);
        Z.push_back(z[c]);
        P.push_back(prim_group[group[t]]);
      }
    }
    const size_t m = X.size();
    if (m < 3) continue;
    double mx = 0, my = 0;
    for (size_t i = 0; i < m; ++i) {
      mx += X[i];
      my += Y[i];
    }
    mx /= m;
    my /= m;
    double suu = 0, suv = 0, svv = 0, su3 = 0, sv3 = 0, sw = 0;
    for (size_t i = 0; i < m; ++i) {
      const double u = X[i] - mx, v = Y[i] - my, w = u * u + v * v;
      suu += u * u;
      suv += u * v;
      svv += v * v;
      su3 += u * w;
      sv3 += v * w;
      sw += w;
    }
    const double det = suu * svv - suv * suv;
    if (!(std::fabs(det) > 0)) continue;
    const double D = (-su3 * svv + sv3 * suv) / det, E = (-sv3 * suu + su3 * suv) / det, F = -sw / m;
    const double xc = mx - 0.5 * D, yc = my - 0.5 * E;
    const double R = std::sqrt(0.25 * (D * D + E * E) - F);
    size_t ref = m;
    for (size_t i = 0; i < m; ++i)
      if (P[i] && (ref == m || std::hypot(X[i], Y[i]) < std::hypot(X[ref], Y[ref]))) ref = i;
    const bool cw = trk_f[7 * first_prim + 5] > 0.0f;
    const double th0 = std::atan2(Y[ref] - yc, X[ref] - xc);
    double ss = 0, sz = 0, sss = 0, ssz = 0;
    for (size_t i = 0; i < m; ++i) {
      double d = cw ? th0 - std::atan2(Y[i] - yc, X[i] - xc) : std::atan2(Y[i] - yc, X[i] - xc) - th0;
      d -= 2.0 * M_PI * std::floor((d + 0.1) / (2.0 * M_PI));
      const double s = R * d;
      ss += s;
      sz += Z[i];
      sss += s * s;
      ssz += s * Z[i];
    }
    const double den = m * sss - ss * ss;
    const double tgl = den > 0 ? (m * ssz - ss * sz) / den : 0.0;
    const double z0 = (sz - tgl * ss) / m;
    double* o = jfit + 7 * root;
    o[0] = xc;
    o[1] = yc;
    o[2] = R;
    o[3] = tgl;
    o[4] = z0;
    o[5] = (double)m;
    o[6] = (double)members[root].size();
    ++n_joined;
  }
  return n_joined;
}
