// FP64 CPU oracle of the TPC sector tracker -- TEST INFRASTRUCTURE ONLY.
//
// Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
// file.  It is a plain single-threaded restatement of the tracker's steps, written
// for a reader to check by eye: std::stable_sort for binning, nested loops for the
// neighbour search, one std::vector per tracklet, a sequential max-key loop for the
// shared-cluster resolution.  It shares nothing with the CUDA library.
//
// The paper (Sec. 3) derives the tracker from the Run 2 HLT cellular-automaton
// tracker and gives no constants; every constant below is a documented reading:
//   * cluster coordinates are quantised to Q = 2^-10 cm integers (the paper's
//     float->integer conversion, Sec. 4 step 2) so that every discrete decision of
//     binning, linking and selection is exact integer arithmetic and cannot differ
//     between CPU and GPU (the order and rounding effects of Sec. 3);
//   * segments with |phi| >= 70 deg are not fitted (Sec. 4, removal list item 3);
//   * numerical failures of the fit end the tracklet (Sec. 4, looper discussion);
//   * an ambiguous cluster goes to the better track (Sec. 4, cluster attachment);
//   * continuous read-out with an unknown vertex position (Abstract): no vertex
//     constraint anywhere, z may carry a drift-time offset.
#include "tpc_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

namespace {

const double QSCALE = 1024.0;            // quanta per cm
const double KB_PER_TESLA = 0.299792458e-2; // curvature [1/cm] per (q/pT [c/GeV] * B [T])
const int SHIFT_MIN = 10;                // smallest bin edge: 2^10 quanta = 1 cm
const int64_t LINK_D = 512;              // chord deviation cut for a link: 0.5 cm in quanta
const double CHI2_CUT = 16.0;            // hit acceptance during extension
const double WIN_MIN = 0.5;              // minimum search half-width [cm]
const int MAX_MISS = 5;                  // consecutive rows without a hit end a pass
const double SIN_MAX = 0.93969262078590838; // sin(70 deg)
const int MIN_HITS = 10;                 // minimum tracklet / track size
const double SNP_LIMIT = 0.9999;         // propagation validity
const double C0_DIAG_ANGLE = 1.0, C0_DIAG_QPT = 100.0;
const double INFLATE = 100.0;            // refit prior: outward variances x100 (at most C0)

struct Row {  // one (item, pad row) of the binning grid
  int pos0 = 0, n = 0, ymin = 0, zmin = 0, shift = SHIFT_MIN, ny = 0, nz = 0;
  std::vector<int> first;  // nbins+1 sorted positions (absolute)
};

struct Tracklet {
  int item = 0, local_id = 0;
  bool valid = false;
  std::vector<int> hits;  // sorted positions, row-descending (downward pass)
  double p[5] = {0, 0, 0, 0, 0}, C[5][5] = {{0}}, chi2 = 0, x_ref = 0;
  int n = 0;
};

struct Track {
  int item, tracklet, first, count;
  double x_ref, p[5], C[5][5], chi2;
  int ndf;
};

}  // namespace

struct orc_result {
  orc_config cfg;
  std::vector<double> row_x;
  std::vector<int> row_qx;
  int n_rows = 0;
  uint32_t n_items = 0;
  std::vector<uint64_t> item_off;
  std::vector<int> qy, qz, id;          // sorted (canonical) order
  std::vector<int> item_of_pos;
  std::vector<Row> rows;                // [item*n_rows + row]
  std::vector<int> up_raw, dn_raw, up, dn;  // sorted positions, -1 = none
  std::vector<int> starts;              // sorted positions, canonical order
  std::vector<Tracklet> tracklets;
  std::vector<Track> tracks;
  std::vector<int> track_ids;           // original ids
};

namespace {

// ---------------------------------------------------------------- track model
// State (y, z, sinphi, tanlambda, q/pT) at sector-local x.  Helix in a uniform Bz:
// along +x the curvature kappa = kB*q/pT turns sinphi by -kappa*dx; y follows the
// circle chord, z grows with the transverse arc length.

double asin_over_u(double u) {  // asin(u)/u
  if (std::fabs(u) < 0.05) {
    double u2 = u * u;
    return 1.0 + u2 * (1.0 / 6.0 + u2 * (3.0 / 40.0 + u2 * (5.0 / 112.0 + u2 * (35.0 / 1152.0))));
  }
  return std::asin(u) / u;
}

double d_asin_over_u(double u) {  // d/du [asin(u)/u]
  if (std::fabs(u) < 0.05) {
    double u2 = u * u;
    return u * (1.0 / 3.0 + u2 * (3.0 / 10.0 + u2 * (15.0 / 56.0 + u2 * (35.0 / 144.0))));
  }
  return (u / std::sqrt(1.0 - u * u) - std::asin(u)) / (u * u);
}

bool propagate(const double* p, double x1, double x2, double bz, double* q, double F[5][5]) {
  const double kB = KB_PER_TESLA * bz;
  const double dx = x2 - x1;
  const double s1 = p[2];
  const double kappa = kB * p[4];
  const double s2 = s1 - kappa * dx;
  if (!(std::fabs(s1) < SNP_LIMIT) || !(std::fabs(s2) < SNP_LIMIT)) return false;
  const double c1 = std::sqrt(1.0 - s1 * s1), c2 = std::sqrt(1.0 - s2 * s2);
  const double T = (s1 + s2) / (c1 + c2);  // tan of the chord direction
  const double w = std::sqrt(1.0 + T * T);
  const double u = 0.5 * kappa * std::fabs(dx) * w;  // sin of half the turning angle
  if (!(std::fabs(u) < 1.0)) return false;
  const double f = asin_over_u(u);
  const double ell = dx * w * f;  // signed transverse arc length
  q[0] = p[0] + dx * T;
  q[1] = p[1] + p[3] * ell;
  q[2] = s2;
  q[3] = p[3];
  q[4] = p[4];
  if (F) {
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) F[i][j] = (i == j) ? 1.0 : 0.0;
    const double num = 1.0 + c1 * c2 + s1 * s2;
    const double den = (c1 + c2) * (c1 + c2);
    const double A1 = num / (c1 * den);  // dT/ds1 at fixed s2
    const double A2 = num / (c2 * den);  // dT/ds2 at fixed s1
    const double dT_ds = A1 + A2;        // s2 moves with s1
    const double dT_dq = A2 * (-kB * dx);
    const double fp = d_asin_over_u(u);
    const double dg_dT = (T / w) * (f + u * fp);
    const double dg_dk = 0.5 * w * w * std::fabs(dx) * fp;
    const double dl_ds = dx * dg_dT * dT_ds;
    const double dl_dq = dx * (dg_dT * dT_dq + dg_dk * kB);
    F[0][2] = dx * dT_ds;
    F[0][4] = dx * dT_dq;
    F[1][2] = p[3] * dl_ds;
    F[1][3] = ell;
    F[1][4] = p[3] * dl_dq;
    F[2][4] = -kB * dx;
  }
  return true;
}

void transport(double C[5][5], double F[5][5]) {  // C <- F C F^T
  double T[5][5], R[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double s = 0;
      for (int k = 0; k < 5; ++k) s += F[i][k] * C[k][j];
      T[i][j] = s;
    }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      double s = 0;
      for (int k = 0; k < 5; ++k) s += T[i][k] * F[j][k];
      R[i][j] = s;
    }
  std::memcpy(C, R, sizeof(R));
}

// chi2 of a measurement (my, mz) against the predicted state; S = H C H^T + V
double chi2_of(const double* p, double C[5][5], double my, double mz, double vy, double vz) {
  const double r0 = my - p[0], r1 = mz - p[1];
  const double S00 = C[0][0] + vy, S01 = C[0][1], S11 = C[1][1] + vz;
  const double det = S00 * S11 - S01 * S01;
  return (S11 * r0 * r0 - 2.0 * S01 * r0 * r1 + S00 * r1 * r1) / det;
}

// Kalman measurement update with H = [I2 0]; returns the chi2 increment.
double update(double* p, double C[5][5], double my, double mz, double vy, double vz) {
  const double r0 = my - p[0], r1 = mz - p[1];
  const double S00 = C[0][0] + vy, S01 = C[0][1], S11 = C[1][1] + vz;
  const double det = S00 * S11 - S01 * S01;
  const double I00 = S11 / det, I01 = -S01 / det, I11 = S00 / det;
  double K[5][2];
  for (int i = 0; i < 5; ++i) {
    K[i][0] = C[i][0] * I00 + C[i][1] * I01;
    K[i][1] = C[i][0] * I01 + C[i][1] * I11;
  }
  for (int i = 0; i < 5; ++i) p[i] += K[i][0] * r0 + K[i][1] * r1;
  double HC[2][5];
  for (int j = 0; j < 5; ++j) {
    HC[0][j] = C[0][j];
    HC[1][j] = C[1][j];
  }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) C[i][j] -= K[i][0] * HC[0][j] + K[i][1] * HC[1][j];
  return r0 * (I00 * r0 + I01 * r1) + r1 * (I01 * r0 + I11 * r1);
}

bool cov_ok(double C[5][5]) {
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j)
      if (!std::isfinite(C[i][j])) return false;
  for (int i = 0; i < 5; ++i)
    if (!(C[i][i] > 0.0)) return false;
  return true;
}

// propagate state and covariance; false if the step is not valid
bool kf_propagate(double* p, double C[5][5], double x1, double x2, double bz) {
  double q[5], F[5][5];
  if (!propagate(p, x1, x2, bz, q, F)) return false;
  std::memcpy(p, q, sizeof(q));
  transport(C, F);
  return true;
}

void set_c0(double C[5][5], double vy, double vz) {
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) C[i][j] = 0.0;
  C[0][0] = vy;
  C[1][1] = vz;
  C[2][2] = C0_DIAG_ANGLE;
  C[3][3] = C0_DIAG_ANGLE;
  C[4][4] = C0_DIAG_QPT;
}

// ---------------------------------------------------------------- helpers
struct Ctx {
  orc_result* R;
  double tanh_, vy, vz, bz;
  const Row& row(int item, int r) const { return R->rows[(size_t)item * R->n_rows + r]; }
  double hy(int pos) const { return R->qy[pos] / QSCALE; }
  double hz(int pos) const { return R->qz[pos] / QSCALE; }
};

// Visit every hit of a row whose bin overlaps the quanta box [ylo,yhi]x[zlo,zhi]
// (or every hit of the row in brute mode).
template <class Fn>
void visit_box(const Ctx& c, int item, int r, int64_t ylo, int64_t yhi, int64_t zlo, int64_t zhi, Fn fn) {
  const Row& rw = c.row(item, r);
  if (rw.n == 0) return;
  if (c.R->cfg.brute) {
    for (int p = rw.pos0; p < rw.pos0 + rw.n; ++p) fn(p);
    return;
  }
  const int64_t ymax = rw.ymin + ((int64_t)rw.ny << rw.shift) - 1;
  const int64_t zmax = rw.zmin + ((int64_t)rw.nz << rw.shift) - 1;
  if (yhi < rw.ymin || ylo > ymax || zhi < rw.zmin || zlo > zmax) return;
  const int iy0 = ylo <= rw.ymin ? 0 : (int)((ylo - rw.ymin) >> rw.shift);
  const int iy1 = std::min<int64_t>(rw.ny - 1, (yhi - rw.ymin) >> rw.shift);
  const int iz0 = zlo <= rw.zmin ? 0 : (int)((zlo - rw.zmin) >> rw.shift);
  const int iz1 = std::min<int64_t>(rw.nz - 1, (zhi - rw.zmin) >> rw.shift);
  for (int iy = iy0; iy <= iy1; ++iy)
    for (int iz = iz0; iz <= iz1; ++iz) {
      const int b = iy * rw.nz + iz;
      for (int p = rw.first[b]; p < rw.first[b + 1]; ++p) fn(p);
    }
}

// ---------------------------------------------------------------- binning
// Per (item,row): extents, bin edge 2^s quanta, counting grid, canonical order
// (row, bin, original id) by a stable sort.  Reading of the bin size: s is the
// smallest s >= 10 with n*4^s >= Ly*Lz (about one hit per bin) and
// ny*nz <= 2n+2 (a bounded grid).
void binning(orc_result* R, const std::vector<int>& qy_in, const std::vector<int>& qz_in,
             const int32_t* row_in) {
  const int NR = R->n_rows;
  R->rows.assign((size_t)R->n_items * NR, Row());
  R->qy.resize(qy_in.size());
  R->qz.resize(qy_in.size());
  R->id.resize(qy_in.size());
  R->item_of_pos.resize(qy_in.size());
  for (uint32_t it = 0; it < R->n_items; ++it) {
    const int64_t a = (int64_t)R->item_off[it], b = (int64_t)R->item_off[it + 1];
    std::vector<std::vector<int>> by_row(NR);
    for (int64_t i = a; i < b; ++i) by_row[row_in[i]].push_back((int)i);
    struct Key { int row, bin, id; };
    std::vector<Key> keys;
    int pos = (int)a;
    for (int r = 0; r < NR; ++r) {
      Row& rw = R->rows[(size_t)it * NR + r];
      const std::vector<int>& h = by_row[r];
      rw.pos0 = pos;
      rw.n = (int)h.size();
      if (rw.n == 0) {
        rw.first.assign(1, pos);
        continue;
      }
      int ymin = qy_in[h[0]], ymax = ymin, zmin = qz_in[h[0]], zmax = zmin;
      for (int i : h) {
        ymin = std::min(ymin, qy_in[i]);
        ymax = std::max(ymax, qy_in[i]);
        zmin = std::min(zmin, qz_in[i]);
        zmax = std::max(zmax, qz_in[i]);
      }
      const int64_t Ly = (int64_t)ymax - ymin + 1, Lz = (int64_t)zmax - zmin + 1;
      int s = SHIFT_MIN;
      for (;; ++s) {
        const int64_t ny = (((int64_t)ymax - ymin) >> s) + 1, nz = (((int64_t)zmax - zmin) >> s) + 1;
        const bool dense_enough = (__int128)rw.n << (2 * s) >= (__int128)Ly * Lz;
        if (dense_enough && ny * nz <= 2 * (int64_t)rw.n + 2) break;
      }
      rw.ymin = ymin;
      rw.zmin = zmin;
      rw.shift = s;
      rw.ny = (int)((((int64_t)ymax - ymin) >> s) + 1);
      rw.nz = (int)((((int64_t)zmax - zmin) >> s) + 1);
      const int nb = rw.ny * rw.nz;
      std::vector<int> count(nb, 0);
      keys.clear();
      for (int i : h) {
        const int bin = ((qy_in[i] - ymin) >> s) * rw.nz + ((qz_in[i] - zmin) >> s);
        keys.push_back({r, bin, i});
        count[bin]++;
      }
      std::stable_sort(keys.begin(), keys.end(), [](const Key& u, const Key& v) {
        if (u.bin != v.bin) return u.bin < v.bin;
        return u.id < v.id;
      });
      rw.first.assign(nb + 1, 0);
      rw.first[0] = pos;
      for (int k = 0; k < nb; ++k) rw.first[k + 1] = rw.first[k] + count[k];
      for (const Key& k : keys) {
        R->qy[pos] = qy_in[k.id];
        R->qz[pos] = qz_in[k.id];
        R->id[pos] = k.id;
        R->item_of_pos[pos] = (int)it;
        ++pos;
      }
    }
  }
}

// ---------------------------------------------------------------- neighbours
// For every hit h on an inner row (1..n_rows-2): the pair (u on r+1, d on r-1),
// each inside the window |dqy| <= 2.75*dqx, |dqz| <= 3.2*dqx, whose chord passes
// closest to h (2.75 = tan 70 deg; 3.2 > sinh(0.9)/cos 70 deg, the steepest z slope
// per unit x of a fitted segment): minimise m = dY^2 + dZ^2 with
//   dY = (qy_u - qy_h)*dx_dn - (qy_h - qy_d)*dx_up  (dx in quanta, exact int64),
// accept if m <= ((dx_up + dx_dn) * D)^2; ties by smaller id_u, then smaller id_d.
void neighbours(orc_result* R) {
  const int NR = R->n_rows;
  const size_t N = R->qy.size();
  R->up_raw.assign(N, -1);
  R->dn_raw.assign(N, -1);
  Ctx c{R};
  for (uint32_t it = 0; it < R->n_items; ++it) {
    for (int r = 1; r + 1 < NR; ++r) {
      const Row& rw = c.row(it, r);
      const int64_t dx_up = R->row_qx[r + 1] - R->row_qx[r];
      const int64_t dx_dn = R->row_qx[r] - R->row_qx[r - 1];
      const int64_t wy_u = dx_up * 11 / 4, wz_u = dx_up * 16 / 5;
      const int64_t wy_d = dx_dn * 11 / 4, wz_d = dx_dn * 16 / 5;
      const int64_t cut = (dx_up + dx_dn) * LINK_D;
      const int64_t cut2 = cut * cut;
      for (int h = rw.pos0; h < rw.pos0 + rw.n; ++h) {
        const int64_t yh = R->qy[h], zh = R->qz[h];
        std::vector<int> U, D;
        visit_box(c, it, r + 1, yh - wy_u, yh + wy_u, zh - wz_u, zh + wz_u, [&](int p) {
          if (std::llabs(R->qy[p] - yh) <= wy_u && std::llabs(R->qz[p] - zh) <= wz_u) U.push_back(p);
        });
        visit_box(c, it, r - 1, yh - wy_d, yh + wy_d, zh - wz_d, zh + wz_d, [&](int p) {
          if (std::llabs(R->qy[p] - yh) <= wy_d && std::llabs(R->qz[p] - zh) <= wz_d) D.push_back(p);
        });
        int64_t best = -1;
        int bu = -1, bd = -1;
        for (int u : U)
          for (int d : D) {
            const int64_t dY = (R->qy[u] - yh) * dx_dn - (yh - R->qy[d]) * dx_up;
            const int64_t dZ = (R->qz[u] - zh) * dx_dn - (zh - R->qz[d]) * dx_up;
            const int64_t m = dY * dY + dZ * dZ;
            if (m > cut2) continue;
            bool better = best < 0 || m < best;
            if (!better && m == best) {
              if (R->id[u] != R->id[bu]) better = R->id[u] < R->id[bu];
              else better = R->id[d] < R->id[bd];
            }
            if (better) {
              best = m;
              bu = u;
              bd = d;
            }
          }
        R->up_raw[h] = bu;
        R->dn_raw[h] = bd;
      }
    }
  }
  // keep only mutual links (reads the raw arrays only, so the result does not
  // depend on the order of processing)
  R->up.assign(N, -1);
  R->dn.assign(N, -1);
  for (size_t h = 0; h < N; ++h) {
    const int u = R->up_raw[h], d = R->dn_raw[h];
    if (u >= 0 && R->dn_raw[u] == (int)h) R->up[h] = u;
    if (d >= 0 && R->up_raw[d] == (int)h) R->dn[h] = d;
  }
  // start hits: an up link, no down link, and a chain of at least 3 hits
  R->starts.clear();
  for (size_t h = 0; h < N; ++h) {
    const int u = R->up[h];
    if (u >= 0 && R->dn[h] < 0 && R->up[u] >= 0) R->starts.push_back((int)h);
  }
}

// ---------------------------------------------------------------- tracklets
// Best hit of a row for the predicted state: smallest chi2 <= 16 (ties: smaller
// original id).  The search box covers max(0.5 cm, 4 sigma) around the prediction;
// chi2 <= 16 implies the hit lies inside it, so the box does not change the result.
int pick(const Ctx& c, int item, int r, const double* p, double C[5][5], double* chi2_out) {
  const double S00 = C[0][0] + c.vy, S11 = C[1][1] + c.vz;
  const double wy = std::max(WIN_MIN, 4.0 * std::sqrt(S00));
  const double wz = std::max(WIN_MIN, 4.0 * std::sqrt(S11));
  const int64_t ylo = (int64_t)std::floor((p[0] - wy) * QSCALE) - 2, yhi = (int64_t)std::ceil((p[0] + wy) * QSCALE) + 2;
  const int64_t zlo = (int64_t)std::floor((p[1] - wz) * QSCALE) - 2, zhi = (int64_t)std::ceil((p[1] + wz) * QSCALE) + 2;
  int best = -1;
  double bchi = 0;
  visit_box(c, item, r, ylo, yhi, zlo, zhi, [&](int h) {
    const double x2 = chi2_of(p, C, c.hy(h), c.hz(h), c.vy, c.vz);
    if (!(x2 <= CHI2_CUT)) return;
    if (best < 0 || x2 < bchi || (x2 == bchi && c.R->id[h] < c.R->id[best])) {
      best = h;
      bchi = x2;
    }
  });
  *chi2_out = bchi;
  return best;
}

int row_of_pos(const orc_result* R, int item, int pos) {
  // rows of an item are contiguous in sorted order
  for (int r = 0; r < R->n_rows; ++r) {
    const Row& rw = R->rows[(size_t)item * R->n_rows + r];
    if (pos >= rw.pos0 && pos < rw.pos0 + rw.n) return r;
  }
  return -1;
}

// One tracklet from a start hit:
//  (i)   initial state from the first, middle and last chain hits, Kalman fit
//        along the chain (chain hits are accepted without a chi2 test);
//  (ii)  extension to outer rows: predict, take the best hit with chi2 <= 16,
//        stop after 5 consecutive misses;
//  (iii) a refit from the outermost hit towards the inner rows, with the
//        outer direction and curvature as starting values and their variances
//        inflated 100-fold (at most C0), re-picking hits as in (ii).
// Why an inflated prior and not C0: the refit re-picks its hits, and from C0
// its first rows are unconstrained (a +-4 cm window around a direction known to
// 1 rad), so where the track's own hit is missing near its outer end the refit
// takes a neighbour's hit and follows it.  With the outward variances x F the
// refit re-uses 1/F of the outward information; F = 100 is where the
// efficiency stops rising (full TPC event: 97.0% from C0, 97.6% at F = 1e4,
// 98.0% at 1e3, 98.25% at 100, 98.3% at 10 and 1), and on short low-pT tracks
// its pulls and chi2/ndf equal those of the fresh fit, while F = 1 makes them
// 1.2-1.7 wide.
// Pieces of one track that start from different chain heads reach the same
// outermost hit in (ii) and would refit the same hits in (iii): only the
// tracklet with the smallest id among those sharing an outermost hit runs
// (iii); the others are dropped.
// The tracklet is the set of hits of (iii); its parameters are those at the
// innermost hit.  Guards end a pass: |sinphi| >= sin 70 deg, |y| > x tan(half
// angle) (the track leaves the sector), an invalid propagation.  A non-finite or
// non-positive covariance diagonal drops the tracklet.
struct Outward {
  bool ok = false;
  int out_hit = -1, out_row = 0;
  double out_p[5] = {0, 0, 0, 0, 0}, out_var[3] = {0, 0, 0};
};

void outward(Ctx& c, int start, Tracklet& T, Outward& O) {
  orc_result* R = c.R;
  const int item = R->item_of_pos[start];
  T.item = item;
  std::vector<int> chain;
  for (int h = start; h >= 0; h = R->up[h]) chain.push_back(h);
  std::vector<int> chain_row(chain.size());
  for (size_t i = 0; i < chain.size(); ++i) chain_row[i] = row_of_pos(R, item, chain[i]);
  auto X = [&](int r) { return R->row_x[r]; };
  // (i) initial state: the circle through the first, middle and last chain hits
  // gives the curvature; the direction is the circle's tangent at the first hit
  // (chord direction plus half the turning angle); tan(lambda) = dz / arc length.
  const size_t L = chain.size();
  const double x1 = X(chain_row[0]), y1 = c.hy(chain[0]), z1 = c.hz(chain[0]);
  const double x2 = X(chain_row[L / 2]), y2 = c.hy(chain[L / 2]);
  const double x3 = X(chain_row[L - 1]), y3 = c.hy(chain[L - 1]), z3 = c.hz(chain[L - 1]);
  const double dx13 = x3 - x1, dy13 = y3 - y1;
  const double d13 = std::sqrt(dx13 * dx13 + dy13 * dy13);
  const double d12 = std::hypot(x2 - x1, y2 - y1), d23 = std::hypot(x3 - x2, y3 - y2);
  const double cross = (x2 - x1) * (y3 - y1) - (y2 - y1) * (x3 - x1);
  const double kB = KB_PER_TESLA * c.bz;
  const double kappa = -2.0 * cross / (d12 * d23 * d13);  // clockwise turn = positive
  const double u = std::min(1.0, std::max(-1.0, 0.5 * kappa * d13));
  const double phi1 = std::atan2(dy13, dx13) + std::asin(u);
  const double arc = d13 * asin_over_u(u);
  double p[5] = {y1, z1, std::sin(phi1), (z3 - z1) / arc, kappa / kB};
  double C[5][5];
  set_c0(C, c.vy, c.vz);
  double x = x1;
  int out_hit = chain[0], out_row = chain_row[0];
  double out_p[5], out_var[3] = {C[2][2], C[3][3], C[4][4]};
  std::memcpy(out_p, p, sizeof(p));
  bool alive = true;
  for (size_t i = 1; i < chain.size(); ++i) {
    const int r = chain_row[i];
    if (!kf_propagate(p, C, x, X(r), c.bz)) { alive = false; break; }
    x = X(r);
    if (!(std::fabs(p[2]) < SIN_MAX) || std::fabs(p[0]) > x * c.tanh_) { alive = false; break; }
    update(p, C, c.hy(chain[i]), c.hz(chain[i]), c.vy, c.vz);
    if (!cov_ok(C)) { T.valid = false; O.ok = false; return; }
    out_hit = chain[i];
    out_row = r;
    std::memcpy(out_p, p, sizeof(p));
    out_var[0] = C[2][2];
    out_var[1] = C[3][3];
    out_var[2] = C[4][4];
  }
  // (ii) extension outwards
  if (alive) {
    int misses = 0;
    for (int r = out_row + 1; r < R->n_rows && misses < MAX_MISS; ++r) {
      if (!kf_propagate(p, C, x, X(r), c.bz)) break;
      x = X(r);
      if (!(std::fabs(p[2]) < SIN_MAX) || std::fabs(p[0]) > x * c.tanh_) break;
      double x2v;
      const int h = pick(c, item, r, p, C, &x2v);
      if (h < 0) { ++misses; continue; }
      update(p, C, c.hy(h), c.hz(h), c.vy, c.vz);
      if (!cov_ok(C)) { T.valid = false; O.ok = false; return; }
      misses = 0;
      out_hit = h;
      out_row = r;
      std::memcpy(out_p, p, sizeof(p));
      out_var[0] = C[2][2];
      out_var[1] = C[3][3];
      out_var[2] = C[4][4];
    }
  }
  O.ok = true;
  O.out_hit = out_hit;
  O.out_row = out_row;
  std::memcpy(O.out_p, out_p, sizeof(out_p));
  std::memcpy(O.out_var, out_var, sizeof(out_var));
}

void inward(Ctx& c, Tracklet& T, const Outward& O) {
  orc_result* R = c.R;
  const int item = T.item;
  auto X = [&](int r) { return R->row_x[r]; };
  const int out_hit = O.out_hit, out_row = O.out_row;
  const double* out_p = O.out_p;
  const double* out_var = O.out_var;
  double C[5][5];
  // (iii) refit inwards from the outermost hit: its measured y, z; the outward
  // direction and curvature with their variances inflated 100-fold (at most the
  // initial ones), so that the refit is well conditioned and the outward fit
  // enters with 1% of its weight.
  double q[5] = {c.hy(out_hit), c.hz(out_hit), out_p[2], out_p[3], out_p[4]};
  set_c0(C, c.vy, c.vz);
  C[2][2] = std::min(C0_DIAG_ANGLE, INFLATE * out_var[0]);
  C[3][3] = std::min(C0_DIAG_ANGLE, INFLATE * out_var[1]);
  C[4][4] = std::min(C0_DIAG_QPT, INFLATE * out_var[2]);
  double x = X(out_row);
  T.hits.assign(1, out_hit);
  T.chi2 = 0.0;
  double in_p[5], in_C[5][5], in_x = x;
  std::memcpy(in_p, q, sizeof(q));
  std::memcpy(in_C, C, sizeof(C));
  int misses = 0;
  for (int r = out_row - 1; r >= 0 && misses < MAX_MISS; --r) {
    if (!kf_propagate(q, C, x, X(r), c.bz)) break;
    x = X(r);
    if (!(std::fabs(q[2]) < SIN_MAX) || std::fabs(q[0]) > x * c.tanh_) break;
    double x2v;
    const int h = pick(c, item, r, q, C, &x2v);
    if (h < 0) { ++misses; continue; }
    T.chi2 += update(q, C, c.hy(h), c.hz(h), c.vy, c.vz);
    if (!cov_ok(C)) { T.valid = false; return; }
    misses = 0;
    T.hits.push_back(h);
    std::memcpy(in_p, q, sizeof(q));
    std::memcpy(in_C, C, sizeof(C));
    in_x = x;
  }
  T.n = (int)T.hits.size();
  T.valid = T.n >= MIN_HITS;
  std::memcpy(T.p, in_p, sizeof(in_p));
  std::memcpy(T.C, in_C, sizeof(in_C));
  T.x_ref = in_x;
}

// ---------------------------------------------------------------- selection
// Each hit goes to the tracklet with the largest key (n_hits, then smaller id);
// a tracklet keeps the hits it owns and becomes a track if it owns >= 10.
void selection(orc_result* R, const int32_t* item_core) {
  const size_t N = R->qy.size();
  std::vector<uint64_t> owner(N, 0);
  auto key = [](const Tracklet& t) {
    return ((uint64_t)t.n << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)t.local_id);
  };
  for (const Tracklet& t : R->tracklets) {
    if (!t.valid) continue;
    for (int h : t.hits) owner[h] = std::max(owner[h], key(t));
  }
  for (size_t ti = 0; ti < R->tracklets.size(); ++ti) {
    const Tracklet& t = R->tracklets[ti];
    if (!t.valid) continue;
    std::vector<int> own;
    for (int k = (int)t.hits.size() - 1; k >= 0; --k)  // ascending rows
      if (owner[t.hits[k]] == key(t)) own.push_back(t.hits[k]);
    if ((int)own.size() < MIN_HITS) continue;
    if (item_core) {  // time-frame slices: report only tracks whose innermost hit is in the core
      const int zin = R->qz[t.hits.back()];
      if (zin < item_core[2 * t.item] || zin >= item_core[2 * t.item + 1]) continue;
    }
    Track tr;
    tr.item = t.item;
    tr.tracklet = t.local_id;
    tr.first = (int)R->track_ids.size();
    tr.count = (int)own.size();
    tr.x_ref = t.x_ref;
    std::memcpy(tr.p, t.p, sizeof(tr.p));
    std::memcpy(tr.C, t.C, sizeof(tr.C));
    tr.chi2 = t.chi2;
    tr.ndf = 2 * t.n - 5;
    for (int h : own) R->track_ids.push_back(R->id[h]);
    R->tracks.push_back(tr);
  }
}

}  // namespace

extern "C" int orc_run(const orc_config* cfg, const float* x, const float* y, const float* z, const int32_t* row,
                       uint64_t n, const uint64_t* item_off, uint32_t n_items, const int32_t* item_core,
                       orc_result** out) {
  *out = nullptr;
  if (cfg->n_rows < 3 || n_items == 0 || item_off[0] != 0 || item_off[n_items] != n) return 1;
  for (uint32_t i = 0; i < n_items; ++i)
    if (item_off[i + 1] < item_off[i]) return 1;
  std::vector<int> qy(n), qz(n);
  for (uint64_t i = 0; i < n; ++i) {
    if (row[i] < 0 || row[i] >= cfg->n_rows) return 7;
    if (!std::isfinite(x[i]) || !std::isfinite(y[i]) || !std::isfinite(z[i])) return 7;
    if (std::fabs(y[i]) > 1e6f || std::fabs(z[i]) > 1e6f) return 7;
    qy[i] = (int)std::nearbyint((double)y[i] * QSCALE);  // exact scale, round half to even
    qz[i] = (int)std::nearbyint((double)z[i] * QSCALE);
  }
  orc_result* R = new orc_result();
  R->cfg = *cfg;
  R->n_rows = cfg->n_rows;
  R->n_items = n_items;
  R->item_off.assign(item_off, item_off + n_items + 1);
  R->row_x.resize(cfg->n_rows);
  R->row_qx.resize(cfg->n_rows);
  for (int r = 0; r < cfg->n_rows; ++r) {
    const double xr = cfg->x_min + r * ((cfg->x_max - cfg->x_min) / (cfg->n_rows - 1));
    R->row_qx[r] = (int)std::nearbyint(xr * QSCALE);
    R->row_x[r] = R->row_qx[r] / QSCALE;
  }
  binning(R, qy, qz, row);
  neighbours(R);
  Ctx c{R, std::tan(cfg->half_angle_deg * M_PI / 180.0), cfg->sigma_y * cfg->sigma_y, cfg->sigma_z * cfg->sigma_z,
        cfg->bz_tesla};
  R->tracklets.resize(R->starts.size());
  std::vector<Outward> O(R->starts.size());
  std::vector<int> local(n_items, 0);
  for (size_t t = 0; t < R->starts.size(); ++t) {
    Tracklet& T = R->tracklets[t];
    T.item = R->item_of_pos[R->starts[t]];
    T.local_id = local[T.item]++;
    outward(c, R->starts[t], T, O[t]);
  }
  // one inward refit per outermost hit: the smallest tracklet id reaching it
  std::vector<int> first_at(R->qy.size(), -1);
  for (size_t t = 0; t < O.size(); ++t)
    if (O[t].ok && first_at[O[t].out_hit] < 0) first_at[O[t].out_hit] = (int)t;
  for (size_t t = 0; t < O.size(); ++t) {
    Tracklet& T = R->tracklets[t];
    if (O[t].ok && first_at[O[t].out_hit] == (int)t) {
      inward(c, T, O[t]);
    } else {
      T.valid = false;
      T.n = 0;
    }
  }
  selection(R, item_core);
  *out = R;
  return 0;
}

extern "C" void orc_free(orc_result* r) { delete r; }

namespace {
template <class T>
int64_t put(const std::vector<T>& v, void* buf, int64_t cap) {
  if (buf) std::memcpy(buf, v.data(), sizeof(T) * (size_t)std::min<int64_t>(cap, (int64_t)v.size()));
  return (int64_t)v.size();
}
}  // namespace

extern "C" int64_t orc_get(const orc_result* R, const char* which, void* buf, int64_t cap) {
  const std::string w(which);
  const size_t N = R->qy.size();
  if (w == "sorted_qy") return put(R->qy, buf, cap);
  if (w == "sorted_qz") return put(R->qz, buf, cap);
  if (w == "sorted_id") return put(R->id, buf, cap);
  if (w == "rows") {
    std::vector<int> v;
    for (const Row& r : R->rows) {
      int e[7] = {r.pos0, r.n, r.ymin, r.zmin, r.shift, r.ny, r.nz};
      v.insert(v.end(), e, e + 7);
    }
    return put(v, buf, cap);
  }
  if (w == "first") {
    std::vector<int> v;
    for (const Row& r : R->rows)
      for (int f : r.first) v.push_back(f - r.pos0);
    return put(v, buf, cap);
  }
  if (w == "up_raw" || w == "dn_raw" || w == "up" || w == "dn") {
    const std::vector<int>& L = w == "up_raw" ? R->up_raw : w == "dn_raw" ? R->dn_raw : w == "up" ? R->up : R->dn;
    std::vector<int> v(N, -1);
    for (size_t p = 0; p < N; ++p) v[R->id[p]] = L[p] >= 0 ? R->id[L[p]] : -1;
    return put(v, buf, cap);
  }
  if (w == "starts") {
    std::vector<int> v;
    for (int s : R->starts) v.push_back(R->id[s]);
    return put(v, buf, cap);
  }
  if (w == "trk_f") {
    std::vector<double> v;
    for (const Track& t : R->tracks) {
      v.push_back(t.x_ref);
      for (int i = 0; i < 5; ++i) v.push_back(t.p[i]);
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) v.push_back(t.C[i][j]);
      v.push_back(t.chi2);
      v.push_back(t.ndf);
      v.push_back(t.item);
    }
    return put(v, buf, cap);
  }
  if (w == "trk_i") {
    std::vector<int64_t> v;
    for (const Track& t : R->tracks) {
      v.push_back(t.item);
      v.push_back(t.first);
      v.push_back(t.count);
      v.push_back(t.tracklet);
    }
    return put(v, buf, cap);
  }
  if (w == "trk_ids") return put(R->track_ids, buf, cap);
  if (w == "tl_n") {
    std::vector<int> v;
    for (const Tracklet& t : R->tracklets) v.push_back(t.valid ? t.n : 0);
    return put(v, buf, cap);
  }
  if (w == "tl_meta") {
    std::vector<int> v;
    for (const Tracklet& t : R->tracklets) {
      v.push_back(t.item);
      v.push_back(t.local_id);
    }
    return put(v, buf, cap);
  }
  if (w == "tl_hits") {
    std::vector<int> v;
    for (const Tracklet& t : R->tracklets)
      if (t.valid)
        for (int h : t.hits) v.push_back(R->id[h]);
    return put(v, buf, cap);
  }
  return -1;
}

extern "C" int orc_propagate(const double* p_in, double x1, double x2, double bz, double* p_out, double* F) {
  double FF[5][5];
  if (!propagate(p_in, x1, x2, bz, p_out, FF)) return 0;
  if (F)
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) F[i * 5 + j] = FF[i][j];
  return 1;
}

extern "C" int orc_fit_hits(int n, const double* x, const double* y, const double* z, const double* p0,
                            const double* C0, double sy, double sz, double bz, double* p_out, double* C_out,
                            double* chi2_out) {
  double p[5], C[5][5];
  std::memcpy(p, p0, sizeof(p));
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) C[i][j] = C0[i * 5 + j];
  double chi2 = 0.0, xc = x[0];
  for (int i = 0; i < n; ++i) {
    if (x[i] != xc) {
      if (!kf_propagate(p, C, xc, x[i], bz)) return 0;
      xc = x[i];
    }
    chi2 += update(p, C, y[i], z[i], sy * sy, sz * sz);
  }
  std::memcpy(p_out, p, sizeof(p));
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) C_out[i * 5 + j] = C[i][j];
  *chi2_out = chi2;
  return 1;
}

extern "C" double orc_chi2(const double* p, const double* C, double my, double mz, double vy, double vz) {
  double CC[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) CC[i][j] = C[i * 5 + j];
  return chi2_of(p, CC, my, mz, vy, vz);
}
