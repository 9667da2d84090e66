/*
 * FP64 CPU oracle of the TPC sector tracker -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded restatement of the tracker's steps (cellular-
 * automaton track finding followed by a Kalman fit, Sec. 3 of the paper and its
 * Abstract), used only by the tests, the smoke check and the CPU-baseline leg of
 * the benchmark.  It shares no code, header or table with the CUDA library; the
 * constants below are this file's own copy of the documented readings.
 *
 * Parity status per function (see the pins in tests/test_oracle_pins.py):
 *   orc_run binning  : pinned (stable-sort definition, invariants, order independence)
 *   orc_run links    : pinned (brute force over all triples on tiny sectors, straight tracks)
 *   orc_propagate    : pinned (RK4 of the Lorentz force; finite-difference Jacobian)
 *   orc_fit_hits     : pinned (straight-line weighted least squares; noise-free helices)
 *   orc_run tracklets: pinned statistically (chi2/ndf ~ 1, pulls N(0,1)), brute search
 *   orc_run selection: pinned (brute force max-key per hit)
 *   orc_trilinear    : pinned (linear fields exact, node values, exact inverse of the field)
 *   orc_mlp_*        : see mlp_oracle.cpp.
 */
#ifndef TPC_ORACLE_H
#define TPC_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n_rows;            /* pad rows per sector */
  double x_min, x_max;   /* radii of first and last row [cm] */
  double half_angle_deg; /* sector half opening angle */
  double bz_tesla;       /* solenoid field */
  double sigma_y, sigma_z; /* cluster resolution used in the Kalman filter [cm] */
  int brute;             /* 1: search every hit of a row instead of the grid window (pins) */
} orc_config;

typedef struct orc_result orc_result;

/* Runs every step on clusters grouped by item (CSR item_off, n_items).
 * item_core (nullable): [n_items][2] slice core [lo,hi) in z quanta.
 * Returns 0 on success, 7 (bad input) if a row is out of range or a value is not finite. */
int orc_run(const orc_config* cfg, const float* x, const float* y, const float* z, const int32_t* row,
            uint64_t n, const uint64_t* item_off, uint32_t n_items, const int32_t* item_core,
            orc_result** out);
void orc_free(orc_result* r);

/* Array access: which = one of the names below; copies up to cap elements, returns the count.
 *   "sorted_qy","sorted_qz","sorted_id"   int32 [n]
 *   "rows"    int32 [n_items*n_rows*7]: pos0,n,ymin,zmin,shift,ny,nz
 *   "first"   int32 concatenated per (item,row): nbins+1 entries relative to pos0
 *   "up_raw","dn_raw","up","dn"  int32 [n] indexed by ORIGINAL id, value = original id or -1
 *   "starts"  int32 original ids of start hits in canonical order
 *   "trk_f"   float64 [n_trk*24]: x_ref,y,z,snp,tgl,qpt,cov[15],chi2,ndf,item
 *   "trk_i"   int64 [n_trk*4]: item, first_cluster, n_clusters, tracklet id (item-local)
 *   "trk_ids" int32 cluster ids (original) of all tracks, concatenated
 *   "tl_n"    int32 [n_tracklets] hits per tracklet (downward pass), 0 = dropped
 *   "tl_meta" int32 [n_tracklets*2]: item, item-local tracklet id
 *   "tl_hits" int32 concatenated original ids of every tracklet (row-descending)
 */
int64_t orc_get(const orc_result* r, const char* which, void* buf, int64_t cap);

/* Helix step of the state (y,z,sinphi,tanlambda,q/pT) from x1 to x2 at field bz.
 * F (nullable) receives the 5x5 Jacobian d(out)/d(in), row-major. Returns 1 if valid. */
int orc_propagate(const double* p_in, double x1, double x2, double bz_tesla, double* p_out, double* F);

/* Kalman filter over given measurements: prior p0,C0 (row-major 5x5) at x[0];
 * for each i: propagate to x[i] and update with (y[i], z[i]).  Returns 1 if valid. */
int orc_fit_hits(int n, const double* x, const double* y, const double* z, const double* p0,
                 const double* C0, double sigma_y, double sigma_z, double bz_tesla,
                 double* p_out, double* C_out, double* chi2_out);

/* Trilinear read of per-sector correction grids (corr_oracle.cpp): grid float32
 * [S][nx][ny][nz][3] over (x, v = y / (x tan_half), z), bounds [S][6]; returns
 * the (dy, dz) components (the pad row fixes x). */
void orc_trilinear(const float* grid, const float* bounds, int nx, int ny, int nz, double tan_half, int n,
                   const int32_t* sector, const double* x, const double* y, const double* z, double* out_dy,
                   double* out_dz);

/* chi2 of measurement (my,mz) against state p with covariance C (row-major 5x5)
 * and measurement variances vy, vz: the hit-selection criterion. */
double orc_chi2(const double* p, const double* C, double my, double mz, double vy, double vz);

#ifdef __cplusplus
}
#endif
#endif
