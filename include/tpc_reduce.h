/*
 * tpc_reduce.h -- data-reduction calls of libtpc.so (arXiv:1910.12214, Sec. 4,
 * "TPC Data Reduction").  They share the context, status codes and conventions
 * of tpc.h: every call returns a tpc_status and never aborts; device work runs
 * on the context's stream.
 */
#ifndef TPC_REDUCE_H
#define TPC_REDUCE_H

#include "tpc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Cluster codec (Sec. 4, step 2) -------------------------------------
 *
 * Converts cluster properties from the reconstruction's floating-point format
 * to integers carrying only the precision the detector resolves.  The paper
 * fixes the dynamic precision of cluster size and charge: in the integer
 * representation every bit more than n places after the leading one is
 * cleared, with rounding, n = 3 for sizes and n = 4 for charges.  Field units
 * and widths are this library's choice (the paper gives none):
 *
 *   field     input        code                      step
 *   y         float  [cm]  int16, nearest (ties even) 2^-6 cm, saturated
 *   z         float  [cm]  int32, nearest (ties even) 2^-6 cm, saturated
 *   row       int32        uint8                      pad row; 0 if out of range
 *   q_tot     float [ADC]  uint16, nearest (ties even) 1 ADC count, saturated,
 *   q_max     float [ADC]  uint16                      then n = 4 dynamic precision
 *   sigma_y   float  [cm]  uint8, nearest (ties even) 2^-7 cm, saturated,
 *   sigma_z   float  [cm]  uint8                      then n = 3 dynamic precision
 *
 * Dynamic precision rounds to the nearest value with n bits after its leading
 * one (ties upward); a carry out of the field gives the largest such value
 * that fits (0xF800 for charges, 0xF0 for sizes).  Negative charges and sizes
 * code as 0; NaN codes as 0 in every field.
 *
 * The decoded value of a code is code x step. */
#define TPC_CODE_POS_STEP_CM (1.0 / 64.0)
#define TPC_CODE_SIZE_STEP_CM (1.0 / 128.0)
#define TPC_CODE_CHARGE_BITS 4 /* bits kept after the leading one */
#define TPC_CODE_SIZE_BITS 3

/* n clusters in SoA form.  Arrays of n values each, all host or all device
 * pointers (see on_device below). */
typedef struct {
  const float* y;
  const float* z;
  const int32_t* row;
  const float* q_tot;
  const float* q_max;
  const float* sigma_y;
  const float* sigma_z;
  uint64_t n;
} tpc_cluster_props;

/* Output codes, n values per array, owned by the caller. */
typedef struct {
  int16_t* y;
  int32_t* z;
  uint8_t* row;
  uint16_t* q_tot;
  uint16_t* q_max;
  uint8_t* sigma_y;
  uint8_t* sigma_z;
} tpc_cluster_codes;

/* Encodes in->n clusters into *out.
 *  on_device = 0: every pointer is a host pointer; the call copies the
 *    properties to the device (staging buffers kept by the context), encodes,
 *    copies the codes back and waits.
 *  on_device = 1: every pointer is a device pointer on the context's device;
 *    the work is enqueued on the context's stream.  With n_bad == NULL the call
 *    returns at once and bad clusters are coded but not reported; otherwise it
 *    waits for the stream.
 * A cluster is bad if its row is outside [0, n_rows) of the context or a value
 * is not finite; it is coded by the rules above all the same.  *n_bad
 * (nullable) receives their number and the call returns TPC_ERR_BAD_INPUT when
 * it is not zero.  n = 0 is valid (nothing happens).  A NULL array with n > 0
 * gives TPC_ERR_INVALID_ARG.  Device arrays aligned to 16 bytes (inputs, z)
 * and 8 bytes (y, charges) take a vectorised path; other alignments are valid
 * and slower. */
tpc_status tpc_encode_clusters(tpc_ctx* ctx, const tpc_cluster_props* in, const tpc_cluster_codes* out, int on_device,
                               uint64_t* n_bad);

/* ---- Cluster association, protection and removal (Sec. 4) ---------------
 *
 * The paper's removal rules: tracking attaches clusters to tracks, an
 * ambiguous cluster going to the higher-momentum track; clusters within a tube
 * of 1.5 cm around a track are adjacent to it, ambiguity again going to the
 * higher-momentum track; clusters adjacent to the primary leg of a track with
 * pT > 50 MeV/c and a local inclination |phi| < 70 degrees are protected.
 * Strategy B removes every cluster that is not protected; strategy A removes
 * the clusters that are not protected and are attached or adjacent to a track
 * with pT <= 50 MeV/c, to a secondary leg, or to a track with |phi| >= 70.
 *
 * This library's reading of the geometry:
 *  - a cluster's candidates are the tracks whose cluster list holds it and
 *    the tracks of its work item whose tube holds it; it goes to the candidate
 *    with the smallest |q/pT| (ties: the smaller track index);
 *  - tube: in the cluster's pad-row plane, distance <= tube_cm between the
 *    cluster (quantised to 2^-10 cm, as the tracker bins it, after any space-
 *    point correction) and the track's crossing point, on the rows from the
 *    track's innermost to its outermost cluster row that the track reaches
 *    (|sin phi| < 0.9999 there; the tracker's helix model at the context's Bz);
 *  - local inclination: |sin phi| of the winning track at the cluster's row,
 *    compared with fl32(sin(max_incl_deg)); pT > min_pt_gev is decided as
 *    |q/pT| < fl32(1 / min_pt_gev) on the float32 track state.
 */
#define TPC_MASK_ASSOCIATED 1u /* attached or adjacent to a track */
#define TPC_MASK_PROTECTED 2u
#define TPC_MASK_REMOVE_A 4u   /* removed by strategy A */
#define TPC_MASK_REMOVE_B 8u   /* removed by strategy B */

typedef struct {
  float tube_cm;      /* adjacency tube radius (1.5) */
  float min_pt_gev;   /* protection needs pT above this (0.05) */
  float max_incl_deg; /* protection needs |phi| below this (70), in (0, 90] */
} tpc_mask_params;

/* Masks of the clusters loaded by tpc_load_clusters, with the tracker's bins
 * of the last tpc_track() (TPC_ERR_STATE if the batch has not been tracked).
 *  prm: NULL = (1.5, 0.05, 70).
 *  tracks: NULL = the context's own tracks of the last tpc_track(), read on the
 *    device (n_tracks, cluster_ids and n_ids ignored).  Otherwise n_tracks
 *    records whose item, first_cluster, n_clusters, x_ref, y, z, snp, tgl and
 *    qpt are used, with cluster_ids (n_ids entries, indices of the loaded
 *    clusters, innermost first per track).  A track whose item or cluster ids
 *    are out of range is skipped and reported (TPC_ERR_BAD_INPUT).
 *  leg: NULL = every track is a primary leg; else one byte per track, 0 =
 *    primary, other = secondary (with tracks == NULL it must hold the number of
 *    tracks tpc_get_tracks reports, and n_tracks must be that number).
 *  mask: one byte per loaded cluster (TPC_MASK_* bits: 3 = protected, 13 =
 *    removed by A and B, 8 = removed by B only); owner (nullable): the winning
 *    track index per cluster, -1 if none.
 *  on_device = 0: every array argument is a host pointer; the call stages it,
 *    computes, copies the results back and waits.  on_device = 1: device
 *    pointers; the work is enqueued on the context's stream and the call
 *    returns at once (a skipped track is then reported by tpc_sync).
 * The result does not depend on the order of the tracks' work on the GPU. */
tpc_status tpc_cluster_masks(tpc_ctx* ctx, const tpc_mask_params* prm, const tpc_track_t* tracks, uint64_t n_tracks,
                             const uint32_t* cluster_ids, uint64_t n_ids, const uint8_t* leg, int on_device,
                             uint8_t* mask, int32_t* owner);

/* ---- Compression of the clusters (Sec. 4, steps 3 and 4) ----------------
 *
 * The paper's steps: clusters not assigned to tracks are ordered in y and z
 * and stored as differences to the previous cluster; clusters assigned to
 * tracks are stored as residuals to the extrapolated track; an ANS entropy
 * coder compresses the result.  This library's format (one self-contained
 * little-endian blob):
 *  - integer codes of every cluster as tpc_encode_clusters makes them;
 *  - unattached clusters (in no track's cluster list) in the tracker's
 *    canonical order of the pad row (the cells of its y-z grid, y-major, then
 *    the cluster index): per (item, row) their number, then per cluster the
 *    zigzag differences (0, -1, 1, -2 -> 0, 1, 2, 3) of the y and z codes to
 *    the previous unattached cluster of the row (the first one to 0);
 *  - attached clusters track by track, innermost first: the zigzag row
 *    increment (the first to row 0) and the zigzag residuals of the y and z
 *    codes to the track's prediction at that row (the tracker's helix from
 *    the track's float32 state, asin(a)/a by two half-angle steps and a series
 *    to a^8, every operation correctly rounded float32 without fused
 *    multiply-add, rounded to the nearest code; 0 if not finite);
 *  - the charge and size codes, unattached clusters first, then attached;
 *  - 11 symbol streams (row counts, dy, dz, row increments, y and z
 *    residuals, q_tot, q_max, sigma_y, sigma_z, clusters per track), each
 *    split into byte planes (as many as its largest value needs, at least
 *    one), each plane coded by rANS: 32-bit states, 16-bit renormalisation,
 *    frequencies scaled to 4096 (f = max(1, floor(count*4096/total)) for
 *    present bytes; an excess is taken one by one from the largest f,
 *    smallest byte first; a shortfall goes to the largest f), chunks of 8192
 *    symbols coded by 32 interleaved states (symbol i by state i mod 32), a
 *    chunk being its final states (2 words each, low first) followed by the
 *    renormalisation words in decoding order;
 *  - layout: header (u32 magic 0x5A435054, u32 version 1, u32 items, u32
 *    rows, u32 tracks, u32 bits of kB = 0.299792458e-2 * Bz as float32, f64
 *    x of the first and last pad row, u64 unattached, u64 attached); per
 *    stream u64 values, u32 planes, per plane u16 f[256], u32 chunks, u32
 *    words per chunk, u16 words; then per track 7 u32: x_ref, y, z, sinphi,
 *    tanlambda, q/pT (float32 bits) and item.
 * Clusters excluded from the binning (bad row or non-finite position) are
 * not stored. */
typedef struct {
  const float* q_tot;   /* one value per loaded cluster */
  const float* q_max;
  const float* sigma_y;
  const float* sigma_z;
} tpc_cluster_charges;

/* Compresses the clusters loaded by tpc_load_clusters, with the tracker's
 * binning of the last tpc_track() (TPC_ERR_STATE otherwise).
 *  charges: charges and sizes of the loaded clusters.
 *  tracks: NULL = the context's own tracks of the last tpc_track()
 *    (n_tracks, cluster_ids, n_ids ignored); else n_tracks records (item,
 *    first_cluster, n_clusters, x_ref, y, z, snp, tgl, qpt used) with
 *    cluster_ids (indices of loaded clusters, innermost first per track).  A
 *    track out of range (item, cluster id or row) gives TPC_ERR_BAD_INPUT.
 *  keep (nullable): one byte per loaded cluster, 0 = removed (Sec. 4, step 5:
 *    clusters not used for physics analysis are discarded), e.g. from the
 *    TPC_MASK_REMOVE_A or _B bit of tpc_cluster_masks.  A removed cluster is
 *    stored neither as unattached nor in its track; a track keeps its place
 *    with the clusters left (its count may be 0), its row increments referring
 *    to its previous stored cluster.
 *  on_device: 1 = charges, tracks, cluster_ids, keep and out are device
 *    pointers; 0 = host pointers.
 *  out, cap: the caller's buffer; *size receives the blob's size; if cap is
 *    smaller nothing is copied and TPC_ERR_CAPACITY is returned (out may be
 *    NULL with cap 0 to ask for the size).  The call waits for its stream. */
tpc_status tpc_compress(tpc_ctx* ctx, const tpc_cluster_charges* charges, const tpc_track_t* tracks,
                        uint64_t n_tracks, const uint32_t* cluster_ids, uint64_t n_ids, const uint8_t* keep,
                        int on_device, uint8_t* out, uint64_t cap, uint64_t* size);

/* ---- Sector-track merger (Sec. 4: the pieces of one track are found in
 * neighbouring sectors separately and must be merged; the removal of clusters
 * of secondary legs works only if the merging works) ---------------------
 *
 * This library's reading (the paper gives no algorithm):
 *  - sectors: 36, 18 per side (0-17 z >= 0, 18-35 z < 0), sector k = s mod
 *    18 centred at azimuth k * 20 degrees; a track's circle in the global
 *    frame from its state (curvature kappa = 0.299792458e-2 Bz q/pT, centre
 *    (x_ref + sinphi/kappa, y - cosphi/kappa) in its sector frame); tracks
 *    with |q/pT| < 1e-4 c/GeV are not merged;
 *  - candidates: tracks of the items of the same event and side in sectors
 *    k+1 and k-1, same sign of q/pT; compatible if (a) (q/pT_A - q/pT_B)^2 <=
 *    16 (var_A + var_B) (the q/pT variances, cov[14]); (b) the reference point
 *    of one lies on the circle of the better measured one within 1 cm + 3 kB
 *    sqrt(var) L^2, L the chord between the reference points; (c) |d tan
 *    lambda| <= 0.02; (d) the outer reference point's z within 2 cm of the inner
 *    track's z + tan(lambda) arc, arc = c (1 + c^2 / (24 R^2)) from the chord c;
 *  - score = chi2(a)/16 + distance(b)/limit + |d tan lambda|/0.02 + |dz|/2 cm;
 *    per direction the compatible candidate with the smallest score (ties:
 *    smaller index); a link joins two tracks that are each other's best in
 *    opposite directions; a group = the tracks connected by links, labelled by
 *    its smallest track index;
 *  - refit of every group in the global frame: the clusters of its tracks
 *    (the pad row fixes x), the algebraic least-squares circle of x^2 + y^2 +
 *    D x + E y + F on coordinates centred on their mean, then z = z0 +
 *    tan(lambda) s by least squares, s the chord-series arc from the innermost
 *    cluster.  The sums are formed in float-float (48-bit significands) and
 *    solved in FP64: the fitted circle matches an FP64 refit to well below
 *    1e-8 cm along the clusters (the radius of a short, nearly straight group
 *    only to a few 1e-9 relative); the compatibility decisions equal exact
 *    ones except within about 1e-13 of a limit. */

/* Merges the tracks of the loaded, tracked batch, which must carry
 * item_sector and item_event (TPC_ERR_STATE otherwise; one item per (event,
 * sector)).
 *  tracks: NULL = the context's own tracks of the last tpc_track() (n_tracks
 *    must be their number, as tpc_get_tracks reports it; cluster_ids, n_ids
 *    ignored); else n_tracks records sorted by item with their cluster_ids
 *    (n_ids entries).  A track out of range (item, cluster, row) or out of
 *    item order gives TPC_ERR_BAD_INPUT.
 *  link: [n_tracks][2] the linked track in sector k+1 and k-1 (-1 none);
 *  group: [n_tracks] the group's smallest track index;
 *  fit: [n_tracks][7] doubles, at each group's smallest index: circle centre
 *    x, y [cm, global frame], radius [cm], tan(lambda), z0 [cm] at the
 *    innermost cluster, clusters, tracks; zero elsewhere (and for straight
 *    tracks).
 *  leg_partner, leg (both nullable; either one asks for the looper legs):
 *    [n_tracks] the other leg of a looper (-1 none) and 1 for its secondary
 *    leg, else 0.  A helix of radius R < 250 cm can turn inside a sector and
 *    come back inward; the tracker fits the returning leg as a track of
 *    opposite q/pT and tan(lambda) sign on the same circle.  Candidates: both
 *    R < 250 cm, same event and side, opposite signs of q/pT and of
 *    tan(lambda); compatible if (|q/pT_A| - |q/pT_B|)^2 <= 16 (var_A + var_B),
 *    the circle centres lie within 1 cm + 3 kB sqrt(var_A + var_B) R^2 (R the
 *    larger radius) and |tan(lambda)_A + tan(lambda)_B| <= 0.02; score =
 *    chi2/16 + centre distance/limit + |sum|/0.02; mutual best pairs are the
 *    two legs; the one whose reference z is farther from 0 (the vertex of an
 *    event) is the secondary leg (ties: the larger index).  Feed `leg` to
 *    tpc_cluster_masks to let strategy A remove the secondary legs.
 *  on_device: 1 = tracks, cluster_ids and the outputs are device pointers
 *    (the call still waits); 0 = host pointers. */
tpc_status tpc_merge_tracks(tpc_ctx* ctx, const tpc_track_t* tracks, uint64_t n_tracks, const uint32_t* cluster_ids,
                            uint64_t n_ids, int on_device, int32_t* link, int32_t* group, double* fit,
                            int32_t* leg_partner, uint8_t* leg);

/* Looper legs joined into one track (Sec. 4: the tracker finds the legs of a
 * looping track separately, and they are merged into one track; the removal
 * of secondary legs relies on it).  Takes the tracks given to
 * tpc_merge_tracks (tracks = NULL: the context's own) and its outputs link,
 * group, leg_partner and leg (all of the same memory kind as on_device says),
 * and joins the groups of every mutual leg pair into one track:
 *  joined: [n_tracks] the joined track's smallest track index (the group label
 *    for tracks of no pair);
 *  jfit: [n_tracks][7] doubles at each joined track's smallest index: the
 *    refit over the clusters of both legs -- the algebraic circle of the
 *    groups (centre x, y, radius, global frame), then tan(lambda) and z0 of
 *    z = z0 + tan(lambda) s, s = R dtheta the arc turned from the primary
 *    legs' innermost cluster in the particle's sense of rotation (clockwise
 *    for q/pT > 0 of the primary leg with the smallest index), z0 at that
 *    cluster; then clusters and tracks; zero elsewhere.  FP64.
 *  n_joined (host, nullable): the number of joined tracks.
 * A joined track holds at most 16 groups and 96 tracks; a larger one, a group
 * or partner out of range, or a cluster out of range gives TPC_ERR_BAD_INPUT.
 * The call waits for its stream. */
tpc_status tpc_join_loopers(tpc_ctx* ctx, const tpc_track_t* tracks, uint64_t n_tracks, const uint32_t* cluster_ids,
                            uint64_t n_ids, int on_device, const int32_t* link, const int32_t* group,
                            const int32_t* leg_partner, const uint8_t* leg, int32_t* joined, double* jfit,
                            uint64_t* n_joined);

#ifdef __cplusplus
}
#endif
#endif /* TPC_REDUCE_H */
