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

#ifdef __cplusplus
}
#endif
#endif /* TPC_REDUCE_H */
