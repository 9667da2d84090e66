/*
 * tpc.h -- C ABI of libtpc.so, a B300-native (sm_103a) TPC sector tracker.
 *
 * The library performs the hot path of the TPC reconstruction described in
 * D. Rohr, "Global Track Reconstruction and Data Compression Strategy in ALICE
 * for LHC Run 3" (arXiv:1910.12214): cellular-automaton track finding followed
 * by a Kalman fit (Sec. 3, derived from the Run 2 HLT tracker), under continuous
 * read-out with no a-priori vertex (Abstract).  Clusters produced by the cluster
 * finder go in (Sec. 4, step 1); tracks and their cluster attachment come out
 * (Sec. 4: the compression steps consume the cluster-to-track attachment, and an
 * ambiguous cluster is given to one track only).
 *
 * Conventions
 *  - Every call returns a tpc_status; the library never aborts or throws.
 *  - A failed call leaves the context usable, except TPC_ERR_CUDA after a
 *    sticky CUDA context error.
 *  - Units: cm, GeV/c, Tesla.  Cluster ids in the output are the caller's
 *    original input indices (0-based, over the whole tpc_clusters batch).
 *  - One context per host thread; a context is not thread-safe.
 *  - Device work runs on the context's stream; tpc_track() is asynchronous and
 *    errors detected on the device (bad input values, capacity) are returned by
 *    the next tpc_get_tracks() or tpc_sync().
 */
#ifndef TPC_H
#define TPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tpc_ctx tpc_ctx;

typedef enum {
  TPC_OK = 0,
  TPC_ERR_INVALID_ARG = 1, /* a NULL pointer, an out-of-range size or an inconsistent CSR */
  TPC_ERR_STATE = 2,       /* call out of order (e.g. tpc_track before tpc_load_clusters) */
  TPC_ERR_CUDA = 3,        /* a CUDA runtime error; see tpc_last_error() */
  TPC_ERR_OOM = 4,         /* the allocator returned NULL */
  TPC_ERR_CAPACITY = 5,    /* an output buffer or an internal limit is too small */
  TPC_ERR_TIMEOUT = 6,     /* a bounded device wait gave up */
  TPC_ERR_BAD_INPUT = 7    /* a cluster has a row out of range or a non-finite coordinate */
} tpc_status;

typedef enum { TPC_MODE_PLAIN = 0, TPC_MODE_BATCHED = 1 } tpc_mode;
typedef enum { TPC_CORR_NONE = 0, TPC_CORR_GRID = 1, TPC_CORR_MLP = 2 } tpc_corr;

/* Optional device-memory allocator (e.g. a framework's caching allocator).
 * alloc(bytes, user) returns a device pointer aligned to >= 256 bytes or NULL;
 * free(ptr, user) releases it.  NULL allocator = cudaMallocAsync on the stream. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} tpc_allocator;

typedef struct {
  int device;                 /* CUDA device ordinal */
  void* stream;               /* cudaStream_t to run on; NULL = a library-owned stream */
  float bz_tesla;             /* solenoid field, e.g. 0.5 */
  int n_rows;                 /* pad rows per sector, 3..256 (152 for the ALICE TPC) */
  float row_x_min, row_x_max; /* radii of the first and last pad row [cm] (85, 246) */
  float sector_half_angle_deg;/* sector half opening angle (10) */
  float sigma_y, sigma_z;     /* cluster resolution used by the Kalman filter [cm] (0.1) */
  tpc_mode mode;              /* PLAIN: one launch per step over all items; BATCHED: the same
                                 stages, the tracklet passes as persistent kernels whose lanes
                                 take tracklets from work queues (outward by chain length,
                                 inward by outermost row) as they finish one; faster on large
                                 batches, slower on one event (identical results) */
  tpc_corr correction;        /* space-point correction applied by tpc_track (see tpc_set_correction) */
  uint64_t max_clusters;      /* initial reservation (0 = grow on demand) */
  uint32_t max_items;         /* initial reservation (0 = grow on demand) */
  const tpc_allocator* allocator; /* NULL = cudaMallocAsync */
  int profile;                /* 1 = record per-step CUDA events for tpc_stage_times */
  const char* tune_cache_path;/* nullable: text file of autotuner results, read and updated by
                                 tpc_autotune (the string is copied at tpc_init) */
} tpc_config;

/* Cluster batch, SoA, grouped by work item (event, sector[, time slice]).
 * Item k owns clusters [item_off[k], item_off[k+1]); item_off[0] = 0 and
 * item_off[n_items] = n.  An empty batch has n = 0 (n_items may be 0).  x is the pad-row radius (only checked to be finite: the
 * row index defines the position along x); y, z are sector-local [cm]; row is the
 * pad-row index 0..n_rows-1.  x, y, z, row are host pointers (copied during the
 * call) or, with on_device = 1, device pointers borrowed until tpc_track() has
 * completed.  item_off, item_sector, item_event and item_core are host arrays.
 * item_core (nullable) holds [n_items][2] z ranges [lo, hi) in units of 2^-10 cm:
 * a track is reported only if its innermost cluster's z lies in its item's range
 * (time-frame slices with overlap report each track once). */
typedef struct {
  const float* x;
  const float* y;
  const float* z;
  const int32_t* row;
  uint64_t n;
  const uint64_t* item_off;
  uint32_t n_items;
  const uint32_t* item_sector; /* nullable: sector id copied into the tracks */
  const uint32_t* item_event;  /* nullable: event id copied into the tracks */
  const int32_t* item_core;    /* nullable */
  int on_device;
} tpc_clusters;

/* One track: Kalman state at the innermost cluster, x_ref = that pad row's radius
 * (sector-local); (y, z, sinphi, tanlambda, q/pT); cov = lower triangle of the 5x5
 * covariance, row by row ((0,0),(1,0),(1,1),(2,0),...,(4,4)).  The track's cluster
 * ids are cluster_ids[first_cluster .. first_cluster + n_clusters), innermost first. */
typedef struct {
  float x_ref, y, z, snp, tgl, qpt;
  float cov[15];
  float chi2;
  int32_t ndf;
  uint32_t item, sector, event, first_cluster, n_clusters;
} tpc_track_t;

/* Creates a context on cfg->device: one GPU of the reconstruction farm that
 * runs the synchronous TPC processing (Sec. 2).  *out receives the context or
 * NULL; the config is copied. */
tpc_status tpc_init(const tpc_config* cfg, tpc_ctx** out);

/* Loads one batch of clusters from the cluster finder (Sec. 4, first step of
 * the processing chain): items of (event, sector) or, under continuous
 * read-out (Abstract, Sec. 2), time-frame slices.  Copied to the device if
 * on_device = 0; resets the previous output; grows the device buffers if
 * needed. */
tpc_status tpc_load_clusters(tpc_ctx* ctx, const tpc_clusters* cl);

/* Loads a continuous read-out time frame (the paper's Abstract and Sec. 2:
 * 50 kHz continuous read-out with no a-priori vertex, so cluster z carries the
 * drift-time offset of its collision) and cuts it into overlapping slices on
 * the device, each an ordinary item of the loaded batch.  fr: the frame's
 * clusters as in tpc_load_clusters, its items normally the 36 sectors with
 * their whole z axis; item_core must be NULL.  Each item is cut along z into
 * cores [c0 + k core_cm, c0 + (k + 1) core_cm) from c0 = floor(zmin / core_cm)
 * core_cm up to the item's largest z (at most 64 per item); slice k holds every
 * cluster of the item with c0 + k core - overlap <= z < c0 + (k + 1) core +
 * overlap (decided as in FP64), in the frame's order, and reports a track only
 * if its innermost cluster's z lies in the core.  With an overlap longer than a
 * track's z extent slicing does not change the result: the tracks are those of
 * the whole frame.  0 <= overlap_cm <= 3 core_cm.  The output cluster ids of
 * tpc_get_tracks / tpc_device_tracks are frame indices; a track's item is its
 * slice (sector and event from the frame item).  tpc_debug_dump shows the
 * sliced batch; the data-reduction calls (tpc_reduce.h) refuse a frame
 * (TPC_ERR_STATE).  The call waits for its stream (it reads the slice sizes).
 * Errors: TPC_ERR_BAD_INPUT for a non-finite z, TPC_ERR_CAPACITY for more than
 * 64 slices in one item. */
tpc_status tpc_load_frame(tpc_ctx* ctx, const tpc_clusters* fr, float core_cm, float overlap_cm);

/* Runs every step of the tracker on the loaded batch (Sec. 3: cellular-
 * automaton track finding followed by a Kalman fit, derived from the Run 2 HLT
 * tracker): quantisation, per-row grids, neighbour links, mutual cleaning,
 * start hits, Kalman tracklets (segments at |phi| >= 70 deg are not fitted and
 * a numerical failure ends a fit, Sec. 4), shared-cluster resolution (a
 * cluster goes to one track only, Sec. 4) and output compaction.
 * Asynchronous. */
tpc_status tpc_track(tpc_ctx* ctx);

/* Waits for the stream and returns a device-side error if one was flagged. */
tpc_status tpc_sync(tpc_ctx* ctx);

/* Waits for the stream and copies the tracks and their cluster ids (the
 * cluster-to-track attachment the compression steps consume, Sec. 4) to the
 * caller's host buffers.  *n_trk and *n_ids always receive the required sizes;
 * if trk_cap or id_cap is too small nothing is copied and TPC_ERR_CAPACITY is
 * returned.  trk / cluster_ids may be NULL with zero capacity (size query). */
tpc_status tpc_get_tracks(tpc_ctx* ctx, tpc_track_t* trk, uint64_t trk_cap, uint32_t* cluster_ids,
                          uint64_t id_cap, uint64_t* n_trk, uint64_t* n_ids);

/* Device pointers of the last output (valid until the next load), for callers
 * that keep the tracks on the GPU.  Any argument may be NULL. */
tpc_status tpc_device_tracks(tpc_ctx* ctx, const tpc_track_t** trk, const uint32_t** cluster_ids,
                             const uint64_t** d_counts);

/* Per-step device times of the last tpc_track() in microseconds (needs
 * cfg.profile = 1): us[i] for the steps named by tpc_stage_name(i); steps the
 * last run's mode does not have read 0 (both modes: 0..8; 9..10, named
 * "unused_9" and "unused_10", are no longer used and read 0).
 * Entries 11..12 are the two kernels of the last tpc_cluster_masks() call and
 * 13..15 the symbol, rANS and layout phases of the last tpc_compress() call
 * (tpc_reduce.h) since the batch was loaded, else 0.  Entry 16 is the
 * space-point correction (grid or network) of the last tpc_track(), 0 when no
 * correction is on. */
tpc_status tpc_stage_times(tpc_ctx* ctx, float* us, int n, int* n_stages);
const char* tpc_stage_name(int i);

/* Intermediate results of the last tpc_track() in a canonical host layout, for
 * parity tests.  stage: 0 sorted (qy,qz,id) int32 x3 per cluster; 1 row records
 * int32 x7 (pos0,n,ymin,zmin,shift,ny,nz) per (item,row); 2 bin starts relative
 * to pos0, nbins+1 per (item,row); 3..6 raw up, raw down, clean up, clean down
 * links as original ids indexed by original id (-1 = none); 7 start hits
 * (original ids, canonical order); 8 hits per tracklet (0 = dropped);
 * 9 tracklet hit lists (original ids, outermost first); 10 tracklet index
 * (canonical order) of every output track; 11 corrected (y, z) of every
 * input cluster as float32 bit patterns (the input when no correction is on).  Copies up to cap int32
 * values into host_buf and sets *n to the full count. */
tpc_status tpc_debug_dump(tpc_ctx* ctx, int stage, int32_t* host_buf, uint64_t cap, uint64_t* n);

/* Space-point correction by per-sector grids (location-dependent calibration,
 * the paper's Abstract; online calibration, Sec. 3).  grid: host float32
 * [n_sectors][nx][ny][nz][3] of (dx, dy, dz) shifts such that corrected =
 * measured + shift, at nodes spanning (x, v = y / (x tan(half angle)), z) in
 * the measured (distorted) space; bounds: host float32 [n_sectors][6] =
 * (x0, x1, v0, v1, z0, z1).  A cluster is corrected by trilinear interpolation
 * at its pad row's radius with coordinates clamped to the grid; the pad row
 * fixes x, so only dy and dz are applied.  Items use the grid of their
 * item_sector (0 when item_sector is NULL).  The grid is copied and kept until
 * replaced or the context is destroyed. */
tpc_status tpc_set_grid_correction(tpc_ctx* ctx, const float* grid, const float* bounds, uint32_t n_sectors, int nx,
                                   int ny, int nz);

/* Selects the correction applied by tpc_track(): TPC_CORR_NONE, TPC_CORR_GRID
 * (needs tpc_set_grid_correction) or TPC_CORR_MLP (needs a trained or loaded
 * network). */
tpc_status tpc_set_correction(tpc_ctx* ctx, tpc_corr mode);

/* Learned surrogate of the grid correction: per sector a 3 -> 64 -> 64 -> 3
 * network with SiLU activations, BF16 operands and FP32 sums, whose output x
 * 10 cm is the (dx, dy, dz) correction (dy, dz applied; the pad row fixes x).
 * Inputs are the measured (x, v = y / (x tan), z) normalised to [-1, 1]^3 by
 * the grid's bounds.  Parameters per sector (float32, 4611): W1[64][3], b1[64],
 * W2[64][64] (out, in), b2[64], W3[3][64], b3[3].
 *
 * tpc_surrogate_train: trains on samples drawn uniformly in each sector's grid
 * box with targets read from the grid (tpc_set_grid_correction must have been
 * called): MSE, Adam (beta 0.9, 0.999), learning rate lr (0 = 3e-2) with a
 * cosine decay over n_samples / 1024 steps of 1024 samples per sector, Xavier-uniform
 * initial weights; samples and initial weights come from a counter-based
 * generator (splitmix64) keyed by seed.  max_steps > 0 stops after that many
 * steps; a later call with the same seed resumes (a call after the last step
 * starts afresh).  The residual |network - grid| of (dy, dz) in cm over
 * held-out points is returned in *max_resid_cm and *rms_resid_cm (nullable).
 * tpc_surrogate_eval: the same residual over n_points per sector.
 * tpc_surrogate_params / set_params: a sector's FP32 master parameters (n >=
 * 4611 floats).  tpc_surrogate_grad: dL/dparams and the loss of the current
 * parameters on the training batch (seed, step) of `batch` samples (a multiple
 * of 128, at most 1024), without updating anything.  save / load: parameters,
 * Adam state, step and input bounds in a binary checkpoint; resuming a run
 * from a checkpoint gives the same parameters bit for bit. */
tpc_status tpc_surrogate_train(tpc_ctx* ctx, uint64_t n_samples, uint64_t seed, int max_steps, float lr,
                               float* max_resid_cm, float* rms_resid_cm);
tpc_status tpc_surrogate_eval(tpc_ctx* ctx, uint64_t n_points, float* max_resid_cm, float* rms_resid_cm);
tpc_status tpc_surrogate_params(tpc_ctx* ctx, int sector, float* out, int n);
tpc_status tpc_surrogate_set_params(tpc_ctx* ctx, int sector, const float* in, int n);
tpc_status tpc_surrogate_grad(tpc_ctx* ctx, int sector, uint64_t seed, uint64_t step, int batch, float* grad, int n,
                              float* loss);
tpc_status tpc_surrogate_save(tpc_ctx* ctx, const char* path);
tpc_status tpc_surrogate_load(tpc_ctx* ctx, const char* path);

/* Launch shapes of the kernels (no effect on results: every shape gives the
 * same output bit for bit).  tracklet_lanes: lanes that share one tracklet
 * (1, 2, 4, 8, 16 or 32; they split the hit search of every row);
 * tracklet_block: threads per block of the tracklet kernel (32, 64, 96
 * or 128); tracklet_blocks_per_sm: grid = this x SM count; sort_smem: dynamic
 * shared memory [bytes] of the per-row sort (rows that do not fit use global
 * memory); link_rows: pad rows per block of the neighbour kernel (-1 = 8; the
 * block's rows are staged in shared memory when they fit); merge_sort_cap:
 * most tracks of one event and side that tpc_merge_tracks sorts by tan(lambda)
 * in shared memory for its candidate search (1 to 16384; larger sets, or -1
 * for every set, are scanned item by item).  0 keeps a field. */
typedef struct {
  int tracklet_lanes;
  int tracklet_block;
  int tracklet_blocks_per_sm;
  int sort_smem;
  int link_rows;
  int mode;          /* 1 = plain, 2 = batched (persistent tracklet kernels fed by work queues) */
  int batch_lanes;   /* lanes per tracklet in the batched form: 1 (persistent refilling kernels),
                        2 or 4 (queued grid-stride kernels) */
  int use_graph;     /* 1 = launch directly, 2 = capture tpc_track once per load and replay it */
  int merge_sort_cap;
} tpc_tuning;

tpc_status tpc_set_tuning(tpc_ctx* ctx, const tpc_tuning* t);
tpc_status tpc_get_tuning(tpc_ctx* ctx, tpc_tuning* t);

/* Autotuner: runs tpc_track() on the loaded batch for every candidate shape
 * (lane groups x block sizes x shared-memory budgets), times each with CUDA
 * events (median of `iters` runs), keeps the fastest in the context and
 * returns it in *best (nullable) with its time in *best_us (nullable).  The
 * last run leaves the batch tracked with the chosen shape.  With a
 * cfg.tune_cache_path, a result stored for the same GPU, mode and batch shape
 * (clusters, items, rows, correction) is used without a search, and a new
 * search's result is stored. */
tpc_status tpc_autotune(tpc_ctx* ctx, int iters, tpc_tuning* best, float* best_us);
/* The same over the shapes of one mode only (1 = plain, 2 = batched; 0 = both,
 * as tpc_autotune), for comparing the two modes at their best shapes. */
tpc_status tpc_autotune_mode(tpc_ctx* ctx, int iters, int mode, tpc_tuning* best, float* best_us);

/* Binning of ONE sector without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate GPU
 * memory while they run (a real-time loop with a memory budget fixed at start,
 * a plug-in inside a framework that owns all device memory, or code that must
 * avoid cudaMalloc/cudaFree because they synchronise the device).  It needs no
 * context: the caller passes device pointers for the inputs (y, z, row: n
 * values each) and the outputs, and the work runs on `stream` (NULL = legacy
 * default stream) on the current device.  The call waits for its stream before
 * returning (it reads an error word).
 *   sorted:    n x 4 int32: (qy, qz, original index, row) in canonical order
 *              (row, bin, index); qy = rint(y * 1024), qz = rint(z * 1024);
 *   rows_out:  n_rows x 8 int32: (pos0, n, ymin, zmin, shift, ny, nz, bin0);
 *   first_out: 2n + 3 n_rows + 1 int32: first sorted position of every bin,
 *              nbins + 1 entries per row starting at its bin0.
 * The temporary storage lives in one fixed device array per GPU inside the
 * library (16 bytes per cluster, TPC_NOALLOC_MAX_CLUSTERS clusters; held by
 * every GPU that loads the library until the process exits).  Larger inputs
 * are rejected with TPC_ERR_CAPACITY before any GPU work; n_rows must be
 * 1..256.  Every call looks up that array's address in the current context
 * and waits for its stream, so it cannot be called during stream capture.
 * Every call uses the same array and it keeps the previous call's contents; calls
 * that overlap on the GPU (other streams, other host threads) race on it, so
 * run them one after another.  Returns TPC_ERR_BAD_INPUT if a row is out of
 * range or a coordinate is not finite (such clusters are left out). */
#define TPC_NOALLOC_MAX_CLUSTERS 65536
tpc_status tpc_bin_sector_noalloc(const float* y, const float* z, const int32_t* row, uint32_t n, int n_rows,
                                  int32_t* sorted, int32_t* rows_out, int32_t* first_out, void* stream);

/* Frees every device buffer and the context. */
void tpc_destroy(tpc_ctx* ctx);

/* Text of the last error of this context (never NULL). */
const char* tpc_last_error(const tpc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TPC_H */
