// Internal device structures of libtpc (not part of the ABI).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#define TPC_MAX_ROWS 256
#define TPC_MAX_ROW_HITS 8192   // hits per (item,row) grid handled in shared memory
#define TPC_QSCALE 1024.0f      // quanta per cm (Q = 2^-10 cm)

// device error bits (OR-ed into a device word, read on the host)
#define TPC_DERR_BAD_INPUT 1u
#define TPC_DERR_ROW_CAP 2u
#define TPC_DERR_TIMEOUT 4u
#define TPC_DERR_BAD_TRACK 8u  // a track given to tpc_cluster_masks refers to an item or cluster out of range
#define TPC_DERR_CAPACITY 16u  // a time-frame item needs more than TF_KMAX slices

// One (item, pad row) of the binning grid: 32 bytes, one load.
struct RowInfo {
  int pos0;   // first sorted position of the row (absolute)
  int n;      // hits in the row
  int ymin, zmin;
  int shift;  // bin edge = 2^shift quanta
  int ny, nz; // grid dimensions; nbins = ny*nz (0 for an empty row)
  int bin0;   // index of the row's first entry in first[] (nbins+1 entries)
};

// Per tracklet result of the Kalman pass (the hit list lives in a separate
// fixed-stride array of n_rows positions per tracklet).
struct TrackletRec {
  float p[5];   // y, z - z_base*Q, sinphi, tanlambda, q/pT at the innermost hit
  float C[15];  // lower triangle
  float chi2, x_ref;
  int n;        // hits of the inward pass (0 = dropped)
  int z_base;   // z origin of the state in quanta (start hit)
  int z_in;     // z of the innermost hit in quanta
  int item, local;
  int pad;
};

// Result of the outward passes (i)+(ii) of a tracklet, input of the inward
// refit (iii).
constexpr int TPC_MAX_SEGS = 1024;  // segments of the batched inward pass (one per SM)

struct TrackletUp {
  int out_hit;   // outermost hit (sorted position), -1 = dropped
  int out_row;
  float snp, tgl, qpt;
  float v2, v3, v4;  // variances of sinphi, tanlambda, q/pT at the outermost hit
  int z_base, item, local, pad;
};

struct DevParams {
  int n_rows;
  float tan_half;   // tan(sector half angle)
  float vy, vz;     // measurement variances
  float kB;         // curvature per unit q/pT [1/cm]
  int qx[TPC_MAX_ROWS];
  float x[TPC_MAX_ROWS];  // qx * Q
};

// Work table entry for cluster-parallel kernels: a CTA handles clusters
// [begin, end) of one item.
struct Chunk {
  int item;
  int begin;
  int end;
};

struct Buffers {
  DevParams par;  // geometry and filter constants (kernel argument, no global state)
  // inputs (device)
  const float *x, *y, *z;
  const int* row;
  const uint64_t* item_off;   // [I+1]
  const int* item_core;       // [I][2] or null
  const uint32_t* item_sector;
  const uint32_t* item_event;
  const Chunk* chunks;
  int n_chunks;
  int N, I;
  // per cluster temporaries
  int* cl_key;    // item*NR+row or -1
  int2* cl_q;     // quantised (qy,qz)
  // per (item,row)
  int* rs_cnt;    // [I*NR]
  int* rs_min;    // [4][I*NR]: ymin, -ymax, zmin, -zmax
  int* row_fill;  // [I*NR]
  int* rs_big;    // rows too large for the warp sort, then their count [I*NR + 1]
  RowInfo* rows;  // [I*NR]
  // grouped (row-major, unsorted) and sorted hits
  int2* g_q;
  int* g_id;
  int4* s_hit;    // sorted hits: (qy, qz, original id, item*NR+row)
  int* first;     // bins
  // links
  int* up_raw;
  int* dn_raw;
  int* up;
  int* dn;
  int* flags;     // start flags -> scan
  int* start_ex;  // exclusive scan of flags [N+1]
  int* starts;    // [T_cap]
  // tracklets
  int T_cap;
  TrackletRec* tl;
  TrackletUp* tlu;                // [T_cap]
  int* out_owner;                 // smallest tracklet reaching each hit as its outermost [N]
  int* tl_hits;   // [T_cap * NR]
  unsigned long long* hit_key;  // [N]
  unsigned long long* tl_cnt;   // packed (1<<32 | owned) per tracklet
  unsigned long long* tl_ex;    // exclusive scan [T_cap+1]
  // outputs
  void* trk;      // tpc_track_t [T_cap]
  uint32_t* trk_ids;  // [N]
  int* trk_tl;        // tracklet index of every track [T_cap]
  unsigned long long* counts;  // [0] n_trk, [1] n_ids, [2] n_tracklets
  unsigned int* err;
  unsigned long long* scan_tmp;  // block sums
  // batched form: tracklets from work queues
  int* chain_len;                 // hits of every start hit's chain [T_cap]
  int* tl_order;                  // tracklet indices in processing order: shortest chains first
                                  // (outward pass), then highest outermost row first per segment
                                  // (inward pass) [T_cap]
  int* seg_next;                  // inward pass: next unclaimed position of every segment [TPC_MAX_SEGS]
  // space-point correction (applied before binning when enabled)
  const float2* grid;             // per-sector (dy, dz) nodes [S][nx][ny][nz]
  const float* grid_bounds;       // [S][6]: x0, x1, v0, v1, z0, z1 (v = y / (x tan_half))
  int grid_nx, grid_ny, grid_nz, grid_sectors;
  const void* mlp;                // per-sector BF16 networks (tpc_mlp.cu), null = none
  int mlp_sectors;
  float* cy;                      // corrected y, z [N]
  float* cz;
};

#define TPC_N_STAGES 11  // the 9 steps of tpc_track, then two slots no longer used (indices kept stable)
#define TPC_N_REPORTED_STAGES 17  // ... then the two kernels of tpc_cluster_masks, the 3 phases of
                                  // tpc_compress, and the space-point correction of tpc_track

struct LaunchCfg {
  int n_rows;
  int num_sms;
  int sort_smem;  // dynamic shared memory of k_row_sort
  int link_smem;  // unused (kept for the ABI's tuning struct)
  int link_rows;  // rows per CTA of k_links (0 = derived from the batch size)
  int grid_scan;  // blocks of the reduce-then-scan (<= 1024)
  int grid_tl;    // blocks of k_tracklets
  int block_tl;   // threads per block of k_tracklets
  int tl_group;   // lanes per tracklet (1, 2, 4, 8, 16, 32)
  int batch_group;  // lanes per tracklet in the batched form (1, 2, 4)
  int merge_sort_cap;   // tracks of one event and side sorted by the merger (0: none)
};

cudaError_t tpc_configure_kernels(int sort_smem, int link_smem);
cudaError_t tpc_launch_plain(const Buffers& b, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev);
cudaError_t tpc_launch_batched(const Buffers& b, const LaunchCfg& c, cudaStream_t s, cudaEvent_t* ev);
cudaError_t tpc_launch_grid_correction(const Buffers& b, cudaStream_t s);

// Continuous read-out time frames cut into overlapping slices on the device
// (tpc_frame.cu; the host side is tpc_load_frame in tpc_capi.cu).
constexpr int TF_KMAX = 64;     // slices of one frame item
constexpr int TF_WMAX = 4;      // overlap <= (TF_WMAX - 1) cores: a cluster is in at most 2 TF_WMAX - 1 slices
constexpr int TF_CHUNK = 4096;  // frame clusters per block
struct FrameArgs {
  const float *x, *y, *z;     // the frame (device)
  const int* row;
  const Chunk* chunks;        // frame chunks of <= TF_CHUNK clusters, one item each, in item order
  int n_chunks;
  const int* chunk_first;     // [F + 1] first chunk of every item
  int F;                      // frame items
  float core, overlap;        // cm
  int W;                      // candidate slices on each side of the estimate: 1 + ceil(overlap / core)
  int* ext;                   // [F][2] order-preserving integers of min z, max z
  double* c0;                 // [F] start of the first core
  int* nslice;                // [F] slices of the item
  float2* bounds;             // [F][TF_KMAX] extended range [lo, hi) of every slice, FP64-exact as floats
  int* cnt;                   // [n_chunks][TF_KMAX] memberships, then the chunk's base inside each slice
  int* size;                  // [F][TF_KMAX] clusters of every slice
  const int* slice_first;     // [F] index of the item's first slice in the sliced batch
  const uint64_t* slice_off;  // [S + 1] first cluster of every slice in the sliced batch
  float *ox, *oy, *oz;        // the sliced batch (device)
  int* orow;
  int* src;                   // frame index of every sliced cluster
  unsigned int* err;
};
cudaError_t tpc_frame_count(const FrameArgs& a, cudaStream_t s);
cudaError_t tpc_frame_scatter(const FrameArgs& a, cudaStream_t s);
cudaError_t tpc_frame_map_ids(const uint32_t* in, const int* src, uint32_t* out, const unsigned long long* counts,
                              int blocks, cudaStream_t s);
cudaError_t tpc_launch_mlp_correction(const Buffers& b, cudaStream_t s);

// MLP surrogate (tpc_mlp.cu)
size_t tpc_mlp_infer_bytes();
int tpc_mlp_nparams();
int tpc_mlp_stride();
cudaError_t tpc_mlp_init(float* master, float* m, float* v, int S, uint64_t seed, cudaStream_t s);
// training workspace of S sectors (device clock, step counter, staged weights)
size_t tpc_mlp_work_bytes(int S);
// n_steps training steps from step `first` of T (cosine schedule from lr);
// work: device block of tpc_mlp_work_bytes(S)
cudaError_t tpc_mlp_train_steps(void* work, uint64_t first, uint64_t T, float lr, uint64_t n_steps, float* master,
                                float* m, float* v, float* partial, float* loss, const float2* grid, int nx, int ny,
                                int nz, int S, int batch, uint64_t seed, bool graph, cudaStream_t s);
cudaError_t tpc_mlp_grad_only(void* work, const float* master, float* partial, float* loss, const float2* grid,
                              int nx, int ny, int nz, int S, int batch, uint64_t seed, uint64_t step, cudaStream_t s);
cudaError_t tpc_mlp_eval(const float* master, const float2* grid, int nx, int ny, int nz, int S, int nblk,
                         uint64_t seed, float* out, cudaStream_t s);
cudaError_t tpc_mlp_prepare(const float* master, const float* bounds, void* infer, int S, cudaStream_t s);

// Cluster codec (tpc_reduce.cu): float properties -> integer codes.
struct CodecIn {
  const float *y, *z;
  const int* row;
  const float *qt, *qm, *sy, *sz;
};
struct CodecOut {
  int16_t* y;
  int* z;
  uint8_t* row;
  uint16_t *qt, *qm;
  uint8_t *sy, *sz;
};
bool codec_vector_ok(const CodecIn& in, const CodecOut& out);
cudaError_t launch_encode(const CodecIn& in, const CodecOut& out, long long n, int n_rows, unsigned long long* n_bad,
                          int num_sms, cudaStream_t s);

// Cluster association and removal masks (tpc_reduce.cu).
struct MaskArgs {
  const RowInfo* rows;        // the tracker's per-(item, row) grids of the loaded batch
  const int* first;
  const int4* s_hit;          // sorted hits (qy, qz, original id, item*NR+row)
  const int* row;             // input pad row of every cluster
  int N, I;
  const void* trk;            // tpc_track_t records
  const uint32_t* ids;        // cluster ids of the tracks
  const unsigned long long* counts;  // device (n_trk, n_ids) of the context's own output, or null
  long long n_trk, n_ids;     // used when counts is null
  const uint8_t* leg;         // per track, 0 = primary; null = all primary
  unsigned long long* assoc;  // per cluster: best (pT, track) key, 0 = none; zero on entry and on exit
  uint8_t* mask;
  int* owner;                 // nullable
  float tube, max_qpt, max_snp;
  unsigned int* err;          // the batch's error word (TPC_DERR_BAD_TRACK)
};
// ev (nullable): 3 events recorded around the two kernels
cudaError_t launch_masks(const MaskArgs& a, const DevParams& par, int num_sms, cudaStream_t s, cudaEvent_t* ev);

// Cluster compression (tpc_reduce.cu): entropy reduction and rANS coding.
#define TPC_CMP_STREAMS 11
#define TPC_CMP_CHUNK 8192
struct CmpArgs {
  // the loaded, tracked batch
  const RowInfo* rows;
  const int4* s_hit;
  const float *y, *z;
  const int* row;
  int N, I, P;  // clusters, items, sorted positions (= N; positions outside every row's range are unused)
  // charges and sizes
  const float *qt, *qm, *sy, *sz;
  const uint8_t* keep;  // per cluster, 0 = removed (not stored); null = keep all
  // tracks
  const void* trk;
  const uint32_t* ids;
  const unsigned long long* counts;  // own output (n_trk, n_ids) or null
  long long n_trk, n_ids;
  unsigned int* err;
  // work arrays
  uint8_t* attached;     // [N]
  int* kpos;             // [P + 1] exclusive scan of the unattached flags over the sorted positions
  int* unatt_id;         // [N]
  uint8_t* unatt_first;  // [N]
  int* trk_n;            // [n_trk + 1] cluster counts -> exclusive scan
  int4* rec;             // [N] per-cluster codes: (z, y | q_tot << 16, q_max | row << 16, sigma_y | sigma_z << 8)
  unsigned long long* val[TPC_CMP_STREAMS];  // symbol streams
  unsigned long long* vmax;                  // [TPC_CMP_STREAMS]
  unsigned long long* hist;                  // [TPC_CMP_STREAMS][8][256]
  int* scan_tmp;                             // block partials
};
cudaError_t cmp_symbols(const CmpArgs& a, const DevParams& par, int num_sms, cudaStream_t s);
// histograms of byte planes 2.. of the streams that need them (stream_planes: host array)
cudaError_t cmp_hist_high(const CmpArgs& a, const DevParams& par, int num_sms, const int* stream_planes,
                          cudaStream_t s);
// plane coding: one warp per chunk of every (stream, plane)
struct CmpPlane {
  const unsigned long long* v;
  long long n;         // values
  int plane;           // byte index
  int chunk0;          // first global chunk index of this plane
  long long scratch0;  // first scratch word of this plane
};
cudaError_t cmp_encode(const CmpPlane* planes, int n_planes, int n_chunks_total, const unsigned long long* hist,
                       const int* plane_stream, uint16_t* ftab, uint16_t* scratch, long long* chunk_ptr, int* chunk_len,
                       const int* chunk_plane, cudaStream_t s);
cudaError_t cmp_layout(const CmpPlane* planes, int n_planes, const int* stream_planes, const long long* stream_n,
                       const uint16_t* ftab, const uint16_t* scratch, const long long* chunk_ptr, const int* chunk_len,
                       int n_chunks_total, const void* trk, long long n_trk, uint32_t kB_bits, double x_min,
                       double x_max, int n_items, int n_rows, long long n_unatt, long long n_att, uint8_t* out,
                       long long* out_size, long long* chunk_dst, cudaStream_t s);

// Sector-track merger (tpc_reduce.cu).
struct MrgArgs {
  const void* trk;            // tpc_track_t records, sorted by item
  const uint32_t* ids;
  long long n_trk, n_ids;
  const uint32_t* item_sector;
  const uint32_t* item_event;
  const int* nb_item;         // [I][2] item of the same event and side in sector k+1 / k-1, -1 none
  int I;
  const float *y, *z;
  const int* row;
  int N;
  double kB;
  float kB3_hi, kB3_lo;       // 3 kB as float-float
  int* item_first;            // [I + 1] first track of every item
  double* geo;                // [n_trk][12] per-track circle (device work array)
  float4* pre;                // [n_trk] (ok ? tan lambda : NaN, q/pT, sqrt(var q/pT), sign): the FP32 prefilter
  float4* geo32;              // [n_trk][2] (xc, yc, R, var q/pT), (x, y, z, radius) of geo rounded to FP32
  int* best;                  // [n_trk][2]
  int* link;                  // [n_trk][2] output
  int* group;                 // [n_trk] output
  double* fit;                // [n_trk][7] output (group roots)
  float* fit_sums;            // [n_trk][MRG_FIT_SUMS] per group root: the refit's float-float sums
  const int* item_seg;        // [I] segment (event and side) of every item
  const int* seg_items;       // [S][19] the segment's items (at most 18, -1 padded), then its item count
  int S;                      // segments
  int legs;                   // pair looper legs
  int* seg_n;                 // [S] tracks of the segment
  int* seg_off;               // [S + 1] offsets of the sorted lists
  int* seg_ok;                // [S] 1: sorted list built (else the candidates are scanned item by item)
  int sort_cap;               // largest segment sorted (at most MRG_SORT_CAP; 0: none)
  unsigned* skey;             // [n_trk] order-preserving tan(lambda) bits, ascending per segment
  int* sidx;                  // [n_trk] the tracks in the same order
  float4* geof2;              // [n_trk][4] float-float circle and reference point for the compatibility tests
  int* lbest;                 // [n_trk] best other-leg candidate
  int* partner;               // [n_trk] output: the other leg of a looper, -1 none
  uint8_t* leg;               // [n_trk] output: 1 for a secondary leg
  unsigned int* err;
};
cudaError_t launch_merge(const MrgArgs& a, const DevParams& par, int num_sms, cudaStream_t s);

// Looper legs joined into one track (tpc_join_loopers; tpc_reduce.cu)
struct JoinArgs {
  const void* trk;            // tpc_track_t [n_trk], sorted by item
  const uint32_t* ids;
  long long n_ids;
  int n_trk;
  const int* link;            // [n_trk][2] merger links
  const int* group;           // [n_trk] merger groups (smallest index)
  const int* partner;         // [n_trk] other leg, -1 none
  const uint8_t* leg;         // [n_trk] 1 = secondary leg
  const uint32_t* item_sector;
  int I;
  const float* y;
  const float* z;
  const int* row;
  int N;
  int* glab;                  // [n_trk] label of every group root
  int* plist;                 // [n_trk] primary legs of mutual pairs
  int* n_pairs;
  int* joined;                // out [n_trk]
  double* jfit;               // out [n_trk][7]
  unsigned int* err;
};
cudaError_t launch_join(const JoinArgs& a, const DevParams& par, int num_sms, cudaStream_t s);
