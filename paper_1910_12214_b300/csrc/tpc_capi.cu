// C ABI of libtpc (include/tpc.h): context, device buffers, launches, copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "tpc.h"
#include "tpc_reduce.h"
#include "tpc_internal.cuh"

struct tpc_ctx {
  tpc_config cfg{};
  std::string tune_path;  // autotuner cache file (cfg.tune_cache_path), empty = none
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool has_alloc = false;
  tpc_allocator alloc{};
  DevParams par{};
  LaunchCfg lc{};
  std::string err;
  // capacity of the current allocation
  long long capN = -1, capI = -1, capChunks = -1;
  std::vector<void*> blocks;
  Buffers b{};
  // buffers owned by the context (b.x.. may point at borrowed device input instead)
  float *own_x = nullptr, *own_y = nullptr, *own_z = nullptr;
  int* own_row = nullptr;
  int* own_core = nullptr;
  uint32_t *own_sec = nullptr, *own_ev = nullptr;
  // host-side copy bookkeeping
  std::vector<Chunk> chunks;
  bool loaded = false, tracked = false;
  bool input_on_device = false;
  cudaEvent_t ev[TPC_N_STAGES + 1] = {};
  cudaEvent_t mask_ev[3] = {};  // around the two kernels of tpc_cluster_masks (profile = 1)
  bool mask_timed = false;
  cudaEvent_t cmp_ev[6] = {};
  cudaEvent_t corr_ev[2] = {};  // around the space-point correction of the last tpc_track (profile = 1)
  bool corr_timed = false;  // around the symbol, rANS and layout phases of tpc_compress (profile = 1)
  bool cmp_timed = false;
  // the merger's item tables of the loaded batch (built on its first call after a load)
  std::vector<int> mrg_nb, mrg_item_seg, mrg_seg_items;
  bool mrg_tab_built = false;
  const void* mrg_tab_dev = nullptr;  // the device copy they were uploaded to
  bool have_events = false;
  // host copies of the item tables (debug dump, merger tables, frames)
  std::vector<uint64_t> h_item_off;
  std::vector<uint32_t> h_item_sector, h_item_event;  // empty if the batch has none
  // execution mode and CUDA graph of tpc_track
  bool batched = false, use_graph = false, last_batched = false;
  cudaGraphExec_t graph = nullptr;
  Buffers graph_b{}, graph_tb{};  // kernel arguments the graph was built with
  const int* graph_src = nullptr;  // frame id map the graph was built with
  // time frames (tpc_load_frame): persistent work buffers, grown on demand;
  // frame_src != null while the loaded batch is a sliced frame
  struct FrameBufs {
    float *x = nullptr, *y = nullptr, *z = nullptr;  // the frame, when given on the host
    int* row = nullptr;
    size_t cap_n = 0;
    Chunk* chunks = nullptr;
    size_t cap_chunks = 0;
    int *chunk_first = nullptr, *ext = nullptr, *nslice = nullptr, *size = nullptr, *slice_first = nullptr;
    double* c0 = nullptr;
    float2* bounds = nullptr;
    size_t cap_f = 0;
    int* cnt = nullptr;
    size_t cap_cnt = 0;
    uint64_t* slice_off = nullptr;
    size_t cap_s = 0;
    float *sx = nullptr, *sy = nullptr, *sz = nullptr;  // the sliced batch
    int *srow = nullptr, *src = nullptr;
    uint32_t* ids = nullptr;  // output cluster ids as frame indices
    size_t cap_ns = 0;
    unsigned int* err = nullptr;
  } fr;
  const int* frame_src = nullptr;
  // space-point correction: mode and model buffers (kept across batch loads)
  tpc_corr corr = TPC_CORR_NONE;
  std::vector<void*> persist;
  void* grid_dev = nullptr;
  void* grid_bounds_dev = nullptr;
  int grid_n[3] = {0, 0, 0}, grid_sectors = 0;
  // MLP surrogate state (master weights, Adam moments, inference copies)
  int mlp_S = 0, mlp_batch = 1024;
  uint64_t mlp_seed = 0, mlp_step = 0, mlp_T = 0;
  void* mlp_work = nullptr;  // training workspace (tpc_mlp.cu: clock, step counter, staged weights)
  float mlp_lr = 3e-2f;
  float *mlp_master = nullptr, *mlp_m = nullptr, *mlp_v = nullptr, *mlp_partial = nullptr, *mlp_loss = nullptr;
  float* mlp_bounds = nullptr;
  void* mlp_infer = nullptr;
  std::vector<float> mlp_bounds_host;
  // cluster codec: staging of host-mode calls (inputs then codes) and the bad-cluster counter
  void* codec_stage = nullptr;
  uint64_t codec_cap = 0;
  unsigned long long* codec_bad = nullptr;
  // cluster masks: per-cluster association words (zero between calls) and host-mode staging
  unsigned long long* mask_assoc = nullptr;
  uint64_t mask_cap = 0;
  bool mask_dirty = false;
  void* mask_stage = nullptr;
  size_t mask_stage_bytes = 0;
  // compression: persistent work buffers, grown on demand
  void* cmp_buf[48] = {};
  size_t cmp_cap[48] = {};
};

namespace {

tpc_status fail(tpc_ctx* c, tpc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

tpc_status cuda_fail(tpc_ctx* c, cudaError_t e, const char* where) {
  return fail(c, TPC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(tpc_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (c->has_alloc) {
    p = c->alloc.alloc(bytes, c->alloc.user);
  } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->blocks.push_back(p);
  return p;
}

void drop_graph(tpc_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
}

bool capturable(cudaStream_t s) { return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread; }

void* persist_alloc(tpc_ctx* c, size_t bytes) {
  const size_t before = c->blocks.size();
  void* p = dev_alloc(c, bytes);
  if (p) {  // move it from the batch list to the persistent list
    c->blocks.resize(before);
    c->persist.push_back(p);
  }
  return p;
}

void persist_free(tpc_ctx* c, void* p) {
  if (!p) return;
  cudaStreamSynchronize(c->stream);
  for (size_t i = 0; i < c->persist.size(); ++i)
    if (c->persist[i] == p) {
      if (c->has_alloc)
        c->alloc.free(p, c->alloc.user);
      else
        cudaFreeAsync(p, c->stream);
      c->persist.erase(c->persist.begin() + i);
      return;
    }
}

void free_all(tpc_ctx* c) {
  drop_graph(c);
  if (!c->blocks.empty()) cudaStreamSynchronize(c->stream);
  for (void* p : c->blocks) {
    if (c->has_alloc)
      c->alloc.free(p, c->alloc.user);
    else
      cudaFreeAsync(p, c->stream);
  }
  c->blocks.clear();
  c->capN = c->capI = c->capChunks = -1;
}

// Allocates every buffer for N clusters, I items and n_chunks CTAs of the
// cluster-parallel kernels.  Sizes per cluster (bytes): inputs 16, temporaries
// 12, grouped 12, sorted 16, bins <= 8, links 20 + 4, tracklets (N/3 starts)
// 4 + 112/3 + 4*n_rows/3, ownership 8 + 16/3, output 112/3 + 4.
tpc_status reserve(tpc_ctx* c, long long N, long long I, long long n_chunks) {
  if (N <= c->capN && I <= c->capI && n_chunks <= c->capChunks) return TPC_OK;
  free_all(c);
  N = std::max<long long>(N, c->capN < 0 ? 0 : c->capN);
  N = std::max<long long>(N, 1);
  I = std::max<long long>(I, 1);
  n_chunks = std::max<long long>(n_chunks, 1);
  const int NR = c->cfg.n_rows;
  const long long M = I * NR;
  const long long Tcap = N / 3 + I + 1;  // starts <= N/3 in total and <= n/3 per item
  Buffers& b = c->b;
  bool ok = true;
  auto A = [&](size_t bytes) -> void* {
    void* p = dev_alloc(c, bytes);
    ok &= p != nullptr;
    return p;
  };
  c->own_x = (float*)A(4 * N);
  c->own_y = (float*)A(4 * N);
  c->own_z = (float*)A(4 * N);
  c->own_row = (int*)A(4 * N);
  b.item_off = (const uint64_t*)A(8 * (I + 1));
  c->own_core = (int*)A(8 * I);
  c->own_sec = (uint32_t*)A(4 * I);
  c->own_ev = (uint32_t*)A(4 * I);
  b.chunks = (const Chunk*)A(sizeof(Chunk) * n_chunks);
  b.cl_key = (int*)A(4 * N);
  b.cl_q = (int2*)A(8 * N);
  b.rs_cnt = (int*)A(4 * M);
  b.rs_min = (int*)A(16 * M);
  b.row_fill = (int*)A(4 * M);
  b.rs_big = (int*)A(4 * (M + 1));
  b.rows = (RowInfo*)A(sizeof(RowInfo) * M);
  b.g_q = (int2*)A(8 * N);
  b.g_id = (int*)A(4 * N);
  b.s_hit = (int4*)A(16 * N);
  b.first = (int*)A(4 * (2 * N + 3 * M + 1));
  b.up_raw = (int*)A(4 * N);
  b.dn_raw = (int*)A(4 * N);
  b.up = (int*)A(4 * N);
  b.dn = (int*)A(4 * N);
  b.flags = (int*)A(4 * N);
  b.start_ex = (int*)A(4 * (N + 1));
  b.starts = (int*)A(4 * Tcap);
  b.tl = (TrackletRec*)A(sizeof(TrackletRec) * Tcap);
  b.tlu = (TrackletUp*)A(sizeof(TrackletUp) * Tcap);
  b.out_owner = (int*)A(4 * N);
  b.tl_hits = (int*)A(4 * (size_t)Tcap * NR);
  b.hit_key = (unsigned long long*)A(8 * N);
  b.tl_cnt = (unsigned long long*)A(8 * Tcap);
  b.tl_ex = (unsigned long long*)A(8 * (Tcap + 1));
  b.trk = A(sizeof(tpc_track_t) * Tcap);
  b.trk_ids = (uint32_t*)A(4 * N);
  b.trk_tl = (int*)A(4 * Tcap);
  b.counts = (unsigned long long*)A(8 * 4);
  b.err = (unsigned int*)A(16);
  b.scan_tmp = (unsigned long long*)A(8 * 1040);
  b.chain_len = (int*)A(4 * Tcap);
  b.tl_order = (int*)A(4 * Tcap);
  b.seg_next = (int*)A(4 * TPC_MAX_SEGS);
  b.cy = (float*)A(4 * N);
  b.cz = (float*)A(4 * N);
  b.T_cap = (int)Tcap;
  if (!ok) {
    free_all(c);
    return fail(c, TPC_ERR_OOM, "device allocation failed");
  }
  c->capN = N;
  c->capI = I;
  c->capChunks = n_chunks;
  return TPC_OK;
}

}  // namespace

extern "C" tpc_status tpc_init(const tpc_config* cfg, tpc_ctx** out) {
  if (!out) return TPC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg) return TPC_ERR_INVALID_ARG;
  if (cfg->n_rows < 3 || cfg->n_rows > TPC_MAX_ROWS || !(cfg->row_x_max > cfg->row_x_min) ||
      !(cfg->row_x_min > 0.f) || !(cfg->sector_half_angle_deg > 0.f) || !(cfg->sector_half_angle_deg < 60.f) ||
      !(cfg->sigma_y > 0.f) || !(cfg->sigma_z > 0.f) || !std::isfinite(cfg->bz_tesla) ||
      (cfg->mode != TPC_MODE_PLAIN && cfg->mode != TPC_MODE_BATCHED) ||
      (cfg->correction != TPC_CORR_NONE && cfg->correction != TPC_CORR_GRID && cfg->correction != TPC_CORR_MLP))
    return TPC_ERR_INVALID_ARG;
  if (cfg->allocator && (!cfg->allocator->alloc || !cfg->allocator->free)) return TPC_ERR_INVALID_ARG;
  tpc_ctx* c = new tpc_ctx();
  c->cfg = *cfg;
  if (cfg->tune_cache_path) c->tune_path = cfg->tune_cache_path;
  c->cfg.tune_cache_path = nullptr;  // the caller's string is not kept
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return TPC_ERR_CUDA;
  }
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return TPC_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cfg->allocator) {
    c->alloc = *cfg->allocator;
    c->has_alloc = true;
  }
  // geometry table: rows at x_min + r*(x_max-x_min)/(n_rows-1), quantised to 2^-10 cm
  DevParams& p = c->par;
  p.n_rows = cfg->n_rows;
  const double x0 = cfg->row_x_min, x1 = cfg->row_x_max;
  for (int r = 0; r < cfg->n_rows; ++r) {
    const double xr = x0 + r * ((x1 - x0) / (cfg->n_rows - 1));
    p.qx[r] = (int)std::nearbyint(xr * 1024.0);
    p.x[r] = (float)(p.qx[r] / 1024.0);
  }
  p.tan_half = (float)std::tan(cfg->sector_half_angle_deg * M_PI / 180.0);
  p.vy = cfg->sigma_y * cfg->sigma_y;
  p.vz = cfg->sigma_z * cfg->sigma_z;
  p.kB = (float)(0.299792458e-2 * cfg->bz_tesla);
  c->b.par = p;
  int dev = cfg->device, sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  LaunchCfg& L = c->lc;
  L.n_rows = cfg->n_rows;
  L.num_sms = sms;
  L.sort_smem = 12 * 1024;
  L.link_smem = 0;
  L.link_rows = 0;
  L.grid_scan = std::min(1024, 2 * sms);
  L.block_tl = 128;
  L.grid_tl = sms * 16;
  L.tl_group = 1;
  L.batch_group = 1;
  L.merge_sort_cap = 16384;
  c->batched = cfg->mode == TPC_MODE_BATCHED;
  c->corr = cfg->correction;
  c->use_graph = capturable(c->stream);
  if ((e = tpc_configure_kernels(L.sort_smem, L.link_smem)) != cudaSuccess) {
    cudaGetLastError();
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return TPC_ERR_CUDA;
  }
  if (cfg->profile) {
    for (int i = 0; i <= TPC_N_STAGES; ++i) cudaEventCreate(&c->ev[i]);
    for (int i = 0; i < 3; ++i) cudaEventCreate(&c->mask_ev[i]);
    for (int i = 0; i < 6; ++i) cudaEventCreate(&c->cmp_ev[i]);
    for (int i = 0; i < 2; ++i) cudaEventCreate(&c->corr_ev[i]);
    c->have_events = true;
  }
  if (cfg->max_clusters || cfg->max_items) {
    tpc_status s = reserve(c, (long long)cfg->max_clusters, (long long)std::max<uint32_t>(1, cfg->max_items),
                           (long long)cfg->max_clusters / 1024 + std::max<uint32_t>(1, cfg->max_items) + 1);
    if (s != TPC_OK) {
      tpc_destroy(c);
      return s;
    }
  }
  *out = c;
  return TPC_OK;
}

extern "C" tpc_status tpc_load_clusters(tpc_ctx* c, const tpc_clusters* cl) {
  if (!c || !cl) return TPC_ERR_INVALID_ARG;
  c->frame_src = nullptr;
  if (!cl->item_off) return fail(c, TPC_ERR_INVALID_ARG, "item_off is required");
  if (cl->n_items == 0 && cl->n != 0) return fail(c, TPC_ERR_INVALID_ARG, "clusters without items");
  if (cl->n > 0 && (!cl->x || !cl->y || !cl->z || !cl->row)) return fail(c, TPC_ERR_INVALID_ARG, "null cluster array");
  if (cl->n >= (1ull << 31) / 3) return fail(c, TPC_ERR_CAPACITY, "at most 715827882 clusters per batch");
  if (cl->item_off[0] != 0 || cl->item_off[cl->n_items] != cl->n)
    return fail(c, TPC_ERR_INVALID_ARG, "item_off must start at 0 and end at n");
  for (uint32_t i = 0; i < cl->n_items; ++i)
    if (cl->item_off[i + 1] < cl->item_off[i]) return fail(c, TPC_ERR_INVALID_ARG, "item_off not monotone");
  if ((unsigned long long)cl->n_items * c->cfg.n_rows >= (1ull << 31) / 4)
    return fail(c, TPC_ERR_CAPACITY, "too many items");
  if (cl->item_core)
    for (uint32_t i = 0; i < cl->n_items; ++i)
      if (cl->item_core[2 * i] > cl->item_core[2 * i + 1]) return fail(c, TPC_ERR_INVALID_ARG, "item_core lo > hi");
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  // work table of the cluster-parallel kernels: chunks of <= 1024 clusters, one item each
  c->chunks.clear();
  for (uint32_t i = 0; i < cl->n_items; ++i)
    for (uint64_t a = cl->item_off[i]; a < cl->item_off[i + 1]; a += 1024)
      c->chunks.push_back({(int)i, (int)a, (int)std::min<uint64_t>(a + 1024, cl->item_off[i + 1])});
  if (c->chunks.empty()) c->chunks.push_back({0, 0, 0});
  tpc_status s = reserve(c, (long long)cl->n, cl->n_items, (long long)c->chunks.size());
  if (s != TPC_OK) return s;
  Buffers& b = c->b;
  b.N = (int)cl->n;
  b.I = (int)std::max<uint32_t>(cl->n_items, 1);
  b.n_chunks = (int)c->chunks.size();
  const size_t n = cl->n;
  // cluster arrays: device pointers are borrowed, host arrays copied into our buffers
  if (cl->on_device) {
    c->input_on_device = true;
    c->b.x = cl->x;
    c->b.y = cl->y;
    c->b.z = cl->z;
    c->b.row = cl->row;
  } else {
    c->b.x = c->own_x;
    c->b.y = c->own_y;
    c->b.z = c->own_z;
    c->b.row = c->own_row;
    c->input_on_device = false;
    if (n) {
      if ((e = cudaMemcpyAsync((void*)b.x, cl->x, 4 * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
          (e = cudaMemcpyAsync((void*)b.y, cl->y, 4 * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
          (e = cudaMemcpyAsync((void*)b.z, cl->z, 4 * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
          (e = cudaMemcpyAsync((void*)b.row, cl->row, 4 * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "cluster upload");
    }
  }
  const size_t I = cl->n_items;
  e = cudaMemcpyAsync((void*)b.item_off, cl->item_off, 8 * (I + 1), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void*)b.chunks, c->chunks.data(), sizeof(Chunk) * c->chunks.size(), cudaMemcpyHostToDevice,
                        c->stream);
  // item metadata: optional arrays become null device pointers when absent
  const int* core_dev = c->own_core;
  const uint32_t* sec_dev = c->own_sec;
  const uint32_t* ev_dev = c->own_ev;
  b.item_core = cl->item_core ? core_dev : nullptr;
  b.item_sector = cl->item_sector ? sec_dev : nullptr;
  b.item_event = cl->item_event ? ev_dev : nullptr;
  if (e == cudaSuccess && cl->item_core)
    e = cudaMemcpyAsync((void*)core_dev, cl->item_core, 8 * I, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && cl->item_sector)
    e = cudaMemcpyAsync((void*)sec_dev, cl->item_sector, 4 * I, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && cl->item_event)
    e = cudaMemcpyAsync((void*)ev_dev, cl->item_event, 4 * I, cudaMemcpyHostToDevice, c->stream);
  c->h_item_off.assign(cl->item_off, cl->item_off + cl->n_items + 1);
  if (cl->item_sector)
    c->h_item_sector.assign(cl->item_sector, cl->item_sector + cl->n_items);
  else
    c->h_item_sector.clear();
  if (cl->item_event)
    c->h_item_event.assign(cl->item_event, cl->item_event + cl->n_items);
  else
    c->h_item_event.clear();
  if (e == cudaSuccess) e = cudaMemsetAsync(b.err, 0, 16, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.counts, 0, 32, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "metadata upload");
  // host arrays must stay valid only during the call
  if (!cl->on_device && (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "sync");
  // a captured graph stays: tpc_track rebuilds or updates it if the kernel
  // arguments changed (a batch of the same sizes into the same buffers reuses it)
  c->loaded = true;
  c->tracked = false;
  c->mask_timed = false;
  c->mrg_tab_built = false;
  c->mrg_tab_dev = nullptr;
  c->cmp_timed = false;
  return TPC_OK;
}

namespace {
template <class T>
bool grow_persist(tpc_ctx* c, T*& p, size_t& cap, size_t n) {
  if (p && n <= cap) return true;
  persist_free(c, p);
  n = std::max<size_t>(n, 1);
  p = static_cast<T*>(persist_alloc(c, sizeof(T) * n));
  cap = p ? n : 0;
  return p != nullptr;
}
}  // namespace

extern "C" tpc_status tpc_load_frame(tpc_ctx* c, const tpc_clusters* fr, float core_cm, float overlap_cm) {
  if (!c || !fr) return TPC_ERR_INVALID_ARG;
  if (!fr->item_off) return fail(c, TPC_ERR_INVALID_ARG, "item_off is required");
  if (fr->item_core) return fail(c, TPC_ERR_INVALID_ARG, "a frame has no item_core: its slices get one");
  if (fr->n_items == 0 && fr->n != 0) return fail(c, TPC_ERR_INVALID_ARG, "clusters without items");
  if (fr->n > 0 && (!fr->x || !fr->y || !fr->z || !fr->row)) return fail(c, TPC_ERR_INVALID_ARG, "null cluster array");
  if (!(core_cm > 0.f) || !(overlap_cm >= 0.f) || !std::isfinite(core_cm) || !std::isfinite(overlap_cm) ||
      std::ceil((double)overlap_cm / core_cm) > TF_WMAX - 1)
    return fail(c, TPC_ERR_INVALID_ARG, "core_cm > 0 and 0 <= overlap_cm <= 3 core_cm");
  if (fr->n >= (1ull << 31) / 8) return fail(c, TPC_ERR_CAPACITY, "frame too large");
  if (fr->item_off[0] != 0 || fr->item_off[fr->n_items] != fr->n)
    return fail(c, TPC_ERR_INVALID_ARG, "item_off must start at 0 and end at n");
  for (uint32_t i = 0; i < fr->n_items; ++i)
    if (fr->item_off[i + 1] < fr->item_off[i]) return fail(c, TPC_ERR_INVALID_ARG, "item_off not monotone");
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  const uint32_t F = fr->n_items;
  const size_t n = fr->n;
  auto& B = c->fr;
  // frame chunks (one item each, in item order) and every item's first chunk
  std::vector<Chunk> chunks;
  std::vector<int> chunk_first(F + 1, 0);
  for (uint32_t i = 0; i < F; ++i) {
    chunk_first[i] = (int)chunks.size();
    for (uint64_t a = fr->item_off[i]; a < fr->item_off[i + 1]; a += TF_CHUNK)
      chunks.push_back({(int)i, (int)a, (int)std::min<uint64_t>(a + TF_CHUNK, fr->item_off[i + 1])});
  }
  chunk_first[F] = (int)chunks.size();
  const size_t nch = chunks.size();
  bool ok = grow_persist(c, B.chunks, B.cap_chunks, nch) && grow_persist(c, B.cnt, B.cap_cnt, nch * TF_KMAX);
  if (ok && (!B.ext || F > B.cap_f)) {  // every per-item array has room for cap_f items
    for (void* p : {(void*)B.chunk_first, (void*)B.ext, (void*)B.nslice, (void*)B.size, (void*)B.slice_first,
                    (void*)B.c0, (void*)B.bounds})
      persist_free(c, p);
    const size_t f = std::max<size_t>(F, 1);
    B.chunk_first = (int*)persist_alloc(c, 4 * (f + 1));
    B.ext = (int*)persist_alloc(c, 8 * f);
    B.nslice = (int*)persist_alloc(c, 4 * f);
    B.size = (int*)persist_alloc(c, 4 * f * TF_KMAX);
    B.slice_first = (int*)persist_alloc(c, 4 * f);
    B.c0 = (double*)persist_alloc(c, 8 * f);
    B.bounds = (float2*)persist_alloc(c, 8 * f * TF_KMAX);
    ok = B.chunk_first && B.ext && B.nslice && B.size && B.slice_first && B.c0 && B.bounds;
    B.cap_f = ok ? f : 0;
    if (!ok) B.ext = nullptr;
  }
  if (ok && !B.err) B.err = (unsigned int*)persist_alloc(c, 16);
  ok = ok && B.err;
  if (ok && !fr->on_device) {
    size_t cap_n = B.cap_n;
    if (!B.x || n > B.cap_n) {
      persist_free(c, B.x);
      persist_free(c, B.y);
      persist_free(c, B.z);
      persist_free(c, B.row);
      const size_t m = std::max<size_t>(n, 1);
      B.x = (float*)persist_alloc(c, 4 * m);
      B.y = (float*)persist_alloc(c, 4 * m);
      B.z = (float*)persist_alloc(c, 4 * m);
      B.row = (int*)persist_alloc(c, 4 * m);
      cap_n = m;
    }
    ok = B.x && B.y && B.z && B.row;
    B.cap_n = ok ? cap_n : 0;
  }
  if (!ok) return fail(c, TPC_ERR_OOM, "device allocation failed (frame buffers)");
  FrameArgs a{};
  if (fr->on_device) {
    a.x = fr->x;
    a.y = fr->y;
    a.z = fr->z;
    a.row = fr->row;
  } else {
    a.x = B.x;
    a.y = B.y;
    a.z = B.z;
    a.row = B.row;
    if (n && ((e = cudaMemcpyAsync(B.x, fr->x, 4 * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
              (e = cudaMemcpyAsync(B.y, fr->y, 4 * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
              (e = cudaMemcpyAsync(B.z, fr->z, 4 * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
              (e = cudaMemcpyAsync(B.row, fr->row, 4 * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess))
      return cuda_fail(c, e, "frame upload");
  }
  a.chunks = B.chunks;
  a.n_chunks = (int)nch;
  a.chunk_first = B.chunk_first;
  a.F = (int)F;
  a.core = core_cm;
  a.overlap = overlap_cm;
  a.W = 1 + (int)std::ceil((double)overlap_cm / core_cm);
  a.ext = B.ext;
  a.c0 = B.c0;
  a.nslice = B.nslice;
  a.bounds = B.bounds;
  a.cnt = B.cnt;
  a.size = B.size;
  a.err = B.err;
  if (nch && (e = cudaMemcpyAsync(B.chunks, chunks.data(), sizeof(Chunk) * nch, cudaMemcpyHostToDevice,
                                  c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "frame chunks");
  if ((e = cudaMemcpyAsync(B.chunk_first, chunk_first.data(), 4 * (F + 1), cudaMemcpyHostToDevice, c->stream)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(B.err, 0, 4, c->stream)) != cudaSuccess || (e = tpc_frame_count(a, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "frame slicing");
  // slice counts and sizes back to the host: the sliced batch's item tables
  std::vector<int> nslice(F), size((size_t)F * TF_KMAX);
  std::vector<double> c0(F);
  unsigned int err = 0;
  if (F && ((e = cudaMemcpyAsync(nslice.data(), B.nslice, 4 * F, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(c0.data(), B.c0, 8 * F, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(size.data(), B.size, 4 * size.size(), cudaMemcpyDeviceToHost, c->stream)) !=
                cudaSuccess))
    return cuda_fail(c, e, "frame sizes");
  if ((e = cudaMemcpyAsync(&err, B.err, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "frame sizes");
  if (err & TPC_DERR_BAD_INPUT) return fail(c, TPC_ERR_BAD_INPUT, "a frame cluster has a non-finite or huge z");
  if (err & TPC_DERR_CAPACITY) return fail(c, TPC_ERR_CAPACITY, "a frame item spans more than 64 slices");
  std::vector<int> slice_first(F);
  std::vector<uint64_t> slice_off(1, 0);
  std::vector<int32_t> core;
  std::vector<uint32_t> sec, ev;
  for (uint32_t i = 0; i < F; ++i) {
    slice_first[i] = (int)slice_off.size() - 1;
    for (int k = 0; k < nslice[i]; ++k) {
      slice_off.push_back(slice_off.back() + (uint64_t)size[(size_t)i * TF_KMAX + k]);
      const double cz = c0[i] + (double)k * core_cm;
      core.push_back((int32_t)std::nearbyint(cz * 1024.0));
      core.push_back((int32_t)std::nearbyint((cz + core_cm) * 1024.0));
      sec.push_back(fr->item_sector ? fr->item_sector[i] : i);
      ev.push_back(fr->item_event ? fr->item_event[i] : 0u);
    }
  }
  const size_t S = slice_off.size() - 1, Ns = slice_off.back();
  if (Ns >= (1ull << 31) / 3) return fail(c, TPC_ERR_CAPACITY, "sliced frame too large");
  size_t cap_s = B.cap_s;
  ok = grow_persist(c, B.slice_off, cap_s, S + 1);
  B.cap_s = ok ? cap_s : 0;
  if (ok && (!B.sx || Ns > B.cap_ns)) {
    for (void* p : {(void*)B.sx, (void*)B.sy, (void*)B.sz, (void*)B.srow, (void*)B.src, (void*)B.ids})
      persist_free(c, p);
    const size_t m = std::max<size_t>(Ns, 1);
    B.sx = (float*)persist_alloc(c, 4 * m);
    B.sy = (float*)persist_alloc(c, 4 * m);
    B.sz = (float*)persist_alloc(c, 4 * m);
    B.srow = (int*)persist_alloc(c, 4 * m);
    B.src = (int*)persist_alloc(c, 4 * m);
    B.ids = (uint32_t*)persist_alloc(c, 4 * m);
    ok = B.sx && B.sy && B.sz && B.srow && B.src && B.ids;
    B.cap_ns = ok ? m : 0;
  }
  if (!ok) return fail(c, TPC_ERR_OOM, "device allocation failed (sliced frame)");
  // slices in place: the frame's chunks scatter into the sliced batch
  a.slice_first = B.slice_first;
  a.slice_off = B.slice_off;
  a.ox = B.sx;
  a.oy = B.sy;
  a.oz = B.sz;
  a.orow = B.srow;
  a.src = B.src;
  if ((F && (e = cudaMemcpyAsync(B.slice_first, slice_first.data(), 4 * F, cudaMemcpyHostToDevice, c->stream)) !=
                cudaSuccess) ||
      (e = cudaMemcpyAsync(B.slice_off, slice_off.data(), 8 * (S + 1), cudaMemcpyHostToDevice, c->stream)) !=
          cudaSuccess ||
      (e = tpc_frame_scatter(a, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "frame scatter");
  // the sliced batch is an ordinary batch on the device (borrowed from the frame buffers)
  tpc_clusters sl{};
  sl.x = B.sx;
  sl.y = B.sy;
  sl.z = B.sz;
  sl.row = B.srow;
  sl.n = Ns;
  sl.item_off = slice_off.data();
  sl.n_items = (uint32_t)S;
  sl.item_sector = sec.data();
  sl.item_event = ev.data();
  sl.item_core = core.data();
  sl.on_device = 1;
  tpc_status st = tpc_load_clusters(c, &sl);
  if (st != TPC_OK) return st;
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "frame load");
  c->frame_src = B.src;
  return TPC_OK;
}

extern "C" tpc_status tpc_track(tpc_ctx* c) {
  if (!c) return TPC_ERR_INVALID_ARG;
  if (!c->loaded) return fail(c, TPC_ERR_STATE, "tpc_track before tpc_load_clusters");
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  if (c->b.N == 0) {
    c->tracked = true;
    return TPC_OK;  // counts were zeroed at load
  }
  if (c->corr == TPC_CORR_GRID && !c->grid_dev)
    return fail(c, TPC_ERR_STATE, "grid correction selected but no grid set (tpc_set_grid_correction)");
  if (c->corr == TPC_CORR_MLP && !c->b.mlp)
    return fail(c, TPC_ERR_STATE, "MLP correction selected but no trained or loaded network");
  Buffers tb = c->b;  // tracking reads corrected coordinates when a correction is on
  if (c->corr != TPC_CORR_NONE) {
    tb.y = c->b.cy;
    tb.z = c->b.cz;
  }
  auto launch = [&]() {
    cudaError_t ce = cudaSuccess;
    const bool tc = c->have_events && c->corr != TPC_CORR_NONE;
    if (tc) cudaEventRecord(c->corr_ev[0], c->stream);
    if (c->corr == TPC_CORR_GRID) ce = tpc_launch_grid_correction(c->b, c->stream);
    if (c->corr == TPC_CORR_MLP) ce = tpc_launch_mlp_correction(c->b, c->stream);
    if (tc) cudaEventRecord(c->corr_ev[1], c->stream);
    if (ce != cudaSuccess) return ce;
    ce = c->batched ? tpc_launch_batched(tb, c->lc, c->stream, c->have_events ? c->ev : nullptr)
                    : tpc_launch_plain(tb, c->lc, c->stream, c->have_events ? c->ev : nullptr);
    if (ce == cudaSuccess && c->frame_src)  // output ids of a sliced frame -> frame indices
      ce = tpc_frame_map_ids(c->b.trk_ids, c->frame_src, c->fr.ids, c->b.counts, 4 * c->lc.num_sms, c->stream);
    return ce;
  };
  if (c->use_graph && capturable(c->stream)) {
    const bool stale = c->graph && (std::memcmp(&c->graph_b, &c->b, sizeof(Buffers)) != 0 ||
                                    std::memcmp(&c->graph_tb, &tb, sizeof(Buffers)) != 0 ||
                                    c->graph_src != c->frame_src);
    if (!c->graph || stale) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
      cudaError_t le = launch();
      e = cudaStreamEndCapture(c->stream, &g);
      if (le != cudaSuccess) e = le;
      if (e == cudaSuccess && stale) {
        // same launch sequence with new arguments: update the executable graph in place
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(c->graph, g, &info) != cudaSuccess) {
          cudaGetLastError();
          drop_graph(c);
        }
      }
      if (e == cudaSuccess && !c->graph) e = cudaGraphInstantiate(&c->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        drop_graph(c);
        return cuda_fail(c, e, "graph build");
      }
      c->graph_b = c->b;
      c->graph_tb = tb;
      c->graph_src = c->frame_src;
    }
    e = cudaGraphLaunch(c->graph, c->stream);
  } else {
    e = launch();
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "launch");
  c->last_batched = c->batched;
  c->corr_timed = c->have_events && c->corr != TPC_CORR_NONE;
  c->tracked = true;
  return TPC_OK;
}

extern "C" tpc_status tpc_sync(tpc_ctx* c) {
  if (!c) return TPC_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream");
  if (!c->loaded) return TPC_OK;
  unsigned int err = 0;
  e = cudaMemcpy(&err, c->b.err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "error word");
  if (err & TPC_DERR_BAD_INPUT) return fail(c, TPC_ERR_BAD_INPUT, "a cluster has a bad row or a non-finite value");
  if (err & TPC_DERR_ROW_CAP) return fail(c, TPC_ERR_CAPACITY, "row too large");
  if (err & TPC_DERR_TIMEOUT) return fail(c, TPC_ERR_TIMEOUT, "device wait timed out");
  if (err & TPC_DERR_BAD_TRACK)
    return fail(c, TPC_ERR_BAD_INPUT, "a track given to tpc_cluster_masks refers to an item or cluster out of range");
  return TPC_OK;
}

extern "C" tpc_status tpc_get_tracks(tpc_ctx* c, tpc_track_t* trk, uint64_t trk_cap, uint32_t* ids, uint64_t id_cap,
                                     uint64_t* n_trk, uint64_t* n_ids) {
  if (!c) return TPC_ERR_INVALID_ARG;
  if (!c->tracked) return fail(c, TPC_ERR_STATE, "tpc_get_tracks before tpc_track");
  tpc_status s = tpc_sync(c);
  if (s != TPC_OK) return s;
  unsigned long long cnt[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpy(cnt, c->b.counts, 32, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "counts");
  if (n_trk) *n_trk = cnt[0];
  if (n_ids) *n_ids = cnt[1];
  if (cnt[0] > trk_cap || cnt[1] > id_cap) return fail(c, TPC_ERR_CAPACITY, "output buffers too small");
  if ((cnt[0] && !trk) || (cnt[1] && !ids)) return fail(c, TPC_ERR_INVALID_ARG, "null output buffer");
  if (cnt[0] && (e = cudaMemcpy(trk, c->b.trk, sizeof(tpc_track_t) * cnt[0], cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(c, e, "track copy");
  const uint32_t* src_ids = c->frame_src ? c->fr.ids : c->b.trk_ids;
  if (cnt[1] && (e = cudaMemcpy(ids, src_ids, 4 * cnt[1], cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(c, e, "id copy");
  return TPC_OK;
}

extern "C" tpc_status tpc_device_tracks(tpc_ctx* c, const tpc_track_t** trk, const uint32_t** ids,
                                        const uint64_t** counts) {
  if (!c) return TPC_ERR_INVALID_ARG;
  if (!c->loaded) return fail(c, TPC_ERR_STATE, "nothing loaded");
  if (trk) *trk = (const tpc_track_t*)c->b.trk;
  if (ids) *ids = c->frame_src ? c->fr.ids : c->b.trk_ids;
  if (counts) *counts = (const uint64_t*)c->b.counts;
  return TPC_OK;
}

static const char* kStageNames[TPC_N_REPORTED_STAGES] = {
    "quantise+row_stats", "row_setup", "group_scatter", "row_sort", "links", "clean+starts", "tracklets",
    "selection", "output", "unused_9", "unused_10", "mask_assoc", "mask_final", "compress_symbols",
    "compress_rans", "compress_layout", "correction"};

extern "C" const char* tpc_stage_name(int i) { return (i >= 0 && i < TPC_N_REPORTED_STAGES) ? kStageNames[i] : ""; }

extern "C" tpc_status tpc_stage_times(tpc_ctx* c, float* us, int n, int* n_stages) {
  if (!c) return TPC_ERR_INVALID_ARG;
  if (n_stages) *n_stages = TPC_N_REPORTED_STAGES;
  if (!c->have_events) return fail(c, TPC_ERR_STATE, "context created without profile = 1");
  if (!c->tracked) return fail(c, TPC_ERR_STATE, "no tpc_track yet");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream");
  for (int i = 0; i < TPC_N_REPORTED_STAGES && i < n; ++i) {
    float ms = 0.f;
    const bool corr = i == TPC_N_REPORTED_STAGES - 1;
    const bool mask = i >= TPC_N_STAGES && i < TPC_N_STAGES + 2, cmp = !corr && i >= TPC_N_STAGES + 2;
    const bool mine = corr ? c->corr_timed : cmp ? c->cmp_timed : (mask ? c->mask_timed : i < 9);
    const int j = i - TPC_N_STAGES - 2;
    const cudaEvent_t a = corr ? c->corr_ev[0]
                               : cmp ? c->cmp_ev[2 * j] : (mask ? c->mask_ev[i - TPC_N_STAGES] : c->ev[i]);
    const cudaEvent_t b = corr ? c->corr_ev[1]
                               : cmp ? c->cmp_ev[2 * j + 1] : (mask ? c->mask_ev[i - TPC_N_STAGES + 1] : c->ev[i + 1]);
    if (mine && cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    us[i] = mine ? ms * 1000.f : 0.f;
  }
  return TPC_OK;
}

extern "C" tpc_status tpc_debug_dump(tpc_ctx* c, int stage, int32_t* buf, uint64_t cap, uint64_t* n_out) {
  if (!c || !n_out) return TPC_ERR_INVALID_ARG;
  if (!c->tracked) return fail(c, TPC_ERR_STATE, "no tpc_track yet");
  tpc_status st = tpc_sync(c);
  if (st != TPC_OK && st != TPC_ERR_BAD_INPUT) return st;
  const Buffers& b = c->b;
  const size_t N = b.N, NR = c->cfg.n_rows, M = (size_t)b.I * NR;
  auto D2H = [&](std::vector<int>& v, const void* src, size_t n) {
    v.resize(n);
    return n ? cudaMemcpy(v.data(), src, 4 * n, cudaMemcpyDeviceToHost) : cudaSuccess;
  };
  std::vector<int> out, sid(N), tmp, hit;
  cudaError_t e = D2H(hit, b.s_hit, 4 * N);
  if (e != cudaSuccess) return cuda_fail(c, e, "dump");
  for (size_t i = 0; i < N; ++i) sid[i] = hit[4 * i + 2];
  std::vector<RowInfo> rows(M);
  if (M && (e = cudaMemcpy(rows.data(), b.rows, sizeof(RowInfo) * M, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(c, e, "dump");
  // tracklet storage index of every tracklet in canonical order (both forms: 0..T-1)
  int T = 0;
  if ((e = cudaMemcpy(&T, b.start_ex + N, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(c, e, "dump");
  std::vector<int> tl_index(T);
  for (int t = 0; t < T; ++t) tl_index[t] = t;
  const int Tmax = tl_index.empty() ? 0 : *std::max_element(tl_index.begin(), tl_index.end()) + 1;
  switch (stage) {
    case 0: {
      out.resize(3 * N);
      for (size_t i = 0; i < N; ++i) {
        out[3 * i] = hit[4 * i];
        out[3 * i + 1] = hit[4 * i + 1];
        out[3 * i + 2] = hit[4 * i + 2];
      }
      break;
    }
    case 1:
      for (const RowInfo& r : rows) {
        const int v[7] = {r.pos0, r.n, r.ymin, r.zmin, r.shift, r.ny, r.nz};
        out.insert(out.end(), v, v + 7);
      }
      break;
    case 2: {
      if ((e = D2H(tmp, b.first, 2 * N + 3 * M + 1)) != cudaSuccess) return cuda_fail(c, e, "dump");
      for (const RowInfo& r : rows) {
        const int nb = r.n > 0 ? r.ny * r.nz : 0;
        for (int j = 0; j <= nb; ++j) out.push_back(tmp[r.bin0 + j] - r.pos0);
      }
      break;
    }
    case 3:
    case 4:
    case 5:
    case 6: {
      const int* src = stage == 3 ? b.up_raw : stage == 4 ? b.dn_raw : stage == 5 ? b.up : b.dn;
      if ((e = D2H(tmp, src, N)) != cudaSuccess) return cuda_fail(c, e, "dump");
      out.assign(N, -1);
      for (size_t p = 0; p < N; ++p)
        if (sid[p] >= 0 && (size_t)sid[p] < N) out[sid[p]] = (tmp[p] >= 0 && (size_t)tmp[p] < N) ? sid[tmp[p]] : -1;
      break;
    }
    case 7: {
      if ((e = D2H(tmp, b.starts, Tmax)) != cudaSuccess) return cuda_fail(c, e, "dump");
      for (int t : tl_index) out.push_back(sid[tmp[t]]);
      break;
    }
    case 8:
    case 9: {  // (tracklets that lost their outermost hit to a smaller id read n = 0)
      std::vector<TrackletRec> tl(Tmax);
      if (Tmax && (e = cudaMemcpy(tl.data(), b.tl, sizeof(TrackletRec) * Tmax, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(c, e, "dump");
      if (stage == 8) {
        for (int t : tl_index) out.push_back(tl[t].n);
      } else {
        if ((e = D2H(tmp, b.tl_hits, (size_t)Tmax * NR)) != cudaSuccess) return cuda_fail(c, e, "dump");
        for (int t : tl_index)
          for (int k = 0; k < tl[t].n; ++k) out.push_back(sid[tmp[(size_t)t * NR + k]]);
      }
      break;
    }
    case 11: {  // corrected (y, z) per input cluster as float bits (input coordinates when no correction)
      const float* ys = c->corr != TPC_CORR_NONE ? b.cy : b.y;
      const float* zs = c->corr != TPC_CORR_NONE ? b.cz : b.z;
      std::vector<int> yy, zz;
      if ((e = D2H(yy, ys, N)) != cudaSuccess || (e = D2H(zz, zs, N)) != cudaSuccess) return cuda_fail(c, e, "dump");
      out.resize(2 * N);
      for (size_t i = 0; i < N; ++i) {
        out[2 * i] = yy[i];
        out[2 * i + 1] = zz[i];
      }
      break;
    }
    case 10: {
      unsigned long long cnt[4] = {0, 0, 0, 0};
      if ((e = cudaMemcpy(cnt, b.counts, 32, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(c, e, "dump");
      if ((e = D2H(out, b.trk_tl, cnt[0])) != cudaSuccess) return cuda_fail(c, e, "dump");
      break;
    }
    default:
      return fail(c, TPC_ERR_INVALID_ARG, "unknown stage");
  }
  *n_out = out.size();
  if (buf && cap) std::memcpy(buf, out.data(), 4 * std::min<size_t>(cap, out.size()));
  if (cap < out.size()) return fail(c, TPC_ERR_CAPACITY, "dump buffer too small");
  return TPC_OK;
}

namespace {
tpc_status apply_tuning(tpc_ctx* c, const tpc_tuning& t) {
  LaunchCfg L = c->lc;
  if (t.tracklet_lanes) {
    if (t.tracklet_lanes != 1 && t.tracklet_lanes != 2 && t.tracklet_lanes != 4 && t.tracklet_lanes != 8 &&
        t.tracklet_lanes != 16 && t.tracklet_lanes != 32)
      return fail(c, TPC_ERR_INVALID_ARG, "tracklet_lanes must be 1, 2, 4, 8, 16 or 32");
    L.tl_group = t.tracklet_lanes;
  }
  if (t.tracklet_block) {
    if (t.tracklet_block % 32 || t.tracklet_block > 128 || t.tracklet_block < 32)
      return fail(c, TPC_ERR_INVALID_ARG, "tracklet_block must be a multiple of 32, at most 128");
    L.block_tl = t.tracklet_block;
  }
  if (t.tracklet_blocks_per_sm) {
    if (t.tracklet_blocks_per_sm < 1 || t.tracklet_blocks_per_sm > 64)
      return fail(c, TPC_ERR_INVALID_ARG, "tracklet_blocks_per_sm out of range");
    L.grid_tl = t.tracklet_blocks_per_sm * L.num_sms;
  }
  if (t.sort_smem) {
    if (t.sort_smem < 1024 || t.sort_smem > 200 * 1024) return fail(c, TPC_ERR_INVALID_ARG, "sort_smem out of range");
    L.sort_smem = t.sort_smem & ~15;
  }
  if (t.link_rows) {
    if (t.link_rows < -1 || t.link_rows > TPC_MAX_ROWS) return fail(c, TPC_ERR_INVALID_ARG, "link_rows out of range");
    L.link_rows = t.link_rows < 0 ? 0 : t.link_rows;
  }
  bool batched = c->batched, use_graph = c->use_graph;
  if (t.mode) {
    if (t.mode != 1 && t.mode != 2) return fail(c, TPC_ERR_INVALID_ARG, "mode must be 1 (plain) or 2 (batched)");
    batched = t.mode == 2;
  }
  if (t.batch_lanes) {
    if (t.batch_lanes != 1 && t.batch_lanes != 2 && t.batch_lanes != 4)
      return fail(c, TPC_ERR_INVALID_ARG, "batch_lanes must be 1, 2 or 4");
    L.batch_group = t.batch_lanes;
  }
  if (t.merge_sort_cap) {
    if (t.merge_sort_cap < -1 || t.merge_sort_cap > 16384)
      return fail(c, TPC_ERR_INVALID_ARG, "merge_sort_cap must be -1 or 1 to 16384");
    L.merge_sort_cap = t.merge_sort_cap < 0 ? 0 : t.merge_sort_cap;
  }
  if (t.use_graph) {
    if (t.use_graph != 1 && t.use_graph != 2) return fail(c, TPC_ERR_INVALID_ARG, "use_graph must be 1 or 2");
    use_graph = t.use_graph == 2 && capturable(c->stream);
  }
  cudaError_t e = tpc_configure_kernels(L.sort_smem, L.link_smem);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel attributes");
  c->lc = L;
  c->batched = batched;
  c->use_graph = use_graph;
  drop_graph(c);
  return TPC_OK;
}
}  // namespace

extern "C" tpc_status tpc_set_tuning(tpc_ctx* c, const tpc_tuning* t) {
  if (!c || !t) return TPC_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  return apply_tuning(c, *t);
}

extern "C" tpc_status tpc_get_tuning(tpc_ctx* c, tpc_tuning* t) {
  if (!c || !t) return TPC_ERR_INVALID_ARG;
  t->tracklet_lanes = c->lc.tl_group;
  t->tracklet_block = c->lc.block_tl;
  t->tracklet_blocks_per_sm = c->lc.grid_tl / std::max(1, c->lc.num_sms);
  t->sort_smem = c->lc.sort_smem;
  t->link_rows = c->lc.link_rows ? c->lc.link_rows : -1;
  t->mode = c->batched ? 2 : 1;
  t->batch_lanes = c->lc.batch_group;
  t->use_graph = c->use_graph ? 2 : 1;
  t->merge_sort_cap = c->lc.merge_sort_cap ? c->lc.merge_sort_cap : -1;
  return TPC_OK;
}

extern "C" tpc_status tpc_autotune(tpc_ctx* c, int iters, tpc_tuning* best_out, float* best_us) {
  return tpc_autotune_mode(c, iters, 0, best_out, best_us);
}

namespace {
// Autotuner cache: one line per key, "key|lanes block per_sm smem link_rows
// mode batch_lanes use_graph merge_cap|best_us".  The key names the GPU, the
// mode searched and the batch's shape (clusters, items, rows, correction), so
// a later process with the same workload skips the search.  File errors only
// disable the cache.
std::string tune_key(const tpc_ctx* c, int mode) {
  cudaDeviceProp p{};
  if (cudaGetDeviceProperties(&p, c->cfg.device) != cudaSuccess) {
    cudaGetLastError();
    return std::string();
  }
  std::ostringstream k;
  std::string name(p.name);
  for (char& ch : name)
    if (ch == ' ' || ch == '|') ch = '_';
  k << name << ":sm" << p.multiProcessorCount << ":mode" << mode << ":n" << c->b.N << ":items" << c->b.I << ":rows"
    << c->cfg.n_rows << ":corr" << (int)c->corr;
  return k.str();
}

bool tune_lookup(const std::string& path, const std::string& key, tpc_tuning* t, float* us) {
  std::ifstream f(path);
  std::string line;
  while (f && std::getline(f, line)) {
    const size_t a = line.find('|'), b = line.rfind('|');
    if (a == std::string::npos || b == a || line.compare(0, a, key) != 0 || a != key.size()) continue;
    std::istringstream v(line.substr(a + 1, b - a - 1));
    tpc_tuning r{};
    if (!(v >> r.tracklet_lanes >> r.tracklet_block >> r.tracklet_blocks_per_sm >> r.sort_smem >> r.link_rows >>
          r.mode >> r.batch_lanes >> r.use_graph >> r.merge_sort_cap))
      continue;
    *t = r;
    *us = std::strtof(line.c_str() + b + 1, nullptr);
    return true;
  }
  return false;
}

void tune_store(const std::string& path, const std::string& key, const tpc_tuning& t, float us) {
  std::vector<std::string> keep;
  {
    std::ifstream f(path);
    std::string line;
    while (f && std::getline(f, line))
      if (line.compare(0, key.size() + 1, key + "|") != 0) keep.push_back(line);
  }
  char buf[256];
  std::snprintf(buf, sizeof(buf), "|%d %d %d %d %d %d %d %d %d|%.9g", t.tracklet_lanes, t.tracklet_block,
                t.tracklet_blocks_per_sm, t.sort_smem, t.link_rows, t.mode, t.batch_lanes, t.use_graph,
                t.merge_sort_cap, us);
  keep.push_back(key + buf);
  const std::string tmp = path + ".tmp";
  {
    std::ofstream o(tmp, std::ios::trunc);
    for (const std::string& l : keep) o << l << "\n";
    if (!o) return;
  }
  std::rename(tmp.c_str(), path.c_str());
}
}  // namespace

extern "C" tpc_status tpc_autotune_mode(tpc_ctx* c, int iters, int mode, tpc_tuning* best_out, float* best_us) {
  if (!c || iters < 1 || mode < 0 || mode > 2) return TPC_ERR_INVALID_ARG;
  if (!c->loaded) return fail(c, TPC_ERR_STATE, "tpc_autotune before tpc_load_clusters");
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  const std::string key = c->tune_path.empty() ? std::string() : tune_key(c, mode);
  {
    tpc_tuning cached{};
    float cached_us = 0.f;
    if (!key.empty() && tune_lookup(c->tune_path, key, &cached, &cached_us)) {
      tpc_status st = apply_tuning(c, cached);
      if (st == TPC_OK) {
        st = tpc_track(c);  // as after a search: the batch is tracked with the chosen shape
        if (best_out) *best_out = cached;
        if (best_us) *best_us = cached_us;
        return st;
      }
    }
  }
  // plain-mode shapes, then shared memory and row blocks, then the batched kernel
  std::vector<tpc_tuning> cand;
  for (int lanes : {1, 2, 4, 8, 16, 32})
    for (int blk : {32, 64, 128})
      for (int per_sm : {8, 16, 32}) cand.push_back({lanes, blk, per_sm, 0, 0, 1, 0, 0});
  for (int sm : {6 * 1024, 12 * 1024, 24 * 1024})
    for (int lr : {-1, 1, 2, 4, 16, 152}) cand.push_back({0, 0, 0, sm, lr, 1, 0, 0});
  for (int bl : {1, 2, 4}) cand.push_back({0, 0, 0, 0, 0, 2, bl, 0});
  if (mode) {  // only the shapes of one mode
    std::vector<tpc_tuning> keep;
    for (const tpc_tuning& t : cand)
      if (t.mode == mode) keep.push_back(t);
    cand.swap(keep);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  tpc_tuning best{};
  tpc_get_tuning(c, &best);
  if (mode) best.mode = mode;
  float best_t = 1e30f;
  const LaunchCfg saved = c->lc;
  auto time_cfg = [&](const tpc_tuning& t, float* us) -> tpc_status {
    tpc_status s = apply_tuning(c, t);
    if (s != TPC_OK) return s;
    std::vector<float> ts;
    for (int k = 0; k < iters + 1; ++k) {
      cudaEventRecord(e0, c->stream);
      s = tpc_track(c);
      if (s != TPC_OK) return s;
      cudaEventRecord(e1, c->stream);
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return cuda_fail(c, e, "autotune");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (k) ts.push_back(ms * 1000.f);  // first run warms up
    }
    std::sort(ts.begin(), ts.end());
    *us = ts[ts.size() / 2];
    return TPC_OK;
  };
  tpc_status st = TPC_OK;
  // lane groups, blocks and grids first (shared memory at its current value), then shared memory
  for (const tpc_tuning& t0 : cand) {
    tpc_tuning t = t0;
    if (!t.tracklet_lanes) {
      t.tracklet_lanes = best.tracklet_lanes;
      t.tracklet_block = best.tracklet_block;
      t.tracklet_blocks_per_sm = best.tracklet_blocks_per_sm;
    }
    if (!t.sort_smem) {
      t.sort_smem = best.sort_smem;
      t.link_rows = best.link_rows;
    }
    if (!t.batch_lanes) t.batch_lanes = best.batch_lanes;
    t.use_graph = best.use_graph;
    float us = 0.f;
    st = time_cfg(t, &us);
    if (st != TPC_OK) break;
    if (us < best_t) {
      best_t = us;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TPC_OK) {
    c->lc = saved;
    tpc_configure_kernels(saved.sort_smem, saved.link_smem);
    return st;
  }
  apply_tuning(c, best);
  st = tpc_track(c);
  if (st == TPC_OK && !key.empty()) tune_store(c->tune_path, key, best, best_t);
  if (best_out) *best_out = best;
  if (best_us) *best_us = best_t;
  return st;
}

extern "C" tpc_status tpc_set_grid_correction(tpc_ctx* c, const float* grid, const float* bounds, uint32_t n_sectors,
                                              int nx, int ny, int nz) {
  if (!c || !grid || !bounds || n_sectors == 0 || nx < 2 || ny < 2 || nz < 2 || nx > 1024 || ny > 1024 || nz > 1024)
    return TPC_ERR_INVALID_ARG;
  for (uint32_t s_ = 0; s_ < n_sectors; ++s_) {
    const float* B = bounds + 6 * s_;
    if (!(B[1] > B[0]) || !(B[3] > B[2]) || !(B[5] > B[4]) || !(B[0] > 0.f))
      return fail(c, TPC_ERR_INVALID_ARG, "grid bounds must be increasing, x0 > 0");
  }
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  const size_t nodes = (size_t)n_sectors * nx * ny * nz;
  std::vector<float> packed(2 * nodes);
  for (size_t k = 0; k < nodes; ++k) {  // keep (dy, dz): the pad row fixes x
    packed[2 * k] = grid[3 * k + 1];
    packed[2 * k + 1] = grid[3 * k + 2];
  }
  persist_free(c, c->grid_dev);
  persist_free(c, c->grid_bounds_dev);
  c->grid_dev = persist_alloc(c, 8 * nodes);
  c->mlp_bounds_host.assign(bounds, bounds + 6 * (size_t)n_sectors);
  c->grid_bounds_dev = persist_alloc(c, 24 * (size_t)n_sectors);
  if (!c->grid_dev || !c->grid_bounds_dev) {
    persist_free(c, c->grid_dev);
    persist_free(c, c->grid_bounds_dev);
    c->grid_dev = c->grid_bounds_dev = nullptr;
    return fail(c, TPC_ERR_OOM, "grid allocation failed");
  }
  if ((e = cudaMemcpyAsync(c->grid_dev, packed.data(), 8 * nodes, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->grid_bounds_dev, bounds, 24 * (size_t)n_sectors, cudaMemcpyHostToDevice, c->stream)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "grid upload");
  c->b.grid = (const float2*)c->grid_dev;
  c->b.grid_bounds = (const float*)c->grid_bounds_dev;
  c->b.grid_nx = nx;
  c->b.grid_ny = ny;
  c->b.grid_nz = nz;
  c->b.grid_sectors = (int)n_sectors;
  drop_graph(c);
  return TPC_OK;
}

extern "C" tpc_status tpc_set_correction(tpc_ctx* c, tpc_corr mode) {
  if (!c) return TPC_ERR_INVALID_ARG;
  if (mode != TPC_CORR_NONE && mode != TPC_CORR_GRID && mode != TPC_CORR_MLP) return TPC_ERR_INVALID_ARG;
  c->corr = mode;
  drop_graph(c);
  return TPC_OK;
}


// ---------------------------------------------------------------- MLP surrogate
namespace {
const uint32_t kMlpMagic = 0x31504C4D;  // "MLP1"

tpc_status mlp_alloc(tpc_ctx* c, int S) {
  if (c->mlp_master && c->mlp_S == S) return TPC_OK;
  if (S > 65535) return fail(c, TPC_ERR_INVALID_ARG, "the surrogate takes at most 65535 sectors");
  for (void* p : {(void*)c->mlp_master, (void*)c->mlp_m, (void*)c->mlp_v, (void*)c->mlp_partial,
                  (void*)c->mlp_loss, (void*)c->mlp_bounds, c->mlp_infer, c->mlp_work})
    persist_free(c, p);
  const size_t np = (size_t)S * tpc_mlp_stride();
  const int nblk = c->mlp_batch / 128;
  c->mlp_master = (float*)persist_alloc(c, 4 * np);
  c->mlp_m = (float*)persist_alloc(c, 4 * np);
  c->mlp_v = (float*)persist_alloc(c, 4 * np);
  c->mlp_partial = (float*)persist_alloc(c, 4 * np * nblk);
  c->mlp_loss = (float*)persist_alloc(c, 4 * (size_t)S * nblk);
  c->mlp_bounds = (float*)persist_alloc(c, 24 * (size_t)S);
  c->mlp_infer = persist_alloc(c, tpc_mlp_infer_bytes() * S);
  c->mlp_work = persist_alloc(c, tpc_mlp_work_bytes(S));
  if (!c->mlp_master || !c->mlp_m || !c->mlp_v || !c->mlp_partial || !c->mlp_loss || !c->mlp_bounds ||
      !c->mlp_infer || !c->mlp_work) {
    c->mlp_master = nullptr;
    return fail(c, TPC_ERR_OOM, "surrogate allocation failed");
  }
  c->mlp_S = S;
  c->b.mlp = nullptr;
  return TPC_OK;
}

tpc_status mlp_publish(tpc_ctx* c) {
  cudaError_t e = tpc_mlp_prepare(c->mlp_master, c->mlp_bounds, c->mlp_infer, c->mlp_S, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "surrogate prepare");
  c->b.mlp = c->mlp_infer;
  c->b.mlp_sectors = c->mlp_S;
  drop_graph(c);
  return TPC_OK;
}

tpc_status mlp_eval(tpc_ctx* c, uint64_t n_points, float* max_resid, float* rms_resid) {
  const int nblk = (int)std::max<uint64_t>(1, (n_points + 127) / 128);
  float* out = (float*)dev_alloc(c, 8 * (size_t)c->mlp_S * nblk);
  if (!out) return fail(c, TPC_ERR_OOM, "evaluation buffer");
  cudaError_t e = tpc_mlp_eval(c->mlp_master, (const float2*)c->grid_dev, c->b.grid_nx, c->b.grid_ny, c->b.grid_nz,
                               c->mlp_S, nblk, c->mlp_seed, out, c->stream);
  std::vector<float> h(2 * (size_t)c->mlp_S * nblk);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), out, 4 * h.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  // return the scratch block to the allocator (it is the last one of the batch list)
  c->blocks.pop_back();
  if (c->has_alloc)
    c->alloc.free(out, c->alloc.user);
  else
    cudaFreeAsync(out, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "surrogate evaluation");
  double mx = 0.0, ss = 0.0;
  for (size_t k = 0; k < h.size() / 2; ++k) {
    mx = std::max(mx, (double)h[2 * k]);
    ss += h[2 * k + 1];
  }
  if (max_resid) *max_resid = (float)mx;
  if (rms_resid) *rms_resid = (float)std::sqrt(ss / (128.0 * nblk * c->mlp_S));
  return TPC_OK;
}
}  // namespace

extern "C" tpc_status tpc_surrogate_train(tpc_ctx* c, uint64_t n_samples, uint64_t seed, int max_steps, float lr,
                                          float* max_resid_cm, float* rms_resid_cm) {
  if (!c || n_samples == 0 || lr < 0.f || !(lr < 1.f)) return TPC_ERR_INVALID_ARG;
  if (!c->grid_dev) return fail(c, TPC_ERR_STATE, "the surrogate learns the grid correction: set a grid first");
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  const int S = c->b.grid_sectors;
  const bool fresh = !c->mlp_master || c->mlp_S != S || c->mlp_seed != seed || c->mlp_step >= c->mlp_T;
  if (fresh) {
    tpc_status st = mlp_alloc(c, S);
    if (st != TPC_OK) return st;
    c->mlp_seed = seed;
    c->mlp_step = 0;
    c->mlp_T = std::max<uint64_t>(1, n_samples / (uint64_t)c->mlp_batch);
    c->mlp_lr = lr > 0.f ? lr : 3e-2f;
    if ((e = tpc_mlp_init(c->mlp_master, c->mlp_m, c->mlp_v, S, seed, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c->mlp_bounds, c->mlp_bounds_host.data(), 24 * (size_t)S, cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "surrogate init");
  }
  const uint64_t end = max_steps > 0 ? std::min<uint64_t>(c->mlp_T, c->mlp_step + (uint64_t)max_steps) : c->mlp_T;
  e = tpc_mlp_train_steps(c->mlp_work, c->mlp_step, c->mlp_T, c->mlp_lr, end - c->mlp_step, c->mlp_master, c->mlp_m,
                          c->mlp_v, c->mlp_partial, c->mlp_loss, (const float2*)c->grid_dev, c->b.grid_nx,
                          c->b.grid_ny, c->b.grid_nz, S, c->mlp_batch, seed, capturable(c->stream), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "surrogate steps");
  c->mlp_step = end;
  tpc_status st = mlp_publish(c);
  if (st != TPC_OK) return st;
  float mx = 0.f, rms = 0.f;
  st = mlp_eval(c, 8192, &mx, &rms);
  if (st != TPC_OK) return st;
  if (max_resid_cm) *max_resid_cm = mx;
  if (rms_resid_cm) *rms_resid_cm = rms;
  if (!std::isfinite(rms)) return fail(c, TPC_ERR_BAD_INPUT, "training diverged (non-finite residual): lower lr");
  return TPC_OK;
}

extern "C" tpc_status tpc_surrogate_eval(tpc_ctx* c, uint64_t n_points, float* max_resid_cm, float* rms_resid_cm) {
  if (!c || n_points == 0) return TPC_ERR_INVALID_ARG;
  if (!c->mlp_master || !c->grid_dev) return fail(c, TPC_ERR_STATE, "needs a trained surrogate and its grid");
  return mlp_eval(c, n_points, max_resid_cm, rms_resid_cm);
}

extern "C" tpc_status tpc_surrogate_params(tpc_ctx* c, int sector, float* out, int n) {
  if (!c || !out || n < tpc_mlp_nparams()) return TPC_ERR_INVALID_ARG;
  if (!c->mlp_master || sector < 0 || sector >= c->mlp_S) return fail(c, TPC_ERR_STATE, "no surrogate for sector");
  cudaError_t e = cudaMemcpyAsync(out, c->mlp_master + (size_t)sector * tpc_mlp_stride(), 4 * tpc_mlp_nparams(),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? TPC_OK : cuda_fail(c, e, "surrogate params");
}

extern "C" tpc_status tpc_surrogate_set_params(tpc_ctx* c, int sector, const float* in, int n) {
  if (!c || !in || n < tpc_mlp_nparams()) return TPC_ERR_INVALID_ARG;
  if (!c->grid_dev) return fail(c, TPC_ERR_STATE, "set a grid first (it fixes the sectors and input bounds)");
  const int S = c->b.grid_sectors;
  if (sector < 0 || sector >= S) return TPC_ERR_INVALID_ARG;
  if (!c->mlp_master || c->mlp_S != S) {
    tpc_status st = mlp_alloc(c, S);
    if (st != TPC_OK) return st;
    cudaError_t e = tpc_mlp_init(c->mlp_master, c->mlp_m, c->mlp_v, S, 0, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->mlp_bounds, c->mlp_bounds_host.data(), 24 * (size_t)S, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "surrogate init");
    c->mlp_step = c->mlp_T = 0;
  }
  cudaError_t e = cudaMemcpyAsync(c->mlp_master + (size_t)sector * tpc_mlp_stride(), in, 4 * tpc_mlp_nparams(),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "surrogate params");
  return mlp_publish(c);
}

extern "C" tpc_status tpc_surrogate_grad(tpc_ctx* c, int sector, uint64_t seed, uint64_t step, int batch, float* grad,
                                         int n, float* loss) {
  if (!c || !grad || n < tpc_mlp_nparams() || batch < 128 || batch % 128 || batch > c->mlp_batch)
    return TPC_ERR_INVALID_ARG;
  if (!c->mlp_master || !c->grid_dev || sector < 0 || sector >= c->mlp_S)
    return fail(c, TPC_ERR_STATE, "needs surrogate parameters and the grid");
  cudaError_t e = tpc_mlp_grad_only(c->mlp_work, c->mlp_master, c->mlp_partial, c->mlp_loss, (const float2*)c->grid_dev,
                                    c->b.grid_nx, c->b.grid_ny, c->b.grid_nz, c->mlp_S, batch, seed, step, c->stream);
  const int nblk = batch / 128, np = tpc_mlp_nparams(), stride = tpc_mlp_stride();
  std::vector<float> part((size_t)nblk * stride), lv(nblk);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), c->mlp_partial + (size_t)sector * nblk * stride, 4 * part.size(),
                        cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lv.data(), c->mlp_loss + (size_t)sector * nblk, 4 * lv.size(), cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "surrogate gradient");
  for (int p = 0; p < np; ++p) {
    double g = 0.0;
    for (int k = 0; k < nblk; ++k) g += part[(size_t)k * stride + p];
    grad[p] = (float)g;
  }
  if (loss) {
    double l = 0.0;
    for (int k = 0; k < nblk; ++k) l += lv[k];
    *loss = (float)(l / batch);
  }
  return TPC_OK;
}

extern "C" tpc_status tpc_surrogate_save(tpc_ctx* c, const char* path) {
  if (!c || !path) return TPC_ERR_INVALID_ARG;
  if (!c->mlp_master) return fail(c, TPC_ERR_STATE, "no surrogate to save");
  const size_t np = (size_t)c->mlp_S * tpc_mlp_stride();
  std::vector<float> w(np), m(np), v(np), bnd(6 * (size_t)c->mlp_S);
  cudaError_t e = cudaMemcpyAsync(w.data(), c->mlp_master, 4 * np, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m.data(), c->mlp_m, 4 * np, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.data(), c->mlp_v, 4 * np, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bnd.data(), c->mlp_bounds, 24 * (size_t)c->mlp_S, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "surrogate save");
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(c, TPC_ERR_INVALID_ARG, std::string("cannot write ") + path);
  const uint64_t hdr[8] = {kMlpMagic, (uint64_t)c->mlp_S, (uint64_t)tpc_mlp_stride(), c->mlp_seed, c->mlp_step,
                           c->mlp_T, (uint64_t)c->mlp_batch, 0};
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(&c->mlp_lr, 4, 1, f) == 1 &&
            std::fwrite(bnd.data(), 4, bnd.size(), f) == bnd.size() && std::fwrite(w.data(), 4, np, f) == np &&
            std::fwrite(m.data(), 4, np, f) == np && std::fwrite(v.data(), 4, np, f) == np;
  ok &= std::fclose(f) == 0;
  return ok ? TPC_OK : fail(c, TPC_ERR_INVALID_ARG, "surrogate write failed");
}

extern "C" tpc_status tpc_surrogate_load(tpc_ctx* c, const char* path) {
  if (!c || !path) return TPC_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(c, TPC_ERR_INVALID_ARG, std::string("cannot read ") + path);
  uint64_t hdr[8];
  float lr = 0.f;
  bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == kMlpMagic && hdr[2] == (uint64_t)tpc_mlp_stride() &&
            hdr[1] > 0 && hdr[1] < 4096 && hdr[6] >= 128 && hdr[6] % 128 == 0 && hdr[6] <= (1u << 20) &&
            std::fread(&lr, 4, 1, f) == 1;
  if (!ok) {
    std::fclose(f);
    return fail(c, TPC_ERR_INVALID_ARG, "not a surrogate checkpoint");
  }
  const int S = (int)hdr[1];
  const size_t np = (size_t)S * tpc_mlp_stride();
  std::vector<float> w(np), m(np), v(np), bnd(6 * (size_t)S);
  ok = std::fread(bnd.data(), 4, bnd.size(), f) == bnd.size() && std::fread(w.data(), 4, np, f) == np &&
       std::fread(m.data(), 4, np, f) == np && std::fread(v.data(), 4, np, f) == np;
  std::fclose(f);
  if (!ok) return fail(c, TPC_ERR_INVALID_ARG, "truncated surrogate checkpoint");
  cudaError_t e = cudaSetDevice(c->cfg.device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  if (hdr[6] < 128 || hdr[6] > (1u << 20) || hdr[6] % 128) return fail(c, TPC_ERR_INVALID_ARG, "bad batch in checkpoint");
  c->mlp_batch = (int)hdr[6];
  if (c->mlp_S != S) c->mlp_master = nullptr;
  tpc_status st = mlp_alloc(c, S);
  if (st != TPC_OK) return st;
  c->mlp_seed = hdr[3];
  c->mlp_step = hdr[4];
  c->mlp_T = hdr[5];
  c->mlp_lr = lr;
  if ((e = cudaMemcpyAsync(c->mlp_master, w.data(), 4 * np, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->mlp_m, m.data(), 4 * np, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->mlp_v, v.data(), 4 * np, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->mlp_bounds, bnd.data(), 24 * (size_t)S, cudaMemcpyHostToDevice, c->stream)) !=
          cudaSuccess)
    return cuda_fail(c, e, "surrogate upload");
  return mlp_publish(c);
}

// ---- cluster codec (Sec. 4, step 2) ----

namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Byte offsets of the 7 input and 7 code arrays of n clusters in one staging block.
void codec_layout(uint64_t n, size_t off[15]) {
  static const int sz[14] = {4, 4, 4, 4, 4, 4, 4, 2, 4, 1, 2, 2, 1, 1};
  size_t o = 0;
  for (int i = 0; i < 14; ++i) {
    off[i] = o;
    o += align256((size_t)n * sz[i]);
  }
  off[14] = o;
}

}  // namespace

extern "C" tpc_status tpc_encode_clusters(tpc_ctx* c, const tpc_cluster_props* in, const tpc_cluster_codes* out,
                                          int on_device, uint64_t* n_bad) {
  if (!c || !in || !out) return fail(c, TPC_ERR_INVALID_ARG, "null argument");
  if (n_bad) *n_bad = 0;
  const uint64_t n = in->n;
  if (n == 0) return TPC_OK;
  if (n > (1ull << 40)) return fail(c, TPC_ERR_INVALID_ARG, "too many clusters");
  if (!in->y || !in->z || !in->row || !in->q_tot || !in->q_max || !in->sigma_y || !in->sigma_z || !out->y ||
      !out->z || !out->row || !out->q_tot || !out->q_max || !out->sigma_y || !out->sigma_z)
    return fail(c, TPC_ERR_INVALID_ARG, "null array");
  cudaError_t e;
  if (!c->codec_bad) {
    c->codec_bad = (unsigned long long*)persist_alloc(c, 256);
    if (!c->codec_bad) return fail(c, TPC_ERR_OOM, "codec counter");
  }
  if ((e = cudaMemsetAsync(c->codec_bad, 0, 8, c->stream)) != cudaSuccess) return cuda_fail(c, e, "codec counter");
  CodecIn di{in->y, in->z, in->row, in->q_tot, in->q_max, in->sigma_y, in->sigma_z};
  CodecOut dout{out->y, out->z, out->row, out->q_tot, out->q_max, out->sigma_y, out->sigma_z};
  size_t off[15];
  if (!on_device) {
    codec_layout(n, off);
    if (n > c->codec_cap) {
      persist_free(c, c->codec_stage);
      c->codec_stage = nullptr;
      c->codec_cap = 0;
      uint64_t cap = std::max<uint64_t>(n, 1 << 16);
      size_t o2[15];
      codec_layout(cap, o2);
      c->codec_stage = persist_alloc(c, o2[14]);
      if (!c->codec_stage) return fail(c, TPC_ERR_OOM, "codec staging");
      c->codec_cap = cap;
    }
    char* base = (char*)c->codec_stage;
    const void* src[7] = {in->y, in->z, in->row, in->q_tot, in->q_max, in->sigma_y, in->sigma_z};
    for (int i = 0; i < 7; ++i)
      if ((e = cudaMemcpyAsync(base + off[i], src[i], 4 * n, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "codec upload");
    di = CodecIn{(const float*)(base + off[0]), (const float*)(base + off[1]), (const int*)(base + off[2]),
                 (const float*)(base + off[3]), (const float*)(base + off[4]), (const float*)(base + off[5]),
                 (const float*)(base + off[6])};
    dout = CodecOut{(int16_t*)(base + off[7]), (int*)(base + off[8]), (uint8_t*)(base + off[9]),
                    (uint16_t*)(base + off[10]), (uint16_t*)(base + off[11]), (uint8_t*)(base + off[12]),
                    (uint8_t*)(base + off[13])};
  }
  if ((e = launch_encode(di, dout, (long long)n, c->cfg.n_rows, c->codec_bad, c->lc.num_sms, c->stream)) !=
      cudaSuccess)
    return cuda_fail(c, e, "codec launch");
  if (!on_device) {
    char* base = (char*)c->codec_stage;
    void* dst[7] = {out->y, out->z, out->row, out->q_tot, out->q_max, out->sigma_y, out->sigma_z};
    static const int w[7] = {2, 4, 1, 2, 2, 1, 1};
    for (int i = 0; i < 7; ++i)
      if ((e = cudaMemcpyAsync(dst[i], base + off[7 + i], (size_t)w[i] * n, cudaMemcpyDeviceToHost, c->stream)) !=
          cudaSuccess)
        return cuda_fail(c, e, "codec download");
  } else if (!n_bad) {
    return TPC_OK;
  }
  unsigned long long bad = 0;
  if ((e = cudaMemcpyAsync(&bad, c->codec_bad, 8, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "codec sync");
  if (n_bad) *n_bad = bad;
  if (bad) return fail(c, TPC_ERR_BAD_INPUT, "a cluster has a bad row or a non-finite value");
  return TPC_OK;
}

// ---- cluster association, protection and removal masks (Sec. 4) ----

extern "C" tpc_status tpc_cluster_masks(tpc_ctx* c, const tpc_mask_params* prm, const tpc_track_t* tracks,
                                        uint64_t n_tracks, const uint32_t* cluster_ids, uint64_t n_ids,
                                        const uint8_t* leg, int on_device, uint8_t* mask, int32_t* owner) {
  if (c && c->frame_src)
    return fail(c, TPC_ERR_STATE, "the data-reduction calls take a batch loaded by tpc_load_clusters, not a frame");
  if (!c || !mask) return fail(c, TPC_ERR_INVALID_ARG, "null argument");
  if (!c->tracked) return fail(c, TPC_ERR_STATE, "tpc_cluster_masks before tpc_track");
  const tpc_mask_params def{1.5f, 0.05f, 70.0f};
  const tpc_mask_params P = prm ? *prm : def;
  if (!(P.tube_cm >= 0.f) || !std::isfinite(P.tube_cm) || !(P.min_pt_gev > 0.f) || !std::isfinite(P.min_pt_gev) ||
      !(P.max_incl_deg > 0.f) || !(P.max_incl_deg <= 90.f))
    return fail(c, TPC_ERR_INVALID_ARG, "mask parameters out of range");
  if (tracks && ((n_tracks && !cluster_ids) || n_tracks > 0x7fffffffull || n_ids > 0xffffffffull))
    return fail(c, TPC_ERR_INVALID_ARG, "track arrays");
  const long long N = c->b.N;
  if (N == 0) return TPC_OK;
  cudaError_t e;
  // association words: zero on entry (each call's second pass clears what the first set)
  if ((uint64_t)N > c->mask_cap || !c->mask_assoc) {
    persist_free(c, c->mask_assoc);
    c->mask_assoc = nullptr;
    c->mask_cap = 0;
    const uint64_t cap = std::max<uint64_t>((uint64_t)N, 1 << 16);
    c->mask_assoc = (unsigned long long*)persist_alloc(c, 8 * cap);
    if (!c->mask_assoc) return fail(c, TPC_ERR_OOM, "mask words");
    c->mask_cap = cap;
    c->mask_dirty = true;
  }
  if (c->mask_dirty) {
    if ((e = cudaMemsetAsync(c->mask_assoc, 0, 8 * (size_t)c->mask_cap, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "mask words");
    c->mask_dirty = false;
  }
  MaskArgs a{};
  a.rows = c->b.rows;
  a.first = c->b.first;
  a.s_hit = c->b.s_hit;
  a.row = c->b.row;
  a.N = (int)N;
  a.I = c->b.I;
  a.assoc = c->mask_assoc;
  a.tube = P.tube_cm;
  a.max_qpt = (float)(1.0 / (double)P.min_pt_gev);
  a.max_snp = (float)std::sin((double)P.max_incl_deg * M_PI / 180.0);
  a.err = c->b.err;
  a.mask = mask;
  a.owner = owner;
  a.leg = leg;
  if (!tracks) {  // the context's own output of the last tpc_track(): counts read on the device
    a.trk = c->b.trk;
    a.ids = c->b.trk_ids;
    a.counts = c->b.counts;
  } else {
    a.trk = tracks;
    a.ids = cluster_ids;
    a.n_trk = (long long)n_tracks;
    a.n_ids = (long long)n_ids;
  }
  char* st = nullptr;
  size_t off_trk = 0, off_ids = 0, off_leg = 0, off_mask = 0, off_own = 0;
  if (!on_device) {  // stage the host arrays
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    const uint64_t nt = tracks ? n_tracks : (leg ? n_tracks : 0);
    off_trk = 0;
    off_ids = off_trk + al(tracks ? sizeof(tpc_track_t) * n_tracks : 0);
    off_leg = off_ids + al(tracks ? 4 * n_ids : 0);
    off_mask = off_leg + al(leg ? nt : 0);
    off_own = off_mask + al((size_t)N);
    const size_t total = off_own + al(owner ? 4 * (size_t)N : 0);
    if (total > c->mask_stage_bytes) {
      persist_free(c, c->mask_stage);
      c->mask_stage = persist_alloc(c, total);
      c->mask_stage_bytes = c->mask_stage ? total : 0;
      if (!c->mask_stage) return fail(c, TPC_ERR_OOM, "mask staging");
    }
    st = (char*)c->mask_stage;
    if (tracks && n_tracks &&
        (e = cudaMemcpyAsync(st + off_trk, tracks, sizeof(tpc_track_t) * n_tracks, cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "track upload");
    if (tracks && n_ids &&
        (e = cudaMemcpyAsync(st + off_ids, cluster_ids, 4 * n_ids, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "id upload");
    if (leg && nt && (e = cudaMemcpyAsync(st + off_leg, leg, nt, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "leg upload");
    if (tracks) {
      a.trk = st + off_trk;
      a.ids = (const uint32_t*)(st + off_ids);
    }
    if (leg) a.leg = (const uint8_t*)(st + off_leg);
    a.mask = (uint8_t*)(st + off_mask);
    a.owner = owner ? (int*)(st + off_own) : nullptr;
  }
  c->mask_timed = c->have_events;
  if ((e = launch_masks(a, c->par, c->lc.num_sms, c->stream, c->have_events ? c->mask_ev : nullptr)) != cudaSuccess) {
    c->mask_dirty = true;
    return cuda_fail(c, e, "mask launch");
  }
  if (on_device) return TPC_OK;
  if ((e = cudaMemcpyAsync(mask, a.mask, (size_t)N, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (owner && (e = cudaMemcpyAsync(owner, a.owner, 4 * (size_t)N, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess))
    return cuda_fail(c, e, "mask download");
  unsigned int err = 0;
  if ((e = cudaMemcpyAsync(&err, c->b.err, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "mask sync");
  if (err & TPC_DERR_BAD_TRACK)
    return fail(c, TPC_ERR_BAD_INPUT, "a track refers to an item or cluster out of range (skipped)");
  return TPC_OK;
}

// ---- compression (Sec. 4, steps 3 and 4) ----

namespace {

// persistent buffer slot i with at least `bytes` bytes (contents not kept on growth)
void* cmp_buffer(tpc_ctx* c, int i, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  if (c->cmp_cap[i] >= bytes) return c->cmp_buf[i];
  persist_free(c, c->cmp_buf[i]);
  c->cmp_buf[i] = persist_alloc(c, bytes + bytes / 4);
  c->cmp_cap[i] = c->cmp_buf[i] ? bytes + bytes / 4 : 0;
  return c->cmp_buf[i];
}

}  // namespace

extern "C" tpc_status tpc_compress(tpc_ctx* c, const tpc_cluster_charges* ch, const tpc_track_t* tracks,
                                   uint64_t n_tracks, const uint32_t* cluster_ids, uint64_t n_ids, const uint8_t* keep,
                                   int on_device, uint8_t* out, uint64_t cap, uint64_t* size) {
  if (c && c->frame_src)
    return fail(c, TPC_ERR_STATE, "the data-reduction calls take a batch loaded by tpc_load_clusters, not a frame");
  if (!c || !ch || !size) return fail(c, TPC_ERR_INVALID_ARG, "null argument");
  if (!c->tracked) return fail(c, TPC_ERR_STATE, "tpc_compress before tpc_track");
  *size = 0;
  const long long N = c->b.N;
  if (N > 0 && (!ch->q_tot || !ch->q_max || !ch->sigma_y || !ch->sigma_z))
    return fail(c, TPC_ERR_INVALID_ARG, "null charge array");
  if (tracks && n_tracks && !cluster_ids) return fail(c, TPC_ERR_INVALID_ARG, "null cluster ids");
  if (cap && !out) return fail(c, TPC_ERR_INVALID_ARG, "null output");
  cudaError_t e;
  // tracks: the context's own (their count read back) or the caller's (staged if on the host)
  const void* trk;
  const uint32_t* ids;
  long long nt, ni;
  if (!tracks) {
    unsigned long long cnt[2];
    if ((e = cudaMemcpyAsync(cnt, c->b.counts, 16, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "track counts");
    trk = c->b.trk;
    ids = c->b.trk_ids;
    nt = (long long)cnt[0];
    ni = (long long)cnt[1];
  } else if (on_device) {
    trk = tracks;
    ids = cluster_ids;
    nt = (long long)n_tracks;
    ni = (long long)n_ids;
  } else {
    nt = (long long)n_tracks;
    ni = (long long)n_ids;
    void* t = cmp_buffer(c, 0, sizeof(tpc_track_t) * (size_t)nt);
    void* d = cmp_buffer(c, 1, 4 * (size_t)ni);
    if (!t || !d) return fail(c, TPC_ERR_OOM, "track staging");
    if ((nt && (e = cudaMemcpyAsync(t, tracks, sizeof(tpc_track_t) * nt, cudaMemcpyHostToDevice, c->stream)) !=
                   cudaSuccess) ||
        (ni && (e = cudaMemcpyAsync(d, cluster_ids, 4 * ni, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess))
      return cuda_fail(c, e, "track upload");
    trk = t;
    ids = (const uint32_t*)d;
  }
  const float* q[4] = {ch->q_tot, ch->q_max, ch->sigma_y, ch->sigma_z};
  if (!on_device && N > 0) {
    float* st = (float*)cmp_buffer(c, 2, 16 * (size_t)N);
    if (!st) return fail(c, TPC_ERR_OOM, "charge staging");
    for (int k = 0; k < 4; ++k) {
      if ((e = cudaMemcpyAsync(st + k * N, q[k], 4 * N, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "charge upload");
      q[k] = st + k * N;
    }
  }
  const uint8_t* d_keep = keep;
  if (keep && !on_device && N > 0) {
    uint8_t* kb = (uint8_t*)cmp_buffer(c, 42, (size_t)N);
    if (!kb) return fail(c, TPC_ERR_OOM, "keep staging");
    if ((e = cudaMemcpyAsync(kb, keep, (size_t)N, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "keep upload");
    d_keep = kb;
  }
  // sorted positions: one per loaded cluster (those of clusters left out of the binning are unused)
  const int NR = c->cfg.n_rows, I = c->b.I;
  const long long P = N;
  const long long NN = std::max<long long>(N, 1), NA = std::max<long long>(std::max(N, ni), 1);
  CmpArgs a{};
  a.rows = c->b.rows;
  a.s_hit = c->b.s_hit;
  a.y = c->b.y;
  a.z = c->b.z;
  a.row = c->b.row;
  a.N = (int)N;
  a.I = I;
  a.P = (int)P;
  a.qt = q[0];
  a.qm = q[1];
  a.sy = q[2];
  a.sz = q[3];
  a.keep = d_keep;
  a.trk = trk;
  a.ids = ids;
  a.counts = nullptr;
  a.n_trk = nt;
  a.n_ids = ni;
  a.err = c->b.err;
  a.attached = (uint8_t*)cmp_buffer(c, 3, NN);
  a.kpos = (int*)cmp_buffer(c, 4, 4 * (size_t)(P + 1));
  a.unatt_id = (int*)cmp_buffer(c, 5, 4 * (size_t)NN);
  a.unatt_first = (uint8_t*)cmp_buffer(c, 6, NN);
  a.trk_n = (int*)cmp_buffer(c, 7, 4 * (size_t)(nt + 1));
  const long long len_cap[TPC_CMP_STREAMS] = {(long long)I * NR, NN, NN, NA, NA, NA, NN + NA, NN + NA, NN + NA, NN + NA,
                                              std::max<long long>(nt, 1)};
  for (int k = 0; k < TPC_CMP_STREAMS; ++k)
    a.val[k] = (unsigned long long*)cmp_buffer(c, 8 + k, 8 * (size_t)len_cap[k]);
  a.vmax = (unsigned long long*)cmp_buffer(c, 19, 8 * TPC_CMP_STREAMS);
  a.hist = (unsigned long long*)cmp_buffer(c, 20, 8ull * TPC_CMP_STREAMS * 2048);
  a.scan_tmp = (int*)cmp_buffer(c, 21, 4 * (size_t)(P / 8192 + nt / 8192 + 8));
  a.rec = (int4*)cmp_buffer(c, 32, 16 * (size_t)NN);
  if (!a.rec) return fail(c, TPC_ERR_OOM, "compression buffers");
  for (int k = 3; k <= 21; ++k)
    if (!c->cmp_buf[k]) return fail(c, TPC_ERR_OOM, "compression buffers");
  unsigned int err0 = 0;
  if ((e = cudaMemcpyAsync(&err0, c->b.err, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "error word");
  const bool timed = c->have_events;
  if (timed) cudaEventRecord(c->cmp_ev[0], c->stream);
  if ((e = cmp_symbols(a, c->par, c->lc.num_sms, c->stream)) != cudaSuccess) return cuda_fail(c, e, "symbols");
  if (timed) cudaEventRecord(c->cmp_ev[1], c->stream);
  // stream lengths and largest values
  unsigned long long vmax[TPC_CMP_STREAMS];
  int n_un = 0, n_att = 0;
  unsigned int err = 0;
  if ((e = cudaMemcpyAsync(vmax, a.vmax, sizeof(vmax), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&n_un, a.kpos + P, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&n_att, a.trk_n + nt, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&err, c->b.err, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "stream sizes");
  if ((err & ~err0) & TPC_DERR_BAD_TRACK) return fail(c, TPC_ERR_BAD_INPUT, "a track refers to an item, cluster or row out of range");
  const long long stream_n[TPC_CMP_STREAMS] = {(long long)I * NR, n_un, n_un, n_att, n_att, n_att, (long long)n_un + n_att,
                                               (long long)n_un + n_att, (long long)n_un + n_att,
                                               (long long)n_un + n_att, nt};
  // planes and chunks
  std::vector<CmpPlane> planes;
  std::vector<int> plane_stream, chunk_plane, stream_planes(TPC_CMP_STREAMS);
  long long scratch = 0, bound = 56 + 12 * TPC_CMP_STREAMS + 28 * nt;
  int n_chunks = 0;
  for (int s = 0; s < TPC_CMP_STREAMS; ++s) {
    int np = 1;
    while (np < 8 && (vmax[s] >> (8 * np))) ++np;
    stream_planes[s] = np;
    const int nch = (int)((stream_n[s] + TPC_CMP_CHUNK - 1) / TPC_CMP_CHUNK);
    for (int p = 0; p < np; ++p) {
      planes.push_back(CmpPlane{a.val[s], stream_n[s], p, n_chunks, scratch});
      plane_stream.push_back(s);
      for (int k = 0; k < nch; ++k) chunk_plane.push_back((int)planes.size() - 1);
      n_chunks += nch;
      scratch += (long long)nch * (TPC_CMP_CHUNK + 64);
      bound += 516 + 4ll * nch + 2ll * (stream_n[s] + 64ll * nch);
    }
  }
  const int NP = (int)planes.size();
  CmpPlane* d_planes = (CmpPlane*)cmp_buffer(c, 22, sizeof(CmpPlane) * NP);
  int* d_pstream = (int*)cmp_buffer(c, 23, 4 * (size_t)NP + 4 * TPC_CMP_STREAMS + 8 * TPC_CMP_STREAMS + 16);
  int* d_cplane = (int*)cmp_buffer(c, 24, 4 * (size_t)std::max(n_chunks, 1));
  uint16_t* d_ftab = (uint16_t*)cmp_buffer(c, 25, 1024 * (size_t)NP);
  uint16_t* d_scratch = (uint16_t*)cmp_buffer(c, 26, 2 * (size_t)std::max<long long>(scratch, 1));
  long long* d_cptr = (long long*)cmp_buffer(c, 27, 8 * (size_t)std::max(n_chunks, 1));
  int* d_clen = (int*)cmp_buffer(c, 28, 4 * (size_t)std::max(n_chunks, 1));
  long long* d_cdst = (long long*)cmp_buffer(c, 29, 8 * (size_t)std::max(n_chunks, 1));
  uint8_t* d_blob = (uint8_t*)cmp_buffer(c, 30, (size_t)bound);
  long long* d_size = (long long*)cmp_buffer(c, 31, 16);
  for (int k = 22; k <= 31; ++k)
    if (!c->cmp_buf[k]) return fail(c, TPC_ERR_OOM, "compression buffers");
  int* d_splanes = d_pstream + NP;
  long long* d_sn = (long long*)(d_splanes + TPC_CMP_STREAMS + (((NP + TPC_CMP_STREAMS) & 1) ? 1 : 0));
  // host copies of the small tables must outlive the asynchronous uploads: wait before returning
  if ((e = cudaMemcpyAsync(d_planes, planes.data(), sizeof(CmpPlane) * NP, cudaMemcpyHostToDevice, c->stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(d_pstream, plane_stream.data(), 4 * NP, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_splanes, stream_planes.data(), 4 * TPC_CMP_STREAMS, cudaMemcpyHostToDevice, c->stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(d_sn, stream_n, 8 * TPC_CMP_STREAMS, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (n_chunks && (e = cudaMemcpyAsync(d_cplane, chunk_plane.data(), 4 * (size_t)n_chunks, cudaMemcpyHostToDevice,
                                        c->stream)) != cudaSuccess))
    return cuda_fail(c, e, "plane tables");
  if (timed) cudaEventRecord(c->cmp_ev[2], c->stream);
  if ((e = cmp_hist_high(a, c->par, c->lc.num_sms, stream_planes.data(), c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "histograms");
  if ((e = cmp_encode(d_planes, NP, n_chunks, a.hist, d_pstream, d_ftab, d_scratch, d_cptr, d_clen, d_cplane,
                      c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "rANS");
  if (timed) cudaEventRecord(c->cmp_ev[3], c->stream);
  const float kBf = c->par.kB;
  uint32_t kb;
  std::memcpy(&kb, &kBf, 4);
  const double xmin = c->cfg.row_x_min, xmax = c->cfg.row_x_max;
  if (timed) cudaEventRecord(c->cmp_ev[4], c->stream);
  if ((e = cmp_layout(d_planes, NP, d_splanes, d_sn, d_ftab, d_scratch, d_cptr, d_clen, n_chunks, trk, nt, kb, xmin,
                      xmax, I, NR, n_un, n_att, d_blob, d_size, d_cdst, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "layout");
  if (timed) cudaEventRecord(c->cmp_ev[5], c->stream);
  c->cmp_timed = timed;
  long long sz[2] = {0, 0};
  if ((e = cudaMemcpyAsync(sz, d_size, 16, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "blob size");
  *size = (uint64_t)sz[0];
  if ((uint64_t)sz[0] > cap) return fail(c, TPC_ERR_CAPACITY, "output buffer too small");
  if ((e = cudaMemcpyAsync(out, d_blob, (size_t)sz[0], on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "blob copy");
  return TPC_OK;
}

// ---- sector-track merger ----

extern "C" tpc_status tpc_merge_tracks(tpc_ctx* c, const tpc_track_t* tracks, uint64_t n_tracks,
                                       const uint32_t* cluster_ids, uint64_t n_ids, int on_device, int32_t* link,
                                       int32_t* group, double* fit, int32_t* leg_partner, uint8_t* leg) {
  if (c && c->frame_src)
    return fail(c, TPC_ERR_STATE, "the data-reduction calls take a batch loaded by tpc_load_clusters, not a frame");
  if (!c) return TPC_ERR_INVALID_ARG;
  if (!c->tracked) return fail(c, TPC_ERR_STATE, "tpc_merge_tracks before tpc_track");
  const int I = (int)c->h_item_sector.size();
  if (I == 0 || c->h_item_event.size() != (size_t)I)
    return fail(c, TPC_ERR_STATE, "the batch has no item_sector / item_event");
  if (n_tracks && (!link || !group || !fit)) return fail(c, TPC_ERR_INVALID_ARG, "null output");
  if (tracks && n_tracks && !cluster_ids) return fail(c, TPC_ERR_INVALID_ARG, "null cluster ids");
  if (n_tracks > 0x7fffffffull) return fail(c, TPC_ERR_INVALID_ARG, "too many tracks");
  cudaError_t e;
  const void* trk;
  const uint32_t* ids;
  long long nt = (long long)n_tracks, ni = (long long)n_ids;
  if (!tracks) {
    unsigned long long cnt[2];
    if ((e = cudaMemcpyAsync(cnt, c->b.counts, 16, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "track counts");
    if (cnt[0] != n_tracks) return fail(c, TPC_ERR_INVALID_ARG, "n_tracks differs from the number of tracks");
    trk = c->b.trk;
    ids = c->b.trk_ids;
    ni = (long long)cnt[1];
  } else if (on_device) {
    trk = tracks;
    ids = cluster_ids;
  } else {
    void* t = cmp_buffer(c, 33, sizeof(tpc_track_t) * (size_t)nt);
    void* d = cmp_buffer(c, 34, 4 * (size_t)ni);
    if (!t || !d) return fail(c, TPC_ERR_OOM, "track staging");
    if ((nt && (e = cudaMemcpyAsync(t, tracks, sizeof(tpc_track_t) * nt, cudaMemcpyHostToDevice, c->stream)) !=
                   cudaSuccess) ||
        (ni && (e = cudaMemcpyAsync(d, cluster_ids, 4 * ni, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess))
      return cuda_fail(c, e, "track upload");
    trk = t;
    ids = (const uint32_t*)d;
  }
  // neighbouring items (same event and side, sector k+1 / k-1) and segments (the items of one event
  // and side, at most 18 listed, for the tan(lambda)-sorted candidate lists): once per load
  const bool legs = leg_partner || leg;
  if (!c->mrg_tab_built) {
    std::vector<int>& nb = c->mrg_nb;
    nb.assign(2 * (size_t)I, -1);
    std::vector<std::pair<uint64_t, int>> key(I);
    for (int i = 0; i < I; ++i) key[i] = {((uint64_t)c->h_item_event[i] << 32) | c->h_item_sector[i], i};
    std::sort(key.begin(), key.end());
    auto find = [&](uint32_t ev, uint32_t sec) {
      const uint64_t k = ((uint64_t)ev << 32) | sec;
      auto it = std::lower_bound(key.begin(), key.end(), std::make_pair(k, INT32_MIN));
      return (it != key.end() && it->first == k) ? it->second : -1;
    };
    for (int i = 0; i < I; ++i) {
      const uint32_t s = c->h_item_sector[i];
      if (s >= 36) continue;
      const uint32_t side = s / 18, k = s % 18;
      nb[2 * i] = find(c->h_item_event[i], side * 18 + (k + 1) % 18);
      nb[2 * i + 1] = find(c->h_item_event[i], side * 18 + (k + 17) % 18);
    }
    std::vector<int>& item_seg = c->mrg_item_seg;
    std::vector<int>& seg_items = c->mrg_seg_items;
    item_seg.assign(I, -1);
    seg_items.clear();
    std::vector<std::pair<uint64_t, int>> es(I);
    for (int i = 0; i < I; ++i)
      es[i] = {((uint64_t)c->h_item_event[i] << 1) | (c->h_item_sector[i] >= 18 ? 1u : 0u), i};
    std::sort(es.begin(), es.end());
    for (size_t lo = 0; lo < es.size();) {
      size_t hi = lo;
      while (hi < es.size() && es[hi].first == es[lo].first) ++hi;
      const size_t sg = seg_items.size() / 19;
      seg_items.resize(seg_items.size() + 19, -1);
      for (size_t j = lo, m = 0; j < hi && m < 18; ++j, ++m) seg_items[19 * sg + m] = es[j].second;
      seg_items[19 * sg + 18] = (int)(hi - lo);
      for (size_t k = lo; k < hi; ++k) item_seg[es[k].second] = (int)sg;
      lo = hi;
    }
    c->mrg_tab_built = true;
    c->mrg_tab_dev = nullptr;
  }
  const std::vector<int>& nb = c->mrg_nb;
  const std::vector<int>& item_seg = c->mrg_item_seg;
  const std::vector<int>& seg_items = c->mrg_seg_items;
  const int S = (int)(seg_items.size() / 19);
  // [nb 2I][item_seg I][seg_items 19S] from the host, then [seg_n S][seg_off S + 1][seg_ok S] on the device
  int* d_nb = (int*)cmp_buffer(c, 35, 4 * (3 * (size_t)I + 22 * (size_t)S + 1));
  int* d_lbest = (int*)cmp_buffer(c, 40, 4 * (size_t)std::max(nt, 1ll));
  int* d_first = (int*)cmp_buffer(c, 36, 4 * (size_t)(I + 1));
  double* d_geo = (double*)cmp_buffer(c, 37, (8 * 12 + 16 + 32 + 64 + 4 + 4 + 136) * (size_t)std::max(nt, 1ll));
  int* d_best = (int*)cmp_buffer(c, 38, 8 * (size_t)std::max(nt, 1ll));
  // outputs: the caller's device arrays, or staging for host arrays
  uint8_t* st = nullptr;
  const size_t o_link = 0, o_group = ((8 * (size_t)nt + 255) & ~size_t(255)),
               o_fit = o_group + ((4 * (size_t)nt + 255) & ~size_t(255));
  const size_t o_part = o_fit + 56 * (size_t)std::max(nt, 1ll), o_leg = o_part + 4 * (size_t)std::max(nt, 1ll);
  if (!on_device) st = (uint8_t*)cmp_buffer(c, 39, o_leg + (size_t)std::max(nt, 1ll));
  if (!d_nb || !d_first || !d_geo || !d_best || !d_lbest || (!on_device && !st))
    return fail(c, TPC_ERR_OOM, "merge buffers");
  if (c->mrg_tab_dev != d_nb) {  // the tables go up once per load (and again if the buffer moved)
    if ((e = cudaMemcpyAsync(d_nb, nb.data(), 8 * (size_t)I, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_nb + 2 * (size_t)I, item_seg.data(), 4 * (size_t)I, cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess ||
        (S && (e = cudaMemcpyAsync(d_nb + 3 * (size_t)I, seg_items.data(), 4 * seg_items.size(),
                                   cudaMemcpyHostToDevice, c->stream)) != cudaSuccess))
      return cuda_fail(c, e, "neighbour table");
    c->mrg_tab_dev = d_nb;
  }
  // the merger's own error word, cleared on the stream (no read of the shared one before the kernels)
  unsigned int* d_merr = (unsigned int*)cmp_buffer(c, 43, 4);
  if (!d_merr) return fail(c, TPC_ERR_OOM, "merge buffers");
  if ((e = cudaMemsetAsync(d_merr, 0, 4, c->stream)) != cudaSuccess) return cuda_fail(c, e, "error word");
  MrgArgs a{};
  a.trk = trk;
  a.ids = ids;
  a.n_trk = nt;
  a.n_ids = ni;
  a.item_sector = c->b.item_sector;
  a.item_event = c->b.item_event;
  a.nb_item = d_nb;
  a.I = I;
  a.y = c->b.y;
  a.z = c->b.z;
  a.row = c->b.row;
  a.N = c->b.N;
  a.kB = 0.299792458e-2 * (double)c->cfg.bz_tesla;
  a.kB3_hi = (float)(3.0 * a.kB);
  a.kB3_lo = (float)(3.0 * a.kB - (double)a.kB3_hi);
  a.item_first = d_first;
  a.geo = d_geo;
  a.pre = (float4*)(d_geo + 12 * (size_t)std::max(nt, 1ll));  // 16-byte aligned: 96 bytes per track before it
  a.geo32 = a.pre + std::max(nt, 1ll);
  a.geof2 = a.geo32 + 2 * std::max(nt, 1ll);
  a.sidx = (int*)(a.geof2 + 4 * std::max(nt, 1ll));
  a.skey = (unsigned*)(a.sidx + std::max(nt, 1ll));
  a.fit_sums = (float*)(a.skey + std::max(nt, 1ll));  // 34 floats per track
  a.item_seg = d_nb + 2 * (size_t)I;
  a.seg_items = d_nb + 3 * (size_t)I;
  a.S = S;
  a.seg_n = d_nb + 3 * (size_t)I + 19 * (size_t)S;
  a.seg_off = a.seg_n + S;
  a.seg_ok = a.seg_off + S + 1;
  a.sort_cap = c->lc.merge_sort_cap;
  a.best = d_best;
  a.link = on_device ? link : (int*)(st + o_link);
  a.group = on_device ? group : (int*)(st + o_group);
  a.fit = on_device ? fit : (double*)(st + o_fit);
  a.legs = legs ? 1 : 0;
  a.lbest = d_lbest;
  // the partner array is needed whenever legs are asked for (the leg flags derive from it)
  a.partner = !legs ? nullptr : (on_device && leg_partner ? leg_partner : (int*)(st ? st + o_part : nullptr));
  a.leg = !leg ? nullptr : (on_device ? leg : st + o_leg);
  if (legs && !a.partner) {  // device call without a partner array: a scratch one
    a.partner = (int*)cmp_buffer(c, 41, 4 * (size_t)std::max(nt, 1ll));
    if (!a.partner) return fail(c, TPC_ERR_OOM, "merge buffers");
  }
  a.err = d_merr;
  if ((e = launch_merge(a, c->par, c->lc.num_sms, c->stream)) != cudaSuccess) return cuda_fail(c, e, "merge");
  if (!on_device && nt &&
      ((e = cudaMemcpyAsync(link, a.link, 8 * (size_t)nt, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
       (e = cudaMemcpyAsync(group, a.group, 4 * (size_t)nt, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
       (e = cudaMemcpyAsync(fit, a.fit, 56 * (size_t)nt, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
       (leg_partner &&
        (e = cudaMemcpyAsync(leg_partner, a.partner, 4 * (size_t)nt, cudaMemcpyDeviceToHost, c->stream)) !=
            cudaSuccess) ||
       (leg && (e = cudaMemcpyAsync(leg, a.leg, (size_t)nt, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)))
    return cuda_fail(c, e, "merge download");
  unsigned int err = 0;
  if ((e = cudaMemcpyAsync(&err, d_merr, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "merge sync");
  if (err & TPC_DERR_BAD_TRACK) return fail(c, TPC_ERR_BAD_INPUT, "a track is out of range or out of item order");
  return TPC_OK;
}

extern "C" tpc_status tpc_join_loopers(tpc_ctx* c, const tpc_track_t* tracks, uint64_t n_tracks,
                                       const uint32_t* cluster_ids, uint64_t n_ids, int on_device, const int32_t* link,
                                       const int32_t* group, const int32_t* leg_partner, const uint8_t* leg,
                                       int32_t* joined, double* jfit, uint64_t* n_joined) {
  if (c && c->frame_src)
    return fail(c, TPC_ERR_STATE, "the data-reduction calls take a batch loaded by tpc_load_clusters, not a frame");
  if (!c) return TPC_ERR_INVALID_ARG;
  if (!c->tracked) return fail(c, TPC_ERR_STATE, "tpc_join_loopers before tpc_track");
  const int I = (int)c->h_item_sector.size();
  if (I == 0) return fail(c, TPC_ERR_STATE, "the batch has no item_sector");
  if (n_tracks && (!link || !group || !leg_partner || !leg || !joined || !jfit))
    return fail(c, TPC_ERR_INVALID_ARG, "null input or output");
  if (tracks && n_tracks && !cluster_ids) return fail(c, TPC_ERR_INVALID_ARG, "null cluster ids");
  if (n_tracks > 0x7fffffffull) return fail(c, TPC_ERR_INVALID_ARG, "too many tracks");
  cudaError_t e;
  const long long nt = (long long)n_tracks;
  long long ni = (long long)n_ids;
  const void* trk;
  const uint32_t* ids;
  if (!tracks) {
    unsigned long long cnt[2];
    if ((e = cudaMemcpyAsync(cnt, c->b.counts, 16, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "track counts");
    if (cnt[0] != n_tracks) return fail(c, TPC_ERR_INVALID_ARG, "n_tracks differs from the number of tracks");
    trk = c->b.trk;
    ids = c->b.trk_ids;
    ni = (long long)cnt[1];
  } else if (on_device) {
    trk = tracks;
    ids = cluster_ids;
  } else {
    void* t = cmp_buffer(c, 33, sizeof(tpc_track_t) * (size_t)nt);
    void* d = cmp_buffer(c, 34, 4 * (size_t)ni);
    if (!t || !d) return fail(c, TPC_ERR_OOM, "track staging");
    if ((nt && (e = cudaMemcpyAsync(t, tracks, sizeof(tpc_track_t) * nt, cudaMemcpyHostToDevice, c->stream)) !=
                   cudaSuccess) ||
        (ni && (e = cudaMemcpyAsync(d, cluster_ids, 4 * ni, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess))
      return cuda_fail(c, e, "track upload");
    trk = t;
    ids = (const uint32_t*)d;
  }
  const size_t m = (size_t)std::max(nt, 1ll);
  // inputs (link 8 B, group 4 B, partner 4 B, leg 1 B per track) and outputs (joined 4 B, jfit 56 B)
  const size_t i_link = 0, i_group = 8 * m, i_part = 12 * m, i_leg = 16 * m;
  const size_t o_jfit = 0, o_joined = 56 * m;
  uint8_t* in_st = nullptr;
  uint8_t* out_st = nullptr;
  if (!on_device) {
    in_st = (uint8_t*)cmp_buffer(c, 44, 17 * m);
    out_st = (uint8_t*)cmp_buffer(c, 46, 60 * m);
  }
  int* work = (int*)cmp_buffer(c, 45, 8 * m + 16);  // glab, plist, pair count
  unsigned int* d_err = (unsigned int*)cmp_buffer(c, 47, 4);
  if ((!on_device && (!in_st || !out_st)) || !work || !d_err) return fail(c, TPC_ERR_OOM, "join buffers");
  JoinArgs a{};
  if (on_device) {
    a.link = link;
    a.group = group;
    a.partner = leg_partner;
    a.leg = leg;
    a.joined = joined;
    a.jfit = jfit;
  } else {
    if (nt && ((e = cudaMemcpyAsync(in_st + i_link, link, 8 * nt, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
               (e = cudaMemcpyAsync(in_st + i_group, group, 4 * nt, cudaMemcpyHostToDevice, c->stream)) !=
                   cudaSuccess ||
               (e = cudaMemcpyAsync(in_st + i_part, leg_partner, 4 * nt, cudaMemcpyHostToDevice, c->stream)) !=
                   cudaSuccess ||
               (e = cudaMemcpyAsync(in_st + i_leg, leg, nt, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess))
      return cuda_fail(c, e, "join upload");
    a.link = (const int*)(in_st + i_link);
    a.group = (const int*)(in_st + i_group);
    a.partner = (const int*)(in_st + i_part);
    a.leg = in_st + i_leg;
    a.jfit = (double*)(out_st + o_jfit);
    a.joined = (int*)(out_st + o_joined);
  }
  a.trk = trk;
  a.ids = ids;
  a.n_ids = ni;
  a.n_trk = (int)nt;
  a.item_sector = c->b.item_sector;
  a.I = I;
  a.y = c->b.y;
  a.z = c->b.z;
  a.row = c->b.row;
  a.N = c->b.N;
  a.glab = work;
  a.plist = work + m;
  a.n_pairs = work + 2 * m;
  a.err = d_err;
  if ((e = cudaMemsetAsync(d_err, 0, 4, c->stream)) != cudaSuccess ||
      (e = launch_join(a, c->par, c->lc.num_sms, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "join");
  if (!on_device && nt &&
      ((e = cudaMemcpyAsync(joined, a.joined, 4 * (size_t)nt, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
       (e = cudaMemcpyAsync(jfit, a.jfit, 56 * (size_t)nt, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess))
    return cuda_fail(c, e, "join download");
  unsigned int err = 0;
  int np = 0;
  if ((e = cudaMemcpyAsync(&err, d_err, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&np, a.n_pairs, 4, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "join sync");
  if (err & TPC_DERR_BAD_TRACK)
    return fail(c, TPC_ERR_BAD_INPUT, "a track, group or partner is out of range, or a joined track is too large");
  if (n_joined) {  // joined tracks: the pairs whose primary is the smallest of its joined track
    std::vector<int> pl(np), gl((size_t)nt);
    *n_joined = 0;
    if (np && ((e = cudaMemcpy(pl.data(), a.plist, 4 * (size_t)np, cudaMemcpyDeviceToHost)) != cudaSuccess ||
               (e = cudaMemcpy(gl.data(), a.joined, 4 * (size_t)nt, cudaMemcpyDeviceToHost)) != cudaSuccess))
      return cuda_fail(c, e, "join count");
    std::vector<int> roots;
    for (int t : pl) roots.push_back(gl[t]);
    std::sort(roots.begin(), roots.end());
    *n_joined = (uint64_t)(std::unique(roots.begin(), roots.end()) - roots.begin());
  }
  return TPC_OK;
}

extern "C" void tpc_destroy(tpc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->cfg.device);
  free_all(c);
  while (!c->persist.empty()) persist_free(c, c->persist.back());
  if (c->have_events) {
    for (int i = 0; i <= TPC_N_STAGES; ++i) cudaEventDestroy(c->ev[i]);
    for (int i = 0; i < 3; ++i) cudaEventDestroy(c->mask_ev[i]);
    for (int i = 0; i < 6; ++i) cudaEventDestroy(c->cmp_ev[i]);
    for (int i = 0; i < 2; ++i) cudaEventDestroy(c->corr_ev[i]);
  }
  if (c->own_stream) {
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
  }
  cudaGetLastError();
  delete c;
}

extern "C" const char* tpc_last_error(const tpc_ctx* c) { return c ? c->err.c_str() : "null context"; }
