// pv_api.cu -- the C ABI declared in include/pv.h.
//
// Host side only: argument checks, context-owned scratch, dispatch to the
// fused or the plain kernels, the host-buffer entry point, and the serving
// layer (continuous batching over several CUDA streams with admission by a
// device memory pool).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pv.h"
#include "pv_kernels.cuh"

using pvdev::Consts;

namespace {

uint64_t now_ns() {
  return static_cast<uint64_t>(std::chrono::duration_cast<std::chrono::nanoseconds>(
                                   std::chrono::steady_clock::now().time_since_epoch())
                                   .count());
}

// A device buffer that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t want = need + need / 4 + 4096;
    cudaError_t err = cudaMalloc(&p, want);
    if (err != cudaSuccess) { p = nullptr; return err; }
    bytes = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

size_t round16(size_t v) { return (v + 15) / 16 * 16; }

// Carves fused-path scratch for a batch out of one buffer.
struct FusedLayout {
  size_t counter, center, cid, slot, A, W, work, total;
  int64_t work_cap;
  int64_t cls_cap[pvk::kWorkClasses];
  FusedLayout(int64_t n, int64_t n_events, int cap) {
    work_cap = 0;
    for (int c = 0; c < pvk::kWorkClasses; ++c) {
      cls_cap[c] = pvk::class_capacity(c, n, n_events, cap);
      work_cap += cls_cap[c];
    }
    size_t o = 0;
    counter = o; o += 256;
    A = o; o += round16(sizeof(float4) * n);
    W = o; o += round16(sizeof(float2) * n);
    center = o; o += round16(sizeof(int16_t) * n);
    cid = o; o += round16(sizeof(int8_t) * n);
    slot = o; o += round16(sizeof(int32_t) * n);
    work = o; o += round16(sizeof(pvk::VertexWork) * work_cap);
    total = o;
  }
  pvk::TrackScratch scratch(void* base) const {
    char* b = static_cast<char*>(base);
    pvk::TrackScratch s;
    s.center = reinterpret_cast<int16_t*>(b + center);
    s.cid = reinterpret_cast<int8_t*>(b + cid);
    s.slot = reinterpret_cast<int32_t*>(b + slot);
    s.A = reinterpret_cast<float4*>(b + A);
    s.W = reinterpret_cast<float2*>(b + W);
    s.work = reinterpret_cast<pvk::VertexWork*>(b + work);
    int64_t first = 0;
    for (int c = 0; c < pvk::kWorkClasses; ++c) {
      s.cls_base[c] = first;
      s.cls_cap[c] = static_cast<int>(cls_cap[c]);
      first += cls_cap[c];
    }
    s.counters = reinterpret_cast<int*>(b + counter);
    for (auto& c : s.stage) c = nullptr;
    return s;
  }
};

struct PlainLayout {
  size_t zpoca, sigma, center, j0, j1, hist, seed_n, seed_lo, seed_hi, seed_bin, seed_z, cid,
      slot, A, W, ev, total;
  PlainLayout(int64_t n, int64_t E, int nbins) {
    size_t o = 0;
    A = o; o += round16(sizeof(float4) * n);
    W = o; o += round16(sizeof(float2) * n);
    zpoca = o; o += round16(4 * n);
    sigma = o; o += round16(4 * n);
    center = o; o += round16(4 * n);
    j0 = o; o += round16(4 * n);
    j1 = o; o += round16(4 * n);
    cid = o; o += round16(4 * n);
    slot = o; o += round16(4 * n);
    hist = o; o += round16(4 * static_cast<size_t>(E) * nbins);
    seed_n = o; o += round16(4 * E);
    ev = o; o += round16(4 * E);
    seed_lo = o; o += round16(4 * E * PV_MAX_SEEDS);
    seed_hi = o; o += round16(4 * E * PV_MAX_SEEDS);
    seed_bin = o; o += round16(4 * E * PV_MAX_SEEDS);
    seed_z = o; o += round16(4 * E * PV_MAX_SEEDS);
    total = o;
  }
  pvk::PlainScratch scratch(void* base) const {
    char* b = static_cast<char*>(base);
    pvk::PlainScratch s;
    s.zpoca = reinterpret_cast<float*>(b + zpoca);
    s.sigma = reinterpret_cast<float*>(b + sigma);
    s.center = reinterpret_cast<int32_t*>(b + center);
    s.j0 = reinterpret_cast<int32_t*>(b + j0);
    s.j1 = reinterpret_cast<int32_t*>(b + j1);
    s.hist = reinterpret_cast<uint32_t*>(b + hist);
    s.seed_n = reinterpret_cast<int32_t*>(b + seed_n);
    s.seed_lo = reinterpret_cast<int32_t*>(b + seed_lo);
    s.seed_hi = reinterpret_cast<int32_t*>(b + seed_hi);
    s.seed_bin = reinterpret_cast<int32_t*>(b + seed_bin);
    s.seed_z = reinterpret_cast<float*>(b + seed_z);
    s.cid = reinterpret_cast<int32_t*>(b + cid);
    s.slot = reinterpret_cast<int32_t*>(b + slot);
    s.A = reinterpret_cast<float4*>(b + A);
    s.W = reinterpret_cast<float2*>(b + W);
    s.ev_status = reinterpret_cast<int32_t*>(b + ev);
    return s;
  }
};

// ---- serving --------------------------------------------------------------

// pv_run_host: event chunks in flight (measured on the nominal batch: 2
// chunks 0.64 ms per step, 3 0.65, 4 0.69, 8 0.81 -- every chunk pays its
// copies' set-up and the kernels' tail, and the host link is the bound)
constexpr int kRunHostChunks = 2;
constexpr int64_t kRunHostChunkEvents = 2048;  // fewest events per chunk
constexpr size_t kMaxQueued = 4096;            // requests waiting for admission
// the serving kernel ends after this long without an event to claim (or
// max_spin_ns if shorter); the next submit or poll starts it again
constexpr uint64_t kServeIdleNs = 2000000;

struct Request {
  uint64_t ticket = 0;
  pv_tracks tracks{};
  pv_vertices out{};
  size_t bytes = 0;
  size_t arena_off = 0;
  uint64_t t_submit = 0;   // host steady clock
  uint64_t t_done = 0;     // host steady clock (from the device's completion stamp)
  uint64_t seq = 0;        // admission number (0: not admitted)
  bool done = false;
};

// First-fit allocator over [0, size) with out-of-order frees.
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free_;   // offset -> length
  void reset(size_t s) {
    size = s;
    free_.clear();
    free_[0] = s;
  }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        size_t rest = it->second - n;
        size_t start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace

struct pv_ctx {
  int device = 0;
  pv_config cfg{};
  pv_beamline beam{};
  Consts C{};
  int n_sm = 0;
  // launch shapes: per event-size bucket, chosen by pv_autotune (default:
  // 128-thread find CTAs, 256-thread fit CTAs, occupancy-sized grids)
  pvk::LaunchCfg bucket_cfg[3];
  int find_per_sm[4][4] = {};         // [mode][64/96/128/256]
  int stage_per_sm[2] = {};           // staged find (kFindFitStaged) at 96/128 threads
  int fit_per_sm[3][2] = {};          // [accumulation mode][128/256]
  // CUDA graphs of the fused launch, keyed by its arguments
  std::map<std::string, cudaGraphExec_t> graphs;
  cudaStream_t capture_stream = nullptr;
  // scratch of the device entry points, one set per CUDA stream, so that calls
  // on different streams may overlap on the GPU
  struct StreamWs {
    DevBuf fused, plain, mv;
  };
  std::map<cudaStream_t, StreamWs> ws;
  DevBuf tpl;                         // template profiles (profile_mode TEMPLATE)
  int mv_per_sm = 0, mv_redo_per_sm = 0;
  // host-buffer entry point staging
  DevBuf host_in, host_out;
  cudaStream_t own_stream = nullptr;
  // pv_run_host's pipeline: copy-in and copy-out streams, per-chunk events and
  // the chunks' event offsets (pinned host memory)
  cudaStream_t rh_in = nullptr, rh_out = nullptr;
  cudaEvent_t rh_ev[2 * kRunHostChunks + 1] = {};
  int64_t* rh_off = nullptr;
  size_t rh_off_cap = 0;
  std::atomic<uint64_t> launches{0};
  std::string last_error;
  // serving: the persistent request loop (pv_serve.cu)
  std::mutex mu;
  DevBuf pool;                          // request scratch, handed out by the arena
  Arena arena;
  bool pool_ready = false;
  pvk::ServeCtl* sctl = nullptr;        // request ring (pinned host memory)
  pvk::ServeCtl* sctl_dev = nullptr;    // its device address
  pvk::ServeDev* sdev = nullptr;        // claim counter and per-slot counts (device)
  cudaStream_t serve_stream = nullptr;
  cudaEvent_t serve_end = nullptr;      // recorded after each launch of the kernel
  bool serve_launched = false;
  int serve_grid = 0;
  unsigned int serve_epoch = 0;         // launches of the serving kernel so far
  uint64_t published = 0;               // events published to the ring
  uint64_t next_seq = 1;                // next admission number
  uint64_t slot_cum[pvk::kServeRing] = {};
  Request* slot_req[pvk::kServeRing] = {};
  std::vector<Request*> inflight;       // admitted, not yet seen complete
  int64_t clock_offset = 0;             // device global timer minus host steady clock, ns
  uint64_t next_ticket = 1;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> requests;
};

namespace {

int fail_cuda(pv_ctx* ctx, cudaError_t err) {
  if (ctx) ctx->last_error = cudaGetErrorString(err);
  return PV_ERR_CUDA;
}

#define PV_CUDA(ctx, call)                              \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return fail_cuda(ctx, _e);   \
  } while (0)

int compute_consts(const pv_config& cfg, const pv_beamline& b, Consts* C) {
  if (!(cfg.dz > 0.0f) || !(cfg.z_max > cfg.z_min)) return PV_ERR_ARG;
  double nb = std::floor((static_cast<double>(cfg.z_max) - static_cast<double>(cfg.z_min)) /
                             static_cast<double>(cfg.dz) + 0.5);
  if (!(nb >= 1.0) || nb > PV_MAX_BINS) return PV_ERR_ARG;
  if (cfg.dip_den <= 0 || cfg.dip_num < 0) return PV_ERR_ARG;
  if (!(cfg.chi2_max > 0.0f) || cfg.max_iter < 0 || cfg.max_iter > 1000) return PV_ERR_ARG;
  if (cfg.accum_mode != PV_ACCUM_FP32 && cfg.accum_mode != PV_ACCUM_KAHAN &&
      cfg.accum_mode != PV_ACCUM_FP64)
    return PV_ERR_ARG;
  if (cfg.path != PV_PATH_FUSED && cfg.path != PV_PATH_PLAIN) return PV_ERR_ARG;
  if (!(cfg.min_integral_pp >= 0.0f) || !(cfg.min_integral_gas >= 0.0f)) return PV_ERR_ARG;
  if (cfg.split_mode != PV_SPLIT_ZORDER && cfg.split_mode != PV_SPLIT_RECURSIVE) return PV_ERR_ARG;
  if (cfg.profile_mode != PV_PROFILE_CUBIC && cfg.profile_mode != PV_PROFILE_TEMPLATE)
    return PV_ERR_ARG;
  if (!(cfg.mv_chi2_cut > 0.0f) || !(cfg.mv_dz_tol >= 0.0f) || !(cfg.mv_w_assoc > 0.0f) ||
      !(cfg.mv_w_assoc <= 1.0f) || !(cfg.mv_dup_sep2 >= 0.0f))
    return PV_ERR_ARG;
  C->z_min = cfg.z_min;
  C->dz = cfg.dz;
  {
    int ex = 0;
    float mant = std::frexp(cfg.dz, &ex);
    C->inv_dz = (mant == 0.5f) ? std::ldexp(1.0f, 1 - ex) : 0.0f;   // dz = 2^(ex-1)
  }
  C->z_gas = cfg.z_gas;
  C->sig_max_pp = cfg.sigma_max_pp;
  C->sig_max_gas = cfg.sigma_max_gas;
  C->x_b = b.x_b;
  C->y_b = b.y_b;
  C->tx_b = b.tx_b;
  C->ty_b = b.ty_b;
  C->chi2_max = cfg.chi2_max;
  C->inv_chi2_max = 1.0f / cfg.chi2_max;
  C->dchi2_tol = cfg.dchi2_tol;
  C->dz_tol = cfg.dz_tol;
  C->max_r_beam = cfg.max_r_beam;
  C->mv_ecut = static_cast<float>(std::exp(-0.5 * static_cast<double>(cfg.mv_chi2_cut)));
  C->mv_dz_tol = cfg.mv_dz_tol;
  C->mv_w_assoc = cfg.mv_w_assoc;
  C->mv_dup_sep2 = cfg.mv_dup_sep2;
  C->split_mode = cfg.split_mode;
  C->profile_mode = cfg.profile_mode;
  C->tpl = nullptr;
  C->thr = cfg.bin_threshold;
  C->t_pp = static_cast<uint32_t>(std::llround(static_cast<double>(cfg.min_integral_pp) * PV_ONE));
  C->t_gas = static_cast<uint32_t>(std::llround(static_cast<double>(cfg.min_integral_gas) * PV_ONE));
  C->dip_num = cfg.dip_num;
  C->dip_den = cfg.dip_den;
  C->min_assoc_pp = cfg.min_assoc_pp;
  C->min_assoc_gas = cfg.min_assoc_gas;
  C->min_pv_pp = cfg.min_pv_tracks_pp;
  C->min_pv_gas = cfg.min_pv_tracks_gas;
  C->nbins = static_cast<int>(nb);
  C->ntiles = (C->nbins + 31) / 32;
  // bin of z_gas by the same binary32 rule as the kernels
  volatile float diff = cfg.z_gas - cfg.z_min;
  volatile float q = diff / cfg.dz;
  int gb;
  if (!(q >= 0.0f)) gb = -1;
  else if (q >= static_cast<float>(C->nbins)) gb = C->nbins;
  else gb = static_cast<int>(q);
  C->gas_bin = gb;
  C->max_iter = cfg.max_iter;
  C->accum_mode = cfg.accum_mode;
  return PV_OK;
}

int check_tracks(const pv_tracks* t) {
  if (!t) return PV_ERR_ARG;
  if (t->n_events < 0 || t->n_tracks < 0) return PV_ERR_ARG;
  if (t->n_tracks > 0x7fffffffLL) return PV_ERR_CAPACITY;   // 32-bit track indices
  if (t->n_events > 0 && !t->event_offsets) return PV_ERR_ARG;
  if (t->n_tracks > 0) {
    const float* p[11] = {t->x, t->y, t->z, t->tx, t->ty, t->cxx, t->cxtx, t->ctxtx,
                          t->cyy, t->cyty, t->ctyty};
    for (auto q : p)
      if (!q) return PV_ERR_ARG;
  }
  return PV_OK;
}

int check_out(const pv_vertices* o, const pv_tracks* t, bool need_xyz) {
  if (!o) return PV_ERR_ARG;
  if (o->capacity < 1 || o->capacity > PV_MAX_SEEDS) return PV_ERR_ARG;
  if (t->n_events > 0 && !o->n_per_event) return PV_ERR_ARG;
  if (t->n_tracks > 0 && !o->track_vertex) return PV_ERR_ARG;
  if (t->n_events > 0 && need_xyz && (!o->x || !o->y || !o->z)) return PV_ERR_ARG;
  return PV_OK;
}

pvk::TrackPtrs track_ptrs(const pv_tracks* t) {
  pvk::TrackPtrs T;
  T.x = t->x; T.y = t->y; T.z = t->z; T.tx = t->tx; T.ty = t->ty;
  T.cxx = t->cxx; T.cxtx = t->cxtx; T.ctxtx = t->ctxtx;
  T.cyy = t->cyy; T.cyty = t->cyty; T.ctyty = t->ctyty;
  T.off = t->event_offsets;
  T.n_tracks = t->n_tracks;
  T.n_events = t->n_events;
  return T;
}

pvk::OutPtrs out_ptrs(const pv_vertices* o) {
  pvk::OutPtrs O;
  O.x = o->x; O.y = o->y; O.z = o->z; O.cov = o->cov; O.chi2 = o->chi2; O.ndof = o->ndof;
  O.n_tracks = o->n_tracks; O.n_iter = o->n_iter; O.status = o->status;
  O.bin_lo = o->bin_lo; O.bin_hi = o->bin_hi; O.bin_max = o->bin_max;
  O.n_per_event = o->n_per_event; O.event_status = o->event_status;
  O.track_vertex = o->track_vertex;
  O.cap = o->capacity;
  return O;
}

pvk::SeedPtrs seed_ptrs(const pv_vertices* s) {
  pvk::SeedPtrs S{};
  if (!s) return S;
  S.x = s->x; S.y = s->y; S.z = s->z;
  S.n_per_event = s->n_per_event;
  S.track_vertex = s->track_vertex;
  S.cap = s->capacity;
  return S;
}

int nt_index(int nt) { return nt == 64 ? 0 : (nt == 96 ? 1 : (nt == 256 ? 3 : 2)); }

int bucket_of(const pv_tracks* t) {
  double mean = t->n_events > 0 ? static_cast<double>(t->n_tracks) / t->n_events : 0.0;
  return mean < 300.0 ? 0 : (mean < 800.0 ? 1 : 2);
}

// Block sizes from the bucket's configuration, grids from occupancy, capped by
// the work there is.
pvk::LaunchCfg launch_cfg(const pv_ctx* ctx, int mode, const pv_tracks* t, int find_nt,
                          int fit_nt) {
  pvk::LaunchCfg L;
  L.find_nt = find_nt;
  L.fit_nt = fit_nt;
  int per = ctx->find_per_sm[mode][nt_index(find_nt)];
  long long g = static_cast<long long>(ctx->n_sm) * (per > 0 ? per : 1);
  if (g > t->n_events) g = t->n_events > 0 ? t->n_events : 1;
  L.find_grid = static_cast<int>(g);
  int fper = ctx->fit_per_sm[ctx->C.accum_mode][fit_nt == 128 ? 0 : 1];
  L.fit_grid = ctx->n_sm * (fper > 0 ? fper : 1);
  return L;
}

pvk::LaunchCfg chosen_cfg(const pv_ctx* ctx, int mode, const pv_tracks* t) {
  const pvk::LaunchCfg& b = ctx->bucket_cfg[bucket_of(t)];
  return launch_cfg(ctx, mode, t, b.find_nt, b.fit_nt);
}

// Enqueue the fused kernels with scratch at `base` (laid out by FusedLayout).
int enqueue_fused_cfg(pv_ctx* ctx, int mode, const pv_tracks* tracks, const pv_vertices* seeds,
                      const pv_vertices* out, void* base, const pvk::LaunchCfg& cfg,
                      cudaStream_t st) {
  FusedLayout L(tracks->n_tracks, tracks->n_events, out->capacity);
  int n = 0;
  PV_CUDA(ctx, pvk::launch_fused(mode, ctx->C, track_ptrs(tracks), seed_ptrs(seeds),
                                 out_ptrs(out), L.scratch(base), cfg, st, &n));
  ctx->launches += n;
  return PV_OK;
}

int enqueue_fused(pv_ctx* ctx, int mode, const pv_tracks* tracks, const pv_vertices* seeds,
                  const pv_vertices* out, void* base, cudaStream_t st) {
  return enqueue_fused_cfg(ctx, mode, tracks, seeds, out, base, chosen_cfg(ctx, mode, tracks), st);
}

void clear_graphs(pv_ctx* ctx) {
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
}

// The fused find+fit as a replayed CUDA graph (one per argument set).
int enqueue_fused_graph(pv_ctx* ctx, const pv_tracks* tracks, const pv_vertices* out, void* base,
                        cudaStream_t st) {
  const pvk::LaunchCfg cfg = chosen_cfg(ctx, pvk::kFindFit, tracks);
  std::string key;
  key.append(reinterpret_cast<const char*>(tracks), sizeof(pv_tracks));
  key.append(reinterpret_cast<const char*>(out), sizeof(pv_vertices));
  key.append(reinterpret_cast<const char*>(&cfg), sizeof(cfg));
  key.append(reinterpret_cast<const char*>(&base), sizeof(base));
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (ctx->graphs.size() >= 64) clear_graphs(ctx);
    if (!ctx->capture_stream)
      PV_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    PV_CUDA(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    FusedLayout L(tracks->n_tracks, tracks->n_events, out->capacity);
    int n = 0;
    cudaError_t err = pvk::launch_fused(pvk::kFindFit, ctx->C, track_ptrs(tracks), seed_ptrs(nullptr),
                                        out_ptrs(out), L.scratch(base), cfg, ctx->capture_stream, &n);
    cudaGraph_t graph = nullptr;
    cudaError_t err2 = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (err != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return fail_cuda(ctx, err); }
    if (err2 != cudaSuccess) return fail_cuda(ctx, err2);
    cudaGraphExec_t exec = nullptr;
    err = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) return fail_cuda(ctx, err);
    it = ctx->graphs.emplace(key, exec).first;
  }
  PV_CUDA(ctx, cudaGraphLaunch(it->second, st));
  ctx->launches += 2;
  return PV_OK;
}

int run_find_or_fit(pv_ctx* ctx, const pv_tracks* tracks, const pv_vertices* seeds,
                    pv_vertices* out, cudaStream_t st, int mode) {
  if (tracks->n_events == 0) return PV_OK;
  if (ctx->cfg.path == PV_PATH_PLAIN) {
    PlainLayout L(tracks->n_tracks, tracks->n_events, ctx->C.nbins);
    DevBuf& pbuf = ctx->ws[st].plain;
    PV_CUDA(ctx, pbuf.ensure(L.total));
    pvk::PlainScratch ws = L.scratch(pbuf.p);
    int n = 0;
    pvk::TrackPtrs T = track_ptrs(tracks);
    if (mode & pvk::kFind) {
      PV_CUDA(ctx, pvk::launch_plain_find(ctx->C, T, out_ptrs(out), ws, st, &n));
    }
    if (mode & pvk::kFit) {
      const pv_vertices* src = (mode & pvk::kFind) ? out : seeds;
      PV_CUDA(ctx, pvk::launch_plain_fit(ctx->C, T, seed_ptrs(src), out_ptrs(out), ws, st, &n));
    }
    ctx->launches += n;
    return PV_OK;
  }
  FusedLayout L(tracks->n_tracks, tracks->n_events, out->capacity);
  DevBuf& fbuf = ctx->ws[st].fused;
  void* before = fbuf.p;
  PV_CUDA(ctx, fbuf.ensure(L.total));
  if (fbuf.p != before) clear_graphs(ctx);   // graphs hold the old scratch
  if (ctx->cfg.use_graph && mode == pvk::kFindFit)
    return enqueue_fused_graph(ctx, tracks, out, fbuf.p, st);
  return enqueue_fused(ctx, mode, tracks, seeds, out, fbuf.p, st);
}

// The device address of pinned host memory the device can reach, or NULL
// (pageable memory, or a pointer CUDA does not know).
void* device_alias(const void* hp) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, hp) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The fused find + fit on tracks that live in host memory the device can
// address: the find kernel reads every column there once (the eight of steps
// (a)-(b) in its fill, writing them to the device copy `stage` (8 columns of
// n_tracks floats) that its fit-input pass reads back, the other three in
// that pass).
int run_staged(pv_ctx* ctx, const pv_tracks* tracks, pv_vertices* out, float* const* stage,
               cudaStream_t st) {
  if (tracks->n_events == 0) return PV_OK;
  FusedLayout L(tracks->n_tracks, tracks->n_events, out->capacity);
  DevBuf& fbuf = ctx->ws[st].fused;
  void* before = fbuf.p;
  PV_CUDA(ctx, fbuf.ensure(L.total));
  if (fbuf.p != before) clear_graphs(ctx);   // graphs hold the old scratch
  pvk::TrackScratch ws = L.scratch(fbuf.p);
  for (int c = 0; c < 8; ++c) ws.stage[c] = stage[c];
  const pvk::LaunchCfg& b = ctx->bucket_cfg[bucket_of(tracks)];
  const int nt = b.find_nt == 96 ? 96 : 128;
  pvk::LaunchCfg cfg = launch_cfg(ctx, pvk::kFindFit, tracks, nt, b.fit_nt);
  const int per = ctx->stage_per_sm[nt == 96 ? 0 : 1];
  long long g = static_cast<long long>(ctx->n_sm) * (per > 0 ? per : 1);
  cfg.find_grid = static_cast<int>(g < tracks->n_events ? g : tracks->n_events);
  int nl = 0;
  PV_CUDA(ctx, pvk::launch_fused(pvk::kFindFitStaged, ctx->C, track_ptrs(tracks), seed_ptrs(nullptr),
                                 out_ptrs(out), ws, cfg, st, &nl));
  ctx->launches += nl;
  return PV_OK;
}

// ---- serving internals (ctx->mu held) ------------------------------------

// Scratch of one request in the pool: per track its center bin, vertex, place
// in vertex order and fit inputs (31 bytes), each array 16-byte aligned.
struct ServeLayout {
  size_t center, cid, slot, A, W, total;
  explicit ServeLayout(int64_t n) {
    size_t o = 0;
    A = o; o += round16(sizeof(float4) * n);
    W = o; o += round16(sizeof(float2) * n);
    slot = o; o += round16(sizeof(int32_t) * n);
    center = o; o += round16(sizeof(int16_t) * n);
    cid = o; o += round16(sizeof(int8_t) * n);
    total = (o + 255) / 256 * 256;
  }
};

uint64_t serve_idle_ns(const pv_ctx* ctx) {
  const uint64_t lim = ctx->cfg.max_spin_ns ? ctx->cfg.max_spin_ns : 10000000000ull;
  return lim < kServeIdleNs ? lim : kServeIdleNs;
}

int ensure_pool(pv_ctx* ctx) {
  if (ctx->pool_ready) return PV_OK;
  size_t bytes = ctx->cfg.pool_bytes ? ctx->cfg.pool_bytes : (size_t(1) << 30);
  PV_CUDA(ctx, ctx->pool.ensure(bytes));
  ctx->arena.reset(ctx->pool.bytes / 256 * 256);
  void* h = nullptr;
  PV_CUDA(ctx, cudaHostAlloc(&h, sizeof(pvk::ServeCtl), cudaHostAllocMapped));
  std::memset(h, 0, sizeof(pvk::ServeCtl));
  ctx->sctl = static_cast<pvk::ServeCtl*>(h);
  void* hd = nullptr;
  PV_CUDA(ctx, cudaHostGetDevicePointer(&hd, h, 0));
  ctx->sctl_dev = static_cast<pvk::ServeCtl*>(hd);
  void* d = nullptr;
  PV_CUDA(ctx, cudaMalloc(&d, sizeof(pvk::ServeDev)));
  ctx->sdev = static_cast<pvk::ServeDev*>(d);
  PV_CUDA(ctx, cudaMemset(d, 0, sizeof(pvk::ServeDev)));
  PV_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->serve_stream, cudaStreamNonBlocking));
  PV_CUDA(ctx, cudaEventCreateWithFlags(&ctx->serve_end, cudaEventDisableTiming));
  const int per = pvk::serve_blocks_per_sm(ctx->C);
  ctx->serve_grid = ctx->n_sm * (per > 0 ? per : 1);
  // the device's global timer against the host clock: the stamp of a one-
  // thread kernel against the midpoint of the host's readings around it (the
  // closest of a few tries)
  int64_t best = -1;
  for (int i = 0; i < 5; ++i) {
    const uint64_t t0 = now_ns();
    PV_CUDA(ctx, pvk::launch_serve_clock(ctx->sctl_dev, ctx->serve_stream));
    PV_CUDA(ctx, cudaStreamSynchronize(ctx->serve_stream));
    const uint64_t t1 = now_ns();
    const uint64_t g = *reinterpret_cast<volatile uint64_t*>(&ctx->sctl->clock_ns);
    if (best < 0 || static_cast<int64_t>(t1 - t0) < best) {
      best = static_cast<int64_t>(t1 - t0);
      ctx->clock_offset = static_cast<int64_t>(g) - static_cast<int64_t>((t0 + t1) / 2);
    }
  }
  ctx->sctl->exit_code = -1;
  ctx->pool_ready = true;
  return PV_OK;
}

// Writes request r into the next ring slot and publishes its events.
void admit(pv_ctx* ctx, Request* r, size_t off) {
  const uint64_t seq = ctx->next_seq++;
  const int slot = static_cast<int>(seq % pvk::kServeRing);
  pvk::ServeDesc* d = &ctx->sctl->ring[slot];
  __atomic_store_n(&d->seq, ~0ull, __ATOMIC_RELEASE);
  char* base = static_cast<char*>(ctx->pool.p) + off;
  const ServeLayout L(r->tracks.n_tracks);
  d->T = track_ptrs(&r->tracks);
  d->O = out_ptrs(&r->out);
  d->center = reinterpret_cast<int16_t*>(base + L.center);
  d->cid = reinterpret_cast<int8_t*>(base + L.cid);
  d->slot = reinterpret_cast<int32_t*>(base + L.slot);
  d->A = reinterpret_cast<float4*>(base + L.A);
  d->W = reinterpret_cast<float2*>(base + L.W);
  d->ev_base = ctx->published;
  ctx->slot_cum[slot] += static_cast<uint64_t>(r->tracks.n_events);
  d->done_target = ctx->slot_cum[slot];
  __atomic_store_n(&d->seq, seq, __ATOMIC_RELEASE);
  ctx->published += static_cast<uint64_t>(r->tracks.n_events);
  __atomic_store_n(&ctx->sctl->published, ctx->published, __ATOMIC_RELEASE);
  r->arena_off = off;
  r->seq = seq;
  ctx->slot_req[slot] = r;
}

bool serve_running(pv_ctx* ctx) {
  if (!ctx->serve_launched) return false;
  const cudaError_t q = cudaEventQuery(ctx->serve_end);
  if (q == cudaErrorNotReady) return true;
  if (q != cudaSuccess) ctx->last_error = cudaGetErrorString(q);
  ctx->serve_launched = false;
  return false;
}

// Starts the serving kernel (if it is not running) from the oldest request
// not yet complete.
int start_server(pv_ctx* ctx) {
  if (serve_running(ctx)) return PV_OK;
  uint64_t start = ctx->next_seq;
  for (const Request* r : ctx->inflight)
    if (r->seq < start) start = r->seq;
  // a new launch: its exit count and orphan list start empty, the previous
  // launch's orphans wait to be taken
  const unsigned int epoch = ++ctx->serve_epoch;
  PV_CUDA(ctx, cudaMemsetAsync(&ctx->sdev->running, 0, sizeof(int), ctx->serve_stream));
  PV_CUDA(ctx, cudaMemsetAsync(&ctx->sdev->orph_n[epoch & 1], 0, sizeof(int), ctx->serve_stream));
  PV_CUDA(ctx, cudaMemsetAsync(&ctx->sdev->orph_take, 0, sizeof(int), ctx->serve_stream));
  PV_CUDA(ctx, pvk::launch_serve(ctx->C, ctx->sctl_dev, ctx->sdev, serve_idle_ns(ctx), start, epoch,
                                 ctx->serve_grid, ctx->serve_stream));
  PV_CUDA(ctx, cudaEventRecord(ctx->serve_end, ctx->serve_stream));
  ctx->serve_launched = true;
  ctx->launches += 1;
  return PV_OK;
}

// Retires completed requests (their pool memory returns to the arena), admits
// waiting requests that fit (any of them: a large one at the head does not
// block smaller ones behind it) and keeps the serving kernel running while
// requests are in flight.
int pump(pv_ctx* ctx) {
  size_t keep = 0;
  for (size_t i = 0; i < ctx->inflight.size(); ++i) {
    Request* r = ctx->inflight[i];
    const int s = static_cast<int>(r->seq % pvk::kServeRing);
    if (__atomic_load_n(&ctx->sctl->done_seq[s], __ATOMIC_ACQUIRE) == r->seq) {
      const uint64_t g = *reinterpret_cast<volatile uint64_t*>(&ctx->sctl->done_ns[s]);
      r->t_done = static_cast<uint64_t>(static_cast<int64_t>(g) - ctx->clock_offset);
      if (r->t_done < r->t_submit) r->t_done = r->t_submit;
      r->done = true;
      ctx->arena.release(r->arena_off, r->bytes);
      ctx->slot_req[s] = nullptr;
    } else {
      ctx->inflight[keep++] = r;
    }
  }
  ctx->inflight.resize(keep);
  bool in_flight = keep > 0;
  for (auto it = ctx->pending.begin(); it != ctx->pending.end();) {
    if (ctx->slot_req[ctx->next_seq % pvk::kServeRing]) break;   // ring full
    size_t off;
    if (!ctx->arena.alloc((*it)->bytes, &off)) {
      ++it;
      continue;
    }
    admit(ctx, *it, off);
    ctx->inflight.push_back(*it);
    in_flight = true;
    it = ctx->pending.erase(it);
  }
  if (in_flight) return start_server(ctx);
  return PV_OK;
}

}  // namespace

// ===========================================================================
// C ABI

extern "C" {

void pv_config_default(pv_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->z_min = -550.0f;
  c->z_max = 300.0f;
  c->dz = 0.25f;
  c->z_gas = -300.0f;
  c->sigma_max_pp = 1.5f;
  c->sigma_max_gas = 10.0f;
  c->min_integral_pp = 2.5f;
  c->min_integral_gas = 1.75f;
  c->bin_threshold = 205;
  c->dip_num = 4;
  c->dip_den = 5;
  c->min_assoc_pp = 3;
  c->min_assoc_gas = 2;
  c->min_pv_tracks_pp = 4;
  c->min_pv_tracks_gas = 3;
  c->chi2_max = 12.0f;
  c->dchi2_tol = 0.01f;
  c->dz_tol = 0.001f;
  c->max_iter = 10;
  c->max_r_beam = 0.3f;
  c->accum_mode = PV_ACCUM_FP32;
  c->path = PV_PATH_FUSED;
  c->use_graph = 0;
  c->reserved = 0;
  c->pool_bytes = 0;
  c->max_spin_ns = 0;
  c->mv_chi2_cut = 4.0f;
  c->mv_dz_tol = 0.0005f;
  c->mv_w_assoc = 0.5f;
  c->mv_dup_sep2 = 25.0f;
  c->split_mode = PV_SPLIT_ZORDER;
  c->profile_mode = PV_PROFILE_CUBIC;
}

int pv_init(const pv_config* cfg, const pv_beamline* beam, int device, pv_ctx** out) {
  if (!out) return PV_ERR_ARG;
  *out = nullptr;
  pv_config c;
  if (cfg) c = *cfg; else pv_config_default(&c);
  pv_beamline b{0.f, 0.f, 0.f, 0.f};
  if (beam) b = *beam;
  Consts C;
  int rc = compute_consts(c, b, &C);
  if (rc != PV_OK) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return PV_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return PV_ERR_CUDA;
  pv_ctx* ctx = new (std::nothrow) pv_ctx();
  if (!ctx) return PV_ERR_NOMEM;
  ctx->device = device;
  ctx->cfg = c;
  ctx->beam = b;
  ctx->C = C;
  if (cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      pvk::fused_setup(C.nbins) != cudaSuccess || pvk::serve_setup(C.nbins) != cudaSuccess) {
    delete ctx;
    return PV_ERR_CUDA;
  }
  if (C.profile_mode == PV_PROFILE_TEMPLATE) {
    // the x86 profile's template table, built once on the device
    int status = 1;
    if (ctx->tpl.ensure(sizeof(pvdev::TplTable)) != cudaSuccess ||
        pvk::build_template_table(static_cast<pvdev::TplTable*>(ctx->tpl.p), C.dz, 0) !=
            cudaSuccess ||
        cudaMemcpy(&status, &static_cast<pvdev::TplTable*>(ctx->tpl.p)->status, sizeof(int),
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
      ctx->tpl.release();
      delete ctx;
      return PV_ERR_CUDA;
    }
    if (status != 0) {            // bins too narrow for the widest template
      ctx->tpl.release();
      delete ctx;
      return PV_ERR_ARG;
    }
    ctx->C.tpl = static_cast<const pvdev::TplTable*>(ctx->tpl.p);
  }
  const int nts[4] = {64, 96, 128, 256};
  const int flav = pvk::flavour_of(C);
  for (int mode = 1; mode <= 3; ++mode)
    for (int i = 0; i < 4; ++i)
      ctx->find_per_sm[mode][i] = pvk::fused_blocks_per_sm(C.nbins, mode, nts[i], flav);
  for (int i = 0; i < 2; ++i)
    ctx->stage_per_sm[i] = pvk::fused_blocks_per_sm(C.nbins, pvk::kFindFitStaged, i ? 128 : 96, 0);
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 2; ++i) ctx->fit_per_sm[k][i] = pvk::fit_blocks_per_sm(k, i == 0 ? 128 : 256);
  for (int b = 0; b < 3; ++b) ctx->bucket_cfg[b] = pvk::LaunchCfg{128, 0, pvk::kFitThreads, 0};
  ctx->mv_per_sm = pvk::mv_blocks_per_sm(false);
  ctx->mv_redo_per_sm = pvk::mv_blocks_per_sm(true);
  *out = ctx;
  return PV_OK;
}

int pv_destroy(pv_ctx* ctx) {
  if (!ctx) return PV_ERR_ARG;
  cudaSetDevice(ctx->device);
  int rc = PV_OK;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    uint64_t limit = ctx->cfg.max_spin_ns ? ctx->cfg.max_spin_ns : 10000000000ull;
    uint64_t t0 = now_ns();
    // the serving kernel finishes the published requests, then sees the stop
    // request; requests still waiting for admission are dropped
    if (ctx->sctl) __atomic_store_n(&ctx->sctl->stop, 1u, __ATOMIC_RELEASE);
    while (serve_running(ctx)) {
      if (now_ns() - t0 > limit) { rc = PV_ERR_TIMEOUT; break; }
      std::this_thread::yield();
    }
    if (rc == PV_OK) {
      for (auto& kv : ctx->requests) delete kv.second;
      ctx->requests.clear();
      ctx->pending.clear();
      ctx->inflight.clear();
      if (ctx->serve_stream) cudaStreamDestroy(ctx->serve_stream);
      if (ctx->serve_end) cudaEventDestroy(ctx->serve_end);
      if (ctx->sctl) cudaFreeHost(ctx->sctl);
      if (ctx->sdev) cudaFree(ctx->sdev);
      ctx->sctl = nullptr;
      ctx->sdev = nullptr;
    }
  }
  if (rc != PV_OK) return rc;   // leave the context alive: its requests still run
  cudaDeviceSynchronize();
  clear_graphs(ctx);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  for (auto& kv : ctx->ws) {
    kv.second.fused.release();
    kv.second.plain.release();
    kv.second.mv.release();
  }
  ctx->ws.clear();
  ctx->tpl.release();
  ctx->host_in.release();
  ctx->host_out.release();
  if (ctx->rh_in) cudaStreamDestroy(ctx->rh_in);
  if (ctx->rh_out) cudaStreamDestroy(ctx->rh_out);
  for (auto& ev : ctx->rh_ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->rh_off) cudaFreeHost(ctx->rh_off);
  ctx->pool.release();
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  delete ctx;
  return PV_OK;
}

int pv_num_bins(const pv_ctx* ctx) { return ctx ? ctx->C.nbins : 0; }

int pv_check_report(uint32_t* count, uint32_t* first_code) {
  if (!count || !first_code) return PV_ERR_ARG;
  unsigned c = 0, f = 0;
  const bool checked = pvk::check_report(&c, &f);
  *count = c;
  *first_code = f;
  return checked ? PV_OK : PV_ERR_ARG;
}

int pv_find_batch(pv_ctx* ctx, const pv_tracks* tracks, pv_vertices* seeds_out, void* stream) {
  if (!ctx) return PV_ERR_ARG;
  int rc = check_tracks(tracks);
  if (rc != PV_OK) return rc;
  rc = check_out(seeds_out, tracks, true);
  if (rc != PV_OK) return rc;
  cudaSetDevice(ctx->device);
  return run_find_or_fit(ctx, tracks, nullptr, seeds_out, static_cast<cudaStream_t>(stream),
                         pvk::kFind);
}

int pv_fit_batch(pv_ctx* ctx, const pv_tracks* tracks, const pv_vertices* seeds, pv_vertices* out,
                 void* stream) {
  if (!ctx) return PV_ERR_ARG;
  int rc = check_tracks(tracks);
  if (rc != PV_OK) return rc;
  rc = check_out(out, tracks, true);
  if (rc != PV_OK) return rc;
  if (seeds) {
    rc = check_out(seeds, tracks, true);
    if (rc != PV_OK) return rc;
  }
  cudaSetDevice(ctx->device);
  return run_find_or_fit(ctx, tracks, seeds, out, static_cast<cudaStream_t>(stream),
                         seeds ? pvk::kFit : pvk::kFindFit);
}

int pv_fit_multi(pv_ctx* ctx, const pv_tracks* tracks, const pv_vertices* seeds, pv_vertices* out,
                 void* stream) {
  if (!ctx) return PV_ERR_ARG;
  int rc = check_tracks(tracks);
  if (rc != PV_OK) return rc;
  rc = check_out(out, tracks, true);
  if (rc != PV_OK) return rc;
  if (seeds) {
    rc = check_out(seeds, tracks, true);
    if (rc != PV_OK) return rc;
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (tracks->n_events == 0) return PV_OK;
  if (!seeds) {
    // the seeds of steps (a)-(c), written into out and read back per event
    rc = run_find_or_fit(ctx, tracks, nullptr, out, st, pvk::kFind);
    if (rc != PV_OK) return rc;
    seeds = out;
  }
  // scratch of the three multi-vertex kernels
  const int64_t E = tracks->n_events, n = tracks->n_tracks;
  const int64_t slots = E * PV_MAX_SEEDS;
  size_t o = 0;
  const size_t o_cnt = o; o += 256;
  const size_t o_K = o; o += round16(sizeof(int) * E);
  const size_t o_P = o; o += round16(3 * sizeof(float4) * n);
  const size_t o_tev = o; o += round16(sizeof(int) * n);
  const size_t o_work = o; o += round16(sizeof(int2) * slots);
  const size_t o_redo = o; o += round16(sizeof(int2) * slots);
  const size_t o_sx = o; o += round16(sizeof(float) * slots);
  const size_t o_sy = o; o += round16(sizeof(float) * slots);
  const size_t o_sz = o; o += round16(sizeof(float) * slots);
  const size_t o_last = o; o += round16(sizeof(pvk::MvLastState) * slots);
  const size_t o_vz = o; o += round16(sizeof(float) * slots);
  const size_t o_vczz = o; o += round16(sizeof(float) * slots);
  const size_t o_vn = o; o += round16(sizeof(int) * slots);
  const size_t o_vst = o; o += round16(sizeof(int) * slots);
  DevBuf& mbuf = ctx->ws[st].mv;
  PV_CUDA(ctx, mbuf.ensure(o));
  char* base = static_cast<char*>(mbuf.p);
  pvk::MvScratch M;
  M.counters = reinterpret_cast<int*>(base + o_cnt);
  M.K = reinterpret_cast<int*>(base + o_K);
  M.P = reinterpret_cast<float4*>(base + o_P);
  M.tev = reinterpret_cast<int*>(base + o_tev);
  M.work = reinterpret_cast<int2*>(base + o_work);
  M.redo = reinterpret_cast<int2*>(base + o_redo);
  M.sx = reinterpret_cast<float*>(base + o_sx);
  M.sy = reinterpret_cast<float*>(base + o_sy);
  M.sz = reinterpret_cast<float*>(base + o_sz);
  M.last = reinterpret_cast<pvk::MvLastState*>(base + o_last);
  M.vz = reinterpret_cast<float*>(base + o_vz);
  M.vczz = reinterpret_cast<float*>(base + o_vczz);
  M.vn = reinterpret_cast<int*>(base + o_vn);
  M.vst = reinterpret_cast<int*>(base + o_vst);
  const int fit_grid = ctx->n_sm * (ctx->mv_per_sm > 0 ? ctx->mv_per_sm : 1);
  const int redo_grid = ctx->n_sm * (ctx->mv_redo_per_sm > 0 ? ctx->mv_redo_per_sm : 1);
  int launches = 0;
  PV_CUDA(ctx, pvk::launch_mv_fit(ctx->C, track_ptrs(tracks), seed_ptrs(seeds), out_ptrs(out), M,
                                  fit_grid, redo_grid, st, &launches));
  ctx->launches += launches;
  return PV_OK;
}

int pv_extrapolate_batch(pv_ctx* ctx, const pv_tracks* tracks, float* zpoca, float* sigma,
                         int32_t* center, void* stream) {
  if (!ctx) return PV_ERR_ARG;
  int rc = check_tracks(tracks);
  if (rc != PV_OK) return rc;
  cudaSetDevice(ctx->device);
  if (tracks->n_tracks == 0) return PV_OK;
  PV_CUDA(ctx, pvk::launch_extrapolate(ctx->C, track_ptrs(tracks), zpoca, sigma, center,
                                       static_cast<cudaStream_t>(stream)));
  ctx->launches += 1;
  return PV_OK;
}

int pv_histogram_batch(pv_ctx* ctx, const pv_tracks* tracks, uint32_t* hist, void* stream) {
  if (!ctx || !hist) return PV_ERR_ARG;
  int rc = check_tracks(tracks);
  if (rc != PV_OK) return rc;
  cudaSetDevice(ctx->device);
  if (tracks->n_events == 0) return PV_OK;
  PlainLayout L(tracks->n_tracks, 0, ctx->C.nbins);
  DevBuf& pbuf = ctx->ws[static_cast<cudaStream_t>(stream)].plain;
  PV_CUDA(ctx, pbuf.ensure(L.total));
  int n = 0;
  PV_CUDA(ctx, pvk::launch_histogram(ctx->C, track_ptrs(tracks), hist, L.scratch(pbuf.p),
                                     static_cast<cudaStream_t>(stream), &n));
  ctx->launches += n;
  return PV_OK;
}

int pv_run_host(pv_ctx* ctx, const pv_tracks* h, pv_vertices* ho, void* stream) {
  if (!ctx) return PV_ERR_ARG;
  int rc = check_tracks(h);
  if (rc != PV_OK) return rc;
  rc = check_out(ho, h, true);
  if (rc != PV_OK) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = h->n_tracks;
  const int64_t E = h->n_events;
  const size_t cap = static_cast<size_t>(ho->capacity);
  const int64_t* hoff = h->event_offsets;
  // events in K chunks, pipelined: chunk k's inputs copy in while chunk k-1
  // runs and chunk k-2's results copy out.  Chunks need offsets that rise
  // within [0, n]; other batches run as one chunk (their kernels flag the
  // events with bad offsets).
  int K = 1;
  if (E >= 2 * kRunHostChunkEvents && hoff[0] == 0 && hoff[E] <= n) {
    bool rising = true;
    for (int64_t e = 0; e < E && rising; ++e) rising = hoff[e + 1] >= hoff[e];
    if (rising) {
      const int64_t k = E / kRunHostChunkEvents;
      K = static_cast<int>(k < kRunHostChunks ? k : kRunHostChunks);
    }
  }
  const float* src[11] = {h->x, h->y, h->z, h->tx, h->ty, h->cxx, h->cxtx, h->ctxtx,
                          h->cyy, h->cyty, h->ctyty};
  // On the fused path of the GPU flavour, tracks in pinned memory the device
  // can address are read there by the find kernel itself, which writes the
  // device copy the fit kernel gathers from: one pass over the host link and
  // no input copies, so the batch runs as one chunk.
  const float* alias[11] = {};
  bool staged = ctx->cfg.path != PV_PATH_PLAIN && pvk::flavour_of(ctx->C) == 0 && n > 0;
  for (int c = 0; c < 11 && staged; ++c) {
    alias[c] = static_cast<const float*>(device_alias(src[c]));
    staged = alias[c] != nullptr;
  }
  if (staged) K = 1;
  // device inputs: 11 float arrays (copies of the host columns, or the staged
  // find's device copy) + the chunks' offsets (E + K entries)
  size_t in_bytes = 11 * round16(4 * n) + round16(8 * (E + K));
  PV_CUDA(ctx, ctx->host_in.ensure(in_bytes));
  char* din = static_cast<char*>(ctx->host_in.p);
  float* dcol[11];
  for (int k = 0; k < 11; ++k) dcol[k] = reinterpret_cast<float*>(din + k * round16(4 * n));
  int64_t* doff = reinterpret_cast<int64_t*>(din + 11 * round16(4 * n));
  // device outputs mirror the non-NULL host outputs; per slot [event][cap],
  // per event, or per track.  On the fused path, pinned host memory that the
  // device can address is written by the kernels in place (they write only
  // the slots of found vertices and read no output back, so nothing is
  // copied back for it); other host memory, and every output of the plain
  // path (whose fit reads the find's outputs), gets a device staging buffer
  // and a copy back.
  const bool in_place = ctx->cfg.path != PV_PATH_PLAIN;
  enum Unit { kSlot, kEvent, kTrack };
  // dev: where the kernels write the column (the host memory's device address,
  // or the staging buffer at off once it is allocated)
  struct Col { void* host; size_t elem; Unit unit; size_t off; char* dev; bool direct; } cols[16];
  int nc = 0;
  size_t o = 0;
  auto plan = [&](void* hp, size_t elem, Unit u) -> int {
    if (!hp) return -1;
    char* alias = in_place ? static_cast<char*>(device_alias(hp)) : nullptr;
    const size_t count = u == kSlot ? static_cast<size_t>(E) * cap
                                    : (u == kEvent ? static_cast<size_t>(E)
                                                   : static_cast<size_t>(n));
    cols[nc] = {hp, elem, u, o, alias, alias != nullptr};
    if (!alias) o += round16(elem * count);
    return nc++;
  };
  const int ix = plan(ho->x, 4, kSlot), iy = plan(ho->y, 4, kSlot), iz = plan(ho->z, 4, kSlot);
  const int icov = plan(ho->cov, 24, kSlot), ichi = plan(ho->chi2, 4, kSlot);
  const int indf = plan(ho->ndof, 4, kSlot), intr = plan(ho->n_tracks, 4, kSlot);
  const int init = plan(ho->n_iter, 4, kSlot), ist = plan(ho->status, 4, kSlot);
  const int ilo = plan(ho->bin_lo, 4, kSlot), ihi = plan(ho->bin_hi, 4, kSlot);
  const int ibm = plan(ho->bin_max, 4, kSlot);
  const int inpe = plan(ho->n_per_event, 4, kEvent), ievs = plan(ho->event_status, 4, kEvent);
  const int itv = plan(ho->track_vertex, 4, kTrack);
  PV_CUDA(ctx, ctx->host_out.ensure(o + 16));
  char* dout = static_cast<char*>(ctx->host_out.p);
  for (int c = 0; c < nc; ++c)
    if (!cols[c].direct) cols[c].dev = dout + cols[c].off;

  if (K > 1) {
    if (!ctx->rh_in)
      PV_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->rh_in, cudaStreamNonBlocking));
    if (!ctx->rh_out)
      PV_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->rh_out, cudaStreamNonBlocking));
    for (auto& ev : ctx->rh_ev)
      if (!ev) PV_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    const size_t need = static_cast<size_t>(E + K);
    if (ctx->rh_off_cap < need) {
      if (ctx->rh_off) cudaFreeHost(ctx->rh_off);
      ctx->rh_off = nullptr;
      ctx->rh_off_cap = 0;
      PV_CUDA(ctx, cudaMallocHost(&ctx->rh_off, sizeof(int64_t) * need));
      ctx->rh_off_cap = need;
    }
    // the copies start after the caller's earlier work on its stream
    PV_CUDA(ctx, cudaEventRecord(ctx->rh_ev[2 * kRunHostChunks], st));
    PV_CUDA(ctx, cudaStreamWaitEvent(ctx->rh_in, ctx->rh_ev[2 * kRunHostChunks], 0));
  }
  for (int k = 0; k < K; ++k) {
    const int64_t e0 = E * k / K, e1 = E * (k + 1) / K;
    const int64_t b0 = K > 1 ? hoff[e0] : 0, b1 = K > 1 ? hoff[e1] : n;
    cudaStream_t s_in = K > 1 ? ctx->rh_in : st;
    cudaStream_t s_out = K > 1 ? ctx->rh_out : st;
    const int64_t nt = b1 - b0;
    if (!staged)
      for (int c = 0; c < 11; ++c)
        if (nt) PV_CUDA(ctx, cudaMemcpyAsync(dcol[c] + b0, src[c] + b0, 4 * nt,
                                             cudaMemcpyHostToDevice, s_in));
    // chunk k's offsets, relative to its first track, at entries e0 + k ..
    int64_t* doff_k = doff + e0 + k;
    if (K > 1) {
      int64_t* ho_k = ctx->rh_off + e0 + k;
      for (int64_t e = e0; e <= e1; ++e) ho_k[e - e0] = hoff[e] - b0;
      PV_CUDA(ctx, cudaMemcpyAsync(doff_k, ho_k, 8 * (e1 - e0 + 1), cudaMemcpyHostToDevice,
                                   s_in));
      PV_CUDA(ctx, cudaEventRecord(ctx->rh_ev[k], s_in));
      PV_CUDA(ctx, cudaStreamWaitEvent(st, ctx->rh_ev[k], 0));
    } else if (E) {
      PV_CUDA(ctx, cudaMemcpyAsync(doff_k, hoff, 8 * (E + 1), cudaMemcpyHostToDevice, st));
    }
    pv_tracks dt = *h;
    const float* const* col = staged ? alias : const_cast<const float* const*>(dcol);
    dt.x = col[0] + b0; dt.y = col[1] + b0; dt.z = col[2] + b0;
    dt.tx = col[3] + b0; dt.ty = col[4] + b0;
    dt.cxx = col[5] + b0; dt.cxtx = col[6] + b0; dt.ctxtx = col[7] + b0;
    dt.cyy = col[8] + b0; dt.cyty = col[9] + b0; dt.ctyty = col[10] + b0;
    dt.event_offsets = doff_k;
    dt.n_tracks = nt;
    dt.n_events = static_cast<int32_t>(e1 - e0);
    const size_t slot0 = static_cast<size_t>(e0) * cap;
    auto sp = [&](int c, size_t first) -> void* {
      return c < 0 ? nullptr : cols[c].dev + cols[c].elem * first;
    };
    pv_vertices dv = *ho;
    dv.x = static_cast<float*>(sp(ix, slot0));
    dv.y = static_cast<float*>(sp(iy, slot0));
    dv.z = static_cast<float*>(sp(iz, slot0));
    dv.cov = static_cast<float*>(sp(icov, slot0));
    dv.chi2 = static_cast<float*>(sp(ichi, slot0));
    dv.ndof = static_cast<float*>(sp(indf, slot0));
    dv.n_tracks = static_cast<int32_t*>(sp(intr, slot0));
    dv.n_iter = static_cast<int32_t*>(sp(init, slot0));
    dv.status = static_cast<int32_t*>(sp(ist, slot0));
    dv.bin_lo = static_cast<int32_t*>(sp(ilo, slot0));
    dv.bin_hi = static_cast<int32_t*>(sp(ihi, slot0));
    dv.bin_max = static_cast<int32_t*>(sp(ibm, slot0));
    dv.n_per_event = static_cast<int32_t*>(sp(inpe, e0));
    dv.event_status = static_cast<int32_t*>(sp(ievs, e0));
    dv.track_vertex = static_cast<int32_t*>(sp(itv, b0));
    rc = staged ? run_staged(ctx, &dt, &dv, dcol, st)
                : run_find_or_fit(ctx, &dt, nullptr, &dv, st, pvk::kFindFit);
    if (rc != PV_OK) return rc;
    if (K > 1) {
      PV_CUDA(ctx, cudaEventRecord(ctx->rh_ev[kRunHostChunks + k], st));
      PV_CUDA(ctx, cudaStreamWaitEvent(s_out, ctx->rh_ev[kRunHostChunks + k], 0));
    }
    for (int c = 0; c < nc; ++c) {
      const Col& col = cols[c];
      if (col.direct) continue;
      size_t first, count;
      if (col.unit == kSlot) { first = slot0; count = static_cast<size_t>(e1 - e0) * cap; }
      else if (col.unit == kEvent) { first = e0; count = static_cast<size_t>(e1 - e0); }
      else { first = b0; count = static_cast<size_t>(nt); }
      if (count)
        PV_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(col.host) + col.elem * first,
                                     col.dev + col.elem * first, col.elem * count,
                                     cudaMemcpyDeviceToHost, s_out));
    }
  }
  if (K > 1) PV_CUDA(ctx, cudaStreamSynchronize(ctx->rh_out));
  PV_CUDA(ctx, cudaStreamSynchronize(st));
  return PV_OK;
}

int pv_submit(pv_ctx* ctx, const pv_tracks* tracks, pv_vertices* out, uint64_t* ticket) {
  if (!ctx || !ticket) return PV_ERR_ARG;
  int rc = check_tracks(tracks);
  if (rc != PV_OK) return rc;
  rc = check_out(out, tracks, true);
  if (rc != PV_OK) return rc;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  rc = ensure_pool(ctx);
  if (rc != PV_OK) return rc;
  const size_t bytes = ServeLayout(tracks->n_tracks).total;
  if (bytes > ctx->arena.size) return PV_ERR_NOMEM;
  if (ctx->pending.size() >= kMaxQueued) {
    rc = pump(ctx);
    if (rc != PV_OK) return rc;
    if (ctx->pending.size() >= kMaxQueued) return PV_ERR_BUSY;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) return PV_ERR_NOMEM;
  r->ticket = ctx->next_ticket++;
  r->tracks = *tracks;
  r->out = *out;
  r->bytes = bytes;
  r->t_submit = now_ns();
  if (tracks->n_events == 0) {
    r->done = true;
    r->t_done = r->t_submit;
  } else {
    ctx->pending.push_back(r);
  }
  ctx->requests[r->ticket] = r;
  *ticket = r->ticket;
  return pump(ctx);
}

int pv_poll(pv_ctx* ctx, uint64_t ticket, int* done) {
  if (!ctx || !done) return PV_ERR_ARG;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->requests.find(ticket);
  if (it == ctx->requests.end()) return PV_ERR_NOTFOUND;
  int rc = it->second->done ? PV_OK : pump(ctx);
  *done = it->second->done ? 1 : 0;
  return rc;
}

int pv_request_latency_ns(pv_ctx* ctx, uint64_t ticket, uint64_t* ns) {
  if (!ctx || !ns) return PV_ERR_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->requests.find(ticket);
  if (it == ctx->requests.end() || !it->second->done) return PV_ERR_NOTFOUND;
  *ns = it->second->t_done - it->second->t_submit;
  delete it->second;
  ctx->requests.erase(it);
  return PV_OK;
}

int pv_serve_start(pv_ctx* ctx) {
  if (!ctx) return PV_ERR_ARG;
  cudaSetDevice(ctx->device);
  std::lock_guard<std::mutex> g(ctx->mu);
  int rc = ensure_pool(ctx);
  if (rc != PV_OK) return rc;
  return start_server(ctx);
}

int pv_serve_status(pv_ctx* ctx, int* running, int* last_exit) {
  if (!ctx) return PV_ERR_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  const bool run = ctx->pool_ready && serve_running(ctx);
  if (running) *running = run ? 1 : 0;
  if (last_exit)
    *last_exit = (ctx->sctl && !run) ? *reinterpret_cast<volatile int*>(&ctx->sctl->exit_code) : -1;
  return PV_OK;
}

const char* pv_strerror(int code) {
  switch (code) {
    case PV_OK: return "ok";
    case PV_ERR_ARG: return "invalid argument";
    case PV_ERR_CUDA: return "CUDA error";
    case PV_ERR_CAPACITY: return "capacity exceeded";
    case PV_ERR_NOMEM: return "out of memory / not admissible";
    case PV_ERR_TIMEOUT: return "timeout";
    case PV_ERR_BUSY: return "busy";
    case PV_ERR_NOTFOUND: return "not found";
    default: return "unknown error";
  }
}

const char* pv_last_cuda_error(const pv_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

uint64_t pv_launch_count(const pv_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

uint64_t pv_device_bytes(const pv_ctx* ctx) {
  if (!ctx) return 0;
  uint64_t b = ctx->tpl.bytes + ctx->host_in.bytes + ctx->host_out.bytes + ctx->pool.bytes;
  for (const auto& kv : ctx->ws) b += kv.second.fused.bytes + kv.second.plain.bytes + kv.second.mv.bytes;
  return b;
}

}  // extern "C"

// ===========================================================================
// Allocation-free variant of the fused find + fit.
//
// Some callers cannot allocate device memory once they are running: a
// real-time loop cannot afford cudaMalloc / cudaFree, which may synchronise
// the whole device, and an application that hands all device memory to its
// own allocator at start-up runs with a fixed budget.  pv_find_fit_static
// serves them: its scratch (the work counter and the per-track arrays of
// events above 256 tracks) lives in the file-scope array below, which every
// GPU that loads this library holds until the process exits.  Host code only
// ever passes the array's device address, obtained with cudaGetSymbolAddress
// once per device (the array's name is a host-side stand-in, not a device
// address) and kept for the life of the process, which assumes the device's
// primary context lives as long.  Calls share the array: two calls whose work
// overlaps on the GPU race, so callers serialise them (one stream, or events
// between streams).

namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;   // 8 MiB
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};

// Device address of g_static_scratch on the current device (set-up on first use).
int static_scratch_for(pv_ctx* ctx, void** out) {
  if (ctx->device < 0 || ctx->device >= kStaticMaxDevices) return PV_ERR_ARG;
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_ptr[ctx->device]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_static_scratch);
    if (err != cudaSuccess || !p) return fail_cuda(ctx, err == cudaSuccess ? cudaErrorUnknown : err);
    g_static_ptr[ctx->device] = p;
  }
  *out = g_static_ptr[ctx->device];
  return PV_OK;
}

}  // namespace

extern "C" int pv_find_fit_static(pv_ctx* ctx, const pv_tracks* tracks, pv_vertices* out,
                                  void* stream) {
  if (!ctx) return PV_ERR_ARG;
  int rc = check_tracks(tracks);
  if (rc != PV_OK) return rc;
  rc = check_out(out, tracks, true);
  if (rc != PV_OK) return rc;
  FusedLayout L(tracks->n_tracks, tracks->n_events, out->capacity);
  if (L.total > kStaticScratchBytes) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "pv_find_fit_static: %lld tracks in %d events need %zu bytes of scratch; "
                  "the static buffer holds %zu bytes", static_cast<long long>(tracks->n_tracks),
                  tracks->n_events, L.total, kStaticScratchBytes);
    ctx->last_error = msg;
    return PV_ERR_CAPACITY;
  }
  PV_CUDA(ctx, cudaSetDevice(ctx->device));
  void* base = nullptr;
  rc = static_scratch_for(ctx, &base);
  if (rc != PV_OK) return rc;
  if (tracks->n_events == 0) return PV_OK;
  // enqueue_fused clears the work counters on the stream before the kernels
  return enqueue_fused(ctx, pvk::kFindFit, tracks, nullptr, out, base,
                       static_cast<cudaStream_t>(stream));
}

extern "C" int pv_launch_config(const pv_ctx* ctx, const pv_tracks* tracks, int* find_threads,
                                int* fit_threads, int* find_grid, int* fit_grid) {
  if (!ctx || !tracks) return PV_ERR_ARG;
  const pvk::LaunchCfg L = chosen_cfg(ctx, pvk::kFindFit, tracks);
  if (find_threads) *find_threads = L.find_nt;
  if (fit_threads) *fit_threads = L.fit_nt;
  if (find_grid) *find_grid = L.find_grid;
  if (fit_grid) *fit_grid = L.fit_grid;
  return PV_OK;
}

extern "C" int pv_autotune(pv_ctx* ctx, const pv_tracks* sample, pv_vertices* out, void* stream) {
  if (!ctx) return PV_ERR_ARG;
  int rc = check_tracks(sample);
  if (rc != PV_OK) return rc;
  rc = check_out(out, sample, true);
  if (rc != PV_OK) return rc;
  if (sample->n_events == 0) return PV_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FusedLayout FL(sample->n_tracks, sample->n_events, out->capacity);
  DevBuf& fbuf = ctx->ws[st].fused;
  void* before = fbuf.p;
  PV_CUDA(ctx, fbuf.ensure(FL.total));
  if (fbuf.p != before) clear_graphs(ctx);
  cudaEvent_t e0, e1;
  PV_CUDA(ctx, cudaEventCreate(&e0));
  PV_CUDA(ctx, cudaEventCreate(&e1));
  const int finds[4] = {64, 96, 128, 256};
  const int fits[2] = {128, 256};
  float best = -1.f;
  pvk::LaunchCfg best_cfg{128, 0, pvk::kFitThreads, 0};
  for (int fi : finds) {
    for (int ft : fits) {
      const pvk::LaunchCfg cfg = launch_cfg(ctx, pvk::kFindFit, sample, fi, ft);
      float t_min = -1.f;
      for (int rep = 0; rep < 4; ++rep) {
        PV_CUDA(ctx, cudaEventRecord(e0, st));
        rc = enqueue_fused_cfg(ctx, pvk::kFindFit, sample, nullptr, out, fbuf.p, cfg, st);
        if (rc != PV_OK) return rc;
        PV_CUDA(ctx, cudaEventRecord(e1, st));
        PV_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        PV_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && (t_min < 0.f || ms < t_min)) t_min = ms;   // the first run warms up
      }
      if (best < 0.f || t_min < best) {
        best = t_min;
        best_cfg = pvk::LaunchCfg{fi, 0, ft, 0};
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->bucket_cfg[bucket_of(sample)] = best_cfg;
  clear_graphs(ctx);
  return PV_OK;
}

extern "C" int pv_set_launch_config(pv_ctx* ctx, int bucket, int find_threads, int fit_threads) {
  if (!ctx || bucket < 0 || bucket > 2) return PV_ERR_ARG;
  if (!pvk::find_block_ok(find_threads) || !pvk::fit_block_ok(fit_threads)) return PV_ERR_ARG;
  ctx->bucket_cfg[bucket] = pvk::LaunchCfg{find_threads, 0, fit_threads, 0};
  clear_graphs(ctx);
  return PV_OK;
}
