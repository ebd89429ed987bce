// pv_kernels.cuh -- kernel parameter blocks and host-side launchers shared by
// the kernels translation unit and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pv_device.cuh"

namespace pvk {

struct TrackPtrs {
  const float *x, *y, *z, *tx, *ty, *cxx, *cxtx, *ctxtx, *cyy, *cyty, *ctyty;
  const int64_t* off;
  int64_t n_tracks;
  int32_t n_events;
};

struct OutPtrs {
  float *x, *y, *z, *cov, *chi2, *ndof;
  int32_t *n_tracks, *n_iter, *status;
  int32_t *bin_lo, *bin_hi, *bin_max;
  int32_t *n_per_event, *event_status, *track_vertex;
  int32_t cap;
};

struct SeedPtrs {            // seeds read by the fit-only kernel
  const float *x, *y, *z;
  const int32_t* n_per_event;
  const int32_t* track_vertex;
  int32_t cap;
};

// One vertex to fit: its fit inputs are A[off .. off + cnt), W[off .. off +
// cnt) (its tracks in track-index order, written by the find kernel) and its
// results go to row e, column k of the outputs; x, y, z are the bit patterns
// of the seed position the inputs are relative to.
struct VertexWork {
  int off;
  int e;
  int kc;           // k | cnt << 8
  int pad0;
  uint32_t x, y, z;
  int pad1;
};

// The vertex work list is split by size class (tracks per vertex: 1-8,
// 9-16, 17-32, 33 and more) so that the four vertices a warp fits together
// need similar numbers of passes over their tracks; the fit kernel takes the
// classes from the largest down.
constexpr int kWorkClasses = 4;
__host__ __device__ inline int work_class(int cnt) {
  return cnt <= 8 ? 0 : (cnt <= 16 ? 1 : (cnt <= 32 ? 2 : 3));
}
constexpr int kClassMinTracks[kWorkClasses] = {1, 9, 17, 33};

// Global scratch of the fused path (indexed by the global track index).
struct TrackScratch {
  int16_t* center;      // per track, events above kSmallCap tracks: center bin
  int8_t* cid;          // and vertex index
  int32_t* slot;        // per track, events above kSmallCap tracks: position of
                        // the track's fit inputs in its event's vertex order
  float4* A;            // per track: fit inputs in vertex order (X, Y, tx, ty)
  float2* W;            //   and their weights (1/V_xx, 1/V_yy) at the seed z
  VertexWork* work;     // vertex work lists, one region per size class
  long long cls_base[kWorkClasses];   // first entry of each class's region
  int cls_cap[kWorkClasses];    // its capacity
  int* counters;        // [0] next event, [1 + c] vertices listed in class c,
                        // [1 + kWorkClasses] next vertex to fit
  float* stage[8];      // kStage: device copy of the first 8 track columns (TrackPtrs order)
};
constexpr int kCounterInts = 8;

// a[c] with constant indices only (a kernel parameter indexed at run time
// would be copied to local memory)
template <typename V>
__host__ __device__ __forceinline__ V class_pick(const V (&a)[kWorkClasses], int c) {
  return c == 0 ? a[0] : (c == 1 ? a[1] : (c == 2 ? a[2] : a[3]));
}

enum Mode : int { kFind = 1, kFit = 2, kFindFit = 3, kStage = 4, kServe = 8 };
// kFindFit | kServe: the serving kernel's event work, which fits the event's
// vertices in the same CTA instead of listing them for the fit kernel
// kFindFit | kStage: the tracks are in host memory the device can address; the
// find kernel reads every column there once: the eight its steps (a)-(b) need
// in the fill, writing them to a device copy (TrackScratch::stage) that its
// fit-input pass reads back, and the other three in that pass
constexpr int kFindFitStaged = kFindFit | kStage;

constexpr int kSmallCap = 256;      // tracks kept in shared memory per event
constexpr int kFusedThreads = 128;

// Flavour of the find kernel: bit 0 the x86 recursive dip split, bit 1 the
// x86 template profile.  The GPU flavour (0) is built for every block size,
// the others for kFlavThreads.
constexpr int kFlavThreads = 128;
__host__ __device__ constexpr int flavour_split(int f) {
  return (f & 1) ? PV_SPLIT_RECURSIVE : PV_SPLIT_ZORDER;
}
__host__ __device__ constexpr int flavour_profile(int f) {
  return (f & 2) ? PV_PROFILE_TEMPLATE : PV_PROFILE_CUBIC;
}
inline int flavour_of(const pvdev::Consts& C) {
  return (C.split_mode == PV_SPLIT_RECURSIVE ? 1 : 0) |
         (C.profile_mode == PV_PROFILE_TEMPLATE ? 2 : 0);
}

// Fills the template table of the x86 profile for bin width dz (one small
// kernel); t->status becomes 1 if the templates do not fit.
cudaError_t build_template_table(pvdev::TplTable* t, float dz, cudaStream_t st);

// Scratch of the plain per-step path.
struct PlainScratch {
  float* zpoca;
  float* sigma;
  int32_t* center;
  int32_t* j0;
  int32_t* j1;
  uint32_t* hist;        // [n_events][nbins]
  int32_t* seed_n;       // [n_events]
  int32_t* seed_lo;      // [n_events][64] ... raw seeds before association
  int32_t* seed_hi;
  int32_t* seed_bin;
  float* seed_z;
  int32_t* cid;          // per track
  int32_t* slot;         // per track
  float4* A;             // per track, fit inputs in vertex order
  float2* W;
  int32_t* ev_status;    // [n_events]
};

size_t fused_smem_bytes(int nbins, int mode, int nt, bool rec);
cudaError_t fused_setup(int nbins);

// Launch shape of the fused path (block sizes and persistent grids); results do
// not depend on it.
struct LaunchCfg {
  int find_nt, find_grid;
  int fit_nt, fit_grid;
};

// Enqueues the fused path: counter reset, find kernel, then (modes with a fit)
// the vertex fit kernel.  *n_launches receives the kernels enqueued.
cudaError_t launch_fused(int mode, const pvdev::Consts& C, const TrackPtrs& T, const SeedPtrs& S,
                         const OutPtrs& O, const TrackScratch& ws, const LaunchCfg& L,
                         cudaStream_t st, int* n_launches);

// The checked build's record of out-of-bounds indices (count, first code),
// reset by the call; false in the default build, which has no checks.
bool check_report(unsigned* count, unsigned* first);
// The same record of the serving kernel's translation unit.
bool serve_check_report(unsigned* count, unsigned* first);

bool find_block_ok(int nt);
bool fit_block_ok(int ft);
int fused_blocks_per_sm(int nbins, int mode, int nt, int flav);
int fit_blocks_per_sm(int accum, int ft);
constexpr int kFitThreads = 256;

// Upper bound of the vertices a batch can list: per event at most
// min(its tracks, capacity) (seeds without tracks are written directly).
inline long long work_capacity(long long n_tracks, long long n_events, int cap) {
  long long c = cap < pvdev::kMaxSeeds ? cap : pvdev::kMaxSeeds;
  long long by_events = n_events * c;
  return by_events < n_tracks ? by_events : n_tracks;
}

// Upper bound of the vertices of size class c: a vertex of the class has at
// least kClassMinTracks[c] tracks.
inline long long class_capacity(int c, long long n_tracks, long long n_events, int cap) {
  long long all = work_capacity(n_tracks, n_events, cap);
  long long by_tracks = n_tracks / kClassMinTracks[c];
  return by_tracks < all ? by_tracks : all;
}

// ---------------------------------------------------------------------------
// Serving: the persistent request loop.  The host writes one descriptor per
// admitted request into a ring in pinned host memory the device reads
// (ServeCtl, mapped), then publishes the request's events by raising
// `published`; the events of all requests form one sequence, request r owning
// [ev_base, ev_base + n_events).  The serving kernel's CTAs claim events of
// that sequence one at a time, run the find and the fit of each, and the CTA
// that completes a request's last event stamps done_ns (the GPU's global
// timer) and done_seq in the ring.  A CTA whose claimed event is not
// published within idle_ns ends; the kernel ends when all have (exit code
// PV_ERR_TIMEOUT), or PV_OK after the host sets `stop`.
constexpr int kServeRing = 1024;
constexpr int kServeThreads = 128;

struct ServeDesc {
  TrackPtrs T;                       // the request's device tracks
  OutPtrs O;                         // its device outputs
  int16_t* center;                   // its scratch (events above kSmallCap tracks)
  int8_t* cid;
  int32_t* slot;
  float4* A;                         // its fit inputs in vertex order
  float2* W;
  unsigned long long ev_base;        // its first event in the sequence
  unsigned long long done_target;    // ServeDev::slot_done of its slot when complete
  unsigned long long seq;            // request number, written last (~0: being written)
};

struct ServeCtl {                    // pinned host memory, mapped for the device
  unsigned long long published;      // events published so far (host)
  unsigned int stop;                 // host: end the kernel
  int exit_code;                     // device: why the kernel ended
  unsigned long long exit_ns;        // device: global timer at the end
  unsigned long long clock_ns;       // device: global timer (clock calibration)
  unsigned long long done_seq[kServeRing];   // device: last request completed in a slot
  unsigned long long done_ns[kServeRing];    // device: its completion time
  ServeDesc ring[kServeRing];
};

// Events are claimed with one atomic add each, so a CTA with nothing to do
// holds the next unpublished event and waits for it; if its wait runs out it
// hands the event to the next launch of the kernel through the orphan list of
// its launch (epoch & 1), which that launch takes first.
constexpr int kServeOrphans = 4096;  // at least the largest grid

struct ServeDev {                    // device memory
  unsigned long long next_event;     // next event of the sequence to claim
  unsigned long long slot_done[kServeRing];  // events completed per slot, cumulative
  int running;                       // CTAs that left the loop (this launch)
  int orph_n[2];                     // events handed on, per launch parity
  int orph_take;                     // orphans of the previous launch taken so far
  unsigned long long orph[2][kServeOrphans];
};

// Launches the serving kernel (grid = SMs x resident CTAs) on st; it reads
// requests from seq_start on.  The flavour and accumulation mode come from C.
cudaError_t launch_serve(const pvdev::Consts& C, ServeCtl* ctl, ServeDev* dev,
                         unsigned long long idle_ns, unsigned long long seq_start,
                         unsigned int epoch, int grid, cudaStream_t st);
// Resident CTAs per SM of the serving kernel; its dynamic shared memory.
int serve_blocks_per_sm(const pvdev::Consts& C);
cudaError_t serve_setup(int nbins);
// Writes the device's global timer to ctl->clock_ns (one thread).
cudaError_t launch_serve_clock(ServeCtl* ctl, cudaStream_t st);

// Multi-vertex fit (GPU flavour of Sec. 3.5) of the seeds S into O.
struct MvLastState {        // the sheared position a vertex's last weights were taken at
  float axp, ayp, az, cx, cy;
};
struct MvScratch {
  int* counters;            // [0] work items listed, [1] next item to fit, [2] vertices
                            // listed for a refit over all tracks, [3] next one to refit
  int* K;                   // per event: seeds fitted
  int* tev;                 // per track: its event (-1: none)
  float4* P;                // per track, three float4: x y z tx | ty cxx cxtx ctxtx |
                            // cyy cyty ctyty S, S = sum over the event's seeds of exp(-chi2/2)
  int2* work;               // (event, seed) per vertex
  int2* redo;               // (event, seed) per vertex to refit over all tracks
  float *sx, *sy, *sz;      // per slot [event][kMaxSeeds]: seed position
  MvLastState* last;        // per slot: last-iteration state
  float *vz, *vczz;         // per slot: fitted z and C_zz
  int *vn, *vst;            // per slot: tracks and status
};
constexpr int kMvThreads = 128;        // per-event kernels: one warp per event
constexpr int kMvFitThreads = 256;
cudaError_t launch_mv_fit(const pvdev::Consts& C, const TrackPtrs& T, const SeedPtrs& S,
                          const OutPtrs& O, const MvScratch& M, int fit_grid, int redo_grid,
                          cudaStream_t st, int* n_launches);
// resident CTAs per SM of the window fits (redo false) or of the refits
int mv_blocks_per_sm(bool redo);

cudaError_t launch_plain_find(const pvdev::Consts& C, const TrackPtrs& T, const OutPtrs& O,
                              const PlainScratch& ws, cudaStream_t st, int* n_launches);
cudaError_t launch_plain_fit(const pvdev::Consts& C, const TrackPtrs& T, const SeedPtrs& S,
                             const OutPtrs& O, const PlainScratch& ws, cudaStream_t st,
                             int* n_launches);
cudaError_t launch_extrapolate(const pvdev::Consts& C, const TrackPtrs& T, float* zpoca,
                               float* sigma, int32_t* center, cudaStream_t st);
cudaError_t launch_histogram(const pvdev::Consts& C, const TrackPtrs& T, uint32_t* hist,
                             const PlainScratch& ws, cudaStream_t st, int* n_launches);

}  // namespace pvk
