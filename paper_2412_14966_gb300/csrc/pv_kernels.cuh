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

// Global scratch for per-track state of events larger than the in-shared
// capacity (indexed by the global track index).
struct TrackScratch {
  int32_t* center;
  int32_t* cid;
  int32_t* slot;
  float4* A;
  float2* W;
};

enum Mode : int { kFind = 1, kFit = 2, kFindFit = 3 };

constexpr int kSmallCap = 256;      // tracks kept in shared memory per event
constexpr int kFusedThreads = 128;

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

size_t fused_smem_bytes(int nbins, int mode);
cudaError_t fused_setup(int nbins);

cudaError_t launch_fused(int mode, const pvdev::Consts& C, const TrackPtrs& T, const SeedPtrs& S,
                         const OutPtrs& O, const TrackScratch& ws, int* work_counter,
                         int grid, cudaStream_t st);

int fused_blocks_per_sm(int nbins, int mode);

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
