// pv_find.cuh -- the find kernel's work on one event, shared by the batched
// find kernel (pv_kernels.cu) and the persistent serving kernel (pv_serve.cu).
#pragma once

#include "pv_kernels.cuh"

namespace pvk {

using namespace pvdev;

// ---------------------------------------------------------------------------
// shared-memory layout of the find kernel
//
// hist    the event's histogram (dense; only the touched 32-bin tiles are
//         written, scanned and cleared)
// tmask   touched-tile mask
// seeds   seed table
// ring    one ring of proto-cluster bounds per warp
// misc    event ring, seed count, association flag, per-warp scan totals
// center, cid   per-track center bin and vertex (events up to kSmallCap tracks)
// uni     during the fill: the prepared tracks of a fill pass (kFillChunk
//         records of 16 bytes); afterwards: the association's arrays and the
//         per-round vertex counts of the placement
// mark    inside uni, after the tile masks: the recursive dip split's
//         pending right-hand sides (x86 flavour; mark_cap int16 entries,
//         shared out among the proto-clusters during the peak search)

constexpr int kFillChunk = 256;             // most tracks one fill pass prepares
constexpr int kPlaceRounds = kSmallCap / 32;
constexpr int kMiscInts = 32;
// misc entries
constexpr int kMiscK = 2, kMiscFlag = 3, kMiscWarpScan = 4;

__host__ __device__ constexpr int fill_per_thread(int nt) { return nt >= 256 ? 1 : 256 / nt; }

struct Layout {
  size_t hist, tmask, seeds, ring, misc, center, cid, uni, mark, total;
  int mark_cap;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// (rec, the recursive (x86) dip split, needs no memory of its own: its
// scratch lies in uni; the argument is kept for the callers)
__host__ __device__ inline Layout make_layout(int nbins, int mode, int nt, bool rec = false) {
  Layout L;
  size_t o = 0;
  const bool find = (mode & kFind) != 0;
  const int ntiles = (nbins + 31) / 32;
  const size_t assoc = sizeof(int) * kMaxSeeds * 5 + sizeof(int16_t) * kPlaceRounds * kMaxSeeds;
  const size_t recs = find ? sizeof(float4) * kFillChunk : 0;
  L.hist = o;   o += find ? sizeof(uint32_t) * ntiles * 32 : 0;
  L.tmask = o;  o += sizeof(uint32_t) * kTileWords;
  L.seeds = o;  o += align_up(sizeof(SeedOut), 16);
  L.ring = o;   o += align_up(sizeof(int16_t) * 2 * kRunRing * (nt / 32), 16);
  L.misc = o;   o += sizeof(int) * kMiscInts;
  L.center = o; o += sizeof(int16_t) * kSmallCap;
  L.cid = o;    o += align_up(sizeof(int8_t) * kSmallCap, 16);
  const size_t uni = align_up(recs > assoc ? recs : assoc, 16);
  const size_t tiles = 2 * sizeof(uint32_t) * kTileWords * 32;   // the peak search's tile masks
  L.uni = o;    o += uni;
  L.mark = L.uni + tiles;
  L.mark_cap = (find && uni > tiles) ? static_cast<int>((uni - tiles) / sizeof(int16_t)) : 0;
  (void)rec;
  L.total = align_up(o, 16);
  return L;
}

// ---------------------------------------------------------------------------
// pieces shared by the fused, the serving and the plain kernels

// Exclusive scan of cnt[0..K) into voff and base (warp 0 only, K <= 64).
__device__ __forceinline__ void warp_offsets(const int* cnt, int K, int* voff, int* base) {
  const int lane = threadIdx.x & 31;
  int c0 = lane < K ? cnt[lane] : 0;
  int c1 = lane + 32 < K ? cnt[lane + 32] : 0;
  int s0 = c0;
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, s0, o);
    if (lane >= o) s0 += v;
  }
  int tot0 = __shfl_sync(0xffffffffu, s0, 31);
  int s1 = c1;
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, s1, o);
    if (lane >= o) s1 += v;
  }
  if (lane < K) { voff[lane] = s0 - c0; base[lane] = s0 - c0; }
  if (lane + 32 < K) { voff[lane + 32] = tot0 + s1 - c1; base[lane + 32] = tot0 + s1 - c1; }
}

// The same placement for the fused path: slot[t] = position of track t among
// its event's tracks in vertex order (SlotT: int16 in shared memory for small
// events, int32 in global scratch above that); warp 0 only.
template <typename CidT, typename SlotT>
__device__ __forceinline__ void warp_place(const CidT* cid, int n, int* base, SlotT* slot) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int t0 = 0; t0 < n; t0 += 32) {
    int t = t0 + lane;
    int c = t < n ? static_cast<int>(cid[t]) : -1;
    unsigned peers = __match_any_sync(0xffffffffu, c);
    int rank = __popc(peers & lt);
    int leader = __ffs(peers) - 1;
    int b = c >= 0 ? base[c] : 0;
    __syncwarp();
    if (c >= 0) {
      if (PV_CHECK(b + rank < n, 6)) slot[t] = static_cast<SlotT>(b + rank);
      if (lane == leader) base[c] = b + __popc(peers);
    }
    __syncwarp();
  }
}

// Step (c) with the whole CTA, on the shared histogram N of one event (whole
// 32-bin tiles).  Every warp scans its share of the touched tiles and records,
// per tile, the bins where a run of bins above the threshold starts and ends
// (smask, emask); warp 0 lists the runs in z order (r_lo, r_hi: NT entries
// each); thread r walks run r (the proto-cluster) and counts its kept pieces,
// keeping the first two; a block-wide scan of the counts gives each piece its
// seed index.  Writes up to cap seeds into S in z order and returns their
// number (which may exceed cap) on every thread, or -1 on every thread when
// the event has more runs than threads (the caller then runs the one-warp
// search).  misc_scan: 2 NT/32 ints; misc_n: one int; mark: mark_cap entries
// of scratch for the recursive split, shared out among the proto-clusters
// (one whose share does not fit splits without scratch).  All threads of the
// CTA must call it.
template <int kSplit, int NT>
__device__ int block_find_seeds(const uint32_t* N, const uint32_t* tmask, const Consts& C,
                                SeedOut* S, int cap, uint32_t* smask, uint32_t* emask,
                                int16_t* r_lo, int16_t* r_hi, int* misc_scan, int* misc_n,
                                int16_t* mark, int mark_cap) {
  constexpr int NW = NT / 32;
  static_assert(kTileWords * 32 <= 4 * 32, "the run list covers at most 128 tiles");
  static_assert(2 * kRunRing * NW >= 2 * NT, "the run list lives in the proto-cluster rings");
  static_assert(kMiscWarpScan + 2 * NW <= kMiscInts, "two per-warp scans in misc");
  static_assert(sizeof(float4) * kFillChunk >= 2 * sizeof(uint32_t) * kTileWords * 32,
                "the tile masks live in the fill records");
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;

  // run starts and ends of the touched tiles, tile i of the mask to warp i mod NW
  int rank = 0;
#pragma unroll 1
  for (int w = 0; w < kTileWords; ++w) {
    uint32_t m = tmask[w];
    while (m) {
      const int tb = __ffs(m) - 1;
      m &= m - 1;
      const bool take = rank == warp;
      rank = rank + 1 == NW ? 0 : rank + 1;
      if (!take) continue;
      const int q = 32 * w + tb;
      const int bin = 32 * q + lane;
      const bool ab = bin < C.nbins && N[bin] > C.thr;
      const bool pa = bin >= 1 && bin - 1 < C.nbins && N[bin - 1] > C.thr;
      const bool na = bin + 1 < C.nbins && N[bin + 1] > C.thr;
      const unsigned st = __ballot_sync(0xffffffffu, ab && !pa);
      const unsigned en = __ballot_sync(0xffffffffu, ab && !na);
      if (lane == 0 && PV_CHECK(q < kTileWords * 32, 18)) {
        smask[q] = st;
        emask[q] = en;
      }
    }
  }
  __syncthreads();

  // warp 0: the runs in z order (lane l the tiles 4l .. 4l + 3)
  if (warp == 0) {
    uint32_t sm[4], em[4];
    int cs = 0, ce = 0;
    const uint32_t tw = (lane >> 3) < kTileWords ? tmask[lane >> 3] : 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = 4 * lane + k;
      const bool touched = ((tw >> (q & 31)) & 1u) != 0u;
      sm[k] = touched ? smask[q] : 0u;
      em[k] = touched ? emask[q] : 0u;
      cs += __popc(sm[k]);
      ce += __popc(em[k]);
    }
    // both counts in one scan (at most 16 runs per tile: 2048 < 2^15)
    int inc = cs | (ce << 16);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    const int tot = __shfl_sync(0xffffffffu, inc, 31);
    const int R = tot & 0xffff;
    if (R <= NT && (tot >> 16) == R) {
      int ps = (inc & 0xffff) - cs, pe = (inc >> 16) - ce;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int q0 = 32 * (4 * lane + k);
        while (sm[k]) {
          const int b = __ffs(sm[k]) - 1;
          sm[k] &= sm[k] - 1;
          if (PV_CHECK(ps < NT, 19)) r_lo[ps] = static_cast<int16_t>(q0 + b);
          ++ps;
        }
        while (em[k]) {
          const int b = __ffs(em[k]) - 1;
          em[k] &= em[k] - 1;
          if (PV_CHECK(pe < NT, 19)) r_hi[pe] = static_cast<int16_t>(q0 + b);
          ++pe;
        }
      }
    }
    if (lane == 0) *misc_n = ((tot >> 16) == R && R <= NT) ? R : -1;
  }
  __syncthreads();
  const int R = *misc_n;
  if (R < 0) return -1;

  // thread r walks run r
  int a = 0, b = -1;
  uint64_t total = 0;
  if (tid < R) {
    a = r_lo[tid];
    b = r_hi[tid];
    // (a run's bounds always lie in the histogram; the test keeps a broken
    // invariant from reading outside it)
    if (!(a >= 0 && a <= b && b < C.nbins)) {
      (void)PV_CHECK(false, 17);
      b = a - 1;
    }
    for (int i = a; i <= b; ++i) total += N[i];
  }
  const uint64_t t_min = C.t_pp < C.t_gas ? C.t_pp : C.t_gas;
  const bool walk = b >= a && total >= t_min;
  // each walked proto-cluster's share of the scratch (recursive split): a
  // block-wide scan of their lengths
  int16_t* my_mark = nullptr;
  if constexpr (kSplit == PV_SPLIT_RECURSIVE) {
    const int len = walk ? b - a + 1 : 0;
    int end = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, end, o);
      if (lane >= o) end += v;
    }
    if (lane == 31) misc_scan[NW + warp] = end;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < NW; ++w)
      if (w < warp) end += misc_scan[NW + w];
    if (walk && end <= mark_cap) my_mark = mark + (end - len);
  }
  int kept = 0, lo1 = 0, hi1 = 0, im1 = 0, lo2 = 0, hi2 = 0, im2 = 0;
  if (walk) {
    split_pieces<kSplit>(N, a, b, total, C,
                         [&](int lo, int hi, uint64_t integral, int im) {
      if (keep_piece(integral, im, C)) {
        if (kept == 0) {
          lo1 = lo; hi1 = hi; im1 = im;
        } else if (kept == 1) {
          lo2 = lo; hi2 = hi; im2 = im;
        }
        ++kept;
      }
    }, my_mark);
  }
  // each piece's index: exclusive scan of the counts in run order
  int incl = kept;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) misc_scan[warp] = incl;
  __syncthreads();
  int pos = incl - kept, n_kept = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const int v = misc_scan[w];
    if (w < warp) pos += v;
    n_kept += v;
  }
  if (kept >= 1 && kept <= 2 && pos < cap) {
    put_seed(N, C, S, pos, lo1, hi1, im1);
    if (kept == 2 && pos + 1 < cap) put_seed(N, C, S, pos + 1, lo2, hi2, im2);
  }
  if (kept > 2 && pos < cap) {
    split_pieces<kSplit>(N, a, b, total, C,
                         [&](int lo, int hi, uint64_t integral, int im) {
      if (keep_piece(integral, im, C)) {
        if (pos < cap) put_seed(N, C, S, pos, lo, hi, im);
        ++pos;
      }
    }, my_mark);
  }
  return n_kept;
}

// What group_fit returns for a vertex without tracks: singular at the first
// iteration (or unconverged with no iteration when max_iter is 0).
__device__ __forceinline__ VertexOut empty_fit(const Consts& C) {
  VertexOut v;
  v.x = v.y = v.z = 0.f;
  for (int c = 0; c < 6; ++c) v.cov[c] = 0.f;
  v.chi2 = 0.f;
  v.ndof = -3.f;
  v.n_tracks = 0;
  v.n_iter = C.max_iter >= 1 ? 1 : 0;
  v.status = C.max_iter >= 1 ? PV_ST_SINGULAR : PV_ST_MAXITER;
  return v;
}

// Write the fit of vertex k of event e (result relative to the seed at
// (xs, ys, zs)) with its selection status.
__device__ __forceinline__ void write_vertex(const Consts& C, const OutPtrs& O, int e, int k,
                                             float xs, float ys, float zs, const VertexOut& v) {
  size_t q = static_cast<size_t>(e) * O.cap + k;
  float x = xs + v.x, y = ys + v.y, z = zs + v.z;
  int st = select_vertex(x, y, z, v.n_tracks, v.status, C);
  O.x[q] = x;
  O.y[q] = y;
  O.z[q] = z;
  if (O.cov) {
#pragma unroll
    for (int c = 0; c < 6; ++c) O.cov[q * 6 + c] = v.cov[c];
  }
  if (O.chi2) O.chi2[q] = v.chi2;
  if (O.ndof) O.ndof[q] = v.ndof;
  if (O.n_tracks) O.n_tracks[q] = v.n_tracks;
  if (O.n_iter) O.n_iter[q] = v.n_iter;
  if (O.status) O.status[q] = st;
}

// A seed without tracks gets the result of an empty fit at its seed
// position.  Rare, and kept out of line so that its registers do not count
// against the find kernel's occupancy.
static __device__ __noinline__ void write_empty_vertex(const Consts& C, const OutPtrs& O,
                                                const SeedOut* S, int e, int k) {
  write_vertex(C, O, e, k, S->x[k], S->y[k], S->z[k], empty_fit(C));
}

// Serving: the vertices a CTA has found and not yet fitted, from up to
// kServeReqs requests.  The serving kernel fits them kServeFitBatch at a time
// (four 8-lane groups in each of its four warps), so it lets them gather
// before a round while more published events wait.
constexpr int kServeFitBatch = 16;
// a round starts once this many are queued (so that most rounds, with the
// vertices of the event that crossed it, still take one pass)
constexpr int kServeRoundAt = 12;
constexpr int kServeQueue = kServeRoundAt - 1 + kMaxSeeds;   // most vertices queued
constexpr int kServeReqs = 4;
struct ServeReq {                    // a request with queued events
  OutPtrs O;
  float4* A;
  float2* W;
  unsigned long long slot, target, seq;
  int events;                        // its events found since the last round
};
struct ServeVertex {                 // one vertex to fit (cnt > 0 tracks)
  int off;                           // fit inputs A[off ..], W[off ..] of its request
  int cnt, e, k, req;
  float x, y, z;                     // seed position
};
struct ServeQueue {
  int n;                             // vertices queued
  int nreq;                          // requests with events since the last round
  int16_t order[kServeQueue];
  ServeVertex v[kServeQueue];
  ServeReq req[kServeReqs];
};

__device__ __forceinline__ bool offsets_bad(int64_t b0, int64_t b1, int64_t n_tracks) {
  return b0 < 0 || b1 < b0 || b1 > n_tracks || b1 - b0 > 0x7fffffffLL;
}


// ---------------------------------------------------------------------------
// find kernel (fused path, stage 1)
//
// kFind:    steps (a)-(d1); outputs seeds and assignments.
// kFindFit: the same, then every associated track's fit inputs (global
//           scratch, vertex order) and one work item per vertex for the fit
//           kernel.
// kFit:     seeds and assignments from the caller, then fit inputs and work.
//
// One event at a time per CTA, claimed from a global counter:
//   fill   in passes of up to CHUNK tracks: each thread prepares its tracks
//          (step a) into records with their place in a block-wide prefix sum
//          of the window sizes; then the pass's (track, bin) items are split
//          evenly over the threads, each walking its range of consecutive
//          items (one CDF per item, the right edge carried over as the next
//          bin's left edge)
//   peaks  every warp scans its share of the touched tiles, warp 0 lists the
//          runs, thread r walks run r (warp 0 alone beyond NT runs)
//   assoc  block-cooperative association with the removal loop
//   place  per 32-track round, the tracks of each vertex are ranked with
//          __match_any_sync and the rounds' counts summed, giving each track
//          its place in vertex order (track-index order within a vertex);
//          events above kSmallCap tracks are placed by warp 0 in one pass
//   inputs every associated track's fit inputs at its vertex's seed

template <int PROFILE>
__device__ __forceinline__ int item_q(int i, int j0, float z, float inv, int tq, const Consts& C) {
  return profile_q<PROFILE>(i, j0, z, inv, tq, C);
}

// 48 registers per thread (a few bytes spill), so that ten 128-thread CTAs
// share an SM: the shared memory of an event (22 KB) allows ten as well
// A CTA's shared state before its first event: an empty histogram and tile mask.
template <int MODE, int NT>
__device__ __forceinline__ void find_prologue(const Consts& C, unsigned char* smem,
                                              const Layout& Lo) {
  if (MODE & kFind) {
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + Lo.hist);
    for (int i = threadIdx.x; i < C.ntiles * 32; i += NT) hist[i] = 0u;
  }
  uint32_t* tmask = reinterpret_cast<uint32_t*>(smem + Lo.tmask);
  if (threadIdx.x < kTileWords) tmask[threadIdx.x] = 0u;
}

// The find kernel's work on one event e (all threads of the CTA; smem is the
// dynamic shared memory laid out by make_layout).  next_slot / e_next: the
// event claimed for the next iteration, published in shared memory after the
// fill (NULL when the caller claims otherwise).  With kServe in MODE the
// event's vertices join the CTA's queue Q (request Q->nreq - 1) instead of the
// fit kernel's work lists.
template <int MODE, int NT, int FLAV>
__device__ __forceinline__ void find_event(const Consts& C, const TrackPtrs& T, const SeedPtrs& SP,
                                           const OutPtrs& O, const TrackScratch& G,
                                           unsigned char* smem, int e, int* next_slot,
                                           int e_next, ServeQueue* Q = nullptr) {
  constexpr int SPLIT = flavour_split(FLAV);
  constexpr int PROFILE = flavour_profile(FLAV);
  constexpr int NW = NT / 32;
  constexpr int KPT = fill_per_thread(NT);       // tracks a thread prepares per fill pass
  constexpr int CHUNK = KPT * NT;
  constexpr int RPW = (kPlaceRounds + NW - 1) / NW;   // placement rounds per warp
  static_assert(CHUNK <= kFillChunk, "fill pass larger than its records");
  const Layout Lo = make_layout(C.nbins, MODE & ~kServe, NT, SPLIT == PV_SPLIT_RECURSIVE);
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem + Lo.hist);
  uint32_t* tmask = reinterpret_cast<uint32_t*>(smem + Lo.tmask);
  SeedOut* S = reinterpret_cast<SeedOut*>(smem + Lo.seeds);
  int* misc = reinterpret_cast<int*>(smem + Lo.misc);
  int16_t* s_center = reinterpret_cast<int16_t*>(smem + Lo.center);
  int8_t* s_cid = reinterpret_cast<int8_t*>(smem + Lo.cid);
  float4* recs = reinterpret_cast<float4*>(smem + Lo.uni);
  int* alive = reinterpret_cast<int*>(smem + Lo.uni);
  int* part = alive + kMaxSeeds;
  int* cnt = part + kMaxSeeds;
  int* voff = cnt + kMaxSeeds;
  int* base = voff + kMaxSeeds;
  int16_t* rc = reinterpret_cast<int16_t*>(base + kMaxSeeds);   // [kPlaceRounds][kMaxSeeds]

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int16_t* pc_lo = reinterpret_cast<int16_t*>(smem + Lo.ring) + warp * 2 * kRunRing;
  int16_t* pc_hi = pc_lo + kRunRing;

    const int64_t b0 = T.off[e], b1 = T.off[e + 1];
    if (offsets_bad(b0, b1, T.n_tracks)) {
      if (tid == 0) {
        O.n_per_event[e] = 0;
        if (O.event_status) O.event_status[e] = PV_EV_BAD_OFFSETS;
      }
      if (tid == NT - 1 && next_slot) *next_slot = e_next;
      __syncthreads();
      return;   // uniform: every thread read the same offsets
    }
    const int n = static_cast<int>(b1 - b0);
    const bool small = n <= kSmallCap;
    int16_t* center = small ? s_center : G.center + b0;
    int8_t* cid = small ? s_cid : G.cid + b0;
    int Ka = 0;

    if (MODE & kFind) {
      // ---- (a) + (b): the fill, in passes of up to CHUNK tracks
      for (int c0 = 0; c0 < n; c0 += CHUNK) {
        // prepare: thread tid's tracks c0 + k NT + tid become records tid KPT
        // + k (window size 0 for a track without one)
        uint32_t tm[kTileWords];
#pragma unroll
        for (int w = 0; w < kTileWords; ++w) tm[w] = 0u;
        int ic = 0;
#pragma unroll 1
        for (int k = 0; k < KPT; ++k) {
          const int t = c0 + k * NT + tid;
          float zr = 0.f, ir = 0.f;
          int jr = 0, nr = 0;
          if (t < n) {
            const int64_t i = b0 + t;
            const float x = T.x[i], y = T.y[i], z = T.z[i], tx = T.tx[i];
            const float ty = T.ty[i], cxx = T.cxx[i], cxtx = T.cxtx[i], ctxtx = T.ctxtx[i];
            if constexpr ((MODE & kStage) != 0) {
              G.stage[0][i] = x; G.stage[1][i] = y; G.stage[2][i] = z; G.stage[3][i] = tx;
              G.stage[4][i] = ty; G.stage[5][i] = cxx; G.stage[6][i] = cxtx; G.stage[7][i] = ctxtx;
            } else if constexpr ((MODE & kFit) != 0) {
              // the fit-input pass reads the y-covariance columns: bring them into L2
              prefetch_l2(T.cyy + i);
              prefetch_l2(T.cyty + i);
              prefetch_l2(T.ctyty + i);
            }
            const Prep p = prepare_track<PROFILE>(x, y, z, tx, ty, cxx, cxtx, ctxtx, C);
            if (PV_CHECK(!small || t < kSmallCap, 7))
              center[t] = static_cast<int16_t>(p.filled ? p.center : -1);
            if (p.filled) {
              zr = p.zpoca;
              jr = p.j0;
              nr = p.j1 - p.j0 + 1;
              if constexpr (PROFILE == PV_PROFILE_TEMPLATE) {
                ir = __int_as_float(p.tq);
              } else {
                float sp = __fmul_rn(kSqrt5, p.sigma);
                if (sp < kSMin) sp = 0.0f;
                ir = (nr > 1 && sp > 0.0f) ? __fdiv_rn(1.0f, sp) : 0.0f;
              }
              // the 32-bin tiles the window touches
              const int q0 = (p.j0 < 0 ? 0 : p.j0) >> 5;
              const int q1 = (p.j1 >= C.nbins ? C.nbins - 1 : p.j1) >> 5;
#pragma unroll
              for (int w = 0; w < kTileWords; ++w) {
                const int lo = q0 > 32 * w ? q0 : 32 * w;
                const int hi = q1 < 32 * w + 31 ? q1 : 32 * w + 31;
                if (lo <= hi) {
                  const int len = hi - lo + 1;
                  tm[w] |= (len == 32 ? 0xffffffffu : ((1u << len) - 1u)) << (lo - 32 * w);
                }
              }
              ic += nr;
            }
          }
          recs[tid * KPT + k] = make_float4(zr, ir, __int_as_float((jr & 0xffff) | (nr << 16)), 0.f);
        }
#pragma unroll
        for (int w = 0; w < kTileWords; ++w) {
          const uint32_t m = __reduce_or_sync(0xffffffffu, tm[w]);
          if (lane == w && m != 0u && (tmask[w] & m) != m) atomicOr(tmask + w, m);
        }
        // block-wide exclusive prefix of the window sizes in record order
        int incl = ic;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        if (lane == 31) misc[kMiscWarpScan + warp] = incl;
        __syncthreads();
        int items = 0, off = incl - ic;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const int v = misc[kMiscWarpScan + w];
          if (w < warp) off += v;
          items += v;
        }
#pragma unroll 1
        for (int k = 0; k < KPT; ++k) {
          float4* r = recs + tid * KPT + k;
          r->w = __int_as_float(off);
          off += __float_as_int(r->z) >> 16;
        }
        __syncthreads();
        // the pass's items split evenly over the threads: each walks its
        // range of consecutive items (the records without a window hold
        // none and are stepped over)
        const int lo = static_cast<int>((static_cast<long long>(items) * tid) / NT);
        const int hi = static_cast<int>((static_cast<long long>(items) * (tid + 1)) / NT);
        if (lo < hi) {
          int a = 0, bb = CHUNK - 1;       // the last record starting at or before lo
          while (a < bb) {
            const int mid = (a + bb + 1) >> 1;
            if (__float_as_int(recs[mid].w) <= lo) a = mid;
            else bb = mid - 1;
          }
          float4 R = recs[a];
          int jj = __float_as_int(R.z);
          int j0 = static_cast<int16_t>(jj & 0xffff), nb = jj >> 16;
          int tq = __float_as_int(R.y);
          int i = lo - __float_as_int(R.w);
          int ql = i > 0 ? item_q<PROFILE>(i, j0, R.x, R.y, tq, C) : 0;
          for (int it = lo; it < hi; ++it) {
            const int qr = (i + 1 < nb) ? item_q<PROFILE>(i + 1, j0, R.x, R.y, tq, C) : kOne;
            const int w = qr - ql;
            const int j = j0 + i;
            if (w > 0 && j >= 0 && j < C.nbins && PV_CHECK(j < C.ntiles * 32, 2))
              atomicAdd(hist + j, static_cast<uint32_t>(w));
            ql = qr;
            if (++i == nb && it + 1 < hi) {
              do {
                if (a + 1 >= CHUNK) {        // (cannot happen: the items are the records')
                  (void)PV_CHECK(false, 14);
                  nb = -1;
                  break;
                }
                R = recs[++a];
                jj = __float_as_int(R.z);
                nb = jj >> 16;
              } while (nb == 0);
              if (nb < 0) break;
              j0 = static_cast<int16_t>(jj & 0xffff);
              tq = __float_as_int(R.y);
              i = 0;
              ql = 0;
            }
          }
        }
        __syncthreads();
      }
      if (tid == NT - 1 && next_slot) *next_slot = e_next;

      // ---- (c): seeds from the touched tiles, with the whole CTA (with warp
      // 0 alone when the event has more runs than threads)
      int16_t* mark = reinterpret_cast<int16_t*>(smem + Lo.mark);   // (x86 flavour)
      int16_t* runs = reinterpret_cast<int16_t*>(smem + Lo.ring);
      uint32_t* tiles = reinterpret_cast<uint32_t*>(smem + Lo.uni);
      int Kall = block_find_seeds<SPLIT, NT>(hist, tmask, C, S, O.cap, tiles,
                                             tiles + kTileWords * 32, runs, runs + NT,
                                             misc + kMiscWarpScan, misc + kMiscFlag, mark,
                                             Lo.mark_cap);
      if (Kall < 0) {
        if (warp == 0) {
          const int K = warp_find_seeds<false, SPLIT>(hist, tmask, C, S, O.cap, pc_lo, pc_hi, mark,
                                                      Lo.mark_cap);
          if (lane == 0) misc[kMiscK] = K;
        }
        __syncthreads();
        Kall = misc[kMiscK];
      } else {
        __syncthreads();
      }
      const int K = Kall < O.cap ? Kall : O.cap;
      // clear the touched tiles for the next event (warp w the tiles of mask
      // word w, w + NW, ...)
      for (int w = warp; w < kTileWords; w += NW) {
        uint32_t m = tmask[w];
        while (m) {
          const int tb = __ffs(m) - 1;
          m &= m - 1;
          hist[(w * 32 + tb) * 32 + lane] = 0u;
        }
      }
      // (d1): association with the removal loop
      Ka = block_associate(center, cid, n, S, K, C, alive, part, cnt, misc + kMiscFlag);
      if (tid < kTileWords) tmask[tid] = 0u;
      // seed positions of the survivors: z from the bins around the maximum
      // in binary64 (Sec. 3.3, R9), x and y on the beamline
      if (tid < Ka) {
        const float zs = seed_z_from(S->nm[tid], S->ni[tid], S->np[tid], S->bin[tid], C);
        S->z[tid] = zs;
        S->x[tid] = __fadd_rn(C.x_b, __fmul_rn(C.tx_b, zs));
        S->y[tid] = __fadd_rn(C.y_b, __fmul_rn(C.ty_b, zs));
      }
      __syncthreads();
      for (int t = tid; t < n; t += NT) O.track_vertex[b0 + t] = cid[t];
      if (tid == 0) {
        O.n_per_event[e] = Ka;
        if (O.event_status) O.event_status[e] = Kall > O.cap ? PV_EV_SEED_OVERFLOW : 0;
      }
      if (tid < Ka) {
        size_t q = static_cast<size_t>(e) * O.cap + tid;
        if (O.bin_lo) O.bin_lo[q] = S->lo[tid];
        if (O.bin_hi) O.bin_hi[q] = S->hi[tid];
        if (O.bin_max) O.bin_max[q] = S->bin[tid];
        if (MODE == kFind) {
          O.x[q] = S->x[tid];
          O.y[q] = S->y[tid];
          O.z[q] = S->z[tid];
        }
      }
    } else {
      // fit only: seeds and assignment from the caller
      int K = SP.n_per_event[e];
      int capk = SP.cap < O.cap ? SP.cap : O.cap;
      capk = capk < kMaxSeeds ? capk : kMaxSeeds;
      K = K < 0 ? 0 : (K > capk ? capk : K);
      if (tid < K) {
        size_t q = static_cast<size_t>(e) * SP.cap + tid;
        S->x[tid] = SP.x[q];
        S->y[tid] = SP.y[q];
        S->z[tid] = SP.z[q];
        S->bin[tid] = -1;             // the seed is given, not a histogram maximum
        cnt[tid] = 0;
      }
      __syncthreads();
      for (int t = tid; t < n; t += NT) {
        int c = SP.track_vertex[b0 + t];
        c = (c >= 0 && c < K) ? c : -1;
        cid[t] = static_cast<int8_t>(c);
        if (c >= 0) atomicAdd(cnt + c, 1);
        if (O.track_vertex != SP.track_vertex) O.track_vertex[b0 + t] = c;
      }
      if (tid == 0 && O.n_per_event != SP.n_per_event) O.n_per_event[e] = K;
      Ka = K;
      if (tid == NT - 1 && next_slot) *next_slot = e_next;
      __syncthreads();
    }

    if (MODE & kFit) {
      // each track's place in vertex order, one work item per vertex with
      // tracks (a vertex without tracks gets the singular result of an empty
      // fit here), then every track's fit inputs at its vertex's seed,
      // written in vertex order for the fit kernel
      if (warp == 0) warp_offsets(cnt, Ka, voff, base);
      if (small) {
        for (int i = tid; i < kPlaceRounds * kMaxSeeds; i += NT) rc[i] = 0;
      }
      __syncthreads();
      int myc[RPW], myrank[RPW];
      if (small) {
        // per round of 32 tracks: each vertex's tracks ranked in track order
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
          const int r = warp + k * NW;
          const int t = 32 * r + lane;
          int c = -1;
          if (r < kPlaceRounds && t < n) c = static_cast<int>(cid[t]);
          const unsigned peers = __match_any_sync(0xffffffffu, c);
          myc[k] = c;
          myrank[k] = __popc(peers & lt);
          if (c >= 0 && lane == __ffs(peers) - 1 && PV_CHECK(c < kMaxSeeds, 16))
            rc[r * kMaxSeeds + c] = static_cast<int16_t>(__popc(peers));
        }
      } else if (warp == 0) {
        warp_place(cid, n, base, G.slot + b0);
      }
      if constexpr ((MODE & kServe) == 0) if (warp == 1 || NW == 1) {
        // one work item per vertex with tracks, in the list of its size class
        const int c0 = (lane < Ka && cnt[lane] > 0) ? work_class(cnt[lane]) : -1;
        const int c1 = (lane + 32 < Ka && cnt[lane + 32] > 0) ? work_class(cnt[lane + 32]) : -1;
        // per class: lane c reserves the class's entries (one round trip for
        // all classes), then each vertex takes its rank within its class
        int mine = 0;
#pragma unroll 1
        for (int c = 0; c < kWorkClasses; ++c) {
          const int k = __popc(__ballot_sync(0xffffffffu, c0 == c)) +
                        __popc(__ballot_sync(0xffffffffu, c1 == c));
          if (lane == c) mine = k;
        }
        int wb = 0;
        if (lane < kWorkClasses && mine > 0) wb = atomicAdd(G.counters + 1 + lane, mine);
        int i0 = 0, i1 = 0;
#pragma unroll 1
        for (int c = 0; c < kWorkClasses; ++c) {
          const unsigned m0 = __ballot_sync(0xffffffffu, c0 == c);
          const unsigned m1 = __ballot_sync(0xffffffffu, c1 == c);
          const int bc = __shfl_sync(0xffffffffu, wb, c);
          if (c0 == c) i0 = bc + __popc(m0 & lt);
          if (c1 == c) i1 = bc + __popc(m0) + __popc(m1 & lt);
        }
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          const int k = lane + 32 * h;
          if (k >= Ka) continue;
          const int cl = h ? c1 : c0;
          const int idx = h ? i1 : i0;
          if (cl >= 0) {
            if (idx < class_pick(G.cls_cap, cl)) {
              VertexWork w;
              w.off = static_cast<int>(b0 + voff[k]);
              w.e = e;
              w.kc = k | (cnt[k] << 8);
              w.pad0 = 0;
              w.x = __float_as_uint(S->x[k]);
              w.y = __float_as_uint(S->y[k]);
              w.z = __float_as_uint(S->z[k]);
              w.pad1 = 0;
              if (PV_CHECK(idx >= 0, 9)) G.work[class_pick(G.cls_base, cl) + idx] = w;
            }
          } else {
            write_empty_vertex(C, O, S, e, k);
          }
        }
      }
      __syncthreads();
      // fit inputs (the staged mode reads its first eight columns back from
      // the device copy the fill wrote, the other three from host memory)
      auto fit_input = [&](int t, int c, int sl) {
        const int64_t i = b0 + t;
        float x, y, z, tx, ty, cxx, cxtx, ctxtx;
        if constexpr ((MODE & kStage) != 0) {
          x = G.stage[0][i]; y = G.stage[1][i]; z = G.stage[2][i]; tx = G.stage[3][i];
          ty = G.stage[4][i]; cxx = G.stage[5][i]; cxtx = G.stage[6][i]; ctxtx = G.stage[7][i];
        } else {
          x = T.x[i]; y = T.y[i]; z = T.z[i]; tx = T.tx[i];
          ty = T.ty[i]; cxx = T.cxx[i]; cxtx = T.cxtx[i]; ctxtx = T.ctxtx[i];
        }
        make_fit_track(x, y, z, tx, ty, cxx, cxtx, ctxtx, T.cyy[i], T.cyty[i], T.ctyty[i],
                       S->x[c], S->y[c], S->z[c], G.A + b0 + sl, G.W + b0 + sl);
      };
      int16_t* s_slot = s_center;      // the center bins are spent
      if (small) {
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
          const int r = warp + k * NW;
          const int c = myc[k];
          if (c < 0) continue;
          int sl = voff[c] + myrank[k];
          for (int q = 0; q < r; ++q) sl += rc[q * kMaxSeeds + c];
          s_slot[32 * r + lane] = static_cast<int16_t>(sl);
        }
        __syncthreads();
      }
      for (int t = tid; t < n; t += NT) {
        const int c = static_cast<int>(cid[t]);
        if (c < 0) continue;
        const int sl = small ? static_cast<int>(s_slot[t]) : G.slot[b0 + t];
        if (!PV_CHECK(sl >= 0 && sl < n && c < kMaxSeeds, 10)) continue;
        fit_input(t, c, sl);
      }
      if constexpr ((MODE & kServe) != 0) {
        // serving: the vertices with tracks join the CTA's queue, a vertex
        // without tracks gets the singular result of an empty fit now
        if (tid < Ka) {
          const int c = cnt[tid];
          if (c > 0) {
            const int qi = atomicAdd(&Q->n, 1);
            if (PV_CHECK(qi < kServeQueue, 20)) {
              ServeVertex& v = Q->v[qi];
              v.off = static_cast<int>(b0 + voff[tid]);
              v.cnt = c;
              v.e = e;
              v.k = tid;
              v.req = Q->nreq - 1;
              v.x = S->x[tid];
              v.y = S->y[tid];
              v.z = S->z[tid];
            }
          } else {
            write_empty_vertex(C, O, S, e, tid);
          }
        }
      }
    }
}

}  // namespace pvk
