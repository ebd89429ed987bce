// pv_kernels.cu -- sm_103a kernels of the primary-vertex library.
//
// Fused path: two persistent kernels.  The find kernel takes one event at a
// time per CTA from a global work counter (uneven event sizes balance
// themselves), keeps the z histogram in shared memory (cleared only where
// tracks wrote, tracked by a 32-bin tile mask), finds seeds with warp ballots,
// associates tracks, and writes each track's fit inputs, in vertex order, to
// an L2-resident scratch with one work item per vertex.  The fit kernel then
// fits vertices of all events, one 8-lane group per vertex, at high
// occupancy.  Per-track association state stays in shared memory for events
// up to kSmallCap tracks and in global scratch for larger events, so no event
// size is refused.
//
// Plain path: one kernel per step (extrapolate / histogram / peaks /
// associate / fit), one CTA per event, histograms and per-track state in
// global memory: the per-step design the fused path is measured against.
#include "pv_find.cuh"

namespace pvk {

using namespace pvdev;

bool check_report(unsigned* count, unsigned* first) {
#if PV_CHECKED
  unsigned zero = 0, c = 0, f = 0;
  cudaDeviceSynchronize();
  cudaMemcpyFromSymbol(&c, g_check_count, sizeof(unsigned));
  cudaMemcpyFromSymbol(&f, g_check_first, sizeof(unsigned));
  cudaMemcpyToSymbol(g_check_count, &zero, sizeof(unsigned));
  cudaMemcpyToSymbol(g_check_first, &zero, sizeof(unsigned));
  unsigned c2 = 0, f2 = 0;
  serve_check_report(&c2, &f2);
  *count = c + c2;
  *first = c ? f : f2;
  return true;
#else
  *count = 0;
  *first = 0;
  return false;
#endif
}

size_t fused_smem_bytes(int nbins, int mode, int nt, bool rec) {
  return make_layout(nbins, mode, nt, rec).total;
}

// ---------------------------------------------------------------------------
// pieces shared by the fused and the plain kernels

// Stable placement of tracks by vertex (track-index order inside a vertex);
// warp 0 only.  base[] is advanced.
__device__ __forceinline__ void warp_slots(const int* cid, int n, int* base, int* slot) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int t0 = 0; t0 < n; t0 += 32) {
    int t = t0 + lane;
    int c = t < n ? cid[t] : -1;
    unsigned peers = __match_any_sync(0xffffffffu, c);
    int rank = __popc(peers & lt);
    int leader = __ffs(peers) - 1;
    int b = c >= 0 ? base[c] : 0;
    __syncwarp();
    if (c >= 0) {
      slot[t] = b + rank;
      if (lane == leader) base[c] = b + __popc(peers);
    }
    __syncwarp();
  }
}

// Fit every vertex of one event (block-cooperative; used by the plain path).
// A, W: per-track fit inputs in vertex order; voff/cnt: vertex ranges.
template <int kAccum>
__device__ void block_fit_event(const Consts& C, const SeedOut* S, int Ka, const int* voff,
                                const int* cnt, const float4* A, const float2* W,
                                const OutPtrs& O, int e) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int vb = warp * kGroupsPerWarp; vb < Ka; vb += nw * kGroupsPerWarp) {
    int k = vb + (lane >> 3);
    bool has = k < Ka;
    int cntk = has ? cnt[k] : -1;
    int o = has ? voff[k] : 0;
    VertexOut v;
    const int r = lane & (kGroup - 1);
    group_fit<kAccum>(A + o + r, W + o + r, kGroup, cntk, C, &v);
    if (has && (lane & 7) == 0) write_vertex(C, O, e, k, S->x[k], S->y[k], S->z[k], v);
  }
}

// Per-track fit inputs in vertex order.
__device__ __forceinline__ void block_fit_inputs(const TrackPtrs& T, int64_t b0, int n,
                                                 const int* cid, const int* slot, const SeedOut* S,
                                                 float4* A, float2* W) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    int c = cid[t];
    if (c < 0) continue;
    int64_t i = b0 + t;
    int s = slot[t];
    make_fit_track(T.x[i], T.y[i], T.z[i], T.tx[i], T.ty[i], T.cxx[i], T.cxtx[i], T.ctxtx[i],
                   T.cyy[i], T.cyty[i], T.ctyty[i], S->x[c], S->y[c], S->z[c], A + s, W + s);
  }
}

// 48 registers per thread (a few bytes spill), so that ten 128-thread CTAs
// share an SM: the shared memory of an event (22 KB) allows ten as well
template <int MODE, int NT, int FLAV = 0>
__global__ void __launch_bounds__(NT, 1280 / NT)
find_kernel(Consts C, TrackPtrs T, SeedPtrs SP, OutPtrs O, TrackScratch G) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout Lo = make_layout(C.nbins, MODE, NT, flavour_split(FLAV) == PV_SPLIT_RECURSIVE);
  find_prologue<MODE, NT>(C, smem, Lo);
  int* misc = reinterpret_cast<int*>(smem + Lo.misc);
  if (threadIdx.x == 0) misc[0] = atomicAdd(G.counters, 1);
  __syncthreads();
  for (int iter = 0;; ++iter) {
    const int e = misc[iter & 1];
    if (e >= T.n_events) break;
    // the next event is claimed while this one runs, by the last thread; the
    // barrier after the fill publishes it
    int e_next = 0;
    if (threadIdx.x == NT - 1) e_next = atomicAdd(G.counters, 1);
    find_event<MODE, NT, FLAV>(C, T, SP, O, G, smem, e, misc + ((iter + 1) & 1), e_next);
    __syncthreads();   // shared state is reused by the next event
  }
}

// ---------------------------------------------------------------------------
// vertex fit kernel (fused path, stage 2): every 8-lane group fits one vertex
// of any event from the fit inputs the find kernel wrote in vertex order;
// warps take 4 work items at a time, largest size class first.

template <int kAccum, int FT>
__global__ void __launch_bounds__(FT)
fit_kernel(Consts C, TrackPtrs T, TrackScratch G, OutPtrs O) {
  const int lane = threadIdx.x & 31;
  const int r = lane & (kGroup - 1);
  // the classes' listed vertices, largest class first
  static_assert(kWorkClasses == 4, "class selection below");
  const int n0 = min(G.counters[1], G.cls_cap[0]), n1 = min(G.counters[2], G.cls_cap[1]);
  const int n2 = min(G.counters[3], G.cls_cap[2]), n3 = min(G.counters[4], G.cls_cap[3]);
  const int n = n0 + n1 + n2 + n3;
  for (;;) {
    int b = 0;
    if (lane == 0) b = atomicAdd(G.counters + 1 + kWorkClasses, kGroupsPerWarp);
    b = __shfl_sync(0xffffffffu, b, 0);
    if (b >= n) break;
    const int v = b + (lane >> 3);
    const bool has = v < n;
    VertexWork w;
    w.off = 0; w.e = 0; w.kc = 0; w.pad0 = 0; w.x = w.y = w.z = 0u; w.pad1 = 0;
    if (has) {
      long long q;
      if (v < n3) q = G.cls_base[3] + v;
      else if (v < n3 + n2) q = G.cls_base[2] + (v - n3);
      else if (v < n3 + n2 + n1) q = G.cls_base[1] + (v - n3 - n2);
      else q = G.cls_base[0] + (v - n3 - n2 - n1);
      w = G.work[q];
    }
    const int k = w.kc & 0xff;
    const int cntk = has ? (w.kc >> 8) : -1;
    // (a checked build that finds a bad vertex range fits no track for it;
    // the warp stays converged for the fit's shuffles)
    const int cnt_g = PV_CHECK(cntk <= 0 || (w.off >= 0 && w.off + cntk <= T.n_tracks), 11)
                          ? cntk : 0;
    VertexOut out;
    group_fit<kAccum>(G.A + w.off + r, G.W + w.off + r, kGroup, cnt_g, C, &out);
    if (has && r == 0)
      write_vertex(C, O, w.e, k, __uint_as_float(w.x), __uint_as_float(w.y), __uint_as_float(w.z),
                   out);
  }
}

// ---------------------------------------------------------------------------
// GPU-flavour multi-vertex fit (Sec. 3.5): every track enters every vertex of
// its event with w_ij = exp(-chi2_ij/2) / (exp(-chi2_cut/2) + sum_k
// exp(-chi2_ik/2)), the other vertices k at their seed positions.

// A track's fit inputs for one vertex and its competing term: the sum over the
// event's seeds of exp(-chi2/2) at the seed positions (S) without this
// vertex's own seed term.
struct MvTrack {
  float X, Y, tx, ty, wx, wy, comp;
};

__device__ __forceinline__ float mv_seed_term(float X, float Y, float wx, float wy) {
  return __expf(-0.5f * (X * X * wx + Y * Y * wy));
}

// a, b, c4: the track's packed record (three float4, written by mv_sums_kernel).
__device__ __forceinline__ bool mv_track_rec(const float4& a, const float4& b, const float4& c4,
                                             float xs, float ys, float zs, MvTrack* m) {
  float4 A;
  float2 W;
  make_fit_track(a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c4.x, c4.y, c4.z, xs, ys, zs, &A, &W);
  if (!(W.x > 0.0f)) return false;
  m->X = A.x; m->Y = A.y; m->tx = A.z; m->ty = A.w; m->wx = W.x; m->wy = W.y;
  const float c = c4.w - mv_seed_term(A.x, A.y, W.x, W.y);
  m->comp = c > 0.0f ? c : 0.0f;
  return true;
}
__device__ __forceinline__ bool mv_track(const float4* p, float xs, float ys, float zs,
                                         MvTrack* m) {
  return mv_track_rec(p[0], p[1], p[2], xs, ys, zs, m);
}

__device__ __forceinline__ float mv_weight(float c2, float comp, const Consts& C) {
  const float e = __expf(-0.5f * c2);
  return e / (C.mv_ecut + comp + e);
}

// The sheared position (and shear) a vertex's last weights were taken at.
using MvLast = MvLastState;

__device__ __forceinline__ float mv_chi2_at(const MvTrack& m, const MvLast& L) {
  const float dtx = m.tx - L.cx, dty = m.ty - L.cy;
  const float rx = m.X + L.az * dtx - L.axp;
  const float ry = m.Y + L.az * dty - L.ayp;
  return rx * rx * m.wx + ry * ry * m.wy;
}

// The window of the multi-vertex fit: a vertex's fit visits the tracks with
// chi2 < kMvWin at its seed; the others must keep chi2 >= kMvSafe at every
// iterate (so each weighs under exp(2 - kMvSafe/2) ~ 7e-13 of a track at the
// vertex, below binary32 resolution of the sums), else the vertex is fitted
// over all tracks.
constexpr float kMvWin = 200.0f;
constexpr float kMvSafe = 60.0f;
constexpr int kMvList = 128;           // most tracks a vertex's window holds
constexpr int kMvRefitAhead = 2;       // tracks a lane loads ahead in a refit
constexpr int kMvWindowBlocks = 4;     // CTAs per SM of the window fits
constexpr int kMvRefitBlocks = 2;      // CTAs per SM of the refits

// Multi-vertex fit of one vertex per G-lane group (binary32 sums), over the
// tracks of the event whose packed records start at rec: all n of them (list
// NULL) or the n listed (list[j] = track index); lane r of the group takes
// every G-th.  Same normal equations, shear and solve as group_fit; the stop
// rule is |dz| < mv_dz_tol alone and a track counts for the vertex from
// weight mv_w_assoc on.  With a list, the fit stops with *escaped set when an
// iterate a (relative to the seed) moves far enough that a track left out
// could come within chi2 kMvSafe: a track's residual changes by
// (a_z t_x - a_x, a_z t_y - a_y), so by Minkowski's inequality its sqrt(chi2)
// drops by at most sqrt(w_max) (|a_x| + |a_y| + 2 |a_z| t_max) (w_max its larger
// weight 1/V, t_max its larger |slope|), which stays below its margin
// m = sqrt(chi2 at the seed) - sqrt(kMvSafe) while
// (|a_x| + |a_y|) i_xy + 2 |a_z| i_z <= 1, i_xy and i_z being the largest
// sqrt(w_max)/m and sqrt(w_max) t_max/m over the tracks left out.  Every lane
// of the warp must call it.
// Sum over the G lanes of a group (G = 8 or 32; xor tree, identical on all its
// lanes).  Every lane of the warp must call it.
template <int G, typename T>
__device__ __forceinline__ T lanes_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A lane's records of its next U tracks (s0, s0 + G, ...; those at or past
// cnt are not loaded), loaded before any is used so that their loads overlap.
template <int G, int U>
__device__ __forceinline__ void mv_load(const float4* rec, const int16_t* list, int s0, int cnt,
                                        float4 (&P)[U][3]) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int s = s0 + u * G;
    if (s < cnt) {
      const float4* p = rec + 3 * (list ? static_cast<int>(list[s]) : s);
      P[u][0] = p[0];
      P[u][1] = p[1];
      P[u][2] = p[2];
    }
  }
}

// U: tracks a lane loads ahead (their terms are still added one by one in
// track order, so U does not change a result's bits).
template <int G, int U = 1>
__device__ void group_fit_multi(const float4* rec, int n, const int16_t* list, float xs,
                                float ys, float zs, bool active, const Consts& C, VertexOut* out,
                                MvLast* last, float i_xy = 0.f, float i_z = 0.f,
                                bool* escaped = nullptr) {
  const int r = threadIdx.x & (G - 1);
  const int cnt = active ? n : 0;
  float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
  for (int s0 = r; s0 < cnt; s0 += U * G) {
    float4 P[U][3];
    mv_load<G, U>(rec, list, s0, cnt, P);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      MvTrack m;
      if (s0 + u * G >= cnt || !mv_track_rec(P[u][0], P[u][1], P[u][2], xs, ys, zs, &m)) continue;
      m0 += m.wx; m1 += m.wx * m.tx; m2 += m.wy; m3 += m.wy * m.ty;
    }
  }
  m0 = lanes_sum<G>(m0); m1 = lanes_sum<G>(m1); m2 = lanes_sum<G>(m2); m3 = lanes_sum<G>(m3);
  float cx = m0 > 0.f ? m1 / m0 : 0.f;
  float cy = m2 > 0.f ? m3 / m2 : 0.f;
  float ax = 0.f, ay = 0.f, az = 0.f;
  bool done = !active;
  int status = 0, n_iter = 0, nw = 0;
  float c2sum = 0.f, sw = 0.f, dchi2 = 0.f;
  float ix = 0.f, iy = 0.f, ux = 0.f, uy = 0.f, is = 0.f;
  MvLast L{0.f, 0.f, 0.f, 0.f, 0.f};
  for (int it = 1; it <= C.max_iter; ++it) {
    float v[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) v[q] = 0.f;
    int cnt_w = 0;
    const MvLast P{ax - cx * az, ay - cy * az, az, cx, cy};
    if (!done && list) {
      // the tracks left out stay out of reach of this iterate?
      const float axy = (ax < 0.f ? -ax : ax) + (ay < 0.f ? -ay : ay);
      const float az_ = az < 0.f ? -az : az;
      if (!(axy * i_xy + 2.0f * az_ * i_z <= 1.0f)) {
        *escaped = true;
        done = true;
      }
    }
    if (!done) {
      for (int s0 = r; s0 < cnt; s0 += U * G) {
        float4 R[U][3];
        mv_load<G, U>(rec, list, s0, cnt, R);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          MvTrack m;
          if (s0 + u * G >= cnt || !mv_track_rec(R[u][0], R[u][1], R[u][2], xs, ys, zs, &m))
            continue;
          const float dtx = m.tx - P.cx, dty = m.ty - P.cy;
          const float rx = m.X + P.az * dtx - P.axp;
          const float ry = m.Y + P.az * dty - P.ayp;
          const float c2 = rx * rx * m.wx + ry * ry * m.wy;
          const float w = mv_weight(c2, m.comp, C);
          const float wx = w * m.wx, wy = w * m.wy;
          v[0] += wx; v[1] += wy;
          v[2] += wx * dtx; v[3] += wy * dty;
          v[4] += wx * dtx * dtx + wy * dty * dty;
          v[5] += wx * rx; v[6] += wy * ry;
          v[7] += wx * dtx * rx + wy * dty * ry;
          v[8] += w * c2; v[9] += w;
          if (w >= C.mv_w_assoc) ++cnt_w;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) v[q] = lanes_sum<G>(v[q]);
    cnt_w = lanes_sum<G>(cnt_w);
    if (!done) {
      const float sxx = v[0], syy = v[1], sxz = v[2], syz = v[3], szz = v[4];
      const float bx = v[5], by = v[6], bz = v[7];
      n_iter = it;
      c2sum = v[8]; sw = v[9]; nw = cnt_w;
      L = P;
      float s_ = 0.f;
      bool ok = sxx > 0.f && syy > 0.f && isfinite(sxx) && isfinite(syy);
      if (ok) {
        ix = 1.0f / sxx;
        iy = 1.0f / syy;
        ux = sxz * ix;
        uy = syz * iy;
        s_ = szz - sxz * ux - syz * uy;
        const float mzz = szz + 2.0f * (cx * sxz + cy * syz) + cx * cx * sxx + cy * cy * syy;
        ok = s_ > kPivotRel * mzz && isfinite(s_);
      }
      if (!ok) {
        status = PV_ST_SINGULAR;
        dchi2 = 0.f;
        done = true;
      } else {
        is = 1.0f / s_;
        const float dz = (ux * bx + uy * by - bz) * is;
        const float dx = (bx + sxz * dz) * ix;
        const float dy = (by + syz * dz) * iy;
        dchi2 = -bx * dx - by * dy + bz * dz;
        ax += dx + cx * dz;
        ay += dy + cy * dz;
        az += dz;
        ux += cx;
        uy += cy;
        cx = ux;
        cy = uy;
        if ((dz < 0.f ? -dz : dz) < C.mv_dz_tol) {
          status = PV_ST_CONVERGED;
          done = true;
        } else if (it == C.max_iter) {
          status = PV_ST_MAXITER;
        }
      }
    }
    if (__all_sync(0xffffffffu, done)) break;
  }
  if (!active) return;
  *last = L;
  out->x = ax;
  out->y = ay;
  out->z = az;
  out->cov[0] = ix + ux * ux * is;
  out->cov[1] = ux * uy * is;
  out->cov[2] = iy + uy * uy * is;
  out->cov[3] = ux * is;
  out->cov[4] = uy * is;
  out->cov[5] = is;
  out->chi2 = c2sum + dchi2;
  out->ndof = 2.0f * sw - 3.0f;
  out->n_tracks = nw;
  out->n_iter = n_iter;
  out->status = status == 0 ? PV_ST_MAXITER : status;
}

// The multi-vertex fit runs as six kernels:
//   mv_event_kernel   one warp per event: its seeds, one work item (event,
//                     vertex) per seed, each track's event;
//   mv_sums_kernel    one thread per track: its packed record with its seed
//                     sum S;
//   mv_fit_kernel     persistent, four vertices per warp from the work list,
//                     any event: the fits over the vertices' windows, then
//                     the refits over all tracks (group_fit_multi);
//   mv_assign_kernel  one thread per track: its vertex from the last-
//                     iteration weights;
//   mv_select_kernel  one thread per event: duplicates in seed order,
//                     selection.

__global__ void __launch_bounds__(kMvThreads)
mv_event_kernel(Consts C, TrackPtrs T, SeedPtrs SP, OutPtrs O, MvScratch M) {
  const int lane = threadIdx.x & 31;
  const int e = (blockIdx.x * kMvThreads + threadIdx.x) >> 5;
  if (e >= T.n_events) return;                       // whole warps
  const int64_t b0 = T.off[e], b1 = T.off[e + 1];
  if (offsets_bad(b0, b1, T.n_tracks)) {
    if (lane == 0) {
      O.n_per_event[e] = 0;
      if (O.event_status) O.event_status[e] = PV_EV_BAD_OFFSETS;
      M.K[e] = 0;
    }
    return;
  }
  const int n = static_cast<int>(b1 - b0);
  int capk = SP.cap < O.cap ? SP.cap : O.cap;
  capk = capk < kMaxSeeds ? capk : kMaxSeeds;
  int K = SP.n_per_event[e];
  K = K < 0 ? 0 : (K > capk ? capk : K);
  // seeds of this event in registers: lane k holds seeds k and k + 32
  float sx0 = 0.f, sy0 = 0.f, sz0 = 0.f, sx1 = 0.f, sy1 = 0.f, sz1 = 0.f;
  if (lane < K) {
    const size_t q = static_cast<size_t>(e) * SP.cap + lane;
    sx0 = SP.x[q]; sy0 = SP.y[q]; sz0 = SP.z[q];
  }
  if (lane + 32 < K) {
    const size_t q = static_cast<size_t>(e) * SP.cap + lane + 32;
    sx1 = SP.x[q]; sy1 = SP.y[q]; sz1 = SP.z[q];
  }
  // the seeds are copied to the per-slot scratch (the output rows may be the
  // seed rows and are overwritten by the fits)
  if (lane < K) {
    const size_t q = static_cast<size_t>(e) * kMaxSeeds + lane;
    M.sx[q] = sx0; M.sy[q] = sy0; M.sz[q] = sz0;
  }
  if (lane + 32 < K) {
    const size_t q = static_cast<size_t>(e) * kMaxSeeds + lane + 32;
    M.sx[q] = sx1; M.sy[q] = sy1; M.sz[q] = sz1;
  }
  // each track's event (the sums follow, one thread per track)
  for (int t = lane; t < n; t += 32) M.tev[b0 + t] = e;
  // work items: one per seed
  int wb = 0;
  if (lane == 0) {
    M.K[e] = K;
    O.n_per_event[e] = K;
    wb = K > 0 ? atomicAdd(M.counters, K) : 0;
  }
  wb = __shfl_sync(0xffffffffu, wb, 0);
  for (int k = lane; k < K; k += 32)
    if (PV_CHECK(K <= kMaxSeeds, 13)) M.work[wb + k] = make_int2(e, k);
}

// Each track's packed record with its seed sum S = sum over the event's seeds
// (in seed order) of exp(-chi2/2) at the seed; one thread per track.
__global__ void __launch_bounds__(256)
mv_sums_kernel(Consts C, TrackPtrs T, MvScratch M) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= T.n_tracks) return;
  const int e = M.tev[i];
  if (e < 0 || e >= T.n_events) return;
  const int K = M.K[e];
  const size_t s0 = static_cast<size_t>(e) * kMaxSeeds;
  const float x = T.x[i], y = T.y[i], z = T.z[i], tx = T.tx[i], ty = T.ty[i];
  const float a = T.cxx[i], b = T.cxtx[i], c = T.ctxtx[i];
  const float d = T.cyy[i], f = T.cyty[i], g = T.ctyty[i];
  float sum = 0.f;
  for (int k = 0; k < K; ++k) {
    float4 A;
    float2 W;
    make_fit_track(x, y, z, tx, ty, a, b, c, d, f, g, M.sx[s0 + k], M.sy[s0 + k], M.sz[s0 + k],
                   &A, &W);
    if (W.x > 0.0f) sum += mv_seed_term(A.x, A.y, W.x, W.y);
  }
  float4* q = M.P + 3 * i;
  q[0] = make_float4(x, y, z, tx);
  q[1] = make_float4(ty, a, b, c);
  q[2] = make_float4(d, f, g, sum);
}

// Multi-vertex fits from the work list: every 8-lane group fits one vertex.
// kRedo = false: over the vertex's window (the tracks with chi2 < kMvWin at
// its seed, listed in shared memory in track order); a vertex whose window
// does not hold -- more than kMvList tracks or none, a track left out came
// within reach, the fit was singular, or the listed tracks' weights sum below
// one half (ndof = 2 sum w - 3), where tracks left out would no longer be
// negligible -- goes to the refit list instead of the outputs.  kRedo = true:
// the refit list, each vertex over every track of its event.  The window fits
// wait on their track loads, so four CTAs per SM (64 registers, a few
// spilled) beat two (97 registers): 1.30 ms against 1.56 ms per nominal step.
// The refits are few and long (the vertices of the largest events, over all
// their tracks): their time is the tail of the longest ones with few warps
// left, so they run two CTAs per SM with 128 registers and each lane loading
// its next kMvRefitAhead tracks ahead (bit for bit the same results; 1.022 ->
// 0.979 ms per nominal call, 1.547 -> 1.477 ms on the mixture).
template <bool kRedo>
__global__ void __launch_bounds__(kMvFitThreads, kRedo ? kMvRefitBlocks : kMvWindowBlocks)
mv_fit_kernel(Consts C, TrackPtrs T, OutPtrs O, MvScratch M) {
  __shared__ int16_t s_list[kRedo ? 1 : kMvFitThreads / kGroup][kRedo ? 1 : kMvList];
  const int lane = threadIdx.x & 31;
  const int r = lane & (kGroup - 1);
  const int n_items = kRedo ? M.counters[2] : M.counters[0];
  int* next = M.counters + (kRedo ? 3 : 1);
  for (;;) {
    int b = 0;
    if (lane == 0) b = atomicAdd(next, kGroupsPerWarp);
    b = __shfl_sync(0xffffffffu, b, 0);
    if (b >= n_items) break;
    const int v = b + (lane >> 3);
    const bool has = v < n_items;
    const int2 it = !has ? make_int2(0, 0) : (kRedo ? M.redo[v] : M.work[v]);
    const int e = it.x, k = it.y;
    const int64_t b0 = has ? T.off[e] : 0;
    const int n = has ? static_cast<int>(T.off[e + 1] - b0) : 0;
    const size_t slot = static_cast<size_t>(e) * kMaxSeeds + k;
    const float xs = has ? M.sx[slot] : 0.f, ys = has ? M.sy[slot] : 0.f;
    const float zs = has ? M.sz[slot] : 0.f;
    const float4* rec = M.P + 3 * b0;
    VertexOut out;
    MvLast L;
    bool keep = has;
    if constexpr (kRedo) {
      group_fit_multi<kGroup, kMvRefitAhead>(rec, n, nullptr, xs, ys, zs, has, C, &out, &L);
    } else {
      // the window, and the bound on the tracks left out (i_xy, i_z)
      int16_t* list = s_list[threadIdx.x >> 3];
      const unsigned gmask = 0xffu << (lane & 24);
      int nn = 0;
      float ixy = 0.f, iz = 0.f;
      for (int j0 = 0; j0 < n; j0 += kGroup) {     // (n is the same on the group's lanes)
        const int sidx = j0 + r;
        bool near = false;
        if (sidx < n) {
          MvTrack m;
          if (mv_track(rec + 3 * sidx, xs, ys, zs, &m)) {
            const float c2 = m.X * m.X * m.wx + m.Y * m.Y * m.wy;
            if (c2 < kMvWin) {
              near = true;
            } else {
              const float rm = 1.0f / (sqrtf(c2) - sqrtf(kMvSafe));
              const float sw = sqrtf(fmaxf(m.wx, m.wy));
              ixy = fmaxf(ixy, sw * rm);
              iz = fmaxf(iz, sw * fmaxf(fabsf(m.tx), fabsf(m.ty)) * rm);
            }
          }
        }
        const unsigned bal = (__ballot_sync(gmask, near) >> (lane & 24)) & 0xffu;
        const int idx = nn + __popc(bal & ((1u << r) - 1u));
        if (near && idx < kMvList) list[idx] = static_cast<int16_t>(sidx);
        nn += __popc(bal);
      }
      ixy = group_max(ixy);
      iz = group_max(iz);
      __syncwarp();
      const bool windowed = has && nn >= 1 && nn <= kMvList && n <= 32767;   // (int16 indices)
      bool escaped = false;
      group_fit_multi<kGroup>(rec, windowed ? nn : 0, windowed ? list : nullptr, xs, ys, zs,
                              windowed, C, &out, &L, ixy, iz, &escaped);
      const bool redo = has && (!windowed || escaped || (out.status & PV_ST_SINGULAR) != 0 ||
                                !(out.ndof >= -2.0f));
      if (redo && r == 0) {
        const int q = atomicAdd(M.counters + 2, 1);
        M.redo[q] = it;
      }
      keep = has && !redo;
    }
    if (keep && r == 0) {
      const size_t q = static_cast<size_t>(e) * O.cap + k;
      O.x[q] = xs + out.x;
      O.y[q] = ys + out.y;
      O.z[q] = zs + out.z;
      if (O.cov) {
#pragma unroll
        for (int c = 0; c < 6; ++c) O.cov[q * 6 + c] = out.cov[c];
      }
      if (O.chi2) O.chi2[q] = out.chi2;
      if (O.ndof) O.ndof[q] = out.ndof;
      if (O.n_tracks) O.n_tracks[q] = out.n_tracks;
      if (O.n_iter) O.n_iter[q] = out.n_iter;
      M.last[slot] = L;
      M.vz[slot] = zs + out.z;
      M.vczz[slot] = out.cov[5];
      M.vn[slot] = out.n_tracks;
      M.vst[slot] = out.status;
    }
  }
}

// Each track's vertex: the vertex of its largest last-iteration weight if
// that is at least mv_w_assoc (the lowest index on ties), else none; one thread
// per track (tracks of events with bad offsets carry no event and are left
// alone).
__global__ void __launch_bounds__(256)
mv_assign_kernel(Consts C, TrackPtrs T, OutPtrs O, MvScratch M) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= T.n_tracks) return;
  const int e = M.tev[i];
  if (e < 0 || e >= T.n_events) return;
  const int K = M.K[e];
  const size_t s0 = static_cast<size_t>(e) * kMaxSeeds;
  const float4* p = M.P + 3 * i;
  const float4 ra = p[0], rb = p[1], rc = p[2];
  int best = -1;
  float wbest = -1.0f;
  for (int j = 0; j < K; ++j) {
    if (M.vst[s0 + j] & PV_ST_SINGULAR) continue;
    MvTrack m;
    if (!mv_track_rec(ra, rb, rc, M.sx[s0 + j], M.sy[s0 + j], M.sz[s0 + j], &m)) continue;
    const float w = mv_weight(mv_chi2_at(m, M.last[s0 + j]), m.comp, C);
    if (w > wbest) {
      wbest = w;
      best = j;
    }
  }
  O.track_vertex[i] = (best >= 0 && wbest >= C.mv_w_assoc) ? best : -1;
}

// Duplicates in seed order, then the final selection; one thread per event.
__global__ void __launch_bounds__(256)
mv_select_kernel(Consts C, TrackPtrs T, OutPtrs O, MvScratch M) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= T.n_events) return;
  const int K = M.K[e];
  const size_t s0 = static_cast<size_t>(e) * kMaxSeeds;
  int kept = -1;
  for (int j = 0; j < K; ++j) {
    int st = M.vst[s0 + j];
    if (st & PV_ST_SINGULAR) continue;
    if (kept >= 0) {
      const float dz = M.vz[s0 + j] - M.vz[s0 + kept];
      if (dz * dz < C.mv_dup_sep2 * (M.vczz[s0 + j] + M.vczz[s0 + kept])) {
        if (M.vn[s0 + j] > M.vn[s0 + kept]) {
          M.vst[s0 + kept] |= PV_ST_DUPLICATE;
          kept = j;
        } else {
          M.vst[s0 + j] |= PV_ST_DUPLICATE;
        }
        continue;
      }
    }
    kept = j;
  }
  for (int j = 0; j < K; ++j) {
    const size_t q = static_cast<size_t>(e) * O.cap + j;
    int st = M.vst[s0 + j];
    if (!(st & (PV_ST_SINGULAR | PV_ST_DUPLICATE)))
      st = select_vertex(O.x[q], O.y[q], M.vz[s0 + j], M.vn[s0 + j], st, C);
    if (O.status) O.status[q] = st;
  }
}

cudaError_t launch_mv_fit(const Consts& C, const TrackPtrs& T, const SeedPtrs& S,
                          const OutPtrs& O, const MvScratch& M, int fit_grid, int redo_grid,
                          cudaStream_t st, int* n_launches) {
  cudaError_t err = cudaMemsetAsync(M.counters, 0, 4 * sizeof(int), st);
  if (err != cudaSuccess) return err;
  const int per_block = kMvThreads / 32;
  const int grid = (T.n_events + per_block - 1) / per_block;
  // (tracks of events the event kernel skips keep event -1)
  err = cudaMemsetAsync(M.tev, 0xff, sizeof(int) * static_cast<size_t>(T.n_tracks), st);
  if (err != cudaSuccess) return err;
  mv_event_kernel<<<grid, kMvThreads, 0, st>>>(C, T, S, O, M);
  if (T.n_tracks > 0)
    mv_sums_kernel<<<static_cast<unsigned>((T.n_tracks + 255) / 256), 256, 0, st>>>(C, T, M);
  mv_fit_kernel<false><<<fit_grid, kMvFitThreads, 0, st>>>(C, T, O, M);
  mv_fit_kernel<true><<<redo_grid, kMvFitThreads, 0, st>>>(C, T, O, M);
  if (T.n_tracks > 0)
    mv_assign_kernel<<<static_cast<unsigned>((T.n_tracks + 255) / 256), 256, 0, st>>>(C, T, O, M);
  mv_select_kernel<<<(T.n_events + 255) / 256, 256, 0, st>>>(C, T, O, M);
  *n_launches += 6;
  return cudaGetLastError();
}

int mv_blocks_per_sm(bool redo) {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &blocks, redo ? mv_fit_kernel<true> : mv_fit_kernel<false>, kMvFitThreads, 0) !=
      cudaSuccess)
    return 0;
  return blocks;
}

// ---------------------------------------------------------------------------
// launch plumbing: kernel instantiations by block size

template <int MODE, int NT, int FLAV>
static cudaError_t setup_find_flav(int nbins) {
  cudaError_t err = cudaFuncSetAttribute(find_kernel<MODE, NT, FLAV>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fused_smem_bytes(nbins, MODE, NT, flavour_split(FLAV) == PV_SPLIT_RECURSIVE));
  if (err != cudaSuccess) return err;
  return cudaFuncSetAttribute(find_kernel<MODE, NT, FLAV>,
                              cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
}

// The GPU flavour (FLAV 0) at every block size; the x86 flavours of the peak
// search and the profile (FLAV 1-3) at kFlavThreads for the modes that find.
template <int MODE, int NT>
static cudaError_t setup_find(int nbins) {
  cudaError_t err = setup_find_flav<MODE, NT, 0>(nbins);
  if constexpr (MODE != kFit && NT == kFlavThreads) {
    if (err == cudaSuccess) err = setup_find_flav<MODE, NT, 1>(nbins);
    if (err == cudaSuccess) err = setup_find_flav<MODE, NT, 2>(nbins);
    if (err == cudaSuccess) err = setup_find_flav<MODE, NT, 3>(nbins);
  }
  return err;
}

template <int NT>
static cudaError_t setup_find_all(int nbins) {
  cudaError_t err;
  if ((err = setup_find<kFind, NT>(nbins)) != cudaSuccess) return err;
  if ((err = setup_find<kFit, NT>(nbins)) != cudaSuccess) return err;
  return setup_find<kFindFit, NT>(nbins);
}

cudaError_t fused_setup(int nbins) {
  cudaError_t err;
  if ((err = setup_find_all<64>(nbins)) != cudaSuccess) return err;
  if ((err = setup_find_all<96>(nbins)) != cudaSuccess) return err;
  if ((err = setup_find_all<128>(nbins)) != cudaSuccess) return err;
  if ((err = setup_find_all<256>(nbins)) != cudaSuccess) return err;
  // the staged find (GPU flavour, 96- and 128-thread blocks)
  if ((err = setup_find_flav<kFindFitStaged, 96, 0>(nbins)) != cudaSuccess) return err;
  return setup_find_flav<kFindFitStaged, 128, 0>(nbins);
}

bool find_block_ok(int nt) { return nt == 64 || nt == 96 || nt == 128 || nt == 256; }
bool fit_block_ok(int ft) { return ft == 128 || ft == 256; }

template <int MODE, int NT, int FLAV = 0>
static int find_blocks(int nbins) {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, find_kernel<MODE, NT, FLAV>, NT,
                                                    fused_smem_bytes(nbins, MODE, NT, flavour_split(FLAV) == PV_SPLIT_RECURSIVE)) != cudaSuccess)
    return 0;
  return blocks;
}

template <int NT>
static int find_blocks_nt(int nbins, int mode) {
  if (mode == kFind) return find_blocks<kFind, NT>(nbins);
  if (mode == kFit) return find_blocks<kFit, NT>(nbins);
  return find_blocks<kFindFit, NT>(nbins);
}

template <int MODE>
static int find_blocks_flav(int nbins, int flav) {
  if (flav == 1) return find_blocks<MODE, kFlavThreads, 1>(nbins);
  if (flav == 2) return find_blocks<MODE, kFlavThreads, 2>(nbins);
  return find_blocks<MODE, kFlavThreads, 3>(nbins);
}

int fused_blocks_per_sm(int nbins, int mode, int nt, int flav) {
  if (mode == kFindFitStaged)
    return nt == 96 ? find_blocks<kFindFitStaged, 96>(nbins) : find_blocks<kFindFitStaged, 128>(nbins);
  if (flav != 0 && mode != kFit)
    return mode == kFind ? find_blocks_flav<kFind>(nbins, flav)
                         : find_blocks_flav<kFindFit>(nbins, flav);
  if (nt == 64) return find_blocks_nt<64>(nbins, mode);
  if (nt == 96) return find_blocks_nt<96>(nbins, mode);
  if (nt == 256) return find_blocks_nt<256>(nbins, mode);
  return find_blocks_nt<128>(nbins, mode);
}

template <int K, int FT>
static int fit_blocks(void) {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fit_kernel<K, FT>, FT, 0) !=
      cudaSuccess)
    return 0;
  return blocks;
}

template <int FT>
static int fit_blocks_ft(int accum) {
  if (accum == PV_ACCUM_KAHAN) return fit_blocks<PV_ACCUM_KAHAN, FT>();
  if (accum == PV_ACCUM_FP64) return fit_blocks<PV_ACCUM_FP64, FT>();
  return fit_blocks<PV_ACCUM_FP32, FT>();
}

int fit_blocks_per_sm(int accum, int ft) {
  return ft == 128 ? fit_blocks_ft<128>(accum) : fit_blocks_ft<256>(accum);
}

template <int FT>
static void launch_fit_ft(int accum, int grid, cudaStream_t st, const Consts& C, const TrackPtrs& T,
                          const TrackScratch& ws, const OutPtrs& O) {
  if (accum == PV_ACCUM_KAHAN)
    fit_kernel<PV_ACCUM_KAHAN, FT><<<grid, FT, 0, st>>>(C, T, ws, O);
  else if (accum == PV_ACCUM_FP64)
    fit_kernel<PV_ACCUM_FP64, FT><<<grid, FT, 0, st>>>(C, T, ws, O);
  else
    fit_kernel<PV_ACCUM_FP32, FT><<<grid, FT, 0, st>>>(C, T, ws, O);
}

template <int MODE, int NT>
static void launch_find_nt(int grid, size_t sm, cudaStream_t st, const Consts& C,
                           const TrackPtrs& T, const SeedPtrs& S, const OutPtrs& O,
                           const TrackScratch& ws) {
  find_kernel<MODE, NT><<<grid, NT, sm, st>>>(C, T, S, O, ws);
}

template <int MODE>
static void launch_find(int nt, int grid, size_t sm, cudaStream_t st, const Consts& C,
                        const TrackPtrs& T, const SeedPtrs& S, const OutPtrs& O,
                        const TrackScratch& ws) {
  if constexpr (MODE != kFit) {
    const int flav = flavour_of(C);
    if (flav != 0) {
      constexpr int NF = kFlavThreads;
      if (flav == 1) find_kernel<MODE, NF, 1><<<grid, NF, sm, st>>>(C, T, S, O, ws);
      else if (flav == 2) find_kernel<MODE, NF, 2><<<grid, NF, sm, st>>>(C, T, S, O, ws);
      else find_kernel<MODE, NF, 3><<<grid, NF, sm, st>>>(C, T, S, O, ws);
      return;
    }
  }
  if (nt == 64) launch_find_nt<MODE, 64>(grid, sm, st, C, T, S, O, ws);
  else if (nt == 96) launch_find_nt<MODE, 96>(grid, sm, st, C, T, S, O, ws);
  else if (nt == 256) launch_find_nt<MODE, 256>(grid, sm, st, C, T, S, O, ws);
  else launch_find_nt<MODE, 128>(grid, sm, st, C, T, S, O, ws);
}

cudaError_t launch_fused(int mode, const Consts& C, const TrackPtrs& T, const SeedPtrs& S,
                         const OutPtrs& O, const TrackScratch& ws, const LaunchCfg& L,
                         cudaStream_t st, int* n_launches) {
  // the x86 flavours of the find are built at kFlavThreads only
  const int nt = (mode != kFit && flavour_of(C) != 0) ? kFlavThreads : L.find_nt;
  size_t sm = fused_smem_bytes(C.nbins, mode & ~kStage, nt,
                               mode != kFit && C.split_mode == PV_SPLIT_RECURSIVE);
  cudaError_t err = cudaMemsetAsync(ws.counters, 0, kCounterInts * sizeof(int), st);
  if (err != cudaSuccess) return err;
  if (mode == kFindFitStaged) {
    // GPU flavour only
    if (L.find_nt == 96)
      find_kernel<kFindFitStaged, 96><<<L.find_grid, 96, sm, st>>>(C, T, S, O, ws);
    else
      find_kernel<kFindFitStaged, 128><<<L.find_grid, 128, sm, st>>>(C, T, S, O, ws);
  } else if (mode == kFind) {
    launch_find<kFind>(L.find_nt, L.find_grid, sm, st, C, T, S, O, ws);
  } else if (mode == kFit) {
    launch_find<kFit>(L.find_nt, L.find_grid, sm, st, C, T, S, O, ws);
  } else {
    launch_find<kFindFit>(L.find_nt, L.find_grid, sm, st, C, T, S, O, ws);
  }
  ++*n_launches;
  if (mode & kFit) {
    if (L.fit_nt == 128) launch_fit_ft<128>(C.accum_mode, L.fit_grid, st, C, T, ws, O);
    else launch_fit_ft<256>(C.accum_mode, L.fit_grid, st, C, T, ws, O);
    ++*n_launches;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// template table of the x86 profile (Sec. 3.2): sigma_k, the class bounds,
// the smallest H_k whose outer edge quantises to 0, and the quantised
// Gaussian CDF at the edges (i - H - 1/2) dz, all in binary64 with
// round-to-nearest intrinsics, quantised with ties to even.

__device__ __forceinline__ long long tpl_quant(int i, int H, double dz, double s) {
  const double x = __ddiv_rn(__dmul_rn(__dsub_rn(static_cast<double>(i - H), 0.5), dz), s);
  const double phi = __dmul_rn(0.5, erfc(__dmul_rn(-x, 0.70710678118654752440)));
  return __double2ll_rn(__dmul_rn(static_cast<double>(kOne), phi));
}

// One thread per class finds sigma_k, its bound and H_k (sigma_k and the bound
// by the same chain of products as a sequential loop); thread 0 lays the
// classes out; all threads fill the quantised CDF values; thread k takes the
// running maximum over class k.
__global__ void __launch_bounds__(256) template_table_kernel(TplTable* t, double dz) {
  __shared__ double sig[kTplClasses];
  __shared__ int first[kTplClasses + 1];
  __shared__ int ok;
  const int k = threadIdx.x;
  if (k < kTplClasses) {
    double s = kTplSigma0, bound = 0.0;
    for (int j = 1; j <= k; ++j) {
      bound = __dmul_rn(s, kTplHalfRatio);
      s = __dmul_rn(s, kTplRatio);
    }
    t->bound[k] = bound;
    sig[k] = s;
    int H = 0;
    while (H < kTplMaxHalf && tpl_quant(0, H, dz, s) != 0) ++H;
    t->half[k] = H;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int total = 0;
    for (int c = 0; c < kTplClasses; ++c) {
      first[c] = total;
      t->first[c] = total;
      total += 2 * t->half[c] + 2;
    }
    first[kTplClasses] = total;
    ok = total <= kTplCap;
    t->status = ok ? 0 : 1;
  }
  __syncthreads();
  if (!ok) return;
  for (int idx = threadIdx.x; idx < first[kTplClasses]; idx += blockDim.x) {
    int c = 0;
    while (first[c + 1] <= idx) ++c;
    const int H = t->half[c];
    const int i = idx - first[c];
    long long v;
    if (i == 0) v = 0;
    else if (i == 2 * H + 1) v = kOne;
    else v = tpl_quant(i, H, dz, sig[c]);
    t->q[idx] = static_cast<int32_t>(v < 0 ? 0 : (v > kOne ? kOne : v));
  }
  __syncthreads();
  // the quantised CDF is non-decreasing in i (monotone Phi, monotone
  // roundings); the running maximum of the definition is taken anyway
  if (k < kTplClasses) {
    int32_t* q = t->q + first[k];
    for (int i = 1; i <= 2 * t->half[k] + 1; ++i)
      if (q[i] < q[i - 1]) q[i] = q[i - 1];
  }
}

cudaError_t build_template_table(TplTable* t, float dz, cudaStream_t st) {
  template_table_kernel<<<1, 256, 0, st>>>(t, static_cast<double>(dz));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// plain per-step kernels

template <int PROFILE>
__global__ void plain_extrapolate_kernel(Consts C, TrackPtrs T, float* zpoca, float* sigma,
                                         int32_t* center, int32_t* j0, int32_t* j1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T.n_tracks;
       i += (int64_t)gridDim.x * blockDim.x) {
    Prep p = prepare_track<PROFILE>(T.x[i], T.y[i], T.z[i], T.tx[i], T.ty[i], T.cxx[i],
                                    T.cxtx[i], T.ctxtx[i], C);
    if (zpoca) zpoca[i] = p.zpoca;
    if (sigma) sigma[i] = p.sigma;
    if (center) center[i] = p.filled ? p.center : -1;
    if (j0) j0[i] = p.j0;
    if (j1) j1[i] = p.j1;
  }
}

__global__ void plain_hist_kernel(Consts C, TrackPtrs T, const float* zpoca, const float* sigma,
                                  const int32_t* center, const int32_t* j0, const int32_t* j1,
                                  uint32_t* hist) {
  const int e = blockIdx.x;
  const int64_t b0 = T.off[e], b1 = T.off[e + 1];
  if (offsets_bad(b0, b1, T.n_tracks)) return;
  uint32_t* h = hist + static_cast<size_t>(e) * C.nbins;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    if (center[i] < 0) continue;
    if (C.profile_mode == PV_PROFILE_TEMPLATE)
      fill_template(h, __ldg(C.tpl->first + tpl_class(sigma[i], C.tpl)), j0[i], j1[i], C);
    else
      fill_profile(h, zpoca[i], sigma[i], j0[i], j1[i], C);
  }
}

template <int SPLIT>
__global__ void __launch_bounds__(32)
plain_peaks_kernel(Consts C, TrackPtrs T, const uint32_t* hist, int cap, int32_t* seed_n,
                   int32_t* seed_lo, int32_t* seed_hi, int32_t* seed_bin, float* seed_z,
                   int32_t* ev_status) {
  __shared__ SeedOut S;
  __shared__ int16_t pc_lo[kRunRing], pc_hi[kRunRing];
  __shared__ int16_t mark[SPLIT == PV_SPLIT_RECURSIVE ? kMaxBins : 1];
  const int e = blockIdx.x;
  const int64_t b0 = T.off[e], b1 = T.off[e + 1];
  const int lane = threadIdx.x;
  if (offsets_bad(b0, b1, T.n_tracks)) {
    if (lane == 0) { seed_n[e] = 0; ev_status[e] = PV_EV_BAD_OFFSETS; }
    return;
  }
  int K = warp_find_seeds<true, SPLIT>(hist + static_cast<size_t>(e) * C.nbins, nullptr, C, &S,
                                       cap, pc_lo, pc_hi, mark,
                                       SPLIT == PV_SPLIT_RECURSIVE ? kMaxBins : 0);
  int Ks = K < cap ? K : cap;
  for (int k = lane; k < Ks; k += 32) {
    size_t q = static_cast<size_t>(e) * kMaxSeeds + k;
    seed_lo[q] = S.lo[k];
    seed_hi[q] = S.hi[k];
    seed_bin[q] = S.bin[k];
    seed_z[q] = S.z[k];
  }
  if (lane == 0) { seed_n[e] = Ks; ev_status[e] = K > cap ? PV_EV_SEED_OVERFLOW : 0; }
}

__global__ void __launch_bounds__(256)
plain_assoc_kernel(Consts C, TrackPtrs T, OutPtrs O, const int32_t* center, int32_t* cid,
                   const int32_t* seed_n, const int32_t* seed_lo, const int32_t* seed_hi,
                   const int32_t* seed_bin, const float* seed_z, const int32_t* ev_status) {
  __shared__ SeedOut S;
  __shared__ int alive[kMaxSeeds], part[kMaxSeeds], cnt[kMaxSeeds], flag;
  const int e = blockIdx.x;
  const int64_t b0 = T.off[e], b1 = T.off[e + 1];
  const int tid = threadIdx.x;
  if (offsets_bad(b0, b1, T.n_tracks)) {
    if (tid == 0) {
      O.n_per_event[e] = 0;
      if (O.event_status) O.event_status[e] = PV_EV_BAD_OFFSETS;
    }
    return;
  }
  const int n = static_cast<int>(b1 - b0);
  const int K = seed_n[e];
  if (tid < K) {
    size_t q = static_cast<size_t>(e) * kMaxSeeds + tid;
    S.lo[tid] = seed_lo[q];
    S.hi[tid] = seed_hi[q];
    S.bin[tid] = seed_bin[q];
    float zs = seed_z[q];
    S.z[tid] = zs;
    S.x[tid] = __fadd_rn(C.x_b, __fmul_rn(C.tx_b, zs));
    S.y[tid] = __fadd_rn(C.y_b, __fmul_rn(C.ty_b, zs));
  }
  __syncthreads();
  int Ka = block_associate(center + b0, cid + b0, n, &S, K, C, alive, part, cnt, &flag);
  for (int t = tid; t < n; t += blockDim.x) O.track_vertex[b0 + t] = cid[b0 + t];
  if (tid == 0) {
    O.n_per_event[e] = Ka;
    if (O.event_status) O.event_status[e] = ev_status[e];
  }
  if (tid < Ka) {
    size_t q = static_cast<size_t>(e) * O.cap + tid;
    O.x[q] = S.x[tid];
    O.y[q] = S.y[tid];
    O.z[q] = S.z[tid];
    if (O.bin_lo) O.bin_lo[q] = S.lo[tid];
    if (O.bin_hi) O.bin_hi[q] = S.hi[tid];
    if (O.bin_max) O.bin_max[q] = S.bin[tid];
  }
}

template <int kAccum>
__global__ void __launch_bounds__(256)
plain_fit_kernel(Consts C, TrackPtrs T, SeedPtrs SP, OutPtrs O, int32_t* cid, int32_t* slot,
                 float4* A, float2* W) {
  __shared__ SeedOut S;
  __shared__ int cnt[kMaxSeeds], voff[kMaxSeeds], base[kMaxSeeds];
  const int e = blockIdx.x;
  const int64_t b0 = T.off[e], b1 = T.off[e + 1];
  const int tid = threadIdx.x;
  if (offsets_bad(b0, b1, T.n_tracks)) return;
  const int n = static_cast<int>(b1 - b0);
  int K = SP.n_per_event[e];
  int capk = SP.cap < O.cap ? SP.cap : O.cap;
  capk = capk < kMaxSeeds ? capk : kMaxSeeds;
  K = K < 0 ? 0 : (K > capk ? capk : K);
  if (tid < K) {
    size_t q = static_cast<size_t>(e) * SP.cap + tid;
    S.x[tid] = SP.x[q];
    S.y[tid] = SP.y[q];
    S.z[tid] = SP.z[q];
    cnt[tid] = 0;
  }
  __syncthreads();
  int32_t* c_e = cid + b0;
  for (int t = tid; t < n; t += blockDim.x) {
    int c = SP.track_vertex[b0 + t];
    c = (c >= 0 && c < K) ? c : -1;
    c_e[t] = c;
    if (c >= 0) atomicAdd(cnt + c, 1);
    if (O.track_vertex != SP.track_vertex) O.track_vertex[b0 + t] = c;
  }
  if (tid == 0 && O.n_per_event != SP.n_per_event) O.n_per_event[e] = K;
  __syncthreads();
  if (tid < 32) warp_offsets(cnt, K, voff, base);
  __syncthreads();
  if (tid < 32) warp_slots(c_e, n, base, slot + b0);
  __syncthreads();
  block_fit_inputs(T, b0, n, c_e, slot + b0, &S, A + b0, W + b0);
  __syncthreads();
  block_fit_event<kAccum>(C, &S, K, voff, cnt, A + b0, W + b0, O, e);
}

static int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 65535 * 16) g = 65535 * 16;
  return static_cast<int>(g);
}

cudaError_t launch_extrapolate(const Consts& C, const TrackPtrs& T, float* zpoca, float* sigma,
                               int32_t* center, cudaStream_t st) {
  if (T.n_tracks == 0) return cudaSuccess;
  // z_poca, sigma_poca and the centre bin do not depend on the profile
  plain_extrapolate_kernel<PV_PROFILE_CUBIC><<<grid_for(T.n_tracks, 256), 256, 0, st>>>(
      C, T, zpoca, sigma, center, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_histogram(const Consts& C, const TrackPtrs& T, uint32_t* hist,
                             const PlainScratch& ws, cudaStream_t st, int* n_launches) {
  cudaError_t err = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)T.n_events * C.nbins, st);
  if (err != cudaSuccess) return err;
  if (T.n_tracks > 0) {
    if (C.profile_mode == PV_PROFILE_TEMPLATE)
      plain_extrapolate_kernel<PV_PROFILE_TEMPLATE><<<grid_for(T.n_tracks, 256), 256, 0, st>>>(
          C, T, ws.zpoca, ws.sigma, ws.center, ws.j0, ws.j1);
    else
      plain_extrapolate_kernel<PV_PROFILE_CUBIC><<<grid_for(T.n_tracks, 256), 256, 0, st>>>(
          C, T, ws.zpoca, ws.sigma, ws.center, ws.j0, ws.j1);
    ++*n_launches;
  }
  plain_hist_kernel<<<T.n_events, 256, 0, st>>>(C, T, ws.zpoca, ws.sigma, ws.center, ws.j0, ws.j1,
                                                 hist);
  ++*n_launches;
  return cudaGetLastError();
}

cudaError_t launch_plain_find(const Consts& C, const TrackPtrs& T, const OutPtrs& O,
                              const PlainScratch& ws, cudaStream_t st, int* n_launches) {
  cudaError_t err = launch_histogram(C, T, ws.hist, ws, st, n_launches);
  if (err != cudaSuccess) return err;
  if (C.split_mode == PV_SPLIT_RECURSIVE)
    plain_peaks_kernel<PV_SPLIT_RECURSIVE><<<T.n_events, 32, 0, st>>>(
        C, T, ws.hist, O.cap, ws.seed_n, ws.seed_lo, ws.seed_hi, ws.seed_bin, ws.seed_z,
        ws.ev_status);
  else
    plain_peaks_kernel<PV_SPLIT_ZORDER><<<T.n_events, 32, 0, st>>>(
        C, T, ws.hist, O.cap, ws.seed_n, ws.seed_lo, ws.seed_hi, ws.seed_bin, ws.seed_z,
        ws.ev_status);
  plain_assoc_kernel<<<T.n_events, 256, 0, st>>>(C, T, O, ws.center, ws.cid, ws.seed_n, ws.seed_lo,
                                                 ws.seed_hi, ws.seed_bin, ws.seed_z, ws.ev_status);
  *n_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_plain_fit(const Consts& C, const TrackPtrs& T, const SeedPtrs& S,
                             const OutPtrs& O, const PlainScratch& ws, cudaStream_t st,
                             int* n_launches) {
  if (C.accum_mode == PV_ACCUM_KAHAN)
    plain_fit_kernel<PV_ACCUM_KAHAN><<<T.n_events, 256, 0, st>>>(C, T, S, O, ws.cid, ws.slot, ws.A,
                                                                  ws.W);
  else if (C.accum_mode == PV_ACCUM_FP64)
    plain_fit_kernel<PV_ACCUM_FP64><<<T.n_events, 256, 0, st>>>(C, T, S, O, ws.cid, ws.slot, ws.A,
                                                                 ws.W);
  else
    plain_fit_kernel<PV_ACCUM_FP32><<<T.n_events, 256, 0, st>>>(C, T, S, O, ws.cid, ws.slot, ws.A,
                                                                 ws.W);
  ++*n_launches;
  return cudaGetLastError();
}

}  // namespace pvk
