// pv_serve.cu -- the persistent serving kernel: continuous batching of
// requests on the device.
//
// Each CTA loops: it claims the next event of the published request
// sequence (ServeCtl / ServeDev in pv_kernels.cuh) and runs steps (a)-(d1) on
// it -- the batched find kernel's event work -- queueing the event's vertices;
// the CTA fits its queue (d2, d3) in rounds of 16 vertices, from whichever
// requests they came, whenever a round's worth has gathered or it would
// otherwise wait, and the round that finishes a request's last events stamps
// the request's completion with the GPU's global timer.  Requests that arrive
// while others run are picked up as CTAs free up, so their events overlap on
// the device; a request's results do not depend on what ran beside it.  Every
// wait is bounded: a CTA that finds nothing to claim for idle_ns leaves the
// loop, and the kernel ends when all have.
#include "pv_find.cuh"

namespace pvk {

bool serve_check_report(unsigned* count, unsigned* first) {
#if PV_CHECKED
  unsigned zero = 0;
  cudaDeviceSynchronize();
  cudaMemcpyFromSymbol(count, g_check_count, sizeof(unsigned));
  cudaMemcpyFromSymbol(first, g_check_first, sizeof(unsigned));
  cudaMemcpyToSymbol(g_check_count, &zero, sizeof(unsigned));
  cudaMemcpyToSymbol(g_check_first, &zero, sizeof(unsigned));
  return true;
#else
  *count = 0;
  *first = 0;
  return false;
#endif
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// loads and stores ordered at system scope (the host writes and reads these)
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int ld_acquire_sys(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void serve_clock_kernel(ServeCtl* ctl) {
  *reinterpret_cast<volatile unsigned long long*>(&ctl->clock_ns) = global_ns();
}

// Warp-cooperative copy of descriptor d into s (8 bytes per lane and load, all
// in flight together); returns, on every lane, whether its sequence number
// read `seq` before and after the copy (the host writes ~0 there first, then
// the fields, then the number).  All 32 lanes of the warp call it.
__device__ __forceinline__ bool read_desc(const ServeDesc* d, ServeDesc* s,
                                          unsigned long long seq) {
  const int lane = threadIdx.x & 31;
  unsigned long long s1 = 0;
  if (lane == 0) s1 = ld_acquire_sys(&d->seq);
  s1 = __shfl_sync(0xffffffffu, s1, 0);
  if (s1 != seq) return false;
  const volatile unsigned long long* src = reinterpret_cast<const volatile unsigned long long*>(d);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(s);
  static_assert(sizeof(ServeDesc) % 8 == 0, "descriptor copied in 8-byte words");
  constexpr int kWords = static_cast<int>(sizeof(ServeDesc) / 8);
  for (int i = lane; i < kWords; i += 32) dst[i] = src[i];
  __syncwarp();
  unsigned long long s2 = 0;
  if (lane == 0) {
    __threadfence_system();
    s2 = ld_acquire_sys(&d->seq);
  }
  return __shfl_sync(0xffffffffu, s2, 0) == seq;
}

// One fitting round of the CTA's queue (all threads): the queued vertices by
// track count, largest first, four to a warp (so that a warp's groups need
// similar numbers of passes), each fitted by an 8-lane group with binary32
// sums per kAccum; then each request with events in the round counts them
// done, and the round that completes a request stamps its completion with the
// global timer.  The queue is empty afterwards.
template <int kAccum>
__device__ __forceinline__ void serve_round(const Consts& C, ServeQueue& Q, ServeCtl* ctl,
                                            ServeDev* dev) {
  constexpr int NW = kServeThreads / 32;
  static_assert(NW * kGroupsPerWarp == kServeFitBatch, "a round fills every group");
  static_assert(kServeQueue <= kServeThreads, "one thread per queued vertex ranks them");
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int n = Q.n < kServeQueue ? Q.n : kServeQueue;
  if (tid < n) {
    const int ck = Q.v[tid].cnt;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const int cj = Q.v[j].cnt;
      rank += (cj > ck || (cj == ck && j < tid)) ? 1 : 0;
    }
    Q.order[rank] = static_cast<int16_t>(tid);
  }
  __syncthreads();
  const int r = lane & (kGroup - 1);
  for (int vb = 0; vb < n; vb += kServeFitBatch) {
    const int sl = vb + warp * kGroupsPerWarp + (lane >> 3);
    const bool has = sl < n;
    const ServeVertex v = Q.v[has ? Q.order[sl] : Q.order[vb]];
    const int q = (v.req >= 0 && v.req < kServeReqs) ? v.req : 0;
    (void)PV_CHECK(v.req == q, 21);
    const ServeReq& R = Q.req[q];
    VertexOut out;
    group_fit<kAccum>(R.A + v.off + r, R.W + v.off + r, kGroup, has ? v.cnt : -1, C, &out);
    if (has && r == 0) write_vertex(C, R.O, v.e, v.k, v.x, v.y, v.z, out);
  }
  // the round's outputs are visible device-wide before its events count as done
  __threadfence();
  __syncthreads();
  if (tid < Q.nreq && tid < kServeReqs) {
    const ServeReq& R = Q.req[tid];
    if (R.events > 0) {
      const unsigned long long ev = static_cast<unsigned long long>(R.events);
      const unsigned long long before = atomicAdd(&dev->slot_done[R.slot], ev);
      if (before + ev == R.target) {
        // the request's last events: its outputs are complete
        __threadfence_system();
        *reinterpret_cast<volatile unsigned long long*>(&ctl->done_ns[R.slot]) = global_ns();
        st_release_sys(&ctl->done_seq[R.slot], R.seq);
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    Q.n = 0;
    Q.nreq = 0;
  }
  __syncthreads();
}

// 64 registers per thread, eight CTAs per SM, which is also what shared memory
// allows (the find's histogram and tables plus the queue: about 25 KB per
// CTA).  Measured on the nominal batch as one request, with the vertices then
// fitted per event: 14.5 M events/s at four CTAs per SM, 17.9 M at six, 19.0 M
// at eight.
template <int FLAV, int kAccum>
__global__ void __launch_bounds__(kServeThreads, 8)
serve_kernel(Consts C, ServeCtl* ctl, ServeDev* dev, unsigned long long idle_ns,
             unsigned long long seq_start, unsigned int epoch) {
  constexpr int NT = kServeThreads;
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout Lo = make_layout(C.nbins, kFindFit, NT, flavour_split(FLAV) == PV_SPLIT_RECURSIVE);
  find_prologue<kFindFit, NT>(C, smem, Lo);
  __shared__ ServeDesc s_d;
  __shared__ TrackScratch s_G;       // the request's scratch, from s_d
  __shared__ ServeQueue Q;
  __shared__ unsigned long long s_g;
  __shared__ int s_code, s_round;
  // warp 0's state: the request the last event fell in, the published count
  // seen last; lane 0's: the event claimed ahead
  unsigned long long cursor = seq_start, pub = 0, ahead = 0;
  bool orphans_left = true;           // lane 0: the previous launch's list not exhausted
  bool have = false, have_ahead = false;
  const int prev = (epoch + 1) & 1, cur = epoch & 1;
  if (threadIdx.x == 0) {
    Q.n = 0;
    Q.nreq = 0;
  }
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) {
      // the next event: first the events the previous launch handed on, then
      // the one claimed ahead, else a new claim
      bool got = false;
      unsigned long long g = 0;
      if (orphans_left) {
        const int i = atomicAdd(&dev->orph_take, 1);
        if (i < dev->orph_n[prev] && i < kServeOrphans) {
          g = dev->orph[prev][i];
          got = true;
        } else {
          orphans_left = false;
        }
      }
      if (!got) {
        if (have_ahead) {
          g = ahead;
          have_ahead = false;
        } else {
          g = atomicAdd(&dev->next_event, 1ull);
        }
      }
      if (g >= pub) pub = ld_acquire_sys(&ctl->published);
      // with plenty of published events left, claim the one after now (its
      // atomic completes while this event runs)
      if (!orphans_left && g + gridDim.x < pub) {
        ahead = atomicAdd(&dev->next_event, 1ull);
        have_ahead = true;
      }
      // fit the queue first when it holds kServeRoundAt vertices, when
      // the event is not published yet (the CTA may wait), or when the event
      // may need a request entry and none is free
      const bool same = have && g >= s_d.ev_base &&
                        g < s_d.ev_base + static_cast<unsigned long long>(s_d.T.n_events);
      s_round = Q.nreq > 0 && (Q.n >= kServeRoundAt || g >= pub || (!same && Q.nreq >= kServeReqs));
      s_g = g;
    }
    __syncthreads();
    if (s_round) serve_round<kAccum>(C, Q, ctl, dev);
    if (threadIdx.x < 32) {
      // the event is processed once published (bounded wait; an event still
      // unpublished when the wait ends, or when the host asks to stop, is
      // handed on to the next launch with the one claimed ahead)
      const unsigned long long g = s_g;
      int code = -1;
      if (threadIdx.x == 0) {
        const unsigned long long t0 = global_ns();
        unsigned int nap = 32;
        while (g >= pub) {
          pub = ld_acquire_sys(&ctl->published);
          if (g < pub) break;
          const bool stop = ld_acquire_sys(&ctl->stop) != 0u;
          if (stop || global_ns() - t0 > idle_ns) {
            int i = atomicAdd(&dev->orph_n[cur], 1);
            if (i < kServeOrphans) dev->orph[cur][i] = g;
            if (have_ahead) {
              i = atomicAdd(&dev->orph_n[cur], 1);
              if (i < kServeOrphans) dev->orph[cur][i] = ahead;
              have_ahead = false;
            }
            code = stop ? PV_OK : PV_ERR_TIMEOUT;
            break;
          }
          __nanosleep(nap);
          if (nap < 1024) nap <<= 1;
        }
        if (code >= 0) {
          // leaving: the previous launch's orphans nobody took move on too
          for (int i = atomicAdd(&dev->orph_take, 1); i < dev->orph_n[prev] && i < kServeOrphans;
               i = atomicAdd(&dev->orph_take, 1)) {
            const int j = atomicAdd(&dev->orph_n[cur], 1);
            if (j < kServeOrphans) dev->orph[cur][j] = dev->orph[prev][i];
          }
        }
      }
      code = __shfl_sync(0xffffffffu, code, 0);
      // (events handed on by the previous launch come in any order: one
      // before the request last found restarts the search at the oldest
      // request of this launch)
      if (have && g < s_d.ev_base) {
        have = false;
        cursor = seq_start;
      }
      // the request holding event g, from the cursor on in sequence order: a
      // slot that no longer holds the cursor's request held a finished one
      // (the host reuses a slot only for a later request, after the earlier
      // one completed).  Bounded: a broken invariant ends the kernel with
      // PV_ERR_NOTFOUND instead of searching on.
      for (unsigned int hops = 0;
           code < 0 && !(have && g >= s_d.ev_base && g < s_d.ev_base + s_d.T.n_events); ++hops) {
        if (hops > (1u << 16)) {
          code = PV_ERR_NOTFOUND;
          break;
        }
        have = read_desc(&ctl->ring[cursor % kServeRing], &s_d, cursor);
        __syncwarp();
        if (!have || g >= s_d.ev_base + static_cast<unsigned long long>(s_d.T.n_events)) {
          have = false;
          ++cursor;
        }
        __syncwarp();
      }
      if (threadIdx.x == 0) {
        s_code = code;
        // the event's request: a queue entry (a new one unless the last is it)
        if (code < 0) {
          s_G = TrackScratch{};
          s_G.center = s_d.center;
          s_G.cid = s_d.cid;
          s_G.slot = s_d.slot;
          s_G.A = s_d.A;
          s_G.W = s_d.W;
        }
        if (code < 0 && (Q.nreq == 0 || Q.req[Q.nreq - 1].seq != s_d.seq) &&
            PV_CHECK(Q.nreq < kServeReqs, 22)) {
          ServeReq& R = Q.req[Q.nreq];
          R.O = s_d.O;
          R.A = s_d.A;
          R.W = s_d.W;
          R.slot = s_d.seq % kServeRing;
          R.target = s_d.done_target;
          R.seq = s_d.seq;
          R.events = 0;
          ++Q.nreq;
        }
      }
    }
    __syncthreads();
    if (s_code >= 0) break;
    // (the event's pointers are read from the shared descriptor where they are
    // used: warp 0 rewrites it only after the event)
    const int e = static_cast<int>(s_g - s_d.ev_base);
    find_event<kFindFit | kServe, NT, FLAV>(C, s_d.T, SeedPtrs{}, s_d.O, s_G, smem, e, nullptr, 0,
                                            &Q);
    __syncthreads();
    if (threadIdx.x == 0) Q.req[Q.nreq - 1].events += 1;
  }
  // the vertices still queued
  if (Q.nreq > 0) serve_round<kAccum>(C, Q, ctl, dev);
  if (threadIdx.x == 0) {
    if (atomicAdd(&dev->running, 1) + 1 == static_cast<int>(gridDim.x)) {
      // the last CTA to leave records why
      *reinterpret_cast<volatile unsigned long long*>(&ctl->exit_ns) = global_ns();
      __threadfence_system();
      *reinterpret_cast<volatile int*>(&ctl->exit_code) = s_code;
    }
  }
}

template <int FLAV>
static cudaError_t setup_serve_flav(int nbins) {
  const int sm = static_cast<int>(
      make_layout(nbins, kFindFit, kServeThreads, flavour_split(FLAV) == PV_SPLIT_RECURSIVE).total);
  cudaError_t err = cudaSuccess;
  for (int a = 0; a < 3 && err == cudaSuccess; ++a) {
    auto k = a == 0 ? serve_kernel<FLAV, PV_ACCUM_FP32>
                    : (a == 1 ? serve_kernel<FLAV, PV_ACCUM_KAHAN> : serve_kernel<FLAV, PV_ACCUM_FP64>);
    err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
  }
  return err;
}

cudaError_t serve_setup(int nbins) {
  cudaError_t err = setup_serve_flav<0>(nbins);
  if (err == cudaSuccess) err = setup_serve_flav<1>(nbins);
  if (err == cudaSuccess) err = setup_serve_flav<2>(nbins);
  if (err == cudaSuccess) err = setup_serve_flav<3>(nbins);
  return err;
}

template <int FLAV>
static void* serve_fn(int accum) {
  if (accum == PV_ACCUM_KAHAN) return reinterpret_cast<void*>(serve_kernel<FLAV, PV_ACCUM_KAHAN>);
  if (accum == PV_ACCUM_FP64) return reinterpret_cast<void*>(serve_kernel<FLAV, PV_ACCUM_FP64>);
  return reinterpret_cast<void*>(serve_kernel<FLAV, PV_ACCUM_FP32>);
}

static void* serve_fn_for(const Consts& C) {
  const int flav = flavour_of(C);
  if (flav == 1) return serve_fn<1>(C.accum_mode);
  if (flav == 2) return serve_fn<2>(C.accum_mode);
  if (flav == 3) return serve_fn<3>(C.accum_mode);
  return serve_fn<0>(C.accum_mode);
}

int serve_blocks_per_sm(const Consts& C) {
  int blocks = 0;
  const size_t sm = make_layout(C.nbins, kFindFit, kServeThreads,
                                C.split_mode == PV_SPLIT_RECURSIVE).total;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, serve_fn_for(C), kServeThreads, sm) !=
      cudaSuccess)
    return 0;
  return blocks;
}

cudaError_t launch_serve(const Consts& C, ServeCtl* ctl, ServeDev* dev, unsigned long long idle_ns,
                         unsigned long long seq_start, unsigned int epoch, int grid,
                         cudaStream_t st) {
  const size_t sm = make_layout(C.nbins, kFindFit, kServeThreads,
                                C.split_mode == PV_SPLIT_RECURSIVE).total;
  Consts Cv = C;
  void* args[] = {&Cv, &ctl, &dev, &idle_ns, &seq_start, &epoch};
  return cudaLaunchKernel(serve_fn_for(C), dim3(grid), dim3(kServeThreads), args, sm, st);
}

cudaError_t launch_serve_clock(ServeCtl* ctl, cudaStream_t st) {
  serve_clock_kernel<<<1, 1, 0, st>>>(ctl);
  return cudaGetLastError();
}

}  // namespace pvk
