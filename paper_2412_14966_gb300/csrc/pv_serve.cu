// pv_serve.cu -- the persistent serving kernel: continuous batching of
// requests on the device.
//
// Each CTA loops: it claims the next event of the published request
// sequence (ServeCtl / ServeDev in pv_kernels.cuh), runs steps (a)-(d3) on it
// -- the batched find kernel's event work, with the event's vertices fitted in
// the same CTA -- and, if the event was its request's last to finish, stamps
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

// 64 registers per thread, eight CTAs per SM (measured on the nominal batch as
// one request: 14.5 M events/s at four CTAs per SM, 17.9 M at six, 19.0 M at
// eight)
template <int FLAV, int kAccum>
__global__ void __launch_bounds__(kServeThreads, 8)
serve_kernel(Consts C, ServeCtl* ctl, ServeDev* dev, unsigned long long idle_ns,
             unsigned long long seq_start, unsigned int epoch) {
  constexpr int NT = kServeThreads;
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout Lo = make_layout(C.nbins, kFindFit, NT, flavour_split(FLAV) == PV_SPLIT_RECURSIVE);
  find_prologue<kFindFit, NT>(C, smem, Lo);
  __shared__ ServeDesc s_d;
  __shared__ unsigned long long s_g;
  __shared__ int s_code;
  // warp 0's state: the request the last event fell in, the published count
  // seen last
  unsigned long long cursor = seq_start, pub = 0;
  bool orphans_left = true;           // lane 0: the previous launch's list not exhausted
  bool have = false;
  const int prev = (epoch + 1) & 1, cur = epoch & 1;
  __syncthreads();
  for (;;) {
    if (threadIdx.x < 32) {
      // the next event (lane 0): first the events the previous launch handed
      // on, then the next of the sequence; it is processed once published
      // (bounded wait; an event still unpublished when the wait ends, or when
      // the host asks to stop, is handed on to the next launch)
      int code = -1;
      unsigned long long g = 0;
      if (threadIdx.x == 0) {
        bool got = false;
        if (orphans_left) {
          const int i = atomicAdd(&dev->orph_take, 1);
          if (i < dev->orph_n[prev] && i < kServeOrphans) {
            g = dev->orph[prev][i];
            got = true;
          } else {
            orphans_left = false;
          }
        }
        if (!got) g = atomicAdd(&dev->next_event, 1ull);
        const unsigned long long t0 = global_ns();
        unsigned int nap = 32;
        while (g >= pub) {
          pub = ld_acquire_sys(&ctl->published);
          if (g < pub) break;
          const bool stop = ld_acquire_sys(&ctl->stop) != 0u;
          if (stop || global_ns() - t0 > idle_ns) {
            const int i = atomicAdd(&dev->orph_n[cur], 1);
            if (i < kServeOrphans) dev->orph[cur][i] = g;
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
      g = __shfl_sync(0xffffffffu, g, 0);
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
        s_g = g;
        s_code = code;
      }
    }
    __syncthreads();
    if (s_code >= 0) break;
    const TrackPtrs T = s_d.T;
    const OutPtrs O = s_d.O;
    const int e = static_cast<int>(s_g - s_d.ev_base);
    TrackScratch G{};
    G.center = s_d.center;
    G.cid = s_d.cid;
    G.slot = s_d.slot;
    G.A = s_d.A;
    G.W = s_d.W;
    const unsigned long long slot = s_d.seq % kServeRing, target = s_d.done_target,
                             seq = s_d.seq;
    __syncthreads();                 // s_d may change once thread 0 claims again
    find_event<kFindFit | kServe, NT, FLAV, kAccum>(C, T, SeedPtrs{}, O, G, smem, e, nullptr, 0);
    // the event's outputs are visible device-wide before it counts as done
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned long long before = atomicAdd(&dev->slot_done[slot], 1ull);
      if (before + 1 == target) {
        // the request's last event: its outputs are complete
        __threadfence_system();
        *reinterpret_cast<volatile unsigned long long*>(&ctl->done_ns[slot]) = global_ns();
        st_release_sys(&ctl->done_seq[slot], seq);
      }
    }
  }
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
