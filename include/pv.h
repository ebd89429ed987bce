/*
 * pv.h -- C ABI of the GB300 primary-vertex library (libpvgb300.so).
 *
 * Primary-vertex finding and fitting for many independent bunch-crossing
 * events, after Dziurda et al., "A parallel algorithm for fast reconstruction
 * of primary vertices on heterogeneous architectures" (arXiv:2412.14966),
 * Sec. 3.  Units: mm for positions, dimensionless slopes, mm^2 (and mm, 1) for
 * covariance terms.
 *
 * Conventions for every entry point:
 *   - Return value: PV_OK (0) or one of the PV_ERR_* codes below; nothing is
 *     thrown across the ABI.  pv_strerror() names a code.
 *   - "device" pointers are CUDA device (or managed) memory on the context's
 *     device; "host" pointers are ordinary or pinned host memory.  The caller
 *     owns every input and output buffer; the context owns only its scratch
 *     memory, CUDA graphs and serving state.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued asynchronously on it unless stated.
 *     The context keeps one set of scratch memory per stream it has seen, so
 *     calls on different streams may overlap on the GPU; calls on one stream
 *     run in stream order.  pv_find_fit_static is the exception (one static
 *     scratch array for all calls, see there).
 *   - A context is not thread-safe: calls from several host threads on one
 *     context must be serialised by the caller, except pv_submit, pv_poll and
 *     pv_request_latency_ns, which lock the context's serving state.
 *   - Per-event and per-track problems are reported in the outputs (event and
 *     vertex status words, track_vertex = -1), not as errors: a non-finite
 *     track is simply not used.
 */
#ifndef PV_H
#define PV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define PV_OK 0
#define PV_ERR_ARG 1        /* invalid argument (NULL pointer, bad size, bad config) */
#define PV_ERR_CUDA 2       /* a CUDA runtime call failed (see pv_last_cuda_error) */
#define PV_ERR_CAPACITY 3   /* request larger than a fixed limit of the library */
#define PV_ERR_NOMEM 4      /* scratch or serving pool could not be allocated / admitted */
#define PV_ERR_TIMEOUT 5    /* a bounded wait ran out */
#define PV_ERR_BUSY 6       /* serving queue full; retry after pv_poll */
#define PV_ERR_NOTFOUND 7   /* unknown serving ticket */

/* ---- vertex status bits (per fitted vertex) ---------------------------- */
#define PV_ST_CONVERGED 1   /* x86 rule of Sec. 3.5: |dchi2| < tol and |dz| < tol */
#define PV_ST_MAXITER 2     /* stopped at max_iter without converging */
#define PV_ST_SINGULAR 4    /* normal matrix not positive definite (e.g. all weights 0) */
#define PV_ST_REJ_BEAM 8    /* pp vertex farther than max_r_beam from the beamline */
#define PV_ST_REJ_NTRK 16   /* fewer than min_pv_tracks tracks with weight > 0 */
#define PV_ST_ACCEPTED 32   /* a primary vertex of the final selection (Sec. 3.5) */
#define PV_ST_DUPLICATE 64  /* multi-vertex fit: rejected as a duplicate of a nearby vertex */

/* ---- event status bits -------------------------------------------------- */
#define PV_EV_SEED_OVERFLOW 1  /* more seed clusters than the capacity; extra ones dropped */
#define PV_EV_BAD_OFFSETS 4    /* offsets not monotone or outside [0, n_tracks]; not processed */

/* ---- fixed limits -------------------------------------------------------- */
#define PV_ONE 4096                   /* histogram weight of one track (fixed point) */
#define PV_MAX_SEEDS 64               /* seed / vertex capacity per event */
#define PV_MAX_BINS 4096              /* histogram bins per event */

/* accumulation of the weighted normal equations in the fit */
#define PV_ACCUM_FP32 0    /* binary32 per lane and across lanes */
#define PV_ACCUM_KAHAN 1   /* compensated binary32 (error-free transformations) */
#define PV_ACCUM_FP64 2    /* binary64 sums, reduction and solve (binary32 per-track terms) */

/* histogram profile (Sec. 3.2) */
#define PV_PROFILE_CUBIC 0     /* GPU flavour: quantised cubic CDF (default) */
#define PV_PROFILE_TEMPLATE 1  /* x86 flavour: template histograms chosen by sigma_poca */

/* dip splitting of proto-clusters (Sec. 3.3) */
#define PV_SPLIT_ZORDER 0     /* GPU flavour: minima in z order (default) */
#define PV_SPLIT_RECURSIVE 1  /* x86 flavour: smallest minimum between the two largest maxima, recursively */

/* execution path */
#define PV_PATH_FUSED 0    /* bucketed persistent kernels, shared-memory histograms */
#define PV_PATH_PLAIN 1    /* one kernel per step, global-memory histograms */

/* Beamline at z = 0 and its slopes (Sec. 3: x_b, y_b, t_x,b, t_y,b). */
typedef struct {
  float x_b, y_b, tx_b, ty_b;
} pv_beamline;

/* Algorithm settings; pv_config_default() fills the paper's values. */
typedef struct {
  float z_min, z_max, dz;           /* histogram range and bin width (Sec. 3.2): -550, 300, 0.25 */
  float z_gas;                      /* p-gas parameters below this z (Table smog-pp): -300 */
  float sigma_max_pp, sigma_max_gas;        /* max sigma_poca to fill (Sec. 3.2): 1.5, 10 */
  float min_integral_pp, min_integral_gas;  /* min cluster integral, tracks (Table smog-pp): 2.5, 1.75 */
  uint32_t bin_threshold;           /* proto-cluster threshold in 1/PV_ONE tracks (unstated): 205 */
  int32_t dip_num, dip_den;         /* dip significant if den*N_min < num*min(N_L, N_R) (unstated): 4, 5 */
  int32_t min_assoc_pp, min_assoc_gas;      /* min tracks per cluster in association (Sec. 3.4): 3, 2 */
  int32_t min_pv_tracks_pp, min_pv_tracks_gas;  /* min tracks with w > 0 (Table smog-pp): 4, 3 */
  float chi2_max;                   /* Tukey cut-off (Sec. 3.5): 12 */
  float dchi2_tol, dz_tol;          /* convergence (Sec. 3.5): 0.01, 0.001 mm */
  int32_t max_iter;                 /* maximal fit iterations (Sec. 3.5): 10 */
  float max_r_beam;                 /* final transverse cut for pp vertices (Sec. 3.5): 0.3 mm */
  int32_t accum_mode;               /* PV_ACCUM_*: default PV_ACCUM_FP32 */
  int32_t path;                     /* PV_PATH_*: default PV_PATH_FUSED */
  int32_t use_graph;                /* 1: the fused find+fit launch is captured once per
                                       argument set as a CUDA graph and replayed: default 0 */
  int32_t reserved;                 /* 0 */
  uint64_t pool_bytes;              /* serving: device bytes admitted requests may pin (0 = 1 GiB) */
  uint64_t max_spin_ns;             /* serving: bound of every wait (0 = 10 s) */
  /* multi-vertex fit (pv_fit_multi, Sec. 3.5 GPU implementation) */
  float mv_chi2_cut;                /* chi2_max of the multi-vertex weight (weight figure): 4 */
  float mv_dz_tol;                  /* convergence |dz| (Sec. 3.5, GPU rule): 0.0005 mm */
  float mv_w_assoc;                 /* weight from which a track counts for a vertex: 0.5 */
  float mv_dup_sep2;                /* duplicates: dz^2 < mv_dup_sep2 (C_zz + C_zz') (Sec. 3.5): 25 */
  int32_t split_mode;               /* PV_SPLIT_*: default PV_SPLIT_ZORDER */
  int32_t profile_mode;             /* PV_PROFILE_*: default PV_PROFILE_CUBIC */
} pv_config;

/* Tracks in structure-of-arrays layout (Sec. 5, x86: one contiguous array per
 * member), grouped by event through CSR offsets.  Track i of the batch has its
 * state (x, y, t_x, t_y) at z (Sec. 2) and the covariance terms V_xx, V_xtx,
 * V_txtx, V_yy, V_yty, V_tyty.  The 11 float arrays and event_offsets live in
 * the same memory space (device for the device entry points, host for
 * pv_run_host).  event_offsets has n_events + 1 entries; event e owns tracks
 * [event_offsets[e], event_offsets[e+1]). */
typedef struct {
  const float *x, *y, *z, *tx, *ty;
  const float *cxx, *cxtx, *ctxtx, *cyy, *cyty, *ctyty;
  const int64_t* event_offsets;
  int64_t n_tracks;
  int32_t n_events;
} pv_tracks;

/* Seeds or vertices, row-major [event][capacity] unless stated.  Any pointer
 * marked optional may be NULL.  cov holds 6 floats per vertex in the order
 * xx, xy, yy, xz, yz, zz (C = (1/2 d2chi2/dalpha2)^-1, Sec. 3.5). */
typedef struct {
  float *x, *y, *z;             /* seed position (find) or fitted position (fit) */
  float* cov;                   /* optional; [event][capacity][6] */
  float *chi2, *ndof;           /* optional; vertex chi2 = chi2_0 + dchi2 and 2 sum(w) - 3 */
  int32_t *n_tracks, *n_iter, *status;   /* optional; tracks with w > 0, iterations, PV_ST_* */
  int32_t *bin_lo, *bin_hi, *bin_max;    /* optional; seed cluster bins and its maximum bin */
  int32_t* n_per_event;         /* [n_events]: seeds (= vertices) of each event */
  int32_t* event_status;        /* optional; [n_events] PV_EV_* bits */
  int32_t* track_vertex;        /* [n_tracks]: seed / vertex index in its event, -1 if none */
  int32_t capacity;             /* per event, 1 .. PV_MAX_SEEDS */
} pv_vertices;

typedef struct pv_ctx pv_ctx;

/* Fill cfg with the paper's settings (values listed in pv_config). */
void pv_config_default(pv_config* cfg);

/* Create a context on CUDA device `device`.  cfg and beam are copied; NULL
 * means defaults / a beamline at the origin with zero slope.  Checks the
 * configuration (PV_ERR_ARG: nbins outside 1..PV_MAX_BINS, dz <= 0, ...).
 * *out receives the context; release it with pv_destroy. */
int pv_init(const pv_config* cfg, const pv_beamline* beam, int device, pv_ctx** out);

/* Release the context, its scratch memory, graphs and serving state.  Waits
 * (bounded by max_spin_ns) for in-flight serving requests. */
int pv_destroy(pv_ctx* ctx);

/* Steps (a)-(d1) of Sec. 3 on a batch: extrapolate each track to the
 * beamline (Eq. zpocadef, sigma_poca of Sec. 3.1), fill each event's z
 * histogram (Sec. 3.2), find seed clusters (Sec. 3.3) and associate tracks
 * (Sec. 3.4).  tracks: device SoA.  seeds_out (device): x, y, z = seed
 * position (beamline at z_seed); bin_lo/hi/max if given; n_per_event;
 * event_status if given; track_vertex.  Asynchronous on cuda_stream.
 * PV_ERR_ARG for NULL required pointers or capacity outside 1..64. */
int pv_find_batch(pv_ctx* ctx, const pv_tracks* tracks, pv_vertices* seeds_out, void* cuda_stream);

/* Steps (d2)-(d3): adaptive Tukey-weighted vertex fit of every seed from its
 * associated tracks (Sec. 3.5) and the final selection.  seeds (device) as
 * written by pv_find_batch (x, y, z, n_per_event, track_vertex are read);
 * out (device) receives one vertex per seed, same indices, with status bits;
 * out->n_per_event and out->track_vertex are written (copies of the seeds').
 * seeds == NULL runs find and fit as one fused pass (the fast path).
 * Asynchronous on cuda_stream. */
int pv_fit_batch(pv_ctx* ctx, const pv_tracks* tracks, const pv_vertices* seeds,
                 pv_vertices* out, void* cuda_stream);

/* The GPU flavour of step (d) (Sec. 3.5): every seed of an event is fitted
 * with weights that share each track among all vertices,
 * w_ij = exp(-chi2_ij/2) / (exp(-mv_chi2_cut/2) + sum_k exp(-chi2_ik/2)),
 * the other vertices k entering at their seed positions; iterations stop at
 * |dz| < mv_dz_tol (at most max_iter).  Then vertices closer than
 * dz^2 < mv_dup_sep2 (C_zz + C_zz') to the last kept one (seed order) lose
 * to the one with more tracks (PV_ST_DUPLICATE), and the final selection of
 * Sec. 3.5 applies.  A vertex's tracks (n_tracks, the track minimum) are those
 * with w >= mv_w_assoc in its last iteration; out->track_vertex receives each
 * track's vertex of largest last-iteration weight if that weight is
 * >= mv_w_assoc, else -1.  Every usable track of an event enters every fit.
 * seeds (device): positions and n_per_event as pv_find_batch writes them, or
 * NULL to find the seeds first (into out).  out (device) as for
 * pv_fit_batch.  Binary32 per-track terms and sums.  Asynchronous on
 * cuda_stream. */
int pv_fit_multi(pv_ctx* ctx, const pv_tracks* tracks, const pv_vertices* seeds,
                 pv_vertices* out, void* cuda_stream);

/* Step (a) alone: z_poca, sigma_poca and the center bin (-1 = not filled) of
 * every track of the batch, in the pinned binary32 sequence.  Device
 * outputs of n_tracks entries; any may be NULL.  Asynchronous. */
int pv_extrapolate_batch(pv_ctx* ctx, const pv_tracks* tracks, float* zpoca, float* sigma_poca,
                         int32_t* center_bin, void* cuda_stream);

/* Steps (a)-(b): the integer histogram of every event (PV_ONE per fully
 * contained track), row-major [n_events][nbins] uint32 in device memory.
 * Asynchronous. */
int pv_histogram_batch(pv_ctx* ctx, const pv_tracks* tracks, uint32_t* hist, void* cuda_stream);

/* Number of histogram bins of the context's configuration. */
int pv_num_bins(const pv_ctx* ctx);

/* Bounds-check record of the checked build (the library compiled with
 * PV_CHECKED=1, a test build): its kernels test the indices of their main
 * shared- and global-memory accesses and skip, and count, any that would leave
 * its buffer.  Synchronises the current device, writes the number of such
 * indices since the last call to *count and the code of the first one to
 * *first_code (both 0 when none), and resets them.  Returns PV_OK in the
 * checked build; the default build has no checks, writes 0 to both and returns
 * PV_ERR_ARG (also for NULL arguments). */
int pv_check_report(uint32_t* count, uint32_t* first_code);

/* The whole method through host memory: copies the host SoA tracks to
 * context-owned device buffers, runs the fused find+fit, delivers the vertex
 * outputs into the host pv_vertices and synchronises cuda_stream.  All
 * pointers in tracks and out are host pointers (pinned memory gives
 * asynchronous copies).  Batches of 4,096 events or more with rising offsets
 * run as two event chunks whose copies overlap the other chunk's kernels.  On
 * the fused path, outputs in pinned (CUDA-registered) memory are written by
 * the kernels in place: only the slots of found vertices (and every event and
 * track entry) are written, the other slots keep their contents.  Other
 * outputs, and all outputs of the plain path, are staged on the device and
 * copied back whole.  Blocking. */
int pv_run_host(pv_ctx* ctx, const pv_tracks* tracks, pv_vertices* out, void* cuda_stream);

/* Serving: continuous batching on the device.  pv_submit queues a request
 * (device tracks and outputs, borrowed until pv_poll reports done) and never
 * blocks.  A request is admitted when the serving pool (pool_bytes of device
 * memory; 31 bytes per track of scratch) has room for it -- any waiting
 * request that fits, not only the oldest -- and then written into a request
 * ring in pinned host memory that a persistent serving kernel reads: its
 * CTAs claim the published events of all admitted requests one at a time, run
 * steps (a)-(d3) on each (the fused path's find and fit, the event's vertices
 * fitted in the same CTA) and stamp a request's completion with the GPU's
 * global timer when its last event finishes.  Requests that arrive while
 * others run overlap with them on the device; a request's results equal those
 * of pv_fit_batch with seeds == NULL on the same context.  *ticket identifies
 * the request.  PV_ERR_BUSY if 4,096 requests already wait for admission,
 * PV_ERR_NOMEM if the request alone exceeds the pool.  The serving kernel
 * occupies the device while it runs; it ends after 2 ms (or max_spin_ns, if
 * shorter) without an event to claim, and pv_submit / pv_poll start it again
 * while requests are in flight. */
int pv_submit(pv_ctx* ctx, const pv_tracks* tracks, pv_vertices* out, uint64_t* ticket);

/* Non-blocking completion check: *done = 1 once the request's outputs are
 * complete in device memory, else 0; also admits waiting requests and keeps
 * the serving kernel running.  PV_ERR_NOTFOUND for an unknown or already
 * retired ticket. */
int pv_poll(pv_ctx* ctx, uint64_t ticket, int* done);

/* Latency of a completed request in nanoseconds, from pv_submit to the
 * device's completion stamp of its last event (the GPU's global timer,
 * calibrated against the host clock when the serving pool is set up), then
 * retires the ticket (later calls with it return PV_ERR_NOTFOUND).
 * PV_ERR_NOTFOUND if the ticket is unknown or not yet done. */
int pv_request_latency_ns(pv_ctx* ctx, uint64_t ticket, uint64_t* ns);

/* Sets up the serving pool and starts the serving kernel now, with or without
 * requests (it ends on its own after its idle bound, see pv_submit). */
int pv_serve_start(pv_ctx* ctx);

/* *running = 1 while the serving kernel runs; *last_exit = how its last run
 * ended when it is not running: PV_OK (stopped by pv_destroy),
 * PV_ERR_TIMEOUT (no event to claim within its idle bound), -1 if it never
 * ended.  Either pointer may be NULL. */
int pv_serve_status(pv_ctx* ctx, int* running, int* last_exit);

/* Steps (a)-(d3) as one fused pass, like pv_fit_batch with seeds == NULL,
 * but without allocating device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while
 * they run (cudaMalloc / cudaFree may synchronise the whole device, which a
 * real-time loop cannot afford; some applications give all device memory to
 * their own allocator and run with a fixed budget).  Its scratch is a static
 * device array of 8 MiB in the library, held by every GPU that loads the
 * library until the process exits.  A batch of n tracks needs 31 bytes per
 * track plus 32 bytes per entry of four vertex work lists (one per size class
 * of at least 1, 9, 17 and 33 tracks) holding min(n / 1, S), min(n / 9, S),
 * min(n / 17, S) and min(n / 33, S) entries, S being the smaller of n and
 * events x out->capacity: about 165,000 tracks of 160-track events at
 * capacity 64.  Batches needing more are refused with PV_ERR_CAPACITY and a
 * message in pv_last_cuda_error.  The first call on a device looks the array up
 * (cudaGetSymbolAddress); make that first call before any stream capture.  The
 * address is kept for the life of the process: it assumes the device's primary
 * context lives as long (do not call this entry point after cudaDeviceReset).
 * All calls share the array, so calls whose work overlaps on the GPU race:
 * run them on one stream or order them with events.  tracks and out are
 * device memory as for pv_fit_batch; the context's path setting is ignored
 * (always the fused kernel).  Asynchronous on cuda_stream. */
int pv_find_fit_static(pv_ctx* ctx, const pv_tracks* tracks, pv_vertices* out, void* cuda_stream);

/* Project-written autotuner of the fused path's launch shape.  Runs the fused
 * find+fit on `sample` (device tracks) into `out` (device) with every
 * candidate pair of block sizes (find kernel 64/96/128/256 threads, fit kernel
 * 128/256), each with its occupancy-sized persistent grid, times them with
 * CUDA events on cuda_stream, and keeps the fastest for the sample's
 * event-size bucket (mean tracks per event below 300, below 800, 800 and
 * more).  Later launches on batches of that bucket use it.  The results of
 * the method do not depend on the launch shape.  Synchronises cuda_stream. */
int pv_autotune(pv_ctx* ctx, const pv_tracks* sample, pv_vertices* out, void* cuda_stream);

/* The launch shape the fused path would use for `tracks`: block sizes of the
 * find and fit kernels (any pointer may be NULL). */
int pv_launch_config(const pv_ctx* ctx, const pv_tracks* tracks, int* find_threads,
                     int* fit_threads, int* find_grid, int* fit_grid);

/* Set the launch shape of an event-size bucket (0: mean tracks per event
 * below 300, 1: below 800, 2: 800 and more) by hand: find kernel 64, 96, 128
 * or 256 threads, fit kernel 128 or 256.  PV_ERR_ARG for other values. */
int pv_set_launch_config(pv_ctx* ctx, int bucket, int find_threads, int fit_threads);

/* Human-readable name of an error code. */
const char* pv_strerror(int code);

/* The last CUDA error string seen by the context (or "" if none). */
const char* pv_last_cuda_error(const pv_ctx* ctx);

/* Number of kernel launches the library enqueued since the context was
 * created (all entry points); used to count launches in a timed region. */
uint64_t pv_launch_count(const pv_ctx* ctx);

/* Device memory the context holds (scratch of every stream it has seen, the
 * template table, pv_run_host's staging and the serving pool), in bytes; 0
 * for NULL.  Grows only when an entry point needs more. */
uint64_t pv_device_bytes(const pv_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PV_H */
