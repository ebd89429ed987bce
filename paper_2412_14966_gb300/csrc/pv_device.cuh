// pv_device.cuh -- device building blocks of the primary-vertex kernels.
//
// Steps (a)-(d1) of the method (extrapolation, histogram, peak search,
// association) follow a pinned IEEE binary32 operation sequence written with
// round-to-nearest intrinsics (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn),
// which the compiler never contracts into FMAs.  Histogram weights are
// integers, so histograms, seeds and track assignments are exact and
// independent of thread order.  The fit (d2) runs in binary32 with a fixed
// lane-to-track mapping and a fixed shuffle tree, so its result depends only
// on the event's own data, not on block size or scheduling.
#pragma once

#include <cstdint>
#include <type_traits>

#include "pv.h"

namespace pvdev {

// Checked build (compiled with PV_CHECKED=1 into a separate library for the
// tests): the kernels test the indices of their main shared- and global-memory
// accesses, skip an access that would leave its buffer and count it (read back
// through pv_check_report).  The default build compiles the tests away.
#ifndef PV_CHECKED
#define PV_CHECKED 0
#endif
#if PV_CHECKED
// out-of-bounds indices met by the checked build: their number and the code
// of the first one (one pair per translation unit, read by its report)
static __device__ unsigned int g_check_count;
static __device__ unsigned int g_check_first;
#if defined(__CUDA_ARCH__)
static __device__ __noinline__ void check_failed(unsigned code) {
  if (atomicAdd(&g_check_count, 1u) == 0u) g_check_first = code;
}
#define PV_CHECK(cond, code) ((cond) ? true : (::pvdev::check_failed(code), false))
#else
#define PV_CHECK(cond, code) true
#endif
#else
#define PV_CHECK(cond, code) true
#endif

constexpr int kOne = PV_ONE;
constexpr int kMaxSeeds = PV_MAX_SEEDS;
constexpr int kMaxBins = PV_MAX_BINS;
constexpr int kMaxTiles = kMaxBins / 32;
constexpr int kTileWords = kMaxTiles / 32;
constexpr float kSqrt5 = 2.23606797749979f;   // half-width of the profile in sigma units
constexpr float kSMin = 1e-6f;                // narrower profiles fill a single bin
constexpr int kGroup = 8;                     // lanes that fit one vertex
constexpr float kPivotRel = 1e-4f;            // z pivot below this share of M_zz: singular
constexpr int kGroupsPerWarp = 32 / kGroup;
// ring of proto-cluster bounds in the peak search: at most 31 are pending
// when a tile is scanned and a 32-bin tile ends at most 16 runs
constexpr int kRunRing = 64;
static_assert(kMaxBins <= 32767, "bin indices are stored as int16");

// Derived settings, passed by value to every kernel.
struct Consts {
  float z_min, dz, z_gas;
  float inv_dz;             // 1/dz when dz is a power of two (exact), else 0
  float sig_max_pp, sig_max_gas;
  float x_b, y_b, tx_b, ty_b;
  float chi2_max, inv_chi2_max, dchi2_tol, dz_tol, max_r_beam;
  uint32_t thr;             // proto-cluster bin threshold (1/ONE units)
  uint32_t t_pp, t_gas;     // minimal cluster integrals (1/ONE units)
  int32_t dip_num, dip_den;
  int32_t min_assoc_pp, min_assoc_gas, min_pv_pp, min_pv_gas;
  int32_t nbins, ntiles, gas_bin;
  int32_t max_iter;
  int32_t accum_mode;
  // multi-vertex fit
  float mv_ecut;            // exp(-chi2_cut / 2)
  float mv_dz_tol, mv_w_assoc, mv_dup_sep2;
  int32_t split_mode;       // PV_SPLIT_*
  int32_t profile_mode;     // PV_PROFILE_*
  const struct TplTable* tpl;   // template profiles (device memory)
};

// ---------------------------------------------------------------------------
// template profiles of the x86 flavour (Sec. 3.2): class k has
// sigma_k = 0.01 mm 2^(k/4) and takes sigma_poca from sigma_{k-1} 2^(1/8) up.
// q holds, per class, the quantised Gaussian CDF Q[0 .. 2H+1] at the bin
// edges (i - H - 1/2) dz around the centre bin, Q[0] = 0, Q[2H+1] = ONE.
constexpr int kTplClasses = 41;
constexpr int kTplMaxHalf = 1024;
constexpr int kTplCap = 16384;               // entries of q
constexpr double kTplSigma0 = 0.01;          // mm
constexpr double kTplRatio = 1.189207115002721;       // 2^(1/4)
constexpr double kTplHalfRatio = 1.0905077326652577;  // 2^(1/8)

struct TplTable {
  double bound[kTplClasses];   // lowest sigma_poca of class k; bound[0] = 0
  int32_t half[kTplClasses];   // H_k
  int32_t first[kTplClasses];  // start of class k in q
  int32_t status;              // 0 ok, 1 the table does not fit
  int32_t q[kTplCap];
};

// class of sigma_poca: the last class whose lower bound it reaches
__device__ __forceinline__ int tpl_class(float sigma, const TplTable* t) {
  const double s = static_cast<double>(sigma);
  int lo = 0, hi = kTplClasses - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s >= __ldg(t->bound + mid)) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Brings the 128-byte line holding *p into L2 (no register result).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ---------------------------------------------------------------------------
// step (a): extrapolation, Eq. zpocadef, Eq. Vxy (diagonal block), sigma_poca

// Bin of v: floor((v - z_min) / dz); -1 below the range, nbins above it.
__device__ __forceinline__ int bin_of(float v, const Consts& C) {
  // dividing by a power of two and multiplying by its exact reciprocal give
  // the same correctly rounded result
  float diff = __fsub_rn(v, C.z_min);
  float q = C.inv_dz != 0.0f ? __fmul_rn(diff, C.inv_dz) : __fdiv_rn(diff, C.dz);
  if (!(q >= 0.0f)) return -1;
  if (q >= __int2float_rn(C.nbins)) return C.nbins;
  return static_cast<int>(q);
}

__device__ __forceinline__ float edge_of(int j, const Consts& C) {
  return __fadd_rn(C.z_min, __fmul_rn(__int2float_rn(j), C.dz));
}

struct Prep {
  float zpoca, sigma;
  int center, j0, j1;
  int tq;                  // template profile: start of its class in q
  bool filled;
};

// The profile window [j0, j1] is z_poca +- sqrt(5) sigma_poca for the cubic
// profile and the class template's c - H .. c + H for kProfile = TEMPLATE.
template <int kProfile = PV_PROFILE_CUBIC>
__device__ __forceinline__ Prep prepare_track(float x, float y, float z, float tx, float ty,
                                              float cxx, float cxtx, float ctxtx,
                                              const Consts& C) {
  Prep r;
  float dtx = __fsub_rn(tx, C.tx_b);
  float dty = __fsub_rn(ty, C.ty_b);
  float t2 = __fadd_rn(__fmul_rn(dtx, dtx), __fmul_rn(dty, dty));
  float xb = __fadd_rn(C.x_b, __fmul_rn(C.tx_b, z));   // beam at the track's z
  float yb = __fadd_rn(C.y_b, __fmul_rn(C.ty_b, z));
  float num = __fadd_rn(__fmul_rn(dtx, __fsub_rn(xb, x)), __fmul_rn(dty, __fsub_rn(yb, y)));
  float zp = __fadd_rn(z, __fdiv_rn(num, t2));
  float d = __fsub_rn(zp, z);
  float vxx = __fadd_rn(__fadd_rn(cxx, __fmul_rn(__fmul_rn(2.0f, d), cxtx)),
                        __fmul_rn(__fmul_rn(d, d), ctxtx));
  float sig = __fsqrt_rn(__fdiv_rn(vxx, t2));
  r.zpoca = zp;
  r.sigma = sig;
  r.filled = false;
  r.center = -1;
  r.j0 = 0;
  r.j1 = -1;
  r.tq = 0;
  if (!(t2 > 0.0f)) return r;
  if (!isfinite(zp) || !isfinite(sig)) return r;
  int c = bin_of(zp, C);
  if (c < 0 || c >= C.nbins) return r;
  float smax = (zp < C.z_gas) ? C.sig_max_gas : C.sig_max_pp;
  if (!(sig <= smax)) return r;
  r.filled = true;
  r.center = c;
  if constexpr (kProfile == PV_PROFILE_TEMPLATE) {
    const int k = tpl_class(sig, C.tpl);
    const int H = __ldg(C.tpl->half + k);
    r.tq = __ldg(C.tpl->first + k);
    r.j0 = c - H;
    r.j1 = c + H;
  } else {
    float s = __fmul_rn(kSqrt5, sig);
    if (s < kSMin) s = 0.0f;
    r.j0 = bin_of(__fsub_rn(zp, s), C);
    r.j1 = bin_of(__fadd_rn(zp, s), C);
  }
  return r;
}

// ---------------------------------------------------------------------------
// step (b): integer profile = quantised cubic CDF of the variance-matched
// Epanechnikov kernel, F(u) = 1/2 + u (3/4 - u^2/4), u in [-1, 1].

// For every binary32 u in (-1, 1) this sequence gives 0 <= q <= ONE (checked
// exhaustively on the host with the same round-to-nearest steps; the test
// suite checks the values next to -1 and 1, where the extremes lie), so q
// needs no clamp.
__device__ __forceinline__ int quant_cdf(float u) {
  if (!(u > -1.0f)) return 0;
  if (u >= 1.0f) return kOne;
  float a = __fmul_rn(u, u);
  float b = __fmul_rn(0.25f, a);
  float c = __fsub_rn(0.75f, b);
  float d = __fmul_rn(u, c);
  float F = __fadd_rn(0.5f, d);
  return __float2int_rn(__fmul_rn(F, static_cast<float>(kOne)));
}

// Add one filled track's profile to hist (shared or global memory).
__device__ __forceinline__ void fill_profile(uint32_t* hist, float zpoca, float sigma, int j0, int j1,
                                             const Consts& C) {
  float s = __fmul_rn(kSqrt5, sigma);
  if (s < kSMin) s = 0.0f;
  float inv_s = (s > 0.0f) ? __fdiv_rn(1.0f, s) : 0.0f;
  int qprev = 0;
  for (int j = j0; j <= j1; ++j) {
    int qnext;
    if (j == j1) {
      qnext = kOne;
    } else {
      float e = edge_of(j + 1, C);
      qnext = quant_cdf(__fmul_rn(__fsub_rn(e, zpoca), inv_s));
    }
    qnext = qnext < qprev ? qprev : qnext;
    int w = qnext - qprev;
    if (w > 0 && j >= 0 && j < C.nbins) atomicAdd(hist + j, static_cast<uint32_t>(w));
    qprev = qnext;
  }
}

// Add one filled track's template profile (class start tq in q) to hist.
__device__ __forceinline__ void fill_template(uint32_t* hist, int tq, int j0, int j1,
                                              const Consts& C) {
  const int32_t* q = C.tpl->q + tq;
  if (!PV_CHECK(tq >= 0 && tq + (j1 - j0) + 1 < kTplCap, 3)) return;
  for (int j = j0; j <= j1; ++j) {
    const int w = __ldg(q + (j - j0) + 1) - __ldg(q + (j - j0));
    if (w > 0 && j >= 0 && j < C.nbins) atomicAdd(hist + j, static_cast<uint32_t>(w));
  }
}

// The quantised CDF value Q_i at edge i of a window starting at bin j0: the
// cubic CDF at the bin edge j0 + i (inv = 1 / (sqrt(5) sigma_poca)), or with
// kProfile = TEMPLATE the class template's Q[i] (tq: the class's start in q).
// Bin j0 + i of a window of nb bins receives Q_{i+1} - Q_i with Q_0 = 0 and
// Q_nb = ONE (fill_profile, fill_template).  Q is non-decreasing along a
// window (F is monotone on [-1, 1], every binary32 step of u and F is a
// monotone rounding, and window edges are at least dz / (sqrt(5) sigma_max) =
// 0.011 apart in u, far above the rounding error of F), so the running-max
// guard of fill_profile never acts and a fill that adds Q_{i+1} - Q_i per bin
// in any order builds the same histogram (integer adds commute).
template <int kProfile>
__device__ __forceinline__ int profile_q(int i, int j0, float zpoca, float inv_s, int tq,
                                         const Consts& C) {
  if constexpr (kProfile == PV_PROFILE_TEMPLATE) {
    return PV_CHECK(tq + i < kTplCap, 1) ? __ldg(C.tpl->q + tq + i) : 0;
  } else {
    return quant_cdf(__fmul_rn(__fsub_rn(edge_of(j0 + i, C), zpoca), inv_s));
  }
}

// ---------------------------------------------------------------------------
// step (c): proto-clusters, dip splitting in z order, seeds

struct SeedOut {   // shared-memory seed table of one event
  int lo[kMaxSeeds], hi[kMaxSeeds], bin[kMaxSeeds];
  float z[kMaxSeeds], x[kMaxSeeds], y[kMaxSeeds];
  uint32_t nm[kMaxSeeds], ni[kMaxSeeds], np[kMaxSeeds];   // N[bin-1], N[bin], N[bin+1]
};

// Walk proto-cluster [a, b] of N; calls emit(lo, hi, integral, im) per piece
// in z order, im being the piece's maximum bin (lowest index on ties).
// Splits at the leftmost bin of a significant minimum between the running
// maximum of the open piece (L, first reached at bin iL) and the next maximum
// (R, first reached at bin kf) if both the piece [s, m] and the rest
// [m+1, b] hold the minimal integral.  A piece's maximum is L: values fall
// after it up to the split point, and the piece after a split starts with
// the minimum's plateau and the ascent to R.
template <class Emit>
__host__ __device__ void split_walk(const uint32_t* N, int a, int b, uint64_t total,
                                    const Consts& C, Emit&& emit) {
  int s = a;
  uint64_t pre_s = 0;                 // sum over [a, s)
  int top = a, iL = a;
  uint64_t pre = N[a];                // sum over [a, top]
  while (top < b && N[top + 1] >= N[top]) {
    ++top;
    pre += N[top];
    if (N[top] > N[top - 1]) iL = top;
  }
  uint32_t L = N[top];
  while (top < b) {
    int j = top, m = top;
    uint64_t pre_j = pre, pre_m = pre;
    while (j < b && N[j + 1] <= N[j]) {
      ++j;
      pre_j += N[j];
      if (N[j] < N[j - 1]) { m = j; pre_m = pre_j; }
    }
    if (j == b) break;
    int k = j, kf = j;
    uint64_t pre_k = pre_j;
    while (k < b && N[k + 1] >= N[k]) {
      ++k;
      pre_k += N[k];
      if (N[k] > N[k - 1]) kf = k;
    }
    uint32_t R = N[k];
    uint32_t lower = L < R ? L : R;
    bool split = false;
    if (static_cast<uint64_t>(C.dip_den) * N[m] < static_cast<uint64_t>(C.dip_num) * lower) {
      uint64_t T = (m < C.gas_bin) ? C.t_gas : C.t_pp;
      if (pre_m - pre_s >= T && total - pre_m >= T) split = true;
    }
    if (split) {
      emit(s, m, pre_m - pre_s, iL);
      s = m + 1;
      pre_s = pre_m;
      L = R;
      iL = kf;
    } else if (R > L) {
      L = R;
      iL = kf;
    }
    top = k;
    pre = pre_k;
  }
  emit(s, b, total - pre_s, iL);
}

// The x86 flavour of the dip splitting (Sec. 3.3): the smallest bin between
// the two largest maxima of [a, b] (a maximum is a run of equal bins higher
// than its neighbours inside [a, b]; equal maxima by lower position; leftmost
// minimum), split there when the dip is significant against the smaller
// maximum and both sides hold the minimal integral, then the same on each
// side, to any depth.  Calls emit(lo, hi, integral, im) per piece in z order;
// total is the integral of [a, b].  A range's first-found largest maximum is
// its argmax (lowest index).  Pieces come out in z order, so every piece but
// the last ends at the split point of the innermost pending right-hand side,
// which starts one bin later: the pending sides need no stack, only their last
// bin, kept in mark[m - a] at their split point m (mark: b - a + 1 int16
// entries of scratch).  A left side's integral is summed while it is split
// off, a right side's during its maxima scan.
template <class Emit>
__host__ __device__ void split_recursive(const uint32_t* N, int a, int b, uint64_t total,
                                         const Consts& C, Emit&& emit, int16_t* mark) {
  int lo = a, hi = b;
  uint64_t integral = total;
  bool known = true;                  // integral of [lo, hi] known
  for (;;) {
    // one pass over the runs of equal bins (one load per bin): a run is a
    // maximum if the bins on both sides are lower (the range ends count as
    // lower); runs come in z order, so equal maxima keep the lower position
    int m1 = -1, m2 = -1;
    uint32_t v1 = 0, v2 = 0;
    {
      int start = lo;
      uint32_t v = N[lo];
      uint64_t sum = v;
      bool left_lower = true;
      for (int i = lo + 1; i <= hi + 1; ++i) {
        const uint32_t nv = i <= hi ? N[i] : 0u;
        sum += nv;
        if (i > hi || nv != v) {
          if (left_lower && (i > hi || nv < v)) {
            if (m1 < 0 || v > v1) {
              m2 = m1; v2 = v1;
              m1 = start; v1 = v;
            } else if (m2 < 0 || v > v2) {
              m2 = start; v2 = v;
            }
          }
          left_lower = v < nv;
          start = i;
          v = nv;
        }
      }
      if (!known) integral = sum;
    }
    if (m2 >= 0) {
      const int l = m1 < m2 ? m1 : m2, h = m1 < m2 ? m2 : m1;
      int m = -1;
      uint32_t vm = 0;
      for (int i = l + 1; i < h; ++i) {
        const uint32_t x = N[i];
        if (m < 0 || x < vm) { m = i; vm = x; }
      }
      const uint32_t lower = v1 < v2 ? v1 : v2;
      if (m >= 0 &&
          static_cast<uint64_t>(C.dip_den) * vm < static_cast<uint64_t>(C.dip_num) * lower) {
        const uint64_t T = (m < C.gas_bin) ? C.t_gas : C.t_pp;
        uint64_t left = 0;
        for (int i = lo; i <= m; ++i) left += N[i];
        const uint64_t right = integral - left;
        if (left >= T && right >= T) {
          mark[m - a] = static_cast<int16_t>(hi);   // the pending side [m + 1, hi]
          hi = m;
          integral = left;
          known = true;
          continue;
        }
      }
    }
    emit(lo, hi, integral, m1);
    if (hi >= b) break;
    lo = hi + 1;
    hi = mark[hi - a];
    known = false;
  }
}

// The same pieces as split_recursive without scratch: each piece is found by
// descending the splitting tree from [a, b] towards the first bin not yet
// emitted (every decision depends only on the range and its integral, so the
// descent meets the same ranges; a right side's integral is the parent's minus
// its left side's).  Each piece costs the scans of its ancestors: for
// proto-clusters longer than the scratch the caller can give.
template <class Emit>
__host__ __device__ void split_recursive_descend(const uint32_t* N, int a, int b, uint64_t total,
                                                 const Consts& C, Emit&& emit) {
  for (int start = a; start <= b;) {
    int lo = a, hi = b;
    uint64_t integral = total;
    for (;;) {
      int m1 = -1, m2 = -1;
      uint32_t v1 = 0, v2 = 0;
      {
        int run = lo;
        uint32_t v = N[lo];
        bool left_lower = true;
        for (int i = lo + 1; i <= hi + 1; ++i) {
          const uint32_t nv = i <= hi ? N[i] : 0u;
          if (i > hi || nv != v) {
            if (left_lower && (i > hi || nv < v)) {
              if (m1 < 0 || v > v1) {
                m2 = m1; v2 = v1;
                m1 = run; v1 = v;
              } else if (m2 < 0 || v > v2) {
                m2 = run; v2 = v;
              }
            }
            left_lower = v < nv;
            run = i;
            v = nv;
          }
        }
      }
      int m = -1;
      uint64_t left = 0;
      bool split = false;
      if (m2 >= 0) {
        const int l = m1 < m2 ? m1 : m2, h = m1 < m2 ? m2 : m1;
        uint32_t vm = 0;
        for (int i = l + 1; i < h; ++i) {
          const uint32_t x = N[i];
          if (m < 0 || x < vm) { m = i; vm = x; }
        }
        const uint32_t lower = v1 < v2 ? v1 : v2;
        if (m >= 0 &&
            static_cast<uint64_t>(C.dip_den) * vm < static_cast<uint64_t>(C.dip_num) * lower) {
          const uint64_t T = (m < C.gas_bin) ? C.t_gas : C.t_pp;
          for (int i = lo; i <= m; ++i) left += N[i];
          split = left >= T && integral - left >= T;
        }
      }
      if (!split) {
        emit(lo, hi, integral, m1);
        start = hi + 1;
        break;
      }
      if (start <= m) {
        hi = m;
        integral = left;
      } else {
        lo = m + 1;
        integral -= left;
      }
    }
  }
}

// The pieces of proto-cluster [a, b] in the chosen flavour (mark: b - a + 1
// entries of scratch for the recursive split, which runs without it when
// mark is NULL; unused by the z-order walk).
template <int kSplit, class Emit>
__host__ __device__ __forceinline__ void split_pieces(const uint32_t* N, int a, int b,
                                                      uint64_t total, const Consts& C,
                                                      Emit&& emit, int16_t* mark) {
  if constexpr (kSplit == PV_SPLIT_RECURSIVE) {
    if (mark) split_recursive(N, a, b, total, C, emit, mark);
    else split_recursive_descend(N, a, b, total, C, emit);
  } else {
    split_walk(N, a, b, total, C, emit);
  }
}

// A piece is a seed cluster if it holds the minimal integral of the region of
// its maximum bin im.
__host__ __device__ __forceinline__ bool keep_piece(uint64_t integral, int im, const Consts& C) {
  uint64_t T = (im < C.gas_bin) ? C.t_gas : C.t_pp;
  return integral >= T;
}

// z_seed = z_mid(i) + delta dz, delta from the exact bin contents in binary64
// (Sec. 3.3), rounded once to binary32.  nm, ni, np = N[i-1], N[i], N[i+1]
// (0 outside the histogram).
__device__ __forceinline__ float seed_z_from(long long nm, long long ni, long long np, int i,
                                             const Consts& C) {
  long long num = np - nm;
  long long den = 2 * ni - np - nm;
  double delta = 0.0;
  if (den > 0) delta = __dmul_rn(0.5, __ddiv_rn(static_cast<double>(num), static_cast<double>(den)));
  double t1 = static_cast<double>(i) + 0.5;
  double t2 = __dmul_rn(t1, static_cast<double>(C.dz));
  double zmid = __dadd_rn(static_cast<double>(C.z_min), t2);
  double t3 = __dmul_rn(delta, static_cast<double>(C.dz));
  return __double2float_rn(__dadd_rn(zmid, t3));
}

__device__ __forceinline__ uint32_t bin_or_zero(const uint32_t* N, int j, const Consts& C) {
  return (j >= 0 && j < C.nbins) ? N[j] : 0u;
}

// Seed record pos of S: the piece [lo, hi], its maximum bin im and the bins
// around it (0 outside the histogram).  False if pos or im is out of range.
__device__ __forceinline__ bool put_seed(const uint32_t* N, const Consts& C, SeedOut* S, int pos,
                                         int lo, int hi, int im) {
  if (!PV_CHECK(pos >= 0 && pos < kMaxSeeds && im >= 0 && im < C.nbins, 4)) return false;
  S->lo[pos] = lo;
  S->hi[pos] = hi;
  S->bin[pos] = im;
  S->nm[pos] = bin_or_zero(N, im - 1, C);
  S->ni[pos] = N[im];
  S->np[pos] = bin_or_zero(N, im + 1, C);
  return true;
}

// Warp-cooperative peak search over a histogram N (shared or global).  If
// tmask is non-null only tiles (32 bins) whose bit is set can hold non-zero
// bins; otherwise every tile is scanned.  pc_lo / pc_hi are a kRunRing-entry
// ring in shared memory; mark (mark_cap int16 entries) is the recursive
// split's scratch, shared out among the proto-clusters walked at once (one
// whose share does not fit splits without scratch).  Writes up to cap seeds
// into S in z order and returns the number found (which may exceed cap).
// All 32 lanes must call it.
template <bool kSeedZ, int kSplit = PV_SPLIT_ZORDER>
__device__ __noinline__ int warp_find_seeds(const uint32_t* N, const uint32_t* tmask, const Consts& C,
                                      SeedOut* S, int cap, int16_t* pc_lo, int16_t* pc_hi,
                                      int16_t* mark = nullptr, int mark_cap = 0) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int n_seeds = 0;
  int n_starts = 0, n_ends = 0, n_done = 0;

  auto put = [&](int pos, int lo, int hi, int im) {
    if (!put_seed(N, C, S, pos, lo, hi, im)) return;
    if (kSeedZ) {
      float zs = seed_z_from(S->nm[pos], S->ni[pos], S->np[pos], im, C);
      S->z[pos] = zs;
      S->x[pos] = __fadd_rn(C.x_b, __fmul_rn(C.tx_b, zs));
      S->y[pos] = __fadd_rn(C.y_b, __fmul_rn(C.ty_b, zs));
    }
  };
  auto process = [&](int count) {
    // lane j walks proto-cluster n_done + j, counting the kept pieces and
    // keeping the first two; only a lane with three or more walks again
    int a = 0, b = -1;
    uint64_t total = 0;
    if (lane < count) {
      a = pc_lo[(n_done + lane) & (kRunRing - 1)];
      b = pc_hi[(n_done + lane) & (kRunRing - 1)];
      // (a run's bounds always lie in the histogram; the test keeps a broken
      // invariant from reading outside it)
      if (!(a >= 0 && a <= b && b < C.nbins)) {
        (void)PV_CHECK(false, 17);
        b = a - 1;
      }
      for (int i = a; i <= b; ++i) total += N[i];
    }
    // no piece of a proto-cluster can hold more than its total integral, so
    // one below the smaller threshold yields no seed: skip its walk
    const uint64_t t_min = C.t_pp < C.t_gas ? C.t_pp : C.t_gas;
    const bool walk = lane < count && total >= t_min;
    // each walked proto-cluster's share of the scratch (recursive split)
    int16_t* lane_mark = nullptr;
    if constexpr (kSplit == PV_SPLIT_RECURSIVE) {
      const int len = walk ? b - a + 1 : 0;
      int end = len;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, end, o);
        if (lane >= o) end += v;
      }
      if (walk && mark && end <= mark_cap) lane_mark = mark + (end - len);
    }
    int kept = 0, lo1 = 0, hi1 = 0, im1 = 0;
    int lo2 = 0, hi2 = 0, im2 = 0;
    if (walk) {
      split_pieces<kSplit>(N, a, b, total, C, [&](int lo, int hi, uint64_t integral, int im) {
        if (keep_piece(integral, im, C)) {
          if (kept == 0) {
            lo1 = lo; hi1 = hi; im1 = im;
          } else if (kept == 1) {
            lo2 = lo; hi2 = hi; im2 = im;
          }
          ++kept;
        }
      }, lane_mark);
    }
    int incl = kept;
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    int n_kept = __shfl_sync(0xffffffffu, incl, 31);
    int pos = n_seeds + incl - kept;
    if (kept >= 1 && kept <= 2 && pos < cap) {
      put(pos, lo1, hi1, im1);
      if (kept == 2 && pos + 1 < cap) put(pos + 1, lo2, hi2, im2);
    }
    if (kept > 2 && pos < cap) {
      split_pieces<kSplit>(N, a, b, total, C, [&](int lo, int hi, uint64_t integral, int im) {
        if (keep_piece(integral, im, C)) {
          if (pos < cap) put(pos, lo, hi, im);
          ++pos;
        }
      }, lane_mark);
    }
    n_seeds += n_kept;
    n_done += count;
    __syncwarp();
  };

  // one tile: the starts and ends of the runs of bins above the threshold
  // (the bins next to the tile come from the adjacent tiles)
  auto scan_tile = [&](int q) {
    const int bin = q * 32 + lane;
    const uint32_t v = (bin < C.nbins) ? N[bin] : 0u;
    const unsigned A = __ballot_sync(0xffffffffu, v > C.thr);
    if (A == 0u) return;
    const int bp = q * 32 - 1, bn = q * 32 + 32;
    const unsigned pa = (bp >= 0 && bp < C.nbins && N[bp] > C.thr) ? 1u : 0u;
    const unsigned na = (bn < C.nbins && N[bn] > C.thr) ? 0x80000000u : 0u;
    const unsigned starts = A & ~((A << 1) | pa);
    const unsigned ends = A & ~((A >> 1) | na);
    if (starts & (1u << lane))
      pc_lo[(n_starts + __popc(starts & lt)) & (kRunRing - 1)] = static_cast<int16_t>(bin);
    if (ends & (1u << lane))
      pc_hi[(n_ends + __popc(ends & lt)) & (kRunRing - 1)] = static_cast<int16_t>(bin);
    n_starts += __popc(starts);
    n_ends += __popc(ends);
    __syncwarp();
    while (n_ends - n_done >= 32) process(32);
  };

  for (int w = 0; w < (C.ntiles + 31) / 32; ++w) {
    uint32_t m;
    if (tmask) {
      m = tmask[w];
    } else {
      int left = C.ntiles - 32 * w;
      m = left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
    }
    while (m) {
      const int tb = __ffs(m) - 1;
      m &= m - 1;
      scan_tile(w * 32 + tb);
    }
  }
  if (n_ends - n_done > 0) process(n_ends - n_done);
  return n_seeds;
}

// ---------------------------------------------------------------------------
// step (d1): association with the removal loop, block-cooperative.
//
// center[t]: center bin or -1; cid[t] receives the index among the surviving
// seeds (z order) or -1.  S holds K seeds on entry and the survivors,
// compacted in z order, on exit.  cnt receives the tracks per survivor.
// Scratch arrays alive/part live in shared memory.  Returns the survivors.
template <typename CenterT, typename CidT>
__device__ int block_associate(const CenterT* center, CidT* cid, int n, SeedOut* S, int K,
                               const Consts& C, int* alive, int* part, int* cnt, int* flag) {
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  if (tid < K) alive[tid] = tid;
  __shared__ int s_ka;
  if (tid == 0) s_ka = K;
  __syncthreads();
  for (;;) {
    int ka = s_ka;
    if (tid + 1 < ka && PV_CHECK(ka <= kMaxSeeds, 5))
      part[tid] = (S->hi[alive[tid]] + S->lo[alive[tid + 1]]) >> 1;
    if (tid < ka) cnt[tid] = 0;
    __syncthreads();
    for (int t = tid; t < n; t += nt) {
      int c = static_cast<int>(center[t]);
      int q = -1;
      if (c >= 0 && ka > 0) {
        int lo = 0, hi = ka - 1;        // number of partition points < c
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (part[mid] < c) lo = mid + 1; else hi = mid;
        }
        q = lo;
        atomicAdd(cnt + q, 1);
      }
      cid[t] = static_cast<CidT>(q);
    }
    __syncthreads();
    if (tid < 32) {
      // fewest tracks among clusters below their threshold, lowest z on ties
      long long best = 0x7fffffffffffffffLL;
      for (int q = tid; q < ka; q += 32) {
        int gas = S->bin[alive[q]] < C.gas_bin;
        int need = gas ? C.min_assoc_gas : C.min_assoc_pp;
        if (cnt[q] < need) {
          long long key = (static_cast<long long>(cnt[q]) << 8) | q;
          best = key < best ? key : best;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v < best ? v : best;
      }
      if (tid == 0) {
        if (best == 0x7fffffffffffffffLL) {
          *flag = 0;
        } else {
          int q = static_cast<int>(best & 0xff);
          for (int r = q; r + 1 < ka; ++r) alive[r] = alive[r + 1];
          s_ka = ka - 1;
          *flag = 1;
        }
      }
    }
    __syncthreads();
    if (!*flag) break;
  }
  int ka = s_ka;
  // compact survivors in z order.  alive is increasing (alive[q] >= q), so
  // the first 32 survivors can be moved once all of them are read, and the
  // rest only read entries at or above 32, which the first half leaves alone.
  if (tid < 32) {
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int q = tid + 32 * h;
      int lo = 0, hi = 0, bn = 0;
      float z = 0.f, x = 0.f, y = 0.f;
      uint32_t nm = 0, ni = 0, np = 0;
      if (q < ka) {
        const int k = alive[q];
        lo = S->lo[k]; hi = S->hi[k]; bn = S->bin[k];
        z = S->z[k]; x = S->x[k]; y = S->y[k];
        nm = S->nm[k]; ni = S->ni[k]; np = S->np[k];
      }
      __syncwarp();
      if (q < ka) {
        S->lo[q] = lo; S->hi[q] = hi; S->bin[q] = bn;
        S->z[q] = z; S->x[q] = x; S->y[q] = y;
        S->nm[q] = nm; S->ni[q] = ni; S->np[q] = np;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  return ka;
}

// ---------------------------------------------------------------------------
// step (d2): per-track fit inputs relative to the seed, and the group fit

struct FitTrack {            // 24 bytes: position at z_seed relative to the seed, slopes, weights
  float X, Y, tx, ty;
  float wx, wy;              // 1/V_xx, 1/V_yy at z_seed; 0 marks an unusable track
};

__device__ __forceinline__ void make_fit_track(float x, float y, float z, float tx, float ty,
                                               float cxx, float cxtx, float ctxtx,
                                               float cyy, float cyty, float ctyty,
                                               float xs, float ys, float zs,
                                               float4* A, float2* W) {
  float d = zs - z;
  float vxx = cxx + 2.0f * d * cxtx + d * d * ctxtx;
  float vyy = cyy + 2.0f * d * cyty + d * d * ctyty;
  float X = x + d * tx - xs;
  float Y = y + d * ty - ys;
  bool ok = (vxx > 0.0f) && (vyy > 0.0f) && isfinite(vxx) && isfinite(vyy) && isfinite(X) &&
            isfinite(Y) && isfinite(tx) && isfinite(ty);
  if (ok) {
    *A = make_float4(X, Y, tx, ty);
    *W = make_float2(1.0f / vxx, 1.0f / vyy);
  } else {
    *A = make_float4(0.f, 0.f, 0.f, 0.f);
    *W = make_float2(0.f, 0.f);
  }
}

struct VertexOut {
  float x, y, z;
  float cov[6];
  float chi2, ndof;
  int n_tracks, n_iter, status;
};

// Sum over the 8 lanes of a group (xor tree; identical on all 8 lanes).
__device__ __forceinline__ float group_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}
__device__ __forceinline__ double group_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}
__device__ __forceinline__ float group_max(float v) {
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 4));
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 2));
  v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
  return v;
}
__device__ __forceinline__ int group_sum_i(int v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// Error-free transformation: s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// Compensated accumulation (Kahan-Babuska-Neumaier style with TwoSum).
struct CSum {
  float hi, lo;
  __device__ __forceinline__ void add(float v) {
    float s, e;
    two_sum(hi, v, s, e);
    hi = s;
    lo += e;
  }
  __device__ __forceinline__ float value() const { return hi + lo; }
};
__device__ __forceinline__ float group_sum_c(CSum v) {
  // reduce (hi, lo) pairs with TwoSum at every level
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    float oh = __shfl_xor_sync(0xffffffffu, v.hi, o);
    float ol = __shfl_xor_sync(0xffffffffu, v.lo, o);
    float s, e;
    two_sum(v.hi, oh, s, e);
    v.hi = s;
    v.lo = v.lo + ol + e;
  }
  return v.hi + v.lo;
}

// Fit of one vertex per 8-lane group.  Every lane of the warp must call it
// (shuffles); lanes of groups without a vertex pass cntk = -1.  Track s of the
// vertex (s = 0 .. cntk-1, in track-index order) is handled by lane s mod 8 of
// the group, which finds its j-th track (s = r + 8 j) at A[j * stride],
// W[j * stride] (the lane's own fit inputs: in global memory in vertex order,
// or in the lane's shared-memory slots).  The result lands in *out on every
// lane of the group.
//
// Each iteration solves the normal equations in sheared coordinates
// x' = x - c_x z, y' = y - c_y z, with c the weighted mean slope of the
// vertex's tracks (weights W for the first iteration, w W of the previous
// iteration afterwards).  The equations keep their structure (the sums use
// t - c instead of t) and the z pivot s = M_zz - M_xz^2/M_xx - M_yz^2/M_yy,
// which the shear leaves unchanged, no longer cancels in binary32 when the
// weighted tracks are nearly parallel.  Step and covariance are mapped back
// with T = [[1,0,c_x],[0,1,c_y],[0,0,1]] (x = x' + c_x z, C = T C' T^T).
template <int kAccum>
__device__ void group_fit(const float4* A, const float2* W, int stride, int cntk,
                          const Consts& C, VertexOut* out) {
  // binary32 per-track terms; sums and solve in binary32 (FP32), compensated
  // binary32 (KAHAN) or binary64 (FP64)
  using T = typename std::conditional<kAccum == PV_ACCUM_FP64, double, float>::type;
  const int r = threadIdx.x & (kGroup - 1);
  // first shear: W-weighted mean slope of the usable tracks
  float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
  for (int s = r, q = 0; s < cntk; s += kGroup, q += stride) {
    float4 a = A[q];
    float2 w2 = W[q];
    if (!(w2.x > 0.0f)) continue;
    m0 += w2.x; m1 += w2.x * a.z; m2 += w2.y; m3 += w2.y * a.w;
  }
  m0 = group_sum(m0); m1 = group_sum(m1); m2 = group_sum(m2); m3 = group_sum(m3);
  T cx = m0 > 0.f ? static_cast<T>(m1 / m0) : T(0);
  T cy = m2 > 0.f ? static_cast<T>(m3 / m2) : T(0);
  T ax = 0, ay = 0, az = 0;           // relative to the seed
  bool done = cntk < 0;
  int status = 0, n_iter = 0;
  T c2sum = 0, sw = 0, dchi2 = 0;
  T ix = 0, iy = 0, ux = 0, uy = 0, is = 0;
  int nw = 0;
  for (int it = 1; it <= C.max_iter; ++it) {
    T v[10];
    int cnt_w = 0;
    const float axp = static_cast<float>(ax - cx * az), ayp = static_cast<float>(ay - cy * az);
    const float fcx = static_cast<float>(cx), fcy = static_cast<float>(cy);
    const float faz = static_cast<float>(az);
    if (kAccum == PV_ACCUM_KAHAN) {
      CSum acc[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) acc[q] = CSum{0.f, 0.f};
      if (!done) {
        for (int s = r, q = 0; s < cntk; s += kGroup, q += stride) {
          float4 a = A[q];
          float2 w2 = W[q];
          if (!(w2.x > 0.0f)) continue;
          float dtx = a.z - fcx, dty = a.w - fcy;
          float rx = a.x + faz * dtx - axp;
          float ry = a.y + faz * dty - ayp;
          float c2 = rx * rx * w2.x + ry * ry * w2.y;
          float w = 0.f;
          if (c2 < C.chi2_max) { float f = 1.0f - c2 * C.inv_chi2_max; w = f * f; }
          if (w > 0.f) {
            float wx = w * w2.x, wy = w * w2.y;
            acc[0].add(wx); acc[1].add(wy);
            acc[2].add(wx * dtx); acc[3].add(wy * dty);
            acc[4].add(wx * dtx * dtx + wy * dty * dty);
            acc[5].add(wx * rx); acc[6].add(wy * ry);
            acc[7].add(wx * dtx * rx + wy * dty * ry);
            acc[8].add(w * c2); acc[9].add(w);
            ++cnt_w;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 10; ++q) v[q] = group_sum_c(acc[q]);
    } else {
#pragma unroll
      for (int q = 0; q < 10; ++q) v[q] = T(0);
      if (!done) {
        for (int s = r, q = 0; s < cntk; s += kGroup, q += stride) {
          float4 a = A[q];
          float2 w2 = W[q];
          if (!(w2.x > 0.0f)) continue;
          float dtx = a.z - fcx, dty = a.w - fcy;
          float rx = a.x + faz * dtx - axp;
          float ry = a.y + faz * dty - ayp;
          float c2 = rx * rx * w2.x + ry * ry * w2.y;
          float w = 0.f;
          if (c2 < C.chi2_max) { float f = 1.0f - c2 * C.inv_chi2_max; w = f * f; }
          if (w > 0.f) {
            float wx = w * w2.x, wy = w * w2.y;
            v[0] += T(wx); v[1] += T(wy);
            v[2] += T(wx * dtx); v[3] += T(wy * dty);
            v[4] += T(wx * dtx * dtx + wy * dty * dty);
            v[5] += T(wx * rx); v[6] += T(wy * ry);
            v[7] += T(wx * dtx * rx + wy * dty * ry);
            v[8] += T(w * c2); v[9] += T(w);
            ++cnt_w;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 10; ++q) v[q] = group_sum(v[q]);
    }
    cnt_w = group_sum_i(cnt_w);
    if (!done) {
      // sheared M = [[Sxx,0,-Sxz],[0,Syy,-Syz],[-Sxz,-Syz,Szz]], rhs (bx, by, -bz)
      T sxx = v[0], syy = v[1], sxz = v[2], syz = v[3], szz = v[4];
      T bx = v[5], by = v[6], bz = v[7];
      n_iter = it;
      c2sum = v[8]; sw = v[9]; nw = cnt_w;
      T s_ = 0;
      bool ok = sxx > T(0) && syy > T(0) && isfinite(sxx) && isfinite(syy);
      if (ok) {
        ix = T(1) / sxx;
        iy = T(1) / syy;
        ux = sxz * ix;
        uy = syz * iy;
        s_ = szz - sxz * ux - syz * uy;      // Schur complement: the z pivot
        // M_zz of the unsheared matrix, for the relative pivot test
        T mzz = szz + T(2) * (cx * sxz + cy * syz) + cx * cx * sxx + cy * cy * syy;
        ok = s_ > T(kPivotRel) * mzz && isfinite(s_);
      }
      if (!ok) {
        status = PV_ST_SINGULAR;
        dchi2 = 0;
        done = true;
      } else {
        is = T(1) / s_;
        T dz = (ux * bx + uy * by - bz) * is;
        T dx = (bx + sxz * dz) * ix;
        T dy = (by + syz * dz) * iy;
        dchi2 = -bx * dx - by * dy + bz * dz;
        ax += dx + cx * dz;
        ay += dy + cy * dz;
        az += dz;
        // covariance terms in the unsheared frame; the next shear is the
        // w W-weighted mean slope of this iteration, ux + c_x
        ux += cx;
        uy += cy;
        cx = ux;
        cy = uy;
        const T adchi2 = dchi2 < T(0) ? -dchi2 : dchi2, adz = dz < T(0) ? -dz : dz;
        if (adchi2 < static_cast<T>(C.dchi2_tol) && adz < static_cast<T>(C.dz_tol)) {
          status = PV_ST_CONVERGED;
          done = true;
        } else if (it == C.max_iter) {
          status = PV_ST_MAXITER;
        }
      }
    }
    if (__all_sync(0xffffffffu, done)) break;
  }
  if (cntk < 0) return;
  // C = T C' T^T with ux, uy already mapped back (M_xz/M_xx of the unsheared M)
  const T uxo = ux, uyo = uy;
  out->x = static_cast<float>(ax);   // relative to the seed; the caller adds the seed position
  out->y = static_cast<float>(ay);
  out->z = static_cast<float>(az);
  out->cov[0] = static_cast<float>(ix + uxo * uxo * is);   // xx
  out->cov[1] = static_cast<float>(uxo * uyo * is);        // xy
  out->cov[2] = static_cast<float>(iy + uyo * uyo * is);   // yy
  out->cov[3] = static_cast<float>(uxo * is);              // xz
  out->cov[4] = static_cast<float>(uyo * is);              // yz
  out->cov[5] = static_cast<float>(is);                    // zz
  out->chi2 = static_cast<float>(c2sum + dchi2);
  out->ndof = static_cast<float>(T(2) * sw - T(3));
  out->n_tracks = nw;
  out->n_iter = n_iter;
  out->status = status == 0 ? PV_ST_MAXITER : status;
}

// Final selection (Sec. 3.5): pp vertices farther than max_r_beam from the
// beamline and vertices with too few tracks are flagged; the rest accepted.
__device__ __forceinline__ int select_vertex(float x, float y, float z, int n_tracks, int status,
                                             const Consts& C) {
  if (status & PV_ST_SINGULAR) return status;
  bool gas = z < C.z_gas;
  if (!gas) {
    float bx = C.x_b + C.tx_b * z, by = C.y_b + C.ty_b * z;
    float r = sqrtf((x - bx) * (x - bx) + (y - by) * (y - by));
    if (r > C.max_r_beam) status |= PV_ST_REJ_BEAM;
  }
  int need = gas ? C.min_pv_gas : C.min_pv_pp;
  if (n_tracks < need) status |= PV_ST_REJ_NTRK;
  if (!(status & (PV_ST_REJ_BEAM | PV_ST_REJ_NTRK))) status |= PV_ST_ACCEPTED;
  return status;
}

}  // namespace pvdev
