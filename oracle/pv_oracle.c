/*
 * pv_oracle.c -- plain, slow CPU oracle for primary-vertex finding and fitting,
 * following Dziurda et al., "A parallel algorithm for fast reconstruction of
 * primary vertices on heterogeneous architectures" (arXiv:2412.14966), Sec. 3.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load this library.  It shares no code, header or table
 * with the CUDA library; the two are compared on the same seeded inputs.
 *
 * Two precisions:
 *   - steps (a)-(c) (extrapolation, histogram, peak search, association) are
 *     written as a pinned IEEE binary32 operation sequence ("contract mode"):
 *     every + - * / sqrt rounds once, in the order written, with no fused
 *     multiply-add (build with -ffp-contract=off).  Histogram weights are
 *     integers, so bins, seeds and track assignments are exact results.
 *     A binary64 version of step (a) exists only to report the binary32 error.
 *   - step (d) (the adaptive vertex fit and the final selection) is binary64
 *     throughout and uses general 3x3 matrix algebra.
 *
 * Readings of points where the paper is silent or garbled:
 *   R1 beam position at the track's z in Eq. zpocadef (x_b is defined at z=0).
 *   R2 Eq. Vxy: only the diagonal x and y blocks are used (x and y independent,
 *      Sec. 3.1); sigma_poca uses V_xx extrapolated to z_poca.
 *   R3 histogram profile: the cubic CDF of the variance-matched Epanechnikov
 *      kernel, F(u) = 1/2 + u (3/4 - u^2/4) on [-1, 1], s = sqrt(5) sigma,
 *      quantised to integers with ONE = 4096 per track.
 *   R4 proto-cluster threshold strict ">" an integer bin_threshold.
 *   R5 dip splitting in z order with integer significance and integral tests.
 *   R6 association: one cluster removed per pass (fewest tracks, lowest z).
 *   R7 fit: M = sum w H^T W H, g = sum w H^T W r, step -M^{-1} g,
 *      C = M^{-1}, dchi2 = g . step, chi2 = sum w chi2_i + dchi2.
 *   R8 final track count = tracks with w > 0 in the last iteration.
 *   R9 seed position: delta and z_seed in binary64 from the exact integer bin
 *      contents, rounded once to binary32; delta = 0 when 2N_i - N_+ - N_- <= 0.
 *   R10 the fit uses a track only if its state is finite and both variances
 *      extrapolated to the seed z are finite and positive.
 *   R11 the normal matrix counts as singular when a Gauss-Jordan pivot is not
 *      above OC_PIVOT_REL times its diagonal element (for example a single
 *      weighted track, or tracks that are all parallel): the vertex gets the
 *      SINGULAR status instead of a step along an undetermined direction.
 *   R16 the x86 dip splitting (split_mode 1): the smallest bin between the two
 *      largest maxima, with the significance and integral tests of R5, applied
 *      recursively to both sides (see oc_split_recursive).
 *   R17 the x86 profile (profile_mode 1): a track adds the template of its
 *      sigma_poca class, centred on the bin of its z_poca.  Class k has
 *      sigma_k = 0.01 mm * 2^(k/4), k = 0 .. 40, and holds the sigma_poca from
 *      sigma_{k-1} 2^(1/8) up; its template is the exact Gaussian integral over
 *      each bin for a mean at the bin centre, quantised like R3 (see oc_tpl_build).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OC_ONE 4096          /* histogram weight of one track, R3 */
#define OC_S_MIN 1e-6f       /* profile half-width below which a track fills one bin */
#define OC_PIVOT_REL 1e-4    /* relative pivot below which M is singular, R11 */

enum {
  OC_CONVERGED = 1, OC_MAXITER = 2, OC_SINGULAR = 4,
  OC_REJ_BEAM = 8, OC_REJ_NTRK = 16, OC_ACCEPTED = 32
};
enum { OC_EV_SEED_OVERFLOW = 1 };

typedef struct {
  /* histogram range and bin width, Sec. 3.2 */
  float z_min, z_max, dz;
  /* boundary of the gas-cell region, Table smog-pp */
  float z_gas;
  /* maximal sigma_poca for filling, Sec. 3.2 */
  float sigma_max_pp, sigma_max_gas;
  /* minimal cluster integral in tracks, Table smog-pp */
  float min_integral_pp, min_integral_gas;
  /* proto-cluster bin threshold in 1/ONE track units, R4 */
  uint32_t bin_threshold;
  /* significant dip: dip_den * N_min < dip_num * min(N_left, N_right), R5 */
  int32_t dip_num, dip_den;
  /* minimal tracks per cluster in the association loop, Sec. 3.4 */
  int32_t min_assoc_pp, min_assoc_gas;
  /* minimal tracks with w > 0 in a final PV, Table smog-pp */
  int32_t min_pv_tracks_pp, min_pv_tracks_gas;
  /* fit, Sec. 3.5 */
  double chi2_max, dchi2_tol, dz_tol;
  int32_t max_iter;
  /* final transverse distance cut for pp vertices, Sec. 3.5 */
  double max_r_beam;
  int32_t max_seeds;
  /* beamline at z = 0 and its slopes, Sec. 3 */
  float x_b, y_b, tx_b, ty_b;
  /* dip splitting: 0 in z order (GPU flavour, R5), 1 recursive (x86, R16) */
  int32_t split_mode;
  /* profile: 0 cubic CDF (GPU flavour, R3), 1 templates chosen by sigma (x86, R17) */
  int32_t profile_mode;
} oc_params;

/* ------------------------------------------------------------------------- */
/* histogram geometry (binary32)                                             */

static int oc_nbins(const oc_params* p) {
  return (int)floor(((double)p->z_max - (double)p->z_min) / (double)p->dz + 0.5);
}

/* bin index of v: floor((v - z_min) / dz); -1 below the range, nbins above. */
static int oc_bin_f32(float v, const oc_params* p, int nbins) {
  float q = (v - p->z_min) / p->dz;
  if (!(q >= 0.0f)) return -1;
  if (q >= (float)nbins) return nbins;
  return (int)q;
}

/* lower edge of bin j */
static float oc_edge_f32(int j, const oc_params* p) {
  float fj = (float)j;
  float w = fj * p->dz;
  return p->z_min + w;
}

/* ------------------------------------------------------------------------- */
/* step (a): extrapolation to the beamline, Eq. zpocadef, Eq. Vxy, sigma_poca */

typedef struct {
  float zpoca, sigma;
  int32_t center, j0, j1, filled;
  int32_t tcls;                                    /* template class (R17), else -1 */
} oc_prep32;

/* ------------------------------------------------------------------------- */
/* template profiles of the x86 flavour, Sec. 3.2, reading R17               */

#define OC_TPL_CLASSES 41
#define OC_TPL_SIGMA0 0.01                      /* mm: sigma of class 0 */
#define OC_TPL_RATIO 1.189207115002721          /* 2^(1/4) between classes */
#define OC_TPL_HALF_RATIO 1.0905077326652577    /* 2^(1/8): class boundaries */
#define OC_TPL_MAX_HALF 1024

typedef struct {
  double sigma[OC_TPL_CLASSES];   /* sigma_k */
  double bound[OC_TPL_CLASSES];   /* lowest sigma_poca of class k (bound[0] = 0) */
  int32_t half[OC_TPL_CLASSES];   /* H_k: the template covers bins c - H_k .. c + H_k */
  int32_t first[OC_TPL_CLASSES];  /* where class k's cumulative values start in q */
  int32_t* q;                     /* Q_k[i], i = 0 .. 2 H_k + 1, at edge (i - H_k - 1/2) dz */
} oc_tpl;

/* standard normal CDF */
static double oc_phi(double x) { return 0.5 * erfc(-x * 0.70710678118654752440); }

/* rint(ONE * Phi) at the edge (i - H - 1/2) dz from the centre of the bin */
static long oc_tpl_q(int i, int H, double dz, double s) {
  double x = ((double)(i - H) - 0.5) * dz / s;
  return lrint((double)OC_ONE * oc_phi(x));
}

/* The templates: H_k is the smallest H whose outer edge holds a quantised
 * CDF of 0; Q_k[0] = 0, Q_k[2 H_k + 1] = ONE and the interior edges hold the
 * quantised Gaussian CDF, made non-decreasing.  Returns 0, -1 on failure. */
static int oc_tpl_build(const oc_params* p, oc_tpl* t) {
  double dz = (double)p->dz;
  double s = OC_TPL_SIGMA0;
  int total = 0;
  for (int k = 0; k < OC_TPL_CLASSES; ++k) {
    if (k > 0) {
      t->bound[k] = s * OC_TPL_HALF_RATIO;
      s = s * OC_TPL_RATIO;
    } else {
      t->bound[k] = 0.0;
    }
    t->sigma[k] = s;
    int H = 0;
    while (H < OC_TPL_MAX_HALF && oc_tpl_q(0, H, dz, s) != 0) H++;
    t->half[k] = H;
    t->first[k] = total;
    total += 2 * H + 2;
  }
  t->q = (int32_t*)malloc(sizeof(int32_t) * (size_t)total);
  if (!t->q) return -1;
  for (int k = 0; k < OC_TPL_CLASSES; ++k) {
    int H = t->half[k];
    int32_t* q = t->q + t->first[k];
    q[0] = 0;
    for (int i = 1; i <= 2 * H; ++i) {
      long v = oc_tpl_q(i, H, dz, t->sigma[k]);
      if (v < 0) v = 0;
      if (v > OC_ONE) v = OC_ONE;
      if (v < q[i - 1]) v = q[i - 1];
      q[i] = (int32_t)v;
    }
    q[2 * H + 1] = OC_ONE;
  }
  return 0;
}

static void oc_tpl_free(oc_tpl* t) { free(t->q); t->q = NULL; }

/* class of sigma_poca: the last class whose lower bound it reaches */
static int oc_tpl_class(float sigma, const oc_tpl* t) {
  int k = 0;
  for (int j = 1; j < OC_TPL_CLASSES; ++j)
    if ((double)sigma >= t->bound[j]) k = j;
  return k;
}

static void oc_prepare_f32(float x, float y, float z, float tx, float ty,
                           float cxx, float cxtx, float ctxtx,
                           const oc_params* p, const oc_tpl* tpl, int nbins, oc_prep32* out) {
  /* slopes relative to the beam */
  float dtx = tx - p->tx_b;
  float dty = ty - p->ty_b;
  float t2 = dtx * dtx + dty * dty;
  /* beam position at the track's z (R1) */
  float xb = p->x_b + p->tx_b * z;
  float yb = p->y_b + p->ty_b * z;
  float num = dtx * (xb - x) + dty * (yb - y);
  float zp = z + num / t2;
  /* V_xx extrapolated to z_poca (Eq. Vxy, diagonal block, R2) */
  float d = zp - z;
  float vxx = cxx + (2.0f * d) * cxtx + (d * d) * ctxtx;
  float sig = sqrtf(vxx / t2);
  out->zpoca = zp;
  out->sigma = sig;
  out->filled = 0;
  out->center = -1;
  out->j0 = 0;
  out->j1 = -1;
  out->tcls = -1;
  if (!(t2 > 0.0f)) return;
  if (!isfinite(zp) || !isfinite(sig)) return;
  int c = oc_bin_f32(zp, p, nbins);
  if (c < 0 || c >= nbins) return;
  float smax = (zp < p->z_gas) ? p->sigma_max_gas : p->sigma_max_pp;
  if (!(sig <= smax)) return;
  out->filled = 1;
  out->center = c;
  if (tpl) {                                       /* R17 */
    int k = oc_tpl_class(sig, tpl);
    out->tcls = k;
    out->j0 = c - tpl->half[k];
    out->j1 = c + tpl->half[k];
    return;
  }
  float s = 2.23606797749979f * sig;
  if (s < OC_S_MIN) s = 0.0f;
  out->j0 = oc_bin_f32(zp - s, p, nbins);
  out->j1 = oc_bin_f32(zp + s, p, nbins);
}

/* binary64 z_poca and sigma_poca of the same formulas, for error reports only */
static void oc_prepare_f64(double x, double y, double z, double tx, double ty,
                           double cxx, double cxtx, double ctxtx,
                           const oc_params* p, double* zpoca, double* sigma) {
  double dtx = tx - (double)p->tx_b, dty = ty - (double)p->ty_b;
  double t2 = dtx * dtx + dty * dty;
  double xb = (double)p->x_b + (double)p->tx_b * z;
  double yb = (double)p->y_b + (double)p->ty_b * z;
  double zp = z + (dtx * (xb - x) + dty * (yb - y)) / t2;
  double d = zp - z;
  double vxx = cxx + 2.0 * d * cxtx + d * d * ctxtx;
  *zpoca = zp;
  *sigma = sqrt(vxx / t2);
}

/* ------------------------------------------------------------------------- */
/* step (b): resolution-weighted profile, Sec. 3.2, reading R3               */

/* quantised cumulative weight at normalised distance u = (edge - z_poca) / s */
static int32_t oc_quant_cdf(float u) {
  if (!(u > -1.0f)) return 0;
  if (u >= 1.0f) return OC_ONE;
  float a = u * u;
  float b = 0.25f * a;
  float c = 0.75f - b;
  float d = u * c;
  float F = 0.5f + d;
  long q = lrintf(F * (float)OC_ONE);
  if (q < 0) q = 0;
  if (q > OC_ONE) q = OC_ONE;
  return (int32_t)q;
}

/* Per-bin integer weights of one filled track.  weights[k] belongs to bin
 * j0 + k, k = 0 .. j1 - j0.  Bins outside [0, nbins) are included here with
 * their weight; the caller drops them.  Returns the number of bins. */
static int oc_profile_weights(const oc_prep32* t, const oc_params* p, const oc_tpl* tpl,
                              uint32_t* weights, int cap) {
  if (tpl) {                                       /* R17: the class template */
    const int32_t* q = tpl->q + tpl->first[t->tcls];
    int n = 2 * tpl->half[t->tcls] + 1;
    if (n > cap) return -1;
    for (int i = 0; i < n; ++i) weights[i] = (uint32_t)(q[i + 1] - q[i]);
    return n;
  }
  float s = 2.23606797749979f * t->sigma;
  if (s < OC_S_MIN) s = 0.0f;
  float inv_s = (s > 0.0f) ? 1.0f / s : 0.0f;
  int n = t->j1 - t->j0 + 1;
  if (n > cap) return -1;
  int32_t qprev = 0;
  for (int j = t->j0; j <= t->j1; ++j) {
    int32_t qnext;
    if (j == t->j1) {
      qnext = OC_ONE;
    } else {
      float e = oc_edge_f32(j + 1, p);
      float u = (e - t->zpoca) * inv_s;
      qnext = oc_quant_cdf(u);
    }
    if (qnext < qprev) qnext = qprev;
    weights[j - t->j0] = (uint32_t)(qnext - qprev);
    qprev = qnext;
  }
  return n;
}

/* ------------------------------------------------------------------------- */
/* step (c): proto-clusters, dip splitting and seeds, Sec. 3.3               */

typedef struct { int32_t lo, hi; } oc_range;

static uint64_t oc_sum(const uint32_t* N, int lo, int hi) {
  uint64_t s = 0;
  for (int i = lo; i <= hi; ++i) s += N[i];
  return s;
}

static int oc_is_gas_bin(int bin, int gas_bin) { return bin < gas_bin; }

static uint64_t oc_min_integral(int gas, const oc_params* p) {
  double v = (double)(gas ? p->min_integral_gas : p->min_integral_pp) * (double)OC_ONE;
  return (uint64_t)llround(v);
}

static int oc_argmax(const uint32_t* N, int lo, int hi) {
  int best = lo;
  for (int i = lo + 1; i <= hi; ++i)
    if (N[i] > N[best]) best = i;
  return best;
}

/* Split proto-cluster [a, b] at significant minima, walking in z order (the
 * GPU variant of Sec. 3.3, reading R5).  Appends pieces to out; returns count. */
static int oc_split(const uint32_t* N, int a, int b, const oc_params* p, int gas_bin,
                    oc_range* out, int cap) {
  int n = 0;
  int s = a;
  int top = a;
  while (top < b && N[top + 1] >= N[top]) top++;   /* first maximum */
  uint64_t L = N[top];                             /* largest value of the open piece */
  while (top < b) {
    int j = top, m = top;
    while (j < b && N[j + 1] <= N[j]) {            /* go down to the minimum */
      j++;
      if (N[j] < N[j - 1]) m = j;                  /* leftmost bin of the lowest plateau */
    }
    if (j == b) break;                             /* no maximum after it */
    int k = j;
    while (k < b && N[k + 1] >= N[k]) k++;         /* up to the next maximum */
    uint64_t R = N[k];
    uint64_t lower = L < R ? L : R;
    int split = 0;
    if ((uint64_t)p->dip_den * (uint64_t)N[m] < (uint64_t)p->dip_num * lower) {
      uint64_t T = oc_min_integral(oc_is_gas_bin(m, gas_bin), p);
      if (oc_sum(N, s, m) >= T && oc_sum(N, m + 1, b) >= T) split = 1;
    }
    if (split) {
      if (n < cap) { out[n].lo = s; out[n].hi = m; }
      n++;
      s = m + 1;
      L = R;
    } else if (R > L) {
      L = R;
    }
    top = k;
  }
  if (n < cap) { out[n].lo = s; out[n].hi = b; }
  n++;
  return n;
}

/* A maximum of N on [a, b]: a maximal run of equal bins higher than the bins
 * next to it inside [a, b] (the ends count as lower); its position is the
 * run's first bin. */
static int oc_is_max_start(const uint32_t* N, int a, int b, int i, int* end) {
  if (i > a && N[i - 1] >= N[i]) return 0;          /* not the run's first bin, or lower */
  int q = i;
  while (q < b && N[q + 1] == N[i]) q++;
  *end = q;
  return q == b || N[q + 1] < N[i];
}

/* Recursive dip splitting (the x86 variant of Sec. 3.3, reading R16): the two
 * largest maxima of [a, b] (lower position first on equal values), the
 * smallest bin strictly between them (leftmost on ties); split there (the
 * minimum goes left) if it is significant against the smaller of the two
 * maxima and both sides hold the minimal integral, then split both sides the
 * same way; otherwise [a, b] is one piece. */
static int oc_split_recursive(const uint32_t* N, int a, int b, const oc_params* p, int gas_bin,
                              oc_range* out, int cap, int n) {
  int m1 = -1, m2 = -1;                            /* positions of the two largest maxima */
  for (int i = a; i <= b; ++i) {
    int end;
    if (!oc_is_max_start(N, a, b, i, &end)) continue;
    if (m1 < 0 || N[i] > N[m1]) { m2 = m1; m1 = i; }
    else if (m2 < 0 || N[i] > N[m2]) m2 = i;
    i = end;
  }
  if (m2 >= 0) {
    int lo = m1 < m2 ? m1 : m2, hi = m1 < m2 ? m2 : m1;
    int m = -1;
    for (int i = lo + 1; i < hi; ++i)
      if (m < 0 || N[i] < N[m]) m = i;
    uint64_t lower = N[m1] < N[m2] ? N[m1] : N[m2];
    if (m >= 0 && (uint64_t)p->dip_den * (uint64_t)N[m] < (uint64_t)p->dip_num * lower) {
      uint64_t T = oc_min_integral(oc_is_gas_bin(m, gas_bin), p);
      if (oc_sum(N, a, m) >= T && oc_sum(N, m + 1, b) >= T) {
        n = oc_split_recursive(N, a, m, p, gas_bin, out, cap, n);
        return oc_split_recursive(N, m + 1, b, p, gas_bin, out, cap, n);
      }
    }
  }
  if (n < cap) { out[n].lo = a; out[n].hi = b; }
  return n + 1;
}

typedef struct {
  int32_t lo, hi, bin;
  float x, y, z;
} oc_seed;

/* z_seed = z_i + delta dz (Sec. 3.3), binary64 from exact integers, R9 */
static float oc_seed_z(const uint32_t* N, int nbins, int i, const oc_params* p) {
  int64_t nm = (i > 0) ? (int64_t)N[i - 1] : 0;
  int64_t np = (i + 1 < nbins) ? (int64_t)N[i + 1] : 0;
  int64_t ni = (int64_t)N[i];
  int64_t num = np - nm;
  int64_t den = 2 * ni - np - nm;
  double delta = 0.0;
  if (den > 0) {
    double q = (double)num / (double)den;
    delta = 0.5 * q;
  }
  double t1 = (double)i + 0.5;
  double t2 = t1 * (double)p->dz;
  double zmid = (double)p->z_min + t2;
  double t3 = delta * (double)p->dz;
  double z = zmid + t3;
  return (float)z;
}

/* z_seed of R9 before its rounding to binary32 (error reports only) */
static double oc_seed_z64(const uint32_t* N, int nbins, int i, const oc_params* p) {
  int64_t nm = (i > 0) ? (int64_t)N[i - 1] : 0;
  int64_t np = (i + 1 < nbins) ? (int64_t)N[i + 1] : 0;
  int64_t ni = (int64_t)N[i];
  int64_t num = np - nm;
  int64_t den = 2 * ni - np - nm;
  double delta = den > 0 ? 0.5 * ((double)num / (double)den) : 0.0;
  return (double)p->z_min + ((double)i + 0.5) * (double)p->dz + delta * (double)p->dz;
}

static int oc_clusters_core(const uint32_t* N, const oc_params* p, oc_seed* seeds, int cap,
                            double* z64);

/* All seeds of one event histogram, z-ordered.  Returns the number of seeds
 * (which may exceed cap; only cap are stored). */
int oc_clusters_from_hist(const uint32_t* N, const oc_params* p, oc_seed* seeds, int cap) {
  return oc_clusters_core(N, p, seeds, cap, NULL);
}

/* The same, also giving each stored seed's z before the binary32 rounding
 * in z64 (when not NULL). */
static int oc_clusters_core(const uint32_t* N, const oc_params* p, oc_seed* seeds, int cap,
                            double* z64) {
  int nbins = oc_nbins(p);
  int gas_bin = oc_bin_f32(p->z_gas, p, nbins);
  int n = 0;
  oc_range pieces[4096];
  for (int i = 0; i < nbins; ++i) {
    if (!(N[i] > p->bin_threshold)) continue;
    int a = i;
    while (i + 1 < nbins && N[i + 1] > p->bin_threshold) i++;
    int b = i;
    int np = p->split_mode == 1 ? oc_split_recursive(N, a, b, p, gas_bin, pieces, 4096, 0)
                                : oc_split(N, a, b, p, gas_bin, pieces, 4096);
    if (np > 4096) np = 4096;
    for (int q = 0; q < np; ++q) {
      int lo = pieces[q].lo, hi = pieces[q].hi;
      int im = oc_argmax(N, lo, hi);
      uint64_t T = oc_min_integral(oc_is_gas_bin(im, gas_bin), p);
      if (oc_sum(N, lo, hi) < T) continue;
      if (n < cap) {
        seeds[n].lo = lo;
        seeds[n].hi = hi;
        seeds[n].bin = im;
        float zs = oc_seed_z(N, nbins, im, p);
        seeds[n].z = zs;
        if (z64) z64[n] = oc_seed_z64(N, nbins, im, p);
        seeds[n].x = p->x_b + p->tx_b * zs;
        seeds[n].y = p->y_b + p->ty_b * zs;
      }
      n++;
    }
  }
  return n;
}

/* ------------------------------------------------------------------------- */
/* step (d1): explicit association with the removal loop, Sec. 3.4, R6       */

/* center: per-track center bin (-1 = not filled).  seeds: K z-ordered seeds.
 * keep[k] receives 1 for surviving seeds; cluster[t] receives the index of the
 * surviving seed among the survivors (z order) or -1.  Returns survivors. */
int oc_associate(const int32_t* center, int64_t n, const oc_seed* seeds, int K,
                 const oc_params* p, int32_t* keep, int32_t* cluster) {
  int nbins = oc_nbins(p);
  int gas_bin = oc_bin_f32(p->z_gas, p, nbins);
  int* alive = (int*)malloc(sizeof(int) * (K > 0 ? K : 1));
  int* count = (int*)malloc(sizeof(int) * (K > 0 ? K : 1));
  for (int k = 0; k < K; ++k) keep[k] = 1;
  int Ka = K;
  for (;;) {
    Ka = 0;
    for (int k = 0; k < K; ++k) if (keep[k]) alive[Ka++] = k;
    for (int q = 0; q < Ka; ++q) count[q] = 0;
    for (int64_t t = 0; t < n; ++t) {
      cluster[t] = -1;
      if (center[t] < 0 || Ka == 0) continue;
      int q = 0;
      /* bins in (p_{q-1}, p_q] belong to cluster q */
      while (q + 1 < Ka) {
        int part = (seeds[alive[q]].hi + seeds[alive[q + 1]].lo) / 2;
        if (center[t] > part) q++; else break;
      }
      cluster[t] = q;
      count[q]++;
    }
    int worst = -1;
    for (int q = 0; q < Ka; ++q) {
      int gas = oc_is_gas_bin(seeds[alive[q]].bin, gas_bin);
      int need = gas ? p->min_assoc_gas : p->min_assoc_pp;
      if (count[q] < need && (worst < 0 || count[q] < count[worst])) worst = q;
    }
    if (worst < 0) break;
    keep[alive[worst]] = 0;
  }
  free(alive);
  free(count);
  return Ka;
}

/* ------------------------------------------------------------------------- */
/* step (d2, d3): adaptive weighted least-squares vertex fit, Sec. 3.5       */

typedef struct {
  double x, y, z;
  double cov[6];        /* xx, xy, yy, xz, yz, zz */
  double chi2, ndof;
  int32_t n_tracks, n_iter, status;
} oc_vertex;

/* Inverse of a symmetric positive definite 3x3 matrix by Gauss-Jordan
 * elimination of [A | I].  Returns 0 if a pivot is not above OC_PIVOT_REL
 * times its diagonal element of A, or not finite (R11). */
static int oc_inverse3(const double A[3][3], double Ainv[3][3]) {
  double a[3][6];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 6; ++c)
      a[r][c] = (c < 3) ? A[r][c] : (c - 3 == r ? 1.0 : 0.0);
  for (int c = 0; c < 3; ++c) {
    double piv = a[c][c];
    if (!(piv > 0.0) || !isfinite(piv) || !(piv > OC_PIVOT_REL * A[c][c])) return 0;
    for (int k = 0; k < 6; ++k) a[c][k] /= piv;
    for (int r = 0; r < 3; ++r) {
      if (r == c) continue;
      double f = a[r][c];
      for (int k = 0; k < 6; ++k) a[r][k] -= f * a[c][k];
    }
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      Ainv[r][c] = a[r][c + 3];
      if (!isfinite(Ainv[r][c])) return 0;
    }
  return 1;
}

typedef struct {
  double x, y, z, tx, ty;
  double wx, wy;        /* inverse of V_xx, V_yy at the seed z (Sec. 3.5) */
  int usable;
} oc_fit_track;

/* Fit one vertex from its tracks, starting at the seed. */
void oc_fit_vertex(const oc_fit_track* trk, int n, double xs, double ys, double zs,
                   const oc_params* p, oc_vertex* out) {
  double alpha[3] = {xs, ys, zs};
  double Minv[3][3] = {{0}};
  double chi2_last = 0.0, dchi2_last = 0.0, sw_last = 0.0;
  int nw_last = 0, status = 0, it_done = 0;
  for (int it = 1; it <= p->max_iter; ++it) {
    double M[3][3] = {{0}}, g[3] = {0, 0, 0};
    double chi2 = 0.0, sw = 0.0;
    int nw = 0;
    for (int i = 0; i < n; ++i) {
      if (!trk[i].usable) continue;
      double r[2];
      r[0] = trk[i].x + (alpha[2] - trk[i].z) * trk[i].tx - alpha[0];
      r[1] = trk[i].y + (alpha[2] - trk[i].z) * trk[i].ty - alpha[1];
      double W[2] = {trk[i].wx, trk[i].wy};
      double c2 = r[0] * r[0] * W[0] + r[1] * r[1] * W[1];
      double w = 0.0;
      if (c2 < p->chi2_max) {
        double f = 1.0 - c2 / p->chi2_max;
        w = f * f;                                  /* Tukey bi-square, Eq. tukey */
      }
      double H[2][3] = {{-1.0, 0.0, trk[i].tx}, {0.0, -1.0, trk[i].ty}};
      for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
          double s = 0.0;
          for (int c = 0; c < 2; ++c) s += H[c][a] * W[c] * H[c][b];
          M[a][b] += w * s;
        }
        double s = 0.0;
        for (int c = 0; c < 2; ++c) s += H[c][a] * W[c] * r[c];
        g[a] += w * s;
      }
      chi2 += w * c2;
      sw += w;
      if (w > 0.0) nw++;
    }
    it_done = it;
    if (!oc_inverse3(M, Minv)) {
      status = OC_SINGULAR;
      chi2_last = chi2; sw_last = sw; nw_last = nw; dchi2_last = 0.0;
      break;
    }
    double step[3];
    for (int a = 0; a < 3; ++a) {
      step[a] = 0.0;
      for (int b = 0; b < 3; ++b) step[a] -= Minv[a][b] * g[b];
    }
    double dchi2 = 0.0;                              /* Eq. deltachisq, R7 */
    for (int a = 0; a < 3; ++a) dchi2 += g[a] * step[a];
    for (int a = 0; a < 3; ++a) alpha[a] += step[a];
    chi2_last = chi2; dchi2_last = dchi2; sw_last = sw; nw_last = nw;
    if (fabs(dchi2) < p->dchi2_tol && fabs(step[2]) < p->dz_tol) {
      status = OC_CONVERGED;
      break;
    }
    if (it == p->max_iter) status = OC_MAXITER;
  }
  if (p->max_iter <= 0) status = OC_MAXITER;
  out->x = alpha[0];
  out->y = alpha[1];
  out->z = alpha[2];
  out->cov[0] = Minv[0][0];
  out->cov[1] = Minv[0][1];
  out->cov[2] = Minv[1][1];
  out->cov[3] = Minv[0][2];
  out->cov[4] = Minv[1][2];
  out->cov[5] = Minv[2][2];
  out->chi2 = chi2_last + dchi2_last;
  out->ndof = 2.0 * sw_last - 3.0;
  out->n_tracks = nw_last;
  out->n_iter = it_done;
  /* final selection, Sec. 3.5 last paragraph and Table smog-pp, R8 */
  if (status & OC_SINGULAR) {
    out->status = status;
    return;
  }
  int gas = out->z < (double)p->z_gas;
  if (!gas) {
    double bx = (double)p->x_b + (double)p->tx_b * out->z;
    double by = (double)p->y_b + (double)p->ty_b * out->z;
    double r = sqrt((out->x - bx) * (out->x - bx) + (out->y - by) * (out->y - by));
    if (r > p->max_r_beam) status |= OC_REJ_BEAM;
  }
  int need = gas ? p->min_pv_tracks_gas : p->min_pv_tracks_pp;
  if (out->n_tracks < need) status |= OC_REJ_NTRK;
  if (!(status & (OC_REJ_BEAM | OC_REJ_NTRK))) status |= OC_ACCEPTED;
  out->status = status;
}

/* Prepare the fit inputs of one track for a vertex whose seed is at zs. */
static void oc_fit_track_from(const float* const* T, int64_t t, double zs, oc_fit_track* f) {
  f->x = T[0][t]; f->y = T[1][t]; f->z = T[2][t];
  f->tx = T[3][t]; f->ty = T[4][t];
  double d = zs - f->z;
  double vxx = (double)T[5][t] + 2.0 * d * (double)T[6][t] + d * d * (double)T[7][t];
  double vyy = (double)T[8][t] + 2.0 * d * (double)T[9][t] + d * d * (double)T[10][t];
  f->wx = 1.0 / vxx;
  f->wy = 1.0 / vyy;
  f->usable = (vxx > 0.0) && (vyy > 0.0) && isfinite(vxx) && isfinite(vyy) &&
              isfinite(f->x) && isfinite(f->y) && isfinite(f->z) &&
              isfinite(f->tx) && isfinite(f->ty);
}

/* ------------------------------------------------------------------------- */
/* exported per-track and per-event entry points                             */

int oc_num_bins(const oc_params* p) { return oc_nbins(p); }
int oc_gas_bin(const oc_params* p) { return oc_bin_f32(p->z_gas, p, oc_nbins(p)); }

/* Step (a) in contract mode for n tracks (T = 11 SoA arrays in the order
 * x y z tx ty cxx cxtx ctxtx cyy cyty ctyty). */
/* The templates of p's profile, or NULL for the cubic profile (built into *t). */
static const oc_tpl* oc_tpl_for(const oc_params* p, oc_tpl* t) {
  t->q = NULL;
  if (p->profile_mode != 1) return NULL;
  if (oc_tpl_build(p, t) != 0) abort();
  return t;
}

/* Step (a) in contract mode for n tracks (T = 11 SoA arrays in the order
 * x y z tx ty cxx cxtx ctxtx cyy cyty ctyty); j0, j1 bound the profile. */
void oc_prepare_tracks_f32(const float* const* T, int64_t n, const oc_params* p,
                           float* zpoca, float* sigma, int32_t* center,
                           int32_t* j0, int32_t* j1, int32_t* filled) {
  int nbins = oc_nbins(p);
  oc_tpl store;
  const oc_tpl* tpl = oc_tpl_for(p, &store);
  for (int64_t t = 0; t < n; ++t) {
    oc_prep32 r;
    oc_prepare_f32(T[0][t], T[1][t], T[2][t], T[3][t], T[4][t], T[5][t], T[6][t], T[7][t],
                   p, tpl, nbins, &r);
    zpoca[t] = r.zpoca; sigma[t] = r.sigma; center[t] = r.center;
    j0[t] = r.j0; j1[t] = r.j1; filled[t] = r.filled;
  }
  oc_tpl_free(&store);
}

/* The template table of the x86 profile (R17): per class sigma_k, its lowest
 * sigma_poca, H_k and the start of its cumulative values in q (q may be NULL
 * to ask for the size).  Returns the number of q entries. */
int oc_template_table(const oc_params* p, double* sigma, double* bound, int32_t* half,
                      int32_t* first, int32_t* q, int cap) {
  oc_tpl t;
  if (oc_tpl_build(p, &t) != 0) return -1;
  int total = t.first[OC_TPL_CLASSES - 1] + 2 * t.half[OC_TPL_CLASSES - 1] + 2;
  for (int k = 0; k < OC_TPL_CLASSES; ++k) {
    if (sigma) sigma[k] = t.sigma[k];
    if (bound) bound[k] = t.bound[k];
    if (half) half[k] = t.half[k];
    if (first) first[k] = t.first[k];
  }
  if (q && cap >= total) memcpy(q, t.q, sizeof(int32_t) * (size_t)total);
  oc_tpl_free(&t);
  return total;
}

int oc_template_classes(void) { return OC_TPL_CLASSES; }

/* Step (a) in binary64, for error reports. */
void oc_prepare_tracks_f64(const float* const* T, int64_t n, const oc_params* p,
                           double* zpoca, double* sigma) {
  for (int64_t t = 0; t < n; ++t)
    oc_prepare_f64(T[0][t], T[1][t], T[2][t], T[3][t], T[4][t], T[5][t], T[6][t], T[7][t],
                   p, &zpoca[t], &sigma[t]);
}

/* Profile weights of one track given z_poca and sigma_poca (contract mode).
 * Returns the number of bins written (first bin in *first), -1 if not filled
 * or cap too small. */
int oc_track_profile(float zpoca, float sigma, const oc_params* p, int32_t* first,
                     uint32_t* weights, int cap) {
  int nbins = oc_nbins(p);
  oc_tpl store;
  const oc_tpl* tpl = oc_tpl_for(p, &store);
  oc_prep32 t;
  t.zpoca = zpoca;
  t.sigma = sigma;
  if (tpl) {
    t.tcls = oc_tpl_class(sigma, tpl);
    t.j0 = oc_bin_f32(zpoca, p, nbins) - tpl->half[t.tcls];
    t.j1 = t.j0 + 2 * tpl->half[t.tcls];
  } else {
    float s = 2.23606797749979f * sigma;
    if (s < OC_S_MIN) s = 0.0f;
    t.j0 = oc_bin_f32(zpoca - s, p, nbins);
    t.j1 = oc_bin_f32(zpoca + s, p, nbins);
  }
  *first = t.j0;
  int n = oc_profile_weights(&t, p, tpl, weights, cap);
  oc_tpl_free(&store);
  return n;
}

/* Histogram of one event (nbins bins, cleared here). */
static void oc_event_histogram_t(const float* const* T, int64_t begin, int64_t end,
                                 const oc_params* p, const oc_tpl* tpl, uint32_t* hist,
                                 int32_t* center) {
  int nbins = oc_nbins(p);
  int cap = nbins + 2 * OC_TPL_MAX_HALF + 8;
  memset(hist, 0, sizeof(uint32_t) * (size_t)nbins);
  uint32_t* w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)cap);
  for (int64_t t = begin; t < end; ++t) {
    oc_prep32 r;
    oc_prepare_f32(T[0][t], T[1][t], T[2][t], T[3][t], T[4][t], T[5][t], T[6][t], T[7][t],
                   p, tpl, nbins, &r);
    center[t - begin] = r.filled ? r.center : -1;
    if (!r.filled) continue;
    int k = oc_profile_weights(&r, p, tpl, w, cap);
    for (int q = 0; q < k; ++q) {
      int j = r.j0 + q;
      if (j >= 0 && j < nbins) hist[j] += w[q];
    }
  }
  free(w);
}

void oc_event_histogram(const float* const* T, int64_t begin, int64_t end, const oc_params* p,
                        uint32_t* hist, int32_t* center) {
  oc_tpl store;
  const oc_tpl* tpl = oc_tpl_for(p, &store);
  oc_event_histogram_t(T, begin, end, p, tpl, hist, center);
  oc_tpl_free(&store);
}

/* Steps (a)-(d1) for a batch of events.
 * Outputs (cap = p->max_seeds seeds per event, row-major [event][cap]):
 *   seed_{x,y,z,lo,hi,bin}, n_seeds[event], event_status[event],
 *   track_cluster[track] (index into the event's seed list or -1),
 *   hist (optional, n_events x nbins). */
int oc_find_batch(const float* const* T, const int64_t* offsets, int32_t n_events,
                  const oc_params* p, float* seed_x, float* seed_y, float* seed_z,
                  int32_t* seed_lo, int32_t* seed_hi, int32_t* seed_bin, int32_t* n_seeds,
                  int32_t* event_status, int32_t* track_cluster, uint32_t* hist_out) {
  int nbins = oc_nbins(p);
  int cap = p->max_seeds;
  uint32_t* hist = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nbins);
  oc_seed* seeds = (oc_seed*)malloc(sizeof(oc_seed) * (size_t)(cap > 0 ? cap : 1));
  int32_t* keep = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
  oc_tpl store;
  const oc_tpl* tpl = oc_tpl_for(p, &store);
  for (int32_t e = 0; e < n_events; ++e) {
    int64_t b = offsets[e], en = offsets[e + 1];
    int64_t n = en - b;
    int32_t* center = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    oc_event_histogram_t(T, b, en, p, tpl, hist, center);
    if (hist_out) memcpy(hist_out + (size_t)e * nbins, hist, sizeof(uint32_t) * (size_t)nbins);
    int K = oc_clusters_from_hist(hist, p, seeds, cap);
    event_status[e] = 0;
    if (K > cap) { event_status[e] |= OC_EV_SEED_OVERFLOW; K = cap; }
    int Ka = oc_associate(center, n, seeds, K, p, keep, track_cluster + b);
    int q = 0;
    for (int k = 0; k < K; ++k) {
      if (!keep[k]) continue;
      size_t o = (size_t)e * cap + q;
      seed_x[o] = seeds[k].x; seed_y[o] = seeds[k].y; seed_z[o] = seeds[k].z;
      seed_lo[o] = seeds[k].lo; seed_hi[o] = seeds[k].hi; seed_bin[o] = seeds[k].bin;
      q++;
    }
    n_seeds[e] = Ka;
    free(center);
  }
  free(hist);
  free(seeds);
  free(keep);
  oc_tpl_free(&store);
  return 0;
}

/* Steps (d2)-(d3) for a batch: fit every seed of every event from the tracks
 * assigned to it.  Vertex outputs are row-major [event][cap] in seed order. */
int oc_fit_batch(const float* const* T, const int64_t* offsets, int32_t n_events,
                 const oc_params* p, const float* seed_x, const float* seed_y,
                 const float* seed_z, const int32_t* n_seeds, const int32_t* track_cluster,
                 double* vx, double* vy, double* vz, double* vcov, double* vchi2,
                 double* vndof, int32_t* vntrk, int32_t* vniter, int32_t* vstatus) {
  int cap = p->max_seeds;
  for (int32_t e = 0; e < n_events; ++e) {
    int64_t b = offsets[e], en = offsets[e + 1];
    int64_t n = en - b;
    oc_fit_track* ft = (oc_fit_track*)malloc(sizeof(oc_fit_track) * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k < n_seeds[e]; ++k) {
      size_t o = (size_t)e * cap + k;
      double zs = seed_z[o];
      int m = 0;
      for (int64_t t = b; t < en; ++t)
        if (track_cluster[t] == k) oc_fit_track_from(T, t, zs, &ft[m++]);
      oc_vertex v;
      oc_fit_vertex(ft, m, seed_x[o], seed_y[o], zs, p, &v);
      vx[o] = v.x; vy[o] = v.y; vz[o] = v.z;
      for (int c = 0; c < 6; ++c) vcov[o * 6 + c] = v.cov[c];
      vchi2[o] = v.chi2; vndof[o] = v.ndof;
      vntrk[o] = v.n_tracks; vniter[o] = v.n_iter; vstatus[o] = v.status;
    }
    free(ft);
  }
  return 0;
}

/* Fit one vertex from explicit track arrays (for the pins). */
void oc_fit_tracks(const float* const* T, int64_t n, float xs, float ys, float zs,
                   const oc_params* p, double* x, double* cov, double* chi2, double* ndof,
                   int32_t* ntrk, int32_t* niter, int32_t* status) {
  oc_fit_track* ft = (oc_fit_track*)malloc(sizeof(oc_fit_track) * (size_t)(n > 0 ? n : 1));
  for (int64_t t = 0; t < n; ++t) oc_fit_track_from(T, t, zs, &ft[t]);
  oc_vertex v;
  oc_fit_vertex(ft, (int)n, xs, ys, zs, p, &v);
  x[0] = v.x; x[1] = v.y; x[2] = v.z;
  for (int c = 0; c < 6; ++c) cov[c] = v.cov[c];
  *chi2 = v.chi2; *ndof = v.ndof; *ntrk = v.n_tracks; *niter = v.n_iter; *status = v.status;
  free(ft);
}

/* Seeds of one histogram (for the pins): arrays of size cap. Returns count. */
int oc_seeds_from_hist(const uint32_t* N, const oc_params* p, int32_t* lo, int32_t* hi,
                       int32_t* bin, float* z, int cap) {
  oc_seed* s = (oc_seed*)malloc(sizeof(oc_seed) * (size_t)(cap > 0 ? cap : 1));
  int n = oc_clusters_from_hist(N, p, s, cap);
  int m = n < cap ? n : cap;
  for (int k = 0; k < m; ++k) { lo[k] = s[k].lo; hi[k] = s[k].hi; bin[k] = s[k].bin; z[k] = s[k].z; }
  free(s);
  return n;
}

/* Association of given center bins to given seeds (for the pins). */
int oc_associate_bins(const int32_t* center, int64_t n, const int32_t* lo, const int32_t* hi,
                      const int32_t* bin, int K, const oc_params* p, int32_t* keep,
                      int32_t* cluster) {
  oc_seed* s = (oc_seed*)malloc(sizeof(oc_seed) * (size_t)(K > 0 ? K : 1));
  for (int k = 0; k < K; ++k) { s[k].lo = lo[k]; s[k].hi = hi[k]; s[k].bin = bin[k]; }
  int r = oc_associate(center, n, s, K, p, keep, cluster);
  free(s);
  return r;
}

/* ========================================================================= */
/* GPU-flavour multi-vertex fit (Sec. 3.5, implicit track association)      */
/*
 * Readings:
 *   R12 weights (Sec. 3.5, Eq. of w_ij): w_ij = exp(-chi2_ij / 2) /
 *       (exp(-chi2_cut / 2) + sum_k exp(-chi2_ik / 2)), k over every seed of
 *       the event.  For a competing vertex k != j, chi2_ik is taken at k's seed
 *       position (the paper keeps the other vertices at their initial
 *       positions, so the fits are independent); for k = j at j's current
 *       position.  W_ik is V^-1 extrapolated to seed k's z (R2); a track that is
 *       not usable for seed k (R10) adds nothing to that term.  chi2_cut = 4,
 *       the value of the paper's weight figure.
 *   R13 the fit stops when |dz| < 0.5 um (no dchi2 condition, Sec. 3.5 GPU
 *       rule), at most max_iter iterations; singular matrices as R11.
 *   R14 a vertex's tracks are those with w_ij >= 0.5 in its last iteration; a
 *       track belongs to the vertex with its largest last-iteration weight when
 *       that weight is >= 0.5 (lowest index on ties), otherwise to none.
 *   R15 duplicates: in seed (z) order every non-singular vertex is compared with
 *       the last one kept; if dz^2 < dup_sep2 (C_zz + C_zz') the one with fewer
 *       tracks is rejected (the earlier one when equal).  The final selection of
 *       Sec. 3.5 then applies to the rest.
 */
typedef struct {
  double chi2_cut;      /* 4 */
  double dz_tol;        /* 0.5e-3 mm */
  double w_assoc;       /* 0.5 */
  double dup_sep2;      /* 25 */
  int32_t max_iter;     /* 10 */
} oc_mv_params;

#define OC_DUPLICATE 64

/* chi2 of a track (fit inputs for some seed) at the point (x, y, z), Eq. chi2 */
static double oc_mv_chi2(const oc_fit_track* f, double x, double y, double z) {
  double rx = f->x + (z - f->z) * f->tx - x;
  double ry = f->y + (z - f->z) * f->ty - y;
  return rx * rx * f->wx + ry * ry * f->wy;
}

/* R12 with comp = sum over the competing seeds of exp(-chi2_ik / 2) */
static double oc_mv_weight(double c2, double comp, const oc_mv_params* m) {
  double e = exp(-0.5 * c2);
  return e / (exp(-0.5 * m->chi2_cut) + comp + e);
}

/* Fit of one vertex with the multi-vertex weights (same normal equations as
 * oc_fit_vertex, R7).  a_prev receives the position the last weights were
 * taken at. */
static void oc_mv_fit_vertex(const oc_fit_track* trk, const double* comp, int n, double xs,
                             double ys, double zs, const oc_mv_params* m, oc_vertex* out,
                             double a_prev[3]) {
  double alpha[3] = {xs, ys, zs};
  double Minv[3][3] = {{0}};
  double chi2_last = 0.0, dchi2_last = 0.0, sw_last = 0.0;
  int nw_last = 0, status = 0, it_done = 0;
  a_prev[0] = xs; a_prev[1] = ys; a_prev[2] = zs;
  for (int it = 1; it <= m->max_iter; ++it) {
    double M[3][3] = {{0}}, g[3] = {0, 0, 0};
    double chi2 = 0.0, sw = 0.0;
    int nw = 0;
    for (int a = 0; a < 3; ++a) a_prev[a] = alpha[a];
    for (int i = 0; i < n; ++i) {
      if (!trk[i].usable) continue;
      double r[2];
      r[0] = trk[i].x + (alpha[2] - trk[i].z) * trk[i].tx - alpha[0];
      r[1] = trk[i].y + (alpha[2] - trk[i].z) * trk[i].ty - alpha[1];
      double W[2] = {trk[i].wx, trk[i].wy};
      double c2 = r[0] * r[0] * W[0] + r[1] * r[1] * W[1];
      double w = oc_mv_weight(c2, comp[i], m);
      double H[2][3] = {{-1.0, 0.0, trk[i].tx}, {0.0, -1.0, trk[i].ty}};
      for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
          double s = 0.0;
          for (int c = 0; c < 2; ++c) s += H[c][a] * W[c] * H[c][b];
          M[a][b] += w * s;
        }
        double s = 0.0;
        for (int c = 0; c < 2; ++c) s += H[c][a] * W[c] * r[c];
        g[a] += w * s;
      }
      chi2 += w * c2;
      sw += w;
      if (w >= m->w_assoc) nw++;
    }
    it_done = it;
    if (!oc_inverse3(M, Minv)) {
      status = OC_SINGULAR;
      chi2_last = chi2; sw_last = sw; nw_last = nw; dchi2_last = 0.0;
      break;
    }
    double step[3];
    for (int a = 0; a < 3; ++a) {
      step[a] = 0.0;
      for (int b = 0; b < 3; ++b) step[a] -= Minv[a][b] * g[b];
    }
    double dchi2 = 0.0;
    for (int a = 0; a < 3; ++a) dchi2 += g[a] * step[a];
    for (int a = 0; a < 3; ++a) alpha[a] += step[a];
    chi2_last = chi2; dchi2_last = dchi2; sw_last = sw; nw_last = nw;
    if (fabs(step[2]) < m->dz_tol) {                 /* R13 */
      status = OC_CONVERGED;
      break;
    }
    if (it == m->max_iter) status = OC_MAXITER;
  }
  if (m->max_iter <= 0) status = OC_MAXITER;
  out->x = alpha[0];
  out->y = alpha[1];
  out->z = alpha[2];
  out->cov[0] = Minv[0][0];
  out->cov[1] = Minv[0][1];
  out->cov[2] = Minv[1][1];
  out->cov[3] = Minv[0][2];
  out->cov[4] = Minv[1][2];
  out->cov[5] = Minv[2][2];
  out->chi2 = chi2_last + dchi2_last;
  out->ndof = 2.0 * sw_last - 3.0;
  out->n_tracks = nw_last;
  out->n_iter = it_done;
  out->status = status;
}

/* Multi-vertex fit of every seed of every event (seeds as oc_find_batch writes
 * them, rows of p->max_seeds), duplicate removal and final selection.
 * track_vertex: per track, R14. */
int oc_mv_fit_batch(const float* const* T, const int64_t* offsets, int32_t n_events,
                    const oc_params* p, const oc_mv_params* m, const float* seed_x,
                    const float* seed_y, const float* seed_z, const int32_t* n_seeds,
                    double* vx, double* vy, double* vz, double* vcov, double* vchi2,
                    double* vndof, int32_t* vntrk, int32_t* vniter, int32_t* vstatus,
                    int32_t* track_vertex) {
  int cap = p->max_seeds;
  for (int32_t e = 0; e < n_events; ++e) {
    int64_t b = offsets[e], n = offsets[e + 1] - b;
    int K = n_seeds[e];
    size_t nn = (size_t)(n > 0 ? n : 1), kk = (size_t)(K > 0 ? K : 1);
    double* E = (double*)malloc(sizeof(double) * nn * kk);     /* exp(-chi2_ik/2) at seed k */
    oc_fit_track* ft = (oc_fit_track*)malloc(sizeof(oc_fit_track) * nn);
    double* comp = (double*)malloc(sizeof(double) * nn);
    double* prev = (double*)malloc(sizeof(double) * 3 * kk);
    for (int k = 0; k < K; ++k) {
      size_t o = (size_t)e * cap + k;
      for (int64_t i = 0; i < n; ++i) {
        oc_fit_track f;
        oc_fit_track_from(T, b + i, seed_z[o], &f);
        E[i * kk + k] = f.usable ? exp(-0.5 * oc_mv_chi2(&f, seed_x[o], seed_y[o], seed_z[o]))
                                 : 0.0;
      }
    }
    for (int j = 0; j < K; ++j) {
      size_t o = (size_t)e * cap + j;
      for (int64_t i = 0; i < n; ++i) {
        oc_fit_track_from(T, b + i, seed_z[o], &ft[i]);
        double c = 0.0;
        for (int k = 0; k < K; ++k)
          if (k != j) c += E[i * kk + k];
        comp[i] = c;
      }
      oc_vertex v;
      oc_mv_fit_vertex(ft, comp, (int)n, seed_x[o], seed_y[o], seed_z[o], m, &v, prev + 3 * j);
      vx[o] = v.x; vy[o] = v.y; vz[o] = v.z;
      for (int c = 0; c < 6; ++c) vcov[o * 6 + c] = v.cov[c];
      vchi2[o] = v.chi2; vndof[o] = v.ndof;
      vntrk[o] = v.n_tracks; vniter[o] = v.n_iter; vstatus[o] = v.status;
    }
    /* R14: each track's vertex from the last-iteration weights */
    for (int64_t i = 0; i < n; ++i) {
      int best = -1;
      double wbest = -1.0;
      for (int j = 0; j < K; ++j) {
        size_t o = (size_t)e * cap + j;
        if (vstatus[o] & OC_SINGULAR) continue;
        oc_fit_track f;
        oc_fit_track_from(T, b + i, seed_z[o], &f);
        if (!f.usable) continue;
        double c = 0.0;
        for (int k = 0; k < K; ++k)
          if (k != j) c += E[i * kk + k];
        double w = oc_mv_weight(oc_mv_chi2(&f, prev[3 * j], prev[3 * j + 1], prev[3 * j + 2]),
                                c, m);
        if (w > wbest) { wbest = w; best = j; }
      }
      track_vertex[b + i] = (best >= 0 && wbest >= m->w_assoc) ? best : -1;
    }
    /* R15: duplicates, then the final selection (Sec. 3.5, Table smog-pp) */
    int last = -1;
    for (int j = 0; j < K; ++j) {
      size_t o = (size_t)e * cap + j;
      if (vstatus[o] & OC_SINGULAR) continue;
      if (last >= 0) {
        size_t ol = (size_t)e * cap + last;
        double dz = vz[o] - vz[ol];
        if (dz * dz < m->dup_sep2 * (vcov[o * 6 + 5] + vcov[ol * 6 + 5])) {
          if (vntrk[o] > vntrk[ol]) {
            vstatus[ol] |= OC_DUPLICATE;
            last = j;
          } else {
            vstatus[o] |= OC_DUPLICATE;
          }
          continue;
        }
      }
      last = j;
    }
    for (int j = 0; j < K; ++j) {
      size_t o = (size_t)e * cap + j;
      int st = vstatus[o];
      if (st & (OC_SINGULAR | OC_DUPLICATE)) continue;
      int gas = vz[o] < (double)p->z_gas;
      if (!gas) {
        double bx = (double)p->x_b + (double)p->tx_b * vz[o];
        double by = (double)p->y_b + (double)p->ty_b * vz[o];
        double r = sqrt((vx[o] - bx) * (vx[o] - bx) + (vy[o] - by) * (vy[o] - by));
        if (r > p->max_r_beam) st |= OC_REJ_BEAM;
      }
      int need = gas ? p->min_pv_tracks_gas : p->min_pv_tracks_pp;
      if (vntrk[o] < need) st |= OC_REJ_NTRK;
      if (!(st & (OC_REJ_BEAM | OC_REJ_NTRK))) st |= OC_ACCEPTED;
      vstatus[o] = st;
    }
    free(E); free(ft); free(comp); free(prev);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* binary64 replay of steps (a)-(d1), for error reports only                 */

/* The cubic profile of R3 evaluated in binary64 from the binary64 z_poca and
 * sigma_poca, quantised with the same rule: every quantity of step (a) and
 * (b) in binary64, the histogram and everything after it integer as before. */
static void oc_event_histogram_f64(const float* const* T, int64_t begin, int64_t end,
                                   const oc_params* p, uint32_t* hist, int32_t* center) {
  int nbins = oc_nbins(p);
  memset(hist, 0, sizeof(uint32_t) * (size_t)nbins);
  const double zmin = p->z_min, dz = p->dz;
  for (int64_t t = begin; t < end; ++t) {
    double zp, sig;
    oc_prepare_f64(T[0][t], T[1][t], T[2][t], T[3][t], T[4][t], T[5][t], T[6][t], T[7][t],
                   p, &zp, &sig);
    center[t - begin] = -1;
    double dtx = (double)T[3][t] - (double)p->tx_b, dty = (double)T[4][t] - (double)p->ty_b;
    if (!(dtx * dtx + dty * dty > 0.0) || !isfinite(zp) || !isfinite(sig)) continue;
    double qc = floor((zp - zmin) / dz);
    if (!(qc >= 0.0) || qc >= (double)nbins) continue;
    double smax = zp < (double)p->z_gas ? (double)p->sigma_max_gas : (double)p->sigma_max_pp;
    if (!(sig <= smax)) continue;
    center[t - begin] = (int32_t)qc;
    double sp = 2.23606797749979 * sig;
    if (sp < (double)OC_S_MIN) sp = 0.0;
    int j0 = (int)floor((zp - sp - zmin) / dz), j1 = (int)floor((zp + sp - zmin) / dz);
    int32_t qprev = 0;
    for (int j = j0; j <= j1; ++j) {
      int32_t qnext = OC_ONE;
      if (j < j1) {
        double u = (zmin + (double)(j + 1) * dz - zp) / sp;
        double F = u <= -1.0 ? 0.0 : (u >= 1.0 ? 1.0 : 0.5 + u * (0.75 - 0.25 * u * u));
        long q = lrint(F * OC_ONE);
        qnext = (int32_t)(q < 0 ? 0 : (q > OC_ONE ? OC_ONE : q));
      }
      if (qnext < qprev) qnext = qprev;
      if (j >= 0 && j < nbins) hist[j] += (uint32_t)(qnext - qprev);
      qprev = qnext;
    }
  }
}

/* Surviving seeds of every event (cap per event, row-major): their maximum bin
 * and z in binary64. */
int oc_find_batch_f64(const float* const* T, const int64_t* offsets, int32_t n_events,
                      const oc_params* p, double* seed_z, int32_t* seed_bin, int32_t* n_seeds) {
  int nbins = oc_nbins(p);
  int cap = p->max_seeds;
  uint32_t* hist = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nbins);
  oc_seed* seeds = (oc_seed*)malloc(sizeof(oc_seed) * (size_t)(cap > 0 ? cap : 1));
  double* z64 = (double*)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
  int32_t* keep = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
  for (int32_t e = 0; e < n_events; ++e) {
    int64_t b = offsets[e], en = offsets[e + 1];
    int64_t n = en - b;
    int32_t* center = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    oc_event_histogram_f64(T, b, en, p, hist, center);
    int K = oc_clusters_core(hist, p, seeds, cap, z64);
    if (K > cap) K = cap;
    int Ka = oc_associate(center, n, seeds, K, p, keep, cl);
    int q = 0;
    for (int k = 0; k < K; ++k) {
      if (!keep[k]) continue;
      seed_z[(size_t)e * cap + q] = z64[k];
      seed_bin[(size_t)e * cap + q] = seeds[k].bin;
      q++;
    }
    n_seeds[e] = Ka;
    free(center);
    free(cl);
  }
  free(hist);
  free(seeds);
  free(z64);
  free(keep);
  return 0;
}

/* Per-bin error of the binary32 profile (R3 cubic, or R17 templates) against
 * the Gaussian bin integral of the binary64 z_poca and sigma_poca, over the
 * bins within 5 sigma of z_poca of every filled track: out[0] = largest
 * |w / ONE - G|, out[1] = sum of squares, out[2] = number of bins, out[3] =
 * largest |sum of the window's weights / ONE - Gaussian mass inside the
 * histogram| (the window's truncation). */
void oc_profile_error(const float* const* T, int64_t n, const oc_params* p, double* out) {
  int nbins = oc_nbins(p);
  oc_tpl store;
  const oc_tpl* tpl = oc_tpl_for(p, &store);
  int cap = nbins + 2 * OC_TPL_MAX_HALF + 8;
  uint32_t* w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)cap);
  double emax = 0.0, ss = 0.0, cnt = 0.0, tmax = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    oc_prep32 r;
    oc_prepare_f32(T[0][t], T[1][t], T[2][t], T[3][t], T[4][t], T[5][t], T[6][t], T[7][t],
                   p, tpl, nbins, &r);
    if (!r.filled) continue;
    double zp, sig;
    oc_prepare_f64(T[0][t], T[1][t], T[2][t], T[3][t], T[4][t], T[5][t], T[6][t], T[7][t],
                   p, &zp, &sig);
    if (!(sig > 0.0)) continue;
    int k = oc_profile_weights(&r, p, tpl, w, cap);
    int g0 = (int)floor((zp - 5.0 * sig - p->z_min) / p->dz);
    int g1 = (int)floor((zp + 5.0 * sig - p->z_min) / p->dz);
    int lo = g0 < r.j0 ? g0 : r.j0, hi = g1 > r.j1 ? g1 : r.j1;
    if (lo < 0) lo = 0;
    if (hi > nbins - 1) hi = nbins - 1;
    double wsum = 0.0, gsum = 0.0;
    for (int j = lo; j <= hi; ++j) {
      double wj = (j >= r.j0 && j <= r.j1 && j - r.j0 < k) ? (double)w[j - r.j0] / OC_ONE : 0.0;
      double e0 = (double)p->z_min + (double)j * p->dz, e1 = e0 + p->dz;
      double g = oc_phi((e1 - zp) / sig) - oc_phi((e0 - zp) / sig);
      double d = fabs(wj - g);
      if (d > emax) emax = d;
      ss += d * d;
      cnt += 1.0;
      wsum += wj;
      gsum += g;
    }
    double tr = fabs(wsum - gsum);
    if (tr > tmax) tmax = tr;
  }
  free(w);
  oc_tpl_free(&store);
  out[0] = emax;
  out[1] = ss;
  out[2] = cnt;
  out[3] = tmax;
}
