/*
 * twinkle.h -- C ABI of the GB300 finite-source binary-lens magnification
 * library (libtwinkle_gb300.so).
 *
 * The problem (paper Sec. 2.1, Eq. 1-2; Sec. 2.3): a binary lens of total mass
 * 1 with mass ratio q = m2/m1 > 0 and projected separation s > 0, in units of
 * the angular Einstein radius (Eq. 3), with the origin at the centre of mass:
 * the primary m1 = 1/(1+q) sits at x = -q s/(1+q), the secondary m2 = q/(1+q)
 * at x = +s/(1+q), both on the real axis.  A uniform disc source of radius
 * rho > 0 centred at zeta0 = y1 + i y2 is magnified by
 *
 *     mu = (total area of its images) / (pi rho^2)          (Sec. 1)
 *
 * which the library computes by contour integration of the images of the
 * source limb (Sec. 2.3-2.5): cancellation-free quintic coefficients (Eq. 6),
 * roots, ghost rejection by the lens-equation residual (Eq. 12-15), linking of
 * real images by parity (Eq. 7), Green's-theorem area with parabolic and
 * cross-caustic corrections (Eq. 8-11), error estimates (Eq. 17-18) and
 * adaptive inverse-transform resampling of the limb until the estimated error
 * is at most rel_tol * mu, or the sample cap is reached (Sec. 3).
 *
 * Memory: every pointer argument is owned by the caller and may point to host
 * memory (pageable or pinned) or to device memory of the current CUDA device;
 * the kind is detected per pointer.  All array arguments of one call must be
 * of the same kind; device memory of another device returns TW_EINVAL.  With host pointers the call is synchronous: inputs are
 * copied to the device and outputs back before it returns.  With device
 * pointers the call is asynchronous on opts->stream (NULL = the legacy default
 * stream) and outputs are valid once that stream reaches the call; buffers
 * must stay valid until then.  The library keeps its own device working
 * memory (sample arenas, staging buffers) for the lifetime of the process; it
 * never frees or retains caller memory.
 *
 * Errors: a negative return code means nothing was written (argument errors
 * are detected before any device work).  The environment variable
 * TW_DEVICE_MEMORY_LIMIT (bytes; unset or 0 = none) caps the device working
 * memory the library allocates for contour integration: a call that would
 * need more returns TW_ENOMEM and writes nothing.  TW_OK means every output element was
 * written; per-position outcomes are reported in opts->pos_status when given.
 * A positive return (warning) is only produced by synchronous (host-pointer)
 * calls, after all outputs were written.
 */
#ifndef TWINKLE_GB300_H
#define TWINKLE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
enum {
    TW_OK = 0,
    TW_EINVAL = -1,   /* invalid argument: n < 0, NULL with n > 0, non-finite or
                         non-positive s, q, rho, tE or rel_tol, mixed pointer
                         kinds, options out of range; nothing written */
    TW_ECUDA = -2,    /* a CUDA runtime call failed (no device, launch error) */
    TW_ENOMEM = -3,   /* device working memory could not be allocated */
    TW_ETIMEOUT = -4, /* a bounded device-side wait gave up */
    TW_ETOOBIG = -5,  /* tw_mag_noalloc: the request needs more scratch than its
                         static array holds (max_samples > 512) */
    TW_WCAP = 1       /* synchronous call: >= 1 position reached the sample cap;
                         its output holds the best estimate */
};

/* Per-position status bits written to tw_opts.pos_status. */
enum {
    TW_POS_OK = 0,
    TW_POS_CAP = 1,        /* sample cap reached: mu is the estimate with the cap's
                              samples, err_out its error estimate (Sec. 3) */
    TW_POS_IMAGECOUNT = 2, /* a limb sample had no image set with 3 or 5 real
                              images and parity sum -1 (Sec. 2.3) */
    TW_POS_NONFINITE = 4,  /* non-finite input position or result (out is NaN) */
    TW_POS_SOLVER = 8,     /* root iteration stopped at its iteration limit */
    TW_POS_SLOPE = 16,     /* a caustic crossing failed the slope test
                              (Sec. 2.4.2): its pair of merging images was
                              not perpendicular to the ghost pair across it;
                              the crossing was moved to the slope jump, or a
                              false image piece removed, where the walk along
                              the five-image run found one */
    TW_POS_EXPANSION = 32, /* tw_surrogate_mag: answered by the point-source
                              expansion (no contour integration) */
    TW_POS_NETWORK = 64    /* tw_surrogate_mag: answered by the network */
};

/* Arithmetic modes. */
enum {
    TW_PREC_FP64 = 0, /* root iterations in FP64 (their pair sums in FP32);
                         coefficients, residuals and area sums in FP64 */
    TW_PREC_MIXED = 1 /* root iterations in FP32, then FP64 polish; coefficients
                         (Eq. 6), residual test (Eq. 12) and area sums in FP64 */
};

typedef struct tw_opts {
    int precision;        /* TW_PREC_FP64 (default) or TW_PREC_MIXED */
    int samples_per_iter; /* limb samples added per iteration and initial sample
                             count: 32, 64 (default, Sec. 3) or 128 */
    int max_samples;      /* sample cap per position, 64..16384 (default 4096, Sec. 3) */
    int autotune;         /* 1: choose the launch shape (samples per iteration,
                             CTAs per SM, work items per grab) by timing a ~5%
                             calibration sub-sample; cached per (GPU, precision,
                             tolerance decade, workload kind) in memory and in
                             $TW_AUTOTUNE_CACHE (default
                             $HOME/.cache/twinkle_gb300_autotune.txt).  It
                             overrides samples_per_iter. */
    int use_graph;        /* 1: replay the launch from a CUDA graph captured on
                             `stream` (needs a non-NULL stream; device pointers) */
    void *stream;         /* cudaStream_t for device-pointer calls, or NULL */
    double *err_out;      /* optional [n]: error estimate of mu (absolute) */
    int32_t *nsamp_out;   /* optional [n]: limb samples used */
    int8_t *pos_status;   /* optional [n]: TW_POS_* bits */
    int warps_per_position; /* 1 (default): one warp integrates each position;
                             2 or 4: that many warps of a CTA integrate each
                             position together, one new limb sample per lane
                             per iteration (32 x warps per iteration;
                             samples_per_iter is then ignored) -- fewer
                             positions in flight, each finished sooner, for
                             workloads too small to fill the GPU (the paper
                             uses a block of threads per source, Sec. 3).
                             With autotune = 1 the autotuner chooses it. */
} tw_opts;

/* Fills *opts with the defaults listed above (all output pointers NULL).
 * tw_opts grows only at its end; fill it with tw_opts_default first. */
void tw_opts_default(tw_opts *opts);

/* Finite-source magnification of n source positions (y1[i], y2[i]) behind
 * one binary lens (s, q) for one source radius rho; out[i] receives mu.
 * rel_tol is the target relative error of mu (the paper's tolerance, Sec. 4.1).
 * Layout: y1, y2, out are contiguous float64 arrays of n elements. */
int tw_mag(double s, double q, double rho, const double *y1, const double *y2, int64_t n,
           double rel_tol, double *out);
int tw_mag_ex(double s, double q, double rho, const double *y1, const double *y2, int64_t n,
              double rel_tol, double *out, const tw_opts *opts);

/* Magnification of a limb-darkened source: brightness I(r) = 1 - u (1 -
 * sqrt(1 - r^2/rho^2)) at distance r from the centre (linear law, 0 <= u <= 1;
 * u = 0 is the uniform disc).  The paper notes that contour integration of a
 * limb-darkened source is costly (Sec. 1) and gives no method; this library
 * writes the image flux, integrated by parts over the radius, as
 *   mu = [(1 - u) mu_1(rho) + u Int_0^{pi/2} sin^3(phi) mu_1(rho sin phi) dphi] / (1 - u/3),
 * mu_1(r) being the uniform-disc magnification of radius r (the contour
 * integral of tw_mag).  mu_1 has kinks at the radii where the circle about
 * the source centre touches a fold of the caustic or passes over a cusp (the
 * stationary points of the distance from the centre along the caustic,
 * found by a sweep of the critical curve); the phi integral is cut there,
 * each piece mapped by a substitution that is flat at its cut ends, and
 * integrated by adaptive Simpson panels (error |S - S_halves| / 15 per
 * panel, up to 40 panels), each uniform disc to rel_tol/2 and the
 * quadrature to rel_tol/2.  One warp per source; opts->err_out receives the
 * summed error estimate, nsamp_out the limb samples of all radii.  Crossings
 * that fail the slope test are reported (TW_POS_SLOPE) and not repaired.
 * Arrays and layout as tw_mag_ex; opts->autotune and warps_per_position are
 * ignored. */
int tw_mag_ld(double s, double q, double rho, double u, const double *y1, const double *y2, int64_t n,
              double rel_tol, double *out, const tw_opts *opts);

/* As tw_mag_ex, with a lens (s[i], q[i]) and source radius rho[i] of its own
 * for every position (contiguous float64 arrays of n elements); positions
 * with an invalid lens or radius give NaN and TW_POS_NONFINITE. */
int tw_mag_multi(const double *s, const double *q, const double *rho, const double *y1, const double *y2, int64_t n,
                 double rel_tol, double *out, const tw_opts *opts);

/* Light curve: magnification at n times of a source moving on a straight
 * line (the paper leaves the convention open; this library uses, with
 * tau = (t - t0)/tE,  y1 = tau cos(alpha) - u0 sin(alpha),
 * y2 = tau sin(alpha) + u0 cos(alpha), in the centre-of-mass frame).
 * times and out are contiguous float64 arrays of n elements; tE > 0. */
int tw_lightcurve(double s, double q, double rho, double u0, double alpha, double t0, double tE,
                  const double *times, int64_t n, double rel_tol, double *out);
int tw_lightcurve_ex(double s, double q, double rho, double u0, double alpha, double t0, double tE,
                     const double *times, int64_t n, double rel_tol, double *out, const tw_opts *opts);

/* Light curve of an orbiting binary lens.  The paper names lens orbital
 * motion as the case contour integration handles flexibly (Sec. 1), without
 * a formula; this library takes the first-order (linear) reading: at time t
 * the separation is s + ds_dt (t - t0) and the binary axis has turned so that
 * the trajectory angle is alpha + dalpha_dt (t - t0), the trajectory being
 * that of tw_lightcurve with these values (ds_dt in Einstein radii per unit
 * of t, dalpha_dt in radians per unit of t).  A time whose separation is not
 * positive gives NaN and TW_POS_NONFINITE.  With ds_dt = dalpha_dt = 0 the
 * results equal tw_lightcurve_ex's. */
int tw_lightcurve_orbital(double s, double q, double rho, double u0, double alpha, double t0, double tE,
                          double ds_dt, double dalpha_dt, const double *times, int64_t n, double rel_tol, double *out,
                          const tw_opts *opts);

/* Many light curves of uneven length in one persistent, work-stealing launch.
 * params: [ncurve][7] float64 rows (s, q, rho, u0, alpha, t0, tE);
 * offsets: [ncurve + 1] int64, offsets[0] = 0, non-decreasing; curve k owns
 * times[offsets[k] .. offsets[k+1]) and the same range of out (and of the
 * optional per-position outputs).  Total positions = offsets[ncurve]. */
int tw_lightcurve_batch(const double *params, const int64_t *offsets, const double *times,
                        int64_t ncurve, double rel_tol, double *out, const tw_opts *opts);

/* tw_mag without any device memory allocation, for callers that cannot
 * allocate: code being captured into a CUDA graph, applications whose device
 * memory belongs to their own pool or arena, and real-time loops in which an
 * allocation could stall or fail.  (The paper has no counterpart: it
 * describes no API.)  It computes what tw_mag_ex computes, with the given
 * precision (TW_PREC_*) and sample cap max_samples (64..512), on `stream`,
 * including the slope-repair pass for up to 4096 positions per call (further
 * positions whose crossing fails the slope test keep the main pass's value).
 * y1, y2 and out must be device pointers of the current device; the call is
 * asynchronous.  The library's scratch for this entry point is one static
 * device array of about 53 MiB (608 warp arenas of 512 limb samples, the
 * repair queue and a work counter), which every GPU that loads the library
 * keeps until the process exits.  Those 608 arenas allow one CTA of four
 * warps per SM on a 152-SM GPU, half the resident warps of tw_mag, which
 * costs throughput on large calls.  max_samples > 512 returns TW_ETOOBIG and
 * writes nothing.
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  Every call reuses the same array
 * (it clears the work counter itself), so calls that overlap on the GPU race
 * and corrupt each other's results: serialise them. */
int tw_mag_noalloc(double s, double q, double rho, const double *y1, const double *y2, int64_t n,
                   double rel_tol, double *out, int precision, int max_samples, void *stream);

/* MLP surrogate (not in the paper; a systems pattern of this library).  A
 * BF16 network 8 -> 256 -> 256 -> 256 -> 256 -> 2 maps (log10 s, log10 q,
 * log10 rho, y1, y2) and three features of the point-source expansion of the
 * same query to (r, l).  The expansion is the hexadecapole approximation
 * A_hex of the finite-source magnification from point-source magnifications
 * (images of Eq. 6, Jacobian of Eq. 7) at the source centre and at 8 points
 * on rings of radius rho/2, rho and 2 rho; its features are the decade of its
 * error estimate, the signed gap between its (rho/2, rho) and (rho, 2 rho)
 * values in units of that estimate, and the signed size of the finite-source
 * correction.  The network predicts mu = A_hex (1 + gap / 15) exp(r) (the
 * factor is the Richardson step between the two ring pairs) with
 * uncertainty sigma = exp(l) in ln mu; the hidden layers run on the tensor
 * cores.
 *
 * tw_surrogate_train draws nsamples positions near caustics (a random point of
 * a random branch of the caustic of a random lens with log10 s ~ U[-0.5, 0.5],
 * log10 q ~ U[-5, -1], log10 rho ~ U[-4, -2], displaced uniformly within three
 * times that branch's size) from `seed`.  The network's band is the positions
 * not flagged as near a caustic (see tw_surrogate_mag) whose expansion error
 * estimate lies in (2.5e-5, 2e-3]: below half of a 1e-4 tolerance the
 * expansion answers by itself, and the bound keeps the correction the
 * network adds small.  Those are labelled by contour integration (FP64,
 * rel_tol 1e-6) in draw order; the last tenth is held out, the rest (a
 * multiple of 4096) trains for `epochs` epochs (Gaussian likelihood of the
 * standardised r, Adam, batch 4096, cosine learning rate).  The held-out rows
 * calibrate kappa_cal: the 99.9% quantile of |r - r_net| / sigma (at least
 * 3), raised until every held-out row it would answer at rel_tol 1e-4 is
 * within 2.5e-5.  The weights file holds magic, shapes, the standardisation record
 * (inputs, target, kappa_cal, band), FP32 weights and a checksum.  stats
 * (optional, [9]): positions drawn, positions in the band, training rows,
 * mean loss of the last epoch, spread of the targets, held-out rows,
 * kappa_cal, the fraction of held-out rows the network would answer at
 * rel_tol 1e-4 and the largest error in ln mu among them.  TW_EINVAL if the
 * band holds fewer than 4096 training or 128 held-out rows.  Synchronous. */
int tw_surrogate_train(const char *weights_path, int64_t nsamples, uint64_t seed, int epochs, double *stats,
                       const tw_opts *opts);

/* Surrogate magnification of n queries with per-query lens and source radius
 * (arrays s, q, rho, y1, y2; host or device, all of one kind).  A query is
 * flagged as near a caustic when the caustic, swept at 64 angles, comes
 * within 4 rho of the centre, the image count differs between the centre and
 * a ring point, min |J| < 0.01 at the centre, or the expansion's error
 * estimate exceeds 5% of the value.  An unflagged query is answered without
 * contour integration by the expansion (mu = A_hex) when its error estimate
 * (the gap between its values from the rings (rho/2, rho) and (rho, 2 rho),
 * floored at a twentieth of the finite-source correction |A_hex - A_0|) is
 * below 0.5 rel_tol, else by the network when the estimate lies in the
 * network's band (2.5e-5, 2e-3] and max(kappa, kappa_cal) * sigma <=
 * rel_tol.  All other
 * queries fall back to contour integration (one persistent launch over them,
 * with opts->precision and opts->max_samples).  out[i] receives mu; counts
 * (optional, [5]) the number of fallbacks, of queries answered by the
 * network, of queries answered by the expansion, and the fallbacks split
 * into those flagged as near a caustic and the unflagged ones that neither
 * the expansion nor the network answered.  opts->pos_status (optional, [n],
 * the kind of the other arrays) receives TW_POS_EXPANSION or TW_POS_NETWORK
 * for answered queries and the contour status bits for fallbacks.  n < 2^31.
 * Synchronous.  The library keeps the call's device buffers for the next
 * call on the device. */
int tw_surrogate_mag(const char *weights_path, const double *s, const double *q, const double *rho,
                     const double *y1, const double *y2, int64_t n, double rel_tol, double kappa, double *out,
                     int64_t *counts, const tw_opts *opts);

/* Timing and work of the latest tw_surrogate_mag call on the current device
 * (the paper has no counterpart; a measurement hook of this library):
 * out[0] device milliseconds of the feature kernels (point images at the
 * centre and on three rings, caustic sweep, expansion), out[1] of the
 * network (input layer, three tensor-core GEMMs, head), out[2] of the three
 * GEMMs alone, each from CUDA events on the call's stream; out[3] point
 * solves, out[4] FP32 Aberth sweeps of those solves, out[5] FP64 Newton root
 * steps, out[6] Aberth iterations of the caustic sweep, out[7] GEMM rows
 * (queries padded to a multiple of 128).  TW_EINVAL if no call completed. */
int tw_last_surrogate_stats(double out[8]);

/* The training-position sampler of tw_surrogate_train, on its own: n seeded
 * positions near caustics into device arrays (asynchronous on `stream`). */
int tw_surrogate_sample(uint64_t seed, int64_t n, double *s, double *q, double *rho, double *y1, double *y2,
                        void *stream);

/* Magnification with a point-source adequacy gate (not in the paper, which
 * leaves such tests to other codes, Sec. 2.3; the expansion is the
 * hexadecapole approximation of Gould 2008 with the error estimate and
 * near-caustic flag of tw_surrogate_mag, without the network).  For each
 * position (per-position lens and radius, as tw_mag_multi) the point-source
 * images at the centre and on three rings give the finite-source expansion
 * and its error estimate; a position not flagged as near a caustic whose
 * estimate is within rel_tol / 2 takes the expansion's value, every other
 * position is integrated by contour (one persistent launch, opts->precision
 * and opts->max_samples).  *n_contour (optional) receives the number of
 * contour-integrated positions.  Host or device arrays (all of one kind);
 * synchronous.  n < 2^31.  The library keeps the call's device buffers
 * (about 60 B per position, plus 48 B per position for host arrays) for the
 * next call on the same device. */
int tw_mag_gated(const double *s, const double *q, const double *rho, const double *y1, const double *y2, int64_t n,
                 double rel_tol, double *out, int64_t *n_contour, const tw_opts *opts);

/* C[M][N] = A[M][K] . B[N][K]^T on the tensor cores (tcgen05.mma, BF16
 * inputs, FP32 accumulation and output), the GEMM of the MLP surrogate; the
 * paper has no counterpart.  A, B (bf16, row-major, K contiguous) and C
 * (float32, row-major) are device pointers; M and N multiples of 128, K a
 * multiple of 64.  Synchronous on `stream`.  TW_ETIMEOUT if a bounded
 * device-side wait gave up (C is then undefined). */
int tw_gemm_bf16(const void *A, const void *B, int M, int N, int K, float *C, void *stream);

/* Text of a return code (TW_OK, TW_E*, TW_WCAP). */
const char *tw_status_str(int code);

/* Library version (major * 10000 + minor * 100 + patch). */
int tw_version(void);

/* Work done by the most recent launch on the current device (waits for it):
 * out[0] limb samples, out[1] FP64 Aberth sweeps (five roots each), out[2]
 * FP32 Aberth sweeps, out[3] edge evaluations (image linking + area + error),
 * out[4] FP64 Newton passes over the five roots (zero: the mixed-precision
 * polish is counted in out[1] as FP64 Aberth sweeps).
 * These are the units of the FLOP accounting of the roofline report; the
 * paper has no counterpart (it reports no operation counts). */
int tw_last_launch_work(int64_t out[5]);

/* Device time, in milliseconds, of the most recent contour integration on
 * the current device (every entry point above that integrates contours,
 * including the fallback of tw_surrogate_mag): its main kernel and its
 * slope-repair kernel, measured by two CUDA events recorded on the launch's
 * stream directly before and after them; waits for it.  TW_EINVAL if no launch has been timed.  No
 * counterpart in the paper (a measurement hook of this library). */
int tw_last_launch_ms(float *ms);

/* Measured peak of a CUDA-core arithmetic pipe on the current device, the
 * denominator of the contour kernel's roofline (the paper has no
 * counterpart; a measurement hook): kind 0 FP64 fused multiply-add, kind 1
 * FP32, as FLOP/s (2 per FMA) of a launch of 8 CTAs per SM whose threads run
 * independent FMA chains.  Synchronous on the legacy default stream; about
 * 100 ms. */
int tw_peak_probe(int kind, double *flops_per_s);

/* Device self-test of the library's FP64 reciprocals against IEEE division,
 * over 2^20 values of magnitude 1e-300..1e300: rcp_max_rel_err[0] receives the
 * largest relative difference of the full reciprocal (the hardware
 * approximation refined by two Newton-Raphson steps, used for the residuals,
 * the areas and every other FP64 division), rcp_max_rel_err[1] that of the
 * one-step reciprocal used for the Aberth correction (about 40 bits).
 * Synchronous.  The paper has no counterpart. */
int tw_selftest(double *rcp_max_rel_err);

/* Device self-test of the library's bounded waits (no counterpart in the
 * paper; a failure-detection hook): one CTA waits on an mbarrier that nothing
 * arrives on, with poll_limit polls (1..2^24), through the wait routine of
 * the tensor-core GEMM, and gives up.  Returns TW_ETIMEOUT when the wait gave
 * up and reported it (the expected outcome), TW_OK if it did not.
 * Synchronous on the legacy default stream; the context stays usable. */
int tw_selftest_timeout(unsigned int poll_limit);

/* Device self-test of the slope test and its repair (Sec. 2.4.2) on a planted
 * misjudgment.  The limb of the source (s, q <= 1, rho, centre y1, y2) is
 * sampled at the n (8..256) host angles theta[] (ascending, in [0, 2 pi)),
 * which must include closely spaced samples (steps < 1e-3) across a caustic
 * crossing; every edge is linked and integrated.  Then the ghost pair of
 * three-image samples next to that crossing is declared real: mode 1 the
 * sample adjacent to the crossing (the crossing moves by one sample), mode 2
 * the two samples beyond it (a false image piece).  out4[0] = 1 when the
 * planted crossing failed the slope test, out4[1] = 1 when the repair gave
 * back the original classification of every sample, out4[2] = relative
 * change of the total area after the repair (-1 when no crossing was found),
 * out4[3] = theta position of the crossing found (-1 none).  Synchronous;
 * the paper has no counterpart (a test hook of this library). */
int tw_selftest_slope(double s, double q, double rho, double y1, double y2, const double *theta, int n, int mode,
                      double *out4);

#ifdef __cplusplus
}
#endif

#endif /* TWINKLE_GB300_H */
