/*
 * cher.h -- C ABI of the GB300 (sm_103a) Cherenkov bunch library.
 *
 * The library runs the data-parallel hot path of air-shower Cherenkov light
 * simulation that Arrabito et al. profile and optimise for CORSIKA/iact
 * ("Optimizing Cherenkov photons generation and propagation in CORSIKA for
 * CTA Monte-Carlo simulations"):
 *
 *   a0  atmosphere tables, built once: the index of refraction on a uniform
 *       fine grid (the paper's "fast interpolation", section 3.3.2) and
 *       refraction-correction tables over height and zenith angle (the
 *       "coefficients for air refraction correction" of section 3.3.1);
 *   a1  per track step: Cherenkov angle and Frank-Tamm photon yield, split
 *       into bunches of about five photons, one per sub-step (CERENK,
 *       section 3.2 and Appendix A);
 *   a2  per bunch: emission point, azimuth and wavelength from a
 *       counter-based Philox4x32-10 stream keyed by (seed, track, bunch), so
 *       that every run and every code version draws the same randoms
 *       (section 5.2);
 *   a3  per bunch: refraction and propagation to the observation level
 *       (RAYBND, section 3.2 and the Appendix B listing), rare conditions
 *       tested first (Algorithms 1-2);
 *   a4  per bunch: fiducial telescope spheres (TELOUT, section 2 and
 *       Appendix A), candidates found through a ground grid;
 *   a5  compaction of the bunches that cross a sphere into per-telescope
 *       record buffers.
 * All steps a1-a5 run in the library's CUDA kernels; a0 runs on the host
 * once per context.
 *
 * Conventions.  Lengths in m, heights above sea level with z pointing up,
 * times in ns, kinetic energies in MeV, wavelengths in nm.  Every function
 * returns a cher_status and never aborts, traps or prints.  Pointers marked
 * "device" must be CUDA device memory (for example from PyTorch) and stay
 * owned by the caller; the context owns only its tables, its telescope grid
 * and a few bytes of scratch.  Functions taking a stream are asynchronous
 * on that stream (NULL = legacy default stream) and do not synchronise.
 * A context is not thread safe: calls on one context must be serialised by
 * the caller; distinct contexts are independent.
 */
#ifndef CHER_H
#define CHER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cher_status {
    CHER_OK = 0,
    CHER_EINVAL = 1,     /* a NULL pointer, a bad size or a bad parameter   */
    CHER_ENOMEM = 2,     /* host or device allocation failed                */
    CHER_ECUDA = 3,      /* a CUDA runtime call failed                      */
    CHER_ESTATE = 4,     /* refraction tables not built yet                 */
    CHER_ERANGE = 5,     /* a size exceeds what the library supports        */
    CHER_EOVERFLOW = 6,  /* a telescope buffer ran out of capacity          */
    CHER_ETIMEOUT = 7,   /* a bounded device-side wait gave up              */
    CHER_EBOUNDS = 8     /* bounds-checked build only: a kernel index check
                            failed (stats[CHER_STAT_DEBUG] says which)      */
} cher_status;

/* Text for a status code (static storage, never NULL). */
const char *cher_status_string(cher_status s);

typedef enum cher_precision {
    CHER_FP64 = 0,       /* everything in double precision                  */
    CHER_FP32_BULK = 1   /* per-bunch arithmetic in single precision; the
                            photon yield (hence the bunch count) and the
                            per-step reference times stay in double         */
} cher_precision;

/* Layered atmosphere: thickness T(h) = a[i] + b[i] exp(-h / c[i]) (g/cm^2,
 * c in m) in layer i, h in [h_bound[i], h_bound[i+1]); the lowest layer
 * extends below h_bound[0] and there is no air above h_bound[5].  The
 * density is rho = -dT/dh and n(h) - 1 = n0_minus_1 rho(h) / rho(0)
 * (section 3.3.1: density, thickness and refractive index versus altitude).
 * Requires c[i] > 0, b[i] >= 0, increasing h_bound, 0 <= n0_minus_1 < 0.01. */
typedef struct cher_atmosphere {
    double h_bound[6];
    double a[5], b[5], c[5];
    double n0_minus_1;
} cher_atmosphere;

/* A fiducial sphere: centre (x, y, h_obs + z), radius r > 0 (section 2). */
typedef struct cher_telescope {
    double x, y, z, r;
} cher_telescope;

/* Options fixed at creation.  Zero fields take the defaults in brackets. */
typedef struct cher_options {
    double bunch_size;       /* photons per bunch at most [5] (Appendix A)   */
    double lambda_min_nm;    /* wavelength band [300, 600] nm               */
    double lambda_max_nm;
    int32_t n_fine;          /* points of the fine n(h) table [10000]
                                (section 3.3.2), 2..1048576                 */
} cher_options;

typedef struct cher_ctx cher_ctx;

/* Create a context on the current CUDA device.
 *   atm       atmosphere (host, copied)
 *   h_obs     observation level, m a.s.l., inside the atmosphere
 *   tel       n_tel telescopes (host, copied); 1 <= n_tel <= 4096
 *   opt       options (host, copied) or NULL for the defaults
 *   out       receives the new context
 * Errors: CHER_EINVAL for bad arguments, CHER_ENOMEM. */
cher_status cher_create(const cher_atmosphere *atm, double h_obs,
                        const cher_telescope *tel, int32_t n_tel,
                        const cher_options *opt, cher_ctx **out);

/* Build (or rebuild) all atmosphere tables on the host in double precision
 * and upload them (one blocking copy per table):
 *   - eta = n - 1 at n_fine uniform heights on [0, h_max];
 *   - refraction tables over n_heights uniform heights on [h_obs, h_max]
 *     and n_zenith observation-level zenith angles whose squared sines are
 *     uniform on [0, sin^2(zenith_max_deg)], holding the horizontal offset
 *     and optical path of the refracted ray minus those of the straight line
 *     at the same observation zenith, each divided by its leading angular
 *     factor (sin/cos^3 and 1/cos^3); a photon arriving steeper than
 *     zenith_max_deg, or emitted above h_max, is counted and dropped;
 *   - the ground grid of telescope candidates.
 * Requires 2 <= n_heights <= 65536, 2 <= n_zenith <= 4096,
 * 0 < zenith_max_deg < 85, h_obs < h_max <= h_bound[5].
 * Errors: CHER_EINVAL, CHER_ERANGE (table too large), CHER_ENOMEM,
 * CHER_ECUDA. */
cher_status cher_build_refraction_tables(cher_ctx *ctx, int32_t n_heights,
                                         int32_t n_zenith,
                                         double zenith_max_deg, double h_max);

/* Release everything the context owns (NULL is accepted). */
cher_status cher_destroy(cher_ctx *ctx);

/* Track steps, structure of arrays, all device pointers with n elements.
 * Step i starts at (x0, y0, z0) at time t0, runs len along the unit
 * direction (ux, uy, uz), for an e+- of kinetic energy ekin.  The direction
 * arrays are float for CHER_FP32_BULK and double for CHER_FP64.
 * shower (optional, NULL = all 0) indexes t_ref (optional, NULL = 0): the
 * arrival times are reported relative to t_ref[shower[i]].
 * track_base is the global index of step 0: the Philox counter of bunch j
 * of step i is (track_base + i, j), so any split of a track list into calls
 * reproduces the same bunches. */
typedef struct cher_tracks {
    const double *x0, *y0, *z0, *t0, *len, *ekin;
    const void *ux, *uy, *uz;
    const uint32_t *shower;
    const double *t_ref;
    int32_t n_showers;
    int64_t n;
    int64_t track_base;
} cher_tracks;

/* Number of counters in cher_output.stats and their meaning. */
#define CHER_NSTATS 16
enum {
    CHER_STAT_STEPS = 0,        /* steps processed                          */
    CHER_STAT_EMITTING = 1,     /* steps above the Cherenkov threshold      */
    CHER_STAT_INVALID = 2,      /* steps with a non-finite or negative field */
    CHER_STAT_BUNCHES = 3,      /* bunches generated (sum of nb)            */
    CHER_STAT_UPWARD = 4,       /* dropped: not travelling downward         */
    CHER_STAT_BELOW_OBS = 5,    /* dropped: emitted below h_obs             */
    CHER_STAT_ABOVE_MAX = 6,    /* dropped: emitted above h_max             */
    CHER_STAT_ANGLE = 7,        /* dropped: zenith beyond the tables        */
    CHER_STAT_GROUND = 8,       /* reached the observation level            */
    CHER_STAT_HITS = 9,         /* (bunch, telescope) crossings found       */
    CHER_STAT_OVERFLOW = 10,    /* crossings not stored (buffer full)       */
    CHER_STAT_ABSORBED = 11,    /* reached h_obs, lost to the transmission  */
    CHER_STAT_FALLBACK = 12,    /* propagated by the beyond-table fallback  */
    CHER_STAT_FB_LOST = 13,     /* past the tables' range, the fallback     */
                                /* queue full: not propagated              */
    CHER_STAT_DEBUG = 14        /* bounds-checked build (compiled with      */
                                /* CHER_DEBUG) only: bit mask of the index  */
                                /* checks that failed (1 fine eta table, 2  */
                                /* refraction tables, 4 grid and candidates, */
                                /* 8 record buffers, 16 trace arrays, 32    */
                                /* shared step constants and offsets, 64    */
                                /* fallback queue); the access is skipped   */
                                /* (index 0 taken instead), nothing traps.  */
                                /* Always 0 in the regular build.           */
};

/* Per-telescope output buffers (device).  Telescope k owns records
 * [k * cap_per_tel, (k + 1) * cap_per_tel).  Record r holds
 *   pos[4 r + 0..3] = x, y, cx, cy
 *   tim[4 r + 0..3] = t, z_emit, photons, lambda_nm
 *   key[r]          = (track_base + i) << 32 | j
 * where (x, y) is where the arrival line crosses the horizontal plane
 * through the sphere centre, relative to the centre; (cx, cy) are the
 * direction cosines at the observation level; t is the arrival time at
 * that plane minus t_ref; z_emit the emission height.  pos and tim are
 * float for CHER_FP32_BULK and double for CHER_FP64, 16-byte (32-byte for
 * double) aligned.  The order of records inside a telescope is not
 * deterministic: sort by key.  count[k] receives the number of crossings
 * found for telescope k, which may exceed cap_per_tel (then only
 * cap_per_tel are stored and the rest counted in stats[OVERFLOW]).
 * count and stats are cleared by every call. */
typedef struct cher_output {
    void *pos;
    void *tim;
    uint64_t *key;
    int64_t cap_per_tel;
    unsigned long long *count;   /* [n_tel]       */
    unsigned long long *stats;   /* [CHER_NSTATS] */
} cher_output;

/* The whole hot path (a1-a5) for n steps in one launch: a persistent,
 * tile-scheduled kernel whose CTAs pull tiles of steps from an atomic queue
 * in the context's scratch word.  Asynchronous on `stream`; the return value
 * reports argument checks and the launch only.  Errors: CHER_EINVAL,
 * CHER_ESTATE, CHER_ERANGE (n > 2^40), CHER_ECUDA. */
cher_status cher_generate_propagate(cher_ctx *ctx, const cher_tracks *tracks,
                                    uint64_t seed, cher_precision prec,
                                    const cher_output *out, void *stream);

/* Longitudinal profile of Cherenkov production (CERLDE; paper section 4:
 * the simulation optionally keeps the number of photons produced versus
 * atmospheric depth, which follows the density profile, and the paper
 * vectorised it with the generation).  The paper gives no formula.  Here a
 * step spreads its photons N uniformly along its straight path, and a
 * photon counts at the atmospheric depth of its emission point,
 * X = T(h) / axis_cos[shower] in g/cm^2 (T the thickness of the layered
 * atmosphere; axis_cos = NULL gives the vertical depth T(h)).  Bin k of a
 * shower's row holds the depths [k bin_gcm2, (k + 1) bin_gcm2); a step adds
 * N times the fraction of its path whose depth falls in bin k.  Photons
 * deeper than the last bin, and steps whose shower index has no row, are
 * not counted.
 *   profile  : device, double [max(n_showers, 1)][n_bins], ADDED to (clear
 *              it before the first call of a batch), 8-byte aligned;
 *   n_bins   : 1 .. 65536, and max(n_showers, 1) * n_bins < 2^31;
 *   bin_gcm2 : finite and > 0;
 *   axis_cos : device, double [max(n_showers, 1)] with values in (0, 1],
 *              or NULL.
 * The sums are FP64 atomic additions, so their rounding order varies from
 * call to call. */
typedef struct cher_profile {
    double *profile;
    int32_t n_bins;
    double bin_gcm2;
    const double *axis_cos;
} cher_profile;

/* cher_generate_propagate plus, when `profile` is not NULL, the
 * longitudinal production profile of the same steps, accumulated in the
 * same launch (per step, from the yield the launch computes).  Errors as
 * cher_generate_propagate; CHER_EINVAL for a profile whose fields are out
 * of range. */
cher_status cher_generate_propagate_ex(cher_ctx *ctx, const cher_tracks *tracks,
                                       uint64_t seed, cher_precision prec,
                                       const cher_output *out, const cher_profile *profile,
                                       void *stream);

/* Shower steps from a parameterised electromagnetic shower, generated on
 * the device (an extension, no counterpart in the paper: its input are the
 * EGS4 electron/positron steps CORSIKA hands to CERENK; this stands in for
 * them so that a batch of showers needs no step arrays from the host).  Per
 * shower: primary energy, axis, core at h_obs and a step count; the steps
 * of shower s follow those of shower s - 1.  Per step g, eight deviates of
 * Philox4x32-10 keyed by `seed`, counters (g, 0, 1) and (g, 1, 1): the
 * depth from the Greisen longitudinal profile (y = ln(E0 / 85 MeV), in
 * isothermal air X = 1030 exp(-h / 8000 m) g/cm^2, X0 = 36.7 g/cm^2, by
 * inverting its CDF tabulated on 1024 uniform depth nodes), the height on
 * the axis (at most 29999 m), an exponential lateral offset of mean 50 m at
 * a uniform azimuth, a log-uniform kinetic energy over 20 MeV - 5 GeV, a
 * direction spread around the axis by Box-Muller normals of width
 * 3 deg x 50 MeV / E, a start time (s_ref - s)/c along the axis (s_ref the
 * distance from 30 km to h_obs) and a length uniform in [1, 20] m.  Per-step
 * arithmetic in FP32 (outputs widened).
 *   showers     : host, n_showers entries, e0_mev > 85, zenith in [0, pi/2),
 *                 finite azimuth and core, n_steps >= 0 (total <= 2^40);
 *   out         : device arrays of the total step count (x0 .. ekin double,
 *                 ux, uy, uz float for CHER_FP32_BULK or double for
 *                 CHER_FP64, shower uint32) and t_ref[n_showers] double (the
 *                 time the axis reaches h_obs), 8-byte aligned.
 * The context holds the per-call tables in its scratch: calls on one
 * context must not overlap on different streams.  Asynchronous on
 * `stream`: the tables (a few KB per shower) go up from the context's
 * pinned staging, and a call first waits, on the host, for the previous
 * call's upload to have read that staging.  Errors: CHER_EINVAL,
 * CHER_ERANGE, CHER_ENOMEM, CHER_ECUDA. */
typedef struct cher_shower {
    double e0_mev;
    double zenith, azimuth;
    double core_x, core_y;
    int64_t n_steps;
} cher_shower;

typedef struct cher_step_buffers {
    double *x0, *y0, *z0, *t0, *len, *ekin;
    void *ux, *uy, *uz;
    uint32_t *shower;
    double *t_ref;
} cher_step_buffers;

cher_status cher_generate_steps(cher_ctx *ctx, const cher_shower *showers, int32_t n_showers,
                                uint64_t seed, cher_precision prec,
                                const cher_step_buffers *out, void *stream);

/* The double -> float rounding that the FP32 path applies to its FP64
 * inputs (positions, lengths, energies, the differences to h_obs and
 * t_ref): round to nearest even, done on the integer pipes because GB300
 * converts on its slow FP64 pipe; results below the smallest normal float
 * flush to zero, beyond the largest float they become infinities.  The
 * paper has no counterpart; it is exposed so that the rounding can be
 * checked against the IEEE conversion.  in, out: device arrays of n
 * elements (n >= 0), 8- and 4-byte aligned; asynchronous on `stream`.
 * Errors: CHER_EINVAL (NULL array with n > 0, n < 0), CHER_ECUDA. */
cher_status cher_round_to_float(const double *in, float *out, int64_t n, void *stream);

/* The float pair the FP32 path splits its FP64 time and height differences
 * into (t0 - t_ref and z0 - h_obs, tens of km and ~1e5 ns), so that its
 * arrival time is summed in float-float: hi = the rounding above and lo the
 * float nearest to in - hi (0 where that would not be a normal float), on
 * the integer pipes.  The paper has no counterpart; exposed for its test.
 * in, hi, lo: device arrays of n elements (n >= 0), 8- and 4-byte aligned;
 * asynchronous on `stream`.  Errors: CHER_EINVAL, CHER_ECUDA. */
cher_status cher_split_to_float(const double *in, float *hi, float *lo, int64_t n,
                                void *stream);

/* The same hot path as cher_generate_propagate (same kernel, same results;
 * see below for the one configuration it refuses) for callers that must
 * not allocate device memory when they run it: pipelines whose device
 * memory is all held by another allocator (a framework's caching pool), and
 * real-time loops that forbid allocation after start-up.  The paper has no
 * counterpart.  The context must have been created and its tables built
 * beforehand; this call allocates nothing and does not use the context's own
 * scratch word.  The persistent kernel's only scratch, its 8-byte tile
 * counter, lives in a fixed 256-byte device array compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 * The first call on each device looks the array's device address up (with
 * that device current).
 * Every call shares the array and clears the counter before its launch:
 * calls that overlap on the GPU (different streams, or several contexts)
 * race on it and must be serialised by the caller.  A step count above
 * 2^40, the library-wide limit, is refused with CHER_ERANGE before anything
 * is launched.  A context whose beyond-table fallback is active
 * (cher_set_fallback past the tables' zenith range, flat layers) is refused
 * with CHER_EINVAL before anything is launched: that fallback queues its
 * bunches in memory the context allocates, and without it those bunches
 * would be dropped where cher_generate_propagate propagates them.  Other
 * errors as cher_generate_propagate. */
cher_status cher_generate_propagate_noalloc(cher_ctx *ctx, const cher_tracks *tracks,
                                            uint64_t seed, cher_precision prec,
                                            const cher_output *out, void *stream);

/* A cher_generate_propagate call captured once into an executable CUDA
 * graph (the counter clears and the persistent kernel), for replaying the
 * same batch of showers with one launch (the batched, graph-captured launch
 * of the independent-shower parallelism of section 2).  The graph keeps the
 * pointers of `tracks` and `out`: the caller keeps those buffers alive and
 * may change their contents between launches, not their addresses.
 * Errors as cher_generate_propagate; CHER_ECUDA if capture fails. */
typedef struct cher_graph cher_graph;
cher_status cher_graph_create(cher_ctx *ctx, const cher_tracks *tracks, uint64_t seed,
                              cher_precision prec, const cher_output *out,
                              cher_graph **graph);
/* Launch the captured graph on `stream` (asynchronous). */
cher_status cher_graph_launch(cher_graph *graph, void *stream);
/* Release the graph (NULL is accepted). */
cher_status cher_graph_destroy(cher_graph *graph);

/* Synchronise `stream`, read out->stats and report CHER_EBOUNDS if an index
 * check of the bounds-checked build failed, else CHER_EOVERFLOW if a
 * telescope buffer overflowed during the last call, else CHER_OK (or
 * CHER_ECUDA if the stream reports an error).  stats_host (optional,
 * CHER_NSTATS entries) receives the counters. */
cher_status cher_sync_status(cher_ctx *ctx, const cher_output *out,
                             unsigned long long *stats_host, void *stream);

/* Launch shape of cher_generate_propagate.  block_threads in {128, 256,
 * 512} is also the number of steps per tile; ctas_per_sm in 0..10 sets the
 * persistent grid (0 = one CTA per tile, no persistence; above 8 only with
 * 128-step tiles in the FP32 path, which has builds for 9 and 10 CTAs per SM
 * with fewer registers per thread; other launches cap at what fits).  A
 * new context starts at 128 / 8 (32 resident warps per SM); cher_autotune
 * measures the shapes on the caller's input and keeps the fastest.  Errors:
 * CHER_EINVAL. */
cher_status cher_set_launch(cher_ctx *ctx, int32_t block_threads,
                            int32_t ctas_per_sm);
cher_status cher_get_launch(const cher_ctx *ctx, int32_t *block_threads,
                            int32_t *ctas_per_sm);

/* ---- differentiable read-out and its adjoint ---------------------------
 * No counterpart in the paper (its path is a forward simulation); these
 * make the path differentiable.  For telescope k and smoothing length sigma
 *   S_k = sum_b w_b G(r_bk),  U_k = sum_b w_b G(r_bk) t_b,
 *   G(r) = exp(-r^2 / (2 sigma^2)) / (2 pi sigma^2) for r < 6 sigma, else 0,
 * over the bunches b that reach the ground, r_bk the distance in the
 * observation plane from the bunch's ground point to the centre (x_k, y_k),
 * w_b its photons, t_b its arrival time (relative to t_ref):
 *   D_k = S_k (photons per m^2),  Tbar_k = U_k / S_k (0 where S_k = 0).
 * nb_frozen (device, n int32, optional) fixes the bunch counts so that the
 * read-out is smooth in the parameters; NULL takes this call's yield.  The
 * bunches within 6 sigma of a centre are listed in an FP32 pass over all
 * bunches, then recomputed one thread each (precision as `prec`) from
 * their Philox counters; sums and gradients accumulate in FP64.  Both calls
 * synchronise `stream` and use scratch the context allocates on first use.
 * n must be below 2^31.  Errors: CHER_EINVAL, CHER_ESTATE, CHER_ERANGE,
 * CHER_ENOMEM, CHER_ECUDA.
 *
 * cher_density: D and Tbar (device, n_tel doubles each). */
cher_status cher_density(cher_ctx *ctx, const cher_tracks *tracks, uint64_t seed,
                         cher_precision prec, double sigma, const int32_t *nb_frozen,
                         double *D, double *Tbar, void *stream);

/* cher_adjoint: for L = sum_k dL_dD[k] D_k + dL_dT[k] Tbar_k (device inputs,
 * n_tel doubles each) the gradients
 *   grad_atm[15]    dL/d(a_0..a_4, b_0..b_4, c_0..c_4) of cher_atmosphere
 *                   (n depends on b and c only: the a entries are 0),
 *   grad_tracks[6n] dL/dx0, dL/dy0, dL/dz0, dL/dux, dL/duy, dL/duz per step,
 *                   stored as six consecutive arrays of n,
 * both device, overwritten.  The direction components are differentiated as
 * independent inputs (no renormalisation). */
cher_status cher_adjoint(cher_ctx *ctx, const cher_tracks *tracks, uint64_t seed,
                         cher_precision prec, double sigma, const int32_t *nb_frozen,
                         const double *dL_dD, const double *dL_dT, double *grad_atm,
                         double *grad_tracks, void *stream);

/* Atmospheric transmission (an extension of the propagation: the paper
 * notes that CORSIKA works with external atmospheric profiles).  With a
 * table set, a bunch that reaches the observation level survives with
 * probability P = exp(-tau / cos(theta_obs)) -- Beer-Lambert along the
 * arrival direction through a flat atmosphere -- and is otherwise counted
 * in stats[CHER_STAT_ABSORBED] and not recorded (trace status 5).  tau is
 * the vertical optical depth between the emission height and h_obs at the
 * bunch's wavelength, interpolated bilinearly in the table and clamped to
 * its range.  The draw is the bunch's fourth Philox deviate u3: it survives
 * when u3 < P, so the same seed gives the same survivors in every code
 * version.
 *   tau       : host, [n_lambda][n_height], finite and >= 0, copied;
 *   node a, b : lambda_a = lambda_min + a (lambda_max - lambda_min) / (n_lambda - 1),
 *               h_b = h_min + b (h_max - h_min) / (n_height - 1);
 *   n_lambda, n_height: 2 .. 4096.
 * NULL removes the table.  Blocking.  Errors: CHER_EINVAL, CHER_ENOMEM,
 * CHER_ECUDA. */
typedef struct cher_transmission {
    int32_t n_lambda, n_height;
    double lambda_min_nm, lambda_max_nm;
    double h_min, h_max;
    const double *tau;
} cher_transmission;

cher_status cher_set_transmission(cher_ctx *ctx, const cher_transmission *table);

/* Beyond-table fallback (the paper's rare-case scalar path, section 3.3.1:
 * the few photons that do not fit the vectorised code take the scalar
 * one).  Bunches whose observation-level zenith lies past the refraction
 * tables' range but within `zenith_max_deg` are propagated by the ray
 * integrals themselves -- n(h) sin(theta(h)) = n_obs sin(theta_obs) in the
 * layered atmosphere, D = int tan(theta) dh, L = int n / cos(theta) dh,
 * 12-point Gauss-Legendre on each layer's part, in FP64 on the FP64 path
 * and in FP32 on the FP32 path (there as the straight line at the arrival
 * zenith plus the integrals of the small corrections) -- instead of being
 * dropped (stats[CHER_STAT_ANGLE]).  The generation launch queues them and
 * a second kernel on the same stream propagates them (stats
 * [CHER_STAT_FALLBACK]); the queue holds `queue_records` bunches per call
 * (0: max(2^20, 4 x the call's steps); 64 B each in FP32, 112 B in FP64,
 * allocated on the first call that needs them), the rest counted in
 * stats[CHER_STAT_FB_LOST].  Trace launches integrate them in place.  The
 * adjoint, the allocation-free launch and the curved atmosphere do not use
 * it (those bunches stay dropped there).
 *   zenith_max_deg: 0 (off) or in (the tables' zenith range, 85];
 *   queue_records : 0 or up to 2^34.
 * Errors: CHER_EINVAL. */
cher_status cher_set_fallback(cher_ctx *ctx, double zenith_max_deg, int64_t queue_records);

/* Wavelength-dependent index of refraction (an extension: the paper's
 * CERENK and RAYBND take n independent of the wavelength).  With kappa set,
 *     n(h, lambda) - 1 = (n(h) - 1) kappa(lambda),
 * n(h) the atmosphere's index (n0_minus_1 at the reference wavelength) and
 * kappa linear in the wavenumber 1/lambda between k nodes, node m at
 *     1/lambda_m = 1/lambda_min - m (1/lambda_min - 1/lambda_max) / (k - 1)
 * (node 0 at the band's short end).  Then, per step, the yield is the
 * Frank-Tamm integral of 1 - 1/(beta n(lambda))^2 over the radiating part of
 * the band (exact: a closed form on each linear piece, the Cherenkov
 * threshold cutting at most one piece); per bunch, the wavelength inverts
 * the step's spectrum with the third Philox deviate (from the short end,
 * like the constant-index 1/lambda^2 draw), the Cherenkov cone, Snell's law
 * and the sphere-plane time use the bunch's own index, and the refraction
 * corrections are interpolated linearly in kappa between tables built for
 * kappa[k-1] and kappa[0] (the context's table sizes; rebuilt with the
 * tables by cher_build_refraction_tables and cher_set_atmosphere).
 *   kappa : host, k values, finite, > 0 and not increasing with m (normal
 *           dispersion: n falls towards long wavelengths), copied;
 *           kappa[0] n0_minus_1 < 0.01;
 *   k     : 2 .. CHER_DISPERSION_MAX_NODES; kappa NULL or k = 0 turns it off.
 * Launches with it run 128-step tiles whatever cher_set_launch chose.  The
 * read-out and its adjoint refuse a context with it (CHER_EINVAL).
 * Blocking.  Errors: CHER_EINVAL, CHER_ESTATE (tables not built yet),
 * CHER_ENOMEM, CHER_ECUDA. */
#define CHER_DISPERSION_MAX_NODES 9
cher_status cher_set_dispersion(cher_ctx *ctx, const double *kappa, int32_t k);

/* Pack the records of every telescope contiguously, telescope after
 * telescope (the order within a telescope as written), so that they come
 * down in one copy per array instead of one per telescope (TELOUT's output,
 * paper Appendix A, is one stream of records).
 *   out         : the buffers and counts of a generation launch (device);
 *                 counts are clipped to cap_per_tel;
 *   prec        : the precision the launch wrote (record layout: 16 B or 32 B
 *                 for pos and tim);
 *   max_records : room in the destinations (records);
 *   dst_pos, dst_tim, dst_key: device, max_records records each;
 *   tel_offset  : device, n_tel + 1 int64: the first packed record of each
 *                 telescope; tel_offset[n_tel] is the total, which may exceed
 *                 max_records (the records past it are not copied).
 * Asynchronous on `stream` (after the launch that wrote `out`).  Errors:
 * CHER_EINVAL, CHER_ECUDA. */
cher_status cher_pack_records(cher_ctx *ctx, const cher_output *out, cher_precision prec,
                              int64_t max_records, void *dst_pos, void *dst_tim,
                              uint64_t *dst_key, int64_t *tel_offset, void *stream);

/* Curved atmosphere (an extension for large zenith angles: the paper's
 * RAYBND works in flat layers).  With an Earth radius R_E set, positions are
 * Cartesian in the core frame (z up, z = height a.s.l. on the core's
 * vertical), the Earth's centre is (0, 0, -R_E), a point's height is its
 * radial height |x - C| - R_E (the steps' index is taken at the radial
 * height of their midpoint), rays keep Bouguer's invariant n r sin(zeta)
 * (zeta the angle to the local vertical) and end on the observation sphere
 * r_o = R_E + h_obs.  The refraction tables become corrections of the
 * central angle and of the optical path to the straight line with the same
 * arrival zenith (three values per node, a zenith axis uniform in
 * sec(zeta_o), the table sizes of the context) and are rebuilt now if built.
 * Records: the arrival point (X, Y) on the observation sphere, which lies
 * (X^2 + Y^2)/2R_E below the tangent plane; the sphere test and the record
 * plane use that point; z_emit is the radial height; the transmission uses
 * the local zenith.  Telescope z stays relative to the tangent plane at h_obs.
 *   earth_radius_m: 0 (flat layers) or in [1e6, 1e8] m.
 * Launches with it run 128-step tiles; the beyond-table fallback is off in
 * it (build the tables up to 85 degrees instead); the read-out, its adjoint
 * and the production profile refuse it (CHER_EINVAL).  Blocking.  Errors:
 * CHER_EINVAL, CHER_ENOMEM, CHER_ECUDA (the previous geometry is kept). */
cher_status cher_set_curved(cher_ctx *ctx, double earth_radius_m);

/* Replace the atmosphere and, if tables were built, rebuild them with the
 * same sizes (blocking).  Errors as cher_build_refraction_tables. */
cher_status cher_set_atmosphere(cher_ctx *ctx, const cher_atmosphere *atm);

/* The host sensitivity tables of the adjoint on their own (no CUDA call):
 * dax[p][j][k] = d ax[j][k] / d p and dal likewise, for the ten parameters
 * p = b_0..b_4, c_0..c_4, each [10][n_heights][n_zenith].  Errors:
 * CHER_EINVAL. */
cher_status cher_build_sensitivity_host(const cher_atmosphere *atm, double h_obs,
                                        int32_t n_fine, int32_t n_heights, int32_t n_zenith,
                                        double zenith_max_deg, double h_max, double *dax,
                                        double *dal);

/* ---- inspection entry points (same device code, for validation) ------- */

/* a1 only: per-step bunch count nb[i] (int32) and photons per bunch w[i]
 * (double), device outputs of n elements.  Errors as above. */
cher_status cher_segment_yield(cher_ctx *ctx, const cher_tracks *tracks,
                               cher_precision prec, int32_t *nb, double *w,
                               void *stream);

/* a2-a4 for every bunch, not only the crossing ones.  bunch_off (device,
 * n + 1 entries) is the exclusive prefix sum of nb from
 * cher_segment_yield; bunch b = bunch_off[i] + j is written at index b of
 *   pos[4 b ..] = X, Y, cx, cy   (ground point at h_obs, direction)
 *   tim[4 b ..] = t, z_emit, photons, lambda_nm
 *   status[b]   = 0 ground, 1 upward, 2 below h_obs, 3 above h_max,
 *                 4 beyond the zenith range, 5 reached h_obs but lost to
 *                 the atmospheric transmission (no ground point then)
 *   nhit[b], first_hit[b] = number of spheres crossed, lowest index or -1.
 * pos/tim are float (CHER_FP32_BULK) or double (CHER_FP64). */
typedef struct cher_trace {
    void *pos;
    void *tim;
    int32_t *status;
    int32_t *nhit;
    int32_t *first_hit;
    int64_t n_bunches;
} cher_trace;

cher_status cher_trace_bunches(cher_ctx *ctx, const cher_tracks *tracks,
                               uint64_t seed, cher_precision prec,
                               const int64_t *bunch_off, const cher_trace *out,
                               void *stream);

/* Copy the double-precision tables of the context to host arrays:
 * eta[n_fine], ax[n_heights * n_zenith], al[n_heights * n_zenith]
 * (row-major, height first); any pointer may be NULL.  Errors:
 * CHER_ESTATE before cher_build_refraction_tables. */
cher_status cher_get_tables(const cher_ctx *ctx, double *eta, double *ax,
                            double *al);

/* The curved atmosphere's host table builder on its own (no CUDA call):
 * ax, al, ag [n_heights * n_zenith] (row-major, height first) as
 * cher_set_curved builds them, zenith nodes uniform in sec.  Errors:
 * CHER_EINVAL. */
cher_status cher_build_curved_tables_host(const cher_atmosphere *atm, double earth_radius_m,
                                          double h_obs, int32_t n_heights, int32_t n_zenith,
                                          double zenith_max_deg, double h_max, double *ax,
                                          double *al, double *ag);

/* The host table builder on its own (no CUDA call): fills eta[n_fine],
 * ax[n_heights * n_zenith], al[n_heights * n_zenith] exactly as
 * cher_build_refraction_tables does.  Errors: CHER_EINVAL. */
cher_status cher_build_tables_host(const cher_atmosphere *atm, double h_obs,
                                   int32_t n_fine, int32_t n_heights,
                                   int32_t n_zenith, double zenith_max_deg,
                                   double h_max, double *eta, double *ax,
                                   double *al);

/* Measure a few launch shapes of cher_generate_propagate on the given
 * input (which must already be resident) and keep the fastest; if
 * cache_path is not NULL the choice is read from / appended to that file
 * (one line per device name, precision and tile count).  Writes into `out`
 * while measuring.  Errors as cher_generate_propagate, plus CHER_EINVAL if
 * the cache file is unreadable garbage. */
cher_status cher_autotune(cher_ctx *ctx, const cher_tracks *tracks,
                          uint64_t seed, cher_precision prec,
                          const cher_output *out, const char *cache_path,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CHER_H */
