/*
 * bhrt.h -- C ABI of the GB300 (sm_103a) ray tracer for rotating
 * dark-matter-dressed black holes.
 *
 * The method (paper "Adaptive ray tracing, image diagnostics, and photon
 * ring signatures of rotating dark-matter-dressed black holes"):
 *   - rotating Kerr-like metric built from a static lapse H_i(R):
 *     Kerr (H = 1 - 2/R), Einasto-type (Eq. 9), cored-NFW (Eq. 13), with
 *     Sigma, F, Delta of Eqs. (23)-(25) and the Boyer-Lindquist components
 *     of Eqs. (27)-(31);
 *   - outer horizon R_+ = largest root of Delta (Eq. 33), extremal spin
 *     Eqs. (34)-(37), stationary-limit surface (Eqs. 38-41), also as
 *     parameter scans over many spacetimes;
 *   - backward null geodesics from a ZAMO screen (Sec. 3.2, Eqs. 63-74),
 *     integrated as Hamilton's equations (Sec. 3.1, Eqs. 46-62);
 *   - capture / escape (Eq. 75) and equatorial crossings (Sec. 3.3, 4.2)
 *     with transfer maps R_em, phi_em, T_em (Eq. 82);
 *   - redshift g (Eq. 89) for circular emitters (Eqs. 90-91) and the
 *     semi-analytic emissivity (Eqs. 83-87), thin-disk intensity
 *     sum over crossings of g^3 j (reading of Eq. 88), or the
 *     finite-thickness integral of Eq. (88) along the ray;
 *   - the shadow boundary along screen directions (Sec. 4.1, Eqs. 78-79);
 *   - adaptive refinement of the screen near class boundaries
 *     (Introduction and Sec. 4; the rule is a documented reading);
 *   - image diagnostics (Sec. 6.2-6.3, Eqs. 92-107), visibilities
 *     (Sec. 6.4, Eqs. 108-109) and their azimuthally averaged and
 *     horizontal-cut amplitude curves (Sec. 6.4).
 * Equation numbers are the paper's, counted in order of appearance.
 *
 * Conventions for every entry point:
 *   - Units are dimensionless with M = 1 (Eq. 1).
 *   - Struct arguments are HOST pointers.  Every array argument is a DEVICE
 *     pointer owned by the caller unless stated otherwise.  The library
 *     allocates no device memory of its own: scratch space is the caller's
 *     workspace, sized by bh_workspace_size.
 *   - Calls are asynchronous on the given stream (NULL = legacy default
 *     stream).  Argument errors are returned synchronously before anything
 *     is enqueued.  Errors detected on the device (queue overflow, time
 *     budget) are written to a status word in the workspace and returned by
 *     bh_workspace_status after the stream has been synchronised.
 *   - The library never aborts and never prints.  Distinct streams with
 *     distinct workspaces may be used concurrently from several threads.
 *   - Screen: cell-centred grid X_i = x_min + (i + 1/2)(x_max - x_min)/nx,
 *     Y_j = y_min + (j + 1/2)(y_max - y_min)/ny; planes are row-major
 *     [ny][nx] with j the row (Y) index.  X is the horizontal celestial
 *     coordinate in the sign convention of Eq. (72).
 */
#ifndef BHRT_H
#define BHRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BH_KERR = 0,    /* H = 1 - 2/R (Kerr reference, Sec. 2.2)              */
  BH_EINASTO = 1, /* Einasto-type regular black hole, Eq. (9)             */
  BH_CNFW = 2     /* cored-NFW black hole, Eq. (13)                       */
} bh_metric;

typedef enum {
  BH_OK = 0,
  BH_ERR_INVALID_ARG = 1,     /* NULL pointer, size or parameter out of range */
  BH_ERR_NO_HORIZON = 2,      /* Delta has no root: |chi| > chi_e (Eqs. 33-37) */
  BH_ERR_OBSERVER_INSIDE = 3, /* R_o <= 10 R_+, or R_o inside the escape test  */
  BH_ERR_WORKSPACE = 4,       /* workspace missing, misaligned or too small    */
  BH_ERR_CUDA = 5,            /* a CUDA runtime call failed                    */
  BH_ERR_TIMEOUT = 6,         /* device time budget exceeded (integrator)      */
  BH_ERR_QUEUE_OVERFLOW = 7,  /* refinement list capacity exceeded             */
  BH_ERR_NO_ISCO = 8          /* no stable circular orbit found for R_in       */
} bh_status;

/* Spacetime: metric family and halo parameters (Sec. 2.1, Eqs. 9-14). */
typedef struct {
  int32_t metric;   /* bh_metric */
  int32_t reserved; /* must be 0 */
  double chi;       /* spin a/M (Eq. 1); |chi| below the extremal spin */
  double lambda_E;  /* Einasto scale l_E/M (Eq. 10), > 0, used by BH_EINASTO */
  double eta;       /* cored-NFW 4 pi rho_0 r_0^2 (Eq. 14), >= 0, BH_CNFW   */
  double lambda_c;  /* cored-NFW core radius r_0/M (Eq. 12), > 0, BH_CNFW   */
} bh_spacetime;

/* Observer and screen (Sec. 3.2 and Sec. 4). */
typedef struct {
  double r_obs;            /* observer radius R_o (> 10 R_+)              */
  double incl;             /* inclination theta_o in radians, (0, pi)      */
  double x_min, x_max;     /* screen extent in X                           */
  double y_min, y_max;     /* screen extent in Y                           */
  int32_t nx, ny;          /* base resolution, 1 .. 16384 each             */
  int32_t refine_levels;   /* adaptive 4x4 refinement depth, 0 .. 3        */
  int32_t reserved;        /* must be 0                                    */
  int64_t refine_capacity; /* max cells per refinement level per call; 0
                              selects, per level L = 1, 2, 3, room for
                              min(16^L, max(4 / 12 / 24, 2^22 / base pixels))
                              cells per base pixel                          */
} bh_camera;

/* Emission (Sec. 5.1, Eqs. 83-87).  The default thin-disk mode evaluates j
 * on the equatorial plane (z = 0) at each trusted crossing, so H0 and h only
 * matter in the volumetric mode. */
typedef struct {
  int32_t r_in_mode;  /* 0: R_in = r_ISCO (prograde); 1: R_in = R_+ + dR_in (Eq. 87) */
  int32_t volumetric; /* 0: thin disk, I = sum over crossings of g^3 j(R_em, 0);
                         1: the finite-thickness integral of Eq. (88),
                         I = int g^3 j(R, theta) dlambda, integrated as a
                         seventh component of the Dormand-Prince system
                         (in its error norm), with the circular emitter at
                         the cylindrical radius rho (Eqs. 90-91), j = 0 where
                         no timelike orbit exists, and steps that may come
                         within 5 H of the plane advancing z by at most H/2.
                         I_n planes stay 0; H0 > 0 and h >= 0 required.
                         The all-FP64 path evaluates the source g^3 j in
                         FP64; the mixed path evaluates it in FP32 on every
                         leg (the promoted FP64 steps keep an FP64
                         geodesic).  Not differentiable by bh_trace_backward. */
  double j0, p, R_s;  /* normalisation, radial power, radial scale (Eq. 83) */
  double sigma_in, sigma_out, R_out; /* tapers, Eqs. (85)-(86)             */
  double dR_in;       /* used when r_in_mode == 1                           */
  double H0, h;       /* disk height H(rho) = H0 + h rho, Eq. (84)          */
} bh_emission;

/* Integrator (the paper names none; these are the build's readings). */
typedef struct {
  int32_t precision;    /* 0: all-FP64; 1: mixed (FP32 bulk, FP64 promoted) */
  int32_t max_steps;    /* attempted steps per ray before status 2          */
  double rtol, atol;    /* Dormand-Prince 5(4) tolerances                   */
  double cap_factor;    /* capture when R < cap_factor * R_+ (Eq. 75)       */
  double esc_factor;    /* escape when R > esc_factor * R_o                 */
  double thetadot_min;  /* trusted crossing needs |dtheta/dlambda| >= this  */
  double dlambda_min;   /* and an affine gap >= this to the previous one    */
  double promote_dr;    /* mixed: FP64 steps while R < R_+ + promote_dr     */
  double time_budget_s; /* device time budget per call (s); 0 = none      */
  int32_t promote_order;/* mixed: rays reaching image order n >= this
                           (n = N_cross - 1, Sec. 4.2) inside R = 5 take
                           FP64 steps until outgoing beyond R = 5;
                           0..1000, 1000 = never                          */
  int32_t reserved;     /* must be 0                                        */
  double promote_turning; /* mixed: radial turning points of near-critical
                           rays.  With the radial potential of the separated
                           Hamiltonian (Eqs. 56-59), Rr(R) = P^2 - Delta K =
                           (Delta p_R)^2, P = (R^2 + chi^2) E - chi ell and K
                           the Carter-type constant p_th^2 + Q^2, a ray inside
                           R = 5 takes FP64 steps once Rr < kappa P^2 and
                           Rr'^2 < 2 kappa Rr'' P^2 (Rr'' with Kerr's
                           Delta'' = 2): it is within kappa of a double root
                           of Rr, i.e. near the photon orbit, about to turn
                           or to plunge; it returns to FP32 once outgoing
                           beyond R = 5 or with Rr > 1.2 kappa P^2 (past the
                           root).  kappa = promote_turning in [0, 1];
                           0 = off.  Every FP32 -> FP64 hand-off also puts
                           p_th and p_R back on the ray's FP64 constants
                           E, ell (Eq. 48) and K from the launch, with
                           the null condition (Eq. 54).                   */
} bh_integrator;

/* Per-pixel output planes (device pointers, caller-owned).  Any pointer
 * marked optional may be NULL. */
typedef struct {
  float* I;               /* [ny*nx] total intensity, leaf mean             */
  float* I_n;             /* optional [3][ny*nx] orders n = 0, 1, 2         */
  uint8_t* ncross;        /* [ny*nx] trusted crossings of the base ray (<=255) */
  uint8_t* status;        /* [ny*nx] 0 escaped, 1 captured, 2 undetermined  */
  uint8_t* refine_level;  /* optional [ny*nx] deepest refinement level      */
  float* R_em;            /* optional [3][ny*nx] transfer maps of the base  */
  float* phi_em;          /*   ray's crossings n = 0, 1, 2 (Eq. 82); 0 where */
  float* T_em;            /*   the crossing does not exist                  */
  float* g;               /* optional [3][ny*nx] redshift factor (Eq. 89)   */
  float* h_drift;         /* optional [ny*nx] max |2 Sigma H| Delta / P^2   */
  uint64_t* refine_keys;  /* optional list of traced refined cells:
                             base_id << 16 | level << 12 | d1 << 8 | d2 << 4 | d3,
                             d_l = 4*row + col of the 4x4 child at level l */
  int64_t refine_keys_cap;   /* capacity of refine_keys                      */
  int64_t* refine_keys_count; /* optional device int64: number of keys (may
                                 exceed the capacity, then the list is cut) */
  int32_t* steps;         /* optional [2][ny*nx]: accepted and rejected
                             Dormand-Prince steps of the base ray (all
                             precisions together)                          */
  uint8_t* promoted;      /* optional [ny*nx]: 1 if the base ray took FP64
                             steps on the mixed path, else 0               */
} bh_image_out;

/* Per-ray record returned by bh_trace_points (device array of structs). */
typedef struct {
  int32_t status, ncross;
  int32_t n_accept, n_reject;
  double I_tot, I_n[3];
  double R_em[3], phi_em[3], T_em[3], g[3];
  double E, ell, h_drift, lambda_end;
} bh_ray_record;

/* ---------------------------------------------------------------------- */

/* Host-side geometry of one spacetime: r_plus = R_+ (Eq. 33), chi_e
 * (Eqs. 36-37, computed with chi ignored), r_isco (prograde circular-orbit
 * energy minimum, from Eqs. 90-91).  Any output may be NULL.
 * Returns BH_ERR_NO_HORIZON (r_plus, r_isco untouched) if |chi| >= chi_e. */
bh_status bh_host_geometry(const bh_spacetime* st, double* r_plus, double* chi_e,
                           double* r_isco);

/* Bytes of device workspace needed by bh_trace_batch with n images of the
 * given cameras (all n cameras must share nx, ny and refine_levels) and
 * integrator precision (integ may be NULL: FP64).  The mixed path needs two
 * hand-off queues on top of the refinement lists.  The workspace must be
 * 256-byte aligned. */
bh_status bh_workspace_size(int32_t n, const bh_camera* cameras, const bh_integrator* integ,
                            size_t* bytes);

/* Traces one image: per-pixel backward geodesics, crossings, g, intensity,
 * refinement and assembly.  Equivalent to bh_trace_batch with n = 1. */
bh_status bh_trace_image(const bh_spacetime* st, const bh_camera* cam, const bh_emission* em,
                         const bh_integrator* integ, const bh_image_out* out, void* workspace,
                         size_t workspace_bytes, void* stream);

/* Traces n images in one persistent work-queue launch per refinement level.
 * st, cam, em, integ, out are host arrays of n structs; all cameras share
 * nx, ny, refine_levels and all integrators share precision.  Images may mix
 * metric families and parameters. */
bh_status bh_trace_batch(int32_t n, const bh_spacetime* st, const bh_camera* cam,
                         const bh_emission* em, const bh_integrator* integ,
                         const bh_image_out* out, void* workspace, size_t workspace_bytes,
                         void* stream);

/* Traces single rays from explicit screen points xy[2*k], xy[2*k+1]
 * (device doubles) into records[k] (device).  Same physics as the image
 * path, no refinement; the mixed precision runs the image path's passes
 * (FP32, FP64 for promoted rays, FP32 after demotion).  Needs
 * bh_points_workspace_size(n) bytes (256-byte aligned). */
bh_status bh_points_workspace_size(int64_t n, size_t* bytes);
bh_status bh_trace_points(const bh_spacetime* st, const bh_camera* cam, const bh_emission* em,
                          const bh_integrator* integ, int64_t n, const double* xy,
                          bh_ray_record* records, void* workspace, size_t workspace_bytes,
                          void* stream);

/* Horizon, extremal-spin and stationary-limit scans (Sec. 2.3, Eqs. 33-41):
 * the parameter-space classification of Figs. 2-4 for n spacetimes st[i]
 * (DEVICE array of structs, any mix of families), one thread each.  Per
 * spacetime: R_e[i], the extremal radius (the maximiser of -R^2 H(R) on
 * (0, 50], where Eq. 36 holds), chi_e[i] = sqrt(-R_e^2 H(R_e)) (Eq. 37, 0 if
 * -R^2 H never becomes positive; R_e then only marks where the scan's
 * maximum fell and has no meaning), r_plus[i] = R_+, the largest root of
 * Delta = R^2 H + chi^2 below R = 50 (Eq. 33; 0 if none), and for each of the
 * n_theta polar angles theta[k] (device, radians) the outer stationary-limit
 * radius R_s[i*n_theta + k], the largest root of R^2 H + chi^2 cos^2 theta
 * (Eq. 40; 0 if none; R_s may be NULL when n_theta is 0).  flags[i]: 0 black
 * hole, 1 no horizon (|chi| > chi_e), 2 invalid parameters (unknown metric,
 * lambda_E <= 0, lambda_c <= 0, eta < 0 or a non-finite value; outputs 0).
 * stats (optional device int64[2], may be NULL) receives the lapse
 * evaluations H(R) of the horizon and of the stationary-limit searches.
 * All arrays are device arrays; no workspace; asynchronous on stream. */
bh_status bh_geometry_scan(int64_t n, const bh_spacetime* st, int32_t n_theta,
                           const double* theta, double* r_plus, double* chi_e, double* R_e,
                           double* R_s, int32_t* flags, int64_t* stats, void* stream);

/* Shadow boundary (Sec. 4.1, Eqs. 78-79).  Along each screen direction
 * psi[k] (device doubles, radians), X = b cos psi, Y = b sin psi, the
 * transition between captured and escaping rays is bracketed in the impact
 * parameter b inside [b_lo, b_hi]: on return (stream-ordered, device
 * outputs) b_in[k] <= b_out[k] with the ray at b_in[k] captured, the ray at
 * b_out[k] not captured (escaped or undetermined) and b_out[k] - b_in[k] <=
 * b_tol, unless flagged.  flags[k]: 1 the ray at b_lo is not captured, 2 the
 * ray at b_hi is captured (with 1 or 2 no transition is bracketed and
 * [b_lo, b_hi] is returned), 4 some traced ray was undetermined, 8 the
 * integrator's time budget ran out first (bracket as far as it got; the
 * workspace status is then BH_ERR_TIMEOUT).  A bracket whose width can no
 * longer shrink in FP64 stops there.  If the fate is not monotone in b along
 * a direction, the transition nearest to b_lo among those the samples see
 * is returned.  Rays are traced by the FP64 integrator (integ->precision
 * must be 0) with the tolerances, step limit and thresholds of integ; the
 * camera gives R_o and the inclination (its screen extent and pixel counts
 * are not used); emission plays no part.  Requires 0 <= b_lo < b_hi,
 * b_tol > 0, all finite (else BH_ERR_INVALID_ARG).  lanes: rays traced per
 * direction and round (1 = bisection, 2 .. 32 = (lanes + 1)-section; a power
 * of two), or 0 for the library's choice: the most lanes, up to 32, with
 * which all directions fit in half of the GPU's resident threads.  stats
 * (optional device int64[3], may be NULL) receives the rays traced and their
 * accepted and rejected Dormand-Prince steps.  Needs
 * bh_shadow_workspace_size(n_psi) bytes of 256-byte aligned workspace. */
bh_status bh_shadow_workspace_size(int64_t n_psi, size_t* bytes);
bh_status bh_shadow_boundary(const bh_spacetime* st, const bh_camera* cam,
                             const bh_integrator* integ, int64_t n_psi, const double* psi,
                             double b_lo, double b_hi, double b_tol, int32_t lanes,
                             double* b_in, double* b_out, int32_t* flags, int64_t* stats,
                             void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------- */
/* Plans: a batch whose per-image constants are computed and uploaded once,
 * then launched any number of times.  bh_plan_launch with use_graph != 0
 * captures the whole launch sequence (persistent trace launch per level,
 * refinement, assembly) into a CUDA graph on first use and replays it
 * afterwards; the stream must then be a non-legacy stream and the output
 * and workspace pointers given at creation must stay valid.  A plan owns
 * host memory only.  Outputs and workspace follow bh_trace_batch. */
typedef struct bh_plan_s* bh_plan;

typedef struct {
  int64_t cells[4];        /* cells per level (level 0 = n * nx * ny)         */
  int64_t rays[4];         /* rays integrated to termination per level        */
  int64_t accepted_fp64;   /* accepted Dormand-Prince steps taken in FP64     */
  int64_t rejected_fp64;   /* rejected FP64 trial steps                       */
  int64_t accepted_fp32;   /* mixed precision: accepted FP32 steps            */
  int64_t rejected_fp32;   /* mixed precision: rejected FP32 trial steps      */
  int64_t promoted_rays;   /* mixed precision: rays handed to the FP64 pass   */
  int64_t spill_full;      /* promotions refused because the queue was full   */
  int64_t max_ray_steps;   /* attempted steps of the longest ray              */
  double trace_ms[4];      /* per-level trace time (all passes) of the last
                              launch when timing is on, else -1               */
  double fp32_ms, fp64_ms; /* trace kernel time by precision (timing on)      */
  int32_t kernel_launches; /* kernels enqueued per launch                     */
  int32_t status;          /* device status word (bh_status)                  */
  int32_t trace_blocks, trace_threads; /* trace launch shape in use           */
  /* Persistent-queue timeline per trace pass (0 main, 1 FP64 promoted,
   * 2 FP32 demoted) and level, from the device clock: bulk = first warp
   * start to the first warp finding the queue empty; tail = from then to
   * the last warp exit (warps running with idle lanes).  -1 if not run. */
  double bulk_ms[3][4];
  double tail_ms[3][4];
  /* Mean fraction of the 32 lanes holding a ray over the stepping-loop
   * iterations of the FP32 and FP64 trace kernels (-1 if not run). */
  double lane_util_fp32, lane_util_fp64;
} bh_run_stats;

/* Validates, computes per-image constants and uploads them to the
 * workspace (synchronises the stream once). */
bh_status bh_plan_create(int32_t n, const bh_spacetime* st, const bh_camera* cam,
                         const bh_emission* em, const bh_integrator* integ,
                         const bh_image_out* out, void* workspace, size_t workspace_bytes,
                         void* stream, bh_plan* plan);
bh_status bh_plan_launch(bh_plan plan, int32_t use_graph, void* stream);
/* Records CUDA events around each trace launch (disables graph replay). */
bh_status bh_plan_set_timing(bh_plan plan, int32_t enable);
/* Fixes the launch shape of a persistent trace kernel of the plan: which = 0
 * the main kernel (FP64, or the FP32 bulk of the mixed path), 1 the FP64
 * promoted pass; blocks >= 1, threads 64 or 128 (a multiple of 32),
 * variant 0 or 1 (the kernel build, as in bh_tune_report).  A grid smaller
 * than the GPU's resident capacity leaves room for other work, e.g. a second
 * plan on another stream.  Any captured graph is discarded. */
bh_status bh_plan_set_launch(bh_plan plan, int32_t which, int32_t blocks, int32_t threads,
                             int32_t variant);
/* Counters of the last launch (blocking copy on `stream`). */
bh_status bh_plan_stats(bh_plan plan, void* stream, bh_run_stats* out);
bh_status bh_plan_destroy(bh_plan plan);

/* Autotuner: runs the plan once per candidate launch shape of the persistent
 * trace kernel (and of the FP64 pass of the mixed path), timing the trace
 * kernels with CUDA events, and keeps the fastest shape for later launches
 * (any captured graph is discarded and re-captured on the next graph launch).
 * Synchronises the stream; outputs hold the last candidate's (identical)
 * results. */
typedef struct {
  int32_t candidates;      /* shapes tried                                    */
  int32_t blocks[2];       /* chosen grid: [0] main trace kernel, [1] FP64 pass */
  int32_t threads[2];      /* chosen block size                               */
  double best_ms[2];       /* trace time of the whole launch with the choice  */
  int32_t variant[2];      /* kernel build chosen: 0 registers unbounded,
                              1 capped (FP64: 3 blocks of 128 per SM; mixed: 4) */
} bh_tune_report;
bh_status bh_plan_autotune(bh_plan plan, void* stream, bh_tune_report* report);

/* ---------------------------------------------------------------------- */
/* Image diagnostics of Sec. 6.2-6.3 from a traced intensity plane I
 * (device float [ny][nx], screen geometry from cam).  out12 (device,
 * 12 doubles) receives, in order:
 *   F (Eq. 92), X_c, Y_c (Eq. 93), C (Eq. 94), rho_bar (Eq. 96),
 *   d_img (Eq. 97), w_img (Eq. 98), A_LR (Eqs. 99-100), P = I_max / mean of
 *   I over pixels with I > 0 (Eq. 101), rho_peak, d_peak = 2 rho_peak
 *   (Eq. 106), theta_peak = d_peak theta_g (Eq. 107).
 * Integrals are pixel sums times dX dY at pixel centres; the left/right split
 * uses strict inequalities; the radial profile bins rho_0 (Eq. 105) with
 * width dX from 0, takes the mean per non-empty bin, resolves argmax ties to
 * the smaller radius and reports the bin centre.  All accumulation is FP64.
 * Needs bh_diagnostics_workspace_size bytes of 256-byte aligned workspace. */
bh_status bh_diagnostics_workspace_size(const bh_camera* cam, size_t* bytes);
bh_status bh_diagnostics(const float* I, const bh_camera* cam, double theta_g, double* out12,
                         void* workspace, size_t workspace_bytes, void* stream);

/* Same diagnostics without a caller workspace; the paper has no counterpart.
 * For callers that cannot allocate device memory when they need the result
 * (a host framework that owns all device memory through its own pool, a
 * plugin that only receives its input and output buffers, a timed loop that
 * must not call cudaMalloc): the reduction scratch is a fixed 256 KiB
 * file-scope device array that every GPU loading the library holds until
 * process exit.  The call allocates nothing.  The first call on each device
 * looks the array's device address up (cudaGetSymbolAddress) and caches it,
 * so make that first call before any stream capture.  The cached address
 * lives as long as the process: after a cudaDeviceReset of a device (which
 * reloads the library's device code there) this entry point must not be
 * used on that device again.  All calls share the
 * array: the histogram is cleared on every call, but calls whose work
 * overlaps on the GPU (different streams, or different host threads on one
 * device) race on it.  Images whose radial profile needs more scratch than
 * the array holds are rejected
 * with BH_ERR_WORKSPACE before anything is enqueued; for a square screen
 * centred on the origin that is a side above about 20,000 pixels. */
bh_status bh_diagnostics_noalloc(const float* I, const bh_camera* cam, double theta_g,
                                 double* out12, void* stream);

/* Visibilities of Eq. (108), FP64 direct sum: V_k = sum_ij I_ij
 * exp[-2 pi i (u_k X_i + v_k Y_j)] dX dY for K baselines uv[2k], uv[2k+1]
 * in cycles per M (device doubles); V[2k], V[2k+1] = Re, Im (device).
 * The normalised amplitude of Eq. (109) is |V_k| / |V(0,0)| with
 * V(0,0) = F.  Cost O(K nx ny) in FP64: the reference mode. */
bh_status bh_visibilities_fp64(const float* I, const bh_camera* cam, const double* uv, int64_t K,
                               double* V, void* stream);

/* Visibilities of Eq. (108) as a tensor-core contraction (tcgen05):
 *   mode 0: FP64 direct sum (bh_visibilities_fp64; workspace unused);
 *   mode 1: operands split hi + lo in BF16, FP32 accumulation;
 *   mode 2: operands split hi + lo in FP16, FP32 accumulation (the image is
 *           divided by image_max first, so intensities far below the maximum
 *           lose relative precision to the FP16 exponent range).
 * image_max > 0 is the image maximum (or any positive scale near it), used
 * to normalise before splitting.  uv and V as in bh_visibilities_fp64.
 * Vnorm (optional device double[K], may be NULL) receives the normalised
 * amplitudes of Eq. (109), |V_k| / |V(0,0)|, with V(0,0) = F = sum I dX dY
 * (Eq. 92) summed in FP64 from the image (not from the split evaluation);
 * an image of zero flux gives inf or NaN there.
 * Modes 1-2 need nx <= 4096 and bh_visibilities_workspace_size bytes of
 * 256-byte aligned workspace.  time_budget_s >= 0 is a device time budget
 * for modes 1-2 (0 = none): each CTA checks it before each reduction
 * chunk issues its copies and products, and once it is spent stops there,
 * waits for the work it has issued and sets BH_ERR_TIMEOUT in the
 * workspace status word (read with bh_workspace_status after
 * synchronising); V is then incomplete.  A pipeline wait that has not
 * completed after 2 s of device time sets the same status. */
bh_status bh_visibilities_workspace_size(const bh_camera* cam, size_t* bytes);
bh_status bh_visibilities(const float* I, const bh_camera* cam, const double* uv, int64_t K,
                          int32_t mode, double image_max, double* V, double* Vnorm,
                          double time_budget_s, void* workspace, size_t workspace_bytes,
                          void* stream);

/* Fourier-domain summaries of Sec. 6.4 at n_q radii q[j] (device doubles,
 * cycles per M): V_avg[j], the normalised amplitude |V|/|V(0,0)| (Eq. 109)
 * averaged over the position angle (midpoint rule at phi_k = (k + 1/2) pi /
 * n_phi, k < n_phi; the amplitude of a real image is symmetric under
 * (u, v) -> (-u, -v)), and V_cut[j] = |V(q_j, 0)| / |V(0,0)|, the horizontal
 * cut (device outputs).  The visibilities are those of bh_visibilities in
 * the given mode (0 FP64 direct, 1 split BF16, 2 split FP16 tensor cores;
 * image_max > 0 as there), with |V(0,0)| from the same evaluation, so
 * q = 0 gives 1 to rounding; an image of zero flux gives NaN.  n_q >= 0, n_phi >= 1.
 * Needs bh_visibility_curves_workspace_size bytes of 256-byte aligned
 * workspace; its leading status word is that of bh_visibilities. */
bh_status bh_visibility_curves_workspace_size(const bh_camera* cam, int32_t n_q, int32_t n_phi,
                                              size_t* bytes);
bh_status bh_visibility_curves(const float* I, const bh_camera* cam, int32_t n_q,
                               const double* q, int32_t n_phi, int32_t mode, double image_max,
                               double* V_avg, double* V_cut, void* workspace,
                               size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------- */
/* Gradients by a hand-written discrete adjoint of the FP64 image path.
 * Loss: L = sum_p dL_dI[p] I[p] + sum_m dL_ddiag[m] D_m with
 *   D = (C (Eq. 94), A_LR (Eq. 99), rho_peak, |V_k|/|V(0,0)| for the 8
 *        baselines uv8 (Eq. 109)),
 * where rho_peak is the vertex of the parabola through the origin-centred
 * profile's peak bin and its two neighbours (a differentiable reading of
 * Eq. 105's bin-centre peak).  grad10 (host) receives dL/d(chi, theta_o,
 * halo1, halo2, j0, p, R_s, sigma_in, sigma_out, R_out); halo1 = lambda_E
 * (Einasto) or eta (cored-NFW), halo2 = lambda_c (cored-NFW); unused halo
 * entries are 0.  The derivative is that of the algorithm with its adaptive
 * decisions frozen (accepted step sizes, refinement pattern, trusted
 * crossings, termination step); R_in = r_ISCO or R_+ + dR_in is
 * differentiated implicitly; the capture radius is held fixed.
 * The forward pass runs in FP64 whatever integ->precision says.  Each ray
 * is replayed with a checkpoint every 64 accepted steps into a per-thread
 * slab sized from the forward image's longest ray (longer rays: fewer
 * threads share the workspace's checkpoint region); BH_ERR_WORKSPACE only
 * if one block of 128 such slabs does not fit there (on a 152-SM GPU, a
 * longest ray of more than about 1.2 million steps, above the default step
 * limit) or a ray has more than 32 trusted crossings.
 * dL_dI (device float [ny][nx]), dL_ddiag (host, 11) and uv8 (host, 8x2
 * cycles/M) may be NULL; diag11 (host) receives D; image_out (device float
 * [ny][nx]) the forward intensity.  Synchronous: returns when grad10 is
 * written.  Needs bh_backward_workspace_size bytes (256-byte aligned). */
bh_status bh_backward_workspace_size(const bh_camera* cam, size_t* bytes);
bh_status bh_trace_backward(const bh_spacetime* st, const bh_camera* cam, const bh_emission* em,
                            const bh_integrator* integ, const float* dL_dI,
                            const double* dL_ddiag, const double* uv8, double* grad10,
                            double* diag11, float* image_out, void* workspace,
                            size_t workspace_bytes, void* stream);

/* Device status word of the last call that used this workspace (blocking
 * copy; call after synchronising the stream). */
bh_status bh_workspace_status(const void* workspace, void* stream);

const char* bh_status_string(bh_status s);

#ifdef __cplusplus
}
#endif
#endif /* BHRT_H */
