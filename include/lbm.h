/*
 * lbm.h -- C ABI of liblbm, a GB300 (sm_103a) implementation of the lattice
 * Boltzmann step with nonequilibrium entropy limiters of Brownlee, Gorban and
 * Levesley, "Nonequilibrium entropy limiters in lattice Boltzmann methods",
 * Physica A 2007 (arXiv:0704.0043).
 *
 * One step (Eq. lbgkLB; the limiter is "a post-processing routine immediately
 * following the collision step", Sec. 4.3.2):
 *   free flight in pull form, halfway bounce-back walls, moving lid (Sec. 2, Sec. 4.4.1)
 *   -> moments (Eq. macro_dis) -> polynomial f* (Eq. polyeq1d / Eq. polyeq2d),
 *      or entropic f* (Eq. entropiceq1d / Eq. maxwellian, LBM_EQ_ENTROPIC)
 *   -> LBGK collision f' = f* + (2 beta - 1)(f* - f)      (Eq. collLBGK)
 *   -> dS(f') = sum_k (f'_k - f*_k)^2 / f*_k              (Sec. 3.6, quadratic form of Eq. DelS;
 *      LBM_EQ_ENTROPIC: sum_k f'_k ln(f'_k / f*_k), Eq. DelS)
 *   -> limiters f -> f* + phi (f - f*)                     (Eq. LimGenF):
 *      positivity rule (Sec. 3.1), median filter (Sec. 3.5), Ehrenfests' trimming (Sec. 3.2)
 *   -> stored field for the next step, plus FP64 sums (Sec. 3.4, Sec. 4.3.1).
 *
 * Conventions shared by every entry point
 *   - Every call returns lbm_status; nothing throws or exits across the ABI.
 *     On failure lbm_last_error(ctx) holds a one-line message.
 *   - The library owns the lattice (populations, scratch) in device memory.
 *     Callers own every buffer they pass in or out.
 *   - All device work is ordered on the CUDA stream given to lbm_create (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).  Calls
 *     that fill host memory synchronise that stream before returning.
 *   - Array arguments may be host or device pointers (detected with
 *     cudaPointerGetAttributes).  Field layout is the oracle layout: site
 *     (i, j) at index j * nx + i (x fastest, y upward, lid at j = ny - 1);
 *     population fields are plane-major, f[k * ny * nx + j * nx + i].
 *   - D2Q9 directions follow Sec. 4.1: 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW,
 *     7 SW, 8 SE.  D1Q3: 0 rest, 1 left (v = -1), 2 right (v = +1), i.e. the
 *     paper's f1, f2, f3.
 *   - A context is used by one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 3

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1, /* a parameter is out of range; nothing was enqueued */
    LBM_ERR_OOM = 2,         /* device allocation failed */
    LBM_ERR_CUDA = 3,        /* a CUDA runtime call failed (message names it) */
    LBM_ERR_NONFINITE = 4,   /* a site had rho <= 0, f*_k <= 0 or a nonfinite value */
    LBM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up: the grid barrier of the tail that
                                preselects dense Ehrenfests' candidates (lattices of 2^20 sites or
                                more, cooperative launch) polls about a second; the pass's results
                                are then not to be trusted (re-initialise the state) */
    LBM_ERR_STATE = 6        /* call out of order (e.g. step before init) */
} lbm_status;

enum { LBM_D1Q3 = 1, LBM_D2Q9 = 2 };

/* Storage precision of the populations.  LBM_FP64 stores f and evaluates
 * every operation in the oracle's order with no FMA contraction.  LBM_FP32,
 * LBM_BF16 and LBM_FP16 store the deviations g_k = f_k - rho_ref W_k from a
 * uniform rest state (in 32, 16 and 16 bits) and compute in FP32 on them (FP64
 * for the global sums and the Ehrenfests' keys); every transfer in or out of
 * the library converts to and from f in FP64. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_BF16 = 2, LBM_FP16 = 3 };

enum {
    LBM_BC_WALLS = 0,    /* D2Q9: still walls left, right, bottom, lid on top, half a link outside
                            the lattice (halfway bounce-back); D1Q3: closed ends */
    LBM_BC_PERIODIC = 1, /* periodic in every direction */
    LBM_BC_CHANNEL = 2,  /* D2Q9: periodic in x, still bottom wall, lid on top */
    /* D2Q9 cavities whose outer ring of nodes lies on the walls (boundary nodes,
     * Sec. 4.4).  Boundary nodes are not collided and not limited, their dS is 0,
     * and the median filter's stencils stay on the other nodes (a node next to one
     * wall: itself and its two neighbours along it; next to two walls: itself and
     * its inward x and y neighbours).  After free flight a boundary node receives
     * the populations it lacks (sources outside the lattice) from the wall rule.
     * The lid is the top row without its two corners and moves with (u_lid, 0);
     * the other walls and the corners are at rest.  The stats' mass counts, at a
     * boundary node, the populations that stream back onto the lattice.  The
     * fused kernel does not take these boundaries (LBM_KERNEL_AUTO picks the
     * tiled kernel). */
    LBM_BC_NODE_WALLS = 3, /* bounce-back: f_k = f_opp(k) + 6 W_k rho_wall (v_k . u_wall) (Sec. 4.4.1) */
    LBM_BC_DIFFUSIVE = 4   /* diffusive Maxwell wall (Sec. 4.4.2): f_k = gamma f*_k(1, u_wall) with
                              gamma = sum of the arrived f_opp(k) / sum of f*_k(1, u_wall) over the
                              returned directions (f* of the configured kind); bounce-back in the
                              corners */
};

/* Limiters (bit set).  LBM_LIM_SMOOTH and LBM_LIM_THRESHOLD are ensemble-dependent: they
 * use E(dS), the mean of dS(f') over the sites with a finite value (not flagged), of the
 * pass being limited, so a pass with either bit first runs a reduction over the lattice.
 *   LBM_LIM_SMOOTH: phi = 1 / (1 + alpha dS^k), alpha = smooth_delta / E^k (Eq. smooth1,
 *     with the ensemble-dependent alpha of Sec. 4.3.2); phi = 1 where E <= 0 or dS = 0.
 *   LBM_LIM_THRESHOLD: dS_t = max(threshold_c E, threshold_delta); phi = sqrt(dS_t / dS)
 *     where dS > dS_t (Sec. 3.4, Eq. entrHom, with dS_0 = c E as in Sec. 4.3.2).
 * Every limiter's phi is combined as the minimum, before Ehrenfests' step.  The
 * ensemble limiters (these two and LBM_LIM_ENTTHRESH) run on the fused kernel where it
 * applies (the E(dS) pass is then the fused kernel's own row streaming), else on the
 * tiled kernel; not in batches, not in lbm_step_noalloc. */
enum { LBM_LIM_POSITIVITY = 1, LBM_LIM_EHRENFEST = 2, LBM_LIM_MEDIAN = 4, LBM_LIM_SMOOTH = 8,
       LBM_LIM_THRESHOLD = 16, LBM_LIM_ENTTHRESH = 32 };
/* LBM_LIM_ENTTHRESH: the threshold filter with dS_0 from Eq. EntThresh, solved on the
 *   pass's own distribution of dS (the sites E(dS) is taken over):
 *   sum_s max(dS_s - dS_0, 0) = entthresh_delta0 (1 - (2 beta - 1)^2) sum_s dS_s, so that the
 *   limiter's entropy production stays within delta_0 of LBGK's (Eq. LimEntLim);
 *   dS_t = max(dS_0, threshold_delta), phi = sqrt(dS_t / dS) where dS > dS_t (or the solve
 *   of LBM_PHI_ENTROPY).  dS_0 is found exactly by a radix descent over the bit patterns
 *   of the dS field (dS_0 = +inf when the right side is 0: nothing is limited); its sums
 *   are added by atomics, so it is reproducible to rounding.  Needs the bit at create
 *   (the field is allocated then); not in batches or lbm_step_noalloc. */

/* Median-filter acceptance rule (Sec. 3.5 with the tolerance of Sec. 4.3.2). */
enum {
    LBM_MEDIAN_THRESHOLD = 0, /* dS_t = max(dS_med, delta); phi = sqrt(dS_t/dS) where dS > dS_t */
    LBM_MEDIAN_GATE = 1       /* phi = sqrt(dS_med/dS) where dS > delta and dS_med < dS */
};

/* Quasiequilibrium and nonequilibrium entropy.
 * LBM_EQ_POLYNOMIAL: f* of Eq. polyeq1d / Eq. polyeq2d, dS(f) = sum_k (f_k - f*_k)^2 / f*_k
 *   (the quadratic form of Eq. DelS, Sec. 3.6).
 * LBM_EQ_ENTROPIC: f* of Eq. entropiceq1d / Eq. maxwellian (the D1Q3 population with
 *   v = +1 takes the printed f2*, the assignment under which sum_k v_k f*_k = rho u),
 *   and the exact dS(f) = sum_k f_k ln(f_k / f*_k) of Eq. DelS, with 0 ln 0 = 0 and
 *   dS = +inf for a state with a negative population (not an error: the limiters act
 *   on it; the median homothety is then 0).  Sites with |u_x| or |u_y| >= 1 have no
 *   entropic f* and are flagged (LBM_ERR_NONFINITE).  The stats are entropy
 *   differences: dS_lbgk = sum [dS(f_in) - dS(f')], dS_lim = sum [dS(f') - dS(f_out)]
 *   plus dS of each Ehrenfests' site's state w.r.t. its own f*, each over the sites
 *   where both values are finite; sum_dS skips infinite values.  FP64 storage and the
 *   tiled kernel only; lbm_init then starts from the entropic f*. */
enum { LBM_EQ_POLYNOMIAL = 0, LBM_EQ_ENTROPIC = 1 };

/* Collision (needs LBM_EQ_ENTROPIC and LBM_FP64 for ELBM).
 * LBM_COLL_LBGK: f' = f* + (2 beta - 1)(f* - f) (Eq. collLBGK, Eq. lbgkLB).
 * LBM_COLL_ELBM: f' = (1 - beta) f + beta f~ with f~ = f + alpha (f* - f) (Eq. elbm),
 *   alpha the nontrivial root of S(f~) = S(f) (Eq. entropy_estimate) found per site by
 *   bisection on [1, alpha_max] to a bracket of 1e-15, keeping the end where the
 *   entropy does not decrease (Sec. 4.2); alpha_max is the positivity boundary of the
 *   line f + alpha (f* - f), taken when the entropy is still above S(f) there (no
 *   root in the positive cone: the positivity rule); f = f* gives alpha = 2. */
enum { LBM_COLL_LBGK = 0, LBM_COLL_ELBM = 1 };

/* Factor of the filters with a target dS_t (median filter, threshold filter).
 * LBM_PHI_HOMOTHETY: phi = sqrt(dS_t / dS) (Eq. entrHom, exact in the quadratic form).
 * LBM_PHI_ENTROPY (LBM_EQ_ENTROPIC only): phi in [0, 1] solves
 *   S(f* + phi (f' - f*)) = S(f*) - dS_t, i.e. dS(f* + phi (f' - f*)) = dS_t with the
 *   exact dS of Eq. DelS (Sec. 3.7), by bisection to a bracket of 1e-15 (the lower end). */
enum { LBM_PHI_HOMOTHETY = 0, LBM_PHI_ENTROPY = 1 };

/* Kernel choice for lbm_step. */
enum {
    LBM_KERNEL_AUTO = 0,    /* the fused D2Q9 cavity kernel or the D1Q3 tube kernel where it applies,
                               else the tiled kernel */
    LBM_KERNEL_TILED = 1,   /* overlapping-tile kernel: every lattice, boundary and precision */
    LBM_KERNEL_FUSED = 2,   /* D2Q9 with LBM_BC_WALLS, FP32/BF16/FP16 storage: row-streaming fused kernel */
    LBM_KERNEL_TUBE = 3     /* D1Q3 with FP32 or FP64 storage, LBM_BC_WALLS or LBM_BC_PERIODIC, no
                               ensemble-dependent limiter: a streaming pass, one chunk of sites per warp
                               (the same populations as the tiled kernel, bit for bit) */
};

typedef struct lbm_config {
    int32_t lattice;         /* LBM_D1Q3 or LBM_D2Q9 */
    int32_t nx, ny;          /* sites; ny must be 1 for D1Q3; nx, ny >= 2 for D2Q9 walls */
    int32_t boundary;        /* LBM_BC_* */
    int32_t precision;       /* LBM_FP64, LBM_FP32, LBM_BF16 or LBM_FP16 */
    uint32_t limiters;       /* LBM_LIM_* bits applied by lbm_step */
    int32_t median_mode;     /* LBM_MEDIAN_* */
    int32_t kernel;          /* LBM_KERNEL_* */
    double beta;             /* LBGK over-relaxation, 0 <= beta <= 1 (Eq. collLBGK) */
    double u_lid;            /* lid x-velocity (D2Q9, LBM_BC_WALLS / LBM_BC_CHANNEL) */
    double rho_wall;         /* density in the moving-wall momentum term 6 W_k rho_wall (v_k . u_lid) */
    double delta_median;     /* median-filter tolerance delta (>= 0) */
    double delta_ehrenfest;  /* Ehrenfests' threshold: sites with dS > delta are candidates */
    int64_t k_max;           /* Ehrenfests' step acts on at most k_max sites per step (>= 0) */
    int32_t stats_history;   /* per-step stats kept on the device (ring length, >= 1) */
    int32_t equilibrium;     /* LBM_EQ_* (LBM_EQ_ENTROPIC needs LBM_FP64) */
    double rho_ref;          /* reference density of the FP32 deviation storage (> 0, default 1) */
    double smooth_delta;     /* LBM_LIM_SMOOTH: alpha = smooth_delta / E(dS)^smooth_k (>= 0, default 0.01) */
    double smooth_k;         /* LBM_LIM_SMOOTH: exponent k (> 0, default 0.5) */
    double threshold_c;      /* LBM_LIM_THRESHOLD: dS_0 = threshold_c * E(dS) (>= 0, default 10) */
    double threshold_delta;  /* LBM_LIM_THRESHOLD: dS_t = max(dS_0, threshold_delta) (>= 0, default 0) */
    int32_t collision;       /* LBM_COLL_* (default LBM_COLL_LBGK) */
    int32_t phi_rule;        /* LBM_PHI_* (default LBM_PHI_HOMOTHETY) */
    double entthresh_delta0; /* LBM_LIM_ENTTHRESH: delta_0 of Eq. EntThresh (>= 0, default 0.1) */
} lbm_config;

typedef struct lbm_step_stats {
    int64_t step;            /* steps taken since lbm_init / lbm_set_populations */
    double mass;             /* sum of rho over sites, after free flight */
    double sum_dS;           /* sum of dS(f') (post-collision, pre-limiter) */
    double dS_lbgk;          /* [1 - (2 beta - 1)^2] * sum of dS(f_in) (Sec. 3.4) */
    double dS_lim;           /* entropy added by the limiters: sum (1 - phi^2) dS(f'),
                                plus phi^2 dS(f') at each Ehrenfests' site */
    int64_t n_pos;           /* sites where the positivity rule acted */
    int64_t n_med;           /* sites where the median filter acted */
    int64_t n_ehr;           /* sites equilibrated by Ehrenfests' step */
    int64_t n_cand;          /* sites with dS(f') > delta_ehrenfest */
    int64_t n_bad;           /* sites flagged nonfinite / nonpositive */
    int32_t status;          /* lbm_status of that step */
    int32_t reserved;
} lbm_step_stats;

typedef struct lbm_ctx lbm_ctx;

/* Fills *cfg with defaults: D2Q9 100 x 100 cavity, FP32, beta = 1, no limiters,
 * delta = 1e-3, k_max = 0, one stats record, rho_wall = rho_ref = 1. */
void lbm_config_default(lbm_config *cfg);

/* Validates cfg, allocates the lattice and scratch on the current device and
 * returns a context bound to `cuda_stream`.  Populations start at zero; call
 * lbm_init or lbm_set_populations before lbm_step (else LBM_ERR_STATE).
 * Errors: LBM_ERR_INVALID_ARG (bad cfg / NULL out), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_config *cfg, void *cuda_stream, lbm_ctx **out);

/* Synchronises the context's stream and frees everything it owns.  NULL is a no-op. */
lbm_status lbm_destroy(lbm_ctx *ctx);

/* Populations at equilibrium f*(rho, u) of the configured kind (Eq. polyeq1d / Eq. polyeq2d;
 * LBM_EQ_ENTROPIC: Eq. entropiceq1d / Eq. maxwellian, NaN where |u_j| >= 1),
 * evaluated in FP64 and stored at the context's precision; resets the step
 * counter and the stats.  rho, ux: nx * ny doubles; uy: nx * ny doubles or NULL
 * (taken as 0; ignored for D1Q3).  Errors: LBM_ERR_INVALID_ARG (NULL rho/ux). */
lbm_status lbm_init(lbm_ctx *ctx, const double *rho, const double *ux, const double *uy);

/* nsteps limited LBGK steps (free flight, collision, the configured limiters,
 * FP64 sums), enqueued asynchronously.  A site that cannot be limited sets the
 * context's sticky status to LBM_ERR_NONFINITE; that status is returned by the
 * next call that synchronises (lbm_stats, lbm_moments, lbm_synchronize, ...).
 * Errors: LBM_ERR_STATE (no init), LBM_ERR_INVALID_ARG (nsteps < 0). */
lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* The dS(f') field (quadratic Kullback form, Sec. 3.6) of the collision the
 * next lbm_step performs on the stored populations, evaluated in FP64 from the
 * stored values: nx * ny doubles into `out`.  No population is modified. */
lbm_status lbm_delta_s(lbm_ctx *ctx, double *out);

/* Applies `limiters` (any LBM_LIM_* bits; Ehrenfests' only if configured at
 * create) to the stored populations themselves, with no free flight and no
 * collision: f' := f, f* := f*(m(f)) of the configured kind, then the same
 * limiter pass as a step (Sec. 3; the ensemble-dependent limiters take E(dS)
 * of the stored state).  Counts and sums go to the stats (step counter
 * unchanged).  Errors: LBM_ERR_INVALID_ARG (unknown bits). */
lbm_status lbm_limit(lbm_ctx *ctx, uint32_t limiters);

/* rho, u (Eq. macro_dis) of the stored populations, FP64, nx * ny each;
 * uy may be NULL.  Synchronises; returns the sticky status. */
lbm_status lbm_moments(lbm_ctx *ctx, double *rho, double *ux, double *uy);

/* Stats of the most recent step (or lbm_limit pass).  Synchronises; returns
 * the sticky status (the stats are written either way). */
lbm_status lbm_stats(lbm_ctx *ctx, lbm_step_stats *out);

/* Up to `cap` most recent per-step stats, oldest first (at most stats_history);
 * *n receives the count written. */
lbm_status lbm_stats_history(lbm_ctx *ctx, lbm_step_stats *out, int64_t cap, int64_t *n);

/* The sites Ehrenfests' step equilibrated in the most recent step, sorted by
 * site index: min(cap, n) int64 indices into idx (host or device), *n = the
 * full count.  Selection (Sec. 3.2, Sec. 4.3.2): the k_max largest dS(f') >
 * delta_ehrenfest, ties to the lower site index. */
lbm_status lbm_limited_sites(lbm_ctx *ctx, int64_t *idx, int64_t cap, int64_t *n);

/* Copies the stored populations out as FP64 (q * nx * ny doubles), or sets
 * them from FP64 (rounded to the storage precision; resets the step counter).
 * Used for checkpoints and for parity checks against the oracle. */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f);
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f);

/* Waits for the context's stream; returns (and clears) the sticky status. */
lbm_status lbm_synchronize(lbm_ctx *ctx);

/* Fills `out` with the context's configuration. */
lbm_status lbm_get_config(const lbm_ctx *ctx, lbm_config *out);

/* Bytes of device memory the context holds (for admission by HBM footprint). */
int64_t lbm_device_bytes(const lbm_ctx *ctx);

/* Device bytes lbm_create would allocate for cfg (0 if cfg is invalid). */
int64_t lbm_footprint_bytes(const lbm_config *cfg);

/* Control-point record (the monitoring point of Sec. 4.4.2): after every
 * subsequent step the tail kernel stores rho, u_x, u_y (Eq. macro_dis, FP64, the
 * values lbm_moments would give) of `site` (index j * nx + i) in a device ring of
 * `capacity` samples, which this call allocates (device memory).  site = -1 stops
 * recording.  Synchronises.  Errors: LBM_ERR_INVALID_ARG (site out of range,
 * capacity < 1), LBM_ERR_OOM. */
lbm_status lbm_probe(lbm_ctx *ctx, int64_t site, int64_t capacity);

/* The most recent min(cap, recorded, capacity) samples of the control point,
 * oldest first, as (rho, u_x, u_y) triples (3 doubles each) into `out` (host or
 * device); *n receives the number of samples written.  Synchronises.
 * Errors: LBM_ERR_STATE (no probe set), LBM_ERR_INVALID_ARG. */
lbm_status lbm_probe_read(lbm_ctx *ctx, double *out, int64_t cap, int64_t *n);

/* CUDA-graph replay for lbm_step: runs of `steps_per_graph` steps (an even
 * number >= 2; 0 turns replay off) are captured once per starting buffer into a
 * CUDA graph on a stream of the context's own and replayed on the context's
 * stream, which removes the per-launch host cost of small lattices.  The steps
 * and their results are those of plain lbm_step calls.  While per-kernel timing
 * (lbm_timing) is on, lbm_step launches plainly.  The first replay of each
 * starting buffer captures its graph; make it before any stream capture of the
 * caller's own.  Errors: LBM_ERR_INVALID_ARG (odd count or 1). */
lbm_status lbm_set_graph(lbm_ctx *ctx, int32_t steps_per_graph);

/* Per-kernel timing with CUDA events recorded on the context's stream.  While
 * enabled, a timed step records an event before its step kernel, one between
 * the step kernel and its one-block tail kernel, and one after the tail.
 * enable = 0 turns timing off, 1 times every step, N > 1 times one step in N
 * (the first, then every N-th: events between the kernels also delay the
 * following launch, so sampling keeps that cost off most steps).
 * lbm_timing_read synchronises, returns the summed milliseconds of each kernel
 * kind and the number of timed steps, and clears the record.
 * Errors: LBM_ERR_INVALID_ARG (NULL context, enable < 0). */
lbm_status lbm_timing(lbm_ctx *ctx, int32_t enable);
lbm_status lbm_timing_read(lbm_ctx *ctx, double *step_kernel_ms, double *tail_kernel_ms, int64_t *steps);

/* The step kernel lbm_step launches for this context: LBM_KERNEL_TILED,
 * LBM_KERNEL_FUSED or LBM_KERNEL_TUBE (-1 for a NULL context). */
int32_t lbm_step_kernel(const lbm_ctx *ctx);

/* Number of kernel launches the context has enqueued so far. */
int64_t lbm_launch_count(const lbm_ctx *ctx);

/* Last error message of ctx (never NULL); lbm_last_error(NULL) reports errors
 * of lbm_create and lbm_footprint_bytes on the calling thread. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Size of the static device scratch array of lbm_step_noalloc, and the
 * largest lattice (nx * ny) it accepts. */
#define LBM_NOALLOC_SCRATCH_BYTES (8u << 20)
#define LBM_NOALLOC_MAX_SITES 262144

/* One limited LBGK step of a lattice held entirely in caller memory, without
 * any device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc (a framework that owns all device
 * memory through its own pool, a host that allows no allocation once running,
 * a process that must not grow its footprint).
 *   cfg:   as for lbm_create; precision must be LBM_FP64 (the arithmetic and the
 *          result are those of an LBM_FP64 context, bit for bit).
 *   f_in:  device pointer, q * nx * ny doubles, the populations before the step
 *          (plane-major oracle layout, as lbm_get_populations writes them).
 *   f_out: device pointer, same size, receives the populations after the step;
 *          must not overlap f_in.
 *   stats: host pointer or NULL; receives this step's sums (stats->step is 1).
 *   cuda_stream: cudaStream_t as void*; the call synchronises it before returning.
 * Scratch (block sums, Ehrenfests' candidates, selected sites, counters, the
 * stats record) comes from one file-scope static device array of
 * LBM_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until
 * the process exits.  Lattices above LBM_NOALLOC_MAX_SITES sites, or whose
 * scratch would not fit the array (any lattice up to 512 x 512 fits), are
 * rejected with LBM_ERR_INVALID_ARG and a message in lbm_last_error(NULL).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  The call never calls cudaMalloc, cudaFree or any
 * allocating routine.  All calls share the one array, and each clears what must
 * start at zero: calls that overlap on the GPU (other threads or streams) race
 * on it and must be serialised by the caller. */
lbm_status lbm_step_noalloc(const lbm_config *cfg, const double *f_in, double *f_out,
                            lbm_step_stats *stats, void *cuda_stream);

/* Static name of a status code. */
const char *lbm_status_string(lbm_status s);

/* LBM_ABI_VERSION of the loaded library. */
int32_t lbm_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
