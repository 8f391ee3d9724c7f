/*
 * lbm_oracle.h -- FP64 CPU oracle for the entropy-limited LBGK step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  It
 * shares no source, header, table or constant with the CUDA library
 * (include/lbm.h, paper_0704_0043_gb300/csrc/); neither side includes or
 * links the other.
 *
 * What it computes (Brownlee, Gorban, Levesley, "Nonequilibrium entropy
 * limiters in lattice Boltzmann methods", Physica A 2007):
 *   - free flight (Sec. 2) in pull form with halfway bounce-back walls and a
 *     moving lid (Sec. 4.4.1),
 *   - moments (Eq. macro_dis), polynomial quasiequilibria (Eq. polyeq1d,
 *     Eq. polyeq2d),
 *   - the LBGK collision with over-relaxation (Eq. collLBGK, Eq. lbgkLB),
 *   - the nonequilibrium entropy in its quadratic Kullback form (Eq. DelS
 *     and the quadratic approximation that follows it in Sec. 3.6),
 *   - optionally entropic quasiequilibria (Eq. entropiceq1d, Eq. maxwellian)
 *     with the exact relative entropy of Eq. DelS,
 *   - the limiters f -> f* + phi (f - f*) (Eq. LimGenF): the positivity rule
 *     (Sec. 3.1), the entropic median filter (Sec. 3.5, Sec. 4.3.2, Sec. 4.4)
 *     and Ehrenfests' trimming with at most k sites per step (Sec. 3.2),
 *   - the dissipation monitors of Sec. 3.4 and Sec. 4.3.1.
 * Every operation is plain IEEE double arithmetic, evaluated left to right,
 * with no contraction into FMA (build with -ffp-contract=off).
 *
 * Population layout: plane-major, f[k * ny * nx + j * nx + i] for direction
 * k, row j (y, upward) and column i (x).  D1Q3 uses ny = 1.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_D1Q3 1
#define ORC_D2Q9 2

#define ORC_BC_WALLS 0    /* D2Q9: cavity (three still walls, lid on top); D1Q3: closed tube ends */
#define ORC_BC_PERIODIC 1 /* periodic in every direction */
#define ORC_BC_CHANNEL 2  /* D2Q9: periodic in x, still wall at the bottom, lid on top */
/* D2Q9 cavities whose outer ring of nodes lies on the walls (boundary nodes, Sec. 4.4):
 * boundary nodes are not collided and not limited; after free flight the
 * populations they lack (those that would come from outside the lattice) are
 * supplied by the wall rule.  The lid is the top row without its two corners,
 * moving with (u_lid, 0); the other walls and the four corners are at rest. */
#define ORC_BC_NODE_WALLS 3 /* bounce-back: f_k = f_opp(k) + 6 W_k rho_wall (v_k . u_wall) (Sec. 4.4.1) */
#define ORC_BC_DIFFUSIVE 4  /* diffusive Maxwell wall: f_k = gamma f*_k(1, u_wall) (Sec. 4.4.2);
                               bounce-back in the corners */

#define ORC_LIM_POSITIVITY 1u
#define ORC_LIM_EHRENFEST 2u
#define ORC_LIM_MEDIAN 4u
#define ORC_LIM_SMOOTH 8u     /* ensemble-dependent smooth limiter, Eq. smooth1 with alpha = delta / E(dS)^k */
#define ORC_LIM_THRESHOLD 16u /* threshold filter, dS_t = max(c E(dS), delta) (Sec. 3.4, Sec. 4.3.2) */
#define ORC_LIM_ENTTHRESH 32u /* threshold filter with dS_0 solving Eq. EntThresh, dS_t = max(dS_0, delta) */

#define ORC_MEDIAN_THRESHOLD 0 /* dS_t = max(dS_med, delta); phi = sqrt(dS_t/dS) where dS > dS_t */
#define ORC_MEDIAN_GATE 1      /* phi = sqrt(dS_med/dS) where dS > delta and dS_med < dS */

#define ORC_EQ_POLYNOMIAL 0 /* Eq. polyeq1d / polyeq2d; dS in its quadratic form */
#define ORC_EQ_ENTROPIC 1   /* Eq. entropiceq1d / maxwellian; dS = sum_k f_k ln(f_k / f*_k) (Eq. DelS) */

#define ORC_COLL_LBGK 0 /* f' = f* + (2 beta - 1)(f* - f), Eq. lbgkLB */
#define ORC_COLL_ELBM 1 /* f' = (1 - beta) f + beta f~, f~ = f + alpha (f* - f), S(f~) = S(f) (Eq. elbm, Eq. entropy_estimate) */

typedef struct {
    int lattice;            /* ORC_D1Q3 or ORC_D2Q9 */
    int nx, ny;             /* lattice size; ny = 1 for D1Q3 */
    int boundary;           /* ORC_BC_* */
    double beta;            /* LBGK over-relaxation parameter, Eq. collLBGK */
    double u_lid;           /* lid x-velocity (D2Q9 top wall) */
    double rho_wall;        /* density used in the moving-wall term */
    unsigned limiters;      /* ORC_LIM_* bit set */
    double delta_median;    /* median-filter tolerance */
    double delta_ehrenfest; /* Ehrenfests' threshold */
    long long k_max;        /* at most this many Ehrenfests' sites per step */
    int median_mode;        /* ORC_MEDIAN_* */
    int equilibrium;        /* ORC_EQ_* */
    double smooth_delta;    /* ORC_LIM_SMOOTH: alpha = smooth_delta / E(dS)^smooth_k */
    double smooth_k;        /* ORC_LIM_SMOOTH: exponent k (> 0) */
    double threshold_c;     /* ORC_LIM_THRESHOLD: dS_0 = threshold_c * E(dS) */
    double threshold_delta; /* ORC_LIM_THRESHOLD / ORC_LIM_ENTTHRESH: dS_t = max(dS_0, threshold_delta) */
    double entthresh_delta0; /* ORC_LIM_ENTTHRESH: delta_0 of Eq. EntThresh (Eq. LimEntLim's bound) */
    int collision;           /* ORC_COLL_* (ELBM needs ORC_EQ_ENTROPIC) */
    int phi_rule;            /* ORC_PHI_*: how the filters with a target dS_t (median, threshold) limit */
} orc_config;

/* ORC_PHI_HOMOTHETY: phi = sqrt(dS_t / dS) (Eq. entrHom, the quadratic approximation).
 * ORC_PHI_ENTROPY (entropic f* only): phi solves dS(f* + phi (f' - f*)) = dS_t, i.e.
 * S(f* + phi (f' - f*)) = S(f*) - dS_t (Sec. 3.7), by bisection on [0, 1]. */
#define ORC_PHI_HOMOTHETY 0
#define ORC_PHI_ENTROPY 1

/*
 * The ensemble-dependent limiters use E(dS), the mean of dS(f') over the
 * sites that are not flagged and have a finite dS, of the state being limited
 * (before any limiter).  Smooth limiter (Eq. smooth1): phi = 1 / (1 + alpha
 * dS^k), alpha = smooth_delta / E^k, phi = 1 where E <= 0 or dS = 0.
 * Threshold filter (Sec. 3.4 with dS_0 = c E as in Sec. 4.3.2): phi =
 * sqrt(dS_t / dS) where dS > dS_t.  ORC_LIM_ENTTHRESH takes dS_0 from Eq.
 * EntThresh on the ensemble's own distribution of dS (the limit of the
 * histogram estimate of Sec. 3.4): sum_s max(dS_s - dS_0, 0) =
 * delta_0 [1 - (2 beta - 1)^2] sum_s dS_s over the same sites as E, solved
 * exactly (its left side is continuous, piecewise linear and decreasing).
 * Parity unpinned against a GPU path: no GPU path implements it yet.  All limiters compose as the minimum of
 * their phi, before Ehrenfests' step.
 *
 * With entropic quasiequilibria (ORC_EQ_ENTROPIC) dS is the exact relative
 * entropy, which is +inf for a state with a negative population (outside the
 * domain of S; such a site is not flagged bad).  The entropy productions are
 * then evaluated as entropy differences at the sites where both entropies are
 * finite:  dS_lbgk = sum [dS(f_in) - dS(f')],  dS_lim = sum [dS(f') - dS(f_out)]
 * over the limited sites plus dS(f_lim) w.r.t. f*(m(f_lim)) at each
 * Ehrenfests' site, and sum_dS skips infinite values.
 */
typedef struct {
    double mass;      /* sum of rho over sites (after free flight) */
    double sum_dS;    /* sum of dS(f') over sites, f' = post-collision, pre-limiter */
    double dS_lbgk;   /* [1 - (2 beta - 1)^2] * sum of dS(f_in), Sec. 3.4 */
    double dS_lim;    /* entropy added by the limiters, quadratic approximation */
    long long n_pos;  /* sites where the positivity rule acted (phi_pos < 1) */
    long long n_med;  /* sites where the median filter acted (phi_med < 1) */
    long long n_ehr;  /* sites equilibrated by Ehrenfests' step */
    long long n_cand; /* sites with dS(f') > delta_ehrenfest */
    long long n_bad;  /* sites with rho <= 0, a nonpositive f*_i or a nonfinite value */
} orc_stats;

/* Polynomial quasiequilibrium f*(rho, u) at one site (Eq. polyeq1d / Eq. polyeq2d). */
void orc_feq(int lattice, double rho, double ux, double uy, double *feq);

/*
 * Entropic quasiequilibrium f*(rho, u) at one site: Eq. entropiceq1d (D1Q3;
 * the printed f2* is the v = +1 population and f3* the v = -1 one, the order
 * in which sum_k v_k f*_k = rho u) and Eq. maxwellian (D2Q9).  Defined for
 * |u_x|, |u_y| < 1; returns 0 there, else 1 (feq is then left unspecified).
 */
int orc_feq_entropic(int lattice, double rho, double ux, double uy, double *feq);

/* Lattice entropy with 0 ln 0 = 0: D2Q9 S(f) = -sum_k f_k ln(f_k / W_k) (Sec. 4.1, Sec. 3.6);
 * D1Q3 S = -H, H = f_rest ln(f_rest / 4) + f_left ln f_left + f_right ln f_right (Sec. 4.1). */
double orc_entropy(int lattice, const double *f);

/* Relative entropy sum_k f_k ln(f_k / fs_k) (Eq. DelS) of q populations, 0 ln 0 = 0, +inf if some f_k < 0. */
double orc_rel_entropy(int q, const double *f, const double *fs);

/*
 * ELBM (Sec. 3.7, Eq. elbm; the LBGK step of Eq. lbgkLB is its alpha = 2 case):
 * the nontrivial root alpha > 1 of S(f + alpha (f* - f)) = S(f) for one site's
 * populations f and their entropic f*, by bisection on [1, alpha_max] to a
 * bracket of 1e-15, returning the end with no entropy decrease (Sec. 4.2).
 * alpha_max is the positivity boundary of the line; where the entropy is still
 * above S(f) there, no root exists in the positive cone and alpha_max is
 * returned (the positivity rule, Sec. 3.1).  f = f* returns 2.  The entropy
 * difference is evaluated as dS(f) - dS(f~) (Eq. DelS, same f*), which equals
 * S(f~) - S(f) for states with the moments of f*.  *pos (may be NULL) is set
 * to 1 when the positivity boundary was taken.
 */
double orc_elbm_alpha(int q, const double *f, const double *fs, int *pos);

/* Sec. 3.7: the phi in [0, 1] with dS(fs + phi (fp - fs)) = target (Eq. DelS), for
 * 0 <= target < dS(fp): bisection to a bracket of 1e-15, returning its lower end
 * (the state it gives has dS at most target). */
double orc_phi_entropy(int q, const double *fp, const double *fs, double target);

/* Moments rho, u of one site's populations (Eq. macro_dis). */
void orc_site_moments(int lattice, const double *f, double *rho, double *ux, double *uy);

/* f = f*(rho(x), u(x)) for every site.  uy may be NULL for D1Q3. */
void orc_init(const orc_config *cfg, const double *rho, const double *ux, const double *uy, double *f);

/* Moments of every site of a stored field.  uy may be NULL for D1Q3. */
void orc_moments(const orc_config *cfg, const double *f, double *rho, double *ux, double *uy);

/*
 * One limited LBGK step: free flight, collision, limiters, store.
 * f_st: stored field (input), f_out: next stored field (may not alias f_st).
 * Optional outputs (NULL to skip): dS_field = dS(f') per site (pre-limiter),
 * phi_field = final phi per site before Ehrenfests' step, sel / n_sel = the
 * sites Ehrenfests' step equilibrated, in selection order (sel needs room for
 * min(k_max, sites) entries), stats.
 * Returns 0, or 1 if any site was flagged (n_bad > 0).
 */
int orc_step(const orc_config *cfg, const double *f_st, double *f_out, double *dS_field,
             double *phi_field, long long *sel, long long *n_sel, orc_stats *stats);

/* nsteps steps in place (ping-pong through an internal buffer); stats of the last step. */
int orc_run(const orc_config *cfg, double *f, long long nsteps, orc_stats *stats);

/* dS(f') of the collision the next step would perform, without limiters. */
int orc_delta_s(const orc_config *cfg, const double *f_st, double *dS_field);

/*
 * Limiters applied to the stored field itself (no free flight, no collision):
 * f' := f_st, f* := f*(m(f_st)).  Same optional outputs as orc_step.
 */
int orc_limit(const orc_config *cfg, unsigned limiters, const double *f_st, double *f_out,
              double *dS_field, double *phi_field, long long *sel, long long *n_sel,
              orc_stats *stats);

#ifdef __cplusplus
}
#endif
#endif
