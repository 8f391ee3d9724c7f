/*
 * lbm_oracle.c -- FP64 CPU oracle for the entropy-limited LBGK step.
 *
 * TEST INFRASTRUCTURE ONLY: see lbm_oracle.h.  Plain, slow, single-threaded
 * C.  Every floating-point expression is written in the order it is meant to
 * be evaluated (left to right) and the file is built with -ffp-contract=off,
 * so no product is fused into an FMA.
 *
 * One step (Eq. lbgkLB with the limiter as a post-processing routine after
 * the collision, Sec. 4.3.2), in the order the paper applies it:
 *   1. free flight, pull form:  f_in_k(x) = f_k(x - v_k)                Sec. 2
 *      a link that leaves the lattice is reflected (halfway bounce-back,
 *      Sec. 4.4.1); a link through the moving lid gains 6 W_k rho_w (v_k . u_w)
 *   2. moments rho, u                                                   Eq. macro_dis
 *   3. polynomial quasiequilibrium f*                                   Eq. polyeq1d / polyeq2d
 *      (or the entropic one                                             Eq. entropiceq1d / maxwellian)
 *   4. LBGK collision  f' = f* + (2 beta - 1)(f* - f_in)                Eq. collLBGK, lbgkLB
 *   5. dS(f') = sum_k (f'_k - f*_k)^2 / f*_k                            Sec. 3.6, quadratic form of Eq. DelS
 *      (entropic f*: dS(f') = sum_k f'_k ln(f'_k / f*_k)                Eq. DelS)
 *   6. phi_pos: positivity rule, closest nonnegative point of the line
 *      through f' and f*                                                Sec. 3.1
 *   7. phi_med: median of dS over the stencil, homothety sqrt(dS_t/dS)  Sec. 3.5, Eq. entrHom
 *      phi_smooth = 1 / (1 + alpha dS^k), alpha = delta / E(dS)^k        Eq. smooth1 (Sec. 4.3.2)
 *      phi_thr = sqrt(dS_t / dS), dS_t = max(c E(dS), delta)            Sec. 3.4, Eq. entrHom
 *   8. phi = min of the limiters' phi;  f_out = f* + phi (f' - f*)      Eq. LimGenF
 *   9. Ehrenfests' step f -> f* at the (at most k) sites of largest
 *      dS > delta, ties broken by lower site index                      Sec. 3.2, Sec. 4.3.2
 *  10. sums: mass, sum dS, LBGK and limiter entropy production          Sec. 3.4, Sec. 4.3.1
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 (Sec. 4.1): 0 rest, 1 east, 2 north, 3 west, 4 south, 5 NE, 6 NW, 7 SW, 8 SE. */
static const int cx9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int cy9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int opp9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* D2Q9 lattice weights W_0 = 4/9, W_1..4 = 1/9, W_5..8 = 1/36 (Sec. 4.1). */
static double w9(int k)
{
    if (k == 0) return 4.0 / 9.0;
    if (k < 5) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

/* D1Q3 (Sec. 4.1): the paper's f1 (rest), f2 (left, v = -1), f3 (right, v = +1) as 0, 1, 2. */
static const int cx3[3] = {0, -1, 1};
static const int opp3[3] = {0, 2, 1};

static int nq(int lattice) { return lattice == ORC_D1Q3 ? 3 : 9; }

void orc_feq(int lattice, double rho, double ux, double uy, double *feq)
{
    if (lattice == ORC_D1Q3) {
        /* Eq. polyeq1d, term by term as printed. */
        double u = ux;
        double uu = u * u;
        feq[0] = ((2.0 * rho) / 3.0) * (1.0 - (3.0 * uu) / 2.0);
        feq[1] = (rho / 6.0) * ((1.0 - 3.0 * u) + 3.0 * uu);
        feq[2] = (rho / 6.0) * ((1.0 + 3.0 * u) + 3.0 * uu);
        return;
    }
    /* Eq. polyeq2d: f*_k = rho W_k (1 + 3 v.u + 9 (v.u)^2 / 2 - 3 u^2 / 2). */
    double usq = ux * ux + uy * uy;
    for (int k = 0; k < 9; ++k) {
        double c = (double)cx9[k] * ux + (double)cy9[k] * uy;
        feq[k] = (rho * w9(k)) * (((1.0 + 3.0 * c) + (9.0 * (c * c)) / 2.0) - (3.0 * usq) / 2.0);
    }
}

int orc_feq_entropic(int lattice, double rho, double ux, double uy, double *feq)
{
    if (lattice == ORC_D1Q3) {
        /* Eq. entropiceq1d.  As printed, f2* - f3* = rho u, i.e. the printed f2*
         * is the population whose velocity makes sum_k v_k f*_k = rho u hold
         * (Eq. macro_dis): v = +1.  Index 1 (v = -1) takes the printed f3*. */
        if (!(fabs(ux) < 1.0)) return 1;
        double u = ux;
        double sq = sqrt(1.0 + 3.0 * (u * u));
        feq[0] = ((2.0 * rho) / 3.0) * (2.0 - sq);
        feq[1] = -(rho / 6.0) * ((3.0 * u + 1.0) - 2.0 * sq);
        feq[2] = (rho / 6.0) * ((3.0 * u - 1.0) + 2.0 * sq);
        return 0;
    }
    /* Eq. maxwellian: f*_k = rho W_k prod_{j = x, y} (2 - sqrt(1 + 3 u_j^2))
     * ((2 u_j + sqrt(1 + 3 u_j^2)) / (1 - u_j))^{v_kj}, v_kj in {-1, 0, 1}. */
    if (!(fabs(ux) < 1.0) || !(fabs(uy) < 1.0)) return 1;
    double u[2] = {ux, uy};
    double A[2], X[2];
    for (int j = 0; j < 2; ++j) {
        double sq = sqrt(1.0 + 3.0 * (u[j] * u[j]));
        A[j] = 2.0 - sq;
        X[j] = (2.0 * u[j] + sq) / (1.0 - u[j]);
    }
    for (int k = 0; k < 9; ++k) {
        int v[2] = {cx9[k], cy9[k]};
        double f = rho * w9(k);
        for (int j = 0; j < 2; ++j) {
            double P = A[j];
            if (v[j] == 1) P = A[j] * X[j];
            if (v[j] == -1) P = A[j] / X[j];
            f = f * P;
        }
        feq[k] = f;
    }
    return 0;
}

double orc_entropy(int lattice, const double *f)
{
    double h = 0.0;
    if (lattice == ORC_D1Q3) {
        /* Sec. 4.1: H = f1 log(f1/4) + f2 log(f2) + f3 log(f3), S = -H */
        if (f[0] > 0.0) h += f[0] * log(f[0] / 4.0);
        if (f[1] > 0.0) h += f[1] * log(f[1]);
        if (f[2] > 0.0) h += f[2] * log(f[2]);
        return -h;
    }
    for (int k = 0; k < 9; ++k)
        if (f[k] > 0.0) h += f[k] * log(f[k] / w9(k));
    return -h;
}

double orc_rel_entropy(int q, const double *f, const double *fs)
{
    /* Eq. DelS: dS = sum_k f_k ln(f_k / f*_k).  A negative population lies
     * outside the domain of S: dS = +inf.  A zero one contributes 0 ln 0 = 0. */
    for (int k = 0; k < q; ++k)
        if (f[k] < 0.0) return INFINITY;
    double s = 0.0;
    for (int k = 0; k < q; ++k) {
        if (f[k] > 0.0) s += f[k] * log(f[k] / fs[k]);
        else if (!(f[k] == 0.0)) return NAN;
    }
    return s;
}

double orc_elbm_alpha(int q, const double *f, const double *fs, int *pos)
{
    if (pos) *pos = 0;
    int same = 1;
    for (int k = 0; k < q; ++k)
        if (f[k] != fs[k]) same = 0;
    if (same) return 2.0;
    /* positivity boundary of f + alpha (f* - f): the smallest f_k / (f_k - f*_k) over f*_k < f_k */
    double amax = INFINITY;
    for (int k = 0; k < q; ++k)
        if (fs[k] < f[k]) {
            double r = f[k] / (f[k] - fs[k]);
            if (r < amax) amax = r;
        }
    double g[9];
    double ds0 = orc_rel_entropy(q, f, fs);
    /* h(alpha) = S(f~) - S(f) = dS(f) - dS(f~) */
    for (int k = 0; k < q; ++k) g[k] = f[k] + amax * (fs[k] - f[k]);
    for (int k = 0; k < q; ++k)
        if (g[k] < 0.0) g[k] = 0.0; /* the boundary itself: the vanishing population is zero */
    if (ds0 - orc_rel_entropy(q, g, fs) >= 0.0) {
        if (pos) *pos = 1;
        return amax;
    }
    double lo = 1.0, hi = amax;
    for (int it = 0; it < 200 && hi - lo > 1e-15; ++it) {
        double mid = 0.5 * (lo + hi);
        for (int k = 0; k < q; ++k) g[k] = f[k] + mid * (fs[k] - f[k]);
        if (ds0 - orc_rel_entropy(q, g, fs) >= 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

double orc_phi_entropy(int q, const double *fp, const double *fs, double target)
{
    /* dS(fs + phi (fp - fs)) grows with phi on [0, 1] (0 at phi = 0, convex) */
    double g[9];
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15; ++it) {
        double mid = 0.5 * (lo + hi);
        for (int k = 0; k < q; ++k) g[k] = fs[k] + mid * (fp[k] - fs[k]);
        if (orc_rel_entropy(q, g, fs) <= target)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* f* of the configured kind; returns 1 where it does not exist. */
static int site_feq(const orc_config *cfg, double rho, double ux, double uy, double *fs)
{
    if (cfg->equilibrium == ORC_EQ_ENTROPIC) return orc_feq_entropic(cfg->lattice, rho, ux, uy, fs);
    orc_feq(cfg->lattice, rho, ux, uy, fs);
    return 0;
}

/* dS(f) of the configured kind (quadratic form, or Eq. DelS for entropic f*). */
static double site_dS(const orc_config *cfg, int q, const double *f, const double *fs)
{
    if (cfg->equilibrium == ORC_EQ_ENTROPIC) return orc_rel_entropy(q, f, fs);
    double s = 0.0;
    for (int k = 0; k < q; ++k) {
        double d = f[k] - fs[k];
        s += (d * d) / fs[k];
    }
    return s;
}

/* A dS value that is allowed to be +inf (entropic f*, population below zero). */
static int dS_ok(const orc_config *cfg, double x)
{
    return cfg->equilibrium == ORC_EQ_ENTROPIC ? !isnan(x) : isfinite(x);
}

void orc_site_moments(int lattice, const double *f, double *rho, double *ux, double *uy)
{
    /* Eq. macro_dis: rho = sum_k f_k, rho u = sum_k v_k f_k, summed in k order. */
    double r = 0.0, jx = 0.0, jy = 0.0;
    if (lattice == ORC_D1Q3) {
        for (int k = 0; k < 3; ++k) {
            r += f[k];
            jx += (double)cx3[k] * f[k];
        }
    } else {
        for (int k = 0; k < 9; ++k) {
            r += f[k];
            jx += (double)cx9[k] * f[k];
            jy += (double)cy9[k] * f[k];
        }
    }
    *rho = r;
    *ux = jx / r;
    *uy = (lattice == ORC_D1Q3) ? 0.0 : jy / r;
}

void orc_init(const orc_config *cfg, const double *rho, const double *ux, const double *uy, double *f)
{
    int q = nq(cfg->lattice);
    long long n = (long long)cfg->nx * cfg->ny;
    double feq[9];
    for (long long s = 0; s < n; ++s) {
        for (int k = 0; k < q; ++k) feq[k] = NAN;
        site_feq(cfg, rho[s], ux[s], uy ? uy[s] : 0.0, feq);
        for (int k = 0; k < q; ++k) f[k * n + s] = feq[k];
    }
}

void orc_moments(const orc_config *cfg, const double *f, double *rho, double *ux, double *uy)
{
    int q = nq(cfg->lattice);
    long long n = (long long)cfg->nx * cfg->ny;
    double fl[9], r, a, b;
    for (long long s = 0; s < n; ++s) {
        for (int k = 0; k < q; ++k) fl[k] = f[k * n + s];
        orc_site_moments(cfg->lattice, fl, &r, &a, &b);
        rho[s] = r;
        ux[s] = a;
        if (uy) uy[s] = b;
    }
}

/* Step 1: the populations that arrive at site (i, j) after free flight. */
static void pull(const orc_config *cfg, const double *f, int i, int j, double *fin)
{
    int nx = cfg->nx, ny = cfg->ny;
    long long n = (long long)nx * ny;
    if (cfg->lattice == ORC_D1Q3) {
        for (int k = 0; k < 3; ++k) {
            int si = i - cx3[k];
            if (cfg->boundary == ORC_BC_PERIODIC) si = (si + nx) % nx;
            if (si < 0 || si >= nx)
                fin[k] = f[opp3[k] * n + i]; /* closed end: halfway bounce-back */
            else
                fin[k] = f[k * n + si];
        }
        return;
    }
    int wrapx = cfg->boundary == ORC_BC_PERIODIC || cfg->boundary == ORC_BC_CHANNEL;
    int wrapy = cfg->boundary == ORC_BC_PERIODIC;
    for (int k = 0; k < 9; ++k) {
        int si = i - cx9[k], sj = j - cy9[k];
        if (wrapx) si = (si + nx) % nx;
        if (wrapy) sj = (sj + ny) % ny;
        if (si >= 0 && si < nx && sj >= 0 && sj < ny) {
            fin[k] = f[k * n + (long long)sj * nx + si];
        } else {
            /* Halfway bounce-back: the population that left (i, j) towards the
             * wall in direction opp(k) comes back as direction k.  A link
             * through the lid (source above the top row) also picks up the
             * moving-wall momentum 6 W_k rho_w (v_k . u_w) with u_w = (u_lid, 0). */
            double v = f[opp9[k] * n + (long long)j * nx + i];
            if (sj > ny - 1) v += ((6.0 * w9(k)) * cfg->rho_wall) * ((double)cx9[k] * cfg->u_lid);
            fin[k] = v;
        }
    }
}

/* Cavities with boundary nodes on the walls (ORC_BC_NODE_WALLS, ORC_BC_DIFFUSIVE). */
static int node_walls(const orc_config *cfg)
{
    return cfg->lattice == ORC_D2Q9 &&
           (cfg->boundary == ORC_BC_NODE_WALLS || cfg->boundary == ORC_BC_DIFFUSIVE);
}

static int boundary_node(const orc_config *cfg, int i, int j)
{
    return node_walls(cfg) && (i == 0 || i == cfg->nx - 1 || j == 0 || j == cfg->ny - 1);
}

static int site_feq(const orc_config *cfg, double rho, double ux, double uy, double *fs);

/*
 * Step 1 at a boundary node (Sec. 4.4): free flight brings the populations whose
 * source lies on the lattice; the others come from the wall rule.  The lid is
 * the top row without its corners and moves with (u_lid, 0); the other walls
 * and the corners are at rest.
 *  - bounce-back (Sec. 4.4.1): f_k = f_opp(k) + 6 W_k rho_wall (v_k . u_wall), the
 *    population that has just arrived moving the other way, plus the momentum
 *    of the moving wall;
 *  - diffusive Maxwell wall (Sec. 4.4.2): f_k = gamma f*_k(1, u_wall) with
 *    gamma = (sum of the arrived f_opp(k)) / (sum of f*_k(1, u_wall)), both sums
 *    over the populations the wall returns, so that the wall returns the mass it
 *    receives; in the corners, bounce-back.
 * In a corner two of the missing populations point out of the lattice again
 * (their opposite is missing too); they never reach the fluid and keep their
 * stored values.
 */
static void wall_node(const orc_config *cfg, const double *f, int i, int j, double *fo)
{
    int nx = cfg->nx, ny = cfg->ny;
    long long n = (long long)nx * ny, s = (long long)j * nx + i;
    int known[9];
    for (int k = 0; k < 9; ++k) {
        int si = i - cx9[k], sj = j - cy9[k];
        known[k] = si >= 0 && si < nx && sj >= 0 && sj < ny;
        fo[k] = known[k] ? f[k * n + (long long)sj * nx + si] : 0.0;
    }
    int corner = (i == 0 || i == nx - 1) && (j == 0 || j == ny - 1);
    int lid = j == ny - 1 && !corner;
    double uw = lid ? cfg->u_lid : 0.0;
    if (cfg->boundary == ORC_BC_DIFFUSIVE && !corner) {
        double fw[9];
        site_feq(cfg, 1.0, uw, 0.0, fw);  /* density is a linear factor of f*: take 1 */
        double arrived = 0.0, returned = 0.0;
        for (int k = 0; k < 9; ++k)
            if (!known[k]) {
                arrived += fo[opp9[k]];
                returned += fw[k];
            }
        double gamma = arrived / returned;
        for (int k = 0; k < 9; ++k)
            if (!known[k]) fo[k] = gamma * fw[k];
        return;
    }
    for (int k = 0; k < 9; ++k) {
        if (known[k]) continue;
        if (known[opp9[k]]) {
            double v = fo[opp9[k]];
            if (lid) v += ((6.0 * w9(k)) * cfg->rho_wall) * ((double)cx9[k] * uw);
            fo[k] = v;
        } else {
            fo[k] = f[k * n + s];
        }
    }
}

/* Mass a boundary node carries into the next step: the populations whose
 * destination lies on the lattice (the others have been returned by the wall
 * rule and are never streamed again). */
static double wall_node_mass(const orc_config *cfg, int i, int j, const double *fo)
{
    double m = 0.0;
    for (int k = 0; k < 9; ++k) {
        int di = i + cx9[k], dj = j + cy9[k];
        if (di >= 0 && di < cfg->nx && dj >= 0 && dj < cfg->ny) m += fo[k];
    }
    return m;
}

/*
 * Steps 2-5 at one site.  Writes f* and f' (q values each), dS(f') and
 * dS(f_in); returns 1 if the site cannot be limited (rho <= 0, no f* or
 * f*_k <= 0 for some k, or a nonfinite value), in which case *dS = +inf.
 * With entropic f*, dS(f') and dS(f_in) may be +inf without the site being
 * flagged (a negative population).
 */
static int site_collide(const orc_config *cfg, const double *fin, double *fs, double *fp,
                        double *dS, double *dS_in, double *rho_out)
{
    int q = nq(cfg->lattice);
    double rho, ux, uy;
    orc_site_moments(cfg->lattice, fin, &rho, &ux, &uy);
    int bad = !(rho > 0.0) || !isfinite(rho) || !isfinite(ux) || !isfinite(uy);
    if (site_feq(cfg, rho, ux, uy, fs)) {
        bad = 1;
        for (int k = 0; k < q; ++k) fs[k] = 0.0;
    }
    double a = 2.0 * cfg->beta - 1.0;
    for (int k = 0; k < q; ++k) fp[k] = fs[k] + a * (fs[k] - fin[k]);
    for (int k = 0; k < q; ++k)
        if (!(fs[k] > 0.0) || !isfinite(fs[k]) || !isfinite(fin[k])) bad = 1;
    if (cfg->collision == ORC_COLL_ELBM && !bad) {
        /* Eq. elbm: F(f) = (1 - beta) f + beta f~ = f + beta alpha (f* - f) */
        double alpha = orc_elbm_alpha(q, fin, fs, NULL);
        for (int k = 0; k < q; ++k) fp[k] = fin[k] + (cfg->beta * alpha) * (fs[k] - fin[k]);
    }
    double s = bad ? 0.0 : site_dS(cfg, q, fp, fs);
    double si = bad ? 0.0 : site_dS(cfg, q, fin, fs);
    if (!dS_ok(cfg, s) || !dS_ok(cfg, si)) bad = 1;
    *rho_out = rho;
    *dS = bad ? INFINITY : s;
    *dS_in = bad ? 0.0 : si;
    return bad;
}

static void sort_small(double *v, int m)
{
    for (int a = 1; a < m; ++a) {
        double x = v[a];
        int b = a - 1;
        while (b >= 0 && v[b] > x) {
            v[b + 1] = v[b];
            --b;
        }
        v[b + 1] = x;
    }
}

/*
 * Median-filter stencil at site (i, j) (Sec. 3.5; wall rules of Sec. 4.4).
 * The paper's boundary nodes sit on the walls and are not filtered; here the
 * walls lie half a link outside the lattice, so every lattice node is a fluid
 * node.  A node next to one wall uses itself and its two neighbours along that
 * wall; a node next to two walls (a corner node) uses itself and its inward
 * neighbour along x and along y; all other nodes use the 3x3 block.  D1Q3:
 * three points; the two end sites are not filtered.
 * Returns the stencil size (0 = not filtered) and the values in v.
 */
static int median_stencil(const orc_config *cfg, const double *dS, int i, int j, double *v)
{
    int nx = cfg->nx, ny = cfg->ny;
    if (cfg->lattice == ORC_D1Q3) {
        if (cfg->boundary == ORC_BC_PERIODIC) {
            v[0] = dS[(i - 1 + nx) % nx];
            v[1] = dS[i];
            v[2] = dS[(i + 1) % nx];
            return 3;
        }
        if (i == 0 || i == nx - 1) return 0;
        v[0] = dS[i - 1];
        v[1] = dS[i];
        v[2] = dS[i + 1];
        return 3;
    }
#define DS(a, b) dS[(long long)(b) * nx + (a)]
    if (node_walls(cfg)) {
        /* Sec. 4.4: boundary nodes are not filtered; a node next to one wall uses
         * the three nodes along that wall (itself and its two neighbours), a node
         * next to two walls itself and its inward neighbours along x and y; all
         * other nodes the 3x3 block. */
        if (boundary_node(cfg, i, j)) return 0;
        int nearx = i == 1 || i == nx - 2, neary = j == 1 || j == ny - 2;
        if (nearx && neary) {
            v[0] = DS(i, j);
            v[1] = DS(i == 1 ? 2 : nx - 3, j);
            v[2] = DS(i, j == 1 ? 2 : ny - 3);
            return 3;
        }
        if (neary) {
            v[0] = DS(i - 1, j);
            v[1] = DS(i, j);
            v[2] = DS(i + 1, j);
            return 3;
        }
        if (nearx) {
            v[0] = DS(i, j - 1);
            v[1] = DS(i, j);
            v[2] = DS(i, j + 1);
            return 3;
        }
        int m = 0;
        for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a) v[m++] = DS(i + a, j + b);
        return 9;
    }
    int wallx = cfg->boundary == ORC_BC_WALLS;
    int wally = cfg->boundary != ORC_BC_PERIODIC;
    int nearx = wallx && (i == 0 || i == nx - 1);
    int neary = wally && (j == 0 || j == ny - 1);
    if (nearx && neary) {
        int ii = (i == 0) ? 1 : nx - 2;
        int jj = (j == 0) ? 1 : ny - 2;
        v[0] = DS(i, j);
        v[1] = DS(ii, j);
        v[2] = DS(i, jj);
        return 3;
    }
    if (neary) {
        v[0] = DS((i - 1 + nx) % nx, j);
        v[1] = DS(i, j);
        v[2] = DS((i + 1) % nx, j);
        return 3;
    }
    if (nearx) {
        v[0] = DS(i, j - 1);
        v[1] = DS(i, j);
        v[2] = DS(i, j + 1);
        return 3;
    }
    int m = 0;
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) v[m++] = DS((i + a + nx) % nx, (j + b + ny) % ny);
    return 9;
#undef DS
}

typedef struct {
    double dS;
    long long s;
} cand_t;

static int dbl_desc(const void *pa, const void *pb)
{
    double a = *(const double *)pa, b = *(const double *)pb;
    return (a < b) - (a > b);
}

/*
 * Eq. EntThresh on the empirical distribution of the n values v: the dS_0 >= 0
 * with sum_s max(v_s - dS_0, 0) = rhs, for 0 <= rhs <= sum_s v_s.  With v
 * sorted in descending order and m values above dS_0 the left side is
 * S_m - m dS_0 (S_m the sum of the m largest), so dS_0 = (S_m - rhs) / m for
 * the m whose segment [v_(m+1), v_m] holds it.
 */
static double entthresh(double *v, long long n, double rhs)
{
    if (n <= 0 || !(rhs > 0.0)) return n > 0 ? INFINITY : 0.0;
    qsort(v, (size_t)n, sizeof(double), dbl_desc);
    double S = 0.0;
    for (long long m = 1; m <= n; ++m) {
        S += v[m - 1];
        double t = (S - rhs) / (double)m;
        double lo = m < n ? v[m] : 0.0;
        if (t >= lo) return t > 0.0 ? t : 0.0;
    }
    return 0.0;
}

static int cand_cmp(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    if (a->dS > b->dS) return -1;
    if (a->dS < b->dS) return 1;
    return (a->s < b->s) ? -1 : (a->s > b->s);
}

/*
 * The factor of a filter that brings dS = x down to the target t < x at site s
 * (fields fp, fs of n sites): the homothety sqrt(t / x) of Eq. entrHom, or, with
 * ORC_PHI_ENTROPY and entropic f*, the exact solve of Sec. 3.7.
 */
static double phi_to(const orc_config *cfg, int q, const double *fp, const double *fs, long long n,
                     long long s, double t, double x)
{
    if (cfg->phi_rule == ORC_PHI_ENTROPY && cfg->equilibrium == ORC_EQ_ENTROPIC) {
        double a[9], b[9];
        for (int k = 0; k < q; ++k) {
            a[k] = fp[k * n + s];
            b[k] = fs[k * n + s];
        }
        return orc_phi_entropy(q, a, b, t);
    }
    return sqrt(t / x);
}

/*
 * Steps 6-9 on per-site fields fs (f*), fp (f'), dS (dS(f')) and the bad-site
 * flags; writes f_out and accumulates the limiter sums into st.
 */
static void limit_core(const orc_config *cfg, unsigned limiters, const double *fs,
                       const double *fp, const double *dS, const unsigned char *bad,
                       double *f_out, double *phi_field, long long *sel, long long *n_sel,
                       orc_stats *st)
{
    int q = nq(cfg->lattice);
    int nx = cfg->nx;
    long long n = (long long)cfg->nx * cfg->ny;
    double *phi = (double *)malloc(sizeof(double) * (size_t)n);
    double v[9];
    /* E(dS): mean of dS(f') over the sites with a finite value, in site order */
    double e_sum = 0.0;
    long long e_cnt = 0;
    for (long long s = 0; s < n; ++s)
        if (!bad[s] && isfinite(dS[s])) {
            e_sum += dS[s];
            e_cnt++;
        }
    double E = e_cnt > 0 ? e_sum / (double)e_cnt : 0.0;
    double t_ent = 0.0;
    if (limiters & ORC_LIM_ENTTHRESH) {
        /* Eq. EntThresh over the same sites as E; dS_t = max(dS_0, delta) */
        double *v = (double *)malloc(sizeof(double) * (size_t)(e_cnt > 0 ? e_cnt : 1));
        long long m = 0;
        for (long long s = 0; s < n; ++s)
            if (!bad[s] && isfinite(dS[s])) v[m++] = dS[s];
        double a = 2.0 * cfg->beta - 1.0;
        double rhs = cfg->entthresh_delta0 * ((1.0 - a * a) * e_sum);
        t_ent = entthresh(v, m, rhs);
        if (t_ent < cfg->threshold_delta) t_ent = cfg->threshold_delta;
        free(v);
    }
    for (long long s = 0; s < n; ++s) {
        double phi_pos = 1.0, phi_med = 1.0, phi_ens = 1.0;
        if (!bad[s]) {
            if ((limiters & ORC_LIM_SMOOTH) && E > 0.0 && dS[s] > 0.0) {
                /* Eq. smooth1 with the ensemble-dependent alpha of Sec. 4.3.2 */
                double alpha = cfg->smooth_delta / pow(E, cfg->smooth_k);
                double p_s = 1.0 / (1.0 + alpha * pow(dS[s], cfg->smooth_k));
                if (p_s < phi_ens) phi_ens = p_s;
            }
            if ((limiters & ORC_LIM_ENTTHRESH) && dS[s] > t_ent) {
                double p_e = phi_to(cfg, q, fp, fs, n, s, t_ent, dS[s]);
                if (p_e < phi_ens) phi_ens = p_e;
            }
            if (limiters & ORC_LIM_THRESHOLD) {
                /* Sec. 3.4: dS_t = max(dS_0, delta), homothety where dS > dS_t */
                double t = cfg->threshold_c * E;
                if (t < cfg->threshold_delta) t = cfg->threshold_delta;
                if (dS[s] > t) {
                    double p_t = phi_to(cfg, q, fp, fs, n, s, t, dS[s]);
                    if (p_t < phi_ens) phi_ens = p_t;
                }
            }
            if (limiters & ORC_LIM_POSITIVITY) {
                /* Sec. 3.1: move along {f* + lambda (f' - f*)} to the positivity boundary. */
                for (int k = 0; k < q; ++k) {
                    double fpk = fp[k * n + s], fsk = fs[k * n + s];
                    if (fpk < 0.0) {
                        double r = fsk / (fsk - fpk);
                        if (r < phi_pos) phi_pos = r;
                    }
                }
            }
            if (limiters & ORC_LIM_MEDIAN) {
                int m = median_stencil(cfg, dS, (int)(s % nx), (int)(s / nx), v);
                if (m > 0) {
                    sort_small(v, m);
                    double med = v[m / 2];
                    double x = dS[s];
                    if (cfg->median_mode == ORC_MEDIAN_GATE) {
                        if (x > cfg->delta_median && med < x) phi_med = phi_to(cfg, q, fp, fs, n, s, med, x);
                    } else {
                        double t = med > cfg->delta_median ? med : cfg->delta_median;
                        if (x > t) phi_med = phi_to(cfg, q, fp, fs, n, s, t, x);
                    }
                }
            }
        }
        double p = phi_pos < phi_med ? phi_pos : phi_med;
        if (phi_ens < p) p = phi_ens;
        phi[s] = p;
        if (phi_pos < 1.0) st->n_pos++;
        if (phi_med < 1.0) st->n_med++;
        if (p < 1.0) {
            double fo[9], fsl[9];
            for (int k = 0; k < q; ++k) {
                double fsk = fs[k * n + s];
                f_out[k * n + s] = fsk + p * (fp[k * n + s] - fsk);
                fo[k] = f_out[k * n + s];
                fsl[k] = fsk;
            }
            if (cfg->equilibrium == ORC_EQ_ENTROPIC) {
                /* entropy difference dS(f') - dS(f_out) at the same f* */
                double d_out = orc_rel_entropy(q, fo, fsl);
                if (isfinite(dS[s]) && isfinite(d_out)) st->dS_lim += dS[s] - d_out;
            } else {
                st->dS_lim += (1.0 - p * p) * dS[s];
            }
        } else {
            /* phi = 1 is the identity: the post-collision state is stored as is. */
            for (int k = 0; k < q; ++k) f_out[k * n + s] = fp[k * n + s];
        }
    }
    if (phi_field)
        for (long long s = 0; s < n; ++s) phi_field[s] = phi[s];

    long long m_sel = 0;
    if (limiters & ORC_LIM_EHRENFEST) {
        cand_t *c = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
        long long nc = 0;
        for (long long s = 0; s < n; ++s) {
            if (!bad[s] && dS[s] > cfg->delta_ehrenfest) {
                c[nc].dS = dS[s];
                c[nc].s = s;
                nc++;
            }
        }
        st->n_cand += nc;
        qsort(c, (size_t)nc, sizeof(cand_t), cand_cmp);
        m_sel = nc < cfg->k_max ? nc : cfg->k_max;
        if (m_sel < 0) m_sel = 0;
        double fl[9], feq[9], r, a, b;
        for (long long t = 0; t < m_sel; ++t) {
            long long s = c[t].s;
            /* Ehrenfests' step: equilibrate the limited state at s, f -> f*(m(f)). */
            for (int k = 0; k < q; ++k) fl[k] = f_out[k * n + s];
            orc_site_moments(cfg->lattice, fl, &r, &a, &b);
            st->n_ehr++;
            if (sel) sel[t] = s;
            /* entropic f*: where the limited state's moments have no f* (|u_j|
             * rounded to 1 or more) the site keeps its populations */
            if (site_feq(cfg, r, a, b, feq)) continue;
            for (int k = 0; k < q; ++k) f_out[k * n + s] = feq[k];
            if (cfg->equilibrium == ORC_EQ_ENTROPIC) {
                /* the entropy the step adds: dS of the limited state w.r.t. its own f* */
                double d_l = orc_rel_entropy(q, fl, feq);
                if (isfinite(d_l)) st->dS_lim += d_l;
            } else {
                st->dS_lim += (phi[s] * phi[s]) * dS[s];
            }
        }
        free(c);
    }
    if (n_sel) *n_sel = m_sel;
    free(phi);
}

static int run_collide_and_limit(const orc_config *cfg, unsigned limiters, int do_stream,
                                 const double *f_st, double *f_out, double *dS_field,
                                 double *phi_field, long long *sel, long long *n_sel,
                                 orc_stats *stats)
{
    int q = nq(cfg->lattice);
    int nx = cfg->nx, ny = cfg->ny;
    long long n = (long long)nx * ny;
    double *fs = (double *)malloc(sizeof(double) * (size_t)(q * n));
    double *fp = (double *)malloc(sizeof(double) * (size_t)(q * n));
    double *dS = (double *)malloc(sizeof(double) * (size_t)n);
    unsigned char *bad = (unsigned char *)malloc((size_t)n);
    orc_stats st;
    memset(&st, 0, sizeof(st));
    double a = 2.0 * cfg->beta - 1.0;
    double sum_in = 0.0;
    double fin[9], fsl[9], fpl[9];
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long long s = (long long)j * nx + i;
            double rho, ds, dsi;
            int b;
            if (boundary_node(cfg, i, j)) {
                /* a boundary node: free flight and the wall rule (step), or its
                 * stored state (limiter pass); no collision, no limiter */
                if (do_stream)
                    wall_node(cfg, f_st, i, j, fin);
                else
                    for (int k = 0; k < 9; ++k) fin[k] = f_st[k * n + s];
                for (int k = 0; k < 9; ++k) {
                    fs[k * n + s] = fin[k];
                    fp[k * n + s] = fin[k];
                }
                dS[s] = 0.0;
                bad[s] = 2;
                st.mass += wall_node_mass(cfg, i, j, fin);
                continue;
            }
            if (do_stream) {
                pull(cfg, f_st, i, j, fin);
                b = site_collide(cfg, fin, fsl, fpl, &ds, &dsi, &rho);
            } else {
                /* Limiter pass on the stored state: f' := f, f* := f*(m(f)). */
                double ux, uy;
                for (int k = 0; k < q; ++k) fin[k] = f_st[k * n + s];
                orc_site_moments(cfg->lattice, fin, &rho, &ux, &uy);
                b = !(rho > 0.0) || !isfinite(rho) || !isfinite(ux) || !isfinite(uy);
                if (site_feq(cfg, rho, ux, uy, fsl)) {
                    b = 1;
                    for (int k = 0; k < q; ++k) fsl[k] = 0.0;
                }
                for (int k = 0; k < q; ++k) {
                    fpl[k] = fin[k];
                    if (!(fsl[k] > 0.0) || !isfinite(fsl[k]) || !isfinite(fin[k])) b = 1;
                }
                ds = b ? 0.0 : site_dS(cfg, q, fpl, fsl);
                if (!dS_ok(cfg, ds)) b = 1;
                if (b) ds = INFINITY;
                dsi = 0.0;
            }
            for (int k = 0; k < q; ++k) {
                fs[k * n + s] = fsl[k];
                fp[k * n + s] = fpl[k];
            }
            dS[s] = ds;
            bad[s] = (unsigned char)b;
            st.mass += rho;
            if (!b) {
                if (cfg->equilibrium == ORC_EQ_ENTROPIC) {
                    /* entropy differences where both entropies are finite */
                    if (isfinite(ds)) st.sum_dS += ds;
                    if (isfinite(ds) && isfinite(dsi)) sum_in += dsi - ds;
                } else {
                    st.sum_dS += ds;
                    sum_in += dsi;
                }
            } else {
                st.n_bad++;
            }
        }
    }
    if (cfg->equilibrium == ORC_EQ_ENTROPIC)
        st.dS_lbgk = do_stream ? sum_in : 0.0;
    else
        st.dS_lbgk = do_stream ? (1.0 - a * a) * sum_in : 0.0;
    limit_core(cfg, limiters, fs, fp, dS, bad, f_out, phi_field, sel, n_sel, &st);
    if (dS_field) memcpy(dS_field, dS, sizeof(double) * (size_t)n);
    if (stats) *stats = st;
    free(fs);
    free(fp);
    free(dS);
    free(bad);
    return st.n_bad > 0;
}

int orc_step(const orc_config *cfg, const double *f_st, double *f_out, double *dS_field,
             double *phi_field, long long *sel, long long *n_sel, orc_stats *stats)
{
    return run_collide_and_limit(cfg, cfg->limiters, 1, f_st, f_out, dS_field, phi_field, sel,
                                 n_sel, stats);
}

int orc_limit(const orc_config *cfg, unsigned limiters, const double *f_st, double *f_out,
              double *dS_field, double *phi_field, long long *sel, long long *n_sel,
              orc_stats *stats)
{
    return run_collide_and_limit(cfg, limiters, 0, f_st, f_out, dS_field, phi_field, sel, n_sel,
                                 stats);
}

int orc_run(const orc_config *cfg, double *f, long long nsteps, orc_stats *stats)
{
    int q = nq(cfg->lattice);
    long long n = (long long)cfg->nx * cfg->ny;
    double *g = (double *)malloc(sizeof(double) * (size_t)(q * n));
    double *cur = f, *nxt = g;
    int rc = 0;
    for (long long t = 0; t < nsteps; ++t) {
        rc |= orc_step(cfg, cur, nxt, NULL, NULL, NULL, NULL, stats);
        double *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    if (cur != f) memcpy(f, cur, sizeof(double) * (size_t)(q * n));
    free(g);
    return rc;
}

int orc_delta_s(const orc_config *cfg, const double *f_st, double *dS_field)
{
    int q = nq(cfg->lattice);
    int nx = cfg->nx, ny = cfg->ny;
    double fin[9], fs[9], fp[9], rho, ds, dsi;
    int rc = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (boundary_node(cfg, i, j)) {  /* not collided: no nonequilibrium entropy */
                dS_field[(long long)j * nx + i] = 0.0;
                continue;
            }
            pull(cfg, f_st, i, j, fin);
            rc |= site_collide(cfg, fin, fs, fp, &ds, &dsi, &rho);
            dS_field[(long long)j * nx + i] = ds;
        }
    (void)q;
    return rc;
}
