// step_tiled.cu -- one limited LBGK step with overlapping tiles, every lattice,
// boundary kind and precision, plus the small field kernels (init, moments,
// population transfer, dS field).
//
// A block computes free flight, collision and dS(f') (Eq. lbgkLB, Sec. 3.6) for
// a tile of sites and keeps the dS values in shared memory; the sites of the
// tile's interior then have their whole median stencil (Sec. 3.5) at hand and
// finish the step: positivity rule (Sec. 3.1), median homothety (Eq. entrHom),
// phi = min of the two, f_out = f* + phi (f' - f*) (Eq. LimGenF), Ehrenfests'
// candidates (Sec. 3.2) and the block's FP64 partial sums (Sec. 3.4).  Tiles
// overlap by one site on each side, so every site is finished by exactly one
// block and the halo ring is recomputed.  In FP64 every operation runs in the
// order of the formulas, unfused (see lattice.cuh).  FP32 storage holds the
// deviations g = f - rho_ref W and the FP32 arithmetic runs on them.
#include <type_traits>

#include "internal.h"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int kTX = 32, kTY = 8;  // D2Q9 tile of computed sites; (kTX-2) x (kTY-2) finished
constexpr int kT1 = 64;           // D1Q3 tile; kT1 - 2 finished (small tiles: a short tube spreads over
                                  // many SMs; GB300's FP64 pipe is narrow per SM)

__device__ __forceinline__ long long fidx(long long plane, int pitch, int k, int y, int x)
{
    return (long long)k * plane + (long long)y * pitch + kLead + x;
}

// Stored value as a compute value: FP64 storage is f itself; FP32 / BF16 /
// FP16 storage is the deviation g, read as g in FP32 or as the absolute
// f = (double) g + rw_k in FP64.
template <typename S, typename T>
__device__ __forceinline__ T load_as(const StepParams &p, S v, int k)
{
    if constexpr (std::is_same<S, double>::value)
        return T(v);
    else if constexpr (std::is_same<T, double>::value)
        return Ar<double>::add((double)s2f(v), p.rw[k]);
    else
        return s2f(v);
}

// Free flight in pull form at site (x, y) (Sec. 2): f_in_k(x) = f_k(x - v_k);
// a link leaving the lattice is reflected, f_in_k(x) = f_opp(k)(x) (halfway
// bounce-back, Sec. 4.4.1), plus the moving-wall term for links through the lid.
// Reads storage type S, returns compute type T (see load_as).
template <int Q, typename S, typename T>
__device__ __forceinline__ void pull(const StepParams &p, const S *__restrict__ f, int x, int y, T fin[Q])
{
    using A = Ar<T>;
    const bool wrapx = bc_wrap_x(p.boundary);
    const bool wrapy = (Q == 9) && bc_wrap_y(p.boundary);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        int sx = x - Lat<Q>::cx(k), sy = y - Lat<Q>::cy(k);
        if (wrapx) sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
        if (wrapy) sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
        if (sx >= 0 && sx < p.nx && sy >= 0 && sy < p.ny) {
            fin[k] = load_as<S, T>(p, f[fidx(p.plane, p.pitch, k, sy, sx)], k);
        } else {
            T v = load_as<S, T>(p, f[fidx(p.plane, p.pitch, Lat<Q>::opp(k), y, x)], Lat<Q>::opp(k));
            if (Q == 9 && sy > p.ny - 1) {
                if constexpr (std::is_same<T, double>::value)
                    v = A::add(v, p.lid[k]);
                else
                    v = A::add(A::add(v, p.lidf[k]), p.lidlo[k]);
            }
            fin[k] = v;
        }
    }
}

// Free flight and the wall rule at a boundary node (x, y) of a cavity whose
// outer ring of nodes lies on the walls (LBM_BC_NODE_WALLS, LBM_BC_DIFFUSIVE;
// Sec. 4.4): the populations whose source is on the lattice arrive; the others
// are supplied by the wall.  The lid is the top row without its corners and
// moves with (u_lid, 0); the other walls and the corners are at rest.
//   bounce-back (Sec. 4.4.1): f_k = f_opp(k) + 6 W_k rho_wall (v_k . u_wall);
//   diffusive (Sec. 4.4.2): f_k = gamma f*_k(1, u_wall), gamma = (sum of the
//     arrived f_opp(k)) / (sum of f*_k(1, u_wall)) over the returned
//     directions, evaluated in FP64 for every storage type; bounce-back in the
//     corners.
// A corner's two missing populations whose opposite is missing too point out
// of the lattice again; they keep their stored values.  `mass` receives the
// populations that stream back onto the lattice (FP64, k order).
template <typename S, typename T>
__device__ void wall_node(const StepParams &p, const S *__restrict__ f, int x, int y, T fin[9], double &mass)
{
    using A = Ar<T>;
    bool known[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int sx = x - Lat<9>::cx(k), sy = y - Lat<9>::cy(k);
        known[k] = sx >= 0 && sx < p.nx && sy >= 0 && sy < p.ny;
        fin[k] = known[k] ? load_as<S, T>(p, f[fidx(p.plane, p.pitch, k, sy, sx)], k) : T(0);
    }
    const bool corner = (x == 0 || x == p.nx - 1) && (y == 0 || y == p.ny - 1);
    const bool lid = y == p.ny - 1 && !corner;
    if (p.boundary == 4 && !corner) {
        const double uw = lid ? p.u_lid : 0.0;
        double fw[9];
        feq_any<9>(p.eq, 1.0, uw, 0.0, fw);  // density is a linear factor of f*: take 1
        double arrived = 0.0, returned = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (!known[k]) {
                const int o = Lat<9>::opp(k);
                arrived = Ar<double>::add(arrived, load_as<S, double>(p, f[fidx(p.plane, p.pitch, o, y - Lat<9>::cy(o), x - Lat<9>::cx(o))], o));
                returned = Ar<double>::add(returned, fw[k]);
            }
        const double gamma = Ar<double>::div(arrived, returned);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (!known[k]) {
                const double v = Ar<double>::mul(gamma, fw[k]);
                if constexpr (std::is_same<T, double>::value)
                    fin[k] = v;
                else
                    fin[k] = (T)Ar<double>::sub(v, p.rw[k]);  // the deviation, rounded once
            }
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (known[k]) continue;
            const int o = Lat<9>::opp(k);
            if (known[o]) {
                T v = fin[o];
                if (lid) {
                    if constexpr (std::is_same<T, double>::value)
                        v = A::add(v, p.lid[k]);
                    else
                        v = A::add(A::add(v, p.lidf[k]), p.lidlo[k]);
                }
                fin[k] = v;
            } else {
                fin[k] = load_as<S, T>(p, f[fidx(p.plane, p.pitch, k, y, x)], k);
            }
        }
    }
    double m = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int dx = x + Lat<9>::cx(k), dy = y + Lat<9>::cy(k);
        if (dx >= 0 && dx < p.nx && dy >= 0 && dy < p.ny) {
            if constexpr (std::is_same<T, double>::value)
                m = Ar<double>::add(m, fin[k]);
            else
                m += (double)fin[k] + p.rw[k];
        }
    }
    mass = m;
}

__device__ __forceinline__ bool is_wall_node(const StepParams &p, int x, int y)
{
    return bc_node_walls(p.boundary) && (x == 0 || x == p.nx - 1 || y == 0 || y == p.ny - 1);
}

// Median of the dS stencil of site (x, y), tile-local position (tx, ty) in a
// shared array with row stride `ld` (Sec. 3.5; wall rules of Sec. 4.4, read for
// walls half a link outside the lattice: a node next to one wall uses itself
// and its two neighbours along that wall, a corner node itself and its inward
// x and y neighbours, every other node the 3x3 block; the two end sites of a
// closed D1Q3 tube are not filtered).  Returns false for sites the filter skips.
template <int Q, typename T>
__device__ __forceinline__ bool stencil_median(const StepParams &p, const T *s, int ld, int tx, int ty,
                                               int x, int y, T &med)
{
#define S_(dx, dy) s[(ty + (dy)) * ld + tx + (dx)]
    if constexpr (Q == 3) {
        if (p.boundary == 0 && (x == 0 || x == p.nx - 1)) return false;
        med = med3(S_(-1, 0), S_(0, 0), S_(1, 0));
        return true;
    } else {
        if (bc_node_walls(p.boundary)) {
            // boundary nodes are not filtered; their neighbours use stencils
            // along the wall (Sec. 4.4)
            if (x == 0 || x == p.nx - 1 || y == 0 || y == p.ny - 1) return false;
            const bool nx1 = x == 1 || x == p.nx - 2, ny1 = y == 1 || y == p.ny - 2;
            if (nx1 && ny1) {
                med = med3(S_(0, 0), S_(x == 1 ? 1 : -1, 0), S_(0, y == 1 ? 1 : -1));
            } else if (ny1) {
                med = med3(S_(-1, 0), S_(0, 0), S_(1, 0));
            } else if (nx1) {
                med = med3(S_(0, -1), S_(0, 0), S_(0, 1));
            } else {
                med = med9(S_(-1, -1), S_(-1, 0), S_(-1, 1), S_(0, -1), S_(0, 0), S_(0, 1), S_(1, -1), S_(1, 0),
                           S_(1, 1));
            }
            return true;
        }
        const bool wallx = p.boundary == 0, wally = p.boundary != 1;
        const bool nearx = wallx && (x == 0 || x == p.nx - 1);
        const bool neary = wally && (y == 0 || y == p.ny - 1);
        if (nearx && neary) {
            const int dx = x == 0 ? 1 : -1, dy = y == 0 ? 1 : -1;
            med = med3(S_(0, 0), S_(dx, 0), S_(0, dy));
        } else if (neary) {
            med = med3(S_(-1, 0), S_(0, 0), S_(1, 0));
        } else if (nearx) {
            med = med3(S_(0, -1), S_(0, 0), S_(0, 1));
        } else {
            med = med9(S_(-1, -1), S_(-1, 0), S_(-1, 1), S_(0, -1), S_(0, 0), S_(0, 1), S_(1, -1), S_(1, 0),
                       S_(1, 1));
        }
        return true;
    }
#undef S_
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// BATCHED: block b runs instance map[b].x of `table` as its block map[b].y
// (tiles numbered row by row); otherwise the single instance (p0, src0, dst0).
template <int Q, typename S, bool BATCHED>
__global__ void __launch_bounds__(256) k_tiled(const StepParams p0, const S *__restrict__ src0, S *__restrict__ dst0,
                                               const TiledArgs *__restrict__ table, const int2 *__restrict__ map)
{
    using T = compute_t<S>;
    using A = Ar<T>;
    constexpr int BX = Q == 9 ? kTX : kT1;
    constexpr int BY = Q == 9 ? kTY : 1;
    __shared__ T sds[BY * BX];
    __shared__ double sred[8][P_NSTAT];
    __shared__ __align__(16) TiledArgs sA;
    int bx = (int)blockIdx.x, by = (int)blockIdx.y, gx = (int)gridDim.x;
    if constexpr (BATCHED) {
        const int2 m = map[blockIdx.x];
        const unsigned *from = reinterpret_cast<const unsigned *>(table + m.x);
        unsigned *to = reinterpret_cast<unsigned *>(&sA);
        for (int i = threadIdx.y * blockDim.x + threadIdx.x; i < (int)(sizeof(TiledArgs) / 4); i += BX * BY)
            to[i] = from[i];
        __syncthreads();
        gx = sA.gx;
        bx = m.y % gx;
        by = m.y / gx;
    }
    const StepParams &p = BATCHED ? sA.p : p0;
    const S *__restrict__ src = BATCHED ? (const S *)sA.src : src0;
    S *__restrict__ dst = BATCHED ? (S *)sA.dst : dst0;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = bx * (BX - 2) - 1 + tx;
    const int y = Q == 9 ? by * (BY - 2) - 1 + ty : 0;
    const bool wrapx = bc_wrap_x(p.boundary);
    const bool wrapy = (Q == 9) && bc_wrap_y(p.boundary);
    bool valid = wrapx ? (x >= -1 && x <= p.nx) : (x >= 0 && x < p.nx);
    if (Q == 9) valid = valid && (wrapy ? (y >= -1 && y <= p.ny) : (y >= 0 && y < p.ny));
    const int xs = wrapx ? (x < 0 ? x + p.nx : (x >= p.nx ? x - p.nx : x)) : x;
    const int ys = wrapy ? (y < 0 ? y + p.ny : (y >= p.ny ? y - p.ny : y)) : y;

    // FP64: fs = f*, fp = f'.  FP32: fs = g*, fp = g' (deviations), fa = absolute f*,
    // nq = corrected nonequilibrium part g - g* (lattice.cuh).
    T fin[Q], fs[Q], fp[Q], fa[Q];
    float nq[Q];
    T ds = T(0), dsin = T(0), rho = T(0);
    bool bad = false;
    // a boundary node of a cavity with nodes on the walls: free flight and the
    // wall rule only (no collision, no limiter, dS = 0)
    const bool wall = Q == 9 && valid && is_wall_node(p, xs, ys);
    double wmass = 0.0;
    if (wall) {
        if constexpr (Q == 9) {
            if (p.collide) {
                wall_node<S, T>(p, src, xs, ys, fin, wmass);
            } else {
#pragma unroll
                for (int k = 0; k < 9; ++k) fin[k] = load_as<S, T>(p, src[fidx(p.plane, p.pitch, k, ys, xs)], k);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const int dx = xs + Lat<9>::cx(k), dy = ys + Lat<9>::cy(k);
                    if (dx >= 0 && dx < p.nx && dy >= 0 && dy < p.ny) {
                        if constexpr (std::is_same<T, double>::value)
                            wmass = Ar<double>::add(wmass, fin[k]);
                        else
                            wmass += (double)fin[k] + p.rw[k];
                    }
                }
            }
        }
    } else if (valid) {
        if (p.collide) {
            pull<Q, S, T>(p, src, xs, ys, fin);
        } else {
#pragma unroll
            for (int k = 0; k < Q; ++k) fin[k] = load_as<S, T>(p, src[fidx(p.plane, p.pitch, k, ys, xs)], k);
        }
        if constexpr (std::is_same<T, double>::value) {
            // entropic f*: the halo ring only supplies dS(f') to the median stencils
            const bool owner = tx >= 1 && tx <= BX - 2 && (Q == 3 || (ty >= 1 && ty <= BY - 2));
            bad = site_collide<Q, T>(fin, T(p.a), p.collide != 0, fs, fp, ds, dsin, rho, p.eq, owner, p.coll, p.beta);
#pragma unroll
            for (int k = 0; k < Q; ++k) fa[k] = fs[k];
        } else {
            bad = site_collide_dev<Q>(fin, (float)p.a, (float)(1.0 + p.a), p.collide != 0, p.rho_ref, p.rwf, fs, nq,
                                      fp, fa, ds, dsin, rho, p.eq);
        }
        if (bad) ds = T(INFINITY);
    }
    sds[ty * BX + tx] = ds;
    // FP32 storage: the block's parameters in FP32, converted once (conversions
    // and compares of doubles run on this GPU's slow FP64 pipe; per thread they
    // bound the kernel).  Each equals the per-thread expression it replaces, so
    // the results do not change: kc[0] = delta_m, kc[1] = the Ehrenfests'
    // recording threshold, kc[2] = 2 beta - 1, kc[3] = alpha of the smooth
    // limiter, kc[4] = dS_t rounded down (for a float dS, dS > kc[4] exactly when
    // (double) dS > dS_t), kc[5] = smooth_k; ke: E > 0, k = 1/2, thresholds on
    __shared__ float kc[9];
    __shared__ int ke[3];
    if constexpr (!std::is_same<T, double>::value) {
        if (tx == 0 && ty == 0) {
            kc[0] = (float)p.delta_m;
            kc[1] = (float)(p.delta_e * (1.0 - 1.0 / 64.0));
            kc[2] = (float)p.a;
            const double E = (p.limiters & 24u) ? p.ens[0] : 0.0;
            // Eq. EntThresh's dS_t rounded down (for a float dS, dS > kc[6] exactly when (double) dS > dS_t)
            kc[6] = (p.limiters & 32u) ? __double2float_rd(p.ent->t) : 0.f;
            kc[7] = (p.limiters & 32u) ? (float)p.ent->t : 0.f;  // the homotheties' dS_t, nearest
            double t = p.threshold_c * E;
            if (t < p.threshold_delta) t = p.threshold_delta;
            kc[3] = (p.limiters & 24u) ? (float)p.ens[1] : 0.f;
            kc[4] = __double2float_rd(t);
            kc[8] = (float)t;
            kc[5] = (float)p.smooth_k;
            ke[0] = E > 0.0;
            ke[1] = p.smooth_k == 0.5;
            ke[2] = (p.limiters & 16u) != 0;
        }
    }
    __syncthreads();

    const bool own_site = valid && tx >= 1 && tx <= BX - 2 && (Q == 3 || (ty >= 1 && ty <= BY - 2)) && x >= 0 &&
                          x < p.nx && y >= 0 && y < p.ny;
    const bool own = own_site && !wall;
    if (own_site && wall) {
        // a boundary node stores what free flight and the wall rule gave it
#pragma unroll
        for (int k = 0; k < Q; ++k) dst[fidx(p.plane, p.pitch, k, y, x)] = f2s<S>(fin[k]);
        if (p.ds_out) p.ds_out[(long long)y * p.nx + x] = 0.0;
    }
    double acc[P_NSTAT];
#pragma unroll
    for (int i = 0; i < P_NSTAT; ++i) acc[i] = 0.0;
    // FP32 storage: the three dS sums as FP32 terms and the counts as flags (see below)
    float fsum_ds = 0.f, fsum_in = 0.f, fsum_lim = 0.f, fmass = 0.f;
    bool c_pos = false, c_med = false, c_bad = false;
    if (own) {
        T phi_pos = T(1), phi_med = T(1);
        if (!bad) {
            if (p.limiters & 1u) {
                if constexpr (std::is_same<T, double>::value) {
                    phi_pos = phi_positivity<Q, T>(fs, fp);
                } else {
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        const float fpa = p.rwf[k] + fp[k];  // absolute f'
                        if (fpa < 0.f) phi_pos = fminf(phi_pos, fa[k] / (fa[k] - fpa));
                    }
                }
            }
            // the homothety acts only where dS > delta_m (both acceptance
            // rules), so the median is formed only there
            T dm;
            if constexpr (std::is_same<T, double>::value)
                dm = p.delta_m;
            else
                dm = kc[0];
            if ((p.limiters & 4u) && ds > dm) {
                T med;
                if (stencil_median<Q, T>(p, sds, BX, tx, ty, x, y, med)) {
                    if constexpr (std::is_same<T, double>::value) {
                        // entropic f* with the solve of Sec. 3.7, else the homothety
                        phi_med = (p.phi_rule == 1 && p.eq == 1)
                                      ? phi_median_entropy<Q>(fp, fs, ds, med, dm, p.median_mode)
                                      : phi_median<T>(ds, med, dm, p.median_mode);
                    } else {
                        phi_med = phi_median<T>(ds, med, dm, p.median_mode);
                    }
                }
            }
        }
        T phi = phi_pos < phi_med ? phi_pos : phi_med;
        if (!bad && (p.limiters & kLimEnsemble)) {
            // ensemble-dependent limiters: ens = {E(dS), alpha = delta / E^k} of this pass
            T pe = T(1);
            if constexpr (std::is_same<T, double>::value) {
                const double E = p.ens[0];
                if ((p.limiters & 8u) && E > 0.0 && ds > 0.0) {
                    // Eq. smooth1 (Sec. 4.3.2); k = 1/2 by a square root
                    const double pk = p.smooth_k == 0.5 ? sqrt(ds) : pow(ds, p.smooth_k);
                    pe = 1.0 / (1.0 + p.ens[1] * pk);
                }
                if ((p.limiters & 32u) && ds > p.ent->t) {
                    // Eq. EntThresh's dS_t (Sec. 3.4), homothety or the solve of Sec. 3.7
                    const double t = p.ent->t;
                    const double pt = (p.phi_rule == 1 && p.eq == 1) ? phi_entropy<Q>(fp, fs, t) : sqrt(t / ds);
                    if (pt < pe) pe = pt;
                }
                if (p.limiters & 16u) {
                    // threshold filter: dS_t = max(c E, delta), homothety where dS > dS_t (Sec. 3.4)
                    double t = p.threshold_c * E;
                    if (t < p.threshold_delta) t = p.threshold_delta;
                    if (ds > t) {
                        const double pt = (p.phi_rule == 1 && p.eq == 1) ? phi_entropy<Q>(fp, fs, t) : sqrt(t / ds);
                        if (pt < pe) pe = pt;
                    }
                }
            } else {
                if ((p.limiters & 8u) && ke[0] && ds > 0.f) {
                    const float pk = ke[1] ? sqrtf(ds) : powf(ds, kc[5]);
                    pe = __fdiv_rn(1.0f, __fmaf_rn(kc[3], pk, 1.0f));  // explicit: the fused kernel's bits
                }
                // the threshold filters: decided exactly against dS_t rounded
                // down, the homothety sqrt(dS_t / dS) in FP32 (the fused kernel's
                // operations)
                if ((p.limiters & 32u) && ds > kc[6]) {
                    const float pt = __fsqrt_rn(__fdiv_rn(kc[7], ds));
                    if (pt < pe) pe = pt;
                }
                if (ke[2] && ds > kc[4]) {
                    const float pt = __fsqrt_rn(__fdiv_rn(kc[8], ds));
                    if (pt < pe) pe = pt;
                }
            }
            if (pe < phi) phi = pe;
        }
        if (phi < T(1)) {
            if constexpr (std::is_same<T, double>::value) {
                double fo[Q];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    fo[k] = A::add(fs[k], A::mul(phi, A::sub(fp[k], fs[k])));
                    dst[fidx(p.plane, p.pitch, k, y, x)] = f2s<S>(fo[k]);
                }
                if (p.eq == 1) {
                    // entropic f*: the entropy difference dS(f') - dS(f_out) at the same f*
                    const double dout = rel_entropy<Q>(fo, fs);
                    if (isfinite(ds) && isfinite(dout)) acc[P_DS_LIM] = A::sub(ds, dout);
                } else {
                    acc[P_DS_LIM] = A::mul(A::sub(1.0, A::mul(phi, phi)), ds);
                }
            } else {
                const float c = limit_weight(phi, kc[2], p.collide != 0);
#pragma unroll
                for (int k = 0; k < Q; ++k) dst[fidx(p.plane, p.pitch, k, y, x)] = f2s<S>(fmaf(-c, nq[k], fin[k]));
                if (p.eq == 1) {
                    // entropic f*: dS(f') - dS(f_out) at the same f*, f_out - f* = phi (f' - f*)
                    float dout[Q];
                    const float m = p.collide ? __fmul_rn(-(float)phi, kc[2]) : (float)phi;
#pragma unroll
                    for (int k = 0; k < Q; ++k) dout[k] = __fmul_rn(m, nq[k]);
                    const float so = rel_entropy_dev<Q>(dout, fa);
                    if (isfinite((float)ds) && isfinite(so)) fsum_lim = __fsub_rn((float)ds, so);
                } else {
                    fsum_lim = __fmul_rn(__fsub_rn(1.f, __fmul_rn((float)phi, (float)phi)), (float)ds);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < Q; ++k) dst[fidx(p.plane, p.pitch, k, y, x)] = f2s<S>(fp[k]);
        }
        acc[P_MASS] = (double)rho;
        if constexpr (!std::is_same<T, double>::value) fmass = __fsub_rn((float)rho, p.rho_ref);  // exact
        if (!bad) {
            if constexpr (std::is_same<T, double>::value) {
                if (p.eq == 1) {
                    // entropic f*: sums of entropy differences where both entropies are finite
                    if (isfinite(ds)) acc[P_SUM_DS] = ds;
                    if (isfinite(ds) && isfinite(dsin)) acc[P_SUM_IN] = Ar<double>::sub(dsin, ds);
                } else {
                    acc[P_SUM_DS] = ds;
                    acc[P_SUM_IN] = dsin;
                }
            } else {
                if (p.eq == 1) {
                    // entropic f*: sums of entropy differences where both entropies are finite
                    if (isfinite(ds)) fsum_ds = ds;
                    if (isfinite(ds) && isfinite(dsin)) fsum_in = __fsub_rn(dsin, ds);
                } else {
                    fsum_ds = ds;
                    fsum_in = dsin;
                }
            }
        } else {
            acc[P_NBAD] = 1.0;
            c_bad = true;
            atomicOr(p.status, kStatNonfinite);
        }
        acc[P_NPOS] = phi_pos < T(1) ? 1.0 : 0.0;
        acc[P_NMED] = phi_med < T(1) ? 1.0 : 0.0;
        c_pos = phi_pos < T(1);
        c_med = phi_med < T(1);
        if ((p.limiters & 2u) && !bad) {
            // Ehrenfests' candidates are decided on an FP64 dS(f').  FP32 storage:
            // sites near or above the threshold recompute their collision in FP64
            // from the same stored values.
            double key = 0.0;
            bool is = false;
            if constexpr (std::is_same<T, double>::value) {
                key = ds;
                is = ds > p.delta_e;
            } else {
                if (ds > kc[1]) {
                    double fin64[Q], fs64[Q], fp64[Q], d64, din64, r64;
                    if (p.collide) {
                        pull<Q, S, double>(p, src, x, y, fin64);
                    } else {
#pragma unroll
                        for (int k = 0; k < Q; ++k) fin64[k] = load_as<S, double>(p, src[fidx(p.plane, p.pitch, k, y, x)], k);
                    }
                    const bool b64 = site_collide<Q, double>(fin64, p.a, p.collide != 0, fs64, fp64, d64, din64, r64,
                                                             p.eq, false);
                    key = d64;
                    is = !b64 && d64 > p.delta_e;
                }
            }
            if (is) {
                const int slot = atomicAdd(p.cand_count, 1);
                if (slot < p.cand_cap) {
                    Cand c;
                    c.key = key;
                    c.site = y * p.nx + x;
                    c.phi = (double)phi;
                    c.ds32 = (float)key;
                    p.cand[slot] = c;
                } else {
                    atomicOr(p.status, kStatCandOverflow);
                }
            }
        }
        if (p.ds_out) p.ds_out[(long long)y * p.nx + x] = (double)ds;
    }
    // block partial sums, fixed order
    const int lin = ty * BX + tx, warp = lin >> 5, lane = lin & 31;
    if constexpr (std::is_same<T, double>::value) {
        if (own_site && wall) acc[P_MASS] = wmass;
#pragma unroll
        for (int i = 0; i < P_NSTAT; ++i) {
            const double v = warp_sum(acc[i]);
            if (lane == 0) sred[warp][i] = v;
        }
    } else {
        // FP32 storage: GB300's FP64 pipe is slow, and seven FP64 warp sums per
        // site bound this kernel.  The dS terms are FP32 values: a warp adds its
        // 32 in FP32 (~1e-6 relative).  The mass is rho_ref times the warp's
        // owned sites plus the FP32 sum of rho - rho_ref (each term exact, the
        // sum of 32 small terms within ~1e-6 of itself, i.e. ~1e-13 of the
        // mass); the counts come from ballots, exactly.  The block adds the
        // warp totals in FP64 in a fixed order.
        const int nown = __popc(__ballot_sync(0xffffffffu, own));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fmass = __fadd_rn(fmass, __shfl_down_sync(0xffffffffu, fmass, o));
            fsum_ds = __fadd_rn(fsum_ds, __shfl_down_sync(0xffffffffu, fsum_ds, o));
            fsum_in = __fadd_rn(fsum_in, __shfl_down_sync(0xffffffffu, fsum_in, o));
            fsum_lim = __fadd_rn(fsum_lim, __shfl_down_sync(0xffffffffu, fsum_lim, o));
        }
        const int npos = __popc(__ballot_sync(0xffffffffu, c_pos));
        const int nmed = __popc(__ballot_sync(0xffffffffu, c_med));
        const int nbad = __popc(__ballot_sync(0xffffffffu, c_bad));
        // boundary nodes carry their mass in FP64 (only warps that hold one add it)
        double wm = 0.0;
        if (__any_sync(0xffffffffu, own_site && wall)) wm = warp_sum(own_site && wall ? wmass : 0.0);
        if (lane == 0) {
            sred[warp][P_MASS] = (double)p.rho_ref * (double)nown + (double)fmass + wm;
            sred[warp][P_SUM_DS] = (double)fsum_ds;
            sred[warp][P_SUM_IN] = (double)fsum_in;
            sred[warp][P_DS_LIM] = (double)fsum_lim;
            sred[warp][P_NPOS] = (double)npos;
            sred[warp][P_NMED] = (double)nmed;
            sred[warp][P_NBAD] = (double)nbad;
        }
    }
    __syncthreads();
    const int bid = by * gx + bx;
    if (lin < P_NSTAT) {
        double v = 0.0;
        for (int w = 0; w < (BX * BY) / 32; ++w) v += sred[w][lin];
        p.partials[(long long)bid * P_NSTAT + lin] = v;
    }
    // The last block of each chunk of kChunkRows blocks to finish sums the
    // chunk's rows in row order (a ticket, no waiting): the tail then reads one
    // row per chunk, and the sums are the same whichever block comes last.
    __shared__ int s_last;
    const int nblk = BATCHED ? sA.blocks : (int)(gridDim.x * gridDim.y);
    const int chunk = bid / kChunkRows;
    const int rows = min(kChunkRows, nblk - chunk * kChunkRows);
    __threadfence();
    __syncthreads();
    if (lin == 0) s_last = atomicAdd(p.chunk_cnt + chunk, 1u) == (unsigned)(rows - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        const double *base = p.partials + (long long)chunk * kChunkRows * P_NSTAT;
        for (int stat = warp; stat < P_NSTAT; stat += (BX * BY) / 32) {
            double v = 0.0;
            for (int r = lane; r < rows; r += 32) v += __ldcg(base + (long long)r * P_NSTAT + stat);
            v = warp_sum(v);
            if (lane == 0) p.partials2[(long long)chunk * P_NSTAT + stat] = v;
        }
        if (lin == 0) p.chunk_cnt[chunk] = 0u;  // for the next launch
    }
}

// E(dS) of a pass (Sec. 3.3, Sec. 4.3.2): the ensemble-dependent limiters need
// the mean of dS(f') over the lattice before any site is limited.  Block b walks
// rows b, b + gridDim.x, ... (its threads along each row, so every warp reads
// consecutive columns of each plane) and sums dS(f') with the same evaluation
// as k_tiled (so the same values), over the sites that are not flagged and have
// a finite dS; k_ens_mean adds the block partials in block order.  With
// LBM_LIM_ENTTHRESH the values also go to the field the EntThresh solve reads.
template <int Q, typename S>
__global__ void __launch_bounds__(256) k_ens_partial(StepParams p, const S *__restrict__ src,
                                                     double *__restrict__ part)
{
    using T = compute_t<S>;
    __shared__ double sw[8][2];
    double sum = 0.0, cnt = 0.0;
    // FP32 storage: a thread's own terms in FP32 and an integer count (GB300's
    // FP64 pipe would otherwise bound this read-once pass)
    float fsum = 0.f;
    int icnt = 0;
    for (int y = blockIdx.x; y < p.ny; y += gridDim.x) {
        for (int x = threadIdx.x; x < p.nx; x += 256) {
            const long long s = (long long)y * p.nx + x;
            if (Q == 9 && is_wall_node(p, x, y)) {  // boundary nodes are not collided
                if (p.ent_field) ((T *)p.ent_field)[s] = T(0);
                continue;
            }
            T fin[Q], fs[Q], fp[Q], fa[Q];
            float nq[Q];
            T ds, dsin, rho;
            bool bad;
            if (p.collide) {
                pull<Q, S, T>(p, src, x, y, fin);
            } else {
#pragma unroll
                for (int k = 0; k < Q; ++k) fin[k] = load_as<S, T>(p, src[fidx(p.plane, p.pitch, k, y, x)], k);
            }
            if constexpr (std::is_same<T, double>::value) {
                bad = site_collide<Q, T>(fin, T(p.a), p.collide != 0, fs, fp, ds, dsin, rho, p.eq, false, p.coll,
                                         p.beta);
                if (!bad && isfinite(ds)) {
                    sum += ds;
                    cnt += 1.0;
                }
            } else {
                bad = site_collide_dev<Q>(fin, (float)p.a, (float)(1.0 + p.a), p.collide != 0, p.rho_ref, p.rwf, fs,
                                          nq, fp, fa, ds, dsin, rho, p.eq);
                if (!bad && isfinite(ds)) {
                    fsum = __fadd_rn(fsum, ds);
                    icnt += 1;
                }
            }
            // Eq. EntThresh works on the same values (0 where the site is left out)
            if (p.ent_field) ((T *)p.ent_field)[s] = (!bad && isfinite(ds) && ds > T(0)) ? ds : T(0);
        }
    }
    if constexpr (!std::is_same<T, double>::value) {
        sum = (double)fsum;
        cnt = (double)icnt;
    }
    sum = warp_sum(sum);
    cnt = warp_sum(cnt);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sw[warp][0] = sum;
        sw[warp][1] = cnt;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += sw[w][threadIdx.x];
        part[2 * blockIdx.x + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(256) k_ens_mean(const double *__restrict__ part, int nblk, double smooth_delta,
                                                  double smooth_k, double *__restrict__ out)
{
    __shared__ double sw[8][2];
    double sum = 0.0, cnt = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 256) {
        sum += part[2 * b];
        cnt += part[2 * b + 1];
    }
    sum = warp_sum(sum);
    cnt = warp_sum(cnt);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sw[warp][0] = sum;
        sw[warp][1] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, c = 0.0;
        for (int w = 0; w < 8; ++w) {
            s += sw[w][0];
            c += sw[w][1];
        }
        const double E = c > 0.0 ? s / c : 0.0;
        out[0] = E;
        out[1] = E > 0.0 ? smooth_delta / pow(E, smooth_k) : 0.0;  // alpha of Eq. smooth1
        out[2] = s;  // sum and count (Eq. EntThresh's right side)
        out[3] = c;
    }
}

template <int Q, typename S>
__global__ void k_delta_s(StepParams p, const S *__restrict__ f, double *__restrict__ out)
{
    const long long n = (long long)p.nx * p.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % p.nx), y = (int)(s / p.nx);
        if (Q == 9 && is_wall_node(p, x, y)) {  // boundary nodes are not collided
            out[s] = 0.0;
            continue;
        }
        double fin[Q], fs[Q], fp[Q], ds, dsin, rho;
        pull<Q, S, double>(p, f, x, y, fin);
        const bool bad = site_collide<Q, double>(fin, p.a, true, fs, fp, ds, dsin, rho, p.eq, true, p.coll, p.beta);
        out[s] = bad ? (double)INFINITY : ds;
    }
}

template <int Q, typename S>
__global__ void k_init(StepParams p, const double *__restrict__ rho, const double *__restrict__ ux,
                       const double *__restrict__ uy, S *__restrict__ f)
{
    const long long n = (long long)p.nx * p.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % p.nx), y = (int)(s / p.nx);
        double fs[Q];
        if (!feq_any<Q>(p.eq, rho[s], ux[s], uy ? uy[s] : 0.0, fs)) {
#pragma unroll
            for (int k = 0; k < Q; ++k) fs[k] = (double)NAN;  // no entropic f* for |u_j| >= 1
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            if constexpr (std::is_same<S, double>::value)
                f[fidx(p.plane, p.pitch, k, y, x)] = fs[k];
            else
                f[fidx(p.plane, p.pitch, k, y, x)] = f2s<S>((float)Ar<double>::sub(fs[k], p.rw[k]));
        }
    }
}

template <int Q, typename S>
__global__ void k_moments(StepParams p, const S *__restrict__ f, double *__restrict__ rho, double *__restrict__ ux,
                          double *__restrict__ uy)
{
    const long long n = (long long)p.nx * p.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % p.nx), y = (int)(s / p.nx);
        double g[Q], r, a, b;
#pragma unroll
        for (int k = 0; k < Q; ++k) g[k] = load_as<S, double>(p, f[fidx(p.plane, p.pitch, k, y, x)], k);
        moments<Q, double>(g, r, a, b);
        rho[s] = r;
        ux[s] = a;
        if (uy) uy[s] = b;
    }
}

template <typename S>
__global__ void k_get(int q, StepParams p, const S *__restrict__ f, double *__restrict__ out)
{
    const long long n = (long long)p.nx * p.ny, tot = n * q;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / n);
        const long long s = e % n;
        out[e] = load_as<S, double>(p, f[fidx(p.plane, p.pitch, k, (int)(s / p.nx), (int)(s % p.nx))], k);
    }
}

template <typename S>
__global__ void k_set(int q, StepParams p, const double *__restrict__ in, S *__restrict__ f)
{
    const long long n = (long long)p.nx * p.ny, tot = n * q;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / n);
        const long long s = e % n;
        S v;
        if constexpr (std::is_same<S, double>::value)
            v = in[e];
        else
            v = f2s<S>((float)Ar<double>::sub(in[e], p.rw[k]));
        f[fidx(p.plane, p.pitch, k, (int)(s / p.nx), (int)(s % p.nx))] = v;
    }
}

inline int grid_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
cudaError_t launch_tiled(int q, const StepParams &p, const T *src, T *dst, int *nblocks, cudaStream_t s)
{
    if (q == 9) {
        dim3 grid((p.nx + kTX - 3) / (kTX - 2), (p.ny + kTY - 3) / (kTY - 2));
        k_tiled<9, T, false><<<grid, dim3(kTX, kTY), 0, s>>>(p, src, dst, nullptr, nullptr);
        *nblocks = (int)(grid.x * grid.y);
    } else {
        dim3 grid((p.nx + kT1 - 3) / (kT1 - 2));
        k_tiled<3, T, false><<<grid, dim3(kT1), 0, s>>>(p, src, dst, nullptr, nullptr);
        *nblocks = (int)grid.x;
    }
    return cudaGetLastError();
}

int tiled_grid_x(int q, int nx) { return q == 9 ? (nx + kTX - 3) / (kTX - 2) : (nx + kT1 - 3) / (kT1 - 2); }

int tiled_blocks_for(int q, int nx, int ny)
{
    return q == 9 ? tiled_grid_x(9, nx) * ((ny + kTY - 3) / (kTY - 2)) : tiled_grid_x(3, nx);
}

cudaError_t launch_tiled_batched_f32(int q, const TiledArgs *table, const int2 *map, int blocks, cudaStream_t s)
{
    if (blocks <= 0) return cudaSuccess;
    const StepParams none{};
    if (q == 9)
        k_tiled<9, float, true><<<blocks, dim3(kTX, kTY), 0, s>>>(none, nullptr, nullptr, table, map);
    else
        k_tiled<3, float, true><<<blocks, dim3(kT1), 0, s>>>(none, nullptr, nullptr, table, map);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_delta_s(int q, const StepParams &p, const T *f, double *out, cudaStream_t s)
{
    const int g = grid_for((long long)p.nx * p.ny, 256);
    if (q == 9)
        k_delta_s<9, T><<<g, 256, 0, s>>>(p, f, out);
    else
        k_delta_s<3, T><<<g, 256, 0, s>>>(p, f, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ens_mean(int q, const StepParams &p, const T *src, double *ens, cudaStream_t s)
{
    if (q == 9)
        k_ens_partial<9, T><<<kEnsBlocks, 256, 0, s>>>(p, src, ens);
    else
        k_ens_partial<3, T><<<kEnsBlocks, 256, 0, s>>>(p, src, ens);
    k_ens_mean<<<1, 256, 0, s>>>(ens, kEnsBlocks, p.smooth_delta, p.smooth_k, ens + 2 * kEnsBlocks);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init(int q, const StepParams &p, const double *rho, const double *ux, const double *uy, T *f,
                        cudaStream_t s)
{
    const int g = grid_for((long long)p.nx * p.ny, 256);
    if (q == 9)
        k_init<9, T><<<g, 256, 0, s>>>(p, rho, ux, uy, f);
    else
        k_init<3, T><<<g, 256, 0, s>>>(p, rho, ux, nullptr, f);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments(int q, const StepParams &p, const T *f, double *rho, double *ux, double *uy,
                           cudaStream_t s)
{
    const int g = grid_for((long long)p.nx * p.ny, 256);
    if (q == 9)
        k_moments<9, T><<<g, 256, 0, s>>>(p, f, rho, ux, uy);
    else
        k_moments<3, T><<<g, 256, 0, s>>>(p, f, rho, ux, uy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_get(int q, const StepParams &p, const T *f, double *out, cudaStream_t s)
{
    k_get<T><<<grid_for((long long)p.nx * p.ny * q, 256), 256, 0, s>>>(q, p, f, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_set(int q, const StepParams &p, const double *in, T *f, cudaStream_t s)
{
    k_set<T><<<grid_for((long long)p.nx * p.ny * q, 256), 256, 0, s>>>(q, p, in, f);
    return cudaGetLastError();
}

#define LBM_INST(T)                                                                                           \
    template cudaError_t launch_tiled<T>(int, const StepParams &, const T *, T *, int *, cudaStream_t);     \
    template cudaError_t launch_delta_s<T>(int, const StepParams &, const T *, double *, cudaStream_t);     \
    template cudaError_t launch_ens_mean<T>(int, const StepParams &, const T *, double *, cudaStream_t);    \
    template cudaError_t launch_init<T>(int, const StepParams &, const double *, const double *,           \
                                        const double *, T *, cudaStream_t);                                  \
    template cudaError_t launch_moments<T>(int, const StepParams &, const T *, double *, double *, double *, \
                                           cudaStream_t);                                                    \
    template cudaError_t launch_get<T>(int, const StepParams &, const T *, double *, cudaStream_t);         \
    template cudaError_t launch_set<T>(int, const StepParams &, const double *, T *, cudaStream_t);
LBM_INST(float)
LBM_INST(double)
LBM_INST(__nv_bfloat16)
LBM_INST(__half)
#undef LBM_INST

}  // namespace lbm
