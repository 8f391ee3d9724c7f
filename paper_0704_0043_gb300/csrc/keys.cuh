// keys.cuh -- the FP64 Ehrenfests' key dS(f') of one D2Q9 site evaluated by a
// whole warp from FP32 / 16-bit storage (Sec. 3.2; dS in the quadratic form
// of Sec. 3.6).  The fused step kernel keys its candidates where it finds them.
#pragma once

#include "internal.h"
#include "lattice.cuh"

namespace lbm {

// What the FP64 key needs of a D2Q9 lattice (walls, channel or periodic):
// layout, boundary, a = 2 beta - 1, rho_ref W_k (rest, axis, diagonal) and the
// moving-lid terms of the links through the lid (directions 4, 7, 8).
struct KeyGeom {
    int nx, ny, pitch, boundary;
    int eq;  // 1: entropic f* and the exact dS of Eq. DelS (key_ent9)
    long long plane;
    double a;
    double rw0, rw1, rw5;
    double lid4, lid7, lid8;
    __device__ double rw(int k) const { return k == 0 ? rw0 : (k <= 4 ? rw1 : rw5); }
    __device__ double lid(int k) const { return k == 4 ? lid4 : (k == 7 ? lid7 : (k == 8 ? lid8 : 0.0)); }
};

// Population k arriving at site (x, y), in FP64 from FP32 / 16-bit storage
// `src` (layout of internal.h): (double) g + rho_ref W, the value the FP64
// path computes from the same stored state.
template <typename S>
__device__ double pull_one_f64(const KeyGeom &p, const S *src, int x, int y, int k)
{
    const bool wrapx = bc_wrap_x(p.boundary), wrapy = bc_wrap_y(p.boundary);
    int sx = x - Lat<9>::cx(k), sy = y - Lat<9>::cy(k);
    if (wrapx) sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
    if (wrapy) sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
    auto at = [&](int q, int yy, int xx) {
        return src[(long long)q * p.plane + (long long)yy * p.pitch + kLead + xx];
    };
    if (sx >= 0 && sx < p.nx && sy >= 0 && sy < p.ny) return Ar<double>::add((double)s2f(at(k, sy, sx)), p.rw(k));
    const int q = Lat<9>::opp(k);
    double v = Ar<double>::add((double)s2f(at(q, y, x)), p.rw(q));
    if (sy > p.ny - 1) v = Ar<double>::add(v, p.lid(k));
    return v;
}

// FP64 key with entropic f* (Eq. maxwellian) and the exact dS of Eq. DelS, from
// the same pulled FP64 populations: the evaluation of the FP64 path
// (site_collide with eq = 1), so the key is the value an LBM_FP64 context
// would compare with delta_e; +inf for a state with a negative population.
template <typename S>
__device__ __noinline__ double key_ent9(const KeyGeom p, const S *src, int site, double delta_e)
{
    const int x = site % p.nx, y = site / p.nx;
    double fin[9], fs[9], fp[9], ds, dsin, rho;
#pragma unroll
    for (int k = 0; k < 9; ++k) fin[k] = pull_one_f64<S>(p, src, x, y, k);
    const bool bad = site_collide<9, double>(fin, p.a, true, fs, fp, ds, dsin, rho, 1, false);
    return !bad && ds > delta_e ? ds : -1.0;
}

// FP64 key dS(f') of `site`, evaluated by the whole (converged) warp: lane k < 9
// pulls population k and evaluates f*_k and its dS term; the moments and the
// final sum run in k order exactly as the sequential FP64 evaluation runs them,
// so the key is the same bit for bit.  Returns the key, or -1 for a site at or
// below delta_e or one that cannot be limited (rho <= 0, some f*_k <= 0,
// nonfinite); every lane returns the same value.  Not inlined: the caller's
// hot loop keeps its registers, and the call is rare.
template <typename S>
__device__ __noinline__ double key_dS9_warp(const KeyGeom p, const S *src, int site, double delta_e)
{
    using A = Ar<double>;
    constexpr unsigned kAll = 0xffffffffu;
    if (p.eq == 1) return key_ent9<S>(p, src, site, delta_e);  // every lane, the same value
    const int lane = threadIdx.x & 31, k = lane < 9 ? lane : 0;
    const int x = site % p.nx, y = site / p.nx;
    const double mine = pull_one_f64<S>(p, src, x, y, k);
    double fin[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) fin[j] = __shfl_sync(kAll, mine, j);
    double rho, ux, uy;
    moments9<double>(fin, rho, ux, uy);
    // f*_k as in feq9<double>
    const double usq = A::add(A::mul(ux, ux), A::mul(uy, uy));
    const double tail = A::mul(A::mul(3.0, usq), 0.5);
    const double c = k == 0 ? 0.0
                   : k == 1 ? ux
                   : k == 2 ? uy
                   : k == 3 ? -ux
                   : k == 4 ? -uy
                   : k == 5 ? A::add(ux, uy)
                   : k == 6 ? A::sub(uy, ux)
                   : k == 7 ? -A::add(ux, uy)
                            : A::sub(ux, uy);
    double poly = A::add(A::add(1.0, A::mul(3.0, c)), A::mul(A::mul(9.0, A::mul(c, c)), 0.5));
    poly = A::sub(poly, tail);
    const double fs = A::mul(A::mul(rho, Lat<9>::w(k)), poly);
    // collision and the dS term as in the sequential evaluation
    const double fp = A::add(fs, A::mul(p.a, A::sub(fs, mine)));
    const double d = A::sub(fp, fs);
    const double term = A::div(A::mul(d, d), fs);
    const bool bad_k = lane < 9 && (!(fs > 0.0) || !isfinite(mine));
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) s = A::add(s, __shfl_sync(kAll, term, j));
    const bool bad = __any_sync(kAll, bad_k) || !(rho > 0.0) || !isfinite(rho) || !isfinite(ux) || !isfinite(uy);
    return !bad && isfinite(s) && s > delta_e ? s : -1.0;
}

// The same key evaluated by one thread alone (lane-parallel keying of many
// candidates: each lane keys its own site).  The operations and their order
// are those of key_dS9_warp, so both give the same bits.
template <typename S>
__device__ __noinline__ double key_dS9_lane(const KeyGeom p, const S *src, int site, double delta_e)
{
    using A = Ar<double>;
    if (p.eq == 1) return key_ent9<S>(p, src, site, delta_e);
    const int x = site % p.nx, y = site / p.nx;
    double fin[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) fin[k] = pull_one_f64<S>(p, src, x, y, k);
    double rho, ux, uy;
    moments9<double>(fin, rho, ux, uy);
    const double usq = A::add(A::mul(ux, ux), A::mul(uy, uy));
    const double tail = A::mul(A::mul(3.0, usq), 0.5);
    bool bad = !(rho > 0.0) || !isfinite(rho) || !isfinite(ux) || !isfinite(uy);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double c = k == 0 ? 0.0
                       : k == 1 ? ux
                       : k == 2 ? uy
                       : k == 3 ? -ux
                       : k == 4 ? -uy
                       : k == 5 ? A::add(ux, uy)
                       : k == 6 ? A::sub(uy, ux)
                       : k == 7 ? -A::add(ux, uy)
                                : A::sub(ux, uy);
        double poly = A::add(A::add(1.0, A::mul(3.0, c)), A::mul(A::mul(9.0, A::mul(c, c)), 0.5));
        poly = A::sub(poly, tail);
        const double fs = A::mul(A::mul(rho, Lat<9>::w(k)), poly);
        const double fp = A::add(fs, A::mul(p.a, A::sub(fs, fin[k])));
        const double d = A::sub(fp, fs);
        s = A::add(s, A::div(A::mul(d, d), fs));
        bad = bad || !(fs > 0.0) || !isfinite(fin[k]);
    }
    return !bad && isfinite(s) && s > delta_e ? s : -1.0;
}

}  // namespace lbm
