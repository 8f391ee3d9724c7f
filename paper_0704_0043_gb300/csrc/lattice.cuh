// lattice.cuh -- per-site arithmetic of the limited LBGK step (device side).
//
// Velocity sets (Sec. 4.1): D2Q9 numbered 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE,
// 6 NW, 7 SW, 8 SE with weights 4/9, 1/9, 1/36; D1Q3 numbered 0 rest, 1 left,
// 2 right (the paper's f1, f2, f3).
//
// Arithmetic policy Ar<T>:
//   Ar<double> rounds every operation on its own (__dadd_rn and friends are
//   never contracted into FMA), so FP64 code written in a fixed order
//   evaluates exactly that order: the FP64 path reproduces a plain
//   left-to-right double evaluation of the same formulas bit for bit.
//   Ar<float> uses the plain operators; the compiler may fuse them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

// Storage types: double (FP64 contexts: f itself), float, __nv_bfloat16 and
// __half (the deviations g = f - rho_ref W).  Arithmetic is FP64 for double
// storage and FP32 otherwise.
template <typename S>
using compute_t = typename std::conditional<std::is_same<S, double>::value, double, float>::type;

__device__ __forceinline__ float s2f(float v) { return v; }
__device__ __forceinline__ float s2f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float s2f(__half v) { return __half2float(v); }
__device__ __forceinline__ double s2f(double v) { return v; }

template <typename S> __device__ __forceinline__ S f2s(compute_t<S> v);
template <> __device__ __forceinline__ double f2s<double>(double v) { return v; }
template <> __device__ __forceinline__ float f2s<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 f2s<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half f2s<__half>(float v) { return __float2half_rn(v); }

template <typename T> struct Ar;

template <> struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
};

template <> struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
    static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
    static __device__ __forceinline__ float div(float a, float b) { return a / b; }
    static __device__ __forceinline__ float sqrt(float a) { return sqrtf(a); }
};

template <int Q> struct Lat;

template <> struct Lat<9> {
    static __host__ __device__ __forceinline__ constexpr int cx(int k)
    {
        return k == 1 || k == 5 || k == 8 ? 1 : (k == 3 || k == 6 || k == 7 ? -1 : 0);
    }
    static __host__ __device__ __forceinline__ constexpr int cy(int k)
    {
        return k == 2 || k == 5 || k == 6 ? 1 : (k == 4 || k == 7 || k == 8 ? -1 : 0);
    }
    static __host__ __device__ __forceinline__ constexpr int opp(int k)
    {
        return k == 0 ? 0 : (k <= 4 ? ((k + 1) % 4) + 1 : ((k - 3) % 4) + 5);
    }
    static __host__ __device__ __forceinline__ constexpr double w(int k)
    {
        return k == 0 ? 4.0 / 9.0 : (k <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

template <> struct Lat<3> {
    static __host__ __device__ __forceinline__ constexpr int cx(int k) { return k == 1 ? -1 : (k == 2 ? 1 : 0); }
    static __host__ __device__ __forceinline__ constexpr int cy(int) { return 0; }
    static __host__ __device__ __forceinline__ constexpr int opp(int k) { return k == 0 ? 0 : 3 - k; }
    static __host__ __device__ __forceinline__ constexpr double w(int k) { return k == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
};

// Eq. macro_dis: rho = sum_k f_k, rho u = sum_k v_k f_k, accumulated in k order
// (terms with v = 0 contribute exactly nothing and are skipped).
template <typename T>
__device__ __forceinline__ void moments9(const T f[9], T &rho, T &ux, T &uy)
{
    using A = Ar<T>;
    T r = f[0];
#pragma unroll
    for (int k = 1; k < 9; ++k) r = A::add(r, f[k]);
    T jx = A::sub(f[1], f[3]);
    jx = A::add(jx, f[5]);
    jx = A::sub(jx, f[6]);
    jx = A::sub(jx, f[7]);
    jx = A::add(jx, f[8]);
    T jy = A::sub(f[2], f[4]);
    jy = A::add(jy, f[5]);
    jy = A::add(jy, f[6]);
    jy = A::sub(jy, f[7]);
    jy = A::sub(jy, f[8]);
    rho = r;
    ux = A::div(jx, r);
    uy = A::div(jy, r);
}

template <typename T>
__device__ __forceinline__ void moments3(const T f[3], T &rho, T &ux, T &uy)
{
    using A = Ar<T>;
    T r = A::add(A::add(f[0], f[1]), f[2]);
    rho = r;
    ux = A::div(A::sub(f[2], f[1]), r);
    uy = T(0);
}

// Eq. polyeq2d: f*_k = rho W_k (1 + 3 v_k.u + 9 (v_k.u)^2 / 2 - 3 u^2 / 2).
// FP32: the rest population is taken as rho minus the other eight, which is
// the same value in exact arithmetic and keeps sum_k f*_k = rho up to unbiased
// rounding (the FP32 weights alone sum to 1 + 7.5e-9, a steady mass gain).
template <typename T>
__device__ __forceinline__ void feq9(T rho, T ux, T uy, T fs[9])
{
    using A = Ar<T>;
    const T usq = A::add(A::mul(ux, ux), A::mul(uy, uy));
    const T tail = A::mul(A::mul(T(3), usq), T(0.5));
    const T c[9] = {T(0), ux, uy, -ux, -uy, A::add(ux, uy), A::sub(uy, ux), -A::add(ux, uy),
                    A::sub(ux, uy)};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        // x / 2 and x * 0.5 round the same real number: identical results
        T poly = A::add(A::add(T(1), A::mul(T(3), c[k])), A::mul(A::mul(T(9), A::mul(c[k], c[k])), T(0.5)));
        poly = A::sub(poly, tail);
        fs[k] = A::mul(A::mul(rho, T(Lat<9>::w(k))), poly);
    }
    if constexpr (std::is_same<T, float>::value) {
        T rest = ((fs[1] + fs[2]) + (fs[3] + fs[4])) + ((fs[5] + fs[6]) + (fs[7] + fs[8]));
        fs[0] = rho - rest;
    }
}

// Eq. polyeq1d, term by term as printed.
template <typename T>
__device__ __forceinline__ void feq3(T rho, T u, T fs[3])
{
    using A = Ar<T>;
    const T uu = A::mul(u, u);
    fs[0] = A::mul(A::div(A::mul(T(2), rho), T(3)), A::sub(T(1), A::mul(A::mul(T(3), uu), T(0.5))));
    const T r6 = A::div(rho, T(6));
    fs[1] = A::mul(r6, A::add(A::sub(T(1), A::mul(T(3), u)), A::mul(T(3), uu)));
    fs[2] = A::mul(r6, A::add(A::add(T(1), A::mul(T(3), u)), A::mul(T(3), uu)));
    if constexpr (std::is_same<T, float>::value) fs[0] = rho - (fs[1] + fs[2]);  // see feq9
}

template <int Q, typename T>
__device__ __forceinline__ void moments(const T f[Q], T &rho, T &ux, T &uy)
{
    if constexpr (Q == 9)
        moments9<T>(f, rho, ux, uy);
    else
        moments3<T>(f, rho, ux, uy);
}

template <int Q, typename T>
__device__ __forceinline__ void feq(T rho, T ux, T uy, T fs[Q])
{
    if constexpr (Q == 9)
        feq9<T>(rho, ux, uy, fs);
    else
        feq3<T>(rho, ux, fs);
}

// Entropic quasiequilibria (FP64 only), in the oracle's operation order.
// Eq. maxwellian: f*_k = rho W_k prod_j A_j X_j^{v_kj} with
// A_j = 2 - sqrt(1 + 3 u_j^2), X_j = (2 u_j + sqrt(1 + 3 u_j^2)) / (1 - u_j);
// v_kj = -1 divides by X_j.  Exists for |u_x|, |u_y| < 1 (returns false otherwise).
__device__ __forceinline__ bool feq_ent9(double rho, double ux, double uy, double fs[9])
{
    using A = Ar<double>;
    if (!(fabs(ux) < 1.0) || !(fabs(uy) < 1.0)) return false;
    const double u[2] = {ux, uy};
    double Aj[2], Xj[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const double sq = A::sqrt(A::add(1.0, A::mul(3.0, A::mul(u[j], u[j]))));
        Aj[j] = A::sub(2.0, sq);
        Xj[j] = A::div(A::add(A::mul(2.0, u[j]), sq), A::sub(1.0, u[j]));
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int v[2] = {Lat<9>::cx(k), Lat<9>::cy(k)};
        double f = A::mul(rho, Lat<9>::w(k));
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double P = v[j] == 1 ? A::mul(Aj[j], Xj[j]) : (v[j] == -1 ? A::div(Aj[j], Xj[j]) : Aj[j]);
            f = A::mul(f, P);
        }
        fs[k] = f;
    }
    return true;
}

// Eq. entropiceq1d, with the printed f2* as the v = +1 population (index 2)
// and the printed f3* as the v = -1 one (index 1): the assignment under which
// sum_k v_k f*_k = rho u.
__device__ __forceinline__ bool feq_ent3(double rho, double u, double fs[3])
{
    using A = Ar<double>;
    if (!(fabs(u) < 1.0)) return false;
    const double sq = A::sqrt(A::add(1.0, A::mul(3.0, A::mul(u, u))));
    fs[0] = A::mul(A::div(A::mul(2.0, rho), 3.0), A::sub(2.0, sq));
    const double r6 = A::div(rho, 6.0);
    fs[1] = A::mul(-r6, A::sub(A::add(A::mul(3.0, u), 1.0), A::mul(2.0, sq)));
    fs[2] = A::mul(r6, A::add(A::sub(A::mul(3.0, u), 1.0), A::mul(2.0, sq)));
    return true;
}

// f* of either kind (eq = 1: entropic); false where the entropic f* does not exist.
template <int Q>
__device__ __forceinline__ bool feq_any(int eq, double rho, double ux, double uy, double fs[Q])
{
    if (eq == 1) {
        if constexpr (Q == 9)
            return feq_ent9(rho, ux, uy, fs);
        else
            return feq_ent3(rho, ux, fs);
    }
    feq<Q, double>(rho, ux, uy, fs);
    return true;
}

// f ln(f / f*) for f > 0, f* > 0 (FP64).  Where f is within 2^-5 of f*
// (almost every site of a flow) by the series of the inverse hyperbolic
// tangent, ln(f / f*) = 2 atanh z = 2 (z + z^3/3 + z^5/5 + ...) with
// z = (f - f*) / (f + f*): f - f* is exact there (Sterbenz), z carries two
// roundings, and with |z| < 0.016 the terms past z^9/9 are below 1e-19 of the
// sum, so the logarithm is within a few ulps of ln(f / f*) itself.  Elsewhere
// the CUDA logarithm of the rounded ratio.  The series costs one division and
// five multiply-adds instead of a division and a general logarithm.
__device__ __forceinline__ double f_ln_ratio(double f, double fs)
{
    const double d = f - fs;
    if (!(fabs(d) < 0.03125 * fs)) return Ar<double>::mul(f, log(Ar<double>::div(f, fs)));
    const double z = d / (f + fs);
    const double w = z * z;
    double p = fma(w, 1.0 / 9.0, 1.0 / 7.0);
    p = fma(p, w, 1.0 / 5.0);
    p = fma(p, w, 1.0 / 3.0);
    const double t = 2.0 * z;
    return f * fma(t * w, p, t);
}

// Eq. DelS: sum_k f_k ln(f_k / f*_k), k order, 0 ln 0 = 0; +inf for a state
// with a negative population (outside the domain of the entropy), NaN for a
// NaN population.
template <int Q>
__device__ __forceinline__ double rel_entropy(const double f[Q], const double fs[Q])
{
    using A = Ar<double>;
    bool neg = false, nan = false;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        neg |= f[k] < 0.0;
        nan |= !(f[k] >= 0.0) && !(f[k] < 0.0);
    }
    if (neg) return (double)INFINITY;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < Q; ++k)
        if (f[k] > 0.0) s = A::add(s, f_ln_ratio(f[k], fs[k]));
    return nan ? (double)NAN : s;
}

// ELBM's alpha (Eq. entropy_estimate, Sec. 4.2): the nontrivial root of
// S(f + alpha (f* - f)) = S(f), i.e. dS(f) - dS(f + alpha (f* - f)) = 0 with the
// exact dS of Eq. DelS, by bisection on [1, alpha_max] to a bracket of 1e-15,
// returning the end where the entropy does not decrease.  alpha_max is the
// positivity boundary of the line (the smallest f_k / (f_k - f*_k) over
// f*_k < f_k); where the entropy is still at least S(f) there, no root lies in
// the positive cone and alpha_max itself is returned (the positivity rule).
// f = f* gives 2, the LBGK step.  The operations are those of the oracle's
// bisection; the logarithms are the device's (f_ln_ratio), so the root agrees
// to the evaluation error of dS.
template <int Q>
__device__ double elbm_alpha(const double f[Q], const double fs[Q])
{
    using A = Ar<double>;
    bool same = true;
#pragma unroll
    for (int k = 0; k < Q; ++k) same = same && f[k] == fs[k];
    if (same) return 2.0;
    double amax = (double)INFINITY;
#pragma unroll
    for (int k = 0; k < Q; ++k)
        if (fs[k] < f[k]) {
            const double r = A::div(f[k], A::sub(f[k], fs[k]));
            if (r < amax) amax = r;
        }
    const double ds0 = rel_entropy<Q>(f, fs);
    double g[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        g[k] = A::add(f[k], A::mul(amax, A::sub(fs[k], f[k])));
        if (g[k] < 0.0) g[k] = 0.0;  // the boundary itself: the vanishing population is zero
    }
    if (A::sub(ds0, rel_entropy<Q>(g, fs)) >= 0.0) return amax;
    double lo = 1.0, hi = amax;
    for (int it = 0; it < 200 && A::sub(hi, lo) > 1e-15; ++it) {
        const double mid = A::mul(0.5, A::add(lo, hi));
#pragma unroll
        for (int k = 0; k < Q; ++k) g[k] = A::add(f[k], A::mul(mid, A::sub(fs[k], f[k])));
        if (A::sub(ds0, rel_entropy<Q>(g, fs)) >= 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Sec. 3.7: the phi in [0, 1] with dS(f* + phi (f' - f*)) = target (Eq. DelS), by
// bisection to a bracket of 1e-15, returning the lower end; dS along the
// segment grows from 0 at f*.
template <int Q>
__device__ double phi_entropy(const double fp[Q], const double fs[Q], double target)
{
    using A = Ar<double>;
    double g[Q];
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200 && A::sub(hi, lo) > 1e-15; ++it) {
        const double mid = A::mul(0.5, A::add(lo, hi));
#pragma unroll
        for (int k = 0; k < Q; ++k) g[k] = A::add(fs[k], A::mul(mid, A::sub(fp[k], fs[k])));
        if (rel_entropy<Q>(g, fs) <= target)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Median-filter factor with the solve of Sec. 3.7 (mode and tolerance as phi_median).
template <int Q>
__device__ double phi_median_entropy(const double fp[Q], const double fs[Q], double x, double med, double delta,
                                     int mode)
{
    if (mode == 1) return (x > delta && med < x) ? phi_entropy<Q>(fp, fs, med) : 1.0;
    const double t = med > delta ? med : delta;
    return x > t ? phi_entropy<Q>(fp, fs, t) : 1.0;
}

// Quadratic nonequilibrium entropy (Sec. 3.6): sum_k (g_k - f*_k)^2 / f*_k, k order.
template <int Q, typename T>
__device__ __forceinline__ T quad_entropy(const T g[Q], const T fs[Q])
{
    using A = Ar<T>;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const T d = A::sub(g[k], fs[k]);
        s = A::add(s, A::div(A::mul(d, d), fs[k]));
    }
    return s;
}

// Collision and entropy at one site from its arriving populations f_in:
// f*, f' = f* + a (f* - f_in) with a = 2 beta - 1 (Eq. collLBGK), dS(f'),
// dS(f_in) and rho.  With collide = false (limiter pass on a stored state)
// f' = f_in.  Returns true for a site that cannot be limited: rho <= 0, no f*
// or f*_k <= 0 for some k, or a nonfinite value.  eq = 1 (FP64 only):
// entropic f* and the exact relative entropy, which is +inf (not an error)
// for a state with a negative population; need_in = false skips dS(f_in).
template <int Q, typename T>
__device__ __forceinline__ bool site_collide(const T fin[Q], T a, bool collide, T fs[Q], T fp[Q],
                                             T &ds, T &ds_in, T &rho, int eq = 0, bool need_in = true,
                                             int coll = 0, double beta = 0.0)
{
    using A = Ar<T>;
    T ux, uy;
    moments<Q, T>(fin, rho, ux, uy);
    bool bad = !(rho > T(0)) || !isfinite(rho) || !isfinite(ux) || !isfinite(uy);
    if constexpr (std::is_same<T, double>::value) {
        if (eq == 1) {
            if (!feq_any<Q>(1, rho, ux, uy, fs)) {
                bad = true;
#pragma unroll
                for (int k = 0; k < Q; ++k) fs[k] = 0.0;
            }
#pragma unroll
            for (int k = 0; k < Q; ++k) fp[k] = collide ? A::add(fs[k], A::mul(a, A::sub(fs[k], fin[k]))) : fin[k];
#pragma unroll
            for (int k = 0; k < Q; ++k) bad |= !(fs[k] > 0.0) || !isfinite(fs[k]) || !isfinite(fin[k]);
            if (coll == 1 && collide && !bad) {
                // Eq. elbm: f' = (1 - beta) f + beta f~ = f + (beta alpha)(f* - f)
                const double ba = A::mul(beta, elbm_alpha<Q>(fin, fs));
#pragma unroll
                for (int k = 0; k < Q; ++k) fp[k] = A::add(fin[k], A::mul(ba, A::sub(fs[k], fin[k])));
            }
            ds = bad ? 0.0 : rel_entropy<Q>(fp, fs);
            // dS(f_in) feeds only the statistics: sites that only supply a
            // stencil value (need_in = false) skip it; with finite populations
            // and f* > 0 it is never NaN, so the flag does not depend on it
            ds_in = (bad || !collide || !need_in) ? 0.0 : rel_entropy<Q>(fin, fs);
            bad |= isnan(ds) || isnan(ds_in);
            return bad;
        }
    }
    feq<Q, T>(rho, ux, uy, fs);
#pragma unroll
    for (int k = 0; k < Q; ++k) fp[k] = collide ? A::add(fs[k], A::mul(a, A::sub(fs[k], fin[k]))) : fin[k];
#pragma unroll
    for (int k = 0; k < Q; ++k) bad |= !(fs[k] > T(0)) || !isfinite(fin[k]);
    ds = quad_entropy<Q, T>(fp, fs);
    ds_in = collide ? quad_entropy<Q, T>(fin, fs) : T(0);
    bad |= !isfinite(ds) || !isfinite(ds_in);
    return bad;
}

// FP64 dS(f') of the collision alone (the Ehrenfests' key): same operations as
// site_collide, without dS(f_in).  Returns false for a site that cannot be limited.
__device__ __forceinline__ bool key_dS9(const double fin[9], double a, double &ds)
{
    using A = Ar<double>;
    double rho, ux, uy, fs[9];
    moments9<double>(fin, rho, ux, uy);
    feq9<double>(rho, ux, uy, fs);
    bool bad = !(rho > 0.0) || !isfinite(rho) || !isfinite(ux) || !isfinite(uy);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        bad |= !(fs[k] > 0.0) || !isfinite(fin[k]);
        const double fp = A::add(fs[k], A::mul(a, A::sub(fs[k], fin[k])));
        const double d = A::sub(fp, fs[k]);
        s = A::add(s, A::div(A::mul(d, d), fs[k]));
    }
    ds = s;
    return !bad && isfinite(s);
}

// Positivity rule (Sec. 3.1): largest lambda <= 1 such that f* + lambda (f' - f*) >= 0.
template <int Q, typename T>
__device__ __forceinline__ T phi_positivity(const T fs[Q], const T fp[Q])
{
    using A = Ar<T>;
    T phi = T(1);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        if (fp[k] < T(0)) {
            const T r = A::div(fs[k], A::sub(fs[k], fp[k]));
            if (r < phi) phi = r;
        }
    }
    return phi;
}

// Median-filter homothety coefficient (Sec. 3.5, Eq. entrHom) for entropy x and
// stencil median med.  mode 0: dS_t = max(med, delta), phi = sqrt(dS_t/x) if
// x > dS_t.  mode 1: phi = sqrt(med/x) if x > delta and med < x.
template <typename T>
__device__ __forceinline__ T phi_median(T x, T med, T delta, int mode)
{
    using A = Ar<T>;
    if (mode == 1) {
        if (x > delta && med < x) return A::sqrt(A::div(med, x));
        return T(1);
    }
    const T t = med > delta ? med : delta;
    return x > t ? A::sqrt(A::div(t, x)) : T(1);
}

// Hardware reciprocal approximation (one special-function instruction,
// relative error below 2^-22): the FP32 entropy denominators.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------------------
// FP32 storage holds deviations g_k = f_k - rho_ref W_k from a uniform rest
// state (the D2Q9 and D1Q3 weights are symmetric under k -> opp(k), so
// bounce-back and the lid term act on g exactly as on f).  Moments, f* and
// the collision are evaluated on the deviations, which keeps three to four
// more significant bits than storing f itself:
//   rho = rho_ref + sum_k g_k,  rho u = sum_k v_k g_k,
//   g*_k = f*_k - rho_ref W_k = W_k (drho + rho e_k) + 3 W_k rho (v_k . u)
// with e_k = 9 (v_k.u)^2 / 2 - 3 u^2 / 2 (Eq. polyeq2d).  The rest deviation
// closes the mass: g*_0 = drho - sum_{k>0} g*_k.

// Explicitly rounded FP32 operations: the compiler fuses nothing, so every
// kernel that evaluates a site with these functions gets the same bits.  F1
// works on one site; F2 on the two sites a lane of the fused kernel carries,
// with the paired FP32 instructions of sm_100 and later (one instruction,
// two independent correctly rounded results).
struct F1 {
    using V = float;
    static __device__ __forceinline__ V add(V a, V b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ V sub(V a, V b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ V s(float x) { return x; }
    static __device__ __forceinline__ V rcp_rn(V a) { return __frcp_rn(a); }
    static __device__ __forceinline__ V rcp_fast(V a) { return rcp_approx(a); }
    static __device__ __forceinline__ V div(V a, V b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ V sqrt(V a) { return __fsqrt_rn(a); }
};

struct F2 {
    using V = float2;
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    // a - b as fma(b, -1, a): the product is exact, so one rounding, as __fsub_rn
    static __device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ V s(float x) { return make_float2(x, x); }
    static __device__ __forceinline__ V rcp_rn(V a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }
    static __device__ __forceinline__ V rcp_fast(V a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
    static __device__ __forceinline__ V div(V a, V b) { return make_float2(__fdiv_rn(a.x, b.x), __fdiv_rn(a.y, b.y)); }
    static __device__ __forceinline__ V sqrt(V a) { return make_float2(__fsqrt_rn(a.x), __fsqrt_rn(a.y)); }
};

template <class O>
__device__ __forceinline__ void moments9_x(const typename O::V g[9], float rho_ref, typename O::V &drho,
                                           typename O::V &rho, typename O::V &ux, typename O::V &uy)
{
    using V = typename O::V;
    drho = O::add(O::add(O::add(O::add(g[0], g[1]), O::add(g[2], g[3])), O::add(O::add(g[4], g[5]), O::add(g[6], g[7]))),
                  g[8]);
    rho = O::add(O::s(rho_ref), drho);
    const V jx = O::add(O::add(O::sub(g[1], g[3]), O::sub(g[5], g[6])), O::sub(g[8], g[7]));
    const V jy = O::sub(O::add(O::sub(g[2], g[4]), O::add(g[5], g[6])), O::add(g[7], g[8]));
    const V inv = O::rcp_rn(rho);
    ux = O::mul(jx, inv);
    uy = O::mul(jy, inv);
}

// The odd part 3 W_k rho (v_k.u) carries all the momentum; its FP32
// coefficients 3 W_1 = 1/3 and 3 W_5 = 1/12 are chosen so that 2 c1 + 4 c5 = 1
// holds exactly for the stored FP32 values (fl(1/3) and 11184810 * 2^-27).
// With the nearest-FP32 weights instead, sum_k v_k f*_k = rho u (1 + 7.5e-9),
// and since f' = f* + a (f* - f_in), every collision would multiply the
// momentum by 1 + 2 beta * 7.5e-9.
template <class O>
__device__ __forceinline__ void feq9_x(typename O::V drho, typename O::V rho, typename O::V ux, typename O::V uy,
                                       typename O::V gs[9])
{
    using V = typename O::V;
    const float w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
    const float c1 = 0x1.555556p-2f, c5 = 0x1.555554p-4f;
    const V m = O::mul(O::s(-1.5f), O::fma(ux, ux, O::mul(uy, uy)));
    const V b1 = O::mul(O::s(c1), rho), b5 = O::mul(O::s(c5), rho);
    const V cp = O::add(ux, uy), cm = O::sub(uy, ux);
    auto pair = [&](float w, V b, V c, V &plus, V &minus) {
        const V e = O::fma(O::mul(O::s(4.5f), c), c, m);
        const V A = O::mul(O::s(w), O::fma(rho, e, drho));
        const V B = O::mul(b, c);
        plus = O::add(A, B);
        minus = O::sub(A, B);
    };
    pair(w1, b1, ux, gs[1], gs[3]);
    pair(w1, b1, uy, gs[2], gs[4]);
    pair(w5, b5, cp, gs[5], gs[7]);
    pair(w5, b5, cm, gs[6], gs[8]);
    gs[0] = O::sub(drho, O::add(O::add(O::add(gs[1], gs[2]), O::add(gs[3], gs[4])),
                                O::add(O::add(gs[5], gs[6]), O::add(gs[7], gs[8]))));
}

// Nonequilibrium part n = g - g* with its mass and momentum sums taken out.
// In exact arithmetic they vanish; in FP32 they carry the rounding of the
// moment sums (up to half an ulp of rho u ~ 0.1, i.e. ~4e-9 per site and
// step).  The collision and the limiters move g along n only (see
// site_collide_dev), so with these sums removed they conserve mass and
// momentum to the rounding of the stored values: on a 1000-step cavity run the
// FP32 error then stays at the level of FP32 storage alone instead of
// several times above it.  The sums of n are small numbers and nearly exact.
template <class O>
__device__ __forceinline__ void neq9_x(const typename O::V g[9], const typename O::V gs[9], typename O::V n[9])
{
    using V = typename O::V;
#pragma unroll
    for (int k = 0; k < 9; ++k) n[k] = O::sub(g[k], gs[k]);
    const V rm = O::add(O::add(O::add(O::add(n[0], n[1]), O::add(n[2], n[3])), O::add(O::add(n[4], n[5]), O::add(n[6], n[7]))),
                        n[8]);
    const V hx = O::mul(O::s(0.5f), O::add(O::add(O::sub(n[1], n[3]), O::sub(n[5], n[6])), O::sub(n[8], n[7])));
    const V hy = O::mul(O::s(0.5f), O::sub(O::add(O::sub(n[2], n[4]), O::add(n[5], n[6])), O::add(n[7], n[8])));
    n[0] = O::sub(n[0], rm);
    n[1] = O::sub(n[1], hx);
    n[3] = O::add(n[3], hx);
    n[2] = O::sub(n[2], hy);
    n[4] = O::add(n[4], hy);
}

// ---------------------------------------------------------------------------
// Entropic quasiequilibria on FP32 deviations.  Eq. maxwellian is the product
// over the axes of A_j X_j^{v_j} with A_j = 2 - s_j, X_j = (2 u_j + s_j) / (1 - u_j),
// s_j = sqrt(1 + 3 u_j^2) (Eq. entropiceq1d is one such factor).  Written as
// 1 + d, each factor has a cancellation-free d (a = s - 1 = 3 u^2 / (1 + s)):
//   v = 0:  d0 = -a
//   v = +1: dp = (u (3 - 2a) - a^2) / (1 - u)
//   v = -1: dm = (u (a - 3) - 2a) / (1 + 2u + a)
// so f*_k = rho W_k (1 + e_k), e_k = dx + dy + dx dy, and the deviation is
// g*_k = W_k (drho + rho e_k); the rest deviation closes the mass as in the
// polynomial form.  Needs |u_x|, |u_y| < 1 (the caller flags the site otherwise).
template <class O>
__device__ __forceinline__ void ent_axis(typename O::V u, typename O::V &d0, typename O::V &dp, typename O::V &dm)
{
    using V = typename O::V;
    const V u2 = O::mul(u, u);
    const V s = O::sqrt(O::fma(O::s(3.f), u2, O::s(1.f)));
    const V a = O::div(O::mul(O::s(3.f), u2), O::add(O::s(1.f), s));
    d0 = O::mul(O::s(-1.f), a);
    dp = O::div(O::fma(u, O::fma(O::s(-2.f), a, O::s(3.f)), O::mul(O::s(-1.f), O::mul(a, a))), O::sub(O::s(1.f), u));
    dm = O::div(O::fma(u, O::sub(a, O::s(3.f)), O::mul(O::s(-2.f), a)),
                O::add(O::fma(O::s(2.f), u, O::s(1.f)), a));
}

template <class O>
__device__ __forceinline__ void feq_ent9_x(typename O::V drho, typename O::V rho, typename O::V ux, typename O::V uy,
                                           typename O::V gs[9])
{
    using V = typename O::V;
    V x0, xp, xm, y0, yp, ym;
    ent_axis<O>(ux, x0, xp, xm);
    ent_axis<O>(uy, y0, yp, ym);
    const float w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
    auto g = [&](float w, V dx, V dy) {
        const V e = O::fma(dx, dy, O::add(dx, dy));
        return O::mul(O::s(w), O::fma(rho, e, drho));
    };
    gs[1] = g(w1, xp, y0);
    gs[2] = g(w1, x0, yp);
    gs[3] = g(w1, xm, y0);
    gs[4] = g(w1, x0, ym);
    gs[5] = g(w5, xp, yp);
    gs[6] = g(w5, xm, yp);
    gs[7] = g(w5, xm, ym);
    gs[8] = g(w5, xp, ym);
    gs[0] = O::sub(drho, O::add(O::add(O::add(gs[1], gs[2]), O::add(gs[3], gs[4])),
                                O::add(O::add(gs[5], gs[6]), O::add(gs[7], gs[8]))));
}

// D1Q3 (Eq. entropiceq1d; index 1 is v = -1, index 2 is v = +1)
__device__ __forceinline__ void feq_ent3_dev(float drho, float rho, float u, float gs[3])
{
    float d0, dp, dm;
    ent_axis<F1>(u, d0, dp, dm);
    gs[1] = __fmul_rn(1.0f / 6.0f, __fmaf_rn(rho, dm, drho));
    gs[2] = __fmul_rn(1.0f / 6.0f, __fmaf_rn(rho, dp, drho));
    gs[0] = __fsub_rn(drho, __fadd_rn(gs[1], gs[2]));
}

// One term of Eq. DelS written without cancellation: with d = f - f* and
// f = f* + d >= 0, f ln(f / f*) - (f - f*) = f* h(f / f*), h(x) = x ln x - x + 1
// >= 0; the terms sum to dS because sum_k (f_k - f*_k) = 0 (shared mass).
// With z = d / (2 f* + d), h = 2 z^2 (1 + z/3 + z^2/3 + z^3/5 + z^4/5 + z^5/7 +
// z^6/7 + ...) / (1 - z) (the series of 2 atanh z multiplied out); for
// |z| < 0.1 the omitted terms are below 1e-8 of the sum.  Farther out the
// logarithm directly.  A negative f gives +inf (outside the entropy's domain);
// f = 0 gives f* (0 ln 0 = 0).
__device__ __forceinline__ float ent_term1(float d, float fs)
{
    const float f = __fadd_rn(fs, d);
    if (!(f >= 0.f)) return f < 0.f ? __int_as_float(0x7f800000) : f;  // +inf, or NaN through
    // the two quotients of the series by the hardware reciprocal (relative error
    // below 2^-22): they scale a term of dS, not a population
    const float z = __fmul_rn(d, rcp_approx(__fadd_rn(__fadd_rn(fs, fs), d)));
    if (fabsf(z) < 0.1f) {
        const float w = __fmul_rn(z, z);
        const float odd = __fmaf_rn(w, __fmaf_rn(w, 1.0f / 7.0f, 1.0f / 5.0f), 1.0f / 3.0f);
        const float even = __fmaf_rn(w, __fmaf_rn(w, __fmaf_rn(w, 1.0f / 7.0f, 1.0f / 5.0f), 1.0f / 3.0f), 1.0f);
        const float P = __fmaf_rn(z, odd, even);
        return __fmul_rn(fs, __fmul_rn(__fmul_rn(__fmul_rn(2.f, w), P), rcp_approx(__fsub_rn(1.f, z))));
    }
    if (f == 0.f) return fs;
    return __fsub_rn(__fmul_rn(f, logf(__fdiv_rn(f, fs))), d);
}

// Eq. DelS of a D2Q9 / D1Q3 state f* + d (absolute f* in fsa), k order; +inf if
// some population is negative.
template <int Q>
__device__ __forceinline__ float rel_entropy_dev(const float d[Q], const float fsa[Q])
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < Q; ++k) s = __fadd_rn(s, ent_term1(d[k], fsa[k]));
    return s;
}

// ent_term1 for the two sites a lane of the fused kernel carries: the series
// branch with paired instructions when both sites take it (the common case),
// else site by site; the same operations per component, so the same bits.
__device__ __forceinline__ float2 ent_term2(float2 d, float2 fs)
{
    using O = F2;
    const float2 f = O::add(fs, d);
    const float2 den = O::add(O::add(fs, fs), d);
    const float2 z = O::mul(d, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
    if (f.x >= 0.f && f.y >= 0.f && fabsf(z.x) < 0.1f && fabsf(z.y) < 0.1f) {
        const float2 w = O::mul(z, z);
        const float2 odd = O::fma(w, O::fma(w, O::s(1.0f / 7.0f), O::s(1.0f / 5.0f)), O::s(1.0f / 3.0f));
        const float2 even =
            O::fma(w, O::fma(w, O::fma(w, O::s(1.0f / 7.0f), O::s(1.0f / 5.0f)), O::s(1.0f / 3.0f)), O::s(1.0f));
        const float2 P = O::fma(z, odd, even);
        const float2 om = O::sub(O::s(1.f), z);
        return O::mul(fs, O::mul(O::mul(O::mul(O::s(2.f), w), P), make_float2(rcp_approx(om.x), rcp_approx(om.y))));
    }
    return make_float2(ent_term1(d.x, fs.x), ent_term1(d.y, fs.y));
}

// The paired form of rel_entropy_dev<9> for the fused kernel.
__device__ __forceinline__ float2 rel_entropy9_x(const float2 d[9], const float2 fsa[9])
{
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 9; ++k) s = F2::add(s, ent_term2(d[k], fsa[k]));
    return s;
}

__device__ __forceinline__ void moments9_dev(const float g[9], float rho_ref, float &drho, float &rho, float &ux,
                                             float &uy)
{
    moments9_x<F1>(g, rho_ref, drho, rho, ux, uy);
}

__device__ __forceinline__ void feq9_dev(float drho, float rho, float ux, float uy, float gs[9])
{
    feq9_x<F1>(drho, rho, ux, uy, gs);
}

// D1Q3 (Eq. polyeq1d): g*_{1,2} = (drho + 3 rho u^2)/6 -/+ rho u / 2.  Every
// operation explicitly rounded, so each kernel that evaluates a D1Q3 site gets
// the same bits.
__device__ __forceinline__ void moments3_dev(const float g[3], float rho_ref, float &drho, float &rho, float &ux,
                                             float &uy)
{
    drho = __fadd_rn(__fadd_rn(g[0], g[1]), g[2]);
    rho = __fadd_rn(rho_ref, drho);
    ux = __fmul_rn(__fsub_rn(g[2], g[1]), __frcp_rn(rho));
    uy = 0.0f;
}

__device__ __forceinline__ void feq3_dev(float drho, float rho, float u, float gs[3])
{
    const float A = __fmul_rn(1.0f / 6.0f, __fmaf_rn(__fmul_rn(__fmul_rn(3.0f, rho), u), u, drho));
    const float B = __fmul_rn(__fmul_rn(0.5f, rho), u);
    gs[1] = __fsub_rn(A, B);
    gs[2] = __fadd_rn(A, B);
    gs[0] = __fsub_rn(drho, __fadd_rn(gs[1], gs[2]));
}

template <int Q>
__device__ __forceinline__ void moments_dev(const float g[Q], float rho_ref, float &drho, float &rho, float &ux,
                                            float &uy)
{
    if constexpr (Q == 9)
        moments9_dev(g, rho_ref, drho, rho, ux, uy);
    else
        moments3_dev(g, rho_ref, drho, rho, ux, uy);
}

template <int Q>
__device__ __forceinline__ void feq_dev(float drho, float rho, float ux, float uy, float gs[Q])
{
    if constexpr (Q == 9)
        feq9_dev(drho, rho, ux, uy, gs);
    else
        feq3_dev(drho, rho, ux, gs);
}

__device__ __forceinline__ void neq9(const float g[9], const float gs[9], float n[9]) { neq9_x<F1>(g, gs, n); }

__device__ __forceinline__ void neq3(const float g[3], const float gs[3], float n[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = __fsub_rn(g[k], gs[k]);
    const float rm = __fadd_rn(__fadd_rn(n[0], n[1]), n[2]);
    const float hx = __fmul_rn(0.5f, __fsub_rn(n[2], n[1]));
    n[0] = __fsub_rn(n[0], rm);
    n[2] = __fsub_rn(n[2], hx);
    n[1] = __fadd_rn(n[1], hx);
}

template <int Q>
__device__ __forceinline__ void neq_dev(const float g[Q], const float gs[Q], float n[Q])
{
    if constexpr (Q == 9)
        neq9(g, gs, n);
    else
        neq3(g, gs, n);
}

// Weight of n in the limited update.  With f* + phi (f' - f*) (Eq. LimGenF)
// and f' = f* + (2 beta - 1)(f* - f) the result is g - c n with
// c = 1 + phi (2 beta - 1) after a collision, c = 1 - phi for a limiter pass
// on stored populations (f' = f); c = 1 (phi = 0) is the Ehrenfests' step.
__device__ __forceinline__ float limit_weight(float phi, float a, bool collide)
{
    return collide ? fmaf(phi, a, 1.f) : 1.f - phi;
}

// FP32 counterpart of site_collide on deviations: g* and the corrected
// nonequilibrium part n, g' = g - 2 beta n (collision, b2 = 2 beta) or g'
// = g, the absolute f* (rw_k + g*_k, for the entropy denominators and the
// positivity rule), dS(f') = (2 beta - 1)^2 dS(f_in) (quadratic form of
// Sec. 3.6 with the denominators by the hardware reciprocal), dS(f_in), rho.
template <int Q>
__device__ __forceinline__ bool site_collide_dev(const float g[Q], float a, float b2, bool collide, float rho_ref,
                                                 const float rw[Q], float gs[Q], float n[Q], float gp[Q],
                                                 float fsa[Q], float &ds, float &ds_in, float &rho, int eq = 0)
{
    float drho, ux, uy;
    moments_dev<Q>(g, rho_ref, drho, rho, ux, uy);
    if (eq == 1) {
        // entropic f* (Eq. maxwellian / Eq. entropiceq1d) and the exact dS of
        // Eq. DelS: dS(f') from f' - f* = -(2 beta - 1) n, dS(f_in) from n;
        // +inf (not a flag) for a state with a negative population
        const bool nofs = !(fabsf(ux) < 1.f) || !(fabsf(uy) < 1.f);
        if (nofs) {
#pragma unroll
            for (int k = 0; k < Q; ++k) gs[k] = 0.f;
        } else if constexpr (Q == 9) {
            feq_ent9_x<F1>(drho, rho, ux, uy, gs);
        } else {
            feq_ent3_dev(drho, rho, ux, gs);
        }
        neq_dev<Q>(g, gs, n);
        float fmin = 3.4e38f, dp[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            fsa[k] = __fadd_rn(rw[k], gs[k]);
            gp[k] = collide ? __fmaf_rn(-b2, n[k], g[k]) : g[k];
            dp[k] = collide ? __fmul_rn(-a, n[k]) : n[k];
            fmin = fminf(fmin, fsa[k]);
        }
        const bool bad = nofs || !(rho > 0.f) || !(fmin > 0.f);
        ds = bad ? 0.f : rel_entropy_dev<Q>(dp, fsa);
        ds_in = (bad || !collide) ? 0.f : rel_entropy_dev<Q>(n, fsa);
        return bad || isnan(ds) || isnan(ds_in);
    }
    feq_dev<Q>(drho, rho, ux, uy, gs);
    neq_dev<Q>(g, gs, n);
    float din = 0.f, fmin = 3.4e38f;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        fsa[k] = __fadd_rn(rw[k], gs[k]);
        din = __fmaf_rn(__fmul_rn(n[k], n[k]), rcp_approx(fsa[k]), din);
        gp[k] = collide ? __fmaf_rn(-b2, n[k], g[k]) : g[k];
        fmin = fminf(fmin, fsa[k]);
    }
    ds_in = collide ? din : 0.f;
    ds = collide ? __fmul_rn(__fmul_rn(a, a), din) : din;
    return !(rho > 0.f) || !(fmin > 0.f) || !isfinite(ds);
}

// min / max selecting one of the two operands (one instruction each; the
// values compared here are never NaN)
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }


template <typename T> __device__ __forceinline__ T med3(T a, T b, T c)
{
    return tmax(tmin(a, b), tmin(tmax(a, b), c));
}

// Median of nine values given as three columns (a, b, c): with each column
// sorted, the median is med3(largest column minimum, median of the column
// medians, smallest column maximum).
template <typename T>
__device__ __forceinline__ T med9(T a0, T a1, T a2, T b0, T b1, T b2, T c0, T c1, T c2)
{
    auto sort3 = [](T &x, T &y, T &z) {
        T lo = tmin(x, y), hi = tmax(x, y);
        T lo2 = tmin(lo, z), t = tmax(lo, z);
        x = lo2;
        y = tmin(hi, t);
        z = tmax(hi, t);
    };
    sort3(a0, a1, a2);
    sort3(b0, b1, b2);
    sort3(c0, c1, c2);
    const T lo = tmax(tmax(a0, b0), c0);
    const T mid = med3(a1, b1, c1);
    const T hi = tmin(tmin(a2, b2), c2);
    return med3(lo, mid, hi);
}

// Adds the FP32 value v exactly to acc, a 128-bit two's-complement fixed-point
// number in units of 2^-64 (bits of v below 2^-64 are dropped, truncating
// toward zero).  A nonfinite v, or |v| >= 2^63, sets `bad` instead.
__device__ __forceinline__ void fx_add(unsigned __int128 &acc, float v, bool &bad)
{
    const unsigned u = __float_as_uint(v);
    const int e = (int)((u >> 23) & 0xffu);  // biased exponent: v = +-m 2^(e - 150)
    if (e == 0xff) {
        bad = true;
        return;
    }
    if (e == 0) return;  // zero or subnormal (below 2^-126)
    const unsigned long long m = (u & 0x7fffffu) | 0x800000u;
    const int sh = e - 150 + 64;  // v = +-m 2^sh units
    if (sh >= 104) {
        bad = true;
        return;
    }
    unsigned __int128 x = 0;
    if (sh >= 0)
        x = (unsigned __int128)m << sh;
    else if (sh > -24)
        x = (unsigned __int128)(m >> -sh);
    acc += (u >> 31) ? (unsigned __int128)0 - x : x;
}

// Value of a 128-bit two's-complement fixed-point number in units of 2^-64:
// the high and low 64-bit magnitudes are converted separately, so the result
// is the same on every run.
__device__ __forceinline__ double fx_value(unsigned __int128 x)
{
    const bool neg = (unsigned long long)(x >> 127) != 0;
    const unsigned __int128 m = neg ? (unsigned __int128)0 - x : x;
    const double d = (double)(unsigned long long)(m >> 64) * 18446744073709551616.0 + (double)(unsigned long long)m;
    return (neg ? -d : d) * 5.42101086242752217003726400434970855712890625e-20;  // 2^-64
}

}  // namespace lbm
