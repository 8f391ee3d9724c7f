// step_tube.cu -- one limited LBGK step of a D1Q3 lattice (the shock tube of
// Sec. 4.3) as a single streaming pass.
//
// The step is that of the tiled kernel for Q = 3 (free flight, Eq. lbgkLB or
// Eq. elbm, dS of Sec. 3.6 / Eq. DelS, the positivity rule of Sec. 3.1, the
// three-point median filter of Sec. 3.5, Ehrenfests' candidates of Sec. 3.2,
// the sums of Sec. 3.4), evaluated per site with the same device functions,
// so the stored populations are the same bit for bit.  What differs is the
// decomposition, made for a one-dimensional lattice:
//   * a warp owns a contiguous chunk of sites and finishes all of them (no
//     overlapping tiles, no shared memory, no block barrier in the step); each
//     lane loads V consecutive sites of every plane as one 16-byte vector
//     (FP32: 4 sites, FP64: 2), or one site with V = 1;
//   * the streamed neighbours come from the adjacent lanes by shuffles; only
//     the two chunk-edge values are loaded on their own;
//   * the median needs dS of the neighbour sites: inside the chunk they are in
//     registers or on the adjacent lane, and dS of a site just outside the
//     chunk is evaluated on demand, only for an edge site whose median is
//     formed (dS above delta_M; rare);
//   * FP64 storage is bound by this GPU's FP64 units, which take a warp's FP64
//     instruction in 64 cycles whatever the number of active lanes: a short
//     tube runs one site per lane (V = 1) and one warp per block, so its warps
//     land on separate SM sub-partitions and the step lasts one site's chain;
//   * FP32 storage with four sites a lane evaluates them as two pairs with the
//     paired FP32 instructions and finishes a pair at once when no limiter
//     acts on it; any other site is finished by an out-of-line function, so
//     the walk's registers hold only what the common case needs.
// Ensemble-dependent limiters and 16-bit storage stay on the tiled kernel.
#include <type_traits>

#include "internal.h"
#include "lattice.cuh"

namespace lbm {
namespace {

__device__ __forceinline__ long long tidx(const StepParams &p, int k, int x) { return (long long)k * p.plane + kLead + x; }

// Stored value as a compute value (as in the tiled kernel): FP64 storage is f,
// FP32 storage the deviation g, read as g in FP32 or as (double) g + rw_k.
template <typename S, typename T>
__device__ __forceinline__ T tload(const StepParams &p, S v, int k)
{
    if constexpr (std::is_same<S, double>::value)
        return T(v);
    else if constexpr (std::is_same<T, double>::value)
        return Ar<double>::add((double)v, p.rw[k]);
    else
        return v;
}

// Free flight of one site (pull, Sec. 2): index 1 moves left (v = -1) and
// arrives from x + 1, index 2 from x - 1; closed ends reflect (halfway
// bounce-back: f_in_k = f_opp(k) of the site itself), periodic ends wrap.
template <typename S, typename T>
__device__ void tube_pull(const StepParams &p, const S *__restrict__ f, int x, T fin[3])
{
    const bool wrap = bc_wrap_x(p.boundary);
    int r = x + 1, l = x - 1;
    if (r >= p.nx) r = wrap ? 0 : -1;
    if (l < 0) l = wrap ? p.nx - 1 : -1;
    fin[0] = tload<S, T>(p, f[tidx(p, 0, x)], 0);
    fin[1] = r >= 0 ? tload<S, T>(p, f[tidx(p, 1, r)], 1) : tload<S, T>(p, f[tidx(p, 2, x)], 2);
    fin[2] = l >= 0 ? tload<S, T>(p, f[tidx(p, 2, l)], 2) : tload<S, T>(p, f[tidx(p, 1, x)], 1);
}

template <typename S, typename T>
__device__ __forceinline__ void tube_read(const StepParams &p, const S *__restrict__ f, int x, T fin[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) fin[k] = tload<S, T>(p, f[tidx(p, k, x)], k);
}

// Per-thread constants of FP32 storage (the FP64 parameters converted once).
struct TubeK {
    float a, b2, dm, thr_e;
};

// Collision and dS of one site (site_collide / site_collide_dev, as the tiled
// kernel calls them).  dS = +inf for a site that cannot be limited.
template <typename T>
__device__ __forceinline__ bool tube_eval(const StepParams &p, const TubeK &kk, const T fin[3], T fs[3], T fp[3],
                                          T fa[3], float nq[3], T &ds, T &dsin, T &rho, bool need_in)
{
    bool bad;
    if constexpr (std::is_same<T, double>::value) {
        bad = site_collide<3, double>(fin, p.a, p.collide != 0, fs, fp, ds, dsin, rho, p.eq, need_in, p.coll, p.beta);
#pragma unroll
        for (int k = 0; k < 3; ++k) fa[k] = fs[k];
        (void)nq;
    } else {
        bad = site_collide_dev<3>(fin, kk.a, kk.b2, p.collide != 0, p.rho_ref, p.rwf, fs, nq, fp, fa, ds, dsin, rho,
                                  p.eq);
    }
    if (bad) ds = T(INFINITY);
    return bad;
}

// dS(f') of site x alone (a median neighbour outside the warp's chunk).
template <typename S>
__device__ compute_t<S> tube_ds(const StepParams &p, const TubeK &kk, const S *__restrict__ src, int x)
{
    using T = compute_t<S>;
    T fin[3], fs[3], fp[3], fa[3], ds, dsin, rho;
    float nq[3];
    if (p.collide)
        tube_pull<S, T>(p, src, x, fin);
    else
        tube_read<S, T>(p, src, x, fin);
    tube_eval<T>(p, kk, fin, fs, fp, fa, nq, ds, dsin, rho, false);
    return ds;
}

// The polynomial FP32 collision of two sites at once: site_collide_dev (eq = 0,
// after a collision) in paired FP32 instructions (F2), the same explicitly
// rounded operations in the same order, so each site gets the same bits.
// Returns f' - rho_ref W (gp), dS(f'), dS(f_in), rho, and whether each site
// cannot be limited (rho <= 0, some f*_k <= 0, dS not finite).
__device__ __forceinline__ void tube_pair_eval(const TubeK &kk, float rho_ref, const float *rwf, const float2 g[3],
                                               float2 gp[3], float2 &ds, float2 &din, float2 &rho, bool &bad_x,
                                               bool &bad_y)
{
    using O = F2;
    const float2 drho = O::add(O::add(g[0], g[1]), g[2]);
    rho = O::add(O::s(rho_ref), drho);
    const float2 u = O::mul(O::sub(g[2], g[1]), O::rcp_rn(rho));
    const float2 A = O::mul(O::s(1.0f / 6.0f), O::fma(O::mul(O::mul(O::s(3.0f), rho), u), u, drho));
    const float2 B = O::mul(O::mul(O::s(0.5f), rho), u);
    float2 gs[3], n[3];
    gs[1] = O::sub(A, B);
    gs[2] = O::add(A, B);
    gs[0] = O::sub(drho, O::add(gs[1], gs[2]));
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = O::sub(g[k], gs[k]);
    const float2 rm = O::add(O::add(n[0], n[1]), n[2]);
    const float2 hx = O::mul(O::s(0.5f), O::sub(n[2], n[1]));
    n[0] = O::sub(n[0], rm);
    n[2] = O::sub(n[2], hx);
    n[1] = O::add(n[1], hx);
    float2 d = O::s(0.f);
    float mx = 3.4e38f, my = 3.4e38f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float2 fsa = O::add(O::s(rwf[k]), gs[k]);
        d = O::fma(O::mul(n[k], n[k]), O::rcp_fast(fsa), d);
        gp[k] = O::fma(O::s(-kk.b2), n[k], g[k]);
        mx = fminf(mx, fsa.x);
        my = fminf(my, fsa.y);
    }
    din = d;
    ds = O::mul(O::s(__fmul_rn(kk.a, kk.a)), d);
    bad_x = !(rho.x > 0.f) || !(mx > 0.f) || !isfinite(ds.x);
    bad_y = !(rho.y > 0.f) || !(my > 0.f) || !isfinite(ds.y);
}

// The sums and counts of one site finished by tube_site32.
struct SiteSums {
    float mass, ds, din, lim;
    int bad, pos, med;
};

// One FP32 site that the paired fast path did not finish (a limiter acts on
// its pair, its lane holds an end of the tube, or the pass is not a
// polynomial collision), from its pull f_in: the evaluation, the positivity
// rule, the three-point median (the neighbours' dS dsl / dsr, or evaluated
// here for the sites xlo / xro outside the warp's chunk, -1 when given), the
// limited or free update, its sums, the Ehrenfests' candidate and the dS
// field.  The operations are those of the tiled kernel's FP32 path.  Not
// inlined: the site's state stays out of the walk's registers.
template <typename S>
__device__ __noinline__ SiteSums tube_site32(const StepParams &p, TubeK kk, const S *__restrict__ src,
                                             S *__restrict__ dst, int x, float f0, float f1, float f2, float dsl,
                                             float dsr, int xlo, int xro, int2 *klist, int *kcount)
{
    SiteSums r{0.f, 0.f, 0.f, 0.f, 0, 0, 0};
    const float fin[3] = {f0, f1, f2};
    float fs[3], fp[3], fa[3], nq[3], ds, dsin, rho;
    const bool bad = tube_eval<float>(p, kk, fin, fs, fp, fa, nq, ds, dsin, rho, true);
    const int nx = p.nx;
    float phi_pos = 1.f, phi_med = 1.f;
    if (!bad) {
        if (p.limiters & 1u) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float fpa = p.rwf[k] + fp[k];  // absolute f'
                if (fpa < 0.f) phi_pos = fminf(phi_pos, fa[k] / (fa[k] - fpa));
            }
        }
        // three-point median (the two end sites of a closed tube are not
        // filtered; a periodic tube's end sites wrap around to each other)
        const bool end = p.boundary == 0 && (x == 0 || x == nx - 1);
        if ((p.limiters & 4u) && ds > kk.dm && !end) {
            const float left = xlo >= 0 ? tube_ds<S>(p, kk, src, xlo) : dsl;
            const float right = xro >= 0 ? tube_ds<S>(p, kk, src, xro) : dsr;
            phi_med = phi_median<float>(ds, med3(left, ds, right), kk.dm, p.median_mode);
        }
    }
    const float phi = phi_pos < phi_med ? phi_pos : phi_med;
    if (phi < 1.f) {
        const float cw = limit_weight(phi, kk.a, p.collide != 0);
#pragma unroll
        for (int k = 0; k < 3; ++k) dst[tidx(p, k, x)] = fmaf(-cw, nq[k], fin[k]);
        if (p.eq == 1) {
            float dout[3];
            const float m = p.collide ? __fmul_rn(-phi, kk.a) : phi;
#pragma unroll
            for (int k = 0; k < 3; ++k) dout[k] = __fmul_rn(m, nq[k]);
            const float so = rel_entropy_dev<3>(dout, fa);
            if (isfinite(ds) && isfinite(so)) r.lim = __fsub_rn(ds, so);
        } else {
            r.lim = __fmul_rn(__fsub_rn(1.f, __fmul_rn(phi, phi)), ds);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) dst[tidx(p, k, x)] = f2s<S>(fp[k]);
    }
    r.mass = __fsub_rn(rho, p.rho_ref);  // exact
    if (!bad) {
        if (p.eq == 1) {
            if (isfinite(ds)) r.ds = ds;
            if (isfinite(ds) && isfinite(dsin)) r.din = __fsub_rn(dsin, ds);
        } else {
            r.ds = ds;
            r.din = dsin;
        }
    } else {
        r.bad = 1;
        atomicOr(p.status, kStatNonfinite);
    }
    r.pos = phi_pos < 1.f;
    r.med = phi_med < 1.f;
    // Ehrenfests' candidate: near or above the threshold, keyed in FP64 after the chunk
    if ((p.limiters & 2u) && !bad && ds > kk.thr_e) klist[atomicAdd(kcount, 1)] = make_int2(x, __float_as_int(phi));
    if (p.ds_out) p.ds_out[x] = (double)ds;
    return r;
}

// Asynchronous copy of N = 4, 8 or 16 bytes global -> shared (cp.async; the
// 16-byte form bypasses L1), and the per-thread group bookkeeping.
template <int N>
__device__ __forceinline__ void tcopy(void *dst_smem, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    if constexpr (N == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(N) : "memory");
}
__device__ __forceinline__ void tcommit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void twait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// V sites per lane, blockDim.x / 32 warps per block.  The grid is at most one
// wave of resident blocks; warp w of the grid takes chunks w, w + W, w + 2W ...
// (W warps in the grid) of 32 V sites each.  Chunks stream through a per-warp
// ring of kTubeRing shared-memory slots filled by asynchronous copies (each
// lane copies its V sites of every plane, lane 0 and lane 31 also the values
// streaming in from the neighbour chunks), kTubeRing - 1 chunks ahead of the
// arithmetic.  `chunked`: the grid has more blocks than one chunk of the
// tail's reduction, so the last block of each kChunkRows blocks sums their
// rows; otherwise the tail reads the block rows.
constexpr int kTubeRing = 3;
constexpr int kTubeWarps = 8;  // the most warps a block has
constexpr int kTubeGroup = 8;  // chunks of a batched work item
// The statistics a warp gathers: FP64 storage sums FP64 terms per lane; FP32
// storage sums a chunk's FP32 terms per lane, adds the lanes in FP32 (a fixed
// butterfly that leaves the four totals in lanes 0, 8, 16, 24) and the chunk
// totals exactly, as 128-bit fixed point (integer instructions: FP64 adds per
// chunk kept this GPU's FP64 units a third busy).
struct TubeAcc {
    double t_mass, t_ds, t_in, t_lim;
    int c_pos, c_med, c_bad, c_own;
    unsigned __int128 fx;  // FP32 storage: lane 0 mass, lane 8 dS, lane 16 dS_in, lane 24 dS_lim
    bool fx_bad;
};

// FP32 storage: the four totals of acc (after the walk), in every lane.
__device__ __forceinline__ void tube_totals(const TubeAcc &acc, double &mass, double &ds, double &din, double &lim)
{
    const double v = acc.fx_bad ? __longlong_as_double(0x7ff8000000000000LL) : fx_value(acc.fx);
    mass = __shfl_sync(0xffffffffu, v, 0);
    ds = __shfl_sync(0xffffffffu, v, 8);
    din = __shfl_sync(0xffffffffu, v, 16);
    lim = __shfl_sync(0xffffffffu, v, 24);
}

// a ring slot: the three planes of a chunk of 32 V sites, then f_2 left of it
// and f_1 right of it
template <typename S, int V>
struct alignas(16) TubeSlot {
    S f[3][32 * V];
    S e[2];
};

// One warp's walk over chunks c0, c0 + stride, ... (< c_end) of lattice p:
// a1-a9 at every site, the Ehrenfests' candidates, the sums into acc.  `my`:
// the warp's ring; klist / kcount: the warp's candidate list (FP32 storage).
// Every lane of the warp takes part.
template <typename S, int V, bool FAST = true>
__device__ __forceinline__ void tube_walk(const StepParams &p, const S *__restrict__ src, S *__restrict__ dst,
                                          int c0, int stride, int c_end, TubeSlot<S, V> *my, int2 *klist,
                                          int *kcount, TubeAcc &acc)
{
    using T = compute_t<S>;
    using A = Ar<T>;
    using Slot = TubeSlot<S, V>;
    constexpr bool F64 = std::is_same<T, double>::value;
    constexpr int CW = 32 * V;  // sites of a chunk
    const int lane = threadIdx.x & 31;
    const int nx = p.nx;
    TubeK kk{};
    if constexpr (!F64) {
        kk.a = (float)p.a;
        kk.b2 = (float)(1.0 + p.a);
        kk.dm = (float)p.delta_m;
        kk.thr_e = (float)(p.delta_e * (1.0 - 1.0 / 64.0));
    }
    T dm;
    if constexpr (F64)
        dm = p.delta_m;
    else
        dm = kk.dm;

    // copies of chunk c into slot `sl` (nothing past the last chunk; the group
    // is committed either way).  The chunk's window lies inside the padded row
    // (kTail zero elements follow the lattice), so whole vectors may be copied
    // past its end.
    auto issue = [&](int c, int sl) {
        if (c < c_end) {
            const int x0 = c * CW, xl = x0 + lane * V;
            if (xl < nx) {
#pragma unroll
                for (int k = 0; k < 3; ++k) tcopy<(int)sizeof(S) * V>(&my[sl].f[k][lane * V], src + tidx(p, k, xl));
            }
            if (lane == 0 && x0 > 0) tcopy<(int)sizeof(S)>(&my[sl].e[0], src + tidx(p, 2, x0 - 1));
            if (lane == 31 && xl + V < nx) tcopy<(int)sizeof(S)>(&my[sl].e[1], src + tidx(p, 1, xl + V));
        }
        tcommit();
    };


    // an Ehrenfests' candidate into the context's list
    auto record = [&](int x, double key, double phi) {
        const int slot = atomicAdd(p.cand_count, 1);
        if (slot < p.cand_cap) {
            Cand cd;
            cd.key = key;
            cd.site = x;
            cd.phi = phi;
            cd.ds32 = (float)key;
            p.cand[slot] = cd;
        } else {
            atomicOr(p.status, kStatCandOverflow);
        }
    };
#pragma unroll
    for (int i = 0; i < kTubeRing - 1; ++i) issue(c0 + i * stride, i);
    int get = 0;
    for (int c = c0; c < c_end; c += stride) {
        __syncwarp();                                                   // every lane is done with the slot refilled now
        issue(c + (kTubeRing - 1) * stride, get == 0 ? kTubeRing - 1 : get - 1);
        twait<kTubeRing - 1>();                                         // this lane's copies of chunk c have landed
        __syncwarp();                                                   // and so have the other lanes'
        const Slot &sl = my[get];
        get = get + 1 == kTubeRing ? 0 : get + 1;
        const int x0 = c * CW, xl = x0 + lane * V;
        S v0[V], v1[V], v2[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            v0[j] = sl.f[0][lane * V + j];
            v1[j] = sl.f[1][lane * V + j];
            v2[j] = sl.f[2][lane * V + j];
        }
        // f_1 of the site right of the lane's last site, f_2 left of its first
        // (the next lane's first and the previous lane's last, or the slot's edges)
        const S r1 = lane == 31 ? sl.e[1] : sl.f[1][lane * V + V];
        const S l2 = lane == 0 ? sl.e[0] : sl.f[2][lane * V - 1];

        // the lane's pull of its site j (free flight with the tube's ends, or
        // the stored values of a limiter pass)
        auto build_fin = [&](int j, T f3[3]) {
            const int x = xl + j;
            if (p.collide) {
                f3[0] = tload<S, T>(p, v0[j], 0);
                f3[1] = tload<S, T>(p, j + 1 < V ? v1[j + 1] : r1, 1);
                f3[2] = tload<S, T>(p, j > 0 ? v2[j - 1] : l2, 2);
                if (x == nx - 1)  // right end: reflect or wrap
                    f3[1] = bc_wrap_x(p.boundary) ? tload<S, T>(p, src[tidx(p, 1, 0)], 1) : tload<S, T>(p, v2[j], 2);
                if (x == 0)  // left end
                    f3[2] = bc_wrap_x(p.boundary) ? tload<S, T>(p, src[tidx(p, 2, nx - 1)], 2) : tload<S, T>(p, v1[j], 1);
            } else {
                f3[0] = tload<S, T>(p, v0[j], 0);
                f3[1] = tload<S, T>(p, v1[j], 1);
                f3[2] = tload<S, T>(p, v2[j], 2);
            }
        };
        T ds[V];
        T s_mass = T(0), s_ds = T(0), s_in = T(0), s_lim = T(0);
        if constexpr (!F64 && FAST) {
            // FP32: a lane inside the tube in a colliding polynomial pass (four sites
            // a lane) evaluates its sites as two pairs (0, 1), (2, 3) with paired
            // instructions, and a pair on which no limiter acts (no bad site, no
            // negative f', no dS above the median filter's delta) is finished here.
            // Every other site keeps only its dS until the neighbours' dS are known
            // and is then finished one at a time by tube_site32.
            bool fastp[2] = {false, false}, paired = false;
            if constexpr (V == 4) {
                paired = p.collide && p.eq == 0 && xl >= 1 && xl + V <= nx - 1;
                if (paired) {
                    // the finished pairs' sums, added pairwise (paired instructions)
                    float2 m2 = F2::s(0.f), d2s = F2::s(0.f), i2s = F2::s(0.f), dmax = F2::s(0.f);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 g[3] = {make_float2(v0[2 * h], v0[2 * h + 1]),
                                             make_float2(v1[2 * h + 1], h == 0 ? v1[2] : r1),
                                             make_float2(h == 0 ? l2 : v2[1], v2[2 * h])};
                        float2 gp[3], d2, i2, r2;
                        bool bx, by;
                        tube_pair_eval(kk, p.rho_ref, p.rwf, g, gp, d2, i2, r2, bx, by);
                        bool act = bx || by;
                        if (p.limiters & 1u) {
#pragma unroll
                            for (int k = 0; k < 3; ++k)
                                act = act || (p.rwf[k] + gp[k].x < 0.f) || (p.rwf[k] + gp[k].y < 0.f);
                        }
                        if (p.limiters & 4u) act = act || d2.x > dm || d2.y > dm;
                        // a site that cannot be limited has dS = +inf (as tube_eval gives it)
                        ds[2 * h] = bx ? T(INFINITY) : d2.x;
                        ds[2 * h + 1] = by ? T(INFINITY) : d2.y;
                        if (act) continue;
                        // f' stored as one 8-byte vector a plane (xl + 2h is even)
                        fastp[h] = true;
                        const int x = xl + 2 * h;
#pragma unroll
                        for (int k = 0; k < 3; ++k) *reinterpret_cast<float2 *>(dst + tidx(p, k, x)) = gp[k];
                        m2 = F2::add(m2, F2::sub(r2, F2::s(p.rho_ref)));  // each term exact
                        d2s = F2::add(d2s, d2);
                        i2s = F2::add(i2s, i2);
                        dmax = make_float2(fmaxf(dmax.x, d2.x), fmaxf(dmax.y, d2.y));
                    }
                    if (fastp[0] || fastp[1]) {
                        s_mass = __fadd_rn(m2.x, m2.y);
                        s_ds = __fadd_rn(d2s.x, d2s.y);
                        s_in = __fadd_rn(i2s.x, i2s.y);
                        acc.c_own += 2 * ((int)fastp[0] + (int)fastp[1]);
                        // Ehrenfests' candidates among the finished sites (rare: one
                        // test a lane), and the dS field when it is asked for
                        if ((p.limiters & 2u) && fmaxf(dmax.x, dmax.y) > kk.thr_e) {
#pragma unroll
                            for (int j = 0; j < V; ++j)
                                if (fastp[j >> 1] && ds[j] > kk.thr_e)
                                    klist[atomicAdd(kcount, 1)] = make_int2(xl + j, __float_as_int(1.f));
                        }
                        if (p.ds_out) {
#pragma unroll
                            for (int j = 0; j < V; ++j)
                                if (fastp[j >> 1]) p.ds_out[xl + j] = (double)ds[j];
                        }
                    }
                }
            }
            if (!paired) {
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    ds[j] = T(0);
                    if (xl + j >= nx) continue;
                    float f3[3], fs3[3], fp3[3], fa3[3], nq3[3], din, r;
                    build_fin(j, f3);
                    tube_eval<float>(p, kk, f3, fs3, fp3, fa3, nq3, ds[j], din, r, false);
                }
            }
            // the median's neighbours: dS of the adjacent lanes' edge sites
            const T dl_lane = __shfl_up_sync(0xffffffffu, ds[V - 1], 1);
            const T dr_lane = __shfl_down_sync(0xffffffffu, ds[0], 1);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int x = xl + j;
                if (fastp[j >> 1] || x >= nx) continue;
                float f3[3];
                build_fin(j, f3);
                // the neighbours' dS, or the site to evaluate (outside the chunk)
                int xlo = -1, xro = -1;
                float dl = 0.f, dr = 0.f;
                if (x == 0)
                    xlo = nx - 1;
                else if (j > 0)
                    dl = ds[j - 1];
                else if (lane > 0)
                    dl = dl_lane;
                else
                    xlo = x - 1;
                if (x == nx - 1)
                    xro = 0;
                else if (j + 1 < V)
                    dr = ds[j + 1];
                else if (lane < 31)
                    dr = dr_lane;
                else
                    xro = x + 1;
                const SiteSums r =
                    tube_site32<S>(p, kk, src, dst, x, f3[0], f3[1], f3[2], dl, dr, xlo, xro, klist, kcount);
                s_lim = __fadd_rn(s_lim, r.lim);
                s_mass = __fadd_rn(s_mass, r.mass);
                s_ds = __fadd_rn(s_ds, r.ds);
                s_in = __fadd_rn(s_in, r.din);
                acc.c_own += 1;
                acc.c_bad += r.bad;
                acc.c_pos += r.pos;
                acc.c_med += r.med;
            }
        } else {
            T fin[V][3], fs[V][3], fp[V][3], fa[V][3], dsin[V], rho[V];
            float nq[V][3];
            bool bad[V];
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int x = xl + j;
                ds[j] = T(0);
                dsin[j] = T(0);
                rho[j] = T(0);
                bad[j] = false;
                if (x >= nx) continue;
                if (p.collide) {
                    fin[j][0] = tload<S, T>(p, v0[j], 0);
                    fin[j][1] = tload<S, T>(p, j + 1 < V ? v1[j + 1] : r1, 1);
                    fin[j][2] = tload<S, T>(p, j > 0 ? v2[j - 1] : l2, 2);
                    if (x == nx - 1)  // right end: reflect or wrap
                        fin[j][1] = bc_wrap_x(p.boundary) ? tload<S, T>(p, src[tidx(p, 1, 0)], 1) : tload<S, T>(p, v2[j], 2);
                    if (x == 0)  // left end
                        fin[j][2] =
                            bc_wrap_x(p.boundary) ? tload<S, T>(p, src[tidx(p, 2, nx - 1)], 2) : tload<S, T>(p, v1[j], 1);
                } else {
                    fin[j][0] = tload<S, T>(p, v0[j], 0);
                    fin[j][1] = tload<S, T>(p, v1[j], 1);
                    fin[j][2] = tload<S, T>(p, v2[j], 2);
                }
                bad[j] = tube_eval<T>(p, kk, fin[j], fs[j], fp[j], fa[j], nq[j], ds[j], dsin[j], rho[j], true);
            }

            // the median's neighbours: dS of the adjacent lanes' edge sites
            const T dl_lane = __shfl_up_sync(0xffffffffu, ds[V - 1], 1);
            const T dr_lane = __shfl_down_sync(0xffffffffu, ds[0], 1);

#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int x = xl + j;
                if (x >= nx) continue;
                ++acc.c_own;
                T phi_pos = T(1), phi_med = T(1);
                if (!bad[j]) {
                    if (p.limiters & 1u) {
                        if constexpr (F64) {
                            phi_pos = phi_positivity<3, T>(fs[j], fp[j]);
                        } else {
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                const float fpa = p.rwf[k] + fp[j][k];  // absolute f'
                                if (fpa < 0.f) phi_pos = fminf(phi_pos, fa[j][k] / (fa[j][k] - fpa));
                            }
                        }
                    }
                    // three-point median (the two end sites of a closed tube are not
                    // filtered; a periodic tube's end sites wrap around to each other)
                    const bool end = p.boundary == 0 && (x == 0 || x == nx - 1);
                    if ((p.limiters & 4u) && ds[j] > dm && !end) {
                        T left, right;
                        if (x == 0)
                            left = tube_ds<S>(p, kk, src, nx - 1);
                        else if (j > 0)
                            left = ds[j - 1];
                        else if (lane > 0)
                            left = dl_lane;
                        else
                            left = tube_ds<S>(p, kk, src, x - 1);
                        if (x == nx - 1)
                            right = tube_ds<S>(p, kk, src, 0);
                        else if (j + 1 < V)
                            right = ds[j + 1];
                        else if (lane < 31)
                            right = dr_lane;
                        else
                            right = tube_ds<S>(p, kk, src, x + 1);
                        const T med = med3(left, ds[j], right);
                        if constexpr (F64) {
                            phi_med = (p.phi_rule == 1 && p.eq == 1)
                                          ? phi_median_entropy<3>(fp[j], fs[j], ds[j], med, dm, p.median_mode)
                                          : phi_median<T>(ds[j], med, dm, p.median_mode);
                        } else {
                            phi_med = phi_median<T>(ds[j], med, dm, p.median_mode);
                        }
                    }
                }
                const T phi = phi_pos < phi_med ? phi_pos : phi_med;
                T lim = T(0);
                if (phi < T(1)) {
                    if constexpr (F64) {
                        double fo[3];
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            fo[k] = A::add(fs[j][k], A::mul(phi, A::sub(fp[j][k], fs[j][k])));
                            dst[tidx(p, k, x)] = fo[k];
                        }
                        if (p.eq == 1) {
                            const double dout = rel_entropy<3>(fo, fs[j]);
                            if (isfinite(ds[j]) && isfinite(dout)) lim = A::sub(ds[j], dout);
                        } else {
                            lim = A::mul(A::sub(1.0, A::mul(phi, phi)), ds[j]);
                        }
                    } else {
                        const float cw = limit_weight(phi, kk.a, p.collide != 0);
#pragma unroll
                        for (int k = 0; k < 3; ++k) dst[tidx(p, k, x)] = fmaf(-cw, nq[j][k], fin[j][k]);
                        if (p.eq == 1) {
                            float dout[3];
                            const float m = p.collide ? __fmul_rn(-phi, kk.a) : phi;
#pragma unroll
                            for (int k = 0; k < 3; ++k) dout[k] = __fmul_rn(m, nq[j][k]);
                            const float so = rel_entropy_dev<3>(dout, fa[j]);
                            if (isfinite(ds[j]) && isfinite(so)) lim = __fsub_rn(ds[j], so);
                        } else {
                            lim = __fmul_rn(__fsub_rn(1.f, __fmul_rn(phi, phi)), ds[j]);
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) dst[tidx(p, k, x)] = f2s<S>(fp[j][k]);
                }
                s_lim = A::add(s_lim, lim);
                if constexpr (F64)
                    s_mass = A::add(s_mass, rho[j]);
                else
                    s_mass = __fadd_rn(s_mass, __fsub_rn(rho[j], p.rho_ref));  // each term exact
                if (!bad[j]) {
                    T tds = T(0), tin = T(0);
                    if (p.eq == 1) {
                        if (isfinite(ds[j])) tds = ds[j];
                        if (isfinite(ds[j]) && isfinite(dsin[j])) tin = A::sub(dsin[j], ds[j]);
                    } else {
                        tds = ds[j];
                        tin = dsin[j];
                    }
                    s_ds = A::add(s_ds, tds);
                    s_in = A::add(s_in, tin);
                } else {
                    ++acc.c_bad;
                    atomicOr(p.status, kStatNonfinite);
                }
                acc.c_pos += phi_pos < T(1);
                acc.c_med += phi_med < T(1);
                if ((p.limiters & 2u) && !bad[j]) {
                    // Ehrenfests' candidates on an FP64 dS(f').  FP64 storage: ds itself.
                    // FP32 storage: sites near and above the threshold go to the warp's list
                    // and are keyed after the chunk, a lane each (below)
                    if constexpr (F64) {
                        if (ds[j] > p.delta_e) record(x, ds[j], (double)phi);
                    } else {
                        if (ds[j] > kk.thr_e) klist[atomicAdd(kcount, 1)] = make_int2(x, __float_as_int(phi));
                    }
                }
                if (p.ds_out) p.ds_out[x] = (double)ds[j];
            }
        }
        if constexpr (!F64) {
            __syncwarp();
            const int nk = *kcount;
            for (int i = lane; i < nk; i += 32) {
                const int2 e = klist[i];
                double fin64[3], fs64[3], fp64[3], d64, din64, r64;
                if (p.collide)
                    tube_pull<S, double>(p, src, e.x, fin64);
                else
                    tube_read<S, double>(p, src, e.x, fin64);
                const bool b64 =
                    site_collide<3, double>(fin64, p.a, p.collide != 0, fs64, fp64, d64, din64, r64, p.eq, false);
                if (!b64 && d64 > p.delta_e) record(e.x, d64, (double)__int_as_float(e.y));
            }
            __syncwarp();
            if (lane == 0) *kcount = 0;
            __syncwarp();
        }
        if constexpr (F64) {
            acc.t_mass = A::add(acc.t_mass, s_mass);
            acc.t_ds = A::add(acc.t_ds, s_ds);
            acc.t_in = A::add(acc.t_in, s_in);
            acc.t_lim = A::add(acc.t_lim, s_lim);
        } else {
            // butterfly: each level halves the sums a lane carries
            const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
            float x0 = hi16 ? s_in : s_mass, x1 = hi16 ? s_lim : s_ds;
            const float y0 = hi16 ? s_mass : s_in, y1 = hi16 ? s_ds : s_lim;
            x0 = __fadd_rn(x0, __shfl_xor_sync(0xffffffffu, y0, 16));
            x1 = __fadd_rn(x1, __shfl_xor_sync(0xffffffffu, y1, 16));
            float z = hi8 ? x1 : x0;
            z = __fadd_rn(z, __shfl_xor_sync(0xffffffffu, hi8 ? x0 : x1, 8));
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) z = __fadd_rn(z, __shfl_xor_sync(0xffffffffu, z, o));
            if ((lane & 7) == 0) fx_add(acc.fx, z, acc.fx_bad);
        }
    }
    twait<0>();
}

template <typename S, int V>
__global__ void __launch_bounds__(256, V > 1 ? 2 : 1)
    k_tube(const __grid_constant__ StepParams p, const S *__restrict__ src, S *__restrict__ dst, int chunked)
{
    constexpr bool F64 = std::is_same<compute_t<S>, double>::value;
    __shared__ TubeSlot<S, V> ring[kTubeWarps][kTubeRing];
    // FP32 storage: the chunk's sites whose FP32 dS(f') lies near or above the
    // threshold (site, phi), keyed in FP64 after the chunk with one lane each:
    // a chunk holding many of them costs one FP64 evaluation per 32, not one per
    // site a lane carries
    __shared__ int2 klist[kTubeWarps][F64 ? 1 : 32 * V];
    __shared__ int kcount[kTubeWarps];
    // the tail of the previous pass may still run (programmatic launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) kcount[warp] = 0;
    __syncwarp();
    TubeAcc acc{};
    tube_walk<S, V>(p, src, dst, blockIdx.x * nw + warp, (int)gridDim.x * nw, (p.nx + 32 * V - 1) / (32 * V),
                    ring[warp], klist[warp], &kcount[warp], acc);
    double t_mass = acc.t_mass, t_ds = acc.t_ds, t_in = acc.t_in, t_lim = acc.t_lim;
    if constexpr (!F64) tube_totals(acc, t_mass, t_ds, t_in, t_lim);
    int c_pos = acc.c_pos, c_med = acc.c_med, c_bad = acc.c_bad, c_own = acc.c_own;

    // block partial row: warp sums, then the warps in order; counts as integers
    __shared__ double sred[8][P_NSTAT];
    if constexpr (F64) {
        t_mass = wsum(t_mass);
        t_ds = wsum(t_ds);
        t_in = wsum(t_in);
        t_lim = wsum(t_lim);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c_pos += __shfl_down_sync(0xffffffffu, c_pos, o);
        c_med += __shfl_down_sync(0xffffffffu, c_med, o);
        c_bad += __shfl_down_sync(0xffffffffu, c_bad, o);
        c_own += __shfl_down_sync(0xffffffffu, c_own, o);
    }
    if (lane == 0) {
        sred[warp][P_MASS] = F64 ? t_mass : (double)p.rho_ref * (double)c_own + t_mass;
        sred[warp][P_SUM_DS] = t_ds;
        sred[warp][P_SUM_IN] = t_in;
        sred[warp][P_DS_LIM] = t_lim;
        sred[warp][P_NPOS] = (double)c_pos;
        sred[warp][P_NMED] = (double)c_med;
        sred[warp][P_NBAD] = (double)c_bad;
    }
    __syncthreads();
    const int bid = blockIdx.x, tid = threadIdx.x;
    if (tid < P_NSTAT) {
        double v = sred[0][tid];
        for (int w = 1; w < nw; ++w) v += sred[w][tid];
        p.partials[(long long)bid * P_NSTAT + tid] = v;
    }
    if (!chunked) return;
    // the last block of each chunk of kChunkRows blocks sums the chunk's rows in
    // row order (a ticket, no waiting)
    __shared__ int s_last;
    const int chunk = bid / kChunkRows;
    const int rows = min(kChunkRows, (int)gridDim.x - chunk * kChunkRows);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(p.chunk_cnt + chunk, 1u) == (unsigned)(rows - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        const double *base = p.partials + (long long)chunk * kChunkRows * P_NSTAT;
        for (int stat = warp; stat < P_NSTAT; stat += nw) {
            double v = 0.0;
            for (int r = lane; r < rows; r += 32) v += __ldcg(base + (long long)r * P_NSTAT + stat);
            v = wsum(v);
            if (lane == 0) p.partials2[(long long)chunk * P_NSTAT + stat] = v;
        }
        if (tid == 0) p.chunk_cnt[chunk] = 0u;  // for the next launch
    }
}

// Batched tubes (FP32 storage): work item i is group map[i].y (kTubeGroup
// chunks of 128 sites) of tube map[i].x of `table`; a warp runs its first item
// (its index in the grid), then takes items from the counter *work (cleared by
// the first tube's tail).  It keeps its tube's arguments in shared memory and
// writes each item's sums into the tube's partial row of that group (a fixed
// evaluation order per item, so the sums do not depend on which warp ran it).
template <int V>
__global__ void __launch_bounds__(256, 2) k_tube_batched(const TubeArgs *__restrict__ table,
                                                         const int2 *__restrict__ map, int items, int *work)
{
    using S = float;
    __shared__ TubeSlot<S, V> ring[kTubeWarps][kTubeRing];
    __shared__ int2 klist[kTubeWarps][32 * V];
    __shared__ int kcount[kTubeWarps];
    __shared__ __align__(16) TubeArgs sA[kTubeWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) kcount[warp] = 0;
    __syncwarp();
    int cur = -1;
    int item = blockIdx.x * nw + warp;
    while (item < items) {
        const int2 m = map[item];
        if (m.x != cur) {
            __syncwarp();
            const unsigned *from = reinterpret_cast<const unsigned *>(table + m.x);
            unsigned *to = reinterpret_cast<unsigned *>(&sA[warp]);
            for (int i = lane; i < (int)(sizeof(TubeArgs) / 4); i += 32) to[i] = from[i];
            __syncwarp();
            cur = m.x;
        }
        const StepParams &p = sA[warp].p;
        const int nch = (p.nx + 32 * V - 1) / (32 * V);
        const int c0 = m.y * kTubeGroup, c1 = min(c0 + kTubeGroup, nch);
        TubeAcc acc{};
        tube_walk<S, V, false>(p, (const S *)sA[warp].src, (S *)sA[warp].dst, c0, 1, c1, ring[warp], klist[warp],
                               &kcount[warp], acc);
        // the item's totals; the counts are per lane
        double t_mass, t_ds, t_in, t_lim;
        tube_totals(acc, t_mass, t_ds, t_in, t_lim);
        const int c_pos = __reduce_add_sync(0xffffffffu, acc.c_pos), c_med = __reduce_add_sync(0xffffffffu, acc.c_med);
        const int c_bad = __reduce_add_sync(0xffffffffu, acc.c_bad), c_own = __reduce_add_sync(0xffffffffu, acc.c_own);
        if (lane == 0) {
            double *row = p.partials + (long long)m.y * P_NSTAT;
            row[P_MASS] = (double)p.rho_ref * (double)c_own + t_mass;
            row[P_SUM_DS] = t_ds;
            row[P_SUM_IN] = t_in;
            row[P_DS_LIM] = t_lim;
            row[P_NPOS] = (double)c_pos;
            row[P_NMED] = (double)c_med;
            row[P_NBAD] = (double)c_bad;
        }
        int next = 0;
        if (lane == 0) next = (int)gridDim.x * nw + atomicAdd(work, 1);
        item = __shfl_sync(0xffffffffu, next, 0);
    }
}

// Launch shape: sites per lane, warps per block and blocks.  A tube of up to
// one chunk per SM sub-partition (4 x 152 chunks of 32 sites) runs one site per
// lane and a warp per block; longer tubes take 16-byte vectors (FP32 4 sites a
// lane, FP64 2) in blocks of 8 / 4 warps, at most one wave of resident blocks.
struct TubeShape {
    int v, warps, blocks;
};

template <typename S, int V>
int resident_blocks(int threads)
{
    static int per_sm = 0;
    if (per_sm == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tube<S, V>, threads, 0) != cudaSuccess || per_sm < 1)) {
        cudaGetLastError();
        per_sm = 2;
    }
    return per_sm * sm_count();
}

TubeShape tube_shape(bool fp64, int nx, bool launch)
{
    TubeShape t{};
    const long long slots = 4LL * sm_count();
    if ((long long)nx <= 32 * slots) {
        t.v = 1;
        t.warps = 1;
    } else {
        t.v = fp64 ? 2 : 4;
        t.warps = fp64 ? 4 : 8;
    }
    const long long per_block = 32LL * t.v * t.warps;
    long long blocks = (nx + per_block - 1) / per_block;
    if (t.v > 1) {
        // one wave: the occupancy of the kernel when launching, a bound (every
        // SM full of blocks of this size) when sizing the partial-sum rows
        const long long cap = !launch ? 2048LL / (32 * t.warps) * sm_count()
                                      : (fp64 ? resident_blocks<double, 2>(32 * t.warps)
                                              : resident_blocks<float, 4>(32 * t.warps));
        blocks = std::min(blocks, cap);
    }
    t.blocks = (int)blocks;
    return t;
}

}  // namespace

bool tube_applies(const lbm_config &c, unsigned limiters)
{
    return c.lattice == LBM_D1Q3 && (c.precision == LBM_FP64 || c.precision == LBM_FP32) &&
           (c.boundary == LBM_BC_WALLS || c.boundary == LBM_BC_PERIODIC) && !(limiters & kLimEnsemble) &&
           (c.kernel == LBM_KERNEL_AUTO || c.kernel == LBM_KERNEL_TUBE);
}

int tube_blocks(bool fp64, int nx) { return tube_shape(fp64, nx, false).blocks; }

template <typename S>
cudaError_t launch_tube(const StepParams &p, const S *src, S *dst, int *nblocks, bool *chunked, cudaStream_t s)
{
    constexpr bool fp64 = std::is_same<S, double>::value;
    const TubeShape t = tube_shape(fp64, p.nx, true);
    const int ch = t.blocks > kChunkRows ? 1 : 0;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)t.blocks);
    cfg.blockDim = dim3((unsigned)(32 * t.warps));
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e;
    if constexpr (fp64)
        e = t.v == 1 ? cudaLaunchKernelEx(&cfg, k_tube<S, 1>, p, src, dst, ch)
                     : cudaLaunchKernelEx(&cfg, k_tube<S, 2>, p, src, dst, ch);
    else
        e = t.v == 1 ? cudaLaunchKernelEx(&cfg, k_tube<S, 1>, p, src, dst, ch)
                     : cudaLaunchKernelEx(&cfg, k_tube<S, 4>, p, src, dst, ch);
    *nblocks = t.blocks;
    *chunked = ch != 0;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

int tube_groups(int nx) { return (nx + 128 * kTubeGroup - 1) / (128 * kTubeGroup); }

cudaError_t launch_tube_batched(const TubeArgs *table, const int2 *map, int items, int *work, cudaStream_t s)
{
    if (items <= 0) return cudaSuccess;
    static int per_sm = 0;
    if (per_sm == 0 &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tube_batched<4>, 256, 0) != cudaSuccess || per_sm < 1)) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int blocks = std::min((items + kTubeWarps - 1) / kTubeWarps, per_sm * sm_count());
    k_tube_batched<4><<<blocks, 32 * kTubeWarps, 0, s>>>(table, map, items, work);
    return cudaGetLastError();
}

template cudaError_t launch_tube<float>(const StepParams &, const float *, float *, int *, bool *, cudaStream_t);
template cudaError_t launch_tube<double>(const StepParams &, const double *, double *, int *, bool *, cudaStream_t);

}  // namespace lbm
