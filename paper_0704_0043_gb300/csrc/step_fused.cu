// step_fused.cu -- row-streaming fused D2Q9 step for the walled cavity.
//
// The same step as the tiled kernel (free flight with halfway bounce-back and
// moving lid, Sec. 2 and Sec. 4.4.1; polynomial f*, Eq. polyeq2d; LBGK
// collision, Eq. collLBGK; dS(f'), Sec. 3.6; positivity rule, Sec. 3.1; median
// filter, Sec. 3.5; Ehrenfests' candidates, Sec. 3.2; FP64 sums, Sec. 3.4),
// with the same per-site FP32 arithmetic, organised for HBM streaming with
// warps that run independently of each other:
//
//  * A block owns a strip of at most 240 columns (a multiple of 8) and walks a
//    segment of rows upward.  It has eight compute warps, a load warp and a
//    store warp.  Compute warp w covers 32 consecutive columns of which lanes
//    1..30 finish their site; lanes 0 and 31 recompute the neighbouring
//    warps' edge columns, so each warp holds the whole 3 x 3 dS stencil of its
//    sites in registers (three rows per lane, the side columns by shuffles)
//    and never waits for another compute warp.
//  * Input: the load warp copies, per row, the strip's nine population rows
//    (bulk asynchronous copies, cp.async.bulk, completion counted on a "full"
//    mbarrier) into an 8-deep ring of shared-memory stages.  Stage s holds the
//    rows the pull of row s reads: planes {0,1,3} of row s, {2,5,6} of row
//    s-1, {4,7,8} of row s+1, so every stored population is read from DRAM
//    once.  A compute warp releases stage s on its "empty" mbarrier after
//    finishing row s+1 (the limiter recomputes that row's pull); the load
//    warp refills a slot once every compute warp has released it.
//  * Output: a compute warp writes the post-collision deviations of its sites
//    into a 4-deep ring of shared-memory output rows, applies the limiters to
//    row r-1 after computing row r (the median needs rows r-2..r), and marks
//    the row done on an mbarrier; the store warp then writes the finished row
//    to global memory with bulk asynchronous stores (one per plane).
//  * Arithmetic is FP32 on the deviations g = f - rho_ref W in nonequilibrium
//    form (lattice.cuh), stored as FP32, BF16 or FP16; no FP64 on the
//    per-site path.  Sites whose FP32 dS is near or above the Ehrenfests'
//    threshold are recorded; the tail kernel recomputes their FP64 key from
//    the pre-step populations.  Sums are kept per thread in FP32 (mass as
//    rho - rho_ref) and folded into FP64 every 32 rows.
//  * Every mbarrier wait is bounded by a clock limit and watches a block-wide
//    abort flag; on expiry the thread sets the timeout status bit and the
//    flag, and every warp leaves its loop.
#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int kW = 8;                // compute warps per block
constexpr int kThreads = 32 * (kW + 2);
constexpr int kMaxWidth = 30 * kW;   // finished columns per strip (at most)
constexpr int kLW = kMaxWidth + 16;  // staged columns per row (halo and 16-byte alignment)
constexpr int kStages = 8;           // input ring
constexpr int kOut = 4;              // output ring
constexpr int kMinSegRows = 16;      // shortest row segment (the halo rows cost 2 / segment)
constexpr long long kWaitLimit = 4000000000LL;  // clock cycles (about 2 s)

template <typename S> struct FusedSmem {
    S in[kStages][9][kLW];
    S out[kOut][9][kMaxWidth];
    unsigned long long full[kStages], empty[kStages], ofull[kOut], oempty[kOut];
    int abort;
};

struct RowState {
    float ds, pp;
    bool bad, cand;
};

__device__ __forceinline__ unsigned smem_addr(const void *ptr)
{
    return (unsigned)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity.  Gives up when another
// thread of the block has set the abort flag, or after kWaitLimit cycles (then
// it sets the flag and the timeout status bit itself).
__device__ __noinline__ bool mbar_wait_slow(unsigned long long *bar, unsigned parity, volatile int *abort,
                                            unsigned *status)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > kWaitLimit) {
            *abort = 1;
            atomicOr(status, kStatTimeout);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, volatile int *abort,
                                          unsigned *status)
{
    return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity, abort, status);
}

// global -> shared bulk copy, completion counted on `bar`
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// shared -> global bulk copy in the issuing thread's bulk-async group
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// orders this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) reads of them
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sorted column (lo <= mid <= hi) of three values.
__device__ __forceinline__ void sort3(float a, float b, float c, float &lo, float &mid, float &hi)
{
    const float t1 = fminf(a, b), t2 = fmaxf(a, b);
    lo = fminf(t1, c);
    const float t3 = fmaxf(t1, c);
    mid = fminf(t2, t3);
    hi = fmaxf(t2, t3);
}

// MED / POS: the median / positivity code is compiled in (each still follows
// the instance's limiter bits).  BATCHED: block b runs instance map[b].x of
// `table` as its block map[b].y; otherwise the single instance A0.
// S: storage type of the deviations (float, __nv_bfloat16 or __half).
template <typename S, bool MED, bool POS, bool BATCHED>
__global__ void __launch_bounds__(kThreads, 2) k_fused(const FusedArgs A0, const FusedArgs *__restrict__ table,
                                                       const int2 *__restrict__ map)
{
    constexpr int E = 16 / (int)sizeof(S);  // elements per 16 bytes
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FusedSmem<S> &sm = *reinterpret_cast<FusedSmem<S> *>(smem_raw);
    __shared__ double red[kW + 2][P_NSTAT];
    __shared__ __align__(16) FusedArgs sA;
    int bid = (int)blockIdx.x;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if constexpr (BATCHED) {
        const int2 m = map[blockIdx.x];
        const unsigned *from = reinterpret_cast<const unsigned *>(table + m.x);
        unsigned *to = reinterpret_cast<unsigned *>(&sA);
        for (int i = t; i < (int)(sizeof(FusedArgs) / 4); i += kThreads) to[i] = from[i];
        bid = m.y;
    }
    // The output ring starts zeroed, and only lattice columns are written to
    // it: the columns a row store carries past the lattice's right edge (up to
    // the next 16 bytes) keep the row padding's zero fill.
    {
        unsigned *o = reinterpret_cast<unsigned *>(&sm.out[0][0][0]);
        for (int i = t; i < (int)(sizeof(sm.out) / 4); i += kThreads) o[i] = 0u;
    }
    __syncthreads();
    const FusedArgs &A = BATCHED ? sA : A0;
    const StepParams &p = A.p;
    const int nx = p.nx, ny = p.ny;
    const int plane = (int)p.plane;  // 9 * plane < 2^31 is checked at launch
    const int strip = bid % A.strips, seg = bid / A.strips;
    const int c0 = strip * A.sw;           // first column of the strip (a multiple of 8)
    const int width = min(A.sw, nx - c0);  // finished columns
    const int nw = (width + 29) / 30;      // compute warps with work
    const int ys = seg * A.seg_rows, ye = min(ys + A.seg_rows, ny);
    const int r0 = max(ys - 1, 0);
    const int rc = min(ye, ny - 1);  // last row whose dS this block computes
    const int s_first = r0 - 1, s_last = rc + 1;
    // staged columns [xs0, xs0 + Lc): 16-byte aligned, inside the padded row
    const int xs0 = c0 - E;
    const int Lc = min(kLW, ((nx + E - 1) & ~(E - 1)) + E - xs0);
    volatile int *abort = &sm.abort;

    if (t == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], (unsigned)nw);
        }
        for (int i = 0; i < kOut; ++i) {
            mbar_init(&sm.ofull[i], (unsigned)nw);
            mbar_init(&sm.oempty[i], 1);
        }
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    float s_mass = 0.f, s_ds = 0.f, s_in = 0.f, s_lim = 0.f;
    int n_pos = 0, n_med = 0, n_bad = 0, n_sites = 0, rows_acc = 0;
    double acc_mass = 0.0, acc_ds = 0.0, acc_in = 0.0, acc_lim = 0.0;

    if (warp == kW) {
        // ---- load warp: stage s into slot (s - s_first) mod kStages ----
        const S *__restrict__ src = (const S *)A.src;
        const unsigned row_bytes = (unsigned)Lc * (unsigned)sizeof(S);
        int issued = 0;
        for (int s = s_first; s <= s_last; ++s) {
            const unsigned j = (unsigned)(s - s_first), slot = j % kStages;
            if (j >= kStages) {  // every compute warp released the slot's previous stage
                bool ok = true;
                if (lane == 0) ok = mbar_wait(&sm.empty[slot], (j / kStages - 1) & 1u, abort, p.status);
                if (!__shfl_sync(kFull, (int)ok, 0)) break;
            }
            unsigned bytes = 0;
            if (s >= 0 && s < ny) bytes += 3u * row_bytes;
            if (s - 1 >= 0 && s - 1 < ny) bytes += 3u * row_bytes;
            if (s + 1 >= 0 && s + 1 < ny) bytes += 3u * row_bytes;
            if (lane == 0) mbar_expect_tx(&sm.full[slot], bytes);
            __syncwarp();
            if (lane < 9) {
                const int k = lane;
                const int row = (k == 0 || k == 1 || k == 3) ? s : ((k == 2 || k == 5 || k == 6) ? s - 1 : s + 1);
                if (row >= 0 && row < ny)
                    bulk_load(&sm.in[slot][k][0], src + (long long)k * plane + (long long)row * p.pitch + kLead + xs0,
                              row_bytes, &sm.full[slot]);
            }
            ++issued;
        }
        // After an abort, wait (bounded) for the copies still in flight: the
        // last kStages issued stages (earlier ones were waited for by the
        // compute warps before their slots were released).
        if (*abort && lane == 0) {
            for (int s = s_first + max(0, issued - kStages); s < s_first + issued; ++s) {
                const unsigned j = (unsigned)(s - s_first);
                const long long t0 = clock64();
                while (!mbar_try_wait(&sm.full[j % kStages], (j / kStages) & 1u) && clock64() - t0 < kWaitLimit) {
                }
            }
        }
    } else if (warp == kW + 1) {
        // ---- store warp: finished row y from output slot (y - ys) mod kOut ----
        S *__restrict__ dst = (S *)A.dst;
        const unsigned bytes = (unsigned)((width + E - 1) & ~(E - 1)) * (unsigned)sizeof(S);
        for (int y = ys; y < ye; ++y) {
            const unsigned j = (unsigned)(y - ys), slot = j % kOut;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&sm.ofull[slot], (j / kOut) & 1u, abort, p.status);
            if (!__shfl_sync(kFull, (int)ok, 0)) break;
            if (lane < 9) {
                bulk_store(dst + (long long)lane * plane + (long long)y * p.pitch + kLead + c0, &sm.out[slot][lane][0],
                           bytes);
                bulk_commit();
                bulk_wait_read_all();  // the slot may be refilled once its bytes are read
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.oempty[slot]);
        }
        if (lane < 9) bulk_wait_all();
    } else if (warp < nw) {
        // ---- compute warp ----
        const int x = c0 - 1 + 30 * warp + lane;  // lattice column of this lane
        const int o = x - xs0;                     // staged index of column x
        const int ox = x - c0;                     // output-row index of column x
        const bool xin = x >= 0 && x < nx;
        const bool xown = xin && lane >= 1 && lane <= 30 && ox < width;
        const bool xwall = x == 0 || x == nx - 1;
        const bool lim_ehr = (p.limiters & 2u) != 0;
        const bool med_on = MED && (p.limiters & 4u) != 0, pos_on = POS && (p.limiters & 1u) != 0;
        const float a = A.a, a2 = A.a * A.a, b2 = A.b2, rho_ref = p.rho_ref;

        auto in_slot = [&](int s) { return (unsigned)(s - s_first) % kStages; };
        auto wait_stage = [&](int s) -> bool {
            if (s > s_last) return true;
            const unsigned j = (unsigned)(s - s_first);
            return mbar_wait(&sm.full[j % kStages], (j / kStages) & 1u, abort, p.status);
        };

        // Free flight into row q: the stored deviations arriving at (x, q).  A
        // link from outside returns the site's own population of the opposite
        // direction (halfway bounce-back; planes {0,1,3} of row q sit in stage
        // q, {2,5,6} in stage q+1, {4,7,8} in stage q-1), plus the lid term.
        auto pull_row = [&](int q, float g[9]) {
            const S(*S0)[kLW] = sm.in[in_slot(q)];
            const S(*Sm)[kLW] = sm.in[in_slot(q - 1)];
            const S(*Sp)[kLW] = sm.in[in_slot(q + 1)];
            g[0] = s2f(S0[0][o]);
            g[1] = s2f(S0[1][o - 1]);
            g[2] = s2f(S0[2][o]);
            g[3] = s2f(S0[3][o + 1]);
            g[4] = s2f(S0[4][o]);
            g[5] = s2f(S0[5][o - 1]);
            g[6] = s2f(S0[6][o + 1]);
            g[7] = s2f(S0[7][o + 1]);
            g[8] = s2f(S0[8][o - 1]);
            const bool edge = xin && (xwall || q == 0 || q == ny - 1);
            if (__any_sync(kFull, edge)) {
                if (edge) {
#pragma unroll
                    for (int k = 1; k < 9; ++k) {
                        const int sx = x - Lat<9>::cx(k), sy = q - Lat<9>::cy(k);
                        if (sx >= 0 && sx < nx && sy >= 0 && sy < ny) continue;
                        const int qq = Lat<9>::opp(k);
                        float v = s2f((qq == 1 || qq == 3) ? S0[qq][o]
                                                            : ((qq == 2 || qq == 5 || qq == 6) ? Sp[qq][o] : Sm[qq][o]));
                        if (sy > ny - 1) {
                            v += k == 4 ? A.lid4 : (k == 7 ? A.lid7 : A.lid8);
                            v += k == 4 ? A.lo4 : (k == 7 ? A.lo7 : A.lo8);
                        }
                        g[k] = v;
                    }
                }
            }
        };

        // Row q: free flight, collision, dS; writes g' of the block's own sites
        // into the output row.  Rare per-site paths sit behind warp votes.
        auto compute_row = [&](int q) -> RowState {
            RowState st{0.f, 1.f, false, false};
            float g[9];
            pull_row(q, g);
            float drho, rho, ux, uy, gs[9], n[9];
            moments9_dev(g, rho_ref, drho, rho, ux, uy);
            feq9_dev(drho, rho, ux, uy, gs);
            neq9(g, gs, n);
            float din = 0.f, fpmin = 3.4e38f;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                din = fmaf(n[k] * n[k], rcp_approx(p.rwf[k] + gs[k]), din);  // / absolute f*
                g[k] = fmaf(-b2, n[k], g[k]);                                // g' = g - 2 beta n
                if (pos_on) fpmin = fminf(fpmin, p.rwf[k] + g[k]);
            }
            float ds = a2 * din;  // dS(f') = (2 beta - 1)^2 dS(f_in) for the same f*
            // f*_k >= rho W_k (1/2 - 3 u^2 / 2) > 0 whenever u^2 < 1/3; only fast
            // flows need the explicit test of every f*_k
            const float usq = fmaf(ux, ux, uy * uy);
            bool bad = !(rho > 0.f) || !isfinite(ds);
            if (__any_sync(kFull, !(usq < 0.3f))) {
                float fsmin = 3.4e38f;
#pragma unroll
                for (int k = 0; k < 9; ++k) fsmin = fminf(fsmin, p.rwf[k] + gs[k]);
                bad = bad || !(fsmin > 0.f);
            }
            if (bad) ds = __int_as_float(0x7f800000);
            if (pos_on && __any_sync(kFull, !bad && fpmin < 0.f)) {
                if (!bad && fpmin < 0.f) {  // positivity rule (Sec. 3.1)
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const float fpa = p.rwf[k] + g[k], fsa = p.rwf[k] + gs[k];
                        if (fpa < 0.f) st.pp = fminf(st.pp, fsa / (fsa - fpa));
                    }
                }
            }
            const bool own = xown && q >= ys && q < ye;
            if (own) {
                S *out = &sm.out[(unsigned)(q - ys) % kOut][0][ox];
#pragma unroll
                for (int k = 0; k < 9; ++k) out[k * kMaxWidth] = f2s<S>(g[k]);
                s_mass += drho;
                ++n_sites;
                if (!bad) {
                    s_ds += ds;
                    s_in += din;
                } else {
                    ++n_bad;
                }
                n_pos += st.pp < 1.f;
            }
            if (__any_sync(kFull, own && bad) && lane == 0) atomicOr(p.status, kStatNonfinite);
            // Ehrenfests' candidates: the tail kernel recomputes the FP64 key of
            // every site recorded here from the pre-step populations
            st.cand = lim_ehr && !bad && own && ds > A.thr_e;
            st.bad = bad;
            st.ds = ds;
            return st;
        };

        // Row y: median of dS (rows y-1, y, y+1 in dm, d0, dp), phi = min(phi_pos,
        // phi_med), limited update where phi < 1, candidate record, sums.
        auto finalise_row = [&](int y, const RowState &st, float dm, float d0, float dp) {
            const bool act = xown && y >= ys && y < ye;
            float pm = 1.f;
            if (med_on) {
                // 3 x 3 median from sorted columns: the median of (largest column
                // minimum, median of the column medians, smallest column maximum);
                // wall rows and columns take the near-wall stencils
                float lo, mid, hi;
                sort3(dm, d0, dp, lo, mid, hi);
                const float lo_l = __shfl_up_sync(kFull, lo, 1), lo_r = __shfl_down_sync(kFull, lo, 1);
                const float mid_l = __shfl_up_sync(kFull, mid, 1), mid_r = __shfl_down_sync(kFull, mid, 1);
                const float hi_l = __shfl_up_sync(kFull, hi, 1), hi_r = __shfl_down_sync(kFull, hi, 1);
                float med = med3(fmaxf(fmaxf(lo_l, lo), lo_r), med3(mid_l, mid, mid_r), fminf(fminf(hi_l, hi), hi_r));
                const bool ywall = y == 0 || y == ny - 1;  // the same for the whole warp
                if (ywall) {
                    const float d_l = __shfl_up_sync(kFull, d0, 1), d_r = __shfl_down_sync(kFull, d0, 1);
                    med = xwall ? med3(d0, x == 0 ? d_r : d_l, y == 0 ? dp : dm) : med3(d_l, d0, d_r);
                } else if (xwall) {
                    med = mid;
                }
                if (act && !st.bad) pm = phi_median<float>(st.ds, med, A.delta_m, p.median_mode);
            }
            const float phi = act ? fminf(st.pp, pm) : 1.f;
            if (__any_sync(kFull, phi < 1.f)) {
                // the limited update g - (1 + phi (2 beta - 1)) n (Eq. LimGenF in
                // nonequilibrium form), with g and n recomputed from the staged
                // rows exactly as the collision computed them (every lane of the
                // warp takes part: pull_row votes across the warp)
                float g[9];
                pull_row(y, g);
                if (phi < 1.f) {
                    float drho, rho, ux, uy, gs[9], n[9];
                    moments9_dev(g, rho_ref, drho, rho, ux, uy);
                    feq9_dev(drho, rho, ux, uy, gs);
                    neq9(g, gs, n);
                    const float c = limit_weight(phi, a, true);
                    S *out = &sm.out[(unsigned)(y - ys) % kOut][0][ox];
#pragma unroll
                    for (int k = 0; k < 9; ++k) out[k * kMaxWidth] = f2s<S>(fmaf(-c, n[k], g[k]));
                    s_lim = fmaf(1.f - phi * phi, st.ds, s_lim);
                }
            }
            if (act) {
                n_med += pm < 1.f;
                if (st.cand) {
                    const int slot = atomicAdd(p.cand_count, 1);
                    if (slot < p.cand_cap) {
                        Cand cd;
                        cd.key = 0.0;
                        cd.phi = (double)phi;
                        cd.site = y * nx + x;
                        cd.pad = 0;
                        p.cand[slot] = cd;
                    } else {
                        atomicOr(p.status, kStatCandOverflow);
                    }
                }
                if (++rows_acc == 32) {
                    acc_mass += (double)s_mass;
                    acc_ds += (double)s_ds;
                    acc_in += (double)s_in;
                    acc_lim += (double)s_lim;
                    s_mass = s_ds = s_in = s_lim = 0.f;
                    rows_acc = 0;
                }
            }
        };

        // Iteration r computes row r, then finishes row r-1, whose dS stencil
        // rows r-2, r-1, r are then in registers.
        RowState prev{0.f, 1.f, false, false};
        float ds_m2 = 0.f, ds_m1 = 0.f;  // dS of rows r-2 and r-1 (this lane's column)
        for (int r = r0; r - 1 < ye; ++r) {
            RowState cur{0.f, 1.f, false, false};
            if (r <= rc) {
                bool ok = wait_stage(r + 1);
                if (r == r0) ok = ok && wait_stage(r - 1) && wait_stage(r);
                const unsigned jo = (unsigned)(r - ys);
                if (ok && r >= ys && r < ye && jo >= kOut)  // output slot free again
                    ok = mbar_wait(&sm.oempty[jo % kOut], (jo / kOut - 1) & 1u, abort, p.status);
                if (!__all_sync(kFull, ok)) break;
                cur = compute_row(r);
            }
            if (r - 1 >= ys) {
                finalise_row(r - 1, prev, ds_m2, ds_m1, cur.ds);
                fence_proxy_async();  // the row's shared-memory writes before the bulk store reads them
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.ofull[(unsigned)(r - 1 - ys) % kOut]);
            }
            if (r - 2 >= s_first) {  // stage r-2 is no longer read by this warp
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.empty[in_slot(r - 2)]);
            }
            ds_m2 = ds_m1;
            ds_m1 = cur.ds;
            prev = cur;
        }
    }

    double acc[P_NSTAT];
    acc[P_MASS] = acc_mass + (double)s_mass + (double)n_sites * (double)p.rho_ref;
    acc[P_SUM_DS] = acc_ds + (double)s_ds;
    acc[P_SUM_IN] = acc_in + (double)s_in;
    acc[P_DS_LIM] = acc_lim + (double)s_lim;
    acc[P_NPOS] = (double)n_pos;
    acc[P_NMED] = (double)n_med;
    acc[P_NBAD] = (double)n_bad;
#pragma unroll
    for (int i = 0; i < P_NSTAT; ++i) {
        const double v = warp_sum_d(acc[i]);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    if (t < P_NSTAT) {
        double v = 0.0;
        for (int w = 0; w < kW + 2; ++w) v += red[w][t];
        p.partials[(long long)bid * P_NSTAT + t] = v;
    }
}

int sm_count()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
            cudaGetLastError();
            sms = 152;
        }
    }
    return sms;
}

template <typename S, bool MED, bool POS, bool BATCHED>
cudaError_t launch_k(const FusedArgs &A, const FusedArgs *table, const int2 *map, int blocks, cudaStream_t s)
{
    const size_t smem = sizeof(FusedSmem<S>);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<S, MED, POS, BATCHED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_fused<S, MED, POS, BATCHED><<<blocks, kThreads, smem, s>>>(A, table, map);
    return cudaGetLastError();
}

// FP32 storage: one kernel per limiter set; 16-bit storage: one kernel that
// follows the limiter bits at run time.
template <typename S>
cudaError_t launch_lim(const FusedArgs &A, int blocks, cudaStream_t s)
{
    if constexpr (std::is_same<S, float>::value) {
        const bool med = (A.p.limiters & 4u) != 0, pos = (A.p.limiters & 1u) != 0;
        if (med && pos) return launch_k<S, true, true, false>(A, nullptr, nullptr, blocks, s);
        if (med) return launch_k<S, true, false, false>(A, nullptr, nullptr, blocks, s);
        if (pos) return launch_k<S, false, true, false>(A, nullptr, nullptr, blocks, s);
        return launch_k<S, false, false, false>(A, nullptr, nullptr, blocks, s);
    } else {
        return launch_k<S, true, true, false>(A, nullptr, nullptr, blocks, s);
    }
}

constexpr int kStripChoices = 8;  // strip counts tried above the fewest possible

}  // namespace

int fused_slots() { return 2 * sm_count(); }

// A launch has at most max(strips, slots) blocks (fused_make_args), strips of
// at least 8 columns, segments of at least kMinSegRows rows, and at most four
// waves of slots (the batch engine's largest budget).
int fused_d2q9_blocks(int nx, int ny)
{
    const long long strips = (nx + 7) / 8, segs = (ny + kMinSegRows - 1) / kMinSegRows;
    const long long most = std::max<long long>(4LL * fused_slots(), strips);
    return (int)std::min(strips * segs, most);
}

bool fused_d2q9_fits(long long plane) { return 9LL * plane < 0x7fffffffLL; }

int fused_make_args(const StepParams &p, const void *src, void *dst, int max_width, int slots, FusedArgs *A)
{
    *A = FusedArgs{};
    A->p = p;
    A->src = src;
    A->dst = dst;
    slots = std::max(1, slots);
    // Strip width (a multiple of 8, at most 240 or max_width) and row
    // segments: the choice with the least work on the busiest block slot,
    // counted as waves of `slots` blocks x (rows + 2 halo rows) x active warps.
    const int cap = max_width > 0 ? std::min(kMaxWidth, std::max(8, max_width & ~7)) : kMaxWidth;
    const int fewest = (p.nx + cap - 1) / cap;
    long long best = -1;
    for (int want = fewest; want < fewest + kStripChoices; ++want) {
        const int sw = std::min(cap, (((p.nx + want - 1) / want) + 7) & ~7);
        const int strips = (p.nx + sw - 1) / sw;
        const int warps = (std::min(sw, p.nx) + 29) / 30;
        int segs = std::max(1, slots / strips);
        const int seg_rows = std::max(kMinSegRows, (p.ny + segs - 1) / segs);
        segs = (p.ny + seg_rows - 1) / seg_rows;
        const long long blocks = (long long)strips * segs;
        const long long waves = (blocks + slots - 1) / slots;
        const long long cost = waves * (seg_rows + 2) * warps;
        if (best < 0 || cost < best || (cost == best && blocks < A->blocks)) {
            best = cost;
            A->sw = sw;
            A->strips = strips;
            A->seg_rows = seg_rows;
            A->blocks = (int)blocks;
        }
        if (sw == 8) break;
    }
    A->a = (float)p.a;
    A->b2 = (float)(1.0 + p.a);
    A->delta_m = (float)p.delta_m;
    A->thr_e = (float)(p.delta_e * (1.0 - 1.0 / 64.0));
    A->rho_ref = p.rho_ref;
    A->lid4 = p.lidf[4];
    A->lid7 = p.lidf[7];
    A->lid8 = p.lidf[8];
    A->lo4 = p.lidlo[4];
    A->lo7 = p.lidlo[7];
    A->lo8 = p.lidlo[8];
    return A->blocks;
}

template <typename S>
cudaError_t launch_fused_d2q9(const StepParams &p, const S *src, S *dst, int *nblocks, cudaStream_t s)
{
    FusedArgs A;
    *nblocks = fused_make_args(p, src, dst, 0, fused_slots(), &A);
    return launch_lim<S>(A, A.blocks, s);
}

template cudaError_t launch_fused_d2q9<float>(const StepParams &, const float *, float *, int *, cudaStream_t);
template cudaError_t launch_fused_d2q9<__nv_bfloat16>(const StepParams &, const __nv_bfloat16 *, __nv_bfloat16 *,
                                                      int *, cudaStream_t);
template cudaError_t launch_fused_d2q9<__half>(const StepParams &, const __half *, __half *, int *, cudaStream_t);

cudaError_t launch_fused_batched(const FusedArgs *table, const int2 *map, int blocks, cudaStream_t s)
{
    if (blocks <= 0) return cudaSuccess;
    const FusedArgs none{};
    return launch_k<float, true, true, true>(none, table, map, blocks, s);
}

}  // namespace lbm
