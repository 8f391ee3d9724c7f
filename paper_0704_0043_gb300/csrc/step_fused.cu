// step_fused.cu -- register-streaming fused D2Q9 step for the walled cavity.
//
// The same step as the tiled kernel (free flight with halfway bounce-back and
// moving lid, Sec. 2 and Sec. 4.4.1; polynomial f*, Eq. polyeq2d; LBGK
// collision, Eq. collLBGK; dS(f'), Sec. 3.6; positivity rule, Sec. 3.1; median
// filter, Sec. 3.5; Ehrenfests' candidates, Sec. 3.2; FP64 sums, Sec. 3.4),
// with the same per-site FP32 arithmetic, organised so that every warp streams
// its own part of the lattice with no shared memory and no barrier:
//
//  * Work item = one warp: a strip of 32 consecutive columns, of which lanes
//    1..30 finish their site (lanes 0 and 31 recompute the neighbouring
//    strips' edge columns), walked upward over a segment of rows.  Row r is
//    computed, then row r-1 is finished: its 3 x 3 dS stencil is then in
//    registers (three rows per lane, the side columns by warp shuffles).
//  * Free flight reads the populations arriving at row r straight from the
//    source field: planes {0,1,3} of row r, {2,5,6} of row r-1, {4,7,8} of
//    row r+1, each a coalesced 32-lane load, so every stored population is
//    read from DRAM once (strips overlap by two columns, segments by two
//    rows).  The loads of row r+1 are issued before row r is computed, so a
//    row of loads is always in flight behind the arithmetic.
//  * The post-collision deviations are stored at once; a site whose phi
//    (decided one row later) is below 1 reloads its row, recomputes the
//    collision exactly and overwrites its populations with the limited ones.
//  * Arithmetic is FP32 on the deviations g = f - rho_ref W in nonequilibrium
//    form (lattice.cuh), stored as FP32, BF16 or FP16; no FP64 on the
//    per-site path.  Sites whose FP32 dS is near or above the Ehrenfests'
//    threshold are recorded; the tail kernel recomputes their FP64 key from
//    the pre-step populations.  Sums are kept per thread in FP32 (mass as
//    rho - rho_ref), folded into FP64 every 128 rows, and reduced per block.
#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int kWarps = 4;  // independent work items per block
constexpr int kThreads = 32 * kWarps;
constexpr int kBlocksPerSM = 6;  // resident blocks per SM (3 for the batched kernel's larger state)
constexpr int kFoldRows = 128;   // FP32 partial sums are folded into FP64 every kFoldRows rows
constexpr int kMinSegRows = 16;  // shortest row segment (the two halo rows cost 2 / segment)

struct RowState {
    float ds, pp;
    bool bad, cand;
};

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
__global__ void __launch_bounds__(kThreads, BATCHED ? 3 : kBlocksPerSM)
    k_fused(const FusedArgs A0, const FusedArgs *__restrict__ table, const int2 *__restrict__ map)
{
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ double red[kWarps][P_NSTAT];
    __shared__ __align__(16) FusedArgs sA;
    int bid = (int)blockIdx.x;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if constexpr (BATCHED) {
        const int2 m = map[blockIdx.x];
        const unsigned *from = reinterpret_cast<const unsigned *>(table + m.x);
        unsigned *to = reinterpret_cast<unsigned *>(&sA);
        for (int i = t; i < (int)(sizeof(FusedArgs) / 4); i += kThreads) to[i] = from[i];
        bid = m.y;
        __syncthreads();
    }
    const FusedArgs &A = BATCHED ? sA : A0;
    const StepParams &p = A.p;

    float s_mass = 0.f, s_ds = 0.f, s_in = 0.f, s_lim = 0.f;
    int n_pos = 0, n_med = 0, n_bad = 0, n_sites = 0, rows_acc = 0;
    double acc_mass = 0.0, acc_ds = 0.0, acc_in = 0.0, acc_lim = 0.0;

    const int item = bid * kWarps + warp;
    if (item < A.items) {
        const S *__restrict__ src = (const S *)A.src;
        S *__restrict__ dst = (S *)A.dst;
        const int nx = p.nx, ny = p.ny, pitch = p.pitch;
        const int plane = (int)p.plane;  // 9 * plane < 2^31 is checked at launch
        const int strip = item % A.strips, seg = item / A.strips;
        const int x = 30 * strip - 1 + lane;  // lattice column of this lane
        const int ys = seg * A.seg_rows, ye = min(ys + A.seg_rows, ny);
        const int r0 = max(ys - 1, 0);
        const int rc = min(ye, ny - 1);  // last row whose dS this warp computes
        const bool xin = x >= 0 && x < nx;
        const bool xown = xin && lane >= 1 && lane <= 30;
        const bool xwall = x == 0 || x == nx - 1;
        const bool lim_ehr = (p.limiters & 2u) != 0;
        const bool med_on = MED && (p.limiters & 4u) != 0, pos_on = POS && (p.limiters & 1u) != 0;
        const float a = A.a, a2 = A.a * A.a, b2 = A.b2, rho_ref = p.rho_ref;
        // element offsets, from (plane 0, row q, column x), of the population of
        // plane k arriving at (x, q): source row q - cy_k, column x - cx_k
        const int o1 = plane - 1, o3 = 3 * plane + 1;
        const int o2 = 2 * plane - pitch, o5 = 5 * plane - pitch - 1, o6 = 6 * plane - pitch + 1;
        const int o4 = 4 * plane + pitch, o7 = 7 * plane + pitch + 1, o8 = 8 * plane + pitch - 1;
        // columns x - 1 and x + 1 stay inside the padded row (x >= -1, x <= nx + 29)

        // Loads of the populations arriving at row q (rows outside the lattice
        // are not read; their links are bounce-back links, set by edge_row).
        auto load_row = [&](int q, float g[9]) {
            const S *b = src + (long long)q * pitch + kLead + x;
            g[0] = s2f(b[0]);
            g[1] = s2f(b[o1]);
            g[3] = s2f(b[o3]);
            if (q >= 1) {
                g[2] = s2f(b[o2]);
                g[5] = s2f(b[o5]);
                g[6] = s2f(b[o6]);
            } else {
                g[2] = g[5] = g[6] = 0.f;
            }
            if (q + 1 < ny) {
                g[4] = s2f(b[o4]);
                g[7] = s2f(b[o7]);
                g[8] = s2f(b[o8]);
            } else {
                g[4] = g[7] = g[8] = 0.f;
            }
        };
        // Halfway bounce-back at wall sites: a link from outside returns the
        // site's own population of the opposite direction, plus the lid term.
        auto edge_row = [&](int q, float g[9]) {
            const bool edge = xin && (xwall || q == 0 || q == ny - 1);
            if (__any_sync(kFull, edge)) {
                if (edge) {
                    const S *b = src + (long long)q * pitch + kLead + x;
#pragma unroll
                    for (int k = 1; k < 9; ++k) {
                        const int sx = x - Lat<9>::cx(k), sy = q - Lat<9>::cy(k);
                        if (sx >= 0 && sx < nx && sy >= 0 && sy < ny) continue;
                        float v = s2f(b[Lat<9>::opp(k) * plane]);
                        if (sy > ny - 1) {
                            v += k == 4 ? A.lid4 : (k == 7 ? A.lid7 : A.lid8);
                            v += k == 4 ? A.lo4 : (k == 7 ? A.lo7 : A.lo8);
                        }
                        g[k] = v;
                    }
                }
            }
        };

        // Row q from its loaded populations: collision, dS; stores g' of the
        // warp's own sites.  Rare per-site paths sit behind warp votes.
        auto compute_row = [&](int q, float g[9]) -> RowState {
            RowState st{0.f, 1.f, false, false};
            edge_row(q, g);
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
                S *out = dst + (long long)q * pitch + kLead + x;
#pragma unroll
                for (int k = 0; k < 9; ++k) out[k * plane] = f2s<S>(g[k]);
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
                // nonequilibrium form), with g and n recomputed exactly as the
                // collision computed them (every lane takes part: edge_row votes)
                float g[9];
                load_row(y, g);
                edge_row(y, g);
                if (phi < 1.f) {
                    float drho, rho, ux, uy, gs[9], n[9];
                    moments9_dev(g, rho_ref, drho, rho, ux, uy);
                    feq9_dev(drho, rho, ux, uy, gs);
                    neq9(g, gs, n);
                    const float c = limit_weight(phi, a, true);
                    S *out = dst + (long long)y * pitch + kLead + x;
#pragma unroll
                    for (int k = 0; k < 9; ++k) out[k * plane] = f2s<S>(fmaf(-c, n[k], g[k]));
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
                if (++rows_acc == kFoldRows) {
                    acc_mass += (double)s_mass;
                    acc_ds += (double)s_ds;
                    acc_in += (double)s_in;
                    acc_lim += (double)s_lim;
                    s_mass = s_ds = s_in = s_lim = 0.f;
                    rows_acc = 0;
                }
            }
        };

        // Iteration r computes row r from the loads issued one iteration
        // earlier and finishes row r-1.  The loop is unrolled twice so that the
        // two load buffers swap roles by name (no copy waits for a load).
        RowState prev{0.f, 1.f, false, false};
        float ds_m2 = 0.f, ds_m1 = 0.f;  // dS of rows r-2 and r-1 (this lane's column)
        auto body = [&](int r, float(&cmp)[9], float(&ld)[9]) {
            RowState st{0.f, 1.f, false, false};
            if (r <= rc) {
                if (r + 1 <= rc) load_row(r + 1, ld);
                st = compute_row(r, cmp);
            }
            if (r - 1 >= ys) finalise_row(r - 1, prev, ds_m2, ds_m1, st.ds);
            ds_m2 = ds_m1;
            ds_m1 = st.ds;
            prev = st;
        };
        float bufA[9], bufB[9];
        load_row(r0, bufA);
        for (int r = r0;;) {
            body(r, bufA, bufB);
            if (++r - 1 >= ye) break;
            body(r, bufB, bufA);
            if (++r - 1 >= ye) break;
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
        for (int w = 0; w < kWarps; ++w) v += red[w][t];
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
    k_fused<S, MED, POS, BATCHED><<<blocks, kThreads, 0, s>>>(A, table, map);
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

}  // namespace

int fused_slots() { return kBlocksPerSM * kWarps * sm_count(); }

// A launch has one block per kWarps work items; items are strips of 30
// columns times row segments of at least kMinSegRows rows.
int fused_d2q9_blocks(int nx, int ny)
{
    const long long strips = (nx + 29) / 30, segs = (ny + kMinSegRows - 1) / kMinSegRows;
    return (int)((strips * segs + kWarps - 1) / kWarps);
}

bool fused_d2q9_fits(long long plane) { return 9LL * plane < 0x7fffffffLL; }

int fused_make_args(const StepParams &p, const void *src, void *dst, int seg_rows, int slots, FusedArgs *A)
{
    *A = FusedArgs{};
    A->p = p;
    A->src = src;
    A->dst = dst;
    // Work items: strips of 30 columns x row segments, about `slots` of them
    // (one wave of resident warps) unless `seg_rows` fixes the segment.
    A->strips = (p.nx + 29) / 30;
    int rows = seg_rows;
    if (rows <= 0) {
        const int segs = std::max(1, std::max(1, slots) / A->strips);
        rows = (p.ny + segs - 1) / segs;
    }
    A->seg_rows = std::max(kMinSegRows, rows);
    A->items = A->strips * ((p.ny + A->seg_rows - 1) / A->seg_rows);
    A->blocks = (A->items + kWarps - 1) / kWarps;
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
