// step_fused.cu -- row-streaming fused D2Q9 step for the walled cavity.
//
// The same step as the tiled kernel (free flight with halfway bounce-back and
// moving lid, Sec. 2 and Sec. 4.4.1; polynomial f*, Eq. polyeq2d; LBGK
// collision, Eq. collLBGK; dS(f'), Sec. 3.6; positivity rule, Sec. 3.1; median
// filter, Sec. 3.5; Ehrenfests' candidates, Sec. 3.2; sums, Sec. 3.4), with
// the same per-site FP32 operations (lattice.cuh), organised so that every
// warp streams its own part of the lattice and never waits for another:
//
//  * Work item = a strip of 64 consecutive columns walked upward over a
//    segment of rows by one warp.  Lane l carries two columns, l and l + 32
//    of the strip, and evaluates both sites with paired FP32 instructions
//    (F2).  The strip's first and last columns recompute the neighbouring
//    strips' edge columns; the other 62 are finished here.  Row r is
//    computed, then row r-1 is finished: its 3 x 3 dS stencil is then in
//    registers (three rows per lane, the side columns by warp shuffles).
//  * Free flight reads the populations arriving at row r straight from the
//    source field: planes {0,1,3} of row r, {2,5,6} of row r-1, {4,7,8} of
//    row r+1, so every stored population is read from DRAM once (strips
//    overlap by two columns; an item's pull also reads three planes of the
//    rows just outside it).  Each plane's row window
//    arrives by 16-byte asynchronous copies (cp.async) in a per-warp ring of
//    shared-memory rows one row ahead of the arithmetic; the lanes read their
//    columns shifted by -cx.
//  * The post-collision deviations are stored at once; a site whose phi
//    (decided one row later) is below 1 reloads its row, recomputes the
//    collision exactly and overwrites its populations with the limited ones.
//  * Arithmetic is FP32 on the deviations g = f - rho_ref W in nonequilibrium
//    form, stored as FP32, BF16 or FP16; no FP64 on the per-site path.  A site
//    whose FP32 dS is near or above the Ehrenfests' threshold is recorded, and
//    its warp evaluates the FP64 key from the pre-step populations after the
//    item.  Sums are kept per thread in FP32 (mass as rho - rho_ref); at the
//    end of a work item (and every 128 rows) the warp adds them up in a fixed
//    order and folds the totals exactly into 128-bit fixed point, so the
//    step's statistics do not depend on which warp ran which item.
//  * Load balance: warps of one SM progress at different rates (the warp
//    scheduler favours older warps), so a static split leaves most warps idle
//    at the end of the launch.  The launch is one wave of resident warps; each
//    warp runs its first item, then takes further (short) items from a
//    counter in device memory until none are left.
#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "keys.cuh"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int kWarps = 4;  // independent work items per block
constexpr int kThreads = 32 * kWarps;
constexpr int kBlocksPerSM = 5;         // resident blocks per SM
constexpr int kBlocksPerSMBatched = 4;  // batched launches (the arguments in shared memory take registers)
constexpr int kRing = 2;         // FP32: rows in each warp's shared-memory load ring
constexpr int kWin = 72;         // FP32: columns of each plane copied per row (16-byte aligned window)
constexpr int kWin16 = 80;       // 16-bit storage: the same window, 8-column aligned
constexpr int kCarveout = -1;    // preferred shared-memory carveout in percent (-1: the driver's choice)
constexpr int kStripCols = 62;   // finished columns per strip (64 computed)
constexpr int kMinSegRows = 4;   // shortest row segment (an item costs a ring prologue and a few atomics)
constexpr int kFoldRows = 128;   // FP32 partial sums are folded into fixed point every kFoldRows rows
constexpr int kItemsPerWarp = 10;  // dynamic work: about this many items per resident warp
constexpr int kLaneKeys = 3;     // candidates of an item from which each lane keys its own
constexpr int kCandList = 32;    // candidates a warp keys itself per item (the tail keys the rest)
constexpr unsigned kFull = 0xffffffffu;

struct RowState {
    float2 ds, pp, pe;  // dS(f'), phi of the positivity rule, phi of the ensemble-dependent limiters
    bool bad_a, bad_b, cand_a, cand_b;
    float2 so;          // entropic f*, no median: dS of the limited state (applied at once)
};

// What the ensemble-dependent limiters need of their pass (read once per
// block from the reduction that ran before the step): E(dS) > 0, alpha and k
// of the smooth limiter, and the threshold filters' dS_t in FP64 with its FP32
// value rounded down (for a float dS, dS > tf exactly when (double) dS > t).
struct EnsParams {
    unsigned lim;  // the pass's ensemble bits
    bool e_pos, k_half;
    float alpha, k;
    double thr_t, ent_t;
    float thr_f, ent_f;    // dS_t rounded down: the decision, exact
    float thr_n, ent_n;    // dS_t rounded to nearest: the homothety's value
};

// phi of the ensemble-dependent limiters at a site with dS(f') = ds (not
// flagged), the same operations as the tiled kernel's: Eq. smooth1 with the
// ensemble's alpha, Eq. EntThresh's dS_t and the threshold dS_t = max(c E,
// delta) with the homothety of Eq. entrHom: which sites it limits is decided
// exactly (against dS_t rounded down), its value sqrt(dS_t / dS) in FP32.
__device__ __forceinline__ float ens_phi(const EnsParams &e, float ds)
{
    float pe = 1.f;
    if ((e.lim & 8u) && e.e_pos && ds > 0.f) {
        const float pk = e.k_half ? sqrtf(ds) : powf(ds, e.k);
        pe = __fdiv_rn(1.f, __fmaf_rn(e.alpha, pk, 1.f));
    }
    if ((e.lim & 32u) && ds > e.ent_f) pe = fminf(pe, __fsqrt_rn(__fdiv_rn(e.ent_n, ds)));
    if ((e.lim & 16u) && ds > e.thr_f) pe = fminf(pe, __fsqrt_rn(__fdiv_rn(e.thr_n, ds)));
    return pe;
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

// Asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst_smem)),
                 "l"(src)
                 : "memory");
}
// cp.async group bookkeeping (per thread).
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Neighbours of the two columns a lane carries (a = strip column l, b = l + 32):
// left of a is a of lane l-1, right of a is a of lane l+1 (b of lane 0 for
// lane 31), left of b is b of lane l-1 (a of lane 31 for lane 0), right of b
// is b of lane l+1.  The strip's outer columns get values they never use.
struct Sides {
    float al, ar, bl, br;
};
__device__ __forceinline__ Sides sides(float a, float b, int lane)
{
    Sides s;
    s.al = __shfl_up_sync(kFull, a, 1);
    s.ar = __shfl_sync(kFull, lane == 0 ? b : a, (lane + 1) & 31);
    s.bl = __shfl_sync(kFull, lane == 31 ? a : b, (lane - 1) & 31);
    s.br = __shfl_down_sync(kFull, b, 1);
    return s;
}

// MED / POS: the median / positivity code is compiled in (each still follows
// the instance's limiter bits).  BATCHED: work item i of the launch is item
// map[i].y of instance map[i].x of `table`, A0.items the launch's item count
// and A0.p.work its item counter; a warp keeps its current instance's
// arguments in shared memory and adds its sums into that instance's
// accumulator rows whenever it moves to another instance.  Otherwise the
// single instance A0.
// S: storage type of the deviations (float, __nv_bfloat16 or __half).
template <typename S, bool MED, bool POS, bool BATCHED, bool ENS = false, bool ENT = false, bool EP = false>
__global__ void __launch_bounds__(kThreads, ENT ? 3 : (BATCHED ? kBlocksPerSMBatched : kBlocksPerSM))
    k_fused(const FusedArgs A0, const FusedArgs *__restrict__ table, const int2 *__restrict__ map)
{
    using O = F2;
    // Ensemble-dependent passes without the median filter apply their
    // site-local limiters as the row is stored (a variant of its own: the
    // code costs registers the median variants cannot spare)
    constexpr bool kFastPhi = !MED && ENS;
    // Launched as a programmatic dependent of the previous kernel: wait for it
    // to finish before any memory access, then let the next kernel (the tail)
    // be scheduled early.  Both are no-ops in an ordinary launch.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // Rows stream through a per-warp ring of shared-memory rows filled by
    // 16-byte asynchronous copies (kRing - 1 rows in flight, no registers
    // held): windows of 72 FP32 or 80 16-bit columns
    constexpr int kChunk = 16 / (int)sizeof(S);          // elements per 16-byte copy
    constexpr int kWinS = sizeof(S) == 4 ? kWin : kWin16;  // window columns (a multiple of kChunk)
    __shared__ __align__(16) S ring[kWarps][kRing][9][kWinS];
    __shared__ unsigned long long sfx[kWarps][kFxWords];
    __shared__ int cand_list[kWarps][kCandList];  // candidate slots of the warp's current item
    __shared__ float2 cand_ds[kWarps][2][32];      // FP32 dS of the lanes' candidates, rows of each parity
    __shared__ __align__(16) FusedArgs sA[BATCHED ? kWarps : 1];
    const int bid = (int)blockIdx.x;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const FusedArgs &A = BATCHED ? sA[warp] : A0;
    const StepParams &p = A.p;
    // ensemble-dependent limiters: this pass's E(dS), alpha and dS_t
    EnsParams ens{};
    if constexpr (ENS) {
        ens.lim = p.limiters & kLimEnsemble;
        if (ens.lim) {
            const double E = p.ens[0];
            ens.e_pos = E > 0.0;
            ens.k_half = p.smooth_k == 0.5;
            ens.alpha = (float)p.ens[1];
            ens.k = (float)p.smooth_k;
            double t = p.threshold_c * E;
            if (t < p.threshold_delta) t = p.threshold_delta;
            ens.thr_t = t;
            ens.thr_f = __double2float_rd(t);
            ens.thr_n = (float)t;
            ens.ent_t = (ens.lim & 32u) ? p.ent->t : 0.0;
            ens.ent_f = (ens.lim & 32u) ? __double2float_rd(ens.ent_t) : 0.f;
            ens.ent_n = (float)ens.ent_t;
        }
    }

    float s_mass = 0.f, s_ds = 0.f, s_in = 0.f, s_lim = 0.f;
    int n_pos = 0, n_med = 0, n_bad = 0, n_sites = 0, rows_acc = 0;
    // fixed-point totals: lane 0 mass, lane 8 dS, lane 16 dS_in, lane 24 dS_lim
    unsigned __int128 fx_acc = 0;
    bool fx_bad = false;
    // Adds the lanes' FP32 sums in a fixed order (a butterfly in which each
    // level halves the sums a lane carries) and folds the four totals into
    // fixed point; every lane takes part.
    auto flush = [&]() {
        const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
        float x0 = hi16 ? s_in : s_mass, x1 = hi16 ? s_lim : s_ds;
        const float y0 = hi16 ? s_mass : s_in, y1 = hi16 ? s_ds : s_lim;
        x0 += __shfl_xor_sync(kFull, y0, 16);
        x1 += __shfl_xor_sync(kFull, y1, 16);
        float z = hi8 ? x1 : x0;
        z += __shfl_xor_sync(kFull, hi8 ? x0 : x1, 8);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) z += __shfl_xor_sync(kFull, z, o);
        if ((lane & 7) == 0) fx_add(fx_acc, z, fx_bad);
        s_mass = s_ds = s_in = s_lim = 0.f;
    };

    int *list = cand_list[warp];
    int n_list = 0;  // candidates recorded in the current item (the same for the whole warp)

    // BATCHED: adds the warp's fixed-point totals and counts into accumulator
    // row (warp % kFxRows) of the instance it worked on, and clears them
    auto commit = [&]() {
        const int tot_sites = __reduce_add_sync(kFull, n_sites), tot_pos = __reduce_add_sync(kFull, n_pos);
        const int tot_med = __reduce_add_sync(kFull, n_med), tot_bad = __reduce_add_sync(kFull, n_bad);
        const unsigned bad_lanes = __ballot_sync(kFull, fx_bad);
        unsigned long long *row = p.fx_rows + (long long)((bid * kWarps + warp) % kFxRows) * kFxWords;
        if ((lane & 7) == 0) {
            const int stat = lane >> 3;  // P_MASS .. P_DS_LIM
            const unsigned long long lo = (unsigned long long)fx_acc, hi = (unsigned long long)(fx_acc >> 64);
            const unsigned long long old = atomicAdd(row + FX_SUM + 2 * stat, lo);
            atomicAdd(row + FX_SUM + 2 * stat + 1, hi + (old + lo < old ? 1ull : 0ull));
        }
        if (lane == 0) {
            atomicAdd(row + FX_SITES, (unsigned long long)tot_sites);
            atomicAdd(row + FX_NPOS, (unsigned long long)tot_pos);
            atomicAdd(row + FX_NMED, (unsigned long long)tot_med);
            atomicAdd(row + FX_NBAD, (unsigned long long)tot_bad);
            const unsigned long long bits = (bad_lanes & 1u) | ((bad_lanes >> 7) & 2u) | ((bad_lanes >> 14) & 4u) |
                                            ((bad_lanes >> 21) & 8u);
            if (bits) atomicOr(row + FX_BAD, bits);
            if (tot_bad) atomicOr(p.status, kStatNonfinite);  // a site was nonfinite
        }
        fx_acc = 0;
        fx_bad = false;
        n_sites = n_pos = n_med = n_bad = 0;
    };
    int cur = -1;  // BATCHED: the instance whose arguments sA[warp] holds

    int item = bid * kWarps + warp;
    while (item < A0.items) {
        int it = item;  // the item within its instance
        if constexpr (BATCHED) {
            const int2 m = map[item];
            if (m.x != cur) {
                if (cur >= 0) commit();
                __syncwarp();
                const unsigned *from = reinterpret_cast<const unsigned *>(table + m.x);
                unsigned *to = reinterpret_cast<unsigned *>(&sA[warp]);
                for (int i = lane; i < (int)(sizeof(FusedArgs) / 4); i += 32) to[i] = from[i];
                __syncwarp();
                cur = m.x;
            }
            it = m.y;
        }
        const S *__restrict__ src = (const S *)A.src;
        S *__restrict__ dst = (S *)A.dst;
        const int nx = p.nx, ny = p.ny, pitch = p.pitch;
        const int plane = (int)p.plane;  // 9 * plane < 2^31 is checked at launch
        const int strip = it % A.strips, seg = it / A.strips;
        const int xa = kStripCols * strip - 1 + lane, xb = xa + 32;  // the lane's two columns
        const int ys = seg * A.seg_rows, ye = min(ys + A.seg_rows, ny);
        // The walk computes its own rows [ys, ye) only.  The median of its first
        // and last row also needs dS of the rows just outside (ys - 1, ye); in
        // the rare rows whose median is formed at all, those are evaluated on
        // demand (halo_ds), so items pay no halo rows in the common case.
        const int r0 = ys;
        const int rc = ye - 1;  // last row whose dS this warp computes
        // every lane reads its columns x - 1 .. x + 1, at most 63 past the
        // lattice's last column: inside the zero row padding (kTail)
        const bool in_a = xa >= 0 && xa < nx, in_b = xb < nx;
        const bool own_a = in_a && lane >= 1, own_b = in_b && lane <= 30;
        const bool wall_a = xa == 0 || xa == nx - 1, wall_b = xb == nx - 1;
        const bool lim_ehr = (p.limiters & 2u) != 0;
        const bool med_on = MED && (p.limiters & 4u) != 0, pos_on = POS && (p.limiters & 1u) != 0;
        const float a = A.a, a2 = A.a * A.a, b2 = A.b2, rho_ref = p.rho_ref;
        // rho_ref W_k takes three values (rest, axis, diagonal), kept in registers
        const float2 rw0 = O::s(p.rwf[0]), rw1 = O::s(p.rwf[1]), rw5 = O::s(p.rwf[5]);
        auto rwk = [&](int k) { return k == 0 ? rw0 : (k <= 4 ? rw1 : rw5); };
        // element offsets, from (plane 0, row q, column x), of the population of
        // plane k arriving at (x, q): source row q - cy_k, column x - cx_k
        const int o1 = plane - 1, o3 = 3 * plane + 1;
        const int o2 = 2 * plane - pitch, o5 = 5 * plane - pitch - 1, o6 = 6 * plane - pitch + 1;
        const int o4 = 4 * plane + pitch, o7 = 7 * plane + pitch + 1, o8 = 8 * plane + pitch - 1;

        // Loads of the populations arriving at row q (rows outside the lattice
        // are not read; their links are bounce-back links, set by edge_row).
        auto load_row = [&](int q, float2 g[9]) {
            const S *ba = src + (long long)q * pitch + kLead + xa;
            auto ld = [&](int off) { return make_float2(s2f(ba[off]), s2f(ba[off + 32])); };
            g[0] = ld(0);
            g[1] = ld(o1);
            g[3] = ld(o3);
            if (q >= 1) {  // the same for the whole warp
                g[2] = ld(o2);
                g[5] = ld(o5);
                g[6] = ld(o6);
            } else {
                g[2] = g[5] = g[6] = make_float2(0.f, 0.f);
            }
            if (q + 1 < ny) {
                g[4] = ld(o4);
                g[7] = ld(o7);
                g[8] = ld(o8);
            } else {
                g[4] = g[7] = g[8] = make_float2(0.f, 0.f);
            }
        };
        // Halfway bounce-back at wall sites: a link from outside returns the
        // site's own population of the opposite direction, plus the lid term.
        auto edge_col = [&](int q, int x, const S *b, float2 g[9], bool second) {
#pragma unroll
            for (int k = 1; k < 9; ++k) {
                const int sx = x - Lat<9>::cx(k), sy = q - Lat<9>::cy(k);
                if (sx >= 0 && sx < nx && sy >= 0 && sy < ny) continue;
                float v = s2f(b[Lat<9>::opp(k) * plane]);
                if (sy > ny - 1) {
                    v += k == 4 ? A.lid4 : (k == 7 ? A.lid7 : A.lid8);
                    v += k == 4 ? A.lo4 : (k == 7 ? A.lo7 : A.lo8);
                }
                if (second)
                    g[k].y = v;
                else
                    g[k].x = v;
            }
        };
        const bool wall_strip = __any_sync(kFull, (in_a && wall_a) || (in_b && wall_b));  // the same for the whole item
        auto edge_row = [&](int q, float2 g[9]) {
            const bool yedge = q == 0 || q == ny - 1;
            const bool ea = in_a && (wall_a || yedge), eb = in_b && (wall_b || yedge);
            if (wall_strip || yedge) {  // the same for the whole warp
                const S *ba = src + (long long)q * pitch + kLead + xa;
                if (ea) edge_col(q, xa, ba, g, false);
                if (eb) edge_col(q, xb, ba + 32, g, true);
            }
        };
        // g*, and the corrected nonequilibrium part of the pulled row q
        auto collide = [&](const float2 g[9], float2 &drho, float2 &rho, float2 &ux, float2 &uy, float2 gs[9],
                           float2 n[9]) {
            moments9_x<O>(g, rho_ref, drho, rho, ux, uy);
            if constexpr (ENT) {
                // entropic f* (Eq. maxwellian); a site with |u_j| >= 1 has none
                // (flagged in row_ds) and takes g* = 0, as in the tiled kernel
                feq_ent9_x<O>(drho, rho, ux, uy, gs);
                const bool na = !(fabsf(ux.x) < 1.f) || !(fabsf(uy.x) < 1.f);
                const bool nb = !(fabsf(ux.y) < 1.f) || !(fabsf(uy.y) < 1.f);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    if (na) gs[k].x = 0.f;
                    if (nb) gs[k].y = 0.f;
                }
            } else {
                feq9_x<O>(drho, rho, ux, uy, gs);
            }
            neq9_x<O>(g, gs, n);
        };

        // Row q from its loaded populations: collision, dS; stores g' of the
        // warp's own sites.  Rare per-site paths sit behind warp votes.
        // dS(f') of a computed row (infinite at sites that cannot be limited:
        // rho <= 0, some f*_k <= 0, nonfinite); din = dS(f_in)
        auto row_ds = [&](const float2 gs[9], const float2 n[9], float2 rho, float2 ux, float2 uy, float2 &din,
                          bool &bad_a, bool &bad_b) -> float2 {
            if constexpr (ENT) {
                // the exact dS of Eq. DelS without cancellation (lattice.cuh): of
                // f' from f' - f* = -(2 beta - 1) n, of f_in from n; +inf (no flag)
                // for a state with a negative population
                float2 fsa[9], d[9];
                float fa = 3.4e38f, fb = 3.4e38f;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    fsa[k] = O::add(rwk(k), gs[k]);
                    d[k] = O::mul(O::s(-a), n[k]);
                    fa = fminf(fa, fsa[k].x);
                    fb = fminf(fb, fsa[k].y);
                }
                bad_a = !(rho.x > 0.f) || !(fabsf(ux.x) < 1.f) || !(fabsf(uy.x) < 1.f) || !(fa > 0.f);
                bad_b = !(rho.y > 0.f) || !(fabsf(ux.y) < 1.f) || !(fabsf(uy.y) < 1.f) || !(fb > 0.f);
                float2 ds = rel_entropy9_x(d, fsa);
                din = rel_entropy9_x(n, fsa);
                bad_a = bad_a || isnan(ds.x) || isnan(din.x);
                bad_b = bad_b || isnan(ds.y) || isnan(din.y);
                ds.x = bad_a ? __int_as_float(0x7f800000) : ds.x;
                ds.y = bad_b ? __int_as_float(0x7f800000) : ds.y;
                return ds;
            }
            din = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 9; ++k)
                din = O::fma(O::mul(n[k], n[k]), O::rcp_fast(O::add(rwk(k), gs[k])), din);  // / absolute f*
            float2 ds = O::mul(O::s(a2), din);  // dS(f') = (2 beta - 1)^2 dS(f_in) for the same f*
            // f*_k >= rho W_k (1/2 - 3 u^2 / 2) > 0 whenever u^2 < 1/3; only fast
            // flows need the explicit test of every f*_k
            const float2 usq = O::fma(ux, ux, O::mul(uy, uy));
            bad_a = !(rho.x > 0.f) || !isfinite(ds.x);
            bad_b = !(rho.y > 0.f) || !isfinite(ds.y);
            if (__any_sync(kFull, !(usq.x < 0.3f) || !(usq.y < 0.3f))) {
                float fa = 3.4e38f, fb = 3.4e38f;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    fa = fminf(fa, p.rwf[k] + gs[k].x);
                    fb = fminf(fb, p.rwf[k] + gs[k].y);
                }
                bad_a = bad_a || !(fa > 0.f);
                bad_b = bad_b || !(fb > 0.f);
            }
            ds.x = bad_a ? __int_as_float(0x7f800000) : ds.x;
            ds.y = bad_b ? __int_as_float(0x7f800000) : ds.y;
            return ds;
        };
        // dS(f') of row q, outside the walk, from global loads (the whole warp)
        auto halo_ds = [&](int q) -> float2 {
            float2 g[9];
            load_row(q, g);
            edge_row(q, g);
            float2 drho, rho, ux, uy, gs[9], n[9], din;
            collide(g, drho, rho, ux, uy, gs, n);
            bool bad_a, bad_b;
            return row_ds(gs, n, rho, ux, uy, din, bad_a, bad_b);
        };

        auto compute_row = [&](int q, float2 g[9]) -> RowState {
            RowState st{make_float2(0.f, 0.f), make_float2(1.f, 1.f), make_float2(1.f, 1.f), false, false, false,
                        false};
            edge_row(q, g);
            float2 drho, rho, ux, uy, gs[9], n[9], din;
            collide(g, drho, rho, ux, uy, gs, n);
            bool bad_a, bad_b;
            float2 ds = row_ds(gs, n, rho, ux, uy, din, bad_a, bad_b);
            if constexpr (EP) {
                // E(dS) pass: the sum and count of dS(f') over the owned sites that
                // are not flagged and have a finite dS, and the Eq. EntThresh field
                const bool rown = q >= ys && q < ye;
                const bool oa = own_a && rown, ob = own_b && rown;
                const bool ga = oa && !bad_a && isfinite(ds.x), gb = ob && !bad_b && isfinite(ds.y);
                s_ds += (ga ? ds.x : 0.f) + (gb ? ds.y : 0.f);
                n_sites += (int)ga + (int)gb;
                if (p.ent_field) {
                    float *fld = (float *)p.ent_field + (long long)q * nx;
                    if (oa) fld[xa] = (ga && ds.x > 0.f) ? ds.x : 0.f;
                    if (ob) fld[xb] = (gb && ds.y > 0.f) ? ds.y : 0.f;
                }
                return st;
            }
            const bool rown = q >= ys && q < ye;
            const bool oa = own_a && rown, ob = own_b && rown;
            if constexpr (kFastPhi) {
                // g stays the arriving g; g' = g - 2 beta n is formed where it is used
                float fpmin_a = 3.4e38f, fpmin_b = 3.4e38f;
                if (pos_on) {
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const float2 gp = O::fma(O::s(-b2), n[k], g[k]);
                        fpmin_a = fminf(fpmin_a, rwk(k).x + gp.x);
                        fpmin_b = fminf(fpmin_b, rwk(k).y + gp.y);
                    }
                }
                if (pos_on && __any_sync(kFull, (!bad_a && fpmin_a < 0.f) || (!bad_b && fpmin_b < 0.f))) {
                    // positivity rule (Sec. 3.1)
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const float2 gp = O::fma(O::s(-b2), n[k], g[k]);
                        const float fpa = p.rwf[k] + gp.x, fsa = p.rwf[k] + gs[k].x;
                        if (!bad_a && fpa < 0.f) st.pp.x = fminf(st.pp.x, fsa / (fsa - fpa));
                        const float fpb = p.rwf[k] + gp.y, fsb = p.rwf[k] + gs[k].y;
                        if (!bad_b && fpb < 0.f) st.pp.y = fminf(st.pp.y, fsb / (fsb - fpb));
                    }
                }
                if (ens.lim) {
                    if (!bad_a) st.pe.x = ens_phi(ens, ds.x);
                    if (!bad_b) st.pe.y = ens_phi(ens, ds.y);
                }
                // no median in this pass: every limiter is site-local, so phi is
                // final here, and the row is stored once: g - (1 + phi (2 beta - 1)) n
                // where phi < 1 (the operations of the deferred update of
                // finalise_row), g - 2 beta n elsewhere
                const float phi_a = oa ? fminf(fminf(st.pp.x, 1.f), st.pe.x) : 1.f;
                const float phi_b = ob ? fminf(fminf(st.pp.y, 1.f), st.pe.y) : 1.f;
                const float2 cs = make_float2(phi_a < 1.f ? -limit_weight(phi_a, a, true) : -b2,
                                              phi_b < 1.f ? -limit_weight(phi_b, a, true) : -b2);
                if constexpr (ENT) {
                    if (__any_sync(kFull, phi_a < 1.f || phi_b < 1.f)) {
                        float2 fsa[9], d[9];
                        const float2 m = make_float2(__fmul_rn(-phi_a, a), __fmul_rn(-phi_b, a));
#pragma unroll
                        for (int k = 0; k < 9; ++k) {
                            fsa[k] = O::add(rwk(k), gs[k]);
                            d[k] = O::mul(m, n[k]);
                        }
                        st.so = rel_entropy9_x(d, fsa);
                    }
                }
                S *out = dst + (long long)q * pitch + kLead + xa;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float2 v = O::fma(cs, n[k], g[k]);
                    if (oa) out[k * plane] = f2s<S>(v.x);
                    if (ob) out[k * plane + 32] = f2s<S>(v.y);
                }
            } else {
                float fpmin_a = 3.4e38f, fpmin_b = 3.4e38f;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    g[k] = O::fma(O::s(-b2), n[k], g[k]);  // g' = g - 2 beta n
                    if (pos_on) {
                        fpmin_a = fminf(fpmin_a, rwk(k).x + g[k].x);
                        fpmin_b = fminf(fpmin_b, rwk(k).y + g[k].y);
                    }
                }
                if (pos_on && __any_sync(kFull, (!bad_a && fpmin_a < 0.f) || (!bad_b && fpmin_b < 0.f))) {
                    // positivity rule (Sec. 3.1)
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const float fpa = p.rwf[k] + g[k].x, fsa = p.rwf[k] + gs[k].x;
                        if (!bad_a && fpa < 0.f) st.pp.x = fminf(st.pp.x, fsa / (fsa - fpa));
                        const float fpb = p.rwf[k] + g[k].y, fsb = p.rwf[k] + gs[k].y;
                        if (!bad_b && fpb < 0.f) st.pp.y = fminf(st.pp.y, fsb / (fsb - fpb));
                    }
                }
                if constexpr (ENS) {
                    // site-local, like the positivity rule: applied with the median's
                    // phi one row later (the row is then recomputed from its sources)
                    if (ens.lim) {
                        if (!bad_a) st.pe.x = ens_phi(ens, ds.x);
                        if (!bad_b) st.pe.y = ens_phi(ens, ds.y);
                    }
                }
                S *out = dst + (long long)q * pitch + kLead + xa;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    if (oa) out[k * plane] = f2s<S>(g[k].x);
                    if (ob) out[k * plane + 32] = f2s<S>(g[k].y);
                }
            }
            const bool ga = oa && !bad_a, gb = ob && !bad_b;
            s_mass += (oa ? drho.x : 0.f) + (ob ? drho.y : 0.f);
            if constexpr (ENT) {
                // entropy differences where both entropies are finite
                const bool fa = ga && isfinite(ds.x), fb = gb && isfinite(ds.y);
                s_ds += (fa ? ds.x : 0.f) + (fb ? ds.y : 0.f);
                s_in += ((fa && isfinite(din.x)) ? __fsub_rn(din.x, ds.x) : 0.f) +
                        ((fb && isfinite(din.y)) ? __fsub_rn(din.y, ds.y) : 0.f);
            } else {
                s_ds += (ga ? ds.x : 0.f) + (gb ? ds.y : 0.f);
                s_in += (ga ? din.x : 0.f) + (gb ? din.y : 0.f);
            }
            n_sites += (int)oa + (int)ob;
            n_bad += (int)(oa && bad_a) + (int)(ob && bad_b);
            if (pos_on) n_pos += (int)(oa && st.pp.x < 1.f) + (int)(ob && st.pp.y < 1.f);
            // Ehrenfests' candidates (FP32 dS near or above the threshold); the
            // FP64 key decides
            st.cand_a = lim_ehr && !bad_a && oa && ds.x > A.thr_e;
            st.cand_b = lim_ehr && !bad_b && ob && ds.y > A.thr_e;
            // their FP32 dS for the record one row later (kept in shared memory,
            // not in registers across the row: row q is recorded after row q + 1
            // is computed, so rows of each parity have their own slot)
            if (st.cand_a || st.cand_b) cand_ds[warp][q & 1][lane] = ds;
            st.bad_a = bad_a;
            st.bad_b = bad_b;
            st.ds = ds;
            return st;
        };

        // Ehrenfests' candidates of row y (flags ca / cb of the lanes' two
        // columns) are recorded at once without their key (NaN), with their
        // FP32 dS; the warp keeps their slots in its list and keys them when
        // the item is done, away from the row loop's registers
        auto record = [&](int y, bool ca, bool cb, float phi_a, float phi_b) {
            const float2 ds = cand_ds[warp][y & 1][lane];
            auto put = [&](bool c, int x, float phi, float ds32) {
                int slot = -1;
                if (c) {
                    slot = atomicAdd(p.cand_count, 1);
                    if (slot < p.cand_cap) {
                        Cand cd;
                        cd.key = __longlong_as_double(0x7ff8000000000000LL);
                        cd.phi = (double)phi;
                        cd.site = y * nx + x;
                        cd.ds32 = ds32;
                        p.cand[slot] = cd;
                    } else {
                        atomicOr(p.status, kStatCandOverflow);
                        slot = -1;
                    }
                }
                const unsigned m = __ballot_sync(kFull, slot >= 0);
                const int at = n_list + __popc(m & ((1u << lane) - 1u));
                if (slot >= 0 && at < kCandList) list[at] = slot;
                n_list += __popc(m);
            };
            put(ca, xa, phi_a, ds.x);
            put(cb, xb, phi_b, ds.y);
        };

        // Row y: median of dS (rows y-1, y, y+1 in dm, d0, dp), phi = min(phi_pos,
        // phi_med), limited update where phi < 1, candidate record, sums.
        auto finalise_row = [&](int y, const RowState &st, float2 dm, float2 d0, float2 dp) {
            if constexpr (EP) return;  // the E(dS) pass stores nothing
            const bool rown = y >= ys && y < ye;
            const bool act_a = own_a && rown, act_b = own_b && rown;
            float pm_a = 1.f, pm_b = 1.f;
            // phi_med < 1 needs dS above delta (and above the median): the
            // median is formed only when some site of the warp's row passes the
            // first, cheap test (rare), and the division and square root only
            // where both hold
            const bool xa_on = act_a && !st.bad_a && st.ds.x > A.delta_m;
            const bool xb_on = act_b && !st.bad_b && st.ds.y > A.delta_m;
            if (med_on && __any_sync(kFull, xa_on || xb_on)) {
                // the rows just outside the walk, when the stencil reaches them
                // (one evaluation site in the code for both)
#pragma unroll 1
                for (int side = 0; side < 2; ++side) {
                    const int hq = side == 0 ? (y == ys && ys > 0 ? ys - 1 : -1) : (y == ye - 1 && ye < ny ? ye : -1);
                    if (hq >= 0) {  // the same for the whole warp
                        const float2 v = halo_ds(hq);
                        if (side == 0)
                            dm = v;
                        else
                            dp = v;
                    }
                }
                // 3 x 3 median from sorted columns: the median of (largest column
                // minimum, median of the column medians, smallest column maximum);
                // wall rows and columns take the near-wall stencils
                float loa, mida, hia, lob, midb, hib;
                sort3(dm.x, d0.x, dp.x, loa, mida, hia);
                sort3(dm.y, d0.y, dp.y, lob, midb, hib);
                const Sides lo = sides(loa, lob, lane), mid = sides(mida, midb, lane), hi = sides(hia, hib, lane);
                float med_a = med3(fmaxf(fmaxf(lo.al, loa), lo.ar), med3(mid.al, mida, mid.ar),
                                   fminf(fminf(hi.al, hia), hi.ar));
                float med_b = med3(fmaxf(fmaxf(lo.bl, lob), lo.br), med3(mid.bl, midb, mid.br),
                                   fminf(fminf(hi.bl, hib), hi.br));
                const bool ywall = y == 0 || y == ny - 1;  // the same for the whole warp
                if (ywall) {
                    const Sides d = sides(d0.x, d0.y, lane);
                    const float vin_a = y == 0 ? dp.x : dm.x, vin_b = y == 0 ? dp.y : dm.y;
                    med_a = wall_a ? med3(d0.x, xa == 0 ? d.ar : d.al, vin_a) : med3(d.al, d0.x, d.ar);
                    med_b = wall_b ? med3(d0.y, d.bl, vin_b) : med3(d.bl, d0.y, d.br);
                } else {
                    if (wall_a) med_a = mida;
                    if (wall_b) med_b = midb;
                }
                if (xa_on && st.ds.x > med_a) pm_a = phi_median<float>(st.ds.x, med_a, A.delta_m, p.median_mode);
                if (xb_on && st.ds.y > med_b) pm_b = phi_median<float>(st.ds.y, med_b, A.delta_m, p.median_mode);
            }
            const float phi_a = act_a ? fminf(fminf(st.pp.x, pm_a), st.pe.x) : 1.f;
            const float phi_b = act_b ? fminf(fminf(st.pp.y, pm_b), st.pe.y) : 1.f;
            if (kFastPhi && !med_on) {
                // the update was stored by compute_row; its entropy, as below
                if constexpr (ENT) {
                    if (phi_a < 1.f && isfinite(st.ds.x) && isfinite(st.so.x)) s_lim += __fsub_rn(st.ds.x, st.so.x);
                    if (phi_b < 1.f && isfinite(st.ds.y) && isfinite(st.so.y)) s_lim += __fsub_rn(st.ds.y, st.so.y);
                } else {
                    if (phi_a < 1.f) s_lim = fmaf(1.f - phi_a * phi_a, st.ds.x, s_lim);
                    if (phi_b < 1.f) s_lim = fmaf(1.f - phi_b * phi_b, st.ds.y, s_lim);
                }
            } else if (__any_sync(kFull, phi_a < 1.f || phi_b < 1.f)) {
                // the limited update g - (1 + phi (2 beta - 1)) n (Eq. LimGenF in
                // nonequilibrium form), with g and n recomputed exactly as the
                // collision computed them (every lane takes part: edge_row votes)
                float2 g[9];
                load_row(y, g);
                edge_row(y, g);
                if (phi_a < 1.f || phi_b < 1.f) {
                    float2 drho, rho, ux, uy, gs[9], n[9];
                    collide(g, drho, rho, ux, uy, gs, n);
                    const float2 mc = make_float2(-limit_weight(phi_a, a, true), -limit_weight(phi_b, a, true));
                    S *out = dst + (long long)y * pitch + kLead + xa;
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const float2 v = O::fma(mc, n[k], g[k]);
                        if (phi_a < 1.f) out[k * plane] = f2s<S>(v.x);
                        if (phi_b < 1.f) out[k * plane + 32] = f2s<S>(v.y);
                    }
                    if constexpr (ENT) {
                        // dS(f') - dS(f_out) at the same f*, f_out - f* = phi (f' - f*)
                        float2 fsa[9], d[9];
                        const float2 m = make_float2(__fmul_rn(-phi_a, a), __fmul_rn(-phi_b, a));
#pragma unroll
                        for (int k = 0; k < 9; ++k) {
                            fsa[k] = O::add(rwk(k), gs[k]);
                            d[k] = O::mul(m, n[k]);
                        }
                        const float2 so = rel_entropy9_x(d, fsa);
                        if (phi_a < 1.f && isfinite(st.ds.x) && isfinite(so.x)) s_lim += __fsub_rn(st.ds.x, so.x);
                        if (phi_b < 1.f && isfinite(st.ds.y) && isfinite(so.y)) s_lim += __fsub_rn(st.ds.y, so.y);
                    } else {
                        if (phi_a < 1.f) s_lim = fmaf(1.f - phi_a * phi_a, st.ds.x, s_lim);
                        if (phi_b < 1.f) s_lim = fmaf(1.f - phi_b * phi_b, st.ds.y, s_lim);
                    }
                }
            }
            n_med += (int)(act_a && pm_a < 1.f) + (int)(act_b && pm_b < 1.f);
            if (__any_sync(kFull, st.cand_a || st.cand_b)) record(y, st.cand_a, st.cand_b, phi_a, phi_b);
            if (rown && ++rows_acc == kFoldRows) {  // the same for the whole warp
                flush();
                rows_acc = 0;
            }
        };

        {
            // Row q's populations arrive by 16-byte asynchronous copies of the
            // window of columns [cb, cb + kWinS) of every plane k, from source
            // row q - cy_k (one 16-byte chunk per copying lane); the lanes then
            // read their two columns shifted by -cx_k.  cb is 16-byte aligned
            // and at most the strip's first pulled column (lane 0's column - 1);
            // the window reaches past its last (lane 31's second column + 1).
            S(*my)[9][kWinS] = ring[warp];
            S *flat = &my[0][0][0];
            for (int i = lane; i < kRing * 9 * kWinS; i += 32) flat[i] = f2s<S>(0.f);
            const int xa0 = kStripCols * strip - 1;  // lane 0's column
            const int cb = (xa0 - 1) & ~(kChunk - 1);
            const int d0 = xa0 - cb + lane;  // window index of the lane's column a
            const bool copier = lane < kWinS / kChunk;
            const int p2 = 2 * plane - pitch, p5 = 5 * plane - pitch, p6 = 6 * plane - pitch;
            const int p4 = 4 * plane + pitch, p7 = 7 * plane + pitch, p8 = 8 * plane + pitch;
            int put = 0, get = 0;  // ring slots of the next row to copy and to read
            auto issue = [&](int q) {
                if (q <= rc) {
                    S(*sl)[kWinS] = my[put];
                    put = put + 1 == kRing ? 0 : put + 1;
                    if (copier) {
                        const S *ba = src + (long long)q * pitch + kLead + cb + kChunk * lane;
                        auto cp = [&](int k, int off) { cp_async16(&sl[k][kChunk * lane], ba + off); };
                        cp(0, 0);
                        cp(1, plane);
                        cp(3, 3 * plane);
                        if (q >= 1) {  // rows outside the lattice are skipped; edge_row sets those links
                            cp(2, p2);
                            cp(5, p5);
                            cp(6, p6);
                        }
                        if (q + 1 < ny) {
                            cp(4, p4);
                            cp(7, p7);
                            cp(8, p8);
                        }
                    }
                }
                cp_async_commit();  // one group per row (empty past the last row)
            };
            // Iteration r computes row r and finishes row r-1.
            RowState prev{make_float2(0.f, 0.f), make_float2(1.f, 1.f), make_float2(1.f, 1.f), false, false, false,
                          false};
            float2 ds_m2 = make_float2(0.f, 0.f), ds_m1 = make_float2(0.f, 0.f);  // dS of rows r-2, r-1
            __syncwarp();
#pragma unroll
            for (int j = 0; j < kRing - 1; ++j) issue(r0 + j);
            for (int r = r0; r - 1 < ye; ++r) {
                RowState st{make_float2(0.f, 0.f), make_float2(1.f, 1.f), make_float2(1.f, 1.f), false, false,
                            false, false};
                if (r <= rc) {
                    __syncwarp();                // every lane is done with the slot row r-1 used
                    issue(r + kRing - 1);        // refills it
                    cp_async_wait<kRing - 1>();  // this thread's copies of row r have landed
                    __syncwarp();                // and so have the other lanes'
                    float2 g[9];
                    const S *sb = &my[get][0][0] + d0;
                    get = get + 1 == kRing ? 0 : get + 1;
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const int o = k * kWinS - Lat<9>::cx(k);
                        g[k] = make_float2(s2f(sb[o]), s2f(sb[o + 32]));
                    }
                    st = compute_row(r, g);
                }
                if (r - 1 >= ys) finalise_row(r - 1, prev, ds_m2, ds_m1, st.ds);
                ds_m2 = ds_m1;
                ds_m1 = st.ds;
                prev = st;
            }
            cp_async_wait<0>();
        }
        // FP64 keys dS(f') of the item's candidates, from the pre-step
        // populations with the FP64 path's operations and order (-1 when the
        // site is at or below the threshold or cannot be limited).  A few are
        // keyed one at a time by the whole warp (a lane per direction, the
        // shortest latency), more lane-parallel; past kCandList the tail
        // kernel keys the rest.  An item with more candidates than that on a
        // lattice with the grid tail keys none: the grid keys only those that
        // can matter (near the k-th largest or near delta).
        const bool dense_item = !BATCHED && n_list > kCandList && (long long)nx * ny >= kSelMinSites;
        if (n_list > 0 && !dense_item) {  // the same for the whole warp
            KeyGeom kg;
            kg.nx = nx;
            kg.ny = ny;
            kg.pitch = pitch;
            kg.boundary = p.boundary;
            kg.plane = p.plane;
            kg.a = p.a;
            kg.rw0 = p.rw[0];
            kg.rw1 = p.rw[1];
            kg.rw5 = p.rw[5];
            kg.lid4 = p.lid[4];
            kg.lid7 = p.lid[7];
            kg.lid8 = p.lid[8];
            kg.eq = p.eq;
            const int n = min(n_list, kCandList);
            __syncwarp();
            if (n >= kLaneKeys) {
                if (lane < n) {
                    const int slot = list[lane];
                    p.cand[slot].key = key_dS9_lane<S>(kg, src, p.cand[slot].site, p.delta_e);
                }
            } else {
                for (int i = 0; i < n; ++i) {
                    const int slot = list[i];
                    const double key = key_dS9_warp<S>(kg, src, p.cand[slot].site, p.delta_e);
                    if (lane == 0) p.cand[slot].key = key;
                }
            }
            __syncwarp();
        }
        n_list = 0;
        // the item's sums, then the next item
        flush();
        rows_acc = 0;
        int *work = BATCHED ? A0.p.work : p.work;
        if (work == nullptr) break;
        int next = 0;
        if (lane == 0) next = (int)gridDim.x * kWarps + atomicAdd(work, 1);
        item = __shfl_sync(kFull, next, 0);
    }
    if constexpr (BATCHED) {
        if (cur >= 0) commit();
        return;
    }

    // Block row of fixed-point totals and counts: integer sums, so the order
    // in which warps and blocks are added does not matter.
    const int tot_sites = __reduce_add_sync(kFull, n_sites), tot_pos = __reduce_add_sync(kFull, n_pos);
    const int tot_med = __reduce_add_sync(kFull, n_med), tot_bad = __reduce_add_sync(kFull, n_bad);
    const unsigned bad_lanes = __ballot_sync(kFull, fx_bad);
    if ((lane & 7) == 0) {
        const int stat = lane >> 3;  // P_MASS .. P_DS_LIM
        sfx[warp][FX_SUM + 2 * stat] = (unsigned long long)fx_acc;
        sfx[warp][FX_SUM + 2 * stat + 1] = (unsigned long long)(fx_acc >> 64);
    }
    if (lane == 0) {
        sfx[warp][FX_SITES] = (unsigned long long)tot_sites;
        sfx[warp][FX_NPOS] = (unsigned long long)tot_pos;
        sfx[warp][FX_NMED] = (unsigned long long)tot_med;
        sfx[warp][FX_NBAD] = (unsigned long long)tot_bad;
        sfx[warp][FX_BAD] = (bad_lanes & 1u) | ((bad_lanes >> 7) & 2u) | ((bad_lanes >> 14) & 4u) |
                            ((bad_lanes >> 21) & 8u);
    }
    __syncthreads();
    // added atomically to accumulator row bid % kFxRows of the instance (a
    // 128-bit sum as two 64-bit adds with the carry passed on); the tail
    // kernel reads the rows and clears them for the next step
    if (t < kFxWords) {
        unsigned long long *row = p.fx_rows + (long long)(bid % kFxRows) * kFxWords;
        if (t < 4) {
            unsigned __int128 v = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w)
                v += ((unsigned __int128)sfx[w][FX_SUM + 2 * t + 1] << 64) | sfx[w][FX_SUM + 2 * t];
            const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
            const unsigned long long old = atomicAdd(row + FX_SUM + 2 * t, lo);
            atomicAdd(row + FX_SUM + 2 * t + 1, hi + (old + lo < old ? 1ull : 0ull));
        } else if (t >= FX_SITES && t <= FX_BAD) {
            unsigned long long v = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) v = t == FX_BAD ? (v | sfx[w][t]) : v + sfx[w][t];
            if (t == FX_NBAD && v != 0) atomicOr(p.status, kStatNonfinite);  // a site was nonfinite
            if (t == FX_BAD) {
                if (v) atomicOr(row + t, v);
            } else {
                atomicAdd(row + t, v);
            }
        }
    }
}

}  // namespace

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

namespace {

template <typename S, bool MED, bool POS, bool BATCHED, bool ENS = false, bool ENT = false, bool EP = false>
cudaError_t launch_k(const FusedArgs &A, const FusedArgs *table, const int2 *map, int blocks, cudaStream_t s)
{
    static bool configured = false;
    if (!configured && kCarveout >= 0) {
        // shared memory vs L1 split (percent of the unified array for shared memory)
        if (cudaFuncSetAttribute(k_fused<S, MED, POS, BATCHED, ENS, ENT, EP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 kCarveout) != cudaSuccess)
            cudaGetLastError();
    }
    configured = true;
    if constexpr (BATCHED) {
        k_fused<S, MED, POS, BATCHED, ENS, ENT, EP><<<blocks, kThreads, 0, s>>>(A, table, map);
    } else {
        // programmatic dependent launch: the blocks may become resident while
        // the previous kernel of the stream (the tail) still runs; they wait
        // for it (griddepcontrol.wait) before touching memory
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const FusedArgs *tab = table;
        const int2 *mp = map;
        return cudaLaunchKernelEx(&cfg, k_fused<S, MED, POS, BATCHED, ENS, ENT, EP>, A, tab, mp);
    }
    return cudaGetLastError();
}

// FP32 storage: one kernel per limiter set; 16-bit storage: one kernel that
// follows the limiter bits at run time.
template <typename S>
cudaError_t launch_lim(const FusedArgs &A, int blocks, cudaStream_t s)
{
    // FP32 passes without the median filter: the variant that stores limited
    // rows at once (every limiter of the pass is site-local)
    const bool nomed = std::is_same<S, float>::value && !(A.p.limiters & 4u);
    if (A.p.eq == 1) {  // entropic f* and the exact dS of Eq. DelS; every limiter bit at run time
        if constexpr (std::is_same<S, float>::value)
            if (nomed) return launch_k<S, false, true, false, true, true>(A, nullptr, nullptr, blocks, s);
        return launch_k<S, true, true, false, true, true>(A, nullptr, nullptr, blocks, s);
    }
    if (A.p.limiters & kLimEnsemble) {  // the ensemble-dependent limiters follow every bit at run time
        if constexpr (std::is_same<S, float>::value)
            if (nomed) return launch_k<S, false, true, false, true>(A, nullptr, nullptr, blocks, s);
        return launch_k<S, true, true, false, true>(A, nullptr, nullptr, blocks, s);
    }
    if constexpr (std::is_same<S, float>::value) {
        const bool med = (A.p.limiters & 4u) != 0, pos = (A.p.limiters & 1u) != 0;
        if (med && pos) return launch_k<S, true, true, false>(A, nullptr, nullptr, blocks, s);
        if (med) return launch_k<S, true, false, false>(A, nullptr, nullptr, blocks, s);
        if (pos) return launch_k<S, false, true, false>(A, nullptr, nullptr, blocks, s);
        return launch_k<S, false, false, false>(A, nullptr, nullptr, blocks, s);
    } else {
        // 16-bit storage: the positivity code is compiled out when the rule is off
        // (the rest of the instruction stream is the kernel's limit, not memory)
        if (!(A.p.limiters & 1u)) return launch_k<S, true, false, false>(A, nullptr, nullptr, blocks, s);
        return launch_k<S, true, true, false>(A, nullptr, nullptr, blocks, s);
    }
}

}  // namespace

int fused_slots(int elem_bytes, bool batched)
{
    (void)elem_bytes;  // every storage type runs kBlocksPerSM blocks per SM
    const int per_sm = batched ? kBlocksPerSMBatched : kBlocksPerSM;  // as in the launch bounds
    return per_sm * kWarps * sm_count();
}

// A launch has one block per kWarps work items; items are strips of 62
// columns times row segments of at least kMinSegRows rows.
int fused_d2q9_blocks(int nx, int ny)
{
    const long long strips = (nx + kStripCols - 1) / kStripCols, segs = (ny + kMinSegRows - 1) / kMinSegRows;
    return (int)((strips * segs + kWarps - 1) / kWarps);
}

bool fused_d2q9_fits(long long plane) { return 9LL * plane < 0x7fffffffLL; }

int fused_make_args(const StepParams &p, const void *src, void *dst, int seg_rows, int slots, FusedArgs *A)
{
    *A = FusedArgs{};
    A->p = p;
    A->src = src;
    A->dst = dst;
    // Work items: strips of 62 columns x row segments, about `slots` of them
    // (one wave of resident warps) unless `seg_rows` fixes the segment.
    A->strips = (p.nx + kStripCols - 1) / kStripCols;
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
    // Dynamic work: one wave of resident blocks over short row segments, about
    // kItemsPerWarp items per warp; warps past their first item take the next
    // from the counter p.work (cleared by the tail kernel after the launch).
    // the entropic variant keeps more registers: three blocks per SM
    const int slots = p.eq == 1 ? 3 * kWarps * sm_count() : fused_slots((int)sizeof(S), false);
    int rows = 0;
    if (p.work != nullptr) {
        const long long strips = (p.nx + kStripCols - 1) / kStripCols;
        rows = (int)std::max<long long>(kMinSegRows, (strips * p.ny + (long long)kItemsPerWarp * slots - 1) /
                                                         ((long long)kItemsPerWarp * slots));
    }
    FusedArgs A;
    fused_make_args(p, src, dst, rows, slots, &A);
    const int blocks = p.work != nullptr ? std::min(A.blocks, slots / kWarps) : A.blocks;
    *nblocks = blocks;
    return launch_lim<S>(A, blocks, s);
}

template cudaError_t launch_fused_d2q9<float>(const StepParams &, const float *, float *, int *, cudaStream_t);
template cudaError_t launch_fused_d2q9<__nv_bfloat16>(const StepParams &, const __nv_bfloat16 *, __nv_bfloat16 *,
                                                      int *, cudaStream_t);
template cudaError_t launch_fused_d2q9<__half>(const StepParams &, const __half *, __half *, int *, cudaStream_t);

// E(dS) of the step about to run (Sec. 3.3), by the fused kernel's row
// streaming with nothing stored: the sum in exact fixed point into the rows
// p.fx_rows (count in FX_SITES), the work items through p.work; k_ens_fx turns
// them into {E, alpha, sum, count} at p.ens and clears rows and counter.
__global__ void k_ens_fx(StepParams p, double *out)
{
    const int lane = threadIdx.x;
    unsigned long long *rows = p.fx_rows;
    // lane r < kFxRows adds row r's sum (128 bits) and count
    unsigned __int128 v = 0;
    unsigned long long cnt = 0;
    if (lane < kFxRows) {
        unsigned long long *row = rows + (long long)lane * kFxWords;
        v = ((unsigned __int128)row[FX_SUM + 2 * P_SUM_DS + 1] << 64) | row[FX_SUM + 2 * P_SUM_DS];
        cnt = row[FX_SITES];
        for (int w = 0; w < kFxWords; ++w) row[w] = 0ull;
    }
#pragma unroll
    for (int o = 1; o < kFxRows; o <<= 1) {
        const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
        const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
        v += ((unsigned __int128)hi << 64) | lo;
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        const double s = fx_value(v);
        const double c = (double)cnt;
        const double E = c > 0.0 ? s / c : 0.0;
        out[0] = E;
        out[1] = E > 0.0 ? p.smooth_delta / pow(E, p.smooth_k) : 0.0;  // alpha of Eq. smooth1
        out[2] = s;
        out[3] = c;
        *p.work = 0;
    }
}

template <typename S>
cudaError_t launch_fused_epass(const StepParams &p, const S *src, cudaStream_t s)
{
    const int slots = p.eq == 1 ? 3 * kWarps * sm_count() : fused_slots((int)sizeof(S), false);
    const long long strips = (p.nx + kStripCols - 1) / kStripCols;
    const int rows = (int)std::max<long long>(kMinSegRows, (strips * p.ny + (long long)kItemsPerWarp * slots - 1) /
                                                               ((long long)kItemsPerWarp * slots));
    FusedArgs A;
    fused_make_args(p, src, nullptr, rows, slots, &A);
    const int blocks = std::min(A.blocks, slots / kWarps);
    cudaError_t e = p.eq == 1 ? launch_k<S, false, false, false, false, true, true>(A, nullptr, nullptr, blocks, s)
                              : launch_k<S, false, false, false, false, false, true>(A, nullptr, nullptr, blocks, s);
    if (e != cudaSuccess) return e;
    k_ens_fx<<<1, 32, 0, s>>>(p, const_cast<double *>(p.ens));
    return cudaGetLastError();
}

template cudaError_t launch_fused_epass<float>(const StepParams &, const float *, cudaStream_t);

cudaError_t launch_fused_batched(const FusedArgs *table, const int2 *map, int items, int *work, cudaStream_t s)
{
    if (items <= 0) return cudaSuccess;
    FusedArgs A0{};
    A0.items = items;
    A0.p.work = work;
    const int blocks = std::min((items + kWarps - 1) / kWarps, fused_slots(4, true) / kWarps);
    return launch_k<float, true, true, true>(A0, table, map, blocks, s);
}

}  // namespace lbm
