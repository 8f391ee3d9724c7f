// step_fused.cu -- row-streaming fused FP32 D2Q9 step for the walled cavity.
//
// The same step as the tiled kernel (free flight with halfway bounce-back and
// moving lid, Sec. 2 and Sec. 4.4.1; polynomial f*, Eq. polyeq2d; LBGK
// collision, Eq. collLBGK; dS(f'), Sec. 3.6; positivity rule, Sec. 3.1; median
// filter, Sec. 3.5; Ehrenfests' candidates, Sec. 3.2; FP64 sums, Sec. 3.4),
// organised for HBM streaming:
//
//  * A block owns a strip of T computed columns (T - 2 finished; strips
//    overlap by two columns so the median has its x halo) and walks a segment
//    of rows upward, one thread per column.
//  * Populations arrive by bulk asynchronous copies (cp.async.bulk, completion
//    counted on an mbarrier) into an 8-deep ring of shared-memory stages.
//    Stage s holds, for the strip's columns, the rows that the pull of row s
//    reads: planes {0,1,3} of row s, {2,5,6} of row s-1, {4,7,8} of row s+1.
//    Every stored population is therefore read from DRAM once; nine lanes of
//    warp 0 issue the copies (one plane each) four to five rows ahead.
//  * Iteration r computes rows r and r+1 (pull, moments, f*, collision, dS),
//    stores the post-collision populations f' of the block's own sites at once,
//    and writes dS into an eight-row ring.  After one block barrier the median stencil of
//    rows r-1 and r is complete: sites whose phi = min(phi_pos, phi_med) is below 1
//    (few) re-read their f', recompute the collision's f* from the moments
//    carried across the barrier and store f* + phi (f' - f*).  Only dS,
//    phi_pos, the moments and a candidate flag of row r-1 stay in registers.
//  * Storage and arithmetic are FP32 on the deviations g = f - rho_ref W
//    (see lattice.cuh); no FP64 on the per-site path.  Sites whose FP32
//    dS is near or above the Ehrenfests' threshold are recorded; the tail
//    kernel recomputes their collision in FP64 from the pre-step populations
//    (the candidate key is FP64, as in the oracle).  Sums are kept per thread
//    in FP32 (mass as rho - rho_ref) and folded into FP64 every 32 rows.
//  * Every mbarrier wait is bounded by a clock limit; on expiry the block sets
//    the timeout status bit and stops.
#include <algorithm>

#include "internal.h"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int kStages = 8;
constexpr int kPad = 8;          // floats staged beyond the strip's T columns
constexpr int kMinSegRows = 16;  // shortest row segment (the halo rows cost 2 / segment)
constexpr long long kWaitLimit = 4000000000LL;  // clock cycles (about 2 s)

template <int T> struct FusedSmem {
    float stage[kStages][9][T + kPad];
    float ds[8][T];  // dS ring: rows r-2 .. r+1 are read while r+2, r+3 are written
    unsigned long long bar[kStages];
    int abort;
};

struct RowState {
    float ds, pp, drho, ux, uy;
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

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
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

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitLimit) return false;
    }
    return true;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// MED / POS: the median / positivity code is compiled in (each still follows
// the instance's limiter bits).  BATCHED: block b runs instance map[b].x of
// `table` as its block map[b].y; otherwise the single instance A0.
template <int T, bool MED, bool POS, bool BATCHED>
__global__ void __launch_bounds__(T, 2) k_fused(const FusedArgs A0, const FusedArgs *__restrict__ table,
                                                const int2 *__restrict__ map)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FusedSmem<T> &sm = *reinterpret_cast<FusedSmem<T> *>(smem_raw);
    __shared__ double red[T / 32][P_NSTAT];
    __shared__ __align__(16) FusedArgs sA;
    int bid = (int)blockIdx.x;
    if constexpr (BATCHED) {
        const int2 m = map[blockIdx.x];
        const unsigned *from = reinterpret_cast<const unsigned *>(table + m.x);
        unsigned *to = reinterpret_cast<unsigned *>(&sA);
        for (int i = threadIdx.x; i < (int)(sizeof(FusedArgs) / 4); i += T) to[i] = from[i];
        bid = m.y;
        __syncthreads();
    }
    const FusedArgs &A = BATCHED ? sA : A0;
    const StepParams &p = A.p;
    const float *__restrict__ src = A.src;
    float *__restrict__ dst = A.dst;
    const int t = threadIdx.x;
    const int nx = p.nx, ny = p.ny;
    const int plane = (int)p.plane;  // 9 * plane < 2^31 is checked at launch
    const int strip = bid % A.strips, seg = bid / A.strips;
    const int cx0 = strip * (T - 2) - 1;  // lattice column of thread 0
    const int x = cx0 + t;
    const int ys = seg * A.seg_rows, ye = min(ys + A.seg_rows, ny);
    // staged columns [xs0, xs0 + Lc): 16-byte aligned, inside the padded row
    const int xs0 = (cx0 - 1) >= 0 ? ((cx0 - 1) & ~3) : -4;
    const int Lc = min(T + kPad, (((nx + 3) & ~3) + 4) - xs0);
    const int o = t + (cx0 - xs0);  // staged index of column x
    const int r0 = max(ys - 1, 0);
    const int rc = min(ye, ny - 1);  // last row whose dS this block computes
    const int s_first = r0 - 1, s_last = rc + 1;
    const bool xin = x >= 0 && x < nx;
    const bool xown = xin && t >= 1 && t <= T - 2;
    const bool xwall = x == 0 || x == nx - 1;
    const int xin_dx = x == 0 ? 1 : -1;  // inward x neighbour of a wall column
    const bool lim_ehr = (p.limiters & 2u) != 0;
    const bool med_on = MED && (p.limiters & 4u) != 0, pos_on = POS && (p.limiters & 1u) != 0;

    // warp 0 stages the rows of stage s: lane 0 posts the byte count, lanes
    // 0..8 copy one plane each (planes {0,1,3} of row s, {2,5,6} of row s-1,
    // {4,7,8} of row s+1)
    auto issue = [&](int s) {
        const int slot = (s - s_first) & (kStages - 1);
        unsigned bytes = 0;
        if (s >= 0 && s < ny) bytes += 3u * (unsigned)Lc * 4u;
        if (s - 1 >= 0 && s - 1 < ny) bytes += 3u * (unsigned)Lc * 4u;
        if (s + 1 >= 0 && s + 1 < ny) bytes += 3u * (unsigned)Lc * 4u;
        if (t == 0) mbar_expect_tx(&sm.bar[slot], bytes);
        __syncwarp();
        if (t < 9) {
            const int k = t;
            const int row = (k == 0 || k == 1 || k == 3) ? s : ((k == 2 || k == 5 || k == 6) ? s - 1 : s + 1);
            if (row >= 0 && row < ny) {
                const float *g_src = src + (long long)k * p.plane + (long long)row * p.pitch + kLead + xs0;
                bulk_copy(&sm.stage[slot][k][0], g_src, (unsigned)Lc * 4u, &sm.bar[slot]);
            }
        }
    };
    auto wait_stage = [&](int s) -> bool {
        if (s > s_last) return true;
        const unsigned j = (unsigned)(s - s_first);
        return mbar_wait(&sm.bar[j & (kStages - 1)], (j / kStages) & 1u);
    };

    if (t == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&sm.bar[i], 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (t < 32)
        for (int s = s_first; s <= s_last && s < s_first + kStages; ++s) issue(s);

    const float a = A.a, a2 = A.a * A.a, rho_ref = p.rho_ref;
    float s_mass = 0.f, s_ds = 0.f, s_in = 0.f, s_lim = 0.f;
    int n_pos = 0, n_med = 0, n_bad = 0, n_sites = 0, rows_acc = 0;
    double acc_mass = 0.0, acc_ds = 0.0, acc_in = 0.0, acc_lim = 0.0;

    // Row q: free flight, collision, dS; stores g' of the block's own sites.
    auto compute_row = [&](int q) -> RowState {
        RowState st{0.f, 1.f, 0.f, 0.f, 0.f, false, false};
        if (q > rc) return st;
        const unsigned jr = (unsigned)(q - s_first);
        const float(*S0)[T + kPad] = sm.stage[jr & (kStages - 1)];
        const float(*Sm)[T + kPad] = sm.stage[(jr - 1u) & (kStages - 1)];
        const float(*Sp)[T + kPad] = sm.stage[(jr + 1u) & (kStages - 1)];
        // stored deviations g = f - rho_ref W arriving at (x, q)
        float g[9];
        g[0] = S0[0][o];
        g[1] = S0[1][o - 1];
        g[2] = S0[2][o];
        g[3] = S0[3][o + 1];
        g[4] = S0[4][o];
        g[5] = S0[5][o - 1];
        g[6] = S0[6][o + 1];
        g[7] = S0[7][o + 1];
        g[8] = S0[8][o - 1];
        if (q == 0 || q == ny - 1 || (xin && xwall)) {
            if (xin) {
                // halfway bounce-back: a link from outside returns the site's own
                // population of the opposite direction (planes {0,1,3} of row q
                // sit in stage q, {2,5,6} in stage q+1, {4,7,8} in stage q-1)
#pragma unroll
                for (int k = 1; k < 9; ++k) {
                    const int sx = x - Lat<9>::cx(k), sy = q - Lat<9>::cy(k);
                    if (sx >= 0 && sx < nx && sy >= 0 && sy < ny) continue;
                    const int qq = Lat<9>::opp(k);
                    float v = (qq == 1 || qq == 3) ? S0[qq][o]
                                                    : ((qq == 2 || qq == 5 || qq == 6) ? Sp[qq][o] : Sm[qq][o]);
                    if (sy > ny - 1) v += (k == 4 ? A.lid4 : (k == 7 ? A.lid7 : A.lid8));
                    g[k] = v;
                }
            }
        }
        float rho, gs[9];
        moments9_dev(g, rho_ref, st.drho, rho, st.ux, st.uy);
        feq9_dev(st.drho, rho, st.ux, st.uy, gs);
        float din = 0.f, fpmin = 3.4e38f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float dk = gs[k] - g[k];
            const float fsa = p.rwf[k] + gs[k];  // absolute f*
            din = fmaf(dk, __fdividef(dk, fsa), din);
            g[k] = fmaf(a, dk, gs[k]);  // g' = g* + (2 beta - 1)(g* - g_in)
            if (pos_on) fpmin = fminf(fpmin, p.rwf[k] + g[k]);
        }
        float ds = a2 * din;  // dS(f') = (2 beta - 1)^2 dS(f_in) for the same f*
        // f*_k >= rho W_k (1/2 - 3 u^2 / 2) > 0 whenever u^2 < 1/3; only fast
        // flows need the explicit test of every f*_k
        const float usq = fmaf(st.ux, st.ux, st.uy * st.uy);
        bool bad = !(rho > 0.f) || !isfinite(ds);
        if (!(usq < 0.3f)) {
            float fsmin = 3.4e38f;
#pragma unroll
            for (int k = 0; k < 9; ++k) fsmin = fminf(fsmin, p.rwf[k] + gs[k]);
            bad = bad || !(fsmin > 0.f);
        }
        if (bad) {
            ds = __int_as_float(0x7f800000);
        } else if (pos_on && fpmin < 0.f) {  // positivity rule (Sec. 3.1)
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float fpa = p.rwf[k] + g[k], fsa = p.rwf[k] + gs[k];
                if (fpa < 0.f) st.pp = fminf(st.pp, fsa / (fsa - fpa));
            }
        }
        const bool own = xown && q >= ys && q < ye;
        if (own) {
            float *out = dst + (long long)q * p.pitch + kLead + x;
#pragma unroll
            for (int k = 0; k < 9; ++k) out[k * plane] = g[k];
            s_mass += st.drho;
            ++n_sites;
            if (!bad) {
                s_ds += ds;
                s_in += din;
            } else {
                ++n_bad;
                atomicOr(p.status, kStatNonfinite);
            }
            n_pos += st.pp < 1.f;
        }
        // Ehrenfests' candidates: the tail kernel recomputes the FP64 key of
        // every site recorded here from the pre-step populations
        st.cand = lim_ehr && !bad && own && ds > A.thr_e;
        st.bad = bad;
        st.ds = ds;
        sm.ds[q & 7][t] = ds;
        return st;
    };

    // Row y: median of dS, phi = min(phi_pos, phi_med), homothety on the stored
    // g' where phi < 1, candidate record, sums.
    auto finalise_row = [&](int y, const RowState &st) {
        if (!(xown && y >= ys && y < ye)) return;
        float pm = 1.f;
        if (med_on && !st.bad) {
            const float *D0 = sm.ds[y & 7], *Dm = sm.ds[(y - 1) & 7], *Dp = sm.ds[(y + 1) & 7];
            const bool ywall = y == 0 || y == ny - 1;
            float med;
            if (xwall || ywall) {
                if (xwall && ywall)
                    med = med3(D0[t], D0[t + xin_dx], (y == 0 ? Dp : Dm)[t]);
                else if (ywall)
                    med = med3(D0[t - 1], D0[t], D0[t + 1]);
                else
                    med = med3(Dm[t], D0[t], Dp[t]);
            } else {
                med = med9(Dm[t - 1], D0[t - 1], Dp[t - 1], Dm[t], D0[t], Dp[t], Dm[t + 1], D0[t + 1], Dp[t + 1]);
            }
            pm = phi_median<float>(st.ds, med, A.delta_m, p.median_mode);
        }
        const float phi = fminf(st.pp, pm);
        if (phi < 1.f) {
            // limiter homothety g* + phi (g' - g*) on the stored g' (Eq. LimGenF),
            // with the same g* as the collision (recomputed from the carried moments)
            float *out = dst + (long long)y * p.pitch + kLead + x;
            float g[9], gs[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) g[k] = out[k * plane];
            feq9_dev(st.drho, rho_ref + st.drho, st.ux, st.uy, gs);
#pragma unroll
            for (int k = 0; k < 9; ++k) out[k * plane] = fmaf(phi, g[k] - gs[k], gs[k]);
            s_lim = fmaf(1.f - phi * phi, st.ds, s_lim);
        }
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
    };

    // Two rows per iteration: compute rows r and r+1, barrier, finish rows r-1
    // (computed in the previous iteration) and r.
    RowState prev{0.f, 1.f, 0.f, 0.f, 0.f, false, false};
    for (int r = r0; r - 1 < ye; r += 2) {
        bool ok = wait_stage(r + 1) && wait_stage(r + 2);
        if (r == r0) ok = ok && wait_stage(r - 1) && wait_stage(r);
        if (!ok) {
            atomicOr(p.status, kStatTimeout);
            sm.abort = 1;
        }
        const RowState ra = compute_row(r);
        const RowState rb = compute_row(r + 1);
        __syncthreads();
        if (sm.abort) break;
        if (t < 32) {
            if (r - 1 + kStages <= s_last) issue(r - 1 + kStages);
            if (r + kStages <= s_last) issue(r + kStages);
        }
        finalise_row(r - 1, prev);
        finalise_row(r, ra);
        prev = rb;
    }
    double acc[P_NSTAT];
    acc[P_MASS] = acc_mass + (double)s_mass + (double)n_sites * (double)rho_ref;
    acc[P_SUM_DS] = acc_ds + (double)s_ds;
    acc[P_SUM_IN] = acc_in + (double)s_in;
    acc[P_DS_LIM] = acc_lim + (double)s_lim;
    acc[P_NPOS] = (double)n_pos;
    acc[P_NMED] = (double)n_med;
    acc[P_NBAD] = (double)n_bad;
    const int warp = t >> 5, lane = t & 31;
#pragma unroll
    for (int i = 0; i < P_NSTAT; ++i) {
        const double v = warp_sum_d(acc[i]);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    if (t < P_NSTAT) {
        double v = 0.0;
        for (int w = 0; w < T / 32; ++w) v += red[w][t];
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

template <int T, bool MED, bool POS, bool BATCHED>
cudaError_t launch_t(const FusedArgs &A, const FusedArgs *table, const int2 *map, int blocks, cudaStream_t s)
{
    const size_t smem = sizeof(FusedSmem<T>);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<T, MED, POS, BATCHED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_fused<T, MED, POS, BATCHED><<<blocks, T, smem, s>>>(A, table, map);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_lim(const FusedArgs &A, int blocks, cudaStream_t s)
{
    const bool med = (A.p.limiters & 4u) != 0, pos = (A.p.limiters & 1u) != 0;
    if (med && pos) return launch_t<T, true, true, false>(A, nullptr, nullptr, blocks, s);
    if (med) return launch_t<T, true, false, false>(A, nullptr, nullptr, blocks, s);
    if (pos) return launch_t<T, false, true, false>(A, nullptr, nullptr, blocks, s);
    return launch_t<T, false, false, false>(A, nullptr, nullptr, blocks, s);
}

}  // namespace

int fused_d2q9_blocks(int nx, int ny) { return ((nx + 253) / 254) * ((ny + kMinSegRows - 1) / kMinSegRows); }

bool fused_d2q9_fits(long long plane) { return 9LL * plane < 0x7fffffffLL; }

int fused_pick_T(int nx)
{
    const int s256 = (nx + 253) / 254, s320 = (nx + 317) / 318;
    return (long long)s320 * 320 < (long long)s256 * 256 ? 320 : 256;
}

int fused_make_args(const StepParams &p, const float *src, float *dst, int T, int slots, FusedArgs *A)
{
    *A = FusedArgs{};
    A->p = p;
    A->src = src;
    A->dst = dst;
    A->strips = (p.nx + T - 3) / (T - 2);
    const int segs = std::max(1, slots / A->strips);
    A->seg_rows = std::max(kMinSegRows, (p.ny + segs - 1) / segs);
    A->blocks = A->strips * ((p.ny + A->seg_rows - 1) / A->seg_rows);
    A->a = (float)p.a;
    A->delta_m = (float)p.delta_m;
    A->thr_e = (float)(p.delta_e * (1.0 - 1.0 / 64.0));
    A->rho_ref = p.rho_ref;
    A->lid4 = (float)p.lid[4];
    A->lid7 = (float)p.lid[7];
    A->lid8 = (float)p.lid[8];
    return A->blocks;
}

cudaError_t launch_fused_d2q9(const StepParams &p, const float *src, float *dst, int *nblocks, cudaStream_t s)
{
    const int T = fused_pick_T(p.nx);
    FusedArgs A;
    *nblocks = fused_make_args(p, src, dst, T, 2 * sm_count(), &A);
    return T == 320 ? launch_lim<320>(A, A.blocks, s) : launch_lim<256>(A, A.blocks, s);
}

cudaError_t launch_fused_batched(int T, const FusedArgs *table, const int2 *map, int blocks, cudaStream_t s)
{
    if (blocks <= 0) return cudaSuccess;
    const FusedArgs none{};
    return T == 320 ? launch_t<320, true, true, true>(none, table, map, blocks, s)
                    : launch_t<256, true, true, true>(none, table, map, blocks, s);
}

}  // namespace lbm
