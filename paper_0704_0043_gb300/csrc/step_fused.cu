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
//    Every stored population is therefore read from DRAM once; one thread
//    issues the copies six rows ahead of the rows being computed.
//  * Iteration r computes row r (pull, moments, f*, collision, dS), stores the
//    post-collision populations f' of the block's own sites at once, and writes
//    dS into a four-row ring.  After one block barrier the median stencil of
//    row r-1 is complete: sites whose phi = min(phi_pos, phi_med) is below 1
//    (few) re-read their f', recompute f* from its moments (the moments of f'
//    are those of f_in) and store f* + phi (f' - f*).  Only dS, phi_pos and the
//    Ehrenfests' key of row r-1 stay in registers across the barrier.
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
    float ds[4][T];
    unsigned long long bar[kStages];
    int abort;
};

struct FusedArgs {
    StepParams p;
    int strips, seg_rows;
    float a, delta_m, thr_e, rho_ref;
    float lid4, lid7, lid8;  // FP32 moving-wall terms of the links through the lid
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

template <int T, bool MED, bool POS>
__global__ void __launch_bounds__(T, 2) k_fused(const FusedArgs A, const float *__restrict__ src,
                                                float *__restrict__ dst)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FusedSmem<T> &sm = *reinterpret_cast<FusedSmem<T> *>(smem_raw);
    __shared__ double red[T / 32][P_NSTAT];
    const StepParams &p = A.p;
    const int t = threadIdx.x;
    const int nx = p.nx, ny = p.ny;
    const int plane = (int)p.plane;  // 9 * plane < 2^31 is checked at launch
    const int strip = (int)blockIdx.x % A.strips, seg = (int)blockIdx.x / A.strips;
    const int cx0 = strip * (T - 2) - 1;  // lattice column of thread 0
    const int x = cx0 + t;
    const int ys = seg * A.seg_rows, ye = min(ys + A.seg_rows, ny);
    // staged columns [xs0, xs0 + Lc): 16-byte aligned, inside the padded row
    const int xs0 = (cx0 - 1) >= 0 ? ((cx0 - 1) & ~3) : -4;
    const int Lc = min(T + kPad, (((nx + 3) & ~3) + 4) - xs0);
    const int o = t + (cx0 - xs0);  // staged index of column x
    const int r0 = max(ys - 1, 0), rl = min(ye, ny);
    const int s_first = r0 - 1, s_last = min(rl, ny - 1) + 1;
    const bool xin = x >= 0 && x < nx;
    const bool xown = xin && t >= 1 && t <= T - 2;
    const bool xwall = x == 0 || x == nx - 1;
    const int xin_dx = x == 0 ? 1 : -1;  // inward x neighbour of a wall column
    const bool lim_ehr = (p.limiters & 2u) != 0;

    auto issue = [&](int s) {
        const int slot = (s - s_first) & (kStages - 1);
        const int rows[3] = {s, s - 1, s + 1};  // rows of plane groups {0,1,3}, {2,5,6}, {4,7,8}
        const int planes[3][3] = {{0, 1, 3}, {2, 5, 6}, {4, 7, 8}};
        unsigned bytes = 0;
#pragma unroll
        for (int g = 0; g < 3; ++g)
            if (rows[g] >= 0 && rows[g] < ny) bytes += 3u * (unsigned)Lc * 4u;
        mbar_expect_tx(&sm.bar[slot], bytes);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            if (rows[g] < 0 || rows[g] >= ny) continue;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int k = planes[g][i];
                const float *g_src = src + (long long)k * p.plane + (long long)rows[g] * p.pitch + kLead + xs0;
                bulk_copy(&sm.stage[slot][k][0], g_src, (unsigned)Lc * 4u, &sm.bar[slot]);
            }
        }
    };
    auto wait_stage = [&](int s) -> bool {
        const unsigned j = (unsigned)(s - s_first);
        return mbar_wait(&sm.bar[j & (kStages - 1)], (j / kStages) & 1u);
    };

    if (t == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&sm.bar[i], 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (t == 0)
        for (int s = s_first; s <= s_last && s < s_first + kStages; ++s) issue(s);

    const float a = A.a, a2 = A.a * A.a, rho_ref = p.rho_ref;
    float ds_p = 0.f, pp_p = 1.f;
    bool bad_p = false, cand_p = false;
    float s_mass = 0.f, s_ds = 0.f, s_in = 0.f, s_lim = 0.f;
    int n_pos = 0, n_med = 0, n_bad = 0, n_sites = 0, rows_acc = 0;
    double acc_mass = 0.0, acc_ds = 0.0, acc_in = 0.0, acc_lim = 0.0;
    bool waited = false;  // stages r-1 and r are ready once stage r+1 of the previous row was

    for (int r = r0; r <= rl; ++r) {
        float ds = 0.f, pp = 1.f;
        bool bad = false, cand = false;
        if (r < ny) {
            bool ok = wait_stage(r + 1);
            if (!waited) ok = ok && wait_stage(r - 1) && wait_stage(r);
            waited = true;
            if (!ok) {
                atomicOr(p.status, kStatTimeout);
                sm.abort = 1;
            }
            const unsigned jr = (unsigned)(r - s_first);
            const float(*S0)[T + kPad] = sm.stage[jr & (kStages - 1)];
            const float(*Sm)[T + kPad] = sm.stage[(jr - 1u) & (kStages - 1)];
            const float(*Sp)[T + kPad] = sm.stage[(jr + 1u) & (kStages - 1)];
            // stored deviations g = f - rho_ref W arriving at (x, r)
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
            if (xin && (xwall || r == 0 || r == ny - 1)) {
                // halfway bounce-back: a link from outside returns the site's own
                // population of the opposite direction (planes {0,1,3} of row r
                // sit in stage r, {2,5,6} in stage r+1, {4,7,8} in stage r-1)
#pragma unroll
                for (int k = 1; k < 9; ++k) {
                    const int sx = x - Lat<9>::cx(k), sy = r - Lat<9>::cy(k);
                    if (sx >= 0 && sx < nx && sy >= 0 && sy < ny) continue;
                    const int q = Lat<9>::opp(k);
                    float v = (q == 1 || q == 3) ? S0[q][o] : ((q == 2 || q == 5 || q == 6) ? Sp[q][o] : Sm[q][o]);
                    if (sy > ny - 1) v += (k == 4 ? A.lid4 : (k == 7 ? A.lid7 : A.lid8));
                    g[k] = v;
                }
            }
            float drho, rho, ux, uy, gs[9];
            moments9_dev(g, rho_ref, drho, rho, ux, uy);
            feq9_dev(drho, rho, ux, uy, gs);
            float din = 0.f, fpmin = 3.4e38f;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float dk = gs[k] - g[k];
                const float fsa = p.rwf[k] + gs[k];  // absolute f*
                din = fmaf(dk, __fdividef(dk, fsa), din);
                g[k] = fmaf(a, dk, gs[k]);  // g' = g* + (2 beta - 1)(g* - g_in)
                if (POS) fpmin = fminf(fpmin, p.rwf[k] + g[k]);
            }
            ds = a2 * din;  // dS(f') = (2 beta - 1)^2 dS(f_in) for the same f*
            // f*_k >= rho W_k (1/2 - 3 u^2 / 2) > 0 whenever u^2 < 1/3; only fast
            // flows need the explicit test of every f*_k
            const float usq = fmaf(ux, ux, uy * uy);
            bad = !(rho > 0.f) || !isfinite(ds);
            if (!(usq < 0.3f)) {
                float fsmin = 3.4e38f;
#pragma unroll
                for (int k = 0; k < 9; ++k) fsmin = fminf(fsmin, p.rwf[k] + gs[k]);
                bad = bad || !(fsmin > 0.f);
            }
            if (bad) {
                ds = __int_as_float(0x7f800000);
            } else if (POS && fpmin < 0.f) {  // positivity rule (Sec. 3.1)
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float fpa = p.rwf[k] + g[k], fsa = p.rwf[k] + gs[k];
                    if (fpa < 0.f) pp = fminf(pp, fsa / (fsa - fpa));
                }
            }
            const bool own = xown && r >= ys && r < ye;
            if (own) {
                float *out = dst + (long long)r * p.pitch + kLead + x;
#pragma unroll
                for (int k = 0; k < 9; ++k) out[k * plane] = g[k];
                s_mass += drho;
                ++n_sites;
                if (!bad) {
                    s_ds += ds;
                    s_in += din;
                } else {
                    ++n_bad;
                    atomicOr(p.status, kStatNonfinite);
                }
                n_pos += pp < 1.f;
            }
            // Ehrenfests' candidates: the tail kernel recomputes the FP64 key of
            // every site recorded here from the pre-step populations
            cand = lim_ehr && !bad && own && ds > A.thr_e;
            sm.ds[r & 3][t] = ds;
        }
        __syncthreads();
        if (sm.abort) break;
        if (t == 0 && r - 1 + kStages <= s_last) issue(r - 1 + kStages);

        const int y = r - 1;
        if (xown && y >= ys && y < ye) {
            float pm = 1.f;
            if (MED && !bad_p) {
                const float *D0 = sm.ds[y & 3], *Dm = sm.ds[(y - 1) & 3], *Dp = sm.ds[(y + 1) & 3];
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
                pm = phi_median<float>(ds_p, med, A.delta_m, p.median_mode);
            }
            const float phi = fminf(pp_p, pm);
            if (phi < 1.f) {
                // limiter homothety g* + phi (g' - g*) on the stored g' (Eq. LimGenF);
                // g* from the moments of g' (equal to those of g_in)
                float *out = dst + (long long)y * p.pitch + kLead + x;
                float g[9], gs[9], drho, rho, ux, uy;
#pragma unroll
                for (int k = 0; k < 9; ++k) g[k] = out[k * plane];
                moments9_dev(g, rho_ref, drho, rho, ux, uy);
                feq9_dev(drho, rho, ux, uy, gs);
#pragma unroll
                for (int k = 0; k < 9; ++k) out[k * plane] = fmaf(phi, g[k] - gs[k], gs[k]);
                s_lim = fmaf(1.f - phi * phi, ds_p, s_lim);
            }
            n_med += pm < 1.f;
            if (cand_p) {
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
        ds_p = ds;
        pp_p = pp;
        bad_p = bad;
        cand_p = cand;
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
        p.partials[(long long)blockIdx.x * P_NSTAT + t] = v;
    }
}

struct Shape {
    int T, strips, segs, seg_rows;
};

Shape choose_shape(int nx, int ny)
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
    const int s256 = (nx + 253) / 254, s320 = (nx + 317) / 318;
    Shape sh{};
    sh.T = (long long)s320 * 320 < (long long)s256 * 256 ? 320 : 256;
    sh.strips = sh.T == 320 ? s320 : s256;
    const int slots = 2 * sms;
    int segs = std::max(1, slots / sh.strips);
    int rows = std::max(kMinSegRows, (ny + segs - 1) / segs);
    sh.seg_rows = rows;
    sh.segs = (ny + rows - 1) / rows;
    return sh;
}

template <int T, bool MED, bool POS>
cudaError_t launch_t(const FusedArgs &A, int blocks, const float *src, float *dst, cudaStream_t s)
{
    const size_t smem = sizeof(FusedSmem<T>);
    static bool configured = false;
    if (!configured) {
        cudaError_t e =
            cudaFuncSetAttribute(k_fused<T, MED, POS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_fused<T, MED, POS><<<blocks, T, smem, s>>>(A, src, dst);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_lim(const FusedArgs &A, int blocks, const float *src, float *dst, cudaStream_t s)
{
    const bool med = (A.p.limiters & 4u) != 0, pos = (A.p.limiters & 1u) != 0;
    if (med && pos) return launch_t<T, true, true>(A, blocks, src, dst, s);
    if (med) return launch_t<T, true, false>(A, blocks, src, dst, s);
    if (pos) return launch_t<T, false, true>(A, blocks, src, dst, s);
    return launch_t<T, false, false>(A, blocks, src, dst, s);
}

}  // namespace

int fused_d2q9_blocks(int nx, int ny) { return ((nx + 253) / 254) * ((ny + kMinSegRows - 1) / kMinSegRows); }

bool fused_d2q9_fits(long long plane) { return 9LL * plane < 0x7fffffffLL; }

cudaError_t launch_fused_d2q9(const StepParams &p, const float *src, float *dst, int *nblocks, cudaStream_t s)
{
    const Shape sh = choose_shape(p.nx, p.ny);
    FusedArgs A{};
    A.p = p;
    A.strips = sh.strips;
    A.seg_rows = sh.seg_rows;
    A.a = (float)p.a;
    A.delta_m = (float)p.delta_m;
    A.thr_e = (float)(p.delta_e * (1.0 - 1.0 / 64.0));
    A.rho_ref = p.rho_ref;
    A.lid4 = (float)p.lid[4];
    A.lid7 = (float)p.lid[7];
    A.lid8 = (float)p.lid[8];
    const int blocks = sh.strips * sh.segs;
    *nblocks = blocks;
    return sh.T == 320 ? launch_lim<320>(A, blocks, src, dst, s) : launch_lim<256>(A, blocks, src, dst, s);
}

}  // namespace lbm
