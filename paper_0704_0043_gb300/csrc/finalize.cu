// finalize.cu -- the per-step tail: fixed-order FP64 reduction of the step
// kernel's block partials, Ehrenfests' selection and step, and the stats record.
//
// Ehrenfests' regularisation (Sec. 3.2; Sec. 4.3.2): among the sites whose
// dS(f') exceeds delta, at most k with the largest dS are equilibrated,
// f -> f*(m(f)).  Ties in dS go to the lower site index, so the chosen set is
// unique.  When there are more than k candidates, a single block finds the k-th
// largest (dS, -site) pair by radix selection: eight 8-bit digit passes over the
// 64-bit pattern of dS (positive doubles order like their bit patterns), then
// four passes over the site index among the candidates tied at the threshold.
//
// The kernel sits between two step launches, so it is built for latency: the
// candidates arrive with their FP64 keys (the step kernels evaluate them where
// they find them), up to kCap of them are kept in shared memory, and sums use
// warp shuffles or exact integer arithmetic.  One block runs the tail.  When a
// pass records more candidates than that (a state far from equilibrium), the
// tail runs as a cooperative grid of one block per SM that first preselects
// them (dense_select): the FP32 dS recorded with each candidate is within 1/64
// of its FP64 key, so a radix search over the FP32 values bounds the k-th
// largest key, and only the candidates near that bound or near delta need
// their FP64 keys; block 0 then selects among the short list.
#include <type_traits>

#include "internal.h"
#include "keys.cuh"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int kFinThreads = 512;
constexpr int kFinWarps = kFinThreads / 32;
constexpr int kCap = 2048;  // candidates held (and selected sets sorted) in shared memory
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kSelSpinLimit = 1u << 21;  // grid-barrier polls (about a second) before giving up

__device__ __forceinline__ unsigned long long key_bits(double d) { return (unsigned long long)__double_as_longlong(d); }

__device__ __forceinline__ long long fidx(long long plane, int pitch, int k, int y, int x)
{
    return (long long)k * plane + (long long)y * pitch + kLead + x;
}

// The pass's input at site (x, y) in FP32: after free flight (collide) with the
// step kernels' FP32 arithmetic (bounce-back, lid term added as hi + lo), or
// the stored populations themselves (limiter pass).
template <int Q, typename S>
__device__ void pull_dev(const FinalParams &p, int x, int y, float g[Q])
{
    const S *src = (const S *)p.src;
    const bool wrapx = bc_wrap_x(p.boundary), wrapy = Q == 9 && bc_wrap_y(p.boundary);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        if (!p.collide) {
            g[k] = s2f(src[fidx(p.plane, p.pitch, k, y, x)]);
            continue;
        }
        int sx = x - Lat<Q>::cx(k), sy = y - Lat<Q>::cy(k);
        if (wrapx) sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
        if (wrapy) sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
        if (sx >= 0 && sx < p.nx && sy >= 0 && sy < p.ny) {
            g[k] = s2f(src[fidx(p.plane, p.pitch, k, sy, sx)]);
        } else {
            float v = s2f(src[fidx(p.plane, p.pitch, Lat<Q>::opp(k), y, x)]);
            if (Q == 9 && sy > p.ny - 1) v = __fadd_rn(__fadd_rn(v, p.lidf[k]), p.lidlo[k]);
            g[k] = v;
        }
    }
}

// Sum over the block in a fixed order (same result every run): warp shuffle
// trees, then a shuffle tree over the warp totals; thread 0 gets the sum.
// FP64 additions are slow on this GPU, so the dependent chain is kept short.
// `warp0_only`: the other warps hold zeros, so warp 0's tree is the sum (the
// same bits: adding the zero totals changes nothing).
__device__ double block_sum0(double v, double *red, bool warp0_only)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (warp0_only && warp != 0) return 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (warp0_only) return v;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double r = lane < kFinWarps ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(kFull, r, o);
        v = r;
    }
    return v;
}


// The digit of a radix-selection pass: hist[d] counts the keys with digit d
// among those still in play, and the rem-th of them is wanted, counting from
// the top digit down (desc) or from digit 0 up.  Threads 0..255 scan the
// counts with warp shuffles (integer sums, so the same on every run) and the
// block picks the digit with __syncthreads_count; every thread of the block
// must call this.  Writes the digit to *digit and the rank left within it to
// *rem_left.
__device__ void pick_digit(const unsigned *hist, long long rem, bool desc, unsigned long long *part,
                           unsigned long long *digit, long long *rem_left)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned long long c = 0;
    if (t < 256) {
        c = hist[desc ? 255 - t : t];  // position t of the scan order
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) c += y;
        }
        if (lane == 31) part[w] = c;
    }
    __syncthreads();
    if (t < 256)
        for (int j = 0; j < w; ++j) c += part[j];
    // c = inclusive count up to scan position t; the wanted digit is the first
    // position whose inclusive count reaches rem
    const int before = __syncthreads_count(t < 256 && (long long)c < rem);
    if (t == before && t < 256) {
        *digit = (unsigned long long)(desc ? 255 - t : t);
        *rem_left = rem - ((long long)c - (long long)hist[desc ? 255 - t : t]);
    }
    __syncthreads();
}

// The geometry of the FP64 key evaluation (D2Q9, FP32 / 16-bit storage).
__device__ KeyGeom key_geom(const FinalParams &p)
{
    KeyGeom kg;
    kg.nx = p.nx;
    kg.ny = p.ny;
    kg.pitch = p.pitch;
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
    return kg;
}

// Grid barrier of the cooperative tail: each block adds one arrival to *bar;
// with `wait` it polls until `target` blocks have arrived.  The poll is
// bounded: past kSelSpinLimit polls the block sets kStatTimeout in *status and
// goes on (the pass's results are then not trusted; the host reports
// LBM_ERR_TIMEOUT).  Every thread of the block calls it; returns whether this
// block gave up.
__device__ bool grid_sync(unsigned *bar, unsigned target, bool wait, unsigned *status, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int gave_up = 0;
        __threadfence();
        atomicAdd(bar, 1u);
        if (wait) {
            unsigned polls = 0;
            while (*(volatile unsigned *)bar < target) {
                if (++polls > kSelSpinLimit) {
                    gave_up = 1;
                    atomicOr(status, kStatTimeout);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *s_flag = gave_up;
    }
    __syncthreads();
    return *s_flag != 0;
}

// The bin holding the rem-th largest entry (rem >= 1) of a kSelBins-bin
// histogram in device memory (bin b counts the keys with digit b, larger
// digits larger keys), and the rank left within that bin.  *s_tot receives the
// histogram's total; when it is below rem no bin holds the entry and *s_bin
// is -1.  Thread t scans bins 8t .. 8t+7 from the top; integer sums, so the
// same on every run.  Every thread of the block calls it.
__device__ void pick_bin(const unsigned *h, long long rem, long long *s_wpart, int *s_bin, long long *s_rem,
                         long long *s_tot)
{
    constexpr int kPer = kSelBins / kFinThreads;
    static_assert(kPer * kFinThreads == kSelBins, "whole bins per thread");
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned c[kPer];
    long long mine = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        c[j] = __ldcg(h + (kSelBins - 1 - (t * kPer + j)));  // written by other blocks' atomics
        mine += c[j];
    }
    long long incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_wpart[w] = incl;
    if (t == 0) *s_bin = -1;
    __syncthreads();
    for (int j = 0; j < w; ++j) incl += s_wpart[j];
    if (t == kFinThreads - 1) *s_tot = incl;
    const long long excl = incl - mine;
    if (excl < rem && rem <= incl) {  // one thread: its bins hold the entry
        long long acc = excl;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            if (acc < rem && rem <= acc + c[j]) {
                *s_bin = kSelBins - 1 - (t * kPer + j);
                *s_rem = rem - acc;
            }
            acc += c[j];
        }
    }
    __syncthreads();
}

// Device-wide preselection of n > kCap recorded candidates (all blocks of the
// cooperative tail call it).  R denotes the candidates whose FP32 dS exceeds
// dhi = delta (1 + 1/64): their FP64 keys exceed delta.  When |R| >= k, the
// k-th largest FP32 dS in R is at least T, the lower end of its bin after two
// 12-bit radix levels (bits 30..19, then 18..7, of the FP32 pattern; positive
// floats order like their patterns), so the k-th largest valid FP64 key is
// at least T / (1 + 1/64), and a candidate whose key reaches it has FP32 dS of
// at least T (1 - 1/64) / (1 + 1/64) > T (1 - 1/32) = Tlow.  The list takes
// every valid candidate with FP32 dS >= Tlow (all valid ones when |R| < k):
// it holds every candidate of the exact top k, ties at the k-th key included.
// The valid candidates are counted exactly: a candidate with a key is valid
// when the key exceeds delta; one without a key is keyed here when it is on
// the list's side of Tlow or within 1/64 of delta (at or below dhi), and
// otherwise valid when its FP32 dS exceeds dhi.  Block 0 then reads the list
// (returns true when it fits in kSelList) and resets the shared state for
// the next pass; the other blocks return false.  Not inlined: the one-block
// tail runs from a cold instruction cache every step, and its code stays
// compact without this rarely taken path.
template <int Q, typename S>
__device__ __noinline__ bool dense_select(const FinalParams &p, int n, unsigned *sh, long long *s_wpart, int *s_bin,
                             long long *s_rem, long long *s_tot, int *s_flag, int *s_qn, unsigned *s_acc,
                             unsigned *s_cnt, unsigned *s_nv)
{
    SelState *ss = p.sel_state;
    const int t = threadIdx.x, lane = t & 31;
    const unsigned nb = gridDim.x;
    const int dhi_bits = __float_as_int((float)(p.delta_e * (1.0 + 1.0 / 64.0)));
    const long long stride = (long long)nb * kFinThreads;
    const long long base0 = (long long)blockIdx.x * kFinThreads;
    auto in_r = [&](int u) { return u > dhi_bits && u < 0x7f800000; };  // FP32 dS above dhi (finite)

    // level 1: bits 30..19 of the candidates in R
    // lanes with the same bin add once (most candidates fall in a few bins)
    auto count_bin = [&](int bin) {
        const unsigned peers = __match_any_sync(kFull, bin);
        if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&sh[bin], (unsigned)__popc(peers));
    };
    for (int b = t; b < kSelBins; b += kFinThreads) sh[b] = 0;
    __syncthreads();
    for (long long base = base0; base < n; base += stride) {  // whole warps per round
        const long long i = base + t;
        int bin = -1;
        if (i < n) {
            const int u = __float_as_int(p.cand[i].ds32);
            if (in_r(u)) bin = u >> 19;
        }
        count_bin(bin);
    }
    __syncthreads();
    for (int b = t; b < kSelBins; b += kFinThreads)
        if (sh[b]) atomicAdd(&ss->hist1[b], sh[b]);
    grid_sync(&ss->bar, nb, true, p.status, s_flag);

    // level 2: bits 18..7 within the level-1 bin of the k-th largest
    pick_bin(ss->hist1, p.k_max, s_wpart, s_bin, s_rem, s_tot);
    const bool all = *s_tot < p.k_max;  // fewer than k in R: every valid candidate is listed
    const int b1 = *s_bin;
    const long long rem1 = *s_rem;
    for (int b = t; b < kSelBins; b += kFinThreads) sh[b] = 0;
    __syncthreads();
    if (!all) {
        for (long long base = base0; base < n; base += stride) {
            const long long i = base + t;
            int bin = -1;
            if (i < n) {
                const int u = __float_as_int(p.cand[i].ds32);
                if (in_r(u) && (u >> 19) == b1) bin = (u >> 7) & (kSelBins - 1);
            }
            count_bin(bin);
        }
        __syncthreads();
        for (int b = t; b < kSelBins; b += kFinThreads)
            if (sh[b]) atomicAdd(&ss->hist2[b], sh[b]);
    }
    grid_sync(&ss->bar, 2 * nb, true, p.status, s_flag);

    // the bound, the keys, the count and the list
    int tlow_bits = 0;
    if (!all) {
        pick_bin(ss->hist2, rem1, s_wpart, s_bin, s_rem, s_tot);
        const unsigned ulb = ((unsigned)b1 << 19) | ((unsigned)*s_bin << 7);
        tlow_bits = __float_as_int(__uint_as_float(ulb) * 0.96875f);
    }
    // Candidates without a key that need one are queued in shared memory (the
    // histogram is no longer needed) and keyed a block at a time, every lane
    // busy: FP64 is slow on this GPU, and keying them where they lie would
    // run most warps' FP64 code for one or two lanes.
    int *queue = reinterpret_cast<int *>(sh);  // at most 2 kFinThreads - 1 entries
    if (t == 0) {
        *s_acc = 0;
        *s_qn = 0;
    }
    __syncthreads();
    constexpr bool kKeyHere = !std::is_same<S, double>::value && Q == 9;  // candidates recorded without a key
    const KeyGeom kg = key_geom(p);
    unsigned nv = 0;
    // warp-aggregated list append (every lane of the warp calls it)
    auto append = [&](bool listed, long long i) {
        const unsigned m = __ballot_sync(kFull, listed);
        unsigned at = 0;
        if (lane == 0 && m) at = atomicAdd(&ss->count, (unsigned)__popc(m));
        at = __shfl_sync(kFull, at, 0) + __popc(m & ((1u << lane) - 1u));
        if (listed && at < (unsigned)kSelList) ss->list[at] = (int)i;
    };
    // key queue entries from .. from + cnt - 1 (cnt <= kFinThreads), one per thread
    auto drain = [&](int from, int cnt) {
        bool listed = false;
        long long i = -1;
        if (t < cnt) {
            i = queue[from + t];
            const Cand c = p.cand[i];
            const double key = key_dS9_lane<S>(kg, (const S *)p.src, c.site, p.delta_e);
            p.cand[i].key = key;
            const bool valid = key > p.delta_e;
            nv += valid;
            listed = valid && __float_as_int(c.ds32) >= tlow_bits;
        }
        append(listed, i);
    };
    for (long long base = base0; base < n; base += stride) {  // whole blocks per round
        const long long i = base + t;
        bool valid = false, listed = false, need = false;
        if (i < n) {
            const Cand c = p.cand[i];
            const int u = __float_as_int(c.ds32);
            const bool top = u >= tlow_bits;
            need = kKeyHere && isnan(c.key) && (top || u <= dhi_bits);
            valid = !need && (isnan(c.key) ? in_r(u) : c.key > p.delta_e);
            listed = top && valid;
        }
        append(listed, i);
        nv += valid;
        if constexpr (kKeyHere) {
            const unsigned m = __ballot_sync(kFull, need);
            int at = 0;
            if (lane == 0 && m) at = atomicAdd(s_qn, __popc(m));
            at = __shfl_sync(kFull, at, 0) + __popc(m & ((1u << lane) - 1u));
            if (need) queue[at] = (int)i;
            __syncthreads();
            const int qn = *s_qn;  // the same for the whole block
            if (qn >= kFinThreads) {
                drain(qn - kFinThreads, kFinThreads);
                __syncthreads();  // the entries are read before new ones overwrite them
                if (t == 0) *s_qn = qn - kFinThreads;
                __syncthreads();
            }
        }
    }
    if constexpr (kKeyHere) drain(0, *s_qn);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nv += __shfl_down_sync(kFull, nv, o);
    if (lane == 0 && nv) atomicAdd(s_acc, nv);
    __syncthreads();
    if (t == 0 && *s_acc) atomicAdd(&ss->n_valid, *s_acc);
    // block 0 waits for every block's list entries and count
    grid_sync(&ss->bar, 3 * nb, blockIdx.x == 0, p.status, s_flag);
    if (blockIdx.x != 0) return false;
    if (t == 0) {
        *s_cnt = __ldcg(&ss->count);
        *s_nv = __ldcg(&ss->n_valid);
        ss->count = 0;
        ss->n_valid = 0;
        ss->bar = 0;
    }
    for (int b = t; b < kSelBins; b += kFinThreads) {
        ss->hist1[b] = 0;
        ss->hist2[b] = 0;
    }
    __syncthreads();
    return *s_cnt <= (unsigned)kSelList;
}

// BATCHED: block b finishes instance b of `table`; otherwise the single (p0, f0).
// GRID: the cooperative grid of one block per SM (dense candidates are
// preselected by all blocks; block 0 runs the tail); otherwise one block.
template <int Q, typename S, bool BATCHED, bool GRID = false>
__global__ void __launch_bounds__(kFinThreads, BATCHED ? 2 : 1) k_finalize(const FinalParams p0, S *__restrict__ f0,
                                                          const FinalArgs *__restrict__ table)
{
    using T = compute_t<S>;
    // Launched as a programmatic dependent of the step kernel: wait for it to
    // finish before any memory access, then let the next step kernel be
    // scheduled early.  Both are no-ops in an ordinary launch.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // The next launch may be scheduled now.  In a grid launch it starts only
    // when every block of this grid has passed this point, i.e. when all of
    // them are resident, so its blocks cannot keep one of ours from running
    // (the grid barriers below wait for resident blocks only).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ double s_key[kCap];
    __shared__ int s_site[kCap];
    __shared__ int s_idx[kCap];
    __shared__ long long s_wpart[kFinWarps], s_rem2, s_tot;
    __shared__ int s_bin, s_flag, s_qn;
    __shared__ unsigned s_acc, s_cnt, s_nv;
    // dense candidates in a grid launch: every block preselects, then block 0
    // runs the tail over the list (use_list) or, when the list overflowed,
    // over all candidates; otherwise block 0 alone runs the tail
    bool use_list = false;
    if constexpr (GRID) {
        const int nrec = p0.ehrenfest ? *p0.cand_count : 0;
        const int n0 = nrec < p0.cand_cap ? nrec : p0.cand_cap;
        const bool dense = n0 > kCap && p0.sel_state != nullptr && p0.k_max > 0;
        if (!dense && blockIdx.x != 0) return;
        if (dense) {
            use_list = dense_select<Q, S>(p0, n0, reinterpret_cast<unsigned *>(s_key), s_wpart, &s_bin, &s_rem2,
                                          &s_tot, &s_flag, &s_qn, &s_acc, &s_cnt, &s_nv);
            if (blockIdx.x != 0) return;
        }
    }
    __shared__ __align__(16) FinalArgs sA;
    if constexpr (BATCHED) {
        const unsigned *from = reinterpret_cast<const unsigned *>(table + blockIdx.x);
        unsigned *to = reinterpret_cast<unsigned *>(&sA);
        for (int i = threadIdx.x; i < (int)(sizeof(FinalArgs) / 4); i += kFinThreads) to[i] = from[i];
        __syncthreads();
    }
    const FinalParams &p = BATCHED ? sA.p : p0;
    S *__restrict__ f = BATCHED ? (S *)sA.f : f0;
    __shared__ double red[kFinWarps + 1];
    __shared__ double tot[P_NSTAT];
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_part[8], s_digit;
    __shared__ long long s_rem, s_step, s_rec;
    __shared__ int s_nsel, s_valid;
    __shared__ unsigned s_status;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    // every thread reads the candidate count (one broadcast load) and loads its
    // first candidate slot at once (any slot below the capacity is readable,
    // so the load does not wait for the count), and both loads overlap the
    // reduction of the step's sums; list entry i is candidate cidx(i) (the
    // preselected list, or all candidates)
    int n = 0;
    if (use_list) {
        n = (int)s_cnt;
    } else if (p.ehrenfest) {
        const int nrec = *p.cand_count;
        n = nrec < p.cand_cap ? nrec : p.cand_cap;
    }
    const int *list = use_list ? p.sel_state->list : nullptr;
    auto cidx = [&](int i) -> int { return use_list ? list[i] : i; };
    Cand first{};
    if (!BATCHED && p.ehrenfest && (use_list ? t < n : t < p.cand_cap)) first = p.cand[cidx(t)];
    if (t == 0) {
        s_step = p.counters[0];
        s_rec = p.counters[1];
        s_status = *p.status;
        s_nsel = 0;
        s_valid = use_list ? (int)s_nv : 0;
    }
    if (p.fixed) {
        // the fused kernel's kFxRows fixed-point accumulator rows (exact integer
        // sums, so the order does not matter), reduced by warp 0 alone: lane l
        // reads 16-byte chunk l % 8 of rows l / 8 and l / 8 + 4 and clears them
        // for the next step.  Chunk c < 4 is FP statistic c (low, high word),
        // chunk 4 the site and positivity counts, chunk 5 the median and
        // nonfinite counts, chunk 6 the nonfinite bits.
        static_assert(kFxRows == 8 && kFxWords == 16, "warp 0 reads 8 rows of 8 chunks");
        if (warp == 0) {
            const int c = lane & 7;
            ulonglong2 *chunks = reinterpret_cast<ulonglong2 *>(p.partials);
            const ulonglong2 w0 = chunks[lane], w1 = chunks[lane + 32];
            chunks[lane] = make_ulonglong2(0ull, 0ull);
            chunks[lane + 32] = make_ulonglong2(0ull, 0ull);
            unsigned __int128 v = 0;
            unsigned long long u0 = 0, u1 = 0;
            if (c < 4) {
                v = (((unsigned __int128)w0.y << 64) | w0.x) + (((unsigned __int128)w1.y << 64) | w1.x);
            } else if (c < 6) {
                u0 = w0.x + w1.x;
                u1 = w0.y + w1.y;
            } else if (c == 6) {
                u0 = w0.x | w1.x;
            }
#pragma unroll
            for (int o = 8; o <= 16; o <<= 1) {  // lanes holding the same chunk
                const unsigned long long lo = __shfl_xor_sync(kFull, (unsigned long long)v, o);
                const unsigned long long hi = __shfl_xor_sync(kFull, (unsigned long long)(v >> 64), o);
                const unsigned long long a0 = __shfl_xor_sync(kFull, u0, o), a1 = __shfl_xor_sync(kFull, u1, o);
                v += ((unsigned __int128)hi << 64) | lo;
                u0 = c == 6 ? (u0 | a0) : u0 + a0;
                u1 += a1;
            }
            // lanes 0..7 hold chunk totals; lanes 0..3 need the site count
            // (chunk 4) and the nonfinite bits (chunk 6)
            const unsigned long long sites = __shfl_sync(kFull, u0, 4), bits = __shfl_sync(kFull, u0, 6);
            if (lane < 4) {  // FP statistic lane
                double d = ((bits >> lane) & 1u) ? __longlong_as_double(0x7ff8000000000000LL) : fx_value(v);
                if (lane == P_MASS) d = Ar<double>::add(d, Ar<double>::mul((double)sites, (double)p.rho_ref));
                tot[lane] = d;
            } else if (lane == 4) {
                tot[P_NPOS] = (double)u1;
            } else if (lane == 5) {
                tot[P_NMED] = (double)u0;
                tot[P_NBAD] = (double)u1;
            }
        }
    } else if (warp < 2 * P_NSTAT) {
        // block partials: warps 2s and 2s+1 reduce statistic s over alternate
        // 32-row groups, in a fixed order (short FP64 dependency chains)
        const int stat = warp >> 1, half = warp & 1;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        int r = lane + 32 * half;
        for (; r + 192 < p.nblocks; r += 256) {
            v0 += p.partials[(long long)r * P_NSTAT + stat];
            v1 += p.partials[(long long)(r + 64) * P_NSTAT + stat];
            v2 += p.partials[(long long)(r + 128) * P_NSTAT + stat];
            v3 += p.partials[(long long)(r + 192) * P_NSTAT + stat];
        }
        for (; r < p.nblocks; r += 64) v0 += p.partials[(long long)r * P_NSTAT + stat];
        double v = (v0 + v1) + (v2 + v3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
        if (lane == 0) red[warp] = v;
    }
    __syncthreads();
    if (!p.fixed && t < P_NSTAT) tot[t] = red[2 * t] + red[2 * t + 1];
    __syncthreads();
    const bool small = n <= kCap;  // candidates held in shared memory
    const long long k = p.k_max;

    // candidate keys: FP64 dS(f'), written with the candidates by the step
    // kernels (sites at or below the threshold carry -1); the fused kernel
    // leaves NaN where a warp had more candidates than it keys itself, and
    // those are keyed here, one thread per candidate, with the same operations.
    // The preselected list holds keyed, valid candidates and their count.
    constexpr bool kLowPrec = !std::is_same<S, double>::value;
    if (use_list) {
        for (int i = t; i < n && small; i += kFinThreads) {
            const Cand c = !BATCHED && i == t ? first : p.cand[list[i]];
            s_key[i] = c.key;
            s_site[i] = c.site;
        }
    } else {
        for (int i = t; i < n; i += kFinThreads) {
            Cand c = !BATCHED && i == t ? first : p.cand[i];
            if constexpr (kLowPrec && Q == 9) {
                if (isnan(c.key)) c.key = key_dS9_lane<S>(key_geom(p), (const S *)p.src, c.site, p.delta_e);
            }
            // below the threshold -> -1, so that from here on a key is valid
            // exactly when its bit pattern is a positive integer (FP64 compares
            // are slow on this GPU; positive doubles order like their patterns)
            if (!(c.key > p.delta_e) && c.key != -1.0) c.key = -1.0;
            if (small) {
                s_key[i] = c.key;
                s_site[i] = c.site;
            } else {
                p.cand[i].key = c.key;
            }
        }
    }
    __syncthreads();
    auto key_of = [&](int i) -> double { return small ? s_key[i] : p.cand[cidx(i)].key; };
    auto site_of = [&](int i) -> int { return small ? s_site[i] : p.cand[cidx(i)].site; };
    if (!use_list) {
        int nv = 0;
        for (int i = t; i < n; i += kFinThreads) nv += (long long)key_bits(key_of(i)) > 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nv += __shfl_down_sync(kFull, nv, o);
        if (lane == 0 && nv) atomicAdd(&s_valid, nv);
    }
    __syncthreads();
    const int n_valid = s_valid;
    double ehr_sum = 0.0;
    const bool ehr_active = p.ehrenfest && k > 0 && n_valid > 0;  // the same for the whole block
    if (ehr_active) {
        unsigned long long kv = 0;  // threshold dS pattern
        int site_thr = 0x7fffffff;
        const bool take_all = (long long)n_valid <= k;
        // few candidates (held in shared memory, at most one per thread): each
        // thread ranks its own by counting the keys that beat it (larger dS, or
        // equal dS at a lower site) -- one pass instead of the digit passes
        const bool by_rank = !take_all && small && n <= kFinThreads;
        if (by_rank) {
            bool chosen = false;
            if (t < n) {
                const unsigned long long u = key_bits(s_key[t]);
                const int st = s_site[t];
                long long rank = 0;
                if ((long long)u > 0) {
                    for (int j = 0; j < n; ++j) {
                        const unsigned long long v = key_bits(s_key[j]);
                        rank += (long long)v > 0 && (v > u || (v == u && s_site[j] < st));
                    }
                    chosen = rank < k;
                }
            }
            if (chosen) {
                const int j = atomicAdd(&s_nsel, 1);
                if (j < p.sel_cap) p.sel[j] = cidx(t);
                if (j < kCap) s_idx[j] = t;
            }
        }
        if (!take_all && !by_rank) {
            unsigned long long prefix = 0, mask = 0;
            long long rem = k;
            for (int shift = 56; shift >= 0; shift -= 8) {
                for (int d = t; d < 256; d += kFinThreads) hist[d] = 0;
                __syncthreads();
                for (int i = t; i < n; i += kFinThreads) {
                    const double key = key_of(i);
                    const unsigned long long u = key_bits(key);
                    if ((long long)u > 0 && (u & mask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
                }
                __syncthreads();
                pick_digit(hist, rem, true, s_part, &s_digit, &s_rem);
                prefix = prefix | (s_digit << shift);
                rem = s_rem;
                mask |= 255ull << shift;
                __syncthreads();
            }
            kv = prefix;
            // among the candidates with dS == kv take the `rem` lowest sites
            unsigned sprefix = 0, smask = 0;
            for (int shift = 24; shift >= 0; shift -= 8) {
                for (int d = t; d < 256; d += kFinThreads) hist[d] = 0;
                __syncthreads();
                for (int i = t; i < n; i += kFinThreads) {
                    const double key = key_of(i);
                    const unsigned s = (unsigned)site_of(i);
                    if ((long long)key_bits(key) > 0 && key_bits(key) == kv && (s & smask) == sprefix)
                        atomicAdd(&hist[(s >> shift) & 255u], 1u);
                }
                __syncthreads();
                pick_digit(hist, rem, false, s_part, &s_digit, &s_rem);
                sprefix = sprefix | ((unsigned)s_digit << shift);
                rem = s_rem;
                smask |= 255u << shift;
                __syncthreads();
            }
            site_thr = (int)sprefix;
        }
        // compaction of the chosen candidates: candidate indices in p.sel, list
        // entries in s_idx (the first kCap)
        for (int i = t; i < n && !by_rank; i += kFinThreads) {
            const double key = key_of(i);
            const unsigned long long u = key_bits(key);
            const bool chosen = (long long)u > 0 && (take_all || u > kv || (u == kv && site_of(i) <= site_thr));
            if (chosen) {
                const int j = atomicAdd(&s_nsel, 1);
                if (j < p.sel_cap) p.sel[j] = cidx(i);
                if (j < kCap) s_idx[j] = i;
            }
        }
        __syncthreads();
        if (t == 0 && s_nsel > p.sel_cap) s_nsel = p.sel_cap;
        __syncthreads();
        const int nsel = s_nsel;
        const bool sorted = nsel <= kCap;
        if (sorted) {
            // bitonic sort of the chosen set by site index (padding sorts last).
            // The payload is s_idx (chosen list entries, -1 for padding); the
            // sort key is the site: read through s_site when the candidates are
            // held in shared memory, else copied into s_site first (then free)
            int m = 1;
            while (m < nsel) m <<= 1;
            for (int i = t; i < m; i += kFinThreads) {
                if (i >= nsel) s_idx[i] = -1;
                if (!small) s_site[i] = i < nsel ? site_of(s_idx[i]) : 0x7fffffff;
            }
            __syncthreads();
            auto skey = [&](int i) -> int {
                if (!small) return s_site[i];
                const int li = s_idx[i];
                return li >= 0 ? s_site[li] : 0x7fffffff;
            };
            for (int size = 2; size <= m; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int i = t; i < m; i += kFinThreads) {
                        const int j = i ^ stride;
                        if (j > i) {
                            const bool up = (i & size) == 0;
                            const int ki = skey(i), kj = skey(j);
                            if ((ki > kj) == up) {
                                int a = s_idx[i]; s_idx[i] = s_idx[j]; s_idx[j] = a;
                                if (!small) {
                                    s_site[i] = kj;
                                    s_site[j] = ki;
                                }
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        }
        // Ehrenfests' step at each chosen site, in site order when sorted
        for (int r = t; r < nsel; r += kFinThreads) {
            // the chosen candidate's site and key (from shared memory when
            // sorted) and its phi
            int site;
            double key, phi;
            if (sorted) {
                const int li = s_idx[r];
                site = small ? s_site[li] : s_site[r];
                key = key_of(li);
                phi = p.cand[cidx(li)].phi;
            } else {
                const Cand c = p.cand[p.sel[r]];
                site = c.site;
                key = c.key;
                phi = c.phi;
            }
            const int x = site % p.nx, y = site / p.nx;
            T g[Q], fs[Q], rho, ux, uy;
            bool write = true;
            if constexpr (std::is_same<T, float>::value) {
                // FP32 / 16-bit storage: f*(m) as g - n (the limiter with phi = 0),
                // m taken from the pass's input (the collision conserves m), so
                // mass and momentum are kept and the result is rounded once
                float drho, nq[Q];
                pull_dev<Q, S>(p, x, y, g);
                moments_dev<Q>(g, p.rho_ref, drho, rho, ux, uy);
                if (p.eq == 1) {
                    // entropic f*: from the limited state in FP64 (the stored values), the
                    // entropy the step adds, dS w.r.t. its own f*; a state whose moments
                    // have no entropic f* keeps its populations
                    double fl[Q], fsd[Q], r2, a2, b2;
#pragma unroll
                    for (int q = 0; q < Q; ++q)
                        fl[q] = Ar<double>::add((double)s2f(f[fidx(p.plane, p.pitch, q, y, x)]), p.rw[q]);
                    moments<Q, double>(fl, r2, a2, b2);
                    write = feq_any<Q>(1, r2, a2, b2, fsd);
                    if (write) {
                        const double d = rel_entropy<Q>(fl, fsd);
                        if (isfinite(d)) ehr_sum = Ar<double>::add(ehr_sum, d);
                        if constexpr (Q == 9)
                            feq_ent9_x<F1>(drho, rho, ux, uy, fs);
                        else
                            feq_ent3_dev(drho, rho, ux, fs);
                    } else {
#pragma unroll
                        for (int q = 0; q < Q; ++q) fs[q] = 0.f;
                    }
                } else {
                    feq_dev<Q>(drho, rho, ux, uy, fs);
                }
                neq_dev<Q>(g, fs, nq);
#pragma unroll
                for (int q = 0; q < Q; ++q) fs[q] = g[q] - nq[q];
            } else {
                // FP64: f*(m(f')) from the stored f', in the oracle's order
#pragma unroll
                for (int q = 0; q < Q; ++q) g[q] = s2f(f[fidx(p.plane, p.pitch, q, y, x)]);
                moments<Q, T>(g, rho, ux, uy);
                if (p.eq == 1) {
                    // entropic f*: the step adds dS of the limited state w.r.t. its own f*
                    // where the limited state's moments have no entropic f* the site keeps its populations
                    write = feq_any<Q>(1, rho, ux, uy, fs);
                    const double d = write ? rel_entropy<Q>(g, fs) : (double)NAN;
                    if (isfinite(d)) ehr_sum = Ar<double>::add(ehr_sum, d);
                } else {
                    feq<Q, T>(rho, ux, uy, fs);
                }
            }
            if (write) {
#pragma unroll
                for (int q = 0; q < Q; ++q) f[fidx(p.plane, p.pitch, q, y, x)] = f2s<S>(fs[q]);
            }
            if (p.eq != 1) ehr_sum = Ar<double>::add(ehr_sum, Ar<double>::mul(Ar<double>::mul(phi, phi), key));
        }
        __syncthreads();
        // the chosen sites, as site indices, for lbm_limited_sites
        if (sorted) {
            for (int r = t; r < nsel; r += kFinThreads) p.sel[r] = small ? s_site[s_idx[r]] : s_site[r];
        } else {
            // unsorted (more than kCap chosen): convert in place, one owner per slot
            for (int r = t; r < nsel; r += kFinThreads) p.sel[r] = p.cand[p.sel[r]].site;
        }
    }
    // thread r applied chosen site r: with at most 32 of them only warp 0
    // holds terms
    const double esum = ehr_active ? block_sum0(ehr_sum, red, s_nsel <= 32) : 0.0;
    if (t == 0) {
        long long step = s_step;
        if (p.collide) {
            step += 1;
            p.counters[0] = step;
        }
        const long long rec = s_rec;
        p.counters[1] = rec + 1;
        DevStats st;
        st.step = step;
        st.mass = tot[P_MASS];
        st.sum_dS = tot[P_SUM_DS];
        st.dS_lbgk = p.collide ? Ar<double>::mul(p.one_minus_a2, tot[P_SUM_IN]) : 0.0;
        st.dS_lim = Ar<double>::add(tot[P_DS_LIM], esum);
        st.n_pos = (long long)tot[P_NPOS];
        st.n_med = (long long)tot[P_NMED];
        st.n_ehr = s_nsel;
        st.n_cand = n_valid;
        st.n_bad = (long long)tot[P_NBAD];
        // the step kernel set its status bits before this launch began
        const unsigned sb = s_status;
        st.status = (sb & kStatNonfinite) ? 4 : ((sb & kStatTimeout) ? 5 : 0);
        st.reserved = 0;
        p.stats_ring[rec % p.ring_len] = st;
        if (p.probe != nullptr && p.collide) {
            // the control point's moments after the whole step (Ehrenfests' writes
            // are visible: the block synchronised after them), as lbm_moments
            // evaluates them
            const int x = p.probe_site % p.nx, y = p.probe_site / p.nx;
            double g[Q], r, a, b;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const S v = f[fidx(p.plane, p.pitch, q, y, x)];
                if constexpr (std::is_same<S, double>::value)
                    g[q] = v;
                else
                    g[q] = Ar<double>::add((double)s2f(v), p.rw[q]);
            }
            moments<Q, double>(g, r, a, b);
            double *slot = p.probe + 3 * ((step - 1) % p.probe_cap);
            slot[0] = r;
            slot[1] = a;
            slot[2] = b;
        }
        *p.sel_count = s_nsel;
        *p.cand_count = 0;
        if (p.work != nullptr) *p.work = 0;  // the next fused launch starts at its first item
    }
}

}  // namespace

template <typename T>
cudaError_t launch_finalize(int q, const FinalParams &p, T *f, cudaStream_t s, int grid)
{
    // programmatic dependent launch (see k_finalize); a grid is a cooperative
    // launch, so that its blocks are resident together for the grid barrier
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid > 1 ? grid : 1);
    cfg.blockDim = dim3(kFinThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeCooperative;
    attr[1].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = grid > 1 ? 2 : 1;
    FinalParams pp = p;
    if (grid <= 1) pp.sel_state = nullptr;
    const FinalArgs *none = nullptr;
    if (grid > 1) {
        if (q == 9) return cudaLaunchKernelEx(&cfg, k_finalize<9, T, false, true>, pp, f, none);
        return cudaLaunchKernelEx(&cfg, k_finalize<3, T, false, true>, pp, f, none);
    }
    if (q == 9) return cudaLaunchKernelEx(&cfg, k_finalize<9, T, false>, pp, f, none);
    return cudaLaunchKernelEx(&cfg, k_finalize<3, T, false>, pp, f, none);
}

template <typename T>
int finalize_grid(int q)
{
    int dev = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    const cudaError_t e = q == 9
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_finalize<9, T, false, true>, kFinThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_finalize<3, T, false, true>, kFinThreads, 0);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    return sm_count();
}

cudaError_t launch_finalize_batched_f32(int q, const FinalArgs *table, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const FinalParams none{};
    if (q == 9)
        k_finalize<9, float, true><<<n, kFinThreads, 0, s>>>(none, nullptr, table);
    else
        k_finalize<3, float, true><<<n, kFinThreads, 0, s>>>(none, nullptr, table);
    return cudaGetLastError();
}

template cudaError_t launch_finalize<float>(int, const FinalParams &, float *, cudaStream_t, int);
template cudaError_t launch_finalize<double>(int, const FinalParams &, double *, cudaStream_t, int);
template cudaError_t launch_finalize<__nv_bfloat16>(int, const FinalParams &, __nv_bfloat16 *, cudaStream_t, int);
template cudaError_t launch_finalize<__half>(int, const FinalParams &, __half *, cudaStream_t, int);
template int finalize_grid<float>(int);
template int finalize_grid<double>(int);
template int finalize_grid<__nv_bfloat16>(int);
template int finalize_grid<__half>(int);

}  // namespace lbm
