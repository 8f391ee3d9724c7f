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
// The kernel is one block and sits between two step launches, so it is built
// for latency: the candidates arrive with their FP64 keys (the step kernels
// evaluate them where they find them), up to kCap of them are kept in shared
// memory, and sums use warp shuffles or exact integer arithmetic.
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

// BATCHED: block b finishes instance b of `table`; otherwise the single (p0, f0).
template <int Q, typename S, bool BATCHED>
__global__ void __launch_bounds__(kFinThreads, BATCHED ? 2 : 1) k_finalize(const FinalParams p0, S *__restrict__ f0,
                                                          const FinalArgs *__restrict__ table)
{
    using T = compute_t<S>;
    // Launched as a programmatic dependent of the step kernel: wait for it to
    // finish before any memory access, then let the next step kernel be
    // scheduled early.  Both are no-ops in an ordinary launch.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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
    __shared__ double s_key[kCap];
    __shared__ int s_site[kCap];
    __shared__ int s_idx[kCap];
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_part[8], s_digit;
    __shared__ unsigned long long s_prefix;
    __shared__ long long s_rem, s_step, s_rec;
    __shared__ int s_n, s_nsel, s_valid;
    __shared__ unsigned s_status;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    if (t == 0) {
        const int nrec = p.ehrenfest ? *p.cand_count : 0;
        s_n = nrec < p.cand_cap ? nrec : p.cand_cap;
        s_step = p.counters[0];
        s_rec = p.counters[1];
        s_status = *p.status;
        s_nsel = 0;
        s_valid = 0;
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
    const int n = s_n;
    const bool small = n <= kCap;  // candidates held in shared memory
    const long long k = p.k_max;

    // candidate keys: FP64 dS(f'), written with the candidates by the step
    // kernels (sites at or below the threshold carry -1); the fused kernel
    // leaves NaN where a warp had more candidates than it keys itself, and
    // those are keyed here, one thread per candidate, with the same operations
    constexpr bool kLowPrec = !std::is_same<S, double>::value;
    for (int i = t; i < n; i += kFinThreads) {
        Cand c = p.cand[i];
        if constexpr (kLowPrec && Q == 9) {
            if (isnan(c.key)) {
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
                c.key = key_dS9_lane<S>(kg, (const S *)p.src, c.site, p.delta_e);
            }
        }
        // below the threshold -> -1, so that from here on a key is valid
        // exactly when its bit pattern is a positive integer (FP64 compares
        // are slow on this GPU; positive doubles order like their patterns)
        if (!(c.key > p.delta_e) && c.key != -1.0) c.key = -1.0;
        if (!small || isnan(p.cand[i].key)) p.cand[i].key = c.key;
        if (small) {
            s_key[i] = c.key;
            s_site[i] = c.site;
        }
    }
    __syncthreads();
    auto key_of = [&](int i) -> double { return small ? s_key[i] : p.cand[i].key; };
    auto site_of = [&](int i) -> int { return small ? s_site[i] : p.cand[i].site; };
    {
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
                if (j < p.sel_cap) p.sel[j] = t;
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
        // compaction of the chosen candidates (indices into the candidate list)
        for (int i = t; i < n && !by_rank; i += kFinThreads) {
            const double key = key_of(i);
            const unsigned long long u = key_bits(key);
            const bool chosen = (long long)u > 0 && (take_all || u > kv || (u == kv && site_of(i) <= site_thr));
            if (chosen) {
                const int j = atomicAdd(&s_nsel, 1);
                if (j < p.sel_cap) p.sel[j] = i;
            }
        }
        __syncthreads();
        if (t == 0 && s_nsel > p.sel_cap) s_nsel = p.sel_cap;
        __syncthreads();
        const int nsel = s_nsel;
        const bool sorted = nsel <= kCap;
        if (sorted) {
            // bitonic sort of the chosen set by site index (padding sorts last);
            // the candidate arrays are no longer read, so they hold the sort keys
            int m = 1;
            while (m < nsel) m <<= 1;
            for (int i = t; i < m; i += kFinThreads) {
                const int ci = i < nsel ? p.sel[i] : -1;
                s_idx[i] = ci;
                s_key[i] = (double)(ci >= 0 ? p.cand[ci].site : 0x7fffffff);
            }
            __syncthreads();
            for (int i = t; i < m; i += kFinThreads) s_site[i] = (int)s_key[i];
            __syncthreads();
            for (int size = 2; size <= m; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int i = t; i < m; i += kFinThreads) {
                        const int j = i ^ stride;
                        if (j > i) {
                            const bool up = (i & size) == 0;
                            if ((s_site[i] > s_site[j]) == up) {
                                int a = s_site[i]; s_site[i] = s_site[j]; s_site[j] = a;
                                a = s_idx[i]; s_idx[i] = s_idx[j]; s_idx[j] = a;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        }
        // Ehrenfests' step at each chosen site, in site order when sorted
        for (int r = t; r < nsel; r += kFinThreads) {
            const int ci = sorted ? s_idx[r] : p.sel[r];
            const Cand c = p.cand[ci];
            const int x = c.site % p.nx, y = c.site / p.nx;
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
            if (p.eq != 1) ehr_sum = Ar<double>::add(ehr_sum, Ar<double>::mul(Ar<double>::mul(c.phi, c.phi), c.key));
        }
        __syncthreads();
        // the chosen sites, as site indices, for lbm_limited_sites
        if (sorted) {
            for (int r = t; r < nsel; r += kFinThreads) p.sel[r] = s_site[r];
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
cudaError_t launch_finalize(int q, const FinalParams &p, T *f, cudaStream_t s)
{
    // programmatic dependent launch (see k_finalize)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(kFinThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const FinalArgs *none = nullptr;
    if (q == 9) return cudaLaunchKernelEx(&cfg, k_finalize<9, T, false>, p, f, none);
    return cudaLaunchKernelEx(&cfg, k_finalize<3, T, false>, p, f, none);
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

template cudaError_t launch_finalize<float>(int, const FinalParams &, float *, cudaStream_t);
template cudaError_t launch_finalize<double>(int, const FinalParams &, double *, cudaStream_t);
template cudaError_t launch_finalize<__nv_bfloat16>(int, const FinalParams &, __nv_bfloat16 *, cudaStream_t);
template cudaError_t launch_finalize<__half>(int, const FinalParams &, __half *, cudaStream_t);

}  // namespace lbm
