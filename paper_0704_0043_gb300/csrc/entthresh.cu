// entthresh.cu -- dS_0 of the threshold filter from Eq. EntThresh, on the device.
//
// Sec. 3.4: with the distribution of dS over the lattice, dS_0 solves
//     sum_s max(dS_s - dS_0, 0) = delta_0 [1 - (2 beta - 1)^2] sum_s dS_s,
// the threshold above which the homothety of Eq. entrHom acts (dS_t =
// max(dS_0, delta)).  The left side G(t) = sum_s max(dS_s - t, 0) falls
// continuously and piecewise linearly with t.  Here it is solved exactly on
// the pass's own dS values (the limit of the paper's histogram estimate), by a
// radix descent over their bit patterns (for values >= 0, the bits order as
// the values do): at each level a histogram pass counts and sums the values
// of each 8-bit digit within the current bin, and one block evaluates G at
// the bins' lower edges, G(e) = S(>= e) - m(>= e) e, and keeps the highest bin
// whose lower edge still has G >= rhs.  After the last digit the bin is a
// single value e with G(e) >= rhs > G(next value), and
//     dS_0 = (S - rhs) / m,  S, m = sum and count of the values above e,
// exactly as the sorted formulation gives.  Values of sites that are flagged
// or not finite are 0 in the field (they add nothing to G for t >= 0).
#include <cmath>

#include "internal.h"

namespace lbm {
namespace {

template <typename T> struct Bits;
template <> struct Bits<float> {
    using U = unsigned;
    static constexpr int kBits = 32;
    static __device__ __forceinline__ U of(float v) { return __float_as_uint(v); }
    static __device__ __forceinline__ double val(U u) { return (double)__uint_as_float(u); }
};
template <> struct Bits<double> {
    using U = unsigned long long;
    static constexpr int kBits = 64;
    static __device__ __forceinline__ U of(double v) { return (U)__double_as_longlong(v); }
    static __device__ __forceinline__ double val(U u) { return __longlong_as_double((long long)u); }
};

// The right side of Eq. EntThresh from the ensemble reduction's sum and count,
// and the special cases of the sorted solve: no value or rhs <= 0 (dS_0 = +inf:
// nothing is limited), and rhs >= sum dS (dS_0 = 0).
__global__ void k_ent_init(const double *ens, double a, double delta0, double t_delta, EntState *st)
{
    const int d = threadIdx.x;
    st->cnt[d] = 0ull;
    st->sum[d] = 0.0;
    if (d != 0) return;
    const double sum = ens[2], count = ens[3];
    const double rhs = delta0 * ((1.0 - a * a) * sum);
    st->rhs = rhs;
    st->s_above = 0.0;
    st->m_above = 0ull;
    st->prefix = 0ull;
    st->done = 0;
    if (count <= 0.0 || !(rhs > 0.0)) {
        st->t = count > 0.0 ? (double)INFINITY : (t_delta > 0.0 ? t_delta : 0.0);
        st->done = 1;
    } else if (rhs >= sum) {
        st->t = t_delta > 0.0 ? t_delta : 0.0;
        st->done = 1;
    }
}

// Histogram of the digit at `shift` among the values whose higher bits equal
// st->prefix, added into st->cnt / st->sum.  dS spans few binades, so at the
// upper levels most values fall into a few crowded bins, where per-value
// atomics would queue on the same addresses.  Instead a warp takes 32
// consecutive values at a time and, for each distinct digit among them (one
// or two, as a rule), adds the lanes holding it (count by ballot, sum by a
// warp reduction) into its own shared histogram, with no atomic; the block
// then adds its warps' bins into the global ones.
template <typename T>
__global__ void __launch_bounds__(256) k_ent_hist(const T *__restrict__ field, long long n, int shift, EntState *st)
{
    using B = Bits<T>;
    using U = typename B::U;
    constexpr int kW = 8;
    __shared__ unsigned cnt[kW][256];
    __shared__ double sum[kW][256];
    if (st->done) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kW * 256; i += 256) {
        (&cnt[0][0])[i] = 0u;
        (&sum[0][0])[i] = 0.0;
    }
    __syncthreads();
    const U prefix = (U)st->prefix;
    const int hi = shift + 8;  // bits above the digit
    const long long stride = (long long)gridDim.x * 256;
    for (long long s0 = blockIdx.x * 256LL + warp * 32; s0 < n; s0 += stride) {
        const long long s = s0 + lane;
        unsigned d = 256u;  // no value
        T v = T(0);
        if (s < n) {
            v = field[s];
            if (v > T(0)) {  // zeros (and excluded sites) add nothing for t >= 0
                const U u = B::of(v);
                if (hi >= B::kBits || ((u ^ prefix) >> hi) == 0) d = (unsigned)((u >> shift) & 255u);
            }
        }
        // the distinct digits of the 32 values, smallest first
        unsigned left = __ballot_sync(0xffffffffu, d < 256u);
        while (left) {
            const unsigned dd = __reduce_min_sync(0xffffffffu, (left >> lane) & 1u ? d : 256u);
            const unsigned mine = __ballot_sync(0xffffffffu, d == dd);
            T x = d == dd ? v : T(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) {
                cnt[warp][dd] += (unsigned)__popc(mine);
                sum[warp][dd] += (double)x;
            }
            left &= ~mine;
        }
    }
    __syncthreads();
    const int d = threadIdx.x;
    unsigned c = 0u;
    double sm = 0.0;
#pragma unroll
    for (int w = 0; w < kW; ++w) {
        c += cnt[w][d];
        sm += sum[w][d];
    }
    if (c) {
        atomicAdd(&st->cnt[d], (unsigned long long)c);
        atomicAdd(&st->sum[d], sm);
    }
}

// One block of 256 threads: G at the lower edge of each bin d of the current
// level, G(d) = S_above + sum_{d' >= d} S_d' - (m_above + sum_{d' >= d} m_d') e_d,
// falls with d; the bin kept is the highest d with G(d) >= rhs.  The histogram
// is cleared for the next level; the last level writes dS_t.
template <typename T>
__global__ void __launch_bounds__(256) k_ent_decide(int shift, int last, double t_delta, EntState *st)
{
    using B = Bits<T>;
    using U = typename B::U;
    __shared__ double ssum[256];
    __shared__ unsigned long long scnt[256];
    __shared__ double wsum[8];
    __shared__ unsigned long long wcnt[8];
    __shared__ int s_keep;
    if (st->done) return;
    const int d = threadIdx.x;
    // suffix sums over the bins above and including each bin, in a fixed order:
    // thread r scans bin 255 - r, a warp-shuffle prefix scan per warp, then the
    // totals of the warps before it
    {
        const int r = d, lane = r & 31, w = r >> 5;
        double v = st->sum[255 - r];
        unsigned long long c = st->cnt[255 - r];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, v, o);
            const unsigned long long yc = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) {
                v += y;
                c += yc;
            }
        }
        if (lane == 31) {
            wsum[w] = v;
            wcnt[w] = c;
        }
        __syncthreads();
        for (int j = 0; j < w; ++j) {
            v += wsum[j];
            c += wcnt[j];
        }
        ssum[255 - r] = v;
        scnt[255 - r] = c;
    }
    __syncthreads();
    const U prefix = (U)st->prefix;
    const double e = B::val(prefix | ((U)d << shift));
    const double S = st->s_above + ssum[d];
    const unsigned long long m = st->m_above + scnt[d];
    const bool ok = S - (double)m * e >= st->rhs;
    const int n_ok = __syncthreads_count(ok);  // G falls with d: the bins 0 .. n_ok - 1 qualify
    if (d == 0) s_keep = n_ok > 0 ? n_ok - 1 : 0;
    __syncthreads();
    const int keep = s_keep;
    if (d == 0) {
        // the values above the kept bin move into the running sum and count
        if (keep < 255) {
            st->s_above += ssum[keep + 1];
            st->m_above += scnt[keep + 1];
        }
        st->prefix = (unsigned long long)(prefix | ((U)keep << shift));
        if (last) {
            double t = st->m_above > 0 ? (st->s_above - st->rhs) / (double)st->m_above : 0.0;
            if (!(t > 0.0)) t = 0.0;
            st->t = t > t_delta ? t : t_delta;
        }
    }
    st->cnt[d] = 0ull;
    st->sum[d] = 0.0;
}

}  // namespace

template <typename T>
cudaError_t launch_entthresh(const StepParams &p, double delta0, long long n, cudaStream_t s)
{
    constexpr int bits = Bits<T>::kBits;
    k_ent_init<<<1, 256, 0, s>>>(p.ens, p.a, delta0, p.threshold_delta, p.ent);
    long long blocks = (n + 255) / 256;
    if (blocks > 4 * 152) blocks = 4 * 152;
    if (blocks < 1) blocks = 1;
    for (int shift = bits - 8; shift >= 0; shift -= 8) {
        k_ent_hist<T><<<(int)blocks, 256, 0, s>>>((const T *)p.ent_field, n, shift, p.ent);
        k_ent_decide<T><<<1, 256, 0, s>>>(shift, shift == 0, p.threshold_delta, p.ent);
    }
    return cudaGetLastError();
}

int entthresh_launches(bool fp64) { return 1 + 2 * (fp64 ? 8 : 4); }

template cudaError_t launch_entthresh<float>(const StepParams &, double, long long, cudaStream_t);
template cudaError_t launch_entthresh<double>(const StepParams &, double, long long, cudaStream_t);

}  // namespace lbm
