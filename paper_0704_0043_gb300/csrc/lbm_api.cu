// lbm_api.cu -- the C ABI of liblbm (include/lbm.h): context, validation,
// device memory ownership, transfers and the per-step launch sequence.
//
// A step is two stream-ordered launches: the step kernel (free flight,
// collision, dS, positivity and median limiters, Ehrenfests' candidates,
// block partial sums; Eq. lbgkLB and Sec. 3) writing the other population
// buffer, then the one-block tail (fixed-order FP64 sums, Ehrenfests' step,
// stats record).  The two buffers swap roles every step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lbm.h"
#include "internal.h"
#include "lattice.cuh"

using namespace lbm;

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_ctx *c, lbm_status s, const std::string &msg)
{
    if (c)
        c->err = msg;
    else
        g_err = msg;
    return s;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + " failed: " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
}

#define CK(c, call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

int lattice_q(int lattice) { return lattice == LBM_D1Q3 ? 3 : 9; }

// Calls fn with a null pointer of the context's storage type.
template <typename F>
cudaError_t with_storage(int precision, F &&fn)
{
    switch (precision) {
    case LBM_FP64: return fn((double *)nullptr);
    case LBM_FP32: return fn((float *)nullptr);
    case LBM_BF16: return fn((__nv_bfloat16 *)nullptr);
    default: return fn((__half *)nullptr);
    }
}
#define STORAGE_T typename std::remove_pointer<decltype(tag)>::type

bool fused_applies(const lbm_config &c)
{
    return c.lattice == LBM_D2Q9 && c.precision != LBM_FP64 && c.boundary == LBM_BC_WALLS &&
           c.kernel != LBM_KERNEL_TILED && fused_d2q9_fits((long long)c.ny * row_pitch(c.nx));
}

std::string validate(const lbm_config *c)
{
    if (!c) return "config is NULL";
    if (c->lattice != LBM_D1Q3 && c->lattice != LBM_D2Q9) return "lattice must be LBM_D1Q3 or LBM_D2Q9";
    if (c->nx < 1 || c->ny < 1) return "nx and ny must be >= 1";
    if ((long long)c->nx * c->ny > 0x7fffffffLL) return "nx * ny must fit a 32-bit site index";
    if (c->precision < LBM_FP64 || c->precision > LBM_FP16)
        return "precision must be LBM_FP64, LBM_FP32, LBM_BF16 or LBM_FP16";
    if (c->lattice == LBM_D1Q3) {
        if (c->ny != 1) return "D1Q3 needs ny == 1";
        if (c->boundary != LBM_BC_WALLS && c->boundary != LBM_BC_PERIODIC)
            return "D1Q3 boundary must be LBM_BC_WALLS or LBM_BC_PERIODIC";
        if (c->boundary == LBM_BC_WALLS && c->nx < 3) return "D1Q3 with closed ends needs nx >= 3";
    } else {
        if (c->boundary < LBM_BC_WALLS || c->boundary > LBM_BC_DIFFUSIVE) return "unknown boundary kind";
        if (c->boundary == LBM_BC_WALLS && (c->nx < 2 || c->ny < 2)) return "D2Q9 cavity needs nx, ny >= 2";
        if (c->boundary >= LBM_BC_NODE_WALLS && (c->nx < 5 || c->ny < 5))
            return "D2Q9 cavity with boundary nodes needs nx, ny >= 5";
        if (c->boundary == LBM_BC_CHANNEL && c->ny < 2) return "D2Q9 channel needs ny >= 2";
    }
    if (c->limiters & ~63u) return "unknown limiter bits";
    if (!(c->smooth_delta >= 0.0) || !std::isfinite(c->smooth_delta)) return "smooth_delta must be finite and >= 0";
    if (!(c->smooth_k > 0.0) || !std::isfinite(c->smooth_k)) return "smooth_k must be finite and > 0";
    if (!(c->threshold_c >= 0.0) || !std::isfinite(c->threshold_c)) return "threshold_c must be finite and >= 0";
    if (!(c->threshold_delta >= 0.0) || !std::isfinite(c->threshold_delta))
        return "threshold_delta must be finite and >= 0";
    if (!(c->beta >= 0.0 && c->beta <= 1.0)) return "beta must lie in [0, 1]";
    if (!std::isfinite(c->u_lid) || !std::isfinite(c->rho_wall)) return "u_lid and rho_wall must be finite";
    if (!(c->delta_median >= 0.0) || !(c->delta_ehrenfest >= 0.0)) return "delta_median and delta_ehrenfest must be >= 0";
    if (c->k_max < 0) return "k_max must be >= 0";
    if (c->median_mode != LBM_MEDIAN_THRESHOLD && c->median_mode != LBM_MEDIAN_GATE) return "unknown median_mode";
    if (c->kernel < LBM_KERNEL_AUTO || c->kernel > LBM_KERNEL_TUBE) return "unknown kernel";
    if (c->equilibrium != LBM_EQ_POLYNOMIAL && c->equilibrium != LBM_EQ_ENTROPIC) return "unknown equilibrium";

    if (c->kernel == LBM_KERNEL_FUSED && !fused_applies(*c))
        return "LBM_KERNEL_FUSED needs D2Q9, FP32/BF16/FP16 storage and LBM_BC_WALLS";
    if (c->kernel == LBM_KERNEL_TUBE && !tube_applies(*c, c->limiters))
        return "LBM_KERNEL_TUBE needs D1Q3, FP32 or FP64 storage and no ensemble-dependent limiter";
    if (c->collision != LBM_COLL_LBGK && c->collision != LBM_COLL_ELBM) return "unknown collision";
    if (c->collision == LBM_COLL_ELBM && (c->equilibrium != LBM_EQ_ENTROPIC || c->precision != LBM_FP64))
        return "ELBM needs entropic quasiequilibria (LBM_EQ_ENTROPIC) and LBM_FP64 storage";
    if (c->phi_rule != LBM_PHI_HOMOTHETY && c->phi_rule != LBM_PHI_ENTROPY) return "unknown phi_rule";
    if (c->phi_rule == LBM_PHI_ENTROPY && (c->equilibrium != LBM_EQ_ENTROPIC || c->precision != LBM_FP64))
        return "LBM_PHI_ENTROPY needs entropic quasiequilibria (LBM_EQ_ENTROPIC) and LBM_FP64 storage";
    if (!(c->entthresh_delta0 >= 0.0) || !std::isfinite(c->entthresh_delta0))
        return "entthresh_delta0 must be finite and >= 0";
    if (c->stats_history < 0) return "stats_history must be >= 0";
    if (!(c->rho_ref > 0.0) || !std::isfinite(c->rho_ref)) return "rho_ref must be finite and > 0";
    return "";
}

size_t ens_bytes()
{
    static_assert(kEnsDoubles >= kEnsFxOffset + kFxRows * kFxWords + 1, "fused E(dS) rows and counter");
    return (size_t)kEnsDoubles * sizeof(double);
}

// E(dS) of a pass by the fused kernel's row streaming: FP32 D2Q9 halfway-wall
// lattices, collision passes (whatever kernel the step itself runs on, so that
// the fused and the tiled step see the same E)
bool epass_applies(const lbm_config &c, int collide)
{
    return collide && c.lattice == LBM_D2Q9 && c.precision == LBM_FP32 && c.boundary == LBM_BC_WALLS &&
           fused_d2q9_fits((long long)c.ny * row_pitch(c.nx));
}
size_t fx_bytes() { return (size_t)kFxRows * kFxWords * sizeof(unsigned long long); }

struct Sizes {
    int q, pitch;
    long long plane;
    size_t elem, field, cand, sel, partials, ring, ent, selstate;
    int cand_cap, sel_cap, rows, ring_len;
    int64_t total() const
    {
        return (int64_t)(2 * field + cand + sel + partials + ring + ens_bytes() + ent + selstate +
                         64 * sizeof(long long) +
                         (size_t)chunks_for(rows) * sizeof(unsigned) + 4096);
    }
};

Sizes sizes_for(const lbm_config &c)
{
    Sizes z{};
    z.q = lattice_q(c.lattice);
    z.pitch = row_pitch(c.nx);
    z.plane = (long long)c.ny * z.pitch;
    z.elem = c.precision == LBM_FP64 ? 8 : (c.precision == LBM_FP32 ? 4 : 2);
    z.field = (size_t)z.q * (size_t)z.plane * z.elem;
    const long long n = (long long)c.nx * c.ny;
    z.cand_cap = (c.limiters & LBM_LIM_EHRENFEST) ? (int)n : 1;
    z.cand = (size_t)z.cand_cap * sizeof(Cand);
    z.selstate = (c.limiters & LBM_LIM_EHRENFEST) && n >= kSelMinSites ? sizeof(SelState) : 0;
    z.sel_cap = (int)std::max<long long>(1, std::min<long long>(c.k_max, n));
    z.sel = (size_t)z.sel_cap * sizeof(int);
    // [fused accumulator rows][tiled block rows][chunk rows]
    z.rows = tiled_blocks_for(z.q, c.nx, c.ny);
    if (z.q == 3) z.rows = std::max(z.rows, tube_blocks(c.precision == LBM_FP64, c.nx));
    z.partials = fx_bytes() + (size_t)(z.rows + chunks_for(z.rows)) * P_NSTAT * sizeof(double);
    z.ring_len = std::max(1, c.stats_history);
    z.ring = (size_t)z.ring_len * sizeof(DevStats);
    // Eq. EntThresh: the pass's dS field (compute precision) and the solve's state
    z.ent = (c.limiters & LBM_LIM_ENTTHRESH)
                ? (size_t)n * (c.precision == LBM_FP64 ? sizeof(double) : sizeof(float)) + sizeof(EntState)
                : 0;
    return z;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

lbm_status ensure_stage(lbm_ctx *c, size_t bytes)
{
    if (c->stage_bytes >= bytes) return LBM_OK;
    if (c->stage) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->stage);
        c->device_bytes -= (int64_t)c->stage_bytes;
        c->stage = nullptr;
        c->stage_bytes = 0;
    }
    CK(c, cudaMalloc(&c->stage, bytes));
    c->stage_bytes = bytes;
    c->device_bytes += (int64_t)bytes;
    return LBM_OK;
}

// Device-side view of a caller array of `count` doubles: the pointer itself
// when it is device memory, else the staging buffer at element offset `off`
// (filled from the host for inputs).
lbm_status dev_in(lbm_ctx *c, const double *src, size_t count, size_t off, const double **out)
{
    if (is_device_ptr(src)) {
        *out = src;
        return LBM_OK;
    }
    CK(c, cudaMemcpyAsync(c->stage + off, src, count * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    *out = c->stage + off;
    return LBM_OK;
}

StepParams step_params(lbm_ctx *c, int collide, unsigned limiters)
{
    StepParams p = cfg_step_params(c->cfg, c->q, c->pitch, c->plane, collide, limiters);
    p.cand = c->cand;
    p.cand_count = c->counts;
    p.cand_cap = c->cand_cap;
    p.fx_rows = reinterpret_cast<unsigned long long *>(c->partials);
    p.partials = c->partials + fx_bytes() / sizeof(double);
    p.partials2 = p.partials + (size_t)c->partial_rows * P_NSTAT;
    p.chunk_cnt = c->chunk_cnt;
    p.status = c->status;
    p.work = c->counts + 2;
    p.ens = c->ens + 2 * kEnsBlocks;
    p.ent_field = (limiters & LBM_LIM_ENTTHRESH) ? c->ent_field : nullptr;
    p.ent = c->ent;
    return p;
}

FinalParams final_params(lbm_ctx *c, int collide, unsigned limiters, int nblocks)
{
    const StepParams p = step_params(c, collide, limiters);
    // the tiled kernel's chunk rows (the fused path points the tail at its accumulator rows)
    FinalParams f = cfg_final_params(c->cfg, p, collide, limiters, chunks_for(nblocks));
    f.partials = p.partials2;
    f.cand = c->cand;
    f.cand_count = c->counts;
    f.cand_cap = c->cand_cap;
    f.sel = c->sel;
    f.sel_cap = c->sel_cap;
    f.sel_count = c->counts + 1;
    f.status = c->status;
    f.stats_ring = c->ring;
    f.ring_len = c->ring_len;
    f.counters = c->counters;
    f.src = c->buf[c->cur];
    f.probe = c->probe_site >= 0 ? c->probe : nullptr;
    f.probe_cap = c->probe_cap;
    f.probe_site = c->probe_site;
    return f;
}

// Next event of the timing record (created on first use).
lbm_status next_event(lbm_ctx *c, cudaEvent_t *ev)
{
    if (c->events_used == c->events.size()) {
        cudaEvent_t e;
        CK(c, cudaEventCreate(&e));
        c->events.push_back(e);
    }
    *ev = c->events[c->events_used++];
    return LBM_OK;
}

lbm_status mark(lbm_ctx *c)
{
    if (!c->timing || !c->timing_now) return LBM_OK;
    cudaEvent_t ev;
    lbm_status s = next_event(c, &ev);
    if (s != LBM_OK) return s;
    CK(c, cudaEventRecord(ev, c->stream));
    return LBM_OK;
}

// One pass (step or limiter pass) from buf[cur] into buf[cur ^ 1].
lbm_status run_pass(lbm_ctx *c, int collide, unsigned limiters)
{
    // timing samples every timing_every-th pass (the events between kernels
    // would otherwise also cost every pass their gap)
    c->timing_now = c->timing && (c->timing_every <= 1 || c->timing_pass++ % c->timing_every == 0);
    lbm_status ms = mark(c);
    if (ms != LBM_OK) return ms;
    StepParams p = step_params(c, collide, limiters);
    int nblocks = 0;
    cudaError_t e;
    void *src = c->buf[c->cur], *dst = c->buf[c->cur ^ 1];
    const bool fused = collide && fused_applies(c->cfg);
    const bool tube = tube_applies(c->cfg, limiters);
    bool chunked = true;
    if (limiters & kLimEnsemble) {
        // E(dS) of this pass, before any site is limited
        if (epass_applies(c->cfg, collide)) {
            StepParams pe = p;
            pe.fx_rows = reinterpret_cast<unsigned long long *>(c->ens + kEnsFxOffset);
            pe.work = reinterpret_cast<int *>(c->ens + kEnsFxOffset + kFxRows * kFxWords);
            e = launch_fused_epass<float>(pe, (const float *)src, c->stream);
        } else {
            e = with_storage(c->cfg.precision, [&](auto tag) -> cudaError_t {
                using S = STORAGE_T;
                return launch_ens_mean<S>(c->q, p, (const S *)src, c->ens, c->stream);
            });
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "ensemble reduction launch");
        c->launches += 2;
        if (limiters & LBM_LIM_ENTTHRESH) {
            // dS_0 of Eq. EntThresh on the field the reduction wrote
            const long long n = (long long)c->cfg.nx * c->cfg.ny;
            const bool fp64 = c->cfg.precision == LBM_FP64;
            e = fp64 ? launch_entthresh<double>(p, c->cfg.entthresh_delta0, n, c->stream)
                     : launch_entthresh<float>(p, c->cfg.entthresh_delta0, n, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "EntThresh launch");
            c->launches += entthresh_launches(fp64);
        }
    }
    e = with_storage(c->cfg.precision, [&](auto tag) -> cudaError_t {
        using S = STORAGE_T;
        if constexpr (!std::is_same<S, double>::value)
            if (fused) return launch_fused_d2q9<S>(p, (const S *)src, (S *)dst, &nblocks, c->stream);
        if constexpr (std::is_same<S, double>::value || std::is_same<S, float>::value)
            if (tube) return launch_tube<S>(p, (const S *)src, (S *)dst, &nblocks, &chunked, c->stream);
        return launch_tiled<S>(c->q, p, (const S *)src, (S *)dst, &nblocks, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
    if ((ms = mark(c)) != LBM_OK) return ms;
    FinalParams f = final_params(c, collide, limiters, nblocks);
    f.fixed = fused ? 1 : 0;
    if (fused) f.partials = c->partials;  // the fixed-point accumulator rows
    if (!chunked) {                        // a short tube: the tail reads the block rows
        f.partials = p.partials;
        f.nblocks = nblocks;
    }
    f.work = fused ? c->counts + 2 : nullptr;
    // the tail: a cooperative grid when the context has one (it preselects
    // dense Ehrenfests' candidates); a graph capture keeps the one-block tail.
    // A device that refuses the cooperative launch keeps the one-block tail
    // from then on.
    const int grid = (c->sel_state && !c->capturing) ? c->fin_grid : 1;
    f.sel_state = c->sel_state;
    e = with_storage(c->cfg.precision, [&](auto tag) -> cudaError_t {
        using S = STORAGE_T;
        cudaError_t le = launch_finalize<S>(c->q, f, (S *)dst, c->stream, grid);
        if (le != cudaSuccess && grid > 1) {
            cudaGetLastError();
            c->fin_grid = 0;
            le = launch_finalize<S>(c->q, f, (S *)dst, c->stream, 1);
        }
        return le;
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernel launch");
    if ((ms = mark(c)) != LBM_OK) return ms;
    c->launches += 2;
    c->cur ^= 1;
    return LBM_OK;
}

lbm_status read_status(lbm_ctx *c, bool clear)
{
    unsigned s = 0;
    CK(c, cudaMemcpyAsync(&s, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (clear && s) CK(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    if (s & kStatNonfinite) return fail(c, LBM_ERR_NONFINITE, "a site had rho <= 0, f*_k <= 0 or a nonfinite value");
    if (s & kStatTimeout) return fail(c, LBM_ERR_TIMEOUT, "a bounded device wait gave up");
    if (s & kStatCandOverflow) return fail(c, LBM_ERR_CUDA, "Ehrenfests' candidate buffer overflowed");
    return LBM_OK;
}

lbm_status reset_counters(lbm_ctx *c)
{
    CK(c, cudaMemsetAsync(c->counters, 0, 2 * sizeof(long long), c->stream));
    CK(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    CK(c, cudaMemsetAsync(c->counts, 0, 4 * sizeof(int), c->stream));
    if (fused_applies(c->cfg))  // the fused kernel's fixed-point accumulators
        CK(c, cudaMemsetAsync(c->partials, 0, fx_bytes(), c->stream));
    CK(c, cudaMemsetAsync(c->ring, 0, (size_t)c->ring_len * sizeof(DevStats), c->stream));
    if (c->sel_state)  // histograms, barrier and counts (a timed-out pass may leave them set)
        CK(c, cudaMemsetAsync(c->sel_state, 0, offsetof(SelState, list), c->stream));
    return LBM_OK;
}

void drop_graphs(lbm_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
        c->gexec[k] = nullptr;
    }
}

// Captures graph_steps passes starting from buffer c->cur into c->gexec[c->cur]
// (the kernels record the buffers they read and write, so a graph is valid for
// one starting buffer; an even step count leaves the context where it began).
lbm_status capture_graph(lbm_ctx *c)
{
    if (!c->gstream) {
        CK(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        CK(c, cudaEventCreateWithFlags(&c->gev, cudaEventDisableTiming));
    }
    const int start = c->cur;
    cudaStream_t user = c->stream;
    c->stream = c->gstream;
    c->capturing = true;
    cudaGraph_t g = nullptr;
    const long long launches = c->launches;
    cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
    lbm_status s = LBM_OK;
    if (e == cudaSuccess) {
        for (int i = 0; i < c->graph_steps && s == LBM_OK; ++i) s = run_pass(c, 1, c->cfg.limiters);
        const cudaError_t ee = cudaStreamEndCapture(c->gstream, &g);
        if (e == cudaSuccess) e = ee;
    }
    c->stream = user;
    c->capturing = false;
    c->cur = start;
    c->graph_launches = c->launches - launches;
    c->launches = launches;
    if (s != LBM_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return s != LBM_OK ? s : cuda_fail(c, e, "graph capture of the step");
    }
    e = cudaGraphInstantiate(&c->gexec[start], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec[start] = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    return LBM_OK;
}

void free_all(lbm_ctx *c)
{
    drop_graphs(c);
    if (c->gev) cudaEventDestroy(c->gev);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    c->events.clear();
    void *ptrs[] = {c->buf[0], c->buf[1], c->cand, c->counts, c->sel, c->partials, c->chunk_cnt,
                    c->status, c->ring, c->counters, c->stage, c->ens, c->probe, c->ent_field, c->ent,
                    c->sel_state};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

void to_public(const DevStats &d, lbm_step_stats *o)
{
    o->step = d.step;
    o->mass = d.mass;
    o->sum_dS = d.sum_dS;
    o->dS_lbgk = d.dS_lbgk;
    o->dS_lim = d.dS_lim;
    o->n_pos = d.n_pos;
    o->n_med = d.n_med;
    o->n_ehr = d.n_ehr;
    o->n_cand = d.n_cand;
    o->n_bad = d.n_bad;
    o->status = d.status;
    o->reserved = 0;
}

}  // namespace

namespace lbm {
StepParams cfg_step_params(const lbm_config &g, int q, int pitch, long long plane, int collide, unsigned limiters)
{
    StepParams p{};
    p.nx = g.nx;
    p.ny = g.ny;
    p.pitch = pitch;
    p.plane = plane;
    p.boundary = g.boundary;
    p.limiters = limiters;
    p.median_mode = g.median_mode;
    p.collide = collide;
    p.eq = g.equilibrium == LBM_EQ_ENTROPIC ? 1 : 0;
    p.a = 2.0 * g.beta - 1.0;
    p.delta_m = g.delta_median;
    p.delta_e = g.delta_ehrenfest;
    p.u_lid = g.u_lid;
    p.beta = g.beta;
    p.coll = g.collision;
    p.phi_rule = g.phi_rule;
    for (int k = 0; k < 9; ++k) {
        const bool lid = q == 9 && g.boundary != LBM_BC_PERIODIC && Lat<9>::cy(k) == -1;
        p.lid[k] = lid ? ((6.0 * Lat<9>::w(k)) * g.rho_wall) * ((double)Lat<9>::cx(k) * g.u_lid) : 0.0;
        p.lidf[k] = (float)p.lid[k];
        p.lidlo[k] = (float)(p.lid[k] - (double)p.lidf[k]);
    }
    p.rho_ref = (float)g.rho_ref;
    for (int k = 0; k < 9; ++k) {
        // offsets of the deviation storage (FP32 / BF16 / FP16); FP64 storage holds f
        // itself and never reads them
        const double w = q == 9 ? Lat<9>::w(k) : (k < 3 ? Lat<3>::w(k) : 0.0);
        p.rw[k] = g.rho_ref * w;
        p.rwf[k] = (float)p.rw[k];
    }
    p.ds_out = nullptr;
    p.smooth_delta = g.smooth_delta;
    p.smooth_k = g.smooth_k;
    p.threshold_c = g.threshold_c;
    p.threshold_delta = g.threshold_delta;
    return p;
}

FinalParams cfg_final_params(const lbm_config &g, const StepParams &p, int collide, unsigned limiters, int nblocks)
{
    FinalParams f{};
    f.nblocks = nblocks;
    // entropic f*: the step kernel sums dS(f_in) - dS(f') itself (no quadratic identity)
    f.one_minus_a2 = g.equilibrium == LBM_EQ_ENTROPIC ? 1.0 : 1.0 - p.a * p.a;
    f.eq = p.eq;
    f.k_max = g.k_max;
    f.ehrenfest = (limiters & LBM_LIM_EHRENFEST) ? 1 : 0;
    f.collide = collide;
    f.nx = g.nx;
    f.ny = g.ny;
    f.pitch = p.pitch;
    f.plane = p.plane;
    f.boundary = g.boundary;
    f.a = p.a;
    f.delta_e = p.delta_e;
    for (int k = 0; k < 9; ++k) {
        f.lid[k] = p.lid[k];
        f.lidf[k] = p.lidf[k];
        f.lidlo[k] = p.lidlo[k];
        f.rw[k] = p.rw[k];
    }
    f.rho_ref = p.rho_ref;
    return f;
}

int set_thread_error_impl(int s, const char *msg)
{
    g_err = msg;
    return s;
}
StepParams ctx_step_params(lbm_ctx *c, int collide, unsigned limiters) { return step_params(c, collide, limiters); }
FinalParams ctx_final_params(lbm_ctx *c, int collide, unsigned limiters, int nblocks)
{
    return final_params(c, collide, limiters, nblocks);
}
bool ctx_uses_fused(const lbm_ctx *c) { return fused_applies(c->cfg); }
double *ctx_fx_rows(lbm_ctx *c) { return c->partials; }
}  // namespace lbm

extern "C" {

void lbm_config_default(lbm_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->lattice = LBM_D2Q9;
    c->nx = 100;
    c->ny = 100;
    c->boundary = LBM_BC_WALLS;
    c->precision = LBM_FP32;
    c->limiters = 0;
    c->median_mode = LBM_MEDIAN_THRESHOLD;
    c->kernel = LBM_KERNEL_AUTO;
    c->beta = 1.0;
    c->u_lid = 0.0;
    c->rho_wall = 1.0;
    c->delta_median = 1e-3;
    c->delta_ehrenfest = 1e-3;
    c->k_max = 0;
    c->stats_history = 1;
    c->equilibrium = LBM_EQ_POLYNOMIAL;
    c->rho_ref = 1.0;
    c->smooth_delta = 1e-2;
    c->smooth_k = 0.5;
    c->threshold_c = 10.0;
    c->threshold_delta = 0.0;
    c->collision = LBM_COLL_LBGK;
    c->phi_rule = LBM_PHI_HOMOTHETY;
    c->entthresh_delta0 = 0.1;
}

int64_t lbm_footprint_bytes(const lbm_config *cfg)
{
    std::string v = validate(cfg);
    if (!v.empty()) {
        g_err = v;
        return 0;
    }
    return sizes_for(*cfg).total();
}

lbm_status lbm_create(const lbm_config *cfg, void *cuda_stream, lbm_ctx **out)
{
    if (!out) return fail(nullptr, LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::string v = validate(cfg);
    if (!v.empty()) return fail(nullptr, LBM_ERR_INVALID_ARG, v);
    lbm_ctx *c = new lbm_ctx();
    c->cfg = *cfg;
    if (c->cfg.stats_history < 1) c->cfg.stats_history = 1;
    c->stream = (cudaStream_t)cuda_stream;
    const Sizes z = sizes_for(c->cfg);
    c->q = z.q;
    c->pitch = z.pitch;
    c->plane = z.plane;
    c->elem = z.elem;
    c->field_bytes = z.field;
    c->cand_cap = z.cand_cap;
    c->sel_cap = z.sel_cap;
    c->partial_rows = z.rows;
    c->ring_len = z.ring_len;
    cudaError_t e = cudaGetDevice(&c->device);
    auto alloc = [&](void **p, size_t bytes) -> cudaError_t {
        if (e != cudaSuccess) return e;
        e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, bytes, c->stream);
        return e;
    };
    alloc(&c->buf[0], z.field);
    alloc(&c->buf[1], z.field);
    alloc((void **)&c->cand, z.cand);
    alloc((void **)&c->counts, 4 * sizeof(int));
    alloc((void **)&c->sel, z.sel);
    alloc((void **)&c->partials, z.partials);
    alloc((void **)&c->chunk_cnt, (size_t)chunks_for(z.rows) * sizeof(unsigned));
    alloc((void **)&c->status, sizeof(unsigned));
    alloc((void **)&c->ring, z.ring);
    alloc((void **)&c->counters, 2 * sizeof(long long));
    alloc((void **)&c->ens, ens_bytes());
    if (z.selstate) {
        alloc((void **)&c->sel_state, z.selstate);
        switch (c->cfg.precision) {
        case LBM_FP64: c->fin_grid = finalize_grid<double>(c->q); break;
        case LBM_FP32: c->fin_grid = finalize_grid<float>(c->q); break;
        case LBM_BF16: c->fin_grid = finalize_grid<__nv_bfloat16>(c->q); break;
        default: c->fin_grid = finalize_grid<__half>(c->q);
        }
    }
    if (z.ent) {
        alloc(&c->ent_field, z.ent - sizeof(EntState));
        alloc((void **)&c->ent, sizeof(EntState));
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        std::string m = std::string("lbm_create: device allocation failed: ") + cudaGetErrorString(e);
        delete c;
        return fail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
    }
    c->device_bytes = z.total();
    *out = c;
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx *c)
{
    if (!c) return LBM_OK;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return LBM_OK;
}

lbm_status lbm_init(lbm_ctx *c, const double *rho, const double *ux, const double *uy)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (!rho || !ux) return fail(c, LBM_ERR_INVALID_ARG, "rho and ux must not be NULL");
    const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
    lbm_status s = ensure_stage(c, 3 * n * sizeof(double));
    if (s != LBM_OK) return s;
    const double *dr, *du, *dv = nullptr;
    if ((s = dev_in(c, rho, n, 0, &dr)) != LBM_OK) return s;
    if ((s = dev_in(c, ux, n, n, &du)) != LBM_OK) return s;
    if (uy && c->q == 9 && (s = dev_in(c, uy, n, 2 * n, &dv)) != LBM_OK) return s;
    cudaError_t e;
    const StepParams sp = step_params(c, 1, 0);
    e = with_storage(c->cfg.precision, [&](auto tag) -> cudaError_t {
        using S = STORAGE_T;
        return launch_init<S>(c->q, sp, dr, du, dv, (S *)c->buf[0], c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel launch");
    c->launches++;
    c->cur = 0;
    if ((s = reset_counters(c)) != LBM_OK) return s;
    CK(c, cudaStreamSynchronize(c->stream));
    c->ready = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *c, int64_t nsteps)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(c, LBM_ERR_INVALID_ARG, "nsteps must be >= 0");
    if (!c->ready) return fail(c, LBM_ERR_STATE, "lbm_step before lbm_init / lbm_set_populations");
    int64_t left = nsteps;
    // graph replay (not while per-kernel timing records its events)
    const int gs = c->graph_steps;
    while (gs > 0 && !c->timing && left >= gs) {
        if (!c->gexec[c->cur]) {
            // the kernels' one-time set-up happens outside the capture: one plain step first
            lbm_status s = run_pass(c, 1, c->cfg.limiters);
            if (s != LBM_OK) return s;
            if (--left < gs) break;
            if (!c->gexec[c->cur] && (s = capture_graph(c)) != LBM_OK) return s;
        }
        CK(c, cudaGraphLaunch(c->gexec[c->cur], c->stream));
        c->launches += c->graph_launches;
        left -= gs;
    }
    for (int64_t i = 0; i < left; ++i) {
        lbm_status s = run_pass(c, 1, c->cfg.limiters);
        if (s != LBM_OK) return s;
    }
    return LBM_OK;
}

lbm_status lbm_limit(lbm_ctx *c, uint32_t limiters)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (limiters & ~63u) return fail(c, LBM_ERR_INVALID_ARG, "unknown limiter bits");
    if (!c->ready) return fail(c, LBM_ERR_STATE, "lbm_limit before lbm_init / lbm_set_populations");
    if ((limiters & LBM_LIM_EHRENFEST) && c->cand_cap < c->cfg.nx * c->cfg.ny)
        return fail(c, LBM_ERR_INVALID_ARG, "Ehrenfests' limiter needs LBM_LIM_EHRENFEST in the config at create");
    if ((limiters & LBM_LIM_ENTTHRESH) && !c->ent)
        return fail(c, LBM_ERR_INVALID_ARG, "LBM_LIM_ENTTHRESH needs the bit in the config at create");
    return run_pass(c, 0, limiters);
}

lbm_status lbm_delta_s(lbm_ctx *c, double *out)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (!out) return fail(c, LBM_ERR_INVALID_ARG, "out is NULL");
    if (!c->ready) return fail(c, LBM_ERR_STATE, "lbm_delta_s before lbm_init / lbm_set_populations");
    const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
    const bool dev = is_device_ptr(out);
    double *dst = out;
    if (!dev) {
        lbm_status s = ensure_stage(c, n * sizeof(double));
        if (s != LBM_OK) return s;
        dst = c->stage;
    }
    StepParams p = step_params(c, 1, 0);
    cudaError_t e = with_storage(c->cfg.precision, [&](auto tag) -> cudaError_t {
        using S = STORAGE_T;
        return launch_delta_s<S>(c->q, p, (const S *)c->buf[c->cur], dst, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "delta_s kernel launch");
    c->launches++;
    if (!dev) CK(c, cudaMemcpyAsync(out, dst, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx *c, double *rho, double *ux, double *uy)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (!rho || !ux) return fail(c, LBM_ERR_INVALID_ARG, "rho and ux must not be NULL");
    if (!c->ready) return fail(c, LBM_ERR_STATE, "lbm_moments before lbm_init / lbm_set_populations");
    const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
    const bool dev = is_device_ptr(rho);
    if (dev != is_device_ptr(ux) || (uy && dev != is_device_ptr(uy)))
        return fail(c, LBM_ERR_INVALID_ARG, "rho, ux, uy must all be host or all be device memory");
    double *dr = rho, *du = ux, *dv = uy;
    if (!dev) {
        lbm_status s = ensure_stage(c, 3 * n * sizeof(double));
        if (s != LBM_OK) return s;
        dr = c->stage;
        du = c->stage + n;
        dv = uy ? c->stage + 2 * n : nullptr;
    }
    const StepParams sp = step_params(c, 1, 0);
    cudaError_t e = with_storage(c->cfg.precision, [&](auto tag) -> cudaError_t {
        using S = STORAGE_T;
        return launch_moments<S>(c->q, sp, (const S *)c->buf[c->cur], dr, du, dv, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel launch");
    c->launches++;
    if (!dev) {
        CK(c, cudaMemcpyAsync(rho, dr, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaMemcpyAsync(ux, du, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (uy) CK(c, cudaMemcpyAsync(uy, dv, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    return read_status(c, false);
}

lbm_status lbm_stats_history(lbm_ctx *c, lbm_step_stats *out, int64_t cap, int64_t *n)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (!out || !n || cap < 0) return fail(c, LBM_ERR_INVALID_ARG, "bad output arguments");
    long long cnt[2] = {0, 0};
    std::vector<DevStats> ring((size_t)c->ring_len);
    CK(c, cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(ring.data(), c->ring, ring.size() * sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const long long recs = cnt[1];
    const long long have = std::min<long long>(recs, c->ring_len);
    const long long take = std::min<long long>(have, cap);
    for (long long i = 0; i < take; ++i) {
        const long long r = recs - take + i;
        to_public(ring[(size_t)(r % c->ring_len)], &out[i]);
    }
    *n = take;
    return read_status(c, false);
}

lbm_status lbm_stats(lbm_ctx *c, lbm_step_stats *out)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (!out) return fail(c, LBM_ERR_INVALID_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    int64_t n = 0;
    return lbm_stats_history(c, out, 1, &n);
}

lbm_status lbm_limited_sites(lbm_ctx *c, int64_t *idx, int64_t cap, int64_t *n)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (!n || cap < 0 || (cap > 0 && !idx)) return fail(c, LBM_ERR_INVALID_ARG, "bad output arguments");
    int cnt = 0;
    CK(c, cudaMemcpyAsync(&cnt, c->counts + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    std::vector<int> s((size_t)std::max(cnt, 0));
    if (cnt > 0) {
        CK(c, cudaMemcpyAsync(s.data(), c->sel, (size_t)cnt * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    std::sort(s.begin(), s.end());
    *n = cnt;
    const int64_t take = std::min<int64_t>(cap, cnt);
    std::vector<int64_t> w((size_t)take);
    for (int64_t i = 0; i < take; ++i) w[(size_t)i] = s[(size_t)i];
    if (take > 0) {
        if (is_device_ptr(idx)) {
            CK(c, cudaMemcpyAsync(idx, w.data(), (size_t)take * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
            CK(c, cudaStreamSynchronize(c->stream));
        } else {
            std::memcpy(idx, w.data(), (size_t)take * sizeof(int64_t));
        }
    }
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx *c, double *f)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (!f) return fail(c, LBM_ERR_INVALID_ARG, "f is NULL");
    const size_t tot = (size_t)c->q * c->cfg.nx * c->cfg.ny;
    const bool dev = is_device_ptr(f);
    double *dst = f;
    if (!dev) {
        lbm_status s = ensure_stage(c, tot * sizeof(double));
        if (s != LBM_OK) return s;
        dst = c->stage;
    }
    const StepParams sp = step_params(c, 1, 0);
    cudaError_t e = with_storage(c->cfg.precision, [&](auto tag) -> cudaError_t {
        using S = STORAGE_T;
        return launch_get<S>(c->q, sp, (const S *)c->buf[c->cur], dst, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "get kernel launch");
    c->launches++;
    if (!dev) CK(c, cudaMemcpyAsync(f, dst, tot * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx *c, const double *f)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (!f) return fail(c, LBM_ERR_INVALID_ARG, "f is NULL");
    const size_t tot = (size_t)c->q * c->cfg.nx * c->cfg.ny;
    const double *src = f;
    if (!is_device_ptr(f)) {
        lbm_status s = ensure_stage(c, tot * sizeof(double));
        if (s != LBM_OK) return s;
        if ((s = dev_in(c, f, tot, 0, &src)) != LBM_OK) return s;
    }
    const StepParams sp = step_params(c, 1, 0);
    cudaError_t e = with_storage(c->cfg.precision, [&](auto tag) -> cudaError_t {
        using S = STORAGE_T;
        return launch_set<S>(c->q, sp, src, (S *)c->buf[0], c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "set kernel launch");
    c->launches++;
    c->cur = 0;
    lbm_status s = reset_counters(c);
    if (s != LBM_OK) return s;
    CK(c, cudaStreamSynchronize(c->stream));
    c->ready = true;
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx *c)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    return read_status(c, true);
}

lbm_status lbm_get_config(const lbm_ctx *c, lbm_config *out)
{
    if (!c || !out) return fail(nullptr, LBM_ERR_INVALID_ARG, "NULL argument");
    *out = c->cfg;
    return LBM_OK;
}

lbm_status lbm_set_graph(lbm_ctx *c, int32_t steps_per_graph)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (steps_per_graph < 0 || steps_per_graph == 1 || (steps_per_graph & 1))
        return fail(c, LBM_ERR_INVALID_ARG, "steps_per_graph must be 0 or an even number >= 2");
    if (steps_per_graph != c->graph_steps) {
        CK(c, cudaStreamSynchronize(c->stream));
        drop_graphs(c);
    }
    c->graph_steps = steps_per_graph;
    return LBM_OK;
}

lbm_status lbm_probe(lbm_ctx *c, int64_t site, int64_t capacity)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    const long long n = (long long)c->cfg.nx * c->cfg.ny;
    if (site < -1 || site >= n) return fail(c, LBM_ERR_INVALID_ARG, "site must be -1 or in [0, nx * ny)");
    if (site >= 0 && capacity < 1) return fail(c, LBM_ERR_INVALID_ARG, "capacity must be >= 1");
    CK(c, cudaStreamSynchronize(c->stream));
    drop_graphs(c);  // the graphs carry the tail's parameters
    if (site < 0) {
        c->probe_site = -1;
        return LBM_OK;
    }
    if (capacity > c->probe_alloc) {
        if (c->probe) {
            cudaFree(c->probe);
            c->device_bytes -= c->probe_alloc * 3 * (int64_t)sizeof(double);
            c->probe = nullptr;
            c->probe_alloc = 0;
        }
        CK(c, cudaMalloc((void **)&c->probe, (size_t)capacity * 3 * sizeof(double)));
        c->probe_alloc = capacity;
        c->device_bytes += capacity * 3 * (int64_t)sizeof(double);
    }
    long long steps = 0;
    CK(c, cudaMemcpy(&steps, c->counters, sizeof(long long), cudaMemcpyDeviceToHost));
    c->probe_site = (int)site;
    c->probe_cap = capacity;
    c->probe_step0 = steps;
    return LBM_OK;
}

lbm_status lbm_probe_read(lbm_ctx *c, double *out, int64_t cap, int64_t *n)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (!n || cap < 0 || (cap > 0 && !out)) return fail(c, LBM_ERR_INVALID_ARG, "bad output arguments");
    *n = 0;
    if (c->probe_site < 0) return fail(c, LBM_ERR_STATE, "no probe set (lbm_probe)");
    long long steps = 0;
    CK(c, cudaMemcpyAsync(&steps, c->counters, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const long long have = std::min<long long>(steps - c->probe_step0, c->probe_cap);
    const long long take = std::min<long long>(std::max<long long>(have, 0), cap);
    std::vector<double> ring((size_t)c->probe_cap * 3);
    if (take > 0) CK(c, cudaMemcpy(ring.data(), c->probe, ring.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> w((size_t)take * 3);
    for (long long i = 0; i < take; ++i) {
        const long long st = steps - take + 1 + i;  // step numbers, oldest first
        const long long slot = (st - 1) % c->probe_cap;
        for (int j = 0; j < 3; ++j) w[(size_t)(3 * i + j)] = ring[(size_t)(3 * slot + j)];
    }
    if (take > 0) {
        if (is_device_ptr(out))
            CK(c, cudaMemcpy(out, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
        else
            std::memcpy(out, w.data(), w.size() * sizeof(double));
    }
    *n = take;
    return LBM_OK;
}

lbm_status lbm_timing(lbm_ctx *c, int32_t enable)
{
    if (!c) return fail(nullptr, LBM_ERR_INVALID_ARG, "ctx is NULL");
    if (enable < 0) return fail(c, LBM_ERR_INVALID_ARG, "enable must be >= 0");
    c->timing = enable != 0;
    c->timing_every = enable > 1 ? enable : 1;
    c->timing_pass = 0;
    c->events_used = 0;
    return LBM_OK;
}

lbm_status lbm_timing_read(lbm_ctx *c, double *step_ms, double *tail_ms, int64_t *steps)
{
    if (!c || !step_ms || !tail_ms || !steps) return fail(c, LBM_ERR_INVALID_ARG, "NULL argument");
    CK(c, cudaStreamSynchronize(c->stream));
    double a = 0.0, b = 0.0;
    const size_t n = c->events_used / 3;
    for (size_t i = 0; i < n; ++i) {
        float t0 = 0.f, t1 = 0.f;
        CK(c, cudaEventElapsedTime(&t0, c->events[3 * i], c->events[3 * i + 1]));
        CK(c, cudaEventElapsedTime(&t1, c->events[3 * i + 1], c->events[3 * i + 2]));
        a += t0;
        b += t1;
    }
    *step_ms = a;
    *tail_ms = b;
    *steps = (int64_t)n;
    c->events_used = 0;
    return LBM_OK;
}

int64_t lbm_device_bytes(const lbm_ctx *c) { return c ? c->device_bytes : 0; }

int64_t lbm_launch_count(const lbm_ctx *c) { return c ? c->launches : 0; }

int32_t lbm_step_kernel(const lbm_ctx *c)
{
    if (!c) return -1;
    if (fused_applies(c->cfg)) return LBM_KERNEL_FUSED;
    return tube_applies(c->cfg, c->cfg.limiters) ? LBM_KERNEL_TUBE : LBM_KERNEL_TILED;
}

const char *lbm_last_error(const lbm_ctx *c) { return c ? c->err.c_str() : g_err.c_str(); }

const char *lbm_status_string(lbm_status s)
{
    switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_ERR_INVALID_ARG: return "LBM_ERR_INVALID_ARG";
    case LBM_ERR_OOM: return "LBM_ERR_OOM";
    case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
    case LBM_ERR_NONFINITE: return "LBM_ERR_NONFINITE";
    case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
    case LBM_ERR_STATE: return "LBM_ERR_STATE";
    }
    return "LBM_ERR_UNKNOWN";
}

int32_t lbm_abi_version(void) { return LBM_ABI_VERSION; }

}  // extern "C"
