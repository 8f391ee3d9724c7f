// batch.cu -- many lattices stepped by shared launches (include/lbm_batch.h).
//
// Each lattice is an ordinary context (lbm_ctx) created on the batch's own
// stream.  A batched step is at most six launches whatever the number of
// lattices: the fused kernel over every FP32 D2Q9 cavity, the tube kernel
// over D1Q3 lattices, the tiled kernel over the rest, and the tail kernel (one
// block per lattice) for D2Q9 and for D1Q3.  The fused launch is one wave of resident
// warps over the work items of all its lattices (strips of 62 columns times
// short row segments), handed out through one device counter, so warps that
// finish early take more work whatever lattice it belongs to; the tube launch
// does the same over groups of 1024 sites of every tube; tiled blocks find
// their lattice and local block number in a device table.  The tables
// exist twice, for even and odd steps, because the two population buffers of
// each lattice swap roles every step.  A lattice's per-site arithmetic is the
// same as when it runs alone, so its populations match a lone run bit for bit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm_batch.h"
#include "internal.h"

using namespace lbm;

struct lbm_batch {
    cudaStream_t user = nullptr;
    cudaStream_t run = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
    std::vector<lbm_ctx *> slots;
    std::vector<lbm_status> slot_status;  // sticky per-lattice status seen by lbm_batch_synchronize
    // launch tables (host copies kept while the device copies are in use)
    bool dirty = true;
    int phase = 0;               // steps since the tables were built, mod 2
    std::vector<int> cur_build;  // each lattice's current buffer when built
    std::vector<FusedArgs> h_fused[2];
    std::vector<TiledArgs> h_t3[2], h_t9[2];
    std::vector<FinalArgs> h_fin9[2], h_fin3[2];
    std::vector<int2> h_fmap, h_t3map, h_t9map, h_tubemap;
    std::vector<TubeArgs> h_tube[2];
    void *table_mem = nullptr;
    size_t table_bytes = 0;
    FusedArgs *fused[2] = {nullptr, nullptr};
    TiledArgs *t3[2] = {nullptr, nullptr}, *t9[2] = {nullptr, nullptr};
    FinalArgs *fin9[2] = {nullptr, nullptr}, *fin3[2] = {nullptr, nullptr};
    int2 *fmap = nullptr, *t3map = nullptr, *t9map = nullptr, *tubemap = nullptr;
    TubeArgs *tube[2] = {nullptr, nullptr};
    int *work = nullptr;   // the fused launch's work-item counter
    int *twork = nullptr;  // the tube launch's
    int fitems = 0, t3blocks = 0, t9blocks = 0, titems = 0, n9 = 0, n3 = 0;
    // shape
    int seg_rows = 0;  // rows per fused work item; 0 = automatic
    int waves = 8;     // automatic segments: about this many work items per resident warp
    // graph replay
    int graph_steps = 0;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch *b, lbm_status s, const std::string &m)
{
    if (b) b->err = m;
    return s;
}

#define BCK(b, call)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,              \
                         std::string(#call) + " failed: " + cudaGetErrorString(e_));                  \
    } while (0)

lbm_ctx *get(lbm_batch *b, int32_t slot)
{
    if (!b || slot < 0 || slot >= (int32_t)b->slots.size()) return nullptr;
    return b->slots[(size_t)slot];
}

// Brings every lattice's `cur` up to date with the steps taken since the
// tables were built.
void materialise(lbm_batch *b)
{
    if (b->dirty) return;
    for (size_t i = 0; i < b->slots.size(); ++i)
        if (b->slots[i]) b->slots[i]->cur = b->cur_build[i] ^ b->phase;
}

void drop_graph(lbm_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

void invalidate(lbm_batch *b)
{
    materialise(b);
    b->dirty = true;
    b->phase = 0;
    drop_graph(b);
}

// Orders the batch stream after the caller's stream.
lbm_status enter(lbm_batch *b)
{
    BCK(b, cudaEventRecord(b->ev_in, b->user));
    BCK(b, cudaStreamWaitEvent(b->run, b->ev_in, 0));
    return LBM_OK;
}

// Orders the caller's stream after the batch stream.
lbm_status leave(lbm_batch *b)
{
    BCK(b, cudaEventRecord(b->ev_out, b->run));
    BCK(b, cudaStreamWaitEvent(b->user, b->ev_out, 0));
    return LBM_OK;
}


lbm_status rebuild(lbm_batch *b)
{
    for (int k = 0; k < 2; ++k) {
        b->h_fused[k].clear();
        b->h_t3[k].clear();
        b->h_tube[k].clear();
        b->h_t9[k].clear();
        b->h_fin9[k].clear();
        b->h_fin3[k].clear();
    }
    b->h_fmap.clear();
    b->h_t3map.clear();
    b->h_tubemap.clear();
    b->h_t9map.clear();
    b->cur_build.assign(b->slots.size(), 0);
    int first_fused = -1;  // index in h_fin9 of the first fused lattice's tail
    int first_tube = -1;   // index in h_fin3 of the first tube's tail
    // one row-segment length for every fused lattice: about `waves` items per
    // resident warp over the strip rows of all of them (unless fixed)
    long long strip_rows = 0;
    for (lbm_ctx *c : b->slots) {
        if (!c) continue;
        if (!c->ready) return bfail(b, LBM_ERR_STATE, "a lattice of the batch was never initialised");
        if (ctx_uses_fused(c)) strip_rows += (long long)((c->cfg.nx + 61) / 62) * c->cfg.ny;
    }
    const long long want = std::max(1LL, (long long)b->waves * fused_slots(4, true));
    const int seg = b->seg_rows > 0 ? b->seg_rows : (int)std::max(4LL, (strip_rows + want - 1) / want);
    for (size_t i = 0; i < b->slots.size(); ++i) {
        lbm_ctx *c = b->slots[i];
        if (!c) continue;
        b->cur_build[i] = c->cur;
        const unsigned lim = c->cfg.limiters;
        const StepParams p = ctx_step_params(c, 1, lim);
        for (int k = 0; k < 2; ++k) {
            void *src = c->buf[c->cur ^ k], *dst = c->buf[c->cur ^ k ^ 1];
            if (ctx_uses_fused(c)) {
                FusedArgs A;
                const int blocks = fused_make_args(p, src, dst, seg, 1, &A);
                b->h_fused[k].push_back(A);
                FinalArgs F{ctx_final_params(c, 1, lim, blocks), dst};
                F.p.src = src;
                F.p.fixed = 1;
                F.p.partials = ctx_fx_rows(c);  // the fused kernel's accumulator rows
                F.p.work = nullptr;             // the first fused lattice's tail clears the counter (below)
                if (first_fused < 0 && k == 0) first_fused = (int)b->h_fin9[0].size();
                b->h_fin9[k].push_back(F);
                if (k == 0)
                    for (int it = 0; it < A.items; ++it)
                        b->h_fmap.push_back(make_int2((int)b->h_fused[0].size() - 1, it));
            } else if (c->q == 3 && tube_applies(c->cfg, lim)) {
                // D1Q3: the tube kernel, groups of chunks from one counter
                TubeArgs A{};
                A.p = p;
                A.src = src;
                A.dst = dst;
                const int groups = tube_groups(c->cfg.nx);
                b->h_tube[k].push_back(A);
                FinalArgs F{ctx_final_params(c, 1, lim, groups), dst};
                F.p.src = src;
                F.p.partials = p.partials;  // one row per group
                F.p.nblocks = groups;
                F.p.work = nullptr;         // the first tube's tail clears the counter (below)
                if (first_tube < 0 && k == 0) first_tube = (int)b->h_fin3[0].size();
                b->h_fin3[k].push_back(F);
                if (k == 0)
                    for (int gi = 0; gi < groups; ++gi)
                        b->h_tubemap.push_back(make_int2((int)b->h_tube[0].size() - 1, gi));
            } else {
                TiledArgs A{};
                A.p = p;
                A.src = src;
                A.dst = dst;
                A.gx = tiled_grid_x(c->q, c->cfg.nx);
                A.blocks = tiled_blocks_for(c->q, c->cfg.nx, c->cfg.ny);
                FinalArgs F{ctx_final_params(c, 1, lim, A.blocks), dst};
                F.p.src = src;
                auto &tab = c->q == 9 ? b->h_t9[k] : b->h_t3[k];
                auto &map = c->q == 9 ? b->h_t9map : b->h_t3map;
                tab.push_back(A);
                (c->q == 9 ? b->h_fin9[k] : b->h_fin3[k]).push_back(F);
                if (k == 0)
                    for (int lb = 0; lb < A.blocks; ++lb) map.push_back(make_int2((int)tab.size() - 1, lb));
            }
        }
    }
    // one device allocation holds every table
    auto sz = [](size_t n, size_t e) { return ((n * e + 255) / 256) * 256; };
    const size_t nf = b->h_fused[0].size(), nt3 = b->h_t3[0].size(), nt9 = b->h_t9[0].size();
    const size_t nf9 = b->h_fin9[0].size(), nf3 = b->h_fin3[0].size(), ntb = b->h_tube[0].size();
    size_t need = 2 * (sz(nf, sizeof(FusedArgs)) + sz(nt3, sizeof(TiledArgs)) + sz(nt9, sizeof(TiledArgs)) +
                       sz(nf9, sizeof(FinalArgs)) + sz(nf3, sizeof(FinalArgs)) + sz(ntb, sizeof(TubeArgs))) +
                  sz(b->h_tubemap.size(), sizeof(int2)) + 256 +
                  sz(b->h_fmap.size(), sizeof(int2)) + sz(b->h_t3map.size(), sizeof(int2)) +
                  sz(b->h_t9map.size(), sizeof(int2)) + 256 + 256;
    if (need > b->table_bytes) {
        BCK(b, cudaStreamSynchronize(b->run));
        if (b->table_mem) cudaFree(b->table_mem);
        b->table_mem = nullptr;
        b->table_bytes = 0;
        BCK(b, cudaMalloc(&b->table_mem, need));
        b->table_bytes = need;
    }
    char *m = (char *)b->table_mem;
    b->work = (int *)m;
    m += 256;
    b->twork = (int *)m;
    m += 256;
    if (first_fused >= 0)
        for (int k = 0; k < 2; ++k) b->h_fin9[k][(size_t)first_fused].p.work = b->work;
    if (first_tube >= 0)
        for (int k = 0; k < 2; ++k) b->h_fin3[k][(size_t)first_tube].p.work = b->twork;
    auto put = [&](const void *h, size_t n, size_t e, void **d) -> cudaError_t {
        *d = m;
        m += sz(n, e);
        return n ? cudaMemcpyAsync(*d, h, n * e, cudaMemcpyHostToDevice, b->run) : cudaSuccess;
    };
    for (int k = 0; k < 2; ++k) {
        BCK(b, put(b->h_fused[k].data(), nf, sizeof(FusedArgs), (void **)&b->fused[k]));
        BCK(b, put(b->h_t3[k].data(), nt3, sizeof(TiledArgs), (void **)&b->t3[k]));
        BCK(b, put(b->h_t9[k].data(), nt9, sizeof(TiledArgs), (void **)&b->t9[k]));
        BCK(b, put(b->h_fin9[k].data(), nf9, sizeof(FinalArgs), (void **)&b->fin9[k]));
        BCK(b, put(b->h_fin3[k].data(), nf3, sizeof(FinalArgs), (void **)&b->fin3[k]));
        BCK(b, put(b->h_tube[k].data(), ntb, sizeof(TubeArgs), (void **)&b->tube[k]));
    }
    BCK(b, put(b->h_fmap.data(), b->h_fmap.size(), sizeof(int2), (void **)&b->fmap));
    BCK(b, put(b->h_t3map.data(), b->h_t3map.size(), sizeof(int2), (void **)&b->t3map));
    BCK(b, put(b->h_t9map.data(), b->h_t9map.size(), sizeof(int2), (void **)&b->t9map));
    BCK(b, put(b->h_tubemap.data(), b->h_tubemap.size(), sizeof(int2), (void **)&b->tubemap));
    BCK(b, cudaMemsetAsync(b->work, 0, sizeof(int), b->run));
    BCK(b, cudaMemsetAsync(b->twork, 0, sizeof(int), b->run));
    b->fitems = (int)b->h_fmap.size();
    b->t3blocks = (int)b->h_t3map.size();
    b->titems = (int)b->h_tubemap.size();
    b->t9blocks = (int)b->h_t9map.size();
    b->n9 = (int)nf9;
    b->n3 = (int)nf3;
    b->dirty = false;
    b->phase = 0;
    drop_graph(b);
    return LBM_OK;
}

int launches_per_step(const lbm_batch *b)
{
    return (b->fitems > 0) + (b->t3blocks > 0) + (b->t9blocks > 0) + (b->titems > 0) + (b->n9 > 0) + (b->n3 > 0);
}

// One batched step on the batch stream (table set `k`).
cudaError_t one_step(lbm_batch *b, int k)
{
    cudaError_t e = cudaSuccess;
    if (b->fitems && e == cudaSuccess) e = launch_fused_batched(b->fused[k], b->fmap, b->fitems, b->work, b->run);
    if (b->t3blocks && e == cudaSuccess) e = launch_tiled_batched_f32(3, b->t3[k], b->t3map, b->t3blocks, b->run);
    if (b->titems && e == cudaSuccess) e = launch_tube_batched(b->tube[k], b->tubemap, b->titems, b->twork, b->run);
    if (b->t9blocks && e == cudaSuccess) e = launch_tiled_batched_f32(9, b->t9[k], b->t9map, b->t9blocks, b->run);
    if (b->n9 && e == cudaSuccess) e = launch_finalize_batched_f32(9, b->fin9[k], b->n9, b->run);
    if (b->n3 && e == cudaSuccess) e = launch_finalize_batched_f32(3, b->fin3[k], b->n3, b->run);
    return e;
}

lbm_status run_steps(lbm_batch *b, int64_t n)
{
    if (b->dirty) {
        lbm_status s = rebuild(b);
        if (s != LBM_OK) return s;
    }
    const int lps = launches_per_step(b);
    int64_t left = n;
    if (b->graph_steps > 0 && left >= b->graph_steps) {
        if (b->phase == 1) {  // graphs start on even steps
            BCK(b, one_step(b, 1));
            b->phase = 0;
            b->launches += lps;
            --left;
        }
        if (!b->exec && left >= b->graph_steps) {
            // the kernels' one-time attribute set-up happens outside the capture
            BCK(b, one_step(b, 0));
            BCK(b, one_step(b, 1));
            b->launches += 2 * lps;
            left -= 2;
            cudaGraph_t g = nullptr;
            BCK(b, cudaStreamBeginCapture(b->run, cudaStreamCaptureModeThreadLocal));
            cudaError_t ce = cudaSuccess;
            for (int i = 0; i < b->graph_steps && ce == cudaSuccess; ++i) ce = one_step(b, i & 1);
            cudaError_t ee = cudaStreamEndCapture(b->run, &g);
            if (ce != cudaSuccess || ee != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return bfail(b, LBM_ERR_CUDA, "graph capture of the batched step failed");
            }
            cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) {
                b->exec = nullptr;
                return bfail(b, LBM_ERR_CUDA, std::string("cudaGraphInstantiate failed: ") + cudaGetErrorString(ie));
            }
        }
        while (b->exec && left >= b->graph_steps) {
            BCK(b, cudaGraphLaunch(b->exec, b->run));
            b->launches += (long long)b->graph_steps * lps;
            left -= b->graph_steps;
        }
    }
    for (int64_t i = 0; i < left; ++i) {
        BCK(b, one_step(b, b->phase));
        b->phase ^= 1;
        b->launches += lps;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(void *cuda_stream, lbm_batch **out)
{
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    lbm_batch *b = new lbm_batch();
    b->user = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&b->run, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess) {
        cudaGetLastError();
        lbm_batch_destroy(b);
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return LBM_OK;
    if (b->run) cudaStreamSynchronize(b->run);
    for (lbm_ctx *c : b->slots)
        if (c) lbm_destroy(c);
    drop_graph(b);
    if (b->table_mem) cudaFree(b->table_mem);
    cudaEvent_t evs[] = {b->ev_in, b->ev_out, b->t0, b->t1};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (b->run) cudaStreamDestroy(b->run);
    delete b;
    return LBM_OK;
}

lbm_status lbm_batch_add(lbm_batch *b, const lbm_config *cfg, int32_t *slot)
{
    if (!b || !cfg || !slot) return bfail(b, LBM_ERR_INVALID_ARG, "NULL argument");
    if (cfg->precision != LBM_FP32) return bfail(b, LBM_ERR_INVALID_ARG, "batched lattices use LBM_FP32");
    if (cfg->equilibrium != LBM_EQ_POLYNOMIAL)
        return bfail(b, LBM_ERR_INVALID_ARG, "batched lattices use polynomial quasiequilibria");
    if (cfg->limiters & kLimEnsemble)
        return bfail(b, LBM_ERR_INVALID_ARG, "the ensemble-dependent limiters are not available in batches");
    lbm_ctx *c = nullptr;
    lbm_status s = lbm_create(cfg, (void *)b->run, &c);
    if (s != LBM_OK) return bfail(b, s, lbm_last_error(nullptr));
    invalidate(b);
    b->slot_status.resize(b->slots.size(), LBM_OK);
    for (size_t i = 0; i < b->slots.size(); ++i) {
        if (!b->slots[i]) {
            b->slots[i] = c;
            b->slot_status[i] = LBM_OK;
            *slot = (int32_t)i;
            return LBM_OK;
        }
    }
    b->slots.push_back(c);
    b->slot_status.push_back(LBM_OK);
    *slot = (int32_t)b->slots.size() - 1;
    return LBM_OK;
}

lbm_status lbm_batch_remove(lbm_batch *b, int32_t slot)
{
    lbm_ctx *c = get(b, slot);
    if (!c) return bfail(b, LBM_ERR_INVALID_ARG, "no lattice in that slot");
    invalidate(b);
    BCK(b, cudaStreamSynchronize(b->run));
    lbm_destroy(c);
    b->slots[(size_t)slot] = nullptr;
    b->slot_status[(size_t)slot] = LBM_OK;
    return LBM_OK;
}

int32_t lbm_batch_size(const lbm_batch *b)
{
    if (!b) return 0;
    int32_t n = 0;
    for (lbm_ctx *c : b->slots) n += c != nullptr;
    return n;
}

int64_t lbm_batch_device_bytes(const lbm_batch *b)
{
    if (!b) return 0;
    int64_t n = (int64_t)b->table_bytes;
    for (lbm_ctx *c : b->slots)
        if (c) n += lbm_device_bytes(c);
    return n;
}

lbm_status lbm_batch_init(lbm_batch *b, int32_t slot, const double *rho, const double *ux, const double *uy)
{
    lbm_ctx *c = get(b, slot);
    if (!c) return bfail(b, LBM_ERR_INVALID_ARG, "no lattice in that slot");
    invalidate(b);
    lbm_status s = enter(b);
    if (s != LBM_OK) return s;
    s = lbm_init(c, rho, ux, uy);
    if (s != LBM_OK) return bfail(b, s, lbm_last_error(c));
    b->slot_status[(size_t)slot] = LBM_OK;
    return leave(b);
}

lbm_status lbm_batch_set_populations(lbm_batch *b, int32_t slot, const double *f)
{
    lbm_ctx *c = get(b, slot);
    if (!c) return bfail(b, LBM_ERR_INVALID_ARG, "no lattice in that slot");
    invalidate(b);
    lbm_status s = enter(b);
    if (s != LBM_OK) return s;
    s = lbm_set_populations(c, f);
    if (s != LBM_OK) return bfail(b, s, lbm_last_error(c));
    b->slot_status[(size_t)slot] = LBM_OK;
    return leave(b);
}

#define BATCH_READ(call)                                                 \
    lbm_ctx *c = get(b, slot);                                           \
    if (!c) return bfail(b, LBM_ERR_INVALID_ARG, "no lattice in that slot"); \
    materialise(b);                                                      \
    lbm_status s = enter(b);                                             \
    if (s != LBM_OK) return s;                                           \
    s = (call);                                                          \
    lbm_status s2 = leave(b);                                            \
    if (s != LBM_OK) return bfail(b, s, lbm_last_error(c));              \
    return s2;

lbm_status lbm_batch_get_populations(lbm_batch *b, int32_t slot, double *f) { BATCH_READ(lbm_get_populations(c, f)) }

lbm_status lbm_batch_moments(lbm_batch *b, int32_t slot, double *rho, double *ux, double *uy)
{
    BATCH_READ(lbm_moments(c, rho, ux, uy))
}

lbm_status lbm_batch_stats(lbm_batch *b, int32_t slot, lbm_step_stats *out) { BATCH_READ(lbm_stats(c, out)) }

lbm_status lbm_batch_limited_sites(lbm_batch *b, int32_t slot, int64_t *idx, int64_t cap, int64_t *n)
{
    BATCH_READ(lbm_limited_sites(c, idx, cap, n))
}

lbm_status lbm_batch_probe(lbm_batch *b, int32_t slot, int64_t site, int64_t capacity)
{
    lbm_ctx *c = get(b, slot);
    if (!c) return bfail(b, LBM_ERR_INVALID_ARG, "no lattice in that slot");
    invalidate(b);  // the launch tables carry each lattice's tail parameters
    lbm_status s = enter(b);
    if (s != LBM_OK) return s;
    s = lbm_probe(c, site, capacity);
    lbm_status s2 = leave(b);
    if (s != LBM_OK) return bfail(b, s, lbm_last_error(c));
    return s2;
}

lbm_status lbm_batch_probe_read(lbm_batch *b, int32_t slot, double *out, int64_t cap, int64_t *n)
{
    BATCH_READ(lbm_probe_read(c, out, cap, n))
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (nsteps < 0) return bfail(b, LBM_ERR_INVALID_ARG, "nsteps must be >= 0");
    if (nsteps == 0 || lbm_batch_size(b) == 0) return LBM_OK;
    lbm_status s = enter(b);
    if (s != LBM_OK) return s;
    s = run_steps(b, nsteps);
    if (s != LBM_OK) return s;
    return leave(b);
}

lbm_status lbm_batch_synchronize(lbm_batch *b)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    BCK(b, cudaStreamSynchronize(b->run));
    materialise(b);
    lbm_status first = LBM_OK;
    for (size_t i = 0; i < b->slots.size(); ++i) {
        lbm_ctx *c = b->slots[i];
        if (!c) continue;
        lbm_status s = lbm_synchronize(c);
        if (s != LBM_OK) {
            b->slot_status[i] = s;
            if (first == LBM_OK) {
                first = s;
                b->err = lbm_last_error(c);
            }
        }
    }
    return first;
}

lbm_status lbm_batch_lattice_status(const lbm_batch *b, int32_t slot)
{
    if (!b || slot < 0 || slot >= (int32_t)b->slots.size() || !b->slots[(size_t)slot]) return LBM_ERR_INVALID_ARG;
    return b->slot_status[(size_t)slot];
}

lbm_status lbm_batch_set_graph(lbm_batch *b, int32_t steps_per_graph)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (steps_per_graph < 0 || steps_per_graph == 1 || (steps_per_graph & 1))
        return bfail(b, LBM_ERR_INVALID_ARG, "steps_per_graph must be 0 or an even number >= 2");
    drop_graph(b);
    b->graph_steps = steps_per_graph;
    return LBM_OK;
}

lbm_status lbm_batch_set_shape(lbm_batch *b, int32_t seg_rows, int32_t waves)
{
    if (!b) return LBM_ERR_INVALID_ARG;
    if (seg_rows != 0 && seg_rows < 4) return bfail(b, LBM_ERR_INVALID_ARG, "seg_rows must be 0 or >= 4");
    if (waves < 1 || waves > 64) return bfail(b, LBM_ERR_INVALID_ARG, "waves must lie in 1 .. 64");
    invalidate(b);
    b->seg_rows = seg_rows;
    b->waves = waves;
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch *b, int32_t trial_steps, double *best_ms)
{
    if (!b || trial_steps < 1) return bfail(b, LBM_ERR_INVALID_ARG, "trial_steps must be >= 1");
    if (lbm_batch_size(b) == 0) return LBM_OK;
    lbm_status s = enter(b);
    if (s != LBM_OK) return s;
    materialise(b);
    // snapshot every lattice: current populations, counters, status, stats ring, counts
    struct Snap {
        lbm_ctx *c;
        int cur;
        void *mem;
    };
    std::vector<Snap> snaps;
    for (lbm_ctx *c : b->slots) {
        if (!c) continue;
        if (!c->ready) return bfail(b, LBM_ERR_STATE, "a lattice of the batch was never initialised");
        const size_t ring = (size_t)c->ring_len * sizeof(DevStats);
        void *mem = nullptr;
        BCK(b, cudaMalloc(&mem, c->field_bytes + ring + 64));
        char *m = (char *)mem;
        BCK(b, cudaMemcpyAsync(m, c->buf[c->cur], c->field_bytes, cudaMemcpyDeviceToDevice, b->run));
        BCK(b, cudaMemcpyAsync(m + c->field_bytes, c->ring, ring, cudaMemcpyDeviceToDevice, b->run));
        BCK(b, cudaMemcpyAsync(m + c->field_bytes + ring, c->counters, 2 * sizeof(long long), cudaMemcpyDeviceToDevice, b->run));
        BCK(b, cudaMemcpyAsync(m + c->field_bytes + ring + 16, c->status, sizeof(unsigned), cudaMemcpyDeviceToDevice, b->run));
        BCK(b, cudaMemcpyAsync(m + c->field_bytes + ring + 32, c->counts, 2 * sizeof(int), cudaMemcpyDeviceToDevice, b->run));
        snaps.push_back({c, c->cur, mem});
    }
    // the work split: automatic segments for 2 .. 16 items per resident warp,
    // or fixed 8- and 16-row segments (an item costs no halo rows; more items
    // even out the warps' different rates, fewer cost less bookkeeping)
    const int Ts[6] = {0, 0, 0, 0, 8, 16};
    const int Ws[6] = {2, 4, 8, 16, 8, 8};
    double best = 1e300;
    int bestT = 0, bestW = 8;
    lbm_status rs = LBM_OK;
    for (int ci = 0; ci < 6; ++ci) {
        const int T = Ts[ci], W = Ws[ci];
        {
            invalidate(b);
            b->seg_rows = T;
            b->waves = W;
            const int gs = b->graph_steps;
            b->graph_steps = 0;
            rs = run_steps(b, 1);  // warm-up (and table build)
            if (rs == LBM_OK) {
                if (cudaEventRecord(b->t0, b->run) != cudaSuccess) rs = LBM_ERR_CUDA;
                if (rs == LBM_OK) rs = run_steps(b, trial_steps);
                if (rs == LBM_OK && cudaEventRecord(b->t1, b->run) != cudaSuccess) rs = LBM_ERR_CUDA;
                float ms = 0.f;
                if (rs == LBM_OK && (cudaEventSynchronize(b->t1) != cudaSuccess ||
                                     cudaEventElapsedTime(&ms, b->t0, b->t1) != cudaSuccess))
                    rs = LBM_ERR_CUDA;
                if (rs == LBM_OK && ms / trial_steps < best) {
                    best = ms / trial_steps;
                    bestT = T;
                    bestW = W;
                }
            }
            b->graph_steps = gs;
            if (rs != LBM_OK) break;
        }
        if (rs != LBM_OK) break;
    }
    // restore the lattices
    materialise(b);
    for (Snap &sn : snaps) {
        lbm_ctx *c = sn.c;
        const size_t ring = (size_t)c->ring_len * sizeof(DevStats);
        char *m = (char *)sn.mem;
        c->cur = sn.cur;
        cudaMemcpyAsync(c->buf[c->cur], m, c->field_bytes, cudaMemcpyDeviceToDevice, b->run);
        cudaMemcpyAsync(c->ring, m + c->field_bytes, ring, cudaMemcpyDeviceToDevice, b->run);
        cudaMemcpyAsync(c->counters, m + c->field_bytes + ring, 2 * sizeof(long long), cudaMemcpyDeviceToDevice, b->run);
        cudaMemcpyAsync(c->status, m + c->field_bytes + ring + 16, sizeof(unsigned), cudaMemcpyDeviceToDevice, b->run);
        cudaMemcpyAsync(c->counts, m + c->field_bytes + ring + 32, 2 * sizeof(int), cudaMemcpyDeviceToDevice, b->run);
    }
    BCK(b, cudaStreamSynchronize(b->run));
    for (Snap &sn : snaps) cudaFree(sn.mem);
    b->dirty = true;  // tables for the restored buffers
    b->phase = 0;
    drop_graph(b);
    b->seg_rows = bestT;
    b->waves = bestW;
    if (rs != LBM_OK) return rs;
    if (best_ms) *best_ms = best;
    return leave(b);
}

int64_t lbm_batch_launch_count(const lbm_batch *b) { return b ? b->launches : 0; }

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err.c_str() : "NULL batch"; }

}  // extern "C"
