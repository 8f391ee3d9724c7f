// noalloc.cu -- one limited step of a lattice held in caller memory, with no
// device allocation (lbm_step_noalloc in include/lbm.h).
//
// Some callers cannot call cudaMalloc: a host framework that owns all device
// memory through its own caching pool and forbids allocations behind its back,
// a real-time or embedded host that allows no allocation once it is running,
// or a process near its memory limit that must not grow its footprint.  For
// them this entry point runs the same step kernels as an LBM_FP64 context (the
// tiled kernel and the one-block tail) directly on the caller's FP64 arrays,
// and takes every scratch buffer (block partial sums, Ehrenfests' candidates,
// the selected sites, counters, status and the stats record) from one
// file-scope static device array of fixed size.
#include <cstdint>
#include <cstring>
#include <string>

#include "../../include/lbm.h"
#include "internal.h"
#include "lattice.cuh"

using namespace lbm;

// Scratch of lbm_step_noalloc: shared by every call on a device, kept (with
// the last call's contents) by every GPU that loads the library until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LBM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr size_t kScratchBytes = LBM_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
    size_t counters, status, counts, chunk_cnt, ring, partials, partials2, sel, cand, total;
};

// Everything before `ring` is cleared by each call.
Layout layout_for(long long sites, int rows, long long k_max, bool ehrenfest)
{
    Layout L{};
    size_t off = 0;
    L.counters = off;
    off = align_up(off + 2 * sizeof(long long), 256);
    L.status = off;
    off = align_up(off + sizeof(unsigned), 256);
    L.counts = off;
    off = align_up(off + 2 * sizeof(int), 256);
    L.chunk_cnt = off;
    off = align_up(off + (size_t)chunks_for(rows) * sizeof(unsigned), 256);
    L.ring = off;
    off = align_up(off + sizeof(DevStats), 256);
    L.partials = off;
    off = align_up(off + (size_t)rows * P_NSTAT * sizeof(double), 256);
    L.partials2 = off;
    off = align_up(off + (size_t)chunks_for(rows) * P_NSTAT * sizeof(double), 256);
    const long long sel = k_max < sites ? k_max : sites;
    L.sel = off;
    off = align_up(off + (size_t)(sel > 1 ? sel : 1) * sizeof(int), 256);
    L.cand = off;
    off = align_up(off + (size_t)(ehrenfest ? sites : 1) * sizeof(Cand), 256);
    L.total = off;
    return L;
}

// A device array of `bytes` bytes on the current device (device or managed
// memory): the kernels below dereference these pointers, so a host address or
// another GPU's memory is rejected before anything is launched.
bool on_current_device(const void *ptr, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

lbm_status cuda_error(cudaError_t e, const char *what)
{
    static thread_local std::string msg;
    msg = std::string("lbm_step_noalloc: ") + what + " failed: " + cudaGetErrorString(e);
    cudaGetLastError();
    return set_thread_error(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, msg.c_str());
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_config *cfg, const double *f_in, double *f_out,
                                       lbm_step_stats *stats, void *cuda_stream)
{
    if (!cfg || !f_in || !f_out) return set_thread_error(LBM_ERR_INVALID_ARG, "lbm_step_noalloc: NULL argument");
    if (cfg->precision != LBM_FP64)
        return set_thread_error(LBM_ERR_INVALID_ARG, "lbm_step_noalloc: needs precision LBM_FP64");
    if (lbm_footprint_bytes(cfg) == 0) return LBM_ERR_INVALID_ARG;  // validates cfg, message already set
    if (cfg->limiters & kLimEnsemble)
        return set_thread_error(LBM_ERR_INVALID_ARG, "lbm_step_noalloc: no ensemble-dependent limiters");
    const long long sites = (long long)cfg->nx * cfg->ny;
    if (sites > LBM_NOALLOC_MAX_SITES)
        return set_thread_error(LBM_ERR_INVALID_ARG,
                                "lbm_step_noalloc: nx * ny exceeds LBM_NOALLOC_MAX_SITES (262144 sites)");
    const int q = cfg->lattice == LBM_D1Q3 ? 3 : 9;
    // one row of block partial sums per tiled-kernel block (the launch below
    // must use exactly this many)
    const int rows = tiled_blocks_for(q, cfg->nx, cfg->ny);
    const bool ehr = (cfg->limiters & LBM_LIM_EHRENFEST) != 0;
    const Layout L = layout_for(sites, rows, cfg->k_max, ehr);
    if (L.total > kScratchBytes)
        return set_thread_error(LBM_ERR_INVALID_ARG,
                                "lbm_step_noalloc: the scratch this lattice needs exceeds LBM_NOALLOC_SCRATCH_BYTES");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return set_thread_error(LBM_ERR_CUDA, "lbm_step_noalloc: device ordinal above the supported 64");
    // Both arrays must be device memory of the current device, and the output
    // must not overlap the input anywhere.
    const size_t bytes = (size_t)q * (size_t)sites * sizeof(double);
    if (!on_current_device(f_in, dev) || !on_current_device(f_out, dev) ||
        !on_current_device((const char *)f_in + bytes - 1, dev) ||
        !on_current_device((const char *)f_out + bytes - 1, dev))
        return set_thread_error(LBM_ERR_INVALID_ARG,
                                "lbm_step_noalloc: f_in and f_out must be device memory of the current device");
    {
        const uintptr_t a0 = (uintptr_t)f_in, b0 = (uintptr_t)f_out;
        if (a0 < b0 + bytes && b0 < a0 + bytes)
            return set_thread_error(LBM_ERR_INVALID_ARG, "lbm_step_noalloc: f_in and f_out overlap");
    }

    // Set-up, once per device with that device current: the device address of
    // the static array (the host-side symbol is only a stand-in for it).
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_error(e, "cudaGetSymbolAddress");
        g_scratch_addr[dev] = (unsigned char *)ptr;
    }
    unsigned char *base = g_scratch_addr[dev];
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // Everything that must start at zero: counters, status, candidate counts,
    // the tiled kernel's chunk counters.
    if ((e = cudaMemsetAsync(base, 0, L.ring, s)) != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");

    // The kernels address element (k, y, x) at k * plane + y * pitch + kLead + x;
    // the caller's arrays are unpadded (pitch nx, plane nx * ny), so they are
    // passed kLead elements early.  Only lattice sites are ever accessed.
    StepParams p = cfg_step_params(*cfg, q, cfg->nx, sites, 1, cfg->limiters);
    p.cand = (Cand *)(base + L.cand);
    p.cand_count = (int *)(base + L.counts);
    p.cand_cap = ehr ? (int)sites : 1;
    p.partials = (double *)(base + L.partials);
    p.partials2 = (double *)(base + L.partials2);
    p.chunk_cnt = (unsigned *)(base + L.chunk_cnt);
    p.fx_rows = nullptr;
    p.status = (unsigned *)(base + L.status);
    p.work = nullptr;
    p.ens = nullptr;
    const double *src = f_in - kLead;
    double *dst = f_out - kLead;
    int nblocks = 0;
    if ((e = launch_tiled<double>(q, p, src, dst, &nblocks, s)) != cudaSuccess) return cuda_error(e, "step kernel launch");
    if (nblocks != rows)
        return set_thread_error(LBM_ERR_CUDA, "lbm_step_noalloc: block count differs from the scratch layout");

    FinalParams f = cfg_final_params(*cfg, p, 1, cfg->limiters, chunks_for(nblocks));
    f.fixed = 0;
    f.work = nullptr;
    f.partials = p.partials2;
    f.cand = p.cand;
    f.cand_count = p.cand_count;
    f.cand_cap = p.cand_cap;
    f.sel = (int *)(base + L.sel);
    {
        const long long sel = cfg->k_max < sites ? cfg->k_max : sites;
        f.sel_cap = (int)(sel > 1 ? sel : 1);
    }
    f.sel_count = p.cand_count + 1;
    f.status = p.status;
    f.stats_ring = (DevStats *)(base + L.ring);
    f.ring_len = 1;
    f.counters = (long long *)(base + L.counters);
    f.src = src;
    if ((e = launch_finalize<double>(q, f, dst, s)) != cudaSuccess) return cuda_error(e, "tail kernel launch");

    DevStats d{};
    unsigned status = 0;
    if ((e = cudaMemcpyAsync(&d, base + L.ring, sizeof(DevStats), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&status, base + L.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_error(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->step = d.step;
        stats->mass = d.mass;
        stats->sum_dS = d.sum_dS;
        stats->dS_lbgk = d.dS_lbgk;
        stats->dS_lim = d.dS_lim;
        stats->n_pos = d.n_pos;
        stats->n_med = d.n_med;
        stats->n_ehr = d.n_ehr;
        stats->n_cand = d.n_cand;
        stats->n_bad = d.n_bad;
        stats->status = d.status;
    }
    if (status & kStatNonfinite)
        return set_thread_error(LBM_ERR_NONFINITE, "lbm_step_noalloc: a site had rho <= 0, f*_k <= 0 or a nonfinite value");
    if (status & kStatTimeout)  // no kernel of this path waits today; kept in step with the context path
        return set_thread_error(LBM_ERR_TIMEOUT, "lbm_step_noalloc: a bounded device wait gave up");
    if (status & kStatCandOverflow)
        return set_thread_error(LBM_ERR_CUDA, "lbm_step_noalloc: Ehrenfests' candidate buffer overflowed");
    return LBM_OK;
}
