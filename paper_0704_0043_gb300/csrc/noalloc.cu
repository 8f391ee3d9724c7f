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
#include <cstring>

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
    size_t counters, status, counts, ring, partials, sel, cand, total;
};

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
    L.ring = off;
    off = align_up(off + sizeof(DevStats), 256);
    L.partials = off;
    off = align_up(off + (size_t)rows * P_NSTAT * sizeof(double), 256);
    const long long sel = k_max < sites ? k_max : sites;
    L.sel = off;
    off = align_up(off + (size_t)(sel > 1 ? sel : 1) * sizeof(int), 256);
    L.cand = off;
    off = align_up(off + (size_t)(ehrenfest ? sites : 1) * sizeof(Cand), 256);
    L.total = off;
    return L;
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_config *cfg, const double *f_in, double *f_out,
                                       lbm_step_stats *stats, void *cuda_stream)
{
    if (!cfg || !f_in || !f_out || f_in == f_out)
        return set_thread_error(LBM_ERR_INVALID_ARG, "lbm_step_noalloc: NULL or aliased arrays");
    if (cfg->precision != LBM_FP64)
        return set_thread_error(LBM_ERR_INVALID_ARG, "lbm_step_noalloc: needs precision LBM_FP64");
    if (lbm_footprint_bytes(cfg) == 0) return LBM_ERR_INVALID_ARG;  // validates cfg, message already set
    if (cfg->limiters & (LBM_LIM_SMOOTH | LBM_LIM_THRESHOLD))
        return set_thread_error(LBM_ERR_INVALID_ARG, "lbm_step_noalloc: no ensemble-dependent limiters");
    const long long sites = (long long)cfg->nx * cfg->ny;
    if (sites > LBM_NOALLOC_MAX_SITES)
        return set_thread_error(LBM_ERR_INVALID_ARG,
                                "lbm_step_noalloc: nx * ny exceeds LBM_NOALLOC_MAX_SITES (262144 sites)");
    const int q = cfg->lattice == LBM_D1Q3 ? 3 : 9;
    const int rows = cfg->lattice == LBM_D2Q9 ? ((cfg->nx + 29) / 30) * ((cfg->ny + 5) / 6) : (cfg->nx + 253) / 254;
    const bool ehr = (cfg->limiters & LBM_LIM_EHRENFEST) != 0;
    const Layout L = layout_for(sites, rows, cfg->k_max, ehr);
    if (L.total > kScratchBytes)
        return set_thread_error(LBM_ERR_INVALID_ARG,
                                "lbm_step_noalloc: the scratch this lattice needs exceeds LBM_NOALLOC_SCRATCH_BYTES");

    // Set-up, once per device with that device current: the device address of
    // the static array (the host-side symbol is only a stand-in for it).
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_thread_error(LBM_ERR_CUDA, "lbm_step_noalloc: no usable current device");
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return set_thread_error(LBM_ERR_CUDA, "lbm_step_noalloc: cudaGetSymbolAddress failed");
        }
        g_scratch_addr[dev] = (unsigned char *)ptr;
    }
    unsigned char *base = g_scratch_addr[dev];
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // Everything that must start at zero: counters, status, candidate counts.
    if (cudaMemsetAsync(base, 0, L.ring, s) != cudaSuccess) return LBM_ERR_CUDA;

    // The kernels address element (k, y, x) at k * plane + y * pitch + kLead + x;
    // the caller's arrays are unpadded (pitch nx, plane nx * ny), so they are
    // passed kLead elements early.  Only lattice sites are ever accessed.
    StepParams p{};
    p.nx = cfg->nx;
    p.ny = cfg->ny;
    p.pitch = cfg->nx;
    p.plane = sites;
    p.boundary = cfg->boundary;
    p.limiters = cfg->limiters;
    p.median_mode = cfg->median_mode;
    p.collide = 1;
    p.eq = cfg->equilibrium == LBM_EQ_ENTROPIC ? 1 : 0;
    p.a = 2.0 * cfg->beta - 1.0;
    p.delta_m = cfg->delta_median;
    p.delta_e = cfg->delta_ehrenfest;
    for (int k = 0; k < 9; ++k) {
        const bool lid = q == 9 && cfg->boundary != LBM_BC_PERIODIC && Lat<9>::cy(k) == -1;
        p.lid[k] = lid ? ((6.0 * Lat<9>::w(k)) * cfg->rho_wall) * ((double)Lat<9>::cx(k) * cfg->u_lid) : 0.0;
        p.lidf[k] = (float)p.lid[k];
        p.lidlo[k] = (float)(p.lid[k] - (double)p.lidf[k]);
        p.rw[k] = 0.0;
        p.rwf[k] = 0.0f;
    }
    p.rho_ref = (float)cfg->rho_ref;
    p.cand = (Cand *)(base + L.cand);
    p.cand_count = (int *)(base + L.counts);
    p.cand_cap = ehr ? (int)sites : 1;
    p.partials = (double *)(base + L.partials);
    p.status = (unsigned *)(base + L.status);
    p.ds_out = nullptr;
    const double *src = f_in - kLead;
    double *dst = f_out - kLead;
    int nblocks = 0;
    if (launch_tiled<double>(q, p, src, dst, &nblocks, s) != cudaSuccess) return LBM_ERR_CUDA;

    FinalParams f{};
    f.nblocks = nblocks;
    f.one_minus_a2 = p.eq ? 1.0 : 1.0 - p.a * p.a;  // entropic f*: the step sums dS(f_in) - dS(f')
    f.eq = p.eq;
    f.k_max = cfg->k_max;
    f.ehrenfest = ehr ? 1 : 0;
    f.collide = 1;
    f.nx = cfg->nx;
    f.ny = cfg->ny;
    f.pitch = cfg->nx;
    f.plane = sites;
    f.partials = p.partials;
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
    f.rho_ref = p.rho_ref;
    if (launch_finalize<double>(q, f, dst, s) != cudaSuccess) return LBM_ERR_CUDA;

    DevStats d{};
    unsigned status = 0;
    if (cudaMemcpyAsync(&d, base + L.ring, sizeof(DevStats), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&status, base + L.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LBM_ERR_CUDA;
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
    if (status & kStatNonfinite) return LBM_ERR_NONFINITE;
    if (status & (kStatTimeout | kStatCandOverflow)) return LBM_ERR_CUDA;
    return LBM_OK;
}
