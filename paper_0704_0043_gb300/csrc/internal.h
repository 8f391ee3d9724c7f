// internal.h -- shared declarations of the liblbm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

// Device layout of a population field: plane-major, rows padded.  Element
// (k, y, x) lives at k * plane + y * pitch + kLead + x.  The kLead elements in
// front of every row and the kTail (at least) after it are zero and never
// written, so a warp may read a window of columns around its strip a few
// elements past either edge of the lattice (the fused kernel's 16-byte
// copies reach up to 68 columns past the last column).
constexpr int kLead = 32;
constexpr int kTail = 96;
__host__ __device__ inline int row_pitch(int nx) { return ((nx + 31) / 32) * 32 + kLead + kTail; }

// Boundary kinds (LBM_BC_*): which directions wrap, and whether the outer
// ring of nodes lies on the walls.
__host__ __device__ inline bool bc_wrap_x(int b) { return b == 1 || b == 2; }
__host__ __device__ inline bool bc_wrap_y(int b) { return b == 1; }
__host__ __device__ inline bool bc_node_walls(int b) { return b == 3 || b == 4; }

// Ensemble-dependent limiter bits (LBM_LIM_SMOOTH | LBM_LIM_THRESHOLD |
// LBM_LIM_ENTTHRESH): a pass with any of them first reduces dS over the lattice.
constexpr unsigned kLimEnsemble = 8u | 16u | 32u;

// State of the device solve of Eq. EntThresh (entthresh.cu): a radix descent
// over the bit patterns of the pass's dS field, 8 bits a level, keeping
// prefix (the determined high bits of the bin that holds dS_0), and the count
// and sum of the values above that bin.
struct EntState {
    double rhs;                  // delta_0 (1 - (2 beta - 1)^2) sum dS
    double s_above;              // sum of the values above the current bin
    unsigned long long m_above;  // their count
    unsigned long long prefix;   // determined high bits (in place)
    double t;                    // result: dS_t = max(dS_0, threshold_delta)
    int done;                    // the solve ended early (no value, rhs <= 0, or dS_0 = 0)
    int pad;
    unsigned long long cnt[256];  // histogram of the current level: counts
    double sum[256];              // and sums
};

// Sticky device status bits.
enum : unsigned { kStatNonfinite = 1u, kStatTimeout = 2u, kStatCandOverflow = 4u };

// Block rows of the tiled kernel are summed in chunks of kChunkRows by the
// last block of each chunk to finish (fixed order within the chunk); the tail
// kernel reduces the chunk rows.
constexpr int kChunkRows = 256;
__host__ __device__ inline int chunks_for(int blocks) { return (blocks + kChunkRows - 1) / kChunkRows; }

// Per-block partial sums written by the step kernels, reduced in a fixed
// order by the finalise kernel.
enum { P_MASS = 0, P_SUM_DS, P_SUM_IN, P_DS_LIM, P_NPOS, P_NMED, P_NBAD, P_NSTAT };

// The fused kernel hands out its work items dynamically, so which warp sums
// which sites varies from run to run.  To keep the step statistics the same
// bit for bit, it sums them exactly: each work item's FP32 sums (a fixed
// evaluation order within the item) are converted to 128-bit two's-complement
// fixed point in units of 2^-64 and added as integers, whose sum does not
// depend on the order.  A fixed-point partial row holds kFxWords words:
// FX_SUM + 2 s (low word) and FX_SUM + 2 s + 1 (high word) for the FP
// statistic s = P_MASS (sum of rho - rho_ref) .. P_DS_LIM; the site and
// limiter counts; and a bit per FP statistic that met a nonfinite or
// out-of-range (>= 2^63) item sum.
// Each block of the fused kernel adds its row atomically into accumulator row
// (block % kFxRows) of its lattice's partials; the tail kernel sums the
// kFxRows rows and clears them.
constexpr int kFxWords = 16;
constexpr int kFxRows = 8;
enum { FX_SUM = 0, FX_SITES = 8, FX_NPOS, FX_NMED, FX_NBAD, FX_BAD };

// Ehrenfests' candidate: FP64 key dS(f') (NaN: not keyed yet), phi of the
// limiter pass, site index, and dS(f') in FP32 (the key rounded, or the FP32
// value the candidate was recorded on; within 1/64 of the key).
struct Cand {
    double key;
    double phi;
    int32_t site;
    float ds32;
};

// Device-wide preselection of Ehrenfests' candidates: when a pass records
// more candidates than the tail's block holds in shared memory, the tail runs
// as a grid of one block per SM.  The grid finds, by two 12-bit radix levels
// over the FP32 dS bit patterns of the candidates certainly above delta, a
// lower bound T of the k-th largest; keys in FP64 the candidates with FP32 dS
// of at least T (1 - 1/32) and those near delta; counts the valid candidates;
// and hands block 0 the short list of valid candidates at or above the bound,
// which holds every candidate the exact top-k can take.
constexpr int kSelBins = 4096;   // bins of one radix level
// Lattices of at least this many sites get the grid tail.  Its launch costs
// one to two microseconds per step, a tenth of a smaller lattice's step; on
// those, one block keys and selects the candidates, about 0.1 us per
// candidate without a key (a tenth of a second when every site of a 2^20-site
// lattice is one).
constexpr long long kSelMinSites = 1ll << 20;
constexpr int kSelList = 65536;  // the longest list block 0 is handed
struct SelState {
    unsigned hist1[kSelBins];  // level 1: bits 30..19 of the FP32 dS pattern
    unsigned hist2[kSelBins];  // level 2: bits 18..7 within level 1's bin
    unsigned bar;              // grid barrier: arrivals so far (block 0 resets it)
    unsigned count;            // list entries (more than kSelList: overflow)
    unsigned n_valid;          // candidates with dS above delta
    unsigned pad;
    int list[kSelList];        // candidate indices
};

struct DevStats {  // mirrors lbm_step_stats
    long long step;
    double mass, sum_dS, dS_lbgk, dS_lim;
    long long n_pos, n_med, n_ehr, n_cand, n_bad;
    int status;
    int reserved;
};

struct StepParams {
    int nx, ny, pitch;
    long long plane;           // elements per population plane
    int boundary;              // LBM_BC_*
    unsigned limiters;
    int median_mode;
    int collide;               // 1: free flight + collision; 0: limiter pass on stored state
    int eq;                    // 0: polynomial f*, quadratic dS; 1: entropic f*, exact dS (FP64 storage)
    double a;                  // 2 beta - 1
    double delta_m, delta_e;
    double u_lid;              // lid x-velocity (wall rule of LBM_BC_DIFFUSIVE)
    double beta;               // LBGK / ELBM relaxation parameter (Eq. elbm)
    int coll;                  // LBM_COLL_* (ELBM: FP64 entropic path)
    int phi_rule;              // LBM_PHI_* (LBM_PHI_ENTROPY: FP64 entropic path)
    double lid[9];             // ((6 W_k) rho_wall) (c_kx u_lid), added on links through the lid
    // the same term for FP32 arithmetic as an unevaluated sum hi + lo: adding
    // both parts keeps the rounding of the constant out of every wall step
    // (a single FP32 constant would bias the lid momentum by ~1e-9 per step)
    float lidf[9], lidlo[9];
    float rho_ref;             // FP32 storage holds g_k = f_k - rho_ref W_k
    double rw[9];              // rho_ref W_k in FP64 (absolute value of FP32 storage: (double) g + rw)
    float rwf[9];              // rho_ref W_k in FP32
    // scratch (library-owned)
    Cand *cand;
    int *cand_count;
    int cand_cap;
    double *partials;          // tiled kernel: [blocks][P_NSTAT] doubles
    double *partials2;         // tiled kernel: [chunks][P_NSTAT] sums of kChunkRows block rows each
    unsigned long long *fx_rows;  // fused kernel: [kFxRows][kFxWords] fixed-point accumulators (own region)
    unsigned *chunk_cnt;       // tiled kernel: blocks of each chunk done this launch (reset by its last block)
    unsigned *status;
    int *work;                 // fused kernel: counter of work items handed out (nullptr: one item per warp)
    double *ds_out;            // optional FP64 dS(f') field (nx * ny) or nullptr
    // ensemble-dependent limiters (LBM_LIM_SMOOTH / LBM_LIM_THRESHOLD)
    double smooth_delta, smooth_k, threshold_c, threshold_delta;
    const double *ens;         // {E(dS), smooth_delta / E^smooth_k, sum dS, count} of this pass (the ensemble reduction)
    void *ent_field;           // LBM_LIM_ENTTHRESH: dS of every site (compute type; 0 where excluded)
    EntState *ent;             // LBM_LIM_ENTTHRESH: the solve's state; ent->t is the pass's dS_t
};

struct FinalParams {
    int nblocks;               // partial rows to reduce
    int fixed;                 // the rows are fixed-point rows of the fused kernel
    int *work;                 // work-item counter to clear for the next step, or nullptr
    double one_minus_a2;       // 1 - (2 beta - 1)^2
    long long k_max;
    int ehrenfest;             // apply Ehrenfests' step
    int collide;
    int eq;                    // as StepParams::eq
    int nx, ny, pitch;
    long long plane;
    double *partials;          // fused kernel: the accumulator rows, cleared once read
    Cand *cand;
    int *cand_count;
    int cand_cap;
    int *sel;                  // selected sites out
    int sel_cap;
    int *sel_count;
    unsigned *status;
    DevStats *stats_ring;
    int ring_len;
    long long *counters;       // [0] steps taken (incremented when collide), [1] records written
    // pre-step populations of the pass (FP32 / BF16 / FP16 storage): the
    // Ehrenfests' step evaluates f*(m) from them, with the same FP32 free
    // flight as the step kernel, so the stored result is rounded once
    const void *src;
    int boundary;
    double a, delta_e;
    double lid[9];
    float lidf[9], lidlo[9];
    float rho_ref;
    double rw[9];
    // control-point record (Sec. 4.4.2): after each step, rho, u_x, u_y of site
    // probe_site into probe[3 ((step - 1) mod probe_cap) ...]; probe == nullptr: off
    double *probe;
    long long probe_cap;
    int probe_site;
    // dense candidates: the grid's shared selection state (launches of more
    // than one block only; nullptr otherwise; FinalParams{} zeroes it)
    SelState *sel_state;
};

// Arguments of one fused-kernel instance (a lattice, its buffers and its
// strip / segment decomposition).
struct FusedArgs {
    StepParams p;
    const void *src;  // float, __nv_bfloat16 or __half deviations
    void *dst;
    int strips, seg_rows, items, blocks;  // work items: strips of 62 finished columns x row segments
    float a, b2, delta_m, thr_e, rho_ref;  // b2 = 2 beta
    float lid4, lid7, lid8;  // FP32 moving-wall terms of the links through the lid (hi + lo)
    float lo4, lo7, lo8;
};

// One tiled-kernel instance (batched launches) and one tail instance.
struct TiledArgs {
    StepParams p;
    const void *src;
    void *dst;
    int gx, blocks;  // blocks along x, blocks in total
};
struct FinalArgs {
    FinalParams p;
    void *f;
};
// One tube-kernel instance of a batched launch (FP32 D1Q3 lattices).
struct TubeArgs {
    StepParams p;
    const void *src;
    void *dst;
};

// Launchers (stream-ordered, no synchronisation).  Return cudaGetLastError().
template <typename T>
cudaError_t launch_tiled(int q, const StepParams &p, const T *src, T *dst, int *nblocks,
                         cudaStream_t s);
// The tail: one block, or (grid > 1, p.sel_state set) a cooperative grid of
// `grid` blocks that preselects dense candidates; the launch returns the
// launch error without a fallback.
template <typename T>
cudaError_t launch_finalize(int q, const FinalParams &p, T *f, cudaStream_t s, int grid = 1);
// Blocks of the tail's cooperative grid on this device: one per SM (0 when a
// block does not fit or the device has no cooperative launch).
template <typename T>
int finalize_grid(int q);
// Field kernels take the StepParams of the context for the layout (nx, ny,
// pitch, plane) and the FP32 storage offsets (rw).
template <typename T>
cudaError_t launch_init(int q, const StepParams &p, const double *rho, const double *ux, const double *uy, T *f,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_moments(int q, const StepParams &p, const T *f, double *rho, double *ux, double *uy,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_get(int q, const StepParams &p, const T *f, double *out, cudaStream_t s);
template <typename T>
cudaError_t launch_set(int q, const StepParams &p, const double *in, T *f, cudaStream_t s);
template <typename T>
cudaError_t launch_delta_s(int q, const StepParams &p, const T *f, double *out, cudaStream_t s);
// E(dS) of the pass p is about to run and the smooth limiter's alpha, into
// ens[2 kEnsBlocks], ens[2 kEnsBlocks + 1] (ens[0 .. 2 kEnsBlocks) is scratch).
constexpr int kEnsBlocks = 608;
// Behind them (in doubles from the start of the E(dS) scratch): {E, alpha, sum,
// count}, then kFxRows fixed-point rows of the fused E(dS) pass and its
// work-item counter (launch_fused_epass).
constexpr int kEnsFxOffset = 2 * kEnsBlocks + 4;
constexpr int kEnsDoubles = kEnsFxOffset + 8 * 16 + 2;
template <typename S>
cudaError_t launch_fused_epass(const StepParams &p, const S *src, cudaStream_t s);
template <typename T>
cudaError_t launch_ens_mean(int q, const StepParams &p, const T *src, double *ens, cudaStream_t s);
// Eq. EntThresh on the field p.ent_field (filled by the ensemble reduction):
// p.ent->t = max(dS_0, threshold_delta).  T is the compute type of the field.
template <typename T>
cudaError_t launch_entthresh(const StepParams &p, double delta0, long long n, cudaStream_t s);
// launches of one EntThresh solve (for the launch count)
int entthresh_launches(bool fp64);

// Sets the calling thread's error message (read by lbm_last_error(NULL)); returns s.
int set_thread_error_impl(int s, const char *msg);
#define set_thread_error(s, msg) ((lbm_status)::lbm::set_thread_error_impl((int)(s), (msg)))

// Fused D2Q9 step for LBM_BC_WALLS (row-streaming kernel; FP32, BF16 or FP16
// storage).
template <typename S>
cudaError_t launch_fused_d2q9(const StepParams &p, const S *src, S *dst, int *nblocks, cudaStream_t s);
int fused_d2q9_blocks(int nx, int ny);  // most blocks (partial-sum rows) any launch of the lattice uses
int fused_slots(int elem_bytes, bool batched);  // resident work items (warps) of one wave
// Fills the instance arguments: row segments of `seg_rows` rows (0: about
// `slots` work items); returns the block count.
int fused_make_args(const StepParams &p, const void *src, void *dst, int seg_rows, int slots, FusedArgs *out);
// Batched launches.  Fused: `items` work items over all instances, item i
// being item map[i].y of instance map[i].x, handed out dynamically through
// the counter *work (cleared by the tail after the launch).  Tiled: `blocks`
// blocks, block b running instance map[b].x as its block map[b].y.
cudaError_t launch_fused_batched(const FusedArgs *table, const int2 *map, int items, int *work, cudaStream_t s);
cudaError_t launch_tiled_batched_f32(int q, const TiledArgs *table, const int2 *map, int blocks, cudaStream_t s);
cudaError_t launch_finalize_batched_f32(int q, const FinalArgs *table, int n, cudaStream_t s);
// D1Q3 streaming step (FP32 / FP64 storage): *chunked is false when the grid
// fits one chunk of the tail's reduction, whose rows the tail then reads itself.
template <typename S>
cudaError_t launch_tube(const StepParams &p, const S *src, S *dst, int *nblocks, bool *chunked, cudaStream_t s);
bool tube_applies(const lbm_config &c, unsigned limiters);  // the pass runs on the tube kernel
// Batched FP32 tubes: `items` work items (groups of chunks, item i = group
// map[i].y of tube map[i].x) handed out through *work; each item writes its
// tube's partial row of its group (the tail reads tube_groups(nx) rows).
cudaError_t launch_tube_batched(const TubeArgs *table, const int2 *map, int items, int *work, cudaStream_t s);
int tube_groups(int nx);
int tube_blocks(bool fp64, int nx);                          // blocks (partial rows) of one launch
int sm_count();
int tiled_grid_x(int q, int nx);
int tiled_blocks_for(int q, int nx, int ny);
bool fused_d2q9_fits(long long plane);  // 32-bit plane offsets inside the kernel

}  // namespace lbm

// Library-owned state of one lattice (opaque to callers, see include/lbm.h).
struct lbm_ctx {
    lbm_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int q = 9;
    int pitch = 0;
    long long plane = 0;
    size_t elem = 4;
    size_t field_bytes = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    lbm::Cand *cand = nullptr;
    int cand_cap = 0;
    lbm::SelState *sel_state = nullptr;  // Ehrenfests' limiter: the cooperative tail's selection state
    int fin_grid = 0;                     // blocks of the cooperative tail (0: one-block tail only)
    bool capturing = false;               // a graph capture is in progress (one-block tail)
    double *ens = nullptr;  // [kEnsBlocks][2] partial sums and counts of dS, then E(dS), alpha, sum, count
    void *ent_field = nullptr;   // LBM_LIM_ENTTHRESH: the pass's dS field
    lbm::EntState *ent = nullptr;  // LBM_LIM_ENTTHRESH: solve state
    int *counts = nullptr;  // [0] candidate count, [1] chosen count, [2] fused work items handed out, [3] unused
    int *sel = nullptr;
    int sel_cap = 0;
    double *partials = nullptr;
    int partial_rows = 0;
    unsigned *chunk_cnt = nullptr;  // tiled kernel: per-chunk block counters
    unsigned *status = nullptr;
    lbm::DevStats *ring = nullptr;
    int ring_len = 1;
    long long *counters = nullptr;  // [0] steps, [1] records
    double *stage = nullptr;
    size_t stage_bytes = 0;
    bool ready = false;
    bool timing = false;
    bool timing_now = false;    // the current pass records its events
    int timing_every = 1;       // record one pass in this many
    long long timing_pass = 0;  // passes since timing was enabled
    std::vector<cudaEvent_t> events;  // three per timed step
    size_t events_used = 0;
    long long launches = 0;
    int64_t device_bytes = 0;
    // CUDA-graph replay of runs of graph_steps steps (0: off): one graph per
    // starting buffer, captured on gstream (the context's own stream may be
    // the legacy default stream, which cannot be captured)
    int graph_steps = 0;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long graph_launches = 0;  // kernel launches one replay performs
    // control-point record (lbm_probe)
    double *probe = nullptr;
    long long probe_cap = 0, probe_alloc = 0, probe_step0 = 0;
    int probe_site = -1;
    std::string err;
};

namespace lbm {
// Geometry and physics of a step for configuration g, stored with row pitch
// `pitch` and `plane` elements per population plane; every scratch pointer is
// left null for the caller to fill.
StepParams cfg_step_params(const lbm_config &g, int q, int pitch, long long plane, int collide, unsigned limiters);
// The tail's parameters that follow from g and from the step's p (scratch
// pointers null).
FinalParams cfg_final_params(const lbm_config &g, const StepParams &p, int collide, unsigned limiters, int nblocks);
// Per-step parameters of a context (collide = 0 for a limiter pass).
StepParams ctx_step_params(lbm_ctx *c, int collide, unsigned limiters);
// The fused kernel's accumulator rows of a context (the tail's partials when fixed = 1).
double *ctx_fx_rows(lbm_ctx *c);
FinalParams ctx_final_params(lbm_ctx *c, int collide, unsigned limiters, int nblocks);
bool ctx_uses_fused(const lbm_ctx *c);
}  // namespace lbm
