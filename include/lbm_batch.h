/*
 * lbm_batch.h -- many independent lattices stepped together (C ABI of liblbm).
 *
 * A batch holds lattices of different kinds and sizes (D2Q9 cavities, D1Q3
 * tubes; FP32 storage) and advances all of them with one launch of each step
 * kernel per step: every block of the launch looks up which lattice it serves
 * in a device table, so a single grid covers all cavities (the fused kernel)
 * and a second one all other lattices (the tiled kernel), followed by one tail
 * launch with a block per lattice (Ehrenfests' step, FP64 sums).  Each lattice
 * evolves exactly as it would alone (same per-site arithmetic, bit for bit).
 * Runs of steps can be captured once into a CUDA graph and replayed.  The
 * paper has no batching; the step itself is the one of include/lbm.h
 * (Eq. lbgkLB with the limiters of Sec. 3).
 *
 * Conventions are those of lbm.h: every call returns lbm_status, callers own
 * their arrays (host or device), the library owns the lattices.  A batch runs
 * its device work on a stream of its own, ordered after the caller's stream at
 * every call and before it on return.  One host thread at a time per batch.
 */
#ifndef LBM_BATCH_H
#define LBM_BATCH_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_batch lbm_batch;

/* Creates an empty batch ordered with `cuda_stream` (cudaStream_t as void*). */
lbm_status lbm_batch_create(void *cuda_stream, lbm_batch **out);

/* Frees every lattice of the batch and the batch itself.  NULL is a no-op. */
lbm_status lbm_batch_destroy(lbm_batch *b);

/* Adds a lattice (allocated as by lbm_create; cfg->precision must be
 * LBM_FP32).  *slot receives its id (stable until removed).  Its populations
 * are zero until lbm_batch_init / lbm_batch_set_populations.
 * Errors: LBM_ERR_INVALID_ARG, LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_batch_add(lbm_batch *b, const lbm_config *cfg, int32_t *slot);

/* Removes and frees a lattice. */
lbm_status lbm_batch_remove(lbm_batch *b, int32_t slot);

/* Number of lattices in the batch, and the device bytes they hold. */
int32_t lbm_batch_size(const lbm_batch *b);
int64_t lbm_batch_device_bytes(const lbm_batch *b);

/* Per-lattice calls: as lbm_init, lbm_set_populations, lbm_get_populations,
 * lbm_moments, lbm_stats and lbm_limited_sites of lbm.h. */
lbm_status lbm_batch_init(lbm_batch *b, int32_t slot, const double *rho, const double *ux, const double *uy);
lbm_status lbm_batch_set_populations(lbm_batch *b, int32_t slot, const double *f);
lbm_status lbm_batch_get_populations(lbm_batch *b, int32_t slot, double *f);
lbm_status lbm_batch_moments(lbm_batch *b, int32_t slot, double *rho, double *ux, double *uy);
lbm_status lbm_batch_stats(lbm_batch *b, int32_t slot, lbm_step_stats *out);
lbm_status lbm_batch_limited_sites(lbm_batch *b, int32_t slot, int64_t *idx, int64_t cap, int64_t *n);

/* Control-point record of one lattice: as lbm_probe / lbm_probe_read of lbm.h. */
lbm_status lbm_batch_probe(lbm_batch *b, int32_t slot, int64_t site, int64_t capacity);
lbm_status lbm_batch_probe_read(lbm_batch *b, int32_t slot, double *out, int64_t cap, int64_t *n);

/* Advances every lattice of the batch by nsteps limited LBGK steps
 * (asynchronous; statuses surface at the next synchronising call).
 * Errors: LBM_ERR_STATE (a lattice was never initialised), LBM_ERR_CUDA. */
lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps);

/* Waits for the batch and collects every lattice's status (a lattice that
 * met a nonfinite site reports LBM_ERR_NONFINITE); returns the first failing
 * one, LBM_OK if none.  The other lattices are unaffected: their steps are
 * independent. */
lbm_status lbm_batch_synchronize(lbm_batch *b);

/* Status of one lattice as collected by lbm_batch_synchronize; it stays set
 * until the lattice is re-initialised (lbm_batch_init /
 * lbm_batch_set_populations) or removed.  LBM_ERR_INVALID_ARG for an empty
 * slot. */
lbm_status lbm_batch_lattice_status(const lbm_batch *b, int32_t slot);

/* CUDA-graph replay: runs of `steps_per_graph` steps (even, >= 2; 0 turns it
 * off) are captured once after the batch changes and replayed. */
lbm_status lbm_batch_set_graph(lbm_batch *b, int32_t steps_per_graph);

/* Work-split autotuner: times `trial_steps` batched steps for each candidate
 * (automatic segments for 2, 4, 8 or 16 work items per resident warp; fixed
 * 8- or 16-row segments),
 * keeps the fastest, and restores every lattice's state, counters and stats
 * to what they were before.  *best_ms receives the winning time per step
 * (may be NULL). */
lbm_status lbm_batch_tune(lbm_batch *b, int32_t trial_steps, double *best_ms);

/* Fixes the fused kernel's work split: seg_rows = rows per work item (a warp
 * walking a strip of 62 columns; 0: automatic, else >= 4), waves 1 .. 64 (with
 * automatic segments: about this many work items per resident warp over the
 * fused lattices together; the items are handed out dynamically).  The split
 * changes the speed only, never a result.  Errors: LBM_ERR_INVALID_ARG. */
lbm_status lbm_batch_set_shape(lbm_batch *b, int32_t seg_rows, int32_t waves);

/* Kernel launches enqueued by lbm_batch_step so far (graph replays count
 * their captured launches). */
int64_t lbm_batch_launch_count(const lbm_batch *b);

/* Last error message of the batch (never NULL). */
const char *lbm_batch_last_error(const lbm_batch *b);

#ifdef __cplusplus
}
#endif
#endif
