/*
 * mdgb_batch.h - ensembles of independent periodic Lennard-Jones systems.
 *
 * Meyer (2013), arXiv:1305.4196, Sec. II.C: the task functor can carry which copy
 * of a system a task works on, so that several systems share one schedule.  Here
 * an ensemble of independent systems of uneven size is advanced together, every
 * call in ONE persistent kernel launch (replayed from a CUDA graph) that takes its
 * work from a device table over all systems:
 *   - a system of at most one_cta_max atoms (2,048 unless md_batch_autotune picks
 *     1,024 or 4,096), or one whose box is under 6 (r_cut + skin) on a side, is one
 *     task: one CTA holds it in shared memory for all steps of the call (linked
 *     cells rebuilt every step, no list);
 *   - a larger system is advanced in phases of tasks that any CTA may take: when
 *     its Verlet lists are due (at the start of a call, and after a step in which
 *     some atom moved more than skin/2), binning in atom chunks, a scan of the cell
 *     counts, an ordering of each cell and the lists of each 2x2x2-cell block; every
 *     step, the forces and velocity Verlet of each block with its 4x4x4-cell
 *     neighbourhood staged in shared memory.  A phase starts when every task of the
 *     one before has finished; no task waits for anything.
 * Both paths use FP32 pair arithmetic, Q31.32 fixed-point forces with the FP64 cutoff
 * decision near r_cut, and FP64 velocity Verlet, so results are bit-reproducible.
 * All systems share the pair parameters (one species), r_cut, skin (the lists of the
 * larger systems) and dt, in mixed precision.
 * Atom arrays are concatenated in system order (system k's atoms after those of
 * systems 0..k-1), N x 3 row-major, host or device as the device_ptrs flag says; the
 * library copies in and out.  Every call returns MD_OK or a negative MD_ERR_* code.
 * A CTA that finds no work for its wait budget (md_batch_set_wait_budget) ends the
 * launch with MD_ERR_TIMEOUT; the ensemble's state is then undefined until the next
 * md_batch_set_state.
 * No counterpart in the paper beyond the replica remark above.
 */
#ifndef MDGB_BATCH_H
#define MDGB_BATCH_H

#include <stdint.h>

#include "mdgb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_batch md_batch;

/*
 * n_systems systems with n_atoms[k] atoms in periodic boxes boxes[3k..3k+2]
 * (each side at least 2 r_cut; systems above 8,192 atoms need sides of at least
 * 6 (r_cut + skin)).  params: one species, MD_MIXED; the stream field selects the
 * stream of the launches.
 */
int md_batch_create(int32_t n_systems, const int64_t *n_atoms, const double *boxes, double r_cut, double skin,
                    const md_params *params, md_batch **out);

/* Positions and velocities (N_total x 3); species may be NULL (all 0). */
int md_batch_set_state(md_batch *b, const double *pos, const double *vel, const int32_t *species,
                       int device_ptrs);

/* Advance every system by n_steps velocity-Verlet steps; synchronises. */
int md_batch_step(md_batch *b, int32_t n_steps);

/* Forces at the current positions (N_total x 3). */
int md_batch_forces(md_batch *b, double *f_out, int device_ptrs);

/* Potential and kinetic energy of every system (host arrays of n_systems). */
int md_batch_energies(md_batch *b, double *pe, double *ke);

/*
 * Positions (wrapped into each box; add image * L for unwrapped coordinates),
 * velocities and image counters (N_total x 3 int32); any output may be NULL.
 */
int md_batch_get_state(md_batch *b, double *pos, double *vel, int32_t *image, int device_ptrs);

/*
 * How each system runs: path[k] = 0 (one CTA for the whole call) or 1 (block
 * tasks over many CTAs); threads[k], the CTA size of the launch; cell_range[k]
 * (path 0: cells at least r_cut / cell_range wide; path 1: 1).  Host arrays of
 * n_systems; any may be NULL.
 */
int md_batch_layout(md_batch *b, int32_t *path, int32_t *threads, int32_t *cell_range);

/*
 * Autotuner: times 10 steps of the whole ensemble per candidate (the state is
 * restored afterwards) and keeps the fastest: the CTA size (128, 256, 512), then
 * the largest system run by one CTA (1,024, 2,048, 4,096 atoms), then for each
 * size bucket of one-CTA systems present ([256, 512), [512, 1024), ..., [4096,
 * 8192] atoms) cells of r_cut or r_cut / 2.  With cache_path non-NULL, a shape
 * found in that JSON file (written for the same GPU name) is used without timing;
 * otherwise the file is written with the chosen shape.
 */
int md_batch_autotune(md_batch *b, const char *cache_path);

/*
 * The wait budget of the launch: a CTA that finds no claimable task for
 * budget_cycles SM clock cycles (0: the default, 2^34) sets a timeout and ends,
 * and the call returns MD_ERR_TIMEOUT.  held_system >= 0 keeps that system's first
 * phase from ever becoming ready (nothing releases it), so that a test can make the
 * wait run out without any fault; -1 holds none.  Calls with a held system or a
 * non-default budget are launched directly, not from the graph.
 */
int md_batch_set_wait_budget(md_batch *b, int64_t budget_cycles, int32_t held_system);

int md_batch_last_error(md_batch *b, char *buf, int64_t len);
void md_batch_destroy(md_batch *b);

#ifdef __cplusplus
}
#endif

#endif
