/*
 * mdgb_batch.h - ensembles of independent periodic Lennard-Jones systems.
 *
 * Meyer (2013), arXiv:1305.4196, Sec. II.C: the task functor can carry which copy
 * of a system a task works on, so that several systems share one schedule.  Here
 * an ensemble of independent systems of uneven size is advanced together:
 *   - systems of at most 8,192 atoms run in one persistent launch per size bucket
 *     in which each CTA owns one whole system for all time steps (linked cells
 *     rebuilt in shared memory every step, FP32 pair arithmetic, Q31.32 fixed-point
 *     forces, FP64 velocity Verlet); the launches are replayed from a CUDA graph;
 *   - larger systems run as ordinary md_system instances (full lists, fused
 *     velocity Verlet), each on its own stream, concurrently with the launch above.
 * All systems share the pair parameters (one species), r_cut, skin (used by the
 * larger systems' lists) and dt, in mixed precision.  Atom arrays are
 * concatenated in system order (system k's atoms after those of systems 0..k-1),
 * N x 3 row-major, host or device as the device_ptrs flag says; the library
 * copies in and out.  Every call returns MD_OK or a negative MD_ERR_* code.
 * The larger systems overlap on the GPU only as far as CUDA's hardware work queues
 * allow: set CUDA_DEVICE_MAX_CONNECTIONS=32 before the process creates its CUDA
 * context (the default, 8, serialises most of the 100+ streams of a large ensemble).
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
 * 4 (r_cut + skin)).  params: one species, MD_MIXED; the stream field selects the
 * stream of the one-CTA-per-system launches (larger systems get their own).
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
 * How each system runs: path[k] = 0 (one CTA per system) or 1 (md_system);
 * threads[k] and cell_range[k] (cells are at least r_cut / cell_range wide) for
 * path 0.  Host arrays of n_systems; any may be NULL.
 */
int md_batch_layout(md_batch *b, int32_t *path, int32_t *threads, int32_t *cell_range);

/*
 * Autotuner: for every size bucket of one-CTA systems ([256, 512), [512, 1024),
 * ..., [4096, 8192] atoms) time 10 steps with 128/256/512 threads and cells of
 * r_cut or r_cut/2 (the state is restored afterwards) and keep the fastest.  With
 * cache_path non-NULL, buckets found in that JSON file (written for the same GPU
 * name) take their choice from it; the other non-empty buckets are timed and the
 * file is rewritten with both.  Buckets that hold no system are not timed and are
 * not written.
 */
int md_batch_autotune(md_batch *b, const char *cache_path);

int md_batch_last_error(md_batch *b, char *buf, int64_t len);
void md_batch_destroy(md_batch *b);

#ifdef __cplusplus
}
#endif

#endif
