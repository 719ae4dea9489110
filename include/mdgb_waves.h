/*
 * mdgb_waves.h - the paper's dependent cell-task schedule as a host tool.
 *
 * Meyer (2013), arXiv:1305.4196, Sec. II.B and the Appendix: the tasks of the
 * CPU cell-task method (one task per grid cell) are grouped into waves of
 * non-overlapping tasks, and each task waits only for the last earlier task
 * that touched one of its cells (the forward and the backward wave methods).
 * These functions build that schedule so that it can be checked against the
 * paper's own examples and compared with the 8 colour phases of the GPU path.
 * Host code only (no device memory, no stream); all arrays are host arrays
 * owned by the caller.  Cells are numbered x fastest: c = x + nx (y + ny z),
 * 0-based.  Errors: MD_ERR_ARG for invalid sizes or arguments.
 *
 * Reading of the Appendix: in one dimension the index stream advances in steps
 * of `spacing` (three; two for the z dimension of the 18-cell variant),
 * wrapping at D when periodic; a set closes when the next index would come
 * closer than `spacing` cells to a member (periodic distance when periodic) or
 * when every cell is covered.  Without periodicity, or when D is a multiple of
 * the spacing, the sets are the residue classes.  When an outer loop advances,
 * the inner dimension's stream restarts at the first index of its previous
 * last set.
 */
#ifndef MDGB_WAVES_H
#define MDGB_WAVES_H

#include <stdint.h>

#include "mdgb.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Index sets covering one dimension of D cells (Appendix).  Writes the set
 * number of every cell to set_of_cell[D] and returns the number of sets, or a
 * negative error.  start (0 <= start < D) is the first index of the stream.
 */
int md_wave_sets_1d(int32_t D, int32_t periodic, int32_t spacing, int32_t start, int32_t *set_of_cell);

/*
 * The waves of an n[0] x n[1] x n[2] grid (Appendix): nested loops, z outer,
 * y middle, x inner, over the index sets.  overlap = 27: a task touches the
 * 3x3x3 cells around it; overlap = 18: the 3x3x2 cells z..z+1 (Sec. II.D.3,
 * half-shell lists), which lets z sets be two cells apart.  Writes the wave
 * of every cell to wave_of_cell[n0 n1 n2]; returns the number of waves.
 */
int md_waves(const int32_t n[3], const int32_t periodic[3], int32_t overlap, int32_t *wave_of_cell);

/*
 * The dependent task schedule by the forward (backward = 0) or backward
 * (backward = 1) wave method (Sec. II.B).  Tasks are numbered in wave order;
 * writes task_cell[T] (the cell of each task, T = n0 n1 n2), n_pred[T] (direct
 * predecessors) and succ_start[T + 1] (CSR offsets of the direct successors).
 * With succ non-NULL (capacity succ_cap entries) also the successor lists,
 * sorted.  Returns the total number of successor entries, or a negative
 * error (MD_ERR_ARG also when succ_cap is too small).  Both methods give the
 * same graph.
 */
int64_t md_wave_schedule(const int32_t n[3], const int32_t periodic[3], int32_t overlap, int32_t backward,
                         int32_t *task_cell, int32_t *n_pred, int64_t *succ_start, int32_t *succ,
                         int64_t succ_cap);

#ifdef __cplusplus
}
#endif

#endif
