/*
 * mdgb_debug.h - host-only introspection of the cell grid and the colour
 * schedule used by libmdgb (no GPU needed).
 *
 * The cell task method lets two tasks run at the same time only if they do
 * not overlap: at least two cells lie between them in every direction
 * (Meyer 2013, Sec. II.A), and waves of such tasks run one after another
 * (Sec. II.B).  libmdgb's 2x2x2-cell blocks (Sec. II.D.2) are split into 8
 * colour classes; these calls expose the exact numbering the kernels use so
 * that a test can check, on the CPU, that the 4x4x4-cell neighbourhoods of
 * all blocks of one colour are pairwise disjoint.
 *
 * All functions are pure host code, return MD_OK (0) or MD_ERR_ARG (-1),
 * write only to the caller's arrays and allocate nothing.
 */
#ifndef MDGB_DEBUG_H
#define MDGB_DEBUG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Cells per dimension md_create() picks for box[3], list radius r_list and list
 * kind list_kind (MD_LIST_*): the largest multiple of 4 with width >= r_list, or 6
 * for MD_LIST_FULL where 6 fit and that multiple is 4 (a homogeneous mixed full-list
 * system may take fewer, coarser cells at its first build; see md_create).
 * MD_ERR_BOX_TOO_SMALL (-2) if < 4. */
int mdgb_grid_shape(const double box[3], double r_list, int32_t list_kind, int32_t nc_out[3]);

/* Cells on a side of length `side` in the coarser grid a mixed full-list system takes at
 * its first build (see md_create): the smallest even count, at least 6, whose width is at
 * most (per_block / (8 rho))^(1/3), so that a 2x2x2-cell block holds about per_block atoms
 * at density rho; never more than fit_nc (>= 4), the count of the first grid.
 * MD_ERR_ARG (-1) for a non-positive or non-finite side, rho or per_block, or fit_nc < 4. */
int mdgb_coarse_cells(double side, double rho, double per_block, int32_t fit_nc, int32_t *nc_out);

/* Number of 2x2x2 blocks for a grid of nc[3] cells (even, >= 4).  Grids with every
 * side a multiple of 4 number their blocks colour class by colour class; the
 * others (full lists only) number them linearly, x fastest. */
int mdgb_num_blocks(const int32_t nc[3], int32_t *nblock_out);

/* Colour class (0..7) of block `block` (colour-major grids only: every nc a
 * multiple of 4). */
int mdgb_block_colour(const int32_t nc[3], int32_t block, int32_t *colour_out);

/* The 64 cells of block `block`'s tile in tile order (own 8 cells first, then the
 * other 35 cells a Newton-3 half list of the own cells reaches, then the remaining 21),
 * as linear cell indices cx + nc[0]*(cy + nc[1]*cz). */
int mdgb_tile_cells(const int32_t nc[3], int32_t block, int32_t cells_out[64]);

/* The mixed path's FP64 decision band around r_cut^2: pairs whose FP32 r^2 lies
 * within r_cut^2 (1 -/+ band) are decided by the FP64 definition (Sec. I: the pair
 * set is fixed by |r| < r_cut).  frame 0: the tile frame of md_system (cells of
 * width up to w_max, atoms at most half_skin from where they were binned); frame 1:
 * the cell frame of the ensemble kernel (cells of width up to w_max, neighbour cells
 * up to R away; half_skin unused).  The band is twice a worst-case bound on
 * |r2_fp32 - r2| / r_cut^2, plus the rounding of the FP32 thresholds. */
int mdgb_cut_band(int32_t frame, double w_max, double half_skin, int32_t R, double r_cut, double *band_out);

#ifdef __cplusplus
}
#endif

#endif /* MDGB_DEBUG_H */
