// mdgb_internal.cuh - shared definitions of the sm_103a kernels and the C-ABI layer.
//
// Cell numbering.  The box is cut into nc[d] cells per dimension (even, at
// least 4).  Cells are grouped into 2x2x2 blocks (the paper's cell-task
// blocking, Sec. II.D.2) and numbered block by block:
//     cell id = block id * 8 + (lx + 2 ly + 4 lz)          (l = cell parity in its block)
// so that the atoms of one block are contiguous after binning.  Blocks are
// numbered in one of two ways.
//   Colour-major (every nc[d] a multiple of 4; all half-list systems): blocks
//   are grouped into 8 colour classes by the parities of their block
//   coordinates,
//       block id = colour * (nblock / 8) + index within colour,
//   so the atoms of one colour class are contiguous too.  Two blocks of the
//   same colour are 4 cells apart in some dimension, so the 4x4x4-cell
//   neighbourhoods ("tiles") of same-colour blocks never overlap: a wave of
//   non-overlapping tasks in the sense of Sec. II.B.
//   Linear (any other even counts; md_create picks them only for full lists
//   with a side of 6 cells): block id = bx + nb[0] (by + nb[1] bz).  Full
//   lists write only their own block's atoms, so they need no colour classes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace mdgb {

// device error bits (sticky, OR-ed into a device word, read by the host)
enum : uint32_t {
    ERR_LIST_OVERFLOW = 1u,   // a neighbour list exceeded the capacity
    ERR_TILE_OVERFLOW = 2u,   // a 4x4x4-cell tile exceeded the on-chip capacity
    ERR_NONFINITE = 4u,       // non-finite pair force or coordinates
    ERR_ESCAPE = 8u,          // an atom moved more than one box length between builds
    ERR_SKIN = 16u,           // displacement > skin/2 under the fixed-interval policy
    ERR_CELL_DENSE = 32u,     // atom-free half list: a cell above 63 atoms or a phase above 255 steps
    ERR_CELL_COUNT = 32u,     // a cell holds more atoms than a list index can address
};

constexpr int MAX_SPECIES = 4;
constexpr int MAX_PAIR = MAX_SPECIES * MAX_SPECIES;

struct Geometry {
    double L[3];       // box sides
    double w[3];       // cell widths L / nc
    double inv_w[3];   // nc / L
    int nc[3];         // cells per dimension (even, >= 4; multiples of 4 unless linear)
    int nb[3];         // blocks per dimension (= nc / 2)
    int nbh[3];        // colour-major: blocks per dimension within one colour class (= nc / 4)
    int linear;        // 1: linear block numbering (no colour classes)
    int nblock;        // number of 2x2x2 blocks
    int ncell;         // number of cells
};

// LJ pair constants per species pair (FP32 copies for the mixed path, FP64 for the FP64 path)
struct PairTable {
    int nsp;
    float sig2_f[MAX_PAIR], c48_f[MAX_PAIR], c24_f[MAX_PAIR], c4_f[MAX_PAIR], rc2_f[MAX_PAIR];
    double sig_d[MAX_PAIR], sig2_d[MAX_PAIR], eps_d[MAX_PAIR], rc2_d[MAX_PAIR];
    double hdtm[MAX_SPECIES];  // (dt/2) / m per species
    double hdtm_q[MAX_SPECIES];  // (dt/2) / m * 2^-32: half kick per unit of Q31.32 force
    double mass[MAX_SPECIES];
    float cut_band;  // mixed path: pairs with FP32 r^2 within r_cut^2 (1 -/+ cut_band) are decided in FP64
    float rc2lo_f[MAX_PAIR], rc2hi_f[MAX_PAIR];  // r_cut^2 (1 -/+ cut_band) in FP32
    // One species: the band as a half width around rc2_f[0] (covering [rc2lo_f, rc2hi_f]),
    // and an r^2 below which a pair's FP32 force term may reach the split's limit
    // (fs2_max); above it |fs2| stays below half that limit.
    float band_half_f, r2_wide_f;
    // One species: the pair force as fs2 = inv^4 (lj_a inv^3 - lj_b) with inv = 1/r^2,
    // lj_a = c48 sigma^12, lj_b = c24 sigma^6 (the 2^11 scale included), and sigma^6.
    float lj_a_f, lj_b_f, sig6_f;
};

// The FP32 thresholds of the band (after pt.cut_band, the pair constants and pt.rc2_f are set).
inline void set_band_thresholds(PairTable& pt) {
    for (int t = 0; t < pt.nsp * pt.nsp; ++t) {
        pt.rc2lo_f[t] = (float)((double)pt.rc2_f[t] * (1.0 - (double)pt.cut_band));
        pt.rc2hi_f[t] = (float)((double)pt.rc2_f[t] * (1.0 + (double)pt.cut_band));
    }
    const float up = pt.rc2hi_f[0] - pt.rc2_f[0], down = pt.rc2_f[0] - pt.rc2lo_f[0];  // exact (Sterbenz)
    pt.band_half_f = up > down ? up : down;
    // fs2(r^2) = 2^11 * 24 eps (2 s6^2 - s6) / r^2, s6 = (sigma^2 / r^2)^3, falls monotonically
    // up to the potential minimum and stays far below the limit beyond it; find where it is
    // half the limit (the same limit as the kernels: 2^22 / r_cut,max * 0.999)
    float rc2max = 0.f;
    for (int t = 0; t < pt.nsp * pt.nsp; ++t) rc2max = pt.rc2_f[t] > rc2max ? pt.rc2_f[t] : rc2max;
    const double half_lim = 0.5 * (double)(4194304.0f / sqrtf(rc2max) * 0.999f);
    const double c48 = pt.c48_f[0], c24 = pt.c24_f[0], sg2 = pt.sig2_f[0];
    double lo = 1e-12 * sg2, hi = 1.2599210498948732 * sg2;  // 2^(1/3) sigma^2: the minimum
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi), s6 = (sg2 / mid) * (sg2 / mid) * (sg2 / mid);
        const double fs = (c48 * s6 - c24) * s6 / mid;
        if (fs > half_lim) lo = mid; else hi = mid;
    }
    pt.r2_wide_f = (float)hi;
    const double sg6 = sg2 * sg2 * sg2;
    pt.lj_a_f = (float)(c48 * sg6 * sg6);
    pt.lj_b_f = (float)(c24 * sg6);
    pt.sig6_f = (float)sg6;
}

// Tight-binding second-moment potential (Cleri and Rosato 1993; the potential of the
// paper's benchmarks, Sec. III), one species, mixed path.  With dr = r - r0:
//   phi(r) = A exp(-p (r/r0 - 1)) = 2^(kp dr + lp),  psi(r) = xi^2 exp(-2q (r/r0 - 1)) = 2^(kq dr + lq)
// E = sum_i [sum_j phi(r_ij) - sqrt(rho_i)], rho_i = sum_j psi(r_ij), and the force of pair
// (i,j) on i along d / r is c_rep phi - c_band psi (1/sqrt(rho_i) + 1/sqrt(rho_j)).
struct TBTable {
    float r0, kp, lp, kq, lq;  // FP32 forms of the two exponentials
    float c_rep, c_band;       // 2 p / r0, q / r0
    float rc2lo_f, rc2hi_f;    // the FP64 decision band around r_cut^2
    double rc2_d;              // r_cut^2
};

// ---- the FP64 decision band around r_cut^2 (host)
// Half an FP32 ulp of the numbers of magnitude up to v > 0: 2^(floor(log2 v) - 24).
inline double f32_half_ulp(double v) {
    int e = 0;
    std::frexp(v, &e);
    return std::ldexp(1.0, e - 25);
}

// |r2_fp32 - r2| bound for a pair at distance up to ~r_cut whose FP32 displacement
// components each carry at most e_d of error, relative to r_cut^2: the error of
// d.d through the components (2 |d|_1 e_d + 3 e_d^2, |d|_1 <= sqrt(3) |d|) and the three
// roundings of r2 = fma(dz, dz, fma(dy, dy, dx * dx)).
inline double r2_rel_bound(double e_d, double rc) {
    const double dmax = rc * 1.001;
    const double err = 2.0 * std::sqrt(3.0) * dmax * e_d + 3.0 * e_d * e_d + 3.0 * f32_half_ulp(dmax * dmax);
    return err / (rc * rc);
}

// Band for the tile frame of the list, force and backward kernels: a coordinate is the
// FP32 rounding of its offset from the build cell's centre (at most w/2 + skin/2 away,
// as the skin/2 rule rebuilds before an atom moves further), plus the FP32 tile offset
// (t - 3/2) w (at most 3w/2), rounded; the displacement is the FP32 difference of two
// coordinates.  Twice the bound, for the smallest cutoff rc_min.
inline double tile_frame_cut_band(double w_max, double half_skin, double rc_min) {
    const double a = 0.5 * w_max + half_skin;
    const double e_coord = f32_half_ulp(a) + f32_half_ulp(1.5 * w_max) + f32_half_ulp(1.5 * w_max + a);
    const double e_d = 2.0 * e_coord + f32_half_ulp(rc_min * 1.001);
    return 2.0 * r2_rel_bound(e_d, rc_min) + 3.0e-7;  // + the FP32 roundings of r_cut^2 (1 -/+ band)
}

// Band for the one-CTA-per-system ensemble kernel: coordinates relative to the centre of
// the cell they were binned into this step (at most w/2 away), the neighbour cell's
// shift k w with |k| <= R (FP32 w, exact multiples for |k| <= 2) added in FP32, then the
// FP32 difference.  Twice the bound.
inline double cell_frame_cut_band(double w_max, int R, double rc) {
    const double e_d = 2.0 * f32_half_ulp(0.5 * w_max) + R * f32_half_ulp(w_max) +
                       f32_half_ulp((0.5 + R) * w_max) + f32_half_ulp(rc * 1.001);
    return 2.0 * r2_rel_bound(e_d, rc) + 3.0e-7;
}

__host__ __device__ inline int block_id_of(const Geometry& g, int bx, int by, int bz) {
    if (g.linear) return bx + g.nb[0] * (by + g.nb[1] * bz);
    int col = (bx & 1) | ((by & 1) << 1) | ((bz & 1) << 2);
    int within = (bx >> 1) + g.nbh[0] * ((by >> 1) + g.nbh[1] * (bz >> 1));
    return col * (g.nblock >> 3) + within;
}

__host__ __device__ inline void block_coords(const Geometry& g, int b, int& bx, int& by, int& bz) {
    if (g.linear) {
        bx = b % g.nb[0];
        const int t = b / g.nb[0];
        by = t % g.nb[1];
        bz = t / g.nb[1];
        return;
    }
    int per = g.nblock >> 3;
    int col = b / per;
    int w = b - col * per;
    int hx = w % g.nbh[0];
    int t = w / g.nbh[0];
    int hy = t % g.nbh[1];
    int hz = t / g.nbh[1];
    bx = 2 * hx + (col & 1);
    by = 2 * hy + ((col >> 1) & 1);
    bz = 2 * hz + ((col >> 2) & 1);
}

// The i-th block in x-fastest spatial order.  Kernels with one CTA per block and no colour
// constraint take their blocks in this order: CTAs that run at the same time then hold
// neighbouring blocks, whose tiles share cells, so the staging reads hit L2.  (Block ids
// themselves are colour-major, for the colour launches of the half-list kernels.)
__host__ __device__ inline int spatial_block(const Geometry& g, int i) {
    if (g.linear) return i;
    const int bx = i % g.nb[0], t = i / g.nb[0];
    return block_id_of(g, bx, t % g.nb[1], t / g.nb[1]);
}

// Cells per side for a box side that fits `fit` cells of width >= r_list: the largest
// multiple of 4, or, for full lists, 6 where that would be 4 and 6 fit.  (Other even counts
// would serve full lists too, but cells of a multiple of 4 per side are wider and fuller:
// at rho* = 0.8442 and r_list = 2.8, 46 cells per side instead of 44 made both the force
// kernel and the list build about 6 % slower.)  A result below 4 means the box is too small.
__host__ __device__ inline int grid_cells(int fit, bool full_list) {
    const int nc4 = fit - fit % 4;
    return (full_list && nc4 == 4 && fit >= 6) ? 6 : nc4;
}

// Cells per side for the coarser grid a mixed full-list system takes at its first build:
// the smallest even count, at least 6, whose width side / count is at most
// (per_block / (8 rho))^(1/3) - a 2x2x2-cell block then holds about per_block atoms at
// density rho - and never more than fit_nc, the count the arrays were sized for.
__host__ __device__ inline int coarse_cells(double side, double rho, double per_block, int fit_nc) {
    const double w = cbrt(per_block / (8.0 * rho));
    int want = (int)ceil(side / w);
    want += want & 1;
    want = want < 6 ? 6 : want;
    return want < fit_nc ? want : fit_nc;
}

// Fill the block fields of g from its cell counts nc[3] (even, >= 4): colour-major
// numbering when every count is a multiple of 4, else linear.
__host__ __device__ inline void set_block_layout(Geometry& g) {
    g.linear = 0;
    for (int d = 0; d < 3; ++d) {
        g.nb[d] = g.nc[d] / 2;
        g.nbh[d] = g.nc[d] / 4;
        if (g.nc[d] % 4) g.linear = 1;
    }
    g.nblock = g.nb[0] * g.nb[1] * g.nb[2];
    g.ncell = g.nblock * 8;
}

__host__ __device__ inline int cell_id_of(const Geometry& g, int cx, int cy, int cz) {
    return block_id_of(g, cx >> 1, cy >> 1, cz >> 1) * 8 + ((cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2));
}

__host__ __device__ inline void cell_coords(const Geometry& g, int c, int& cx, int& cy, int& cz) {
    int bx, by, bz;
    block_coords(g, c >> 3, bx, by, bz);
    int l = c & 7;
    cx = 2 * bx + (l & 1);
    cy = 2 * by + ((l >> 1) & 1);
    cz = 2 * bz + ((l >> 2) & 1);
}

// FP32 offsets (t - 3/2) * w of the 4 tile coordinates per dimension (see tile.cuh).
struct TileOffsets {
    float off[3][4];
};

// Per-CTA tile bookkeeping in shared memory.
struct TileMeta {
    int prefix[65];  // tile slot -> first tile index (prefix[64] = tile size)
    int start[64];   // tile slot -> first global (cell-ordered) atom index
};

// Device state shared by the kernels (all arrays in cell order unless noted).
struct DevState {
    int64_t n;
    int np;                 // row stride of the neighbour-list matrix (n rounded up to 64)
    double *x, *y, *z;      // positions, unwrapped since the last build
    double *vx, *vy, *vz;   // velocities
    double *rx, *ry, *rz;   // reference positions of the last build (FP64 path displacement test)
    int32_t *ix, *iy, *iz;  // periodic image counters
    int32_t *species;       // species id
    int32_t *orig;          // original index of each cell-ordered atom
    int32_t *cell_of;       // cell id of each atom at the last build
    float4 *xr;             // FP32 coordinates relative to the centre of the atom's build cell (mixed path)
    float4 *xr_ref;         // xr at the last build (mixed path displacement test)
    long long *fq;          // mixed path: forces, 3 x n, Q31.32 fixed point (x block, y block, z block)
    double *f;              // FP64 path: forces, 3 x n
    int32_t *cell_start;    // ncell + 1
    double *centre;         // cell centres, 3 x ncell (x block, y block, z block)
    int ncell;
    uint16_t *nl;           // neighbour lists, tile-local indices, in chunks of 8: entry k of atom s at
                            // nl[((k / 8) * np + s) * 8 + k % 8]; the last chunk is padded with the
                            // tile's dummy slot (a point far outside every cutoff)
    uint16_t *nl_cnt;       // list length per atom
    float *pe_atom_f;       // per-atom energy share (mixed, on demand)
    float *vir_atom_f;      // per-atom virial share, 6 x n (mixed, on demand)
    double *pe_atom_d;      // FP64 path
    double *vir_atom_d;     // FP64 path, 6 x n
    uint32_t *err;          // sticky error bits
    int32_t *rebuild_flag;  // set when some atom moved more than skin/2
    int32_t *stats;         // [0] max list length, [1] max tile size, [2..3] sum of list lengths (u64),
                            // [4] occupied blocks (k_classify_blocks)
    // The occupied blocks (own atoms > 0) in spatial order, listed after every binning.  With
    // compact > 0 the full-list mixed force kernel and the list builder run a grid of
    // `compact` CTAs over this list instead of one CTA per block: a system that is mostly
    // vacuum then pays nothing for its empty blocks.
    int32_t *blk_list;
    int compact;
    uint8_t *af_steps;      // atom-free half list: steps per (block, warp, phase, pass)
};

// ---- kernel launchers (defined in the .cu files)
void launch_bin_assign(const DevState& s, const Geometry& g, int32_t* atom_cell, int32_t* cell_count,
                       cudaStream_t st);
void launch_scan(const int32_t* in, int32_t* out_exclusive, int n, int32_t* scratch, cudaStream_t st);
size_t scan_scratch_ints(int n);
void launch_scatter(const DevState& s, const int32_t* atom_cell, const int32_t* cell_start, int32_t* cursor,
                    int32_t* slot_key, int32_t* slot_src, cudaStream_t st);
void launch_cell_sort(const Geometry& g, const int32_t* cell_start, const int32_t* slot_key,
                      const int32_t* slot_src, int32_t* sorted_src, cudaStream_t st);
void launch_gather(const DevState& s, const DevState& scratch, const Geometry& g, const int32_t* sorted_src,
                   const int32_t* atom_cell, cudaStream_t st);
void launch_classify_blocks(const DevState& s, const Geometry& g, cudaStream_t st);
void launch_step_ctrl(int policy, int every_k, int32_t* rebuild_flag, long long* step_counter,
                      long long* n_builds, uint32_t* err, cudaGraphConditionalHandle handle, cudaStream_t st);
void launch_count_build(long long* n_builds, cudaStream_t st);
void launch_copy_state(const DevState& dst, const DevState& src, cudaStream_t st);
void launch_build_lists(const DevState& s, const Geometry& g, const TileOffsets& to, double rl2, int list_cap,
                        int tile_cap, int half, cudaStream_t st);
size_t build_lists_smem(int list_cap, int tile_cap);
void launch_forces_mixed(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                         int tile_cap, int half, int with_energy, cudaStream_t st);
size_t force_smem_bytes(int mixed, int half, int with_energy, int tile_cap);
// Where a kick-kick-drift step writes the new positions: the other pair of position
// buffers (FP32 cell-relative and FP64), because CTAs that are still running read the
// current ones (their tiles, and the FP64 cutoff test of pairs near r_cut).
struct StepOut {
    float4* xr;
    double *x, *y, *z;
};
void launch_forces_mixed_fused(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                               int tile_cap, int mode, StepOut out, double dt, double lim2, cudaStream_t st);
enum { FUSE_KICK = 1, FUSE_KICK_KICK_DRIFT = 2 };  // modes of launch_forces_mixed_fused
// TB-SMA forces (full lists, mixed): the density pass writes emb[i] = 1/sqrt(rho_i) (0 for an
// atom without neighbours), the force pass the Q31.32 forces; with_energy also writes the
// per-atom energies and virial shares.  Two launches.
void launch_tbsma(const DevState& s, const Geometry& g, const TBTable& tb, const TileOffsets& to, int tile_cap,
                  float* emb, int with_energy, cudaStream_t st);
size_t tbsma_smem_bytes(int tile_cap);
// Colour-schedule race detector: blocks [block0, block0 + nblocks) tag their tile atoms.
void launch_colour_tags(const DevState& s, const Geometry& g, int block0, int nblocks, int32_t* tags,
                        unsigned long long* conflicts, cudaStream_t st);
void init_tbsma_kernels();
void launch_forces_fp64(const DevState& s, const Geometry& g, const PairTable& pt, int tile_cap, int half,
                        int with_energy, cudaStream_t st);
void launch_integrate(const DevState& s, const Geometry& g, const PairTable& pt, int mode, int mixed,
                      double dt, double lim2, cudaStream_t st);
void launch_reduce_energy(const DevState& s, const PairTable& pt, int mixed, double* partials, int nparts,
                          double* out8, cudaStream_t st);
void launch_set_state(const DevState& s, const double* pos, const double* vel, const int32_t* species,
                      int nsp, cudaStream_t st);
void launch_get_state(const DevState& s, double* pos, double* vel, int32_t* image, cudaStream_t st);
void launch_forces_out(const DevState& s, int mixed, double* f_out, cudaStream_t st);
void launch_cells_out(const DevState& s, const Geometry& g, int32_t* cells, cudaStream_t st);
void launch_pairs_out(const DevState& s, const Geometry& g, int half, unsigned long long* counter,
                      int32_t* pairs, long long cap, cudaStream_t st);

void init_force_kernels();
float fs2_max_of(const PairTable& pt);  // largest |fs2| the two-part split takes (k_force.cu)
// atom-free half lists (k_half_af.cu)
void launch_build_sched(const DevState& s, const Geometry& g, const TileOffsets& to, double rl2, int list_cap,
                        int tile_cap, cudaStream_t st);
void launch_forces_half_af(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                           int tile_cap, float fs2_max, int with_energy, cudaStream_t st);
size_t af_sched_smem_bytes(int tile_cap);
size_t af_force_smem_bytes(int tile_cap);
void init_half_af_kernels();
void init_force_fp64_kernels();
void init_grad_kernels();
size_t backward_smem_bytes(int fp64, int tile_cap);
size_t backward_scratch_doubles(int64_t n, int nsp, int nparts);
void launch_force_backward(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                           int tile_cap, int fp64, const double* G, double* gx_orig, int want_energy,
                           double* scratch, int nparts, cudaStream_t st);
void init_list_kernels();

// integrate modes
enum { INT_KICK_DRIFT = 0, INT_KICK_KICK_DRIFT = 1, INT_KICK = 2 };

}  // namespace mdgb
