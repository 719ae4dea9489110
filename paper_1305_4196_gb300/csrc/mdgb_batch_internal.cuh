// mdgb_batch_internal.cuh - ensembles of independent systems (k_batch.cu, api_batch.cu).
#pragma once

#include "mdgb_internal.cuh"

namespace mdgb {

constexpr int BATCH_MAX_THREADS = 512;
constexpr int BATCH_MAX_ATOMS = 8192;   // atoms of a system run by one CTA (shared memory)
constexpr int BATCH_MAX_CELLS = 4096;   // cells of such a system
enum { BATCH_HAVE_FORCES = 1, BATCH_ENERGY = 2 };

// One system of the ensemble (device array, one entry per CTA).
struct BatchSys {
    int64_t a0;        // first atom in the ensemble's atom arrays
    int id;            // index of the system in the ensemble (energy outputs)
    int n;             // atoms
    int nc[3];         // cells per dimension, each at least r_cut / R wide
    int ncell;
    int R;             // neighbour range in cells
    double L[3], w[3], inv_w[3];
    float wf[3];       // cell width in FP32 (the shift of a neighbour cell)
};

// A system spread over many CTAs (block tasks): cells at least r_cut + skin wide, an even
// count of at least 4 per side, linear cell and 2x2x2-block numbering (x fastest).
struct EnsBlockSys {
    int64_t a0;        // first atom in the ensemble's atom arrays
    int64_t c0;        // first cell in the ensemble's cell arrays (counts, cursors)
    int64_t s0;        // first entry of its cell starts (ncell + 1 of them)
    int id;            // index of the system in the ensemble (energy outputs)
    int n;
    int nc[3], nb[3];  // cells and blocks per dimension
    int ncell, nblock;
    double L[3], w[3], inv_w[3];
    float off[3][4];   // FP32 tile offsets (t - 3/2) w of the 4 tile coordinates
};

// One entry of the launch's work table: a system and the task counts of its phases.
struct EnsEntry {
    int kind;          // 0: one CTA for the whole call (BatchSys), 1: block tasks (EnsBlockSys)
    int idx;           // index into the BatchSys or EnsBlockSys array
    int n_atom_chunks, n_cell_chunks, nblock;
};

// The ensemble's atom arrays (original order within each system, systems one after another).
struct BatchState {
    int64_t ntot;
    double *x, *y, *z, *vx, *vy, *vz;
    int32_t *ix, *iy, *iz, *species;
    long long* fq;     // 3 x ntot, Q31.32
    uint32_t* err;
};

// Work arrays of the block systems and the launch's scheduler words.
struct EnsArrays {
    double *xa, *ya, *za;        // second position buffer (ntot)
    int32_t* cell_of;            // ntot: an atom's cell for the next binning
    int32_t *perm_u, *perm_s;    // ntot: slot -> atom within its system (unordered / ordered in a cell)
    int32_t* scell;              // ntot: slot -> cell
    float4 *xs, *xsb;            // ntot: FP32 coordinates relative to the slot's build cell centre,
                                 // by slot, for even / odd steps
    float4* xs_ref;              // ntot: the same at the last build (skin/2 test)
    uint4* nl;                   // Verlet lists: chunk c of slot i of a system at a0 * list_chunks + c * n + i
    int32_t* nl_cnt;             // ntot: list length by slot
    int32_t* rebuild;            // per block system: some atom moved more than skin/2
    int32_t* valid;              // per block system: its lists and coordinates carry over between calls
    int list_chunks;             // list capacity in chunks of 8 entries
    float lim2_f;                // (skin/2)^2
    double rl2;                  // r_list^2
    float rl2_lo, rl2_hi;        // r_list^2 (1 -/+ 1e-4): candidates in between are re-tested in FP64
    int32_t *count, *cursor;     // cells of all block systems
    int32_t* cstart;             // cells + one per block system
    float* pe_atom;              // ntot: half pair energies per atom (energy calls)
    unsigned long long* ctl;     // per entry: (phase << 32) | next task
    int32_t* done;               // per entry: tasks of the current phase completed
    int32_t* g_done;             // entries finished
    long long budget;            // cycles a CTA may find no work before it reports a timeout
};

constexpr int ENS_ATOM_CHUNK = 2048;  // atoms per binning / scatter / wrap task
constexpr int ENS_CELL_CHUNK = 64;    // cells per in-cell ordering task
constexpr uint32_t ERR_TIMEOUT = 64u; // a CTA found no work for longer than its budget
constexpr uint32_t ENS_DONE = 0xffffffffu, ENS_HOLD = 0xfffffffeu, ENS_START = 0xfffffffdu;

// Shared memory of a system of at most nmax atoms (nmax a multiple of 8): three FP32
// coordinate arrays and the slot -> cell map of nmax + 2 slots, three u16 arrays of nmax,
// then the int arrays (cell starts and counts).
__host__ __device__ inline size_t batch_smem_ints_offset(int nmax) {
    const size_t np2 = (size_t)nmax + 2;
    return (np2 * (3 * 4 + 2) + (size_t)nmax * 3 * 2 + 15) & ~(size_t)15;
}
size_t batch_smem_bytes(int nmax, int cmax);
// Dynamic shared memory of a block task's tile of at most tile_slots slots (float4 each,
// plus the far slot after the last).
size_t ens_tile_smem_bytes(int tile_slots);
// Dynamic shared memory of a block system's list build for a tile of T atoms.
size_t ens_list_smem(int T);
// One persistent launch over every system of the ensemble (k_batch.cu).
void launch_ensemble(const EnsEntry* ent, int nent, const BatchSys* one, const EnsBlockSys* blk,
                     const BatchState& st, const EnsArrays& ea, const PairTable& pt, int n_steps, int flags,
                     double dt, int threads, int grid, int nmax, int cmax, int tile_slots, size_t smem,
                     double* pe_out, double* ke_out, cudaStream_t s);
// CTAs of the launch that fit one SM at once for this shape.
int ensemble_ctas_per_sm(int threads, size_t smem);
void init_batch_kernels();

}  // namespace mdgb
