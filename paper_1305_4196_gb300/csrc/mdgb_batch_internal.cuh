// mdgb_batch_internal.cuh - ensembles of independent small systems (k_batch.cu, api_batch.cu).
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

// The ensemble's atom arrays (original order within each system, systems one after another).
struct BatchState {
    int64_t ntot;
    double *x, *y, *z, *vx, *vy, *vz;
    int32_t *ix, *iy, *iz, *species;
    long long* fq;     // 3 x ntot, Q31.32
    uint32_t* err;
};

// Shared memory of a system of at most nmax atoms (nmax a multiple of 8): three FP32
// coordinate arrays and the slot -> cell map of nmax + 2 slots, three u16 arrays of nmax,
// then the int arrays (cell starts and counts).
__host__ __device__ inline size_t batch_smem_ints_offset(int nmax) {
    const size_t np2 = (size_t)nmax + 2;
    return (np2 * (3 * 4 + 2) + (size_t)nmax * 3 * 2 + 15) & ~(size_t)15;
}
size_t batch_smem_bytes(int nmax, int cmax);
void launch_batch_run(const BatchSys* sys, int nsys, const BatchState& st, const PairTable& pt, int n_steps,
                      int flags, double dt, int threads, int nmax, int cmax, double* pe_out, double* ke_out,
                      float* pe_atom, cudaStream_t s);
void init_batch_kernels();

}  // namespace mdgb
