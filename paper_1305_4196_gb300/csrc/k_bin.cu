// k_bin.cu - linked-cell binning on the GPU (Sec. II.A, step 1 of the cell task algorithm).
//
// The paper bins particles into a grid of cells at least as wide as the
// interaction range and keeps one linked list per cell.  On the GPU the
// linked lists become a counting sort: every atom gets its cell, cells get
// their atom counts and an exclusive scan turns counts into start offsets;
// atoms are then scattered to their cell's slot range and all per-atom state
// is gathered into that cell order, so that one cell (and one 2x2x2 block of
// cells) is a contiguous range of atoms.  Inside a cell atoms are ordered by
// original index, which makes the layout a function of the positions alone.
#include "mdgb_internal.cuh"

namespace mdgb {

// ---------------------------------------------------------------- assign
// Map x into [0, L) (one box length at most, counted in the image counters:
// the same operation the oracle applies at a rebuild) and find the cell.
__global__ void k_bin_assign(DevState s, Geometry g, int32_t* __restrict__ atom_cell,
                             int32_t* __restrict__ cell_count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    double* X[3] = {s.x, s.y, s.z};
    int32_t* I[3] = {s.ix, s.iy, s.iz};
    int c[3];
    uint32_t bad = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double x = X[d][i];
        const double L = g.L[d];
        // The FP64 pipe is the scarce one on this GPU: most atoms need only the cell,
        // x * nc / L truncated (two FP64 operations).  The exact comparisons of the wrap run
        // for the atoms that may need it: negative or non-finite x, and the last cell column
        // (x * nc / L >= nc - 1 holds for every x >= L).
        int cc = (int)(x * g.inv_w[d]);
        const long long bits = __double_as_longlong(x);
        if (bits < 0 || cc >= g.nc[d] - 1 || ((bits >> 52) & 0x7ff) == 0x7ff) {
            if (x >= L) {
                x = __dsub_rn(x, L);
                I[d][i] += 1;
                X[d][i] = x;
            } else if (x < 0.0) {
                x = __dadd_rn(x, L);
                I[d][i] -= 1;
                X[d][i] = x;
            }
            if (!(x >= 0.0 && x <= L)) bad |= isfinite(x) ? ERR_ESCAPE : ERR_NONFINITE;
            cc = (int)(x * g.inv_w[d]);
        }
        cc = cc < 0 ? 0 : (cc >= g.nc[d] ? g.nc[d] - 1 : cc);
        c[d] = cc;
    }
    if (bad) atomicOr(s.err, bad);
    int id = cell_id_of(g, c[0], c[1], c[2]);
    atom_cell[i] = id;
    // atoms arrive in the previous cell order: most of a warp shares a cell, so one
    // atomic per cell and warp instead of one per atom
    const unsigned peers = __match_any_sync(__activemask(), id);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cell_count[id], __popc(peers));
}

void launch_bin_assign(const DevState& s, const Geometry& g, int32_t* atom_cell, int32_t* cell_count,
                       cudaStream_t st) {
    if (s.n == 0) return;
    int bs = 256;
    k_bin_assign<<<(unsigned)((s.n + bs - 1) / bs), bs, 0, st>>>(s, g, atom_cell, cell_count);
}

// ---------------------------------------------------------------- scan
// Exclusive scan of n int32 counts into out[0..n] (out[n] = total): a
// three-kernel scan (tile sums, scan of tile sums, add-back), deterministic.
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_PER_THREAD = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    int warp_off = warp > 0 ? warp_sums[warp - 1] : 0;
    total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const int32_t* __restrict__ in,
                                                             int32_t* __restrict__ out, int n,
                                                             int32_t* __restrict__ tile_sums) {
    __shared__ int warp_sums[32];
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER_THREAD;
    int v[SCAN_PER_THREAD];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        sum += v[k];
    }
    int total;
    int off = block_exclusive_scan(sum, warp_sums, total);
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        if (base + k < n) out[base + k] = off;
        off += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// single CTA: exclusive scan of the tile sums in place, total to out[n]
__global__ void __launch_bounds__(1024) k_scan_sums(int32_t* __restrict__ tile_sums, int ntiles,
                                                    int32_t* __restrict__ out, int n) {
    __shared__ int warp_sums[32];
    int carry = 0;
    for (int base = 0; base < ntiles; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < ntiles ? tile_sums[i] : 0;
        int total;
        int off = block_exclusive_scan(v, warp_sums, total);
        if (i < ntiles) tile_sums[i] = carry + off;
        carry += total;
    }
    if (threadIdx.x == 0) out[n] = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_add(int32_t* __restrict__ out, int n,
                                                           const int32_t* __restrict__ tile_sums) {
    int add = tile_sums[blockIdx.x];
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER_THREAD;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k)
        if (base + k < n) out[base + k] += add;
}

size_t scan_scratch_ints(int n) { return (size_t)(n + SCAN_TILE - 1) / SCAN_TILE + 1; }

void launch_scan(const int32_t* in, int32_t* out, int n, int32_t* scratch, cudaStream_t st) {
    int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles == 0) ntiles = 1;
    k_scan_tiles<<<ntiles, SCAN_THREADS, 0, st>>>(in, out, n, scratch);
    k_scan_sums<<<1, 1024, 0, st>>>(scratch, ntiles, out, n);
    k_scan_add<<<ntiles, SCAN_THREADS, 0, st>>>(out, n, scratch);
}

// ---------------------------------------------------------------- scatter
__global__ void k_scatter(DevState s, const int32_t* __restrict__ atom_cell,
                          const int32_t* __restrict__ cell_start, int32_t* __restrict__ cursor,
                          int32_t* __restrict__ slot_key, int32_t* __restrict__ slot_src) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    int c = atom_cell[i];
    // one atomic per cell and warp; the order within a cell is set by k_cell_sort
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, c);
    const int lane = (int)(threadIdx.x & 31), leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&cursor[c], __popc(peers));
    base = __shfl_sync(act, base, leader);
    int slot = cell_start[c] + base + __popc(peers & ((1u << lane) - 1u));
    slot_key[slot] = s.orig[i];
    slot_src[slot] = (int32_t)i;
}

void launch_scatter(const DevState& s, const int32_t* atom_cell, const int32_t* cell_start, int32_t* cursor,
                    int32_t* slot_key, int32_t* slot_src, cudaStream_t st) {
    if (s.n == 0) return;
    int bs = 256;
    k_scatter<<<(unsigned)((s.n + bs - 1) / bs), bs, 0, st>>>(s, atom_cell, cell_start, cursor, slot_key,
                                                              slot_src);
}

// ---------------------------------------------------------------- in-cell order
// One warp per cell: the rank of an atom is the number of atoms of its cell
// with a smaller original index (original indices are unique).
__global__ void k_cell_sort(int ncell, const int32_t* __restrict__ cell_start,
                            const int32_t* __restrict__ slot_key, const int32_t* __restrict__ slot_src,
                            int32_t* __restrict__ sorted_src) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= ncell) return;
    int start = cell_start[warp];
    int cnt = cell_start[warp + 1] - start;
    for (int e = lane; e < cnt; e += 32) {
        int key = slot_key[start + e];
        int rank = 0;
        for (int f = 0; f < cnt; ++f) rank += slot_key[start + f] < key;
        sorted_src[start + rank] = slot_src[start + e];
    }
}

void launch_cell_sort(const Geometry& g, const int32_t* cell_start, const int32_t* slot_key,
                      const int32_t* slot_src, int32_t* sorted_src, cudaStream_t st) {
    int bs = 256;
    int64_t threads = (int64_t)g.ncell * 32;
    k_cell_sort<<<(unsigned)((threads + bs - 1) / bs), bs, 0, st>>>(g.ncell, cell_start, slot_key, slot_src,
                                                                    sorted_src);
}

// ---------------------------------------------------------------- gather
// New slot t takes the atom that was at src = sorted_src[t].  Permuted state
// (positions, velocities, images, species, original ids) goes to the scratch
// copy d and comes back with k_copy_back; state derived from the new layout
// (reference positions, cell, FP32 cell-relative coordinates) is written to s.
__global__ void k_gather(DevState d, DevState s, Geometry g, const int32_t* __restrict__ sorted_src,
                         const int32_t* __restrict__ atom_cell) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    int src = sorted_src[t];
    double x = s.x[src], y = s.y[src], z = s.z[src];
    d.x[t] = x;
    d.y[t] = y;
    d.z[t] = z;
    d.vx[t] = s.vx[src];
    d.vy[t] = s.vy[src];
    d.vz[t] = s.vz[src];
    d.ix[t] = s.ix[src];
    d.iy[t] = s.iy[src];
    d.iz[t] = s.iz[src];
    int sp = s.species[src];
    d.species[t] = sp;
    d.orig[t] = s.orig[src];
    s.rx[t] = x;
    s.ry[t] = y;
    s.rz[t] = z;
    int c = atom_cell[src];
    s.cell_of[t] = c;
    float4 p;
    p.x = __double2float_rn(__dsub_rn(x, s.centre[c]));
    p.y = __double2float_rn(__dsub_rn(y, s.centre[g.ncell + c]));
    p.z = __double2float_rn(__dsub_rn(z, s.centre[2 * g.ncell + c]));
    p.w = __int_as_float(sp);
    s.xr[t] = p;
    s.xr_ref[t] = p;
}

__global__ void k_copy_back(DevState s, DevState d) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    s.x[t] = d.x[t];
    s.y[t] = d.y[t];
    s.z[t] = d.z[t];
    s.vx[t] = d.vx[t];
    s.vy[t] = d.vy[t];
    s.vz[t] = d.vz[t];
    s.ix[t] = d.ix[t];
    s.iy[t] = d.iy[t];
    s.iz[t] = d.iz[t];
    s.species[t] = d.species[t];
    s.orig[t] = d.orig[t];
}

void launch_gather(const DevState& s, const DevState& scratch, const Geometry& g, const int32_t* sorted_src,
                   const int32_t* atom_cell, cudaStream_t st) {
    if (s.n == 0) return;
    int bs = 256;
    unsigned nb = (unsigned)((s.n + bs - 1) / bs);
    k_gather<<<nb, bs, 0, st>>>(scratch, s, g, sorted_src, atom_cell);
    k_copy_back<<<nb, bs, 0, st>>>(s, scratch);
}

// ---------------------------------------------------------------- occupied blocks
// Own-atom count of every block after binning (its 8 cells are consecutive in the
// block-major cell numbering); the ids of the blocks with atoms go to blk_list (spatial
// order within each warp's 32 blocks, warps in the order they reach the counter) and their
// number to stats[4].  The order of the list does not affect any result: each block writes
// only its own atoms.
__global__ void k_classify_blocks(DevState s, Geometry g) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    bool occ = false;
    int b = 0;
    if (k < g.nblock) {
        b = spatial_block(g, k);
        occ = s.cell_start[8 * b + 8] > s.cell_start[8 * b];
    }
    const unsigned mo = __ballot_sync(0xffffffffu, occ);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && mo) base = atomicAdd(&s.stats[4], __popc(mo));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (occ) s.blk_list[base + __popc(mo & ((1u << lane) - 1u))] = b;
}

void launch_classify_blocks(const DevState& s, const Geometry& g, cudaStream_t st) {
    cudaMemsetAsync(s.stats + 4, 0, sizeof(int32_t), st);
    k_classify_blocks<<<(g.nblock + 255) / 256, 256, 0, st>>>(s, g);
}

}  // namespace mdgb
