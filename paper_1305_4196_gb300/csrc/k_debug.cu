// k_debug.cu - the colour-schedule race detector (debug only, never on a timed path).
//
// The half-list kernel lets the blocks of one colour class run at the same time because
// their 4x4x4-cell tiles are disjoint, so no atom is written by two CTAs of one wave
// (Sec. II.A, Sec. II.B).  Here every block of a phase claims each atom of its tile with a
// compare-and-swap on a per-atom tag; an atom another block of the phase already claimed
// is a conflict.  It uses the kernels' own device-side block and tile mapping.
#include "tile.cuh"

namespace mdgb {

__global__ void k_colour_tags(DevState s, Geometry g, int block0, int32_t* __restrict__ tags,
                              unsigned long long* __restrict__ conflicts) {
    __shared__ TileMeta m;
    const int b = block0 + blockIdx.x;
    tile_meta(g, s.cell_start, b, m);
    unsigned long long mine = 0;
    for (int u = threadIdx.x; u < m.prefix[64]; u += blockDim.x) {
        const int j = tile_global_index(m, u);
        const int prev = atomicCAS(&tags[j], -1, b);
        if (prev != -1 && prev != b) ++mine;
    }
    if (mine) atomicAdd(conflicts, mine);
}

void launch_colour_tags(const DevState& s, const Geometry& g, int block0, int nblocks, int32_t* tags,
                        unsigned long long* conflicts, cudaStream_t st) {
    if (nblocks <= 0) return;
    k_colour_tags<<<nblocks, 128, 0, st>>>(s, g, block0, tags, conflicts);
}

}  // namespace mdgb
