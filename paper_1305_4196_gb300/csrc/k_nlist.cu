// k_nlist.cu - neighbour-list construction by cell tasks (Sec. II.A).
//
// The paper builds the neighbour lists of all particles of one cell per task
// (Sec. II.A) and gives each task its own list storage so that no two tasks
// update the same structure (Sec. II.A, Sec. II.C).  Here one CTA is the task
// of one 2x2x2-cell block: it stages the block's 4x4x4-cell tile in shared
// memory, each of its 8 warps takes one cell of the block (lanes = the cell's
// atoms), and every candidate of the 27 surrounding cells is broadcast from
// shared memory to the warp.  Each atom's list is written only by its own
// lane, so the lists need no synchronisation at all.
//
// The set is exactly the FP64 definition: pairs with minimum-image
// |x_i - x_j|^2 < r_list^2 evaluated as ((dx*dx)+dy*dy)+dz*dz.  The FP32
// tile test decides every candidate whose r^2 is further than a relative
// 1e-4 from r_list^2 (the FP32 coordinate error is below 1e-6); candidates
// inside that band are re-tested with the FP64 positions in exactly the
// definition's operation order (minimum image d - L*rint(d/L)).
//
// Full lists hold every neighbour of every atom.  Half lists (Newton's third
// law, Sec. II.D.3) hold each pair once: a neighbour in the same cell only if
// it comes later in cell order, plus all neighbours of the 13 "forward" cells.
#include "nl_scan.cuh"

namespace mdgb {

// The lists of the own atoms of block b (the CTA's task).
template <int HALF>
__device__ __forceinline__ void build_block(const DevState& s, const Geometry& g, const TileOffsets& to, double rl2,
                                            float band_lo, float band_hi, int list_cap, int tile_cap, int b) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    __shared__ int pp[65];
    const int SL = soa_len(tile_cap);
    float* tx = reinterpret_cast<float*>(smem);
    float* ty = tx + SL;
    float* tz = ty + SL;
    uint16_t* buf = reinterpret_cast<uint16_t*>(tz + SL);  // NL_WARPS x NL_RING x 32

    tile_meta(g, s.cell_start, b, m);
    const int T = m.prefix[64];
    // the tile capacity this block needs: its atoms and the dummy slot, and for half lists
    // also room for the mixed kernel's reaction sums over the cells a half list reaches
    const int need = HALF ? max(T + 1, tile_cap_for_recv(m.prefix[TILE_RECV_CELLS])) : T + 1;
    if (threadIdx.x == 0) atomicMax(&s.stats[1], need);
    if (need > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    if (m.prefix[8] == 0) return;  // empty block (vacuum): no lists to build
    tile_pad_prefix(m, pp);
    tile_stage_soa(m, pp, s.xr, to, tx, ty, tz);
    __syncthreads();

    const unsigned sx = (unsigned)__cvta_generic_to_shared(tx);
    const unsigned sy = (unsigned)__cvta_generic_to_shared(ty);
    const unsigned sz = (unsigned)__cvta_generic_to_shared(tz);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = warp & 1, ly = (warp >> 1) & 1, lz = warp >> 2;
    const int own_begin = m.prefix[warp], own_count = m.prefix[warp + 1] - own_begin;
    const int own_pbegin = pp[warp];
    uint16_t* col = buf + (size_t)warp * NL_RING * 32 + lane;
    const int blk0 = m.start[0];
    const int own_coord = (lx + 1) + 4 * (ly + 1) + 16 * (lz + 1);
    const f2_t hi2 = f2_pack(band_hi, band_hi), lo2 = f2_pack(band_lo, band_lo);
    int max_cnt = 0;
    unsigned long long sum_cnt = 0;

    for (int base = 0; base < own_count; base += 32) {
        const int e = base + lane;
        const bool active = e < own_count;
        const int ei = active ? e : 0;
        const int ui = own_begin + ei;
        const int own_p = own_pbegin + ei;
        const float xi = tx[own_p], yi = ty[own_p], zi = tz[own_p];
        const f2_t pix = f2_pack(xi, xi), piy = f2_pack(yi, yi), piz = f2_pack(zi, zi);
        const int gi = blk0 + ui;
        ListOut o{col, reinterpret_cast<uint4*>(s.nl) + gi, (size_t)s.np, list_cap, 0, 0};
        {
            const int slot = c_tiles.idx_of_coord[own_coord];
            const int jadj = m.start[slot] - pp[slot];  // cell-ordered atom index = padded index + jadj
            scan_cell<HALF, true>(sx, sy, sz, pp[slot], m.prefix[slot + 1] - m.prefix[slot],
                                  m.prefix[slot] - pp[slot], pix, piy, piz, hi2, lo2, own_p, active, o,
                                  [&](int q) {
                                      return fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gi, q + jadj, rl2);
                                  });
        }
#pragma unroll 1
        for (int key = HALF ? 1 : -13; key <= 13; ++key) {
            if (key == 0) continue;
            const int oz = (key + 13) / 9 - 1, oy = ((key + 13) / 3) % 3 - 1, ox = (key + 13) % 3 - 1;
            const int slot = c_tiles.idx_of_coord[own_coord + ox + 4 * oy + 16 * oz];
            const int jadj = m.start[slot] - pp[slot];
            scan_cell<HALF, false>(sx, sy, sz, pp[slot], m.prefix[slot + 1] - m.prefix[slot],
                                   m.prefix[slot] - pp[slot], pix, piy, piz, hi2, lo2, own_p, active, o,
                                   [&](int q) {
                                       return fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gi, q + jadj, rl2);
                                   });
        }
        // the last chunk, padded with the tile's dummy slot T
        flush_chunks(o, (unsigned)T, true);
        const int cnt = o.cnt;
        if (active) {
            if (cnt > list_cap) atomicOr(s.err, ERR_LIST_OVERFLOW);
            s.nl_cnt[gi] = (uint16_t)(cnt < list_cap ? cnt : list_cap);
            max_cnt = cnt > max_cnt ? cnt : max_cnt;
            sum_cnt += (unsigned long long)cnt;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        max_cnt = max(max_cnt, __shfl_xor_sync(0xffffffffu, max_cnt, o));
        sum_cnt += __shfl_xor_sync(0xffffffffu, sum_cnt, o);
    }
    if (lane == 0) {
        atomicMax(&s.stats[0], max_cnt);
        atomicAdd(reinterpret_cast<unsigned long long*>(&s.stats[2]), sum_cnt);
    }
}

// One CTA per block in spatial order.
template <int HALF>
__global__ void __launch_bounds__(NL_WARPS * 32, 3) k_build_lists(DevState s, Geometry g, TileOffsets to,
                                                                  double rl2, float band_lo, float band_hi,
                                                                  int list_cap, int tile_cap) {
    build_block<HALF>(s, g, to, rl2, band_lo, band_hi, list_cap, tile_cap, spatial_block(g, blockIdx.x));
}

// A compact system: a grid of s.compact CTAs over the occupied blocks.
template <int HALF>
__global__ void __launch_bounds__(NL_WARPS * 32, 3) k_build_lists_occ(DevState s, Geometry g, TileOffsets to,
                                                                      double rl2, float band_lo, float band_hi,
                                                                      int list_cap, int tile_cap) {
    const int count = s.stats[4];
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        build_block<HALF>(s, g, to, rl2, band_lo, band_hi, list_cap, tile_cap, s.blk_list[k]);
        __syncthreads();  // the next block reuses the shared memory
    }
}

static size_t nl_smem_bytes(int list_cap, int tile_cap) {
    (void)list_cap;
    return (size_t)soa_len(tile_cap) * 3 * sizeof(float) + (size_t)NL_WARPS * 32 * NL_RING * 2;
}

void launch_build_lists(const DevState& s, const Geometry& g, const TileOffsets& to, double rl2, int list_cap,
                        int tile_cap, int half, cudaStream_t st) {
    if (s.n == 0) return;
    size_t smem = nl_smem_bytes(list_cap, tile_cap);
    float lo = (float)(rl2 * (1.0 - 1e-4));
    float hi = (float)(rl2 * (1.0 + 1e-4));
    if (s.compact) {
        if (half) k_build_lists_occ<1><<<s.compact, NL_WARPS * 32, smem, st>>>(s, g, to, rl2, lo, hi, list_cap, tile_cap);
        else k_build_lists_occ<0><<<s.compact, NL_WARPS * 32, smem, st>>>(s, g, to, rl2, lo, hi, list_cap, tile_cap);
        return;
    }
    if (half) k_build_lists<1><<<g.nblock, NL_WARPS * 32, smem, st>>>(s, g, to, rl2, lo, hi, list_cap, tile_cap);
    else k_build_lists<0><<<g.nblock, NL_WARPS * 32, smem, st>>>(s, g, to, rl2, lo, hi, list_cap, tile_cap);
}

size_t build_lists_smem(int list_cap, int tile_cap) { return nl_smem_bytes(list_cap, tile_cap); }

template <typename K>
static void allow_max_smem(K kernel) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

void init_list_kernels() {
    allow_max_smem(k_build_lists<0>);
    allow_max_smem(k_build_lists<1>);
    allow_max_smem(k_build_lists_occ<0>);
    allow_max_smem(k_build_lists_occ<1>);
}

// ---------------------------------------------------------------- export
// The list as unordered pairs of original ids (i < j).  A full list holds
// each pair twice and reports it from the side with the smaller id.
__global__ void k_pairs_out(DevState s, Geometry g, int half, unsigned long long* __restrict__ counter,
                            int32_t* __restrict__ pairs, long long cap) {
    __shared__ TileMeta m;
    const int b = blockIdx.x;
    tile_meta(g, s.cell_start, b, m);
    const int blk0 = m.start[0];
    const int nown = m.prefix[8];
    for (int ui = threadIdx.x; ui < nown; ui += blockDim.x) {
        const int gi = blk0 + ui;
        const int oi = s.orig[gi];
        const int cnt = s.nl_cnt[gi];
        const uint16_t* rows = s.nl;
        for (int k = 0; k < cnt; ++k) {
            const int u = rows[((size_t)(k >> 3) * s.np + gi) * 8 + (k & 7)];
            if (u >= m.prefix[64]) continue;  // an idle step of an atom-free schedule
            const int slot = tile_slot_of(m, u);
            const int gj = m.start[slot] + (u - m.prefix[slot]);
            const int oj = s.orig[gj];
            if (!half && oi > oj) continue;
            const unsigned long long at = atomicAdd(counter, 1ull);
            if ((long long)at < cap) {
                pairs[2 * at] = oi < oj ? oi : oj;
                pairs[2 * at + 1] = oi < oj ? oj : oi;
            }
        }
    }
}

void launch_pairs_out(const DevState& s, const Geometry& g, int half, unsigned long long* counter,
                      int32_t* pairs, long long cap, cudaStream_t st) {
    if (s.n == 0) return;
    k_pairs_out<<<g.nblock, 128, 0, st>>>(s, g, half, counter, pairs, cap);
}

}  // namespace mdgb
