// tile.cuh - the on-chip neighbourhood of one 2x2x2-cell block.
//
// A cell task of the paper (Sec. II.A) reads the particles of its cell and
// of the 26 surrounding cells.  Blocking 2x2x2 cells into one task
// (Sec. II.D.2) widens that neighbourhood to the 4x4x4 cells around the
// block: the "tile".  One CTA stages its tile in shared memory once and
// serves every list build / force evaluation of its block from there, so the
// neighbour lists can hold 16-bit tile-local indices.
//
// Tile order: the block's own 8 cells first (in the block's cell order, so
// the block's atoms keep their cell-sorted order and own atom k has tile
// index k), then the other 56 cells of the 4x4x4 neighbourhood, x fastest.
// Coordinates in the tile are FP32, relative to the block centre: each
// atom's FP32 offset from its own cell centre plus the (t - 3/2) cell-width
// offset of its tile cell, which is the same for every periodic image.
#pragma once

#include "mdgb_internal.cuh"

namespace mdgb {

struct TileTables {
    int8_t idx_of_coord[64];  // tile coordinate (tx + 4 ty + 16 tz) -> tile slot
    int8_t coord_of_idx[64];  // tile slot -> tile coordinate
};

// Tile cell (x, y, z) (0..3 each; the block's own cells are 1..2) is a Newton-3 half-shell
// target of some own cell: the cell itself, or a forward neighbour (dz > 0; dz = 0 and
// dy > 0; dz = dy = 0 and dx > 0; Sec. II.D.3).  Half-list reactions only reach these.
__host__ __device__ constexpr bool tile_receives(int x, int y, int z) {
    for (int oz = 1; oz <= 2; ++oz)
        for (int oy = 1; oy <= 2; ++oy)
            for (int ox = 1; ox <= 2; ++ox) {
                const int dx = x - ox, dy = y - oy, dz = z - oz;
                if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) continue;
                if (dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx >= 0)))) return true;
            }
    return false;
}

// Slots: the 8 own cells first, then the other cells a half list reaches, then the rest.
// So the own atoms are tile entries 0 .. prefix[8] - 1 and every half-list target lies in
// entries 0 .. prefix[TILE_RECV_CELLS] - 1.
constexpr int TILE_RECV_CELLS = 43;

__host__ __device__ constexpr TileTables make_tile_tables() {
    TileTables t{};
    int k = 8, r = TILE_RECV_CELLS;
    for (int c = 0; c < 64; ++c) {
        int x = c & 3, y = (c >> 2) & 3, z = c >> 4;
        bool own = x >= 1 && x <= 2 && y >= 1 && y <= 2 && z >= 1 && z <= 2;
        int i = own ? (x - 1) + 2 * (y - 1) + 4 * (z - 1) : (tile_receives(x, y, z) ? k++ : r++);
        t.idx_of_coord[c] = (int8_t)i;
        t.coord_of_idx[i] = (int8_t)c;
    }
    return t;
}

__host__ __device__ constexpr int count_tile_receivers() {
    int k = 0;
    for (int c = 0; c < 64; ++c) k += tile_receives(c & 3, (c >> 2) & 3, c >> 4) ? 1 : 0;
    return k;
}
static_assert(count_tile_receivers() == TILE_RECV_CELLS, "half-shell targets of a 2x2x2 block");

// Entries of the reaction sums a mixed half-list CTA keeps for a tile capacity: 11/16 of
// it (the 43 of 64 cells a half list reaches hold about 2/3 of a tile's atoms), and the
// smallest tile capacity whose share holds `recv` entries.
__host__ __device__ inline int half_recv_cap(int tile_cap) { return ((tile_cap * 11 + 15) / 16 + 31) & ~31; }
__host__ __device__ inline int tile_cap_for_recv(int recv) { return (recv * 16 + 10) / 11; }

static __constant__ TileTables c_tiles = make_tile_tables();

// Cell id of tile slot t of the block with coordinates (bx, by, bz).
__device__ __forceinline__ int tile_cell_id(const Geometry& g, int bx, int by, int bz, int t) {
    const int c = c_tiles.coord_of_idx[t];
    const int tx = c & 3, ty = (c >> 2) & 3, tz = c >> 4;
    int cx = 2 * bx - 1 + tx, cy = 2 * by - 1 + ty, cz = 2 * bz - 1 + tz;
    cx += cx < 0 ? g.nc[0] : (cx >= g.nc[0] ? -g.nc[0] : 0);
    cy += cy < 0 ? g.nc[1] : (cy >= g.nc[1] ? -g.nc[1] : 0);
    cz += cz < 0 ? g.nc[2] : (cz >= g.nc[2] ? -g.nc[2] : 0);
    return cell_id_of(g, cx, cy, cz);
}

// Fill meta for block b (threads 0..63 of the CTA take part; ends with __syncthreads).
__device__ __forceinline__ void tile_meta(const Geometry& g, const int32_t* __restrict__ cell_start, int b,
                                          TileMeta& m) {
    const int t = threadIdx.x;
    if (t < 64) {
        int bx, by, bz;
        block_coords(g, b, bx, by, bz);
        int id = tile_cell_id(g, bx, by, bz, t);
        int st = cell_start[id];
        int cnt = cell_start[id + 1] - st;
        m.start[t] = st;
        // inclusive scan of the 64 counts over two warps
        int lane = t & 31;
        int v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        m.prefix[t + 1] = v;  // warp-local inclusive prefix for now
    }
    __syncthreads();
    if (t >= 32 && t < 64) m.prefix[t + 1] += m.prefix[32];
    if (t == 0) m.prefix[0] = 0;
    __syncthreads();
}

// The same meta filled by one warp (lanes take slots lane and lane + 32; ends with __syncwarp).
__device__ __forceinline__ void tile_meta_warp(const Geometry& g, const int32_t* __restrict__ cell_start, int b,
                                               TileMeta& m) {
    const int lane = threadIdx.x & 31;
    int bx, by, bz;
    block_coords(g, b, bx, by, bz);
    int below = 0;  // atoms in slots 0..31
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int t = lane + 32 * h;
        const int id = tile_cell_id(g, bx, by, bz, t);
        const int st = cell_start[id];
        int v = cell_start[id + 1] - st;
        m.start[t] = st;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        m.prefix[t + 1] = v + below;
        below = __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) m.prefix[0] = 0;
    __syncwarp();
}

// Tile slot holding tile index u (binary search in the 65-entry prefix).
__device__ __forceinline__ int tile_slot_of(const TileMeta& m, int u) {
    int lo = 0, hi = 64;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (m.prefix[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// The FP64 pair test of the definition, in the oracle's operation order: minimum image
// d - L*rint(d/L) per dimension, r^2 = ((dx*dx) + dy*dy) + dz*dz, strict r^2 < cut2.
// Used wherever an FP32 distance lies too close to a threshold (list radius or cutoff)
// to decide the comparison.
__device__ __forceinline__ double mic_rn(double d, double L) {
    return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

__device__ __forceinline__ bool fp64_pair_test(const double* __restrict__ x, const double* __restrict__ y,
                                            const double* __restrict__ z, double Lx, double Ly, double Lz, int i,
                                            int j, double rl2) {
    double dx = mic_rn(__dsub_rn(x[i], x[j]), Lx);
    double dy = mic_rn(__dsub_rn(y[i], y[j]), Ly);
    double dz = mic_rn(__dsub_rn(z[i], z[j]), Lz);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < rl2;
}


// Cell-ordered global index of tile index u.
__device__ __forceinline__ int tile_global_index(const TileMeta& m, int u) {
    const int slot = tile_slot_of(m, u);
    return m.start[slot] + (u - m.prefix[slot]);
}

// o[t] for t in 0..3 without dynamic indexing (which would copy the table to local memory)
__device__ __forceinline__ float pick4(const float (&o)[4], int t) {
    return t == 0 ? o[0] : (t == 1 ? o[1] : (t == 2 ? o[2] : o[3]));
}

// Block-frame FP32 coordinates of tile index u, the same additions as the staging below.
__device__ __forceinline__ float4 tile_coord(const TileMeta& m, const TileOffsets& to, const float4* __restrict__ xr,
                                             int u) {
    const int slot = tile_slot_of(m, u);
    const int c = c_tiles.coord_of_idx[slot];
    const float4 p = xr[m.start[slot] + (u - m.prefix[slot])];
    return make_float4(p.x + pick4(to.off[0], c & 3), p.y + pick4(to.off[1], (c >> 2) & 3),
                       p.z + pick4(to.off[2], c >> 4), p.w);
}

// Stage the block-frame FP32 coordinates of the tile, one warp per tile cell (lanes
// over the cell's atoms, two cells per step so that two loads are in flight).
__device__ __forceinline__ void tile_stage_f32_cells(const TileMeta& m, const float4* __restrict__ xr,
                                                     const TileOffsets& to, float4* __restrict__ tile) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int slot = warp; slot < 64; slot += 2 * nw) {
        const int slot2 = slot + nw;
        const int c = c_tiles.coord_of_idx[slot];
        const int u0 = m.prefix[slot], cnt = m.prefix[slot + 1] - u0, j0 = m.start[slot];
        const int c2 = slot2 < 64 ? c_tiles.coord_of_idx[slot2] : 0;
        const int v0 = slot2 < 64 ? m.prefix[slot2] : 0;
        const int cnt2 = slot2 < 64 ? m.prefix[slot2 + 1] - v0 : 0;
        const int k0 = slot2 < 64 ? m.start[slot2] : 0;
        const float ox = pick4(to.off[0], c & 3), oy = pick4(to.off[1], (c >> 2) & 3), oz = pick4(to.off[2], c >> 4);
        const float ox2 = pick4(to.off[0], c2 & 3), oy2 = pick4(to.off[1], (c2 >> 2) & 3),
                    oz2 = pick4(to.off[2], c2 >> 4);
        const int most = cnt > cnt2 ? cnt : cnt2;
        for (int e = lane; e < most; e += 32) {
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f), q = p;
            if (e < cnt) p = xr[j0 + e];
            if (e < cnt2) q = xr[k0 + e];
            if (e < cnt) tile[u0 + e] = make_float4(p.x + ox, p.y + oy, p.z + oz, p.w);
            if (e < cnt2) tile[v0 + e] = make_float4(q.x + ox2, q.y + oy2, q.z + oz2, q.w);
        }
    }
}

// One FP32 value per tile atom into the .w of its tile entry (a single-species tile does
// not need the species there), one warp per tile cell.
__device__ __forceinline__ void tile_stage_w(const TileMeta& m, const float* __restrict__ v,
                                             float4* __restrict__ tile) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int slot = warp; slot < 64; slot += nw) {
        const int u0 = m.prefix[slot], cnt = m.prefix[slot + 1] - u0, j0 = m.start[slot];
        for (int e = lane; e < cnt; e += 32) tile[u0 + e].w = v[j0 + e];
    }
}

// Stage the block-frame FP32 coordinates of the tile (T = m.prefix[64] <= cap).
__device__ __forceinline__ void tile_stage_f32(const TileMeta& m, const float4* __restrict__ xr,
                                               const TileOffsets& to, float4* __restrict__ tile,
                                               int32_t* __restrict__ gidx) {
    const int T = m.prefix[64];
    for (int u = threadIdx.x; u < T; u += blockDim.x) {
        int slot = tile_slot_of(m, u);
        int c = c_tiles.coord_of_idx[slot];
        int j = m.start[slot] + (u - m.prefix[slot]);
        float4 p = xr[j];
        p.x += pick4(to.off[0], c & 3);
        p.y += pick4(to.off[1], (c >> 2) & 3);
        p.z += pick4(to.off[2], c >> 4);
        tile[u] = p;
        if (gidx) gidx[u] = j;
    }
}

// Stage the FP64 tile of block b: coordinates relative to the block centre (periodic
// images shifted by one box length where the tile wraps), species, and a dummy slot T
// far outside every cutoff.
__device__ __forceinline__ void tile_stage_f64(const DevState& s, const Geometry& g, const TileMeta& m, int b,
                                               double* __restrict__ tx_, double* __restrict__ ty_,
                                               double* __restrict__ tz_, int* __restrict__ tsp) {
    int bx, by, bz;
    block_coords(g, b, bx, by, bz);
    const int T = m.prefix[64];
    for (int u = threadIdx.x; u < T; u += blockDim.x) {
        const int slot = tile_slot_of(m, u);
        const int c = c_tiles.coord_of_idx[slot];
        const int j = m.start[slot] + (u - m.prefix[slot]);
        const int t3[3] = {c & 3, (c >> 2) & 3, c >> 4};
        const int b3[3] = {bx, by, bz};
        const double* X[3] = {s.x, s.y, s.z};
        double* out[3] = {tx_, ty_, tz_};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int raw = 2 * b3[d] - 1 + t3[d];
            const double shift = raw < 0 ? -g.L[d] : (raw >= g.nc[d] ? g.L[d] : 0.0);
            const double centre = (2.0 * b3[d] + 1.0) * g.w[d];
            out[d][u] = (X[d][j] + shift) - centre;
        }
        tsp[u] = s.species[j];
    }
    if (threadIdx.x == 0) {
        tx_[T] = ty_[T] = tz_[T] = 1.0e4;
        tsp[T] = 0;
    }
}

}  // namespace mdgb
