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
#include "tile.cuh"

namespace mdgb {

constexpr int NL_WARPS = 8;

__device__ __forceinline__ double mic_rn(double d, double L) {
    return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

// FP64 test in the oracle's operation order.
__device__ __forceinline__ bool fp64_pair_test(const double* __restrict__ x, const double* __restrict__ y,
                                            const double* __restrict__ z, double Lx, double Ly, double Lz, int i,
                                            int j, double rl2) {
    double dx = mic_rn(__dsub_rn(x[i], x[j]), Lx);
    double dy = mic_rn(__dsub_rn(y[i], y[j]), Ly);
    double dz = mic_rn(__dsub_rn(z[i], z[j]), Lz);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < rl2;
}

typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float a, float b) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Per-warp list staging: each own atom of the warp has a 64-slot ring of list
// entries in shared memory; whole chunks of 8 entries are flushed to the list
// matrix as soon as they fill (chunk c of atom gi at uint4 index c * np + gi).
constexpr int RING = 64;
constexpr int WARP_ATOMS = 32;  // own atoms handled by one warp pass

// One neighbour cell (tile indices u0 .. u1-1) against the warp's own atoms
// own_begin .. own_begin+na-1.  Lanes hold candidates; the warp steps through the
// own atoms, and __ballot_sync / __popc turn each atom's accepted candidates into
// consecutive list slots with no per-lane loop.  OWN marks the atoms' own cell,
// where the atom itself (full lists) or every atom up to it (half lists) is excluded.
// Candidates inside the FP64 re-test band are re-tested in the definition's order.
template <int HALF, bool OWN>
__device__ __forceinline__ void scan_cell_ballot(const float4* __restrict__ tile, const int32_t* __restrict__ gidx,
                                                 const DevState& s, const Geometry& g, double rl2, int u0, int u1,
                                                 int own_begin, int na, int lane, float band_lo, float band_hi,
                                                 uint16_t* __restrict__ ring, int* __restrict__ cnt_s,
                                                 uint4* __restrict__ out0, int list_cap, int T) {
    const unsigned lt = (1u << lane) - 1u;
    for (int g0 = u0; g0 < u1; g0 += 32) {
        const int u = g0 + lane;
        const bool valid = u < u1;
        const float4 pj = tile[valid ? u : u0];
        for (int a = 0; a < na; ++a) {
            const int ui = own_begin + a;
            const float4 pi = tile[ui];  // broadcast
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            bool maybe = valid && r2 <= band_hi;
            if (OWN) maybe = maybe && (HALF ? u > ui : u != ui);
            unsigned bm = __ballot_sync(0xffffffffu, maybe);
            if (bm == 0u) continue;
            const bool sure = r2 < band_lo;
            if (__ballot_sync(0xffffffffu, maybe && !sure)) {
                bool take = maybe && (sure || fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gidx[ui],
                                                            gidx[valid ? u : u0], rl2));
                bm = __ballot_sync(0xffffffffu, take);
                maybe = take;
            }
            const int c = cnt_s[a];
            const int cn = c + __popc(bm);
            uint16_t* r = ring + a * RING;
            if (maybe) {
                const int k = c + __popc(bm & lt);
                if (k < list_cap) r[k & (RING - 1)] = (uint16_t)u;
            }
            __syncwarp();
            // flush the chunks this atom completed
            const int f0 = c >> 3, f1 = (cn < list_cap ? cn : list_cap) >> 3;
            if (lane < f1 - f0) {
                const int ch = f0 + lane;
                const uint16_t* q = r + ((ch * 8) & (RING - 1));
                uint4 v;
                v.x = q[0] | ((unsigned)q[1] << 16);
                v.y = q[2] | ((unsigned)q[3] << 16);
                v.z = q[4] | ((unsigned)q[5] << 16);
                v.w = q[6] | ((unsigned)q[7] << 16);
                out0[(size_t)ch * s.np + a] = v;
            }
            if (lane == 0) cnt_s[a] = cn;
            __syncwarp();
        }
    }
    (void)T;
}

template <int HALF>
__global__ void __launch_bounds__(NL_WARPS * 32, 2) k_build_lists(DevState s, Geometry g, TileOffsets to,
                                                               double rl2, float band_lo, float band_hi,
                                                               int list_cap, int tile_cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    float4* tile = reinterpret_cast<float4*>(smem);                    // tile_cap
    int32_t* gidx = reinterpret_cast<int32_t*>(tile + tile_cap);       // tile_cap
    int* cnt_all = reinterpret_cast<int*>(gidx + tile_cap);            // NL_WARPS x 32
    uint16_t* ring_all = reinterpret_cast<uint16_t*>(cnt_all + NL_WARPS * WARP_ATOMS);  // NL_WARPS x 32 x RING

    const int b = blockIdx.x;
    tile_meta(g, s.cell_start, b, m);
    const int T = m.prefix[64];
    if (threadIdx.x == 0) atomicMax(&s.stats[1], T + 1);
    if (T + 1 > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    tile_stage_f32(m, s.xr, to, tile, gidx);
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = warp & 1, ly = (warp >> 1) & 1, lz = warp >> 2;
    const int own_begin0 = m.prefix[warp], own_count = m.prefix[warp + 1] - own_begin0;
    const int blk0 = m.start[0];
    const int own_coord = (lx + 1) + 4 * (ly + 1) + 16 * (lz + 1);
    int* cnt_s = cnt_all + warp * WARP_ATOMS;
    uint16_t* ring = ring_all + (size_t)warp * WARP_ATOMS * RING;
    int max_cnt = 0;
    unsigned long long sum_cnt = 0;

    for (int base = 0; base < own_count; base += WARP_ATOMS) {
        const int na = own_count - base < WARP_ATOMS ? own_count - base : WARP_ATOMS;
        const int own_begin = own_begin0 + base;
        uint4* out0 = reinterpret_cast<uint4*>(s.nl) + (blk0 + own_begin);
        cnt_s[lane] = 0;
        __syncwarp();
        {
            const int slot = c_tiles.idx_of_coord[own_coord];
            scan_cell_ballot<HALF, true>(tile, gidx, s, g, rl2, m.prefix[slot], m.prefix[slot + 1], own_begin, na,
                                         lane, band_lo, band_hi, ring, cnt_s, out0, list_cap, T);
        }
#pragma unroll 1
        for (int key = HALF ? 1 : -13; key <= 13; ++key) {
            if (key == 0) continue;
            const int oz = (key + 13) / 9 - 1, oy = ((key + 13) / 3) % 3 - 1, ox = (key + 13) % 3 - 1;
            const int slot = c_tiles.idx_of_coord[own_coord + ox + 4 * oy + 16 * oz];
            scan_cell_ballot<HALF, false>(tile, gidx, s, g, rl2, m.prefix[slot], m.prefix[slot + 1], own_begin, na,
                                          lane, band_lo, band_hi, ring, cnt_s, out0, list_cap, T);
        }
        // lane a finishes atom a: last partial chunk (padded with the dummy slot T), count, stats
        if (lane < na) {
            const int cnt = cnt_s[lane];
            const int ccnt = cnt < list_cap ? cnt : list_cap;
            if (ccnt & 7) {
                const int ch = ccnt >> 3;
                const uint16_t* q = ring + lane * RING + ((ch * 8) & (RING - 1));
                unsigned e[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) e[k] = k < (ccnt & 7) ? q[k] : (unsigned)T;
                out0[(size_t)ch * s.np + lane] =
                    make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16), e[4] | (e[5] << 16), e[6] | (e[7] << 16));
            }
            if (cnt > list_cap) atomicOr(s.err, ERR_LIST_OVERFLOW);
            s.nl_cnt[blk0 + own_begin + lane] = (uint16_t)ccnt;
            max_cnt = cnt > max_cnt ? cnt : max_cnt;
            sum_cnt += (unsigned long long)cnt;
        }
        __syncwarp();
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

static size_t nl_smem_bytes(int list_cap, int tile_cap) {
    (void)list_cap;
    return (size_t)tile_cap * (sizeof(float4) + sizeof(int32_t)) + (size_t)NL_WARPS * WARP_ATOMS * sizeof(int) +
           (size_t)NL_WARPS * WARP_ATOMS * RING * sizeof(uint16_t);
}

void launch_build_lists(const DevState& s, const Geometry& g, const TileOffsets& to, double rl2, int list_cap,
                        int tile_cap, int half, cudaStream_t st) {
    if (s.n == 0) return;
    size_t smem = nl_smem_bytes(list_cap, tile_cap);
    float lo = (float)(rl2 * (1.0 - 1e-4));
    float hi = (float)(rl2 * (1.0 + 1e-4));
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
