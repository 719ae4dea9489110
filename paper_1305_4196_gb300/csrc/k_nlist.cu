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
__device__ __forceinline__ float pi_x(f2_t v) {
    float a, b;
    f2_unpack(v, a, b);
    return a;
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

// Scan of one group of 32 consecutive tile candidates g0 .. g0+31 against a lane's
// atom, two per step in packed FP32x2.  Candidate k of the group lands in bit
// 31-k of the masks: `maybe` has r^2 <= band_hi (inside the list radius or in the
// FP64 re-test band), `sure` has r^2 < band_lo (inside for certain).  Each bit is
// the sign of r^2 - threshold shifted in, so a candidate costs one integer op on
// top of its distance arithmetic.
__device__ __forceinline__ void scan_group(const float4* __restrict__ tile, int g0, f2_t pix, f2_t piy, f2_t piz,
                                           f2_t hi2, f2_t lo2, unsigned& maybe, unsigned& sure) {
    unsigned mm = 0u, ms = 0u;
#pragma unroll
    for (int k = 0; k < 32; k += 2) {
        const float4 pa = tile[g0 + k];
        const float4 pb = tile[g0 + k + 1];
        const f2_t dx = f2_sub(pix, f2_pack(pa.x, pb.x));
        const f2_t dy = f2_sub(piy, f2_pack(pa.y, pb.y));
        const f2_t dz = f2_sub(piz, f2_pack(pa.z, pb.z));
        const f2_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
        float ha, hb, la, lb;
        f2_unpack(f2_sub(r2, hi2), ha, hb);
        f2_unpack(f2_sub(r2, lo2), la, lb);
        mm = (mm << 1) | (__float_as_uint(ha) >> 31);
        mm = (mm << 1) | (__float_as_uint(hb) >> 31);
        ms = (ms << 1) | (__float_as_uint(la) >> 31);
        ms = (ms << 1) | (__float_as_uint(lb) >> 31);
    }
    maybe = mm;
    sure = ms;
}

// Candidates u0 .. u1-1 of one neighbour cell: scan in groups of 32, then append
// the accepted ones to the lane's column of the list buffer in candidate order.
// OWN marks the atom's own cell, where the atom itself (full lists) or every atom
// up to it (half lists) is excluded.  Band candidates are re-tested in FP64.
template <int HALF, bool OWN>
__device__ __forceinline__ void scan_cell(const float4* __restrict__ tile, const int32_t* __restrict__ gidx,
                                          const DevState& s, const Geometry& g, double rl2, int u0, int u1, f2_t pix,
                                          f2_t piy, f2_t piz, f2_t hi2, f2_t lo2, int ui, bool active,
                                          uint16_t* __restrict__ col, int list_cap, int& cnt) {
    for (int g0 = u0; g0 < u1; g0 += 32) {
        unsigned mm, ms;
        scan_group(tile, g0, pix, piy, piz, hi2, lo2, mm, ms);
        const int nvalid = u1 - g0;
        if (nvalid < 32) mm &= ~0u << (32 - nvalid);
        if (OWN) {
            const int rel = ui - g0;  // own atom's bit is 31 - rel
            if (HALF) {
                if (rel >= 31) mm = 0u;
                else if (rel >= 0) mm &= ~0u >> (rel + 1);
            } else if (rel >= 0 && rel < 32) {
                mm &= ~(0x80000000u >> rel);
            }
        }
        if (!active) mm = 0u;
        const unsigned band = mm & ~ms;
        while (mm) {
            const int k = __clz(mm);
            const unsigned bit = 0x80000000u >> k;
            mm &= ~bit;
            const int u = g0 + k;
            if (band & bit) {
                if (!fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gidx[ui], gidx[u], rl2)) continue;
            }
            if (cnt < list_cap) col[cnt * 32] = (uint16_t)u;
            ++cnt;
        }
    }
}

template <int HALF>
__global__ void __launch_bounds__(NL_WARPS * 32, 2) k_build_lists(DevState s, Geometry g, TileOffsets to,
                                                                  double rl2, float band_lo, float band_hi,
                                                                  int list_cap, int tile_cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    float4* tile = reinterpret_cast<float4*>(smem);                   // tile_cap + 32: groups read past T
    int32_t* gidx = reinterpret_cast<int32_t*>(tile + tile_cap + 32);  // tile_cap
    uint16_t* buf = reinterpret_cast<uint16_t*>(gidx + tile_cap);     // NL_WARPS x list_cap x 32

    const int b = blockIdx.x;
    tile_meta(g, s.cell_start, b, m);
    const int T = m.prefix[64];
    if (threadIdx.x == 0) atomicMax(&s.stats[1], T + 1);
    if (T + 1 > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    tile_stage_f32(m, s.xr, to, tile, gidx);
    for (int u = T + threadIdx.x; u < T + 32; u += blockDim.x)
        tile[u] = make_float4(1.0e4f, 1.0e4f, 1.0e4f, __int_as_float(0));
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = warp & 1, ly = (warp >> 1) & 1, lz = warp >> 2;
    const int own_begin = m.prefix[warp], own_count = m.prefix[warp + 1] - own_begin;
    uint16_t* col = buf + (size_t)warp * list_cap * 32 + lane;
    const int blk0 = m.start[0];
    const int own_coord = (lx + 1) + 4 * (ly + 1) + 16 * (lz + 1);
    const f2_t hi2 = f2_pack(band_hi, band_hi), lo2 = f2_pack(band_lo, band_lo);
    int max_cnt = 0;
    unsigned long long sum_cnt = 0;

    for (int base = 0; base < own_count; base += 32) {
        const int e = base + lane;
        const bool active = e < own_count;
        const int ui = own_begin + (active ? e : 0);
        const float4 pi = tile[ui];
        const f2_t pix = f2_pack(pi.x, pi.x), piy = f2_pack(pi.y, pi.y), piz = f2_pack(pi.z, pi.z);
        int cnt = 0;
        {
            const int slot = c_tiles.idx_of_coord[own_coord];
            scan_cell<HALF, true>(tile, gidx, s, g, rl2, m.prefix[slot], m.prefix[slot + 1], pix, piy, piz, hi2,
                                  lo2, ui, active, col, list_cap, cnt);
        }
#pragma unroll 1
        for (int key = HALF ? 1 : -13; key <= 13; ++key) {
            if (key == 0) continue;
            const int oz = (key + 13) / 9 - 1, oy = ((key + 13) / 3) % 3 - 1, ox = (key + 13) % 3 - 1;
            const int slot = c_tiles.idx_of_coord[own_coord + ox + 4 * oy + 16 * oz];
            scan_cell<HALF, false>(tile, gidx, s, g, rl2, m.prefix[slot], m.prefix[slot + 1], pix, piy, piz, hi2,
                                   lo2, ui, active, col, list_cap, cnt);
        }
        const int gi = blk0 + ui;
        if (active) {
            if (cnt > list_cap) atomicOr(s.err, ERR_LIST_OVERFLOW);
            s.nl_cnt[gi] = (uint16_t)(cnt < list_cap ? cnt : list_cap);
            max_cnt = cnt > max_cnt ? cnt : max_cnt;
            sum_cnt += (unsigned long long)cnt;
        }
        // write the lists in chunks of 8 (one 16-byte store per chunk), padding the
        // last chunk with the tile's dummy slot T
        const int ccnt = active ? (cnt < list_cap ? cnt : list_cap) : 0;
        const int nch = (ccnt + 7) >> 3;
        int wch = nch;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wch = max(wch, __shfl_xor_sync(0xffffffffu, wch, o));
        __syncwarp();
        uint4* out = reinterpret_cast<uint4*>(s.nl) + gi;
        for (int c = 0; c < wch; ++c) {
            if (c < nch) {
                unsigned v[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int k0 = 8 * c + 2 * h, k1 = k0 + 1;
                    const unsigned a0 = k0 < ccnt ? col[k0 * 32] : (unsigned)T;
                    const unsigned a1 = k1 < ccnt ? col[k1 * 32] : (unsigned)T;
                    v[h] = a0 | (a1 << 16);
                }
                out[(size_t)c * s.np] = make_uint4(v[0], v[1], v[2], v[3]);
            }
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
    return (size_t)(tile_cap + 32) * sizeof(float4) + (size_t)tile_cap * sizeof(int32_t) +
           (size_t)NL_WARPS * 32 * list_cap * 2;
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
