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
#include "fixpt.cuh"
#include "tile.cuh"

namespace mdgb {

constexpr int NL_WARPS = 8;

// Two packed FP32 pairs from 16 bytes of shared memory (one 128-bit load).
__device__ __forceinline__ void lds_f2x2(unsigned addr, f2_t& lo, f2_t& hi) {
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "r"(addr));
}

__device__ __forceinline__ unsigned sign_in(unsigned mask, float v) {
    return __funnelshift_l(__float_as_uint(v), mask, 1);  // (mask << 1) | sign bit of v
}

// Scan of one group of up to 32 consecutive candidates of the padded tile (padded
// index g0, a multiple of 4; nvalid of them are real) against a lane's atom, four per
// step: one 128-bit broadcast load per coordinate, packed FP32x2 arithmetic.  The scan
// stops after the step holding the last real candidate (nvalid is the same for the
// whole warp).  Candidate k of the group lands in bit 31-k of the masks: `maybe` has
// r^2 <= band_hi (inside the list radius or in the FP64 re-test band), `sure` has
// r^2 < band_lo (inside for certain).  Each bit is the sign of r^2 - threshold
// shifted in; bits past the scanned steps are zero.
__device__ __forceinline__ void scan_group(unsigned sx, unsigned sy, unsigned sz, int g0, int nvalid, f2_t pix,
                                           f2_t piy, f2_t piz, f2_t hi2, f2_t lo2, unsigned& maybe,
                                           unsigned& sure) {
    unsigned mm = 0u, ms = 0u;
    const unsigned off0 = (unsigned)g0 * 4u;
    int k = 0;
#pragma unroll
    for (; k < 32; k += 4) {
        if (k >= nvalid) break;
        f2_t x01, x23, y01, y23, z01, z23;
        lds_f2x2(sx + off0 + 4u * k, x01, x23);
        lds_f2x2(sy + off0 + 4u * k, y01, y23);
        lds_f2x2(sz + off0 + 4u * k, z01, z23);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const f2_t dx = f2_sub(pix, h ? x23 : x01);
            const f2_t dy = f2_sub(piy, h ? y23 : y01);
            const f2_t dz = f2_sub(piz, h ? z23 : z01);
            const f2_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
            float ha, hb, la, lb;
            f2_unpack(f2_sub(r2, hi2), ha, hb);
            f2_unpack(f2_sub(r2, lo2), la, lb);
            mm = sign_in(sign_in(mm, ha), hb);
            ms = sign_in(sign_in(ms, la), lb);
        }
    }
    // k candidates were shifted in (k >= 4): move candidate 0 to bit 31
    maybe = k < 32 ? mm << (32 - k) : mm;
    sure = k < 32 ? ms << (32 - k) : ms;
}

// A lane's list output.  Accepted entries go to a ring of NL_RING slots in shared
// memory (slot r at col[r * 32]) and leave for global memory in full chunks of 8 as
// soon as they are complete, so the CTA never holds whole lists on chip.
constexpr int NL_RING = 64;

struct ListOut {
    uint16_t* col;  // this lane's ring
    uint4* out;     // chunk 0 of this atom's list; chunk c at out[c * np]
    size_t np;
    int list_cap;
    int cnt;      // entries accepted so far (may exceed list_cap: overflow)
    int flushed;  // entries already written to global memory (a multiple of 8)
};

__device__ __forceinline__ unsigned ring_pair(const uint16_t* __restrict__ col, int k, int stored, unsigned pad) {
    const unsigned a = k < stored ? (unsigned)col[(k & (NL_RING - 1)) * 32] : pad;
    const unsigned b = k + 1 < stored ? (unsigned)col[((k + 1) & (NL_RING - 1)) * 32] : pad;
    return a | (b << 16);
}

// Write every complete chunk; with pad < 65536 also the last partial chunk, padded.
__device__ __forceinline__ void flush_chunks(ListOut& o, unsigned pad, bool last) {
    const int stored = o.cnt < o.list_cap ? o.cnt : o.list_cap;
    while (stored - o.flushed >= 8 || (last && stored > o.flushed)) {
        const int k = o.flushed;
        o.out[(size_t)(k >> 3) * o.np] = make_uint4(ring_pair(o.col, k, stored, pad), ring_pair(o.col, k + 2, stored, pad),
                                                    ring_pair(o.col, k + 4, stored, pad),
                                                    ring_pair(o.col, k + 6, stored, pad));
        o.flushed = k + 8;
    }
}

// Candidates of one neighbour cell (padded indices p0 .. p0+cnt-1; canonical tile
// index = padded index + adj, cell-ordered atom index = padded index + jadj): scan in
// groups of 32, re-test the band candidates in FP64, then append the accepted ones to
// the lane's list in candidate order.  OWN marks the atom's own cell, where the atom
// itself (full lists) or every atom up to it (half lists) is excluded; own_p is the
// atom's padded index.
template <int HALF, bool OWN>
__device__ __forceinline__ void scan_cell(unsigned sx, unsigned sy, unsigned sz, const DevState& s,
                                          const Geometry& g, double rl2, int p0, int cnt_c, int adj, int jadj,
                                          f2_t pix, f2_t piy, f2_t piz, f2_t hi2, f2_t lo2, int own_p, int gi_own,
                                          bool active, ListOut& o) {
    const int p1 = p0 + cnt_c;
    for (int g0 = p0; g0 < p1; g0 += 32) {
        unsigned mm, ms;
        const int nvalid = p1 - g0;
        scan_group(sx, sy, sz, g0, nvalid, pix, piy, piz, hi2, lo2, mm, ms);
        if (nvalid < 32) mm &= ~0u << (32 - nvalid);
        if (OWN) {
            const int rel = own_p - g0;  // own atom's bit is 31 - rel
            if (HALF) {
                if (rel >= 31) mm = 0u;
                else if (rel >= 0) mm &= ~0u >> (rel + 1);
            } else if (rel >= 0 && rel < 32) {
                mm &= ~(0x80000000u >> rel);
            }
        }
        if (!active) mm = 0u;
        const int ubase = g0 + adj;
        unsigned band = mm & ~ms;
        while (band) {  // rare: within 1e-4 of r_list^2 in relative terms
            const int k = __clz(band);
            const unsigned bit = 0x80000000u >> k;
            band ^= bit;
            if (!fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gi_own, g0 + jadj + k, rl2)) mm ^= bit;
        }
        if (!mm) continue;
        const int nb = __popc(mm);
        int c = o.cnt;
        if (c + nb <= o.list_cap) {
            while (mm) {
                const int k = __clz(mm);
                mm ^= 0x80000000u >> k;
                o.col[(c & (NL_RING - 1)) * 32] = (uint16_t)(ubase + k);
                ++c;
            }
        } else {
            while (mm) {
                const int k = __clz(mm);
                mm ^= 0x80000000u >> k;
                if (c < o.list_cap) o.col[(c & (NL_RING - 1)) * 32] = (uint16_t)(ubase + k);
                ++c;
            }
        }
        o.cnt = c;
        flush_chunks(o, 0u, false);
    }
}

// Padded cell starts of the tile: every cell's first atom at a multiple of 4, so
// that candidate groups start on 16-byte boundaries.  Threads 0..63; ends with
// __syncthreads.
__device__ __forceinline__ void tile_pad_prefix(const TileMeta& m, int* __restrict__ pp) {
    const int t = threadIdx.x;
    if (t < 64) {
        const int cnt = m.prefix[t + 1] - m.prefix[t];
        int v = (cnt + 3) & ~3;
        const int lane = t & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        pp[t + 1] = v;
    }
    __syncthreads();
    if (t >= 32 && t < 64) pp[t + 1] += pp[32];
    if (t == 0) pp[0] = 0;
    __syncthreads();
}

// Padded SoA staging, one warp per tile cell (no search for the cell of an atom).
__device__ __forceinline__ void tile_stage_soa(const TileMeta& m, const int* __restrict__ pp,
                                               const float4* __restrict__ xr, const TileOffsets& to,
                                               float* __restrict__ tx, float* __restrict__ ty,
                                               float* __restrict__ tz) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int slot = warp; slot < 64; slot += NL_WARPS) {
        const int c = c_tiles.coord_of_idx[slot];
        const float ox = pick4(to.off[0], c & 3), oy = pick4(to.off[1], (c >> 2) & 3),
                    oz = pick4(to.off[2], c >> 4);
        const int j0 = m.start[slot], cnt = m.prefix[slot + 1] - m.prefix[slot], q0 = pp[slot];
        for (int e = lane; e < cnt; e += 32) {
            const float4 p = xr[j0 + e];
            tx[q0 + e] = p.x + ox;
            ty[q0 + e] = p.y + oy;
            tz[q0 + e] = p.z + oz;
        }
    }
}

// Padded SoA array length for a tile of at most tile_cap atoms: 3 padding slots per
// cell at most, plus one group of read-ahead past the last cell.
__host__ __device__ inline int soa_len(int tile_cap) { return (tile_cap + 64 * 3 + 32 + 3) & ~3; }

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
    if (threadIdx.x == 0) atomicMax(&s.stats[1], T + 1);
    if (T + 1 > tile_cap) {
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
            scan_cell<HALF, true>(sx, sy, sz, s, g, rl2, pp[slot], m.prefix[slot + 1] - m.prefix[slot],
                                  m.prefix[slot] - pp[slot], m.start[slot] - pp[slot], pix, piy, piz, hi2, lo2,
                                  own_p, gi, active, o);
        }
#pragma unroll 1
        for (int key = HALF ? 1 : -13; key <= 13; ++key) {
            if (key == 0) continue;
            const int oz = (key + 13) / 9 - 1, oy = ((key + 13) / 3) % 3 - 1, ox = (key + 13) % 3 - 1;
            const int slot = c_tiles.idx_of_coord[own_coord + ox + 4 * oy + 16 * oz];
            scan_cell<HALF, false>(sx, sy, sz, s, g, rl2, pp[slot], m.prefix[slot + 1] - m.prefix[slot],
                                   m.prefix[slot] - pp[slot], m.start[slot] - pp[slot], pix, piy, piz, hi2, lo2,
                                   own_p, gi, active, o);
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
