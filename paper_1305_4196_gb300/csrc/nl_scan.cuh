// nl_scan.cuh - the candidate scan of the neighbour-list builders (k_nlist.cu, and the
// block systems of the ensemble kernel in k_batch.cu).
//
// A CTA stages its block's tile as three FP32 arrays with every cell starting on a 16-byte
// boundary (padded indices), so that one 128-bit broadcast load yields two packed FP32x2
// operands; a warp takes one own cell, one lane per atom, and scans the candidates of each
// neighbour cell in groups of 32, four per step.  Accepted entries go to a ring of slots per
// lane in shared memory and leave for global memory in chunks of 8 tile indices.
#pragma once

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
// index = padded index + adj): scan in groups of 32, re-test the band candidates in FP64
// (retest(padded index) gives the definition's answer), then append the accepted ones to
// the lane's list in candidate order.  OWN marks the atom's own cell, where the atom
// itself (full lists) or every atom up to it (half lists) is excluded; own_p is the
// atom's padded index.
template <int HALF, bool OWN, typename Retest>
__device__ __forceinline__ void scan_cell(unsigned sx, unsigned sy, unsigned sz, int p0, int cnt_c, int adj,
                                          f2_t pix, f2_t piy, f2_t piz, f2_t hi2, f2_t lo2, int own_p, bool active,
                                          ListOut& o, Retest&& retest) {
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
            if (!retest(g0 + k)) mm ^= bit;
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

// Padded SoA staging, one warp per tile cell (no search for the cell of an atom); CG:
// coordinates written by other CTAs of the same launch, read from L2.
template <bool CG = false>
__device__ __forceinline__ void tile_stage_soa(const TileMeta& m, const int* __restrict__ pp,
                                               const float4* __restrict__ xr, const TileOffsets& to,
                                               float* __restrict__ tx, float* __restrict__ ty,
                                               float* __restrict__ tz) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int slot = warp; slot < 64; slot += (int)(blockDim.x >> 5)) {
        const int c = c_tiles.coord_of_idx[slot];
        const float ox = pick4(to.off[0], c & 3), oy = pick4(to.off[1], (c >> 2) & 3),
                    oz = pick4(to.off[2], c >> 4);
        const int j0 = m.start[slot], cnt = m.prefix[slot + 1] - m.prefix[slot], q0 = pp[slot];
        for (int e = lane; e < cnt; e += 32) {
            const float4 p = CG ? __ldcg(xr + j0 + e) : xr[j0 + e];
            tx[q0 + e] = p.x + ox;
            ty[q0 + e] = p.y + oy;
            tz[q0 + e] = p.z + oz;
        }
    }
}

// Padded SoA array length for a tile of at most tile_cap atoms: 3 padding slots per
// cell at most, plus one group of read-ahead past the last cell.
__host__ __device__ inline int soa_len(int tile_cap) { return (tile_cap + 64 * 3 + 32 + 3) & ~3; }

}  // namespace mdgb
