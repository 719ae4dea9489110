// k_half_af.cu - Newton-3 half lists evaluated with no atomic operation at all.
//
// The paper's schedule never lets two workers touch one particle at the same time
// (Sec. II.A), so it needs no locks; its tasks run in waves separated by barriers
// (Sec. II.B), and with Newton's third law a task writes the forces of its own cell and of
// the forward half of its neighbourhood (Sec. II.D.3).  This file carries that rule down to
// the threads of a CTA:
//
//  * the 8 colour launches give each CTA a 2x2x2-cell block whose 4x4x4-cell tile no other
//    CTA of the launch touches (as for k_force_mixed_half);
//  * inside the CTA, warp w owns cell w of the block.  The pairs of the block are split into
//    14 phases, one per offset of the half shell (the cell itself, then the 13 forward
//    cells), separated by __syncthreads: in phase p every warp writes only the atoms of cell
//    w + offset(p), and these 8 cells are different, so no two warps write one atom;
//  * inside a warp, the pairs of one (own cell, target cell) phase are laid out in steps such
//    that the 32 lanes of a step name 32 different target atoms (a matching of the bipartite
//    pair graph, built with the lists).  A lane then adds its reaction to the target's
//    shared-memory accumulator with a plain read-modify-write: no lane of the warp touches
//    that atom in the same step.
//
// Each pair is evaluated once; the force on the owning atom accumulates in registers and
// the reaction, its exact negative, in the tile's 32-bit split sums, so the fixed-point
// total force is exactly zero.  Large terms wait in a per-warp queue of exact 64-bit terms
// whose slots come from ballots.  The force kernel performs no atomic operation; an atomic
// OR sets an error bit only when a kernel finds a fault, and the schedule build sums its
// statistics (longest schedule, pair count) with one atomic per warp.
//
// The schedule is stored like a neighbour list (entry k of atom i at chunk k/8 of the
// chunked matrix): the atom's target for each step of its phases, the tile's dummy slot T
// for a step in which its lane is idle.  Cells hold at most AF_MAX_CELL atoms; cells of more
// than 32 take a second pass per phase, whose atoms keep their sums in lane-private shared
// memory.
#include "fixpt.cuh"
#include "tile.cuh"

namespace mdgb {

constexpr int AF_WARPS = 8;
constexpr int AF_PHASES = 14;
constexpr int AF_MAX_CELL = 63;  // 8 cells of at most 63 atoms: at most 504 terms per tile sum
constexpr int AF_QUEUE = 32;     // large terms per warp and launch

// Half-shell offset of phase p: p = 0 the cell itself, p = 1..13 the forward cells, with
// p = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1) - 13.
__device__ __forceinline__ void af_offset(int p, int& dx, int& dy, int& dz) {
    const int k = p + 13;
    dz = k / 9 - 1;
    dy = (k / 3) % 3 - 1;
    dx = k % 3 - 1;
}

// A pair inside one cell belongs to the atom chosen by the parity of the two tile indices
// (the lower one when the sum is odd, the higher one when it is even), so that both atoms
// own about half of their same-cell pairs.
__device__ __forceinline__ bool af_owns(int ui, int uj) { return ((ui + uj) & 1) ? ui < uj : ui > uj; }

__host__ __device__ inline size_t af_steps_per_block() { return (size_t)AF_WARPS * AF_PHASES * 2; }

// ---------------------------------------------------------------- schedule
// One CTA per block (every block, any order): warp w builds the steps of own cell w.
// steps[(b * 8 + w) * 28 + p * 2 + q] = steps of pass q of phase p.  stats: [0] the longest
// schedule, [2..3] the number of pairs (each once).
__global__ void __launch_bounds__(AF_WARPS * 32) k_build_sched(DevState s, Geometry g, TileOffsets to, double rl2,
                                                               float band_lo, float band_hi, int list_cap,
                                                               int tile_cap) {
    extern __shared__ __align__(16) float af_smem[];
    __shared__ TileMeta m;
    float* tx = af_smem;
    float* ty = tx + tile_cap;
    float* tz = ty + tile_cap;
    const int b = spatial_block(g, blockIdx.x);
    tile_meta(g, s.cell_start, b, m);
    const int T = m.prefix[64];
    if (threadIdx.x == 0) atomicMax(&s.stats[1], T + 1);
    if (T + 1 > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* steps = s.af_steps + ((size_t)b * AF_WARPS + warp) * AF_PHASES * 2;
    if (m.prefix[8] == 0) {
        for (int k = lane; k < AF_PHASES * 2; k += 32) steps[k] = 0;
        return;
    }
    for (int slot = warp; slot < 64; slot += AF_WARPS) {  // the tile's FP32 coordinates, as everywhere
        const int c = c_tiles.coord_of_idx[slot];
        const float ox = pick4(to.off[0], c & 3), oy = pick4(to.off[1], (c >> 2) & 3),
                    oz = pick4(to.off[2], c >> 4);
        const int j0 = m.start[slot], u0 = m.prefix[slot], cnt = m.prefix[slot + 1] - u0;
        for (int e = lane; e < cnt; e += 32) {
            const float4 q = s.xr[j0 + e];
            tx[u0 + e] = q.x + ox;
            ty[u0 + e] = q.y + oy;
            tz[u0 + e] = q.z + oz;
        }
    }
    __syncthreads();

    const int own_c = c_tiles.coord_of_idx[warp];
    const int cx = own_c & 3, cy = (own_c >> 2) & 3, cz = own_c >> 4;
    const int own0 = m.prefix[warp], nw = m.prefix[warp + 1] - own0;
    const int blk0 = m.start[0];
    if (nw > AF_MAX_CELL) {
        if (lane == 0) atomicOr(s.err, ERR_CELL_DENSE);
        return;
    }
    int max_len = 0;
    unsigned long long pairs = 0;
    for (int q = 0; q < 2; ++q) {
        if (q == 1 && nw <= 32) {
            for (int k = lane; k < AF_PHASES; k += 32) steps[2 * k + 1] = 0;
            break;
        }
        const int a = q * 32 + lane;
        const bool va = a < nw;
        const int ui = own0 + (va ? a : 0), gi = blk0 + ui;
        const float xi = tx[ui], yi = ty[ui], zi = tz[ui];
        uint4* const out = reinterpret_cast<uint4*>(s.nl) + gi;
        unsigned w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;  // the open chunk of this atom's schedule
        int k = 0;                                    // entries so far (the same in every lane)
        int real = 0;
        for (int p = 0; p < AF_PHASES; ++p) {
            int dx, dy, dz;
            af_offset(p, dx, dy, dz);
            const int ts = c_tiles.idx_of_coord[(cx + dx) + 4 * (cy + dy) + 16 * (cz + dz)];
            const int t0 = m.prefix[ts], mt = m.prefix[ts + 1] - t0;
            if (mt > AF_MAX_CELL) {
                if (lane == 0) atomicOr(s.err, ERR_CELL_DENSE);
                return;
            }
            // the lane's neighbours in the target cell: FP32 test, FP64 re-test in the band
            unsigned long long M = 0ull;
            for (int j = 0; j < mt; ++j) {
                const int uj = t0 + j;
                const float ex = xi - tx[uj], ey = yi - ty[uj], ez = zi - tz[uj];
                const float r2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                bool in = va && r2 < band_hi && (p != 0 || (uj != ui && af_owns(ui, uj)));
                if (in && !(r2 < band_lo))
                    in = fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gi, tile_global_index(m, uj), rl2);
                M |= (unsigned long long)in << j;
            }
            // steps: every lane with pairs left proposes one, starting its search at a
            // lane- and step-dependent position; of the lanes proposing one target the
            // lowest takes it, the others try again in the next step
            int S = 0;
            while (__any_sync(0xffffffffu, M != 0ull)) {
                int prop = -1 - lane;  // unique: matches no other lane
                if (M) {
                    const int r = (lane + S) % mt;
                    const unsigned long long rot = r ? ((M >> r) | (M << (64 - r))) : M;
                    prop = (__ffsll((long long)rot) - 1 + r) & 63;
                }
                const unsigned peers = __match_any_sync(0xffffffffu, prop);
                const bool win = prop >= 0 && lane == __ffs(peers) - 1;
                unsigned e = (unsigned)T;
                if (win) {
                    M &= ~(1ull << prop);
                    e = (unsigned)(t0 + prop);
                    ++real;
                }
                const int h = k & 7;  // uniform
                if (h == 0) w0 = e;
                else if (h == 1) w0 |= e << 16;
                else if (h == 2) w1 = e;
                else if (h == 3) w1 |= e << 16;
                else if (h == 4) w2 = e;
                else if (h == 5) w2 |= e << 16;
                else if (h == 6) w3 = e;
                else w3 |= e << 16;
                ++k;
                if ((k & 7) == 0 && va && k <= list_cap) out[(size_t)((k >> 3) - 1) * s.np] = make_uint4(w0, w1, w2, w3);
                ++S;
            }
            if (S > 255) {
                if (lane == 0) atomicOr(s.err, ERR_CELL_DENSE);
                S = 255;
            }
            if (lane == 0) steps[2 * p + q] = (uint8_t)S;
        }
        if (k & 7) {  // the last chunk, its open entries set to the dummy slot
            const int h = k & 7;
            const unsigned pad = (unsigned)T | ((unsigned)T << 16);
            auto fin = [&](unsigned& w, int wi) {
                if (2 * wi >= h) w = pad;
                else if (2 * wi + 1 >= h) w = (w & 0xffffu) | ((unsigned)T << 16);
            };
            fin(w0, 0);
            fin(w1, 1);
            fin(w2, 2);
            fin(w3, 3);
            const int kk = (k + 7) & ~7;
            if (va && kk <= list_cap) out[(size_t)((kk >> 3) - 1) * s.np] = make_uint4(w0, w1, w2, w3);
        }
        if (va) {
            if (k > list_cap) atomicOr(s.err, ERR_LIST_OVERFLOW);
            s.nl_cnt[gi] = (uint16_t)(k < list_cap ? k : list_cap);
            max_len = k > max_len ? k : max_len;
            pairs += (unsigned long long)real;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        max_len = max(max_len, __shfl_xor_sync(0xffffffffu, max_len, o));
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    }
    if (lane == 0) {
        atomicMax(&s.stats[0], max_len);
        atomicAdd(reinterpret_cast<unsigned long long*>(&s.stats[2]), pairs);
    }
}

// ---------------------------------------------------------------- forces
// The three components' split terms of one pair: t1 (high part) and t2 (low part) bits with
// the MAGIC offset, as fix_add computes them.
struct AfTerm {
    unsigned h[3], l[3];
};

__device__ __forceinline__ void af_split(float fs2, float d, unsigned& h, unsigned& l) {
    const float t1 = __fmaf_rn(fs2, d, MAGIC);
    const float hh = __fsub_rn(t1, MAGIC);
    const float r = __fmaf_rn(fs2, d, -hh);
    const float t2 = __fmaf_rn(r, TWO21, MAGIC);
    h = __float_as_uint(t1);
    l = __float_as_uint(t2);
}

struct AfWide {  // one warp's queue of large terms
    long long q[AF_QUEUE][3];
    int u[AF_QUEUE];
    int n;
};

// Shared memory: tile coordinates (float4), then the tile's six 32-bit split sums (SoA,
// each the true sum of its parts: no term counts are needed), then the lane-private split
// sums of second-pass atoms (8 warps x 6 x 32).
size_t af_force_smem_bytes(int tile_cap) {
    return (size_t)tile_cap * sizeof(float4) + (size_t)6 * tile_cap * sizeof(unsigned) +
           (size_t)AF_WARPS * 6 * 32 * sizeof(unsigned);
}

template <bool SINGLE, bool EV>
__global__ void __launch_bounds__(AF_WARPS * 32) k_force_half_af(DevState s, Geometry g, PairTable pt, TileOffsets to,
                                                                 int tile_cap, float fs2_max, int block0) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    __shared__ uint8_t st[AF_WARPS * AF_PHASES * 2];
    __shared__ AfWide wide[AF_WARPS];
    float4* tile = reinterpret_cast<float4*>(smem);
    unsigned* acc = reinterpret_cast<unsigned*>(tile + tile_cap);  // hx, lx, hy, ly, hz, lz: tile_cap each
    unsigned* priv = acc + 6 * tile_cap;                             // second-pass atoms' sums
    const int b = block0 + blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    tile_meta(g, s.cell_start, b, m);
    const int T = m.prefix[64];
    if (T + 1 > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    if (m.prefix[8] == 0) return;
    tile_stage_f32_cells(m, s.xr, to, tile);
    if (threadIdx.x == 0) tile[T] = make_float4(1.0e4f, 1.0e4f, 1.0e4f, __int_as_float(0));
    for (int u = threadIdx.x; u < 6 * tile_cap; u += blockDim.x) acc[u] = 0u;
    for (int k = threadIdx.x; k < AF_WARPS * 6 * 32; k += blockDim.x) priv[k] = 0u;
    for (int k = threadIdx.x; k < AF_WARPS * AF_PHASES * 2; k += blockDim.x)
        st[k] = s.af_steps[(size_t)b * AF_WARPS * AF_PHASES * 2 + k];
    if (lane == 0) wide[warp].n = 0;
    __syncthreads();

    const int own0 = m.prefix[warp], nw = m.prefix[warp + 1] - own0;
    const int blk0 = m.start[0];
    const int64_t n = s.n;
    const size_t np = s.np;
    const int nsp = pt.nsp;
    unsigned* const hx = acc;
    unsigned* const lx = acc + tile_cap;
    unsigned* const hy = acc + 2 * tile_cap;
    unsigned* const ly = acc + 3 * tile_cap;
    unsigned* const hz = acc + 4 * tile_cap;
    unsigned* const lz = acc + 5 * tile_cap;
    const unsigned MB = __float_as_uint(MAGIC);
    // pass 0: the lane's atom of the first 32 (sums in registers, schedule chunk by chunk)
    const bool v0 = lane < nw;
    const int ui0 = own0 + (v0 ? lane : 0), gi0 = blk0 + ui0;
    const float4 p0 = tile[ui0];
    const uint4* lp0 = reinterpret_cast<const uint4*>(s.nl) + gi0;
    uint4 cur = make_uint4(0u, 0u, 0u, 0u);
    int k0 = 0;
    FixAcc ax{0u, 0u}, ay{0u, 0u}, az{0u, 0u};
    float pe0 = 0.f, w00 = 0.f, w01 = 0.f, w02 = 0.f, w03 = 0.f, w04 = 0.f, w05 = 0.f;
    // pass 1 (cells of more than 32 atoms): the lane's second atom
    const bool v1 = 32 + lane < nw;
    const int ui1 = own0 + (v1 ? 32 + lane : 0), gi1 = blk0 + ui1;
    int k1 = 0;
    float pe1 = 0.f, w10 = 0.f, w11 = 0.f, w12 = 0.f, w13 = 0.f, w14 = 0.f, w15 = 0.f;
    unsigned* const my = priv + (size_t)warp * 6 * 32 + lane;  // its six sums, stride 32

    // One step of the atom (ui, gi, pi) against tile index u (u == T: an idle step).  The
    // reaction goes to u's tile sums; the caller adds the own terms.
    auto pair_step = [&](int ui, int gi, const float4& pi, int u, AfTerm& t, float& pe, float& w0, float& w1,
                         float& w2, float& w3, float& w4, float& w5) {
        const float4 pj = tile[u];
        const float dx = __fsub_rn(pi.x, pj.x), dy = __fsub_rn(pi.y, pj.y), dz = __fsub_rn(pi.z, pj.z);
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const int ty = SINGLE ? 0 : __float_as_int(pi.w) * nsp + __float_as_int(pj.w);
        const float inv = rcp_approx(r2);
        float fs, s6;  // the full-list kernel's formula (single species) or the tables
        if (SINGLE) {
            const float inv2 = __fmul_rn(inv, inv), inv3 = __fmul_rn(inv2, inv);
            fs = __fmul_rn(__fmaf_rn(pt.lj_a_f, inv3, -pt.lj_b_f), __fmul_rn(inv2, inv2));
            s6 = __fmul_rn(pt.sig6_f, inv3);
        } else {
            const float s2 = __fmul_rn(pt.sig2_f[ty], inv);
            s6 = __fmul_rn(__fmul_rn(s2, s2), s2);
            fs = __fmul_rn(__fmul_rn(__fmaf_rn(pt.c48_f[ty], s6, -pt.c24_f[ty]), s6), inv);
        }
        bool inside = u < T && r2 < pt.rc2hi_f[ty];
        if (inside && !(r2 < pt.rc2lo_f[ty]))  // rare: the cutoff decided by the FP64 definition
            inside = fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gi, tile_global_index(m, u),
                                    pt.rc2_d[ty]);
        float fs2 = inside ? fs : 0.0f;
        const bool big = !(fabsf(fs2) < fs2_max);  // beyond the split (or not finite): the queue
        const unsigned bigs = __ballot_sync(0xffffffffu, big);
        if (bigs) {
            if (big) {
                AfWide& wq = wide[warp];
                const int at = wq.n + 2 * __popc(bigs & ((1u << lane) - 1u));
                const long long qx = fix_term_wide(fs2, dx, s.err), qy = fix_term_wide(fs2, dy, s.err),
                                qz = fix_term_wide(fs2, dz, s.err);
                if (at + 1 < AF_QUEUE) {
                    wq.u[at] = ui;
                    wq.q[at][0] = qx;
                    wq.q[at][1] = qy;
                    wq.q[at][2] = qz;
                    wq.u[at + 1] = u;
                    wq.q[at + 1][0] = -qx;
                    wq.q[at + 1][1] = -qy;
                    wq.q[at + 1][2] = -qz;
                } else {
                    atomicOr(s.err, ERR_NONFINITE);
                }
            }
            __syncwarp();
            if (lane == 0) wide[warp].n += 2 * __popc(bigs);
            __syncwarp();
            if (big) fs2 = 0.0f;  // the split sums take a zero term
        }
        af_split(fs2, dx, t.h[0], t.l[0]);
        af_split(fs2, dy, t.h[1], t.l[1]);
        af_split(fs2, dz, t.h[2], t.l[2]);
        if (u < T) {  // the reaction: the only lane of the warp writing atom u in this step
            hx[u] += MB - t.h[0];
            lx[u] += MB - t.l[0];
            hy[u] += MB - t.h[1];
            ly[u] += MB - t.l[1];
            hz[u] += MB - t.h[2];
            lz[u] += MB - t.l[2];
        }
        if (EV && inside && !big) {
            const float c4 = SINGLE ? pt.c4_f[0] : pt.c4_f[ty];
            const float gq = fs2 * (1.0f / FS_SCALE);
            pe += c4 * s6 * (s6 - 1.0f);
            w0 = fmaf(dx, gq * dx, w0);
            w1 = fmaf(dy, gq * dy, w1);
            w2 = fmaf(dz, gq * dz, w2);
            w3 = fmaf(dx, gq * dy, w3);
            w4 = fmaf(dx, gq * dz, w4);
            w5 = fmaf(dy, gq * dz, w5);
        }
    };

    for (int p = 0; p < AF_PHASES; ++p) {
        const int S0 = st[(warp * AF_PHASES + p) * 2], S1 = st[(warp * AF_PHASES + p) * 2 + 1];
        for (int sidx = 0; sidx < S0; ++sidx, ++k0) {  // k0 is the same in every lane
            if ((k0 & 7) == 0) cur = v0 ? __ldcs(lp0 + (size_t)(k0 >> 3) * np) : make_uint4(0u, 0u, 0u, 0u);
            const unsigned wv = (k0 & 4) ? ((k0 & 2) ? cur.w : cur.z) : ((k0 & 2) ? cur.y : cur.x);
            const int u = v0 ? (int)((k0 & 1) ? (wv >> 16) : (wv & 0xffffu)) : T;
            AfTerm t;
            pair_step(ui0, gi0, p0, u, t, pe0, w00, w01, w02, w03, w04, w05);
            ax.hi += t.h[0];
            ax.lo += t.l[0];
            ay.hi += t.h[1];
            ay.lo += t.l[1];
            az.hi += t.h[2];
            az.lo += t.l[2];
        }
        for (int sidx = 0; sidx < S1; ++sidx, ++k1) {  // rare: a cell of more than 32 atoms
            const int u = v1 ? (int)s.nl[((size_t)(k1 >> 3) * np + gi1) * 8 + (k1 & 7)] : T;
            AfTerm t;
            pair_step(ui1, gi1, tile[ui1], u, t, pe1, w10, w11, w12, w13, w14, w15);
#pragma unroll
            for (int c = 0; c < 3; ++c) {  // lane-private: plain adds, with the offsets removed
                my[(2 * c) * 32] += t.h[c] - MB;
                my[(2 * c + 1) * 32] += t.l[c] - MB;
            }
        }
        __syncthreads();  // the next phase writes other cells
    }
    // the own atoms' sums into their tile sums (the phases are over: nobody else writes them)
    if (v0) {
        hx[ui0] += ax.hi - (unsigned)k0 * MB;
        lx[ui0] += ax.lo - (unsigned)k0 * MB;
        hy[ui0] += ay.hi - (unsigned)k0 * MB;
        ly[ui0] += ay.lo - (unsigned)k0 * MB;
        hz[ui0] += az.hi - (unsigned)k0 * MB;
        lz[ui0] += az.lo - (unsigned)k0 * MB;
        if (EV) {
            s.pe_atom_f[gi0] = pe0;
            s.vir_atom_f[gi0] = w00;
            s.vir_atom_f[n + gi0] = w01;
            s.vir_atom_f[2 * n + gi0] = w02;
            s.vir_atom_f[3 * n + gi0] = w03;
            s.vir_atom_f[4 * n + gi0] = w04;
            s.vir_atom_f[5 * n + gi0] = w05;
        }
    }
    if (v1) {
        hx[ui1] += my[0];
        lx[ui1] += my[32];
        hy[ui1] += my[64];
        ly[ui1] += my[96];
        hz[ui1] += my[128];
        lz[ui1] += my[160];
        if (EV) {
            s.pe_atom_f[gi1] = pe1;
            s.vir_atom_f[gi1] = w10;
            s.vir_atom_f[n + gi1] = w11;
            s.vir_atom_f[2 * n + gi1] = w12;
            s.vir_atom_f[3 * n + gi1] = w13;
            s.vir_atom_f[4 * n + gi1] = w14;
            s.vir_atom_f[5 * n + gi1] = w15;
        }
    }
    __syncthreads();
    // add the tile back: this CTA is the only one of its colour touching these atoms
    for (int u = threadIdx.x; u < T; u += blockDim.x) {
        const unsigned a0 = hx[u], a1 = lx[u], a2 = hy[u], a3 = ly[u], a4 = hz[u], a5 = lz[u];
        if ((a0 | a1 | a2 | a3 | a4 | a5) == 0u) continue;
        const int slot = tile_slot_of(m, u);
        const int gj = m.start[slot] + (u - m.prefix[slot]);
        s.fq[gj] += (long long)(int)a0 * 2097152LL + (long long)(int)a1;
        s.fq[n + gj] += (long long)(int)a2 * 2097152LL + (long long)(int)a3;
        s.fq[2 * n + gj] += (long long)(int)a4 * 2097152LL + (long long)(int)a5;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // the queued large terms, exact in 64 bits, one writer
        for (int w = 0; w < AF_WARPS; ++w) {
            const int nq = wide[w].n < AF_QUEUE ? wide[w].n : AF_QUEUE;
            for (int k = 0; k < nq; ++k) {
                const int u = wide[w].u[k];
                const int slot = tile_slot_of(m, u);
                const int gj = m.start[slot] + (u - m.prefix[slot]);
                s.fq[gj] += wide[w].q[k][0];
                s.fq[n + gj] += wide[w].q[k][1];
                s.fq[2 * n + gj] += wide[w].q[k][2];
            }
        }
    }
}

// ---------------------------------------------------------------- launchers
size_t af_sched_smem_bytes(int tile_cap) { return (size_t)3 * tile_cap * sizeof(float); }

void launch_build_sched(const DevState& s, const Geometry& g, const TileOffsets& to, double rl2, int list_cap,
                        int tile_cap, cudaStream_t st) {
    if (s.n == 0) return;
    const float lo = (float)(rl2 * (1.0 - 1e-4)), hi = (float)(rl2 * (1.0 + 1e-4));
    k_build_sched<<<g.nblock, AF_WARPS * 32, af_sched_smem_bytes(tile_cap), st>>>(s, g, to, rl2, lo, hi, list_cap,
                                                                                  tile_cap);
}

void launch_forces_half_af(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                           int tile_cap, float fs2_max, int with_energy, cudaStream_t st) {
    if (s.n == 0) return;
    cudaMemsetAsync(s.fq, 0, sizeof(long long) * 3 * (size_t)s.n, st);
    const size_t smem = af_force_smem_bytes(tile_cap);
    const bool single = pt.nsp == 1;
    const int per = g.nblock / 8;
    for (int col = 0; col < 8; ++col) {
        const int b0 = col * per;
        if (single && !with_energy)
            k_force_half_af<true, false><<<per, AF_WARPS * 32, smem, st>>>(s, g, pt, to, tile_cap, fs2_max, b0);
        else if (single)
            k_force_half_af<true, true><<<per, AF_WARPS * 32, smem, st>>>(s, g, pt, to, tile_cap, fs2_max, b0);
        else if (!with_energy)
            k_force_half_af<false, false><<<per, AF_WARPS * 32, smem, st>>>(s, g, pt, to, tile_cap, fs2_max, b0);
        else
            k_force_half_af<false, true><<<per, AF_WARPS * 32, smem, st>>>(s, g, pt, to, tile_cap, fs2_max, b0);
    }
}

template <typename K>
static void af_allow_max_smem(K kernel) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

void init_half_af_kernels() {
    af_allow_max_smem(k_build_sched);
    af_allow_max_smem(k_force_half_af<true, false>);
    af_allow_max_smem(k_force_half_af<true, true>);
    af_allow_max_smem(k_force_half_af<false, false>);
    af_allow_max_smem(k_force_half_af<false, true>);
}

}  // namespace mdgb
