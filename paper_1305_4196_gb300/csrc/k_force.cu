// k_force.cu - Lennard-Jones forces by cell tasks (Sec. II.A, step 2).
//
// One CTA is the task of one 2x2x2-cell block (Sec. II.D.2 blocking): it
// stages the block's 4x4x4-cell tile in shared memory and evaluates the
// neighbour lists of the block's own atoms against it.
//
//  * Full lists: one thread per atom i, accumulating only F_i.  No thread
//    ever writes an atom it does not own, so the paper's requirement that no
//    particle is updated by two workers at once (Sec. II.A) holds with no
//    synchronisation at all.
//  * Half lists (Newton's third law, Sec. II.D.3): each pair once; the
//    reaction -f_ij goes to the tile copy of j in shared memory, and the tile
//    is added back to global memory at the end.  Blocks of one colour class
//    have disjoint tiles, so one launch per colour runs only non-overlapping
//    tasks - the barrier-separated waves of Sec. II.B, 8 of them.  No global
//    atomics are used; within a CTA the tile accumulators take shared-memory
//    integer adds.
//
// Mixed precision: pair arithmetic in FP32 on block-frame coordinates; every
// pair force component q = rint(f * 2^32) is added in Q31.32 fixed point,
// split exactly into a high part (multiples of 2^21) and a low part, each
// summed in a 32-bit integer.  Integer sums do not depend on order, so the
// result is bit-reproducible for any list order, thread mapping or list kind,
// and f_ji = -f_ij bit for bit makes the total force exactly zero.
//
// FP64: the same structure with FP64 tile coordinates and FP64 sums (k_force_fp64.cu).
#include "fixpt.cuh"
#include "tile.cuh"

namespace mdgb {

constexpr int F_THREADS = 256;
enum { FM_FORCE = 0, FM_KICK = 1, FM_KKD = 2 };  // what the full-list mixed kernel does after the force
constexpr int FULL_THREADS = 256;  // CTA size of the full-list mixed kernel
// Register cap of the full-list mixed kernel: 48 keeps 5 CTAs (40 warps) resident per SM.
// The kernel is latency bound, and more resident warps beat longer per-thread schedules.
#define MDGB_FULL_MAX_REGS 48
// With several species the pair constants come from shared memory, and 48 registers spill.
#define MDGB_FULL_MAX_REGS_SPECIES 64
// per-pair LJ in FP32: returns fs2 = (|f|/r) * 2^11 (not masked) and whether the FP32
// r^2 is inside the cutoff
template <bool SINGLE>
__device__ __forceinline__ float lj_fs_unmasked(const PairTable& pt, int t, float r2, float& s6_out, bool& inside) {
    const float sig2 = SINGLE ? pt.sig2_f[0] : pt.sig2_f[t];
    const float c48 = SINGLE ? pt.c48_f[0] : pt.c48_f[t];
    const float c24 = SINGLE ? pt.c24_f[0] : pt.c24_f[t];
    const float rc2 = SINGLE ? pt.rc2_f[0] : pt.rc2_f[t];
    const float inv = rcp_approx(r2);
    const float s2 = sig2 * inv;
    const float s6 = s2 * s2 * s2;
    inside = r2 < rc2;
    s6_out = s6;
    return (c48 * s6 - c24) * s6 * inv;  // constants carry the 2^11 scale
}

__device__ __forceinline__ void stage_dummy_f32(float4* tile, int T) {
    if (threadIdx.x == 0) tile[T] = make_float4(1.0e4f, 1.0e4f, 1.0e4f, __int_as_float(0));
}

// Species constants of a CTA in shared memory (dynamic indexing of kernel parameters
// would go through local memory).
struct SpeciesTable {
    float sig2[MAX_PAIR], c48[MAX_PAIR], c24[MAX_PAIR], c4[MAX_PAIR], rc2[MAX_PAIR];
    float rc2lo[MAX_PAIR], rc2hi[MAX_PAIR];  // r_cut^2 (1 -/+ cut_band): the FP64 decision band
    double rc2d[MAX_PAIR];                   // FP64 r_cut^2
};

__device__ __forceinline__ void load_species_table(const PairTable& pt, SpeciesTable& st) {
    const int t = threadIdx.x;
    if (t < MAX_PAIR) {
        st.sig2[t] = pt.sig2_f[t];
        st.c48[t] = pt.c48_f[t];
        st.c24[t] = pt.c24_f[t];
        st.c4[t] = pt.c4_f[t];
        st.rc2[t] = pt.rc2_f[t];
        st.rc2lo[t] = pt.rc2lo_f[t];
        st.rc2hi[t] = pt.rc2hi_f[t];
        st.rc2d[t] = pt.rc2_d[t];
    }
}

// What follows an atom's force in the full-list mixed kernels (MODE as below); one
// function so that every kernel applies exactly the same operations.
template <bool SINGLE, int MODE>
__device__ __forceinline__ void full_epilogue(const DevState& s, const PairTable& pt, int gi, int si, long long qx,
                                              long long qy, long long qz, const StepOut& out, double dt,
                                              float lim2_f) {
    const int64_t n = s.n;
    if (MODE != FM_KKD) {
        s.fq[gi] = qx;
        s.fq[n + gi] = qy;
        s.fq[2 * n + gi] = qz;
    }
    if (MODE != FM_FORCE) {
        const double hq = pt.hdtm_q[SINGLE ? 0 : si];
        const double kq = MODE == FM_KKD ? 2.0 * hq : hq;
        const double vx = fma(kq, (double)qx, s.vx[gi]);
        const double vy = fma(kq, (double)qy, s.vy[gi]);
        const double vz = fma(kq, (double)qz, s.vz[gi]);
        s.vx[gi] = vx;
        s.vy[gi] = vy;
        s.vz[gi] = vz;
        if (MODE == FM_KKD) {
            const double x = fma(dt, vx, s.x[gi]), y = fma(dt, vy, s.y[gi]), z = fma(dt, vz, s.z[gi]);
            out.x[gi] = x;
            out.y[gi] = y;
            out.z[gi] = z;
            const int c = s.cell_of[gi];
            const float4 r = s.xr_ref[gi];
            float4 q;
            q.x = __double2float_rn(x - s.centre[c]);
            q.y = __double2float_rn(y - s.centre[s.ncell + c]);
            q.z = __double2float_rn(z - s.centre[2 * s.ncell + c]);
            q.w = r.w;
            out.xr[gi] = q;
            const float ex = q.x - r.x, ey = q.y - r.y, ez = q.z - r.z;
            if (!(fmaf(ez, ez, fmaf(ey, ey, ex * ex)) <= lim2_f)) *s.rebuild_flag = 1;
        }
    }
}

// Exact finish of one atom by one warp (all 32 lanes), for an atom that the FP32 loop
// below cannot finish: a pair whose FP32 r^2 lies within the band around r_cut^2 (the
// cutoff is decided by the FP64 definition) or a pair force component that may reach
// 2048 eps/sigma (beyond the two-part split; or not finite).  About one atom in 1,500 of
// a liquid.  The neighbours come from the CTA's tile, so every other pair gets exactly
// the term the FP32 loop adds; band pairs are decided in FP64 in the oracle's operation
// order; large terms are rounded in FP64 (fix_term_wide).  Each lane keeps the 32-bit
// split sums of the FP32 loop, and the terms they cannot take - large terms, and the
// lane's split sums every FIX_SPLIT_MAX_TERMS terms - go to the warp's exact 64-bit sums
// in shared memory (WarpWide), so this rare path adds no 64-bit registers to the kernel
// it is inlined into.  All sums are exact integers, so the warp total does not depend on
// how the list is spread over the lanes.  The same epilogue follows.  This runs after the
// loop, not inside it: a call from the loop cost the kernel half its speed.
struct WarpWide {
    unsigned long long q[3];
    int nwide;
};

template <bool SINGLE, bool EV, int MODE>
__device__ __forceinline__ void finish_atom_warp(const DevState& s, const Geometry& g, const PairTable& pt,
                                                 const float4* __restrict__ tile, const SpeciesTable& stab,
                                                 const TileMeta& m, int ui, float fs2_max, const StepOut& out,
                                                 double dt, float lim2_f, WarpWide& ww) {
    const int lane = threadIdx.x & 31;
    const int T = m.prefix[64];
    const int gi = m.start[0] + ui;
    const float4 pi = tile[ui];
    const int si = __float_as_int(pi.w);
    const int nsp = pt.nsp;
    const int nent = ((s.nl_cnt[gi] + 7) >> 3) * 8;
    if (lane == 0) {
        ww.q[0] = ww.q[1] = ww.q[2] = 0ull;
        ww.nwide = 0;
    }
    __syncwarp();
    FixAcc ax{0u, 0u}, ay{0u, 0u}, az{0u, 0u};
    int nterms = 0;
    float pe = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;
    for (int k = lane; k < nent; k += 32) {
        const int u = s.nl[((size_t)(k >> 3) * s.np + gi) * 8 + (k & 7)];
        if (u >= T) continue;  // padding (the tile's dummy slot): no force
        const float4 pj = tile[u];
        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const int t = SINGLE ? 0 : si * nsp + __float_as_int(pj.w);
        const float inv = rcp_approx(r2);
        float fs, s6;  // the FP32 loop's operations, term for term
        if (SINGLE) {
            const float inv2 = __fmul_rn(inv, inv), inv3 = __fmul_rn(inv2, inv);
            fs = __fmul_rn(__fmaf_rn(pt.lj_a_f, inv3, -pt.lj_b_f), __fmul_rn(inv2, inv2));
            s6 = __fmul_rn(pt.sig6_f, inv3);
        } else {
            const float s2 = __fmul_rn(stab.sig2[t], inv);
            s6 = __fmul_rn(__fmul_rn(s2, s2), s2);
            fs = __fmul_rn(__fmul_rn(__fmaf_rn(stab.c48[t], s6, -stab.c24[t]), s6), inv);
        }
        bool inside = r2 < stab.rc2lo[t];
        if (!inside && r2 < stab.rc2hi[t])
            inside = fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gi, tile_global_index(m, u),
                                    stab.rc2d[t]);
        const float fs2 = inside ? fs : 0.0f;
        if (fabsf(fs2) < fs2_max) {
            fix_add(ax, fs2, dx);
            fix_add(ay, fs2, dy);
            fix_add(az, fs2, dz);
            if (++nterms == FIX_SPLIT_MAX_TERMS) {  // only for lists of more than 16,000 entries
                atomicAdd(&ww.q[0], (unsigned long long)fix_final(ax, nterms));
                atomicAdd(&ww.q[1], (unsigned long long)fix_final(ay, nterms));
                atomicAdd(&ww.q[2], (unsigned long long)fix_final(az, nterms));
                ax = ay = az = FixAcc{0u, 0u};
                nterms = 0;
            }
        } else {
            atomicAdd(&ww.q[0], (unsigned long long)fix_term_wide(fs2, dx, s.err));
            atomicAdd(&ww.q[1], (unsigned long long)fix_term_wide(fs2, dy, s.err));
            atomicAdd(&ww.q[2], (unsigned long long)fix_term_wide(fs2, dz, s.err));
            atomicAdd(&ww.nwide, 1);
        }
        if (EV && inside) {
            const float gq = fs2 * (1.0f / FS_SCALE);
            pe += stab.c4[t] * s6 * (s6 - 1.0f);
            w0 += dx * (gq * dx);
            w1 += dy * (gq * dy);
            w2 += dz * (gq * dz);
            w3 += dx * (gq * dy);
            w4 += dx * (gq * dz);
            w5 += dy * (gq * dz);
        }
    }
    long long qx = fix_final(ax, nterms), qy = fix_final(ay, nterms), qz = fix_final(az, nterms);
    __syncwarp();
    if (lane == 0) {
        fix_wide_count_ok(ww.nwide, s.err);
        qx += (long long)ww.q[0];
        qy += (long long)ww.q[1];
        qz += (long long)ww.q[2];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        qx += __shfl_xor_sync(0xffffffffu, qx, o);
        qy += __shfl_xor_sync(0xffffffffu, qy, o);
        qz += __shfl_xor_sync(0xffffffffu, qz, o);
        if (EV) {  // a fixed butterfly: the FP32 sums are reproducible
            pe += __shfl_xor_sync(0xffffffffu, pe, o);
            w0 += __shfl_xor_sync(0xffffffffu, w0, o);
            w1 += __shfl_xor_sync(0xffffffffu, w1, o);
            w2 += __shfl_xor_sync(0xffffffffu, w2, o);
            w3 += __shfl_xor_sync(0xffffffffu, w3, o);
            w4 += __shfl_xor_sync(0xffffffffu, w4, o);
            w5 += __shfl_xor_sync(0xffffffffu, w5, o);
        }
    }
    if (lane == 0) {
        full_epilogue<SINGLE, MODE>(s, pt, gi, si, qx, qy, qz, out, dt, lim2_f);
        if (EV) {
            const int64_t n = s.n;
            s.pe_atom_f[gi] = 0.5f * pe;
            s.vir_atom_f[gi] = 0.5f * w0;
            s.vir_atom_f[n + gi] = 0.5f * w1;
            s.vir_atom_f[2 * n + gi] = 0.5f * w2;
            s.vir_atom_f[3 * n + gi] = 0.5f * w3;
            s.vir_atom_f[4 * n + gi] = 0.5f * w4;
            s.vir_atom_f[5 * n + gi] = 0.5f * w5;
        }
    }
}

// ---------------------------------------------------------------- mixed, full list
// One thread per atom, two neighbours per iteration in packed FP32x2 arithmetic; each
// neighbour is one 128-bit shared-memory load.
//
// MODE selects what follows each atom's force (fused velocity Verlet, the same
// operations as k_integrate's mixed path, so fused and separate steps agree bit for
// bit):
//   FM_FORCE  store the fixed-point force;
//   FM_KICK   store it and apply the closing half kick v += (dt/2m) F;
//   FM_KKD    closing and next opening kick in one, v += 2 (dt/2m) F, then the drift
//             x += dt v into out (the other position buffers: other CTAs may still be
//             staging this atom's current FP32 coordinates or testing a pair near r_cut
//             with its current FP64 position), the new FP32 coordinates beside it, and
//             the skin/2 displacement test.  The force itself is not stored.
//
// full_block is the task of block b for the CTA that calls it; k_force_mixed_full runs one
// block per CTA in spatial order, k_force_mixed_occ loops over the occupied blocks of a
// compact system.
template <bool SINGLE, bool EV, int MODE>
__device__ __forceinline__ void full_block(const DevState& s, const Geometry& g, const PairTable& pt,
                                           const TileOffsets& to, int tile_cap, float fs2_max, const StepOut& out,
                                           double dt, float lim2_f, int b) {
    static_assert(!EV || MODE == FM_FORCE, "energy/virial launches only evaluate forces");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    __shared__ SpeciesTable stab;
    __shared__ WarpWide wwide[FULL_THREADS / 32];
    float4* tile = reinterpret_cast<float4*>(smem);
    // own atoms left to finish_atom_warp: bit ui % 32 of word ui / 32.  Own atom ui runs on
    // thread ui % blockDim.x, so word w is written and read by warp w % (warps) alone
    unsigned* qmask = reinterpret_cast<unsigned*>(tile + tile_cap);
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    load_species_table(pt, stab);
    tile_meta(g, s.cell_start, b, m);
    const int T = m.prefix[64];
    if (T + 1 > tile_cap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    const int nown = m.prefix[8];
    if (nown == 0) return;
    tile_stage_f32_cells(m, s.xr, to, tile);
    stage_dummy_f32(tile, T);
    __syncthreads();
    const unsigned tile_s = (unsigned)__cvta_generic_to_shared(tile);
    const int blk0 = m.start[0];
    const int64_t n = s.n;
    const size_t np = s.np;
    const int nsp = pt.nsp;
    const f2_t magic2 = f2_pack(MAGIC, MAGIC);
    const f2_t two21 = f2_pack(TWO21, TWO21);
    for (int w = warp; w < (nown + 31) >> 5; w += nwarps)
        if ((threadIdx.x & 31) == 0) qmask[w] = 0u;
    __syncwarp();
    for (int ui = threadIdx.x; ui < nown; ui += blockDim.x) {
        const int gi = blk0 + ui;
        const float4 pi = tile[ui];
        const int si = __float_as_int(pi.w);
        const int nch = (s.nl_cnt[gi] + 7) >> 3;
        const uint4* lp = reinterpret_cast<const uint4*>(s.nl) + gi;
        if (MODE == FM_KKD) {
            // the velocity Verlet update's state into L2 while the pairs run (an L2 prefetch
            // holds no register: 0.3012 -> 0.2991 ms per fused step at 2,048,000 atoms)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s.vx + gi));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s.vy + gi));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s.vz + gi));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s.x + gi));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s.y + gi));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s.z + gi));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s.xr_ref + gi));
        }
        FixAcc ax{0u, 0u}, ay{0u, 0u}, az{0u, 0u};
        float pe = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;
        // the 32-bit split sums are exact up to FIX_SPLIT_MAX_TERMS terms; a longer list
        // (only at densities several times a liquid's) goes to the exact finish
        bool bad = nch * 8 > FIX_SPLIT_MAX_TERMS;
        // one species: the band and large-force tests as two running minima, checked once
        float mdist = 3.0e38f, mr2 = 3.0e38f;
        for_each_neighbour_pair(lp, np, nch, [&](int u0, int u1) {
            const float4 pa = lds_tile(tile_s, u0);
            const float4 pb = lds_tile(tile_s, u1);
            // scalar differences land directly in the register pairs of the packed operands
            const f2_t dx = f2_pack(__fsub_rn(pi.x, pa.x), __fsub_rn(pi.x, pb.x));
            const f2_t dy = f2_pack(__fsub_rn(pi.y, pa.y), __fsub_rn(pi.y, pb.y));
            const f2_t dz = f2_pack(__fsub_rn(pi.z, pa.z), __fsub_rn(pi.z, pb.z));
            const f2_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
            float r2a, r2b;
            f2_unpack(r2, r2a, r2b);
            const f2_t inv = f2_pack(rcp_approx(r2a), rcp_approx(r2b));
            float fa, fb;
            f2_t s6;  // (sigma^2 / r^2)^3, for the energy
            bool ina, inb;
            if (SINGLE) {
                // fs2 = inv^4 (a inv^3 - b): the constants are kernel parameters
                const f2_t inv2 = f2_mul(inv, inv);
                const f2_t inv3 = f2_mul(inv2, inv);
                const f2_t t = f2_fma(f2_pack(pt.lj_a_f, pt.lj_a_f), inv3, f2_pack(-pt.lj_b_f, -pt.lj_b_f));
                f2_unpack(f2_mul(t, f2_mul(inv2, inv2)), fa, fb);
                if (EV) s6 = f2_mul(f2_pack(pt.sig6_f, pt.sig6_f), inv3);
                // inside for certain below the band, tentatively inside up to its top: a pair
                // in the band leaves the atom to finish_atom_warp (FP64 cutoff decision)
                ina = r2a < pt.rc2hi_f[0];
                inb = r2b < pt.rc2hi_f[0];
                float dca, dcb;
                f2_unpack(f2_sub(r2, f2_pack(pt.rc2_f[0], pt.rc2_f[0])), dca, dcb);  // exact near r_cut
                mdist = fminf(mdist, fminf(fabsf(dca), fabsf(dcb)));
                mr2 = fminf(mr2, fminf(r2a, r2b));
            } else {
                const int ta = si * nsp + __float_as_int(pa.w);
                const int tb = si * nsp + __float_as_int(pb.w);
                const f2_t s2 = f2_mul(f2_pack(stab.sig2[ta], stab.sig2[tb]), inv);
                s6 = f2_mul(f2_mul(s2, s2), s2);
                f2_unpack(f2_mul(f2_mul(f2_fma(f2_pack(stab.c48[ta], stab.c48[tb]), s6,
                                               f2_pack(-stab.c24[ta], -stab.c24[tb])),
                                        s6),
                                 inv),
                          fa, fb);
                ina = r2a < stab.rc2hi[ta];
                inb = r2b < stab.rc2hi[tb];
                bad |= !(fabsf(fa) < fs2_max) | !(fabsf(fb) < fs2_max) | (ina != (r2a < stab.rc2lo[ta])) |
                       (inb != (r2b < stab.rc2lo[tb]));
            }
            fa = ina ? fa : 0.0f;
            fb = inb ? fb : 0.0f;
            const f2_t fs2 = f2_pack(fa, fb);
            fix_add2(ax, fs2, dx, magic2, two21);
            fix_add2(ay, fs2, dy, magic2, two21);
            fix_add2(az, fs2, dz, magic2, two21);
            if (EV) {
                float s6a, s6b, dxa, dxb, dya, dyb, dza, dzb;
                f2_unpack(s6, s6a, s6b);
                f2_unpack(dx, dxa, dxb);
                f2_unpack(dy, dya, dyb);
                f2_unpack(dz, dza, dzb);
                const int ta = SINGLE ? 0 : si * nsp + __float_as_int(pa.w);
                const int tb = SINGLE ? 0 : si * nsp + __float_as_int(pb.w);
                const float c4a = SINGLE ? pt.c4_f[0] : stab.c4[ta], c4b = SINGLE ? pt.c4_f[0] : stab.c4[tb];
                const float ua = ina ? c4a * s6a * (s6a - 1.0f) : 0.0f;
                const float ub = inb ? c4b * s6b * (s6b - 1.0f) : 0.0f;
                const float ga = fa * (1.0f / FS_SCALE), gb = fb * (1.0f / FS_SCALE);
                pe += ua + ub;
                w0 += dxa * (ga * dxa) + dxb * (gb * dxb);
                w1 += dya * (ga * dya) + dyb * (gb * dyb);
                w2 += dza * (ga * dza) + dzb * (gb * dzb);
                w3 += dxa * (ga * dya) + dxb * (gb * dyb);
                w4 += dxa * (ga * dza) + dxb * (gb * dzb);
                w5 += dya * (ga * dza) + dyb * (gb * dzb);
            }
        });
        // a pair in the band (|r^2 - r_cut^2| up to its half width) or close enough for a
        // term beyond the split sends the atom to the exact finish; NaN distances give no
        // force on either path
        if (SINGLE) bad |= (mdist <= pt.band_half_f) | (mr2 < pt.r2_wide_f);
        if (bad) {  // finished after the loop by finish_atom_warp, epilogue included
            atomicOr(&qmask[ui >> 5], 1u << (ui & 31));
            continue;
        }
        const int nterms = nch * 8;
        const long long qx = fix_final(ax, nterms), qy = fix_final(ay, nterms), qz = fix_final(az, nterms);
        full_epilogue<SINGLE, MODE>(s, pt, gi, si, qx, qy, qz, out, dt, lim2_f);
        if (EV) {
            // full lists see every pair twice: each atom keeps half of each pair energy / virial
            s.pe_atom_f[gi] = 0.5f * pe;
            s.vir_atom_f[gi] = 0.5f * w0;
            s.vir_atom_f[n + gi] = 0.5f * w1;
            s.vir_atom_f[2 * n + gi] = 0.5f * w2;
            s.vir_atom_f[3 * n + gi] = 0.5f * w3;
            s.vir_atom_f[4 * n + gi] = 0.5f * w4;
            s.vir_atom_f[5 * n + gi] = 0.5f * w5;
        }
    }
    // the warp's queued atoms, as soon as its own loop is done (the tile stays unchanged
    // until the CTA ends)
    __syncwarp();
    for (int w = warp; w < (nown + 31) >> 5; w += nwarps) {
        unsigned bits = qmask[w];
        while (bits) {
            const int ui = (w << 5) + __ffs(bits) - 1;
            bits &= bits - 1u;
            finish_atom_warp<SINGLE, EV, MODE>(s, g, pt, tile, stab, m, ui, fs2_max, out, dt, lim2_f, wwide[warp]);
        }
    }
}

template <bool SINGLE, bool EV, int MODE>
__global__ void __maxnreg__(SINGLE ? MDGB_FULL_MAX_REGS : MDGB_FULL_MAX_REGS_SPECIES) k_force_mixed_full(DevState s, Geometry g, PairTable pt,
                                                                TileOffsets to, int tile_cap, float fs2_max,
                                                                StepOut out, double dt,
                                                                float lim2_f) {
    full_block<SINGLE, EV, MODE>(s, g, pt, to, tile_cap, fs2_max, out, dt, lim2_f, spatial_block(g, blockIdx.x));
}

// The same over the occupied blocks of a compact system: a grid of s.compact CTAs, each
// taking every gridDim-th entry of the list.  (A separate kernel: the loop in the
// one-block kernel cost the dense case 10 % through its register allocation.)
template <bool SINGLE, bool EV, int MODE>
__global__ void __maxnreg__(SINGLE ? MDGB_FULL_MAX_REGS : MDGB_FULL_MAX_REGS_SPECIES) k_force_mixed_occ(DevState s, Geometry g, PairTable pt,
                                                                TileOffsets to, int tile_cap, float fs2_max,
                                                                StepOut out, double dt,
                                                                float lim2_f) {
    const int count = s.stats[4];
    for (int k = blockIdx.x; k < count; k += gridDim.x) {
        full_block<SINGLE, EV, MODE>(s, g, pt, to, tile_cap, fs2_max, out, dt, lim2_f, s.blk_list[k]);
        __syncthreads();  // the next block reuses the shared memory
    }
}

// ---------------------------------------------------------------- mixed, half list, one colour
// Shared memory: tile coordinates, then the tile's fixed-point accumulators
// (hi and lo parts per component, 32-bit) and their term counts.  Pair energies
// and virials are booked in full on the listing atom (only totals are reported).
template <bool SINGLE, bool EV>
__global__ void __launch_bounds__(F_THREADS) k_force_mixed_half(DevState s, Geometry g, PairTable pt,
                                                                TileOffsets to, int tile_cap, float fs2_max,
                                                                int block0) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileMeta m;
    // terms beyond the two-part split (atoms closer than about 0.75 sigma) do not go
    // through the 32-bit tile sums: they wait here as exact 64-bit values
    constexpr int WQ = 64;
    __shared__ long long wq[WQ][3];
    __shared__ int wq_u[WQ];
    __shared__ int nwq;
    // Reaction sums only for the tile entries a half list reaches (the own cells and their
    // forward neighbours come first in the tile, Sec. II.D.3): 6 x rcap, hx, lx, hy, ly, hz,
    // lz, with the split's offset taken off each term; then, where a block needs them,
    // each entry's term count in 16 bits, two to a word (fewer than the tile's atoms, < 2^15).
    const int rcap = half_recv_cap(tile_cap);
    float4* tile = reinterpret_cast<float4*>(smem);
    unsigned* acc = reinterpret_cast<unsigned*>(tile + tile_cap);
    unsigned* cnt2 = acc + 6 * rcap;
    __shared__ int max_nch;  // the longest own list, in chunks
    const int b = block0 + blockIdx.x;
    if (threadIdx.x == 0) {
        nwq = 0;
        max_nch = 0;
    }
    tile_meta(g, s.cell_start, b, m);
    const int T = m.prefix[64];
    const int recv = m.prefix[TILE_RECV_CELLS];
    if (T + 1 > tile_cap || recv > rcap) {
        if (threadIdx.x == 0) atomicOr(s.err, ERR_TILE_OVERFLOW);
        return;
    }
    for (int ui = threadIdx.x; ui < m.prefix[8]; ui += blockDim.x)
        atomicMax(&max_nch, (s.nl_cnt[m.start[0] + ui] + 7) >> 3);
    tile_stage_f32_cells(m, s.xr, to, tile);
    stage_dummy_f32(tile, T);
    for (int u = threadIdx.x; u < recv; u += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c * rcap + u] = 0u;
        if ((u & 1) == 0) cnt2[u >> 1] = 0u;
    }
    __syncthreads();
    const unsigned magic_bits = __float_as_uint(MAGIC);
    const int blk0 = m.start[0];
    const int nown = m.prefix[8];
    const int64_t n = s.n;
    const int np = s.np;
    // Each term's high part is below 2^22 in magnitude, so a 32-bit sum stays exact up to
    // FIX_SPLIT_MAX_TERMS terms.  An entry takes at most its own list's terms (own atoms)
    // and one reaction per own atom, so the counts are only kept for blocks where that
    // bound exceeds the limit (small boxes with whole-box tiles, high densities)
    const bool count = nown + 8 * max_nch > FIX_SPLIT_MAX_TERMS;
    for (int ui = threadIdx.x; ui < nown; ui += blockDim.x) {
        const int gi = blk0 + ui;
        const float4 pi = tile[ui];
        const int si = __float_as_int(pi.w);
        const int nch = (s.nl_cnt[gi] + 7) >> 3;
        FixAcc ax{0u, 0u}, ay{0u, 0u}, az{0u, 0u};
        float pe = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f, w4 = 0.f, w5 = 0.f;
        MDGB_FOR_EACH_NEIGHBOUR(reinterpret_cast<const uint4*>(s.nl) + gi, np, nch, {
            const float4 pj = tile[u];
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const int t = SINGLE ? 0 : si * pt.nsp + __float_as_int(pj.w);
            float s6;
            bool inside;
            const float fs = lj_fs_unmasked<SINGLE>(pt, t, r2, s6, inside);
            if (r2 < pt.rc2hi_f[t] && !(r2 < pt.rc2lo_f[t]))  // rare: decide the cutoff in FP64
                inside = fp64_pair_test(s.x, s.y, s.z, g.L[0], g.L[1], g.L[2], gi, tile_global_index(m, u),
                                        SINGLE ? pt.rc2_d[0] : pt.rc2_d[t]);
            const float fs2 = inside ? fs : 0.0f;
            FixAcc bx{0u, 0u}, by{0u, 0u}, bz{0u, 0u};
            if (fabsf(fs2) < fs2_max) {
                fix_add(ax, fs2, dx);
                fix_add(ay, fs2, dy);
                fix_add(az, fs2, dz);
                fix_sub(bx, fs2, dx);
                fix_sub(by, fs2, dy);
                fix_sub(bz, fs2, dz);
            } else {  // rare: both atoms' terms into the queue (its count bounds the 64-bit sums)
                const long long qx = fix_term_wide(fs2, dx, s.err), qy = fix_term_wide(fs2, dy, s.err),
                                qz = fix_term_wide(fs2, dz, s.err);
                // the split sums count this pair as a zero term (offset bits only)
                fix_add(ax, 0.0f, 0.0f);
                fix_add(ay, 0.0f, 0.0f);
                fix_add(az, 0.0f, 0.0f);
                fix_add(bx, 0.0f, 0.0f);
                fix_add(by, 0.0f, 0.0f);
                fix_add(bz, 0.0f, 0.0f);
                const int k = atomicAdd(&nwq, 2);
                if (k + 1 < WQ && k + 2 <= FIX_WIDE_MAX_TERMS) {
                    wq_u[k] = ui;
                    wq[k][0] = qx;
                    wq[k][1] = qy;
                    wq[k][2] = qz;
                    wq_u[k + 1] = u;
                    wq[k + 1][0] = -qx;
                    wq[k + 1][1] = -qy;
                    wq[k + 1][2] = -qz;
                } else {
                    atomicOr(s.err, ERR_NONFINITE);
                }
            }
            if (u < recv) {  // else the padding's dummy slot: a zero term
                atomicAdd(&acc[0 * rcap + u], bx.hi - magic_bits);
                atomicAdd(&acc[1 * rcap + u], bx.lo - magic_bits);
                atomicAdd(&acc[2 * rcap + u], by.hi - magic_bits);
                atomicAdd(&acc[3 * rcap + u], by.lo - magic_bits);
                atomicAdd(&acc[4 * rcap + u], bz.hi - magic_bits);
                atomicAdd(&acc[5 * rcap + u], bz.lo - magic_bits);
                if (count) atomicAdd(&cnt2[u >> 1], 1u << ((u & 1) << 4));
            }
            if (EV) {
                const float c4 = SINGLE ? pt.c4_f[0] : pt.c4_f[t];
                const float fs = fs2 * (1.0f / FS_SCALE);
                pe += inside ? c4 * s6 * (s6 - 1.0f) : 0.0f;
                w0 = fmaf(dx, fs * dx, w0);
                w1 = fmaf(dy, fs * dy, w1);
                w2 = fmaf(dz, fs * dz, w2);
                w3 = fmaf(dx, fs * dy, w3);
                w4 = fmaf(dx, fs * dz, w4);
                w5 = fmaf(dy, fs * dz, w5);
            }
        })
        // own atom's part goes through the same tile accumulator, its nch * 8 offsets removed
        const unsigned bias = (unsigned)(nch * 8) * magic_bits;
        atomicAdd(&acc[0 * rcap + ui], ax.hi - bias);
        atomicAdd(&acc[1 * rcap + ui], ax.lo - bias);
        atomicAdd(&acc[2 * rcap + ui], ay.hi - bias);
        atomicAdd(&acc[3 * rcap + ui], ay.lo - bias);
        atomicAdd(&acc[4 * rcap + ui], az.hi - bias);
        atomicAdd(&acc[5 * rcap + ui], az.lo - bias);
        if (count) atomicAdd(&cnt2[ui >> 1], (unsigned)(nch * 8) << ((ui & 1) << 4));
        if (EV) {
            s.pe_atom_f[gi] = pe;
            s.vir_atom_f[gi] = w0;
            s.vir_atom_f[n + gi] = w1;
            s.vir_atom_f[2 * n + gi] = w2;
            s.vir_atom_f[3 * n + gi] = w3;
            s.vir_atom_f[4 * n + gi] = w4;
            s.vir_atom_f[5 * n + gi] = w5;
        }
    }
    __syncthreads();
    // add the tile back: this CTA is the only one of its colour touching these atoms
    for (int u = threadIdx.x; u < recv; u += blockDim.x) {
        if (count) {
            const unsigned nt = (cnt2[u >> 1] >> ((u & 1) << 4)) & 0xffffu;
            if (nt == 0) continue;
            // more than FIX_SPLIT_MAX_TERMS terms on one atom could wrap its 32-bit sums
            if (nt > FIX_SPLIT_MAX_TERMS) atomicOr(s.err, ERR_NONFINITE);
        }
        const int slot = tile_slot_of(m, u);
        const int gj = m.start[slot] + (u - m.prefix[slot]);
        FixAcc fx{acc[0 * rcap + u], acc[1 * rcap + u]};
        FixAcc fy{acc[2 * rcap + u], acc[3 * rcap + u]};
        FixAcc fz{acc[4 * rcap + u], acc[5 * rcap + u]};
        s.fq[gj] += fix_final(fx, 0);
        s.fq[n + gj] += fix_final(fy, 0);
        s.fq[2 * n + gj] += fix_final(fz, 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // the queued large terms, exact in 64 bits
        const int nq = nwq < WQ ? nwq : WQ;
        for (int k = 0; k < nq; ++k) {
            const int u = wq_u[k];
            const int slot = tile_slot_of(m, u);
            const int gj = m.start[slot] + (u - m.prefix[slot]);
            s.fq[gj] += wq[k][0];
            s.fq[n + gj] += wq[k][1];
            s.fq[2 * n + gj] += wq[k][2];
        }
    }
}

size_t force_smem_bytes(int mixed, int half, int with_energy, int tile_cap) {
    (void)with_energy;
    if (mixed) {
        size_t b = (size_t)tile_cap * sizeof(float4);
        if (half) {  // reaction sums and 16-bit term counts of the entries a half list reaches
            const size_t r = (size_t)half_recv_cap(tile_cap);
            b += r * 6 * sizeof(unsigned) + (((r + 1) / 2 * sizeof(unsigned) + 15) & ~(size_t)15);
        }
        else b += ((size_t)(tile_cap + 31) / 32 * sizeof(unsigned) + 15) & ~(size_t)15;  // own atoms to finish
        return b;
    }
    size_t b = (size_t)tile_cap * (3 * sizeof(double) + sizeof(int));
    if (half) b += (size_t)tile_cap * 3 * sizeof(double);
    return b;
}

// Raise every force kernel's dynamic shared-memory limit to what the SM allows
// (once per device, before any launch or stream capture).
template <typename K>
static void allow_max_smem(K kernel) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

void init_force_kernels() {
    allow_max_smem(k_force_mixed_full<true, false, FM_FORCE>);
    allow_max_smem(k_force_mixed_full<true, true, FM_FORCE>);
    allow_max_smem(k_force_mixed_full<false, false, FM_FORCE>);
    allow_max_smem(k_force_mixed_full<false, true, FM_FORCE>);
    allow_max_smem(k_force_mixed_full<true, false, FM_KICK>);
    allow_max_smem(k_force_mixed_full<false, false, FM_KICK>);
    allow_max_smem(k_force_mixed_full<true, false, FM_KKD>);
    allow_max_smem(k_force_mixed_full<false, false, FM_KKD>);
    allow_max_smem(k_force_mixed_occ<true, false, FM_FORCE>);
    allow_max_smem(k_force_mixed_occ<true, true, FM_FORCE>);
    allow_max_smem(k_force_mixed_occ<false, false, FM_FORCE>);
    allow_max_smem(k_force_mixed_occ<false, true, FM_FORCE>);
    allow_max_smem(k_force_mixed_occ<true, false, FM_KICK>);
    allow_max_smem(k_force_mixed_occ<false, false, FM_KICK>);
    allow_max_smem(k_force_mixed_occ<true, false, FM_KKD>);
    allow_max_smem(k_force_mixed_occ<false, false, FM_KKD>);
    allow_max_smem(k_force_mixed_half<true, false>);
    allow_max_smem(k_force_mixed_half<true, true>);
    allow_max_smem(k_force_mixed_half<false, false>);
    allow_max_smem(k_force_mixed_half<false, true>);
    init_force_fp64_kernels();
}

// |fs2 * d| < 2^22 (the exact range of the two-part split) is guaranteed when |fs2| < 2^22 / r_cut
float fs2_max_of(const PairTable& pt) {
    float rcmax2 = 0.f;
    for (int t = 0; t < pt.nsp * pt.nsp; ++t) rcmax2 = pt.rc2_f[t] > rcmax2 ? pt.rc2_f[t] : rcmax2;
    return 4194304.0f / sqrtf(rcmax2) * 0.999f;
}

// One full-list launch: a CTA per block, or with a compact system a grid of s.compact CTAs
// over the occupied blocks.
template <bool SINGLE, bool EV, int MODE>
static void launch_full(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                        int tile_cap, float fs2_max, StepOut out, double dt, float lim2_f, size_t smem,
                        cudaStream_t st) {
    if (s.compact)
        k_force_mixed_occ<SINGLE, EV, MODE><<<s.compact, FULL_THREADS, smem, st>>>(s, g, pt, to, tile_cap, fs2_max,
                                                                                 out, dt, lim2_f);
    else
        k_force_mixed_full<SINGLE, EV, MODE><<<g.nblock, FULL_THREADS, smem, st>>>(s, g, pt, to, tile_cap, fs2_max,
                                                                                 out, dt, lim2_f);
}

void launch_forces_mixed(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                         int tile_cap, int half, int with_energy, cudaStream_t st) {
    if (s.n == 0) return;
    const size_t smem = force_smem_bytes(1, half, with_energy, tile_cap);
    const float fs2_max = fs2_max_of(pt);
    const bool single = pt.nsp == 1;
    if (!half) {
        if (single && !with_energy)
            launch_full<true, false, FM_FORCE>(s, g, pt, to, tile_cap, fs2_max, StepOut{}, 0.0, 0.f, smem, st);
        else if (single)
            launch_full<true, true, FM_FORCE>(s, g, pt, to, tile_cap, fs2_max, StepOut{}, 0.0, 0.f, smem, st);
        else if (!with_energy)
            launch_full<false, false, FM_FORCE>(s, g, pt, to, tile_cap, fs2_max, StepOut{}, 0.0, 0.f, smem, st);
        else
            launch_full<false, true, FM_FORCE>(s, g, pt, to, tile_cap, fs2_max, StepOut{}, 0.0, 0.f, smem, st);
        return;
    }
    cudaMemsetAsync(s.fq, 0, sizeof(long long) * 3 * (size_t)s.n, st);
    const int per = g.nblock / 8;
    for (int col = 0; col < 8; ++col) {
        const int b0 = col * per;
        if (single && !with_energy)
            k_force_mixed_half<true, false><<<per, F_THREADS, smem, st>>>(s, g, pt, to, tile_cap, fs2_max, b0);
        else if (single)
            k_force_mixed_half<true, true><<<per, F_THREADS, smem, st>>>(s, g, pt, to, tile_cap, fs2_max, b0);
        else if (!with_energy)
            k_force_mixed_half<false, false><<<per, F_THREADS, smem, st>>>(s, g, pt, to, tile_cap, fs2_max, b0);
        else
            k_force_mixed_half<false, true><<<per, F_THREADS, smem, st>>>(s, g, pt, to, tile_cap, fs2_max, b0);
    }
}

// Full-list mixed forces fused with velocity Verlet (mode FM_KICK: closing half kick;
// FM_KKD: closing + opening kick and drift, the new positions into out).
template <bool SINGLE, int MODE>
static void launch_full_mode(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                             int tile_cap, float fs2_max, StepOut out, double dt, float lim2_f, size_t smem,
                             cudaStream_t st) {
    launch_full<SINGLE, false, MODE>(s, g, pt, to, tile_cap, fs2_max, out, dt, lim2_f, smem, st);
}

void launch_forces_mixed_fused(const DevState& s, const Geometry& g, const PairTable& pt, const TileOffsets& to,
                               int tile_cap, int mode, StepOut out, double dt, double lim2, cudaStream_t st) {
    if (s.n == 0) return;
    const size_t smem = force_smem_bytes(1, 0, 0, tile_cap);
    const float fs2_max = fs2_max_of(pt);
    // the FP32 displacement test is slightly stricter than skin/2 (as in k_integrate)
    const float lim2_f = (float)(lim2 * (1.0 - 1e-4));
    const bool single = pt.nsp == 1;
    if (mode == FM_KICK) {
        if (single)
            launch_full_mode<true, FM_KICK>(s, g, pt, to, tile_cap, fs2_max, out, dt, lim2_f, smem, st);
        else
            launch_full_mode<false, FM_KICK>(s, g, pt, to, tile_cap, fs2_max, out, dt, lim2_f, smem, st);
    } else {
        if (single)
            launch_full_mode<true, FM_KKD>(s, g, pt, to, tile_cap, fs2_max, out, dt, lim2_f, smem, st);
        else
            launch_full_mode<false, FM_KKD>(s, g, pt, to, tile_cap, fs2_max, out, dt, lim2_f, smem, st);
    }
}

}  // namespace mdgb
