// k_batch.cu - ensembles of independent systems in one persistent launch.
//
// The paper notes that its task functor can carry which copy of a system a task
// works on, so that replicas share one schedule (Sec. II.C).  Here every call on an
// ensemble is one launch of k_ensemble_run (at the end of this file), whose CTAs take
// tasks from a device work table over all systems.  Two kinds of system:
//
// A small system (a few hundred to a few thousand atoms) is one task: one CTA owns it
// for all time steps of the call; its FP32 coordinates and linked cells live in shared
// memory and no other CTA touches it.  Per step the CTA
//   * re-bins its atoms into cells at least r_cut / R wide (counting sort in shared
//     memory; atoms of a cell kept in index order),
//   * evaluates the cutoff LJ force on every atom over the (2R+1)^3 surrounding cells:
//     two candidates per step in packed FP32x2 arithmetic on cell-relative coordinates
//     (structure-of-arrays copies in shared memory, so one 64-bit load brings a pair),
//     with no branches, every pair force component added as rint(f * 2^32) through
//     the main path's exact two-part integer split (forces do not depend on order);
//     an atom with a pair in the FP64 cutoff band or a force beyond the split's range
//     is finished after the loop by an exact scalar pass,
//   * and integrates velocity Verlet in FP64.
// There is no neighbour list: the cells are rebuilt every step, which for systems of
// this size costs less than a list build would.
//
// A larger system is advanced in phases of tasks that any CTA may take, with Verlet
// lists (the block systems below).
#include "mdgb_batch_internal.cuh"
#include "nl_scan.cuh"

namespace mdgb {

namespace {

// block-wide exclusive scan of cnt[0..m) into start[0..m], start[m] = total (CG: counts
// written by other CTAs of the launch, read from L2)
template <bool CG = false>
__device__ void block_scan(const int* __restrict__ cnt, int* __restrict__ start, int m, int* warp_tot) {
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5, nw = nt >> 5;
    const int per = (m + nt - 1) / nt;
    const int lo = t * per, hi = min(lo + per, m);
    int s = 0;
    for (int k = lo; k < hi; ++k) s += CG ? __ldcg(cnt + k) : cnt[k];
    int v = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    int run = (warp > 0 ? warp_tot[warp - 1] : 0) + v - s;
    for (int k = lo; k < hi; ++k) {
        start[k] = run;
        run += CG ? __ldcg(cnt + k) : cnt[k];
    }
    if (t == nt - 1) start[m] = run;
    __syncthreads();
}

struct Smem {
    float *px, *py, *pz;  // n + 2: FP32 coordinates relative to the cell centre, by slot (slot n: far away)
    uint16_t* perm;       // n: slot -> local atom
    uint16_t* cell;       // n: local atom -> cell, then local atom -> slot
    uint16_t* scell;      // n + 2: slot -> cell
    uint16_t* queue;      // n: slots left to the exact pass
    int* nqueued;
    int* cstart;          // ncell + 1
    int* ccount;          // ncell
    int* warp_tot;        // 32
};

// Wrap every atom into the box (one box length at most, counted in the image
// counters), find its cell, and sort the atoms into cells, within a cell in index
// order; write the slot-ordered FP32 coordinates.
__device__ void batch_bin(const BatchSys& y, BatchState st, Smem& sm) {
    const int n = y.n, m = y.ncell;
    for (int k = threadIdx.x; k < m; k += blockDim.x) sm.ccount[k] = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        const int64_t g = y.a0 + a;
        double* X[3] = {st.x, st.y, st.z};
        int32_t* I[3] = {st.ix, st.iy, st.iz};
        int c[3];
        uint32_t bad = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double x = X[d][g];
            if (x >= y.L[d]) {
                x = __dsub_rn(x, y.L[d]);
                I[d][g] += 1;
                X[d][g] = x;
            } else if (x < 0.0) {
                x = __dadd_rn(x, y.L[d]);
                I[d][g] -= 1;
                X[d][g] = x;
            }
            if (!(x >= 0.0 && x <= y.L[d])) bad |= isfinite(x) ? ERR_ESCAPE : ERR_NONFINITE;
            const int cc = (int)(x * y.inv_w[d]);
            c[d] = cc < 0 ? 0 : (cc >= y.nc[d] ? y.nc[d] - 1 : cc);
        }
        if (bad) atomicOr(st.err, bad);
        const int id = c[0] + y.nc[0] * (c[1] + y.nc[1] * c[2]);
        sm.cell[a] = (uint16_t)id;
        atomicAdd(&sm.ccount[id], 1);
    }
    __syncthreads();
    block_scan(sm.ccount, sm.cstart, m, sm.warp_tot);
    for (int k = threadIdx.x; k < m; k += blockDim.x) sm.ccount[k] = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        const int id = sm.cell[a];
        sm.perm[sm.cstart[id] + atomicAdd(&sm.ccount[id], 1)] = (uint16_t)a;  // any order within the cell
    }
    __syncthreads();
    // rank within the cell by atom index (one warp per cell; perm only read here):
    // the coordinates go straight to the ranked slot, and cell[] becomes atom -> slot
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int id = warp; id < m; id += nw) {
        const int s0 = sm.cstart[id], cnt = sm.cstart[id + 1] - s0;
        const int cx = id % y.nc[0], cy = (id / y.nc[0]) % y.nc[1], cz = id / (y.nc[0] * y.nc[1]);
        const double ox = (cx + 0.5) * y.w[0], oy = (cy + 0.5) * y.w[1], oz = (cz + 0.5) * y.w[2];
        for (int e = lane; e < cnt; e += 32) {
            const int mine = sm.perm[s0 + e];
            int rank = 0;
            for (int f = 0; f < cnt; ++f) rank += (int)sm.perm[s0 + f] < mine;
            const int64_t g = y.a0 + mine;
            sm.px[s0 + rank] = __double2float_rn(st.x[g] - ox);
            sm.py[s0 + rank] = __double2float_rn(st.y[g] - oy);
            sm.pz[s0 + rank] = __double2float_rn(st.z[g] - oz);
            sm.scell[s0 + rank] = (uint16_t)id;
            sm.cell[mine] = (uint16_t)(s0 + rank);
        }
    }
    if (threadIdx.x == 0) {  // slot n: read as the second of a pair at the last cell's end
        sm.px[n] = sm.py[n] = sm.pz[n] = 1.0e4f;
        sm.scell[n] = 0;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < n; a += blockDim.x) sm.perm[sm.cell[a]] = (uint16_t)a;
    __syncthreads();
}

// Cell coordinates of slot p's cell.
__device__ __forceinline__ void slot_cell(const BatchSys& y, const Smem& sm, int p, int& cx, int& cy, int& cz) {
    const int id = sm.scell[p];
    cx = id % y.nc[0];
    cy = (id / y.nc[0]) % y.nc[1];
    cz = id / (y.nc[0] * y.nc[1]);
}

__device__ __forceinline__ int wrap_cell(int c, int nc) { return c < 0 ? c + nc : (c >= nc ? c - nc : c); }

// Exact force on the atom of slot p, one candidate at a time: a pair whose FP32 r^2 lies in
// the band around r_cut^2 is decided in FP64 by the definition, a large term is rounded in
// FP64 (fix_term_wide); every other term is the one the packed loop would add.
template <bool ENERGY>
__device__ __noinline__ void batch_force_exact(const BatchSys& y, const BatchState& st, const PairTable& pt,
                                               float fs2_max, const Smem& sm, float* __restrict__ pe_out, int p) {
    const int R = y.R;
    const float sig2 = pt.sig2_f[0], c48 = pt.c48_f[0], c24 = pt.c24_f[0], c4 = pt.c4_f[0];
    const int a = sm.perm[p];
    const int64_t g = y.a0 + a;
    int cx, cy, cz;
    slot_cell(y, sm, p, cx, cy, cz);
    const float xi = sm.px[p], yi = sm.py[p], zi = sm.pz[p];
    long long qx = 0, qy = 0, qz = 0;  // exact 64-bit sums
    int nwide = 0;
    float pe = 0.f;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                const int id = wrap_cell(cx + dx, y.nc[0]) +
                               y.nc[0] * (wrap_cell(cy + dy, y.nc[1]) + y.nc[1] * wrap_cell(cz + dz, y.nc[2]));
                const float sx = (float)dx * y.wf[0], sy = (float)dy * y.wf[1], sz = (float)dz * y.wf[2];
                const int q1 = sm.cstart[id + 1];
                for (int q = sm.cstart[id]; q < q1; ++q) {
                    if (q == p) continue;
                    const float ex = xi - (sm.px[q] + sx), ey = yi - (sm.py[q] + sy), ez = zi - (sm.pz[q] + sz);
                    const float r2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                    if (!(r2 < pt.rc2hi_f[0])) continue;
                    if (!(r2 < pt.rc2lo_f[0]) &&
                        !fp64_pair_test(st.x, st.y, st.z, y.L[0], y.L[1], y.L[2], g, y.a0 + sm.perm[q], pt.rc2_d[0]))
                        continue;
                    const float inv = rcp_approx(r2);
                    const float s2 = sig2 * inv;
                    const float s6 = s2 * s2 * s2;
                    const float fs2 = __fmul_rn(__fmul_rn(__fmaf_rn(c48, s6, -c24), s6), inv);  // (|f|/r) * 2^11
                    qx += fix_term_any(fs2, ex, fs2_max, st.err);
                    qy += fix_term_any(fs2, ey, fs2_max, st.err);
                    qz += fix_term_any(fs2, ez, fs2_max, st.err);
                    nwide += fabsf(fs2) < fs2_max ? 0 : 1;
                    if (ENERGY) pe += c4 * s6 * (s6 - 1.0f);
                }
            }
    fix_wide_count_ok(nwide, st.err);
    st.fq[g] = qx;
    st.fq[st.ntot + g] = qy;
    st.fq[2 * st.ntot + g] = qz;
    if (ENERGY) pe_out[a] = 0.5f * pe;
}

// Force on every atom (fixed point into st.fq); with energy, also its half pair energies
// (FP32 per atom, neighbours in slot order: deterministic).  Two candidates per step:
// the pair (q, q+1) with q even, masked to the cell's range and away from the atom itself.
template <bool ENERGY>
__device__ void batch_forces(const BatchSys& y, BatchState st, const PairTable& pt, float fs2_max, Smem& sm,
                             float* __restrict__ pe_out) {
    const int n = y.n, R = y.R;
    const f2_t magic2 = f2_pack(MAGIC, MAGIC), two21 = f2_pack(TWO21, TWO21);
    const f2_t sig2 = f2_pack(pt.sig2_f[0], pt.sig2_f[0]), c48 = f2_pack(pt.c48_f[0], pt.c48_f[0]);
    const f2_t nc24 = f2_pack(-pt.c24_f[0], -pt.c24_f[0]);
    const float rc2_lo = pt.rc2lo_f[0], rc2_hi = pt.rc2hi_f[0], c4 = pt.c4_f[0];
    const unsigned spx = (unsigned)__cvta_generic_to_shared(sm.px);
    const unsigned spy = (unsigned)__cvta_generic_to_shared(sm.py);
    const unsigned spz = (unsigned)__cvta_generic_to_shared(sm.pz);
    if (threadIdx.x == 0) *sm.nqueued = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        int cx, cy, cz;
        slot_cell(y, sm, p, cx, cy, cz);
        const float xi = sm.px[p], yi = sm.py[p], zi = sm.pz[p];
        const f2_t pix = f2_pack(xi, xi), piy = f2_pack(yi, yi), piz = f2_pack(zi, zi);
        FixAcc ax{0u, 0u}, ay{0u, 0u}, az{0u, 0u};
        int nterms = 0, nin = 0;  // nin: non-zero terms, which bound the 32-bit split sums
        float pe = 0.f;
        bool bad = false;
        for (int dz = -R; dz <= R; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    const int id = wrap_cell(cx + dx, y.nc[0]) +
                                   y.nc[0] * (wrap_cell(cy + dy, y.nc[1]) + y.nc[1] * wrap_cell(cz + dz, y.nc[2]));
                    const float sxf = (float)dx * y.wf[0], syf = (float)dy * y.wf[1], szf = (float)dz * y.wf[2];
                    const f2_t sx = f2_pack(sxf, sxf), sy = f2_pack(syf, syf), sz = f2_pack(szf, szf);
                    const int c0 = sm.cstart[id], c1 = sm.cstart[id + 1];
                    for (int q = c0 & ~1; q < c1; q += 2) {
                        f2_t X, Y, Z;
                        asm volatile("ld.shared.b64 %0, [%1];" : "=l"(X) : "r"(spx + 4u * (unsigned)q));
                        asm volatile("ld.shared.b64 %0, [%1];" : "=l"(Y) : "r"(spy + 4u * (unsigned)q));
                        asm volatile("ld.shared.b64 %0, [%1];" : "=l"(Z) : "r"(spz + 4u * (unsigned)q));
                        const f2_t ex = f2_sub(pix, f2_add(X, sx));
                        const f2_t ey = f2_sub(piy, f2_add(Y, sy));
                        const f2_t ez = f2_sub(piz, f2_add(Z, sz));
                        const f2_t r2 = f2_fma(ez, ez, f2_fma(ey, ey, f2_mul(ex, ex)));
                        float r2a, r2b;
                        f2_unpack(r2, r2a, r2b);
                        const bool ina = (q >= c0) & (q != p) & (r2a < rc2_hi);
                        const bool inb = (q + 1 < c1) & (q + 1 != p) & (r2b < rc2_hi);
                        const f2_t inv = f2_pack(rcp_approx(r2a), rcp_approx(r2b));
                        const f2_t s2 = f2_mul(sig2, inv);
                        const f2_t s6 = f2_mul(f2_mul(s2, s2), s2);
                        const f2_t fsv = f2_mul(f2_mul(f2_fma(c48, s6, nc24), s6), inv);
                        float fa, fb;
                        f2_unpack(fsv, fa, fb);
                        fa = ina ? fa : 0.0f;
                        fb = inb ? fb : 0.0f;
                        bad |= (ina & !(r2a < rc2_lo)) | (inb & !(r2b < rc2_lo)) | !(fabsf(fa) < fs2_max) |
                               !(fabsf(fb) < fs2_max);
                        const f2_t fs2 = f2_pack(fa, fb);
                        fix_add2(ax, fs2, ex, magic2, two21);
                        fix_add2(ay, fs2, ey, magic2, two21);
                        fix_add2(az, fs2, ez, magic2, two21);
                        nterms += 2;
                        nin += (int)ina + (int)inb;
                        if (ENERGY) {
                            float s6a, s6b;
                            f2_unpack(s6, s6a, s6b);
                            pe += (ina ? c4 * s6a * (s6a - 1.0f) : 0.0f) + (inb ? c4 * s6b * (s6b - 1.0f) : 0.0f);
                        }
                    }
                }
        bad |= nin > FIX_SPLIT_MAX_TERMS;  // the split sums could wrap: the exact 64-bit pass
        if (bad) {  // finished by batch_force_exact after the loop
            sm.queue[atomicAdd(sm.nqueued, 1)] = (uint16_t)p;
            continue;
        }
        const int a = sm.perm[p];
        const int64_t g = y.a0 + a;
        st.fq[g] = fix_final(ax, nterms);
        st.fq[st.ntot + g] = fix_final(ay, nterms);
        st.fq[2 * st.ntot + g] = fix_final(az, nterms);
        if (ENERGY) pe_out[a] = 0.5f * pe;
    }
    __syncthreads();
    const int nq = *sm.nqueued;
    for (int k = threadIdx.x; k < nq; k += blockDim.x)
        batch_force_exact<ENERGY>(y, st, pt, fs2_max, sm, pe_out, sm.queue[k]);
}

// v += k F (FP64, F in Q31.32); with drift also x += dt v
__device__ void batch_kick(const BatchSys& y, BatchState st, const PairTable& pt, double dt, bool drift) {
    const double hq = pt.hdtm_q[0];
    for (int a = threadIdx.x; a < y.n; a += blockDim.x) {
        const int64_t g = y.a0 + a;
        const double vx = fma(hq, (double)st.fq[g], st.vx[g]);
        const double vy = fma(hq, (double)st.fq[st.ntot + g], st.vy[g]);
        const double vz = fma(hq, (double)st.fq[2 * st.ntot + g], st.vz[g]);
        st.vx[g] = vx;
        st.vy[g] = vy;
        st.vz[g] = vz;
        if (drift) {
            st.x[g] = fma(dt, vx, st.x[g]);
            st.y[g] = fma(dt, vy, st.y[g]);
            st.z[g] = fma(dt, vz, st.z[g]);
        }
    }
}

// Fixed-order block sum of per-thread FP64 values
__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = 1; w < (int)blockDim.x; w <<= 1) {
        const int t = threadIdx.x;
        if ((t & (2 * w - 1)) == 0 && t + w < (int)blockDim.x) sh[t] += sh[t + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

}  // namespace


// ---------------------------------------------------------------- one-CTA systems
namespace {

// The whole call for a system held by one CTA: flags BATCH_HAVE_FORCES (st.fq holds F at
// the current positions), BATCH_ENERGY (potential and kinetic energy at the end).
__device__ void run_one_system(const BatchSys& y, const BatchState& st, const PairTable& pt, int n_steps, int flags,
                               double dt, float fs2_max, int nmax, int cmax, float* __restrict__ pe_atom,
                               double* __restrict__ pe_out, double* __restrict__ ke_out, unsigned char* smem,
                               int* warp_tot, int* nqueued, double* red) {
    if (y.n == 0) return;
    if (y.n > nmax || y.ncell > cmax) {  // the host sizes the launch for its systems
        if (threadIdx.x == 0) atomicOr(st.err, ERR_TILE_OVERFLOW);
        return;
    }
    Smem sm;
    const int np2 = nmax + 2;  // even: the three coordinate arrays stay 8-byte aligned
    sm.px = reinterpret_cast<float*>(smem);
    sm.py = sm.px + np2;
    sm.pz = sm.py + np2;
    sm.perm = reinterpret_cast<uint16_t*>(sm.pz + np2);
    sm.cell = sm.perm + nmax;
    sm.scell = sm.cell + nmax;
    sm.queue = sm.scell + np2;
    sm.nqueued = nqueued;
    sm.cstart = reinterpret_cast<int*>(smem + batch_smem_ints_offset(nmax));
    sm.ccount = sm.cstart + cmax + 1;
    sm.warp_tot = warp_tot;
    if (!(flags & BATCH_HAVE_FORCES) || n_steps == 0) {
        batch_bin(y, st, sm);
        batch_forces<false>(y, st, pt, fs2_max, sm, nullptr);
        __syncthreads();
    }
    for (int step = 0; step < n_steps; ++step) {
        batch_kick(y, st, pt, dt, true);  // opening half kick and drift
        __syncthreads();
        batch_bin(y, st, sm);
        batch_forces<false>(y, st, pt, fs2_max, sm, nullptr);
        __syncthreads();
        batch_kick(y, st, pt, dt, false);  // closing half kick
        __syncthreads();
    }
    if (flags & BATCH_ENERGY) {
        batch_bin(y, st, sm);
        batch_forces<true>(y, st, pt, fs2_max, sm, pe_atom + y.a0);
        __syncthreads();
        double pe = 0.0, ke = 0.0;
        const double m = pt.mass[0];
        for (int a = threadIdx.x; a < y.n; a += blockDim.x) {
            const int64_t g = y.a0 + a;
            pe += (double)pe_atom[g];
            ke += 0.5 * m * (st.vx[g] * st.vx[g] + st.vy[g] * st.vy[g] + st.vz[g] * st.vz[g]);
        }
        pe = block_sum(pe, red);
        ke = block_sum(ke, red);
        if (threadIdx.x == 0) {
            pe_out[y.id] = pe;
            ke_out[y.id] = ke;
        }
    }
}

// ---------------------------------------------------------------- block systems
// A system too large for one CTA is advanced in phases of tasks that any CTA of the launch
// may take; a phase starts when every task of the one before it is done.  Phase p = 8 k + s
// of time step k (k = 0 .. K) is stage s:
//   BIN   (atom chunks)  wrap the positions into the box, find each atom's cell, count;
//   SCAN  (one task)     exclusive scan of the counts into cell starts;
//   SCAT  (atom chunks)  each atom takes a slot of its cell;
//   SORT  (cell chunks)  a warp per cell orders its atoms by index (so that every sum is
//                        deterministic) and writes their FP32 coordinates relative to the
//                        cell centre, also as the reference of the skin/2 test;
//   LIST  (blocks)       the Verlet lists of the block's atoms: pairs closer than r_cut +
//                        skin by the FP64 definition (an FP32 test, and an FP64 re-test of
//                        candidates within 1e-4 of the threshold), as 16-bit indices into the
//                        block's tile;
//   FORCE (blocks)       the tile (the block's 4x4x4 cells, current coordinates in the frame
//                        of the block) is staged in shared memory; one thread per own atom
//                        walks its list two entries per step in packed FP32x2 and adds every
//                        pair force component as rint(f 2^32) through the exact two-part
//                        split; an atom with a pair in the FP64 cutoff band or a force beyond
//                        the split is finished by an exact scalar pass.  Then velocity Verlet
//                        in FP64: the closing half kick of step k - 1 and, for k < K, the
//                        opening half kick and the drift of step k into the other position
//                        buffers (other tasks of the phase still read this step's), and the
//                        skin/2 test against the reference.
// A call starts with a one-task START phase that goes on with FORCE of step 0 when the lists
// and coordinates of the previous call are still valid, else with BIN of step 0.  After
// FORCE of step k < K comes BIN of step k + 1 if some atom of the system moved more than
// skin/2, else FORCE of step k + 1.  After FORCE of step K: for odd K, FINAL (atom chunks:
// the positions and coordinates back into the first buffers); then ESUM (one task, energy
// calls: fixed-order sums of the potential and kinetic energy).  Positions are wrapped into
// the box at each BIN only, so between builds they stay in the frame of the lists; the
// host wraps them on output.
// No task waits for anything: the scheduler only hands out tasks of phases that are ready.
// Data written by one task and read by another goes through L2 (__ldcg), never through a
// CTA's L1.
enum { ST_BIN = 0, ST_SCAN = 1, ST_SCAT = 2, ST_SORT = 3, ST_LIST = 4, ST_FORCE = 5 };

__device__ __forceinline__ uint32_t ens_p_end(int K) { return 8u * (uint32_t)(K + 1); }  // FINAL; ESUM after it

__device__ __forceinline__ bool ens_fp64_pair_test(const double* __restrict__ x, const double* __restrict__ y,
                                                   const double* __restrict__ z, const EnsBlockSys& s, int64_t i,
                                                   int64_t j, double r2max) {
    const double dx = mic_rn(__dsub_rn(__ldcg(x + i), __ldcg(x + j)), s.L[0]);
    const double dy = mic_rn(__dsub_rn(__ldcg(y + i), __ldcg(y + j)), s.L[1]);
    const double dz = mic_rn(__dsub_rn(__ldcg(z + i), __ldcg(z + j)), s.L[2]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < r2max;
}

// Wrap one coordinate into [0, L) (one box length at most, counted in the image counter)
// and return its cell index; out-of-box or non-finite coordinates set *bad.
__device__ __forceinline__ int ens_wrap_cell(double& x, int32_t& img, double L, double inv_w, int nc, uint32_t& bad) {
    if (x >= L) {
        x = __dsub_rn(x, L);
        img += 1;
    } else if (x < 0.0) {
        x = __dadd_rn(x, L);
        img -= 1;
    }
    if (!(x >= 0.0 && x <= L)) bad |= isfinite(x) ? ERR_ESCAPE : ERR_NONFINITE;
    const int c = (int)(x * inv_w);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

struct PosBuf {
    double *x, *y, *z;
};

__device__ __forceinline__ PosBuf ens_pos(const BatchState& st, const EnsArrays& ea, bool odd) {
    return odd ? PosBuf{ea.xa, ea.ya, ea.za} : PosBuf{st.x, st.y, st.z};
}

// BIN: wrap the positions of the odd / even buffer in place, cells and counts.
__device__ void ens_bin(const EnsBlockSys& y, const BatchState& st, const EnsArrays& ea, bool odd, int task) {
    const int lo = task * ENS_ATOM_CHUNK, hi = min(y.n, lo + ENS_ATOM_CHUNK);
    const PosBuf P = ens_pos(st, ea, odd);
    double* X[3] = {P.x, P.y, P.z};
    int32_t* I[3] = {st.ix, st.iy, st.iz};
    for (int a = lo + (int)threadIdx.x; a < hi; a += blockDim.x) {
        const int64_t g = y.a0 + a;
        int c[3];
        uint32_t bad = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double x = __ldcg(X[d] + g);
            const double x0 = x;
            int32_t img = __ldcg(I[d] + g);
            const int32_t img0 = img;
            c[d] = ens_wrap_cell(x, img, y.L[d], y.inv_w[d], y.nc[d], bad);
            if (x != x0) X[d][g] = x;
            if (img != img0) I[d][g] = img;
        }
        if (bad) atomicOr(st.err, bad);
        const int id = c[0] + y.nc[0] * (c[1] + y.nc[1] * c[2]);
        ea.cell_of[g] = id;
        atomicAdd(&ea.count[y.c0 + id], 1);
    }
}

// FINAL (odd K): the second buffers' positions and coordinates into the first.
__device__ void ens_final(const EnsBlockSys& y, const BatchState& st, const EnsArrays& ea, int task) {
    const int lo = task * ENS_ATOM_CHUNK, hi = min(y.n, lo + ENS_ATOM_CHUNK);
    for (int a = lo + (int)threadIdx.x; a < hi; a += blockDim.x) {
        const int64_t g = y.a0 + a;
        st.x[g] = __ldcg(ea.xa + g);
        st.y[g] = __ldcg(ea.ya + g);
        st.z[g] = __ldcg(ea.za + g);
        ea.xs[g] = __ldcg(ea.xsb + g);
    }
}

__device__ void ens_scan(const EnsBlockSys& y, const EnsArrays& ea, int* warp_tot) {
    block_scan<true>(ea.count + y.c0, ea.cstart + y.s0, y.ncell, warp_tot);
    for (int k = threadIdx.x; k < y.ncell; k += blockDim.x) {
        ea.count[y.c0 + k] = 0;
        ea.cursor[y.c0 + k] = 0;
    }
}

__device__ void ens_scatter(const EnsBlockSys& y, const EnsArrays& ea, uint32_t* st_err, int task) {
    const int lo = task * ENS_ATOM_CHUNK, hi = min(y.n, lo + ENS_ATOM_CHUNK);
    for (int a = lo + (int)threadIdx.x; a < hi; a += blockDim.x) {
        const int64_t g = y.a0 + a;
        const int c = __ldcg(ea.cell_of + g);
        const int slot = __ldcg(ea.cstart + y.s0 + c) + atomicAdd(&ea.cursor[y.c0 + c], 1);
        // counts and cells disagree only after a task gave up (an error already raised)
        if (slot < __ldcg(ea.cstart + y.s0 + c + 1)) ea.perm_u[y.a0 + slot] = a;
        else atomicOr(st_err, ERR_TILE_OVERFLOW);
    }
}

__device__ void ens_sort(const EnsBlockSys& y, const BatchState& st, const EnsArrays& ea, bool odd, int task) {
    const PosBuf P = ens_pos(st, ea, odd);
    float4* xs = odd ? ea.xsb : ea.xs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c_hi = min(y.ncell, (task + 1) * ENS_CELL_CHUNK);
    for (int c = task * ENS_CELL_CHUNK + warp; c < c_hi; c += nw) {
        const int s0 = __ldcg(ea.cstart + y.s0 + c), cnt = __ldcg(ea.cstart + y.s0 + c + 1) - s0;
        const int cx = c % y.nc[0], cy = (c / y.nc[0]) % y.nc[1], cz = c / (y.nc[0] * y.nc[1]);
        const double ox = (cx + 0.5) * y.w[0], oy = (cy + 0.5) * y.w[1], oz = (cz + 0.5) * y.w[2];
        const int* seg = ea.perm_u + y.a0 + s0;
        for (int e0 = 0; e0 < cnt; e0 += 32) {
            const int e = e0 + lane;
            const int mine = e < cnt ? __ldcg(seg + e) : 0x7fffffff;
            int rank = 0;
            if (cnt <= 32) {  // the cell's ids are in the lanes: rank by shuffles
                for (int f = 0; f < cnt; ++f) rank += __shfl_sync(0xffffffffu, mine, f) < mine;
            } else {
                for (int f = 0; f < cnt; ++f) rank += __ldcg(seg + f) < mine;
            }
            if (e >= cnt || mine < 0 || mine >= y.n) continue;  // (an id out of range: a slot left
                                                                // unfilled after an error)
            const int64_t g = y.a0 + mine;
            const int64_t sl = y.a0 + s0 + rank;
            ea.perm_s[sl] = mine;
            ea.scell[sl] = c;
            const float4 q = make_float4(__double2float_rn(__ldcg(P.x + g) - ox), __double2float_rn(__ldcg(P.y + g) - oy),
                                         __double2float_rn(__ldcg(P.z + g) - oz), 0.0f);
            xs[sl] = q;
            ea.xs_ref[sl] = q;
        }
    }
}

// Tile of a block task: the 64 cells (own 8 first, tile order of tile.cuh) and their atoms
// by slot (TileMeta: prefix = first tile index of each cell, start = its first slot in the
// system's cell order); tile index T = prefix[64] is a point far outside every cutoff.
using EnsTile = TileMeta;

constexpr int ENS_QUEUE = 512;  // own atoms of a block left to the exact pass

// Tile slot of tile index u (binary search in the prefix).
__device__ __forceinline__ int ens_slot_of(const EnsTile& mt, int u) {
    int lo = 0, hi = 64;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (mt.prefix[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The tile meta of block b (threads 0..63 take part; ends with __syncthreads).
__device__ void ens_meta(const EnsBlockSys& y, const EnsArrays& ea, int b, EnsTile& mt) {
    const int bx = b % y.nb[0], t_ = b / y.nb[0], by = t_ % y.nb[1], bz = t_ / y.nb[1];
    const int t = threadIdx.x;
    if (t < 64) {
        const int c = c_tiles.coord_of_idx[t];
        int cx = 2 * bx - 1 + (c & 3), cy = 2 * by - 1 + ((c >> 2) & 3), cz = 2 * bz - 1 + (c >> 4);
        cx += cx < 0 ? y.nc[0] : (cx >= y.nc[0] ? -y.nc[0] : 0);
        cy += cy < 0 ? y.nc[1] : (cy >= y.nc[1] ? -y.nc[1] : 0);
        cz += cz < 0 ? y.nc[2] : (cz >= y.nc[2] ? -y.nc[2] : 0);
        const int id = cx + y.nc[0] * (cy + y.nc[1] * cz);
        const int s0 = __ldcg(ea.cstart + y.s0 + id);
        const int cnt = __ldcg(ea.cstart + y.s0 + id + 1) - s0;
        mt.start[t] = s0;
        const int lane = t & 31;
        int v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int w = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += w;
        }
        mt.prefix[t + 1] = v;
    }
    __syncthreads();
    if (t >= 32 && t < 64) mt.prefix[t + 1] += mt.prefix[32];
    if (t == 0) mt.prefix[0] = 0;
    __syncthreads();
}

// Fill the tile of block b from the FP32 coordinates xs (by slot) in the frame of the block;
// returns the tile size T, or -1 if it exceeds tile_slots.  Ends with __syncthreads.
__device__ int ens_stage(const EnsBlockSys& y, const EnsArrays& ea, const float4* xs, int b, int tile_slots,
                         float4* tile, EnsTile& mt, uint32_t* err) {
    ens_meta(y, ea, b, mt);
    const int T = mt.prefix[64];
    if (T + 1 > tile_slots) {
        if (threadIdx.x == 0) atomicOr(err, ERR_TILE_OVERFLOW);
        return -1;
    }
    // all threads over the tile's atoms (its cell by binary search), so that the L2 loads of
    // a task overlap
    for (int u = threadIdx.x; u < T; u += blockDim.x) {
        const int sl = ens_slot_of(mt, u);
        const int c = c_tiles.coord_of_idx[sl];
        const float ox = pick4(y.off[0], c & 3), oy = pick4(y.off[1], (c >> 2) & 3), oz = pick4(y.off[2], c >> 4);
        const float4 p = __ldcg(xs + y.a0 + mt.start[sl] + (u - mt.prefix[sl]));
        tile[u] = make_float4(p.x + ox, p.y + oy, p.z + oz, 0.0f);
    }
    if (threadIdx.x == 0) tile[T] = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.0f);
    __syncthreads();
    return T;
}

// Shared memory of a LIST task for a tile of T atoms: the padded FP32 arrays and the
// lanes' rings of list entries (8 warps).
__host__ __device__ inline size_t ens_list_smem_bytes(int T) {
    return (size_t)soa_len(T + 1) * 3 * sizeof(float) + (size_t)NL_WARPS * 32 * NL_RING * sizeof(uint16_t);
}

// LIST: the Verlet lists of the own atoms of block b, by the candidate scan of the main
// builder (nl_scan.cuh): warp w takes own cell w, one lane per atom; entries are tile
// indices in chunks of 8 (the last padded with T), by slot.
__device__ void ens_list(const EnsBlockSys& y, const BatchState& st, const EnsArrays& ea, bool odd, int b,
                         size_t smem_bytes, unsigned char* smem, EnsTile& mt, int* pp) {
    ens_meta(y, ea, b, mt);
    const int T = mt.prefix[64];
    if (ens_list_smem_bytes(T) > smem_bytes || T > 65535) {
        if (threadIdx.x == 0) atomicOr(st.err, ERR_TILE_OVERFLOW);
        return;
    }
    const int SL = soa_len(T + 1);
    float* tx = reinterpret_cast<float*>(smem);
    float* ty = tx + SL;
    float* tz = ty + SL;
    uint16_t* buf = reinterpret_cast<uint16_t*>(tz + SL);  // NL_WARPS x NL_RING x 32
    TileOffsets to;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int q = 0; q < 4; ++q) to.off[d][q] = y.off[d][q];
    tile_pad_prefix(mt, pp);
    tile_stage_soa<true>(mt, pp, (odd ? ea.xsb : ea.xs) + y.a0, to, tx, ty, tz);
    __syncthreads();
    const PosBuf P = ens_pos(st, ea, odd);
    const unsigned sx = (unsigned)__cvta_generic_to_shared(tx);
    const unsigned sy = (unsigned)__cvta_generic_to_shared(ty);
    const unsigned sz = (unsigned)__cvta_generic_to_shared(tz);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (warp >= NL_WARPS) return;
    uint16_t* col = buf + (size_t)warp * NL_RING * 32 + lane;
    const int cap = ea.list_chunks * 8;
    uint4* nl = ea.nl + y.a0 * (int64_t)ea.list_chunks;
    const f2_t hi2 = f2_pack(ea.rl2_hi, ea.rl2_hi), lo2 = f2_pack(ea.rl2_lo, ea.rl2_lo);
    for (int oc = warp; oc < 8; oc += min(nw, NL_WARPS)) {
        const int lx = oc & 1, ly = (oc >> 1) & 1, lz = oc >> 2;
        const int own_coord = (lx + 1) + 4 * (ly + 1) + 16 * (lz + 1);
        const int own_begin = mt.prefix[oc], own_count = mt.prefix[oc + 1] - own_begin;
        for (int base = 0; base < own_count; base += 32) {
            const int e = base + lane;
            const bool active = e < own_count;
            const int ei = active ? e : 0;
            const int own_p = pp[oc] + ei;
            const int slot_i = mt.start[oc] + ei;
            const int64_t gi = y.a0 + __ldcg(ea.perm_s + y.a0 + slot_i);
            const float xi = tx[own_p], yi = ty[own_p], zi = tz[own_p];
            const f2_t pix = f2_pack(xi, xi), piy = f2_pack(yi, yi), piz = f2_pack(zi, zi);
            ListOut o{col, nl + slot_i, (size_t)y.n, cap, 0, 0};
#pragma unroll 1
            for (int key = 0; key < 27; ++key) {  // the own cell first, then the 26 neighbours
                const int kk = key == 0 ? 0 : (key <= 13 ? key - 14 : key - 13);
                const int oz = (kk + 13) / 9 - 1, oy = ((kk + 13) / 3) % 3 - 1, ox = (kk + 13) % 3 - 1;
                const int sl = c_tiles.idx_of_coord[own_coord + ox + 4 * oy + 16 * oz];
                const int s_adj = mt.start[sl] - pp[sl];  // system slot = padded index + s_adj
                auto retest = [&](int q) {
                    const int64_t gj = y.a0 + __ldcg(ea.perm_s + y.a0 + q + s_adj);
                    return ens_fp64_pair_test(P.x, P.y, P.z, y, gi, gj, ea.rl2);
                };
                if (key == 0)
                    scan_cell<0, true>(sx, sy, sz, pp[sl], mt.prefix[sl + 1] - mt.prefix[sl], mt.prefix[sl] - pp[sl],
                                       pix, piy, piz, hi2, lo2, own_p, active, o, retest);
                else
                    scan_cell<0, false>(sx, sy, sz, pp[sl], mt.prefix[sl + 1] - mt.prefix[sl], mt.prefix[sl] - pp[sl],
                                        pix, piy, piz, hi2, lo2, own_p, active, o, retest);
            }
            flush_chunks(o, (unsigned)T, true);
            if (active) {
                if (o.cnt > cap) atomicOr(st.err, ERR_LIST_OVERFLOW);
                ea.nl_cnt[y.a0 + slot_i] = o.cnt < cap ? o.cnt : cap;
            }
        }
    }
}

// The state an own atom's Verlet update reads, loaded before its force loop so that the
// loads overlap it.
struct AtomState {
    double vx, vy, vz, x, y, z;
};

__device__ __forceinline__ AtomState ens_load_state(const BatchState& st, const EnsArrays& ea, int k, int K,
                                                    int64_t g) {
    AtomState a{0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (K == 0) return a;
    a.vx = __ldcg(st.vx + g);
    a.vy = __ldcg(st.vy + g);
    a.vz = __ldcg(st.vz + g);
    if (k < K) {
        const PosBuf P = ens_pos(st, ea, (k & 1) != 0);
        a.x = __ldcg(P.x + g);
        a.y = __ldcg(P.y + g);
        a.z = __ldcg(P.z + g);
    }
    return a;
}

// Velocity Verlet for one own atom (slot, atom g, state a) after its force at step k of K.
__device__ __forceinline__ void ens_epilogue(const EnsBlockSys& y, const BatchState& st, const EnsArrays& ea,
                                             const PairTable& pt, int k, int K, bool energy, double dt, int slot,
                                             int64_t g, long long qx, long long qy, long long qz, float pe,
                                             int bidx, const AtomState& a) {
    if (k == K) {
        st.fq[g] = qx;
        st.fq[st.ntot + g] = qy;
        st.fq[2 * st.ntot + g] = qz;
        if (energy) ea.pe_atom[g] = 0.5f * pe;
    }
    if (K == 0) return;
    const double hq = pt.hdtm_q[0];
    double vx = a.vx, vy = a.vy, vz = a.vz;
    if (k > 0) {  // closing half kick of step k - 1
        vx = fma(hq, (double)qx, vx);
        vy = fma(hq, (double)qy, vy);
        vz = fma(hq, (double)qz, vz);
    }
    if (k < K) {  // opening half kick of step k
        vx = fma(hq, (double)qx, vx);
        vy = fma(hq, (double)qy, vy);
        vz = fma(hq, (double)qz, vz);
    }
    st.vx[g] = vx;
    st.vy[g] = vy;
    st.vz[g] = vz;
    if (k == K) return;
    // drift into the other buffers: FP64 positions, and FP32 coordinates relative to the
    // centre of the cell the atom was binned into at the last build
    const bool odd = (k & 1) != 0;
    const PosBuf Pn = ens_pos(st, ea, !odd);
    const double x = fma(dt, vx, a.x), yv = fma(dt, vy, a.y), z = fma(dt, vz, a.z);
    Pn.x[g] = x;
    Pn.y[g] = yv;
    Pn.z[g] = z;
    const int64_t sl = y.a0 + slot;
    const int c = __ldcg(ea.scell + sl);
    const int cx = c % y.nc[0], cy = (c / y.nc[0]) % y.nc[1], cz = c / (y.nc[0] * y.nc[1]);
    const float4 q = make_float4(__double2float_rn(x - (cx + 0.5) * y.w[0]), __double2float_rn(yv - (cy + 0.5) * y.w[1]),
                                 __double2float_rn(z - (cz + 0.5) * y.w[2]), 0.0f);
    (odd ? ea.xs : ea.xsb)[sl] = q;
    const float4 r = __ldcg(ea.xs_ref + sl);
    const float ex = q.x - r.x, ey = q.y - r.y, ez = q.z - r.z;
    if (!(fmaf(ez, ez, fmaf(ey, ey, ex * ex)) <= ea.lim2_f)) ea.rebuild[bidx] = 1;
}

// Chunks 0 .. nch-1 of one list (chunk c at lp[c * stride]), two entries per call of body;
// the chunks were written by other CTAs of the launch, so they are read from L2, two chunks
// ahead of their use (a task holds few warps, so load latency is not hidden by others).
template <typename Body>
__device__ __forceinline__ void ens_for_each_pair(const uint4* __restrict__ lp, size_t stride, int nch, Body&& body) {
    uint4 cur = make_uint4(0u, 0u, 0u, 0u), n1 = cur, n2 = cur;
    if (nch > 0) cur = __ldcg(lp);
    if (nch > 1) n1 = __ldcg(lp + stride);
    for (int c = 0; c < nch; ++c) {
        if (c + 2 < nch) n2 = __ldcg(lp + (size_t)(c + 2) * stride);
        body((int)(cur.x & 0xffffu), (int)(cur.x >> 16));
        body((int)(cur.y & 0xffffu), (int)(cur.y >> 16));
        body((int)(cur.z & 0xffffu), (int)(cur.z >> 16));
        body((int)(cur.w & 0xffffu), (int)(cur.w >> 16));
        cur = n1;
        n1 = n2;
    }
}

// FORCE of block b at step k.  The pair step is the main path's one-species form: fs2 =
// inv^4 (a inv^3 - b) with inv = 1/r^2, and the cutoff-band and large-force tests as two
// running minima (min |r^2 - r_cut^2| and min r^2) checked once per atom.
template <bool ENERGY>
__device__ void ens_force(const EnsBlockSys& y, const BatchState& st, const EnsArrays& ea, const PairTable& pt,
                          float fs2_max, int k, int K, double dt, int b, int bidx, int tile_slots, float4* tile,
                          EnsTile& mt, uint16_t* queue, int* nqueued) {
    const bool odd = (k & 1) != 0;
    if (threadIdx.x == 0) *nqueued = 0;
    const int T = ens_stage(y, ea, odd ? ea.xsb : ea.xs, b, tile_slots, tile, mt, st.err);
    if (T < 0) return;
    const unsigned tile_s = (unsigned)__cvta_generic_to_shared(tile);
    const uint4* nl = ea.nl + y.a0 * (int64_t)ea.list_chunks;
    for (int u = threadIdx.x; u < mt.prefix[8]; u += blockDim.x) {
        int os = 0;
        while (os < 7 && u >= mt.prefix[os + 1]) ++os;
        const int slot = mt.start[os] + (u - mt.prefix[os]);
        const float4 pi = tile[u];
        const int nch = (__ldcg(ea.nl_cnt + y.a0 + slot) + 7) >> 3;
        const int64_t g = y.a0 + __ldcg(ea.perm_s + y.a0 + slot);
        const AtomState as = ens_load_state(st, ea, k, K, g);
        FixAcc ax{0u, 0u}, ay{0u, 0u}, az{0u, 0u};
        float pe = 0.f, mdist = 3.0e38f, mr2 = 3.0e38f;
        ens_for_each_pair(nl + slot, (size_t)y.n, nch, [&](int u0, int u1) {
            const float4 pa = lds_tile(tile_s, u0);
            const float4 pb = lds_tile(tile_s, u1);
            const f2_t ex = f2_pack(__fsub_rn(pi.x, pa.x), __fsub_rn(pi.x, pb.x));
            const f2_t ey = f2_pack(__fsub_rn(pi.y, pa.y), __fsub_rn(pi.y, pb.y));
            const f2_t ez = f2_pack(__fsub_rn(pi.z, pa.z), __fsub_rn(pi.z, pb.z));
            const f2_t r2 = f2_fma(ez, ez, f2_fma(ey, ey, f2_mul(ex, ex)));
            float r2a, r2b;
            f2_unpack(r2, r2a, r2b);
            const f2_t inv = f2_pack(rcp_approx(r2a), rcp_approx(r2b));
            const f2_t inv2 = f2_mul(inv, inv);
            const f2_t inv3 = f2_mul(inv2, inv);
            const f2_t t = f2_fma(f2_pack(pt.lj_a_f, pt.lj_a_f), inv3, f2_pack(-pt.lj_b_f, -pt.lj_b_f));
            float fa, fb;
            f2_unpack(f2_mul(t, f2_mul(inv2, inv2)), fa, fb);
            const bool ina = r2a < pt.rc2hi_f[0], inb = r2b < pt.rc2hi_f[0];
            float dca, dcb;
            f2_unpack(f2_sub(r2, f2_pack(pt.rc2_f[0], pt.rc2_f[0])), dca, dcb);  // exact near r_cut
            mdist = fminf(mdist, fminf(fabsf(dca), fabsf(dcb)));
            mr2 = fminf(mr2, fminf(r2a, r2b));
            fa = ina ? fa : 0.0f;
            fb = inb ? fb : 0.0f;
            const f2_t fs2 = f2_pack(fa, fb);
            fix_add2(ax, fs2, ex, f2_pack(MAGIC, MAGIC), f2_pack(TWO21, TWO21));
            fix_add2(ay, fs2, ey, f2_pack(MAGIC, MAGIC), f2_pack(TWO21, TWO21));
            fix_add2(az, fs2, ez, f2_pack(MAGIC, MAGIC), f2_pack(TWO21, TWO21));
            if (ENERGY) {
                float s6a, s6b;
                f2_unpack(f2_mul(f2_pack(pt.sig6_f, pt.sig6_f), inv3), s6a, s6b);
                pe += (ina ? pt.c4_f[0] * s6a * (s6a - 1.0f) : 0.0f) + (inb ? pt.c4_f[0] * s6b * (s6b - 1.0f) : 0.0f);
            }
        });
        // a pair in the band or close enough for a term beyond the split, or a list longer
        // than the split sums take, sends the atom to the exact pass
        if ((mdist <= pt.band_half_f) | (mr2 < pt.r2_wide_f) | (nch * 8 > FIX_SPLIT_MAX_TERMS)) {
            const int at = atomicAdd(nqueued, 1);
            if (at < ENS_QUEUE) queue[at] = (uint16_t)u;
            else atomicOr(st.err, ERR_TILE_OVERFLOW);
            continue;
        }
        const int nterms = nch * 8;
        ens_epilogue(y, st, ea, pt, k, K, ENERGY, dt, slot, g, fix_final(ax, nterms), fix_final(ay, nterms),
                     fix_final(az, nterms), pe, bidx, as);
    }
    __syncthreads();
    // the exact pass: every entry one at a time, the same FP32 operations for ordinary pairs,
    // FP64 decisions in the cutoff band, large terms rounded in FP64
    const PosBuf P = ens_pos(st, ea, odd);
    const int nq = min(*nqueued, ENS_QUEUE);
    for (int j = threadIdx.x; j < nq; j += blockDim.x) {
        const int u = queue[j];
        int os = 0;
        while (os < 7 && u >= mt.prefix[os + 1]) ++os;
        const int slot = mt.start[os] + (u - mt.prefix[os]);
        const int64_t gi = y.a0 + __ldcg(ea.perm_s + y.a0 + slot);
        const float4 pi = tile[u];
        const int cnt = __ldcg(ea.nl_cnt + y.a0 + slot);
        long long qx = 0, qy = 0, qz = 0;
        float pe = 0.f;
        int nwide = 0;
        for (int e = 0; e < cnt; ++e) {
            const uint4 ch = __ldcg(nl + (int64_t)(e >> 3) * y.n + slot);
            const unsigned w = (e & 7) < 4 ? ((e & 7) < 2 ? ch.x : ch.y) : ((e & 7) < 6 ? ch.z : ch.w);
            const int q = (int)((w >> (16 * (e & 1))) & 0xffffu);
            const float4 pj = tile[q];
            const float ex = __fsub_rn(pi.x, pj.x), ey = __fsub_rn(pi.y, pj.y), ez = __fsub_rn(pi.z, pj.z);
            const float r2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
            if (!(r2 < pt.rc2hi_f[0])) continue;
            if (!(r2 < pt.rc2lo_f[0])) {
                const int sl = ens_slot_of(mt, q);
                const int64_t gj = y.a0 + __ldcg(ea.perm_s + y.a0 + mt.start[sl] + (q - mt.prefix[sl]));
                if (!ens_fp64_pair_test(P.x, P.y, P.z, y, gi, gj, pt.rc2_d[0])) continue;
            }
            const float inv = rcp_approx(r2);
            const float inv2 = __fmul_rn(inv, inv);
            const float inv3 = __fmul_rn(inv2, inv);
            const float fs2 = __fmul_rn(__fmaf_rn(pt.lj_a_f, inv3, -pt.lj_b_f), __fmul_rn(inv2, inv2));
            qx += fix_term_any(fs2, ex, fs2_max, st.err);
            qy += fix_term_any(fs2, ey, fs2_max, st.err);
            qz += fix_term_any(fs2, ez, fs2_max, st.err);
            nwide += fabsf(fs2) < fs2_max ? 0 : 1;
            if (ENERGY) {
                const float s6 = __fmul_rn(pt.sig6_f, inv3);
                pe += pt.c4_f[0] * s6 * (s6 - 1.0f);
            }
        }
        fix_wide_count_ok(nwide, st.err);
        ens_epilogue(y, st, ea, pt, k, K, ENERGY, dt, slot, gi, qx, qy, qz, pe, bidx, ens_load_state(st, ea, k, K, gi));
    }
}

__device__ void ens_esum(const EnsBlockSys& y, const BatchState& st, const EnsArrays& ea, const PairTable& pt,
                         double* pe_out, double* ke_out, double* red) {
    double pe = 0.0, ke = 0.0;
    const double m = pt.mass[0];
    for (int a = threadIdx.x; a < y.n; a += blockDim.x) {
        const int64_t g = y.a0 + a;
        const double vx = __ldcg(st.vx + g), vy = __ldcg(st.vy + g), vz = __ldcg(st.vz + g);
        pe += (double)__ldcg(ea.pe_atom + g);
        ke += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    }
    pe = block_sum(pe, red);
    ke = block_sum(ke, red);
    if (threadIdx.x == 0) {
        pe_out[y.id] = pe;
        ke_out[y.id] = ke;
    }
}

// Tasks in phase p of an entry (one-CTA entries: p = 0, one task).
__device__ __forceinline__ int ens_ntasks(const EnsEntry& e, uint32_t p, int K) {
    if (e.kind == 0) return p == 0 ? 1 : 0;
    if (p == ENS_START) return 1;
    const uint32_t pe = ens_p_end(K);
    if (p == pe) return e.n_atom_chunks;  // FINAL
    if (p == pe + 1) return 1;             // ESUM
    switch (p & 7) {
        case ST_BIN: return e.n_atom_chunks;
        case ST_SCAN: return 1;
        case ST_SCAT: return e.n_atom_chunks;
        case ST_SORT: return e.n_cell_chunks;
        default: return e.nblock;  // LIST, FORCE
    }
}

// The phase after p, chosen by the CTA that completed p's last task.
__device__ __forceinline__ uint32_t ens_next_phase(const EnsEntry& e, uint32_t p, int K, int flags,
                                                  const EnsArrays& ea) {
    if (e.kind == 0) return ENS_DONE;
    const uint32_t pe = ens_p_end(K);
    volatile int* rebuild = ea.rebuild + e.idx;
    volatile int* valid = ea.valid + e.idx;
    if (p == ENS_START) {
        if (*valid && !*rebuild) return ST_FORCE;
        *rebuild = 0;
        return ST_BIN;
    }
    if (p == pe) return (flags & BATCH_ENERGY) ? pe + 1 : ENS_DONE;
    if (p == pe + 1) return ENS_DONE;
    if ((p & 7) == ST_LIST) *valid = 1;
    if ((p & 7) != ST_FORCE) return p + 1;
    const uint32_t k = p >> 3;
    if ((int)k == K) return (K & 1) ? pe : ((flags & BATCH_ENERGY) ? pe + 1 : ENS_DONE);
    if (*rebuild) {
        *rebuild = 0;
        return 8u * (k + 1) + ST_BIN;
    }
    return 8u * (k + 1) + ST_FORCE;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace

// One persistent launch for the whole ensemble.  Every CTA loops: warp 0 looks through the
// work table (32 entries per probe, starting at the entry it last worked on) for a phase
// with an unclaimed task and claims it by compare-and-swap on the entry's word; the CTA runs
// the task; the CTA that completes a phase's last task publishes the next phase.  No task
// ever waits.  A CTA that finds no work keeps looking until every entry is done; if it finds
// none for ea.budget cycles it sets ERR_TIMEOUT and ends (as do all others, once they see
// the bit), so the host gets MD_ERR_TIMEOUT instead of a hung launch.
#ifndef CLAIM_MANY
#define CLAIM_MANY 4
#endif
// Up to 128 registers a thread: capped at 64 (four 256-thread CTAs per SM) the block tasks
// spill and the 512-system ensemble ran 20 % slower (2.66 against 2.20 ms per step) than
// with two CTAs per SM unspilled.
__global__ void __launch_bounds__(BATCH_MAX_THREADS, 1)
    k_ensemble_run(const EnsEntry* __restrict__ ent, int nent, const BatchSys* __restrict__ one,
                   const EnsBlockSys* __restrict__ blk, BatchState st, EnsArrays ea, PairTable pt, int K, int flags,
                   double dt, float fs2_max, int nmax, int cmax, int tile_slots, double* __restrict__ pe_out,
                   double* __restrict__ ke_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int warp_tot[32];
    __shared__ double red[BATCH_MAX_THREADS];
    __shared__ int nqueued;
    __shared__ EnsTile mt;
    __shared__ int pp[65];
    const size_t smem_bytes = (size_t)(tile_slots + 1) * sizeof(float4);
    __shared__ uint16_t queue[ENS_QUEUE];
    __shared__ int s_ent, s_task, s_take, s_quit;
    __shared__ uint32_t s_phase;
    const int lane = threadIdx.x & 31;
    int cursor = (int)((blockIdx.x * 37u) % (unsigned)max(nent, 1));
    long long idle_since = clock64();
    const bool energy_call = (flags & BATCH_ENERGY) != 0;
    while (true) {
        if (threadIdx.x < 32) {
            int got = -1, task = 0, ntake = 1;
            uint32_t ph = 0;
            int quit = 0;
            if (lane == 0)
                quit = ld_relaxed_s32(ea.g_done) >= nent || (ld_relaxed_s32(reinterpret_cast<const int*>(st.err)) &
                                                             (int)ERR_TIMEOUT) != 0;
            quit = __shfl_sync(0xffffffffu, quit, 0);
            for (int r = 0; !quit && got < 0 && r < nent; r += 32) {
                const int e = (cursor + r + lane) % nent;
                const bool live = r + lane < nent;
                unsigned long long w = live ? ld_relaxed_u64(ea.ctl + e) : 0ull;
                const uint32_t p = (uint32_t)(w >> 32), nx = (uint32_t)w;
                const int T = live && p < ENS_HOLD ? ens_ntasks(ent[e], p, K) : 0;
                // several tasks at once from large phases: fewer claims
                const int want = (int)nx + CLAIM_MANY <= T && T >= 16 * CLAIM_MANY ? CLAIM_MANY
                                 : ((int)nx + 2 <= T && T >= 8 ? 2 : 1);
                bool can = (int)nx < T;
                unsigned m = __ballot_sync(0xffffffffu, can);
                while (m) {
                    const int l = __ffs(m) - 1;
                    int ok = 0;
                    if (lane == l) ok = atomicCAS(ea.ctl + e, w, w + (unsigned long long)want) == w;
                    ok = __shfl_sync(0xffffffffu, ok, l);
                    if (ok) {
                        got = __shfl_sync(0xffffffffu, e, l);
                        ph = __shfl_sync(0xffffffffu, p, l);
                        task = (int)__shfl_sync(0xffffffffu, nx, l);
                        ntake = __shfl_sync(0xffffffffu, want, l);
                        break;
                    }
                    m &= m - 1;
                }
            }
            if (lane == 0) {
                s_ent = got;
                s_phase = ph;
                s_task = task;
                s_take = ntake;
                s_quit = quit;
            }
        }
        __syncthreads();
        const int e = s_ent;
        const uint32_t p = s_phase;
        const int task0 = s_task, take = s_take;
        const int quit = s_quit;
        __syncthreads();
        if (quit) break;
        if (e < 0) {
            if (clock64() - idle_since > ea.budget) {
                if (threadIdx.x == 0) atomicOr(st.err, ERR_TIMEOUT);
                break;
            }
            __nanosleep(2000);
            continue;
        }
        __threadfence();  // what the phase before this one wrote is visible from here on
        const EnsEntry en = ent[e];
        for (int task = task0; task < task0 + take; ++task) {
            if (en.kind == 0) {
                run_one_system(one[en.idx], st, pt, K, flags, dt, fs2_max, nmax, cmax, ea.pe_atom, pe_out, ke_out, smem,
                               warp_tot, &nqueued, red);
            } else {
                const EnsBlockSys& y = blk[en.idx];
                const uint32_t pend = ens_p_end(K);
                float4* tile = reinterpret_cast<float4*>(smem);
                if (p == ENS_START) {
                    // only the decision of ens_next_phase
                } else if (p == pend) {
                    ens_final(y, st, ea, task);
                } else if (p == pend + 1) {
                    ens_esum(y, st, ea, pt, pe_out, ke_out, red);
                } else {
                    const int k = (int)(p >> 3);
                    const bool odd = (k & 1) != 0;
                    switch (p & 7) {
                        case ST_BIN: ens_bin(y, st, ea, odd, task); break;
                        case ST_SCAN: ens_scan(y, ea, warp_tot); break;
                        case ST_SCAT: ens_scatter(y, ea, st.err, task); break;
                        case ST_SORT: ens_sort(y, st, ea, odd, task); break;
                        case ST_LIST: ens_list(y, st, ea, odd, task, smem_bytes, smem, mt, pp); break;
                        default:
                            if (energy_call && k == K)
                                ens_force<true>(y, st, ea, pt, fs2_max, k, K, dt, task, en.idx, tile_slots, tile, mt,
                                                queue, &nqueued);
                            else
                                ens_force<false>(y, st, ea, pt, fs2_max, k, K, dt, task, en.idx, tile_slots, tile, mt,
                                                 queue, &nqueued);
                    }
                }
            }
            if (task + 1 < task0 + take) __syncthreads();  // the next task reuses the shared memory
        }
        __threadfence();  // this task's writes before its completion is counted
        __syncthreads();
        if (threadIdx.x == 0) {
            const int T = ens_ntasks(en, p, K);
            if (atomicAdd(ea.done + e, take) + take == T) {  // the phase's last task: publish the next
                const uint32_t np = ens_next_phase(en, p, K, flags, ea);
                ea.done[e] = 0;
                __threadfence();
                atomicExch(ea.ctl + e, (unsigned long long)np << 32);
                if (np == ENS_DONE) atomicAdd(ea.g_done, 1);
            }
        }
        cursor = e;
        idle_since = clock64();
    }
}

size_t batch_smem_bytes(int nmax, int cmax) {
    return batch_smem_ints_offset(nmax) + (size_t)(2 * cmax + 1) * sizeof(int);
}

size_t ens_tile_smem_bytes(int tile_slots) { return (size_t)(tile_slots + 1) * sizeof(float4); }

size_t ens_list_smem(int T) { return ens_list_smem_bytes(T); }

void launch_ensemble(const EnsEntry* ent, int nent, const BatchSys* one, const EnsBlockSys* blk,
                     const BatchState& st, const EnsArrays& ea, const PairTable& pt, int n_steps, int flags,
                     double dt, int threads, int grid, int nmax, int cmax, int tile_slots, size_t smem,
                     double* pe_out, double* ke_out, cudaStream_t s) {
    if (nent == 0 || grid <= 0) return;
    const float fs2_max = 4194304.0f / sqrtf(pt.rc2_f[0]) * 0.999f;
    k_ensemble_run<<<grid, threads, smem, s>>>(ent, nent, one, blk, st, ea, pt, n_steps, flags, dt, fs2_max, nmax,
                                               cmax, tile_slots, pe_out, ke_out);
}

int ensemble_ctas_per_sm(int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ensemble_run, threads, smem) != cudaSuccess) return 0;
    return n;
}

void init_batch_kernels() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_ensemble_run) != cudaSuccess) return;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(k_ensemble_run, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

}  // namespace mdgb
