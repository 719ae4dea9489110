// k_batch.cu - ensembles of small independent systems, one CTA per system.
//
// The paper notes that its task functor can carry which copy of a system a task
// works on, so that replicas share one schedule (Sec. II.C).  On the GPU an ensemble
// of small periodic systems (a few hundred to a few thousand atoms) is run by one
// persistent launch in which each CTA owns one whole system for all of its time
// steps: the system's FP32 coordinates and linked cells live in shared memory, and
// no two CTAs ever touch the same particle, so the launch needs no synchronisation
// between CTAs at all.  Per step the CTA
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
#include "fixpt.cuh"
#include "mdgb_batch_internal.cuh"
#include "tile.cuh"

namespace mdgb {

namespace {

// block-wide exclusive scan of cnt[0..m) into start[0..m], start[m] = total
__device__ void block_scan(const int* __restrict__ cnt, int* __restrict__ start, int m, int* warp_tot) {
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5, nw = nt >> 5;
    const int per = (m + nt - 1) / nt;
    const int lo = t * per, hi = min(lo + per, m);
    int s = 0;
    for (int k = lo; k < hi; ++k) s += cnt[k];
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
        run += cnt[k];
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

// One CTA per system.  flags: BATCH_HAVE_FORCES (st.fq holds F at the current
// positions), BATCH_ENERGY (potential and kinetic energy per system at the end).
__global__ void __launch_bounds__(BATCH_MAX_THREADS) k_batch_run(const BatchSys* __restrict__ sys, int nsys,
                                                                 BatchState st, PairTable pt, int n_steps,
                                                                 int flags, double dt, float fs2_max,
                                                                 int nmax, int cmax, double* __restrict__ pe_out,
                                                                 double* __restrict__ ke_out,
                                                                 float* __restrict__ pe_atom) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int warp_tot[32];
    __shared__ double red[BATCH_MAX_THREADS];
    const int b = blockIdx.x;
    if (b >= nsys) return;
    const BatchSys y = sys[b];
    if (y.n == 0) return;
    if (y.n > nmax || y.ncell > cmax) {  // the host sizes every launch for its systems
        if (threadIdx.x == 0) atomicOr(st.err, ERR_TILE_OVERFLOW);
        return;
    }
    __shared__ int nqueued;
    Smem sm;
    const int np2 = nmax + 2;  // even: the three coordinate arrays stay 8-byte aligned
    sm.px = reinterpret_cast<float*>(smem);
    sm.py = sm.px + np2;
    sm.pz = sm.py + np2;
    sm.perm = reinterpret_cast<uint16_t*>(sm.pz + np2);
    sm.cell = sm.perm + nmax;
    sm.scell = sm.cell + nmax;
    sm.queue = sm.scell + np2;
    sm.nqueued = &nqueued;
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

size_t batch_smem_bytes(int nmax, int cmax) {
    return batch_smem_ints_offset(nmax) + (size_t)(2 * cmax + 1) * sizeof(int);
}

void launch_batch_run(const BatchSys* sys, int nsys, const BatchState& st, const PairTable& pt, int n_steps,
                      int flags, double dt, int threads, int nmax, int cmax, double* pe_out, double* ke_out,
                      float* pe_atom, cudaStream_t s) {
    if (nsys == 0) return;
    const float fs2_max = 4194304.0f / sqrtf(pt.rc2_f[0]) * 0.999f;
    k_batch_run<<<nsys, threads, batch_smem_bytes(nmax, cmax), s>>>(sys, nsys, st, pt, n_steps, flags, dt, fs2_max,
                                                                     nmax, cmax, pe_out, ke_out, pe_atom);
}

void init_batch_kernels() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_batch_run) != cudaSuccess) return;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(k_batch_run, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

}  // namespace mdgb
