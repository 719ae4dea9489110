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
//   * evaluates the cutoff LJ force on every atom over the (2R+1)^3 surrounding cells
//     (FP32 pair arithmetic on cell-relative coordinates, every pair force component
//     added as rint(f * 2^32) through the same exact two-part integer split as the
//     main path, so forces do not depend on summation order),
//   * and integrates velocity Verlet in FP64.
// There is no neighbour list: the cells are rebuilt every step, which for systems of
// this size costs less than a list build would.
#include "mdgb_batch_internal.cuh"
#include "tile.cuh"

namespace mdgb {

namespace {

constexpr float BMAGIC = 12582912.0f;  // 1.5 * 2^23
constexpr float BTWO21 = 2097152.0f;   // 2^21

struct Fix2 {
    unsigned hi, lo;
};

// add rint(a * 2^21) in units of 2^-32 for a = fs2 * d (|a| < 2^22): exact two-part split
__device__ __forceinline__ void bfix_add(Fix2& acc, float fs2, float d) {
    const float t1 = __fmaf_rn(fs2, d, BMAGIC);
    const float h = __fsub_rn(t1, BMAGIC);
    const float r = __fmaf_rn(fs2, d, -h);
    const float t2 = __fmaf_rn(r, BTWO21, BMAGIC);
    acc.hi += __float_as_uint(t1);
    acc.lo += __float_as_uint(t2);
}

// the same sum for |fs2 * d| >= 2^22 (or non-finite): FP64 rounding, same two-part form
__device__ __noinline__ uint2 bfix_wide(float fs2, float d, uint32_t* err) {
    double a = (double)fs2 * (double)d * 2097152.0;
    if (!(fabs(a) < 9.0e15)) {
        atomicOr(err, ERR_NONFINITE);
        a = 0.0;
    }
    const long long q = __double2ll_rn(a);
    const long long qh = q >> 21;
    return make_uint2(__float_as_uint(BMAGIC) + (unsigned)(int)qh,
                      __float_as_uint(BMAGIC) + (unsigned)(int)(q - qh * 2097152LL));
}

__device__ __forceinline__ long long bfix_final(const Fix2& a, int nterms) {
    const int hi = (int)(a.hi - (unsigned)nterms * __float_as_uint(BMAGIC));
    const int lo = (int)(a.lo - (unsigned)nterms * __float_as_uint(BMAGIC));
    return (long long)hi * 2097152LL + (long long)lo;
}

__device__ __forceinline__ float brcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

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
    float4* xr;        // n: FP32 coordinates relative to the cell centre, by slot (species in w)
    uint16_t* perm;    // n: slot -> local atom
    uint16_t* cell;    // n: local atom -> cell, then local atom -> slot
    int* cstart;       // ncell + 1
    int* ccount;       // ncell
    int* warp_tot;     // 32
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
            float4 p;
            p.x = __double2float_rn(st.x[g] - ox);
            p.y = __double2float_rn(st.y[g] - oy);
            p.z = __double2float_rn(st.z[g] - oz);
            p.w = __int_as_float(st.species[g]);
            sm.xr[s0 + rank] = p;
            sm.cell[mine] = (uint16_t)(s0 + rank);
        }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < n; a += blockDim.x) sm.perm[sm.cell[a]] = (uint16_t)a;
    __syncthreads();
}

// Force on every atom (fixed point into st.fq); with energy, also its half pair
// energies (FP32 per atom, neighbours in slot order: deterministic).
template <bool ENERGY>
__device__ void batch_forces(const BatchSys& y, BatchState st, const PairTable& pt, float fs2_max, Smem& sm,
                             float* __restrict__ pe_out) {
    const int n = y.n, R = y.R;
    const float sig2 = pt.sig2_f[0], c48 = pt.c48_f[0], c24 = pt.c24_f[0], c4 = pt.c4_f[0];
    const float rc2_lo = pt.rc2lo_f[0], rc2_hi = pt.rc2hi_f[0];
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int a = sm.perm[p];
        const float4 pi = sm.xr[p];
        // cell of slot p: find it from the cell of atom a (binary search would also do)
        const int64_t g = y.a0 + a;
        int cc[3];
        {
            const double* X[3] = {st.x, st.y, st.z};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int v = (int)(X[d][g] * y.inv_w[d]);
                cc[d] = v < 0 ? 0 : (v >= y.nc[d] ? y.nc[d] - 1 : v);
            }
        }
        Fix2 ax{0u, 0u}, ay{0u, 0u}, az{0u, 0u};
        int nterms = 0;
        float pe = 0.f;
        for (int dz = -R; dz <= R; ++dz) {
            int z = cc[2] + dz;
            z += z < 0 ? y.nc[2] : (z >= y.nc[2] ? -y.nc[2] : 0);
            for (int dy = -R; dy <= R; ++dy) {
                int yy = cc[1] + dy;
                yy += yy < 0 ? y.nc[1] : (yy >= y.nc[1] ? -y.nc[1] : 0);
                for (int dx = -R; dx <= R; ++dx) {
                    int x = cc[0] + dx;
                    x += x < 0 ? y.nc[0] : (x >= y.nc[0] ? -y.nc[0] : 0);
                    const int id = x + y.nc[0] * (yy + y.nc[1] * z);
                    const float sx = (float)dx * y.wf[0], sy = (float)dy * y.wf[1], sz = (float)dz * y.wf[2];
                    const bool self_cell = (dx | dy | dz) == 0;
                    const int q1 = sm.cstart[id + 1];
                    for (int q = sm.cstart[id]; q < q1; ++q) {
                        if (self_cell && q == p) continue;
                        const float4 pj = sm.xr[q];
                        const float ex = pi.x - (pj.x + sx), ey = pi.y - (pj.y + sy), ez = pi.z - (pj.z + sz);
                        const float r2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                        if (!(r2 < rc2_hi)) continue;
                        if (!(r2 < rc2_lo) &&  // rare: decide the cutoff in FP64, as the definition
                            !fp64_pair_test(st.x, st.y, st.z, y.L[0], y.L[1], y.L[2], g, y.a0 + sm.perm[q],
                                            pt.rc2_d[0]))
                            continue;
                        const float inv = brcp(r2);
                        const float s2 = sig2 * inv;
                        const float s6 = s2 * s2 * s2;
                        const float fs2 = (c48 * s6 - c24) * s6 * inv;  // (|f|/r) * 2^11
                        if (fabsf(fs2) < fs2_max) {
                            bfix_add(ax, fs2, ex);
                            bfix_add(ay, fs2, ey);
                            bfix_add(az, fs2, ez);
                        } else {
                            uint2 t = bfix_wide(fs2, ex, st.err);
                            ax.hi += t.x;
                            ax.lo += t.y;
                            t = bfix_wide(fs2, ey, st.err);
                            ay.hi += t.x;
                            ay.lo += t.y;
                            t = bfix_wide(fs2, ez, st.err);
                            az.hi += t.x;
                            az.lo += t.y;
                        }
                        ++nterms;
                        if (ENERGY) pe += c4 * s6 * (s6 - 1.0f);
                    }
                }
            }
        }
        st.fq[g] = bfix_final(ax, nterms);
        st.fq[st.ntot + g] = bfix_final(ay, nterms);
        st.fq[2 * st.ntot + g] = bfix_final(az, nterms);
        if (ENERGY) pe_out[a] = 0.5f * pe;
    }
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
    Smem sm;
    sm.xr = reinterpret_cast<float4*>(smem);
    sm.perm = reinterpret_cast<uint16_t*>(sm.xr + nmax);
    sm.cell = sm.perm + nmax;
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
