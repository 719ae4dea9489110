// k_integrate.cu - velocity Verlet, displacement test, FP64 reductions and state I/O.
//
// The paper integrates the equations of motion with a plain particle-parallel
// loop (Sec. II.A, Sec. II.C).  The integrator is textbook velocity Verlet:
//     v += (dt/2m) F;  x += dt v;  [rebuild test];  F = F(x);  v += (dt/2m) F
// with every operation rounded exactly as written (no contraction), so that
// given identical forces the FP64 trajectory matches the definition bit for bit.
// Consecutive steps fuse the closing half kick of one step with the opening
// half kick and drift of the next (the same operations, one kernel).
//
// Energies use the paper's thread-local accumulators (Sec. II.C) in a fixed
// order: per-atom shares, then per-CTA FP64 partials, then one CTA.
#include "mdgb_internal.cuh"

namespace mdgb {

__device__ __forceinline__ double force_of(const DevState& s, int mixed, int64_t i) {
    return mixed ? (double)s.fq[i] * 2.3283064365386963e-10 /* 2^-32 */ : s.f[i];
}

// mode: INT_KICK_DRIFT (first step), INT_KICK_KICK_DRIFT (close step, open next), INT_KICK (close)
__global__ void k_integrate(DevState s, Geometry g, PairTable pt, int mode, int mixed, double dt, double lim2,
                            float lim2_f) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int64_t n = s.n;
    const double h = pt.hdtm[s.species[i]];
    double v[3] = {s.vx[i], s.vy[i], s.vz[i]};
    double F[3] = {force_of(s, mixed, i), force_of(s, mixed, n + i), force_of(s, mixed, 2 * n + i)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (mode != INT_KICK_DRIFT) v[d] = __dadd_rn(v[d], __dmul_rn(h, F[d]));
        if (mode != INT_KICK) v[d] = __dadd_rn(v[d], __dmul_rn(h, F[d]));
    }
    s.vx[i] = v[0];
    s.vy[i] = v[1];
    s.vz[i] = v[2];
    if (mode == INT_KICK) return;
    double x[3] = {s.x[i], s.y[i], s.z[i]};
#pragma unroll
    for (int d = 0; d < 3; ++d) x[d] = __dadd_rn(x[d], __dmul_rn(dt, v[d]));
    s.x[i] = x[0];
    s.y[i] = x[1];
    s.z[i] = x[2];
    bool moved;
    if (mixed) {
        // FP32 coordinates relative to the build cell's centre, and the displacement test on them
        int cx, cy, cz;
        cell_coords(g, s.cell_of[i], cx, cy, cz);
        float4 p;
        p.x = __double2float_rn(__dsub_rn(x[0], __dmul_rn((double)cx + 0.5, g.w[0])));
        p.y = __double2float_rn(__dsub_rn(x[1], __dmul_rn((double)cy + 0.5, g.w[1])));
        p.z = __double2float_rn(__dsub_rn(x[2], __dmul_rn((double)cz + 0.5, g.w[2])));
        const float4 r = s.xr_ref[i];
        p.w = r.w;
        s.xr[i] = p;
        const float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
        moved = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) > lim2_f;
    } else {
        const double dx = __dsub_rn(x[0], s.rx[i]);
        const double dy = __dsub_rn(x[1], s.ry[i]);
        const double dz = __dsub_rn(x[2], s.rz[i]);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        moved = d2 > lim2;
    }
    if (moved) *s.rebuild_flag = 1;
}

void launch_integrate(const DevState& s, const Geometry& g, const PairTable& pt, int mode, int mixed,
                      double dt, double lim2, cudaStream_t st) {
    if (s.n == 0) return;
    int bs = 256;
    // the FP32 test is made slightly stricter so that FP32 rounding can never let an atom
    // move further than skin/2 without a rebuild
    float lim2_f = (float)(lim2 * (1.0 - 1e-4));
    k_integrate<<<(unsigned)((s.n + bs - 1) / bs), bs, 0, st>>>(s, g, pt, mode, mixed, dt, lim2, lim2_f);
}

// ---------------------------------------------------------------- reductions
// partial[b][0..7] = (PE, KE, W_xx, W_yy, W_zz, W_xy, W_xz, W_yz) over a contiguous chunk,
// each thread summing a fixed strided subset in order, then a fixed-shape tree.
constexpr int RED_THREADS = 256;

__global__ void __launch_bounds__(RED_THREADS) k_reduce_partials(DevState s, PairTable pt, int mixed,
                                                                 int64_t chunk, double* __restrict__ partials) {
    __shared__ double sh[8][RED_THREADS];
    const int64_t n = s.n;
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = lo + threadIdx.x; i < hi; i += RED_THREADS) {
        const double m = pt.mass[s.species[i]];
        const double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
        acc[1] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        if (mixed) {
            acc[0] += (double)s.pe_atom_f[i];
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[2 + c] += (double)s.vir_atom_f[c * n + i];
        } else {
            acc[0] += s.pe_atom_d[i];
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[2 + c] += s.vir_atom_d[c * n + i];
        }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 8) partials[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_reduce_final(const double* __restrict__ partials, int nparts, double* __restrict__ out8) {
    if (threadIdx.x < 8) {
        double a = 0.0;
        for (int b = 0; b < nparts; ++b) a += partials[b * 8 + threadIdx.x];
        out8[threadIdx.x] = a;
    }
}

void launch_reduce_energy(const DevState& s, const PairTable& pt, int mixed, double* partials, int nparts,
                          double* out8, cudaStream_t st) {
    int64_t chunk = (s.n + nparts - 1) / nparts;
    if (chunk < 1) chunk = 1;
    k_reduce_partials<<<nparts, RED_THREADS, 0, st>>>(s, pt, mixed, chunk, partials);
    k_reduce_final<<<1, 32, 0, st>>>(partials, nparts, out8);
}

// ---------------------------------------------------------------- state I/O
__global__ void k_set_state(DevState s, const double* __restrict__ pos, const double* __restrict__ vel,
                            const int32_t* __restrict__ species, int nsp) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    s.x[i] = pos[3 * i];
    s.y[i] = pos[3 * i + 1];
    s.z[i] = pos[3 * i + 2];
    s.vx[i] = vel ? vel[3 * i] : 0.0;
    s.vy[i] = vel ? vel[3 * i + 1] : 0.0;
    s.vz[i] = vel ? vel[3 * i + 2] : 0.0;
    s.ix[i] = 0;
    s.iy[i] = 0;
    s.iz[i] = 0;
    int sp = species ? species[i] : 0;
    if (sp < 0 || sp >= nsp) {
        atomicOr(s.err, 0x80000000u);
        sp = 0;
    }
    s.species[i] = sp;
    s.orig[i] = (int32_t)i;
}

void launch_set_state(const DevState& s, const double* pos, const double* vel, const int32_t* species, int nsp,
                      cudaStream_t st) {
    if (s.n == 0) return;
    int bs = 256;
    k_set_state<<<(unsigned)((s.n + bs - 1) / bs), bs, 0, st>>>(s, pos, vel, species, nsp);
}

__global__ void k_get_state(DevState s, double* __restrict__ pos, double* __restrict__ vel,
                            int32_t* __restrict__ image) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int64_t o = s.orig[i];
    if (pos) {
        pos[3 * o] = s.x[i];
        pos[3 * o + 1] = s.y[i];
        pos[3 * o + 2] = s.z[i];
    }
    if (vel) {
        vel[3 * o] = s.vx[i];
        vel[3 * o + 1] = s.vy[i];
        vel[3 * o + 2] = s.vz[i];
    }
    if (image) {
        image[3 * o] = s.ix[i];
        image[3 * o + 1] = s.iy[i];
        image[3 * o + 2] = s.iz[i];
    }
}

void launch_get_state(const DevState& s, double* pos, double* vel, int32_t* image, cudaStream_t st) {
    if (s.n == 0) return;
    int bs = 256;
    k_get_state<<<(unsigned)((s.n + bs - 1) / bs), bs, 0, st>>>(s, pos, vel, image);
}

__global__ void k_forces_out(DevState s, int mixed, double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int64_t o = s.orig[i];
    const int64_t n = s.n;
    out[3 * o] = force_of(s, mixed, i);
    out[3 * o + 1] = force_of(s, mixed, n + i);
    out[3 * o + 2] = force_of(s, mixed, 2 * n + i);
}

void launch_forces_out(const DevState& s, int mixed, double* f_out, cudaStream_t st) {
    if (s.n == 0) return;
    int bs = 256;
    k_forces_out<<<(unsigned)((s.n + bs - 1) / bs), bs, 0, st>>>(s, mixed, f_out);
}

__global__ void k_cells_out(DevState s, Geometry g, int32_t* __restrict__ cells) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    int cx, cy, cz;
    cell_coords(g, s.cell_of[i], cx, cy, cz);
    cells[s.orig[i]] = cx + g.nc[0] * (cy + g.nc[1] * cz);
}

void launch_cells_out(const DevState& s, const Geometry& g, int32_t* cells, cudaStream_t st) {
    if (s.n == 0) return;
    int bs = 256;
    k_cells_out<<<(unsigned)((s.n + bs - 1) / bs), bs, 0, st>>>(s, g, cells);
}

}  // namespace mdgb
