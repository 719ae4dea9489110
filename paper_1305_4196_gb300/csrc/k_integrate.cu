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
//
// FP64 path: every operation rounded exactly as written, as the definition.
// Mixed path: the same update in fused form (one FMA per kick of the fixed-point
// force, one per drift, a fused double kick between steps); GB300 runs FP64 at
// 1/64 of the FP32 rate, so the FP64 instruction count sets this kernel's time.
__global__ void k_integrate(DevState s, Geometry g, PairTable pt, int mode, int mixed, double dt, double lim2,
                            float lim2_f) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int64_t n = s.n;
    const int sp = s.species[i];
    double v[3] = {s.vx[i], s.vy[i], s.vz[i]};
    if (mixed) {
        const double hq = pt.hdtm_q[sp];
        const double kq = mode == INT_KICK_KICK_DRIFT ? 2.0 * hq : hq;
        const double F[3] = {(double)s.fq[i], (double)s.fq[n + i], (double)s.fq[2 * n + i]};
#pragma unroll
        for (int d = 0; d < 3; ++d) v[d] = fma(kq, F[d], v[d]);
    } else {
        const double h = pt.hdtm[sp];
        const double F[3] = {s.f[i], s.f[n + i], s.f[2 * n + i]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (mode != INT_KICK_DRIFT) v[d] = __dadd_rn(v[d], __dmul_rn(h, F[d]));
            if (mode != INT_KICK) v[d] = __dadd_rn(v[d], __dmul_rn(h, F[d]));
        }
    }
    s.vx[i] = v[0];
    s.vy[i] = v[1];
    s.vz[i] = v[2];
    if (mode == INT_KICK) return;
    double x[3] = {s.x[i], s.y[i], s.z[i]};
    bool moved;
    if (mixed) {
#pragma unroll
        for (int d = 0; d < 3; ++d) x[d] = fma(dt, v[d], x[d]);
        // FP32 coordinates relative to the build cell's centre, and the displacement test on them
        const int c = s.cell_of[i];
        float4 p;
        p.x = __double2float_rn(x[0] - s.centre[c]);
        p.y = __double2float_rn(x[1] - s.centre[s.ncell + c]);
        p.z = __double2float_rn(x[2] - s.centre[2 * s.ncell + c]);
        const float4 r = s.xr_ref[i];
        p.w = r.w;
        s.xr[i] = p;
        const float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
        moved = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) > lim2_f;
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) x[d] = __dadd_rn(x[d], __dmul_rn(dt, v[d]));
        const double dx = __dsub_rn(x[0], s.rx[i]);
        const double dy = __dsub_rn(x[1], s.ry[i]);
        const double dz = __dsub_rn(x[2], s.rz[i]);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        moved = d2 > lim2;
    }
    s.x[i] = x[0];
    s.y[i] = x[1];
    s.z[i] = x[2];
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

// ---------------------------------------------------------------- step control (graph mode)
// One thread decides whether this step rebuilds the lists: the skin/2 flag raised
// by k_integrate, or every k-th step.  It sets the graph's IF-node condition,
// clears the flag for the next step and advances the device step counter.
__global__ void k_step_ctrl(int policy, int every_k, int32_t* rebuild_flag, long long* step_counter,
                            uint32_t* err, cudaGraphConditionalHandle handle) {
    const long long step = *step_counter + 1;
    const int moved = *rebuild_flag;
    int rebuild;
    if (policy == 1) {
        rebuild = (step % every_k) == 0;
        if (moved && !rebuild) atomicOr(err, ERR_SKIN);
    } else {
        rebuild = moved != 0;
    }
    *rebuild_flag = 0;
    *step_counter = step;
    cudaGraphSetConditional(handle, rebuild ? 1u : 0u);
}

__global__ void k_count_build(long long* n_builds) { *n_builds += 1; }

void launch_step_ctrl(int policy, int every_k, int32_t* rebuild_flag, long long* step_counter,
                      long long* n_builds, uint32_t* err, cudaGraphConditionalHandle handle, cudaStream_t st) {
    (void)n_builds;
    k_step_ctrl<<<1, 1, 0, st>>>(policy, every_k, rebuild_flag, step_counter, err, handle);
}

void launch_count_build(long long* n_builds, cudaStream_t st) { k_count_build<<<1, 1, 0, st>>>(n_builds); }

// snapshot copy of the permuted state (positions, velocities, images, species, ids)
__global__ void k_copy_state(DevState d, DevState s) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    d.x[t] = s.x[t];
    d.y[t] = s.y[t];
    d.z[t] = s.z[t];
    d.vx[t] = s.vx[t];
    d.vy[t] = s.vy[t];
    d.vz[t] = s.vz[t];
    d.ix[t] = s.ix[t];
    d.iy[t] = s.iy[t];
    d.iz[t] = s.iz[t];
    d.species[t] = s.species[t];
    d.orig[t] = s.orig[t];
}

void launch_copy_state(const DevState& dst, const DevState& src, cudaStream_t st) {
    if (src.n == 0) return;
    int bs = 256;
    k_copy_state<<<(unsigned)((src.n + bs - 1) / bs), bs, 0, st>>>(dst, src);
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

__global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double* __restrict__ partials, int nparts,
                                                               double* __restrict__ out8) {
    __shared__ double sh[8][RED_THREADS];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nparts; b += RED_THREADS)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] += partials[b * 8 + c];
#pragma unroll
    for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 8) out8[threadIdx.x] = sh[threadIdx.x][0];
}

void launch_reduce_energy(const DevState& s, const PairTable& pt, int mixed, double* partials, int nparts,
                          double* out8, cudaStream_t st) {
    int64_t chunk = (s.n + nparts - 1) / nparts;
    if (chunk < 1) chunk = 1;
    k_reduce_partials<<<nparts, RED_THREADS, 0, st>>>(s, pt, mixed, chunk, partials);
    k_reduce_final<<<1, RED_THREADS, 0, st>>>(partials, nparts, out8);
}

// ---------------------------------------------------------------- state I/O
__global__ void k_set_state(DevState s, const double* __restrict__ pos, const double* __restrict__ vel,
                            const int32_t* __restrict__ species, int nsp) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    double q[6] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], vel ? vel[3 * i] : 0.0, vel ? vel[3 * i + 1] : 0.0,
                   vel ? vel[3 * i + 2] : 0.0};
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if (!isfinite(q[k])) {  // refused by md_set_state; kept finite meanwhile
            atomicOr(s.err, 0x40000000u);
            q[k] = 0.0;
        }
    s.x[i] = q[0];
    s.y[i] = q[1];
    s.z[i] = q[2];
    s.vx[i] = q[3];
    s.vy[i] = q[4];
    s.vz[i] = q[5];
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
